// FP32 ERMC ray-trace kernel with converged ray initialisation and lane refill.
//
// Same estimator as trace.cu (Silvestri & Pecnik, arXiv:1810.00188: Eqs. 2, 3,
// 12-17 and Algorithm 1), scheduled for SIMT efficiency.  The paper identifies
// warp divergence from rays of very different lengths as the dominant loss of a
// GPU ERMC (Section 4.2) and reorders rays by absorption coefficient; here the
// divergence is removed structurally instead:
//
//  * each warp owns a persistent sequence of work items = (emitting cell, block
//    of up to NB rays), at most two items in flight;
//  * ray initialisation (Philox draws, band/g sampling, direction, origin, the
//    emitting cell's kappa and B, the DDA set-up) runs converged: 32 lanes
//    initialise 32 rays at once and push 48-byte states into a per-warp ring
//    buffer in shared memory;
//  * the march advances every active lane by one cell per iteration; a lane
//    whose ray ends pops the next prepared state, so all lanes stay busy;
//  * a finished ray stores its sample Y at its index in a per-block array in
//    shared memory; when the block's rays are all done the warp sums the array in
//    a fixed order (compensated binary32 pairs per lane, binary64 across lanes).
//    Results are therefore independent of scheduling and of the box: a cell's Q
//    is bit-identical whichever warp computes it.
//
// A loop iteration that makes no progress cannot happen; if it did, the warp
// sets an error flag (counters[5]) and returns instead of spinning.
#include <math.h>
#include <stdint.h>

#include "mcrt_internal.h"

namespace mcrt {
namespace {

constexpr int POOL = 64;   // prepared ray states per warp
constexpr int NB = 256;    // rays per work item
constexpr int WARPS = 8;   // warps per CTA
constexpr int BRICK = 8;   // cells are enumerated in 8x8x8 bricks; each warp takes a
                           // contiguous run, so an SM's rays stay near its cells and
                           // the field gathers hit L1 (rays average a few cells)

struct WarpSmem {
  float4 A[POOL];     // t0x, t0y, t0z, tsx
  float4 B[POOL];     // tsy, tsz, B_i, wgt * kappa_i
  uint4 C[POOL];      // n | g << 16, ray index, flags, unused
  float ybuf[2][NB];  // per-slot samples Y by ray index within the block
};

// flags: bits 0-5 axis signs (+1 each, 2 bits per axis), bit 6 slot,
// bits 8-15 ray index within the block.

__device__ __forceinline__ uint4 philox10(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// The hot path avoids integer<->float conversion instructions, which GB300
// executes on its narrow FP64 pipe, with exact bit constructions:
//  * uniform (w>>9 + 1/2) 2^-23: the 23 draw bits as the mantissa of a number
//    in [1, 2), minus (1 - 2^-24); exact (Sterbenz);
//  * u < 2^23 as a float: mantissa bits of 2^23 + u, minus 2^23; exact;
//  * floor of f in [0, 2^22]: adding 1.5 * 2^23 with round-down puts floor(f)
//    in the low mantissa bits (the sum's ulp is 1); exact.
__device__ __forceinline__ float unif(unsigned w) {
  return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994f;
}

__device__ __forceinline__ float u23_to_float(unsigned u) {
  return __uint_as_float(0x4B000000u | u) - 8388608.f;
}

// A count in [0, 2^32] as a float (16-bit halves, each exact).
__device__ __forceinline__ float u33_to_float(unsigned long long c) {
  if (c >> 32) return 4294967296.f;
  const unsigned v = (unsigned)c;
  return u23_to_float(v >> 16) * 65536.f + u23_to_float(v & 0xffffu);
}

// Linear-interpolation position on the uniform T nodes, clamped to the end
// nodes (same result as clamp(floor(f), 0, nT-2) and clamp(f - floor, 0, 1)).
__device__ __forceinline__ void tpos(float T, float T0, float inv_dT, float tmax_node, int &it,
                                     float &fr) {
  const float f = (T - T0) * inv_dT;
  const float fc = fminf(fmaxf(f, 0.f), tmax_node);
  const float big = __fadd_rd(fc, 12582912.f);
  it = __float_as_int(big) - 0x4B400000;
  fr = fminf(fmaxf(f - (big - 12582912.f), 0.f), 1.f);
}

__device__ __forceinline__ int pick(const unsigned long long *__restrict__ cum, int K, unsigned u) {
  int lo = 0, hi = K - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((unsigned long long)u < cum[mid])
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ void absorb(float x, float &alpha, float &trans) {
  const float e = __expf(-x);
  const float sr = x * (1.f - x * (0.5f - x * (0.16666667f - x * 0.041666668f)));
  const bool small = x < 0.05f;
  alpha = small ? sr : 1.f - e;
  trans = small ? 1.f - sr : e;
}

__device__ __forceinline__ void axis_setup(float d, float fr, float delta, int &s, float &t0,
                                           float &ts) {
  if (d > 0.f) {
    s = 1;
    ts = __fdividef(delta, d);
    t0 = (1.f - fr) * ts;
  } else if (d < 0.f) {
    s = -1;
    ts = __fdividef(delta, -d);
    t0 = fr * ts;
  } else {
    s = 0;
    ts = INFINITY;
    t0 = INFINITY;
  }
}

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += err;
}

struct Item {  // warp-uniform description of one work item
  int lin, ix, iy, iz;  // emitting cell
  int bc;               // index in the box (x fastest)
  int b, nr;            // ray block and its number of rays
};

// Position p of the brick-ordered enumeration -> box coordinates; false when the
// position falls outside the box (ragged edge bricks).
__device__ __forceinline__ bool brick_cell(const TraceArgs &a, long long p, int nbx, int nby,
                                           int &bx, int &by, int &bz) {
  const long long brick = p / (BRICK * BRICK * BRICK);
  const int off = (int)(p - brick * (BRICK * BRICK * BRICK));
  const int gx = (int)(brick % nbx), gy = (int)((brick / nbx) % nby), gz = (int)(brick / ((long long)nbx * nby));
  bx = gx * BRICK + off % BRICK;
  by = gy * BRICK + (off / BRICK) % BRICK;
  bz = gz * BRICK + off / (BRICK * BRICK);
  return bx < a.bnx && by < a.bny && bz < a.bnz;
}

__device__ __forceinline__ Item make_item(const TraceArgs &a, int bx, int by, int bz, int b) {
  Item it;
  it.bc = bx + a.bnx * (by + a.bny * bz);
  it.b = b;
  it.ix = a.bi0 + bx;
  it.iy = a.bj0 + by;
  it.iz = a.bk0 + bz;
  it.lin = it.ix + a.nx * (it.iy + a.ny * it.iz);
  const int left = a.rays - b * NB;
  it.nr = left < NB ? left : NB;
  return it;
}

template <int MINB, int KSTEPS>
__global__ void __launch_bounds__(WARPS * 32, MINB) trace_pool_kernel(const TraceArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem *wsm = reinterpret_cast<WarpSmem *>(smem_raw);
  unsigned long long *s_counts = reinterpret_cast<unsigned long long *>(smem_raw + WARPS * sizeof(WarpSmem));
  const bool plain = a.cell_cn == nullptr;
  if (plain && a.counts_in_smem) {
    const int ncount = a.nb + a.nb * a.ng;
    for (int i = threadIdx.x; i < ncount; i += blockDim.x)
      s_counts[i] = i < a.nb ? a.cn[i] : a.cg[i - a.nb];
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  WarpSmem &S = wsm[warp];
  const unsigned lt_mask = (1u << lane) - 1u;
  const long long W = (long long)gridDim.x * WARPS;
  const long long wg = (long long)blockIdx.x * WARPS + warp;
  const int nblk = (a.rays + NB - 1) / NB;
  const int nbx = (a.bnx + BRICK - 1) / BRICK, nby = (a.bny + BRICK - 1) / BRICK,
            nbz = (a.bnz + BRICK - 1) / BRICK;
  const long long P = (long long)nbx * nby * nbz * (BRICK * BRICK * BRICK);
  const long long chunk = (P + W - 1) / W;
  long long p_next = wg * chunk;
  const long long p_end = min(P, p_next + chunk);
  int cur_bx = 0, cur_by = 0, cur_bz = 0, cur_b = nblk;  // cell being initialised
  bool exhausted = p_next >= p_end;
  unsigned my_cells = 0;

  const int nx = a.nx, ny = a.ny, nz = a.nz, nxy = nx * ny, nxyz = nxy * nz, nb = a.nb,
            ng = a.ng, nT = a.nT;
  const float2 *__restrict__ field = a.field32;
  const float2 *__restrict__ ktab = a.ktab32;
  const float2 *__restrict__ btab = a.btab32;
  const float T0 = (float)a.T0, inv_dT = (float)a.inv_dT, inv_xref = (float)a.inv_xref,
              tol = (float)a.tol, tmax_node = (float)(a.nT - 2);
  const float DX = (float)a.dx, DY = (float)a.dy, DZ = (float)a.dz;
  const float eps0 = (float)a.eps_wall[0], eps1 = (float)a.eps_wall[1];

  // warp-uniform scheduling state
  int it_init = 0, it_done = 0;  // item sequence numbers
  int r_init = 0;
  unsigned head = 0, tail = 0;  // ring positions (mod POOL); count = tail - head
  Item item0 = make_item(a, 0, 0, 0, 0), item1 = item0;  // the two slots' items
  int done0 = 0, done1 = 0;                          // finished rays per slot
  double cell_S = 0.0, cell_S2 = 0.0;  // running sums of the oldest item's cell
  unsigned long long cell_steps_lane = 0;
  unsigned steps0 = 0u, steps1 = 0u;   // this lane's steps per slot

  // per-lane ray registers
  bool active = false;
  int lin = 0, ix = 0, iy = 0, iz = 0, sx = 0, sy = 0, sz = 0, steps = 0, slot = 0, rl = 0;
  int krow = 0, n = 0;
  unsigned ray = 0, nrefl = 0, cellid = 0;
  float t0x = 0, t0y = 0, t0z = 0, tsx = 0, tsy = 0, tsz = 0, cntx = 0, cnty = 0, cntz = 0;
  float tnx = 0, tny = 0, tnz = 0, tprev = 0, tau = 1, X = 0, B_i = 0, B_last = 0, scale = 0;
  unsigned long long tot_steps = 0;
  unsigned tot_cap = 0, tot_wall = 0, max_ray = 0;

  while (!(exhausted && r_init == 0 && it_done == it_init)) {
    bool progress = false;
    // ---- A. converged initialisation of up to 32 rays into the ring ----
    const bool room = (int)(tail - head) <= POOL - 32 && it_init < it_done + 2;
    if (room && r_init == 0 && !exhausted && cur_b >= nblk) {
      // next emitting cell of this warp's brick-ordered run
      bool found = false;
      while (!found && p_next < p_end) {
        found = brick_cell(a, p_next, nbx, nby, cur_bx, cur_by, cur_bz);
        ++p_next;
      }
      if (found) {
        cur_b = 0;
        ++my_cells;
      } else {
        exhausted = true;
      }
      progress = true;
    }
    if (room && (r_init > 0 || cur_b < nblk)) {
      progress = true;
      const int s = (int)(it_init & 1);
      if (r_init == 0) {
        const Item nI = make_item(a, cur_bx, cur_by, cur_bz, cur_b);
        ++cur_b;
        if (s)
          item1 = nI;
        else
          item0 = nI;
      }
      const Item I = s ? item1 : item0;
      const int r = r_init + lane;
      if (r < I.nr) {
        const unsigned cell = (unsigned)I.lin;
        const unsigned rayid = (unsigned)(a.ray_offset + (unsigned long long)(I.b * NB + r));
        const float2 fi = __ldg(field + cell);
        int it_i;
        float fr_i;
        tpos(fi.x, T0, inv_dT, tmax_node, it_i, fr_i);
        const unsigned long long *__restrict__ cn =
            plain ? (a.counts_in_smem ? s_counts : a.cn) : a.cell_cn + (size_t)cell * nb;
        const unsigned long long *__restrict__ cg =
            plain ? (a.counts_in_smem ? s_counts + nb : a.cg) : a.cell_cg + (size_t)cell * nb * ng;
        const unsigned hemi = a.cell_hemi ? __ldg(a.cell_hemi + cell) : 4194304u;
        const uint4 u = philox10(make_uint4(cell, rayid, 0u, a.snapshot), a.key0, a.key1);
        const unsigned m0 = u.x >> 9;
        float mu, ph;
        if (m0 < hemi) {
          const float h = u23_to_float(hemi);
          mu = 1.f - (u23_to_float(m0) + 0.5f) * __frcp_rn(h);
          ph = h * 1.1920928955078125e-07f;
        } else {
          const float h = u23_to_float(8388608u - hemi);
          mu = -((u23_to_float(m0 - hemi) + 0.5f) * __frcp_rn(h));
          ph = h * 1.1920928955078125e-07f;
        }
        float sphi, cphi;
        sincospif(2.f * unif(u.y), &sphi, &cphi);
        const float st = sqrtf(fmaxf(0.f, 1.f - mu * mu));
        const int nn = pick(cn, nb, u.z);
        const unsigned long long *cgn = cg + (size_t)nn * ng;
        const int gg = pick(cgn, ng, u.w);
        float wgt;
        if (plain) {
          wgt = __ldg(a.wgt32 + nn * ng + gg);
        } else {
          const unsigned long long mn = cn[nn] - (nn ? cn[nn - 1] : 0ull);
          const unsigned long long mg = cgn[gg] - (gg ? cgn[gg - 1] : 0ull);
          const float p = u33_to_float(mn) * 2.3283064365386963e-10f * (u33_to_float(mg) * 2.3283064365386963e-10f);
          wgt = __fdividef(__ldg(a.w_g32 + gg), p) * __fdividef(6.2831855f, ph);
        }
        float fx = 0.5f, fy = 0.5f, fz = 0.5f;
        if (a.origin == 0) {
          const uint4 v = philox10(make_uint4(cell, rayid, 1u, a.snapshot), a.key0, a.key1);
          fx = unif(v.x);
          fy = unif(v.y);
          fz = unif(v.z);
        }
        const float2 ki = __ldg(ktab + (size_t)(nn * ng + gg) * nT + it_i);
        const float2 bi = __ldg(btab + (size_t)nn * nT + it_i);
        const float kap_i = (ki.x + fr_i * ki.y) * (fi.y * inv_xref);
        int ssx, ssy, ssz;
        float a0x, a0y, a0z, asx, asy, asz;
        axis_setup(st * cphi, fx, DX, ssx, a0x, asx);
        axis_setup(mu, fy, DY, ssy, a0y, asy);
        axis_setup(st * sphi, fz, DZ, ssz, a0z, asz);
        const int pos = (tail + lane) & (POOL - 1);
        S.A[pos] = make_float4(a0x, a0y, a0z, asx);
        S.B[pos] = make_float4(asy, asz, bi.x + fr_i * bi.y, wgt * kap_i);
        const unsigned flags = (unsigned)(ssx + 1) | ((unsigned)(ssy + 1) << 2) |
                               ((unsigned)(ssz + 1) << 4) | ((unsigned)s << 6) | ((unsigned)r << 8);
        S.C[pos] = make_uint4((unsigned)nn | ((unsigned)gg << 16), rayid, flags, 0u);
      }
      const int cnt = min(32, I.nr - r_init);
      tail += (unsigned)cnt;
      r_init += 32;
      if (r_init >= I.nr) {
        r_init = 0;
        ++it_init;
      }
      __syncwarp();
    }

    // ---- B. idle lanes take prepared rays ----
    const unsigned idle = __ballot_sync(0xffffffffu, !active);
    const int avail = (int)(tail - head);
    if (idle && avail > 0) {
      const int rank = __popc(idle & lt_mask);
      if (!active && rank < avail) {
        const int pos = (head + rank) & (POOL - 1);
        const float4 A = S.A[pos];
        const float4 Bv = S.B[pos];
        const uint4 Cv = S.C[pos];
        t0x = A.x;
        t0y = A.y;
        t0z = A.z;
        tsx = A.w;
        tsy = Bv.x;
        tsz = Bv.y;
        B_i = Bv.z;
        scale = Bv.w;
        n = (int)(Cv.x & 0xffffu);
        krow = (n * ng + (int)(Cv.x >> 16)) * nT;
        ray = Cv.y;
        sx = (int)(Cv.z & 3u) - 1;
        sy = (int)((Cv.z >> 2) & 3u) - 1;
        sz = (int)((Cv.z >> 4) & 3u) - 1;
        slot = (int)((Cv.z >> 6) & 1u);
        rl = (int)((Cv.z >> 8) & 0xffu);
        const Item I = slot ? item1 : item0;
        lin = I.lin;
        ix = I.ix;
        iy = I.iy;
        iz = I.iz;
        cellid = (unsigned)I.lin;
        tnx = t0x;
        tny = t0y;
        tnz = t0z;
        cntx = cnty = cntz = 0.f;
        tprev = 0.f;
        tau = 1.f;
        X = 0.f;
        B_last = B_i;
        steps = 0;
        nrefl = 0;
        active = true;
      }
      const int taken = min(__popc(idle), avail);
      head += (unsigned)taken;
      progress = true;
      __syncwarp();
    }

    // ---- C. up to KSTEPS march steps per active lane (Algorithm 1 "March") ----
    bool finished = false;
    if (__any_sync(0xffffffffu, active)) progress = true;  // warp-uniform
    for (int kstep = 0; kstep < KSTEPS; ++kstep) {
      if (!active) break;
        float tn;
        int ax;
        if (tnx <= tny && tnx <= tnz) {
          ax = 0;
          tn = tnx;
        } else if (tny <= tnz) {
          ax = 1;
          tn = tny;
        } else {
          ax = 2;
          tn = tnz;
        }
        const float ds = fmaxf(tn - tprev, 0.f);
        const float2 f = __ldg(field + lin);
        int it;
        float fr;
        tpos(f.x, T0, inv_dT, tmax_node, it, fr);
        const float2 kk = __ldg(ktab + krow + it);
        const float2 bb = __ldg(btab + n * nT + it);
        const float kap = (kk.x + fr * kk.y) * (f.y * inv_xref);
        const float Bj = bb.x + fr * bb.y;
        float alpha, trans;
        absorb(kap * ds, alpha, trans);
        X += (B_i - Bj) * (tau * alpha);  // Eq. 14 term / kappa_i
        tau *= trans;                     // Eq. 3
        B_last = Bj;
        ++steps;
        bool done = tau <= tol;
        if (!done && steps >= a.max_steps) {
          done = true;
          ++tot_cap;
        }
        if (!done) {
          tprev = tn;
          if (ax == 0) {
            cntx += 1.f;
            tnx = fmaf(cntx, tsx, t0x);
            ix += sx;
            lin += sx;
            if (ix >= nx) {
              ix -= nx;
              lin -= nx;
            } else if (ix < 0) {
              ix += nx;
              lin += nx;
            }
          } else if (ax == 2) {
            cntz += 1.f;
            tnz = fmaf(cntz, tsz, t0z);
            iz += sz;
            lin += sz * nxy;
            if (iz >= nz) {
              iz -= nz;
              lin -= nxyz;
            } else if (iz < 0) {
              iz += nz;
              lin += nxyz;
            }
          } else {
            cnty += 1.f;
            tny = fmaf(cnty, tsy, t0y);
            iy += sy;
            lin += sy * nx;
            if (iy < 0 || iy >= ny) {
              // wall: absorbs eps of the ray and emits at T_wall (Eq. 3 wall factor)
              const int wl = iy < 0 ? 0 : 1;
              const float eps = wl ? eps1 : eps0;
              const float Bw = __ldg(a.bwall32 + wl * nb + n);
              X += (B_i - Bw) * (tau * eps);
              tau *= 1.f - eps;
              ++tot_wall;
              if (eps >= 1.f || tau <= tol) {
                done = true;
              } else {
                float nfx = 0.5f, nfz = 0.5f;
                if (sx > 0)
                  nfx = 1.f - (tnx - tprev) / tsx;
                else if (sx < 0)
                  nfx = (tnx - tprev) / tsx;
                if (sz > 0)
                  nfz = 1.f - (tnz - tprev) / tsz;
                else if (sz < 0)
                  nfz = (tnz - tprev) / tsz;
                nfx = fminf(fmaxf(nfx, 0.f), 1.f);
                nfz = fminf(fmaxf(nfz, 0.f), 1.f);
                const float nfy = wl == 0 ? 0.f : 1.f;
                iy = wl == 0 ? 0 : ny - 1;
                lin = ix + nx * iy + nxy * iz;
                float ddx, ddy, ddz;
                if (a.reflect == 1) {
                  // specular: |d| per axis unchanged, the y component flips
                  ddx = sx > 0 ? DX / tsx : (sx < 0 ? -DX / tsx : 0.f);
                  ddz = sz > 0 ? DZ / tsz : (sz < 0 ? -DZ / tsz : 0.f);
                  ddy = wl == 0 ? DY / tsy : -DY / tsy;
                } else {
                  const uint4 v = philox10(make_uint4(cellid, ray, 2u + nrefl, a.snapshot), a.key0, a.key1);
                  const float mr = sqrtf(unif(v.x));
                  float sp, cp;
                  sincospif(2.f * unif(v.y), &sp, &cp);
                  const float sr = sqrtf(fmaxf(0.f, 1.f - mr * mr));
                  ddx = sr * cp;
                  ddy = wl == 0 ? mr : -mr;
                  ddz = sr * sp;
                }
                ++nrefl;
                axis_setup(ddx, nfx, DX, sx, t0x, tsx);
                axis_setup(ddy, nfy, DY, sy, t0y, tsy);
                axis_setup(ddz, nfz, DZ, sz, t0z, tsz);
                cntx = cnty = cntz = 0.f;
                tnx = t0x;
                tny = t0y;
                tnz = t0z;
                tprev = 0.f;
              }
            }
          }
        }
        if (done) {
          if (tau > 0.f) X += (B_i - B_last) * tau;  // residual dump (Algorithm 1)
          S.ybuf[slot][rl] = scale * X;
          if (slot)
            steps1 += (unsigned)steps;
          else
            steps0 += (unsigned)steps;
          tot_steps += (unsigned long long)steps;
          max_ray = max(max_ray, (unsigned)steps);
          active = false;
          finished = true;
        }
    
    }
    // ---- D. bookkeeping and in-order completion of work items ----
    const unsigned fin0 = __ballot_sync(0xffffffffu, finished && slot == 0);
    const unsigned fin1 = __ballot_sync(0xffffffffu, finished && slot == 1);
    done0 += __popc(fin0);
    done1 += __popc(fin1);
    for (;;) {
      const int so = (int)(it_done & 1);
      if (it_done >= it_init) break;  // not fully initialised yet
      const Item I = so ? item1 : item0;
      if ((so ? done1 : done0) < I.nr) break;
      progress = true;
      __syncwarp();
      float hi = 0.f, lo = 0.f, hi2 = 0.f, lo2 = 0.f;
      for (int k = lane; k < I.nr; k += 32) {
        const float y = S.ybuf[so][k];
        two_sum_acc(hi, lo, y);
        const float p = y * y;
        two_sum_acc(hi2, lo2, p);
        lo2 += fmaf(y, y, -p);
      }
      double bs = (double)hi + (double)lo, bs2 = (double)hi2 + (double)lo2;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        bs += __shfl_xor_sync(0xffffffffu, bs, off);
        bs2 += __shfl_xor_sync(0xffffffffu, bs2, off);
      }
      cell_S += bs;
      cell_S2 += bs2;
      cell_steps_lane += so ? steps1 : steps0;
      if (so) {
        steps1 = 0u;
        done1 = 0;
      } else {
        steps0 = 0u;
        done0 = 0;
      }
      if (I.b == nblk - 1) {
        unsigned long long cs = cell_steps_lane;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, off);
        if (lane == 0) {
          const double N = (double)a.rays;
          const double Q = cell_S / N;
          a.q[I.bc] = Q;  // Eq. 8: mean of the per-ray samples
          if (a.sigma)
            a.sigma[I.bc] = a.rays > 1 ? sqrt(fmax(cell_S2 / N - Q * Q, 0.0) / (N - 1.0)) : 0.0;
          if (a.steps_cell) a.steps_cell[I.bc] = cs;
        }
        cell_S = cell_S2 = 0.0;
        cell_steps_lane = 0;
      }
      ++it_done;
      __syncwarp();
    }
    if (!progress) {  // unreachable by construction; never spin
      if (lane == 0) atomicOr(a.counters + 5, 1ull);
      break;
    }
  }

  // kernel-wide counters
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tot_steps += __shfl_xor_sync(0xffffffffu, tot_steps, off);
    tot_cap += __shfl_xor_sync(0xffffffffu, tot_cap, off);
    tot_wall += __shfl_xor_sync(0xffffffffu, tot_wall, off);
    max_ray = max(max_ray, __shfl_xor_sync(0xffffffffu, max_ray, off));
  }
  if (lane == 0 && my_cells > 0) {
    atomicMax(a.counters + 4, (unsigned long long)max_ray);
    atomicAdd(a.counters + 0, tot_steps);
    if (tot_cap) atomicAdd(a.counters + 1, (unsigned long long)tot_cap);
    if (tot_wall) atomicAdd(a.counters + 2, (unsigned long long)tot_wall);
    atomicAdd(a.counters + 3, (unsigned long long)my_cells * (unsigned long long)a.rays);
  }
}

template <int MINB, int KSTEPS>
cudaError_t launch_pool_variant(const TraceArgs &a, cudaStream_t s, size_t smem) {
  // per-device launch shape, computed once per device and shared-memory size
  static int configured_smem[64], blocks_per_sm[64], num_sms[64];
  static bool init_done = false;
  if (!init_done) {
    for (int i = 0; i < 64; ++i) configured_smem[i] = -1;
    init_done = true;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (configured_smem[dev] != (int)smem) {
    e = cudaFuncSetAttribute(trace_pool_kernel<MINB, KSTEPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[dev], trace_pool_kernel<MINB, KSTEPS>,
                                                      WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm[dev] < 1) blocks_per_sm[dev] = 1;
    configured_smem[dev] = (int)smem;
  }
  const long long need = (a.ncells_box + WARPS - 1) / WARPS;
  long long blocks = (long long)num_sms[dev] * blocks_per_sm[dev];
  if (blocks > need) blocks = need;
  trace_pool_kernel<MINB, KSTEPS><<<(unsigned)blocks, WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_trace_pool(const TraceArgs &a, int min_blocks, int steps_per_round,
                              cudaStream_t s) {
  if (a.ncells_box <= 0) return cudaSuccess;
  const size_t smem = WARPS * sizeof(WarpSmem) +
                      (a.counts_in_smem ? sizeof(unsigned long long) * (size_t)(a.nb + a.nb * a.ng) : 0);
#define MCRT_POOL_K(MB)                                                   \
  switch (steps_per_round) {                                              \
    case 2: return launch_pool_variant<MB, 2>(a, s, smem);                \
    case 4: return launch_pool_variant<MB, 4>(a, s, smem);                \
    default: return launch_pool_variant<MB, 1>(a, s, smem);               \
  }
  switch (min_blocks) {
    case 1: MCRT_POOL_K(1)
    case 3: MCRT_POOL_K(3)
    default: MCRT_POOL_K(2)
  }
#undef MCRT_POOL_K
}

}  // namespace mcrt

// Device helpers shared by the FP32 trace kernels of trace_fp32.cu (one solve)
// and batch.cu (many snapshots in one launch): the per-warp ray ring, exact bit
// constructions of uniforms and small integers, the interpolation position, the
// azimuth's sine and cosine, the guided inverse CDF, the absorption of a segment, the
// axis set-up of the parametric ray, compensated binary32 sums, and the
// brick-order enumeration of cells.
#pragma once

#include <math.h>
#include <stdint.h>

#include "mcrt_internal.h"

namespace mcrt {
namespace {

constexpr int POOL = 64;   // prepared ray states per warp
constexpr int WARPS = 8;   // warps per CTA
constexpr int BRICK = 8;   // cells are enumerated in 8x8x8 bricks
constexpr int GUIDE_BITS = 11;           // the top bits of R_n that index the guide table
constexpr int GUIDE = 1 << GUIDE_BITS;   // guide-table buckets of the band CDF
constexpr int GG_BITS = 5;               // the top bits of R_g that index a band's g guide
constexpr int GG = 1 << GG_BITS;         // g guide entries per band (bytes)
constexpr int REFILL = 8;  // idle lanes of a warp before they take prepared rays

struct WarpRing {
  float4 A[POOL];  // t0x, t0y, t0z, tsx
  float4 B[POOL];  // tsy, tsz, B_i, w * kappa_i
  uint4 C[POOL];   // n | g << 16, Philox ray index, axis signs, emitting cell (linear)
  int4 D[POOL];    // sample slot (cell position in the chunk), ix, iy, iz
};

// Exact bit constructions instead of conversion instructions:
//  * uniform (w>>9 + 1/2) 2^-23: the 23 draw bits as the mantissa of a number in
//    [1, 2), minus (1 - 2^-24); exact (Sterbenz);
//  * u < 2^23 as a float: mantissa bits of 2^23 + u, minus 2^23; exact;
//  * floor / nearest integer of f in [0, 2^22]: adding 1.5 * 2^23 with directed
//    or nearest rounding puts the integer in the low mantissa bits (the sum's ulp
//    is 1); exact.
__device__ __forceinline__ float unif(unsigned w) {
  return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994f;
}

__device__ __forceinline__ float u23_to_float(unsigned u) {
  return __uint_as_float(0x4B000000u | u) - 8388608.f;
}

__device__ __forceinline__ float u33_to_float(unsigned long long c) {
  if (c >> 32) return 4294967296.f;
  const unsigned v = (unsigned)c;
  return u23_to_float(v >> 16) * 65536.f + u23_to_float(v & 0xffffu);
}

// A cell's precomputed interpolation position (Section 2.2's linear
// interpolation in T; see pack_positions_kernel): node index in the top 9 bits,
// the fraction towards the next node as 23 mantissa bits (exact).
__device__ __forceinline__ void tpos(unsigned packed, unsigned &it, float &fr) {
  it = packed >> 23;
  fr = __uint_as_float(0x3F800000u | (packed & 0x7FFFFFu)) - 1.f;
}

// sin(2 pi u), cos(2 pi u) for u in (0, 1) with the hardware approximations
// (absolute error about 4e-7): the angle is reduced to 2 pi (u - 1/2) in
// (-pi, pi), the range where __sincosf is accurate, and both signs flip back.
__device__ __forceinline__ void sincos_2pi(float u, float &s, float &c) {
  float s0, c0;
  __sincosf(6.28318530717958647f * (u - 0.5f), &s0, &c0);
  s = -s0;
  c = -c0;
}

// First k with u < cum[k] (the inverse CDF of Eq. 17), started from a guide
// table: guide[m] = first k with cum[k] > m 2^(32 - GUIDE_BITS), so the scan
// is short.
__device__ __forceinline__ int pick_guided(const unsigned long long *__restrict__ cum,
                                           const unsigned short *__restrict__ guide, unsigned u) {
  int k = guide[u >> (32 - GUIDE_BITS)];
  while ((unsigned long long)u >= cum[k]) ++k;
  return k;
}

// First g with u < cum[g] within one band's g counts (Eq. 17), started from the
// band's guide: gg[m] = first g with cum[g] > m 2^(32 - GG_BITS).
__device__ __forceinline__ int pick_gguided(const unsigned long long *__restrict__ cum,
                                            const unsigned char *__restrict__ gg, unsigned u) {
  int k = gg[u >> (32 - GG_BITS)];
  while ((unsigned long long)u >= cum[k]) ++k;
  return k;
}

__device__ __forceinline__ void absorb(float x, float &alpha, float &trans) {
  // alpha = 1 - exp(-x) (Eq. 2), trans = exp(-x) (Eq. 3); a 4-term series below
  // x = 0.05 avoids the cancellation of 1 - exp(-x)
  const float e = __expf(-x);
  const float sr = x * (1.f - x * (0.5f - x * (0.16666667f - x * 0.041666668f)));
  const bool small = x < 0.05f;
  alpha = small ? sr : 1.f - e;
  trans = small ? 1.f - sr : e;
}

// Parametric ray o + t d along one axis: the m-th face crossing is at t0 + m ts.
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

// Brick-order position p (relative to a bnx x bny x bnz box) -> box coordinates;
// false for positions outside the box (ragged edge bricks).
__device__ __forceinline__ bool brick_cell_d(int bnx, int bny, int bnz, long long p, int &bx, int &by,
                                             int &bz) {
  const unsigned nbx = (unsigned)(bnx + BRICK - 1) / BRICK, nby = (unsigned)(bny + BRICK - 1) / BRICK;
  unsigned off, gx, gy, gz;
  if (p < (1LL << 31)) {
    // 32-bit arithmetic: boxes of fewer than 2^31 positions (64-bit divisions
    // are long instruction sequences)
    const unsigned pu = (unsigned)p, brick = pu / (BRICK * BRICK * BRICK), t = brick / nbx;
    off = pu % (BRICK * BRICK * BRICK);
    gx = brick - t * nbx;
    gy = t % nby;
    gz = t / nby;
  } else {
    const long long brick = p / (BRICK * BRICK * BRICK);
    off = (unsigned)(p - brick * (BRICK * BRICK * BRICK));
    gx = (unsigned)(brick % nbx);
    gy = (unsigned)((brick / nbx) % nby);
    gz = (unsigned)(brick / ((long long)nbx * nby));
  }
  bx = (int)(gx * BRICK + off % BRICK);
  by = (int)(gy * BRICK + (off / BRICK) % BRICK);
  bz = (int)(gz * BRICK + off / (BRICK * BRICK));
  return bx < bnx && by < bny && bz < bnz;
}

__device__ __forceinline__ bool brick_cell(const TraceArgs &a, long long p, int &bx, int &by,
                                           int &bz) {
  return brick_cell_d(a.bnx, a.bny, a.bnz, p, bx, by, bz);
}

// Batched solves: the snapshot that owns global position p (starts[k] is
// snapshot k's first position; starts[n] the end).
__device__ __forceinline__ int snapshot_of(const long long *starts, int n, long long p) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= p)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Compensated binary32 pair (hi + lo) plus another pair, renormalised.
__device__ __forceinline__ void pair_add(float &hi, float &lo, float bhi, float blo) {
  const float s = hi + bhi;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (bhi - bb) + (lo + blo);
  hi = s + err;
  lo = err - (hi - s);
}

// Long rays (long_rays.cu).  A ray whose flight to the next y face still crosses
// at least `need` x/z faces: (t_y - t) (1/ts_x + 1/ts_z), an axis the ray does
// not cross having ts = inf.  A flight with no y face ahead (d_y = 0) is long
// unless the ray crosses nothing at all.
__device__ __forceinline__ bool long_flight(float tny, float tprev, float tsx, float tsz, float need) {
  return (tny - tprev) * (__frcp_rn(tsx) + __frcp_rn(tsz)) >= need;
}

// Stores a lane's ray state for the warp-parallel march; false when the buffer
// is full (the ray then marches on where it is).
__device__ __forceinline__ bool hand_off(const TraceArgs &a, const LongRay &L) {
  const unsigned long long k = atomicAdd(a.counters + 7, 1ull);
  if (k >= (unsigned long long)a.long_cap) return false;
  const float4 *src = reinterpret_cast<const float4 *>(&L);
  float4 *dst = reinterpret_cast<float4 *>(a.long_rays + k);
#pragma unroll
  for (int i = 0; i < 8; ++i) dst[i] = src[i];
  return true;
}

// Sum of one cell's N samples y[0..N) and of their squares over a warp, as
// compensated binary32 pairs.  Each lane reads its samples lane, lane + 32, ...
// in batches of LOADS (with the streaming hint: each sample is read once, and a
// batch keeps enough bytes in flight for HBM), sums a batch and its squares
// pairwise in binary32, and adds the two batch sums to its compensated pairs.
// The lanes then combine in a lane-independent tree, so every lane returns
// identical bits, and the order never depends on the launch.  A pairwise sum of
// 8 values errs by at most 3 units in the last place of the sum of their
// magnitudes, so the tally is within 2e-7 of sum |y| (the FP32 tolerance on Q is
// 1e-4 of the cell's mean |Y|), at a quarter of the additions of compensating
// every sample.
__device__ __forceinline__ void warp_cell_sums(const float *__restrict__ y, int N, int lane, float &hi,
                                               float &lo, float &hi2, float &lo2) {
  constexpr int LOADS = 8;
  hi = 0.f; lo = 0.f; hi2 = 0.f; lo2 = 0.f;
  for (int k0 = lane; k0 < N; k0 += 32 * LOADS) {
    float v[LOADS], sq[LOADS];
#pragma unroll
    for (int j = 0; j < LOADS; ++j) v[j] = k0 + 32 * j < N ? __ldcs(y + k0 + 32 * j) : 0.f;
#pragma unroll
    for (int j = 0; j < LOADS; ++j) sq[j] = v[j] * v[j];
#pragma unroll
    for (int w = 1; w < LOADS; w <<= 1) {
#pragma unroll
      for (int j = 0; j < LOADS; j += 2 * w) {
        v[j] += v[j + w];
        sq[j] += sq[j + w];
      }
    }
    two_sum_acc(hi, lo, v[0]);
    two_sum_acc(hi2, lo2, sq[0]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, off), ol = __shfl_xor_sync(0xffffffffu, lo, off);
    const float oh2 = __shfl_xor_sync(0xffffffffu, hi2, off), ol2 = __shfl_xor_sync(0xffffffffu, lo2, off);
    // combine in a lane-independent order so every lane holds identical bits
    if (lane & off) {
      float th = oh, tl = ol, th2 = oh2, tl2 = ol2;
      pair_add(th, tl, hi, lo);
      pair_add(th2, tl2, hi2, lo2);
      hi = th; lo = tl; hi2 = th2; lo2 = tl2;
    } else {
      pair_add(hi, lo, oh, ol);
      pair_add(hi2, lo2, oh2, ol2);
    }
  }
}

// ---- absorption-based estimate (ARMC) -----------------------------------------

// Index of `cell`'s per-batch sum for the ray with index r in its cell: batch
// r mod 16 (with fewer than 16 rays per cell, r < K and the batch is r itself).
__device__ __forceinline__ size_t armc_slot(const TraceArgs &a, unsigned r, unsigned cell) {
  return (size_t)(r & 15u) * (size_t)a.armc_nc + cell;
}

// V_i / V_j of the emitting cell i (linear index cellid) and an absorbing cell in
// row j, for the absorption-based deposits: cells differ only in their
// wall-normal height, and only on a stretched grid (faces yfs; null: 1).
__device__ __forceinline__ float volume_ratio(const float *__restrict__ yfs, int nx, int ny, unsigned cellid, int j) {
  if (!yfs) return 1.f;
  const int ie = (int)((cellid / (unsigned)nx) % (unsigned)ny);
  return (__ldg(yfs + ie + 1) - __ldg(yfs + ie)) / (__ldg(yfs + j + 1) - __ldg(yfs + j));
}

// binary32 -> binary64, exactly, from the bits (the conversion instruction runs
// on the narrow binary64 pipe); zeros, subnormals, infinities and NaN take the
// instruction.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e - 1u < 254u) {
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  return (double)f;
}

// ---- one march round of a lane (both FP32 trace kernels) ----------------------

// A ray in flight: the registers of one lane.  Table and field indices are
// unsigned: widening them to 64-bit addresses is free, while sign-extending an
// int costs a conversion on GB300's narrow pipe.
struct LaneRay {
  bool active = false;
  unsigned lin = 0, krow = 0, n = 0, slot = 0, r = 0;
  uint2 fcur = make_uint2(0u, 0u);  // field entry of the current cell, loaded a step ahead
  int ix = 0, iy = 0, iz = 0, sx = 0, sy = 0, sz = 0, steps = 0;
  unsigned ray = 0, nrefl = 0, cellid = 0;
  float t0x = 0, t0y = 0, t0z = 0, tsx = 0, tsy = 0, tsz = 0, cntx = 0, cnty = 0, cntz = 0;
  float tnx = 0, tny = 0, tnz = 0, tprev = 0, tau = 1, X = 0, B_i = 0, B_last = 0, scale = 0;
  // multigrid: current grid, segments marched on it, offset of its fields, and
  // the face counter step (grid lev keeps every inc-th face of the grid the
  // axis parameters were set up on)
  int lev = 0, lsteps = 0;
  unsigned loff = 0;
  float inc = 1.f;
};

// A lane's counts for the solve's statistics and the per-cell step sums.
struct LaneStats {
  unsigned long long tot_steps = 0;
  unsigned tot_cap = 0, tot_wall = 0, max_ray = 0, tot_rays = 0;
  int acc_slot = -1;  // run of steps for the per-cell step counts
  unsigned acc_steps = 0;
};

// What a march round reads besides the ray and the launch arguments: the grid,
// fields and walls of the solve, or of the snapshot a batched warp is on.
struct MarchGrid {
  int nx, ny, nz, nxy;
  const uint2 *field;        // table positions and x of every multigrid grid
  const float *yfs;          // stretched y faces, or null
  const float *bwall;        // wall band intensities [faces][nb]
  float DX, DY, DZ, eps0, eps1;
  int reflect;               // 0 diffuse, 1 specular
  unsigned snapw;            // fourth Philox counter word
};

// Up to KSTEPS march steps of the lane's ray (Algorithm 1 "March"): per segment
// the absorption of Eq. 2, the term of Eq. 14 and the transmissivity of Eq. 3;
// face crossings with the periodic wrap, wall events (Eq. 3 wall factor,
// diffuse or specular reflection), the multigrid switch (Section 4.3), the
// hand-off of long rays, and at the end the residual dump and the sample.
// GEN: stretched y faces and closed boxes; AR: the absorption-based deposits;
// BATCH: a batched launch (the snapshot of a handed-off ray from its position
// among the snapshots' first positions, `starts`).
template <int KSTEPS, bool MG, bool GEN, bool AR, bool BATCH>
__device__ __forceinline__ void march_round(const TraceArgs &a, const MarchGrid &g, LaneRay &s, LaneStats &ls,
                                            const long long *starts = nullptr) {
  const float *__restrict__ yfs = GEN ? g.yfs : nullptr;
  const float4 *__restrict__ kbtab = a.kbtab32;
  const uint2 *__restrict__ field = g.field;
  const float *__restrict__ bwall = g.bwall;
  float *__restrict__ Ybuf = a.ybuf;
  const float tol = a.tol32;
  const int nb = a.nb;
  const unsigned N = (unsigned)a.rays;
  auto dyl = [&](int j, int l) -> float {
    return __ldg(yfs + ((unsigned)(j + 1) << l)) - __ldg(yfs + ((unsigned)j << l));
  };
  for (int kstep = 0; kstep < KSTEPS; ++kstep) {
    if (!s.active) break;
    float tn;
    int ax;
    if (s.tnx <= s.tny && s.tnx <= s.tnz) {
      ax = 0;
      tn = s.tnx;
    } else if (s.tny <= s.tnz) {
      ax = 1;
      tn = s.tny;
    } else {
      ax = 2;
      tn = s.tnz;
    }
    const float ds = fmaxf(tn - s.tprev, 0.f);
    const uint2 f = s.fcur;
    unsigned it;
    float fr;
    tpos(f.x, it, fr);
    const float4 kb = __ldg(kbtab + (s.krow + it));
    const float kap = (kb.x + fr * kb.y) * __uint_as_float(f.y);
    const float Bj = kb.z + fr * kb.w;
    float alpha, trans;
    absorb(kap * ds, alpha, trans);
    const float term = (s.B_i - Bj) * (s.tau * alpha);
    s.X += term;     // Eq. 14 term / kappa_i
    s.tau *= trans;  // Eq. 3
    if (AR && s.lin != s.cellid)  // the exchange absorbed in cell j, seen from j
      atomicAdd(a.armc_acc + armc_slot(a, s.r, s.lin),
                f32_to_f64(-s.scale * term * volume_ratio(yfs, g.nx, g.ny, s.cellid, s.iy)));
    s.B_last = Bj;
    ++s.steps;
    if (MG) ++s.lsteps;
    bool done = s.tau <= tol;
    if (!done && s.steps >= a.max_steps) {
      done = true;
      ++ls.tot_cap;
    }
    if (!done) {
      s.tprev = tn;
      // dimensions of the current grid
      const int nxl = MG ? g.nx >> s.lev : g.nx, nyl = MG ? g.ny >> s.lev : g.ny, nzl = MG ? g.nz >> s.lev : g.nz;
      const int nxyl = MG ? nxl * nyl : g.nxy;
      {
        // branch-free advance of the crossed axis (lanes cross different axes)
        const bool mx = ax == 0, my = ax == 1, mz = ax == 2;
        const float step = MG ? s.inc : 1.f;
        s.cntx += mx ? step : 0.f;
        s.cnty += my ? step : 0.f;
        s.cntz += mz ? step : 0.f;
        s.tnx = mx ? fmaf(s.cntx, s.tsx, s.t0x) : s.tnx;
        s.tny = my ? fmaf(s.cnty, s.tsy, s.t0y) : s.tny;
        s.tnz = mz ? fmaf(s.cntz, s.tsz, s.t0z) : s.tnz;
        s.ix += mx ? s.sx : 0;
        s.iy += my ? s.sy : 0;
        s.iz += mz ? s.sz : 0;
        if (yfs && my && (unsigned)s.iy < (unsigned)nyl) s.tny = s.tprev + dyl(s.iy, MG ? s.lev : 0) * s.tsy;
        // periodic wrap: an index can only leave the grid in the ray's direction
        const int wx = (unsigned)s.ix < (unsigned)nxl ? 0 : -s.sx * nxl;
        s.ix += wx;
        const int wz = (unsigned)s.iz < (unsigned)nzl ? 0 : -s.sz * nzl;
        s.iz += wz;
        // the linear index from the three indices (multiply-adds, off the ALU pipe)
        s.lin = (unsigned)(s.ix + nxl * (s.iy + nyl * s.iz));
        if (GEN && !BATCH && a.xz_walls && (wx | wz)) {
          // closed box: a black x or z wall absorbs the rest of the ray and
          // emits at its temperature (Eq. 3 wall factor with eps = 1)
          const int f = wx ? (wx > 0 ? 2 : 3) : (wz > 0 ? 4 : 5);
          const float tw = (s.B_i - __ldg(bwall + ((unsigned)(f * nb) + s.n))) * s.tau;
          s.X += tw;
          if (AR)  // the cell's own exchange with the wall
            atomicAdd(a.armc_acc + armc_slot(a, s.r, s.cellid), f32_to_f64(s.scale * tw));
          s.tau = 0.f;
          ++ls.tot_wall;
          done = true;
        } else if ((unsigned)s.iy >= (unsigned)nyl) {
          // wall: absorbs eps of the ray and emits at T_wall (Eq. 3 wall factor)
          const int wl = s.iy < 0 ? 0 : 1;
          const float eps = wl ? g.eps1 : g.eps0;
          const float Bw = __ldg(bwall + ((unsigned)(wl * nb) + s.n));
          s.X += (s.B_i - Bw) * (s.tau * eps);
          if (AR)  // the cell's own exchange with the wall
            atomicAdd(a.armc_acc + armc_slot(a, s.r, s.cellid), f32_to_f64(s.scale * ((s.B_i - Bw) * (s.tau * eps))));
          s.tau *= 1.f - eps;
          ++ls.tot_wall;
          if (eps >= 1.f || s.tau <= tol) {
            done = true;
          } else {
            // fractions of the current grid's cell, whose extent along an
            // axis is inc face steps of the axis parameters
            const float cx = MG ? s.tsx * s.inc : s.tsx, cz = MG ? s.tsz * s.inc : s.tsz;
            float nfx = 0.5f, nfz = 0.5f;
            if (s.sx > 0)
              nfx = 1.f - (s.tnx - s.tprev) / cx;
            else if (s.sx < 0)
              nfx = (s.tnx - s.tprev) / cx;
            if (s.sz > 0)
              nfz = 1.f - (s.tnz - s.tprev) / cz;
            else if (s.sz < 0)
              nfz = (s.tnz - s.tprev) / cz;
            nfx = fminf(fmaxf(nfx, 0.f), 1.f);
            nfz = fminf(fmaxf(nfz, 0.f), 1.f);
            const float nfy = wl == 0 ? 0.f : 1.f;
            s.iy = wl == 0 ? 0 : nyl - 1;
            s.lin = (unsigned)(s.ix + nxl * s.iy + nxyl * s.iz);
            // cell size of the current grid over the finest, and of the grid
            // the axis parameters were set up on
            const float gl = MG ? (float)(1 << s.lev) : 1.f, gb = MG ? gl / s.inc : 1.f;
            float ddx, ddy, ddz;
            if (g.reflect == 1) {
              // specular: |d| per axis unchanged, the y component flips
              ddx = s.sx > 0 ? gb * g.DX / s.tsx : (s.sx < 0 ? -gb * g.DX / s.tsx : 0.f);
              ddz = s.sz > 0 ? gb * g.DZ / s.tsz : (s.sz < 0 ? -gb * g.DZ / s.tsz : 0.f);
              const float ady = yfs ? 1.f / s.tsy : gb * g.DY / s.tsy;
              ddy = wl == 0 ? ady : -ady;
            } else {
              // Lambertian: cos(theta) = sqrt(U), azimuth 2 pi U (block 2 + k)
              const uint4 v = philox10r(make_uint4(s.cellid, s.ray, 2u + s.nrefl, g.snapw), a.rkey);
              const float mr = sqrtf(unif(v.x));
              float sp, cp;
              sincos_2pi(unif(v.y), sp, cp);
              const float sr = sqrtf(fmaxf(0.f, 1.f - mr * mr));
              ddx = sr * cp;
              ddy = wl == 0 ? mr : -mr;
              ddz = sr * sp;
            }
            ++s.nrefl;
            axis_setup(ddx, nfx, gl * g.DX, s.sx, s.t0x, s.tsx);
            axis_setup(ddy, nfy, yfs ? dyl(s.iy, MG ? s.lev : 0) : gl * g.DY, s.sy, s.t0y, s.tsy);
            axis_setup(ddz, nfz, gl * g.DZ, s.sz, s.t0z, s.tsz);
            if (yfs && s.sy != 0) s.tsy = __frcp_rn(fabsf(ddy));
            s.cntx = s.cnty = s.cntz = 0.f;
            s.tnx = s.t0x;
            s.tny = s.t0y;
            s.tnz = s.t0z;
            s.tprev = 0.f;
            if (MG) s.inc = 1.f;
          }
        }
      }
      if (MG && !done && s.lev + 1 < a.mg_levels && s.lsteps >= a.mg_steps) {
        // multigrid (Section 4.3): fall onto the next coarser grid here.  Its
        // faces are the even-numbered faces of this grid, so an axis whose
        // next face is odd-numbered skips it; the cell is the one containing
        // this one.
        if (s.sx != 0 && ((s.sx > 0 ? s.ix + 1 : s.ix) & 1)) {
          s.cntx += s.inc;
          s.tnx = fmaf(s.cntx, s.tsx, s.t0x);
        }
        if (s.sy != 0 && ((s.sy > 0 ? s.iy + 1 : s.iy) & 1)) {
          if (yfs) {
            s.tny += dyl(s.sy > 0 ? s.iy + 1 : s.iy - 1, s.lev) * s.tsy;  // the skipped row's height
          } else {
            s.cnty += s.inc;
            s.tny = fmaf(s.cnty, s.tsy, s.t0y);
          }
        }
        if (s.sz != 0 && ((s.sz > 0 ? s.iz + 1 : s.iz) & 1)) {
          s.cntz += s.inc;
          s.tnz = fmaf(s.cntz, s.tsz, s.t0z);
        }
        s.loff += (unsigned)(nxyl * nzl);
        s.ix >>= 1;
        s.iy >>= 1;
        s.iz >>= 1;
        s.lin = (unsigned)(s.ix + (nxl >> 1) * (s.iy + (nyl >> 1) * s.iz));
        s.inc *= 2.f;
        ++s.lev;
        s.lsteps = 0;
      }
    }
    if (!MG && !done && s.steps >= a.long_steps && (s.steps == a.long_steps || ax == 1) &&
        long_flight(s.tny, s.tprev, s.tsx, s.tsz, a.long_flight)) {
      // a long flight ahead (a grazing ray of a thin band): the warp-parallel
      // march of long_rays.cu finishes this ray; checked when the ray reaches
      // long_steps segments and at each later y face (a reflection is one)
      LongRay L;
      L.t0x = s.t0x; L.t0y = s.t0y; L.t0z = s.t0z; L.tsx = s.tsx;
      L.tsy = s.tsy; L.tsz = s.tsz; L.cntx = s.cntx; L.cnty = s.cnty;
      L.cntz = s.cntz; L.tnx = s.tnx; L.tny = s.tny; L.tnz = s.tnz;
      L.tprev = s.tprev; L.tau = s.tau; L.X = s.X; L.B_i = s.B_i;
      L.B_last = s.B_last; L.scale = s.scale; L.krow = s.krow; L.n = s.n;
      L.ix = s.ix; L.iy = s.iy; L.iz = s.iz;
      L.signs = (unsigned)(s.sx + 1) | ((unsigned)(s.sy + 1) << 2) | ((unsigned)(s.sz + 1) << 4);
      L.lin = s.lin; L.slot = s.slot; L.r = s.r; L.ray = s.ray;
      L.cellid = s.cellid; L.steps = (unsigned)s.steps; L.nrefl = s.nrefl; L.snap = BATCH ? (unsigned)snapshot_of(starts, a.nsnaps, a.chunk_p0 + s.slot) : 0u;
      if (hand_off(a, L)) s.active = false;
    }
    // the next step's field entry, loaded now so that its latency overlaps the
    // rest of this march round
    if (!done && s.active) s.fcur = __ldg(field + (MG ? s.loff + s.lin : s.lin));
    if (done) {
      if (s.tau > 0.f) s.X += (s.B_i - s.B_last) * s.tau;  // residual dump (Algorithm 1)
      if (AR) {
        // the residual is absorbed in the last medium cell crossed (the row is
        // clamped: after a wall event iy lies outside the grid)
        const int jres = min(max(s.iy, 0), g.ny - 1);
        const unsigned lres = (unsigned)(s.ix + g.nx * (jres + g.ny * s.iz));
        if (s.tau > 0.f && lres != s.cellid)
          atomicAdd(a.armc_acc + armc_slot(a, s.r, lres),
                    f32_to_f64(-s.scale * ((s.B_i - s.B_last) * s.tau) * volume_ratio(yfs, g.nx, g.ny, s.cellid, jres)));
        atomicAdd(a.ermc_acc + armc_slot(a, s.r, s.cellid), f32_to_f64(s.scale * s.X));
      }
      Ybuf[(size_t)s.slot * (unsigned)N + s.r] = s.scale * s.X;  // the ray's sample Y (Eq. 14)
      if (a.ray_steps) a.ray_steps[(size_t)s.slot * (unsigned)N + s.r] = (unsigned)s.steps;
      if (a.steps_cell) {
        if ((int)s.slot != ls.acc_slot) {
          if (ls.acc_slot >= 0 && ls.acc_steps) atomicAdd(a.step_acc + ls.acc_slot, (unsigned long long)ls.acc_steps);
          ls.acc_slot = (int)s.slot;
          ls.acc_steps = 0;
        }
        ls.acc_steps += (unsigned)s.steps;
      }
      ls.tot_steps += (unsigned long long)s.steps;
      ls.max_ray = max(ls.max_ray, (unsigned)s.steps);
      ++ls.tot_rays;
      s.active = false;
    }
  }
}

// ---- binary64 per-cell tallies (Eq. 8: Q_i is the mean of the samples) -------
//
// Binary64 Neumaier summation of every sample would keep GB300's narrow binary64
// pipe busy for longer than the trace itself, so the tally is built in two
// stages that give binary64 accuracy at a few binary64 operations per 32
// samples:
//  1. a tile of 32 consecutive samples of one cell is summed EXACTLY in 64-bit
//     fixed point (integer arithmetic): each binary32 y = m 2^(e - 150) is
//     shifted to the unit 2^(E - 184), E the tile's largest exponent field, and
//     its square m^2 2^(2e - 300) to the unit 2^(2E - 310).  Bits below the unit
//     are dropped (at most one unit per sample: 2^-57 of the tile's largest |y|,
//     2^-56 of its largest y^2); 32 terms below 2^58 in magnitude cannot overflow;
//  2. each tile sum is rounded once to binary64 (the integer-to-binary64
//     conversion, then an exact power-of-two scaling) and added to its
//     segment's running sum with Neumaier's compensated summation in binary64
//     (a segment: a run of up to 64 consecutive tiles, tally_segments);
//  3. the segments' sums are added in order the same way (one segment for
//     N <= 2048: the cell sum is that segment's sum).
// The result is within about 2^-51 of sum |y| (and of sum y^2) of the exact sums
// of the binary32 samples -- binary64 quality -- and the order is fixed (samples
// 0..N-1 of the cell, tile by tile, segment by segment), so it never depends on
// the launch, nor on whether a cell's segments are summed by one warp or many.

// s + c += b (Neumaier).  |s| >= |b| is decided on the bit patterns (integer
// compare of the magnitudes; both finite).
__device__ __forceinline__ void neumaier_add(double &s, double &c, double b) {
  const double t = s + b;
  const unsigned long long ms = (unsigned long long)__double_as_longlong(s) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long mb = (unsigned long long)__double_as_longlong(b) & 0x7FFFFFFFFFFFFFFFull;
  const bool ge = ms >= mb;
  const double big = ge ? s : b, small = ge ? b : s;
  c += (big - t) + small;
  s = t;
}

// 2^k as a binary64 for k in [-1022, 1023] (exact, built from its bits).
__device__ __forceinline__ double pow2d(int k) {
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// Exact sums of 32 binary32 values v[0..31] and of their squares (stage 1),
// rounded to binary64 (stage 2's input).  Sets `bad` when a value is not finite.
// Each value enters as its signed significand placed at bit 34 of a 64-bit word
// and shifted right (arithmetically) by its exponent's distance d from the
// largest; its square as m^2 placed at bit 10 and shifted right by 2d.
__device__ __forceinline__ void tile_sums_exact(const unsigned (&v)[32], double &s1, double &s2, bool &bad) {
  unsigned vmax = 0u;  // largest magnitude's bits: the largest exponent field
#pragma unroll
  for (int k = 0; k < 32; ++k) vmax = max(vmax, v[k] & 0x7FFFFFFFu);
  const unsigned E = max(vmax >> 23, 1u);
  bad |= E == 0xFFu;
  long long acc = 0;
  unsigned long long acc2 = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const unsigned e = (v[k] >> 23) & 0xFFu;
    const unsigned m = (v[k] & 0x7FFFFFu) | (e ? 0x800000u : 0u);
    const unsigned d = E - max(e, 1u);  // >= 0
    // y in units of 2^(E - 184): (+-m 2^34) >> d, truncated towards -inf
    const int sm = (int)v[k] < 0 ? -(int)m : (int)m;
    acc += ((long long)sm << 34) >> min(d, 63u);
    // y^2 in units of 2^(2E - 310): (m^2 2^10) >> 2d
    acc2 += (((unsigned long long)m * m) << 10) >> min(2u * d, 63u);
  }
  const int Ei = (int)min(E, 254u);
  s1 = __ll2double_rn(acc) * pow2d(Ei - 184);
  s2 = __ull2double_rn(acc2) * pow2d(2 * Ei - 310);
}

// One tally segment of the warp's cells: lane c owns the cell whose N samples
// start at y0 + c * N when bit c of `cells` is set, and gets the compensated
// sums s + c of the exact sums of its tiles t0 .. t1 - 1 (of y and of y^2).
// Tiles of 32 samples are staged through the warp's shared-memory tile
// ([cell][sample], rows padded to 36 words: the row stores and the lanes' 16-byte
// row reads are conflict-free) from coalesced loads of each cell's 32
// consecutive samples (128 bytes, streaming hint: read once).  `bad` is set when
// a sample is not finite.
__device__ __forceinline__ void warp_segment64(const float *__restrict__ y0, int N, unsigned cells, int lane,
                                               float (*tile)[36], int t0, int t1, double &v1, double &v2,
                                               bool &bad) {
  double s = 0.0, c = 0.0, s2 = 0.0, c2 = 0.0;
  const bool mine = (cells >> lane) & 1u;
  for (int t = t0; t < t1; ++t) {
    const int r0 = t * 32;
    const bool in = r0 + lane < N;
    float ld[32];
#pragma unroll
    for (int cc = 0; cc < 32; ++cc)
      ld[cc] = ((cells >> cc) & 1u) && in ? __ldcs(y0 + (size_t)cc * (unsigned)N + (unsigned)(r0 + lane)) : 0.f;
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) tile[cc][lane] = ld[cc];
    __syncwarp();
    if (mine) {
      unsigned v[32];
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        const float4 f = *reinterpret_cast<const float4 *>(&tile[lane][k]);
        v[k] = __float_as_uint(f.x);
        v[k + 1] = __float_as_uint(f.y);
        v[k + 2] = __float_as_uint(f.z);
        v[k + 3] = __float_as_uint(f.w);
      }
      double t1s, t2s;
      tile_sums_exact(v, t1s, t2s, bad);
      neumaier_add(s, c, t1s);
      neumaier_add(s2, c2, t2s);
    }
    __syncwarp();
  }
  v1 = s + c;
  v2 = s2 + c2;
}

// Binary64 tallies of the warp's cells (cells, tiles and staging as in
// warp_segment64): the tiles' exact sums added in order within each segment
// (tally_segments), the segments' sums in order across them (the same bits as
// warp_segment64 per segment followed by combine_segments_kernel).  Returns the
// lane's sum of y and of y^2 (NaN when a sample is not finite); lanes without a
// cell return zeros.
__device__ __forceinline__ void warp_tally64(const float *__restrict__ y0, int N, unsigned cells, int lane,
                                             float (*tile)[36], double &sum, double &sum2) {
  double S = 0.0, C = 0.0, S2 = 0.0, C2 = 0.0;  // over segments
  double s = 0.0, c = 0.0, s2 = 0.0, c2 = 0.0;  // within the current segment
  bool bad = false;
  const bool mine = (cells >> lane) & 1u;
  const int ntile = (N + 31) / 32, L = tally_seg_len(ntile);
  for (int r0 = 0, t = 0; r0 < N; r0 += 32, ++t) {
    const bool in = r0 + lane < N;
    float ld[32];
#pragma unroll
    for (int cc = 0; cc < 32; ++cc)
      ld[cc] = ((cells >> cc) & 1u) && in ? __ldcs(y0 + (size_t)cc * (unsigned)N + (unsigned)(r0 + lane)) : 0.f;
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) tile[cc][lane] = ld[cc];
    __syncwarp();
    if (mine) {
      unsigned v[32];
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        const float4 f = *reinterpret_cast<const float4 *>(&tile[lane][k]);
        v[k] = __float_as_uint(f.x);
        v[k + 1] = __float_as_uint(f.y);
        v[k + 2] = __float_as_uint(f.z);
        v[k + 3] = __float_as_uint(f.w);
      }
      double t1, t2;
      tile_sums_exact(v, t1, t2, bad);
      neumaier_add(s, c, t1);
      neumaier_add(s2, c2, t2);
      if ((t + 1) % L == 0 || t == ntile - 1) {  // the segment's last tile
        neumaier_add(S, C, s + c);
        neumaier_add(S2, C2, s2 + c2);
        s = c = s2 = c2 = 0.0;
      }
    }
    __syncwarp();
  }
  sum = bad ? __longlong_as_double(0x7FF8000000000000ll) : S + C;
  sum2 = bad ? sum : S2 + C2;
}

}  // namespace
}  // namespace mcrt

// Batched FP32 solve: many snapshots (fields of possibly different grid sizes
// that share the k-distribution) in ONE persistent trace launch and one
// per-cell reduction.  Warps claim runs of brick-ordered positions from the
// concatenation of all snapshots (the largest first); the estimator, the ring
// scheduling and the fixed-order reduction are those of trace_fp32.cu, so every
// snapshot's result equals its own single solve bit for bit.  Kept apart from
// trace_fp32.cu so that the single-solve kernel does not carry the snapshot
// bookkeeping.
#include <math.h>
#include <stdint.h>

#include "draws.cuh"
#include "mcrt_internal.h"
#include "trace_common.cuh"

namespace mcrt {
namespace {

// The FP32 trace kernel of trace_fp32.cu, run as one persistent launch over the
// snapshots a.snaps.  Every warp works on one snapshot at a time and lets its
// rays finish before it moves to the next one, so the snapshot's grid, fields,
// walls and proposal are warp-uniform values.  MG: the multigrid march of
// Section 4.3.
// GEN: some snapshot has stretched y faces; the uniform variant drops the
// row-height lookups from the step.
template <int MINB, int KSTEPS, bool MG, bool GEN>
__global__ void __launch_bounds__(WARPS * 32, MINB) trace_batch_kernel(const TraceArgs a) {
  constexpr bool BATCH = true;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpRing *rings = reinterpret_cast<WarpRing *>(smem_raw);
  const bool plain = a.snaps[0].cell_cn == nullptr;
  // plain-proposal counts and guide table: staged in shared memory when they fit
  // (counts_in_smem bit 0); a per-cell proposal is staged per warp, one emitting
  // cell at a time (bit 1), in the same space
  const unsigned long long *s_cn = a.cn, *s_cg = a.cg;
  const unsigned short *s_guide = a.guide;
  const bool cell_stage = !plain && (a.counts_in_smem & 2);
  unsigned long long *w_cn = reinterpret_cast<unsigned long long *>(smem_raw + WARPS * sizeof(WarpRing)) +
                             (size_t)(threadIdx.x >> 5) * (a.nb + a.nb * a.ng);
  unsigned long long *w_cg = w_cn + a.nb;
  // batched solves: the table of snapshot starts follows the per-warp slices of
  // the per-cell proposal (present only when cells are staged)
  const size_t wslice = cell_stage ? sizeof(unsigned long long) * (size_t)(a.nb + a.nb * a.ng) : 0;
  long long *starts = reinterpret_cast<long long *>(smem_raw + WARPS * sizeof(WarpRing) + WARPS * wslice);
  if (BATCH) {
    for (int i = threadIdx.x; i <= a.nsnaps; i += blockDim.x)
      starts[i] = a.snaps[i].p0;  // snaps[nsnaps].p0 is the end of the last snapshot
  } else if (plain && (a.counts_in_smem & 1)) {
    unsigned long long *cn_sh = reinterpret_cast<unsigned long long *>(smem_raw + WARPS * sizeof(WarpRing));
    unsigned short *g_sh = reinterpret_cast<unsigned short *>(cn_sh + a.nb + a.nb * a.ng);
    const int ncount = a.nb + a.nb * a.ng;
    for (int i = threadIdx.x; i < ncount; i += blockDim.x)
      cn_sh[i] = i < a.nb ? a.cn[i] : a.cg[i - a.nb];
    for (int i = threadIdx.x; i < GUIDE; i += blockDim.x) g_sh[i] = a.guide[i];
    s_cn = cn_sh;
    s_cg = cn_sh + a.nb;
    s_guide = g_sh;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  WarpRing &R = rings[threadIdx.x >> 5];
  const unsigned lt_mask = (1u << lane) - 1u;
  // Runs of brick-order positions are claimed from a launch-wide counter
  // (counters[6], zeroed before each launch): a warp whose cells hold longer rays
  // takes fewer cells, and the runs keep neighbouring cells together.
  // positions per claim: about claim_rays rays (at least one cell), and at
  // least 8 claims per warp
  const long long G = max(1LL, min((long long)((a.claim_rays > 0 ? a.claim_rays : 1024) / a.rays),
                                   (a.chunk_p1 - a.chunk_p0) / ((long long)gridDim.x * WARPS * 8)));
  long long p_next = 0, p_end = 0;

  const int nb = a.nb, ng = a.ng, nT = a.nT, N = a.rays;
  const float4 *__restrict__ kbtab = a.kbtab32;  // {kappa, slope, B, slope} per (n, g, t)
  const float tol = a.tol32;
  // the grid, fields, walls and proposal of the snapshot being solved (a batch
  // loads them when a warp moves to another snapshot; a single solve never does)
  int nx = a.nx, ny = a.ny, nz = a.nz, nxy = nx * ny;
  int bi0_b = 0, bj0_b = 0, bk0_b = 0, bnx_b = 0, bny_b = 0, bnz_b = 0;
  const uint2 *__restrict__ field = a.fpos32;
  float DX = a.dx32, DY = a.dy32, DZ = a.dz32;
  const float *__restrict__ yfs = a.yf32;
  float eps0 = a.eps32[0], eps1 = a.eps32[1];
  const float *__restrict__ bwall_b = nullptr;
  const float *__restrict__ wgt_b = nullptr;
  const unsigned long long *__restrict__ ccn_b = nullptr;
  const unsigned long long *__restrict__ ccg_b = nullptr;
  const unsigned *__restrict__ chemi_b = nullptr;
  int reflect_b = 0;
  unsigned snapw_b = 0;
  long long sp0 = 0, sp1 = BATCH ? 0 : 0x7fffffffffffffffLL;  // positions of this snapshot
  bool pending = false;  // the next claimed position lies in another snapshot
  // stretched y (faces non-null): tsy holds 1/|d_y| and each y crossing adds the
  // next row's height; the height of row j of grid l from the faces
  auto dyl = [&](int j, int l) -> float {
    return __ldg(yfs + ((unsigned)(j + 1) << l)) - __ldg(yfs + ((unsigned)j << l));
  };
  float *__restrict__ Ybuf = a.ybuf;
  const unsigned long long ray_off = a.ray_offset_dev ? *a.ray_offset_dev : a.ray_offset;

  // warp-uniform: the emitting cell being initialised, its next ray, and (per-cell
  // proposal) its hemisphere count
  int c_bx = 0, c_by = 0, c_bz = 0, c_lin = 0, c_slot = 0, c_r = N;
  unsigned c_hemi = 4194304u;
  bool exhausted = false;
  unsigned head = 0, tail = 0;  // ring positions (mod POOL)

  // per-lane ray registers
  bool active = false;
  // table and field indices are unsigned: widening them to 64-bit addresses is
  // free, while sign-extending an int costs a conversion on GB300's narrow pipe
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
  unsigned long long tot_steps = 0;
  unsigned tot_cap = 0, tot_wall = 0, max_ray = 0, tot_rays = 0;
  int acc_slot = -1;  // run of steps for the per-cell step counts
  unsigned acc_steps = 0;

  for (;;) {
    bool progress = false;
    if (BATCH && pending && tail == head && !__any_sync(0xffffffffu, active)) {
      // every ray of the previous snapshot has finished: take over the snapshot
      // that owns the next claimed position
      const int snap_i = snapshot_of(starts, a.nsnaps, p_next);
      const SnapArgs &sn = a.snaps[snap_i];
      nx = sn.nx;
      ny = sn.ny;
      nz = sn.nz;
      nxy = nx * ny;
      bnx_b = nx;
      bny_b = ny;
      bnz_b = nz;
      bi0_b = bj0_b = bk0_b = 0;
      field = sn.fpos32;
      DX = sn.dx;
      DY = sn.dy;
      DZ = sn.dz;
      yfs = sn.yf32;
      eps0 = sn.eps0;
      eps1 = sn.eps1;
      bwall_b = sn.bwall32;
      wgt_b = sn.wgt32;
      ccn_b = sn.cell_cn;
      ccg_b = sn.cell_cg;
      chemi_b = sn.cell_hemi;
      reflect_b = sn.reflect;
      snapw_b = sn.snapshot;
      sp0 = sn.p0;
      sp1 = starts[snap_i + 1];
      // the plain proposal's counts are read through L1 (shared memory stays
      // small, leaving L1 to the field gathers)
      s_cn = sn.cn;
      s_cg = sn.cg;
      s_guide = sn.guide;
      pending = false;
      progress = true;
    }
    // ---- A. converged initialisation of up to 32 rays of one cell ----
    if ((int)(tail - head) <= POOL - 32 && !exhausted && !pending) {
      progress = true;
      if (c_r >= N) {  // next emitting cell of this warp's brick-ordered run
        bool found = false;
        long long p = p_next;
        for (;;) {
          // a batch moves to another snapshot only once this one's rays are done
          if (BATCH && p < p_end && (p < sp0 || p >= sp1)) break;
          while (!found && p < p_end && (!BATCH || p < sp1)) {
            found = brick_cell_d(bnx_b, bny_b, bnz_b,
                                 p - sp0, c_bx, c_by, c_bz);
            ++p;
          }
          if (found) break;
          if (BATCH && p < p_end) break;
          unsigned long long base = 0;  // claim the next run (warp-uniform)
          if (lane == 0) base = atomicAdd(a.counters + 6, (unsigned long long)G);
          base = __shfl_sync(0xffffffffu, base, 0);
          p = a.chunk_p0 + (long long)base;
          p_end = min(a.chunk_p1, p + G);
          if (p >= a.chunk_p1) break;
        }
        p_next = p;
        if (found) {
          c_r = 0;
          c_slot = (int)(p - 1 - a.chunk_p0);
          c_lin = (bi0_b + c_bx) +
                  nx * ((bj0_b + c_by) + ny * (bk0_b + c_bz));
          if (!plain) {
            c_hemi = __ldg(chemi_b + c_lin);
            if (cell_stage) {  // all of this cell's rays are initialised before the next cell's
              const unsigned long long *gcn = ccn_b + (size_t)c_lin * nb;
              const unsigned long long *gcg = ccg_b + (size_t)c_lin * nb * ng;
              for (int i = lane; i < nb; i += 32) w_cn[i] = __ldg(gcn + i);
              for (int i = lane; i < nb * ng; i += 32) w_cg[i] = __ldg(gcg + i);
              __syncwarp();
            }
          }
        } else if (BATCH && p < p_end) {
          pending = true;  // the run continues in another snapshot
        } else {
          exhausted = true;
        }
      }
      if (!exhausted && !pending) {
        const int rr = c_r + lane;
        if (rr < N) {
          const unsigned cell = (unsigned)c_lin;
          const unsigned rayid = (unsigned)(ray_off + (unsigned long long)rr);
          const uint2 fi = __ldg(field + cell);
          unsigned it_i;
          float fr_i;
          tpos(fi.x, it_i, fr_i);
          const uint4 u = philox10r(make_uint4(cell, rayid, 0u, snapw_b), a.rkey);
          unsigned hemi = 4194304u;
          int nn, gg;
          float wgt;
          if (plain) {
            nn = pick_guided(s_cn, s_guide, u.z);
            gg = pick(s_cg + nn * ng, ng, u.w);
          } else if (cell_stage) {
            hemi = c_hemi;
            nn = pick(w_cn, nb, u.z);
            gg = pick(w_cg + nn * ng, ng, u.w);
          } else {
            hemi = c_hemi;
            const unsigned long long *cn = ccn_b + (size_t)cell * nb;
            const unsigned long long *cgn0 = ccg_b + (size_t)cell * nb * ng;
            nn = pick(cn, nb, u.z);
            gg = pick(cgn0 + (size_t)nn * ng, ng, u.w);
          }
          // direction: hemisphere of the y axis by the integer count `hemi` of
          // 2^23, mu uniform inside it (plain: mu = 1 - 2 U); phi = 2 pi R_phi
          const unsigned m0 = u.x >> 9;
          const bool up = m0 < hemi;
          const float h = u23_to_float(up ? hemi : 8388608u - hemi);
          // the plain proposal's hemisphere count is 2^22, whose reciprocal is
          // exact; a per-cell count takes a correctly rounded reciprocal (a
          // warp-uniform branch, so the plain path never evaluates it)
          float rh = 2.384185791015625e-07f;
          if (!plain) rh = __frcp_rn(h);
          const float mt = (u23_to_float(up ? m0 : m0 - hemi) + 0.5f) * rh;
          const float mu = up ? 1.f - mt : -mt;
          const float ph = h * 1.1920928955078125e-07f;
          if (plain) {
            wgt = __ldg(wgt_b + nn * ng + gg);
          } else {
            const unsigned long long *cn = cell_stage ? w_cn : ccn_b + (size_t)cell * nb;
            const unsigned long long *cgn =
                cell_stage ? w_cg + nn * ng : ccg_b + ((size_t)cell * nb + nn) * ng;
            const unsigned long long mn = cn[nn] - (nn ? cn[nn - 1] : 0ull);
            const unsigned long long mg = cgn[gg] - (gg ? cgn[gg - 1] : 0ull);
            const float p = u33_to_float(mn) * 2.3283064365386963e-10f * (u33_to_float(mg) * 2.3283064365386963e-10f);
            wgt = __fdividef(__ldg(a.w_g32 + gg), p) * __fdividef(6.2831855f, ph);
          }
          float sphi, cphi;
          sincos_2pi(unif(u.y), sphi, cphi);
          const float st = sqrtf(fmaxf(0.f, 1.f - mu * mu));
          float fx = 0.5f, fy = 0.5f, fz = 0.5f;
          if (a.origin == 0) {
            const uint4 v = philox10r(make_uint4(cell, rayid, 1u, snapw_b), a.rkey);
            fx = unif(v.x);
            fy = unif(v.y);
            fz = unif(v.z);
          }
          const float4 kbi = __ldg(kbtab + ((unsigned)(nn * ng + gg) * (unsigned)nT + it_i));
          const float kap_i = (kbi.x + fr_i * kbi.y) * __uint_as_float(fi.y);
          int ssx, ssy, ssz;
          float a0x, a0y, a0z, asx, asy, asz;
          axis_setup(st * cphi, fx, DX, ssx, a0x, asx);
          axis_setup(mu, fy, yfs ? dyl(bj0_b + c_by, 0) : DY, ssy, a0y, asy);
          axis_setup(st * sphi, fz, DZ, ssz, a0z, asz);
          if (yfs && ssy != 0) asy = __frcp_rn(fabsf(mu));
          const int pos = (tail + lane) & (POOL - 1);
          R.A[pos] = make_float4(a0x, a0y, a0z, asx);
          R.B[pos] = make_float4(asy, asz, kbi.z + fr_i * kbi.w, wgt * kap_i);
          const unsigned flags = (unsigned)(ssx + 1) | ((unsigned)(ssy + 1) << 2) |
                                 ((unsigned)(ssz + 1) << 4);
          R.C[pos] = make_uint4((unsigned)nn | ((unsigned)gg << 16), rayid, flags, cell);
          R.D[pos] = make_int4(c_slot, bi0_b + c_bx, bj0_b + c_by,
                               bk0_b + c_bz);
        }
        tail += (unsigned)min(32, N - c_r);
        c_r += 32;
      }
      __syncwarp();
    }

    // ---- B. idle lanes take prepared rays ----
    // The take-over runs on the idle lanes only, so a warp waits until REFILL of
    // its lanes are idle (or it is draining): one pass then serves more rays, at
    // the cost of a round or two with idle lanes (2.6% less time at 64^3 x 1000
    // rays than a take-over in every round).
    const unsigned idle = __ballot_sync(0xffffffffu, !active);
    const int avail = (int)(tail - head);
    if (idle && avail > 0 && (__popc(idle) >= REFILL || idle == 0xffffffffu || exhausted || pending)) {
      progress = true;
      const int rank = __popc(idle & lt_mask);
      if (!active && rank < avail) {
        const int pos = (head + rank) & (POOL - 1);
        const float4 A = R.A[pos];
        const float4 Bv = R.B[pos];
        const uint4 Cv = R.C[pos];
        const int4 Dv = R.D[pos];
        t0x = A.x;
        t0y = A.y;
        t0z = A.z;
        tsx = A.w;
        tsy = Bv.x;
        tsz = Bv.y;
        B_i = Bv.z;
        scale = Bv.w;
        n = Cv.x & 0xffffu;
        krow = (n * (unsigned)ng + (Cv.x >> 16)) * (unsigned)nT;
        ray = Cv.y;
        sx = (int)(Cv.z & 3u) - 1;
        sy = (int)((Cv.z >> 2) & 3u) - 1;
        sz = (int)((Cv.z >> 4) & 3u) - 1;
        cellid = Cv.w;
        lin = Cv.w;
        slot = (unsigned)Dv.x;
        ix = Dv.y;
        iy = Dv.z;
        iz = Dv.w;
        r = ray - (unsigned)ray_off;
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
        fcur = __ldg(field + lin);
        if (MG) {
          lev = 0;
          lsteps = 0;
          loff = 0;
          inc = 1.f;
        }
      }
      head += (unsigned)min(__popc(idle), avail);
      __syncwarp();
    }

    const unsigned busy = __ballot_sync(0xffffffffu, active);
    if (!busy && exhausted && tail == head) break;
    if (busy) progress = true;

    // ---- C. up to KSTEPS march steps per active lane (Algorithm 1 "March") ----
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
      const uint2 f = fcur;
      unsigned it;
      float fr;
      tpos(f.x, it, fr);
      const float4 kb = __ldg(kbtab + (krow + it));
      const float kap = (kb.x + fr * kb.y) * __uint_as_float(f.y);
      const float Bj = kb.z + fr * kb.w;
      float alpha, trans;
      absorb(kap * ds, alpha, trans);
      X += (B_i - Bj) * (tau * alpha);  // Eq. 14 term / kappa_i
      tau *= trans;                     // Eq. 3
      B_last = Bj;
      ++steps;
      if (MG) ++lsteps;
      bool done = tau <= tol;
      if (!done && steps >= a.max_steps) {
        done = true;
        ++tot_cap;
      }
      if (!done) {
        tprev = tn;
        // dimensions of the current grid
        const int nxl = MG ? nx >> lev : nx, nyl = MG ? ny >> lev : ny, nzl = MG ? nz >> lev : nz;
        const int nxyl = MG ? nxl * nyl : nxy;
        {
          // branch-free advance of the crossed axis (lanes cross different axes)
          const bool mx = ax == 0, my = ax == 1, mz = ax == 2;
          const float step = MG ? inc : 1.f;
          cntx += mx ? step : 0.f;
          cnty += my ? step : 0.f;
          cntz += mz ? step : 0.f;
          tnx = mx ? fmaf(cntx, tsx, t0x) : tnx;
          tny = my ? fmaf(cnty, tsy, t0y) : tny;
          tnz = mz ? fmaf(cntz, tsz, t0z) : tnz;
          ix += mx ? sx : 0;
          iy += my ? sy : 0;
          iz += mz ? sz : 0;
          if (GEN && yfs && my && (unsigned)iy < (unsigned)nyl) tny = tprev + dyl(iy, MG ? lev : 0) * tsy;
          // periodic wrap: an index can only leave the grid in the ray's direction
          const int wx = (unsigned)ix < (unsigned)nxl ? 0 : -sx * nxl;
          ix += wx;
          const int wz = (unsigned)iz < (unsigned)nzl ? 0 : -sz * nzl;
          iz += wz;
          // the linear index from the three indices (multiply-adds, off the ALU pipe)
          lin = (unsigned)(ix + nxl * (iy + nyl * iz));
          if ((unsigned)iy >= (unsigned)nyl) {
            // wall: absorbs eps of the ray and emits at T_wall (Eq. 3 wall factor)
            const int wl = iy < 0 ? 0 : 1;
            const float eps = wl ? eps1 : eps0;
            const float Bw = __ldg(bwall_b + ((unsigned)(wl * nb) + n));
            X += (B_i - Bw) * (tau * eps);
            tau *= 1.f - eps;
            ++tot_wall;
            if (eps >= 1.f || tau <= tol) {
              done = true;
            } else {
              // fractions of the current grid's cell, whose extent along an
              // axis is inc face steps of the axis parameters
              const float cx = MG ? tsx * inc : tsx, cz = MG ? tsz * inc : tsz;
              float nfx = 0.5f, nfz = 0.5f;
              if (sx > 0)
                nfx = 1.f - (tnx - tprev) / cx;
              else if (sx < 0)
                nfx = (tnx - tprev) / cx;
              if (sz > 0)
                nfz = 1.f - (tnz - tprev) / cz;
              else if (sz < 0)
                nfz = (tnz - tprev) / cz;
              nfx = fminf(fmaxf(nfx, 0.f), 1.f);
              nfz = fminf(fmaxf(nfz, 0.f), 1.f);
              const float nfy = wl == 0 ? 0.f : 1.f;
              iy = wl == 0 ? 0 : nyl - 1;
              lin = (unsigned)(ix + nxl * iy + nxyl * iz);
              // cell size of the current grid over the finest, and of the grid
              // the axis parameters were set up on
              const float gl = MG ? (float)(1 << lev) : 1.f, gb = MG ? gl / inc : 1.f;
              float ddx, ddy, ddz;
              if (reflect_b == 1) {
                // specular: |d| per axis unchanged, the y component flips
                ddx = sx > 0 ? gb * DX / tsx : (sx < 0 ? -gb * DX / tsx : 0.f);
                ddz = sz > 0 ? gb * DZ / tsz : (sz < 0 ? -gb * DZ / tsz : 0.f);
                const float ady = yfs ? 1.f / tsy : gb * DY / tsy;
                ddy = wl == 0 ? ady : -ady;
              } else {
                // Lambertian: cos(theta) = sqrt(U), azimuth 2 pi U (block 2 + k)
                const uint4 v = philox10r(make_uint4(cellid, ray, 2u + nrefl, snapw_b), a.rkey);
                const float mr = sqrtf(unif(v.x));
                float sp, cp;
                sincos_2pi(unif(v.y), sp, cp);
                const float sr = sqrtf(fmaxf(0.f, 1.f - mr * mr));
                ddx = sr * cp;
                ddy = wl == 0 ? mr : -mr;
                ddz = sr * sp;
              }
              ++nrefl;
              axis_setup(ddx, nfx, gl * DX, sx, t0x, tsx);
              axis_setup(ddy, nfy, yfs ? dyl(iy, MG ? lev : 0) : gl * DY, sy, t0y, tsy);
              axis_setup(ddz, nfz, gl * DZ, sz, t0z, tsz);
              if (yfs && sy != 0) tsy = __frcp_rn(fabsf(ddy));
              cntx = cnty = cntz = 0.f;
              tnx = t0x;
              tny = t0y;
              tnz = t0z;
              tprev = 0.f;
              if (MG) inc = 1.f;
            }
          }
        }
        if (MG && !done && lev + 1 < a.mg_levels && lsteps >= a.mg_steps) {
          // multigrid (Section 4.3): fall onto the next coarser grid here.  Its
          // faces are the even-numbered faces of this grid, so an axis whose
          // next face is odd-numbered skips it; the cell is the one containing
          // this one.
          if (sx != 0 && ((sx > 0 ? ix + 1 : ix) & 1)) {
            cntx += inc;
            tnx = fmaf(cntx, tsx, t0x);
          }
          if (sy != 0 && ((sy > 0 ? iy + 1 : iy) & 1)) {
            if (yfs) {
              tny += dyl(sy > 0 ? iy + 1 : iy - 1, lev) * tsy;  // the skipped row's height
            } else {
              cnty += inc;
              tny = fmaf(cnty, tsy, t0y);
            }
          }
          if (sz != 0 && ((sz > 0 ? iz + 1 : iz) & 1)) {
            cntz += inc;
            tnz = fmaf(cntz, tsz, t0z);
          }
          loff += (unsigned)(nxyl * nzl);
          ix >>= 1;
          iy >>= 1;
          iz >>= 1;
          lin = (unsigned)(ix + (nxl >> 1) * (iy + (nyl >> 1) * iz));
          inc *= 2.f;
          ++lev;
          lsteps = 0;
        }
      }
      if (!MG && !done && steps >= a.long_steps && (steps == a.long_steps || ax == 1) &&
          long_flight(tny, tprev, tsx, tsz, a.long_flight)) {
        // a long flight ahead (a grazing ray of a thin band): the warp-parallel
        // march of long_rays.cu finishes this ray; checked when the ray reaches
        // long_steps segments and at each later y face (a reflection is one)
        LongRay L;
        L.t0x = t0x; L.t0y = t0y; L.t0z = t0z; L.tsx = tsx;
        L.tsy = tsy; L.tsz = tsz; L.cntx = cntx; L.cnty = cnty;
        L.cntz = cntz; L.tnx = tnx; L.tny = tny; L.tnz = tnz;
        L.tprev = tprev; L.tau = tau; L.X = X; L.B_i = B_i;
        L.B_last = B_last; L.scale = scale; L.krow = krow; L.n = n;
        L.ix = ix; L.iy = iy; L.iz = iz;
        L.signs = (unsigned)(sx + 1) | ((unsigned)(sy + 1) << 2) | ((unsigned)(sz + 1) << 4);
        L.lin = lin; L.slot = slot; L.r = r; L.ray = ray;
        L.cellid = cellid; L.steps = (unsigned)steps; L.nrefl = nrefl; L.snap = (unsigned)snapshot_of(starts, a.nsnaps, a.chunk_p0 + slot);
        if (hand_off(a, L)) active = false;
      }
      // the next step's field entry, loaded now so that its latency overlaps the
      // rest of this march round
      if (!done && active) fcur = __ldg(field + (MG ? loff + lin : lin));
      if (done) {
        if (tau > 0.f) X += (B_i - B_last) * tau;  // residual dump (Algorithm 1)
        Ybuf[(size_t)slot * (unsigned)N + r] = scale * X;  // the ray's sample Y (Eq. 14)
        if (a.ray_steps) a.ray_steps[(size_t)slot * (unsigned)N + r] = (unsigned)steps;
        if (a.steps_cell) {
          if ((int)slot != acc_slot) {
            if (acc_slot >= 0 && acc_steps) atomicAdd(a.step_acc + acc_slot, (unsigned long long)acc_steps);
            acc_slot = (int)slot;
            acc_steps = 0;
          }
          acc_steps += (unsigned)steps;
        }
        tot_steps += (unsigned long long)steps;
        max_ray = max(max_ray, (unsigned)steps);
        ++tot_rays;
        active = false;
      }
    }
    if (!progress) {  // unreachable by construction; never spin
      if (lane == 0) atomicOr(a.counters + 5, 1ull);
      break;
    }
  }
  if (a.steps_cell && acc_slot >= 0 && acc_steps)
    atomicAdd(a.step_acc + acc_slot, (unsigned long long)acc_steps);

#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    tot_steps += __shfl_xor_sync(0xffffffffu, tot_steps, off);
    tot_cap += __shfl_xor_sync(0xffffffffu, tot_cap, off);
    tot_wall += __shfl_xor_sync(0xffffffffu, tot_wall, off);
    max_ray = max(max_ray, __shfl_xor_sync(0xffffffffu, max_ray, off));
    tot_rays += __shfl_xor_sync(0xffffffffu, tot_rays, off);
  }
  if (lane == 0 && tot_rays) {
    atomicAdd(a.counters + 0, tot_steps);
    atomicAdd(a.counters + 3, (unsigned long long)tot_rays);
    if (tot_cap) atomicAdd(a.counters + 1, (unsigned long long)tot_cap);
    if (tot_wall) atomicAdd(a.counters + 2, (unsigned long long)tot_wall);
    atomicMax(a.counters + 4, (unsigned long long)max_ray);
  }
}

// Per-cell reduction of a batched launch (as reduce_cells_kernel of
// trace_fp32.cu: lane c of a warp takes the cell at chunk position c and sums its
// N samples in order into binary64 tallies, warp_tally64); each position goes
// to the outputs of the snapshot that owns it.  The order never depends on
// scheduling, so Q and sigma are reproducible bit for bit and equal the single
// solve's.
__global__ void __launch_bounds__(256) reduce_cells_batch_kernel(const TraceArgs a) {
  __shared__ __align__(16) float tiles[WARPS][32][36];
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int N = a.rays;
  const long long P = a.chunk_p1 - a.chunk_p0;
  for (long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < P;
       base += nwarps * 32) {
    int bx = 0, by = 0, bz = 0;
    long long bc = 0;
    double *oq = nullptr, *osig = nullptr;
    bool mine = false;
    if (base + lane < P) {
      const long long pos = a.chunk_p0 + base + lane;
      int lo = 0, hi = a.nsnaps - 1;  // the owning snapshot (binary search over the start positions)
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.snaps[mid].p0 <= pos)
          lo = mid;
        else
          hi = mid - 1;
      }
      const SnapArgs &sn = a.snaps[lo];
      mine = brick_cell_d(sn.nx, sn.ny, sn.nz, pos - sn.p0, bx, by, bz);
      bc = bx + (long long)sn.nx * (by + (long long)sn.ny * bz);
      oq = sn.q;
      osig = sn.sigma;
    }
    const unsigned cells = __ballot_sync(0xffffffffu, mine);
    if (!cells) continue;  // warp-uniform
    double S, S2;
    warp_tally64(a.ybuf + (size_t)base * (unsigned)N, N, cells, lane, tiles[threadIdx.x >> 5], S, S2);
    if (mine) {
      const double Nd = (double)N;
      const double Q = S / Nd;
      oq[bc] = Q;
      if (osig) osig[bc] = N > 1 ? sqrt(fmax(S2 / Nd - Q * Q, 0.0) / (Nd - 1.0)) : 0.0;
    }
  }
}

// The binary32 tally of a batched launch, on request (mcrt_tuning.tally_binary32;
// as reduce_cells32_kernel of trace_fp32.cu).
__global__ void __launch_bounds__(256) reduce_cells_batch32_kernel(const TraceArgs a) {
  constexpr bool BATCH = true;
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int N = a.rays;
  const long long P = a.chunk_p1 - a.chunk_p0;
  for (long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < P;
       base += nwarps * 32) {
    float mh = 0.f, ml = 0.f, mh2 = 0.f, ml2 = 0.f;
    bool mine = false;
    long long mbc = 0;
    double *mq = a.q, *msig = a.sigma;
    const int ncell = (int)min(32LL, P - base);
    for (int c = 0; c < ncell; ++c) {
      int bx, by, bz;
      const long long pos = a.chunk_p0 + base + c;
      long long bc;
      double *oq = a.q, *osig = a.sigma;
      if (BATCH) {
        // the owning snapshot (binary search over the start positions)
        int lo = 0, hi = a.nsnaps - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.snaps[mid].p0 <= pos)
            lo = mid;
          else
            hi = mid - 1;
        }
        const SnapArgs &sn = a.snaps[lo];
        if (!brick_cell_d(sn.nx, sn.ny, sn.nz, pos - sn.p0, bx, by, bz)) continue;  // warp-uniform
        bc = bx + (long long)sn.nx * (by + (long long)sn.ny * bz);
        oq = sn.q;
        osig = sn.sigma;
      } else {
        if (!brick_cell(a, pos, bx, by, bz)) continue;  // warp-uniform
        bc = bx + (long long)a.bnx * (by + (long long)a.bny * bz);
      }
      float hi, lo, hi2, lo2;
      warp_cell_sums(a.ybuf + (size_t)(base + c) * N, N, lane, hi, lo, hi2, lo2);
      if (lane == c) {
        mh = hi; ml = lo; mh2 = hi2; ml2 = lo2;
        mine = true;
        mbc = bc;
        mq = oq;
        msig = osig;
      }
    }
    if (mine) {
      const double S = (double)mh + (double)ml, S2 = (double)mh2 + (double)ml2;
      const double Nd = (double)N;
      const double Q = S / Nd;
      mq[mbc] = Q;
      if (msig) msig[mbc] = N > 1 ? sqrt(fmax(S2 / Nd - Q * Q, 0.0) / (Nd - 1.0)) : 0.0;
      if (!BATCH && a.steps_cell) a.steps_cell[mbc] = a.step_acc[base + lane];
    }
  }
}

template <int MINB, int KSTEPS, bool MG, bool GEN>
cudaError_t configure_variant(size_t smem, int *bps, int *nsm) {
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
    e = cudaFuncSetAttribute(trace_batch_kernel<MINB, KSTEPS, MG, GEN>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[dev],
                                                      trace_batch_kernel<MINB, KSTEPS, MG, GEN>, WARPS * 32,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm[dev] < 1) blocks_per_sm[dev] = 1;
    configured_smem[dev] = (int)smem;
  }
  *bps = blocks_per_sm[dev];
  *nsm = num_sms[dev];
  return cudaSuccess;
}

template <int MINB, int KSTEPS, bool MG, bool GEN>
cudaError_t launch_variant(const TraceArgs &a, cudaStream_t s, size_t smem) {
  // per-device launch shape, computed once per device and shared-memory size
  int bps = 0, nsm = 0;
  cudaError_t e = configure_variant<MINB, KSTEPS, MG, GEN>(smem, &bps, &nsm);
  if (e != cudaSuccess) return e;
  const long long P = a.chunk_p1 - a.chunk_p0;
  const long long need = (P + WARPS - 1) / WARPS;
  long long blocks = a.grid_blocks > 0 ? a.grid_blocks : (long long)nsm * bps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  trace_batch_kernel<MINB, KSTEPS, MG, GEN><<<(unsigned)blocks, WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int fp32_batch_max_snapshots() { return 1024; }

// Ring states, one slice per warp for its snapshot's counts and guide table, and
// the table of snapshot start positions.
static size_t fp32_batch_smem_bytes(int nb, int ng, int nsnaps, int counts_in_smem) {
  const size_t wslice = (counts_in_smem & 2) ? sizeof(unsigned long long) * (size_t)(nb + nb * ng) : 0;
  return WARPS * sizeof(WarpRing) + WARPS * wslice + sizeof(long long) * (size_t)(nsnaps + 1);
}

// CTAs per SM (3 when min_blocks >= 3, else 2), march steps per refill round (2
// when steps_per_round >= 2, else 1), multigrid, stretched snapshots.  prepare =
// true sets the variant's launch attributes; false launches it.
template <bool MG, bool GEN>
cudaError_t run_batch_variant(bool prepare, const TraceArgs *a, bool mb3, bool k2, cudaStream_t s, size_t smem,
                              int *bps, int *nsm) {
  if (prepare) {
    if (mb3) return k2 ? configure_variant<3, 2, MG, GEN>(smem, bps, nsm) : configure_variant<3, 1, MG, GEN>(smem, bps, nsm);
    return k2 ? configure_variant<2, 2, MG, GEN>(smem, bps, nsm) : configure_variant<2, 1, MG, GEN>(smem, bps, nsm);
  }
  if (mb3) return k2 ? launch_variant<3, 2, MG, GEN>(*a, s, smem) : launch_variant<3, 1, MG, GEN>(*a, s, smem);
  return k2 ? launch_variant<2, 2, MG, GEN>(*a, s, smem) : launch_variant<2, 1, MG, GEN>(*a, s, smem);
}

static cudaError_t batch_dispatch(bool prepare, const TraceArgs *a, int min_blocks, int steps_per_round,
                                  bool multigrid, bool stretched, cudaStream_t s, size_t smem, int *bps, int *nsm) {
  const bool mb3 = min_blocks >= 3, k2 = steps_per_round >= 2;
  if (multigrid)
    return stretched ? run_batch_variant<true, true>(prepare, a, mb3, k2, s, smem, bps, nsm)
                     : run_batch_variant<true, false>(prepare, a, mb3, k2, s, smem, bps, nsm);
  return stretched ? run_batch_variant<false, true>(prepare, a, mb3, k2, s, smem, bps, nsm)
                   : run_batch_variant<false, false>(prepare, a, mb3, k2, s, smem, bps, nsm);
}

cudaError_t prepare_trace_fp32_batch(int min_blocks, int steps_per_round, int nb, int ng, int nsnaps,
                                     int counts_in_smem, int multigrid, int *blocks_per_sm, int *num_sms) {
  const size_t smem = fp32_batch_smem_bytes(nb, ng, nsnaps, counts_in_smem);
  // both geometry variants: the captured launch takes one of them
  int bps_gen = 0, nsm_gen = 0;
  cudaError_t e = batch_dispatch(true, nullptr, min_blocks, steps_per_round, multigrid != 0, true, nullptr, smem,
                                 &bps_gen, &nsm_gen);
  if (e != cudaSuccess) return e;
  return batch_dispatch(true, nullptr, min_blocks, steps_per_round, multigrid != 0, false, nullptr, smem,
                        blocks_per_sm, num_sms);
}

cudaError_t launch_trace_fp32_batch(const TraceArgs &args, int min_blocks, int steps_per_round,
                                    cudaStream_t s) {
  if (args.chunk_p1 <= args.chunk_p0) return cudaSuccess;
  TraceArgs a = args;
  if (!long_rays_on(a)) a.long_steps = 0x7fffffff;  // no hand-off
  const size_t smem = fp32_batch_smem_bytes(a.nb, a.ng, a.nsnaps, a.counts_in_smem);
  cudaError_t e = cudaMemsetAsync(a.counters + 6, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  e = batch_dispatch(false, &a, min_blocks, steps_per_round, a.mg_levels > 1, a.batch_stretched != 0, s, smem,
                     nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (long_rays_on(a)) {
    e = launch_long_rays(a, s);
    if (e != cudaSuccess) return e;
  }
  const long long P = a.chunk_p1 - a.chunk_p0;
  long long blocks = ((P + 31) / 32 + 7) / 8;  // one warp per 32 positions
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();
  if (a.tally32)
    reduce_cells_batch32_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  else
    reduce_cells_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mcrt

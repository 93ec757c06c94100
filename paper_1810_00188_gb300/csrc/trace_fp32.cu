// FP32 ERMC ray-trace kernel (converged initialisation, lane refill) and the
// per-cell reduction of its samples.
//
// Same estimator as trace.cu (Silvestri & Pecnik, arXiv:1810.00188: Eqs. 2, 3,
// 12-17 and Algorithm 1), scheduled for the SIMT machine.  The paper identifies
// warp divergence from rays of very different lengths as the dominant loss of a
// GPU ERMC (Section 4.2) and reorders rays by absorption coefficient; here the
// divergence is removed structurally:
//
//  * emitting cells are enumerated in 8x8x8-brick order and warps claim short
//    runs of them from a launch-wide counter, with all their rays (rays travel a
//    few cells on average, so an SM's field gathers stay in L1, and a warp whose
//    cells hold long rays takes fewer cells);
//  * ray initialisation (Philox draws, band/g sampling, direction, origin, the
//    emitting cell's kappa and B, the DDA set-up) runs converged: 32 lanes
//    initialise 32 rays at once into a per-warp ring of prepared states in
//    shared memory;
//  * the march advances every active lane by up to KSTEPS cells per round; a lane
//    whose ray ends stores its sample Y and takes the next prepared state; the
//    field entry of the next cell is loaded a step ahead, and kappa and B of the
//    ray's (n, g) come in one 16-byte load from an interleaved table;
//  * the channel geometry (uniform y, periodic x and z) is a compile-time
//    variant whose step has no stretched-face or closed-box tests;
//  * a ray that has marched long_steps segments with a long flight ahead (a
//    grazing ray of a thin band, up to ~10^5 steps) is handed to the
//    warp-parallel march of long_rays.cu instead of holding its lane to the end;
//  * samples go to a scratch array indexed by (cell, ray); reduce_cells_kernel
//    sums each cell's samples in a fixed order into binary64 tallies (exact
//    32-sample tiles, Neumaier-compensated binary64 sums), so Q and sigma do
//    not depend on scheduling, launch shape or box.
//
// GB300 issues binary64 arithmetic and int<->float conversions on a narrow pipe,
// so the per-ray and per-step code uses neither: ray weights come from a
// host-built FP64 table rounded once, each cell's table position is precomputed
// (tpos), tol, the cell sizes and the wall emissivities arrive as binary32 copies
// (converting the binary64 launch arguments in the kernel put a binary64
// conversion wherever the compiler rematerialised them: 18M of them in a 48^3
// solve, the binary64 pipe 37% busy), and the remaining conversions are exact bit
// constructions (unif, u23_to_float).
//
// A round that makes no progress cannot happen; if it did, the warp sets an
// error flag (counters[5]) and returns instead of spinning.  Warps claim runs
// of cells from a launch-wide counter (counters[6]).
#include <math.h>
#include <stdint.h>

#include "draws.cuh"
#include "mcrt_internal.h"
#include "trace_common.cuh"

namespace mcrt {
namespace {

// GEN: the general geometry (stretched y faces, closed-box x and z walls).  The
// channel variant (uniform y, periodic x and z) drops those tests from the step.
// AR: the absorption-based estimate (Section 2, ARMC): besides its own sample,
// each ray deposits, into every other cell it crosses, minus the term it adds to
// its own cell's emission-based estimate (the exchange seen from the absorbing
// cell), its residual into the last cell it crossed, and its wall terms into
// its own cell; deposits go to per-batch binary64 sums (batch = ray index mod K)
// with atomic adds, and the ray's sample to its cell's per-batch emission-based
// sum; on a stretched grid each deposit carries the volume ratio of the emitting
// and the absorbing cell.  One grid; a ray handed to the long-ray march makes
// its remaining deposits there.
template <int MINB, int KSTEPS, bool MG, bool GEN, bool AR = false>
__global__ void __launch_bounds__(WARPS * 32, MINB) trace_fp32_kernel(const TraceArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpRing *rings = reinterpret_cast<WarpRing *>(smem_raw);
  const bool plain = a.cell_cn == nullptr;
  // plain-proposal counts and guide table: staged in shared memory when they fit
  // (counts_in_smem bit 0); a per-cell proposal is staged per warp, one emitting
  // cell at a time (bit 1), in the same space
  const unsigned long long *s_cn = a.cn, *s_cg = a.cg;
  const unsigned short *s_guide = a.guide;
  const unsigned char *s_gg = a.gguide;
  const bool cell_stage = !plain && (a.counts_in_smem & 2);
  unsigned long long *w_cn = reinterpret_cast<unsigned long long *>(smem_raw + WARPS * sizeof(WarpRing)) +
                             (size_t)(threadIdx.x >> 5) * (a.nb + a.nb * a.ng);
  unsigned long long *w_cg = w_cn + a.nb;
  if (plain && (a.counts_in_smem & 1)) {
    unsigned long long *cn_sh = reinterpret_cast<unsigned long long *>(smem_raw + WARPS * sizeof(WarpRing));
    unsigned short *g_sh = reinterpret_cast<unsigned short *>(cn_sh + a.nb + a.nb * a.ng);
    const int ncount = a.nb + a.nb * a.ng;
    for (int i = threadIdx.x; i < ncount; i += blockDim.x)
      cn_sh[i] = i < a.nb ? a.cn[i] : a.cg[i - a.nb];
    for (int i = threadIdx.x; i < GUIDE; i += blockDim.x) g_sh[i] = a.guide[i];
    unsigned char *gg_sh = reinterpret_cast<unsigned char *>(g_sh + GUIDE);
    for (int i = threadIdx.x; i < a.nb * GG; i += blockDim.x) gg_sh[i] = a.gguide[i];
    s_cn = cn_sh;
    s_cg = cn_sh + a.nb;
    s_guide = g_sh;
    s_gg = gg_sh;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  WarpRing &R = rings[threadIdx.x >> 5];
  const unsigned lt_mask = (1u << lane) - 1u;
  // Runs of brick-order positions are claimed from a launch-wide counter
  // (counters[6], zeroed before each launch): a warp whose cells hold longer rays
  // takes fewer cells, and the runs keep neighbouring cells together.
  // positions per claim: about claim_rays rays (at least one cell), and at
  // least 8 claims per warp.  A cell with more rays than that is claimed in
  // nblk blocks of equal size RB (a multiple of 32; claim k: block k mod nblk of
  // position k / nblk), so that a chunk of few cells with many rays each still
  // spreads over every warp; the samples, and so Q and sigma, do not depend on
  // who traces which rays.
  const int claim = a.claim_rays > 0 ? a.claim_rays : 1024;
  const int RB0 = (claim + 31) / 32 * 32;
  const bool by_block = a.rays > RB0;
  const long long nblk = by_block ? (a.rays + RB0 - 1) / RB0 : 1;
  const int RB = by_block ? (int)(((a.rays + nblk - 1) / nblk + 31) / 32 * 32) : RB0;  // blocks of equal size
  const long long G = max(1LL, min((long long)(claim / a.rays),
                                   (a.chunk_p1 - a.chunk_p0) / ((long long)gridDim.x * WARPS * 8)));
  long long p_next = 0, p_end = 0;

  const int nx = a.nx, ny = a.ny, nz = a.nz, nxy = nx * ny, nb = a.nb,
            ng = a.ng, nT = a.nT, N = a.rays;
  const uint2 *__restrict__ field = a.fpos32;
  const float4 *__restrict__ kbtab = a.kbtab32;  // {kappa, slope, B, slope} per (n, g, t)
  const float tol = a.tol32;
  const float DX = a.dx32, DY = a.dy32, DZ = a.dz32;
  // stretched y (faces non-null): tsy holds 1/|d_y| and each y crossing adds the
  // next row's height; the height of row j of grid l from the faces
  const float *__restrict__ yfs = GEN ? a.yf32 : nullptr;
  auto dyl = [&](int j, int l) -> float {
    return __ldg(yfs + ((unsigned)(j + 1) << l)) - __ldg(yfs + ((unsigned)j << l));
  };
  const float eps0 = a.eps32[0], eps1 = a.eps32[1];
  float *__restrict__ Ybuf = a.ybuf;
  const unsigned long long ray_off = a.ray_offset_dev ? *a.ray_offset_dev : a.ray_offset;

  // warp-uniform: the emitting cell being initialised, its next ray, and (per-cell
  // proposal) its hemisphere count
  int c_bx = 0, c_by = 0, c_bz = 0, c_lin = 0, c_slot = 0, c_r = N, c_end = N;
  unsigned c_hemi = 4194304u;
  // 1 / (hemisphere count) of each hemisphere, per cell (the plain proposal's
  // 2^22 has the exact reciprocal 2^-22): one correctly rounded reciprocal per
  // cell instead of one per ray
  float c_rup = 2.384185791015625e-07f, c_rdn = 2.384185791015625e-07f;
  bool exhausted = false;
  unsigned head = 0, tail = 0;  // ring positions (mod POOL)

  // the lane's ray and counts; the grid the march reads
  LaneRay lr;
  LaneStats ls;
  const MarchGrid mg_grid{nx, ny, nz, nxy, field, yfs, a.bwall32, DX, DY, DZ, eps0, eps1, a.reflect,
                          a.snapshot};

  for (;;) {
    bool progress = false;
    // ---- A. converged initialisation of up to 32 rays of one cell ----
    if ((int)(tail - head) <= POOL - 32 && !exhausted) {
      progress = true;
      if (c_r >= c_end) {  // next emitting cell of this warp's brick-ordered run
        bool found = false;
        long long p = p_next;
        int r0 = 0;
        if (by_block) {
          for (;;) {  // claim the next block of one cell's rays (warp-uniform)
            unsigned long long k = 0;
            if (lane == 0) k = atomicAdd(a.counters + 6, 1ull);
            k = __shfl_sync(0xffffffffu, k, 0);
            p = a.chunk_p0 + (long long)(k / (unsigned long long)nblk);
            if (p >= a.chunk_p1) break;
            found = brick_cell(a, p, c_bx, c_by, c_bz);
            ++p;
            if (found) {
              r0 = (int)(k % (unsigned long long)nblk) * RB;
              break;
            }
          }
        } else {
          for (;;) {
            while (!found && p < p_end) {
              found = brick_cell(a, p, c_bx, c_by, c_bz);
              ++p;
            }
            if (found) break;
            unsigned long long base = 0;  // claim the next run (warp-uniform)
            if (lane == 0) base = atomicAdd(a.counters + 6, (unsigned long long)G);
            base = __shfl_sync(0xffffffffu, base, 0);
            p = a.chunk_p0 + (long long)base;
            p_end = min(a.chunk_p1, p + G);
            if (p >= a.chunk_p1) break;
          }
        }
        p_next = p;
        if (found) {
          c_r = r0;
          c_end = min(N, r0 + (by_block ? RB : N));
          c_slot = (int)(p - 1 - a.chunk_p0);
          c_lin = (a.bi0 + c_bx) + nx * ((a.bj0 + c_by) + ny * (a.bk0 + c_bz));
          c_rup = c_rdn = 2.384185791015625e-07f;
          if (!plain) {
            c_hemi = __ldg(a.cell_hemi + c_lin);
            c_rup = __frcp_rn(u23_to_float(c_hemi));
            c_rdn = __frcp_rn(u23_to_float(8388608u - c_hemi));
            if (cell_stage) {  // all of this cell's rays are initialised before the next cell's
              const unsigned long long *gcn = a.cell_cn + (size_t)c_lin * nb;
              const unsigned long long *gcg = a.cell_cg + (size_t)c_lin * nb * ng;
              for (int i = lane; i < nb; i += 32) w_cn[i] = __ldg(gcn + i);
              for (int i = lane; i < nb * ng; i += 32) w_cg[i] = __ldg(gcg + i);
              __syncwarp();
            }
          }
        } else {
          exhausted = true;
        }
      }
      if (!exhausted) {
        const int rr = c_r + lane;
        bool keep = false, inst = false;  // through the ring and the march / ended in its cell
        float4 sA, sB;
        unsigned sCx = 0u, sCz = 0u;
        if (rr < c_end) {
          const unsigned cell = (unsigned)c_lin;
          const unsigned rayid = (unsigned)(ray_off + (unsigned long long)rr);
          const uint2 fi = __ldg(field + cell);
          unsigned it_i;
          float fr_i;
          tpos(fi.x, it_i, fr_i);
          const uint4 u = philox10r(make_uint4(cell, rayid, 0u, a.snapshot), a.rkey);
          unsigned hemi = 4194304u;
          int nn, gg;
          float wgt;
          if (plain) {
            nn = pick_guided(s_cn, s_guide, u.z);
            gg = pick_gguided(s_cg + nn * ng, s_gg + nn * GG, u.w);
          } else if (cell_stage) {
            hemi = c_hemi;
            nn = pick(w_cn, nb, u.z);
            gg = pick(w_cg + nn * ng, ng, u.w);
          } else {
            hemi = c_hemi;
            const unsigned long long *cn = a.cell_cn + (size_t)cell * nb;
            const unsigned long long *cgn0 = a.cell_cg + (size_t)cell * nb * ng;
            nn = pick(cn, nb, u.z);
            gg = pick(cgn0 + (size_t)nn * ng, ng, u.w);
          }
          // direction: hemisphere of the y axis by the integer count `hemi` of
          // 2^23, mu uniform inside it (plain: mu = 1 - 2 U); phi = 2 pi R_phi
          const unsigned m0 = u.x >> 9;
          const bool up = m0 < hemi;
          const float h = u23_to_float(up ? hemi : 8388608u - hemi);
          const float mt = (u23_to_float(up ? m0 : m0 - hemi) + 0.5f) * (up ? c_rup : c_rdn);
          const float mu = up ? 1.f - mt : -mt;
          const float ph = h * 1.1920928955078125e-07f;
          if (plain) {
            wgt = __ldg(a.wgt32 + nn * ng + gg);
          } else {
            const unsigned long long *cn = cell_stage ? w_cn : a.cell_cn + (size_t)cell * nb;
            const unsigned long long *cgn =
                cell_stage ? w_cg + nn * ng : a.cell_cg + ((size_t)cell * nb + nn) * ng;
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
            const uint4 v = philox10r(make_uint4(cell, rayid, 1u, a.snapshot), a.rkey);
            fx = unif(v.x);
            fy = unif(v.y);
            fz = unif(v.z);
          }
          const float4 kbi = __ldg(kbtab + ((unsigned)(nn * ng + gg) * (unsigned)nT + it_i));
          const float kap_i = (kbi.x + fr_i * kbi.y) * __uint_as_float(fi.y);
          int ssx, ssy, ssz;
          float a0x, a0y, a0z, asx, asy, asz;
          axis_setup(st * cphi, fx, DX, ssx, a0x, asx);
          axis_setup(mu, fy, yfs ? dyl(a.bj0 + c_by, 0) : DY, ssy, a0y, asy);
          axis_setup(st * sphi, fz, DZ, ssz, a0z, asz);
          if (yfs && ssy != 0) asy = __frcp_rn(fabsf(mu));
          // A ray whose first segment, inside its own cell, leaves tau <= tol ends
          // there with X = 0 exactly: that segment's B_j is B_i and the residual
          // dump uses B_last = B_i.  Its sample (0) and its one step are recorded
          // below from the same expressions the march evaluates (same bits), and
          // the ray skips the ring and the march (about 40% of the rays of the
          // 64^3 channel: optically thick bands).
          float al0, tr0;
          absorb(kap_i * fminf(fminf(a0x, a0y), a0z), al0, tr0);
          inst = tr0 <= tol;
          keep = !inst;
          sA = make_float4(a0x, a0y, a0z, asx);
          sB = make_float4(asy, asz, kbi.z + fr_i * kbi.w, wgt * kap_i);
          sCx = (unsigned)nn | ((unsigned)gg << 16);
          sCz = (unsigned)(ssx + 1) | ((unsigned)(ssy + 1) << 2) | ((unsigned)(ssz + 1) << 4);
        }
        // the rays that go on are packed into the ring in lane order (the ray
        // index and the cell are rebuilt here rather than held across the ballot)
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
          const int pos = (tail + __popc(km & lt_mask)) & (POOL - 1);
          R.A[pos] = sA;
          R.B[pos] = sB;
          R.C[pos] = make_uint4(sCx, (unsigned)(ray_off + (unsigned long long)rr), sCz, (unsigned)c_lin);
          R.D[pos] = make_int4(c_slot, a.bi0 + c_bx, a.bj0 + c_by, a.bk0 + c_bz);
        }
        tail += (unsigned)__popc(km);
        if (inst) {
          Ybuf[(size_t)c_slot * (unsigned)N + (unsigned)rr] = 0.f;
          if (a.ray_steps) a.ray_steps[(size_t)c_slot * (unsigned)N + (unsigned)rr] = 1u;
          if (a.steps_cell) {
            if (c_slot != ls.acc_slot) {
              if (ls.acc_slot >= 0 && ls.acc_steps)
                atomicAdd(a.step_acc + ls.acc_slot, (unsigned long long)ls.acc_steps);
              ls.acc_slot = c_slot;
              ls.acc_steps = 0;
            }
            ls.acc_steps += 1u;
          }
          ls.tot_steps += 1ull;
          ls.max_ray = max(ls.max_ray, 1u);
          ++ls.tot_rays;
        }
        c_r += 32;
      }
      __syncwarp();
    }

    // ---- B. idle lanes take prepared rays ----
    // The take-over runs on the idle lanes only, so a warp waits until REFILL of
    // its lanes are idle (or it is draining): one pass then serves more rays, at
    // the cost of a round or two with idle lanes (2.6% less time at 64^3 x 1000
    // rays than a take-over in every round).
    const unsigned idle = __ballot_sync(0xffffffffu, !lr.active);
    const int avail = (int)(tail - head);
    if (idle && avail > 0 && (__popc(idle) >= REFILL || idle == 0xffffffffu || exhausted)) {
      progress = true;
      const int rank = __popc(idle & lt_mask);
      if (!lr.active && rank < avail) {
        const int pos = (head + rank) & (POOL - 1);
        const float4 A = R.A[pos];
        const float4 Bv = R.B[pos];
        const uint4 Cv = R.C[pos];
        const int4 Dv = R.D[pos];
        lr.t0x = A.x;
        lr.t0y = A.y;
        lr.t0z = A.z;
        lr.tsx = A.w;
        lr.tsy = Bv.x;
        lr.tsz = Bv.y;
        lr.B_i = Bv.z;
        lr.scale = Bv.w;
        lr.n = Cv.x & 0xffffu;
        lr.krow = (lr.n * (unsigned)ng + (Cv.x >> 16)) * (unsigned)nT;
        lr.ray = Cv.y;
        lr.sx = (int)(Cv.z & 3u) - 1;
        lr.sy = (int)((Cv.z >> 2) & 3u) - 1;
        lr.sz = (int)((Cv.z >> 4) & 3u) - 1;
        lr.cellid = Cv.w;
        lr.lin = Cv.w;
        lr.slot = (unsigned)Dv.x;
        lr.ix = Dv.y;
        lr.iy = Dv.z;
        lr.iz = Dv.w;
        lr.r = lr.ray - (unsigned)ray_off;
        lr.tnx = lr.t0x;
        lr.tny = lr.t0y;
        lr.tnz = lr.t0z;
        lr.cntx = lr.cnty = lr.cntz = 0.f;
        lr.tprev = 0.f;
        lr.tau = 1.f;
        lr.X = 0.f;
        lr.B_last = lr.B_i;
        lr.steps = 0;
        lr.nrefl = 0;
        lr.active = true;
        lr.fcur = __ldg(field + lr.lin);
        if (MG) {
          lr.lev = 0;
          lr.lsteps = 0;
          lr.loff = 0;
          lr.inc = 1.f;
        }
      }
      head += (unsigned)min(__popc(idle), avail);
      __syncwarp();
    }

    const unsigned busy = __ballot_sync(0xffffffffu, lr.active);
    if (!busy && exhausted && tail == head) break;
    if (busy) progress = true;

    // ---- C. up to KSTEPS march steps per active lane (Algorithm 1 "March") ----
    march_round<KSTEPS, MG, GEN, AR, false>(a, mg_grid, lr, ls);
    if (!progress) {  // unreachable by construction; never spin
      if (lane == 0) atomicOr(a.counters + 5, 1ull);
      break;
    }
  }
  if (a.steps_cell && ls.acc_slot >= 0 && ls.acc_steps)
    atomicAdd(a.step_acc + ls.acc_slot, (unsigned long long)ls.acc_steps);
  unsigned long long tot_steps = ls.tot_steps;
  unsigned tot_cap = ls.tot_cap, tot_wall = ls.tot_wall, max_ray = ls.max_ray, tot_rays = ls.tot_rays;

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

// Per-cell reduction (Eq. 8: Q_i is the mean of the cell's samples; sigma_i its
// standard error).  A warp takes 32 consecutive chunk positions, lane c the cell
// at position c, and each lane sums its cell's N samples in order into binary64
// tallies (warp_tally64: exact 32-sample tiles, Neumaier-compensated binary64
// sums).  Q = sum / N and the standard error follow in binary64.  The order
// never depends on scheduling, so Q and sigma are reproducible bit for bit.
__global__ void __launch_bounds__(256) reduce_cells_kernel(const TraceArgs a) {
  __shared__ __align__(16) float tiles[WARPS][32][36];
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int N = a.rays;
  const long long P = a.chunk_p1 - a.chunk_p0;
  for (long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < P;
       base += nwarps * 32) {
    int bx = 0, by = 0, bz = 0;
    const bool mine = base + lane < P && brick_cell(a, a.chunk_p0 + base + lane, bx, by, bz);
    const unsigned cells = __ballot_sync(0xffffffffu, mine);
    if (!cells) continue;  // warp-uniform
    double S, S2;
    warp_tally64(a.ybuf + (size_t)base * (unsigned)N, N, cells, lane, tiles[threadIdx.x >> 5], S, S2);
    if (mine) {
      const long long bc = bx + (long long)a.bnx * (by + (long long)a.bny * bz);
      const double Nd = (double)N;
      const double Q = S / Nd;
      a.q[bc] = Q;
      if (a.sigma) a.sigma[bc] = N > 1 ? sqrt(fmax(S2 / Nd - Q * Q, 0.0) / (Nd - 1.0)) : 0.0;
      if (a.steps_cell) a.steps_cell[bc] = a.step_acc[base + lane];
    }
  }
}

// The split form of reduce_cells_kernel (a.tally_part non-null, more than one
// tally segment): each segment of each group of 32 positions is an item of its
// own; its sums go to a.tally_part and combine_segments_kernel adds a cell's
// segments in order (the same bits as one warp adding them).
__global__ void __launch_bounds__(256) reduce_segments_kernel(const TraceArgs a) {
  __shared__ __align__(16) float tiles[WARPS][32][36];
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int N = a.rays;
  const long long P = a.chunk_p1 - a.chunk_p0;
  const int ntile = (N + 31) / 32, nseg = tally_segments(ntile), L = tally_seg_len(ntile);
  const long long nitems = ((P + 31) / 32) * nseg;
  for (long long item = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < nitems; item += nwarps) {
    const long long base = (item / nseg) * 32;
    const int k = (int)(item % nseg);
    int bx = 0, by = 0, bz = 0;
    const bool mine = base + lane < P && brick_cell(a, a.chunk_p0 + base + lane, bx, by, bz);
    const unsigned cells = __ballot_sync(0xffffffffu, mine);
    if (!cells) continue;  // warp-uniform
    double v1, v2;
    bool bad = false;
    warp_segment64(a.ybuf + (size_t)base * (unsigned)N, N, cells, lane, tiles[threadIdx.x >> 5], k * L,
                   min(ntile, (k + 1) * L), v1, v2, bad);
    if (mine) {
      const double nan = __longlong_as_double(0x7FF8000000000000ll);
      a.tally_part[(size_t)k * (size_t)P + (size_t)(base + lane)] = make_double2(bad ? nan : v1, bad ? nan : v2);
    }
  }
}

// The binary32 tally, on request (mcrt_tuning.tally_binary32): for each cell the
// lanes sum its N samples in a fixed order (lane l takes samples l, l + 32, ...,
// sums each batch of 8 pairwise in binary32 and adds the batch sums to
// compensated binary32 pairs, then a fixed butterfly of pair additions), and
// lane c keeps cell c's totals, converted to binary64 for Q and sigma.  Its
// error is within about 2e-7 of sum |y| (warp_cell_sums).
__global__ void __launch_bounds__(256) reduce_cells32_kernel(const TraceArgs a) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int N = a.rays;
  const long long P = a.chunk_p1 - a.chunk_p0;
  for (long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < P;
       base += nwarps * 32) {
    float mh = 0.f, ml = 0.f, mh2 = 0.f, ml2 = 0.f;
    bool mine = false;
    int mbx = 0, mby = 0, mbz = 0;
    const int ncell = (int)min(32LL, P - base);
    for (int c = 0; c < ncell; ++c) {
      int bx, by, bz;
      if (!brick_cell(a, a.chunk_p0 + base + c, bx, by, bz)) continue;  // warp-uniform
      float hi, lo, hi2, lo2;
      warp_cell_sums(a.ybuf + (size_t)(base + c) * N, N, lane, hi, lo, hi2, lo2);
      if (lane == c) {
        mh = hi; ml = lo; mh2 = hi2; ml2 = lo2;
        mine = true;
        mbx = bx; mby = by; mbz = bz;
      }
    }
    if (mine) {
      const double S = (double)mh + (double)ml, S2 = (double)mh2 + (double)ml2;
      const long long bc = mbx + (long long)a.bnx * (mby + (long long)a.bny * mbz);
      const double Nd = (double)N;
      const double Q = S / Nd;
      a.q[bc] = Q;
      if (a.sigma) a.sigma[bc] = N > 1 ? sqrt(fmax(S2 / Nd - Q * Q, 0.0) / (Nd - 1.0)) : 0.0;
      if (a.steps_cell) a.steps_cell[bc] = a.step_acc[base + lane];
    }
  }
}

// The absorption-based estimate of each cell and its combination with the
// emission-based one (Section 2), from the per-batch sums the AR trace launches
// accumulated: batch b holds the rays r = b (mod K), n_b of them per cell.
//   ARMC:   Q = sum_b A_b / N; sigma^2 = var_b(A_b / n_b) / K (batch means)
//   hybrid: lam Q_E + (1 - lam) Q_A with lam = (T - T_min) / (T_max - T_min),
//           sigma from the batch means of the combined batch estimates.
// One thread per cell; binary64.
__global__ void armc_finalize_kernel(const double *__restrict__ acc, const double *__restrict__ eacc,
                                     long long nc, int K, int N, int hybrid, const double2 *__restrict__ field,
                                     double T_min, double inv_dT, double *q, double *sigma) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    double lam = 0.0;
    if (hybrid) lam = fmin(fmax((field[c].x - T_min) * inv_dT, 0.0), 1.0);
    double sum = 0.0, mean = 0.0, m2 = 0.0;
    for (int b = 0; b < K; ++b) {
      const double nb = (double)((N - b + K - 1) / K);
      const double vb = lam * eacc[(size_t)b * nc + c] + (1.0 - lam) * acc[(size_t)b * nc + c];
      sum += vb;
      const double xb = vb / nb, d = xb - mean;  // Welford over the batch estimates
      mean += d / (double)(b + 1);
      m2 += d * (xb - mean);
    }
    q[c] = sum / (double)N;
    if (sigma) sigma[c] = K > 1 ? sqrt(m2 / ((double)(K - 1) * (double)K)) : 0.0;
  }
}

template <int MINB, int KSTEPS, bool MG, bool GEN, bool AR = false>
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
    e = cudaFuncSetAttribute(trace_fp32_kernel<MINB, KSTEPS, MG, GEN, AR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[dev],
                                                      trace_fp32_kernel<MINB, KSTEPS, MG, GEN, AR>, WARPS * 32,
                                                      smem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm[dev] < 1) blocks_per_sm[dev] = 1;
    configured_smem[dev] = (int)smem;
  }
  *bps = blocks_per_sm[dev];
  *nsm = num_sms[dev];
  return cudaSuccess;
}

template <int MINB, int KSTEPS, bool MG, bool GEN, bool AR = false>
cudaError_t launch_variant(const TraceArgs &a, cudaStream_t s, size_t smem) {
  // per-device launch shape, computed once per device and shared-memory size
  int bps = 0, nsm = 0;
  cudaError_t e = configure_variant<MINB, KSTEPS, MG, GEN, AR>(smem, &bps, &nsm);
  if (e != cudaSuccess) return e;
  const long long P = a.chunk_p1 - a.chunk_p0;
  const long long need = (P + WARPS - 1) / WARPS;
  long long blocks = a.grid_blocks > 0 ? a.grid_blocks : (long long)nsm * bps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  trace_fp32_kernel<MINB, KSTEPS, MG, GEN, AR><<<(unsigned)blocks, WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// One of the variants: CTAs per SM (1..4, default 2), march steps per refill
// round (1, 2, 4), multigrid, general geometry.  prepare = true sets the
// variant's launch attributes; false launches it.
template <bool MG, bool GEN>
cudaError_t run_variant(bool prepare, const TraceArgs *a, int min_blocks, int steps_per_round, cudaStream_t s,
                        size_t smem, int *bps, int *nsm) {
#define MCRT_V(MB, K) \
  return prepare ? configure_variant<MB, K, MG, GEN>(smem, bps, nsm) : launch_variant<MB, K, MG, GEN>(*a, s, smem)
#define MCRT_VK(MB)        \
  switch (steps_per_round) { \
    case 2: MCRT_V(MB, 2);   \
    case 4: MCRT_V(MB, 4);   \
    default: MCRT_V(MB, 1);  \
  }
  switch (min_blocks) {
    case 1: MCRT_VK(1)
    case 3: MCRT_VK(3)
    case 4: MCRT_VK(4)
    default: MCRT_VK(2)
  }
#undef MCRT_VK
#undef MCRT_V
  return cudaErrorInvalidValue;  // not reached
}

cudaError_t dispatch(bool prepare, const TraceArgs *a, int min_blocks, int steps_per_round, bool multigrid,
                     bool general, cudaStream_t s, size_t smem, int *bps, int *nsm) {
  // the absorption-based estimate: the default launch shape on one grid, the
  // channel or the general geometry (the host refuses multigrid)
  if (!prepare && a->armc_acc)
    return general ? launch_variant<3, 1, false, true, true>(*a, s, smem)
                   : launch_variant<3, 1, false, false, true>(*a, s, smem);
  if (multigrid)
    return general ? run_variant<true, true>(prepare, a, min_blocks, steps_per_round, s, smem, bps, nsm)
                   : run_variant<true, false>(prepare, a, min_blocks, steps_per_round, s, smem, bps, nsm);
  return general ? run_variant<false, true>(prepare, a, min_blocks, steps_per_round, s, smem, bps, nsm)
                 : run_variant<false, false>(prepare, a, min_blocks, steps_per_round, s, smem, bps, nsm);
}

}  // namespace

cudaError_t launch_armc_finalize(const double *acc, const double *eacc, long long nc, int K, int N,
                                 int hybrid, const double2 *field, double T_min, double T_max, double *q,
                                 double *sigma, cudaStream_t s) {
  if (nc <= 0) return cudaSuccess;
  long long blocks = (nc + 255) / 256;
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();
  const double inv = T_max > T_min ? 1.0 / (T_max - T_min) : 0.0;
  armc_finalize_kernel<<<(unsigned)blocks, 256, 0, s>>>(acc, eacc, nc, K, N, hybrid, field, T_min, inv, q,
                                                        sigma);
  return cudaGetLastError();
}

long long fp32_bricks_positions(int bnx, int bny, int bnz) {
  const long long nbx = (bnx + BRICK - 1) / BRICK, nby = (bny + BRICK - 1) / BRICK,
                  nbz = (bnz + BRICK - 1) / BRICK;
  return nbx * nby * nbz * (BRICK * BRICK * BRICK);
}

int fp32_brick_volume() { return BRICK * BRICK * BRICK; }

int fp32_guide_size() { return GUIDE; }

int fp32_guide_bits() { return GUIDE_BITS; }

int fp32_gguide_size() { return GG; }

int fp32_gguide_bits() { return GG_BITS; }

int fp32_plain_stage_fits(int nb, int ng) {
  return sizeof(unsigned long long) * (size_t)(nb + nb * ng) + sizeof(unsigned short) * GUIDE + (size_t)nb * GG <=
         48 * 1024;
}

// Ring states, then (bit 0) the plain counts and guide table or (bit 1) one
// cell's counts per warp.
static size_t fp32_smem_bytes(int nb, int ng, int counts_in_smem) {
  const size_t rows = sizeof(unsigned long long) * (size_t)(nb + nb * ng);
  const size_t plain = (counts_in_smem & 1) ? rows + sizeof(unsigned short) * GUIDE + (size_t)nb * GG : 0;
  const size_t cell = (counts_in_smem & 2) ? WARPS * rows : 0;
  return WARPS * sizeof(WarpRing) + (plain > cell ? plain : cell);
}

int fp32_cell_stage_fits(int nb, int ng) {
  return (size_t)WARPS * sizeof(unsigned long long) * (size_t)(nb + nb * ng) <= 48 * 1024;
}

cudaError_t prepare_trace_fp32(int min_blocks, int steps_per_round, int nb, int ng, int counts_in_smem,
                               int multigrid, int *blocks_per_sm, int *num_sms) {
  const size_t smem = fp32_smem_bytes(nb, ng, counts_in_smem);
  // both geometry variants: the launches that follow may take either
  int bps_gen = 0, nsm_gen = 0;
  cudaError_t e = dispatch(true, nullptr, min_blocks, steps_per_round, multigrid != 0, true, nullptr, smem,
                           &bps_gen, &nsm_gen);
  if (e != cudaSuccess) return e;
  return dispatch(true, nullptr, min_blocks, steps_per_round, multigrid != 0, false, nullptr, smem,
                  blocks_per_sm, num_sms);
}

cudaError_t launch_trace_fp32(const TraceArgs &args, int min_blocks, int steps_per_round,
                              cudaStream_t s, cudaEvent_t *marks, int *kernels) {
  if (kernels) *kernels = 0;
  if (args.chunk_p1 <= args.chunk_p0) return cudaSuccess;
  TraceArgs a = args;
  if (!long_rays_on(a)) a.long_steps = 0x7fffffff;  // no hand-off
  const size_t smem = fp32_smem_bytes(a.nb, a.ng, a.counts_in_smem);
  // the claim counter of this launch's position runs and its hand-off count
  cudaError_t e = cudaMemsetAsync(a.counters + 6, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const bool general = a.yf32 != nullptr || a.xz_walls != 0;
  if (marks && (e = cudaEventRecord(marks[0], s)) != cudaSuccess) return e;
  e = dispatch(false, &a, min_blocks, steps_per_round, a.mg_levels > 1, general, s, smem, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (marks && (e = cudaEventRecord(marks[1], s)) != cudaSuccess) return e;
  if (long_rays_on(a)) {
    e = launch_long_rays(a, s);
    if (e != cudaSuccess) return e;
  }
  if (marks && (e = cudaEventRecord(marks[2], s)) != cudaSuccess) return e;
  const long long P = a.chunk_p1 - a.chunk_p0;
  long long blocks = ((P + 31) / 32 + 7) / 8;  // one warp per 32 positions
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();
  int tally = 1;
  if (a.tally32) {
    reduce_cells32_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
  } else {
    int tma = 0;
    e = a.reduce_plain ? cudaSuccess : launch_reduce_tma(a, s, &tma);
    if (e != cudaSuccess) return e;
    if (!tma) {
      const int nseg = tally_segments((a.rays + 31) / 32);
      if (a.tally_part && nseg > 1) {  // every segment of every group an item of its own
        long long b2 = ((P + 31) / 32 * nseg + 7) / 8;
        if (b2 > grid_stride_blocks()) b2 = grid_stride_blocks();
        reduce_segments_kernel<<<(unsigned)b2, 256, 0, s>>>(a);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_combine_segments(a, s);
        if (e != cudaSuccess) return e;
        tally = 2;
      } else {
        reduce_cells_kernel<<<(unsigned)blocks, 256, 0, s>>>(a);
      }
    } else {
      tally = tma;
    }
  }
  e = cudaGetLastError();
  if (e == cudaSuccess && marks) e = cudaEventRecord(marks[3], s);
  if (e == cudaSuccess && kernels) *kernels = 1 + (long_rays_on(a) ? 1 : 0) + tally;
  return e;
}

}  // namespace mcrt

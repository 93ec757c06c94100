// The warp-parallel march of long rays.
//
// A ray of an optically thin band that runs nearly parallel to the walls makes
// up to ~10^5 steps through the periodic x and z directions before its
// transmissivity falls below tol (Algorithm 1) or it reaches a wall.  In the
// trace kernel every step waits on the previous one (field gather -> table
// gather -> exponential), about 0.3 us, so one such ray can outlast the whole
// rest of the solve.  The trace kernel therefore hands a ray off when it has
// marched long_steps segments and a long flight lies ahead (trace_common.cuh),
// and this kernel finishes it with a whole warp.
//
// Within one flight (the path between two y faces) the ray crosses only x and
// z faces, whose crossing times are fma(m, ts, t0) for consecutive integers m.
// The warp splits a window of the flight into 32 consecutive time intervals; each
// lane finds its start cell from the face counts at its start time, marches its
// interval with a local transmissivity starting at 1, and the lanes combine:
//   tau at lane j's start = tau * prod_{i<j} T_i,   X += sum_j tau_j X_j,
// which is the sum of Eq. 14 over the same segments (a segment cut by a lane
// boundary contributes twice, exp(-k s1) exp(-k s2) = exp(-k (s1 + s2))).  The
// stopping rules of Algorithm 1 (tau <= tol after a segment; max_steps) are
// found from the scans, and the lane where the ray stops re-marches its interval
// with the running values.  Flights with few crossings left, y faces and wall
// events are marched one segment at a time by the whole warp, exactly as the
// trace kernel does.  Every lane holds the same ray state; all reductions run in
// a fixed order, so a ray's result does not depend on the warp or launch.
//
// With the absorption-based estimate (AR) the march also makes the ray's
// deposits: one lane for the segments marched one at a time, the walls and the
// residual; in a window each lane walks its pieces again once the scan has given
// the transmissivity at its start, and deposits each piece's term (the two
// pieces of a segment cut at a lane boundary deposit it in two parts).
#include <math.h>
#include <stdint.h>

#include "draws.cuh"
#include "mcrt_internal.h"
#include "trace_common.cuh"

namespace mcrt {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int PIECES = 32;   // nominal x/z crossings per lane and window
constexpr int SERIAL = 32;   // flights with fewer crossings left march one segment at a time
constexpr int LANE_MAX = 8 * PIECES + 16;  // bound of a lane's loop (expected: PIECES + 2)
constexpr int GATHER = 4;    // pieces of a lane whose loads are issued together

struct Geom {
  const uint2 *field;
  const float *yfs;
  const float *bwall;
  int nx, ny, nz, reflect;
  float DX, DY, DZ, eps0, eps1;
  unsigned snapw;
};

__device__ __forceinline__ Geom geom_of(const TraceArgs &a, unsigned snap) {
  Geom g;
  if (a.snaps) {
    const SnapArgs &sn = a.snaps[snap];
    g.field = sn.fpos32;
    g.yfs = sn.yf32;
    g.bwall = sn.bwall32;
    g.nx = sn.nx;
    g.ny = sn.ny;
    g.nz = sn.nz;
    g.reflect = sn.reflect;
    g.DX = sn.dx;
    g.DY = sn.dy;
    g.DZ = sn.dz;
    g.eps0 = sn.eps0;
    g.eps1 = sn.eps1;
    g.snapw = sn.snapshot;
  } else {
    g.field = a.fpos32;
    g.yfs = a.yf32;
    g.bwall = a.bwall32;
    g.nx = a.nx;
    g.ny = a.ny;
    g.nz = a.nz;
    g.reflect = a.reflect;
    g.DX = a.dx32;
    g.DY = a.dy32;
    g.DZ = a.dz32;
    g.eps0 = a.eps32[0];
    g.eps1 = a.eps32[1];
    g.snapw = a.snapshot;
  }
  return g;
}

// kappa and B of the cell `lin` for the ray's (n, g) row (Section 2.2's linear
// interpolation in T; kappa scales with x / x_ref)
__device__ __forceinline__ void medium(const uint2 *__restrict__ field, const float4 *__restrict__ kbtab,
                                       unsigned lin, unsigned krow, float &kap, float &Bj) {
  const uint2 f = __ldg(field + lin);
  unsigned it;
  float fr;
  tpos(f.x, it, fr);
  const float4 kb = __ldg(kbtab + (krow + it));
  kap = (kb.x + fr * kb.y) * __uint_as_float(f.y);
  Bj = kb.z + fr * kb.w;
}

__device__ __forceinline__ float row_height(const float *yfs, int j) {
  return __ldg(yfs + j + 1) - __ldg(yfs + j);
}

__device__ __forceinline__ int wrap1(int i, int n) { return i >= n ? i - n : (i < 0 ? i + n : i); }

// The first crossing of an axis after time ts, counted from the window's next
// crossing index c0: the smallest m >= c0 with fma(m, ts_a, t0) > ts, its time,
// and the cell index i moved by (m - c0) faces in direction s (periodic).
__device__ __forceinline__ void first_after(float ts, float t0, float tsa, float ra, float c0, int s, int n,
                                            float &c, float &t, int &i) {
  float m = fmaxf(c0, floorf((ts - t0) * ra) + 1.f);
  for (int k = 0; k < 4 && m > c0 && fmaf(m - 1.f, tsa, t0) > ts; ++k) m -= 1.f;
  for (int k = 0; k < 4 && !(fmaf(m, tsa, t0) > ts); ++k) m += 1.f;
  const int d = (int)(m - c0) % n;
  int v = (i + s * d) % n;
  if (v < 0) v += n;
  i = v;
  c = m;
  t = fmaf(m, tsa, t0);
}

// AR: the absorption-based estimate's deposits (a.armc_acc non-null).
template <bool AR>
__global__ void __launch_bounds__(256) long_march_kernel(const TraceArgs a) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long handed = a.counters[7];
  const long long total = (long long)min(handed, (unsigned long long)a.long_cap);
  if (gw == 0 && lane == 0 && handed) {
    atomicAdd(a.counters + 8, (unsigned long long)total);
    if (handed > (unsigned long long)total) atomicAdd(a.counters + 9, handed - (unsigned long long)total);
  }
  const float4 *__restrict__ kbtab = a.kbtab32;
  const float tol = a.tol32;
  const int nb = a.nb, N = a.rays;
  const long long guard_max = 2LL * a.max_steps + 64;
  unsigned long long w_steps = 0;
  unsigned w_rays = 0, w_cap = 0, w_wall = 0, w_max = 0;

  for (long long i = gw; i < total; i += nw) {
    const LongRay L = a.long_rays[i];
    const Geom g = geom_of(a, L.snap);
    float t0x = L.t0x, t0y = L.t0y, t0z = L.t0z, tsx = L.tsx, tsy = L.tsy, tsz = L.tsz;
    float cntx = L.cntx, cnty = L.cnty, cntz = L.cntz, tnx = L.tnx, tny = L.tny, tnz = L.tnz;
    float tprev = L.tprev, tau = L.tau, X = L.X, B_last = L.B_last;
    const float B_i = L.B_i;
    const unsigned krow = L.krow;
    int ix = L.ix, iy = L.iy, iz = L.iz;
    int sx = (int)(L.signs & 3u) - 1, sy = (int)((L.signs >> 2) & 3u) - 1, sz = (int)((L.signs >> 4) & 3u) - 1;
    int steps = (int)L.steps;
    unsigned nrefl = L.nrefl, capped = 0, walls = 0;
    bool done = false;
    // the absorption-based estimate: deposits into the per-batch sums, as the
    // trace kernel makes them (one lane deposits what all lanes hold)
    auto deposit = [&](unsigned cell, float v) { atomicAdd(a.armc_acc + armc_slot(a, L.r, cell), f32_to_f64(v)); };
    // the volume ratio of the emitting cell and one in row j (stretched grids)
    auto vratio = [&](int j) { return volume_ratio(g.yfs, g.nx, g.ny, L.cellid, j); };

    // wall event at the y face just crossed (iy outside the grid): the wall
    // factor of Eq. 3, then stop or reflect, as in the trace kernel
    auto wall = [&]() {
      const int wl = iy < 0 ? 0 : 1;
      const float eps = wl ? g.eps1 : g.eps0;
      const float Bw = __ldg(g.bwall + ((unsigned)(wl * nb) + L.n));
      X += (B_i - Bw) * (tau * eps);
      if (AR && lane == 0) deposit(L.cellid, L.scale * ((B_i - Bw) * (tau * eps)));  // own exchange with the wall
      tau *= 1.f - eps;
      ++walls;
      if (eps >= 1.f || tau <= tol) {
        done = true;
        return;
      }
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
      iy = wl == 0 ? 0 : g.ny - 1;
      float ddx, ddy, ddz;
      if (g.reflect == 1) {
        ddx = sx > 0 ? g.DX / tsx : (sx < 0 ? -g.DX / tsx : 0.f);
        ddz = sz > 0 ? g.DZ / tsz : (sz < 0 ? -g.DZ / tsz : 0.f);
        const float ady = g.yfs ? 1.f / tsy : g.DY / tsy;
        ddy = wl == 0 ? ady : -ady;
      } else {
        const uint4 v = philox10r(make_uint4(L.cellid, L.ray, 2u + nrefl, g.snapw), a.rkey);
        const float mr = sqrtf(unif(v.x));
        float sp, cp;
        sincos_2pi(unif(v.y), sp, cp);
        const float sr = sqrtf(fmaxf(0.f, 1.f - mr * mr));
        ddx = sr * cp;
        ddy = wl == 0 ? mr : -mr;
        ddz = sr * sp;
      }
      ++nrefl;
      axis_setup(ddx, nfx, g.DX, sx, t0x, tsx);
      axis_setup(ddy, nfy, g.yfs ? row_height(g.yfs, iy) : g.DY, sy, t0y, tsy);
      axis_setup(ddz, nfz, g.DZ, sz, t0z, tsz);
      if (g.yfs && sy != 0) tsy = __frcp_rn(fabsf(ddy));
      cntx = cnty = cntz = 0.f;
      tnx = t0x;
      tny = t0y;
      tnz = t0z;
      tprev = 0.f;
    };
    // the y face at tny: as the trace kernel advances a y crossing
    auto cross_y = [&]() {
      cnty += 1.f;
      tny = fmaf(cnty, tsy, t0y);
      iy += sy;
      if (g.yfs && iy >= 0 && iy < g.ny) tny = tprev + row_height(g.yfs, iy) * tsy;
      if (iy < 0 || iy >= g.ny) wall();
    };

    for (long long guard = 0; !done; ++guard) {
      if (guard > guard_max) {  // unreachable: every pass advances the ray
        if (lane == 0) atomicOr(a.counters + 5, 2ull);
        break;
      }
      const float rx = __frcp_rn(tsx), rz = __frcp_rn(tsz);  // 0 on an axis not crossed
      const float rate = rx + rz;                            // x/z crossings per unit length
      const float left = (tny - tprev) * rate;               // crossings before the next y face
      if (!(left >= (float)SERIAL)) {
        // ---- one segment, exactly as the trace kernel marches it ----
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
        float kap, Bj;
        const unsigned lin = (unsigned)(ix + g.nx * (iy + g.ny * iz));
        medium(g.field, kbtab, lin, krow, kap, Bj);
        float alpha, trans;
        absorb(kap * fmaxf(tn - tprev, 0.f), alpha, trans);
        const float term = (B_i - Bj) * (tau * alpha);
        X += term;
        if (AR && lane == 0 && lin != L.cellid) deposit(lin, -L.scale * term * vratio(iy));  // absorbed in cell lin
        tau *= trans;
        B_last = Bj;
        ++steps;
        done = tau <= tol;
        if (!done && steps >= a.max_steps) {
          done = true;
          ++capped;
        }
        if (!done) {
          tprev = tn;
          if (ax == 0) {
            cntx += 1.f;
            tnx = fmaf(cntx, tsx, t0x);
            ix = wrap1(ix + sx, g.nx);
          } else if (ax == 2) {
            cntz += 1.f;
            tnz = fmaf(cntz, tsz, t0z);
            iz = wrap1(iz + sz, g.nz);
          } else {
            cross_y();
          }
        }
        continue;
      }

      // ---- a window of the flight, 32 lanes at once ----
      float t_end = tprev + (32.f * PIECES) * __frcp_rn(rate);
      const bool to_face = !(t_end < tny);  // the window reaches the next y face
      if (to_face) t_end = tny;
      const float h = (t_end - tprev) * (1.f / 32.f);
      auto bound = [&](int j) -> float {
        return j == 0 ? tprev : (j >= 32 ? t_end : fminf(fmaf((float)j, h, tprev), t_end));
      };
      const float ts = bound(lane), te = bound(lane + 1);
      // this lane's first crossings after ts and its cell there
      float cx = cntx, tx = tnx, cz = cntz, tz = tnz;
      int jx = ix, jz = iz;
      if (lane > 0) {
        if (sx != 0) first_after(ts, t0x, tsx, rx, cntx, sx, g.nx, cx, tx, jx);
        if (sz != 0) first_after(ts, t0z, tsz, rz, cntz, sz, g.nz, cz, tz, jz);
      }
      const float cx0 = cx, tx0 = tx, cz0 = cz, tz0 = tz;
      const int jx0 = jx, jz0 = jz;
      // the lane whose interval ends at the y face: a z crossing there comes
      // after the y crossing (axis order x, y, z on ties), and its last piece
      // ends a segment
      const bool y_end = to_face && lane == 31;
      const unsigned row = (unsigned)(g.nx * iy);
      const unsigned plane = (unsigned)(g.nx * g.ny);
      // pieces of this lane's interval: segments ending at a crossing count as
      // steps; the piece ending at te continues in the next lane
      float lt = 1.f, ltc = 1.f, lX = 0.f, lB = B_last;
      int lst = 0;
      bool closed = false;
      {
        // GATHER pieces at a time: their cells and lengths first (face-count
        // arithmetic only), then all their field entries, then all their table
        // rows, so that the loads of a batch are in flight together instead of
        // one piece's two dependent loads after another's; the pieces are then
        // added in order, as one at a time would add them
        float tp = ts;
        for (int k = 0; k < LANE_MAX && !closed; k += GATHER) {
          unsigned lin[GATHER];
          float len[GATHER];
          int np = 0;
          bool last_in = true;
#pragma unroll
          for (int b = 0; b < GATHER; ++b) {
            if (np == b && last_in) {
              const bool xf = tx <= tz;
              const float tn = xf ? tx : tz;
              const bool in = (xf || !y_end) ? tn <= te : tn < te;
              lin[b] = (unsigned)jx + row + plane * (unsigned)jz;
              len[b] = fmaxf((in ? tn : te) - tp, 0.f);
              np = b + 1;
              last_in = in;
              if (in) {
                if (xf) {
                  cx += 1.f;
                  tx = fmaf(cx, tsx, t0x);
                  jx = wrap1(jx + sx, g.nx);
                } else {
                  cz += 1.f;
                  tz = fmaf(cz, tsz, t0z);
                  jz = wrap1(jz + sz, g.nz);
                }
                tp = tn;
              }
            }
          }
          uint2 fe[GATHER];
#pragma unroll
          for (int b = 0; b < GATHER; ++b)
            if (b < np) fe[b] = __ldg(g.field + lin[b]);
          float4 kb[GATHER];
#pragma unroll
          for (int b = 0; b < GATHER; ++b)
            if (b < np) kb[b] = __ldg(kbtab + (krow + (fe[b].x >> 23)));
#pragma unroll
          for (int b = 0; b < GATHER; ++b) {
            if (b < np) {
              unsigned it;
              float fr;
              tpos(fe[b].x, it, fr);
              const float kap = (kb[b].x + fr * kb[b].y) * __uint_as_float(fe[b].y);
              const float Bj = kb[b].z + fr * kb[b].w;
              float alpha, trans;
              absorb(kap * len[b], alpha, trans);
              lX += (B_i - Bj) * (lt * alpha);
              lt *= trans;
              lB = Bj;
              const bool in = b < np - 1 || last_in;
              if (in || y_end) {
                ++lst;
                ltc = lt;
              }
              if (!in) closed = true;
            }
          }
        }
      }
      if (!__all_sync(FULL, closed)) {  // unreachable: an interval holds about PIECES crossings
        if (lane == 0) atomicOr(a.counters + 5, 2ull);
        break;
      }
      // exclusive product of the lanes' transmissivities, inclusive sum of their steps
      float pin = lt;
      int sinc = lst;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const float po = __shfl_up_sync(FULL, pin, off);
        const int so = __shfl_up_sync(FULL, sinc, off);
        if (lane >= off) {
          pin *= po;
          sinc += so;
        }
      }
      float pex = __shfl_up_sync(FULL, pin, 1);
      if (lane == 0) pex = 1.f;
      const float tb = tau * pex;         // transmissivity at the lane's start
      const int sb = steps + sinc - lst;  // segments before the lane
      // the first lane with a segment end where Algorithm 1 stops the ray
      const bool stop = lst > 0 && (tb * ltc <= tol || sb + lst >= a.max_steps);
      const unsigned sm = __ballot_sync(FULL, stop);
      const int js = sm ? __ffs((int)sm) - 1 : 32;
      float c = lane < js ? tb * lX : 0.f;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
      if (AR && lane < js) {
        // the deposits of this lane's pieces: the walk again, with the
        // transmissivity at its start (tb); the two pieces of a segment cut at a
        // lane boundary deposit its term in two parts
        float dcx = cx0, dtx = tx0, dcz = cz0, dtz = tz0, gt = tb, tp = ts;
        int djx = jx0, djz = jz0;
        for (int k = 0; k < LANE_MAX; ++k) {
          const bool xf = dtx <= dtz;
          const float tn = xf ? dtx : dtz;
          const bool in = (xf || !y_end) ? tn <= te : tn < te;
          float kap, Bj;
          const unsigned lin = (unsigned)djx + row + plane * (unsigned)djz;
          medium(g.field, kbtab, lin, krow, kap, Bj);
          float alpha, trans;
          absorb(kap * fmaxf((in ? tn : te) - tp, 0.f), alpha, trans);
          if (lin != L.cellid) deposit(lin, -L.scale * ((B_i - Bj) * (gt * alpha)) * vratio(iy));
          gt *= trans;
          if (!in) break;
          if (xf) {
            dcx += 1.f;
            dtx = fmaf(dcx, tsx, t0x);
            djx = wrap1(djx + sx, g.nx);
          } else {
            dcz += 1.f;
            dtz = fmaf(dcz, tsz, t0z);
            djz = wrap1(djz + sz, g.nz);
          }
          tp = tn;
        }
      }
      if (js < 32) {
        // the ray stops in lane js's interval: march it again with the running
        // transmissivity and step count, applying the stopping rules
        float gt = tb, gX = 0.f, gB = lB;
        int gs = sb;
        unsigned gcap = 0;
        if (lane == js) {
          cx = cx0;
          tx = tx0;
          cz = cz0;
          tz = tz0;
          jx = jx0;
          jz = jz0;
          float tp = ts;
          for (int k = 0; k < LANE_MAX; ++k) {
            const bool xf = tx <= tz;
            const float tn = xf ? tx : tz;
            const bool in = (xf || !y_end) ? tn <= te : tn < te;
            float kap, Bj;
            const unsigned lin = (unsigned)jx + row + plane * (unsigned)jz;
            medium(g.field, kbtab, lin, krow, kap, Bj);
            float alpha, trans;
            absorb(kap * fmaxf((in ? tn : te) - tp, 0.f), alpha, trans);
            const float term = (B_i - Bj) * (gt * alpha);
            gX += term;
            if (AR && lin != L.cellid) deposit(lin, -L.scale * term * vratio(iy));
            gt *= trans;
            gB = Bj;
            if (in || y_end) {
              ++gs;
              if (gt <= tol) break;
              if (gs >= a.max_steps) {
                gcap = 1;
                break;
              }
            }
            if (!in) break;
            if (xf) {
              cx += 1.f;
              tx = fmaf(cx, tsx, t0x);
              jx = wrap1(jx + sx, g.nx);
            } else {
              cz += 1.f;
              tz = fmaf(cz, tsz, t0z);
              jz = wrap1(jz + sz, g.nz);
            }
            tp = tn;
          }
        }
        gX = __shfl_sync(FULL, gX, js);
        gt = __shfl_sync(FULL, gt, js);
        gB = __shfl_sync(FULL, gB, js);
        gs = __shfl_sync(FULL, gs, js);
        gcap = __shfl_sync(FULL, gcap, js);
        X = (X + c) + gX;
        tau = gt;
        B_last = gB;
        steps = gs;
        capped += gcap;
        done = true;
      } else {
        X += c;
        tau *= __shfl_sync(FULL, pin, 31);
        steps += __shfl_sync(FULL, sinc, 31);
        B_last = __shfl_sync(FULL, lB, 31);
        cntx = __shfl_sync(FULL, cx, 31);
        tnx = __shfl_sync(FULL, tx, 31);
        ix = __shfl_sync(FULL, jx, 31);
        cntz = __shfl_sync(FULL, cz, 31);
        tnz = __shfl_sync(FULL, tz, 31);
        iz = __shfl_sync(FULL, jz, 31);
        tprev = t_end;
        if (to_face) cross_y();  // the segment ending at the face was counted by lane 31
      }
    }
    if (tau > 0.f) X += (B_i - B_last) * tau;  // residual dump (Algorithm 1)
    if (AR && lane == 0) {
      // the residual is absorbed in the last medium cell crossed (the row clamped
      // after a wall event); the ray's sample to its cell's emission-based sum
      const int jres = min(max(iy, 0), g.ny - 1);
      const unsigned lres = (unsigned)(ix + g.nx * (jres + g.ny * iz));
      if (tau > 0.f && lres != L.cellid) deposit(lres, -L.scale * ((B_i - B_last) * tau) * vratio(jres));
      atomicAdd(a.ermc_acc + armc_slot(a, L.r, L.cellid), f32_to_f64(L.scale * X));
    }
    if (lane == 0) {
      a.ybuf[(size_t)L.slot * (unsigned)N + L.r] = L.scale * X;  // the ray's sample Y (Eq. 14)
      if (a.ray_steps) a.ray_steps[(size_t)L.slot * (unsigned)N + L.r] = (unsigned)steps;
      if (a.steps_cell) atomicAdd(a.step_acc + L.slot, (unsigned long long)steps);
    }
    w_steps += (unsigned long long)steps;
    ++w_rays;
    w_cap += capped;
    w_wall += walls;
    w_max = max(w_max, (unsigned)steps);
  }
  if (lane == 0 && w_rays) {
    atomicAdd(a.counters + 0, w_steps);
    atomicAdd(a.counters + 3, (unsigned long long)w_rays);
    if (w_cap) atomicAdd(a.counters + 1, (unsigned long long)w_cap);
    if (w_wall) atomicAdd(a.counters + 2, (unsigned long long)w_wall);
    atomicMax(a.counters + 4, (unsigned long long)w_max);
  }
}

}  // namespace

long long long_ray_capacity(long long rays, int long_steps) {
  // rays that reach L segments fall off roughly like 1/L (grazing directions)
  // times the share of thin bands (a 1 m slab with 119 x 16 bands hands off
  // about 1 ray in 1.2e4 at L = 1024); rays 256 / L^2 leaves a margin of three
  // at the default L = 1024 and holds every ray for L <= 16, at least 2^16
  // entries (128 B each)
  const long long L = long_steps > 1 ? long_steps : 1;
  long long c = L <= 16 ? rays : rays / ((L * L + 255) / 256);
  if (c < 65536) c = 65536;
  if (c > rays) c = rays > 0 ? rays : 1;
  if (c > (1LL << 24)) c = 1LL << 24;
  return c;
}

cudaError_t launch_long_rays(const TraceArgs &a, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // one warp per long ray, up to four 256-thread CTAs per SM; warps stride over
  // the rays beyond that
  long long blocks = ((long long)a.long_cap + 7) / 8;
  if (blocks > 4LL * sms) blocks = 4LL * sms;
  if (blocks < 1) blocks = 1;
  if (a.armc_acc)
    long_march_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(a);
  else
    long_march_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mcrt

// ERMC ray-trace kernel: the per-cell ray loop that produces Q_rad.
//
// Silvestri & Pecnik (arXiv:1810.00188): Section 2 (Eqs. 2, 3, 12-14), Section
// 2.1 (band / quadrature-point sampling, Eqs. 15-17), Algorithm 1 (initialise,
// march, residual dump) and the domain parallelisation of Section 3 (all rays of
// a cell owned by one worker, so the per-cell tally needs no atomics).
//
// GB300 mapping: one warp per emitting cell, its 32 lanes stride over the cell's
// rays; a warp-shuffle reduction in binary64 and a single store of Q and sigma
// per cell.  Everything is binary64: this is the parity mode (binary64 issues at
// about 1/64 of the binary32 rate on GB300; FP32 solves run the scheduled
// kernels of trace_fp32.cu).  Random numbers come from a counter-based
// Philox4x32-10 keyed by (cell, ray, draw block, snapshot), so each ray's draws
// are independent of the launch shape.  The k-distribution tables are read
// through the read-only path as {value, next-minus-value} pairs so a lookup is one
// 8- or 16-byte load and one fused multiply-add.
#include <math.h>
#include <stdint.h>

#include "mcrt_internal.h"

namespace mcrt {
namespace {

// ---- counter-based random numbers -----------------------------------------
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): each round multiplies counter words 0
// and 2 by the round constants, mixes the high halves into words 1 and 3 with
// the key, and the key advances by the Weyl increments between rounds.
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

// Uniform on (0, 1) from the top 23 bits of a word: (w>>9 + 1/2) 2^-23, exact
// in binary32 and binary64.
template <typename R>
__device__ __forceinline__ R unif(unsigned w) {
  return ((R)(w >> 9) + (R)0.5) * (R)1.1920928955078125e-07;
}

// ---- precision-specific pieces ---------------------------------------------
template <typename R> struct Prec;
template <> struct Prec<double> {
  typedef double2 R2;
  __device__ static const double2 *field(const TraceArgs &a) { return a.field64; }
  __device__ static const double2 *ktab(const TraceArgs &a) { return a.ktab64; }
  __device__ static const double2 *btab(const TraceArgs &a) { return a.btab64; }
  __device__ static const double *bwall(const TraceArgs &a) { return a.bwall64; }
  __device__ static const double *yf(const TraceArgs &a) { return a.yf64; }
  __device__ static void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
  __device__ static double div(double a, double b) { return a / b; }
  __device__ static void absorb(double x, double &alpha, double &trans) {
    alpha = -expm1(-x);
    trans = exp(-x);
  }
};

// Linear-interpolation position on the uniform T nodes (Section 2.2); clamps
// to the end nodes outside the table.
template <typename R>
__device__ __forceinline__ void tpos(R T, R T0, R inv_dT, int nT, int &it, R &fr) {
  const R f = (T - T0) * inv_dT;
  const R fl = fmin(fmax(floor(f), (R)0), (R)(nT - 2));
  it = (int)fl;
  fr = fmin(fmax(f - fl, (R)0), (R)1);
}

// First k with u < cum[k] (cum non-decreasing, cum[K-1] = 2^32): the inverse
// CDF of a discrete pdf held as integer counts (Eq. 17 with R_n, R_g).
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

__device__ __forceinline__ void neumaier(double &s, double &c, double v) {
  const double t = s + v;
  if (fabs(s) >= fabs(v))
    c += (s - t) + v;
  else
    c += (v - t) + s;
  s = t;
}

// Per-lane tally of sum(Y) and sum(Y^2): Neumaier sums in binary64.
template <typename R> struct Tally;
template <> struct Tally<double> {
  double s = 0.0, c = 0.0, s2 = 0.0, c2 = 0.0;
  __device__ void add(double y) {
    neumaier(s, c, y);
    neumaier(s2, c2, y * y);
  }
  __device__ double sum() const { return s + c; }
  __device__ double sum2() const { return s2 + c2; }
};

// Ray weight w_g / (p(n,g) q(Omega)) from the integer counts (Eq. 14 with the
// pdfs of Eqs. 4, 9, 16).
template <typename R>
__device__ __forceinline__ R ray_weight(const TraceArgs &a, bool plain, int n, int g,
                                        unsigned long long mn, unsigned long long mg, double ph);
template <>
__device__ __forceinline__ double ray_weight<double>(const TraceArgs &a, bool, int, int g,
                                                     unsigned long long mn, unsigned long long mg,
                                                     double ph) {
  const double p = ((double)mn * 2.3283064365386963e-10) * ((double)mg * 2.3283064365386963e-10);
  return (__ldg(a.w_g + g) / p) * (6.283185307179586 / ph);
}

// Distance parameters of one axis of the parametric ray o + t d: the m-th face
// crossing is at t = t0 + m * ts.
template <typename R>
__device__ __forceinline__ void axis_setup(R d, R fr, R delta, int &s, R &t0, R &ts) {
  if (d > (R)0) {
    s = 1;
    ts = Prec<R>::div(delta, d);
    t0 = ((R)1 - fr) * ts;
  } else if (d < (R)0) {
    s = -1;
    ts = Prec<R>::div(delta, -d);
    t0 = fr * ts;
  } else {
    s = 0;
    ts = (R)INFINITY;
    t0 = (R)INFINITY;
  }
}

constexpr int START_LANES = 8;  // waiting lanes that set up their next rays together

// AR: the absorption-based estimate's deposits (a.armc_acc non-null).
template <typename R, bool AR>
__global__ void __launch_bounds__(256) trace_kernel(const TraceArgs a) {
  typedef typename Prec<R>::R2 R2;
  extern __shared__ unsigned long long s_counts[];  // plain band counts, then g counts
  const bool plain = a.cell_cn == nullptr;
  if (plain && a.counts_in_smem) {
    const int ncount = a.nb + a.nb * a.ng;
    for (int i = threadIdx.x; i < ncount; i += blockDim.x)
      s_counts[i] = i < a.nb ? a.cn[i] : a.cg[i - a.nb];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.ncells_box) return;  // whole warps only

  const int ci = a.bi0 + (int)(w % a.bnx);
  const int cj = a.bj0 + (int)((w / a.bnx) % a.bny);
  const int ck = a.bk0 + (int)(w / ((long long)a.bnx * a.bny));
  const int nx = a.nx, ny = a.ny, nz = a.nz, nxy = nx * ny, nb = a.nb, ng = a.ng, nT = a.nT;
  const unsigned cell = (unsigned)(ci + nx * cj + nxy * ck);

  const R2 *__restrict__ field = Prec<R>::field(a);
  const R2 *__restrict__ ktab = Prec<R>::ktab(a);
  const R2 *__restrict__ btab = Prec<R>::btab(a);
  const R *__restrict__ bwall = Prec<R>::bwall(a);
  const R T0 = (R)a.T0, inv_dT = (R)a.inv_dT, inv_xref = (R)a.inv_xref, tol = (R)a.tol;
  const R DX = (R)a.dx, DY = (R)a.dy, DZ = (R)a.dz;
  // stretched y: faces (null: uniform DY); the height of row j of grid l
  const R *__restrict__ yfs = Prec<R>::yf(a);
  auto dyl = [&](int j, int l) -> R {
    return __ldg(yfs + ((size_t)(j + 1) << l)) - __ldg(yfs + ((size_t)j << l));
  };

  // emitting cell state
  const R2 fi = __ldg(field + cell);
  int it_i;
  R fr_i;
  tpos<R>(fi.x, T0, inv_dT, nT, it_i, fr_i);
  const R xr_i = fi.y * inv_xref;

  const unsigned long long *__restrict__ cn =
      plain ? (a.counts_in_smem ? s_counts : a.cn) : a.cell_cn + (size_t)cell * nb;
  const unsigned long long *__restrict__ cg =
      plain ? (a.counts_in_smem ? s_counts + nb : a.cg) : a.cell_cg + (size_t)cell * nb * ng;
  const unsigned hemi = a.cell_hemi ? __ldg(a.cell_hemi + cell) : 4194304u;
  const R inv_hemi = (R)1 / (R)hemi, inv_lo = (R)1 / (R)(8388608u - hemi);

  Tally<R> tally;
  unsigned long long nsteps = 0, ncap = 0, nwall = 0, max_ray = 0;
  // the absorption-based estimate (a.armc_acc non-null): each ray's deposits
  // into the per-batch sums [16][cells] of the cells that absorb (batch: the
  // ray's index mod 16), on a stretched grid with the volume ratio V_i / V_j
  // (the rows' heights), and its sample into its own cell's emission-based sum
  auto deposit = [&](double *acc, int r, unsigned c, double v) {
    atomicAdd(acc + (size_t)(r & 15) * (size_t)a.armc_nc + c, v);
  };
  auto vratio = [&](int j) -> R { return yfs ? dyl(cj, 0) / dyl(j, 0) : (R)1; };

  // Each lane marches its rays r = lane, lane + 32, ... one after another, and a
  // lane whose ray has ended starts its next one without waiting for the rest of
  // the warp's current rays (a heavy-tailed ray length otherwise idles most
  // lanes at the end of each round of 32 rays): the same rays in the same order
  // on each lane, hence the same tallies.
  unsigned ray = 0, nrefl = 0;
  R ddx = 0, ddy = 0, ddz = 0, fx = 0, fy = 0, fz = 0, wgt = 0, kap_i = 0, B_i = 0;
  int n = 0;
  size_t krow = 0, brow = 0;
  int ix = 0, iy = 0, iz = 0, lin = 0, sx = 0, sy_ = 0, sz = 0, steps = 0;
  R t0x = 0, t0y = 0, t0z = 0, tsx = 0, tsy = 0, tsz = 0, cntx = 0, cnty = 0, cntz = 0;
  R tnx = 0, tny = 0, tnz = 0, tprev = 0, X = 0, tau = 1, B_last = 0;
  // multigrid (Section 4.3): current grid, its dimensions and the offset of its
  // fields, segments marched on it, and the face counter step: grid l keeps
  // every inc-th face of the grid the axis parameters were set up on
  int lev = 0, lsteps = 0, nxl = nx, nyl = ny, nzl = nz;
  long long loff = 0;
  R inc = 1;
  // the set-up of ray r (Algorithm 1 "Initialize")
  auto start = [&](int r) {
    ray = (unsigned)(a.ray_offset + (unsigned long long)r);
    const uint4 u = philox10(make_uint4(cell, ray, 0u, a.snapshot), a.key0, a.key1);

    // direction: hemisphere of the y axis by the integer count `hemi` of 2^23,
    // mu uniform inside it; azimuth phi = 2 pi R_phi (Eq. 9)
    const unsigned m0 = u.x >> 9;
    R mu;
    double ph;
    if (m0 < hemi) {
      mu = (R)1 - ((R)m0 + (R)0.5) * inv_hemi;
      ph = (double)hemi * 1.1920928955078125e-07;
    } else {
      mu = -(((R)(m0 - hemi) + (R)0.5) * inv_lo);
      ph = (double)(8388608u - hemi) * 1.1920928955078125e-07;
    }
    R sphi, cphi;
    Prec<R>::sincospi_((R)2 * unif<R>(u.y), &sphi, &cphi);
    const R st = sqrt(fmax((R)0, (R)1 - mu * mu));
    ddx = st * cphi;
    ddy = mu;
    ddz = st * sphi;

    // band and quadrature point from two words (Eq. 17); weight w_g / (p q)
    n = pick(cn, nb, u.z);
    const unsigned long long *cgn = cg + (size_t)n * ng;
    const int g = pick(cgn, ng, u.w);
    const unsigned long long mn = cn[n] - (n ? cn[n - 1] : 0ull);
    const unsigned long long mg = cgn[g] - (g ? cgn[g - 1] : 0ull);
    wgt = ray_weight<R>(a, plain, n, g, mn, mg, ph);

    // origin: uniform in the cell (block 1 draws) or the centre
    fx = fy = fz = (R)0.5;
    if (a.origin == 0) {
      const uint4 v = philox10(make_uint4(cell, ray, 1u, a.snapshot), a.key0, a.key1);
      fx = unif<R>(v.x);
      fy = unif<R>(v.y);
      fz = unif<R>(v.z);
    }

    krow = (size_t)(n * ng + g) * nT;
    brow = (size_t)n * nT;
    const R2 ki = __ldg(ktab + krow + it_i);
    const R2 bi = __ldg(btab + brow + it_i);
    kap_i = (ki.x + fr_i * ki.y) * xr_i;
    B_i = bi.x + fr_i * bi.y;

    // the march starts in the emitting cell on the finest grid
    ix = ci;
    iy = cj;
    iz = ck;
    lin = (int)cell;
    axis_setup<R>(ddx, fx, DX, sx, t0x, tsx);
    axis_setup<R>(ddy, fy, yfs ? dyl(cj, 0) : DY, sy_, t0y, tsy);
    axis_setup<R>(ddz, fz, DZ, sz, t0z, tsz);
    // stretched y: tsy is 1/|d_y|, and each y crossing adds the next row's height
    if (yfs && sy_ != 0) tsy = (R)1 / fabs(ddy);
    cntx = cnty = cntz = 0;
    tnx = t0x;
    tny = t0y;
    tnz = t0z;
    tprev = 0;
    X = 0;
    tau = 1;
    B_last = B_i;
    steps = 0;
    nrefl = 0;
    lev = 0;
    lsteps = 0;
    nxl = nx;
    nyl = ny;
    nzl = nz;
    loff = 0;
    inc = 1;
  };
  int r = lane;
  bool live = r < a.rays;  // the lane holds a ray (marching, or waiting to start it)
  bool wait = live;        // the lane's next ray is not set up yet
  while (__any_sync(0xffffffffu, live)) {
    // the waiting lanes set up their rays together once START_LANES of them
    // wait or none marches: the set-up's binary64 work then runs on more lanes
    const unsigned wm = __ballot_sync(0xffffffffu, wait);
    const unsigned mm = __ballot_sync(0xffffffffu, live && !wait);
    if (wm && (__popc(wm) >= START_LANES || mm == 0) && wait) {
      start(r);
      wait = false;
    }
    if (!live || wait) continue;
    // one segment of the march (Algorithm 1 "March")
    bool end = false;
    do {
      int ax;
      R tn;
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
      const R ds = fmax(tn - tprev, (R)0);
      const R2 f = __ldg(field + loff + lin);
      int it;
      R fr;
      tpos<R>(f.x, T0, inv_dT, nT, it, fr);
      const R2 kk = __ldg(ktab + krow + it);
      const R2 bb = __ldg(btab + brow + it);
      const R kap = (kk.x + fr * kk.y) * (f.y * inv_xref);
      const R Bj = bb.x + fr * bb.y;
      R alpha, trans;
      Prec<R>::absorb(kap * ds, alpha, trans);
      const R term = (B_i - Bj) * (tau * alpha);
      X += term;  // Eq. 14 term / kappa_i
      if (AR && lin != (int)cell) deposit(a.armc_acc, r, (unsigned)lin, -(wgt * kap_i) * term * vratio(iy));
      tau *= trans;  // Eq. 3
      B_last = Bj;
      ++steps;
      ++lsteps;
      if (tau <= tol) { end = true; break; }
      if (steps >= a.max_steps) {
        ++ncap;
        {
          end = true;
          break;
        }
      }
      tprev = tn;
      const int nxyl = nxl * nyl;
      if (a.xz_walls && ax != 1 && (ax == 0 ? (unsigned)(ix + sx) >= (unsigned)nxl
                                             : (unsigned)(iz + sz) >= (unsigned)nzl)) {
        // closed box: a black x or z wall absorbs the rest of the ray and emits
        // at its temperature (Eq. 3 wall factor with eps = 1)
        const int f = ax == 0 ? (ix + sx < 0 ? 2 : 3) : (iz + sz < 0 ? 4 : 5);
        const R tw = (B_i - __ldg(bwall + f * nb + n)) * tau;
        X += tw;
        if (AR) deposit(a.armc_acc, r, cell, (wgt * kap_i) * tw);  // the cell's own exchange with the wall
        tau = 0;
        ++nwall;
        {
          end = true;
          break;
        }
      }
      if (ax == 0) {
        cntx += inc;
        tnx = fma(cntx, tsx, t0x);
        ix += sx;
        lin += sx;
        if (ix >= nxl) {
          ix -= nxl;
          lin -= nxl;
        } else if (ix < 0) {
          ix += nxl;
          lin += nxl;
        }
      } else if (ax == 2) {
        cntz += inc;
        tnz = fma(cntz, tsz, t0z);
        iz += sz;
        lin += sz * nxyl;
        if (iz >= nzl) {
          iz -= nzl;
          lin -= nxyl * nzl;
        } else if (iz < 0) {
          iz += nzl;
          lin += nxyl * nzl;
        }
      } else {
        cnty += inc;
        tny = fma(cnty, tsy, t0y);
        iy += sy_;
        lin += sy_ * nxl;
        if (yfs && iy >= 0 && iy < nyl) tny = tprev + dyl(iy, lev) * tsy;
        if (iy < 0 || iy >= nyl) {
          // wall event: the wall absorbs eps of the ray and emits at T_wall
          const int wl = iy < 0 ? 0 : 1;
          const R eps = (R)a.eps_wall[wl];
          const R Bw = __ldg(bwall + wl * nb + n);
          X += (B_i - Bw) * (tau * eps);
          if (AR) deposit(a.armc_acc, r, cell, (wgt * kap_i) * ((B_i - Bw) * (tau * eps)));
          tau *= (R)1 - eps;
          ++nwall;
          if (eps >= (R)1 || tau <= tol) { end = true; break; }
          // reflect from the crossing point at t = tprev (fractions of the
          // current grid's cell, whose extent along an axis is inc face steps)
          R nfx = fx, nfz = fz;
          if (sx > 0)
            nfx = (R)1 - (tnx - tprev) / (tsx * inc);
          else if (sx < 0)
            nfx = (tnx - tprev) / (tsx * inc);
          if (sz > 0)
            nfz = (R)1 - (tnz - tprev) / (tsz * inc);
          else if (sz < 0)
            nfz = (tnz - tprev) / (tsz * inc);
          fx = fmin(fmax(nfx, (R)0), (R)1);
          fz = fmin(fmax(nfz, (R)0), (R)1);
          fy = wl == 0 ? (R)0 : (R)1;
          iy = wl == 0 ? 0 : nyl - 1;
          lin = ix + nxl * iy + nxyl * iz;
          if (a.reflect == 1) {
            ddy = -ddy;
          } else {
            // Lambertian: cos(theta) = sqrt(U), azimuth 2 pi U (block 2 + k)
            const uint4 v =
                philox10(make_uint4(cell, ray, 2u + nrefl, a.snapshot), a.key0, a.key1);
            const R mr = sqrt(unif<R>(v.x));
            R sp, cp;
            Prec<R>::sincospi_((R)2 * unif<R>(v.y), &sp, &cp);
            const R sr = sqrt(fmax((R)0, (R)1 - mr * mr));
            ddx = sr * cp;
            ddy = wl == 0 ? mr : -mr;
            ddz = sr * sp;
          }
          ++nrefl;
          const R gl = (R)(1 << lev);  // cell size of the current grid / finest
          axis_setup<R>(ddx, fx, DX * gl, sx, t0x, tsx);
          axis_setup<R>(ddy, fy, yfs ? dyl(iy, lev) : DY * gl, sy_, t0y, tsy);
          axis_setup<R>(ddz, fz, DZ * gl, sz, t0z, tsz);
          if (yfs && sy_ != 0) tsy = (R)1 / fabs(ddy);
          cntx = cnty = cntz = 0;
          tnx = t0x;
          tny = t0y;
          tnz = t0z;
          tprev = 0;
          inc = 1;
        }
      }
      if (lev + 1 < a.mg_levels && lsteps >= a.mg_steps) {
        // multigrid (Section 4.3): fall onto the next coarser grid here.  Its
        // faces are the even-numbered faces of this grid, so an axis whose next
        // face is odd-numbered skips it; the cell is the one containing this one.
        if (sx != 0 && ((sx > 0 ? ix + 1 : ix) & 1)) {
          cntx += inc;
          tnx = fma(cntx, tsx, t0x);
        }
        if (sy_ != 0 && ((sy_ > 0 ? iy + 1 : iy) & 1)) {
          if (yfs) {
            tny += dyl(sy_ > 0 ? iy + 1 : iy - 1, lev) * tsy;  // the skipped row's height
          } else {
            cnty += inc;
            tny = fma(cnty, tsy, t0y);
          }
        }
        if (sz != 0 && ((sz > 0 ? iz + 1 : iz) & 1)) {
          cntz += inc;
          tnz = fma(cntz, tsz, t0z);
        }
        loff += (long long)nxl * nyl * nzl;
        nxl >>= 1;
        nyl >>= 1;
        nzl >>= 1;
        ix >>= 1;
        iy >>= 1;
        iz >>= 1;
        lin = ix + nxl * (iy + nyl * iz);
        inc *= (R)2;
        ++lev;
        lsteps = 0;
      }
    } while (false);
    if (!end) continue;
    if (tau > (R)0) X += (B_i - B_last) * tau;  // residual dump (Algorithm 1)
    if (AR) {
      // the residual is absorbed in the last medium cell crossed (the row
      // clamped after a wall event)
      const int jres = min(max(iy, 0), ny - 1);
      const unsigned lres = (unsigned)(ix + nx * (jres + ny * iz));
      if (tau > (R)0 && lres != cell)
        deposit(a.armc_acc, r, lres, -(wgt * kap_i) * ((B_i - B_last) * tau) * vratio(jres));
      deposit(a.ermc_acc, r, cell, wgt * (kap_i * X));
    }

    tally.add(wgt * (kap_i * X));
    nsteps += (unsigned long long)steps;
    max_ray = max(max_ray, (unsigned long long)steps);
    r += 32;
    live = r < a.rays;
    wait = live;
  }

  // warp reduction of the lanes' tallies
  double S = tally.sum(), S2 = tally.sum2();
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    S += __shfl_xor_sync(0xffffffffu, S, off);
    S2 += __shfl_xor_sync(0xffffffffu, S2, off);
    nsteps += __shfl_xor_sync(0xffffffffu, nsteps, off);
    ncap += __shfl_xor_sync(0xffffffffu, ncap, off);
    nwall += __shfl_xor_sync(0xffffffffu, nwall, off);
    max_ray = max(max_ray, __shfl_xor_sync(0xffffffffu, max_ray, off));
  }
  if (lane == 0) {
    atomicMax(a.counters + 4, max_ray);
    const double N = (double)a.rays;
    const double Q = S / N;
    a.q[w] = Q;  // Eq. 8: mean of the per-ray samples
    if (a.sigma)
      a.sigma[w] = a.rays > 1 ? sqrt(fmax(S2 / N - Q * Q, 0.0) / (N - 1.0)) : 0.0;
    if (a.steps_cell) a.steps_cell[w] = nsteps;
    atomicAdd(a.counters + 0, nsteps);
    if (ncap) atomicAdd(a.counters + 1, ncap);
    if (nwall) atomicAdd(a.counters + 2, nwall);
    atomicAdd(a.counters + 3, (unsigned long long)a.rays);
  }
}

}  // namespace

cudaError_t launch_trace(const TraceArgs &a, int precision, cudaStream_t s) {
  if (a.ncells_box <= 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = (a.ncells_box * 32 + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const size_t smem =
      a.counts_in_smem ? sizeof(unsigned long long) * (size_t)(a.nb + a.nb * a.ng) : 0;
  if (precision != 1) return cudaErrorInvalidValue;  // FP32 solves run trace_fp32.cu's kernels
  if (a.armc_acc)
    trace_kernel<double, true><<<(unsigned)blocks, threads, smem, s>>>(a);
  else
    trace_kernel<double, false><<<(unsigned)blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mcrt

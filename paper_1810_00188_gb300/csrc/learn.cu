// Learned spectral/directional proposal: cell features, second-moment and cost
// tallies of a solve, the network's forward pass (straight into a per-cell
// integer proposal), and its training (fused forward + loss + backward, a
// fixed-order gradient reduction, Adam).
//
// The paper draws (n, g) from Zhang's T_max pdf (Section 2.1, Eqs. 13, 16) and
// the direction isotropically (Eq. 9).  Eq. 14 stays unbiased for any other pdf
// if the ray weight divides by the probabilities actually used and every
// contributing (n, g, hemisphere) keeps a non-zero probability; here the pdf of
// each emitting cell is
//     q(n,g) = (1 - mix) softmax(z)_(n,g) + mix p0(n,g),
//     q(h)   = (1 - mix) softmax(z_up, z_down)_h + mix / 2,
// z the output of a 12 -> 64 -> 64 -> (K + 2) perceptron with GELU activations
// and FP16 weights (FP32 arithmetic), quantised to integer counts (the trace
// kernel's weights use the quantised probabilities exactly).  The network is
// trained to minimise, per cell, (second moment per ray) x (steps per ray)
// relative to the plain pdf, from unbiased tallies of plain solves:
//     m[k][h] = (1/N) sum_(rays in k,h) Y^2 p_k p_h   ->  E_q[Y^2] = sum m / (q_k q_h)
//     c[k][h] = (1/N) sum_(rays in k,h) steps / (p_k p_h) -> E_q[steps] = sum c q_k q_h
//     L = A(q) C(q) / (A(p0) C(p0)),  A = sum m / (q_k q_h),  C = c0 + sum c q_k q_h.
//
// The tiny contractions (12x64, 64x64, 64x(K+2) per cell) run as FP32 FMAs on
// shared-memory tiles; the work is a few milliseconds next to the solves that
// produce its data, so they do not go to the tensor cores.
#include <cuda_fp16.h>
#include <math.h>

#include "draws.cuh"
#include "mcrt_internal.h"

namespace mcrt {
namespace {

constexpr int NF = kNFeat, NH = kNHidden;
constexpr int IT = 32;   // cells per inference tile
constexpr int TT = 16;   // samples per training tile
constexpr int NTHR = 256;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678f)); }

__device__ __forceinline__ float gelu_prime(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678f)) + x * 0.39894228f * expf(-0.5f * x * x);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---- features ------------------------------------------------------------------
// 0 T_i/1000, 1 x_i, 2 y_c/h - 1, 3-4 wall T/1000, 5 eps of the nearer wall,
// 6 h dT/dy / 1000 (centred, one-sided at the walls; on a stretched grid over
// the distance of the face-midpoint centres), 7 h |grad_xz T| / 1000
// (centred, periodic), 8-9 mean and standard deviation of T over the 3^3
// neighbourhood (periodic in x, z; cut at the walls) / T_i, 10 the Planck-mean
// absorption coefficient at (T_i, x_i) times h, 11 T_max / T_i.

__global__ void __launch_bounds__(NTHR) features_kernel(const FeatArgs f) {
  const long long ncell = (long long)f.nx * f.ny * f.nz;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < f.n;
       q += (long long)gridDim.x * blockDim.x) {
    const long long c = f.cells ? (long long)f.cells[q] : q;
    float *o = f.out + q * NF;
    if (c < 0 || c >= ncell) {
      atomicOr(f.err, 1ull);
      for (int i = 0; i < NF; ++i) o[i] = __int_as_float(0x7fc00000);
      continue;
    }
    const int nx = f.nx, ny = f.ny, nz = f.nz;
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    auto T = [&](int ii, int jj, int kk) {
      return f.field64[(size_t)ii + (size_t)nx * ((size_t)jj + (size_t)ny * kk)].x;
    };
    // row centres: midpoints of the faces on a stretched grid
    auto ycen = [&](int jj) { return f.yf ? 0.5 * (f.yf[jj] + f.yf[jj + 1]) : (jj + 0.5) * f.dy; };
    const double2 v = f.field64[c];
    const double Ti = v.x, yc = ycen(j);
    o[0] = (float)(Ti / 1000.0);
    o[1] = (float)v.y;
    o[2] = (float)(yc / f.h - 1.0);
    o[3] = (float)(f.T_wall[0] / 1000.0);
    o[4] = (float)(f.T_wall[1] / 1000.0);
    o[5] = (float)(yc < f.h ? f.eps_wall[0] : f.eps_wall[1]);
    double dTdy = 0.0;
    if (ny > 1 && !f.yf) {
      if (j == 0)
        dTdy = (T(i, 1, k) - T(i, 0, k)) / f.dy;
      else if (j == ny - 1)
        dTdy = (T(i, ny - 1, k) - T(i, ny - 2, k)) / f.dy;
      else
        dTdy = (T(i, j + 1, k) - T(i, j - 1, k)) / (2.0 * f.dy);
    } else if (ny > 1) {
      // stretched grid: differences over the distance of the centres used
      const int j0 = j == 0 ? 0 : j - 1, j1 = j == ny - 1 ? ny - 1 : j + 1;
      dTdy = (T(i, j1, k) - T(i, j0, k)) / (ycen(j1) - ycen(j0));
    }
    o[6] = (float)(f.h * dTdy / 1000.0);
    const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
    const int kp = k + 1 == nz ? 0 : k + 1, km = k == 0 ? nz - 1 : k - 1;
    const double dTdx = (T(ip, j, k) - T(im, j, k)) / (2.0 * f.dx);
    const double dTdz = (T(i, j, kp) - T(i, j, km)) / (2.0 * f.dz);
    o[7] = (float)(f.h * sqrt(dTdx * dTdx + dTdz * dTdz) / 1000.0);
    double sum = 0.0;
    int cnt = 0;
    const int xs[3] = {im, i, ip}, zs[3] = {km, k, kp};
    for (int c2 = 0; c2 < 3; ++c2)
      for (int b2 = -1; b2 <= 1; ++b2) {
        const int jj = j + b2;
        if (jj < 0 || jj >= ny) continue;
        for (int a2 = 0; a2 < 3; ++a2) {
          sum += T(xs[a2], jj, zs[c2]);
          ++cnt;
        }
      }
    const double mean = sum / cnt;
    double var = 0.0;
    for (int c2 = 0; c2 < 3; ++c2)
      for (int b2 = -1; b2 <= 1; ++b2) {
        const int jj = j + b2;
        if (jj < 0 || jj >= ny) continue;
        for (int a2 = 0; a2 < 3; ++a2) {
          const double d = T(xs[a2], jj, zs[c2]) - mean;
          var += d * d;
        }
      }
    o[8] = (float)(mean / Ti);
    o[9] = (float)(sqrt(var / cnt) / Ti);
    // Planck mean at T_i: sum_n B_n sum_g w_g kappa_(n,g) / sum_n B_n with B and
    // kappa linear in the fraction between nodes, i.e. a quadratic over a linear
    // polynomial per node (coefficients summed on the host in FP64)
    const uint2 pk = f.fpos32[c];
    const unsigned it = pk.x >> 23;
    const float fr = __uint_as_float(0x3F800000u | (pk.x & 0x7FFFFFu)) - 1.f;
    const float4 k0 = f.kptab[2 * it], k1 = f.kptab[2 * it + 1];
    const float num = k0.x + fr * (k0.y + fr * k0.z), den = k0.w + fr * k1.x;
    o[10] = den > 0.f ? (float)((double)(num / den) * (double)__uint_as_float(pk.y) * f.h) : 0.f;
    o[11] = (float)(f.T_max / Ti);
  }
}

// ---- second-moment and cost tallies ----------------------------------------------
// One warp per listed cell whose samples are in this chunk: recomputes each
// ray's (n, g, hemisphere) from its Philox draw exactly as the trace kernel did,
// and adds Y^2 p_k p_h / N and steps / (p_k p_h) / N to its bin.  The 32 rays of
// a round are added one after another by the lane that owns the bin, so the
// sums have a fixed order.

constexpr int TALLY_WARPS = 4;

__global__ void __launch_bounds__(TALLY_WARPS * 32) tally_kernel(const TallyArgs t) {
  extern __shared__ double tsm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int K2 = 2 * t.nb * t.ng;
  double *sm = tsm + (size_t)w * 2 * K2, *sc = sm + K2;
  const long long ncell = (long long)t.nx * t.ny * t.nz;
  const int nbx = (t.nx + 7) / 8, nby = (t.ny + 7) / 8;
  const unsigned N = (unsigned)t.N;
  for (long long q = (long long)blockIdx.x * TALLY_WARPS + w; q < t.n;
       q += (long long)gridDim.x * TALLY_WARPS) {
    const long long c = t.cells[q];
    if (c < 0 || c >= ncell) {
      if (lane == 0) atomicOr(t.err, 1ull);
      continue;
    }
    const int x = (int)(c % t.nx), y = (int)((c / t.nx) % t.ny), z = (int)(c / ((long long)t.nx * t.ny));
    const long long p = ((long long)(x >> 3) + nbx * ((long long)(y >> 3) + (long long)nby * (z >> 3))) * 512 +
                        (x & 7) + 8 * ((y & 7) + 8 * (z & 7));
    if (p < t.chunk_p0 || p >= t.chunk_p1) continue;
    const size_t slot = (size_t)(p - t.chunk_p0);
    for (int e = lane; e < K2; e += 32) sm[e] = sc[e] = 0.0;
    __syncwarp();
    const unsigned long long *cn = t.cell_cn ? t.cell_cn + (size_t)c * t.nb : t.cn;
    const unsigned long long *cg = t.cell_cg ? t.cell_cg + (size_t)c * t.nb * t.ng : t.cg;
    const unsigned hemi = t.cell_hemi ? t.cell_hemi[c] : 4194304u;
    for (unsigned r0 = 0; r0 < N; r0 += 32) {
      const unsigned r = r0 + lane;
      int bin = 0;
      double vm = 0.0, vc = 0.0;
      if (r < N) {
        const unsigned rayid = (unsigned)(t.ray_off + r);
        const uint4 u = philox10(make_uint4((unsigned)c, rayid, 0u, t.snapshot), t.key0, t.key1);
        const unsigned m0 = u.x >> 9;
        const int h = m0 < hemi ? 0 : 1;
        const double ph = (double)(h ? 8388608u - hemi : hemi) * 0x1p-23;
        const int nn = pick(cn, t.nb, u.z);
        const unsigned long long *cgn = cg + (size_t)nn * t.ng;
        const int gg = pick(cgn, t.ng, u.w);
        const double pn = (double)(cn[nn] - (nn ? cn[nn - 1] : 0ull)) * 0x1p-32;
        const double pg = (double)(cgn[gg] - (gg ? cgn[gg - 1] : 0ull)) * 0x1p-32;
        const double png = pn * pg;
        const double Y = (double)t.ybuf[slot * N + r];
        const double st = (double)t.ray_steps[slot * N + r];
        vm = Y * Y * png * ph / (double)N;
        vc = st / (png * ph) / (double)N;
        bin = (nn * t.ng + gg) * 2 + h;
      }
      const int cntr = N - r0 < 32u ? (int)(N - r0) : 32;
      for (int jr = 0; jr < cntr; ++jr) {
        const int bj = __shfl_sync(0xffffffffu, bin, jr);
        const double mj = __shfl_sync(0xffffffffu, vm, jr);
        const double cj = __shfl_sync(0xffffffffu, vc, jr);
        if ((bj & 31) == lane) {
          sm[bj] += mj;
          sc[bj] += cj;
        }
      }
    }
    __syncwarp();
    for (int e = lane; e < K2; e += 32) {
      t.m_out[q * K2 + e] = (float)sm[e];
      t.c_out[q * K2 + e] = (float)sc[e];
    }
    __syncwarp();
  }
}

// ---- integer proposal of one cell ------------------------------------------------
// Counts of 2^32 proportional to the weights, at least one for every positive
// weight, the rounding remainder on the first largest weight; W is the sum of
// the weights in order.  Per-cell proposals take this decision in binary32 (the
// host's plain proposal takes it once, in binary64): count = floor(RN(w / W)
// 2^32) with a correctly rounded binary32 quotient (the scaling by 2^32 is
// exact).  GB300 issues binary64 on a narrow pipe, and a proposal has 360
// counts per cell.
// floor(y) for 0 <= y < 2^32 from the bits (the significand shifted by the
// exponent): the same value as the float-to-integer conversion, which runs on
// GB300's narrow pipe.
__device__ __forceinline__ unsigned floor_u32(float y) {
  const unsigned u = __float_as_uint(y);
  const int e = (int)(u >> 23) - 127;  // y in [2^e, 2^(e+1))
  if (e < 0) return 0u;
  const unsigned m = (u & 0x7FFFFFu) | 0x800000u;
  return e >= 23 ? m << (e - 23) : m >> (23 - e);
}

__device__ __forceinline__ long long count32(float w, float W) {
  const float y = __fdiv_rn(w, W) * 4294967296.0f;
  return y >= 4294967296.0f ? 4294967296LL : (long long)floor_u32(y);  // y >= 0
}

__device__ bool quantize_row(const float *w, int K, float W, unsigned long long *cum) {
  if (!(W > 0.f)) return false;
  int kmax = 0;
  float wmax = w[0];
  long long total = 0;
  if (K <= 16) {  // the counts in registers (the same sums as below)
    long long m[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < K) {
        const float wk = w[k];
        if (wk > wmax) {
          wmax = wk;
          kmax = k;
        }
        long long mk = 0;
        if (wk > 0.f) {
          mk = count32(wk, W);
          mk = mk < 1 ? 1 : mk;
        }
        m[k] = mk;
        total += mk;
      }
    }
    unsigned long long acc = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < K) {
        acc += (unsigned long long)m[k] + (k == kmax ? (unsigned long long)(4294967296LL - total) : 0ull);
        cum[k] = acc;
      }
    }
    return true;
  }
  for (int k = 0; k < K; ++k) {  // counts (kept in cum), their total, the first largest weight
    const float wk = w[k];
    if (wk > wmax) {
      wmax = wk;
      kmax = k;
    }
    long long mk = 0;
    if (wk > 0.f) {
      mk = count32(wk, W);
      mk = mk < 1 ? 1 : mk;
    }
    cum[k] = (unsigned long long)mk;
    total += mk;
  }
  unsigned long long acc = 0;
  for (int k = 0; k < K; ++k) {
    acc += cum[k] + (k == kmax ? (unsigned long long)(4294967296LL - total) : 0ull);
    cum[k] = acc;
  }
  return true;
}

// The band counts of quantize_cell for nb <= 64, with lane l holding bands l
// and l + 32 in registers: the same sums as the general path (the total of the
// band weights in band order, each band's count once, the exact integer total,
// the first largest weight), with the total formed on every lane from the
// lanes' registers instead of one lane reading shared memory.
__device__ __forceinline__ void quantize_bands64(const float *wn, int nb, int lane, unsigned long long *cn,
                                                 unsigned long long *err) {
  const float w0 = lane < nb ? wn[lane] : 0.f, w1 = lane + 32 < nb ? wn[lane + 32] : 0.f;
  float W = 0.f;
#pragma unroll 8
  for (int n = 0; n < nb; ++n) W += __shfl_sync(0xffffffffu, n < 32 ? w0 : w1, n & 31);  // band order
  if (!(W > 0.f)) {
    if (lane == 0) atomicOr(err, 2ull);
    return;
  }
  long long m0 = 0, m1 = 0;
  if (w0 > 0.f) {
    m0 = count32(w0, W);
    m0 = m0 < 1 ? 1 : m0;
  }
  if (w1 > 0.f) {
    m1 = count32(w1, W);
    m1 = m1 < 1 ? 1 : m1;
  }
  long long tot = m0 + m1;
  // the first largest weight: band lane, then lane + 32, then across lanes
  float bw = lane < nb ? w0 : -1.f;
  int bk = lane < nb ? lane : nb;
  if (lane + 32 < nb && w1 > bw) {
    bw = w1;
    bk = lane + 32;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const float ow = __shfl_xor_sync(0xffffffffu, bw, o);
    const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
    if (ow > bw || (ow == bw && ok < bk)) {
      bw = ow;
      bk = ok;
    }
  }
  // cumulative counts: a warp scan of bands 0..31, then of bands 32..63 on
  // top of the first round's total; the remainder goes to the first largest band
  const unsigned long long rem = (unsigned long long)(4294967296LL - tot);
  unsigned long long carry = 0;
#pragma unroll
  for (int round = 0; round < 2; ++round) {
    const int n = 32 * round + lane;
    unsigned long long v = (unsigned long long)(round ? m1 : m0) + (n == bk ? rem : 0ull);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (n < nb) cn[n] = carry + v;
    carry += __shfl_sync(0xffffffffu, v, 31);
  }
}

// Warp-cooperative: q [nb * ng] spectral probabilities and q_up of one cell ->
// cumulative band counts cn [nb], g counts within each band cg [nb][ng], and the
// upward-hemisphere count of 2^23.  wn: nb floats of scratch (the binary32 band
// weights).  Each band's weight is the binary32 sum of its points in
// order of g, the total the binary32 sum of the band weights in band order on
// one lane; the counts, their exact integer total and the first largest weight
// are formed across lanes.
__device__ void quantize_cell(const float *q, float q_up, int nb, int ng, float *wn,
                              unsigned long long *cn, unsigned long long *cg, unsigned *hemi,
                              unsigned long long *err) {
  const int lane = threadIdx.x & 31;
  for (int n = lane; n < nb; n += 32) {
    const float *qn = q + (size_t)n * ng;
    float W = 0.f;
    for (int g = 0; g < ng; ++g) W += qn[g];
    wn[n] = W;
    if (!quantize_row(qn, ng, W, cg + (size_t)n * ng)) {
      // a band that is never drawn gets uniform g counts (weights 1, so the
      // remainder goes to g = 0)
      const long long mk = count32(1.f, (float)ng);
      unsigned long long acc = 0;
      for (int g = 0; g < ng; ++g) {
        acc += (unsigned long long)(g == 0 ? mk + (4294967296LL - mk * ng) : mk);
        cg[(size_t)n * ng + g] = acc;
      }
    }
  }
  __syncwarp();
  if (nb <= 64) {
    quantize_bands64(wn, nb, lane, cn, err);
  } else {
  float W = 0.f;
  if (lane == 0)
    for (int n = 0; n < nb; ++n) W += wn[n];  // binary32, in band order
  W = __shfl_sync(0xffffffffu, W, 0);
  if (!(W > 0.f)) {
    if (lane == 0) atomicOr(err, 2ull);
  } else {
    // band counts (lane l: bands l, l + 32, ...), their exact total and the
    // first largest band weight
    long long tot = 0;
    float bw = -1.f;
    int bk = nb;
    for (int n = lane; n < nb; n += 32) {
      const float w = wn[n];
      if (w > bw) {
        bw = w;
        bk = n;
      }
      long long mk = 0;
      if (w > 0.f) {
        mk = count32(w, W);
        mk = mk < 1 ? 1 : mk;
      }
      tot += mk;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
      const float ow = __shfl_xor_sync(0xffffffffu, bw, o);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
      if (ow > bw || (ow == bw && ok < bk)) {
        bw = ow;
        bk = ok;
      }
    }
    // cumulative counts: a warp scan per round of 32 bands, the rounds in order
    // (integer sums: the same values in any order); the remainder goes to the
    // first largest band
    unsigned long long carry = 0;
    for (int n0 = 0; n0 < nb; n0 += 32) {
      const int n = n0 + lane;
      unsigned long long v = 0;
      if (n < nb) {
        const float w = wn[n];
        long long mk = 0;
        if (w > 0.f) {
          mk = count32(w, W);
          mk = mk < 1 ? 1 : mk;
        }
        v = (unsigned long long)mk + (n == bk ? (unsigned long long)(4294967296LL - tot) : 0ull);
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (n < nb) cn[n] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  }
  if (lane == 0) {
    // round half up of q_up 2^23 (exact in binary32: the scaling is a power of
    // two and the sum is below 2^23 + 1/2 with an ulp of at most 1/2)
    const float hq = fminf(fmaxf(floorf(q_up * 8388608.f + 0.5f), 1.f), 8388607.f);
    *hemi = floor_u32(hq);
  }
  __syncwarp();
}

__global__ void __launch_bounds__(NTHR, 4) quantize_cells_kernel(const float *q, long long n, int nb,
                                                             int ng, unsigned long long *cell_cn,
                                                             unsigned long long *cell_cg,
                                                             unsigned *cell_hemi,
                                                             unsigned long long *err) {
  extern __shared__ float qsm[];  // per warp: the band weights
  const int w = threadIdx.x >> 5;
  const int K = nb * ng;
  float *wn = qsm + (size_t)w * nb;
  for (long long c = (long long)blockIdx.x * (NTHR / 32) + w; c < n;
       c += (long long)gridDim.x * (NTHR / 32)) {
    const float *qc = q + c * (K + 2);
    quantize_cell(qc, qc[K], nb, ng, wn, cell_cn + c * nb, cell_cg + c * (long long)K, cell_hemi + c,
                  err);
  }
}

// ---- spectral proposals at each cell's own temperature ---------------------------
// The paper's estimator draws (n, g) from the emission spectrum at T_max
// (Zhang's proposal, Eq. 13 discretised as Eq. 16) because the classic ERMC
// draw, from the emitting cell's own spectrum kappa_(n,g)(T_i) B_n(T_i), has a
// large variance in cold cells (Section 2).  Per cell (one warp):
//   local:  p_c(n,g) ~ w_g B_n(T_i) kappa_(n,g)(T_i)          (x_i cancels)
//   hybrid: (1 - lam) p0(n,g) + lam p_local, lam = (T_i - T_min) / (T_max - T_min)
// with p0 the T_max proposal; both quantised like any cell proposal (the ray
// weight divides by the quantised probability, so the estimate stays unbiased),
// hemispheres 1/2 each.
__global__ void __launch_bounds__(NTHR, 4) spectral_proposal_kernel(const SpectralArgs a) {
  extern __shared__ float ssm[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int K = a.nb * a.ng;
  // per warp: the band weights, the cell's K probabilities
  float *wn = ssm + (size_t)w * a.nb;
  float *qw = ssm + (size_t)(NTHR / 32) * a.nb + (size_t)w * K;
  for (long long c = (long long)blockIdx.x * (NTHR / 32) + w; c < a.n;
       c += (long long)gridDim.x * (NTHR / 32)) {
    const uint2 pk = a.fpos32[c];
    const unsigned it = pk.x >> 23;
    const float fr = __uint_as_float(0x3F800000u | (pk.x & 0x7FFFFFu)) - 1.f;
    const double T = a.field64[c].x;
    double lam = 1.0;
    if (a.mode == 1) {
      lam = a.T_max > a.T_min ? (T - a.T_min) / (a.T_max - a.T_min) : 1.0;
      lam = fmin(fmax(lam, 0.0), 1.0);
    }
    // the local weights; the hybrid also needs their sum (lane-strided, then a
    // fixed-order warp sum in binary64), the local proposal only whether one is
    // positive (the weights are >= 0, so that is the sum's sign)
    double part = 0.0;
    bool any = false;
    for (int k = lane; k < K; k += 32) {
      const int n = k / a.ng, g = k - n * a.ng;
      const float2 kk = a.ktab32[(size_t)k * a.nT + it];
      const float2 bb = a.btab32[(size_t)n * a.nT + it];
      const float v = a.w_g32[g] * fmaf(fr, bb.y, bb.x) * fmaf(fr, kk.y, kk.x);
      const float qk = v > 0.f ? v : 0.f;
      qw[k] = qk;
      any = any || qk > 0.f;
      if (a.mode == 1) part += (double)qk;
    }
    if (a.mode == 1) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    }
    const bool pos = __any_sync(0xffffffffu, any);
    __syncwarp();
    if (a.mode == 1 || !pos) {
      // hybrid (or a cell whose own spectrum is empty: the T_max proposal), in
      // binary32 from two per-cell factors (a binary64 division per point would
      // keep the narrow binary64 pipe busy for most of the kernel)
      const double l = pos ? lam : 0.0;
      const float c0 = (float)(1.0 - l), c1 = pos ? (float)(l / part) : 0.f;
      for (int k = lane; k < K; k += 32) qw[k] = fmaf(c1, qw[k], c0 * a.p0[k]);
      __syncwarp();
    }
    quantize_cell(qw, 0.5f, a.nb, a.ng, wn, a.cell_cn + c * a.nb, a.cell_cg + c * (long long)K,
                  a.cell_hemi + c, a.err);
  }
}

// ---- network: shared-memory weights ------------------------------------------------
// W1T [12][64], W2T [64][64] (input-major, for the forward pass), W3T [64][LDO]
// with LDO an odd number of 32-bit words so that both the forward pass (lanes
// along outputs) and the backward pass (lanes along inputs) are free of bank
// conflicts.

__host__ __device__ inline int ldo_halves(int K) { return 2 * ((((K + 2) + 1) / 2) | 1); }

struct MlpSmem {
  __half *W1T, *W2T, *W2, *W3T;
  float *b1, *b2, *b3;
};

__device__ void load_weights(const __half *th, int K, const MlpSmem &S, bool need_w2) {
  const int ldo = ldo_halves(K);
  const __half *W1 = th, *W2 = W1 + NH * NF + NH, *W3 = W2 + NH * NH + NH;
  const __half *b1 = W1 + NH * NF, *b2 = W2 + NH * NH, *b3 = W3 + (size_t)(K + 2) * NH;
  for (int e = threadIdx.x; e < NH * NF; e += blockDim.x) {
    const int o = e / NF, i = e % NF;
    S.W1T[i * NH + o] = W1[e];
  }
  for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) {
    const int o = e / NH, i = e % NH;
    S.W2T[i * NH + o] = W2[e];
    if (need_w2) S.W2[e] = W2[e];
  }
  for (int e = threadIdx.x; e < (K + 2) * NH; e += blockDim.x) {
    const int o = e / NH, i = e % NH;
    S.W3T[i * ldo + o] = W3[e];
  }
  for (int e = threadIdx.x; e < NH; e += blockDim.x) {
    S.b1[e] = __half2float(b1[e]);
    S.b2[e] = __half2float(b2[e]);
  }
  for (int e = threadIdx.x; e < K + 2; e += blockDim.x) S.b3[e] = __half2float(b3[e]);
}

// Forward pass of `rows` cells whose normalised features are in X [T][12]:
// A1, H1, A2, H2 [T][64] (A* may be null) and logits Z [T][K+2].
template <int T>
__device__ void forward_tile(const MlpSmem &S, int K, const float *X, float *A1, float *H1,
                             float *A2, float *H2, float *Z) {
  const int ldo = ldo_halves(K);
  for (int e = threadIdx.x; e < T * NH; e += blockDim.x) {
    const int c = e / NH, o = e % NH;
    float a = S.b1[o];
#pragma unroll
    for (int i = 0; i < NF; ++i) a += __half2float(S.W1T[i * NH + o]) * X[c * NF + i];
    if (A1) A1[e] = a;
    H1[e] = gelu(a);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < T * NH; e += blockDim.x) {
    const int c = e / NH, o = e % NH;
    float a = S.b2[o];
#pragma unroll 8
    for (int i = 0; i < NH; ++i) a += __half2float(S.W2T[i * NH + o]) * H1[c * NH + i];
    if (A2) A2[e] = a;
    H2[e] = gelu(a);
  }
  __syncthreads();
  const int KO = K + 2;
  for (int e = threadIdx.x; e < T * KO; e += blockDim.x) {
    const int c = e / KO, o = e % KO;
    float a = S.b3[o];
#pragma unroll 8
    for (int i = 0; i < NH; ++i) a += __half2float(S.W3T[i * ldo + o]) * H2[c * NH + i];
    Z[e] = a;
  }
  __syncthreads();
}

// Inference form of forward_tile (same sums in the same order, so the same
// bits): the two 64-wide layers are blocked over CB = 8 cells, each thread holding
// CB accumulators of one output column, so a weight read from shared memory
// serves CB cells and the activations are broadcast reads.
template <int T>
__device__ void forward_tile_infer(const MlpSmem &S, int K, const float *X, float *H1, float *H2,
                                   float *Z) {
  constexpr int CB = 8;
  static_assert(T % CB == 0, "cell blocks");
  const int ldo = ldo_halves(K);
  for (int e = threadIdx.x; e < T * NH; e += blockDim.x) {
    const int c = e / NH, o = e % NH;
    float a = S.b1[o];
#pragma unroll
    for (int i = 0; i < NF; ++i) a += __half2float(S.W1T[i * NH + o]) * X[c * NF + i];
    H1[e] = gelu(a);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (T / CB) * NH; e += blockDim.x) {
    const int cb = e / NH, o = e % NH;
    float acc[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) acc[j] = S.b2[o];
    const float *h = H1 + (size_t)cb * CB * NH;
#pragma unroll 4
    for (int i = 0; i < NH; ++i) {
      const float w = __half2float(S.W2T[i * NH + o]);
#pragma unroll
      for (int j = 0; j < CB; ++j) acc[j] += w * h[j * NH + i];
    }
#pragma unroll
    for (int j = 0; j < CB; ++j) H2[(cb * CB + j) * NH + o] = gelu(acc[j]);
  }
  __syncthreads();
  const int KO = K + 2;
  for (int e = threadIdx.x; e < (T / CB) * KO; e += blockDim.x) {
    const int cb = e / KO, o = e % KO;
    float acc[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) acc[j] = S.b3[o];
    const float *h = H2 + (size_t)cb * CB * NH;
#pragma unroll 4
    for (int i = 0; i < NH; ++i) {
      const float w = __half2float(S.W3T[i * ldo + o]);
#pragma unroll
      for (int j = 0; j < CB; ++j) acc[j] += w * h[j * NH + i];
    }
#pragma unroll
    for (int j = 0; j < CB; ++j) Z[(size_t)(cb * CB + j) * KO + o] = acc[j];
  }
  __syncthreads();
}

size_t infer_smem_bytes(int K) {
  const size_t halves = (size_t)NF * NH + NH * NH + (size_t)NH * ldo_halves(K);
  const size_t floats = 2 * NH + (K + 2) + IT * NF + 2 * IT * NH + (size_t)IT * (K + 2) + K + 2 * NF;
  return ((halves * 2 + 15) / 16) * 16 + floats * 4 + 64;
}

__global__ void __launch_bounds__(NTHR) mlp_infer_kernel(const MlpInferArgs a) {
  extern __shared__ __align__(16) unsigned char ism[];
  const int K = a.K, KO = K + 2, ldo = ldo_halves(K);
  MlpSmem S;
  __half *hp = reinterpret_cast<__half *>(ism);
  S.W1T = hp;
  S.W2T = S.W1T + NF * NH;
  S.W2 = nullptr;
  S.W3T = S.W2T + NH * NH;
  const size_t halves = (size_t)NF * NH + NH * NH + (size_t)NH * ldo;
  float *fp = reinterpret_cast<float *>(ism + ((halves * 2 + 15) / 16) * 16);
  S.b1 = fp;
  S.b2 = S.b1 + NH;
  S.b3 = S.b2 + NH;
  float *X = S.b3 + KO;
  float *H1 = X + IT * NF, *H2 = H1 + IT * NH, *Z = H2 + IT * NH;
  float *p0s = Z + (size_t)IT * KO;
  float *nrm = p0s + K;  // fmean [12], finv [12]
  load_weights(a.theta16, K, S, false);
  for (int e = threadIdx.x; e < NF; e += blockDim.x) {
    nrm[e] = a.fmean[e];
    nrm[NF + e] = a.finv[e];
  }
  if (a.p0_stride == 0)
    for (int e = threadIdx.x; e < K; e += blockDim.x) p0s[e] = a.p0[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long ntiles = (a.n + IT - 1) / IT;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long t0 = tile * IT;
    const int rows = (int)min((long long)IT, a.n - t0);
    for (int e = threadIdx.x; e < IT * NF; e += blockDim.x) {
      const int c = e / NF, i = e % NF;
      X[e] = c < rows ? (a.feat[(t0 + c) * NF + i] - nrm[i]) * nrm[NF + i] : 0.f;
    }
    __syncthreads();
    forward_tile_infer<IT>(S, K, X, H1, H2, Z);
    // softmax over the spectral logits and the hemisphere pair, then the mixture
    for (int c = w; c < rows; c += NTHR / 32) {
      float *z = Z + (size_t)c * KO;
      const float *p0 = a.p0_stride ? a.p0 + (t0 + c) * (long long)a.p0_stride : p0s;
      float mx = -INFINITY;
      for (int k = lane; k < K; k += 32) mx = fmaxf(mx, z[k]);
      mx = warp_max(mx);
      float sum = 0.f;
      for (int k = lane; k < K; k += 32) sum += expf(z[k] - mx);
      sum = warp_sum(sum);
      const float inv = 1.f / sum;
      const float hm = fmaxf(z[K], z[K + 1]);
      const float eu = expf(z[K] - hm), ed = expf(z[K + 1] - hm);
      __syncwarp();
      for (int k = lane; k < K; k += 32)
        z[k] = (1.f - a.mix) * (expf(z[k] - mx) * inv) + a.mix * p0[k];
      __syncwarp();
      if (lane == 0) {
        z[K] = (1.f - a.mix) * (eu / (eu + ed)) + a.mix * 0.5f;
        z[K + 1] = (1.f - a.mix) * (ed / (eu + ed)) + a.mix * 0.5f;
      }
      __syncwarp();
      for (int k = lane; k < KO; k += 32) a.q_out[(t0 + c) * KO + k] = z[k];
    }
    __syncthreads();
  }
}

// ---- inference on the tensor cores ------------------------------------------------
// The two 64-wide layers and the output layer are contractions of FP16 weights
// with FP32 activations: mma.sync m16n8k16 (FP16 operands, FP32 accumulation)
// over tiles of 16 cells.  Each activation h is split into FP16 parts hi =
// RN16(h), lo = RN16(h - hi) (h = hi + lo to about 2^-22 relative) and every
// product is taken twice, W hi + W lo: the weights are FP16 numbers already, so
// the layers keep about binary32 accuracy.  The 12-wide input layer stays on the
// FP32 units (3% of the work).  Weights W2 [64][LDK] and W3 [n-tiles * 8][LDK]
// are stored row by output ([n][k], the m16n8k16 B operand), activations
// [cell][LDK]: with LDK = 72 halves (36 words) the fragment loads are free of
// bank conflicts; the logits go to Z [16][LDZ] with LDZ = 8 (mod 32) words.
constexpr int ITC = 16;   // cells per tensor-core tile
constexpr int LDK = 72;   // halves per row of W2, W3 and the activations
__host__ __device__ inline int tc_ntiles(int K) { return (K + 2 + 7) / 8; }
__host__ __device__ inline int tc_ldz(int K) { return ((K + 2 + 23) / 32) * 32 + 8; }

__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// hi/lo FP16 parts of two neighbouring activations, stored as half2 words
__device__ __forceinline__ void split_store(__half *hi, __half *lo, int off, float v0, float v1) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  *reinterpret_cast<__half2 *>(hi + off) = h;
  *reinterpret_cast<__half2 *>(lo + off) = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
}

// One 16 x 8 output tile of a 64-deep layer: D = sum_k (Ahi + Alo)[16][k] W[n0 + .][k]
__device__ __forceinline__ void mma_tile64(const __half *Ahi, const __half *Alo, const __half *W, int n0,
                                           int lane, float (&d)[4]) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int k0 = 0; k0 < NH; k0 += 16) {
    const __half *wrow = W + (size_t)(n0 + g) * LDK + k0 + 2 * t;
    const unsigned b0 = *reinterpret_cast<const unsigned *>(wrow);
    const unsigned b1 = *reinterpret_cast<const unsigned *>(wrow + 8);
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      const __half *A = part ? Alo : Ahi;
      unsigned a[4];
      a[0] = *reinterpret_cast<const unsigned *>(A + g * LDK + k0 + 2 * t);
      a[1] = *reinterpret_cast<const unsigned *>(A + (g + 8) * LDK + k0 + 2 * t);
      a[2] = *reinterpret_cast<const unsigned *>(A + g * LDK + k0 + 2 * t + 8);
      a[3] = *reinterpret_cast<const unsigned *>(A + (g + 8) * LDK + k0 + 2 * t + 8);
      mma16816(d, a, b0, b1);
    }
  }
}

// The A fragments of a 16 x 64 activation tile (hi and lo parts) for every k0,
// loaded once per warp and reused for all of its output n-tiles.
__device__ __forceinline__ void load_afrag(const __half *A, int lane, unsigned (&f)[NH / 16][4]) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < NH / 16; ++j) {
    const int k0 = 16 * j;
    f[j][0] = *reinterpret_cast<const unsigned *>(A + g * LDK + k0 + 2 * t);
    f[j][1] = *reinterpret_cast<const unsigned *>(A + (g + 8) * LDK + k0 + 2 * t);
    f[j][2] = *reinterpret_cast<const unsigned *>(A + g * LDK + k0 + 2 * t + 8);
    f[j][3] = *reinterpret_cast<const unsigned *>(A + (g + 8) * LDK + k0 + 2 * t + 8);
  }
}

// mma_tile64 with the A fragments in registers: the same products in the same
// order (k0 ascending, the hi part before the lo part).
__device__ __forceinline__ void mma_tile64_frag(const unsigned (&ahi)[NH / 16][4], const unsigned (&alo)[NH / 16][4],
                                                const __half *W, int n0, int lane, float (&d)[4]) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < NH / 16; ++j) {
    const __half *wrow = W + (size_t)(n0 + g) * LDK + 16 * j + 2 * t;
    const unsigned b0 = *reinterpret_cast<const unsigned *>(wrow);
    const unsigned b1 = *reinterpret_cast<const unsigned *>(wrow + 8);
    mma16816(d, ahi[j], b0, b1);
    mma16816(d, alo[j], b0, b1);
  }
}

size_t infer_tc_smem_bytes(int K) {
  const size_t halves = (size_t)NF * NH + (size_t)NH * LDK + (size_t)tc_ntiles(K) * 8 * LDK + 4 * ITC * LDK;
  const size_t floats = 2 * NH + (size_t)tc_ntiles(K) * 8 + ITC * NF + (size_t)ITC * tc_ldz(K) + K + 2 * NF;
  return ((halves * 2 + 15) / 16) * 16 + floats * 4 + 64;
}

__global__ void __launch_bounds__(NTHR, 1) mlp_infer_tc_kernel(const MlpInferArgs a) {
  extern __shared__ __align__(16) unsigned char tcs[];
  const int K = a.K, KO = K + 2, NT = tc_ntiles(K), ldz = tc_ldz(K);
  __half *W1T = reinterpret_cast<__half *>(tcs);  // [12][64]
  __half *W2 = W1T + NF * NH;                     // [64][LDK]
  __half *W3 = W2 + NH * LDK;                     // [NT * 8][LDK]
  __half *H1h = W3 + (size_t)NT * 8 * LDK, *H1l = H1h + ITC * LDK;
  __half *H2h = H1l + ITC * LDK, *H2l = H2h + ITC * LDK;
  const size_t halves = (size_t)NF * NH + (size_t)NH * LDK + (size_t)NT * 8 * LDK + 4 * ITC * LDK;
  float *b1 = reinterpret_cast<float *>(tcs + ((halves * 2 + 15) / 16) * 16);
  float *b2 = b1 + NH, *b3 = b2 + NH;  // b3 [NT * 8]
  float *X = b3 + NT * 8, *Z = X + ITC * NF;  // Z [16][ldz]
  float *p0s = Z + (size_t)ITC * ldz, *nrm = p0s + K;
  {
    const __half *tW1 = a.theta16, *tW2 = tW1 + NH * NF + NH, *tW3 = tW2 + NH * NH + NH;
    const __half *tb1 = tW1 + NH * NF, *tb2 = tW2 + NH * NH, *tb3 = tW3 + (size_t)KO * NH;
    for (int e = threadIdx.x; e < NH * NF; e += blockDim.x) W1T[(e % NF) * NH + e / NF] = tW1[e];
    for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) W2[(e / NH) * LDK + e % NH] = tW2[e];
    for (int e = threadIdx.x; e < NT * 8 * NH; e += blockDim.x) {
      const int o = e / NH, i = e % NH;
      W3[o * LDK + i] = o < KO ? tW3[(size_t)o * NH + i] : __float2half(0.f);
    }
    for (int e = threadIdx.x; e < NH; e += blockDim.x) {
      b1[e] = __half2float(tb1[e]);
      b2[e] = __half2float(tb2[e]);
    }
    for (int e = threadIdx.x; e < NT * 8; e += blockDim.x) b3[e] = e < KO ? __half2float(tb3[e]) : 0.f;
    for (int e = threadIdx.x; e < NF; e += blockDim.x) {
      nrm[e] = a.fmean[e];
      nrm[NF + e] = a.finv[e];
    }
    if (a.p0_stride == 0)
      for (int e = threadIdx.x; e < K; e += blockDim.x) p0s[e] = a.p0[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const long long ntiles = (a.n + ITC - 1) / ITC;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long t0 = tile * ITC;
    const int rows = (int)min((long long)ITC, a.n - t0);
    for (int e = threadIdx.x; e < ITC * NF; e += blockDim.x) {
      const int c = e / NF, i = e % NF;
      X[e] = c < rows ? (a.feat[(t0 + c) * NF + i] - nrm[i]) * nrm[NF + i] : 0.f;
    }
    __syncthreads();
    // input layer (FP32): two neighbouring outputs per thread
    for (int e = threadIdx.x; e < ITC * NH / 2; e += blockDim.x) {
      const int c = e / (NH / 2), o = 2 * (e % (NH / 2));
      float h0 = b1[o], h1 = b1[o + 1];
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const float x = X[c * NF + i];
        h0 += __half2float(W1T[i * NH + o]) * x;
        h1 += __half2float(W1T[i * NH + o + 1]) * x;
      }
      split_store(H1h, H1l, c * LDK + o, gelu(h0), gelu(h1));
    }
    __syncthreads();
    // hidden layer: warp w computes outputs 8w .. 8w + 7
    {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tile64(H1h, H1l, W2, 8 * w, lane, d);
      const int o = 8 * w + 2 * t;
      split_store(H2h, H2l, g * LDK + o, gelu(d[0] + b2[o]), gelu(d[1] + b2[o + 1]));
      split_store(H2h, H2l, (g + 8) * LDK + o, gelu(d[2] + b2[o]), gelu(d[3] + b2[o + 1]));
    }
    __syncthreads();
    // output layer: the n-tiles round-robin over the warps
    unsigned ahi[NH / 16][4], alo[NH / 16][4];
    load_afrag(H2h, lane, ahi);
    load_afrag(H2l, lane, alo);
    for (int nt = w; nt < NT; nt += NTHR / 32) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tile64_frag(ahi, alo, W3, 8 * nt, lane, d);
      const int o = 8 * nt + 2 * t;
      *reinterpret_cast<float2 *>(Z + g * ldz + o) = make_float2(d[0] + b3[o], d[1] + b3[o + 1]);
      *reinterpret_cast<float2 *>(Z + (g + 8) * ldz + o) = make_float2(d[2] + b3[o], d[3] + b3[o + 1]);
    }
    __syncthreads();
    // softmax over the spectral logits and the hemisphere pair, then the mixture
    // (mlp_infer_kernel's expressions; each lane keeps to its own logits, so each
    // exponential is evaluated once and kept in place, and the mixture is
    // written straight out)
    for (int c = w; c < rows; c += NTHR / 32) {
      float *z = Z + (size_t)c * ldz;
      float *qo = a.q_out + (t0 + c) * KO;
      const float *p0 = a.p0_stride ? a.p0 + (t0 + c) * (long long)a.p0_stride : p0s;
      float mx = -INFINITY;
      for (int k = lane; k < K; k += 32) mx = fmaxf(mx, z[k]);
      mx = warp_max(mx);
      float sum = 0.f;
      for (int k = lane; k < K; k += 32) {
        const float e = expf(z[k] - mx);
        z[k] = e;
        sum += e;
      }
      sum = warp_sum(sum);
      const float inv = 1.f / sum;
      for (int k = lane; k < K; k += 32) qo[k] = (1.f - a.mix) * (z[k] * inv) + a.mix * p0[k];
      if (lane == 0) {
        const float hm = fmaxf(z[K], z[K + 1]);
        const float eu = expf(z[K] - hm), ed = expf(z[K + 1] - hm);
        qo[K] = (1.f - a.mix) * (eu / (eu + ed)) + a.mix * 0.5f;
        qo[K + 1] = (1.f - a.mix) * (ed / (eu + ed)) + a.mix * 0.5f;
      }
    }
    __syncthreads();
  }
}

// ---- training ------------------------------------------------------------------
// Persistent CTAs; each takes tiles of TT samples of the batch, runs the forward
// pass, the loss gradient with respect to the logits, and the backward pass,
// accumulating its share of the gradient in shared memory (each entry owned by
// one thread, samples added in order), then writes it to partial[blockIdx.x].
// grad_reduce_kernel adds the CTAs' partials in order: the gradient does not
// depend on timing.

size_t train_smem_bytes(int K) {
  const int KO = K + 2;
  const size_t halves = (size_t)NF * NH + 2 * NH * NH + (size_t)NH * ldo_halves(K);
  const size_t grads = (size_t)NF * NH + NH + NH * NH + NH + (size_t)NH * KO + KO;
  const size_t floats = 2 * NH + KO + grads + TT * NF + 6 * TT * NH + (size_t)TT * KO + 2 * NF + 8;
  return ((halves * 2 + 15) / 16) * 16 + floats * 4 + 16;
}

__global__ void __launch_bounds__(NTHR, 1) mlp_train_kernel(const MlpTrainArgs a) {
  extern __shared__ __align__(16) unsigned char tsm2[];
  const int K = a.K, KO = K + 2, ldo = ldo_halves(K);
  MlpSmem S;
  __half *hp = reinterpret_cast<__half *>(tsm2);
  S.W1T = hp;
  S.W2T = S.W1T + NF * NH;
  S.W2 = S.W2T + NH * NH;
  S.W3T = S.W2 + NH * NH;
  const size_t halves = (size_t)NF * NH + 2 * NH * NH + (size_t)NH * ldo;
  float *fp = reinterpret_cast<float *>(tsm2 + ((halves * 2 + 15) / 16) * 16);
  S.b1 = fp;
  S.b2 = S.b1 + NH;
  S.b3 = S.b2 + NH;
  float *gW1T = S.b3 + KO, *gb1 = gW1T + NF * NH, *gW2T = gb1 + NH, *gb2 = gW2T + NH * NH,
        *gW3T = gb2 + NH, *gb3 = gW3T + (size_t)NH * KO;
  float *X = gb3 + KO, *A1 = X + TT * NF, *H1 = A1 + TT * NH, *A2 = H1 + TT * NH, *H2 = A2 + TT * NH,
        *dA2 = H2 + TT * NH, *dA1 = dA2 + TT * NH, *Z = dA1 + TT * NH;
  float *nrm = Z + (size_t)TT * KO;
  __shared__ double s_loss;
  __shared__ float s_lsamp[TT];
  __shared__ double s_stat[TT][4];
  __shared__ double s_tot[4];
  __shared__ double s_bs[4];
  load_weights(a.theta16, K, S, true);
  const long long ngrad = (long long)NF * NH + NH + NH * NH + NH + (long long)NH * KO + KO;
  for (long long e = threadIdx.x; e < ngrad; e += blockDim.x) gW1T[e] = 0.f;
  for (int e = threadIdx.x; e < NF; e += blockDim.x) {
    nrm[e] = a.fmean[e];
    nrm[NF + e] = a.finv[e];
  }
  if (threadIdx.x == 0) {
    s_loss = 0.0;
    for (int j = 0; j < 4; ++j) {
      s_tot[j] = 0.0;
      s_bs[j] = a.bsum ? a.bsum[j] : 0.0;
    }
  }
  const bool stats_only = a.mode == 1 && a.pass == 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float invB = 1.f / (float)a.n;
  const long long ntiles = (a.n + TT - 1) / TT;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long t0 = tile * TT;
    const int rows = (int)min((long long)TT, a.n - t0);
    for (int e = threadIdx.x; e < TT * NF; e += blockDim.x) {
      const int c = e / NF, i = e % NF;
      float v = 0.f;
      if (c < rows) {
        const long long smp = a.idx ? (long long)a.idx[t0 + c] : t0 + c;
        if (smp >= 0 && smp < a.n_data) v = (a.feat[smp * NF + i] - nrm[i]) * nrm[NF + i];
      }
      X[e] = v;
    }
    __syncthreads();
    forward_tile<TT>(S, K, X, A1, H1, A2, H2, Z);
    // loss and its gradient with respect to the logits, one warp per sample
    for (int c = w; c < TT; c += NTHR / 32) {
      float *z = Z + (size_t)c * KO;
      if (lane == 0) {
        s_lsamp[c] = 0.f;
        for (int j = 0; j < 4; ++j) s_stat[c][j] = 0.0;
      }
      if (c >= rows) {
        for (int k = lane; k < KO; k += 32) z[k] = 0.f;
        continue;
      }
      const long long smp = a.idx ? (long long)a.idx[t0 + c] : t0 + c;
      if (smp < 0 || smp >= a.n_data) {  // outside the dataset: no contribution
        if (lane == 0) atomicOr(a.err, 1ull);
        for (int k = lane; k < KO; k += 32) z[k] = 0.f;
        continue;
      }
      const float *m = a.mom + smp * 2 * K;
      const float *cs = a.cost ? a.cost + smp * 2 * K : nullptr;
      const float *p0 = a.p0 + smp * (long long)a.p0_stride;
      float mx = -INFINITY;
      for (int k = lane; k < K; k += 32) mx = fmaxf(mx, z[k]);
      mx = warp_max(mx);
      float sum = 0.f;
      for (int k = lane; k < K; k += 32) sum += expf(z[k] - mx);
      sum = warp_sum(sum);
      const float inv = 1.f / sum;
      const float hm = fmaxf(z[K], z[K + 1]);
      const float eu = expf(z[K] - hm), ed = expf(z[K + 1] - hm);
      const float tu = eu / (eu + ed), td = ed / (eu + ed);
      const float qu = (1.f - a.mix) * tu + a.mix * 0.5f, qd = (1.f - a.mix) * td + a.mix * 0.5f;
      float A0 = 0.f, Aq = 0.f, C0 = 0.f, Cq = 0.f;
      for (int k = lane; k < K; k += 32) {
        const float pk = p0[k];
        if (!(pk > 0.f)) continue;
        const float qk = (1.f - a.mix) * (expf(z[k] - mx) * inv) + a.mix * pk;
        const float mu = m[2 * k], md = m[2 * k + 1];
        A0 += (mu + md) / (pk * 0.5f);
        Aq += mu / (qk * qu) + md / (qk * qd);
        if (cs) {
          C0 += (cs[2 * k] + cs[2 * k + 1]) * (pk * 0.5f);
          Cq += cs[2 * k] * (qk * qu) + cs[2 * k + 1] * (qk * qd);
        }
      }
      A0 = warp_sum(A0);
      Aq = warp_sum(Aq);
      if (cs) {
        C0 = warp_sum(C0) + a.c0;
        Cq = warp_sum(Cq) + a.c0;
      } else {
        C0 = Cq = 1.f;
      }
      // multipliers dL/dA(q), dL/dC(q) of this sample
      float gA, gC;
      if (a.mode == 1) {
        const float wc = a.wgt ? a.wgt[smp] : 1.f;
        if (lane == 0) {
          s_stat[c][0] = (double)wc * Aq;
          s_stat[c][1] = (double)wc * A0;
          s_stat[c][2] = Cq;
          s_stat[c][3] = C0;
        }
        if (stats_only) continue;
        const float den = (float)(s_bs[1] * s_bs[3]);
        gA = wc * (float)s_bs[2] / den;
        gC = cs ? (float)s_bs[0] / den : 0.f;
      } else {
        if (!(A0 > 0.f) || !(C0 > 0.f)) {
          __syncwarp();
          for (int k = lane; k < KO; k += 32) z[k] = 0.f;
          continue;
        }
        const float norm = A0 * C0;
        if (lane == 0) s_lsamp[c] = Aq * Cq / norm;
        gA = invB * Cq / norm;
        gC = cs ? invB * Aq / norm : 0.f;
      }
      // dL/dq_k and the hemisphere gradients; then through the softmaxes
      float dot = 0.f, gu = 0.f, gd = 0.f;
      for (int k = lane; k < K; k += 32) {
        const float pk = p0[k];
        if (!(pk > 0.f)) continue;
        const float sk = expf(z[k] - mx) * inv;
        const float qk = (1.f - a.mix) * sk + a.mix * pk;
        const float mu = m[2 * k], md = m[2 * k + 1];
        float g = -gA * (mu / (qk * qk * qu) + md / (qk * qk * qd));
        gu -= gA * mu / (qk * qu * qu);
        gd -= gA * md / (qk * qd * qd);
        if (cs) {
          g += gC * (cs[2 * k] * qu + cs[2 * k + 1] * qd);
          gu += gC * cs[2 * k] * qk;
          gd += gC * cs[2 * k + 1] * qk;
        }
        dot += sk * g;
      }
      dot = warp_sum(dot);
      gu = warp_sum(gu);
      gd = warp_sum(gd);
      __syncwarp();
      for (int k = lane; k < K; k += 32) {
        const float pk = p0[k];
        const float sk = expf(z[k] - mx) * inv;
        float g = 0.f;
        if (pk > 0.f) {
          const float qk = (1.f - a.mix) * sk + a.mix * pk;
          const float mu = m[2 * k], md = m[2 * k + 1];
          g = -gA * (mu / (qk * qk * qu) + md / (qk * qk * qd));
          if (cs) g += gC * (cs[2 * k] * qu + cs[2 * k + 1] * qd);
        }
        z[k] = (1.f - a.mix) * sk * (g - dot);
      }
      __syncwarp();
      if (lane == 0) {
        const float dh = tu * gu + td * gd;
        z[K] = (1.f - a.mix) * tu * (gu - dh);
        z[K + 1] = (1.f - a.mix) * td * (gd - dh);
      }
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int c = 0; c < rows; ++c) s_loss += (double)s_lsamp[c] * (double)invB;
      for (int c = 0; c < rows; ++c)
        for (int j = 0; j < 4; ++j) s_tot[j] += s_stat[c][j];
    }
    if (stats_only) {
      __syncthreads();
      continue;
    }
    // layer 3: gW3T[i][o] += sum_c H2[c][i] dz[c][o]; gb3; dH2 -> dA2
    for (int e = threadIdx.x; e < NH * KO; e += blockDim.x) {
      const int i = e / KO, o = e % KO;
      float acc = gW3T[e];
#pragma unroll
      for (int c = 0; c < TT; ++c) acc += H2[c * NH + i] * Z[c * KO + o];
      gW3T[e] = acc;
    }
    for (int o = threadIdx.x; o < KO; o += blockDim.x) {
      float acc = gb3[o];
#pragma unroll
      for (int c = 0; c < TT; ++c) acc += Z[c * KO + o];
      gb3[o] = acc;
    }
    for (int e = threadIdx.x; e < TT * NH; e += blockDim.x) {
      const int c = e / NH, i = e % NH;
      float acc = 0.f;
      const float *zc = Z + (size_t)c * KO;
      const __half *wr = S.W3T + (size_t)i * ldo;
      for (int o = 0; o < KO; ++o) acc += __half2float(wr[o]) * zc[o];
      dA2[e] = acc * gelu_prime(A2[e]);
    }
    __syncthreads();
    // layer 2
    for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) {
      const int i = e / NH, o = e % NH;
      float acc = gW2T[e];
#pragma unroll
      for (int c = 0; c < TT; ++c) acc += H1[c * NH + i] * dA2[c * NH + o];
      gW2T[e] = acc;
    }
    for (int o = threadIdx.x; o < NH; o += blockDim.x) {
      float acc = gb2[o];
#pragma unroll
      for (int c = 0; c < TT; ++c) acc += dA2[c * NH + o];
      gb2[o] = acc;
    }
    for (int e = threadIdx.x; e < TT * NH; e += blockDim.x) {
      const int c = e / NH, i = e % NH;
      float acc = 0.f;
#pragma unroll 8
      for (int o = 0; o < NH; ++o) acc += __half2float(S.W2[o * NH + i]) * dA2[c * NH + o];
      dA1[e] = acc * gelu_prime(A1[e]);
    }
    __syncthreads();
    // layer 1
    for (int e = threadIdx.x; e < NF * NH; e += blockDim.x) {
      const int i = e / NH, o = e % NH;
      float acc = gW1T[e];
#pragma unroll
      for (int c = 0; c < TT; ++c) acc += X[c * NF + i] * dA1[c * NH + o];
      gW1T[e] = acc;
    }
    for (int o = threadIdx.x; o < NH; o += blockDim.x) {
      float acc = gb1[o];
#pragma unroll
      for (int c = 0; c < TT; ++c) acc += dA1[c * NH + o];
      gb1[o] = acc;
    }
    __syncthreads();
  }
  if (stats_only) {
    __syncthreads();
    if (threadIdx.x < 4) a.stat_partial[(size_t)blockIdx.x * 4 + threadIdx.x] = s_tot[threadIdx.x];
    return;
  }
  // this CTA's share, in theta's layout
  float *out = a.partial + (size_t)blockIdx.x * ngrad;
  const long long oW1 = 0, ob1 = NH * NF, oW2 = ob1 + NH, ob2 = oW2 + NH * NH, oW3 = ob2 + NH,
                  ob3 = oW3 + (long long)KO * NH;
  for (int e = threadIdx.x; e < NH * NF; e += blockDim.x) {
    const int o = e / NF, i = e % NF;
    out[oW1 + e] = gW1T[i * NH + o];
  }
  for (int e = threadIdx.x; e < NH; e += blockDim.x) {
    out[ob1 + e] = gb1[e];
    out[ob2 + e] = gb2[e];
  }
  for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) {
    const int o = e / NH, i = e % NH;
    out[oW2 + e] = gW2T[i * NH + o];
  }
  for (int e = threadIdx.x; e < KO * NH; e += blockDim.x) {
    const int o = e / NH, i = e % NH;
    out[oW3 + e] = gW3T[(size_t)i * KO + o];
  }
  for (int e = threadIdx.x; e < KO; e += blockDim.x) out[ob3 + e] = gb3[e];
  __syncthreads();
  if (threadIdx.x == 0) a.loss_partial[blockIdx.x] = s_loss;
}

__global__ void grad_reduce_kernel(const float *partial, const double *loss_partial, int grid,
                                   long long np, const double *bsum, float *grad, double *loss) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np;
       j += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int b = 0; b < grid; ++b) acc += partial[(size_t)b * np + j];
    grad[j] = acc;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double l = 0.0;
    if (bsum) {
      l = (bsum[0] / bsum[1]) * (bsum[2] / bsum[3]);
    } else {
      for (int b = 0; b < grid; ++b) l += loss_partial[b];
    }
    *loss = l;
  }
}

__global__ void stat_reduce_kernel(const double *stat_partial, int grid, double *bsum) {
  if (threadIdx.x < 4) {
    double acc = 0.0;
    for (int b = 0; b < grid; ++b) acc += stat_partial[(size_t)b * 4 + threadIdx.x];
    bsum[threadIdx.x] = acc;
  }
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the FP32 master weights; the FP16
// copy the network runs with is refreshed in the same pass.
__global__ void adam_kernel(float *theta, __half *theta16, const float *grad, float *m1, float *m2,
                            long long np, float lr, float beta1, float beta2, float eps, float c1,
                            float c2) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np;
       j += (long long)gridDim.x * blockDim.x) {
    const float g = grad[j];
    const float a = beta1 * m1[j] + (1.f - beta1) * g;
    const float b = beta2 * m2[j] + (1.f - beta2) * g * g;
    m1[j] = a;
    m2[j] = b;
    const float t = theta[j] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    theta[j] = t;
    theta16[j] = __float2half_rn(t);
  }
}

__global__ void to_half_kernel(const float *theta, __half *theta16, long long np) {
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < np;
       j += (long long)gridDim.x * blockDim.x)
    theta16[j] = __float2half_rn(theta[j]);
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  }
  return n;
}

unsigned grid_for(long long items, int per_block, int per_sm = 8) {
  long long b = (items + per_block - 1) / per_block;
  const long long cap = (long long)num_sms() * per_sm;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

long long mlp_nparams(int K) {
  return (long long)NH * NF + NH + (long long)NH * NH + NH + (long long)(K + 2) * NH + (K + 2);
}

int mlp_train_grid() { return num_sms(); }

cudaError_t launch_features(const FeatArgs &f, cudaStream_t s) {
  if (f.n <= 0) return cudaSuccess;
  features_kernel<<<grid_for(f.n, NTHR), NTHR, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_tally(const TallyArgs &t, cudaStream_t s) {
  if (t.n <= 0) return cudaSuccess;
  const size_t smem = (size_t)TALLY_WARPS * 2 * 2 * t.nb * t.ng * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(tally_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  tally_kernel<<<grid_for(t.n, TALLY_WARPS, 4), TALLY_WARPS * 32, smem, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const MlpInferArgs &a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const size_t tsmem = infer_tc_smem_bytes(a.K);
  if (tsmem <= 200 * 1024) {  // the tensor-core kernel (every K a network here uses)
    cudaError_t e = cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tsmem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_infer_tc_kernel, NTHR, tsmem);
    if (e != cudaSuccess) return e;
    mlp_infer_tc_kernel<<<grid_for(a.n, ITC, per_sm > 0 ? per_sm : 1), NTHR, tsmem, s>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = infer_smem_bytes(a.K);
  cudaError_t e = cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // as many resident CTAs per SM as shared memory allows (two at K = 320)
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_infer_kernel, NTHR, smem);
  if (e != cudaSuccess) return e;
  mlp_infer_kernel<<<grid_for(a.n, IT, per_sm > 0 ? per_sm : 1), NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_quantize_cells(const float *q, long long n, int nb, int ng,
                                  unsigned long long *cell_cn, unsigned long long *cell_cg,
                                  unsigned *cell_hemi, unsigned long long *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = (size_t)(NTHR / 32) * nb * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(quantize_cells_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  quantize_cells_kernel<<<grid_for(n, NTHR / 32, 4), NTHR, smem, s>>>(q, n, nb, ng, cell_cn, cell_cg,
                                                                       cell_hemi, err);
  return cudaGetLastError();
}

cudaError_t launch_spectral_proposal(const SpectralArgs &a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const size_t smem = (size_t)(NTHR / 32) * ((size_t)a.nb + (size_t)a.nb * a.ng) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(spectral_proposal_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  spectral_proposal_kernel<<<grid_for(a.n, NTHR / 32, 4), NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mlp_train(const MlpTrainArgs &a, cudaStream_t s) {
  const size_t smem = train_smem_bytes(a.K);
  cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  mlp_train_kernel<<<a.grid, NTHR, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const float *partial, const double *loss_partial, int grid,
                               long long np, const double *bsum, float *grad, double *loss,
                               cudaStream_t s) {
  grad_reduce_kernel<<<grid_for(np, 256, 2), 256, 0, s>>>(partial, loss_partial, grid, np, bsum, grad,
                                                          loss);
  return cudaGetLastError();
}

cudaError_t launch_stat_reduce(const double *stat_partial, int grid, double *bsum, cudaStream_t s) {
  stat_reduce_kernel<<<1, 32, 0, s>>>(stat_partial, grid, bsum);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *theta, __half *theta16, const float *grad, float *m1, float *m2,
                        long long np, float lr, float beta1, float beta2, float eps, float c1,
                        float c2, cudaStream_t s) {
  adam_kernel<<<grid_for(np, 256, 2), 256, 0, s>>>(theta, theta16, grad, m1, m2, np, lr, beta1, beta2,
                                                   eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_theta_to_half(const float *theta, __half *theta16, long long np, cudaStream_t s) {
  to_half_kernel<<<grid_for(np, 256, 2), 256, 0, s>>>(theta, theta16, np);
  return cudaGetLastError();
}

}  // namespace mcrt

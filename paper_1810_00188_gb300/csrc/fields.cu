// Field staging: packs the temperature T and H2O mole fraction x of every cell
// into the interleaved {T, x} layouts the trace kernel gathers (one 8- or
// 16-byte load per traversed cell), and reduces the maximum / minimum valid
// temperature and the number of rejected cells in the same pass.  The maximum
// feeds T_max of the spectral proposal (Eq. 13).
#include <math.h>

#include "mcrt_internal.h"

namespace mcrt {
namespace {

__global__ void __launch_bounds__(256) pack_fields_kernel(const void *T, const void *x, int fp64_in,
                                                          double x_ref, long long n, double2 *f64,
                                                          unsigned long long *stats) {
  unsigned long long tmax = 0ull, tmin = ~0ull, bad = 0ull;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double t, xv;
    if (fp64_in) {
      t = ((const double *)T)[i];
      xv = x ? ((const double *)x)[i] : x_ref;
    } else {
      t = (double)((const float *)T)[i];
      xv = x ? (double)((const float *)x)[i] : x_ref;
    }
    const bool ok = isfinite(t) && t > 0.0 && isfinite(xv) && xv >= 0.0;
    if (ok) {
      // positive doubles order like their bit patterns
      const unsigned long long b = (unsigned long long)__double_as_longlong(t);
      tmax = b > tmax ? b : tmax;
      tmin = b < tmin ? b : tmin;
    } else {
      ++bad;
    }
    f64[i] = make_double2(t, xv);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, tmax, off);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, tmin, off);
    tmax = a > tmax ? a : tmax;
    tmin = b < tmin ? b : tmin;
    bad += __shfl_xor_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(stats + 0, tmax);
    atomicMin(stats + 1, tmin);
    if (bad) atomicAdd(stats + 2, bad);
  }
}

// Interpolation position of every cell for the FP32 trace kernel: the node index
// t and the fraction of the way to node t+1 (Section 2.2's linear interpolation
// in T), packed as (t << 23) | round(fraction * 2^23), next to x / x_ref.  A
// temperature at or beyond the last node maps to (nT-1, 0), which reads the same
// value as (nT-2, 1) because the last node's slope is stored as 0.  Computed once
// per field / table change, so the march does no floor, clamp or multiply.
__global__ void __launch_bounds__(256) pack_positions_kernel(const double2 *f64, long long n, double T0,
                                                             double inv_dT, int nT, double inv_xref,
                                                             uint2 *pos) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = f64[i];
    double f = (v.x - T0) * inv_dT;
    if (!(f > 0.0)) f = 0.0;
    if (f > (double)(nT - 1)) f = (double)(nT - 1);
    const double fl = floor(f);
    unsigned t = (unsigned)fl;
    unsigned q = (unsigned)rint((f - fl) * 8388608.0);
    if (q >= 8388608u) {
      q = 0u;
      ++t;
    }
    if (t > (unsigned)(nT - 1)) {
      t = (unsigned)(nT - 1);
      q = 0u;
    }
    pos[i] = make_uint2((t << 23) | q, __float_as_uint((float)(v.y * inv_xref)));
  }
}

// Multigrid (Section 4.3): the fields of the next coarser grid, each coarse cell
// the mean T and mean x of the 2x2x2 finer cells it covers (the coarse
// temperatures come from the fine solution); on a stretched grid the mean is
// weighted by the children's heights (volumes).  The eight values are summed z
// outermost, x innermost.
__global__ void __launch_bounds__(256) coarsen_kernel(const double2 *__restrict__ fine, int n0, int n1,
                                                      int n2, double2 *__restrict__ coarse,
                                                      const double *__restrict__ yf, int level) {
  const int c0 = n0 / 2, c1 = n1 / 2, c2 = n2 / 2;
  const long long nc = (long long)c0 * c1 * c2;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
       i += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(i % c0), J = (int)((i / c0) % c1), K = (int)(i / ((long long)c0 * c1));
    double t = 0.0, x = 0.0, ws = 0.0, w[2] = {1.0, 1.0};
    if (yf) {
      w[0] = yf[(size_t)(2 * J + 1) << level] - yf[(size_t)(2 * J) << level];
      w[1] = yf[(size_t)(2 * J + 2) << level] - yf[(size_t)(2 * J + 1) << level];
    }
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const double2 v =
              fine[(size_t)(2 * I + a) + (size_t)n0 * ((size_t)(2 * J + b) + (size_t)n1 * (2 * K + c))];
          if (yf) {
            t += w[b] * v.x;
            x += w[b] * v.y;
            ws += w[b];
          } else {
            t += v.x;
            x += v.y;
          }
        }
    coarse[i] = yf ? make_double2(t / ws, x / ws) : make_double2(t * 0.125, x * 0.125);
  }
}

}  // namespace

int multigrid_levels(int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1) return 0;
  int n[3] = {nx, ny, nz}, L = 1;
  while (L < 16) {
    bool ok = true;
    for (int a = 0; a < 3; ++a)
      if (n[a] % 2 != 0 || n[a] / 2 < 3) ok = false;
    if (!ok) break;
    for (int a = 0; a < 3; ++a) n[a] /= 2;
    ++L;
  }
  return L;
}

long long grid_stride_blocks() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 16;
  if (sms[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    sms[dev] = n;
  }
  return 16LL * sms[dev];
}

long long multigrid_cells(int nx, int ny, int nz, int levels) {
  long long total = 0;
  for (int l = 0; l < levels; ++l) total += (long long)(nx >> l) * (ny >> l) * (nz >> l);
  return total;
}

cudaError_t launch_coarsen(const double2 *fine, int n0, int n1, int n2, double2 *coarse,
                           const double *yf, int level, cudaStream_t s) {
  const long long nc = (long long)(n0 / 2) * (n1 / 2) * (n2 / 2);
  if (nc <= 0) return cudaSuccess;
  long long blocks = (nc + 255) / 256;
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();
  coarsen_kernel<<<(unsigned)blocks, 256, 0, s>>>(fine, n0, n1, n2, coarse, yf, level);
  return cudaGetLastError();
}

cudaError_t launch_pack_positions(const double2 *f64, long long n, double T0, double inv_dT, int nT,
                                  double inv_xref, uint2 *pos, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();
  pack_positions_kernel<<<(unsigned)blocks, 256, 0, s>>>(f64, n, T0, inv_dT, nT, inv_xref, pos);
  return cudaGetLastError();
}

cudaError_t launch_pack_fields(const void *T, const void *x, int fp64_in, double x_ref,
                               long long n, double2 *f64,
                               unsigned long long *stats, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(stats, 0, 3 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(stats + 1, 0xff, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();  // grid-stride
  pack_fields_kernel<<<(unsigned)blocks, 256, 0, s>>>(T, x, fp64_in, x_ref, n, f64, stats);
  return cudaGetLastError();
}

}  // namespace mcrt

// Machine ceilings for the traversal's roofline: the special-function unit's
// base-2 exponential rate (a march step evaluates one exponential, for the
// transmissivity of the segment, Eq. 10) and the rate of random 8-byte loads
// (a march step gathers the {T, x} of the cell it crosses and two table
// entries).  Neither is part of the method; they are measured on the machine
// the solve runs on, because the nominal rates of these units are not what a
// dependent gather loop sees.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mcrt.h"

namespace {

constexpr int CHAINS = 8;   // independent dependency chains per thread
constexpr int THREADS = 256;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Each thread iterates x <- 2^(-x) on CHAINS independent values (the fixed point
// is near 0.64, so every value stays finite).  Thread 0 of block 0 records SM
// cycles and global nanoseconds around its loop for the clock estimate.
__global__ void __launch_bounds__(THREADS) ex2_rate_kernel(float *out, int iters,
                                                           unsigned long long *clk) {
  float x[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) x[j] = 0.05f * j + 1e-7f * threadIdx.x;
  const bool rec = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long c0 = 0, t0 = 0;
  if (rec) {
    t0 = global_ns();
    c0 = clock64();
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) x[j] = ex2_approx(-x[j]);
  }
  if (rec) {
    const unsigned long long c1 = clock64(), t1 = global_ns();
    clk[0] = c1 - c0;
    clk[1] = t1 - t0;
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += x[j];
  out[(size_t)blockIdx.x * THREADS + threadIdx.x] = s;
}

// Each thread issues CHAINS independent 8-byte loads per iteration at indices
// from per-chain 32-bit LCGs (the top log2(n) bits), so the loads of a warp
// fall in different sectors and each index is independent of loaded data.
__global__ void __launch_bounds__(THREADS) gather_rate_kernel(const uint2 *__restrict__ buf, int shift,
                                                              int iters, unsigned *out) {
  const unsigned tid = blockIdx.x * THREADS + threadIdx.x;
  unsigned s[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s[j] = tid * 2654435761u + 0x9E3779B9u * (j + 1);
  unsigned acc = 0;
  for (int it = 0; it < iters; ++it) {
    uint2 v[CHAINS];
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) {
      s[j] = s[j] * 1664525u + 1013904223u;
      v[j] = __ldg(buf + (s[j] >> shift));
    }
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) acc ^= v[j].x + v[j].y;
  }
  out[tid] = acc;
}

struct DeviceScope {
  int prev = -1;
  bool ok = false;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return MCRT_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? MCRT_E_OOM : MCRT_E_CUDA;
}

// Full-occupancy grid: resident CTAs per SM x SMs.
cudaError_t full_grid(const void *fn, int dev, int *blocks) {
  int sms = 0, per_sm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, 0);
  if (e != cudaSuccess) return e;
  *blocks = sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

// Times launch(): one untimed launch, then one timed with events on a private
// stream.  Returns milliseconds in *ms.
template <class F>
cudaError_t time_launch(cudaStream_t st, F launch, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" int mcrt_probe_ex2(int device, double *per_s, double *sm_mhz) {
  if (!per_s || !sm_mhz) return MCRT_E_ARG;
  DeviceScope g(device);
  if (!g.ok) return MCRT_E_CUDA;
  int blocks = 0;
  cudaError_t e = full_grid((const void *)ex2_rate_kernel, device, &blocks);
  if (e != cudaSuccess) return status_of(e);
  const int iters = 1 << 15;
  float *out = nullptr;
  unsigned long long *clk = nullptr;
  cudaStream_t st = nullptr;
  e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * THREADS);
  if (e == cudaSuccess) e = cudaMalloc(&clk, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  float ms = 0.f;
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess)
    e = time_launch(st, [&] { ex2_rate_kernel<<<blocks, THREADS, 0, st>>>(out, iters, clk); }, &ms);
  if (e == cudaSuccess) e = cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost);
  if (st) cudaStreamDestroy(st);
  if (clk) cudaFree(clk);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return status_of(e);
  if (!(ms > 0.f) || h[1] == 0) return MCRT_E_CUDA;
  *per_s = (double)blocks * THREADS * CHAINS * iters / (ms * 1e-3);
  *sm_mhz = 1e3 * (double)h[0] / (double)h[1];
  return MCRT_OK;
}

extern "C" int mcrt_probe_gather(int device, uint64_t bytes, double *per_s) {
  if (!per_s) return MCRT_E_ARG;
  if (bytes < (1ull << 12) || bytes > (1ull << 35) || (bytes & (bytes - 1))) return MCRT_E_ARG;
  DeviceScope g(device);
  if (!g.ok) return MCRT_E_CUDA;
  int blocks = 0;
  cudaError_t e = full_grid((const void *)gather_rate_kernel, device, &blocks);
  if (e != cudaSuccess) return status_of(e);
  // n = bytes / 8 elements, a power of two: index = the top log2(n) bits
  int log2n = 0;
  while ((1ull << (log2n + 1)) <= bytes / 8) ++log2n;
  const int shift = 32 - log2n;  // 9 <= log2n <= 32: the index fits 32 bits
  const int iters = 1 << 12;
  uint2 *buf = nullptr;
  unsigned *out = nullptr;
  cudaStream_t st = nullptr;
  e = cudaMalloc(&buf, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(unsigned) * (size_t)blocks * THREADS);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x3c, bytes, st);
  float ms = 0.f;
  if (e == cudaSuccess)
    e = time_launch(st, [&] { gather_rate_kernel<<<blocks, THREADS, 0, st>>>(buf, shift, iters, out); }, &ms);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (buf) cudaFree(buf);
  if (e != cudaSuccess) return status_of(e);
  if (!(ms > 0.f)) return MCRT_E_CUDA;
  *per_s = (double)blocks * THREADS * CHAINS * iters / (ms * 1e-3);
  return MCRT_OK;
}

// Host-side state of a context and the helpers shared by the C-ABI source
// files (mcrt_api.cpp, learn_api.cpp).  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mcrt.h"
#include "mcrt_internal.h"

namespace mcrt_host {

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace mcrt_host

struct mcrt_ctx {
  using DevBuf = mcrt_host::DevBuf;
  mcrt_grid_desc grid{};
  std::vector<double> yf;  // stretched grid: the ny + 1 wall-normal faces (empty: uniform)
  // k-distribution (host copy, FP64)
  bool have_kdist = false;
  int nb = 0, ng = 0, nT = 0;
  double T0 = 0, dT = 1, x_ref = 1;
  std::vector<double> w_g, kappa, B;
  // fields
  bool have_fields = false;
  double T_max_field = 0, T_min_field = 0;
  // cell proposal
  bool have_cell_prop = false;
  // plain proposal cache (valid for prop_T_max); p0 its (n, g) probabilities
  bool prop_valid = false;
  double prop_T_max = -1;
  std::vector<float> p0_host;
  double p0_T_max = -1;  // T_max that p0_host / p0_32 were built for
  // device buffers
  DevBuf field64, fpos32, ktab64, ktab32, kbtab32, btab64, btab32, bwall64, bwall32, wg, wg32, wgt32, cn, cg,
      guide, gguide, ybuf, step_acc,
      cell_cn, cell_cg, cell_hemi, counters, fstats, q, sigma, steps;
  // learned proposal: plain probabilities, feature scratch, per-ray steps, error flag
  DevBuf p0_32, feat, ray_steps, lerr, kptab;
  // learned proposal: network outputs of one chunk of cells, before quantisation
  DevBuf qprop;
  // stretched grid: faces in FP64 and FP32
  DevBuf yf64, yf32;
  // long rays handed off by the FP32 exact march (LongRay entries)
  DevBuf longbuf;
  // absorption-based estimate: per-batch sums [2][16][cells]
  DevBuf armcbuf;
  // mcrt_set_fields from host memory: the device copy of T and x before packing
  DevBuf fstage;
  // binary64 tallies of cells with more than one segment: the segments' sums
  DevBuf tpart;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-kernel marks of the last FP32 solve: four events per chunk (launch_trace_fp32)
  std::vector<cudaEvent_t> kev;
  int kev_chunks = 0;
  cudaStream_t last_stream = nullptr;
  bool solved = false;
  int last_launches = 0;
  int min_blocks = 3;
  int steps_per_round = 1;
  int scratch_mib = 4096;
  int long_steps = 1024;    // hand-off threshold in segments (<= 0: never)
  float long_flight = 32;   // x/z crossings left in the flight for a hand-off
  int tally32 = 0;          // per-cell tallies in binary32 pairs instead of binary64
  int claim_rays = 1024;    // FP32 kernels: rays per claimed run of cells
  int tally_plain = 0;      // binary64 tallies by plain loads instead of TMA
  int batch_per_snapshot = 0;  // batches: per-item launches even for one k-distribution
  double last_T_max = 0;
  std::string err;
};

namespace mcrt_host {

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline int fail(mcrt_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

inline int cuda_fail(mcrt_ctx *c, cudaError_t e, const char *where) {
  cudaGetLastError();  // clear a sticky non-fatal error
  const int code = e == cudaErrorMemoryAllocation ? MCRT_E_OOM : MCRT_E_CUDA;
  return fail(c, code, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                      \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

inline cudaError_t ensure(DevBuf &b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

inline void release(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// Zhang's T_max proposal (Eq. 13 as Eq. 16) for the current fields, built and
// uploaded when stale (mcrt_api.cpp).
int build_plain_proposal(mcrt_ctx *ctx, double Tm, cudaStream_t s);
double proposal_T_max(const mcrt_ctx *ctx);
int ensure_plain_proposal(mcrt_ctx *ctx, cudaStream_t s);

// Launch arguments of an FP32/FP64 solve over the box b (i0,i1,j0,j1,k0,k1);
// outputs and scratch are left for the caller (mcrt_api.cpp).
void fill_trace_args(const mcrt_ctx *ctx, const mcrt_solve_params *p, const int b[6],
                     mcrt::TraceArgs *a);
// Sizes the long-ray buffer for chunks of chunk_rays rays and points the launch
// arguments at it (the hand-off is off for multigrid, closed boxes or by the
// tuning: mcrt::long_rays_on).
int setup_long_rays(mcrt_ctx *ctx, long long chunk_rays, mcrt::TraceArgs *a);
// Validates solve parameters common to every solve entry point.
int check_solve_params(mcrt_ctx *ctx, const mcrt_solve_params *p, int b[6]);

}  // namespace mcrt_host

// Per-cell binary64 tallies (Eq. 8: Q_i is the mean of the cell's samples) with
// the samples streamed into shared memory by the tensor memory accelerator.
//
// The samples of a solve chunk form a 2-D array [positions][N] of binary32
// (position = a cell's place in the chunk's brick order).  A warp owns 32
// consecutive positions; its 32-sample tiles ([32 positions][32 samples],
// 4 KB) arrive by cp.async.bulk.tensor into two shared buffers per warp, so the
// next tile is in flight while lane c adds its position's 32 samples exactly
// (tile_sums_exact) and compensates the tile sums (Neumaier): the same
// arithmetic in the same order as reduce_cells_kernel, hence the same bits.
// The tiles are written with the 128-byte swizzle (16-byte chunk j of row r
// lands at chunk j ^ (r mod 8)), so each lane's reads of its own row are free of
// bank conflicts.  Samples past N and positions past the chunk come in as zeros
// (the tensor's bounds); positions outside the box (ragged bricks) are loaded
// and ignored.
//
// Requirements of the copy: the sample array 16-byte aligned, the row pitch
// N * 4 bytes a multiple of 16 (N % 4 == 0); the x coordinate of every tile is a
// multiple of 32 samples (128 bytes).  Otherwise the caller uses
// reduce_cells_kernel.  Every wait on a tile is bounded: a tile that does not
// arrive sets bit 3 of counters[5] (reported as MCRT_E_TIMEOUT) and the warp
// stops after another bounded wait for its copies in flight.
#include <cuda.h>
#include <math.h>
#include <stdint.h>

#include "draws.cuh"
#include "mcrt_internal.h"
#include "trace_common.cuh"

namespace mcrt {
namespace {

constexpr int TW = 8;                  // warps per CTA
constexpr unsigned TILE_BYTES = 32 * 32 * 4;
constexpr long long WAIT_TRIES = 1 << 22;  // with 64 ns sleeps: a quarter of a second

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait of the whole warp for phase `parity` of bar; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  for (long long i = 0; i < WAIT_TRIES; ++i) {
    if (__all_sync(0xffffffffu, mbar_test(bar, parity))) return true;
    __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_tile(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(TW * 32, 3) reduce_cells_tma_kernel(const TraceArgs a,
                                                                  const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  // 1024-byte aligned buffers (the swizzle's period), then the barriers
  unsigned char *base_sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tsm) + 1023) & ~static_cast<uintptr_t>(1023));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *buf = base_sm + (size_t)w * 2 * TILE_BYTES;
  uint64_t *bar = reinterpret_cast<uint64_t *>(base_sm + (size_t)TW * 2 * TILE_BYTES) + 2 * w;
  const int N = a.rays;
  const long long P = a.chunk_p1 - a.chunk_p0;
  const int ntile = (N + 31) / 32;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long ngroups = (P + 31) / 32;
  const long long mygroups = gw < ngroups ? (ngroups - gw + nwarps - 1) / nwarps : 0;
  const long long T = mygroups * ntile;  // this warp's tiles, group by group
  if (T == 0) return;
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  auto issue = [&](long long t) {  // lane 0: tile t into buffer t & 1
    const long long g = gw + (t / ntile) * nwarps;
    const int r0 = (int)(t % ntile) * 32;
    uint64_t *b = bar + (t & 1);
    mbar_expect_tx(b, TILE_BYTES);
    tma_tile(buf + (t & 1) * TILE_BYTES, &tmap, r0, (int)(g * 32), b);
  };
  if (lane == 0) {
    issue(0);
    if (T > 1) issue(1);
  }
  double s = 0.0, c = 0.0, s2 = 0.0, c2 = 0.0;
  bool bad = false, mine = false;
  int bx = 0, by = 0, bz = 0;
  for (long long t = 0; t < T; ++t) {
    const long long g = gw + (t / ntile) * nwarps;
    const int tile = (int)(t % ntile);
    if (tile == 0) {  // a new group of 32 positions
      const long long p = g * 32 + lane;
      mine = p < P && brick_cell(a, a.chunk_p0 + p, bx, by, bz);
      s = c = s2 = c2 = 0.0;
      bad = false;
    }
    if (!mbar_wait(bar + (t & 1), (unsigned)((t >> 1) & 1))) {
      if (lane == 0) atomicOr(a.counters + 5, 8ull);
      // the copies still in flight (tiles t and t + 1) land in this CTA's shared
      // memory: wait for them once more, bounded, before leaving
      mbar_wait(bar + (t & 1), (unsigned)((t >> 1) & 1));
      if (t + 1 < T) mbar_wait(bar + ((t + 1) & 1), (unsigned)(((t + 1) >> 1) & 1));
      return;
    }
    if (mine) {
      const unsigned char *row = buf + (t & 1) * TILE_BYTES + lane * 128;
      unsigned v[32];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint4 f = *reinterpret_cast<const uint4 *>(row + ((j ^ (lane & 7)) << 4));
        v[4 * j] = f.x;
        v[4 * j + 1] = f.y;
        v[4 * j + 2] = f.z;
        v[4 * j + 3] = f.w;
      }
      double t1, t2;
      tile_sums_exact(v, t1, t2, bad);
      neumaier_add(s, c, t1);
      neumaier_add(s2, c2, t2);
    }
    __syncwarp();  // every lane has read the buffer
    if (lane == 0 && t + 2 < T) {
      // order the lanes' reads of the buffer before the copy engine's writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + 2);
    }
    if (tile == ntile - 1 && mine) {
      const double S = bad ? __longlong_as_double(0x7FF8000000000000ll) : s + c;
      const double S2 = bad ? S : s2 + c2;
      const long long cell = bx + (long long)a.bnx * (by + (long long)a.bny * bz);
      const double Nd = (double)N;
      const double Q = S / Nd;
      a.q[cell] = Q;
      if (a.sigma) a.sigma[cell] = N > 1 ? sqrt(fmax(S2 / Nd - Q * Q, 0.0) / (Nd - 1.0)) : 0.0;
      if (a.steps_cell) a.steps_cell[cell] = a.step_acc[g * 32 + lane];
    }
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

size_t tma_smem_bytes() { return (size_t)TW * 2 * TILE_BYTES + TW * 2 * sizeof(uint64_t) + 1024; }

}  // namespace

cudaError_t launch_reduce_tma(const TraceArgs &a, cudaStream_t s, bool *launched) {
  *launched = false;
  const long long P = a.chunk_p1 - a.chunk_p0;
  if (P <= 0 || a.rays < 1 || (a.rays & 3) || (reinterpret_cast<uintptr_t>(a.ybuf) & 15) || P > (1LL << 31))
    return cudaSuccess;
  EncodeTiled enc = encode_fn();
  if (!enc) return cudaSuccess;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)a.rays, (cuuint64_t)P};
  const cuuint64_t strides[1] = {(cuuint64_t)a.rays * sizeof(float)};
  const cuuint32_t box[2] = {32, 32}, estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.ybuf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaSuccess;
  const size_t smem = tma_smem_bytes();
  static int configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    e = cudaFuncSetAttribute(reduce_cells_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[dev] = 1;
  }
  // one group of 32 positions per warp where the grid allows (grid-stride
  // beyond): short blocks spread over whatever SMs are free, which matters when
  // the tally runs beside other solves' kernels in a batch graph
  const long long groups = (P + 31) / 32;
  long long blocks = (groups + TW - 1) / TW;
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();
  reduce_cells_tma_kernel<<<(unsigned)blocks, TW * 32, smem, s>>>(a, map);
  e = cudaGetLastError();
  if (e == cudaSuccess) *launched = true;
  return e;
}

}  // namespace mcrt

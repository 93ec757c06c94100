// Per-cell binary64 tallies (Eq. 8: Q_i is the mean of the cell's samples) with
// the samples streamed into shared memory by the tensor memory accelerator.
//
// The samples of a solve chunk form a 2-D array [positions][N] of binary32
// (position = a cell's place in the chunk's brick order).  A warp owns 32
// consecutive positions; its 32-sample tiles ([32 positions][32 samples],
// 4 KB) arrive by cp.async.bulk.tensor into two shared buffers per warp, so the
// next tile is in flight while lane c adds its position's 32 samples exactly
// (tile_sums_exact) and compensates the tile sums (Neumaier) segment by segment:
// the same arithmetic in the same order as reduce_cells_kernel, hence the same
// bits.  Cells of several segments (more than 2048 samples) have each segment
// summed by a warp of its own when the caller provides the segment scratch
// (a.tally_part), and combine_segments_kernel adds the segments in order: a chunk
// of few cells with many rays each is then spread over the whole GPU.
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

// The work of a warp is a sequence of items: an item is a group of 32
// consecutive positions and either all of their tiles or, in a split tally
// (MODE 2: a.tally_part non-null and more than one segment), one segment of
// them, so that cells with many samples are summed by many warps.  MODE 0: one
// segment (the cell sum is that segment's compensated sum, s + c); MODE 1:
// several segments added in order by the warp itself.  The items' tiles form one
// sequence per warp, so the copy of the next tile is in flight across item
// boundaries too.  A split item's last segment is padded to the common length
// with tiles past N, which the copy fills with zeros and whose sums (exact
// zeros) leave the compensated sums unchanged.
template <int MODE>
__global__ void __launch_bounds__(TW * 32, MODE == 1 ? 2 : 3) reduce_cells_tma_kernel(const TraceArgs a,
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
  const int L = MODE == 0 ? ntile : tally_seg_len(ntile);
  const int ipg = MODE == 2 ? tally_segments(ntile) : 1;  // items per group
  const int ilen = MODE == 2 ? L : ntile;                  // tiles per item
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nitems = ((P + 31) / 32) * ipg;
  const long long myitems = gw < nitems ? (nitems - gw + nwarps - 1) / nwarps : 0;
  const long long T = myitems * ilen;  // this warp's tiles, item by item
  if (T == 0) return;
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // the copy cursor (lane 0): the tile after the last one issued, as the
  // item's group row, its first tile and the tile within the item
  long long ci = gw;  // item of the copy cursor
  int ct = 0, cy = 0, cx0 = 0;
  auto cursor_item = [&]() {
    cy = (int)((ci / ipg) * 32);
    cx0 = (int)(ci % ipg) * L;
  };
  cursor_item();
  auto issue = [&](long long t) {  // lane 0: the cursor's tile (tile t) into buffer t & 1
    uint64_t *b = bar + (t & 1);
    mbar_expect_tx(b, TILE_BYTES);
    tma_tile(buf + (t & 1) * TILE_BYTES, &tmap, (cx0 + ct) * 32, cy, b);
    if (++ct == ilen) {
      ct = 0;
      ci += nwarps;
      cursor_item();
    }
  };
  if (lane == 0) {
    issue(0);
    if (T > 1) issue(1);
  }
  double S = 0.0, C = 0.0, S2 = 0.0, C2 = 0.0;  // over segments (MODE 1)
  double s = 0.0, c = 0.0, s2 = 0.0, c2 = 0.0;  // within the current segment
  bool bad = false, mine = false;
  int bx = 0, by = 0, bz = 0;
  long long i = gw, p = 0;  // the item being summed and the lane's position
  int tt = 0;               // tile within the item
  for (long long t = 0; t < T; ++t) {
    if (tt == 0) {  // a new item
      p = (i / ipg) * 32 + lane;
      mine = p < P && brick_cell(a, a.chunk_p0 + p, bx, by, bz);
      S = C = S2 = C2 = s = c = s2 = c2 = 0.0;
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
    const bool last = tt == ilen - 1;
    if (mine) {
      if (MODE == 2) {
        if (last) {  // the item is one segment: its sums, for the second kernel
          const double nan = __longlong_as_double(0x7FF8000000000000ll);
          a.tally_part[(size_t)(i % ipg) * (size_t)P + (size_t)p] =
              make_double2(bad ? nan : s + c, bad ? nan : s2 + c2);
        }
      } else {
        if (MODE == 1 && ((tt + 1) % L == 0 || last)) {  // the segment's last tile
          neumaier_add(S, C, s + c);
          neumaier_add(S2, C2, s2 + c2);
          s = c = s2 = c2 = 0.0;
        }
        if (last) {
          const double nan = __longlong_as_double(0x7FF8000000000000ll);
          const double Sy = bad ? nan : (MODE == 1 ? S + C : s + c);
          const double Sy2 = bad ? nan : (MODE == 1 ? S2 + C2 : s2 + c2);
          const long long cell = bx + (long long)a.bnx * (by + (long long)a.bny * bz);
          const double Nd = (double)N;
          const double Q = Sy / Nd;
          a.q[cell] = Q;
          if (a.sigma) a.sigma[cell] = N > 1 ? sqrt(fmax(Sy2 / Nd - Q * Q, 0.0) / (Nd - 1.0)) : 0.0;
          if (a.steps_cell) a.steps_cell[cell] = a.step_acc[p];
        }
      }
    }
    if (last) {
      tt = 0;
      i += nwarps;
    } else {
      ++tt;
    }
  }
}

// The second kernel of a split tally: one thread per position adds the
// segments' sums in order (the same compensated sum as a warp that adds its
// cell's segments itself) and writes Q and sigma.
__global__ void __launch_bounds__(256) combine_segments_kernel(const TraceArgs a) {
  const int N = a.rays;
  const long long P = a.chunk_p1 - a.chunk_p0;
  const int nseg = tally_segments((N + 31) / 32);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long long)gridDim.x * blockDim.x) {
    int bx = 0, by = 0, bz = 0;
    if (!brick_cell(a, a.chunk_p0 + p, bx, by, bz)) continue;
    double S = 0.0, C = 0.0, S2 = 0.0, C2 = 0.0;
    bool bad = false;
    for (int k = 0; k < nseg; ++k) {
      const double2 v = a.tally_part[(size_t)k * (size_t)P + (size_t)p];
      bad |= isnan(v.x);
      neumaier_add(S, C, v.x);
      neumaier_add(S2, C2, v.y);
    }
    const double Sy = bad ? __longlong_as_double(0x7FF8000000000000ll) : S + C;
    const double Sy2 = bad ? Sy : S2 + C2;
    const long long cell = bx + (long long)a.bnx * (by + (long long)a.bny * bz);
    const double Nd = (double)N;
    const double Q = Sy / Nd;
    a.q[cell] = Q;
    if (a.sigma) a.sigma[cell] = N > 1 ? sqrt(fmax(Sy2 / Nd - Q * Q, 0.0) / (Nd - 1.0)) : 0.0;
    if (a.steps_cell) a.steps_cell[cell] = a.step_acc[p];
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

cudaError_t launch_reduce_tma(const TraceArgs &a, cudaStream_t s, int *kernels) {
  *kernels = 0;
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
    e = cudaFuncSetAttribute(reduce_cells_tma_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(reduce_cells_tma_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(reduce_cells_tma_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[dev] = 1;
  }
  // one group of 32 positions per warp where the grid allows (grid-stride
  // beyond): short blocks spread over whatever SMs are free, which matters when
  // the tally runs beside other solves' kernels in a batch graph
  const int nseg = tally_segments((a.rays + 31) / 32);
  const bool split = a.tally_part != nullptr && nseg > 1;
  const long long items = ((P + 31) / 32) * (split ? nseg : 1);
  long long blocks = (items + TW - 1) / TW;
  if (blocks > grid_stride_blocks()) blocks = grid_stride_blocks();
  if (split)
    reduce_cells_tma_kernel<2><<<(unsigned)blocks, TW * 32, smem, s>>>(a, map);
  else if (nseg > 1)
    reduce_cells_tma_kernel<1><<<(unsigned)blocks, TW * 32, smem, s>>>(a, map);
  else
    reduce_cells_tma_kernel<0><<<(unsigned)blocks, TW * 32, smem, s>>>(a, map);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  *kernels = 1;
  if (split) {
    e = launch_combine_segments(a, s);
    if (e == cudaSuccess) *kernels = 2;
  }
  return e;
}

cudaError_t launch_combine_segments(const TraceArgs &a, cudaStream_t s) {
  const long long P = a.chunk_p1 - a.chunk_p0;
  if (P <= 0) return cudaSuccess;
  // 64 positions per CTA: a chunk of few cells (many rays each) still spreads
  // its binary64 sums over the SMs' narrow binary64 pipes
  long long cb = (P + 63) / 64;
  if (cb > grid_stride_blocks()) cb = grid_stride_blocks();
  combine_segments_kernel<<<(unsigned)cb, 64, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mcrt

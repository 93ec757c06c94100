// Draw decoding shared by the FP32 trace kernel and the learned-proposal
// kernels, which must reproduce the trace kernel's (n, g, hemisphere) choices
// exactly: Philox4x32-10 (Salmon et al., SC'11: ten rounds of the 4x32 Philox
// bijection with the published multipliers and Weyl key increments) and the
// inverse CDF of integer cumulative counts (Eq. 17 with the pdf quantised to
// counts of 2^32).
#pragma once

#include <cuda_runtime.h>

namespace mcrt {
namespace {

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

// The same bijection with the round keys precomputed: rk[2 r], rk[2 r + 1] are
// k0 + r W0 and k1 + r W1 (mod 2^32).  Given a kernel argument, each round's
// keys are operands read from the constant bank instead of two additions.
__device__ __forceinline__ uint4 philox10r(uint4 c, const unsigned *rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

// First k with u < cum[k] (binary search; cum[K-1] = 2^32 > u).
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

}  // namespace
}  // namespace mcrt

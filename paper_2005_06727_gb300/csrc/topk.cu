// Top-k nearest documents: the k smallest WMD values of one query and their
// document ids (the k-nearest-neighbour use of the distance, Sec. 1 and 2).
//
// One CTA of 1024 threads selects from WMD[N] (written by the fused loop):
//   1. every value is mapped to a 64-bit key whose unsigned order is the
//      numeric order (-0 counts as +0, every NaN after every number);
//   2. a radix select over the key's eight bytes, most significant first,
//      finds the k-th smallest key K* (a 256-bin shared-memory histogram of
//      the keys that match the bytes chosen so far, per pass);
//   3. one pass in document order takes every key below K* and the first
//      keys equal to K* (lowest document ids) until k are taken;
//   4. a bitonic sort in shared memory orders the k by (key, document id).
// Ties are broken by the lower document id, so the result is unique.  When
// N keys fit in shared memory (N <= kCacheMax) they are read from global
// memory once and kept there for all passes.
#include "wmd_internal.h"

namespace wmd {
namespace {

constexpr int kThreads = 1024;
constexpr int kCacheMax = 12288;  // keys kept in shared memory (96 KB)
static_assert(kTopkMaxK <= kThreads * 4, "sort loop bound");

__device__ __forceinline__ unsigned long long order_key(double x) {
  if (x != x) return ~0ull;          // NaN: after every number
  if (x == 0.0) x = 0.0;             // -0 and +0 are equal
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Block-wide exclusive prefix count of `flag` (every thread calls it);
// returns this thread's rank and writes the block total to *total.
__device__ __forceinline__ unsigned block_rank(bool flag, unsigned* warp_sums, unsigned* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned ball = __ballot_sync(0xffffffffu, flag);
  const unsigned before = __popc(ball & ((1u << lane) - 1u));
  if (lane == 0) warp_sums[warp] = __popc(ball);
  __syncthreads();
  if (warp == 0) {
    const unsigned v = warp_sums[lane];
    unsigned s = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += o;
    }
    warp_sums[lane] = s - v;  // exclusive
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const unsigned r = warp_sums[warp] + before;
  __syncthreads();  // warp_sums is reused by the next call
  return r;
}

template <bool CACHED>
__global__ void __launch_bounds__(kThreads, 1)
    topk_kernel(const double* __restrict__ wmd, int64_t N, int k, int64_t* __restrict__ out_idx,
                double* __restrict__ out_val) {
  extern __shared__ unsigned long long cache[];  // N keys when CACHED
  __shared__ unsigned hist[256];
  __shared__ unsigned warp_sums[32];
  __shared__ unsigned s_total, s_digit, s_need, s_taken;
  __shared__ unsigned long long s_key[kTopkMaxK];
  __shared__ long long s_idx[kTopkMaxK];
  const int tid = threadIdx.x;

  auto key_at = [&](int64_t i) { return CACHED ? cache[i] : order_key(wmd[i]); };
  if (CACHED) {
    for (int64_t i = tid; i < N; i += kThreads) cache[i] = order_key(wmd[i]);
  }

  // 2. radix select of the k-th smallest key, one byte per pass
  unsigned long long prefix = 0, mask = 0;
  unsigned need = (unsigned)k;  // rank of the target among the keys matching prefix
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int b = tid; b < 256; b += kThreads) hist[b] = 0;
    __syncthreads();
    // warp-aggregated counts: WMD values share their leading bytes, so most
    // keys of a pass land in few bins; lanes with the same byte add once
    for (int64_t base = 0; base < N; base += kThreads) {
      const int64_t i = base + tid;
      int digit = -1;
      if (i < N) {
        const unsigned long long key = key_at(i);
        if ((key & mask) == prefix) digit = (int)((key >> shift) & 255u);
      }
      const unsigned same = __match_any_sync(0xffffffffu, digit);
      if (digit >= 0 && (tid & 31) == __ffs(same) - 1) atomicAdd(&hist[digit], (unsigned)__popc(same));
    }
    __syncthreads();
    if (tid < 32) {
      // lane l holds bins 8 l .. 8 l + 7; find the bin where the running
      // count first reaches `need`
      unsigned c[8], sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        c[q] = hist[8 * tid + q];
        sum += c[q];
      }
      unsigned incl = sum;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
        if (tid >= off) incl += o;
      }
      const unsigned excl = incl - sum;
      const unsigned hit = __ballot_sync(0xffffffffu, excl < need && need <= incl);
      if (tid == __ffs(hit) - 1) {
        unsigned run = excl;
        int q = 0;
        while (run + c[q] < need) run += c[q++];
        s_digit = 8 * tid + q;
        s_need = need - run;
      }
    }
    __syncthreads();
    prefix |= (unsigned long long)s_digit << shift;
    mask |= 255ull << shift;
    need = s_need;
    __syncthreads();
  }
  const unsigned long long kth = prefix;  // the k-th smallest key

  // 3. take every key below kth (exactly k - need of them, in any slot
  //    order) and the first `need` keys equal to it in document order
  if (tid == 0) s_taken = 0;
  for (int t = tid; t < kTopkMaxK; t += kThreads) {
    s_key[t] = ~0ull;
    s_idx[t] = 0;
  }
  __syncthreads();
  const unsigned n_less = (unsigned)k - need;
  unsigned eq_seen = 0;  // equal keys met in earlier tiles (block-uniform)
  for (int64_t base = 0; base < N; base += kThreads) {
    const int64_t i = base + tid;
    const unsigned long long key = i < N ? key_at(i) : ~0ull;
    if (i < N && key < kth) {
      const unsigned slot = atomicAdd(&s_taken, 1u);
      if (slot < (unsigned)kTopkMaxK) {  // always: fewer than k keys lie below kth
        s_key[slot] = key;
        s_idx[slot] = i;
      }
    }
    const bool eq = i < N && key == kth && eq_seen < need;
    const int n_eq = __syncthreads_count(eq);
    if (n_eq) {  // block-uniform
      const unsigned r = block_rank(eq, warp_sums, &s_total);
      const unsigned slot = n_less + eq_seen + r;
      if (eq && eq_seen + r < need && slot < (unsigned)kTopkMaxK) {
        s_key[slot] = key;
        s_idx[slot] = i;
      }
      eq_seen += (unsigned)n_eq;
    }
  }
  __syncthreads();

  // 4. bitonic sort of the k taken (padded to a power of two) by (key, id)
  int P = 1;
  while (P < k) P <<= 1;
  for (int t = k + tid; t < P; t += kThreads) {
    s_key[t] = ~0ull;
    s_idx[t] = 0x7fffffffffffffffll;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int a = tid; a < P; a += kThreads) {
        const int b = a ^ stride;
        if (b > a) {
          const bool up = (a & size) == 0;
          const unsigned long long ka = s_key[a], kb = s_key[b];
          const long long ia = s_idx[a], ib = s_idx[b];
          const bool a_after = ka > kb || (ka == kb && ia > ib);
          if (a_after == up) {
            s_key[a] = kb;
            s_key[b] = ka;
            s_idx[a] = ib;
            s_idx[b] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = tid; t < k; t += kThreads) {
    const long long j = s_idx[t];
    out_idx[t] = j;
    out_val[t] = (j >= 0 && j < N) ? wmd[j] : __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace

cudaError_t launch_topk(const double* wmd, int64_t N, int k, int64_t* out_idx, double* out_val,
                        cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  if (N <= kCacheMax) {
    const size_t smem = (size_t)N * sizeof(unsigned long long);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
      attr_err = cudaFuncSetAttribute(topk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kCacheMax * sizeof(unsigned long long)));
    });
    if (attr_err != cudaSuccess) return attr_err;
    topk_kernel<true><<<1, kThreads, smem, s>>>(wmd, N, k, out_idx, out_val);
  } else {
    topk_kernel<false><<<1, kThreads, 0, s>>>(wmd, N, k, out_idx, out_val);
  }
  return cudaGetLastError();
}

}  // namespace wmd

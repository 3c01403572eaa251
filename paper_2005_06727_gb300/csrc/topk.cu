// Top-k nearest documents: the k smallest WMD values of one query and their
// document ids (the k-nearest-neighbour use of the distance, Sec. 1 and 2).
//
// One CTA of 1024 threads selects from WMD[N] (written by the fused loop):
//   1. every value is mapped to a 64-bit key whose unsigned order is the
//      numeric order (-0 counts as +0, every NaN after every number); one
//      sweep finds the smallest and largest key, whose common leading bits
//      every key shares (WMD values lie close together, so this skips the
//      sign, the exponent and a few mantissa bits);
//   2. a radix select over the remaining bits, 8 per pass, most significant
//      first: each pass builds a 256-bin shared-memory histogram of the
//      current candidates (plain shared-memory atomics: below the common
//      prefix the keys spread over many bins, and aggregating equal bytes per
//      warp with match.any cost more than the collisions it saved), every
//      warp scans it for itself and finds the bin of the
//      k-th smallest key (one barrier per pass; three histogram buffers
//      rotate), and a second sweep emits the keys of the lower bins (they
//      are among the k) and moves the keys of that bin to a shared-memory
//      index list, the next pass's candidates;
//   3. once at most kSmall candidates remain (or every bit is decided), the
//      rest of the k are the candidates of smallest (key, document id); with
//      many exact ties they are taken in document order instead;
//   4. the k taken are ordered by (key, document id): by counting ranks for
//      k <= 256, else by a bitonic sort.
// Ties are broken by the lower document id, so the result is unique.  When
// N keys fit in shared memory (N <= kCacheMax) they are read from global
// memory once and kept there for all passes.
#include "wmd_internal.h"

namespace wmd {
namespace {

// Threads per CTA for keys streamed from global memory and for keys kept in
// shared memory (256 for the latter was measured slower at N = 5000: 22.6
// against 21.1 us for k = 10, 50.6 against 42.1 us for k = 1024).
constexpr int kThreadsStream = 1024;
constexpr int kThreadsCached = 1024;
constexpr int kCacheMax = 12288;   // keys kept in shared memory (96 KB)
constexpr int kUnroll = 8;         // independent key loads in flight per thread
constexpr int kRankSortMax = 256;  // k up to this: rank counting (one entry per thread), else bitonic
static_assert(kRankSortMax <= kThreadsCached && kRankSortMax <= kThreadsStream, "rank sort");
constexpr int kCandMax = 8192;     // candidate list capacity (indices)
constexpr int kSmall = 256;        // candidates few enough to rank directly
static_assert(kTopkMaxK * 12 <= kCandMax * 4, "the spare list holds kTopkMaxK keys and ids");

// From the value's bits, loaded as an integer: the FP64 pipe of this GPU is
// too slow to test every value with floating-point compares (and integer tests
// on a reinterpreted double may be folded back into them by the compiler).
__device__ __forceinline__ unsigned long long order_key(unsigned long long b) {
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  if (mag > 0x7ff0000000000000ull) return ~0ull;  // NaN: after every number
  if (mag == 0) b = 0;                              // -0 and +0 are equal
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Block-wide exclusive prefix count of `flag` (every thread calls it);
// returns this thread's rank and writes the block total to *total.
template <int NT>
__device__ __forceinline__ unsigned block_rank(bool flag, unsigned* warp_sums, unsigned* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned ball = __ballot_sync(0xffffffffu, flag);
  const unsigned before = __popc(ball & ((1u << lane) - 1u));
  if (lane == 0) warp_sums[warp] = __popc(ball);
  __syncthreads();
  if (warp == 0) {
    const unsigned v = lane < NT / 32 ? warp_sums[lane] : 0u;
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

// Visits the keys of the current candidate set in blocks of NT *
// kUnroll (every thread runs the same number of iterations, so warp
// collectives inside `f` are safe).  The set is either the whole array
// filtered by (key & mask) == prefix (full) or an explicit index list.
template <bool CACHED, int NT, typename F>
__device__ __forceinline__ void sweep(const unsigned long long* __restrict__ bits,
                                      const unsigned long long* cache,
                                      int64_t N, bool full, const int* list, unsigned nlist,
                                      unsigned long long mask, unsigned long long prefix, F&& f) {
  const int64_t n = full ? N : (int64_t)nlist;
  for (int64_t base = 0; base < n; base += (int64_t)NT * kUnroll) {
    unsigned long long key[kUnroll];
    int64_t idx[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t t = base + u * NT + threadIdx.x;
      idx[u] = t < n ? (full ? t : (int64_t)list[t]) : -1;
      key[u] = idx[u] >= 0 ? (CACHED ? cache[idx[u]] : order_key(__ldg(bits + idx[u]))) : ~0ull;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const bool in = idx[u] >= 0 && (!full || (key[u] & mask) == prefix);
      f(in, key[u], idx[u]);
    }
  }
}

template <bool CACHED, int NT>
__global__ void __launch_bounds__(NT, 1)
    topk_kernel(const double* __restrict__ wmd, int64_t N, int k, int64_t* __restrict__ out_idx,
                double* __restrict__ out_val) {
  // dynamic: [N keys if CACHED][two candidate lists of kCandMax indices]
  extern __shared__ __align__(16) unsigned char dyn[];
  unsigned long long* cache = reinterpret_cast<unsigned long long*>(dyn);
  int* cand[2];
  cand[0] = reinterpret_cast<int*>(dyn + (CACHED ? (size_t)N * sizeof(unsigned long long) : 0));
  cand[1] = cand[0] + kCandMax;
  __shared__ unsigned hist[3][256];
  __shared__ unsigned warp_sums[32];
  constexpr int kWarps = NT / 32;
  __shared__ unsigned long long s_min[kWarps], s_max[kWarps];
  __shared__ unsigned s_total, s_taken, s_ncand[2];
  __shared__ unsigned long long s_key[kTopkMaxK];
  __shared__ long long s_idx[kTopkMaxK];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(wmd);
  auto key_at = [&](int64_t i) { return CACHED ? cache[i] : order_key(__ldg(bits + i)); };

  // 1. smallest and largest key (and the shared-memory copy of the keys)
  unsigned long long kmin = ~0ull, kmax = 0;
  for (int64_t base = 0; base < N; base += (int64_t)NT * kUnroll) {
    unsigned long long key[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + u * NT + tid;
      key[u] = i < N ? order_key(__ldg(bits + i)) : ~0ull;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + u * NT + tid;
      if (i < N) {
        if (CACHED) cache[i] = key[u];
        kmin = key[u] < kmin ? key[u] : kmin;
        kmax = key[u] > kmax ? key[u] : kmax;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, off);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, off);
    kmin = a < kmin ? a : kmin;
    kmax = b > kmax ? b : kmax;
  }
  if (lane == 0) {
    s_min[warp] = kmin;
    s_max[warp] = kmax;
  }
  for (int t = tid; t < 2 * 256; t += NT) hist[t >> 8][t & 255] = 0;
  for (int t = tid; t < kTopkMaxK; t += NT) {
    s_key[t] = ~0ull;
    s_idx[t] = 0;
  }
  if (tid == 0) {
    s_taken = 0;
    s_ncand[0] = s_ncand[1] = 0;
  }
  __syncthreads();
  kmin = lane < kWarps ? s_min[lane] : ~0ull;  // one warp's total per lane, then a butterfly
  kmax = lane < kWarps ? s_max[lane] : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, off);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, off);
    kmin = a < kmin ? a : kmin;
    kmax = b > kmax ? b : kmax;
  }

  // 2. radix select over the bits below the common prefix of kmin and kmax.
  //    Each pass histograms the next byte of the current candidates, emits
  //    the keys of the bins below the k-th key's bin (they are among the k)
  //    and moves the keys of its bin to the next candidate list, until at
  //    most kSmall candidates are left or every bit is decided.
  int hi = kmin == kmax ? 0 : 64 - __clzll((long long)(kmin ^ kmax));  // undecided low bits
  unsigned long long mask = hi == 64 ? 0ull : ~((1ull << hi) - 1ull);
  unsigned long long prefix = kmin & mask;
  unsigned need = (unsigned)k;  // rank of the k-th key among the candidates
  bool full = true;             // candidates: all keys matching prefix, else cand[cur]
  int cur = 0;
  unsigned ncand = (unsigned)N;
  int pass = 0;
  while (hi > 0 && (full || ncand > (unsigned)kSmall)) {
    const int width = hi < 8 ? hi : 8;
    const int shift = hi - width;
    const unsigned dmask = (1u << width) - 1u;
    unsigned* h = hist[pass % 3];
    for (int t = tid; t < 256; t += NT) hist[(pass + 1) % 3][t] = 0;  // nobody reads it now
    sweep<CACHED, NT>(bits, cache, N, full, cand[cur], ncand, mask, prefix,
                  [&](bool in, unsigned long long key, int64_t) {
                    if (in) atomicAdd(&h[(unsigned)(key >> shift) & dmask], 1u);
                  });
    __syncthreads();
    // every warp finds the bin where the running count reaches `need`
    // (lane l holds bins 8 l .. 8 l + 7)
    unsigned c[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      c[q] = h[8 * lane + q];
      sum += c[q];
    }
    unsigned incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    const unsigned excl = incl - sum;
    const unsigned hit = __ballot_sync(0xffffffffu, excl < need && need <= incl);
    const int src = hit ? __ffs(hit) - 1 : 0;
    unsigned run = excl;
    int q = 0;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
      if (q == t && run + c[t] < need) {
        run += c[t];
        ++q;
      }
    }
    unsigned cq = c[0];
#pragma unroll
    for (int t = 1; t < 8; ++t) cq = q == t ? c[t] : cq;
    const unsigned bin = (unsigned)__shfl_sync(0xffffffffu, 8 * lane + q, src);
    const unsigned below = __shfl_sync(0xffffffffu, run, src);
    const unsigned cnt = __shfl_sync(0xffffffffu, cq, src);
    // emit the keys below the bin; move the bin's keys to the next list
    const bool compact = cnt <= (unsigned)kCandMax;
    int* next = cand[cur ^ 1];
    unsigned* nnext = &s_ncand[pass & 1];
    sweep<CACHED, NT>(bits, cache, N, full, cand[cur], ncand, mask, prefix,
                  [&](bool in, unsigned long long key, int64_t i) {
                    if (!in) return;
                    const unsigned digit = (unsigned)(key >> shift) & dmask;
                    if (digit < bin) {
                      const unsigned slot = atomicAdd(&s_taken, 1u);
                      if (slot < (unsigned)kTopkMaxK) {  // always: fewer than k lie below
                        s_key[slot] = key;
                        s_idx[slot] = i;
                      }
                    } else if (digit == bin && compact) {
                      const unsigned p = atomicAdd(nnext, 1u);
                      if (p < (unsigned)kCandMax) next[p] = (int)i;
                    }
                  });
    if (tid == 0) s_ncand[(pass + 1) & 1] = 0;  // the counter of the pass after next
    __syncthreads();
    need -= below;
    prefix |= (unsigned long long)bin << shift;
    mask |= (unsigned long long)dmask << shift;
    hi = shift;
    ncand = cnt;
    if (compact) {
      full = false;
      cur ^= 1;
    }
    ++pass;
  }
  if (need < 1) need = 1;  // (always in [1, k]; kept there for the slots below)
  if (need > (unsigned)k) need = (unsigned)k;
  const unsigned base_slot = (unsigned)k - need;

  // 3. the last `need` of the k among the remaining candidates
  if (ncand <= (unsigned)kSmall || (!full && ncand <= (unsigned)kTopkMaxK)) {
    // few candidates: gather them with their keys (into the spare list's
    // memory) and take those of rank < need by (key, id)
    unsigned long long* tkey = reinterpret_cast<unsigned long long*>(cand[cur ^ 1]);
    int* tidx = reinterpret_cast<int*>(tkey + kTopkMaxK);
    if (tid == 0) s_total = 0;
    __syncthreads();
    sweep<CACHED, NT>(bits, cache, N, full, cand[cur], ncand, mask, prefix,
                  [&](bool in, unsigned long long key, int64_t i) {
                    if (!in) return;
                    const unsigned p = atomicAdd(&s_total, 1u);
                    if (p < (unsigned)kTopkMaxK) {
                      tkey[p] = key;
                      tidx[p] = (int)i;
                    }
                  });
    __syncthreads();
    const unsigned m = s_total < (unsigned)kTopkMaxK ? s_total : (unsigned)kTopkMaxK;
    for (unsigned t = tid; t < m; t += NT) {
      const unsigned long long kt = tkey[t];
      const int it = tidx[t];
      unsigned rank = 0;
      for (unsigned j = 0; j < m; ++j) {
        const unsigned long long kj = tkey[j];
        rank += (kj < kt || (kj == kt && tidx[j] < it)) ? 1u : 0u;
      }
      if (rank < need && base_slot + rank < (unsigned)kTopkMaxK) {
        s_key[base_slot + rank] = kt;
        s_idx[base_slot + rank] = it;
      }
    }
  } else {
    // every bit decided and many keys equal to the k-th: the lowest ids win,
    // so take them in document order
    unsigned eq_seen = 0;  // block-uniform
    for (int64_t base = 0; base < N; base += NT) {
      const int64_t i = base + tid;
      const bool eq = i < N && key_at(i) == prefix && eq_seen < need;
      const int cnt = __syncthreads_count(eq);
      if (cnt) {  // block-uniform
        const unsigned r = block_rank<NT>(eq, warp_sums, &s_total);
        const unsigned slot = base_slot + eq_seen + r;
        if (eq && eq_seen + r < need && slot < (unsigned)kTopkMaxK) {
          s_key[slot] = prefix;
          s_idx[slot] = i;
        }
        eq_seen += (unsigned)cnt;
      }
    }
  }
  __syncthreads();

  // 4. order the k taken by (key, document id)
  if (k <= kRankSortMax) {
    // the rank of an entry is the number of entries before it (all distinct)
    unsigned long long kt = 0;
    long long it = 0;
    int rank = 0;
    if (tid < k) {
      kt = s_key[tid];
      it = s_idx[tid];
      for (int j = 0; j < k; ++j) {
        const unsigned long long kj = s_key[j];
        const long long ij = s_idx[j];
        rank += (kj < kt || (kj == kt && ij < it)) ? 1 : 0;
      }
    }
    __syncthreads();
    if (tid < k) {
      s_key[rank] = kt;
      s_idx[rank] = it;
    }
    __syncthreads();
  } else {
    int P = 1;
    while (P < k) P <<= 1;
    for (int t = k + tid; t < P; t += NT) {
      s_key[t] = ~0ull;
      s_idx[t] = 0x7fffffffffffffffll;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int a = tid; a < P; a += NT) {
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
  }
  for (int t = tid; t < k; t += NT) {
    const long long j = s_idx[t];
    out_idx[t] = j;
    out_val[t] = (j >= 0 && j < N) ? wmd[j] : __longlong_as_double(0x7ff8000000000000ll);
  }
}

}  // namespace

cudaError_t launch_topk(const double* wmd, int64_t N, int k, int64_t* out_idx, double* out_val,
                        cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const size_t lists = 2 * (size_t)kCandMax * sizeof(int);
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [lists] {
    attr_err = cudaFuncSetAttribute(topk_kernel<true, kThreadsCached>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(kCacheMax * sizeof(unsigned long long) + lists));
    if (attr_err == cudaSuccess)
      attr_err = cudaFuncSetAttribute(topk_kernel<false, kThreadsStream>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lists);
  });
  if (attr_err != cudaSuccess) return attr_err;
  if (N <= kCacheMax) {
    topk_kernel<true, kThreadsCached>
        <<<1, kThreadsCached, (size_t)N * sizeof(unsigned long long) + lists, s>>>(wmd, N, k,
                                                                                 out_idx, out_val);
  } else {
    topk_kernel<false, kThreadsStream><<<1, kThreadsStream, lists, s>>>(wmd, N, k, out_idx,
                                                                       out_val);
  }
  return cudaGetLastError();
}

}  // namespace wmd

// Top-k nearest documents: the k smallest WMD values of one query and their
// document ids (the k-nearest-neighbour use of the distance, Sec. 1 and 2).
//
// Three kernels, by the size of WMD[N] (written by the fused loop), all
// launched as programmatic dependents of the work before them:
//   * N <= 16384: one CTA keeps the keys in registers (topk_small_kernel);
//   * N <= 262144: the same over a thread-block cluster of 16 (or 8) CTAs,
//     histograms merged through distributed shared memory
//     (topk_cluster_kernel);
//   * larger N: the kernel described next (topk_kernel).
// Each kernel's own comment gives its steps.
//
// topk_kernel: one CTA of 1024 threads:
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
#include <cooperative_groups.h>

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

// WMD[] is written by the kernel before this one in the stream, which may
// still run when this kernel starts (programmatic dependent launch): wait for
// it, then read the values with ordinary coherent loads kept in order with
// the wait (volatile asm; no __ldg, whose data must be read-only for the
// kernel's lifetime).
__device__ __forceinline__ void wait_for_values() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ unsigned long long ld_bits(const unsigned long long* a) {
  unsigned long long v;
  asm volatile("ld.global.u64 %0, [%1];" : "=l"(v) : "l"(a));
  return v;
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
__device__ __forceinline__ void sweep(const unsigned long long* bits,
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
      key[u] = idx[u] >= 0 ? (CACHED ? cache[idx[u]] : order_key(ld_bits(bits + idx[u]))) : ~0ull;
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
    topk_kernel(const double* wmd, int64_t N, int k, int64_t* __restrict__ out_idx,
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
  wait_for_values();
  const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(wmd);
  auto key_at = [&](int64_t i) { return CACHED ? cache[i] : order_key(ld_bits(bits + i)); };

  // 1. smallest and largest key (and the shared-memory copy of the keys)
  unsigned long long kmin = ~0ull, kmax = 0;
  for (int64_t base = 0; base < N; base += (int64_t)NT * kUnroll) {
    unsigned long long key[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + u * NT + tid;
      key[u] = i < N ? order_key(ld_bits(bits + i)) : ~0ull;
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

// ---------------------------------------------------------------- small N
// N <= kSmallThreads * kSmallE keys, kept in registers: thread t holds keys
// t E ... t E + E - 1 (E = ceil(N / 1024), a compile-time count so that no
// loop over a thread's keys runs empty slots), and thread order is
// document order.
// A radix select on 11-bit digits of key - (smallest key), most significant
// first from the top bit of the range (largest - smallest): the first pass
// spreads the keys over all 2048 bins whatever their exponents, and usually
// leaves the k-th key's bin with a few keys, which are then ranked by
// (key, id) directly; repeated exact ties fall through to document order.
// About ten barriers in all, against two sweeps per 8-bit pass above.
constexpr int kSmallThreads = 512;
constexpr int kSmallE = 32;        // keys per thread at most (one instance per count)
constexpr int kSmallBits = 10;
constexpr int kSmallBins = 1 << kSmallBits;
constexpr int kSmallCand = 64;     // candidates ranked directly (16 threads each)
constexpr int64_t kSmallMaxN = (int64_t)kSmallThreads * kSmallE;
static_assert(kSmallBins == 2 * kSmallThreads, "two bins per thread in the scan");
static_assert(kSmallCand * 8 == kSmallThreads && kSmallThreads % kRankSortMax == 0, "rank split");

__device__ __forceinline__ bool before(unsigned long long ka, int ia, unsigned long long kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// The k taken (keys and ids in s_key / s_idx, any order, all distinct by
// (key, id)), written out ordered by (key, document id), by a whole block of
// NT threads: rank counting, NT / 256 threads per entry, for k <= 256; a
// bitonic sort of the next power of two for larger k.
template <int NT>
__device__ __forceinline__ void order_taken(unsigned long long* s_key, int* s_idx, int k,
                                            const double* wmd, int N, int64_t* out_idx,
                                            double* out_val) {
  const int tid = threadIdx.x;
  if (k <= kRankSortMax) {
    constexpr int kPer = NT / kRankSortMax;  // threads per entry (a power of two)
    const int en = tid / kPer, part = tid % kPer;
    unsigned long long kt = 0;
    int it = 0, rank = 0;
    if (en < k) {
      kt = s_key[en];
      it = s_idx[en];
      for (int j = part; j < k; j += kPer) rank += before(s_key[j], s_idx[j], kt, it) ? 1 : 0;
    }
#pragma unroll
    for (int off = 1; off < kPer; off <<= 1) rank += __shfl_xor_sync(0xffffffffu, rank, off);
    if (en < k && part == 0) {
      out_idx[rank] = it;
      out_val[rank] = (it >= 0 && it < N) ? wmd[it] : __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  int P = 1;
  while (P < k) P <<= 1;
  for (int t = k + tid; t < P; t += NT) {
    s_key[t] = ~0ull;
    s_idx[t] = 0x7fffffff;
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int a = tid; a < P; a += NT) {
        const int b = a ^ stride;
        if (b > a) {
          const unsigned long long ka = s_key[a], kb = s_key[b];
          const int ia = s_idx[a], ib = s_idx[b];
          if (before(kb, ib, ka, ia) == ((a & size) == 0)) {
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
  for (int t = tid; t < k; t += NT) {
    const int j = s_idx[t];
    out_idx[t] = j;
    out_val[t] = (j >= 0 && j < N) ? wmd[j] : __longlong_as_double(0x7ff8000000000000ll);
  }
}


template <int E>
__global__ void __launch_bounds__(kSmallThreads, 1)
    topk_small_kernel(const double* wmd, int N, int k, int64_t* out_idx, double* out_val) {
  __shared__ unsigned hist[kSmallBins];
  constexpr int kW = kSmallThreads / 32;
  __shared__ unsigned warp_sums[kW];
  __shared__ unsigned long long s_min[kW], s_max[kW];
  __shared__ unsigned s_sel[3];   // bin, keys below it, keys in it
  __shared__ unsigned s_taken, s_ncand;
  __shared__ unsigned long long s_key[kTopkMaxK];
  __shared__ int s_idx[kTopkMaxK];
  __shared__ unsigned long long c_key[kSmallCand];
  __shared__ int c_idx[kSmallCand];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = tid * E;

  hist[2 * tid] = 0;
  hist[2 * tid + 1] = 0;
  if (tid == 0) {
    s_taken = 0;
    s_ncand = 0;
  }
  wait_for_values();
  const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(wmd);
  unsigned long long key[E];
  unsigned valid = 0;  // bit e: key e exists
  unsigned long long kmin = ~0ull, kmax = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const bool v = i0 + e < N;
    key[e] = v ? order_key(ld_bits(bits + i0 + e)) : ~0ull;
    valid |= (v ? 1u : 0u) << e;
    if (v) {
      kmin = key[e] < kmin ? key[e] : kmin;
      kmax = key[e] > kmax ? key[e] : kmax;
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
  __syncthreads();
  kmin = lane < kW ? s_min[lane] : ~0ull;  // a full butterfly: every lane gets the total
  kmax = lane < kW ? s_max[lane] : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, off);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, off);
    kmin = a < kmin ? a : kmin;
    kmax = b > kmax ? b : kmax;
  }
  // from here on the keys are offsets from the smallest (same order)
#pragma unroll
  for (int e = 0; e < E; ++e) key[e] -= kmin;
  const unsigned long long range = kmax - kmin;

  unsigned cm = valid;  // bit e: key e is a candidate (matches the decided prefix)
  int hi = range == 0 ? 0 : 64 - __clzll((long long)range);  // undecided low bits
  unsigned long long mask = hi == 64 ? 0ull : ~((1ull << hi) - 1ull);
  unsigned long long prefix = 0;
  unsigned need = (unsigned)k;  // rank of the k-th key among the candidates
  unsigned ncand = (unsigned)N;
  while (hi > 0 && ncand > (unsigned)kSmallCand) {
    const int width = hi < kSmallBits ? hi : kSmallBits;
    const int shift = hi - width;
    const unsigned dmask = (1u << width) - 1u;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if ((cm >> e) & 1u) atomicAdd(&hist[(unsigned)(key[e] >> shift) & dmask], 1u);
    __syncthreads();
    // block-wide scan of the bins (thread t: bins 2t and 2t + 1); the thread
    // whose bins hold the need-th candidate publishes its bin
    const unsigned h0 = hist[2 * tid], h1 = hist[2 * tid + 1];
    hist[2 * tid] = 0;  // only this thread reads them in this pass
    hist[2 * tid + 1] = 0;
    const unsigned sum = h0 + h1;
    unsigned incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned v = lane < kW ? warp_sums[lane] : 0u;
      unsigned w = v;
#pragma unroll
      for (int off = 1; off < kW; off <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += o;
      }
      if (lane < kW) warp_sums[lane] = w - v;  // exclusive
    }
    __syncthreads();
    const unsigned excl = warp_sums[warp] + incl - sum;
    if (excl < need && need <= excl + h0) {
      s_sel[0] = 2 * tid;
      s_sel[1] = excl;
      s_sel[2] = h0;
    } else if (excl + h0 < need && need <= excl + sum) {
      s_sel[0] = 2 * tid + 1;
      s_sel[1] = excl + h0;
      s_sel[2] = h1;
    }
    __syncthreads();
    const unsigned bin = s_sel[0];
    need -= s_sel[1];
    ncand = s_sel[2];
    prefix |= (unsigned long long)bin << shift;
    mask |= (unsigned long long)dmask << shift;
    hi = shift;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (((unsigned)(key[e] >> shift) & dmask) != bin) cm &= ~(1u << e);
    // warp_sums and s_sel are rewritten only after the next pass's first
    // barrier, which every thread reaches after reading them
  }

  // the keys below the decided prefix are among the k; the candidates (keys
  // equal to it in the decided bits) supply the last `need` by (key, id)
  const unsigned base = (unsigned)k - need;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (((valid >> e) & 1u) && (key[e] & mask) < prefix) {
      const unsigned slot = atomicAdd(&s_taken, 1u);
      if (slot < (unsigned)kTopkMaxK) {  // always: fewer than k lie below
        s_key[slot] = key[e];
        s_idx[slot] = i0 + e;
      }
    }
  }
  if (ncand <= (unsigned)kSmallCand) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((cm >> e) & 1u) {
        const unsigned p = atomicAdd(&s_ncand, 1u);
        if (p < (unsigned)kSmallCand) {
          c_key[p] = key[e];
          c_idx[p] = i0 + e;
        }
      }
    }
    __syncthreads();
    // candidate tid / 8, its rank summed over 8 threads
    const unsigned m = s_ncand < (unsigned)kSmallCand ? s_ncand : (unsigned)kSmallCand;
    const unsigned c = (unsigned)tid >> 3, part = (unsigned)tid & 7u;
    unsigned long long kt = 0;
    int it = 0;
    unsigned r = 0;
    if (c < m) {
      kt = c_key[c];
      it = c_idx[c];
      for (unsigned j = part; j < m; j += 8) r += before(c_key[j], c_idx[j], kt, it) ? 1u : 0u;
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    if (c < m && part == 0 && r < need && base + r < (unsigned)kTopkMaxK) {
      s_key[base + r] = kt;
      s_idx[base + r] = it;
    }
  } else {
    // every bit decided and more than kSmallCand keys equal to the k-th:
    // the lowest document ids win; thread order is document order, so a
    // block-wide prefix count of each thread's candidates ranks them
    const unsigned mine = __popc(cm);
    unsigned incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned v = lane < kW ? warp_sums[lane] : 0u;
      unsigned w = v;
#pragma unroll
      for (int off = 1; off < kW; off <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += o;
      }
      if (lane < kW) warp_sums[lane] = w - v;
    }
    __syncthreads();
    unsigned r = warp_sums[warp] + incl - mine;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((cm >> e) & 1u) {
        if (r < need && base + r < (unsigned)kTopkMaxK) {
          s_key[base + r] = key[e];
          s_idx[base + r] = i0 + e;
        }
        ++r;
      }
    }
  }
  __syncthreads();

  order_taken<kSmallThreads>(s_key, s_idx, k, wmd, N, out_idx, out_val);
}

// ---------------------------------------------------------------- large N
// The same selection spread over a thread-block cluster of CS CTAs (16 where
// the GPU allows clusters that large, else 8), one SM each: CTA r keeps keys
// [r S, (r + 1) S) in registers (S = ceil(N / CS), E keys per thread, 512
// threads), and the CTAs meet through distributed shared memory:
//   * every CTA publishes its smallest and largest key; each reads all CS of
//     them and forms the global range itself;
//   * per digit pass every CTA histograms its own keys in its shared memory;
//     after a cluster barrier CTA 0 sums the CS histograms bin by bin (remote
//     loads), scans them and publishes the bin of the k-th key, which every
//     CTA reads after a second barrier;
//   * the keys below that bin and the candidates in it are written into CTA
//     0's shared memory with remote atomics on its counters; after a last
//     barrier the other CTAs leave (nothing reads their shared memory any
//     more) and CTA 0 ranks the candidates and orders the k.
// Every wait is a hardware cluster barrier (barrier.cluster); the kernel has
// no spin loop.
constexpr int kClusterThreads = 512;
constexpr int kClusterMaxE = 32;

template <int E>
__global__ void __launch_bounds__(kClusterThreads, 1)
    topk_cluster_kernel(const double* wmd, int N, int k, int64_t* out_idx, double* out_val) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int CS = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  constexpr int kW = kClusterThreads / 32;
  __shared__ unsigned hist[kSmallBins];
  __shared__ unsigned warp_sums[kW];
  __shared__ unsigned long long s_min[kW], s_max[kW];
  __shared__ unsigned long long blk_min, blk_max;
  __shared__ unsigned blk_cnt;
  __shared__ unsigned s_sel[3];   // CTA 0: bin, keys below it, keys in it
  __shared__ unsigned s_taken, s_ncand;
  __shared__ unsigned long long s_key[kTopkMaxK];
  __shared__ int s_idx[kTopkMaxK];
  __shared__ unsigned long long c_key[kSmallCand];
  __shared__ int c_idx[kSmallCand];
  static_assert(kSmallBins == 2 * kClusterThreads, "two bins per thread in the scan");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int span = (N + CS - 1) / CS;
  const int lo = rank * span;
  const int end = min(N, lo + span);
  const int i0 = lo + tid * E;

  hist[2 * tid] = 0;
  hist[2 * tid + 1] = 0;
  if (tid == 0) {
    s_taken = 0;
    s_ncand = 0;
  }
  wait_for_values();
  const unsigned long long* bits = reinterpret_cast<const unsigned long long*>(wmd);
  unsigned long long key[E];
  unsigned valid = 0;
  unsigned long long kmin = ~0ull, kmax = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const bool v = i0 + e < end;
    key[e] = v ? order_key(ld_bits(bits + i0 + e)) : ~0ull;
    valid |= (v ? 1u : 0u) << e;
    if (v) {
      kmin = key[e] < kmin ? key[e] : kmin;
      kmax = key[e] > kmax ? key[e] : kmax;
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
  __syncthreads();
  if (warp == 0) {
    kmin = lane < kW ? s_min[lane] : ~0ull;
    kmax = lane < kW ? s_max[lane] : 0ull;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, off);
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, off);
      kmin = a < kmin ? a : kmin;
      kmax = b > kmax ? b : kmax;
    }
    if (lane == 0) {
      blk_min = kmin;
      blk_max = kmax;
    }
  }
  cluster.sync();  // every CTA's range and zeroed counters are visible
  // the global range: lane l reads CTA l's (CS <= 32), then a butterfly
  kmin = lane < CS ? *cluster.map_shared_rank(&blk_min, lane) : ~0ull;
  kmax = lane < CS ? *cluster.map_shared_rank(&blk_max, lane) : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, off);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, off);
    kmin = a < kmin ? a : kmin;
    kmax = b > kmax ? b : kmax;
  }
#pragma unroll
  for (int e = 0; e < E; ++e) key[e] -= kmin;
  const unsigned long long range = kmax - kmin;

  unsigned cm = valid;
  int hi = range == 0 ? 0 : 64 - __clzll((long long)range);
  unsigned long long mask = hi == 64 ? 0ull : ~((1ull << hi) - 1ull);
  unsigned long long prefix = 0;
  unsigned need = (unsigned)k;
  unsigned ncand = (unsigned)N;
  while (hi > 0 && ncand > (unsigned)kSmallCand) {
    const int width = hi < kSmallBits ? hi : kSmallBits;
    const int shift = hi - width;
    const unsigned dmask = (1u << width) - 1u;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if ((cm >> e) & 1u) atomicAdd(&hist[(unsigned)(key[e] >> shift) & dmask], 1u);
    cluster.sync();  // every CTA's histogram is complete
    if (rank == 0) {
      unsigned h0 = 0, h1 = 0;
      for (int r = 0; r < CS; ++r) {
        const unsigned* rh = cluster.map_shared_rank(hist, r);
        h0 += rh[2 * tid];
        h1 += rh[2 * tid + 1];
      }
      const unsigned sum = h0 + h1;
      unsigned incl = sum;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
      }
      if (lane == 31) warp_sums[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        const unsigned v = lane < kW ? warp_sums[lane] : 0u;
        unsigned w = v;
#pragma unroll
        for (int off = 1; off < kW; off <<= 1) {
          const unsigned o = __shfl_up_sync(0xffffffffu, w, off);
          if (lane >= off) w += o;
        }
        if (lane < kW) warp_sums[lane] = w - v;
      }
      __syncthreads();
      const unsigned excl = warp_sums[warp] + incl - sum;
      if (excl < need && need <= excl + h0) {
        s_sel[0] = 2 * tid;
        s_sel[1] = excl;
        s_sel[2] = h0;
      } else if (excl + h0 < need && need <= excl + sum) {
        s_sel[0] = 2 * tid + 1;
        s_sel[1] = excl + h0;
        s_sel[2] = h1;
      }
    }
    cluster.sync();  // the bin is published; no CTA reads another's histogram any more
    const unsigned* sel = cluster.map_shared_rank(s_sel, 0);
    const unsigned bin = sel[0];
    need -= sel[1];
    ncand = sel[2];
    hist[2 * tid] = 0;
    hist[2 * tid + 1] = 0;
    __syncthreads();  // every bin is zero before any thread counts the next pass
    prefix |= (unsigned long long)bin << shift;
    mask |= (unsigned long long)dmask << shift;
    hi = shift;
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (((unsigned)(key[e] >> shift) & dmask) != bin) cm &= ~(1u << e);
    // CTA 0 rewrites s_sel only after the next pass's first barrier, which
    // every CTA reaches after reading it
  }

  // the keys below the decided prefix and the candidates, into CTA 0
  const unsigned base = (unsigned)k - need;
  unsigned* r_taken = cluster.map_shared_rank(&s_taken, 0);
  unsigned long long* r_key = cluster.map_shared_rank(s_key, 0);
  int* r_idx = cluster.map_shared_rank(s_idx, 0);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (((valid >> e) & 1u) && (key[e] & mask) < prefix) {
      const unsigned slot = atomicAdd(r_taken, 1u);
      if (slot < (unsigned)kTopkMaxK) {  // always: fewer than k lie below
        r_key[slot] = key[e];
        r_idx[slot] = i0 + e;
      }
    }
  }
  if (ncand <= (unsigned)kSmallCand) {
    unsigned* r_ncand = cluster.map_shared_rank(&s_ncand, 0);
    unsigned long long* r_ckey = cluster.map_shared_rank(c_key, 0);
    int* r_cidx = cluster.map_shared_rank(c_idx, 0);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((cm >> e) & 1u) {
        const unsigned p = atomicAdd(r_ncand, 1u);
        if (p < (unsigned)kSmallCand) {
          r_ckey[p] = key[e];
          r_cidx[p] = i0 + e;
        }
      }
    }
    cluster.sync();  // everything for CTA 0 has arrived
    if (rank != 0) return;
    // candidate tid / 8, its rank summed over 8 threads
    const unsigned m = s_ncand < (unsigned)kSmallCand ? s_ncand : (unsigned)kSmallCand;
    const unsigned c = (unsigned)tid >> 3, part = (unsigned)tid & 7u;
    unsigned long long kt = 0;
    int it = 0;
    unsigned r = 0;
    if (c < m) {
      kt = c_key[c];
      it = c_idx[c];
      for (unsigned j = part; j < m; j += 8) r += before(c_key[j], c_idx[j], kt, it) ? 1u : 0u;
    }
#pragma unroll
    for (int off = 1; off < 8; off <<= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    if (c < m && part == 0 && r < need && base + r < (unsigned)kTopkMaxK) {
      s_key[base + r] = kt;
      s_idx[base + r] = it;
    }
  } else {
    // every bit decided and more than kSmallCand keys equal to the k-th: the
    // lowest document ids win.  CTA r holds a contiguous id range, so a
    // candidate's rank is the candidates of the CTAs before it plus its rank
    // in its own CTA (thread order is document order).
    const unsigned mine = __popc(cm);
    unsigned incl = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned v = lane < kW ? warp_sums[lane] : 0u;
      unsigned w = v;
#pragma unroll
      for (int off = 1; off < kW; off <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += o;
      }
      if (lane < kW) warp_sums[lane] = w - v;
      if (lane == kW - 1) blk_cnt = w;
    }
    cluster.sync();  // every CTA's count is visible
    unsigned before_me = 0;
    for (int r = 0; r < rank; ++r) before_me += *cluster.map_shared_rank(&blk_cnt, r);
    unsigned rr = before_me + warp_sums[warp] + incl - mine;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((cm >> e) & 1u) {
        if (rr < need && base + rr < (unsigned)kTopkMaxK) {
          r_key[base + rr] = key[e];
          r_idx[base + rr] = i0 + e;
        }
        ++rr;
      }
    }
    cluster.sync();  // everything for CTA 0 has arrived; nobody reads blk_cnt any more
    if (rank != 0) return;
  }
  __syncthreads();

  // CTA 0: the k taken, ordered by (key, document id)
  order_taken<kClusterThreads>(s_key, s_idx, k, wmd, N, out_idx, out_val);
}

template <int E>
cudaError_t launch_cluster(const double* wmd, int n, int k, int64_t* out_idx, double* out_val,
                           int cs, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cs);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, topk_cluster_kernel<E>, wmd, n, k, out_idx, out_val);
}

// Per device, once: the dynamic shared memory the 8-bit kernels need, and the
// cluster size the selection uses (16 CTAs where the GPU can run such a
// cluster, a non-portable size; else 8; 0 if neither fits).  Function
// attributes are set per device, so a process that selects on several GPUs
// sets them on each.
struct TopkSetup {
  bool done = false;
  cudaError_t err = cudaSuccess;
  int cs = 0;
};

TopkSetup topk_setup() {
  static std::mutex mu;
  static TopkSetup per_dev[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  dev = dev < 64 ? dev : 63;
  std::lock_guard<std::mutex> lock(mu);
  TopkSetup& st = per_dev[dev];
  if (st.done) return st;
  const size_t lists = 2 * (size_t)kCandMax * sizeof(int);
  st.err = cudaFuncSetAttribute(topk_kernel<true, kThreadsCached>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kCacheMax * sizeof(unsigned long long) + lists));
  if (st.err == cudaSuccess)
    st.err = cudaFuncSetAttribute(topk_kernel<false, kThreadsStream>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lists);
  const void* kerns[] = {(const void*)topk_cluster_kernel<4>, (const void*)topk_cluster_kernel<8>,
                         (const void*)topk_cluster_kernel<12>, (const void*)topk_cluster_kernel<16>,
                         (const void*)topk_cluster_kernel<20>, (const void*)topk_cluster_kernel<24>,
                         (const void*)topk_cluster_kernel<28>, (const void*)topk_cluster_kernel<32>};
  bool ok16 = true;
  for (const void* f : kerns)
    ok16 = ok16 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                       cudaSuccess;
  for (int want : {16, 8}) {
    if (want == 16 && !ok16) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)want);
    cfg.blockDim = dim3(kClusterThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)want;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, topk_cluster_kernel<32>, &cfg) == cudaSuccess && n > 0) {
      st.cs = want;
      break;
    }
  }
  cudaGetLastError();  // a refused cluster size leaves no error behind
  st.done = true;
  return st;
}

}  // namespace

cudaError_t launch_topk(const double* wmd, int64_t N, int k, int64_t* out_idx, double* out_val,
                        cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const size_t lists = 2 * (size_t)kCandMax * sizeof(int);
  const TopkSetup st = topk_setup();
  if (st.err != cudaSuccess) return st.err;
  // programmatic dependent launch: the CTA may become resident while the
  // kernel that writes WMD[] (the fused loop) drains; it waits for it first
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (N <= kSmallMaxN) {
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = 0;
    const int n = (int)N;
    const int e = (n + kSmallThreads - 1) / kSmallThreads;
    auto go = [&](auto kern) { return cudaLaunchKernelEx(&cfg, kern, wmd, n, k, out_idx, out_val); };
    if (e <= 1) return go(topk_small_kernel<1>);
    if (e <= 2) return go(topk_small_kernel<2>);
    if (e <= 3) return go(topk_small_kernel<3>);
    if (e <= 4) return go(topk_small_kernel<4>);
    if (e <= 6) return go(topk_small_kernel<6>);
    if (e <= 8) return go(topk_small_kernel<8>);
    if (e <= 10) return go(topk_small_kernel<10>);
    if (e <= 12) return go(topk_small_kernel<12>);
    if (e <= 16) return go(topk_small_kernel<16>);
    if (e <= 20) return go(topk_small_kernel<20>);
    if (e <= 24) return go(topk_small_kernel<24>);
    return go(topk_small_kernel<32>);
  }
  const int cs = N > kSmallMaxN ? st.cs : 0;
  if (cs > 0 && N <= (int64_t)cs * kClusterThreads * kClusterMaxE) {
    const int n = (int)N;
    const int e = ((n + cs - 1) / cs + kClusterThreads - 1) / kClusterThreads;
    if (e <= 4) return launch_cluster<4>(wmd, n, k, out_idx, out_val, cs, s);
    if (e <= 8) return launch_cluster<8>(wmd, n, k, out_idx, out_val, cs, s);
    if (e <= 12) return launch_cluster<12>(wmd, n, k, out_idx, out_val, cs, s);
    if (e <= 16) return launch_cluster<16>(wmd, n, k, out_idx, out_val, cs, s);
    if (e <= 20) return launch_cluster<20>(wmd, n, k, out_idx, out_val, cs, s);
    if (e <= 24) return launch_cluster<24>(wmd, n, k, out_idx, out_val, cs, s);
    if (e <= 28) return launch_cluster<28>(wmd, n, k, out_idx, out_val, cs, s);
    return launch_cluster<32>(wmd, n, k, out_idx, out_val, cs, s);
  }
  if (N <= kCacheMax) {
    cfg.blockDim = dim3(kThreadsCached);
    cfg.dynamicSmemBytes = (size_t)N * sizeof(unsigned long long) + lists;
    return cudaLaunchKernelEx(&cfg, topk_kernel<true, kThreadsCached>, wmd, N, k, out_idx, out_val);
  }
  cfg.blockDim = dim3(kThreadsStream);
  cfg.dynamicSmemBytes = lists;
  return cudaLaunchKernelEx(&cfg, topk_kernel<false, kThreadsStream>, wmd, N, k, out_idx, out_val);
}

}  // namespace wmd

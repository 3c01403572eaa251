// K1 on the 5th-generation tensor cores: cdist + K = exp(-lambda M).
//
// Sec. 5 of the paper turns the Euclidean distance into a matrix-multiply-like
// kernel, m^2(i, w) = |e_i|^2 + |e_w|^2 - 2 e_i . e_w, so that the v_r x V
// block of M comes out of one GEMM of the query rows (v_r x d) against the
// vocabulary (V x d), and the same kernel also emits K (Algorithm 1).  Here
// that GEMM runs on tcgen05 (kind::f16, float32 accumulation in TMEM) with
// float32 accuracy from an fp16 pair per operand, prepared once when the
// corpus is loaded: every row is scaled by a power of two 2^e so that its
// largest entry lies in [2^14, 2^15), and x = hi + lo 2^-11 with hi = fp16(x)
// and lo = fp16((x - hi) 2^11).  Then
//   a . b = 2^-(e_a + e_b) (a_hi . b_hi + 2^-11 (a_hi . b_lo + a_lo . b_hi))
// up to the dropped a_lo . b_lo term (2^-22 relative).  B (the query side)
// is kept as one 2N-row operand [B_hi; B_lo], so a_hi . b_hi and a_hi . b_lo
// come out of a single N = 2N MMA; a_lo . b_hi is a second MMA that
// accumulates into the a_hi . b_lo columns, so the large term and the two
// small ones are summed apart.  Both halves of the vocabulary tile arrive by
// TMA in their final form: no conversion pass touches shared memory.
//
// One persistent CTA per SM walks 128-row tiles of the active vocabulary:
//   warp 8        TMA producer: 128 x 64 fp16 k-blocks of vecs_hi and vecs_lo
//                 (128B-swizzled), into an S-stage ring in shared memory
//   warp 9        MMA issuer (one thread) and TMEM owner
//   warps 0..7    epilogue (two warps per TMEM lane quarter, half the columns
//                 each): TMEM -> registers, m, K, word-major stores
// The query side (B, N x d) is gathered once per CTA by the epilogue and MMA
// warps into shared memory and kept resident; the producer primes a few
// stages and holds the rest of the stream until those gathers are in flight,
// so that they do not queue behind it.  Accumulators are double buffered in
// TMEM so the epilogue of tile t overlaps the MMAs of tile t+1.  Every wait is
// bounded: on a timeout the CTA raises a flag, drains what it issued, frees
// its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "wmd_internal.h"

namespace wmd {
namespace tc {

constexpr int kM = 128;                   // vocabulary rows per tile (MMA M)
constexpr int kKB = 64;                   // fp16 elements per 128-byte k-block
constexpr int kHalfBytes = kM * 128;      // one k-block of the hi (or lo) tile
constexpr int kStageBytes = 2 * kHalfBytes;
constexpr int kThreads = 320;             // 10 warps
constexpr int kBuildThreads = 288;        // warps 0..7 and 9 gather the query operand
constexpr int kPrime = 2;                 // stages issued before the query gathers
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz (drains; default role limit)
constexpr float kLoScale = 1.f / 2048.f;  // 2^-11

struct Params {
  const uint16_t* vhi;  // fp16 pair of the (permuted) vocabulary rows, V x ldv
  const uint16_t* vlo;
  const float* rscale;  // 2^-e per row
  int ldv;
  const float* norms;
  const float* vecs;    // the float32 rows (near pairs are recomputed from them)
  int d;
  int64_t U;
  const int32_t* perm;
  int64_t V;
  const int32_t* q_ids;
  const float* q_w;
  int v_r;
  int VR;
  float lambda;
  void* K;
  int ldk;
  int kcol0;
  float* r_out;
  float* lam_out;
  int num_tiles;
  int KB;
  int S;  // stages of the A ring
  int* err;              // this launch's error slots, one per CTA, written by every CTA
                         // at its end: 0, or a timeout code and/or kRangeFlag
  long long wait_cycles; // limit of every wait between roles (drains keep kWaitCycles)
  // read-only data the next kernel (the fused loop) starts from: prefetched
  // into L2 with the evict-last priority while the vocabulary streams
  const void* pf_ptr[3];
  size_t pf_bytes[3];
};

#ifdef WMD_TC_TRACE
// Timeline of the first CTAs (globaltimer, ns) for tuning: [cta][event][index].
__device__ long long g_tc_trace[4][8][64];
__device__ __forceinline__ void trace(int ev, int idx) {
  if (blockIdx.x < 4 && idx < 64) {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    g_tc_trace[blockIdx.x][ev][idx] = t;
  }
}
#define TC_TRACE(ev, idx) trace(ev, idx)
#else
#define TC_TRACE(ev, idx) ((void)0)
#endif

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of the same phase (mbarrier.test_wait never suspends).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Limits below this many cycles poll with test_wait: try_wait may suspend the
// thread for longer than such a limit, which would then never run out.
constexpr long long kPollBelow = 1000000;

// Bounded wait: false if the phase did not complete in time or another role
// of the CTA gave up (the shared abort flag).  The first wait that runs out
// records which role and iteration gave up in the abort flag:
// 0x40000000 | role << 24 | (iteration & 0xffffff).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         int role, int iter, long long limit) {
  const long long t0 = clock64();
  const bool poll = limit < kPollBelow;
  while (!(poll ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity))) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      atomicCAS(const_cast<int*>(abort_flag), 0, 0x40000000 | (role << 24) | (iter & 0xffffff));
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, A: 128 x 16 fp16, B: N x 16 fp16, both
// K-major, float32 accumulation.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride-dimension offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // swizzle: 128 bytes
  return d;
}

// Instruction descriptor for kind::f16: D float32, A and B fp16 (format 0),
// both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int NC>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_load<8>(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Hardware square root and base-2 exponential (PTX sqrt.approx / ex2.approx,
// relative errors near 2^-23 and 2^-22): the epilogue's two transcendental
// steps in one instruction each, since at 128-column queries the epilogue,
// not the vocabulary stream, sets the kernel's pace.
__device__ __forceinline__ float sqrt_fast(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float exp2_fast(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kLog2e = 1.4426950408889634f;

// Stores the first n (a multiple of 4, n <= CH) values of a row chunk.
template <int CH>
__device__ __forceinline__ void store_chunk(float* dst, const float (&v)[CH], int n) {
#pragma unroll
  for (int j = 0; j < CH; j += 4)
    if (j < n) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
}

template <int CH>
__device__ __forceinline__ void store_chunk(__nv_bfloat16* dst, const float (&v)[CH], int n) {
#pragma unroll
  for (int j = 0; j < CH; j += 4) {
    if (j < n) {
      __nv_bfloat162 a = __floats2bfloat162_rn(v[j], v[j + 1]);
      __nv_bfloat162 b = __floats2bfloat162_rn(v[j + 2], v[j + 3]);
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&a);
      u.y = *reinterpret_cast<uint32_t*>(&b);
      *reinterpret_cast<uint2*>(dst + j) = u;
    }
  }
}

// ------------------------------------------------------------------ kernel
// N: query columns of the tile (B holds 2N rows, the MMAs are N = 2N and N).
template <int N>
__host__ __device__ constexpr int tmem_cols() {
  return 4 * N;  // two buffers of [a.b_hi-part | cross terms]
}

template <int N, typename KT>
__global__ void __launch_bounds__(kThreads, 1)
    cdist_tc_kernel(const __grid_constant__ CUtensorMap tmap_hi,
                    const __grid_constant__ CUtensorMap tmap_lo, const Params p) {
  constexpr uint32_t kIdesc2 = idesc_f16(kM, 2 * N);  // a_hi . [b_hi | b_lo]
  constexpr uint32_t kIdesc = idesc_f16(kM, N);       // a_lo . b_hi
  constexpr int kCols = tmem_cols<N>();
  static_assert(kCols >= 32 && kCols <= 512 && (kCols & (kCols - 1)) == 0, "TMEM allocation");
  constexpr int kHalfN = N / 2;                       // columns per epilogue warp
  constexpr int CH = kHalfN < 32 ? kHalfN : 32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  const int KB = p.KB;
  const int S = p.S;
  const int bblock = 2 * N * 128;               // bytes of one [B_hi; B_lo] k-block
  uint8_t* Bcat = smem;
  uint8_t* Abuf = Bcat + KB * bblock;           // S stages: hi tile, then lo tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(Abuf + S * kStageBytes);
  uint64_t* full = bars;
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  int32_t* qrow_s = reinterpret_cast<int32_t*>(drain + 1);
  float* qn_s = reinterpret_cast<float*>(qrow_s + N);
  float* qrs_s = qn_s + N;
  uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(qrs_s + N);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_base_s + 1);
  int* consumed_s = const_cast<int*>(abort_flag) + 1;
  volatile int* issued_s = consumed_s + 1;      // gathering warps whose loads are in flight
  int* range_s = const_cast<int*>(issued_s) + 1; // kRangeFlag once an epilogue thread saw lambda m too large

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  if (tid == 0) TC_TRACE(5, 0);

  // the device rows of the query words (ids -> permutation) are looked up
  // first, so that these dependent loads overlap the prologue
  int qrow = -1;
  if (tid < N && tid < p.v_r) {
    const int64_t id = p.q_ids[tid];
    qrow = (id >= 0 && id < p.V) ? p.perm[id] : -2;
  }
  // CTA 0 also copies the padded weights for the loop kernel: loaded here,
  // beside the ids, so that their store below does not wait for a load
  float qw = 0.f;
  if (p.r_out && blockIdx.x == 0 && tid < p.VR && tid < p.v_r) qw = p.q_w[tid];

  // ---- prologue: barriers and TMEM only, so that the producer starts at once
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 256);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    *consumed_s = 0;
    *issued_s = 0;
    *range_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == 9) tmem_alloc(tmem_base_s, kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_base_s;
  const int nlt = (p.num_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  if (warp != 8) {
    // ---------------------------------------------------------------- B, all but the producer
    // query columns (device row, norm, inverse scale), the padded weights,
    // then the resident B = the query rows' fp16 pairs in the 128B-swizzled
    // K-major layout (chunk c of row n lands at chunk c ^ (n % 8)): hi rows
    // 0..N-1, lo rows N..2N-1 of every k-block
    const int bt = tid < 256 ? tid : tid - 32;  // 0 .. 287 (bt = tid below N)
    float qn = 0.f, qrs = 0.f;
    if (bt < N) {
      const int row = qrow;
      qrow_s[bt] = row;
      // these two loads stay in flight behind the B loads below
      if (row >= 0) {
        qn = __ldg(p.norms + row);
        qrs = __ldg(p.rscale + row);
      } else if (row == -2) {
        qn = __int_as_float(0x7fc00000);
      }
    }
    if (p.r_out && blockIdx.x == 0 && bt < p.VR) p.r_out[bt] = qw;
    if (p.lam_out && blockIdx.x == 0 && bt == 0) {
      // lambda, and the final step's scale -ln 2 / lambda as a double two
      // floats further on (8-byte aligned), for the loop kernel
      *p.lam_out = p.lambda;
      *reinterpret_cast<double*>(p.lam_out + 2) = -0.69314718055994530942 / (double)p.lambda;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kBuildThreads) : "memory");
    if (tid == 0) TC_TRACE(6, 0);
    // every 16-byte chunk of B goes straight from global to shared memory
    // (cp.async, all of a thread's chunks in flight at once); the chunks of
    // padding rows and of ids outside [0, V) are zero-filled (source size 0)
    const int per_row = KB * 8;                 // 16-byte chunks of one row's hi (or lo) part
    const int total = 2 * N * per_row;
    for (int idx = bt; idx < total; idx += kBuildThreads) {
      const int nn = idx / per_row;             // 0..2N-1: hi rows, then lo rows
      const int n = nn < N ? nn : nn - N;
      const int rem = idx - nn * per_row;
      const int kb = rem >> 3;
      const int ch = rem & 7;
      const int k = kb * kKB + ch * 8;
      const int row = qrow_s[n];
      const bool ok = row >= 0 && k < p.ldv;
      const uint16_t* src = (nn < N ? p.vhi : p.vlo) + (ok ? (size_t)row * p.ldv + k : 0);
      const uint32_t dst = smem_u32(Bcat + kb * bblock + nn * 128 + ((ch ^ (nn & 7)) << 4));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                   "r"(ok ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // the producer may stream the vocabulary now: the query copies are ahead of it
    __syncwarp();
    if (lane == 0) atomicAdd(const_cast<int*>(issued_s), 1);
    if (tid == 0) TC_TRACE(6, 1);
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (bt < N) {
      qn_s[bt] = qn;
      qrs_s[bt] = qrs;
    }
    fence_async_smem();
    asm volatile("bar.sync 1, %0;" ::"r"(kBuildThreads) : "memory");  // B resident for everyone
    if (tid == 0) TC_TRACE(5, 1);
  }

  if (warp == 8) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmap_hi) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmap_lo) : "memory");
      int it = 0;
      bool ok = true;
      for (int lt = 0; lt < nlt && ok; ++lt) {
        const int w0 = ((int)blockIdx.x + lt * (int)gridDim.x) * kM;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          if (it == kPrime) {
            // hold the stream until every gathering warp has its loads in flight
            const long long t0 = clock64();
            while (*issued_s < kBuildThreads / 32) {
              if (*abort_flag) {
                ok = false;
                break;
              }
              if (clock64() - t0 > p.wait_cycles) {
                atomicCAS(const_cast<int*>(abort_flag), 0, 0x40000000 | (7 << 24));
                ok = false;
                break;
              }
            }
            if (!ok) break;
          }
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, 1, it, p.wait_cycles)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], kStageBytes);
          tma_load_2d(Abuf + s * kStageBytes, &tmap_hi, &full[s], kb * kKB, w0);
          tma_load_2d(Abuf + s * kStageBytes + kHalfBytes, &tmap_lo, &full[s], kb * kKB, w0);
          TC_TRACE(0, it);
        }
      }
      // the vocabulary stream of this CTA is issued: the next kernel in the
      // stream (the fused loop) may start its CTAs once every CTA is here,
      // so that they share the SMs with this grid's last tiles only (started
      // earlier, they slowed this kernel more than they gained); they wait
      // for this grid's results before reading them
      asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
      if (*abort_flag) {
        // let the loads already issued land before the CTA leaves
        for (int j = *consumed_s; j < it; ++j) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[j % S], (uint32_t)(j / S) & 1u) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp == 9) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int lt = 0; lt < nlt && ok; ++lt) {
        const int ab = lt & 1;
        const uint32_t tph = (uint32_t)(lt >> 1) & 1u;
        if (!mbar_wait(&tempty[ab], tph ^ 1u, abort_flag, 3, lt, p.wait_cycles)) break;
        tc_fence_after();
        // columns [0, N): a_hi . b_hi; [N, 2N): a_hi . b_lo + a_lo . b_hi (scaled 2^11)
        const uint32_t d_tmem = tmem_base + (uint32_t)(ab * 2 * N);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          const uint32_t a_hi = smem_u32(Abuf + s * kStageBytes);
          const uint32_t a_lo = a_hi + kHalfBytes;
          const uint32_t b_cat = smem_u32(Bcat + kb * bblock);  // rows 0..N-1 are b_hi
          if (!mbar_wait(&full[s], ph, abort_flag, 4, it, p.wait_cycles)) {
            ok = false;
            break;
          }
          TC_TRACE(2, it);
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < kKB / 16; ++ks) {
            const uint32_t o = ks * 32;  // 16 fp16 = 32 bytes along K
            mma_f16(d_tmem, sw128_desc(a_hi + o), sw128_desc(b_cat + o), kIdesc2, (kb | ks) != 0);
            mma_f16(d_tmem + N, sw128_desc(a_lo + o), sw128_desc(b_cat + o), kIdesc, 1);
          }
          mma_commit(&empty[s]);
          if (ok) *consumed_s = it + 1;
        }
        if (ok) mma_commit(&tfull[ab]);
      }
      // every MMA issued by this thread completes before TMEM is released
      mma_commit(drain);
      const long long t0 = clock64();
      while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
    __syncwarp();
    // the vocabulary stream is over; while the last epilogue runs, the warp
    // prefetches this CTA's share of the next kernel's read-only inputs into
    // L2 (evict-last), one 128-byte line per prefetch
    for (int r = 0; r < 3; ++r) {
      const char* base = static_cast<const char*>(p.pf_ptr[r]);
      if (!base) continue;
      const size_t lines = (p.pf_bytes[r] + 127) / 128;
      for (size_t l = (size_t)blockIdx.x * 32 + lane; l < lines; l += (size_t)gridDim.x * 32)
        asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(base + l * 128));
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and the columns
    // [kHalfN (w / 4), kHalfN (w / 4 + 1)) of both accumulator parts
    const int q = warp & 3;
    const int c0 = (warp >> 2) * kHalfN;
    const int row_in_tile = q * 32 + lane;
    const int ncols = min(N, p.VR);             // columns this launch owns in K
    bool out_of_range = false;                  // some lambda m reached the float32 limit of K
    for (int lt = 0; lt < nlt; ++lt) {
      const int ab = lt & 1;
      const uint32_t tph = (uint32_t)(lt >> 1) & 1u;
      const int64_t w = (int64_t)((int)blockIdx.x + lt * (int)gridDim.x) * kM + row_in_tile;
      const bool live = w < p.U;
      const float nw = live ? p.norms[w] : 0.f;  // issued before the wait
      const float rsw = live ? p.rscale[w] : 0.f;
      if (!mbar_wait(&tfull[ab], tph, abort_flag, 5, lt, p.wait_cycles)) break;
      if (tid == 0) TC_TRACE(3, lt);
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * 2 * N);
#pragma unroll
      for (int cc = 0; cc < kHalfN; cc += CH) {
        const int c = c0 + cc;
        float big[CH], small[CH];
        tmem_load<CH>(taddr + c, big);
        tmem_load<CH>(taddr + N + c, small);
        if (cc + CH == kHalfN) {
          tc_fence_before();
          mbar_arrive(&tempty[ab]);
        }
        if (live && c < ncols) {
          // a.b = 2^-(e_w + e_q) (big + 2^-11 small); m^2 = |a|^2 + |b|^2 - 2 a.b
          // (clamped), K = exp(-lambda m); the query's own word is exactly
          // m = 0 (K = 1); padding columns are 0 and an id outside [0, V) gives
          // NaN.  Where the GEMM form has cancelled more than two bits (m^2
          // below a quarter of |a|^2 + |b|^2: a near pair, Sec. 5), m^2 is
          // recomputed from the float32 rows by direct differences (Sec. 2).
          // Three passes, so that the rare recomputation stays out of the two
          // straight-line ones: m^2 by the GEMM form, the near pairs again,
          // then K.
          float kv[CH];
          uint32_t near = 0;  // bit j: column c + j is a near pair
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            const int col = c + j;
            const float dot = (fmaf(small[j], kLoScale, big[j]) * rsw) * qrs_s[col];
            const int qr = qrow_s[col];
            const float nsum = nw + qn_s[col];
            kv[j] = nsum - 2.f * dot;  // m^2 for now
            near |= (kv[j] < kNearPair * nsum && qr >= 0 && qr != (int)w && col < p.v_r ? 1u : 0u) << j;
          }
          if (near) {
#pragma unroll
            for (int j = 0; j < CH; ++j)
              if ((near >> j) & 1u) kv[j] = direct_m2(p.vecs, p.ldv, p.d, w, qrow_s[c + j]);
          }
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            const int col = c + j;
            const int qr = qrow_s[col];
            const float lm = p.lambda * sqrt_fast(fmaxf(kv[j], 0.f));
            const float e = exp2_fast(-lm * kLog2e);  // exp(-lambda m)
            const float k = qr == (int)w ? 1.f : (qr == -2 ? __int_as_float(0x7fc00000) : e);
            out_of_range |= col < p.v_r && qr >= 0 && qr != (int)w && lm > kRangeLimit;
            kv[j] = col < p.v_r ? k : 0.f;
          }
          store_chunk<CH>(static_cast<KT*>(p.K) + (size_t)w * p.ldk + p.kcol0 + c, kv, ncols - c);
        }
      }
    }
    if (out_of_range) atomicOr(range_s, kRangeFlag);
  }

  if (warp == 0 && lane == 0) TC_TRACE(4, 0);
  tc_fence_before();
  __syncthreads();
  if (tid == 0) TC_TRACE(5, 2);
  if (warp == 9) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kCols);
  }
  // this CTA's error slot, written whatever happened, so that nothing has to
  // clear it before the launch
  if (tid == 0) p.err[blockIdx.x] = *abort_flag | *range_s;
}

// Shared memory of one CTA for S stages.
template <int N>
size_t smem_bytes(int KB, int S) {
  return 1024 + 2 * (size_t)KB * N * 128 + (size_t)S * kStageBytes + (2 * S + 5) * 8 + N * 12 + 32;
}

constexpr size_t kSmemLimit = 232448;
constexpr int kMaxStages = 6;

// Stages that fit next to the resident B for this width (0 if fewer than 2).
template <int N>
int stages_for(int KB) {
  int S = kMaxStages;
  while (S >= 2 && smem_bytes<N>(KB, S) > kSmemLimit) --S;
  return S >= 2 ? S : 0;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

template <int N, typename KT>
cudaError_t launch_t(const wmd_corpus* c, Params p, cudaStream_t s) {
  p.S = stages_for<N>(p.KB);
  if (p.S == 0) return cudaErrorNotSupported;
  const size_t bytes = smem_bytes<N>(p.KB, p.S);
  // the shared-memory limit is raised once per device and size (never inside
  // a stream capture: the first launch of a shape always runs eagerly)
  static std::mutex mu;
  static size_t set_bytes[64] = {};
  {
    std::lock_guard<std::mutex> lock(mu);
    const int dev = c->device < 64 ? c->device : 63;
    if (set_bytes[dev] < bytes) {
      cudaError_t e = cudaFuncSetAttribute(cdist_tc_kernel<N, KT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      set_bytes[dev] = bytes;
    }
  }
  const int grid = cdist_tc_grid(c);
  const CUtensorMap* mh = reinterpret_cast<const CUtensorMap*>(c->tmap_hi);
  const CUtensorMap* ml = reinterpret_cast<const CUtensorMap*>(c->tmap_lo);
  cdist_tc_kernel<N, KT><<<grid, kThreads, bytes, s>>>(*mh, *ml, p);
  return cudaGetLastError();
}

int num_kblocks(const wmd_corpus* c) { return (c->ldv + kKB - 1) / kKB; }

}  // namespace tc

bool make_vecs_tensor_map(wmd_corpus* c) {
  auto fn = tc::encode_fn();
  if (!fn) return false;
  static_assert(sizeof(CUtensorMap) <= sizeof(c->tmap_hi), "tensor map storage");
  cuuint64_t dims[2] = {(cuuint64_t)c->ldv, (cuuint64_t)c->V};
  cuuint64_t strides[1] = {(cuuint64_t)c->ldv * sizeof(uint16_t)};
  cuuint32_t box[2] = {tc::kKB, tc::kM};
  cuuint32_t estr[2] = {1, 1};
  for (int part = 0; part < 2; ++part) {
    CUtensorMap map;
    CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, part ? c->vecs_lo : c->vecs_hi,
                    dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::memcpy(part ? c->tmap_lo : c->tmap_hi, &map, sizeof(map));
  }
  return true;
}

int cdist_tc_grid(const wmd_corpus* c) {
  const int tiles = (int)((c->U + tc::kM - 1) / tc::kM);
  return std::max(1, std::min(tiles, c->num_sms));
}

int cdist_tc_max_width(const wmd_corpus* c) {
  if (!c->tmap_ok || c->U == 0) return 0;
  const int KB = tc::num_kblocks(c);
  if (tc::stages_for<128>(KB)) return 128;
  if (tc::stages_for<64>(KB)) return 64;
  if (tc::stages_for<32>(KB)) return 32;
  if (tc::stages_for<16>(KB)) return 16;
  return 0;
}

// Tensor-core path for one slice of at most cdist_tc_max_width(c) query
// columns (B stays resident in shared memory); cudaErrorNotSupported otherwise.
cudaError_t launch_cdist_tc(const wmd_corpus* c, const int32_t* q_ids, const float* q_w, int v_r,
                            int VR, float lambda, wmd_precision prec, void* K, int ldk, int kcol0,
                            float* r_out, float* lam_out, int* err, const L2Prefetch* pf,
                            cudaStream_t s) {
  if (!c->tmap_ok || VR > 128 || c->U == 0) return cudaErrorNotSupported;
  tc::Params p;
  p.vhi = c->vecs_hi;
  p.vlo = c->vecs_lo;
  p.rscale = c->rscale;
  p.ldv = c->ldv;
  p.norms = c->norms;
  p.vecs = c->vecs;
  p.d = c->d;
  p.U = c->U;
  p.perm = c->perm;
  p.V = c->V;
  p.q_ids = q_ids;
  p.q_w = q_w;
  p.v_r = v_r;
  p.VR = VR;
  p.lambda = lambda;
  p.K = K;
  p.ldk = ldk;
  p.kcol0 = kcol0;
  p.r_out = r_out;
  p.lam_out = lam_out;
  p.num_tiles = (int)((c->U + tc::kM - 1) / tc::kM);
  p.KB = tc::num_kblocks(c);
  p.S = 0;
  p.err = err;
  p.wait_cycles = c->wait_cycles > 0 ? c->wait_cycles : tc::kWaitCycles;
  for (int r = 0; r < 3; ++r) {
    p.pf_ptr[r] = pf ? pf->ptr[r] : nullptr;
    p.pf_bytes[r] = pf ? pf->bytes[r] : 0;
  }
  const bool bf = prec == WMD_PREC_BF16_K;
  if (VR <= 16) return bf ? tc::launch_t<16, __nv_bfloat16>(c, p, s) : tc::launch_t<16, float>(c, p, s);
  if (VR <= 32) return bf ? tc::launch_t<32, __nv_bfloat16>(c, p, s) : tc::launch_t<32, float>(c, p, s);
  if (VR <= 64) return bf ? tc::launch_t<64, __nv_bfloat16>(c, p, s) : tc::launch_t<64, float>(c, p, s);
  return bf ? tc::launch_t<128, __nv_bfloat16>(c, p, s) : tc::launch_t<128, float>(c, p, s);
}

}  // namespace wmd

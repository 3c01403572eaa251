// K1 on the 5th-generation tensor cores: cdist + K = exp(-lambda M).
//
// Sec. 5 of the paper turns the Euclidean distance into a matrix-multiply-like
// kernel, m^2(i, w) = |e_i|^2 + |e_w|^2 - 2 e_i . e_w, so that the v_r x V
// block of M comes out of one GEMM of the query rows (v_r x d) against the
// vocabulary (V x d), and the same kernel also emits K (Algorithm 1).  Here
// that GEMM runs on tcgen05 with float32 accuracy from TF32 inputs
// (3xTF32: a = a_hi + a_lo, a.b ~ a_hi.b_hi + a_hi.b_lo + a_lo.b_hi, dropping
// only a_lo.b_lo, which is 2^-20 relative), accumulating in TMEM.  B is kept
// as one 2N-row operand [B_hi; B_lo], so a_hi.b_hi and a_hi.b_lo come out of
// a single N = 2N MMA that reads the A tile once; a_lo.b_hi is a second MMA.
//
// One persistent CTA per SM walks 128-row tiles of the active vocabulary:
//   warp 8        TMA producer: 128 x 32 float32 k-blocks of vecs, 128B-swizzled
//   warps 4..7    converters: split each landed k-block into hi and lo parts
//   warp 9        MMA issuer (one thread) and TMEM owner
//   warps 0..3    epilogue: TMEM -> registers, m, K, word-major stores
// The query side (B, N x d) is gathered once per CTA into shared memory, split
// into hi/lo parts and kept resident.  The hi part of A is the landed float32
// tile itself (the tensor core reads the tf32 bits of each operand).  Accumulators are double buffered in
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
constexpr int kKB = 32;                   // float32 elements per 128-byte k-block
constexpr int kStageBytes = kM * kKB * 4; // one k-block of the A tile
constexpr int kThreads = 320;             // 10 warps
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

struct Params {
  const float* vecs;
  int ldv;
  const float* norms;
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
  int* err;
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

// Bounded wait: false if the phase did not complete in time or another role
// of the CTA gave up (the shared abort flag).  The first wait that runs out
// records which role and iteration gave up in the abort flag:
// 0x40000000 | role << 24 | (iteration & 0xffffff).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         int role, int iter) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
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

// D[tmem] (+)= A[smem] * B[smem]^T, A: 128 x 8 tf32, B: N x 8 tf32, both K-major.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
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

// Instruction descriptor for kind::tf32: D float32, A and B tf32, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int NC>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float* v);

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

// TMEM columns per tile buffer: 2N for a_hi.[b_hi | b_lo] and N for
// a_lo.b_hi; two buffers, rounded up to a power of two.
template <int N>
__host__ __device__ constexpr int tmem_cols() {
  return 6 * N <= 32 ? 32 : (6 * N <= 64 ? 64 : (6 * N <= 128 ? 128 : (6 * N <= 256 ? 256 : 512)));
}

// Stores the first n (a multiple of 4, n <= N) values of a row.
template <int N>
__device__ __forceinline__ void store_row(float* dst, const float (&v)[N], int n) {
#pragma unroll
  for (int j = 0; j < N; j += 4)
    if (j < n) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
}

template <int N>
__device__ __forceinline__ void store_row(__nv_bfloat16* dst, const float (&v)[N], int n) {
#pragma unroll
  for (int j = 0; j < N; j += 4) {
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
// N: query columns of the tile (MMA N); S: TMA stages of A; LS: slots of the
// lo-part ring (the hi part is the landed float32 tile itself: the tensor
// core reads only the tf32 bits of each operand, and lo = a - tf32(a)).
template <int N, int S, int LS, typename KT>
__global__ void __launch_bounds__(kThreads, 1)
    cdist_tc_kernel(const __grid_constant__ CUtensorMap tmap_a, const Params p) {
  constexpr uint32_t kIdesc2 = idesc_tf32(kM, 2 * N);  // a_hi . [b_hi | b_lo]
  constexpr uint32_t kIdesc = idesc_tf32(kM, N);       // a_lo . b_hi
  constexpr int kCols = tmem_cols<N>();
  static_assert(LS < S, "the lo ring must be shorter than the stage ring");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  const int KB = p.KB;
  const int bblock = 2 * N * 128;               // bytes of one [B_hi; B_lo] k-block
  uint8_t* Bcat = smem;
  uint8_t* Abuf = Bcat + KB * bblock;           // S stages of landed float32 tiles
  uint8_t* Lbuf = Abuf + S * kStageBytes;       // LS slots of lo parts
  uint64_t* bars = reinterpret_cast<uint64_t*>(Lbuf + LS * kStageBytes);
  uint64_t* full = bars;
  uint64_t* conv = full + S;
  uint64_t* empty = conv + S;
  uint64_t* tfull = empty + S;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  int32_t* qrow_s = reinterpret_cast<int32_t*>(drain + 1);
  float* qn_s = reinterpret_cast<float*>(qrow_s + N);
  uint32_t* tmem_base_s = reinterpret_cast<uint32_t*>(qn_s + N);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_base_s + 1);
  int* consumed_s = const_cast<int*>(abort_flag) + 1;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  if (tid == 0) TC_TRACE(5, 0);

  // ---- prologue: barriers and TMEM only, so that the producer starts at once
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    *consumed_s = 0;
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
    // query columns (device row, norm), the padded weights, then the resident
    // B = query rows split into tf32 hi and lo parts in the 128B-swizzled
    // K-major layout (chunk c of row n lands at chunk c ^ (n % 8)); every
    // thread issues all its loads before its first store
    constexpr int kBT = kThreads - 32;
    const int bt = tid < 256 ? tid : tid - 32;  // 0 .. 287
    if (bt < N) {
      int row = -1;
      if (bt < p.v_r) {
        const int64_t id = p.q_ids[bt];
        row = (id >= 0 && id < p.V) ? p.perm[id] : -2;
      }
      qrow_s[bt] = row;
    }
    if (p.r_out && blockIdx.x == 0 && bt < p.VR) p.r_out[bt] = bt < p.v_r ? p.q_w[bt] : 0.f;
    if (p.lam_out && blockIdx.x == 0 && bt == 0) *p.lam_out = p.lambda;
    asm volatile("bar.sync 1, %0;" ::"r"(kBT) : "memory");
    const int total = N * KB * 8;
    for (int base = bt; base < total; base += kBT * 12) {
      float4 v[12];
#pragma unroll
      for (int j = 0; j < 12; ++j) {
        const int idx = base + j * kBT;
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < total) {
          const int n = idx / (KB * 8);
          const int rem = idx - n * KB * 8;
          const int k = (rem >> 3) * kKB + (rem & 7) * 4;
          const int row = qrow_s[n];
          if (row >= 0 && k < p.ldv)
            v[j] = __ldg(reinterpret_cast<const float4*>(p.vecs + (size_t)row * p.ldv + k));
          else if (row == -2)
            v[j] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int j = 0; j < 12; ++j) {
        const int idx = base + j * kBT;
        if (idx < total) {
          const int n = idx / (KB * 8);
          const int rem = idx - n * KB * 8;
          const int kb = rem >> 3;
          const int ch = rem & 7;
          float4 hi;
          hi.x = __uint_as_float(__float_as_uint(v[j].x) & 0xFFFFE000u);
          hi.y = __uint_as_float(__float_as_uint(v[j].y) & 0xFFFFE000u);
          hi.z = __uint_as_float(__float_as_uint(v[j].z) & 0xFFFFE000u);
          hi.w = __uint_as_float(__float_as_uint(v[j].w) & 0xFFFFE000u);
          const float4 lo = make_float4(v[j].x - hi.x, v[j].y - hi.y, v[j].z - hi.z, v[j].w - hi.w);
          const int nl = n + N;  // row of the lo part in the 2N-row operand
          *reinterpret_cast<float4*>(Bcat + kb * bblock + n * 128 + ((ch ^ (n & 7)) << 4)) = hi;
          *reinterpret_cast<float4*>(Bcat + kb * bblock + nl * 128 + ((ch ^ (nl & 7)) << 4)) = lo;
        }
      }
    }
    // norms of the query words (off the load chain of B)
    if (bt < N) {
      const int row = qrow_s[bt];
      qn_s[bt] = row >= 0 ? p.norms[row] : (row == -2 ? __int_as_float(0x7fc00000) : 0.f);
    }
    fence_async_smem();
    asm volatile("bar.sync 1, %0;" ::"r"(kBT) : "memory");  // B resident for everyone
    if (tid == 0) TC_TRACE(5, 1);
  }

  if (warp == 8) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmap_a) : "memory");
      int it = 0;
      bool ok = true;
      for (int lt = 0; lt < nlt && ok; ++lt) {
        const int w0 = ((int)blockIdx.x + lt * (int)gridDim.x) * kM;
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, 1, it)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], kStageBytes);
          tma_load_2d(Abuf + s * kStageBytes, &tmap_a, &full[s], kb * kKB, w0);
          TC_TRACE(0, it);
        }
      }
      if (*abort_flag) {
        // let the loads already issued land before the CTA leaves
        for (int j = *consumed_s; j < it; ++j) {
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[j % S], (uint32_t)(j / S) & 1u) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // ---------------------------------------------------------------- converters
    // lo = a - tf32(a) of every landed tile, into ring slot it % LS once the
    // MMAs that read that slot (iteration it - LS) have completed
    const int ct = tid - 128;
    int it = 0;
    bool ok = true;
    for (int lt = 0; lt < nlt && ok; ++lt) {
      for (int kb = 0; kb < KB; ++kb, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!mbar_wait(&full[s], ph, abort_flag, 2, it)) {
          ok = false;
          break;
        }
        if (ct == 0) TC_TRACE(1, it);
        if (it >= LS) {
          const int j = it - LS;
          if (!mbar_wait(&empty[j % S], (uint32_t)(j / S) & 1u, abort_flag, 6, it)) {
            ok = false;
            break;
          }
        }
        const float4* A4 = reinterpret_cast<const float4*>(Abuf + s * kStageBytes);
        float4* L4 = reinterpret_cast<float4*>(Lbuf + (it % LS) * kStageBytes);
        float4 v[kStageBytes / 16 / 128];
#pragma unroll
        for (int j = 0; j < kStageBytes / 16 / 128; ++j) v[j] = A4[ct + 128 * j];
#pragma unroll
        for (int j = 0; j < kStageBytes / 16 / 128; ++j) {
          const float4 a = v[j];
          L4[ct + 128 * j] = make_float4(a.x - __uint_as_float(__float_as_uint(a.x) & 0xFFFFE000u),
                                         a.y - __uint_as_float(__float_as_uint(a.y) & 0xFFFFE000u),
                                         a.z - __uint_as_float(__float_as_uint(a.z) & 0xFFFFE000u),
                                         a.w - __uint_as_float(__float_as_uint(a.w) & 0xFFFFE000u));
        }
        fence_async_smem();
        mbar_arrive(&conv[s]);
        if (ct == 0) *consumed_s = it + 1;
      }
    }
  } else if (warp == 9) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int lt = 0; lt < nlt && ok; ++lt) {
        const int ab = lt & 1;
        const uint32_t aph = (uint32_t)(lt >> 1) & 1u;
        if (!mbar_wait(&tempty[ab], aph ^ 1u, abort_flag, 3, lt)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(ab * 3 * N);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          const uint32_t a_hi = smem_u32(Abuf + s * kStageBytes);
          const uint32_t a_lo = smem_u32(Lbuf + (it % LS) * kStageBytes);
          const uint32_t b_cat = smem_u32(Bcat + kb * bblock);  // rows 0..N-1 are b_hi
          // a_hi . [b_hi | b_lo] as soon as the tile lands ...
          if (!mbar_wait(&full[s], ph, abort_flag, 4, it)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < kKB / 8; ++ks) {
            const uint32_t o = ks * 32;  // 8 tf32 = 32 bytes along K
            mma_tf32(d_tmem, sw128_desc(a_hi + o), sw128_desc(b_cat + o), kIdesc2, (kb | ks) != 0);
          }
          // ... a_lo . b_hi once the converters wrote the lo part
          if (!mbar_wait(&conv[s], ph, abort_flag, 4, it)) {
            ok = false;
            break;
          }
          TC_TRACE(2, it);
          tc_fence_after();
#pragma unroll
          for (int ks = 0; ks < kKB / 8; ++ks) {
            const uint32_t o = ks * 32;
            mma_tf32(d_tmem + 2 * N, sw128_desc(a_lo + o), sw128_desc(b_cat + o), kIdesc, (kb | ks) != 0);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&tfull[ab]);
      }
      // every MMA issued by this thread completes before TMEM is released
      mma_commit(drain);
      const long long t0 = clock64();
      while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int row_in_tile = warp * 32 + lane;
    float acc[N];
    for (int lt = 0; lt < nlt; ++lt) {
      const int ab = lt & 1;
      const uint32_t aph = (uint32_t)(lt >> 1) & 1u;
      const int64_t w = (int64_t)((int)blockIdx.x + lt * (int)gridDim.x) * kM + row_in_tile;
      const float nw = w < p.U ? p.norms[w] : 0.f;  // issued before the wait
      if (!mbar_wait(&tfull[ab], aph, abort_flag, 5, lt)) break;
      if (tid == 0) TC_TRACE(3, lt);
      tc_fence_after();
      // a.b = a_hi.b_hi (columns 0..N-1) + a_hi.b_lo (N..2N-1) + a_lo.b_hi (2N..3N-1)
      const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * 3 * N);
      constexpr int CH = N < 32 ? N : 32;
#pragma unroll
      for (int c = 0; c < N; c += CH) {
        float t1[CH], t2[CH];
        tmem_load<CH>(taddr + c, acc + c);
        tmem_load<CH>(taddr + N + c, t1);
        tmem_load<CH>(taddr + 2 * N + c, t2);
#pragma unroll
        for (int j = 0; j < CH; ++j) acc[c + j] = (t2[j] + t1[j]) + acc[c + j];
      }
      tc_fence_before();
      mbar_arrive(&tempty[ab]);

      if (w < p.U) {
        // m^2 = |a|^2 + |b|^2 - 2 a.b (clamped), K = exp(-lambda m); the
        // query's own word is exactly m = 0 (K = 1); padding columns are 0 and
        // an id outside [0, V) gives NaN
        float kv[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float e = expf(-p.lambda * sqrtf(fmaxf((nw + qn_s[j]) - 2.f * acc[j], 0.f)));
          const int qr = qrow_s[j];
          const float k = qr == (int)w ? 1.f : (qr == -2 ? __int_as_float(0x7fc00000) : e);
          kv[j] = j < p.v_r ? k : 0.f;
        }
        store_row<N>(static_cast<KT*>(p.K) + (size_t)w * p.ldk + p.kcol0, kv, N < p.VR ? N : p.VR);
      }
    }
  }

  if (warp == 0 && lane == 0) TC_TRACE(4, 0);
  tc_fence_before();
  __syncthreads();
  if (tid == 0) TC_TRACE(5, 2);
  if (warp == 9) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kCols);
  }
  if (tid == 0 && *abort_flag) atomicCAS(p.err, 0, *abort_flag);
}

template <int N, int S, int LS>
size_t smem_bytes(int KB) {
  return 1024 + 2 * (size_t)KB * N * 128 + (size_t)(S + LS) * kStageBytes + (3 * S + 5) * 8 +
         N * 8 + 16;
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

template <int N, int S, int LS, typename KT>
cudaError_t launch_t(const wmd_corpus* c, const Params& p, cudaStream_t s) {
  const size_t bytes = smem_bytes<N, S, LS>(p.KB);
  // the shared-memory limit is raised once per device and size (never inside
  // a stream capture: the first launch of a shape always runs eagerly)
  static std::mutex mu;
  static size_t set_bytes[64] = {};
  {
    std::lock_guard<std::mutex> lock(mu);
    const int dev = c->device < 64 ? c->device : 63;
    if (set_bytes[dev] < bytes) {
      cudaError_t e = cudaFuncSetAttribute(cdist_tc_kernel<N, S, LS, KT>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      set_bytes[dev] = bytes;
    }
  }
  const int grid = std::max(1, std::min(p.num_tiles, c->num_sms));
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(c->tmap_vecs);
  cdist_tc_kernel<N, S, LS, KT><<<grid, kThreads, bytes, s>>>(*map, p);
  return cudaGetLastError();
}

}  // namespace tc

bool make_vecs_tensor_map(wmd_corpus* c) {
  auto fn = tc::encode_fn();
  if (!fn) return false;
  static_assert(sizeof(CUtensorMap) <= sizeof(c->tmap_vecs), "tensor map storage");
  CUtensorMap map;
  cuuint64_t dims[2] = {(cuuint64_t)c->ldv, (cuuint64_t)c->V};
  cuuint64_t strides[1] = {(cuuint64_t)c->ldv * sizeof(float)};
  cuuint32_t box[2] = {tc::kKB, tc::kM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->vecs, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  std::memcpy(c->tmap_vecs, &map, sizeof(map));
  return true;
}

// Tensor-core path when the query fits one N <= 64 tile and B stays resident
// in shared memory; returns cudaErrorNotSupported otherwise.
cudaError_t launch_cdist_tc(const wmd_corpus* c, const int32_t* q_ids, const float* q_w, int v_r,
                            int VR, float lambda, wmd_precision prec, void* K, int ldk, int kcol0,
                            float* r_out, float* lam_out, int* err, cudaStream_t s) {
  if (!c->tmap_ok || VR > 64 || c->U == 0) return cudaErrorNotSupported;
  tc::Params p;
  p.vecs = c->vecs;
  p.ldv = c->ldv;
  p.norms = c->norms;
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
  p.KB = (c->ldv + tc::kKB - 1) / tc::kKB;
  p.err = err;
  const bool bf = prec == WMD_PREC_BF16_K;
  const size_t limit = 232448;
  if (VR <= 16) {
    if (tc::smem_bytes<16, 8, 3>(p.KB) > limit) return cudaErrorNotSupported;
    return bf ? tc::launch_t<16, 8, 3, __nv_bfloat16>(c, p, s) : tc::launch_t<16, 8, 3, float>(c, p, s);
  }
  if (VR <= 32) {
    if (tc::smem_bytes<32, 6, 3>(p.KB) > limit) return cudaErrorNotSupported;
    return bf ? tc::launch_t<32, 6, 3, __nv_bfloat16>(c, p, s) : tc::launch_t<32, 6, 3, float>(c, p, s);
  }
  if (tc::smem_bytes<64, 3, 1>(p.KB) > limit) return cudaErrorNotSupported;
  return bf ? tc::launch_t<64, 3, 1, __nv_bfloat16>(c, p, s) : tc::launch_t<64, 3, 1, float>(c, p, s);
}

}  // namespace wmd

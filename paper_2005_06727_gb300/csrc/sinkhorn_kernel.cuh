// The fused Sinkhorn-Knopp loop kernel (K2 + K3), shared by the translation
// units that instantiate it: sinkhorn.cu (a fixed number of loop bodies, the
// form of Sec. 3) and sinkhorn_conv.cu (Algorithm 1's "while x changes", tested
// per document).  Everything here lives in an anonymous namespace, so each
// unit compiles its own instances.
//
// Algorithm 1 iterates x = diag(1/r) K (c .* (1 ./ (K^T (1./x)))).  Sec. 3
// replaces the dense K^T u by an SDDMM evaluated only at the nonzeros of c and
// forms x with an SpMM; its SDDMM_SpMM kernel fuses the two so that v is
// consumed as soon as it is produced.  Here the fusion goes one step further:
// every column j of x, u and v depends only on column j of c, so one team of
// warps owns one document for the whole solve.  It gathers the document's
// block K[w, :] (n_j rows of the word-major K) once, keeps it in registers
// for all max_iter + 1 SDDMMs and max_iter SpMMs, and finishes with the
// reduction WMD_j = sum_i u_ij ((K .* M) v)_ij.  v, x and u never reach
// global memory; nothing is shared between documents, so no atomics are
// needed (the paper's nnz-balanced partition avoids them the same way).
//
// Register tile of one lane: R rows (document words) x C columns (query
// words).  Lane = pw * PI + pi: the PI lanes of a row group split the row's
// columns, the PW = 32 / PI row groups split the rows (SpMM
// partial sums are finished column by column through shared memory for
// one-warp teams of queries up to 32 wide, else with PW-lane butterflies and,
// for teams of several warps, across the warps through shared memory; the
// lane that finishes a column also forms its u = r / x once).  Column j of
// lane pi is c(j) = (j / 4) * 4 PI + 4 pi + j % 4, so one float4 load per 4
// columns reads 16 PI contiguous bytes of a row.
//
// The SDDMM row sums end in a reduce-scatter instead of a full butterfly, so
// that fewer reciprocals are computed twice.  A butterfly over the high bits
// of pi (xor PX, 2 PX, ... below PI) comes first; then the PX lanes p that
// differ in the low bits of pi hold the group's R rows in slots
// (d, k), d < PX, k < R / PX, slot (d, k) of lane p holding row
// ((p ^ d) R / PX + k).  A shuffle with lane p ^ d then brings lane p the
// partial sums of its own rows (d = 0), so PX - 1 shuffles per own row
// finish the sums, each lane forms v = c / s for its R / PX own rows only,
// and the same xor pattern hands every lane the v of its other slots (an
// all-gather).  K rows are gathered in plain row order (the PI lanes of a row
// group read one row together) and then moved to their slots inside each
// lane with log2(PX) levels of conditional swaps.  PX is 4 for 64-wide
// queries and 2 otherwise, as timed: four lanes save more shuffles and
// reciprocals but need R in steps of 4, which costs more padding rows than it
// saves for the 32-, 128- and 256-wide tiles (and ties at 16); one lane (the
// full butterfly) was slower for every width.
//
// The kernel is launched as a programmatic dependent of the cdist kernel: a
// warp reads its task record and its rows' word ids and weights (corpus data,
// which cdist prefetched into L2) and only then waits for cdist's K, r,
// lambda and error slots.
//
// K .* M for the final step is recovered from the K block already in
// registers: M = -ln(K) / lambda = -log2(K) ln 2 / lambda, exact for K = 1
// (the query's own word) and within a few float32 ulps of m while K is a
// normal float (the cdist kernel computed K = exp(-lambda m) in float32, so
// -ln K returns lambda m up to the rounding of that product and of expf).
#pragma once

#include <mutex>

#include "wmd_internal.h"

namespace wmd {
namespace {

struct LoopParams {
  const int64_t* doc_ptr;
  const int32_t* doc_words;
  const float* doc_vals;
  const void* K;
  int ldk;
  int kcol0;
  const float* r;
  const float* lam;  // lambda of the single query, then the double -ln 2 / lambda at
                     // lam + 2 (both written by the cdist kernel)
  int v_r;
  int T;
  const WarpTask* tasks;  // [item][warp]
  double* out;
  const int* err;  // the query's error slots, one per cdist CTA (a wait ran out,
  int n_err;       // or K left the float32 range): if any is set, every result is
                   // NaN.  Batched launches do not read them: the host turns a
                   // failed query of a batch into NaN results and an error.
  int* err_out;    // optional summary of the slots for the host (warp 0 of block 0)
  const QueryDesc* queries;  // blockIdx.y selects the query; NULL: the fields above
  // convergence-tested instances (CONV) only, single query: a document stops
  // once x changes by at most tol relative to its previous value, and
  // iters[doc] (optional) receives the loop bodies it ran
  float tol;
  int32_t* iters;
};

// K is written by the cdist kernel, which may still be running when this
// kernel starts (programmatic dependent launch), so K is not read-only for
// this kernel's lifetime: no __ldg / ld.global.nc, which the compiler may
// schedule above griddepcontrol.wait.  These loads are volatile asm, kept in
// program order with the wait (itself volatile asm).
__device__ __forceinline__ float4 ld_k4(const float4* a) {
  float4 v;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a));
  return v;
}
__device__ __forceinline__ uint2 ld_k2(const uint2* a) {
  uint2 v;
  asm volatile("ld.global.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(a));
  return v;
}

// Loads the C columns of K row `row` that lane pi owns, as C/2 float2 pairs.
template <typename KT, int C, int PI>
__device__ __forceinline__ void load_krow(const KT* Kb, int64_t row, int ldk,
                                          int kcol0, int pi, float2 (&dst)[C / 2]) {
  if constexpr (sizeof(KT) == 4) {
    const float4* src =
        reinterpret_cast<const float4*>(reinterpret_cast<const float*>(Kb) + row * ldk + kcol0);
#pragma unroll
    for (int g = 0; g < C / 4; ++g) {
      const float4 t = ld_k4(src + g * PI + pi);
      dst[2 * g + 0] = make_float2(t.x, t.y);
      dst[2 * g + 1] = make_float2(t.z, t.w);
    }
  } else {
    const uint2* src = reinterpret_cast<const uint2*>(
        reinterpret_cast<const __nv_bfloat16*>(Kb) + row * ldk + kcol0);
#pragma unroll
    for (int g = 0; g < C / 4; ++g) {
      const uint2 t = ld_k2(src + g * PI + pi);
      dst[2 * g + 0] = make_float2(__uint_as_float(t.x << 16), __uint_as_float(t.x & 0xffff0000u));
      dst[2 * g + 1] = make_float2(__uint_as_float(t.y << 16), __uint_as_float(t.y & 0xffff0000u));
    }
  }
}

// OR of a query's error slots (one per cdist CTA, written by every CTA at
// its end, so nothing clears them before a query), read by a whole warp.
// Eight loads per lane are issued before any is used, so that up to 256
// slots (every single-launch query) cost one trip to L2, not one per slot.
__device__ __forceinline__ int read_errors(const int* err, int n, int lane) {
  int v = 0;
  for (int base = lane; base < n; base += 256) {
    int w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = base + 32 * k < n ? err[base + 32 * k] : 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) v |= w[k];
  }
  return __reduce_or_sync(0xffffffffu, v);
}

// Programmatic dependent launch: the kernel may start while the cdist
// kernel before it in the stream still runs; from this wait on, everything
// that kernel wrote (K, r, lambda, the error slots) is visible.  A no-op when
// the launch has no programmatic predecessor.
__device__ __forceinline__ void wait_for_producer() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void team_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// The same barrier, returning whether `pred` held for any of its threads
// (PTX bar.red.or.pred).
__device__ __forceinline__ bool team_barrier_any(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, %2, %3, pi;\n\t"
      "selp.u32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Whether a column's u still moves: |u' - u| > tol u'.  With u = r / x this is
// |x' - x| > tol x, the relative change of x against its previous value; NaN
// counts as moving.
__device__ __forceinline__ bool still_moving(float un, float uo, float tol) {
  return !(fabsf(un - uo) <= tol * un);
}

// Hardware base-2 logarithm (PTX lg2.approx.ftz) of a normal float.
__device__ __forceinline__ float fast_log2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// K log2 K = -lambda K M / ln 2 for two entries of K.  K below the smallest
// normal float is clamped there, so that the logarithm needs no subnormal
// handling and the term stays finite (and below 1.5e-36 in magnitude).
__device__ __forceinline__ float2 k_log2k(float2 k) {
  // opaque to the compiler, so that the logarithms stay in the last pass
  // instead of being hoisted out of the iterations (96 live values per lane
  // would not fit in registers)
  asm volatile("" : "+f"(k.x), "+f"(k.y));
  const float2 l = make_float2(fast_log2(fmaxf(k.x, 1.17549435e-38f)), fast_log2(fmaxf(k.y, 1.17549435e-38f)));
  return __fmul2_rn(k, l);
}


// Knuth's TwoSum: s + e == a + b exactly (s = fl(a + b)).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Hardware reciprocal (PTX rcp.approx, about 1 ulp); operands here are never
// zero: padding rows and columns are seeded so that their sums stay positive.
__device__ __forceinline__ float fast_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Row stride (floats) of the per-warp partial sums of x in shared memory.  A
// quarter warp (8 / PI row groups pw of PI lanes pi) stores 16 bytes per lane
// at column 4 PI h + 4 pi, i.e. 16-byte piece pw S/4 + PI h + pi of the
// buffer: a stride S with S/4 = PI (mod 8) puts the eight pieces on distinct
// banks.
__host__ __device__ constexpr int wpart_stride(int VR, int PI) {
  int s4 = VR / 4;
  while (s4 % 8 != PI % 8) ++s4;
  return 4 * s4;
}

// Lanes of the SDDMM reduce-scatter for a query tile VR wide (1 would be the
// plain butterfly over all PI lanes).
__host__ __device__ constexpr int scatter_lanes(int VR) { return VR == 64 ? 4 : 2; }

// Moves the K rows of a lane from plain order (slot d holds row group rows
// d RK .. d RK + RK - 1) to the reduce-scatter order (slot d holds those of
// d ^ px): one level of conditional swaps per bit of px.
template <int R, int PX, int C2>
__device__ __forceinline__ void permute_slots(float2 (&kt)[R][C2], int px) {
  constexpr int RK = R / PX;
#pragma unroll
  for (int b = 1; b < PX; b <<= 1) {
    const bool f = (px & b) != 0;
#pragma unroll
    for (int d = 0; d < PX; ++d) {
      if (d & b) continue;
#pragma unroll
      for (int k = 0; k < RK; ++k) {
#pragma unroll
        for (int q = 0; q < C2; ++q) {
          const float2 a = kt[d * RK + k][q], c = kt[(d | b) * RK + k][q];
          kt[d * RK + k][q] = f ? c : a;
          kt[(d | b) * RK + k][q] = f ? a : c;
        }
      }
    }
  }
}

struct TeamCtx {
  int doc;
  int64_t beg;
  int n;
  int W;
  int kw;
  int team;
  int warp;
  int lane;
  int pi;
  int pw;
  QueryDesc q;  // the query this CTA works for (q.lambda: batched launches only)
  int rpw_res;  // rows per warp when the document is register resident
  int nch;      // chunks this warp handles
  float* red;   // [NW][VR] partial x of every warp, then [NW / 2][VR] u of every team
  double* wred; // [NW] partial WMD of every warp of the CTA
  float* wpart; // [NW][PW + 1][wpart_stride] per warp: row-group partial x, then u
  int nw;       // warps in the CTA
};

// The whole solve of one document by one team, with R rows per lane known at
// compile time (no per-row guards, so every phase is one straight-line block).
// RELOAD: the document is longer than the team's registers; each pass re-reads
// its chunks of K (from L2) instead of keeping them resident.
// CONV: the loop stops early once x has stopped changing (Algorithm 1's "while
// x changes", tested per document after every body: all columns must satisfy
// |x' - x| <= tol x), and the team writes the number of bodies it ran.
template <int VR, int PI, int R, bool RELOAD, bool CONV, typename KT>
__device__ __forceinline__ void solve(const LoopParams& p, const TeamCtx& t) {
  constexpr int C = VR / PI;
  constexpr int C2 = C / 2;
  constexpr int PW = 32 / PI;
  constexpr int PX = scatter_lanes(VR);  // lanes of the row-sum reduce-scatter
  constexpr int RK = R / PX;             // rows whose sums a lane finishes
  static_assert(R % PX == 0, "rows per lane must split over the reduce-scatter lanes");
  const KT* Kb = static_cast<const KT*>(p.K);
  const int px = t.pi & (PX - 1);
  // row of slot rI within the warp's chunk: slot (d, k) = (rI / RK, rI % RK)
  // holds the group's row (px ^ d) RK + k; K is gathered in plain order (row
  // rI PW + pw into slot rI) and permuted afterwards
  auto slot_row = [&](int rI) { return ((px ^ (rI / RK)) * RK + rI % RK) * PW + t.pw; };
  auto plain_row = [&](int rI) { return rI * PW + t.pw; };
  // first column of float2 pair q of this lane
  auto lane_col = [&](int q) { return (q >> 1) * 4 * PI + 4 * t.pi + 2 * (q & 1); };

  // corpus data first (the previous kernel does not write it): the word ids
  // and weights of my rows, then wait for that kernel's K and r
  float cw[R];
  int wrow[R];
  if (!RELOAD && t.nch) {
    const int start = t.kw * t.rpw_res;
    const int len = min(t.rpw_res, t.n - start);
#pragma unroll
    for (int rI = 0; rI < R; ++rI) {
      const int srow = slot_row(rI), prow = plain_row(rI);
      cw[rI] = srow < len ? p.doc_vals[t.beg + start + srow] : 0.f;
      wrow[rI] = prow < len ? p.doc_words[t.beg + start + prow] : -1;
    }
  }
  wait_for_producer();
  // the cdist kernel gave up waiting, or K left the float32 range: no result
  // (whole teams leave together).  The resident path reads the error slots
  // after it has issued its K gathers, so that both share one trip to L2.
  auto failed = [&]() {
    if (p.queries || !read_errors(p.err, p.n_err, t.lane)) return false;
    if (t.kw == 0 && t.lane == 0) {
      t.q.out[t.doc] = __longlong_as_double(0x7ff8000000000000ll);
      if (CONV && p.iters) p.iters[t.doc] = p.T;
    }
    return true;
  };
  if ((RELOAD || !t.nch) && failed()) return;

  // query weights and the initial u = 1 / x = v_r for my columns; one lane
  // per column seeds the SpMM sums of padding columns with 1 so that 1/x stays
  // finite there (their r is 0, so u = r / x = 0, and K = 0 keeps them out of
  // every sum); bit 2q+h of `seed` marks those columns
  // narrow queries finish x through shared memory (below: one-warp teams
  // entirely, teams of several warps within each warp); wider ones keep the
  // query weights of their columns in registers
  constexpr bool kSmemFinish = VR <= 32;
  float2 rr[C2], u[C2];
  uint32_t seed = 0;
#pragma unroll
  for (int q = 0; q < C2; ++q) {
    const int col = lane_col(q);
    const bool l0 = col < t.q.v_r, l1 = col + 1 < t.q.v_r;
    if (!kSmemFinish) rr[q] = make_float2(l0 ? t.q.r[col] : 0.f, l1 ? t.q.r[col + 1] : 0.f);
    u[q] = make_float2(l0 ? (float)t.q.v_r : 0.f, l1 ? (float)t.q.v_r : 0.f);
    if (t.pw == 0 && t.kw == 0) seed |= (l0 ? 0u : 1u) << (2 * q) | (l1 ? 0u : 1u) << (2 * q + 1);
  }

  float2 kt[R][C2];
  // long documents (RELOAD): chunk m of this warp, re-read from L2 each pass
  auto load_chunk = [&](int m) {
    const int start = (m * t.W + t.kw) * (PW * R);
    const int len = min(PW * R, t.n - start);
#pragma unroll
    for (int rI = 0; rI < R; ++rI) {
      const int srow = slot_row(rI), prow = plain_row(rI);
      cw[rI] = srow < len ? p.doc_vals[t.beg + start + srow] : 0.f;
      if (prow < len) {
        load_krow<KT, C, PI>(Kb, p.doc_words[t.beg + start + prow], p.ldk, t.q.kcol0, t.pi, kt[rI]);
      } else {
        // padding row: c = 0 gives v = 0, and K = 1 keeps s > 0 so that
        // c / s needs no guard
#pragma unroll
        for (int q = 0; q < C2; ++q) kt[rI][q] = make_float2(1.f, 1.f);
      }
    }
    permute_slots<R, PX, C2>(kt, px);
  };
  if (!RELOAD && t.nch) {
    // K rows of the resident block; padding rows: c = 0 gives v = 0, and
    // K = 1 keeps s > 0 so that c / s needs no guard
#pragma unroll
    for (int rI = 0; rI < R; ++rI) {
      if (wrow[rI] >= 0) {
        load_krow<KT, C, PI>(Kb, wrow[rI], p.ldk, t.q.kcol0, t.pi, kt[rI]);
      } else {
#pragma unroll
        for (int q = 0; q < C2; ++q) kt[rI][q] = make_float2(1.f, 1.f);
      }
    }
    if (failed()) return;
    permute_slots<R, PX, C2>(kt, px);
  }

  // u is finished column by column: lane tl of the team (of the warp for
  // one-warp teams of narrow queries) owns columns tl, tl + 32 W, ... (at
  // most kLaneCols of them: teams of several warps have W >= 2, and queries
  // above 32 wide finish one-warp teams in registers)
  constexpr int kLaneCols = (VR + 63) / 64;
  const int tl = t.kw * 32 + t.lane;
  float* red = t.red;                        // [NW][VR] partial x of every warp
  float* ured = t.red + t.nw * VR + t.team * VR;  // u of this team
  // [PW][kWS] partial x of the warp's row groups, then [VR] u of a one-warp
  // team; rows padded so that a quarter warp's 16-byte stores hit distinct banks
  constexpr int kWS = wpart_stride(VR, PI);
  float* wpart = t.wpart + t.warp * (PW + 1) * kWS;
  float* wu = wpart + PW * kWS;
  float rcol[kLaneCols];
  float uold[kLaneCols];  // CONV: u of those columns before the current body
#pragma unroll
  for (int j = 0; j < kLaneCols; ++j) {
    const int col = tl + j * 32 * t.W;
    rcol[j] = col < t.q.v_r ? t.q.r[col] : 0.f;
    uold[j] = col < t.q.v_r ? (float)t.q.v_r : 0.f;
  }
  float wacc = 0.f;
  bool done = false;  // CONV: x stopped changing (the whole team agrees)
  int it = 0;
  for (; it <= p.T; ++it) {
    const bool last = it == p.T || (CONV && done);
    float2 xp[C2];
#pragma unroll
    for (int q = 0; q < C2; ++q)
      xp[q] = make_float2((seed >> (2 * q)) & 1u ? 1.f : 0.f, (seed >> (2 * q + 1)) & 1u ? 1.f : 0.f);

    for (int m = 0; m < t.nch; ++m) {
      if (RELOAD) load_chunk(m);
      // SDDMM: s_w = sum_i K[w, i] u_i, my columns then the PI lanes of the row
      float s[R];
#pragma unroll
      for (int rI = 0; rI < R; ++rI) {
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < C2; ++q) a = __ffma2_rn(kt[rI][q], u[q], a);
        s[rI] = a.x + a.y;
      }
#pragma unroll
      for (int off = PX; off < PI; off <<= 1) {
#pragma unroll
        for (int rI = 0; rI < R; ++rI) s[rI] += __shfl_xor_sync(0xffffffffu, s[rI], off);
      }
      // reduce-scatter over the PX lanes: lane px ^ d holds my row k in its
      // slot (d, k); v_w = c_w / s_w for my RK rows (padding rows carry c = 0
      // and give v = 0), then the all-gather of the other slots' v
      float v[R];
#pragma unroll
      for (int k = 0; k < RK; ++k) {
        float sk = s[k];
#pragma unroll
        for (int d = 1; d < PX; ++d) sk += __shfl_xor_sync(0xffffffffu, s[d * RK + k], d);
        v[k] = cw[k] * fast_rcp(sk);
      }
#pragma unroll
      for (int d = 1; d < PX; ++d) {
#pragma unroll
        for (int k = 0; k < RK; ++k) v[d * RK + k] = __shfl_xor_sync(0xffffffffu, v[k], d);
      }

      if (!last) {
        // SpMM: x_i += K[w, i] v_w over my rows
#pragma unroll
        for (int rI = 0; rI < R; ++rI) {
          const float2 vv = make_float2(v[rI], v[rI]);
#pragma unroll
          for (int q = 0; q < C2; ++q) xp[q] = __ffma2_rn(kt[rI][q], vv, xp[q]);
        }
      } else {
        // final reduction: sum_w v_w sum_i u_i K[w, i] log2 K[w, i] (= -lambda /
        // ln 2 times the WMD); a lane's few terms are summed in float32, lanes
        // in double-float and warps in float64
#pragma unroll
        for (int rI = 0; rI < R; ++rI) {
          float2 tt = make_float2(0.f, 0.f);
#pragma unroll
          for (int q = 0; q < C2; ++q) tt = __ffma2_rn(u[q], k_log2k(kt[rI][q]), tt);
          wacc = fmaf(v[rI], tt.x + tt.y, wacc);
        }
      }
    }

    if (kSmemFinish && !last && t.W == 1) {
      // x = sum over the PW row groups of the warp, finished through shared
      // memory: every lane stores its partial sums, lane L sums column L (and
      // L + 32, ...) in fixed row-group order and writes u = r / x, every lane
      // reads back its columns' u
      // (u = 1 / x with x = diag(1/r) (K v):  u_i = r_i / (K v)_i)
#pragma unroll
      for (int h = 0; h < C2 / 2; ++h)
        *reinterpret_cast<float4*>(&wpart[t.pw * kWS + lane_col(2 * h)]) =
            make_float4(xp[2 * h].x, xp[2 * h].y, xp[2 * h + 1].x, xp[2 * h + 1].y);
      __syncwarp();
      bool moving = false;
#pragma unroll
      for (int j = 0; j < kLaneCols; ++j) {
        const int col = t.lane + 32 * j;
        if (col < VR) {
          float x = 0.f;
#pragma unroll
          for (int k2 = 0; k2 < PW; ++k2) x += wpart[k2 * kWS + col];
          const float un = rcol[j] * fast_rcp(x);
          if constexpr (CONV) {
            moving |= still_moving(un, uold[j], p.tol);
            uold[j] = un;
          }
          wu[col] = un;
        }
      }
      __syncwarp();
      if constexpr (CONV) done = !__any_sync(0xffffffffu, moving);
#pragma unroll
      for (int h = 0; h < C2 / 2; ++h) {
        const float4 uu = *reinterpret_cast<const float4*>(&wu[lane_col(2 * h)]);
        u[2 * h] = make_float2(uu.x, uu.y);
        u[2 * h + 1] = make_float2(uu.z, uu.w);
      }
    } else if (!last) {
      // x: sum over the PW row groups of the warp ...
      if constexpr (kSmemFinish) {
        // (teams of several warps, narrow queries) through shared memory, as
        // for one-warp teams: every lane stores its partials, lane L sums
        // column L over the row groups in order and leaves the warp's sum in
        // the team's exchange buffer
#pragma unroll
        for (int h = 0; h < C2 / 2; ++h)
          *reinterpret_cast<float4*>(&wpart[t.pw * kWS + lane_col(2 * h)]) =
              make_float4(xp[2 * h].x, xp[2 * h].y, xp[2 * h + 1].x, xp[2 * h + 1].y);
        __syncwarp();
        if (t.lane < VR) {
          float xs = 0.f;
#pragma unroll
          for (int k2 = 0; k2 < PW; ++k2) xs += wpart[k2 * kWS + t.lane];
          red[t.warp * VR + t.lane] = xs;
        }
      } else {
#pragma unroll
        for (int off = PI; off < 32; off <<= 1) {
#pragma unroll
          for (int q = 0; q < C2; ++q) {
            const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, xp[q].x, off),
                                         __shfl_xor_sync(0xffffffffu, xp[q].y, off));
            xp[q] = __fadd2_rn(xp[q], o);
          }
        }
      }
      // u = 1 / x with x = diag(1/r) (K v):  u_i = r_i / (K v)_i
      if (t.W == 1) {
        bool moving = false;
#pragma unroll
        for (int q = 0; q < C2; ++q) {
          const float2 un = __fmul2_rn(rr[q], make_float2(fast_rcp(xp[q].x), fast_rcp(xp[q].y)));
          if constexpr (CONV)
            moving |= still_moving(un.x, u[q].x, p.tol) || still_moving(un.y, u[q].y, p.tol);
          u[q] = un;
        }
        if constexpr (CONV) done = !__any_sync(0xffffffffu, moving);
      } else {
        // ... and over the warps of the team: each lane of the team finishes
        // whole columns (the team's partial sums in fixed warp order, so
        // deterministic, then u), and every lane reads back its columns' u
        if (!kSmemFinish && t.pw == 0) {
#pragma unroll
          for (int q = 0; q < C2; ++q)
            *reinterpret_cast<float2*>(&red[t.warp * VR + lane_col(q)]) = xp[q];
        }
        team_barrier(1 + t.team, 32 * t.W);
        bool moving = false;
#pragma unroll
        for (int j = 0; j < kLaneCols; ++j) {
          const int col = tl + j * 32 * t.W;
          if (col < VR) {
            float x = 0.f;
            for (int k2 = 0; k2 < t.W; ++k2) x += red[(t.team * t.W + k2) * VR + col];
            const float un = rcol[j] * fast_rcp(x);
            if constexpr (CONV) {
              moving |= still_moving(un, uold[j], p.tol);
              uold[j] = un;
            }
            ured[col] = un;
          }
        }
        if constexpr (CONV) done = !team_barrier_any(1 + t.team, 32 * t.W, moving);
        else team_barrier(1 + t.team, 32 * t.W);
#pragma unroll
        for (int q = 0; q < C2; ++q) u[q] = *reinterpret_cast<const float2*>(&ured[lane_col(q)]);
      }
    }
    if (CONV && last) break;  // stopped early: `it` is the number of bodies run
  }
  if constexpr (CONV) {
    if (p.iters && t.kw == 0 && t.lane == 0) p.iters[t.doc] = it;
  }

  // WMD_j: sum over the lanes of the warp in double-float (hi + lo pairs
  // combined with TwoSum, as accurate as float64 for these 32 terms and
  // without the GPU's slow float64 pipe), then over the team's warps in
  // float64
  float hi = wacc, lo = 0.f;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, off);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, off);
    float sh, se;
    two_sum(hi, h2, sh, se);
    two_sum(sh, se + (lo + l2), hi, lo);
  }
  // (float64 only in lane 0: this GPU's FP64 pipe is narrow).  The factor
  // -ln 2 / lambda was computed once per query outside this kernel (a float64
  // division per document would load that pipe) and is read only here, so
  // that it occupies no registers during the loop.
  auto scale = [&]() {
    return p.queries ? p.queries[blockIdx.y].scale : *reinterpret_cast<const double*>(p.lam + 2);
  };
  if (t.W > 1) {
    if (t.lane == 0) t.wred[t.warp] = (double)hi + (double)lo;
    team_barrier(1 + t.team, 32 * t.W);
    if (t.kw == 0 && t.lane == 0) {
      double acc = 0.0;
      for (int k2 = 0; k2 < t.W; ++k2) acc += t.wred[t.team * t.W + k2];
      t.q.out[t.doc] = acc * scale();
    }
  } else if (t.lane == 0) {
    t.q.out[t.doc] = ((double)hi + (double)lo) * scale();
  }
}

template <int VR, int PI, int RMAX, int MINB, int NW, bool CONV, typename KT>
__global__ void __launch_bounds__(NW * 32, MINB) sinkhorn_fused_kernel(LoopParams p) {
  constexpr int C = VR / PI;
  constexpr int PW = 32 / PI;
  constexpr int RPW = PW * RMAX;
  // resident tiles come in up to 4 row-count steps of about RMAX / 4, each
  // rounded up to a multiple of the reduce-scatter width
  constexpr int PX = scatter_lanes(VR);
  constexpr int R1 = round_up(RMAX / 4, PX), R2 = round_up(RMAX / 2, PX),
                R3 = round_up(3 * RMAX / 4, PX);
  static_assert(C % 4 == 0, "columns per lane must be a multiple of 4");
  static_assert(RMAX % PX == 0, "RMAX must split over the reduce-scatter lanes");

  __shared__ __align__(16) float red[2 * NW * VR];
  __shared__ __align__(16) float wpart[VR <= 32 ? NW * (PW + 1) * wpart_stride(VR, PI) : 4];
  __shared__ double wred[NW];

  // a programmatic dependent of this launch (the top-k selection, or the
  // next width class of a batch) may start once every CTA of this grid has
  // started; it waits for this grid's results itself
  asm volatile("griddepcontrol.launch_dependents;");
  TeamCtx t;
  t.warp = threadIdx.x >> 5;
  t.lane = threadIdx.x & 31;
  t.pi = t.lane % PI;
  t.pw = t.lane / PI;
  if (p.err_out && blockIdx.x == 0 && blockIdx.y == 0 && t.warp == 0) {
    // summary for the host: the first CTA code found, with the range flag
    wait_for_producer();
    int v = 0;
    for (int i = t.lane; i < p.n_err; i += 32) v |= p.err[i];  // one CTA, once: plain loop
    const unsigned nz = __ballot_sync(0xffffffffu, v != 0);
    const int first = __shfl_sync(0xffffffffu, v, nz ? __ffs(nz) - 1 : 0);
    const int range = __reduce_or_sync(0xffffffffu, v) & kRangeFlag;
    if (t.lane == 0) *p.err_out = first | range;
  }
  const WarpTask task = p.tasks[blockIdx.x * NW + t.warp];
  t.W = task.n_w >> kTaskWShift;
  if (t.W == 0) return;  // no team in this item (whole teams leave together)
  t.team = t.warp / t.W;
  t.kw = t.warp - t.team * t.W;
  t.doc = task.doc;
  t.beg = task.beg;
  t.n = task.n_w & ((1 << kTaskWShift) - 1);
  if (p.queries) {
    t.q = p.queries[blockIdx.y];  // written by the host before the cdist kernel
  } else {
    t.q.r = p.r;
    t.q.out = p.out;
    t.q.kcol0 = p.kcol0;
    t.q.v_r = p.v_r;
  }
  if (t.n == 0) {
    wait_for_producer();  // the error slots come from the cdist kernel
    const bool bad = !p.queries && read_errors(p.err, p.n_err, t.lane);
    if (t.kw == 0 && t.lane == 0) {
      t.q.out[t.doc] = bad || p.T >= 1 ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
      // x of an empty document goes 1/v_r -> 0 -> 0/0: it never settles
      if (CONV && p.iters) p.iters[t.doc] = p.T;
    }
    return;
  }
  t.red = red;
  t.wred = wred;
  t.wpart = wpart;
  t.nw = NW;

  if (t.n <= t.W * RPW) {
    // register resident: one chunk of rpw_res rows per warp
    t.rpw_res = (t.n + t.W - 1) / t.W;
    const int start = t.kw * t.rpw_res;
    t.nch = start < t.n ? 1 : 0;
    const int len = t.nch ? min(t.rpw_res, t.n - start) : 0;
    const int reff = (len + PW - 1) / PW;
    if (reff <= R1) solve<VR, PI, R1, false, CONV, KT>(p, t);
    else if (reff <= R2) solve<VR, PI, R2, false, CONV, KT>(p, t);
    else if (reff <= R3) solve<VR, PI, R3, false, CONV, KT>(p, t);
    else solve<VR, PI, RMAX, false, CONV, KT>(p, t);
  } else {
    t.rpw_res = 0;
    const int nchunks_total = (t.n + RPW - 1) / RPW;
    t.nch = max(0, (nchunks_total - t.kw + t.W - 1) / t.W);
    solve<VR, PI, RMAX, true, CONV, KT>(p, t);
  }
}

// Tile variants per width class: {VR, PI, RMAX, CTAs per SM, warps per CTA}.
// RMAX * (VR / PI) floats of K per lane; the variants trade register tile
// size (work per cross-lane reduction) against resident warps (latency
// hiding), and wide queries use 8-warp CTAs so that a team of up to 8 warps
// keeps a long document's K block resident.  Two lanes per row (no butterfly
// before the reduce-scatter) pay off for 16-wide queries but not for 32-wide
// ones (RMAX 6: 2.54 against 2.16 us per iteration).  The 48-, 96- and
// 192-wide classes have 12 columns per lane (4, 8 and 16 lanes per row), so
// that a query just above a power of two does not pay for a quarter of
// padding columns; the 96-wide one also runs as three 4-warp CTAs per SM,
// whose K block is as large as the 64-wide class's.  (A 24-wide tile, two
// lanes per row, was slower than the 32-wide one for 19-word queries.)  The autotuner (wmd_autotune) picks one per class and
// precision by timing.
template <int CLS, int V> struct Var;
template <> struct Var<0, 0> { static constexpr int VR = 8, PI = 2, RMAX = 12, MINB = 4, NW = 4; };
template <> struct Var<0, 1> { static constexpr int VR = 8, PI = 2, RMAX = 24, MINB = 2, NW = 4; };
template <> struct Var<1, 0> { static constexpr int VR = 16, PI = 4, RMAX = 24, MINB = 3, NW = 4; };
template <> struct Var<1, 1> { static constexpr int VR = 16, PI = 2, RMAX = 12, MINB = 3, NW = 4; };
template <> struct Var<2, 0> { static constexpr int VR = 32, PI = 4, RMAX = 12, MINB = 3, NW = 4; };
template <> struct Var<2, 1> { static constexpr int VR = 32, PI = 4, RMAX = 8, MINB = 4, NW = 4; };
template <> struct Var<3, 0> { static constexpr int VR = 48, PI = 4, RMAX = 8, MINB = 3, NW = 4; };
template <> struct Var<3, 1> { static constexpr int VR = 48, PI = 4, RMAX = 4, MINB = 4, NW = 4; };
template <> struct Var<4, 0> { static constexpr int VR = 64, PI = 8, RMAX = 12, MINB = 3, NW = 4; };
template <> struct Var<4, 1> { static constexpr int VR = 64, PI = 8, RMAX = 8, MINB = 4, NW = 4; };
template <> struct Var<5, 0> { static constexpr int VR = 96, PI = 8, RMAX = 8, MINB = 1, NW = 8; };
template <> struct Var<5, 1> { static constexpr int VR = 96, PI = 8, RMAX = 8, MINB = 3, NW = 4; };
template <> struct Var<6, 0> { static constexpr int VR = 128, PI = 8, RMAX = 8, MINB = 1, NW = 8; };
template <> struct Var<6, 1> { static constexpr int VR = 128, PI = 8, RMAX = 8, MINB = 2, NW = 4; };
template <> struct Var<7, 0> { static constexpr int VR = 192, PI = 16, RMAX = 8, MINB = 1, NW = 8; };
template <> struct Var<7, 1> { static constexpr int VR = 192, PI = 16, RMAX = 8, MINB = 2, NW = 4; };
template <> struct Var<8, 0> { static constexpr int VR = 256, PI = 16, RMAX = 8, MINB = 1, NW = 8; };
template <> struct Var<8, 1> { static constexpr int VR = 256, PI = 16, RMAX = 8, MINB = 2, NW = 4; };

template <int CLS, int V, bool CONV, typename KT>
cudaError_t launch_var(const LoopParams& p, int n_items, int nq, cudaStream_t s) {
  using Cf = Var<CLS, V>;
  auto kern = sinkhorn_fused_kernel<Cf::VR, Cf::PI, Cf::RMAX, Cf::MINB, Cf::NW, CONV, KT>;
  if (n_items == 0 || nq == 0) return cudaSuccess;
  // the same shared-memory carveout as the cdist kernel, so that the first
  // CTAs can share SMs with it (once per device, never inside a capture: the
  // first launch of a shape always runs eagerly)
  static std::mutex mu;
  static bool set_on[64] = {};
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    dev = dev < 64 ? dev : 63;
    std::lock_guard<std::mutex> lock(mu);
    if (!set_on[dev]) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                 (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      set_on[dev] = true;
    }
  }
  // programmatic dependent launch: CTAs may start while the kernel before
  // them (the cdist kernel) finishes; they wait for its results in solve()
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n_items, (unsigned)nq);
  cfg.blockDim = dim3(Cf::NW * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int CLS, bool CONV, typename KT>
cudaError_t launch_cls(int var, const LoopParams& p, int n_items, int nq, cudaStream_t s) {
  if constexpr (kClassVariants[CLS] > 2) {
    if (var == 2) return launch_var<CLS, 2, CONV, KT>(p, n_items, nq, s);
  }
  return var ? launch_var<CLS, 1, CONV, KT>(p, n_items, nq, s)
             : launch_var<CLS, 0, CONV, KT>(p, n_items, nq, s);
}

template <bool CONV, typename KT>
cudaError_t dispatch_loop(int cls, int var, const LoopParams& p, int n_items, int nq,
                          cudaStream_t s) {
  switch (cls) {
    case 0: return launch_cls<0, CONV, KT>(var, p, n_items, nq, s);
    case 1: return launch_cls<1, CONV, KT>(var, p, n_items, nq, s);
    case 2: return launch_cls<2, CONV, KT>(var, p, n_items, nq, s);
    case 3: return launch_cls<3, CONV, KT>(var, p, n_items, nq, s);
    case 4: return launch_cls<4, CONV, KT>(var, p, n_items, nq, s);
    case 5: return launch_cls<5, CONV, KT>(var, p, n_items, nq, s);
    case 6: return launch_cls<6, CONV, KT>(var, p, n_items, nq, s);
    case 7: return launch_cls<7, CONV, KT>(var, p, n_items, nq, s);
    default: return launch_cls<8, CONV, KT>(var, p, n_items, nq, s);
  }
}

// Parameters shared by every launch of the loop for query class cls.
inline LoopParams base_params(const wmd_corpus* c, int cls, int var, const void* K, int ldk,
                              int T, const int* err, int n_err) {
  LoopParams p;
  p.doc_ptr = c->doc_ptr;
  p.doc_words = c->doc_words;
  p.doc_vals = c->doc_vals;
  p.K = K;
  p.ldk = ldk;
  p.kcol0 = 0;
  p.r = nullptr;
  p.lam = nullptr;
  p.v_r = 0;
  p.T = T;
  p.tasks = c->sched[cls][var].d_tasks;
  p.out = nullptr;
  p.err = err;
  p.n_err = n_err;
  p.err_out = nullptr;
  p.queries = nullptr;
  p.tol = 0.f;
  p.iters = nullptr;
  return p;
}

}  // namespace
}  // namespace wmd

// K2 + K3: the fused Sinkhorn-Knopp loop and the final WMD reduction.
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
// Register tile of one lane: RMAX rows (document words) x C columns (query
// words).  Lane = pw * PI + pi: the PI lanes of a row group split the row's
// columns (SDDMM partial dots are combined with PI-lane butterflies), the
// PW = 32 / PI row groups split the rows (SpMM partial sums are combined with
// PW-lane butterflies and, for teams of several warps, through shared memory).
// Column j of lane pi is c(j) = (j / 4) * 4 PI + 4 pi + j % 4, so one float4
// load per 4 columns reads 16 PI contiguous bytes per row group.
//
// K .* M for the final step is recovered from K itself: M = -ln(K) / lambda,
// exact for K = 1 (the query's own word) and within a few float32 ulps while
// K is a normal float.
#include <cfloat>

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
  int v_r;
  int T;
  double inv_lambda;
  const LoopItem* items;
  const int32_t* order;
  double* out;
};

template <typename KT, int C, int PI>
__device__ __forceinline__ void load_krow(const KT* __restrict__ Kb, int64_t row, int ldk,
                                          int kcol0, int pi, float (&dst)[C]) {
  if constexpr (sizeof(KT) == 4) {
    const float4* src =
        reinterpret_cast<const float4*>(reinterpret_cast<const float*>(Kb) + row * ldk + kcol0);
#pragma unroll
    for (int g = 0; g < C / 4; ++g) {
      const float4 t = __ldg(src + g * PI + pi);
      dst[4 * g + 0] = t.x;
      dst[4 * g + 1] = t.y;
      dst[4 * g + 2] = t.z;
      dst[4 * g + 3] = t.w;
    }
  } else {
    const uint2* src = reinterpret_cast<const uint2*>(
        reinterpret_cast<const __nv_bfloat16*>(Kb) + row * ldk + kcol0);
#pragma unroll
    for (int g = 0; g < C / 4; ++g) {
      const uint2 t = __ldg(src + g * PI + pi);
      dst[4 * g + 0] = __uint_as_float(t.x << 16);
      dst[4 * g + 1] = __uint_as_float(t.x & 0xffff0000u);
      dst[4 * g + 2] = __uint_as_float(t.y << 16);
      dst[4 * g + 3] = __uint_as_float(t.y & 0xffff0000u);
    }
  }
}

__device__ __forceinline__ void team_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int VR, int PI, int RMAX, typename KT>
__global__ void __launch_bounds__(128, 2) sinkhorn_fused_kernel(LoopParams p) {
  constexpr int C = VR / PI;
  constexpr int PW = 32 / PI;
  constexpr int RPW = PW * RMAX;
  static_assert(C % 4 == 0, "columns per lane must be a multiple of 4");

  __shared__ float red[2][4][VR];
  __shared__ double wred[4];

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int pi = lane % PI;
  const int pw = lane / PI;
  const LoopItem item = p.items[blockIdx.x];
  const int W = item.W;
  const int team = warp / W;
  const int kw = warp - team * W;  // warp index inside the team
  const int slot = item.begin + team;
  if (team >= 4 / W || slot >= item.end) return;  // whole team leaves together

  const int doc = p.order[slot];
  const int64_t beg = p.doc_ptr[doc];
  const int n = (int)(p.doc_ptr[doc + 1] - beg);
  if (n == 0) {
    if (kw == 0 && lane == 0) p.out[doc] = p.T >= 1 ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
    return;
  }
  const KT* Kb = static_cast<const KT*>(p.K);

  // rows of this warp: one resident chunk, or several chunks re-read per pass
  const bool resident = n <= W * RPW;
  int rpw_res = (n + W - 1) / W;
  int nch;
  if (resident) {
    nch = (kw * rpw_res < n) ? 1 : 0;
  } else {
    const int nchunks_total = (n + RPW - 1) / RPW;
    nch = (nchunks_total - kw + W - 1) / W;
    if (nch < 0) nch = 0;
  }

  // query weights and the initial u = 1 / x = v_r for my columns
  float rr[C], u[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int col = (j >> 2) * 4 * PI + 4 * pi + (j & 3);
    const bool live = col < p.v_r;
    rr[j] = live ? p.r[col] : 0.f;
    u[j] = live ? (float)p.v_r : 0.f;
  }

  float kt[RMAX][C];
  float cw[RMAX];
  int reff = 0;  // rows of the current chunk held by each row group

  auto load_chunk = [&](int m) {
    int start, len;
    if (resident) {
      start = kw * rpw_res;
      len = min(rpw_res, n - start);
    } else {
      start = (m * W + kw) * RPW;
      len = min(RPW, n - start);
    }
    reff = (len + PW - 1) / PW;
#pragma unroll
    for (int rI = 0; rI < RMAX; ++rI) {
      const int row = rI * PW + pw;
      if (rI < reff && row < len) {
        const int64_t e = beg + start + row;
        const int wrow = p.doc_words[e];
        cw[rI] = p.doc_vals[e];
        load_krow<KT, C, PI>(Kb, wrow, p.ldk, p.kcol0, pi, kt[rI]);
      } else {
        cw[rI] = 0.f;
#pragma unroll
        for (int j = 0; j < C; ++j) kt[rI][j] = 0.f;
      }
    }
  };

  if (resident && nch) load_chunk(0);

  int buf = 0;
  double wacc = 0.0;
  for (int it = 0; it <= p.T; ++it) {
    const bool last = it == p.T;
    float xp[C];
#pragma unroll
    for (int j = 0; j < C; ++j) xp[j] = 0.f;

    for (int m = 0; m < nch; ++m) {
      if (!resident) load_chunk(m);
      // SDDMM: s_w = sum_i K[w, i] u_i over my columns, then over the PI lanes
      float s[RMAX];
#pragma unroll
      for (int rI = 0; rI < RMAX; ++rI) {
        if (rI < reff) {
          float a0 = 0.f, a1 = 0.f;
#pragma unroll
          for (int j = 0; j < C; j += 2) {
            a0 = fmaf(kt[rI][j], u[j], a0);
            a1 = fmaf(kt[rI][j + 1], u[j + 1], a1);
          }
          s[rI] = a0 + a1;
        }
      }
#pragma unroll
      for (int off = 1; off < PI; off <<= 1) {
#pragma unroll
        for (int rI = 0; rI < RMAX; ++rI)
          if (rI < reff) s[rI] += __shfl_xor_sync(0xffffffffu, s[rI], off);
      }
      // v_w = c_w / s_w (rows past the document end carry c = 0, v = 0)
      float v[RMAX];
#pragma unroll
      for (int rI = 0; rI < RMAX; ++rI)
        v[rI] = (rI < reff && cw[rI] > 0.f) ? __fdividef(cw[rI], s[rI]) : 0.f;

      if (!last) {
        // SpMM: x_i += K[w, i] v_w over my rows
#pragma unroll
        for (int rI = 0; rI < RMAX; ++rI) {
          if (rI < reff) {
#pragma unroll
            for (int j = 0; j < C; ++j) xp[j] = fmaf(kt[rI][j], v[rI], xp[j]);
          }
        }
      } else {
        // final reduction: sum_w v_w sum_i u_i K[w,i] M[w,i], M = -ln(K)/lambda
#pragma unroll
        for (int rI = 0; rI < RMAX; ++rI) {
          if (rI < reff) {
            float t = 0.f;
#pragma unroll
            for (int j = 0; j < C; ++j) {
              const float kk = kt[rI][j];
              const float km = kk >= FLT_MIN ? -kk * __logf(kk) : 0.f;
              t = fmaf(u[j], km, t);
            }
            wacc += (double)v[rI] * (double)t;
          }
        }
      }
    }

    if (!last) {
      // x: sum over the PW row groups of this warp ...
#pragma unroll
      for (int off = PI; off < 32; off <<= 1) {
#pragma unroll
        for (int j = 0; j < C; ++j) xp[j] += __shfl_xor_sync(0xffffffffu, xp[j], off);
      }
      // ... and over the warps of the team
      if (W > 1) {
        if (pw == 0) {
#pragma unroll
          for (int j = 0; j < C; ++j) {
            const int col = (j >> 2) * 4 * PI + 4 * pi + (j & 3);
            red[buf][warp][col] = xp[j];
          }
        }
        team_barrier(1 + team, 32 * W);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int col = (j >> 2) * 4 * PI + 4 * pi + (j & 3);
          float x = 0.f;
          for (int k2 = 0; k2 < W; ++k2) x += red[buf][team * W + k2][col];
          xp[j] = x;
        }
        buf ^= 1;
      }
      // u = 1 / x with x = diag(1/r) (K v):  u_i = r_i / (K v)_i
#pragma unroll
      for (int j = 0; j < C; ++j) u[j] = rr[j] > 0.f ? __fdividef(rr[j], xp[j]) : 0.f;
    }
  }

  // WMD_j: sum over the lanes of the warp, then over the team's warps
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) wacc += __shfl_xor_sync(0xffffffffu, wacc, off);
  if (W > 1) {
    if (lane == 0) wred[warp] = wacc;
    team_barrier(1 + team, 32 * W);
    if (kw == 0 && lane == 0) {
      double t = 0.0;
      for (int k2 = 0; k2 < W; ++k2) t += wred[team * W + k2];
      p.out[doc] = t * p.inv_lambda;
    }
  } else if (lane == 0) {
    p.out[doc] = wacc * p.inv_lambda;
  }
}

// Per-class tile shapes: {VR, PI, RMAX}; RMAX * (VR / PI) = 96 registers of K.
template <int CLS> struct ClassCfg;
template <> struct ClassCfg<0> { static constexpr int VR = 8, PI = 2, RMAX = 24; };
template <> struct ClassCfg<1> { static constexpr int VR = 16, PI = 4, RMAX = 24; };
template <> struct ClassCfg<2> { static constexpr int VR = 32, PI = 4, RMAX = 12; };
template <> struct ClassCfg<3> { static constexpr int VR = 64, PI = 8, RMAX = 12; };
template <> struct ClassCfg<4> { static constexpr int VR = 128, PI = 8, RMAX = 6; };
template <> struct ClassCfg<5> { static constexpr int VR = 256, PI = 16, RMAX = 6; };

template <int CLS, typename KT>
cudaError_t launch_cls(const LoopParams& p, int n_items, cudaStream_t s) {
  using Cf = ClassCfg<CLS>;
  if (n_items == 0) return cudaSuccess;
  sinkhorn_fused_kernel<Cf::VR, Cf::PI, Cf::RMAX, KT><<<n_items, 128, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename KT>
cudaError_t dispatch_loop(int cls, const LoopParams& p, int n_items, cudaStream_t s) {
  switch (cls) {
    case 0: return launch_cls<0, KT>(p, n_items, s);
    case 1: return launch_cls<1, KT>(p, n_items, s);
    case 2: return launch_cls<2, KT>(p, n_items, s);
    case 3: return launch_cls<3, KT>(p, n_items, s);
    case 4: return launch_cls<4, KT>(p, n_items, s);
    default: return launch_cls<5, KT>(p, n_items, s);
  }
}

}  // namespace

int rows_per_warp(int cls) {
  switch (cls) {
    case 0: return (32 / ClassCfg<0>::PI) * ClassCfg<0>::RMAX;
    case 1: return (32 / ClassCfg<1>::PI) * ClassCfg<1>::RMAX;
    case 2: return (32 / ClassCfg<2>::PI) * ClassCfg<2>::RMAX;
    case 3: return (32 / ClassCfg<3>::PI) * ClassCfg<3>::RMAX;
    case 4: return (32 / ClassCfg<4>::PI) * ClassCfg<4>::RMAX;
    default: return (32 / ClassCfg<5>::PI) * ClassCfg<5>::RMAX;
  }
}

cudaError_t launch_loop(const wmd_corpus* c, int cls, const void* K, int ldk, int kcol0,
                        const float* r, int v_r, float lambda, int T, wmd_precision prec,
                        double* out, cudaStream_t s) {
  LoopParams p;
  p.doc_ptr = c->doc_ptr;
  p.doc_words = c->doc_words;
  p.doc_vals = c->doc_vals;
  p.K = K;
  p.ldk = ldk;
  p.kcol0 = kcol0;
  p.r = r;
  p.v_r = v_r;
  p.T = T;
  p.inv_lambda = 1.0 / (double)lambda;
  p.items = c->sched[cls].d_items;
  p.order = c->order;
  p.out = out;
  if (prec == WMD_PREC_BF16_K) return dispatch_loop<__nv_bfloat16>(cls, p, c->sched[cls].n_items, s);
  return dispatch_loop<float>(cls, p, c->sched[cls].n_items, s);
}

}  // namespace wmd

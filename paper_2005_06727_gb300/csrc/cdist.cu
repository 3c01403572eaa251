// K1: query gather and the cdist + K = exp(-lambda M) build.
//
// Sec. 2 defines m(i, w) = sqrt(sum_k (e_i[k] - e_w[k])^2); Sec. 5 rewrites the
// distance as a GEMM, ||a||^2 + ||b||^2 - 2 a.b, so that the v_r x V block of M
// comes out of one blocked matrix product and the same kernel also emits K.
// Algorithm 1 then needs K = exp(-lambda M) restricted to the query rows.
//
// Output layout is word-major: K[w * ldk + kcol0 + i] for active word row w
// and query column i (the "on the fly transpose" of Sec. 3: the v_r values a
// document word needs are contiguous).  Columns i >= v_r are written as 0.
// A query word equal to the vocabulary word gets M = 0 exactly (K = 1).
#include <algorithm>

#include "wmd_internal.h"

namespace wmd {
namespace {

template <typename KT>
__device__ __forceinline__ KT to_k(float x);
template <>
__device__ __forceinline__ float to_k<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_k<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// -------------------------------------------------------------- cdist (CUDA cores)
// CTA tile: 128 vocabulary rows x VRB query columns, k-slabs of 32.
// Thread (wg, cg): rows 4wg..4wg+3, columns TC*cg..TC*cg+TC-1.
constexpr int kTileW = 128;
constexpr int kSlab = 32;
constexpr int kAStride = kTileW + 4;

template <int VRB, typename KT>
__global__ void __launch_bounds__(256) cdist_kernel(
    const float* __restrict__ vecs, int ldv, int d, const float* __restrict__ norms, int64_t U,
    const int32_t* __restrict__ perm, int64_t V, const int32_t* __restrict__ q_ids,
    const float* __restrict__ q_w, int v_r, int VR, float lambda, KT* __restrict__ K, int ldk,
    int kcol0, float* __restrict__ r_out, float* __restrict__ lam_out, int* __restrict__ err) {
  constexpr int TC = VRB / 8;
  constexpr int BStride = VRB + 4;
  __shared__ __align__(16) float As[kSlab][kAStride];
  __shared__ __align__(16) float Bs[kSlab][BStride];
  __shared__ int32_t qrow_s[VRB];
  __shared__ float qn_s[VRB];

  const int tid = threadIdx.x;
  const int wg = tid & 31;
  const int cg = tid >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * kTileW;
  const int c0 = blockIdx.y * VRB;

  // query compaction output: device row of every query column (-1 padding,
  // -2 an id outside [0, V), whose column becomes NaN) and its norm
  if (tid < VRB) {
    const int col = c0 + tid;
    int row = -1;
    float nq = 0.f;
    if (col < v_r) {
      const int64_t id = q_ids[col];
      if (id >= 0 && id < V) {
        row = perm[id];
        nq = norms[row];
      } else {
        row = -2;
        nq = __int_as_float(0x7fc00000);
      }
    }
    qrow_s[tid] = row;
    qn_s[tid] = nq;
  }
  // the loop kernel reads 1/r through this padded copy of the weights
  if (r_out && blockIdx.x == 0) {
    for (int i = tid + c0; i < c0 + VRB; i += 256) r_out[i] = i < v_r ? q_w[i] : 0.f;
  }
  if (lam_out && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
    // lambda, and the final step's scale -ln 2 / lambda as a double two
    // floats further on (8-byte aligned), for the loop kernel
    *lam_out = lambda;
    *reinterpret_cast<double*>(lam_out + 2) = -0.69314718055994530942 / (double)lambda;
  }
  __syncthreads();

  float acc[4][TC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < TC; ++b) acc[a][b] = 0.f;

  float4 pa[4];
  constexpr int BLoads = (VRB * 8 + 255) / 256;
  float4 pb[BLoads];

  auto fetch = [&](int k0) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int l = tid + 256 * p;
      const int row = l >> 3, kq = l & 7;
      const int64_t w = w0 + row;
      const int k = k0 + 4 * kq;
      pa[p] = (w < U && k < ldv) ? __ldg(reinterpret_cast<const float4*>(vecs + w * ldv + k))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int p = 0; p < BLoads; ++p) {
      const int l = tid + 256 * p;
      const int col = l >> 3, kq = l & 7;
      const int k = k0 + 4 * kq;
      const int row = col < VRB ? qrow_s[col] : -1;
      if (row >= 0 && k < ldv)
        pb[p] = __ldg(reinterpret_cast<const float4*>(vecs + (size_t)row * ldv + k));
      else if (row == -2)
        pb[p] = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
      else
        pb[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int l = tid + 256 * p;
      const int row = l >> 3, kq = l & 7;
      As[4 * kq + 0][row] = pa[p].x;
      As[4 * kq + 1][row] = pa[p].y;
      As[4 * kq + 2][row] = pa[p].z;
      As[4 * kq + 3][row] = pa[p].w;
    }
#pragma unroll
    for (int p = 0; p < BLoads; ++p) {
      const int l = tid + 256 * p;
      const int col = l >> 3, kq = l & 7;
      if (col < VRB) {
        Bs[4 * kq + 0][col] = pb[p].x;
        Bs[4 * kq + 1][col] = pb[p].y;
        Bs[4 * kq + 2][col] = pb[p].z;
        Bs[4 * kq + 3][col] = pb[p].w;
      }
    }
  };

  const int nslab = (ldv + kSlab - 1) / kSlab;
  fetch(0);
  for (int s = 0; s < nslab; ++s) {
    __syncthreads();
    stash();
    __syncthreads();
    if (s + 1 < nslab) fetch((s + 1) * kSlab);
#pragma unroll 8
    for (int kk = 0; kk < kSlab; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][4 * wg]);
      float b[TC];
      if constexpr (TC >= 4) {
#pragma unroll
        for (int q = 0; q < TC / 4; ++q) {
          const float4 t = *reinterpret_cast<const float4*>(&Bs[kk][TC * cg + 4 * q]);
          b[4 * q + 0] = t.x; b[4 * q + 1] = t.y; b[4 * q + 2] = t.z; b[4 * q + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < TC; ++q) b[q] = Bs[kk][TC * cg + q];
      }
#pragma unroll
      for (int q = 0; q < TC; ++q) {
        acc[0][q] = fmaf(a.x, b[q], acc[0][q]);
        acc[1][q] = fmaf(a.y, b[q], acc[1][q]);
        acc[2][q] = fmaf(a.z, b[q], acc[2][q]);
        acc[3][q] = fmaf(a.w, b[q], acc[3][q]);
      }
    }
  }

  // epilogue: M^2 = |a|^2 + |b|^2 - 2 a.b (by direct differences for near
  // pairs, where that form has cancelled more than two bits), clamp, sqrt,
  // exact zero on the query's own word, K = exp(-lambda M)
  bool out_of_range = false;
  float qnv[TC];
  int qrw[TC];
#pragma unroll
  for (int q = 0; q < TC; ++q) {
    qnv[q] = qn_s[TC * cg + q];
    qrw[q] = qrow_s[TC * cg + q];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t w = w0 + 4 * wg + a;
    if (w >= U) continue;
    const float nw = norms[w];
    KT outk[TC];
#pragma unroll
    for (int q = 0; q < TC; ++q) {
      const int col = c0 + TC * cg + q;
      float kv;
      if (col < v_r) {
        if (qrw[q] == (int)w) {
          kv = 1.f;
        } else if (qrw[q] == -2) {
          kv = __int_as_float(0x7fc00000);  // id outside [0, V): NaN column
        } else {
          const float nsum = nw + qnv[q];
          float m2 = nsum - 2.f * acc[a][q];
          if (m2 < kNearPair * nsum && qrw[q] >= 0) m2 = direct_m2(vecs, ldv, d, w, qrw[q]);
          const float lm = lambda * sqrtf(fmaxf(m2, 0.f));
          out_of_range |= qrw[q] >= 0 && lm > kRangeLimit;
          kv = expf(-lm);
        }
      } else {
        kv = 0.f;
      }
      outk[q] = to_k<KT>(kv);
    }
    const size_t o = (size_t)w * ldk + kcol0 + c0 + TC * cg;
#pragma unroll
    for (int q = 0; q < TC; ++q) K[o + q] = outk[q];
  }
  if (out_of_range) atomicOr(err, kRangeFlag);
}

template <int VRB, typename KT>
cudaError_t launch_cdist_t(const wmd_corpus* c, const int32_t* q_ids, const float* q_w, int v_r,
                           int VR, float lambda, KT* K, int ldk, int kcol0, float* r_out, float* lam_out,
                           int* err, cudaStream_t s) {
  // at least one CTA row so that r_out is written even without active words
  const int64_t tiles = std::max<int64_t>((c->U + kTileW - 1) / kTileW, 1);
  dim3 grid((unsigned)tiles, (unsigned)(VR / VRB));
  cdist_kernel<VRB, KT><<<grid, 256, 0, s>>>(c->vecs, c->ldv, c->d, c->norms, c->U, c->perm, c->V,
                                            q_ids, q_w, v_r, VR, lambda, K, ldk, kcol0, r_out, lam_out,
                                            err);
  return cudaGetLastError();
}

template <typename KT>
cudaError_t dispatch_cdist(const wmd_corpus* c, const int32_t* q_ids, const float* q_w, int v_r,
                           int VR, float lambda, KT* K, int ldk, int kcol0, float* r_out, float* lam_out,
                           int* err, cudaStream_t s) {
  switch (VR) {
    case 8: return launch_cdist_t<8, KT>(c, q_ids, q_w, v_r, VR, lambda, K, ldk, kcol0, r_out, lam_out, err, s);
    case 16: return launch_cdist_t<16, KT>(c, q_ids, q_w, v_r, VR, lambda, K, ldk, kcol0, r_out, lam_out, err, s);
    case 32: return launch_cdist_t<32, KT>(c, q_ids, q_w, v_r, VR, lambda, K, ldk, kcol0, r_out, lam_out, err, s);
    default: return launch_cdist_t<64, KT>(c, q_ids, q_w, v_r, VR, lambda, K, ldk, kcol0, r_out, lam_out, err, s);
  }
}

}  // namespace

cudaError_t launch_cdist(const wmd_corpus* c, const int32_t* q_ids, const float* q_w, int v_r,
                         int VR, float lambda, wmd_precision prec, void* K, int ldk, int kcol0,
                         float* r_out, float* lam_out, int* err, const L2Prefetch* pf,
                         cudaStream_t s) {
  // tensor cores (cdist_tc.cu): the query's columns in slices as wide as the
  // resident query operand allows (128 at most); every slice streams the
  // active vocabulary once and writes its own cdist_tc_grid error slots.
  // The choice must match cdist_err_slots.
  const int width = cdist_tc_max_width(c);
  if (width >= VR || (width > 0 && VR <= 16))
    return launch_cdist_tc(c, q_ids, q_w, v_r, VR, lambda, prec, K, ldk, kcol0, r_out, lam_out,
                           err, pf, s);
  if (width > 0) {
    const size_t esz = prec == WMD_PREC_BF16_K ? 2 : 4;
    const int G = cdist_tc_grid(c);
    for (int j0 = 0; j0 < VR; j0 += width) {
      const int vr_slice = std::max(0, std::min(width, v_r - j0));
      // a slice past the last query word still writes its zero padding
      const cudaError_t e = launch_cdist_tc(
          c, q_ids + std::min(j0, v_r), q_w + std::min(j0, v_r), vr_slice, width, lambda, prec,
          static_cast<char*>(K) + (size_t)j0 * esz, ldk, kcol0, r_out ? r_out + j0 : nullptr,
          j0 == 0 ? lam_out : nullptr, err + (j0 / width) * G, j0 == 0 ? pf : nullptr, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // CUDA cores: one slot, cleared here and ORed into by every CTA
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (prec == WMD_PREC_BF16_K)
    return dispatch_cdist<__nv_bfloat16>(c, q_ids, q_w, v_r, VR, lambda,
                                         static_cast<__nv_bfloat16*>(K), ldk, kcol0, r_out,
                                         lam_out, err, s);
  return dispatch_cdist<float>(c, q_ids, q_w, v_r, VR, lambda, static_cast<float*>(K), ldk,
                               kcol0, r_out, lam_out, err, s);
}

int cdist_err_slots(const wmd_corpus* c, int VR) {
  const int width = cdist_tc_max_width(c);
  if (width >= VR || (width > 0 && VR <= 16)) return cdist_tc_grid(c);
  if (width > 0) return (VR + width - 1) / width * cdist_tc_grid(c);
  return 1;
}

}  // namespace wmd

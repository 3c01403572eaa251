// Algorithm 1 in its dense form, on the GPU: the comparator for the sparse
// fused loop.
//
// Sec. 3 ("Dense to Sparse Kernel", Table 1) argues that the dense form wastes
// almost all of its time computing K^T u at every (word, document) position
// and scaling the dense c with it, although only the nonzeros of c are ever
// used.  This file computes the dense form literally, so that the argument
// can be measured on the same GPU:
//
//   x = 1/v_r
//   repeat max_iter times:
//     S = K^T u                 (dense U x N: cuBLAS SGEMM, k = VR)
//     v = c .* (1 ./ S)         (dense U x N, elementwise)
//     x = diag(1/r) (K v)       (VR x N: cuBLAS SGEMM, k = U);  u = 1 ./ x
//   S = K^T u;  v = c .* (1 ./ S)
//   WMD_j = sum_i u_ij ((K .* M) v)_ij      (SGEMM, then an FP64 column sum)
//
// The rows are the corpus's active vocabulary (U words, the device-row order
// of the resident embeddings): the dense c is zero on every other word, whose
// rows only ever multiply zeros.  K (word-major U x VR, exactly the K that the
// sparse path uses) is a column-major VR x U matrix with leading dimension VR.
// K .* M is recovered from K as K (-ln K) / lambda, as in the fused loop.  The
// GEMMs are plain library GEMMs in FP32 (cuBLAS's default math: no TF32); the
// elementwise steps are this file's kernels.
#include <cublas_v2.h>

#include <mutex>

#include "wmd_internal.h"

namespace wmd {
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct DenseLayout {
  size_t c_off, s_off, q_off, u_off, x_off, km_off, total;
};

// [c: U x N][S: U x N][query workspace: r, lambda, K][u: VR x N][X: VR x N][KM: VR x U]
DenseLayout dense_layout(const wmd_corpus* c, int VR) {
  DenseLayout L;
  const size_t un = (size_t)std::max<int64_t>(c->U, 1) * (size_t)std::max<int64_t>(c->N, 1);
  const size_t vn = (size_t)VR * (size_t)std::max<int64_t>(c->N, 1);
  size_t o = 0;
  L.c_off = o;  o = align256(o + un * sizeof(float));
  L.s_off = o;  o = align256(o + un * sizeof(float));
  L.q_off = o;  o = align256(o + ws_layout(c, VR, WMD_PREC_FP32).total);
  L.u_off = o;  o = align256(o + vn * sizeof(float));
  L.x_off = o;  o = align256(o + vn * sizeof(float));
  L.km_off = o; o = align256(o + (size_t)VR * std::max<int64_t>(c->U, 1) * sizeof(float));
  L.total = o;
  return L;
}

// dense c, column j = document j (U entries); one warp per document
__global__ void scatter_c_kernel(const int64_t* __restrict__ doc_ptr,
                                 const int32_t* __restrict__ doc_words,
                                 const float* __restrict__ doc_vals, int64_t N, int64_t U,
                                 float* __restrict__ cd) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= N) return;
  for (int64_t k = doc_ptr[j] + lane; k < doc_ptr[j + 1]; k += 32)
    cd[j * U + doc_words[k]] = doc_vals[k];
}

// x = 1 / v_r, i.e. u = v_r on the query rows (0 on padding rows)
__global__ void init_u_kernel(float* __restrict__ u, int VR, int v_r, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    u[t] = (int)(t % VR) < v_r ? (float)v_r : 0.f;
}

// S <- c .* (1 ./ S), elementwise over the dense U x N block
__global__ void ratio_kernel(const float* __restrict__ cd, float* __restrict__ s, int64_t n) {
  const int64_t n4 = n / 4;
  const float4* c4 = reinterpret_cast<const float4*>(cd);
  float4* s4 = reinterpret_cast<float4*>(s);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
    const float4 a = c4[t];
    float4 b = s4[t];
    b.x = a.x * (1.f / b.x);
    b.y = a.y * (1.f / b.y);
    b.z = a.z * (1.f / b.z);
    b.w = a.w * (1.f / b.w);
    s4[t] = b;
  }
  for (int64_t t = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    s[t] = cd[t] * (1.f / s[t]);
}

// x = diag(1/r) X, u = 1 ./ x on the query rows (0 on padding rows)
__global__ void update_u_kernel(const float* __restrict__ X, const float* __restrict__ r,
                                float* __restrict__ u, int VR, int v_r, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % VR);
    u[t] = i < v_r ? 1.f / ((1.f / r[i]) * X[t]) : 0.f;
  }
}

// K .* M with M = -ln(K) / lambda (0 where K is 0: padding rows)
__global__ void km_kernel(const float* __restrict__ K, const float* __restrict__ lam,
                          float* __restrict__ km, int64_t n) {
  const float l = *lam;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float k = K[t];
    km[t] = k > 0.f ? k * (-logf(k) / l) : 0.f;
  }
}

// WMD_j = sum_i u_ij Y_ij, accumulated in FP64; one thread per document
__global__ void column_sum_kernel(const float* __restrict__ u, const float* __restrict__ Y, int VR,
                                  int64_t N, double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double acc = 0.0;
  for (int i = 0; i < VR; ++i) acc += (double)u[j * VR + i] * (double)Y[j * VR + i];
  out[j] = acc;
}

std::mutex g_blas_mu;
cublasHandle_t g_blas[64] = {};

int grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16);
}

wmd_status blas_error(cublasStatus_t st, const char* what) {
  return set_error(st == CUBLAS_STATUS_ALLOC_FAILED ? WMD_ERR_OUT_OF_MEMORY : WMD_ERR_CUDA,
                   std::string(what) + ": cuBLAS status " + std::to_string((int)st));
}

#define WMD_BLAS_TRY(expr)                                        \
  do {                                                            \
    cublasStatus_t st_ = (expr);                                  \
    if (st_ != CUBLAS_STATUS_SUCCESS) return blas_error(st_, #expr); \
  } while (0)

}  // namespace

}  // namespace wmd

using namespace wmd;

extern "C" {

size_t wmd_dense_workspace_bytes(const wmd_corpus* c, int32_t v_r) {
  if (!c || v_r <= 0 || v_r > WMD_MAX_VR) return 0;
  return dense_layout(c, kClassKVR[vr_class(v_r)]).total;
}

wmd_status wmd_dense_load_c(wmd_corpus* c, void* d_ws, size_t ws_bytes, void* stream) {
  wmd::NvtxRange nvtx_range("wmd_dense_load_c");
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  const DenseLayout L = dense_layout(c, 8);
  if (!d_ws || ws_bytes < L.s_off) return set_error(WMD_ERR_INVALID_ARG, "workspace too small");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) WMD_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* cd = reinterpret_cast<float*>(static_cast<char*>(d_ws) + L.c_off);
  cudaError_t e = cudaMemsetAsync(cd, 0, (size_t)c->U * c->N * sizeof(float), s);
  if (e == cudaSuccess && c->N > 0) {
    const int threads = 256;
    const int64_t blocks = (c->N * 32 + threads - 1) / threads;
    scatter_c_kernel<<<(unsigned)blocks, threads, 0, s>>>(c->doc_ptr, c->doc_words, c->doc_vals,
                                                          c->N, c->U, cd);
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_error(e, "wmd_dense_load_c");
  return WMD_OK;
}

wmd_status wmd_query_dense(wmd_corpus* c, const int32_t* d_q_ids, const float* d_q_w,
                           int32_t v_r, float lambda, int32_t max_iter, void* d_ws,
                           size_t ws_bytes, double* d_out, void* stream) {
  wmd::NvtxRange nvtx_range("wmd_query_dense");
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  if (v_r <= 0 || v_r > WMD_MAX_VR) return set_error(WMD_ERR_INVALID_ARG, "v_r out of range");
  if (max_iter < 0) return set_error(WMD_ERR_INVALID_ARG, "max_iter must be >= 0");
  const int VR = kClassKVR[vr_class(v_r)];
  const DenseLayout L = dense_layout(c, VR);
  if (!d_ws || ws_bytes < L.total) return set_error(WMD_ERR_INVALID_ARG, "workspace too small");
  if (!d_out && c->N > 0) return set_error(WMD_ERR_INVALID_ARG, "d_out is NULL");
  if (c->U > INT32_MAX || c->N > INT32_MAX)
    return set_error(WMD_ERR_UNSUPPORTED, "dense form limited to 2^31 - 1 words and documents");
  char* ws = static_cast<char*>(d_ws);
  const WsLayout Q = ws_layout(c, VR, WMD_PREC_FP32);
  wmd_status st = wmd_build_kernel_matrix(c, d_q_ids, d_q_w, v_r, lambda, WMD_PREC_FP32,
                                          ws + L.q_off, Q.total, stream);
  if (st != WMD_OK) return st;
  if (c->N == 0) return WMD_OK;

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) WMD_CUDA_TRY(cudaSetDevice(c->device));
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, c->device};

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_blas_mu);
  if (c->device < 0 || c->device >= 64) return set_error(WMD_ERR_UNSUPPORTED, "device ordinal");
  cublasHandle_t& h = g_blas[c->device];
  if (!h) {
    WMD_BLAS_TRY(cublasCreate(&h));
    WMD_BLAS_TRY(cublasSetMathMode(h, CUBLAS_DEFAULT_MATH));
  }
  WMD_BLAS_TRY(cublasSetStream(h, s));

  const int U = (int)c->U, N = (int)c->N;
  const float* cd = reinterpret_cast<const float*>(ws + L.c_off);
  float* S = reinterpret_cast<float*>(ws + L.s_off);
  const float* r = reinterpret_cast<const float*>(ws + L.q_off + Q.r_off);
  const float* lam = r + VR;
  const float* K = reinterpret_cast<const float*>(ws + L.q_off + Q.k_off);
  float* u = reinterpret_cast<float*>(ws + L.u_off);
  float* X = reinterpret_cast<float*>(ws + L.x_off);
  float* KM = reinterpret_cast<float*>(ws + L.km_off);
  const int64_t un = (int64_t)U * N, vn = (int64_t)VR * N;
  const float one = 1.f, zero = 0.f;
  const int T = 256;

  init_u_kernel<<<grid_for(vn, T), T, 0, s>>>(u, VR, v_r, vn);
  WMD_CUDA_TRY(cudaGetLastError());
  for (int it = 0; it <= max_iter; ++it) {
    // S = K^T u  (U x N)
    WMD_BLAS_TRY(cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, U, N, VR, &one, K, VR, u, VR, &zero,
                             S, U));
    // v = c .* (1 ./ S), in place
    ratio_kernel<<<grid_for(un / 4 + 1, T), T, 0, s>>>(cd, S, un);
    WMD_CUDA_TRY(cudaGetLastError());
    if (it == max_iter) break;
    // X = K v  (VR x N), then u = 1 ./ (diag(1/r) X)
    WMD_BLAS_TRY(cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, VR, N, U, &one, K, VR, S, U, &zero,
                             X, VR));
    update_u_kernel<<<grid_for(vn, T), T, 0, s>>>(X, r, u, VR, v_r, vn);
    WMD_CUDA_TRY(cudaGetLastError());
  }
  // WMD = sum(u .* ((K .* M) v))
  km_kernel<<<grid_for((int64_t)VR * U, T), T, 0, s>>>(K, lam, KM, (int64_t)VR * U);
  WMD_CUDA_TRY(cudaGetLastError());
  WMD_BLAS_TRY(cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, VR, N, U, &one, KM, VR, S, U, &zero, X,
                           VR));
  column_sum_kernel<<<(N + T - 1) / T, T, 0, s>>>(u, X, VR, N, d_out);
  WMD_CUDA_TRY(cudaGetLastError());
  return WMD_OK;
}

}  // extern "C"

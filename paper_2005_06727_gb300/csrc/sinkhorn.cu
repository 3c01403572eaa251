// K2 + K3: the fused Sinkhorn-Knopp loop and the final WMD reduction, with a
// fixed number of loop bodies (Sec. 3: max_iter bodies, then one more u/v
// update and the reduction).  The kernel itself, and how it maps Algorithm 1
// onto warps, registers and shared memory, is in sinkhorn_kernel.cuh.
#include "sinkhorn_kernel.cuh"

namespace wmd {
namespace {

template <int CLS, int V>
constexpr int rpw() { return (32 / Var<CLS, V>::PI) * Var<CLS, V>::RMAX; }

}  // namespace

int rows_per_warp(int cls, int var) {
  switch (cls) {
    case 0: return var ? rpw<0, 1>() : rpw<0, 0>();
    case 1: return var ? rpw<1, 1>() : rpw<1, 0>();
    case 2: return var ? rpw<2, 1>() : rpw<2, 0>();
    case 3: return var ? rpw<3, 1>() : rpw<3, 0>();
    case 4: return var ? rpw<4, 1>() : rpw<4, 0>();
    default: return var ? rpw<5, 1>() : rpw<5, 0>();
  }
}

int warps_per_cta(int cls, int var) {
  switch (cls) {
    case 4: return var ? Var<4, 1>::NW : Var<4, 0>::NW;
    case 5: return var ? Var<5, 1>::NW : Var<5, 0>::NW;
    default: return 4;
  }
}

L2Prefetch loop_inputs(const wmd_corpus* c, int cls, wmd_precision prec) {
  L2Prefetch pf{};
  if (cls < 0 || cls >= kNumClasses) return pf;
  const int var = c->loop_variant[cls][prec == WMD_PREC_BF16_K];
  pf.ptr[0] = c->sched[cls][var].d_tasks;
  pf.bytes[0] = (size_t)c->sched[cls][var].n_items * warps_per_cta(cls, var) * sizeof(WarpTask);
  pf.ptr[1] = c->doc_words;
  pf.bytes[1] = (size_t)c->nnz * sizeof(int32_t);
  pf.ptr[2] = c->doc_vals;
  pf.bytes[2] = (size_t)c->nnz * sizeof(float);
  return pf;
}

cudaError_t launch_loop(const wmd_corpus* c, int cls, const void* K, int ldk, int kcol0,
                        const float* r, const float* lam, int v_r, int T, wmd_precision prec,
                        double* out, const int* err, int* err_out, cudaStream_t s) {
  const int var = c->loop_variant[cls][prec == WMD_PREC_BF16_K];
  LoopParams p = base_params(c, cls, var, K, ldk, T, err);
  p.kcol0 = kcol0;
  p.r = r;
  p.lam = lam;
  p.v_r = v_r;
  p.out = out;
  p.err_out = err_out;
  const int n_items = c->sched[cls][var].n_items;
  if (prec == WMD_PREC_BF16_K) return dispatch_loop<false, __nv_bfloat16>(cls, var, p, n_items, 1, s);
  return dispatch_loop<false, float>(cls, var, p, n_items, 1, s);
}

cudaError_t launch_loop_batch(const wmd_corpus* c, int cls, const void* K, int ldk,
                              const QueryDesc* d_queries, int nq, int T, wmd_precision prec,
                              cudaStream_t s) {
  const int var = c->loop_variant[cls][prec == WMD_PREC_BF16_K];
  LoopParams p = base_params(c, cls, var, K, ldk, T, nullptr);  // errors: per query descriptor
  p.queries = d_queries;
  const int n_items = c->sched[cls][var].n_items;
  if (prec == WMD_PREC_BF16_K) return dispatch_loop<false, __nv_bfloat16>(cls, var, p, n_items, nq, s);
  return dispatch_loop<false, float>(cls, var, p, n_items, nq, s);
}

}  // namespace wmd

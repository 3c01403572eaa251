// K2 + K3: the fused Sinkhorn-Knopp loop and the final WMD reduction, with a
// fixed number of loop bodies (Sec. 3: max_iter bodies, then one more u/v
// update and the reduction).  The kernel itself, and how it maps Algorithm 1
// onto warps, registers and shared memory, is in sinkhorn_kernel.cuh.
#include "sinkhorn_kernel.cuh"

namespace wmd {
namespace {

template <int CLS, int V>
constexpr int rpw() { return (32 / Var<CLS, V>::PI) * Var<CLS, V>::RMAX; }

// rows per warp and warps per CTA of variant `var` of class CLS
template <int CLS>
int cls_rows(int var) {
  if constexpr (kClassVariants[CLS] > 2) {
    if (var == 2) return rpw<CLS, 2>();
  }
  return var ? rpw<CLS, 1>() : rpw<CLS, 0>();
}
template <int CLS>
int cls_warps(int var) {
  if constexpr (kClassVariants[CLS] > 2) {
    if (var == 2) return Var<CLS, 2>::NW;
  }
  return var ? Var<CLS, 1>::NW : Var<CLS, 0>::NW;
}

}  // namespace

int rows_per_warp(int cls, int var) {
  switch (cls) {
    case 0: return cls_rows<0>(var);
    case 1: return cls_rows<1>(var);
    case 2: return cls_rows<2>(var);
    case 3: return cls_rows<3>(var);
    case 4: return cls_rows<4>(var);
    case 5: return cls_rows<5>(var);
    case 6: return cls_rows<6>(var);
    case 7: return cls_rows<7>(var);
    default: return cls_rows<8>(var);
  }
}

int warps_per_cta(int cls, int var) {
  switch (cls) {
    case 0: return cls_warps<0>(var);
    case 1: return cls_warps<1>(var);
    case 2: return cls_warps<2>(var);
    case 3: return cls_warps<3>(var);
    case 4: return cls_warps<4>(var);
    case 5: return cls_warps<5>(var);
    case 6: return cls_warps<6>(var);
    case 7: return cls_warps<7>(var);
    default: return cls_warps<8>(var);
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
                        double* out, const int* err, int n_err, int* err_out, cudaStream_t s) {
  const int var = c->loop_variant[cls][prec == WMD_PREC_BF16_K];
  LoopParams p = base_params(c, cls, var, K, ldk, T, err, n_err);
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
  // errors: the host reads every batched query's slots
  LoopParams p = base_params(c, cls, var, K, ldk, T, nullptr, 0);
  p.queries = d_queries;
  const int n_items = c->sched[cls][var].n_items;
  if (prec == WMD_PREC_BF16_K) return dispatch_loop<false, __nv_bfloat16>(cls, var, p, n_items, nq, s);
  return dispatch_loop<false, float>(cls, var, p, n_items, nq, s);
}

}  // namespace wmd

// K2 + K3 with Algorithm 1's loop condition "while x changes": the fused loop
// of sinkhorn_kernel.cuh instantiated with the per-document convergence test.
//
// Every column of x depends only on its own document, so the test is taken per
// document: after each loop body the team that owns the document checks all
// its query rows for |x' - x| <= tol x (in the form |u' - u| <= tol u', the
// same inequality since u = r / x) and, once it holds, runs the final u/v
// update and the WMD reduction instead of another body.  max_iter still caps
// the loop.  The team writes the number of bodies it ran, so a caller can see
// which documents converged.  These instances live in their own translation
// unit so that they compile in parallel with the fixed-count ones.
#include "sinkhorn_kernel.cuh"

namespace wmd {

cudaError_t launch_loop_conv(const wmd_corpus* c, int cls, const void* K, int ldk,
                             const float* r, const float* lam, int v_r, int T, float tol,
                             wmd_precision prec, double* out, int32_t* iters, const int* err,
                             int n_err, cudaStream_t s) {
  const int var = c->loop_variant[cls][prec == WMD_PREC_BF16_K];
  LoopParams p = base_params(c, cls, var, K, ldk, T, err, n_err);
  p.r = r;
  p.lam = lam;
  p.v_r = v_r;
  p.out = out;
  p.tol = tol;
  p.iters = iters;
  const int n_items = c->sched[cls][var].n_items;
  if (prec == WMD_PREC_BF16_K) return dispatch_loop<true, __nv_bfloat16>(cls, var, p, n_items, 1, s);
  return dispatch_loop<true, float>(cls, var, p, n_items, 1, s);
}

}  // namespace wmd

// Internal declarations shared by the translation units of the WMD library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wmd.h"

namespace wmd {

// ---------------------------------------------------------------- tracing
// A named NVTX range over a host-side scope: profilers (nsys, ncu --nvtx)
// show the library's phases under these names.  NVTX is header-only here and
// costs a few nanoseconds per range when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- errors
wmd_status set_error(wmd_status st, const std::string& msg);
wmd_status cuda_error(cudaError_t e, const char* what);

#define WMD_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t e_ = (expr);                                \
    if (e_ != cudaSuccess) return ::wmd::cuda_error(e_, #expr); \
  } while (0)

// ---------------------------------------------------------------- query width classes
// The fused loop pads the query to one of these widths (its register tile,
// kClassVR); the cdist kernel, K and the workspace use the power of two at or
// above it (kClassKVR: K rows have that many entries, and the loop reads the
// first kClassVR of them).  The 48-, 96- and 192-wide tiles save a quarter
// of the loop's work for queries just above 32, 64 and 128 words.
constexpr int kNumClasses = 9;
constexpr int kClassVR[kNumClasses] = {8, 16, 32, 48, 64, 96, 128, 192, 256};
constexpr int kClassKVR[kNumClasses] = {8, 16, 32, 64, 64, 128, 128, 256, 256};

inline int vr_class(int v_r) {
  for (int c = 0; c < kNumClasses; ++c)
    if (v_r <= kClassVR[c]) return c;
  return -1;
}

// The class whose loop tile is `width` wide, or -1.
inline int class_of_width(int width) {
  for (int c = 0; c < kNumClasses; ++c)
    if (kClassVR[c] == width) return c;
  return -1;
}

// Fused-loop tile variants per class (sinkhorn.cu) and the rows one warp of
// variant `var` keeps in registers (row groups x rows per lane).
constexpr int kMaxVariants = 2;
constexpr int kClassVariants[kNumClasses] = {2, 2, 2, 2, 2, 2, 2, 2, 2};
int rows_per_warp(int cls, int var);
int warps_per_cta(int cls, int var);  // 4 or 8

// The task of one warp in one CTA work item of the fused loop: the document
// its team solves (its range in the document-major CSR, its length and id)
// and the team size W (warps per document).  A CTA's NW/W teams take
// consecutive documents of the length-sorted order; W = 0 marks a warp with
// no team in the item.  One 16-byte load per warp at item start.
struct WarpTask {
  int64_t beg;
  int32_t n_w;  // n | W << 24
  int32_t doc;
};
constexpr int kTaskWShift = 24;

// The partition of the documents into teams: a document of n words gets the
// smallest team of W warps (W = 1, 2, 4, ... up to the CTA's warps) with
// n <= W x rows_per_warp x fill / 100.  fill = 100 keeps every document that
// fits in registers resident with as few warps as possible; below 100 spreads
// documents over more warps (fewer rows per warp, more cross-warp sums);
// above 100 gives long documents fewer warps, which then re-read chunks of K
// from L2 each pass.  The autotuner picks one per class and tile variant.
constexpr int kNumFills = 4;
constexpr int kFills[kNumFills] = {100, 75, 50, 200};
inline bool valid_fill(int f) {
  for (int i = 0; i < kNumFills; ++i)
    if (kFills[i] == f) return true;
  return false;
}

struct Schedule {
  WarpTask* d_tasks = nullptr;  // n_items x (warps per CTA)
  int32_t n_items = 0;
  int32_t fill = 100;           // the partition this schedule was built with
};

}  // namespace wmd

struct wmd_corpus {
  int device = 0;
  int64_t V = 0, N = 0, nnz = 0, U = 0;
  int32_t d = 0, ldv = 0;  // embedding width and padded row stride (floats)

  // device, resident
  float* vecs = nullptr;       // V x ldv, rows permuted: active words first
  float* norms = nullptr;      // V, squared row norms (fp64 sum, rounded)
  // the same rows as an fp16 pair for the tensor cores: row w scaled by 2^e_w
  // (its largest entry in [2^14, 2^15)), x = hi + lo * 2^-11 up to 2^-22
  // relative; rscale[w] = 2^-e_w
  uint16_t* vecs_hi = nullptr; // V x ldv fp16 bits
  uint16_t* vecs_lo = nullptr; // V x ldv fp16 bits
  float* rscale = nullptr;     // V
  int32_t* perm = nullptr;     // V: word id -> device row
  int64_t* doc_ptr = nullptr;  // N+1, document-major CSR of c^T
  int32_t* doc_words = nullptr;// nnz, device rows (< U) sorted within a doc
  float* doc_vals = nullptr;   // nnz
  wmd::Schedule sched[wmd::kNumClasses][wmd::kMaxVariants];
  // host copies kept for rebuilding schedules with another partition
  std::vector<int64_t> h_dptr;   // N+1, document-major CSR offsets
  std::vector<int32_t> h_order;  // documents by decreasing length (stable)
  int loop_variant[wmd::kNumClasses][2] = {};  // chosen variant per class and precision
  size_t device_bytes = 0;
  int num_sms = 0;
  bool tmap_ok = false;        // tensor-core cdist available (TMA descriptors built)
  // options (wmd_options)
  bool use_graphs = true;
  long long wait_cycles = 0;   // device-side wait limit of the tensor-core cdist (0: default)
  std::string autotune_cache;  // file of tuned loop variants ("" = none)
  wmd_server_options server_defaults{};
  alignas(64) unsigned char tmap_hi[128];  // CUtensorMap of vecs_hi (128-byte tiles of 128 rows)
  alignas(64) unsigned char tmap_lo[128];  // CUtensorMap of vecs_lo

  // host path (wmd_query) state, guarded by mu
  std::mutex mu;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int32_t* h_stage = nullptr;  // pinned, mapped: WMD_MAX_VR ids and WMD_MAX_VR weights (read by the cdist kernel), error word (written by the loop kernel)
  double* h_out = nullptr;     // pinned, mapped N doubles: the loop kernel writes the results here (host path)
  int32_t* dh_stage = nullptr; // device addresses of the two mapped blocks
  double* dh_out = nullptr;
  // captured host-path sequences, keyed by query shape (second use onwards)
  struct QueryGraph {
    int v_r, T, prec, variant;
    float lambda;
    double* dout;  // where the loop kernel writes the results
    int uses;
    cudaGraphExec_t exec;
    uint64_t last;
  };
  std::vector<QueryGraph> qgraphs;
  uint64_t qtick = 0;
};

namespace wmd {

// Workspace carve-up for one query whose K rows are VR wide (kClassKVR of its
// class): the padded query weights r (VR floats) followed by lambda (float VR)
// and the final step's scale -ln 2 / lambda (a double at float VR + 2); the
// query's error slots (cdist_err_slots ints); and the word-major K (U x VR).
struct WsLayout {
  size_t r_off, err_off, k_off, total;
  int n_err;
};
// Error slot codes: a cdist wait that ran out (0x40000000 | role << 24 |
// iteration) and/or kRangeFlag once some lambda * M reached the float32 range
// limit of K.  The tensor-core cdist writes one slot per CTA at its end, so
// nothing clears the slots before a query; the CUDA-core cdist ORs into one
// slot that a memset clears first.
constexpr int kRangeFlag = 0x20000000;
constexpr float kRangeLimit = 87.33654f;  // -ln(FLT_MIN): K = exp(-lambda M) below is subnormal
// Error slots one query of K width VR uses (the cdist kernel's CTAs over
// all its column slices, or 1 for the CUDA-core kernel).
int cdist_err_slots(const wmd_corpus* c, int VR);
// CTAs of one tensor-core cdist launch.
int cdist_tc_grid(const wmd_corpus* c);
// Host summary of a query's error slots: the first nonzero code, with the
// range flag if any slot has it (0: no error).
inline int error_summary(const int* slots, size_t n) {
  int first = 0, any = 0;
  for (size_t i = 0; i < n; ++i) {
    if (!first) first = slots[i];
    any |= slots[i];
  }
  return first | (any & kRangeFlag);
}
WsLayout ws_layout(const wmd_corpus* c, int VR, wmd_precision prec);

// Read-only regions (up to three) that the kernel after cdist starts from;
// the tensor-core cdist prefetches them into L2 while it streams.
struct L2Prefetch {
  const void* ptr[3];
  size_t bytes[3];
};
// The fused loop's inputs for query class cls: its work items and the
// document-major CSR.
L2Prefetch loop_inputs(const wmd_corpus* c, int cls, wmd_precision prec);

// Kernel launchers (cdist.cu / sinkhorn.cu).  err: the query's error slots
// (cdist_err_slots of them).
cudaError_t launch_cdist(const wmd_corpus* c, const int32_t* q_ids, const float* q_w, int v_r,
                         int VR, float lambda, wmd_precision prec, void* K, int ldk, int kcol0,
                         float* r_out, float* lam_out, int* err, const L2Prefetch* pf,
                         cudaStream_t s);
cudaError_t launch_cdist_tc(const wmd_corpus* c, const int32_t* q_ids, const float* q_w, int v_r,
                            int VR, float lambda, wmd_precision prec, void* K, int ldk, int kcol0,
                            float* r_out, float* lam_out, int* err, const L2Prefetch* pf,
                            cudaStream_t s);
bool make_vecs_tensor_map(wmd_corpus* c);
// Widest query slice the tensor-core cdist takes for this corpus (0: none).
int cdist_tc_max_width(const wmd_corpus* c);
void release_batch_state(const wmd_corpus* c);  // serve.cu: cached batch buffers and graphs
// One query of a batched loop launch: its padded weights r, output row, first
// column of its block in the word-major K, and its number of words.
struct QueryDesc {
  const float* r;
  double* out;
  int kcol0;
  int v_r;
  float lambda;
  double scale;    // -ln 2 / lambda, the final step's factor
};
cudaError_t launch_loop_batch(const wmd_corpus* c, int cls, const void* K, int ldk,
                              const QueryDesc* d_queries, int nq, int T, wmd_precision prec,
                              cudaStream_t s);
// err: the query's error slots; err_out (optional, device-visible): receives
// their summary (the first CTA's code found, with the range flag, or 0)
cudaError_t launch_loop(const wmd_corpus* c, int cls, const void* K, int ldk, int kcol0,
                        const float* r, const float* lam, int v_r, int T, wmd_precision prec,
                        double* out, const int* err, int n_err, int* err_out, cudaStream_t s);
// Top-k selection of WMD[N] (topk.cu): the k smallest values (ties: lower
// document id first; NaN last) into out_idx / out_val, ascending.
constexpr int kTopkMaxK = 1024;
cudaError_t launch_topk(const double* wmd, int64_t N, int k, int64_t* out_idx, double* out_val,
                        cudaStream_t s);
// The convergence-tested loop (sinkhorn_conv.cu): at most T bodies, a
// document stopping once |x' - x| <= tol x for all its query rows; iters
// (optional, device) receives the bodies run per document.
cudaError_t launch_loop_conv(const wmd_corpus* c, int cls, const void* K, int ldk,
                             const float* r, const float* lam, int v_r, int T, float tol,
                             wmd_precision prec, double* out, int32_t* iters, const int* err,
                             int n_err, cudaStream_t s);
// Host-side message for a nonzero error word summary (timeout or range).
wmd_status device_error(int code);
// Looks up the no-allocation entry point's scratch array on `device` (once
// per device; the lookup makes the driver reserve the array there).
cudaError_t noalloc_reserve(int device);
// The squared distance of two embedding rows by direct differences (Sec. 2),
// used by the cdist kernels where the GEMM form |a|^2 + |b|^2 - 2 a.b has
// cancelled more than two bits (near pairs, Sec. 5's concern).
__device__ __forceinline__ float direct_m2(const float* __restrict__ vecs, int ldv, int d,
                                           int64_t a, int64_t b) {
  const float* pa = vecs + a * ldv;
  const float* pb = vecs + b * ldv;
  float acc = 0.f;
  for (int k = 0; k < d; ++k) {
    const float t = __ldg(pa + k) - __ldg(pb + k);
    acc = fmaf(t, t, acc);
  }
  return acc;
}
// Below this fraction of |a|^2 + |b|^2 the GEMM form is replaced by direct_m2.
constexpr float kNearPair = 0.25f;

}  // namespace wmd

/*
 * wmd.h -- C ABI of the GB300 sparse Sinkhorn-Knopp Word Mover's Distance.
 *
 * The library computes, for one query histogram r and many target histograms
 * c (the columns of a V x N sparse matrix), the Sinkhorn distance of
 * Algorithm 1 of Tithi & Petrini, "An Efficient Shared-memory Parallel
 * Sinkhorn-Knopp Algorithm to Compute the Word Mover's Distance"
 * (arXiv 2005.06727), in the sparse SDDMM + SpMM form of its Sec. 3:
 *
 *   I = (r > 0); M[i, w] = ||vecs[q_i] - vecs[w]||_2 (Sec. 2, unsquared);
 *   K = exp(-lambda M);  x = 1/v_r;
 *   repeat max_iter times:  u = 1/x;  v = c ./ (K^T u) at the nonzeros of c
 *                           (SDDMM);  x = diag(1/r) K v  (SpMM)
 *   u = 1/x;  v = c ./ (K^T u);  WMD_j = sum_i u_ij ((K .* M) v)_ij.
 *
 * Besides that fixed-count form (single, device-resident, batched and served
 * queries), the library offers Algorithm 1's own loop condition "while x
 * changes" per document (wmd_query_device_tol), the k nearest documents of a
 * query (wmd_topk, wmd_query_device_topk), Algorithm 1 in its dense form as a
 * measured comparator (wmd_query_dense), and a device query for callers that
 * cannot allocate (wmd_query_device_noalloc).
 *
 * Conventions shared by every entry point:
 *  - All functions return a wmd_status; on failure wmd_last_error() returns a
 *    thread-local message describing the first error.  No entry point aborts
 *    or traps; CUDA errors are reported as WMD_ERR_CUDA.
 *  - "host" pointers are ordinary CPU memory borrowed for the duration of the
 *    call; "device" pointers are CUDA global memory on the corpus's device.
 *    The caller owns every buffer it passes; the library owns the corpus and
 *    server objects and the device copies inside them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device-path entry points only enqueue work on it.
 *  - No renormalisation: r and the columns of c are used exactly as given,
 *    the paper assumes both sum to 1 (Sec. 3).
 *  - lambda > 0 and K = exp(-lambda M) (Algorithm 1; the paper's Python passes
 *    lambda negated, which this API does not).
 *  - Results follow the IEEE arithmetic of the formula: a document without
 *    words gives NaN when max_iter >= 1 (u = 1/0 meets a zero column) and 0
 *    when max_iter == 0.
 *  - Arithmetic: float32 for the loop (the BF16_K precision stores K in
 *    bfloat16 and still accumulates in float32), float64 for the final
 *    per-document sum.  Valid while lambda * M < 87.3 for every query word
 *    and active vocabulary word, so that K = exp(-lambda M) stays a normal
 *    float32.  The cdist kernel checks this for every entry it writes; a
 *    query that leaves the range gets NaN for every document, and the host
 *    entry points (wmd_query, wmd_query_batch, the server) report
 *    WMD_ERR_RANGE.
 *  - Device-side errors are per query: every CTA of a query's cdist kernel
 *    writes its own error slot in the query's workspace at every launch
 *    (nothing has to clear them), so a failed query never affects a later
 *    one or one running beside it; a query of a batch that fails gets NaN
 *    results and the batch call reports it.
 */
#ifndef WMD_GB300_H
#define WMD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum wmd_status {
  WMD_OK = 0,
  WMD_ERR_INVALID_ARG = 1,   /* a size, pointer, id or weight is invalid       */
  WMD_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed, or an
                                admission budget is exceeded                    */
  WMD_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed     */
  WMD_ERR_NOT_READY = 4,     /* a served request has not finished yet          */
  WMD_ERR_TIMEOUT = 5,       /* a bounded wait ran out                         */
  WMD_ERR_SHUTDOWN = 6,      /* the server is shutting down                    */
  WMD_ERR_UNSUPPORTED = 7,   /* e.g. v_r above WMD_MAX_VR                      */
  WMD_ERR_RANGE = 8          /* lambda * M reached 87.3 for some word pair: K
                                would leave the float32 range (results NaN)   */
} wmd_status;

typedef enum wmd_precision {
  WMD_PREC_FP32 = 0,   /* K stored and used in float32                        */
  WMD_PREC_BF16_K = 1  /* K stored in bfloat16, loop arithmetic in float32     */
} wmd_precision;

/* Largest number of query words (after dropping zero weights) per query. */
#define WMD_MAX_VR 256

typedef struct wmd_corpus wmd_corpus; /* opaque, owned by the library */
typedef struct wmd_server wmd_server; /* opaque, owned by the library */

typedef struct wmd_corpus_info {
  int64_t V;        /* vocabulary size (rows of vecs and of c)               */
  int32_t d;        /* embedding width                                       */
  int64_t N;        /* number of target documents (columns of c)             */
  int64_t nnz;      /* nonzeros of c                                         */
  int64_t U;        /* active vocabulary: words that occur in some document  */
  int32_t device;   /* CUDA device holding the corpus                        */
  size_t device_bytes; /* device memory held by the corpus                   */
  int32_t cdist_kernel; /* which kernel builds K for this corpus:
                           WMD_CDIST_TENSOR_CORES (tcgen05, the default) or
                           WMD_CDIST_CUDA_CORES (chosen by the options, or
                           because the tensor map of the vocabulary could not
                           be built)                                          */
} wmd_corpus_info;

#define WMD_CDIST_TENSOR_CORES 0
#define WMD_CDIST_CUDA_CORES 1

/* ---------------------------------------------------------------------------
 * Library options, given to wmd_corpus_load (NULL = the defaults that
 * wmd_options_default writes).  They configure the services around the
 * method, not the method itself.
 *
 * device            CUDA device ordinal that holds the corpus (default 0).
 * use_graphs        1 (default): wmd_query and wmd_query_batch capture their
 *                   kernel sequence into a CUDA graph on the second call of a
 *                   query shape and replay it afterwards; 0: always launch
 *                   the kernels one by one.
 * cdist_kernel      WMD_CDIST_TENSOR_CORES (default) or WMD_CDIST_CUDA_CORES
 *                   (the float32 FMA kernel; for comparison and for widths
 *                   the tensor-core kernel cannot hold).  The environment
 *                   variable WMD_CDIST_KERNEL=simt also selects it.
 * autotune_cache    path of a text file of tuned fused-loop tile variants
 *                   and partitions
 *                   (NULL: the environment variable WMD_AUTOTUNE_CACHE, else
 *                   no file).  wmd_corpus_load applies the entries recorded
 *                   for a corpus of the same shape (V, d, N, nnz, active
 *                   words); wmd_autotune appends its choice.  A missing or
 *                   unreadable file is ignored; a line that does not parse is
 *                   skipped.
 * wait_limit_cycles limit, in SM clock cycles, of each device-side wait of
 *                   the tensor-core cdist kernel between its roles (0: the
 *                   default, 4e9 cycles, about 2 s).  A wait that runs out
 *                   makes the query return WMD_ERR_TIMEOUT with NaN results;
 *                   the kernel still retires every copy and tensor-core
 *                   operation it issued before it returns.  Tests set it low
 *                   to exercise that path.
 * server            defaults of wmd_server_create(corpus, NULL, ...).
 * ------------------------------------------------------------------------- */
typedef struct wmd_server_options {
  int32_t max_batch;   /* most requests in one batch (default 64)              */
  int32_t slots;       /* batches in flight at once (default 2, at most 16)    */
  size_t mem_budget;   /* device bytes shared by all slots (default 8 GiB)     */
  int64_t max_pending; /* waiting requests before submit refuses (default 65536) */
} wmd_server_options;

typedef struct wmd_options {
  int32_t device;
  int32_t use_graphs;
  int32_t cdist_kernel;
  const char* autotune_cache;
  int64_t wait_limit_cycles;
  wmd_server_options server;
} wmd_options;

/* Writes the defaults listed above into *opt. */
void wmd_options_default(wmd_options* opt);

/* Thread-local description of the last failure in this thread ("" if none). */
const char* wmd_last_error(void);

/* Library version string. */
const char* wmd_version(void);

/* Measured FP32 fused multiply-add rate of GPU `device` in TFLOP/s (2 flops
 * per FMA), the roof of the fused Sinkhorn loop, which is bound by FP32
 * issue (Sec. 3's SDDMM and SpMM are one FMA per K element each).  packed = 0
 * times scalar FFMA, packed != 0 packed float2 FFMA2.  Runs a few launches of
 * a register-only kernel on a private stream of that device (about 10 ms in
 * all; the calling thread's current device is restored) and reports the
 * fastest.  *tflops is written on success only.  Errors: WMD_ERR_INVALID_ARG
 * (null tflops, device out of range), WMD_ERR_CUDA, WMD_ERR_OUT_OF_MEMORY is
 * reported as WMD_ERR_CUDA (4 bytes per CTA of scratch). */
wmd_status wmd_measure_fp32_peak(int32_t device, int32_t packed, double* tflops);

/* ---------------------------------------------------------------------------
 * Query compaction (Algorithm 1, the selection I = (r > 0)).  Host only, no GPU.
 * q_ids[n_q], q_w[n_q]: the sparse query r as (word id, weight) pairs, host.
 * Entries with weight 0 are dropped; the kept pairs are written, in input
 * order, to out_ids / out_w (host, capacity n_q each) and their count to
 * *out_vr.  Errors (WMD_ERR_INVALID_ARG): an id outside [0, V), a duplicate id
 * among the kept entries, a negative, NaN or infinite weight, n_q < 0.
 * WMD_ERR_UNSUPPORTED: more than WMD_MAX_VR kept entries.
 * ------------------------------------------------------------------------- */
wmd_status wmd_compact_query(const int32_t* q_ids, const float* q_w, int32_t n_q,
                             int64_t V, int32_t* out_ids, float* out_w,
                             int32_t* out_vr);

/* ---------------------------------------------------------------------------
 * Corpus load (Sec. 3 inputs `vecs` and `c`).  Host buffers, synchronous.
 * vecs:    V x d float32, row-major (row w = embedding of word w), host.
 * c:       the paper's V x N CSR with rows = words: row_ptr[V+1] (int64,
 *          row_ptr[0] = 0, non-decreasing, row_ptr[V] = nnz), doc_idx[nnz]
 *          (int32 document ids in [0, N), strictly increasing within a row),
 *          val[nnz] (float32, finite and > 0).  All host.
 * opt:     library options (device, graphs, cdist kernel, autotune cache,
 *          device wait limit, server defaults); NULL = wmd_options_default.
 * On success *out receives a corpus that keeps resident on the device, until
 * wmd_corpus_free: vecs (rows permuted so that words occurring in some
 * document come first), the row norms, the same rows as fp16 hi/lo pairs with
 * a power-of-two scale per row (the tensor-core cdist operands), a
 * document-major copy of c, and the fused loop's work items.
 * Errors: WMD_ERR_INVALID_ARG for any malformed input (checked on the host
 * before anything is copied), WMD_ERR_UNSUPPORTED for a document of 2^24 or
 * more distinct words, WMD_ERR_OUT_OF_MEMORY, WMD_ERR_CUDA.
 * ------------------------------------------------------------------------- */
wmd_status wmd_corpus_load(const float* vecs, int64_t V, int32_t d,
                           const int64_t* row_ptr, const int32_t* doc_idx,
                           const float* val, int64_t N, int64_t nnz,
                           const wmd_options* opt, wmd_corpus** out);

/* ---------------------------------------------------------------------------
 * Document sharding.  The paper parallelises the SDDMM_SpMM kernel by
 * splitting the documents (the columns of c) into ranges of about equal
 * nonzeros, one per thread and, across sockets, per socket (Sec. 3 and 4):
 * every column of x, u and v depends only on its own column of c, so the
 * ranges need no communication until the results are put together.  These
 * calls make that split across corpora (one per GPU, or several on one GPU).
 *
 * wmd_shard_plan: host only.  c as in wmd_corpus_load (host); S >= 1 shards.
 *   doc_begin[S + 1] (host) receives the boundaries: shard s holds documents
 *   [doc_begin[s], doc_begin[s + 1]), contiguous, each with about nnz / S
 *   nonzeros (a range may be empty when S is large).  WMD_ERR_INVALID_ARG
 *   for a malformed input.
 * wmd_corpus_load_shard: wmd_corpus_load of documents [doc_begin, doc_end)
 *   only, renumbered from 0 (document doc_begin + j of c is document j of
 *   the shard), with the whole vocabulary.  A shard's results equal the
 *   corresponding slice of the unsharded corpus's bit for bit when both use
 *   the same fused-loop tile variant and partition (wmd_set_loop_variant,
 *   wmd_set_loop_partition).  Errors as
 *   wmd_corpus_load, plus WMD_ERR_INVALID_ARG for a range outside [0, N].
 * The k nearest documents of the whole corpus are the k nearest among the
 * shards' own k nearest (ids shifted by doc_begin): wmd_topk over the
 * shards' candidate values concatenated in shard order returns them, since
 * that order is also ascending document order between equal values.
 * ------------------------------------------------------------------------- */
wmd_status wmd_shard_plan(const int64_t* row_ptr, const int32_t* doc_idx, int64_t V, int64_t N,
                          int32_t S, int64_t* doc_begin);
wmd_status wmd_corpus_load_shard(const float* vecs, int64_t V, int32_t d,
                                 const int64_t* row_ptr, const int32_t* doc_idx,
                                 const float* val, int64_t N, int64_t nnz, int64_t doc_begin,
                                 int64_t doc_end, const wmd_options* opt, wmd_corpus** out);

/* Frees a corpus (NULL is accepted).  The caller must not free a corpus that
 * a server or an in-flight device call still uses. */
void wmd_corpus_free(wmd_corpus* corpus);

wmd_status wmd_corpus_get_info(const wmd_corpus* corpus, wmd_corpus_info* out);

/* Changes the corpus's wait_limit_cycles (see wmd_options; 0 = the default)
 * for every later query, and drops the CUDA graphs captured with the old
 * limit.  Not thread-safe against queries running on this corpus or a server
 * using it. */
wmd_status wmd_corpus_set_wait_limit(wmd_corpus* corpus, int64_t cycles);

/* ---------------------------------------------------------------------------
 * One query, host buffers, synchronous (Sec. 3 `sinkhorn_wmd(r, c, vecs,
 * lamda, max_iter)`).  q_ids/q_w: sparse query as in wmd_compact_query (host).
 * out_wmd: host array of N doubles, WMD_j for every document j.
 * The call compacts and validates the query on the host into a pinned,
 * device-mapped staging block that the kernels read directly, and runs the
 * cdist/K build and the fused loop (from a captured CUDA graph from the
 * second call of a query shape on).  The loop kernel writes
 * the result straight into out_wmd when out_wmd is pinned host memory mapped
 * into the device's address space (cudaHostAlloc, or cudaHostRegister with
 * mapping), else into a pinned staging block that is then copied to out_wmd.
 * Calls on one corpus are serialised by an internal lock.
 * Errors: those of wmd_compact_query, WMD_ERR_INVALID_ARG for lambda <= 0 or
 * non-finite, max_iter < 0 or an empty query (v_r = 0), WMD_ERR_CUDA.
 * ------------------------------------------------------------------------- */
wmd_status wmd_query(wmd_corpus* corpus, const int32_t* q_ids, const float* q_w,
                     int32_t n_q, float lambda, int32_t max_iter,
                     wmd_precision prec, double* out_wmd);

/* ---------------------------------------------------------------------------
 * Device-resident path.  Stream ordered; nothing is synchronised.
 *
 * wmd_workspace_bytes: size of the caller-provided device workspace that the
 * calls below need for a query of v_r words (0 < v_r <= WMD_MAX_VR).
 *
 * d_q_ids[v_r], d_q_w[v_r]: the COMPACTED query on the device (ids in [0, V),
 * unique, weights > 0 -- e.g. the output of wmd_compact_query).  The kernels
 * never read outside the corpus for an out-of-range id: its column of K
 * becomes NaN and so does every result, but uniqueness is not re-checked.
 * d_ws: device workspace of at least wmd_workspace_bytes(...) bytes, 256-byte
 * aligned; it holds r, lambda and K between the two stages.
 * d_out: device-visible array of N doubles (device memory, or pinned host
 * memory mapped into the device's address space).
 * The loop kernel is launched as a programmatic dependent of the kernel
 * before it on the stream: it may start early, but reads nothing that
 * kernel (or anything before it) wrote, and writes d_out, only after it has
 * completed.
 *
 * wmd_build_kernel_matrix (Sec. 2 distance, Sec. 5 GEMM-type cdist,
 * Algorithm 1's K = exp(-lambda M)): K[w, i] for every active word w (a word
 * that occurs in some document), word-major (the "on the fly transpose" of
 * Sec. 3), plus the padded weights r and lambda, into d_ws.
 * wmd_sinkhorn_loop (Algorithm 1 loop and final reduction; the fused
 * SDDMM_SpMM kernel of Sec. 3): max_iter iterations plus the final reduction
 * for all N documents, reading K, r and lambda from the workspace that
 * wmd_build_kernel_matrix filled (same v_r and precision); K .* M of the
 * final step is recovered from K as K (-ln K) / lambda.
 * wmd_query_device: both stages.
 * ------------------------------------------------------------------------- */
size_t wmd_workspace_bytes(const wmd_corpus* corpus, int32_t v_r, wmd_precision prec);

wmd_status wmd_build_kernel_matrix(wmd_corpus* corpus, const int32_t* d_q_ids,
                                   const float* d_q_w, int32_t v_r, float lambda,
                                   wmd_precision prec, void* d_ws, size_t ws_bytes,
                                   void* stream);

wmd_status wmd_sinkhorn_loop(wmd_corpus* corpus, int32_t v_r, int32_t max_iter,
                             wmd_precision prec, void* d_ws, size_t ws_bytes,
                             double* d_out, void* stream);

wmd_status wmd_query_device(wmd_corpus* corpus, const int32_t* d_q_ids,
                            const float* d_q_w, int32_t v_r, float lambda,
                            int32_t max_iter, wmd_precision prec, void* d_ws,
                            size_t ws_bytes, double* d_out, void* stream);

/* ---------------------------------------------------------------------------
 * Convergence-tested query: Algorithm 1's loop condition "while x changes",
 * with max_iter as the cap that Sec. 3 puts on the loop.
 *
 * The test is taken per document j (every column of x depends only on its
 * own document): after loop body k has produced x^(k), document j stops when
 *     max_i |x^(k)_ij - x^(k-1)_ij| / x^(k-1)_ij <= tol       (i < v_r),
 * or when k = max_iter, and its WMD is then formed as after exactly k bodies
 * (u = 1/x^(k), one more SDDMM for v, the reduction).  x^(0) = 1/v_r.
 * The test runs in float32 on the GPU: a document whose relative change lies
 * within float32 rounding of tol may stop one body earlier or later than an
 * exact evaluation would.  An empty document never settles (x: 1/v_r, 0,
 * 0/0) and runs max_iter bodies (its WMD is NaN, as in wmd_query).
 *
 * Arguments as wmd_query_device (device pointers, the same workspace size
 * and layout, stream-ordered, asynchronous), plus:
 *   tol      in [0, 1); 0 stops a document only when x no longer changes at
 *            all in float32 (the result then equals wmd_query_device's).
 *   d_iters  device int32[N] or NULL: the number of loop bodies each
 *            document ran (1..max_iter, 0 when max_iter = 0).
 * Errors: WMD_ERR_INVALID_ARG for a tol outside [0, 1) or NaN, and every
 * error of wmd_query_device.
 * ------------------------------------------------------------------------- */
wmd_status wmd_query_device_tol(wmd_corpus* corpus, const int32_t* d_q_ids,
                                const float* d_q_w, int32_t v_r, float lambda,
                                int32_t max_iter, float tol, wmd_precision prec,
                                void* d_ws, size_t ws_bytes, double* d_out,
                                int32_t* d_iters, void* stream);

/* ---------------------------------------------------------------------------
 * k nearest documents.  The paper uses the WMD to find the documents closest
 * to a query (k-nearest-neighbour retrieval, Sec. 1 and 2): these calls return
 * the k smallest WMD values and their document ids.
 *
 * wmd_topk: selects from WMD[N] already on the device (d_wmd, e.g. the d_out
 *   of wmd_query_device).  Output, ascending by value: d_idx[k] (int64
 *   document ids) and d_val[k] (their WMD values, as stored in d_wmd).  Ties
 *   go to the lower document id, -0 equals +0, and NaN (empty documents)
 *   sorts after every number, so the result is unique.  Runs on the calling
 *   thread's current device, stream-ordered on `stream` (NULL = legacy
 *   default stream), asynchronous.  1 <= k <= min(N, 1024), else
 *   WMD_ERR_INVALID_ARG; k = 0 does nothing; N above 2^31 - 1 gives
 *   WMD_ERR_UNSUPPORTED.  Allocates nothing.  The selection runs in one CTA
 *   for N <= 16384, on a thread-block cluster of 16 (else 8) CTAs for N up
 *   to 262144 where the GPU can run such clusters, and in one CTA otherwise;
 *   it is launched as a programmatic dependent of the work before it on the
 *   stream and reads d_wmd only after that work has completed.
 * wmd_query_device_topk: wmd_query_device (same arguments; d_out receives
 *   all N values) followed by wmd_topk on its output, on the corpus's device.
 * ------------------------------------------------------------------------- */
wmd_status wmd_topk(const double* d_wmd, int64_t N, int32_t k, int64_t* d_idx, double* d_val,
                    void* stream);

wmd_status wmd_query_device_topk(wmd_corpus* corpus, const int32_t* d_q_ids,
                                 const float* d_q_w, int32_t v_r, float lambda,
                                 int32_t max_iter, wmd_precision prec, void* d_ws,
                                 size_t ws_bytes, double* d_out, int32_t k, int64_t* d_idx,
                                 double* d_val, void* stream);

/* ---------------------------------------------------------------------------
 * Dense Algorithm 1 on the GPU: a comparator for the sparse path.  Sec. 3
 * ("Dense to Sparse Kernel", Table 1) argues that the dense form spends its
 * time computing K^T u at every (word, document) position although only the
 * nonzeros of c are used.  These calls run that dense form literally, so the
 * argument can be measured on one GPU: per loop body S = K^T u (U x N),
 * v = c .* (1 ./ S), x = diag(1/r) K v, u = 1 ./ x; then the final update and
 * WMD_j = sum_i u_ij ((K .* M) v)_ij.  U is the corpus's active vocabulary
 * (the dense c is zero on every other word).  The two GEMMs per body are
 * cuBLAS SGEMM in FP32; the elementwise steps are this library's kernels.
 * K is the FP32 K of wmd_build_kernel_matrix; results match wmd_query_device
 * within the FP32 tolerance (summation order differs).
 *
 * wmd_dense_workspace_bytes: device bytes for a query of v_r words, 0 if v_r
 *   is out of range: 8 U N (dense c and S) + the query workspace + 8 VR N +
 *   4 VR U, each region 256-byte aligned.
 * wmd_dense_load_c: writes the dense U x N c (column j = document j) at the
 *   start of d_ws (asynchronous on `stream`).  Call once per workspace; the
 *   query calls read it and never write it.
 * wmd_query_dense: the dense Algorithm 1 for one query (device pointers as
 *   wmd_query_device, asynchronous on `stream`); d_out receives WMD[N].  The
 *   first call on a device creates a cuBLAS handle (allocates).  Errors:
 *   WMD_ERR_INVALID_ARG (arguments, max_iter < 0, workspace too small), WMD_ERR_UNSUPPORTED
 *   (U or N above 2^31 - 1), WMD_ERR_CUDA / WMD_ERR_OUT_OF_MEMORY from CUDA or
 *   cuBLAS.  Calls on one device are serialised by a lock while they enqueue.
 * ------------------------------------------------------------------------- */
size_t wmd_dense_workspace_bytes(const wmd_corpus* corpus, int32_t v_r);
wmd_status wmd_dense_load_c(wmd_corpus* corpus, void* d_ws, size_t ws_bytes, void* stream);
wmd_status wmd_query_dense(wmd_corpus* corpus, const int32_t* d_q_ids, const float* d_q_w,
                           int32_t v_r, float lambda, int32_t max_iter, void* d_ws,
                           size_t ws_bytes, double* d_out, void* stream);

/* ---------------------------------------------------------------------------
 * Tile variants of the fused loop and their autotuner.  Every query width
 * class (v_r rounded up to 8, 16, 32, 48, 64, 96, 128, 192 or 256: the
 * width of the loop's register tile; K itself is computed for v_r rounded up
 * to a power of two, and the 48-, 96- and 192-wide tiles read the first
 * columns of it) has one or more register-tile shapes for the fused
 * SDDMM/SpMM loop (same arithmetic, same results within rounding); they trade
 * work per cross-lane reduction against resident warps.  wmd_loop_width: the
 * class's tile width for queries of v_r words (the columns every SDDMM and
 * SpMM works on; 0 for v_r outside [1, WMD_MAX_VR]); host only, needs no GPU.
 * wmd_loop_variant_count: how many tile variants exist for queries of v_r
 * words.  wmd_set_loop_variant: use `variant` for v_r's class and `prec` on
 * this corpus (all later calls; not thread-safe against running queries).
 * wmd_get_loop_variant: the variant in use for v_r's class and `prec` (-1
 * for a NULL corpus, v_r out of range or an unknown precision).
 *
 * Partition (the paper's split of the documents over threads, Sec. 3, here
 * over warps): documents are taken in decreasing length and a document of n
 * words gets a team of W warps, the smallest power of two (up to the tile
 * variant's warps per CTA) with n <= W x rows_per_warp x fill / 100.
 * fill = 100 (the default) is the fewest warps that keep the document's K
 * block in registers; 75 and 50 spread documents over more warps; 200 gives
 * long documents half the warps, which then re-read chunks of K from L2
 * each pass.  The partition belongs to a class and tile variant (both
 * precisions).  wmd_set_loop_partition: rebuild the work items of v_r's
 * class and `variant` with `fill` (50, 75, 100 or 200; else
 * WMD_ERR_INVALID_ARG); waits for all work on the device first and drops
 * the corpus's captured CUDA graphs.  wmd_get_loop_partition: the fill in
 * use (-1 for a NULL corpus or an invalid class or variant).  Results of
 * different partitions agree within rounding (the sums across warps run in
 * another order).
 *
 * wmd_autotune: synchronous; builds K for the given query (host buffers, as
 * wmd_query), times every variant of its class with every partition on
 * this corpus with CUDA events, keeps the fastest partition for each
 * variant and the fastest variant for that class and precision, and writes
 * the variant's index to *chosen (may be NULL).  Allocates a temporary
 * workspace; waits for all work on the device first and drops the corpus's
 * captured CUDA graphs, and must not overlap other calls on the corpus.
 * With an autotune cache (wmd_options) the choice (variant and partition)
 * is appended to the cache file, and corpora of the same shape loaded later
 * start from it.
 * ------------------------------------------------------------------------- */
int32_t wmd_loop_width(int32_t v_r);
int32_t wmd_loop_variant_count(int32_t v_r);
wmd_status wmd_set_loop_variant(wmd_corpus* corpus, int32_t v_r, wmd_precision prec,
                                int32_t variant);
int32_t wmd_get_loop_variant(const wmd_corpus* corpus, int32_t v_r, wmd_precision prec);
wmd_status wmd_set_loop_partition(wmd_corpus* corpus, int32_t v_r, int32_t variant,
                                  int32_t fill);
int32_t wmd_get_loop_partition(const wmd_corpus* corpus, int32_t v_r, int32_t variant);
wmd_status wmd_autotune(wmd_corpus* corpus, const int32_t* q_ids, const float* q_w,
                        int32_t n_q, float lambda, int32_t max_iter, wmd_precision prec,
                        int32_t* chosen);

/* ---------------------------------------------------------------------------
 * Batched queries (many queries of uneven v_r, one resident corpus).  The
 * paper computes one query against many documents (Sec. 3); a batch is that
 * computation for every query, with each query's K block laid out next to the
 * others' and one fused-loop launch per query-width class covering every
 * (query, document) pair.  A query's results do not depend on the rest of the
 * batch (bit-identical to wmd_query).
 *
 * nq queries in CSR form: query q is q_ids[q_ptr[q] .. q_ptr[q+1]) with weights
 * q_w[...] (host; compacted and validated like wmd_compact_query), lambda[q]
 * its regulariser.  out: host, nq x N doubles, row-major (row q = query q).
 * Synchronous.  Repeated calls with the same shape (widths, lambdas,
 * max_iter, precision) replay a captured CUDA graph.  Errors: those of
 * wmd_query for any query, WMD_ERR_INVALID_ARG for a malformed q_ptr.
 * ------------------------------------------------------------------------- */
wmd_status wmd_query_batch(wmd_corpus* corpus, int32_t nq, const int64_t* q_ptr,
                           const int32_t* q_ids, const float* q_w, const float* lambda,
                           int32_t max_iter, wmd_precision prec, double* out);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching over a resident corpus.
 *
 * wmd_serve_submit copies and validates one query (host buffers, same rules
 * as wmd_query) and returns a ticket at once.  A scheduler thread owned by the
 * server admits waiting requests, oldest first, into batches whenever one of
 * its `slots` is free (a slot = one CUDA stream with its own buffers), up to
 * `max_batch` requests and the slot's share of `mem_budget` device bytes
 * (mem_budget / slots; a request needs 2 U VR sizeof(K) + 8 N bytes).  New
 * batches start while earlier ones still run on other streams.
 * wmd_serve_poll waits at most timeout_us for the ticket: WMD_OK (out_wmd,
 * host, N doubles, filled; the ticket is retired), WMD_ERR_NOT_READY
 * (timeout_us == 0 and not finished), WMD_ERR_TIMEOUT (timeout_us > 0 ran
 * out), or the request's own error; WMD_ERR_INVALID_ARG for an unknown ticket.
 * wmd_serve_cancel retires a ticket (a request already on the GPU finishes
 * and its result is dropped).  Submit answers WMD_ERR_OUT_OF_MEMORY for a
 * request larger than one slot's budget, WMD_ERR_NOT_READY when max_pending
 * requests already wait, WMD_ERR_SHUTDOWN during wmd_server_destroy.
 * wmd_server_destroy finishes the batches on the GPU, fails the requests
 * still waiting with WMD_ERR_SHUTDOWN and frees the server (not the corpus).
 * Device-side errors (WMD_ERR_TIMEOUT, WMD_ERR_RANGE) are kept per slot and
 * cleared before each batch: they fail the requests of that batch only.
 * ------------------------------------------------------------------------- */

typedef struct wmd_server_stats {
  int64_t submitted;
  int64_t completed;
  int64_t cancelled;
  int64_t batches;
  int64_t max_batch_seen;
  int64_t pending;
  int64_t in_flight_batches;
} wmd_server_stats;

/* opt: NULL for the defaults given to wmd_corpus_load (wmd_options.server). */
wmd_status wmd_server_create(wmd_corpus* corpus, const wmd_server_options* opt,
                             wmd_server** out);
wmd_status wmd_serve_submit(wmd_server* server, const int32_t* q_ids, const float* q_w,
                            int32_t n_q, float lambda, int32_t max_iter,
                            wmd_precision prec, uint64_t* ticket);
wmd_status wmd_serve_poll(wmd_server* server, uint64_t ticket, double* out_wmd,
                          int64_t timeout_us);
wmd_status wmd_serve_cancel(wmd_server* server, uint64_t ticket);
wmd_status wmd_server_get_stats(wmd_server* server, wmd_server_stats* out);
void wmd_server_destroy(wmd_server* server);

/* ---------------------------------------------------------------------------
 * Device-resident query that allocates nothing (the paper has no counterpart;
 * this is a service for callers that may not call cudaMalloc, e.g. because
 * their own memory manager already owns all device memory, or because an
 * allocation would synchronise the device in a latency-critical thread).
 *
 * Same computation, arguments and preconditions as wmd_query_device, without
 * d_ws: the workspace is a 16 MiB scratch array compiled into the library
 * (every GPU that loads the library holds it until the process exits).
 * Queries whose workspace (wmd_workspace_bytes) exceeds 16 MiB are rejected
 * with WMD_ERR_UNSUPPORTED.  wmd_corpus_load, which allocates anyway, looks
 * up the array's device address on the corpus's device, so the driver
 * reserves the array there at load time and this call itself never touches
 * the allocator; the call only reads that recorded address.  All calls share
 * the one array and each call overwrites what it reads (its error slots
 * included: every cdist CTA rewrites its own), so calls whose
 * kernels overlap on the GPU (different streams, or different corpora on the
 * same device) race and must be serialised by the caller.  Allocates no
 * memory: no cudaMalloc, no cudaFree.
 * ------------------------------------------------------------------------- */
wmd_status wmd_query_device_noalloc(wmd_corpus* corpus, const int32_t* d_q_ids,
                                    const float* d_q_w, int32_t v_r, float lambda,
                                    int32_t max_iter, wmd_precision prec,
                                    double* d_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* WMD_GB300_H */

// Host side of the C ABI: validation, corpus load, schedules and the query
// entry points.  All device work is done by the kernels in cdist.cu and
// sinkhorn.cu; nothing here computes a distance or a scaling vector.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include <cuda_fp16.h>

#include "wmd_internal.h"

namespace wmd {

namespace {
thread_local std::string g_last_error;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t count, size_t* bytes) {
  *dst = nullptr;
  size_t b = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), b);
  if (e != cudaSuccess) return e;
  *bytes += b;
  if (count) e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

void free_corpus_device(wmd_corpus* c) {
  cudaFree(c->vecs);
  cudaFree(c->norms);
  cudaFree(c->vecs_hi);
  cudaFree(c->vecs_lo);
  cudaFree(c->rscale);
  cudaFree(c->perm);
  cudaFree(c->doc_ptr);
  cudaFree(c->doc_words);
  cudaFree(c->doc_vals);
  for (auto& sc : c->sched)
    for (auto& s : sc) cudaFree(s.d_tasks);
  cudaFree(c->ws);
  cudaFreeHost(c->h_stage);
  cudaFreeHost(c->h_out);
  for (auto& g : c->qgraphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->qgraphs.clear();
  if (c->stream) cudaStreamDestroy(c->stream);
}

// ---------------------------------------------------------------- schedules
// The CTA work items of class `cls`, tile variant `var`, partition `fill`:
// documents in decreasing length, each with the smallest team allowed by
// the partition (see kFills); a CTA's NW / W teams take consecutive
// documents of one team size.  Replaces the class's previous schedule; the
// caller makes sure that no launch still reads it.
cudaError_t build_schedule(wmd_corpus* c, int cls, int var, int fill) {
  const std::vector<int64_t>& dptr = c->h_dptr;
  const std::vector<int32_t>& order = c->h_order;
  const int64_t N = c->N;
  const int64_t rpw = rows_per_warp(cls, var);
  const int nw = warps_per_cta(cls, var);
  auto team = [&](int64_t n) {
    int W = 1;
    while (W < nw && n * 100 > W * rpw * fill) W *= 2;
    return W;
  };
  std::vector<WarpTask> tasks;
  int32_t n_items = 0;
  int64_t i = 0;
  while (i < N) {
    const int W = team(dptr[order[i] + 1] - dptr[order[i]]);
    const int per = nw / W;
    int64_t j = i;
    while (j < N && team(dptr[order[j] + 1] - dptr[order[j]]) == W) ++j;
    for (int64_t b = i; b < j; b += per, ++n_items) {
      for (int warp = 0; warp < nw; ++warp) {
        const int64_t slot = b + warp / W;
        if (slot < std::min<int64_t>(b + per, j)) {
          const int32_t d = order[slot];
          const int32_t len = (int32_t)(dptr[d + 1] - dptr[d]);
          tasks.push_back(WarpTask{dptr[d], len | (W << kTaskWShift), d});
        } else {
          tasks.push_back(WarpTask{0, 0, 0});
        }
      }
    }
    i = j;
  }
  Schedule& sc = c->sched[cls][var];
  if (sc.d_tasks) {
    c->device_bytes -= std::max<size_t>(size_t(sc.n_items) * nw, 1) * sizeof(WarpTask);
    cudaFree(sc.d_tasks);
    sc.d_tasks = nullptr;
  }
  sc.n_items = n_items;
  sc.fill = fill;
  return upload(&sc.d_tasks, tasks.data(), tasks.size(), &c->device_bytes);
}

// Drops everything that captured a schedule's address: the host path's CUDA
// graphs and the batch path's cached graphs.
void drop_captured(wmd_corpus* c) {
  for (auto& g : c->qgraphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->qgraphs.clear();
  release_batch_state(c);
}

// ---------------------------------------------------------------- autotune cache
// One line per tuned choice: "wmd-loop V d N nnz U width precision variant
// fill" (width: the class's loop tile width, kClassVR; fill: the partition;
// lines without it mean 100).  A corpus applies the lines recorded for its
// own shape; the last one wins.
void load_autotune_cache(wmd_corpus* c) {
  if (c->autotune_cache.empty()) return;
  FILE* f = std::fopen(c->autotune_cache.c_str(), "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    long long V, N, nnz, U;
    int d, width, prec, var, fill = 100;
    const int got = std::sscanf(line, "wmd-loop %lld %d %lld %lld %lld %d %d %d %d", &V, &d, &N,
                                &nnz, &U, &width, &prec, &var, &fill);
    if (got != 8 && got != 9) continue;  // lines without a partition keep fill = 100
    if (V != c->V || d != c->d || N != c->N || nnz != c->nnz || U != c->U) continue;
    const int cls = class_of_width(width);
    if (cls < 0 || prec < 0 || prec > 1 || var < 0 ||
        var >= kClassVariants[cls] || !valid_fill(fill))
      continue;
    c->loop_variant[cls][prec] = var;
    if (c->sched[cls][var].fill != fill && build_schedule(c, cls, var, fill) != cudaSuccess) break;
  }
  std::fclose(f);
}

void save_autotune_choice(const wmd_corpus* c, int cls, int prec, int var) {
  if (c->autotune_cache.empty()) return;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  FILE* f = std::fopen(c->autotune_cache.c_str(), "a");
  if (!f) return;
  std::fprintf(f, "wmd-loop %lld %d %lld %lld %lld %d %d %d %d\n", (long long)c->V, (int)c->d,
               (long long)c->N, (long long)c->nnz, (long long)c->U, kClassVR[cls], prec, var,
               (int)c->sched[cls][var].fill);
  std::fclose(f);
}

wmd_status check_query_args(const wmd_corpus* c, int v_r, float lambda, int T) {
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  if (v_r <= 0) return set_error(WMD_ERR_INVALID_ARG, "query has no word with positive weight");
  if (v_r > WMD_MAX_VR) return set_error(WMD_ERR_UNSUPPORTED, "v_r exceeds WMD_MAX_VR");
  if (!(lambda > 0.f) || !std::isfinite(lambda))
    return set_error(WMD_ERR_INVALID_ARG, "lambda must be positive and finite");
  if (T < 0) return set_error(WMD_ERR_INVALID_ARG, "max_iter must be >= 0");
  return WMD_OK;
}

wmd_status check_ws(const wmd_corpus* c, int v_r, wmd_precision prec, const void* ws,
                    size_t ws_bytes) {
  if (prec != WMD_PREC_FP32 && prec != WMD_PREC_BF16_K)
    return set_error(WMD_ERR_INVALID_ARG, "unknown precision");
  if (!ws) return set_error(WMD_ERR_INVALID_ARG, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256)
    return set_error(WMD_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  const WsLayout L = ws_layout(c, kClassKVR[vr_class(v_r)], prec);
  if (ws_bytes < L.total) return set_error(WMD_ERR_INVALID_ARG, "workspace too small");
  return WMD_OK;
}

}  // namespace

wmd_status set_error(wmd_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

wmd_status cuda_error(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? WMD_ERR_OUT_OF_MEMORY : WMD_ERR_CUDA;
}

wmd_status device_error(int err) {
  if (err & 0x40000000) {
    static const char* roles[] = {"?", "producer (stage free)", "?",
                                  "MMA (accumulator free)", "MMA (tile landed)",
                                  "epilogue (accumulator full)", "?",
                                  "producer (query gathers in flight)"};
    const int role = (err >> 24) & 0x3f;
    char msg[160];
    std::snprintf(msg, sizeof msg,
                  "a device-side wait in the cdist kernel timed out: %s, iteration %d (code 0x%08x)",
                  roles[role < 8 ? role : 0], err & 0xffffff, (unsigned)err);
    return set_error(WMD_ERR_TIMEOUT, msg);
  }
  if (err & kRangeFlag)
    return set_error(WMD_ERR_RANGE,
                     "lambda * M reached 87.3 for some query word and vocabulary word: "
                     "K = exp(-lambda M) leaves the float32 range (lower lambda)");
  return WMD_OK;
}

WsLayout ws_layout(const wmd_corpus* c, int VR, wmd_precision prec) {
  WsLayout L;
  size_t o = 0;
  L.r_off = o;                                        // r, lambda, scale
  L.err_off = o + (size_t)(VR + 4) * sizeof(float);   // error slots
  L.n_err = cdist_err_slots(c, VR);
  o = align_up(L.err_off + (size_t)L.n_err * sizeof(int), 256);
  const size_t kelem = prec == WMD_PREC_BF16_K ? 2 : 4;
  const size_t kbytes = align_up((size_t)std::max<int64_t>(c->U, 1) * VR * kelem, 256);
  L.k_off = o;
  o += kbytes;
  L.total = o;
  return L;
}

}  // namespace wmd

using namespace wmd;

extern "C" {

const char* wmd_last_error(void) { return g_last_error.c_str(); }

const char* wmd_version(void) { return "wmd-gb300 0.2 (sm_103a)"; }

void wmd_options_default(wmd_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->device = 0;
  opt->use_graphs = 1;
  opt->cdist_kernel = WMD_CDIST_TENSOR_CORES;
  opt->autotune_cache = nullptr;
  opt->wait_limit_cycles = 0;
  opt->server.max_batch = 64;
  opt->server.slots = 2;
  opt->server.mem_budget = size_t(8) << 30;
  opt->server.max_pending = 65536;
}

wmd_status wmd_compact_query(const int32_t* q_ids, const float* q_w, int32_t n_q, int64_t V,
                             int32_t* out_ids, float* out_w, int32_t* out_vr) {
  if (n_q < 0) return set_error(WMD_ERR_INVALID_ARG, "n_q < 0");
  if (!out_vr || (n_q > 0 && (!q_ids || !q_w || !out_ids || !out_w)))
    return set_error(WMD_ERR_INVALID_ARG, "NULL pointer");
  int32_t k = 0;
  std::vector<int32_t> seen;
  seen.reserve(n_q);
  for (int32_t i = 0; i < n_q; ++i) {
    const float w = q_w[i];
    if (!std::isfinite(w) || w < 0.f)
      return set_error(WMD_ERR_INVALID_ARG, "query weight " + std::to_string(i) + " is negative or not finite");
    if (q_ids[i] < 0 || q_ids[i] >= V)
      return set_error(WMD_ERR_INVALID_ARG, "query id " + std::to_string(q_ids[i]) + " outside [0, V)");
    if (w == 0.f) continue;  // I = (r > 0)
    seen.push_back(q_ids[i]);
    out_ids[k] = q_ids[i];
    out_w[k] = w;
    ++k;
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
    return set_error(WMD_ERR_INVALID_ARG, "duplicate query word id");
  *out_vr = k;
  if (k > WMD_MAX_VR) return set_error(WMD_ERR_UNSUPPORTED, "more than WMD_MAX_VR query words");
  return WMD_OK;
}

wmd_status wmd_corpus_load(const float* vecs, int64_t V, int32_t d, const int64_t* row_ptr,
                           const int32_t* doc_idx, const float* val, int64_t N, int64_t nnz,
                           const wmd_options* opt, wmd_corpus** out) {
  wmd::NvtxRange nvtx_range("wmd_corpus_load");
  if (!out) return set_error(WMD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  wmd_options o;
  wmd_options_default(&o);
  if (opt) o = *opt;
  if (o.device < 0) return set_error(WMD_ERR_INVALID_ARG, "device ordinal < 0");
  if (o.cdist_kernel != WMD_CDIST_TENSOR_CORES && o.cdist_kernel != WMD_CDIST_CUDA_CORES)
    return set_error(WMD_ERR_INVALID_ARG, "unknown cdist kernel");
  if (o.wait_limit_cycles < 0) return set_error(WMD_ERR_INVALID_ARG, "wait_limit_cycles < 0");
  if (o.server.max_batch <= 0 || o.server.slots <= 0 || o.server.slots > 16 ||
      o.server.mem_budget == 0 || o.server.max_pending <= 0)
    return set_error(WMD_ERR_INVALID_ARG, "server options out of range");
  const int32_t device = o.device;
  if (V <= 0 || V > INT32_MAX) return set_error(WMD_ERR_INVALID_ARG, "V must be in [1, 2^31)");
  if (d <= 0) return set_error(WMD_ERR_INVALID_ARG, "d must be positive");
  if (N < 0 || N > INT32_MAX) return set_error(WMD_ERR_INVALID_ARG, "N must be in [0, 2^31)");
  if (nnz < 0) return set_error(WMD_ERR_INVALID_ARG, "nnz < 0");
  if (!vecs || !row_ptr || (nnz > 0 && (!doc_idx || !val)))
    return set_error(WMD_ERR_INVALID_ARG, "NULL input pointer");
  if (row_ptr[0] != 0 || row_ptr[V] != nnz)
    return set_error(WMD_ERR_INVALID_ARG, "row_ptr must start at 0 and end at nnz");
  for (int64_t w = 0; w < V; ++w) {
    if (row_ptr[w + 1] < row_ptr[w]) return set_error(WMD_ERR_INVALID_ARG, "row_ptr decreases");
    for (int64_t e = row_ptr[w]; e < row_ptr[w + 1]; ++e) {
      if (doc_idx[e] < 0 || doc_idx[e] >= N)
        return set_error(WMD_ERR_INVALID_ARG, "doc_idx outside [0, N)");
      if (e > row_ptr[w] && doc_idx[e] <= doc_idx[e - 1])
        return set_error(WMD_ERR_INVALID_ARG, "doc_idx not strictly increasing within a row");
      if (!(val[e] > 0.f) || !std::isfinite(val[e]))
        return set_error(WMD_ERR_INVALID_ARG, "c values must be finite and > 0");
    }
  }
  for (int64_t i = 0; i < V * (int64_t)d; ++i)
    if (!std::isfinite(vecs[i])) return set_error(WMD_ERR_INVALID_ARG, "vecs holds a non-finite value");

  wmd_corpus* c = new (std::nothrow) wmd_corpus();
  if (!c) return set_error(WMD_ERR_OUT_OF_MEMORY, "host allocation failed");
  c->device = device;
  c->use_graphs = o.use_graphs != 0;
  c->wait_cycles = o.wait_limit_cycles;
  c->server_defaults = o.server;
  if (o.autotune_cache) {
    c->autotune_cache = o.autotune_cache;
  } else if (const char* env = std::getenv("WMD_AUTOTUNE_CACHE")) {
    c->autotune_cache = env;
  }
  c->V = V;
  c->N = N;
  c->nnz = nnz;
  c->d = d;
  // rows padded to 32 elements: 128-byte float32 rows for the CUDA-core
  // cdist, and 16-byte aligned fp16 rows (64-byte strides) for the TMA tiles
  // of the tensor-core cdist
  c->ldv = (int32_t)align_up((size_t)d, 32);

  // active vocabulary first: device row of word w
  std::vector<int32_t> perm(V);
  int64_t U = 0;
  for (int64_t w = 0; w < V; ++w)
    if (row_ptr[w + 1] > row_ptr[w]) perm[w] = (int32_t)U++;
  int64_t nxt = U;
  for (int64_t w = 0; w < V; ++w)
    if (row_ptr[w + 1] == row_ptr[w]) perm[w] = (int32_t)nxt++;
  c->U = U;

  // permuted, padded embeddings and their squared norms (float64 sums)
  std::vector<float> hv((size_t)V * c->ldv, 0.f);
  std::vector<float> hn(V);
  for (int64_t w = 0; w < V; ++w) {
    const float* src = vecs + (size_t)w * d;
    float* dst = hv.data() + (size_t)perm[w] * c->ldv;
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
      dst[k] = src[k];
      s += (double)src[k] * (double)src[k];
    }
    hn[perm[w]] = (float)s;
  }

  // fp16 pair of every row for the tensor-core cdist: scale the row by 2^e so
  // that its largest magnitude lies in [2^14, 2^15) (exact), hi = fp16(x),
  // lo = fp16((x - hi) * 2^11) (x - hi is exact in float32); the dropped part
  // is below 2^-22 of the row's largest entry.  Host arithmetic only, so the
  // pair is the same on every machine.
  std::vector<uint16_t> hhi((size_t)V * c->ldv, 0), hlo((size_t)V * c->ldv, 0);
  std::vector<float> hrs(V, 1.f);
  auto split_rows = [&](int64_t r0, int64_t r1) {
    for (int64_t r = r0; r < r1; ++r) {
      const float* x = hv.data() + (size_t)r * c->ldv;
      float mx = 0.f;
      for (int k = 0; k < d; ++k) mx = std::max(mx, std::fabs(x[k]));
      int ex = 0;
      if (mx > 0.f) std::frexp(mx, &ex);  // mx < 2^ex
      const int e = std::min(120, std::max(-120, 15 - ex));
      hrs[r] = std::ldexp(1.f, -e);
      for (int k = 0; k < d; ++k) {
        const float xs = std::ldexp(x[k], e);
        const __half h = __float2half_rn(xs);
        const float rem = (xs - __half2float(h)) * 2048.f;
        const __half l = __float2half_rn(rem);
        hhi[(size_t)r * c->ldv + k] = __half_as_ushort(h);
        hlo[(size_t)r * c->ldv + k] = __half_as_ushort(l);
      }
    }
  };
  {
    const int64_t nt = std::max<int64_t>(
        1, std::min<int64_t>({16, (int64_t)std::thread::hardware_concurrency(), V / 4096 + 1}));
    std::vector<std::thread> pool;
    for (int64_t t = 1; t < nt; ++t) pool.emplace_back(split_rows, V * t / nt, V * (t + 1) / nt);
    split_rows(0, V / nt);
    for (auto& th : pool) th.join();
  }

  // document-major copy of c (CSR of c^T), words as device rows
  std::vector<int64_t> dptr(N + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) dptr[doc_idx[e] + 1]++;
  for (int64_t j = 0; j < N; ++j) dptr[j + 1] += dptr[j];
  std::vector<int64_t> fill(dptr.begin(), dptr.end() - 1);
  std::vector<int32_t> dwords(nnz);
  std::vector<float> dvals(nnz);
  for (int64_t w = 0; w < V; ++w)
    for (int64_t e = row_ptr[w]; e < row_ptr[w + 1]; ++e) {
      const int64_t pos = fill[doc_idx[e]]++;
      dwords[pos] = perm[w];
      dvals[pos] = val[e];
    }

  for (int64_t j = 0; j < N; ++j)
    if (dptr[j + 1] - dptr[j] >= (int64_t(1) << kTaskWShift)) {
      delete c;
      return set_error(WMD_ERR_UNSUPPORTED, "a document has 2^24 or more distinct words");
    }

  // documents by decreasing length (longest first), ties by id
  std::vector<int32_t> order(N);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return (dptr[a + 1] - dptr[a]) > (dptr[b + 1] - dptr[b]);
  });

  DeviceGuard g(device);
  cudaError_t e = cudaSetDevice(device);
  size_t bytes = 0;
  if (e == cudaSuccess) e = upload(&c->vecs, hv.data(), hv.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->norms, hn.data(), hn.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->vecs_hi, hhi.data(), hhi.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->vecs_lo, hlo.data(), hlo.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->rscale, hrs.data(), hrs.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->perm, perm.data(), perm.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->doc_ptr, dptr.data(), dptr.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->doc_words, dwords.data(), dwords.size(), &bytes);
  if (e == cudaSuccess) e = upload(&c->doc_vals, dvals.data(), dvals.size(), &bytes);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    // the options (or WMD_CDIST_KERNEL=simt, used by the tests that compare
    // both kernels) keep cdist on the CUDA cores; otherwise the tensor-core
    // kernel is used wherever its tensor map can be built
    const char* kern = std::getenv("WMD_CDIST_KERNEL");
    const bool simt = o.cdist_kernel == WMD_CDIST_CUDA_CORES || (kern && std::strcmp(kern, "simt") == 0);
    c->tmap_ok = !simt && make_vecs_tensor_map(c);
  }
  // the no-allocation entry point's scratch array is reserved now, while
  // allocating is allowed anyway (its first query then allocates nothing)
  if (e == cudaSuccess) e = noalloc_reserve(device);

  // per query-width class and tile variant: the CTA work items of the
  // default partition (fill = 100)
  c->device_bytes = bytes;
  c->h_dptr = std::move(dptr);
  c->h_order = std::move(order);
  for (int cls = 0; cls < kNumClasses && e == cudaSuccess; ++cls)
    for (int var = 0; var < kClassVariants[cls] && e == cudaSuccess; ++var)
      e = build_schedule(c, cls, var, 100);
  if (e != cudaSuccess) {
    wmd_status st = cuda_error(e, "corpus upload");
    free_corpus_device(c);
    delete c;
    return st;
  }
  load_autotune_cache(c);
  *out = c;
  return WMD_OK;
}

wmd_status wmd_shard_plan(const int64_t* row_ptr, const int32_t* doc_idx, int64_t V, int64_t N,
                          int32_t S, int64_t* doc_begin) {
  if (!row_ptr || !doc_begin || V <= 0 || N < 0 || S <= 0)
    return set_error(WMD_ERR_INVALID_ARG, "shard plan: bad arguments");
  const int64_t nnz = row_ptr[V];
  if (nnz < 0 || (nnz > 0 && !doc_idx)) return set_error(WMD_ERR_INVALID_ARG, "shard plan: bad CSR");
  // nonzeros per document (the SDDMM/SpMM work of a document is its length
  // times v_r, so equal nonzeros mean equal work, as in Sec. 3's split)
  std::vector<int64_t> pre(N + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) {
    const int64_t j = doc_idx[e];
    if (j < 0 || j >= N) return set_error(WMD_ERR_INVALID_ARG, "shard plan: doc_idx outside [0, N)");
    pre[j + 1]++;
  }
  for (int64_t j = 0; j < N; ++j) pre[j + 1] += pre[j];
  // boundary s: the first document whose prefix reaches s nnz / S (rounded to
  // the nearer side), never before the previous boundary
  doc_begin[0] = 0;
  for (int32_t sh = 1; sh < S; ++sh) {
    const double target = (double)nnz * sh / S;
    int64_t j = std::lower_bound(pre.begin(), pre.end(), (int64_t)std::ceil(target)) - pre.begin();
    if (j > 0 && j <= N && target - pre[j - 1] < pre[j] - target) --j;
    doc_begin[sh] = std::min<int64_t>(N, std::max<int64_t>(doc_begin[sh - 1], j));
  }
  doc_begin[S] = N;
  return WMD_OK;
}

wmd_status wmd_corpus_load_shard(const float* vecs, int64_t V, int32_t d, const int64_t* row_ptr,
                                 const int32_t* doc_idx, const float* val, int64_t N, int64_t nnz,
                                 int64_t doc_begin, int64_t doc_end, const wmd_options* opt,
                                 wmd_corpus** out) {
  wmd::NvtxRange nvtx_range("wmd_corpus_load_shard");
  if (!out) return set_error(WMD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (V <= 0 || V > INT32_MAX || !row_ptr || nnz < 0 || (nnz > 0 && (!doc_idx || !val)))
    return set_error(WMD_ERR_INVALID_ARG, "shard load: bad CSR arguments");
  if (N < 0 || doc_begin < 0 || doc_end < doc_begin || doc_end > N)
    return set_error(WMD_ERR_INVALID_ARG, "shard load: document range outside [0, N]");
  if (row_ptr[0] != 0 || row_ptr[V] != nnz)
    return set_error(WMD_ERR_INVALID_ARG, "row_ptr must start at 0 and end at nnz");
  // the shard's V x (doc_end - doc_begin) CSR: every word row keeps its
  // entries inside the range, documents renumbered from 0 (the full
  // validation happens in wmd_corpus_load)
  std::vector<int64_t> rp(V + 1, 0);
  std::vector<int32_t> di;
  std::vector<float> vv;
  for (int64_t w = 0; w < V; ++w) {
    if (row_ptr[w + 1] < row_ptr[w]) return set_error(WMD_ERR_INVALID_ARG, "row_ptr decreases");
    for (int64_t e = row_ptr[w]; e < row_ptr[w + 1]; ++e) {
      const int64_t j = doc_idx[e];
      if (j >= doc_begin && j < doc_end) {
        di.push_back((int32_t)(j - doc_begin));
        vv.push_back(val[e]);
      }
    }
    rp[w + 1] = (int64_t)di.size();
  }
  return wmd_corpus_load(vecs, V, d, rp.data(), di.data(), vv.data(), doc_end - doc_begin,
                         (int64_t)di.size(), opt, out);
}

void wmd_corpus_free(wmd_corpus* c) {
  if (!c) return;
  release_batch_state(c);
  {
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_corpus_device(c);
  }
  delete c;
}

wmd_status wmd_corpus_set_wait_limit(wmd_corpus* c, int64_t cycles) {
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  if (cycles < 0) return set_error(WMD_ERR_INVALID_ARG, "wait limit < 0");
  std::lock_guard<std::mutex> lock(c->mu);
  DeviceGuard g(c->device);
  // captured sequences hold the old limit in their kernel parameters
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& q : c->qgraphs)
    if (q.exec) cudaGraphExecDestroy(q.exec);
  c->qgraphs.clear();
  release_batch_state(c);
  c->wait_cycles = cycles;
  return WMD_OK;
}

wmd_status wmd_corpus_get_info(const wmd_corpus* c, wmd_corpus_info* out) {
  if (!c || !out) return set_error(WMD_ERR_INVALID_ARG, "NULL pointer");
  out->V = c->V;
  out->d = c->d;
  out->N = c->N;
  out->nnz = c->nnz;
  out->U = c->U;
  out->device = c->device;
  out->device_bytes = c->device_bytes;
  out->cdist_kernel = cdist_tc_max_width(c) > 0 ? WMD_CDIST_TENSOR_CORES : WMD_CDIST_CUDA_CORES;
  return WMD_OK;
}

size_t wmd_workspace_bytes(const wmd_corpus* c, int32_t v_r, wmd_precision prec) {
  if (!c || v_r <= 0 || v_r > WMD_MAX_VR) return 0;
  return ws_layout(c, kClassKVR[vr_class(v_r)], prec).total;
}

wmd_status wmd_build_kernel_matrix(wmd_corpus* c, const int32_t* d_q_ids, const float* d_q_w,
                                   int32_t v_r, float lambda, wmd_precision prec, void* d_ws,
                                   size_t ws_bytes, void* stream) {
  wmd::NvtxRange nvtx_range("K1 cdist + K");
  wmd_status st = check_query_args(c, v_r, lambda, 0);
  if (st != WMD_OK) return st;
  if (!d_q_ids || !d_q_w) return set_error(WMD_ERR_INVALID_ARG, "NULL query pointer");
  if ((st = check_ws(c, v_r, prec, d_ws, ws_bytes)) != WMD_OK) return st;
  DeviceGuard g(c->device);
  const int VR = kClassKVR[vr_class(v_r)];
  const WsLayout L = ws_layout(c, VR, prec);
  char* ws = static_cast<char*>(d_ws);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* r = reinterpret_cast<float*>(ws + L.r_off);
  int* err = reinterpret_cast<int*>(ws + L.err_off);
  const L2Prefetch pf = loop_inputs(c, vr_class(v_r), prec);
  WMD_CUDA_TRY(launch_cdist(c, d_q_ids, d_q_w, v_r, VR, lambda, prec, ws + L.k_off, VR, 0, r,
                            r + VR, err, &pf, s));
  return WMD_OK;
}

namespace {

// The fused loop of wmd_sinkhorn_loop; err_out (optional, device-visible)
// receives the cdist timeout word.
wmd_status sinkhorn_loop(wmd_corpus* c, int32_t v_r, int32_t max_iter, wmd_precision prec,
                         void* d_ws, size_t ws_bytes, double* d_out, int* err_out, void* stream) {
  wmd_status st = check_query_args(c, v_r, 1.f, max_iter);
  if (st != WMD_OK) return st;
  if (!d_out && c->N > 0) return set_error(WMD_ERR_INVALID_ARG, "d_out is NULL");
  if ((st = check_ws(c, v_r, prec, d_ws, ws_bytes)) != WMD_OK) return st;
  DeviceGuard g(c->device);
  const int cls = vr_class(v_r);
  const int VR = kClassKVR[cls];
  const WsLayout L = ws_layout(c, VR, prec);
  char* ws = static_cast<char*>(d_ws);
  const float* r = reinterpret_cast<const float*>(ws + L.r_off);
  const int* err = reinterpret_cast<const int*>(ws + L.err_off);
  WMD_CUDA_TRY(launch_loop(c, cls, ws + L.k_off, VR, 0, r, r + VR, v_r, max_iter, prec, d_out,
                           err, L.n_err, err_out, static_cast<cudaStream_t>(stream)));
  return WMD_OK;
}

}  // namespace

wmd_status wmd_sinkhorn_loop(wmd_corpus* c, int32_t v_r, int32_t max_iter, wmd_precision prec,
                             void* d_ws, size_t ws_bytes, double* d_out, void* stream) {
  wmd::NvtxRange nvtx_range("K2+K3 fused loop");
  return sinkhorn_loop(c, v_r, max_iter, prec, d_ws, ws_bytes, d_out, nullptr, stream);
}

wmd_status wmd_query_device(wmd_corpus* c, const int32_t* d_q_ids, const float* d_q_w,
                            int32_t v_r, float lambda, int32_t max_iter, wmd_precision prec,
                            void* d_ws, size_t ws_bytes, double* d_out, void* stream) {
  wmd::NvtxRange nvtx_range("wmd_query_device");
  wmd_status st = check_query_args(c, v_r, lambda, max_iter);
  if (st != WMD_OK) return st;
  // every argument is checked before the first launch, so that a refused call
  // writes nothing (not even the workspace)
  if (!d_out && c->N > 0) return set_error(WMD_ERR_INVALID_ARG, "d_out is NULL");
  if (!d_q_ids || !d_q_w) return set_error(WMD_ERR_INVALID_ARG, "NULL query pointer");
  if ((st = check_ws(c, v_r, prec, d_ws, ws_bytes)) != WMD_OK) return st;
  st = wmd_build_kernel_matrix(c, d_q_ids, d_q_w, v_r, lambda, prec, d_ws, ws_bytes, stream);
  if (st != WMD_OK) return st;
  return wmd_sinkhorn_loop(c, v_r, max_iter, prec, d_ws, ws_bytes, d_out, stream);
}

wmd_status wmd_query_device_tol(wmd_corpus* c, const int32_t* d_q_ids, const float* d_q_w,
                                int32_t v_r, float lambda, int32_t max_iter, float tol,
                                wmd_precision prec, void* d_ws, size_t ws_bytes, double* d_out,
                                int32_t* d_iters, void* stream) {
  wmd::NvtxRange nvtx_range("wmd_query_device_tol");
  wmd_status st = check_query_args(c, v_r, lambda, max_iter);
  if (st != WMD_OK) return st;
  if (!(tol >= 0.f && tol < 1.f)) return set_error(WMD_ERR_INVALID_ARG, "tol must lie in [0, 1)");
  if (!d_out && c->N > 0) return set_error(WMD_ERR_INVALID_ARG, "d_out is NULL");
  if (!d_q_ids || !d_q_w) return set_error(WMD_ERR_INVALID_ARG, "NULL query pointer");
  if ((st = check_ws(c, v_r, prec, d_ws, ws_bytes)) != WMD_OK) return st;
  st = wmd_build_kernel_matrix(c, d_q_ids, d_q_w, v_r, lambda, prec, d_ws, ws_bytes, stream);
  if (st != WMD_OK) return st;
  DeviceGuard g(c->device);
  const int cls = vr_class(v_r);
  const int VR = kClassKVR[cls];
  const WsLayout L = ws_layout(c, VR, prec);
  char* ws = static_cast<char*>(d_ws);
  const float* r = reinterpret_cast<const float*>(ws + L.r_off);
  const int* err = reinterpret_cast<const int*>(ws + L.err_off);
  WMD_CUDA_TRY(launch_loop_conv(c, cls, ws + L.k_off, VR, r, r + VR, v_r, max_iter, tol, prec,
                                d_out, d_iters, err, L.n_err, static_cast<cudaStream_t>(stream)));
  return WMD_OK;
}

wmd_status wmd_topk(const double* d_wmd, int64_t N, int32_t k, int64_t* d_idx, double* d_val,
                    void* stream) {
  wmd::NvtxRange nvtx_range("wmd_topk");
  if (k == 0) return WMD_OK;
  if (N < 0 || k < 0 || k > N || k > kTopkMaxK)
    return set_error(WMD_ERR_INVALID_ARG, "k must satisfy 0 <= k <= min(N, 1024)");
  if (!d_wmd || !d_idx || !d_val) return set_error(WMD_ERR_INVALID_ARG, "NULL pointer");
  if (N > INT32_MAX) return set_error(WMD_ERR_UNSUPPORTED, "N above 2^31 - 1");
  WMD_CUDA_TRY(launch_topk(d_wmd, N, k, d_idx, d_val, static_cast<cudaStream_t>(stream)));
  return WMD_OK;
}

wmd_status wmd_query_device_topk(wmd_corpus* c, const int32_t* d_q_ids, const float* d_q_w,
                                 int32_t v_r, float lambda, int32_t max_iter, wmd_precision prec,
                                 void* d_ws, size_t ws_bytes, double* d_out, int32_t k,
                                 int64_t* d_idx, double* d_val, void* stream) {
  wmd::NvtxRange nvtx_range("wmd_query_device_topk");
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  if (k < 0 || k > c->N || k > kTopkMaxK)
    return set_error(WMD_ERR_INVALID_ARG, "k must satisfy 0 <= k <= min(N, 1024)");
  if (k > 0 && (!d_idx || !d_val)) return set_error(WMD_ERR_INVALID_ARG, "NULL output pointer");
  wmd_status st = wmd_query_device(c, d_q_ids, d_q_w, v_r, lambda, max_iter, prec, d_ws, ws_bytes,
                                   d_out, stream);
  if (st != WMD_OK) return st;
  DeviceGuard g(c->device);
  return wmd_topk(d_out, c->N, k, d_idx, d_val, stream);
}

int32_t wmd_loop_width(int32_t v_r) {
  const int cls = v_r > 0 && v_r <= WMD_MAX_VR ? vr_class(v_r) : -1;
  return cls >= 0 ? kClassVR[cls] : 0;
}

int32_t wmd_loop_variant_count(int32_t v_r) {
  const int cls = vr_class(v_r);
  return v_r > 0 && cls >= 0 ? kClassVariants[cls] : 0;
}

wmd_status wmd_set_loop_variant(wmd_corpus* c, int32_t v_r, wmd_precision prec, int32_t variant) {
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  const int cls = v_r > 0 ? vr_class(v_r) : -1;
  if (cls < 0) return set_error(WMD_ERR_INVALID_ARG, "v_r out of range");
  if (prec != WMD_PREC_FP32 && prec != WMD_PREC_BF16_K)
    return set_error(WMD_ERR_INVALID_ARG, "unknown precision");
  if (variant < 0 || variant >= kClassVariants[cls])
    return set_error(WMD_ERR_INVALID_ARG, "no such variant for this query width");
  c->loop_variant[cls][prec == WMD_PREC_BF16_K] = variant;
  return WMD_OK;
}

wmd_status wmd_set_loop_partition(wmd_corpus* c, int32_t v_r, int32_t variant, int32_t fill) {
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  const int cls = v_r > 0 ? vr_class(v_r) : -1;
  if (cls < 0) return set_error(WMD_ERR_INVALID_ARG, "v_r out of range");
  if (variant < 0 || variant >= kClassVariants[cls])
    return set_error(WMD_ERR_INVALID_ARG, "no such variant for this query width");
  if (!valid_fill(fill)) return set_error(WMD_ERR_INVALID_ARG, "fill must be 50, 75, 100 or 200");
  if (c->sched[cls][variant].fill == fill) return WMD_OK;
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lock(c->mu);
  // the old work items may still be read by launches in flight on any stream
  WMD_CUDA_TRY(cudaDeviceSynchronize());
  drop_captured(c);
  WMD_CUDA_TRY(build_schedule(c, cls, variant, fill));
  return WMD_OK;
}

int32_t wmd_get_loop_partition(const wmd_corpus* c, int32_t v_r, int32_t variant) {
  const int cls = v_r > 0 ? vr_class(v_r) : -1;
  if (!c || cls < 0 || variant < 0 || variant >= kClassVariants[cls]) return -1;
  return c->sched[cls][variant].fill;
}

int32_t wmd_get_loop_variant(const wmd_corpus* c, int32_t v_r, wmd_precision prec) {
  const int cls = v_r > 0 ? vr_class(v_r) : -1;
  if (!c || cls < 0 || (prec != WMD_PREC_FP32 && prec != WMD_PREC_BF16_K)) return -1;
  return c->loop_variant[cls][prec == WMD_PREC_BF16_K];
}

wmd_status wmd_autotune(wmd_corpus* c, const int32_t* q_ids, const float* q_w, int32_t n_q,
                        float lambda, int32_t max_iter, wmd_precision prec, int32_t* chosen) {
  wmd::NvtxRange nvtx_range("wmd_autotune");
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  std::vector<int32_t> ids(std::max(n_q, 1));
  std::vector<float> w(std::max(n_q, 1));
  int32_t v_r = 0;
  wmd_status st = wmd_compact_query(q_ids, q_w, n_q, c->V, ids.data(), w.data(), &v_r);
  if (st != WMD_OK) return st;
  if ((st = check_query_args(c, v_r, lambda, max_iter)) != WMD_OK) return st;
  if (prec != WMD_PREC_FP32 && prec != WMD_PREC_BF16_K)
    return set_error(WMD_ERR_INVALID_ARG, "unknown precision");
  const int cls = vr_class(v_r);
  DeviceGuard g(c->device);
  // the timed partitions replace the class's work items: nothing else may
  // use the corpus meanwhile (the host path waits on the lock), and launches
  // in flight on other streams finish first
  std::lock_guard<std::mutex> lock(c->mu);
  WMD_CUDA_TRY(cudaDeviceSynchronize());
  drop_captured(c);
  const size_t ws_bytes = wmd_workspace_bytes(c, v_r, prec);
  void* ws = nullptr;
  int32_t* d_ids = nullptr;
  float* d_w = nullptr;
  double* d_out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best = 0;
  float best_ms = 0.f;
  cudaError_t e = cudaMalloc(&ws, ws_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&d_ids, v_r * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_w, v_r * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, std::max<int64_t>(c->N, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ids, ids.data(), v_r * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, w.data(), v_r * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    // every tile variant of the class with every partition: the fastest
    // partition stays with each variant, the fastest pair is chosen
    st = wmd_build_kernel_matrix(c, d_ids, d_w, v_r, lambda, prec, ws, ws_bytes, s);
    const int pi = prec == WMD_PREC_BF16_K;
    const int keep = c->loop_variant[cls][pi];
    float best_var_ms[kMaxVariants] = {};
    for (int var = 0; var < kClassVariants[cls] && st == WMD_OK && e == cudaSuccess; ++var) {
      c->loop_variant[cls][pi] = var;
      int best_fill = c->sched[cls][var].fill;
      for (int fi = 0; fi < kNumFills && st == WMD_OK && e == cudaSuccess; ++fi) {
        if (c->sched[cls][var].fill != kFills[fi]) {
          e = cudaStreamSynchronize(s);
          if (e == cudaSuccess) e = build_schedule(c, cls, var, kFills[fi]);
          if (e != cudaSuccess) break;
        }
        for (int k = 0; k < 2 && st == WMD_OK; ++k)
          st = wmd_sinkhorn_loop(c, v_r, max_iter, prec, ws, ws_bytes, d_out, s);
        if (st != WMD_OK) break;
        e = cudaEventRecord(e0, s);
        for (int k = 0; k < 5 && st == WMD_OK; ++k)
          st = wmd_sinkhorn_loop(c, v_r, max_iter, prec, ws, ws_bytes, d_out, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (fi == 0 || ms < best_var_ms[var])) {
          best_var_ms[var] = ms;
          best_fill = kFills[fi];
        }
      }
      if (st == WMD_OK && e == cudaSuccess && c->sched[cls][var].fill != best_fill) {
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = build_schedule(c, cls, var, best_fill);
      }
      if (st == WMD_OK && e == cudaSuccess && (var == 0 || best_var_ms[var] < best_ms)) {
        best_ms = best_var_ms[var];
        best = var;
      }
    }
    c->loop_variant[cls][pi] = (st == WMD_OK && e == cudaSuccess) ? best : keep;
    if (st == WMD_OK && e == cudaSuccess) save_autotune_choice(c, cls, pi, best);
  }
  if (s) cudaStreamSynchronize(s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(ws);
  cudaFree(d_ids);
  cudaFree(d_w);
  cudaFree(d_out);
  if (e != cudaSuccess) return cuda_error(e, "autotune");
  if (st != WMD_OK) return st;
  if (chosen) *chosen = best;
  return WMD_OK;
}

wmd_status wmd_query(wmd_corpus* c, const int32_t* q_ids, const float* q_w, int32_t n_q,
                     float lambda, int32_t max_iter, wmd_precision prec, double* out_wmd) {
  wmd::NvtxRange nvtx_range("wmd_query");
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  if (!out_wmd && c->N > 0) return set_error(WMD_ERR_INVALID_ARG, "out_wmd is NULL");
  if (n_q > WMD_MAX_VR) {
    // compaction may still bring it under the limit: use a temporary
    std::vector<int32_t> ids(n_q);
    std::vector<float> w(n_q);
    int32_t v_r = 0;
    wmd_status st = wmd_compact_query(q_ids, q_w, n_q, c->V, ids.data(), w.data(), &v_r);
    if (st != WMD_OK) return st;
    return wmd_query(c, ids.data(), w.data(), v_r, lambda, max_iter, prec, out_wmd);
  }
  std::lock_guard<std::mutex> lock(c->mu);
  DeviceGuard g(c->device);
  if (!c->stream) WMD_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  if (!c->h_stage) {
    WMD_CUDA_TRY(cudaHostAlloc(&c->h_stage, (2 * WMD_MAX_VR + 4) * sizeof(int32_t), cudaHostAllocMapped));
    const cudaError_t e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->dh_stage), c->h_stage, 0);
    if (e != cudaSuccess) {
      cudaFreeHost(c->h_stage);
      c->h_stage = nullptr;
      return cuda_error(e, "cudaHostGetDevicePointer");
    }
  }
  // compact straight into the pinned staging block: ids, then weights
  int32_t* h_ids = c->h_stage;
  float* h_w = reinterpret_cast<float*>(c->h_stage + WMD_MAX_VR);
  int32_t* h_err = c->h_stage + 2 * WMD_MAX_VR;
  int32_t v_r = 0;
  wmd_status st = wmd_compact_query(q_ids, q_w, n_q, c->V, h_ids, h_w, &v_r);
  if (st != WMD_OK) return st;
  if ((st = check_query_args(c, v_r, lambda, max_iter)) != WMD_OK) return st;
  if (prec != WMD_PREC_FP32 && prec != WMD_PREC_BF16_K)
    return set_error(WMD_ERR_INVALID_ARG, "unknown precision");
  const size_t need = wmd_workspace_bytes(c, v_r, prec);
  if (c->ws_bytes < need) {
    // a new workspace invalidates the captured sequences that point into it
    cudaStreamSynchronize(c->stream);
    for (auto& g2 : c->qgraphs)
      if (g2.exec) cudaGraphExecDestroy(g2.exec);
    c->qgraphs.clear();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
    WMD_CUDA_TRY(cudaMalloc(&c->ws, need));
    c->ws_bytes = need;
  }
  if (!c->h_out) {
    WMD_CUDA_TRY(cudaHostAlloc(&c->h_out, std::max<int64_t>(c->N, 1) * sizeof(double), cudaHostAllocMapped));
    const cudaError_t e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->dh_out), c->h_out, 0);
    if (e != cudaSuccess) {
      cudaFreeHost(c->h_out);
      c->h_out = nullptr;
      return cuda_error(e, "cudaHostGetDevicePointer");
    }
  }

  // the query comes from, and the results and the error word go to, host
  // memory directly: the kernels read the mapped staging block (no copy in)
  // and the loop kernel writes the mapped output blocks (no copy back)
  double* dh_out = c->dh_out;
  int32_t* dh_stage = c->dh_stage;
  int* dh_err = dh_stage + 2 * WMD_MAX_VR;
  // a caller buffer that is pinned and mapped into the device's address space
  // takes the results directly (no copy out of the staging block)
  bool direct = false;
  if (c->N > 0) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, out_wmd) == cudaSuccess) {
      if (pa.type == cudaMemoryTypeHost && pa.devicePointer) {
        dh_out = static_cast<double*>(pa.devicePointer);
        direct = true;
      }
    } else {
      cudaGetLastError();
    }
  }

  // the whole sequence (cdist, loop) runs eagerly on the first use of a
  // query shape and from a captured CUDA graph from the second use on
  const int cls = vr_class(v_r);
  const int variant = c->loop_variant[cls][prec == WMD_PREC_BF16_K];
  const int32_t* dh_ids = dh_stage;
  const float* dh_w = reinterpret_cast<const float*>(dh_stage + WMD_MAX_VR);
  auto enqueue = [&]() -> wmd_status {
    wmd_status s2 = check_query_args(c, v_r, lambda, max_iter);
    if (s2 == WMD_OK)
      s2 = wmd_build_kernel_matrix(c, dh_ids, dh_w, v_r, lambda, prec, c->ws, c->ws_bytes, c->stream);
    if (s2 == WMD_OK)
      s2 = sinkhorn_loop(c, v_r, max_iter, prec, c->ws, c->ws_bytes, dh_out, dh_err, c->stream);
    return s2;
  };
  wmd_corpus::QueryGraph* qg = nullptr;
  for (auto& g2 : c->qgraphs)
    if (g2.v_r == v_r && g2.T == max_iter && g2.prec == (int)prec && g2.variant == variant &&
        g2.lambda == lambda && g2.dout == dh_out)
      qg = &g2;
  if (!qg) {
    if (c->qgraphs.size() >= 8) {
      auto oldest = std::min_element(c->qgraphs.begin(), c->qgraphs.end(),
                                     [](const wmd_corpus::QueryGraph& a, const wmd_corpus::QueryGraph& b) {
                                       return a.last < b.last;
                                     });
      if (oldest->exec) cudaGraphExecDestroy(oldest->exec);
      c->qgraphs.erase(oldest);
    }
    c->qgraphs.push_back(
        wmd_corpus::QueryGraph{v_r, max_iter, (int)prec, variant, lambda, dh_out, 0, nullptr, 0});
    qg = &c->qgraphs.back();
  }
  qg->last = ++c->qtick;
  if (!c->use_graphs) {
    st = enqueue();
    if (st != WMD_OK) {
      cudaStreamSynchronize(c->stream);
      return st;
    }
  } else if (qg->exec) {
    WMD_CUDA_TRY(cudaGraphLaunch(qg->exec, c->stream));
  } else if (qg->uses >= 1) {
    cudaGraph_t graph = nullptr;
    WMD_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    st = enqueue();
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (st != WMD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&qg->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      qg->exec = nullptr;
      return cuda_error(e, "cudaGraphInstantiate");
    }
    WMD_CUDA_TRY(cudaGraphLaunch(qg->exec, c->stream));
  } else {
    st = enqueue();
    if (st != WMD_OK) {
      cudaStreamSynchronize(c->stream);
      return st;
    }
  }
  qg->uses += 1;
  WMD_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->N > 0 && !direct) std::memcpy(out_wmd, c->h_out, c->N * sizeof(double));
  const int err = *reinterpret_cast<volatile int32_t*>(h_err);
  if (err) return device_error(err);
  return WMD_OK;
}

}  // extern "C"

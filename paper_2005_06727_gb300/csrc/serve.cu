// Batched and served queries: many queries of uneven v_r against one resident
// corpus (the paper answers one query at a time, Sec. 3 and Sec. 4; running
// several is the same computation repeated per query).
//
// A batch lays every query's block of K side by side in one
// word-major matrix (row w holds the VR_q columns of query q at offset col0_q),
// runs one cdist launch per query (tensor cores where they apply) and then ONE
// fused-loop launch per query-width class that covers every (query, document)
// pair of that class (blockIdx.y = query).  No reduction order depends on the
// composition of the batch, so a query's WMD values are bit-identical alone,
// in a batch and in the server's mix.
//
// wmd_query_batch replays a captured CUDA graph when the same batch shape
// (widths, lambdas, max_iter, precision) comes again.  The server runs a
// scheduler thread: requests wait in a queue, and whenever one of its stream
// slots is free it admits as many waiting requests as fit the slot's share of
// the memory budget (continuous batching: new batches start while earlier
// ones are still on the GPU, on other streams).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wmd_internal.h"

namespace wmd {
namespace {

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// One compacted query of a batch.
struct Req {
  std::vector<int32_t> ids;
  std::vector<float> w;
  float lambda = 0.f;
  int v_r = 0;
  int cls = 0;
  int VR = 0;
};

size_t k_elem(wmd_precision prec) { return prec == WMD_PREC_BF16_K ? 2 : 4; }

// Device bytes one query adds to a batch (its K columns, r, output).
size_t request_bytes(const wmd_corpus* c, int VR, wmd_precision prec) {
  return (size_t)std::max<int64_t>(c->U, 1) * VR * k_elem(prec) + VR * 4 +
         (size_t)std::max<int64_t>(c->N, 1) * 8 + 64;
}

// Buffers of one batch in flight (grow-only), device and pinned host.
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int32_t* d_ids = nullptr;
  float* d_w = nullptr;
  size_t ids_cap = 0, w_cap = 0;
  QueryDesc* d_desc = nullptr;
  size_t desc_cap = 0;
  char* d_ws = nullptr;  // r_all | K_all
  size_t ws_cap = 0;
  double* d_out = nullptr;
  size_t out_cap = 0;
  int32_t* h_ids = nullptr;
  float* h_w = nullptr;
  QueryDesc* h_desc = nullptr;
  double* h_out = nullptr;
  int* h_err = nullptr;  // pinned copy of every query's error words (read after `done`)
  size_t h_err_cap = 0;
  size_t h_ids_cap = 0, h_w_cap = 0, h_desc_cap = 0, h_out_cap = 0;

  void release() {
    if (stream) cudaStreamSynchronize(stream);
    cudaFree(d_ids);
    cudaFree(d_w);
    cudaFree(d_desc);
    cudaFree(d_ws);
    cudaFree(d_out);
    cudaFreeHost(h_ids);
    cudaFreeHost(h_w);
    cudaFreeHost(h_desc);
    cudaFreeHost(h_out);
    cudaFreeHost(h_err);
    if (done) cudaEventDestroy(done);
    if (stream) cudaStreamDestroy(stream);
    *this = Slot();
  }
};

template <typename T>
cudaError_t grow_dev(T** p, size_t* cap, size_t need) {
  if (*cap >= need) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(need, 1) * sizeof(T));
  if (e == cudaSuccess) *cap = need;
  return e;
}

template <typename T>
cudaError_t grow_host(T** p, size_t* cap, size_t need) {
  if (*cap >= need) return cudaSuccess;
  cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(p), std::max<size_t>(need, 1) * sizeof(T));
  if (e == cudaSuccess) *cap = need;
  return e;
}

// Column layout of a batch: query q owns columns [col0[q], col0[q] + VR_q).
struct Layout {
  std::vector<int> col0;
  int ldk = 0;
  size_t words = 0;
  size_t r_off = 0, err_off = 0, k_off = 0, ws_bytes = 0;
  std::vector<size_t> err_first;   // query -> its first error slot (prefix sums; [nq] = total)
  std::vector<int> desc_of;        // query -> index in the descriptor table
  int cls_begin[kNumClasses + 1];  // descriptor ranges per class
};

Layout plan(const wmd_corpus* c, const std::vector<const Req*>& qs, wmd_precision prec) {
  Layout L;
  L.col0.resize(qs.size());
  int col = 0;
  for (size_t q = 0; q < qs.size(); ++q) {
    L.col0[q] = col;
    col += qs[q]->VR;
    L.words += qs[q]->v_r;
  }
  L.ldk = std::max(col, 8);
  L.r_off = 0;
  // after every query's r: every query's error slots (one per cdist CTA)
  L.err_off = (size_t)L.ldk * 4;
  L.err_first.assign(qs.size() + 1, 0);
  for (size_t q = 0; q < qs.size(); ++q)
    L.err_first[q + 1] = L.err_first[q] + cdist_err_slots(c, qs[q]->VR);
  L.k_off = round_up(L.err_off + L.err_first.back() * sizeof(int), 256);
  const size_t kb = round_up((size_t)std::max<int64_t>(c->U, 1) * L.ldk * k_elem(prec), 256);
  L.ws_bytes = L.k_off + kb;
  // descriptors grouped by width class
  L.desc_of.assign(qs.size(), 0);
  int n = 0;
  for (int cls = 0; cls < kNumClasses; ++cls) {
    L.cls_begin[cls] = n;
    for (size_t q = 0; q < qs.size(); ++q)
      if (qs[q]->cls == cls) L.desc_of[q] = n++;
  }
  L.cls_begin[kNumClasses] = n;
  return L;
}

// Fills the slot's staging buffers and enqueues the whole batch on its stream:
// H2D of ids, weights and descriptors, one cdist per query, one loop per
// class, D2H of the nq x N results into the slot's pinned buffer.
wmd_status enqueue_batch(wmd_corpus* c, Slot& s, const std::vector<const Req*>& qs,
                         const Layout& L, int T, wmd_precision prec) {
  wmd::NvtxRange nvtx_range("batch enqueue");
  const size_t nq = qs.size();
  const size_t N1 = (size_t)std::max<int64_t>(c->N, 1);
  WMD_CUDA_TRY(grow_dev(&s.d_ids, &s.ids_cap, L.words));
  WMD_CUDA_TRY(grow_dev(&s.d_w, &s.w_cap, L.words));
  WMD_CUDA_TRY(grow_dev(&s.d_desc, &s.desc_cap, nq));
  WMD_CUDA_TRY(grow_dev(&s.d_ws, &s.ws_cap, L.ws_bytes));
  WMD_CUDA_TRY(grow_dev(&s.d_out, &s.out_cap, nq * N1));
  WMD_CUDA_TRY(grow_host(&s.h_ids, &s.h_ids_cap, L.words));
  WMD_CUDA_TRY(grow_host(&s.h_w, &s.h_w_cap, L.words));
  WMD_CUDA_TRY(grow_host(&s.h_desc, &s.h_desc_cap, nq));
  WMD_CUDA_TRY(grow_host(&s.h_out, &s.h_out_cap, nq * N1));
  WMD_CUDA_TRY(grow_host(&s.h_err, &s.h_err_cap, L.err_first.back()));

  // staging: compacted words of every query, and the descriptor table
  size_t off = 0;
  std::vector<size_t> word_off(nq);
  for (size_t q = 0; q < nq; ++q) {
    word_off[q] = off;
    std::memcpy(s.h_ids + off, qs[q]->ids.data(), qs[q]->v_r * sizeof(int32_t));
    std::memcpy(s.h_w + off, qs[q]->w.data(), qs[q]->v_r * sizeof(float));
    off += qs[q]->v_r;
  }
  char* ws = s.d_ws;
  float* r_all = reinterpret_cast<float*>(ws + L.r_off);
  int* err = reinterpret_cast<int*>(ws + L.err_off);  // every query's slots
  for (size_t q = 0; q < nq; ++q) {
    QueryDesc& d = s.h_desc[L.desc_of[q]];
    d.r = r_all + L.col0[q];
    d.out = s.d_out + q * N1;
    d.kcol0 = L.col0[q];
    d.v_r = qs[q]->v_r;
    d.lambda = qs[q]->lambda;
    d.scale = -0.69314718055994530942 / (double)qs[q]->lambda;
  }
  cudaStream_t st = s.stream;
  WMD_CUDA_TRY(cudaMemcpyAsync(s.d_ids, s.h_ids, L.words * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  WMD_CUDA_TRY(cudaMemcpyAsync(s.d_w, s.h_w, L.words * sizeof(float), cudaMemcpyHostToDevice, st));
  WMD_CUDA_TRY(cudaMemcpyAsync(s.d_desc, s.h_desc, nq * sizeof(QueryDesc), cudaMemcpyHostToDevice, st));
  // the first cdist launch prefetches the loop's document CSR into L2; every
  // query's cdist writes its own error slots (a failure fails that query only)
  const L2Prefetch pf = loop_inputs(c, vr_class(qs[0]->v_r), prec);
  for (size_t q = 0; q < nq; ++q)
    WMD_CUDA_TRY(launch_cdist(c, s.d_ids + word_off[q], s.d_w + word_off[q], qs[q]->v_r, qs[q]->VR,
                              qs[q]->lambda, prec, ws + L.k_off, L.ldk, L.col0[q],
                              r_all + L.col0[q], nullptr, err + L.err_first[q],
                              q == 0 ? &pf : nullptr, st));
  for (int cls = 0; cls < kNumClasses; ++cls) {
    const int n = L.cls_begin[cls + 1] - L.cls_begin[cls];
    if (n)
      WMD_CUDA_TRY(launch_loop_batch(c, cls, ws + L.k_off, L.ldk, s.d_desc + L.cls_begin[cls], n, T,
                                     prec, st));
  }
  if (c->N > 0)
    WMD_CUDA_TRY(cudaMemcpyAsync(s.h_out, s.d_out, nq * N1 * sizeof(double), cudaMemcpyDeviceToHost, st));
  WMD_CUDA_TRY(cudaMemcpyAsync(s.h_err, err, L.err_first.back() * sizeof(int),
                               cudaMemcpyDeviceToHost, st));
  return WMD_OK;
}

wmd_status compact(const wmd_corpus* c, const int32_t* ids, const float* w, int32_t n, float lambda,
                   Req* out) {
  out->ids.resize(std::max(n, 1));
  out->w.resize(std::max(n, 1));
  int32_t vr = 0;
  wmd_status st = wmd_compact_query(ids, w, n, c->V, out->ids.data(), out->w.data(), &vr);
  if (st != WMD_OK) return st;
  if (vr <= 0) return set_error(WMD_ERR_INVALID_ARG, "query has no word with positive weight");
  if (!(lambda > 0.f) || !(lambda < 3.4e38f))
    return set_error(WMD_ERR_INVALID_ARG, "lambda must be positive and finite");
  out->ids.resize(vr);
  out->w.resize(vr);
  out->v_r = vr;
  out->cls = vr_class(vr);
  out->VR = kClassKVR[out->cls];
  out->lambda = lambda;
  return WMD_OK;
}

// -------------------------------------------------------------- batch API state
struct GraphEntry {
  std::vector<int> shape;  // v_r of every query
  std::vector<float> lambdas;
  int T = 0;
  int prec = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

struct BatchState {
  std::mutex mu;
  Slot slot;
  std::vector<GraphEntry> graphs;
  uint64_t tick = 0;
};

std::mutex g_batch_mu;
std::unordered_map<const wmd_corpus*, std::unique_ptr<BatchState>> g_batch;

BatchState* batch_state(const wmd_corpus* c) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  auto& p = g_batch[c];
  if (!p) p.reset(new BatchState());
  return p.get();
}

}  // namespace

void release_batch_state(const wmd_corpus* c) {
  std::unique_ptr<BatchState> st;
  {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    auto it = g_batch.find(c);
    if (it == g_batch.end()) return;
    st = std::move(it->second);
    g_batch.erase(it);
  }
  for (auto& g : st->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  st->slot.release();
}

}  // namespace wmd

using namespace wmd;

// ================================================================ server
struct wmd_server {
  struct Request {
    Req q;
    int T = 0;
    wmd_precision prec = WMD_PREC_FP32;
    uint64_t ticket = 0;
    wmd_status status = WMD_ERR_NOT_READY;  // NOT_READY while queued or running
    std::string error;
    std::vector<double> result;
    size_t bytes = 0;
  };
  struct InFlight {
    int slot = -1;
    std::vector<std::shared_ptr<Request>> reqs;
    std::vector<size_t> err_first;  // each request's error slots in the slot's copy
  };

  wmd_corpus* corpus = nullptr;
  wmd_server_options opt;
  std::vector<Slot> slots;
  std::vector<bool> slot_busy;
  std::mutex mu;
  std::condition_variable cv_work;   // scheduler: new requests or shutdown
  std::condition_variable cv_done;   // pollers: a request finished
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
  std::vector<InFlight> inflight;
  uint64_t next_ticket = 1;
  bool shutdown = false;
  std::thread worker;
  wmd_server_stats stats;

  void run();
  void retire_finished(std::unique_lock<std::mutex>& lock, bool block);
  bool launch_one(std::unique_lock<std::mutex>& lock);
};

void wmd_server::retire_finished(std::unique_lock<std::mutex>& lock, bool block) {
  for (size_t i = 0; i < inflight.size();) {
    Slot& s = slots[inflight[i].slot];
    cudaError_t e = cudaEventQuery(s.done);
    if (e == cudaErrorNotReady && block) {
      lock.unlock();
      // bounded wait on the oldest batch: poll the event with short sleeps
      const auto t0 = std::chrono::steady_clock::now();
      while ((e = cudaEventQuery(s.done)) == cudaErrorNotReady &&
             std::chrono::steady_clock::now() - t0 < std::chrono::seconds(30))
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      lock.lock();
      block = false;
    }
    if (e == cudaErrorNotReady) {
      ++i;
      continue;
    }
    const size_t N1 = (size_t)std::max<int64_t>(corpus->N, 1);
    auto& reqs = inflight[i].reqs;
    for (size_t q = 0; q < reqs.size(); ++q) {
      Request& r = *reqs[q];
      // the request's own error slots (copied back with the results)
      const auto& ef = inflight[i].err_first;
      const int err = e == cudaSuccess ? error_summary(s.h_err + ef[q], ef[q + 1] - ef[q]) : 0;
      if (e != cudaSuccess) {
        r.status = WMD_ERR_CUDA;
        r.error = std::string("batch failed: ") + cudaGetErrorString(e);
      } else if (err) {
        r.status = device_error(err);
        r.error = wmd_last_error();
      } else {
        r.result.assign(s.h_out + q * N1, s.h_out + q * N1 + corpus->N);
        r.status = WMD_OK;
      }
    }
    stats.completed += reqs.size();
    slot_busy[inflight[i].slot] = false;
    inflight.erase(inflight.begin() + i);
    cv_done.notify_all();
  }
}

bool wmd_server::launch_one(std::unique_lock<std::mutex>& lock) {
  if (pending.empty()) return false;
  int free_slot = -1;
  for (size_t i = 0; i < slots.size(); ++i)
    if (!slot_busy[i]) {
      free_slot = (int)i;
      break;
    }
  if (free_slot < 0) return false;
  // admit, in arrival order, the requests of the oldest one's kind
  // (precision, max_iter) that fit the slot's memory share and batch size
  const size_t budget = opt.mem_budget / std::max(opt.slots, 1);
  const wmd_precision prec = pending.front()->prec;
  const int T = pending.front()->T;
  std::vector<std::shared_ptr<Request>> batch;
  size_t bytes = 0;
  for (auto it = pending.begin(); it != pending.end() && (int)batch.size() < opt.max_batch;) {
    Request& r = **it;
    if (r.prec == prec && r.T == T && (batch.empty() || bytes + r.bytes <= budget)) {
      bytes += r.bytes;
      batch.push_back(*it);
      it = pending.erase(it);
    } else {
      ++it;
    }
  }
  Slot& s = slots[free_slot];
  std::vector<const Req*> qs;
  for (auto& r : batch) qs.push_back(&r->q);
  const Layout L = plan(corpus, qs, prec);
  wmd_status st;
  {
    lock.unlock();
    DevGuard g(corpus->device);
    st = enqueue_batch(corpus, s, qs, L, T, prec);
    if (st == WMD_OK) {
      cudaError_t e = cudaEventRecord(s.done, s.stream);
      if (e != cudaSuccess) st = cuda_error(e, "cudaEventRecord");
    }
    lock.lock();
  }
  if (st != WMD_OK) {
    for (auto& r : batch) {
      r->status = st;
      r->error = wmd_last_error();
    }
    cv_done.notify_all();
    return true;
  }
  slot_busy[free_slot] = true;
  InFlight f;
  f.slot = free_slot;
  f.err_first = L.err_first;
  f.reqs = std::move(batch);
  stats.batches += 1;
  stats.max_batch_seen = std::max<int64_t>(stats.max_batch_seen, (int64_t)f.reqs.size());
  inflight.push_back(std::move(f));
  return true;
}

void wmd_server::run() {
  std::unique_lock<std::mutex> lock(mu);
  while (true) {
    retire_finished(lock, false);
    if (shutdown && pending.empty() && inflight.empty()) break;
    if (launch_one(lock)) continue;
    if (!inflight.empty() && (pending.empty() || inflight.size() == slots.size())) {
      // every slot is busy (or nothing waits): finish the oldest batch first
      retire_finished(lock, true);
      continue;
    }
    cv_work.wait_for(lock, std::chrono::microseconds(200));
  }
  // leftover requests after shutdown
  for (auto& r : pending) {
    r->status = WMD_ERR_SHUTDOWN;
    r->error = "server shut down";
  }
  pending.clear();
  cv_done.notify_all();
}

extern "C" {

wmd_status wmd_query_batch(wmd_corpus* c, int32_t nq, const int64_t* q_ptr, const int32_t* q_ids,
                           const float* q_w, const float* lambda, int32_t max_iter,
                           wmd_precision prec, double* out) {
  wmd::NvtxRange nvtx_range("wmd_query_batch");
  if (!c) return set_error(WMD_ERR_INVALID_ARG, "corpus is NULL");
  if (nq < 0) return set_error(WMD_ERR_INVALID_ARG, "nq < 0");
  if (nq == 0) return WMD_OK;
  if (!q_ptr || !lambda || (c->N > 0 && !out)) return set_error(WMD_ERR_INVALID_ARG, "NULL pointer");
  if (max_iter < 0) return set_error(WMD_ERR_INVALID_ARG, "max_iter must be >= 0");
  if (prec != WMD_PREC_FP32 && prec != WMD_PREC_BF16_K)
    return set_error(WMD_ERR_INVALID_ARG, "unknown precision");
  if (q_ptr[0] != 0) return set_error(WMD_ERR_INVALID_ARG, "q_ptr[0] must be 0");
  std::vector<Req> reqs(nq);
  for (int32_t q = 0; q < nq; ++q) {
    const int64_t b = q_ptr[q], e = q_ptr[q + 1];
    if (e < b || e - b > INT32_MAX) return set_error(WMD_ERR_INVALID_ARG, "q_ptr must not decrease");
    wmd_status st = compact(c, q_ids + b, q_w + b, (int32_t)(e - b), lambda[q], &reqs[q]);
    if (st != WMD_OK) return st;
  }
  std::vector<const Req*> qs;
  for (auto& r : reqs) qs.push_back(&r);
  const Layout L = plan(c, qs, prec);

  BatchState* B = batch_state(c);
  std::lock_guard<std::mutex> lock(B->mu);
  DevGuard g(c->device);
  Slot& s = B->slot;
  if (!s.stream) {
    WMD_CUDA_TRY(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    WMD_CUDA_TRY(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
  }
  // a captured graph replays the same shape: widths, lambdas, T, precision
  std::vector<int> shape(nq);
  std::vector<float> lams(nq);
  for (int q = 0; q < nq; ++q) {
    shape[q] = reqs[q].v_r;
    lams[q] = reqs[q].lambda;
  }
  GraphEntry* ge = nullptr;
  for (auto& g2 : B->graphs)
    if (g2.shape == shape && g2.lambdas == lams && g2.T == max_iter && g2.prec == (int)prec) ge = &g2;
  // buffers must not move under a captured graph: size them before capture
  const bool fresh = !ge;
  if (!c->use_graphs) {
    wmd_status st = enqueue_batch(c, s, qs, L, max_iter, prec);
    if (st != WMD_OK) return st;
  } else if (fresh) {
    // run once eagerly (allocates and sizes every buffer), then capture
    wmd_status st = enqueue_batch(c, s, qs, L, max_iter, prec);
    if (st != WMD_OK) return st;
    WMD_CUDA_TRY(cudaStreamSynchronize(s.stream));
    cudaGraph_t graph = nullptr;
    WMD_CUDA_TRY(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
    st = enqueue_batch(c, s, qs, L, max_iter, prec);
    cudaError_t e = cudaStreamEndCapture(s.stream, &graph);
    if (st != WMD_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
    GraphEntry entry;
    entry.shape = shape;
    entry.lambdas = lams;
    entry.T = max_iter;
    entry.prec = (int)prec;
    e = cudaGraphInstantiate(&entry.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
    if (B->graphs.size() >= 8) {
      auto oldest = std::min_element(B->graphs.begin(), B->graphs.end(),
                                     [](const GraphEntry& a, const GraphEntry& b) { return a.last_use < b.last_use; });
      cudaGraphExecDestroy(oldest->exec);
      B->graphs.erase(oldest);
    }
    B->graphs.push_back(entry);
    ge = &B->graphs.back();
  } else {
    // same shape: refresh the staged query words, then replay
    size_t off = 0;
    for (int q = 0; q < nq; ++q) {
      std::memcpy(s.h_ids + off, reqs[q].ids.data(), reqs[q].v_r * sizeof(int32_t));
      std::memcpy(s.h_w + off, reqs[q].w.data(), reqs[q].v_r * sizeof(float));
      off += reqs[q].v_r;
    }
    WMD_CUDA_TRY(cudaGraphLaunch(ge->exec, s.stream));
  }
  if (ge) ge->last_use = ++B->tick;
  WMD_CUDA_TRY(cudaStreamSynchronize(s.stream));
  // a query whose cdist reported an error gets NaN results (the loop kernel
  // of a batch does not read the error slots) and the call reports the first
  // such query
  const size_t N1 = (size_t)std::max<int64_t>(c->N, 1);
  wmd_status first = WMD_OK;
  std::string msg;
  for (int q = 0; q < nq; ++q) {
    double* row = out + (size_t)q * c->N;
    const int err = error_summary(s.h_err + L.err_first[q], L.err_first[q + 1] - L.err_first[q]);
    if (err) {
      if (c->N > 0) std::fill(row, row + c->N, std::numeric_limits<double>::quiet_NaN());
      if (first == WMD_OK) {
        first = device_error(err);
        msg = "query " + std::to_string(q) + " of the batch: " + wmd_last_error();
      }
    } else if (c->N > 0) {
      std::memcpy(row, s.h_out + q * N1, c->N * sizeof(double));
    }
  }
  if (first != WMD_OK) return set_error(first, msg);
  return WMD_OK;
}

wmd_status wmd_server_create(wmd_corpus* c, const wmd_server_options* opt, wmd_server** out) {
  if (!c || !out) return set_error(WMD_ERR_INVALID_ARG, "NULL pointer");
  *out = nullptr;
  wmd_server_options o = c->server_defaults;
  if (opt) o = *opt;
  if (o.max_batch <= 0 || o.slots <= 0 || o.slots > 16 || o.mem_budget == 0 || o.max_pending <= 0)
    return set_error(WMD_ERR_INVALID_ARG, "server options out of range");
  std::unique_ptr<wmd_server> s(new (std::nothrow) wmd_server());
  if (!s) return set_error(WMD_ERR_OUT_OF_MEMORY, "host allocation failed");
  s->corpus = c;
  s->opt = o;
  std::memset(&s->stats, 0, sizeof(s->stats));
  s->slots.resize(o.slots);
  s->slot_busy.assign(o.slots, false);
  {
    DevGuard g(c->device);
    for (auto& sl : s->slots) {
      WMD_CUDA_TRY(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
      WMD_CUDA_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
    }
  }
  wmd_server* raw = s.get();
  s->worker = std::thread([raw] {
    cudaSetDevice(raw->corpus->device);
    raw->run();
  });
  *out = s.release();
  return WMD_OK;
}

wmd_status wmd_serve_submit(wmd_server* s, const int32_t* q_ids, const float* q_w, int32_t n_q,
                            float lambda, int32_t max_iter, wmd_precision prec, uint64_t* ticket) {
  if (!s || !ticket) return set_error(WMD_ERR_INVALID_ARG, "NULL pointer");
  if (max_iter < 0) return set_error(WMD_ERR_INVALID_ARG, "max_iter must be >= 0");
  if (prec != WMD_PREC_FP32 && prec != WMD_PREC_BF16_K)
    return set_error(WMD_ERR_INVALID_ARG, "unknown precision");
  auto r = std::make_shared<wmd_server::Request>();
  wmd_status st = compact(s->corpus, q_ids, q_w, n_q, lambda, &r->q);
  if (st != WMD_OK) return st;
  r->T = max_iter;
  r->prec = prec;
  r->bytes = request_bytes(s->corpus, r->q.VR, prec);
  if (r->bytes > s->opt.mem_budget / s->opt.slots)
    return set_error(WMD_ERR_OUT_OF_MEMORY,
                     "query needs " + std::to_string(r->bytes) +
                         " device bytes, more than one slot's share of the memory budget");
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->shutdown) return set_error(WMD_ERR_SHUTDOWN, "server is shutting down");
  if ((int64_t)s->pending.size() >= s->opt.max_pending)
    return set_error(WMD_ERR_NOT_READY, "request queue is full; retry later");
  r->ticket = s->next_ticket++;
  s->tickets[r->ticket] = r;
  s->pending.push_back(r);
  s->stats.submitted += 1;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return WMD_OK;
}

wmd_status wmd_serve_poll(wmd_server* s, uint64_t ticket, double* out_wmd, int64_t timeout_us) {
  if (!s) return set_error(WMD_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return set_error(WMD_ERR_INVALID_ARG, "unknown ticket");
  std::shared_ptr<wmd_server::Request> r = it->second;
  if (r->status == WMD_ERR_NOT_READY && timeout_us > 0)
    s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us),
                        [&] { return r->status != WMD_ERR_NOT_READY; });
  if (r->status == WMD_ERR_NOT_READY)
    return timeout_us > 0 ? set_error(WMD_ERR_TIMEOUT, "request not finished within the timeout")
                          : set_error(WMD_ERR_NOT_READY, "request not finished yet");
  s->tickets.erase(it);
  if (r->status != WMD_OK) return set_error(r->status, r->error);
  if (s->corpus->N > 0) {
    if (!out_wmd) return set_error(WMD_ERR_INVALID_ARG, "out_wmd is NULL");
    std::memcpy(out_wmd, r->result.data(), s->corpus->N * sizeof(double));
  }
  return WMD_OK;
}

wmd_status wmd_serve_cancel(wmd_server* s, uint64_t ticket) {
  if (!s) return set_error(WMD_ERR_INVALID_ARG, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return set_error(WMD_ERR_INVALID_ARG, "unknown ticket");
  auto r = it->second;
  auto pit = std::find(s->pending.begin(), s->pending.end(), r);
  if (pit != s->pending.end()) s->pending.erase(pit);  // never launched
  // a running request finishes on the GPU; its result is dropped
  s->tickets.erase(it);
  s->stats.cancelled += 1;
  return WMD_OK;
}

wmd_status wmd_server_get_stats(wmd_server* s, wmd_server_stats* out) {
  if (!s || !out) return set_error(WMD_ERR_INVALID_ARG, "NULL pointer");
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  out->pending = (int64_t)s->pending.size();
  out->in_flight_batches = (int64_t)s->inflight.size();
  return WMD_OK;
}

void wmd_server_destroy(wmd_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->shutdown = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  {
    DevGuard g(s->corpus->device);
    for (auto& sl : s->slots) sl.release();
  }
  delete s;
}

}  // extern "C"

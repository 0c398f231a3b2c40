// Serving loop over many resident graphs: a native worker pool takes update
// requests as they arrive (continuous batching: a request starts as soon as a
// worker and its graph are free, while others are on the GPU), keeps each
// admitted graph's CSR and tracked pairs on the device in its own context and
// stream, and admits graphs by a device-memory budget: a graph becomes
// resident when its context fits beside the resident ones (or when nothing
// else is resident), and memory returns to the budget when a graph is
// removed or, with eviction on, when an idle resident graph is checkpointed
// to host memory (least recently used first) to make room for a graph whose
// requests are the oldest waiting; an evicted graph is restored from its
// checkpoint at its next admission.  Requests of one graph run in
// submission order, one at a time; different graphs run concurrently.  Built
// only on the public C ABI.
#include <condition_variable>
#include <chrono>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Ticket {
  int32_t graph = -1;
  // owned copies of the update's host arrays
  std::vector<int32_t> ins_u, ins_v, del_u, del_v, del_nodes;
  std::vector<double> ins_w;
  int64_t n_new = 0;
  bool has_w = false;
  Clock::time_point t_submit, t_start, t_end;
  grest_status status = GREST_OK;
  grest_stats stats{};
  bool done = false;
};

struct Graph {
  grest_config cfg{};
  int64_t n = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val, U0, theta0;
  bool has_val = false, has_pairs = false;
  grest_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  int64_t bytes = 0;      // device bytes of its context (0 until measured)
  bool resident = false, busy = false, removed = false;
  std::deque<int64_t> queue;  // pending tickets, in submission order
  std::vector<uint8_t> ckpt;  // grest_checkpoint of an evicted graph (empty otherwise)
  Clock::time_point last_used{};
  bool evict_failed = false;  // a checkpoint failed: not evicted again until its next request ran
};

}  // namespace

struct grest_server {
  int dev = 0;
  int64_t budget = 0, used = 0;
  int n_resident = 0;
  bool evict = false;  // checkpoint idle resident graphs to host memory to admit waiting ones
  int64_t freeing = 0;  // bytes of evictions in progress
  int64_t n_admissions = 0, n_evictions = 0, n_restores = 0;
  std::vector<std::unique_ptr<Graph>> graphs;
  std::vector<std::unique_ptr<Ticket>> tickets;
  std::mutex mu;
  std::condition_variable cv;  // work available / ticket done / graph idle
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace {

void release(grest_server* sv, Graph& g) {  // mu held; the graph is idle
  if (!g.resident) return;
  grest_destroy(g.ctx);
  cudaStreamDestroy(g.stream);
  g.ctx = nullptr;
  g.stream = nullptr;
  g.resident = false;
  sv->used -= g.bytes;
  sv->n_resident -= 1;
}

void fail_queue(grest_server* sv, Graph& g, grest_status st) {  // mu held
  const Clock::time_point now = Clock::now();
  for (int64_t t : g.queue) {
    Ticket& tk = *sv->tickets[t];
    tk.status = st;
    tk.t_start = tk.t_end = now;
    tk.done = true;
  }
  g.queue.clear();
}

enum Action { kRun, kAdmit, kEvict };

// What a worker does next (mu held).  Among graphs that are not busy and
// have requests: the oldest pending ticket of a graph that is resident (run
// it) or fits the budget (admit it first).  With eviction on, when the oldest
// pending ticket of all belongs to a graph that does not fit, the least
// recently used idle resident graph is evicted instead.  Returns the graph
// index, or -1 when there is nothing to do.
int pick(grest_server* sv, Action* act) {
  int best = -1, starved = -1;
  Clock::time_point tb{}, ts{};
  for (int i = 0; i < (int)sv->graphs.size(); ++i) {
    Graph& g = *sv->graphs[i];
    if (g.busy || g.queue.empty()) continue;
    const Clock::time_point t = sv->tickets[g.queue.front()]->t_submit;
    if (!g.resident) {
      const bool fits = sv->n_resident == 0 || (g.bytes > 0 ? sv->used + g.bytes <= sv->budget : sv->used < sv->budget);
      if (!fits) {
        if (starved < 0 || t < ts) {
          starved = i;
          ts = t;
        }
        continue;
      }
    }
    if (best < 0 || t < tb) {
      best = i;
      tb = t;
    }
  }
  // evict only when the evictions already under way would not make room
  bool room_soon = false;
  if (starved >= 0 && sv->freeing > 0) {
    const Graph& w = *sv->graphs[starved];
    const int64_t after = sv->used - sv->freeing;
    room_soon = w.bytes > 0 ? after + w.bytes <= sv->budget : after < sv->budget;
  }
  if (sv->evict && starved >= 0 && !room_soon && (best < 0 || ts < tb)) {
    int v = -1;
    Clock::time_point tv{};
    for (int j = 0; j < (int)sv->graphs.size(); ++j) {
      Graph& g = *sv->graphs[j];
      if (!g.resident || g.busy || !g.queue.empty() || g.removed || g.evict_failed) continue;
      if (v < 0 || g.last_used < tv) {
        v = j;
        tv = g.last_used;
      }
    }
    if (v >= 0) {
      *act = kEvict;
      return v;
    }
  }
  if (best >= 0) *act = sv->graphs[best]->resident ? kRun : kAdmit;
  return best;
}

void worker(grest_server* sv) {
  cudaSetDevice(sv->dev);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    Action act = kRun;
    int gi = -1;
    sv->cv.wait(lk, [&] { return sv->stop || (gi = pick(sv, &act)) >= 0; });
    if (sv->stop) return;
    Graph& g = *sv->graphs[gi];
    g.busy = true;
    if (act == kEvict) {
      // checkpoint to host memory, then free the context; on failure the
      // graph stays resident and is not chosen again until a request of it
      // has run
      sv->freeing += g.bytes;
      lk.unlock();
      std::vector<uint8_t> blob;
      int64_t nb = 0;
      grest_status s0 = grest_checkpoint(g.ctx, nullptr, &nb);
      if (s0 == GREST_OK) {
        blob.resize((size_t)nb);
        s0 = grest_checkpoint(g.ctx, blob.data(), &nb);
      }
      if (s0 == GREST_OK) {
        grest_destroy(g.ctx);
        cudaStreamDestroy(g.stream);
      }
      lk.lock();
      sv->freeing -= g.bytes;
      if (s0 == GREST_OK) {
        if (!g.removed) g.ckpt.swap(blob);  // removed while it was being evicted: nothing to keep
        g.ctx = nullptr;
        g.stream = nullptr;
        g.resident = false;
        sv->used -= g.bytes;
        sv->n_resident -= 1;
        sv->n_evictions += 1;
      } else {
        g.evict_failed = true;
      }
      g.busy = false;
      sv->cv.notify_all();
      continue;
    }
    if (act == kAdmit) {
      lk.unlock();
      cudaStream_t st = nullptr;
      grest_ctx* ctx = nullptr;
      grest_status s0 = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess ? GREST_OK
                                                                                                : GREST_ERR_CUDA;
      const bool from_ckpt = !g.ckpt.empty();
      if (s0 == GREST_OK && from_ckpt)
        s0 = grest_restore(g.ckpt.data(), (int64_t)g.ckpt.size(), st, &ctx);
      else if (s0 == GREST_OK)
        s0 = grest_init(&g.cfg, g.n, g.rowptr.data(), g.col.data(), g.has_val ? g.val.data() : nullptr,
                        g.has_pairs ? g.U0.data() : nullptr, g.has_pairs ? g.theta0.data() : nullptr, st, &ctx);
      int64_t bytes = 0;
      if (s0 == GREST_OK) grest_get_device_bytes(ctx, &bytes);
      lk.lock();
      if (s0 != GREST_OK) {
        if (ctx) grest_destroy(ctx);
        if (st) cudaStreamDestroy(st);
        fail_queue(sv, g, s0);
      } else if (sv->n_resident > 0 && sv->used + bytes > sv->budget) {
        // does not fit beside the resident graphs: give the memory back; the
        // graph waits until removals make room for its measured size
        g.bytes = bytes;
        lk.unlock();
        grest_destroy(ctx);
        cudaStreamDestroy(st);
        lk.lock();
      } else {
        g.ctx = ctx;
        g.stream = st;
        g.bytes = bytes;
        g.resident = true;
        g.last_used = Clock::now();
        sv->used += bytes;
        sv->n_resident += 1;
        sv->n_admissions += 1;
        if (from_ckpt) {
          sv->n_restores += 1;
          std::vector<uint8_t>().swap(g.ckpt);
        }
      }
      g.busy = false;
      sv->cv.notify_all();
      continue;
    }
    const int64_t t = g.queue.front();
    g.queue.pop_front();
    Ticket& tk = *sv->tickets[t];
    lk.unlock();
    grest_update u{};
    u.n_new_nodes = tk.n_new;
    u.n_ins = (int64_t)tk.ins_u.size();
    u.ins_u = tk.ins_u.data();
    u.ins_v = tk.ins_v.data();
    u.ins_w = tk.has_w ? tk.ins_w.data() : nullptr;
    u.n_del = (int64_t)tk.del_u.size();
    u.del_u = tk.del_u.data();
    u.del_v = tk.del_v.data();
    u.n_del_nodes = (int64_t)tk.del_nodes.size();
    u.del_nodes = tk.del_nodes.data();
    u.on_device = 0;
    tk.t_start = Clock::now();
    const grest_status st = grest_apply_update(g.ctx, &u, &tk.stats);
    tk.t_end = Clock::now();
    int64_t nb = g.bytes;
    grest_get_device_bytes(g.ctx, &nb);  // buffers may have grown for this batch
    lk.lock();
    sv->used += nb - g.bytes;
    g.bytes = nb;
    tk.status = st;
    tk.done = true;
    g.busy = false;
    g.last_used = tk.t_end;
    g.evict_failed = false;
    if (g.removed && g.queue.empty()) release(sv, g);
    sv->cv.notify_all();
  }
}

template <typename T>
void copy_in(std::vector<T>& dst, const T* src, int64_t n) {
  dst.assign(src, src + n);
}

}  // namespace

grest_status grest_server_create(int32_t n_workers, int64_t hbm_budget_bytes, grest_server** out) {
  if (!out || n_workers < 1 || hbm_budget_bytes < 0) return GREST_ERR_INVALID_ARG;
  *out = nullptr;
  grest_server* sv = new grest_server;
  if (cudaGetDevice(&sv->dev) != cudaSuccess) {
    delete sv;
    return GREST_ERR_CUDA;
  }
  sv->budget = hbm_budget_bytes;
  for (int i = 0; i < n_workers; ++i) sv->workers.emplace_back(worker, sv);
  *out = sv;
  return GREST_OK;
}

grest_status grest_server_add_graph(grest_server* sv, const grest_config* cfg, int64_t n, const int64_t* rowptr,
                                    const int32_t* col, const double* val, const double* U0, const double* theta0,
                                    int32_t* graph_id) {
  if (!sv || !cfg || !graph_id || n < 1 || !rowptr || (!col && rowptr[n] > 0)) return GREST_ERR_INVALID_ARG;
  if ((U0 == nullptr) != (theta0 == nullptr)) return GREST_ERR_INVALID_ARG;
  std::unique_ptr<Graph> g(new Graph);
  g->cfg = *cfg;
  g->n = n;
  copy_in(g->rowptr, rowptr, n + 1);
  copy_in(g->col, col, rowptr[n]);
  if (val) {
    copy_in(g->val, val, rowptr[n]);
    g->has_val = true;
  }
  if (U0) {
    copy_in(g->U0, U0, n * (int64_t)cfg->k);
    copy_in(g->theta0, theta0, cfg->k);
    g->has_pairs = true;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  *graph_id = (int32_t)sv->graphs.size();
  sv->graphs.push_back(std::move(g));
  return GREST_OK;
}

grest_status grest_server_submit(grest_server* sv, int32_t graph_id, const grest_update* u, int64_t* ticket) {
  if (!sv || !u || !ticket || u->on_device) return GREST_ERR_INVALID_ARG;
  if (u->n_new_nodes < 0 || u->n_ins < 0 || u->n_del < 0 || u->n_del_nodes < 0) return GREST_ERR_INVALID_ARG;
  if ((u->n_ins > 0 && (!u->ins_u || !u->ins_v)) || (u->n_del > 0 && (!u->del_u || !u->del_v)) ||
      (u->n_del_nodes > 0 && !u->del_nodes))
    return GREST_ERR_INVALID_ARG;
  std::unique_ptr<Ticket> tk(new Ticket);
  tk->n_new = u->n_new_nodes;
  copy_in(tk->ins_u, u->ins_u, u->n_ins);
  copy_in(tk->ins_v, u->ins_v, u->n_ins);
  if (u->ins_w) {
    copy_in(tk->ins_w, u->ins_w, u->n_ins);
    tk->has_w = true;
  }
  copy_in(tk->del_u, u->del_u, u->n_del);
  copy_in(tk->del_v, u->del_v, u->n_del);
  copy_in(tk->del_nodes, u->del_nodes, u->n_del_nodes);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (graph_id < 0 || graph_id >= (int32_t)sv->graphs.size() || sv->graphs[graph_id]->removed)
    return GREST_ERR_INVALID_ARG;
  tk->graph = graph_id;
  tk->t_submit = Clock::now();
  *ticket = (int64_t)sv->tickets.size();
  sv->tickets.push_back(std::move(tk));
  sv->graphs[graph_id]->queue.push_back(*ticket);
  sv->cv.notify_all();
  return GREST_OK;
}

grest_status grest_server_wait(grest_server* sv, int64_t ticket, grest_status* result, grest_stats* stats,
                               double* wait_ms, double* run_ms) {
  if (!sv) return GREST_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (ticket < 0 || ticket >= (int64_t)sv->tickets.size()) return GREST_ERR_INVALID_ARG;
  Ticket& tk = *sv->tickets[ticket];
  sv->cv.wait(lk, [&] { return tk.done; });
  if (result) *result = tk.status;
  if (stats) *stats = tk.stats;
  if (wait_ms) *wait_ms = std::chrono::duration<double, std::milli>(tk.t_start - tk.t_submit).count();
  if (run_ms) *run_ms = std::chrono::duration<double, std::milli>(tk.t_end - tk.t_start).count();
  return GREST_OK;
}

grest_status grest_server_poll(grest_server* sv, int64_t ticket, int32_t* done) {
  if (!sv || !done) return GREST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (ticket < 0 || ticket >= (int64_t)sv->tickets.size()) return GREST_ERR_INVALID_ARG;
  *done = sv->tickets[ticket]->done ? 1 : 0;
  return GREST_OK;
}

grest_status grest_server_remove_graph(grest_server* sv, int32_t graph_id) {
  if (!sv) return GREST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (graph_id < 0 || graph_id >= (int32_t)sv->graphs.size() || sv->graphs[graph_id]->removed)
    return GREST_ERR_INVALID_ARG;
  Graph& g = *sv->graphs[graph_id];
  g.removed = true;
  std::vector<uint8_t>().swap(g.ckpt);
  if (!g.busy && g.queue.empty()) release(sv, g);
  sv->cv.notify_all();
  return GREST_OK;
}

grest_status grest_server_get_embedding(grest_server* sv, int32_t graph_id, double* U, double* theta, uint8_t* live,
                                        int64_t* n_out) {
  if (!sv || !n_out) return GREST_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (graph_id < 0 || graph_id >= (int32_t)sv->graphs.size()) return GREST_ERR_INVALID_ARG;
  Graph& g = *sv->graphs[graph_id];
  sv->cv.wait(lk, [&] { return !g.busy && g.queue.empty(); });
  if (!g.resident && !g.ckpt.empty())  // evicted: read the checkpoint
    return grest_checkpoint_embedding(g.ckpt.data(), (int64_t)g.ckpt.size(), U, theta, live, n_out, nullptr);
  if (!g.resident) return GREST_ERR_INVALID_ARG;  // never admitted, or removed
  g.busy = true;  // no worker takes it while the copy runs
  lk.unlock();
  const grest_status st = grest_get_embedding(g.ctx, U, theta, live, n_out, 0);
  lk.lock();
  g.busy = false;
  sv->cv.notify_all();
  return st;
}

grest_status grest_server_resident(grest_server* sv, int64_t* bytes, int32_t* n_resident) {
  if (!sv) return GREST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (bytes) *bytes = sv->used;
  if (n_resident) *n_resident = sv->n_resident;
  return GREST_OK;
}

grest_status grest_server_set_eviction(grest_server* sv, int32_t on) {
  if (!sv || (on != 0 && on != 1)) return GREST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->evict = on != 0;
  sv->cv.notify_all();
  return GREST_OK;
}

grest_status grest_server_counters(grest_server* sv, int64_t* admissions, int64_t* evictions, int64_t* restores) {
  if (!sv) return GREST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (admissions) *admissions = sv->n_admissions;
  if (evictions) *evictions = sv->n_evictions;
  if (restores) *restores = sv->n_restores;
  return GREST_OK;
}

void grest_server_destroy(grest_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (auto& t : sv->workers) t.join();
  cudaSetDevice(sv->dev);
  for (auto& g : sv->graphs) {
    fail_queue(sv, *g, GREST_ERR_INVALID_ARG);
    release(sv, *g);
  }
  delete sv;
}

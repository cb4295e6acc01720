// serve.cu -- many constructions at once on one GPU.
//
// A server owns W worker threads; each worker owns a context (its own CUDA
// stream and scratch), so the kernels of up to W requests run concurrently
// on the device.  A request is admitted when its worst-case device footprint
// fits the memory budget next to what is already charged (continuous
// admission: a request that arrives while others run starts as soon as a
// worker and enough memory are free).  A finished graph stays charged at its
// real size until dbg_graph_free.  A request whose footprint exceeds the
// whole budget is built by the key-range bucket path (dbg_build_bucketed),
// with the part of the budget that is free when it starts.  A build that
// still runs out of device memory (memory taken outside the budget) waits
// until another request finishes and runs again; alone, it fails.
// dbg_build_batch runs a set of read sets through a transient server.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dbg_internal.h"

namespace dbg {
namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t) {
  return std::chrono::duration<double>(t - t0).count();
}

struct Request {
  uint64_t ticket = 0;
  const char *reads = nullptr;
  const uint32_t *lengths = nullptr;
  uint64_t n = 0;
  uint32_t k = 0;
  uint64_t footprint = 0;  // worst-case peak bytes of the in-memory build
  uint64_t charge = 0;     // bytes charged while it runs
  uint64_t retry_after = 0;  // ran out of memory: wait for a finish after this count
  uint32_t retries = 0;
  bool bucketed = false;
  Clock::time_point submitted, started, finished;
  bool done = false;
  dbg_status status = DBG_OK;
  dbg_graph *graph = nullptr;
  std::string error;
};

}  // namespace
}  // namespace dbg

struct dbg_server {
  int device = 0;
  uint64_t budget = 0;
  // charged bytes, and the lock and wake-up of the queue; graphs the server
  // built hold a reference until they are freed
  std::shared_ptr<dbg::BudgetShare> bud = std::make_shared<dbg::BudgetShare>();
  uint32_t running = 0, peak_running = 0;
  uint64_t finishes = 0, peak_charged = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::condition_variable cv_done;
  cudaStream_t admit_stream = nullptr;  // copies of device-resident lengths at submission
  std::deque<std::shared_ptr<dbg::Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<dbg::Request>> all;
  std::vector<std::thread> workers;
  std::vector<dbg_ctx *> ctxs;
  dbg::Clock::time_point t0 = dbg::Clock::now();
  uint32_t tune_variants[4] = {0, 0, 0, 0};
  bool have_tuning = false;
};

namespace dbg {

// Worst-case peak device bytes of one in-memory build (dbg_build), from
// the buffers it holds at once when every edge instance is a distinct edge
// (E = N, R = 2N + I node records, V <= R nodes) and every group of the
// hybrid sort's local pass is too long for shared memory (its copies
// gathered and sorted over every digit).  The fullest points are the
// edge-key sort (A), the node-record sort (B) and the node-ID pass (C).
uint64_t build_footprint(uint64_t n, uint64_t bases, uint64_t N, uint64_t I, uint32_t k, bool reads_on_host,
                         bool lengths_on_host) {
  const uint64_t w = k <= 31 ? 8 : 16;
  const uint64_t E = N, R = 2 * N + I, V = R;
  // per-read offsets, packed reads, the device copy of host lengths, the
  // two staging buffers of host reads
  const uint64_t inputs = 16 * (n + 1) + bases / 4 + 64 + (lengths_on_host ? 4 * n : 0) +
                          (reads_on_host ? 2 * std::min<uint64_t>(bases, 256ull << 20) : 0);
  // two key buffers, the local pass's count staging, gathered oversize keys
  // (two buffers, their distinct keys and run heads)
  const uint64_t A = 2 * N * w + 4 * N + 3 * N * w + 4 * N;
  // the distinct keys' buffer and counts, the graph's edge arrays, two
  // record buffers (key + payload) and the gathered oversize records
  const uint64_t B = N * w + 4 * E + E * (w + 5) + 4 * R * (w + 4);
  // records, row offsets, edge arrays, src / dst, adjacency with its sides,
  // partitioned edge ends, node keys and row_ptr
  const uint64_t C = 2 * R * (w + 4) + 8 * (R + 1) + E * (w + 5) + 8 * E + 20 * E + 16 * E + V * (w + 8);
  const uint64_t tiles = N / 2048 + 1;  // per-tile bounds, counts and scan words
  return inputs + std::max({A, B, C}) + 64 * tiles + (64ull << 20);
}

// Bytes to charge for request r now (bucketed: what is free, once that is
// at least a quarter of what it would like), or 0 if it must wait.  Called under the
// budget lock.
static uint64_t admit_charge(const dbg_server *srv, const Request &r) {
  const uint64_t in_use = srv->bud->in_use;
  const bool alone = srv->running == 0;
  if (srv->finishes < r.retry_after && !alone) return 0;
  if (!r.bucketed) return (alone || in_use + r.footprint <= srv->budget) ? std::max<uint64_t>(1, r.footprint) : 0;
  const uint64_t want = std::min(r.footprint, srv->budget);
  const uint64_t free_b = srv->budget > in_use ? srv->budget - in_use : 0;
  if (free_b > 0 && free_b >= want / 4) return free_b;
  return alone ? std::max<uint64_t>({free_b, want / 4, 1ull << 20}) : 0;
}

static void worker_main(dbg_server *srv, int idx) {
  cudaSetDevice(srv->device);
  dbg_ctx *ctx = srv->ctxs[idx];
  BudgetShare &bud = *srv->bud;
  for (;;) {
    std::shared_ptr<Request> req;
    {
      std::unique_lock<std::mutex> lk(bud.mu);
      for (;;) {
        if (srv->stopping && srv->queue.empty()) return;
        // admission: the first queued request that fits next to what is charged
        auto it = srv->queue.begin();
        uint64_t charge = 0;
        for (; it != srv->queue.end(); ++it)
          if ((charge = admit_charge(srv, **it)) != 0) break;
        if (it != srv->queue.end()) {
          req = *it;
          srv->queue.erase(it);
          req->charge = charge;
          bud.in_use += charge;
          srv->running++;
          srv->peak_running = std::max(srv->peak_running, srv->running);
          srv->peak_charged = std::max(srv->peak_charged, bud.in_use);
          break;
        }
        bud.cv.wait(lk);
      }
    }
    req->started = Clock::now();
    dbg_graph *g = nullptr;
    dbg_status st;
    if (req->bucketed)
      st = dbg_build_bucketed(ctx, req->reads, req->lengths, req->n, req->k, req->charge, &g);
    else
      st = dbg_build(ctx, req->reads, req->lengths, req->n, req->k, &g);
    if (g) {
      // the graph outlives this worker's stream: free it in legacy-stream order
      g->al.stream = nullptr;
      g->budget = srv->bud;
      g->charged = g->device_bytes();
    }
    bool requeued = false;
    {
      std::lock_guard<std::mutex> lk(bud.mu);
      bud.in_use -= std::min(bud.in_use, req->charge);
      srv->running--;
      if (st == DBG_ENOMEM && srv->running > 0) {
        // memory taken outside the budget: run again after another finish
        req->retry_after = srv->finishes + 1;
        req->retries++;
        srv->queue.push_front(req);
        requeued = true;
      } else {
        srv->finishes++;
        req->finished = Clock::now();
        req->status = st;
        req->graph = g;
        if (g) bud.in_use += g->charged;
        if (st != DBG_OK) req->error = dbg_last_error();
        req->done = true;
      }
    }
    (void)requeued;
    srv->cv_done.notify_all();
    bud.cv.notify_all();
  }
}

}  // namespace dbg

using namespace dbg;

extern "C" {

void dbg_server_options_init(dbg_server_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(dbg_server_options);
  o->device = -1;
  o->workers = 4;
}

dbg_status dbg_server_create(dbg_server **out, const dbg_server_options *opt) {
  if (!out) return DBG_EINVAL;
  *out = nullptr;
  dbg_server_options o;
  dbg_server_options_init(&o);
  if (opt) std::memcpy(&o, opt, std::min<size_t>(opt->struct_size ? opt->struct_size : sizeof(o), sizeof(o)));
  int dev = o.device;
  if (dev < 0) DBG_CUDA_TRY(cudaGetDevice(&dev));
  DBG_CUDA_TRY(cudaSetDevice(dev));
  if (o.workers < 1 || o.workers > 64) {
    set_error("workers must be in [1, 64]");
    return DBG_EINVAL;
  }
  dbg_server *srv = new (std::nothrow) dbg_server();
  if (!srv) return DBG_ENOMEM;
  srv->device = dev;
  if (cudaStreamCreateWithFlags(&srv->admit_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete srv;
    set_error("cudaStreamCreateWithFlags failed");
    return DBG_ECUDA;
  }
  size_t free_b = 0, total_b = 0;
  DBG_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
  srv->budget = o.mem_budget ? o.mem_budget : (uint64_t)(0.8 * (double)free_b);
  for (uint32_t i = 0; i < o.workers; i++) {
    dbg_options co;
    dbg_options_init(&co);
    co.device = dev;
    co.spin_limit = o.spin_limit;
    dbg_ctx *c = nullptr;
    dbg_status st = dbg_create(&c, &co);
    if (st != DBG_OK) {
      for (dbg_ctx *x : srv->ctxs) dbg_destroy(x);
      cudaStreamDestroy(srv->admit_stream);
      delete srv;
      return st;
    }
    for (int kd = 0; kd < 4; kd++) c->sort_variant[kd] = o.sort_variant[kd];
    srv->ctxs.push_back(c);
  }
  for (uint32_t i = 0; i < o.workers; i++) srv->workers.emplace_back(worker_main, srv, (int)i);
  *out = srv;
  return DBG_OK;
}

void dbg_server_destroy(dbg_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->bud->mu);
    srv->stopping = true;
  }
  srv->bud->cv.notify_all();
  for (auto &t : srv->workers) t.join();
  for (auto &kv : srv->all)
    if (kv.second->graph) dbg_graph_free(kv.second->graph);
  for (dbg_ctx *c : srv->ctxs) dbg_destroy(c);
  cudaStreamDestroy(srv->admit_stream);
  delete srv;
}

uint64_t dbg_server_budget(const dbg_server *srv) { return srv ? srv->budget : 0; }

uint64_t dbg_server_charged(const dbg_server *srv) {
  if (!srv) return 0;
  std::lock_guard<std::mutex> lk(srv->bud->mu);
  return srv->bud->in_use;
}

dbg_status dbg_server_stats(const dbg_server *srv, dbg_server_counters *out) {
  if (!srv || !out) return DBG_EINVAL;
  std::lock_guard<std::mutex> lk(srv->bud->mu);
  out->charged = srv->bud->in_use;
  out->peak_charged = srv->peak_charged;
  out->finished = srv->finishes;
  out->running = srv->running;
  out->peak_running = srv->peak_running;
  out->queued = (uint32_t)srv->queue.size();
  return DBG_OK;
}

dbg_status dbg_submit(dbg_server *srv, const dbg_readset *req, uint64_t *ticket) {
  if (!srv || !req || !ticket) return DBG_EINVAL;
  if (req->k < 1 || req->k > 63 || (req->k % 2) == 0) {
    set_error("k = %u: k must be odd and in [1, 63]", req->k);
    return DBG_EINVAL;
  }
  if (req->n > 0 && (!req->reads || !req->lengths)) {
    set_error("reads or lengths is NULL");
    return DBG_EINVAL;
  }
  auto on_device = [](const void *p) {
    cudaPointerAttributes a;
    const bool dev = cudaPointerGetAttributes(&a, p) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return dev;
  };
  const bool host_len = req->n == 0 || !on_device(req->lengths);
  const bool host_reads = req->n > 0 && !on_device(req->reads);
  // the sums the footprint needs: bases, edge instances, reads of length k
  // (device-resident lengths are copied to the host first)
  std::vector<uint32_t> staged;
  const uint32_t *len = req->lengths;
  if (!host_len) {
    staged.resize(req->n);
    DBG_CUDA_TRY(cudaMemcpyAsync(staged.data(), req->lengths, req->n * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                 srv->admit_stream));
    DBG_CUDA_TRY(cudaStreamSynchronize(srv->admit_stream));
    len = staged.data();
  }
  uint64_t bases = 0, N = 0, I = 0;
  for (uint64_t i = 0; i < req->n; i++) {
    bases += len[i];
    N += len[i] > req->k ? len[i] - req->k : 0;
    I += len[i] == req->k;
  }
  auto r = std::make_shared<Request>();
  r->reads = req->reads;
  r->lengths = req->lengths;
  r->n = req->n;
  r->k = req->k;
  r->footprint = build_footprint(req->n, bases, N, I, req->k, host_reads, host_len);
  r->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(srv->bud->mu);
    r->bucketed = r->footprint > srv->budget || (req->flags & DBG_REQ_BUCKETED);
    r->ticket = srv->next_ticket++;
    srv->all[r->ticket] = r;
    srv->queue.push_back(r);
    *ticket = r->ticket;
  }
  srv->bud->cv.notify_all();
  return DBG_OK;
}

dbg_status dbg_poll(dbg_server *srv, uint64_t ticket, int wait, dbg_graph **out, dbg_request_stats *stats) {
  if (!srv || !out) return DBG_EINVAL;
  *out = nullptr;
  std::unique_lock<std::mutex> lk(srv->bud->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return DBG_EINVAL;
  }
  auto r = it->second;
  if (!r->done) {
    if (!wait) return DBG_EAGAIN;
    srv->cv_done.wait(lk, [&] { return r->done; });
  }
  if (stats) {
    stats->queue_s = seconds_since(r->submitted, r->started);
    stats->run_s = seconds_since(r->started, r->finished);
    stats->latency_s = seconds_since(r->submitted, r->finished);
    stats->footprint = r->footprint;
    stats->bucketed = r->bucketed ? 1 : 0;
    stats->retries = r->retries;
    stats->charged = r->charge;
  }
  srv->all.erase(it);
  if (r->status != DBG_OK) {
    set_error("%s", r->error.c_str());
    return r->status;
  }
  *out = r->graph;
  r->graph = nullptr;
  return DBG_OK;
}

dbg_status dbg_build_batch(dbg_ctx *ctx, const dbg_readset *sets, uint32_t nsets, uint32_t workers,
                           dbg_graph **outs) {
  if (!ctx || (nsets > 0 && (!sets || !outs))) return DBG_EINVAL;
  for (uint32_t i = 0; i < nsets; i++) outs[i] = nullptr;
  if (nsets == 0) return DBG_OK;
  dbg_server_options o;
  dbg_server_options_init(&o);
  o.device = ctx->device;
  o.workers = workers ? workers : 4;
  o.mem_budget = ctx->mem_budget;
  o.spin_limit = ctx->spin_limit;
  for (int kd = 0; kd < 4; kd++) o.sort_variant[kd] = ctx->sort_variant[kd];
  dbg_server *srv = nullptr;
  DBG_TRY(dbg_server_create(&srv, &o));
  std::vector<uint64_t> tickets(nsets);
  dbg_status st = DBG_OK;
  for (uint32_t i = 0; i < nsets && st == DBG_OK; i++) st = dbg_submit(srv, &sets[i], &tickets[i]);
  for (uint32_t i = 0; i < nsets; i++) {
    if (!tickets[i]) continue;
    dbg_graph *g = nullptr;
    dbg_status s = dbg_poll(srv, tickets[i], 1, &g, nullptr);
    if (s != DBG_OK && st == DBG_OK) st = s;
    outs[i] = g;
  }
  dbg_server_destroy(srv);
  if (st != DBG_OK) {
    for (uint32_t i = 0; i < nsets; i++) {
      dbg_graph_free(outs[i]);
      outs[i] = nullptr;
    }
  }
  return st;
}

}  // extern "C"

// serve.cu -- many constructions at once on one GPU.
//
// A server owns W worker threads; each worker owns a context (its own CUDA
// stream and scratch), so the kernels of up to W requests run concurrently
// on the device.  A request is admitted when its estimated device footprint
// fits the memory budget next to the requests already running (continuous
// admission: a request that arrives while others run starts as soon as a
// worker and enough memory are free).  A request whose footprint exceeds the
// whole budget is built by the key-range bucket path (dbg_build_bucketed),
// which keeps only one key range of its edges on the device at a time.
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
  uint64_t footprint = 0;
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
  uint64_t in_use = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<dbg::Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<dbg::Request>> all;
  std::vector<std::thread> workers;
  std::vector<dbg_ctx *> ctxs;
  dbg::Clock::time_point t0 = dbg::Clock::now();
  uint32_t tune_variants[4] = {0, 0, 0, 0};
  bool have_tuning = false;
};

namespace dbg {

// Estimated peak device bytes of one in-memory build: two key buffers and
// run heads for N edge instances, packed and ASCII reads, per-read
// offsets, and node records of up to 2 per instance (the worst case when
// every instance is a distinct edge is 2N records; builds of real read sets
// keep far fewer, and a quarter of that bound is charged).
uint64_t build_footprint(const uint32_t *lengths, uint64_t n, uint32_t k, bool lengths_on_host) {
  uint64_t bases = 0, N = 0;
  if (lengths_on_host) {
    for (uint64_t r = 0; r < n; r++) {
      bases += lengths[r];
      N += lengths[r] > k ? lengths[r] - k : 0;
    }
  }
  const uint64_t w = k <= 31 ? 8 : 16;
  const uint64_t keys = N * (2 * w + 4);
  const uint64_t reads = bases + bases / 4 + n * 24;
  const uint64_t records = (2 * N / 4) * (w + 4) * 2;
  const uint64_t graph = (N / 4) * (w + 13 + 2 * 9) + (N / 4) * (w + 8);
  return keys + reads + records + graph + (64ull << 20);
}

static void worker_main(dbg_server *srv, int idx) {
  cudaSetDevice(srv->device);
  dbg_ctx *ctx = srv->ctxs[idx];
  for (;;) {
    std::shared_ptr<Request> req;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      for (;;) {
        if (srv->stopping && srv->queue.empty()) return;
        // admission: the first queued request that fits next to the running ones
        auto it = srv->queue.begin();
        for (; it != srv->queue.end(); ++it) {
          const auto &r = *it;
          const uint64_t need = r->bucketed ? std::min<uint64_t>(r->footprint, srv->budget) : r->footprint;
          if (srv->in_use + need <= srv->budget || srv->in_use == 0) break;
        }
        if (it != srv->queue.end()) {
          req = *it;
          srv->queue.erase(it);
          srv->in_use += req->bucketed ? std::min<uint64_t>(req->footprint, srv->budget) : req->footprint;
          break;
        }
        srv->cv_work.wait(lk);
      }
    }
    req->started = Clock::now();
    dbg_graph *g = nullptr;
    dbg_status st;
    if (req->bucketed)
      st = dbg_build_bucketed(ctx, req->reads, req->lengths, req->n, req->k, srv->budget, &g);
    else
      st = dbg_build(ctx, req->reads, req->lengths, req->n, req->k, &g);
    if (g) {
      // the graph outlives this worker's stream: free it in legacy-stream order
      g->al.stream = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      req->finished = Clock::now();
      req->status = st;
      req->graph = g;
      if (st != DBG_OK) req->error = dbg_last_error();
      req->done = true;
      srv->in_use -= req->bucketed ? std::min<uint64_t>(req->footprint, srv->budget) : req->footprint;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
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
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stopping = true;
  }
  srv->cv_work.notify_all();
  for (auto &t : srv->workers) t.join();
  for (auto &kv : srv->all)
    if (kv.second->graph) dbg_graph_free(kv.second->graph);
  for (dbg_ctx *c : srv->ctxs) dbg_destroy(c);
  delete srv;
}

uint64_t dbg_server_budget(const dbg_server *srv) { return srv ? srv->budget : 0; }

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
  cudaPointerAttributes a;
  bool host_len = true;
  if (req->n > 0 && cudaPointerGetAttributes(&a, req->lengths) == cudaSuccess)
    host_len = !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  auto r = std::make_shared<Request>();
  r->reads = req->reads;
  r->lengths = req->lengths;
  r->n = req->n;
  r->k = req->k;
  r->footprint = build_footprint(req->lengths, req->n, req->k, host_len);
  r->submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    r->bucketed = r->footprint > srv->budget || (req->flags & DBG_REQ_BUCKETED);
    r->ticket = srv->next_ticket++;
    srv->all[r->ticket] = r;
    srv->queue.push_back(r);
    *ticket = r->ticket;
  }
  srv->cv_work.notify_one();
  return DBG_OK;
}

dbg_status dbg_poll(dbg_server *srv, uint64_t ticket, int wait, dbg_graph **out, dbg_request_stats *stats) {
  if (!srv || !out) return DBG_EINVAL;
  *out = nullptr;
  std::unique_lock<std::mutex> lk(srv->mu);
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

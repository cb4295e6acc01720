// api.cu -- the C ABI: contexts, device memory, dbg_build and the graph
// accessors.  Every compute step runs in the CUDA kernels of this library.
#include <initializer_list>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "dbg_device.cuh"
#include "dbg_internal.h"

namespace dbg {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void *Allocator::get(size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (alloc) return alloc(user, bytes, (void *)stream);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void Allocator::put(void *p, size_t bytes) {
  if (!p) return;
  if (free) {
    free(user, p, bytes, (void *)stream);
    return;
  }
  cudaFreeAsync(p, stream);
}

dbg_status alloc_buf(dbg_ctx *ctx, DevBuf &b, size_t bytes) {
  b.release();
  b.al = &ctx->al;
  b.p = ctx->al.get(bytes);
  if (!b.p) {
    set_error("device allocation of %zu bytes failed", bytes);
    return DBG_ENOMEM;
  }
  b.bytes = bytes;
  return DBG_OK;
}

dbg_status ensure_status(dbg_ctx *ctx, size_t words) {
  if (words <= ctx->status_words) return DBG_OK;
  size_t want = std::max(words, ctx->status_words * 2);
  if (ctx->d_status) cudaFreeAsync(ctx->d_status, ctx->stream);
  ctx->d_status = nullptr;
  ctx->status_words = 0;
  DBG_CUDA_TRY(cudaMallocAsync((void **)&ctx->d_status, want * sizeof(uint64_t), ctx->stream));
  DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, want * sizeof(uint64_t), ctx->stream));
  ctx->status_words = want;
  return DBG_OK;
}

dbg_status copy_spread(cudaStream_t *streams, int n_streams, int *next, void *dst, const void *src, size_t bytes) {
  // chunks of at least 32 MB, at most one per stream and array
  const size_t chunk = std::max<size_t>((size_t)32 << 20, (bytes + n_streams - 1) / n_streams);
  for (size_t off = 0; off < bytes; off += chunk) {
    const size_t b = std::min(chunk, bytes - off);
    DBG_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off, b,
                                 cudaMemcpyDefault, streams[*next]));
    *next = (*next + 1) % n_streams;
  }
  return DBG_OK;
}

dbg_status ensure_copy_stream(dbg_ctx *ctx) {
  if (!ctx->copy_stream) DBG_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  return DBG_OK;
}

dbg_status next_epoch(dbg_ctx *ctx, uint32_t *epoch) {
  if (ctx->epoch >= 0x3fffffffu) {
    // the 30-bit epoch wrapped: old words could look current again
    if (ctx->d_status)
      DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, ctx->status_words * sizeof(uint64_t), ctx->stream));
    ctx->epoch = 1;
  }
  *epoch = ctx->epoch++;
  return DBG_OK;
}

dbg_status check_device_error(dbg_ctx *ctx) {
  DBG_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
  DBG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  uint32_t e = ctx->h_pinned[0];
  if (e == 0) return DBG_OK;
  DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream));
  if (e & ERR_BAD_BASE) {
    set_error("a read holds a byte outside {A,C,G,T}");
    return DBG_EINVAL;
  }
  if (e & ERR_TIMEOUT) {
    set_error("a device-side wait reached its spin limit");
    return DBG_ETIMEOUT;
  }
  if (e & ERR_OVERFLOW) {
    set_error("a device count overflowed its 32-bit field");
    return DBG_EOVERFLOW;
  }
  set_error("device consistency check failed (code %u)", e);
  return DBG_EINTERNAL;
}

const char *const kStageNames[ST_COUNT] = {
    "offsets", "pack", "emit", "sort_edges", "rle", "endpoints", "sort_nodes", "node_ids",
    "adjacency", "copies", "compact_links", "compact_rank", "compact_cycles", "compact_output",
    "local_sort_edges", "local_sort_nodes", "partition_edges", "node_mult"};

static cudaEvent_t pool_event(dbg_ctx *ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

Span::Span(dbg_ctx *c, int st, double algo_bytes, uint32_t n_launches)
    : ctx(c), stage(st), bytes(algo_bytes), launches(n_launches) {
  ctx->launches += n_launches;
  if (ctx->prof && (a = pool_event(ctx))) cudaEventRecord(a, ctx->stream);
}

Span::~Span() {
  if (!a) return;
  cudaEvent_t b = pool_event(ctx);
  if (!b) {
    ctx->ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, ctx->stream);
  ctx->pending.push_back(ProfRecord{stage, a, b, bytes, launches});
}

void prof_resolve(dbg_ctx *ctx) {
  for (auto &r : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      dbg_stage_stat &st = ctx->stats[r.stage];
      st.launches += r.launches;
      st.ms += ms;
      st.bytes += r.bytes;
    } else {
      cudaGetLastError();
    }
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->pending.clear();
}

dbg_status read_small(dbg_ctx *ctx, const void *d_src, size_t bytes, void *h_dst) {
  DBG_CUDA_TRY(cudaMemcpyAsync(ctx->h_pinned, d_src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  DBG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  std::memcpy(h_dst, ctx->h_pinned, bytes);
  return DBG_OK;
}

dbg_status copy_out(dbg_ctx *ctx, void *dst, const void *src, size_t bytes) {
  if (!bytes) return DBG_OK;
  DBG_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
  DBG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return DBG_OK;
}

// Sets the context's device for the scope of one call.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

static bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace dbg

using namespace dbg;

extern "C" {

void dbg_options_init(dbg_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->struct_size = sizeof(dbg_options);
  opt->device = -1;
}

const char *dbg_last_error(void) { return g_last_error.c_str(); }

dbg_status dbg_create(dbg_ctx **out, const dbg_options *opt) {
  if (!out) return DBG_EINVAL;
  *out = nullptr;
  dbg_options o;
  dbg_options_init(&o);
  if (opt) {
    if (opt->struct_size < offsetof(dbg_options, reserved)) {
      set_error("dbg_options.struct_size too small");
      return DBG_EINVAL;
    }
    std::memcpy(&o, opt, std::min<size_t>(opt->struct_size, sizeof(o)));
  }
  int dev = o.device;
  if (dev < 0) DBG_CUDA_TRY(cudaGetDevice(&dev));
  DeviceScope scope(dev);
  dbg_ctx *ctx = new (std::nothrow) dbg_ctx();
  if (!ctx) return DBG_ENOMEM;
  ctx->device = dev;
  dbg_status st = DBG_OK;
  auto fail = [&](const char *what, cudaError_t e) {
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    st = DBG_ECUDA;
  };
  cudaError_t e;
  if (o.stream) {
    ctx->stream = (cudaStream_t)o.stream;
  } else if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess) {
    fail("cudaStreamCreate", e);
  } else {
    ctx->own_stream = true;
  }
  ctx->al.alloc = o.alloc;
  ctx->al.free = o.free;
  ctx->al.user = o.alloc_user;
  ctx->al.stream = ctx->stream;
  ctx->mem_budget = o.mem_budget;
  if (o.spin_limit) ctx->spin_limit = o.spin_limit;
  if (st == DBG_OK && (e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    fail("cudaDeviceGetAttribute", e);
  if (st == DBG_OK && !o.alloc) {
    // keep freed blocks in the device pool instead of returning them to the driver
    cudaMemPool_t pool;
    if ((e = cudaDeviceGetDefaultMemPool(&pool, dev)) != cudaSuccess) fail("cudaDeviceGetDefaultMemPool", e);
    uint64_t thr = UINT64_MAX;
    if (st == DBG_OK && (e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr)) != cudaSuccess)
      fail("cudaMemPoolSetAttribute", e);
  }
  if (st == DBG_OK && (e = cudaMalloc((void **)&ctx->d_err, 256)) != cudaSuccess) fail("cudaMalloc", e);
  if (st == DBG_OK && (e = cudaMemset(ctx->d_err, 0, 256)) != cudaSuccess) fail("cudaMemset", e);
  if (st == DBG_OK) ctx->d_counters = ctx->d_err + 16;
  if (st == DBG_OK && (e = cudaMallocHost((void **)&ctx->h_pinned, 4096)) != cudaSuccess) fail("cudaMallocHost", e);
  if (st == DBG_OK && (e = cudaEventCreateWithFlags(&ctx->ev, cudaEventDisableTiming)) != cudaSuccess)
    fail("cudaEventCreate", e);
  if (st != DBG_OK) {
    dbg_destroy(ctx);
    return st;
  }
  *out = ctx;
  return DBG_OK;
}

dbg_status dbg_profile_enable(dbg_ctx *ctx, int on) {
  if (!ctx) return DBG_EINVAL;
  DeviceScope scope(ctx->device);
  DBG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  prof_resolve(ctx);
  ctx->prof = on != 0;
  std::memset(ctx->stats, 0, sizeof(ctx->stats));
  for (int i = 0; i < ST_COUNT; i++) std::snprintf(ctx->stats[i].name, sizeof(ctx->stats[i].name), "%s", kStageNames[i]);
  return DBG_OK;
}

uint32_t dbg_profile_read(dbg_ctx *ctx, dbg_stage_stat *out, uint32_t cap) {
  if (!ctx) return 0;
  DeviceScope scope(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  for (uint32_t i = 0; i < cap && i < ST_COUNT; i++) {
    out[i] = ctx->stats[i];
    std::snprintf(out[i].name, sizeof(out[i].name), "%s", kStageNames[i]);
  }
  return ST_COUNT;
}

uint64_t dbg_launch_count(const dbg_ctx *ctx) { return ctx ? ctx->launches : 0; }

void dbg_destroy(dbg_ctx *ctx) {
  if (!ctx) return;
  DeviceScope scope(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->d_status) cudaFreeAsync(ctx->d_status, ctx->stream);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->ev) cudaEventDestroy(ctx->ev);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

dbg_status dbg_build(dbg_ctx *ctx, const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k,
                     dbg_graph **out) {
  if (!out) {
    set_error("out is NULL");
    return DBG_EINVAL;
  }
  *out = nullptr;
  if (!ctx) {
    set_error("ctx is NULL");
    return DBG_EINVAL;
  }
  if (k < 1 || k > 63 || (k % 2) == 0) {
    set_error("k = %u: k must be odd and in [1, 63]", k);
    return DBG_EINVAL;
  }
  if (n > 0 && (!reads || !lengths)) {
    set_error("reads or lengths is NULL");
    return DBG_EINVAL;
  }
  if (n >= 0xffffffffull) {
    set_error("n = %llu reads exceed one in-memory build", (unsigned long long)n);
    return DBG_EOVERFLOW;
  }
  DeviceScope scope(ctx->device);
  cudaStream_t s = ctx->stream;
  dbg_graph *g = new (std::nothrow) dbg_graph();
  if (!g) return DBG_ENOMEM;
  g->al = ctx->al;
  g->device = ctx->device;
  g->n_copy = ctx->copy_streams;
  // graph arrays must be freed through the graph's own allocator copy
  auto rebind = [&](DevBuf &b) { b.al = &g->al; };

  dbg_status st = DBG_OK;
  DevBuf d_len;
  const uint32_t *len_dev = lengths;
  bool reads_on_dev = true;
  if (n > 0) {
    reads_on_dev = is_device_ptr(reads);
    if (!is_device_ptr(lengths)) {
      st = alloc_buf(ctx, d_len, n * sizeof(uint32_t));
      if (st == DBG_OK && cudaMemcpyAsync(d_len.p, lengths, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        set_error("copy of the read lengths to the device failed");
        st = DBG_ECUDA;
      }
      len_dev = d_len.as<uint32_t>();
    }
  }
  if (st == DBG_OK) {
    // host reads are streamed in by the build once it knows their length
    BuildInput in{reinterpret_cast<const uint8_t *>(reads), len_dev, n, !reads_on_dev, k};
    st = k <= 31 ? build_graph_u64(ctx, in, g) : build_graph_u128(ctx, in, g);
  }
  for (DevBuf *b : {&g->node_keys, &g->edge_keys, &g->src, &g->dst, &g->orient, &g->mult, &g->row_ptr,
                    &g->adj_nbr, &g->adj_edge, &g->adj_role, &g->adj_side, &g->node_mult, &g->node_reads})
    rebind(*b);
  d_len.release();
  cudaStreamSynchronize(s);
  prof_resolve(ctx);
  if (st != DBG_OK) {
    cudaGetLastError();
    cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s);
    dbg_graph_free(g);
    return st;
  }
  *out = g;
  return DBG_OK;
}

dbg_status dbg_build_bucketed(dbg_ctx *ctx, const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k,
                              uint64_t mem_budget, dbg_graph **out) {
  if (!out) {
    set_error("out is NULL");
    return DBG_EINVAL;
  }
  *out = nullptr;
  if (!ctx) {
    set_error("ctx is NULL");
    return DBG_EINVAL;
  }
  if (k < 1 || k > 63 || (k % 2) == 0) {
    set_error("k = %u: k must be odd and in [1, 63]", k);
    return DBG_EINVAL;
  }
  if (n > 0 && (!reads || !lengths)) {
    set_error("reads or lengths is NULL");
    return DBG_EINVAL;
  }
  if (n >= 0xffffffffull) {
    set_error("n = %llu reads exceed one build", (unsigned long long)n);
    return DBG_EOVERFLOW;
  }
  DeviceScope scope(ctx->device);
  cudaStream_t s = ctx->stream;
  if (mem_budget == 0) {
    size_t free_b = 0, total_b = 0;
    DBG_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    mem_budget = free_b / 2;
  }
  dbg_graph *g = new (std::nothrow) dbg_graph();
  if (!g) return DBG_ENOMEM;
  g->al = ctx->al;
  g->device = ctx->device;
  g->n_copy = ctx->copy_streams;
  dbg_status st = DBG_OK;
  DevBuf d_len;
  const uint32_t *len_dev = lengths;
  const bool reads_on_dev = n > 0 && is_device_ptr(reads);
  if (n > 0 && !is_device_ptr(lengths)) {
    st = alloc_buf(ctx, d_len, n * sizeof(uint32_t));
    if (st == DBG_OK && cudaMemcpyAsync(d_len.p, lengths, n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("copy of the read lengths to the device failed");
      st = DBG_ECUDA;
    }
    len_dev = d_len.as<uint32_t>();
  }
  if (st == DBG_OK) {
    BucketInput in{reads, reads_on_dev, len_dev, n, k};
    st = k <= 31 ? build_bucketed_u64(ctx, in, mem_budget, g, &g->edge_buckets, &g->node_buckets)
                 : build_bucketed_u128(ctx, in, mem_budget, g, &g->edge_buckets, &g->node_buckets);
  }
  for (DevBuf *b : {&g->node_keys, &g->edge_keys, &g->src, &g->dst, &g->orient, &g->mult, &g->row_ptr,
                    &g->adj_nbr, &g->adj_edge, &g->adj_role, &g->adj_side})
    b->al = &g->al;
  d_len.release();
  cudaStreamSynchronize(s);
  prof_resolve(ctx);
  if (st != DBG_OK) {
    cudaGetLastError();
    cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s);
    dbg_graph_free(g);
    return st;
  }
  *out = g;
  return DBG_OK;
}

void dbg_graph_buckets(const dbg_graph *g, uint32_t *edge_ranges, uint32_t *node_ranges) {
  if (edge_ranges) *edge_ranges = g ? g->edge_buckets : 0;
  if (node_ranges) *node_ranges = g ? g->node_buckets : 0;
}

namespace dbg {
// one look-back wait on tile 0's word, which nothing writes in this epoch
__global__ void k_selftest_wait(uint64_t *status, uint32_t epoch, uint32_t spin_limit, uint32_t *err) {
  if (threadIdx.x == 0 && blockIdx.x == 0) lookback_exclusive(status, 1, 1, epoch, spin_limit, err);
}
}  // namespace dbg

dbg_status dbg_selftest_wait(dbg_ctx *ctx, uint32_t spin_limit) {
  if (!ctx || spin_limit == 0 || spin_limit > (1u << 20)) {
    set_error("spin_limit must be in [1, 2^20]");
    return DBG_EINVAL;
  }
  DeviceScope scope(ctx->device);
  DBG_TRY(ensure_status(ctx, 2));
  uint32_t epoch;
  DBG_TRY(next_epoch(ctx, &epoch));
  DBG_LAUNCH(ctx, ST_COPIES, 0.0, k_selftest_wait<<<1, 32, 0, ctx->stream>>>(ctx->d_status, epoch, spin_limit, ctx->d_err));
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  prof_resolve(ctx);
  return check_device_error(ctx);
}

uint32_t dbg_graph_k(const dbg_graph *g) { return g ? g->k : 0; }
uint32_t dbg_graph_key_words(const dbg_graph *g) { return g ? g->key_words : 0; }
uint64_t dbg_graph_num_nodes(const dbg_graph *g) { return g ? g->num_nodes : 0; }
uint64_t dbg_graph_num_edges(const dbg_graph *g) { return g ? g->num_edges : 0; }
uint64_t dbg_graph_num_instances(const dbg_graph *g) { return g ? g->num_instances : 0; }

static dbg_status copy_plain(int device, void *dst, const void *src, size_t bytes) {
  if (!dst || !bytes) return DBG_OK;
  DeviceScope scope(device);
  DBG_CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
  return DBG_OK;
}

dbg_status dbg_graph_nodes(const dbg_graph *g, uint64_t *keys) {
  if (!g || (!keys && g->num_nodes)) return DBG_EINVAL;
  return copy_plain(g->device, keys, g->node_keys.p, g->num_nodes * g->key_words * sizeof(uint64_t));
}

dbg_status dbg_graph_edges(const dbg_graph *g, uint64_t *keys, uint32_t *src, uint32_t *dst, uint8_t *orient,
                           uint32_t *mult) {
  if (!g) return DBG_EINVAL;
  const uint64_t E = g->num_edges;
  DBG_TRY(copy_plain(g->device, keys, g->edge_keys.p, E * g->key_words * sizeof(uint64_t)));
  DBG_TRY(copy_plain(g->device, src, g->src.p, E * sizeof(uint32_t)));
  DBG_TRY(copy_plain(g->device, dst, g->dst.p, E * sizeof(uint32_t)));
  DBG_TRY(copy_plain(g->device, orient, g->orient.p, E));
  DBG_TRY(copy_plain(g->device, mult, g->mult.p, E * sizeof(uint32_t)));
  return DBG_OK;
}

dbg_status dbg_graph_node_mult(const dbg_graph *g, uint32_t *mult) {
  if (!g) return DBG_EINVAL;
  if (!g->node_mult.p) {
    set_error("node multiplicities were not counted for this graph (dbg_node_mult_set before dbg_build)");
    return DBG_EINVAL;
  }
  if (g->num_nodes && !mult) return DBG_EINVAL;
  return copy_plain(g->device, mult, g->node_mult.p, g->num_nodes * sizeof(uint32_t));
}

namespace {
struct CopyPart {
  void *dst;
  const void *src;
  size_t bytes;
};
// starts the copies of the given parts on the graph's own copy streams
dbg_status copy_parts_async(dbg_graph *g, std::initializer_list<CopyPart> parts) {
  DeviceScope scope(g->device);
  for (int i = 0; i < g->n_copy; i++)
    if (!g->copy_streams[i]) DBG_CUDA_TRY(cudaStreamCreateWithFlags(&g->copy_streams[i], cudaStreamNonBlocking));
  for (const CopyPart &c : parts)
    if (c.dst && c.bytes) DBG_TRY(copy_spread(g->copy_streams, g->n_copy, &g->copy_next, c.dst, c.src, c.bytes));
  return DBG_OK;
}
}  // namespace



dbg_status dbg_graph_edges_async(dbg_graph *g, uint64_t *keys, uint32_t *src, uint32_t *dst, uint8_t *orient,
                                 uint32_t *mult) {
  if (!g) return DBG_EINVAL;
  const uint64_t E = g->num_edges;
  return copy_parts_async(g, {{keys, g->edge_keys.p, E * g->key_words * sizeof(uint64_t)},
                              {src, g->src.p, E * sizeof(uint32_t)},
                              {dst, g->dst.p, E * sizeof(uint32_t)},
                              {orient, g->orient.p, E},
                              {mult, g->mult.p, E * sizeof(uint32_t)}});
}

dbg_status dbg_graph_nodes_async(dbg_graph *g, uint64_t *keys) {
  if (!g) return DBG_EINVAL;
  return copy_parts_async(g, {{keys, g->node_keys.p, g->num_nodes * g->key_words * sizeof(uint64_t)}});
}

dbg_status dbg_graph_csr_async(dbg_graph *g, uint64_t *row_ptr, uint32_t *nbr, uint32_t *edge, uint8_t *role) {
  if (!g) return DBG_EINVAL;
  const uint64_t A = 2 * g->num_edges;
  return copy_parts_async(g, {{row_ptr, g->row_ptr.p, (g->num_nodes + 1) * sizeof(uint64_t)},
                              {nbr, g->adj_nbr.p, A * sizeof(uint32_t)},
                              {edge, g->adj_edge.p, A * sizeof(uint32_t)},
                              {role, g->adj_role.p, A}});
}

dbg_status dbg_graph_wait(dbg_graph *g) {
  if (!g) return DBG_EINVAL;
  DeviceScope scope(g->device);
  for (cudaStream_t cs : g->copy_streams)
    if (cs) DBG_CUDA_TRY(cudaStreamSynchronize(cs));
  return DBG_OK;
}

dbg_status dbg_graph_csr(const dbg_graph *g, uint64_t *row_ptr, uint32_t *nbr, uint32_t *edge, uint8_t *role) {
  if (!g) return DBG_EINVAL;
  const uint64_t A = 2 * g->num_edges;
  DBG_TRY(copy_plain(g->device, row_ptr, g->row_ptr.p, (g->num_nodes + 1) * sizeof(uint64_t)));
  DBG_TRY(copy_plain(g->device, nbr, g->adj_nbr.p, A * sizeof(uint32_t)));
  DBG_TRY(copy_plain(g->device, edge, g->adj_edge.p, A * sizeof(uint32_t)));
  DBG_TRY(copy_plain(g->device, role, g->adj_role.p, A));
  return DBG_OK;
}

dbg_status dbg_graph_device_view(const dbg_graph *g, dbg_graph_view *v) {
  if (!g || !v) return DBG_EINVAL;
  v->k = g->k;
  v->key_words = g->key_words;
  v->num_nodes = g->num_nodes;
  v->num_edges = g->num_edges;
  v->num_instances = g->num_instances;
  v->node_keys = g->node_keys.as<uint64_t>();
  v->edge_keys = g->edge_keys.as<uint64_t>();
  v->row_ptr = g->row_ptr.as<uint64_t>();
  v->src = g->src.as<uint32_t>();
  v->dst = g->dst.as<uint32_t>();
  v->mult = g->mult.as<uint32_t>();
  v->adj_nbr = g->adj_nbr.as<uint32_t>();
  v->adj_edge = g->adj_edge.as<uint32_t>();
  v->orient = g->orient.as<uint8_t>();
  v->adj_role = g->adj_role.as<uint8_t>();
  return DBG_OK;
}

void dbg_graph_free(dbg_graph *g) {
  if (!g) return;
  DeviceScope scope(g->device);
  for (cudaStream_t cs : g->copy_streams)
    if (cs) {  // read-backs in flight finish before the arrays go
      cudaStreamSynchronize(cs);
      cudaStreamDestroy(cs);
    }
  std::shared_ptr<BudgetShare> budget = std::move(g->budget);
  const uint64_t charged = g->charged;
  delete g;  // DevBuf destructors release in stream order
  if (budget) budget->release(charged);
}

static const char *variant_name_of(uint32_t kind, uint32_t v, uint32_t *count) {
  *count = 0;
  switch (kind) {
    case 0: return sort_variant_name_u64(false, v, count);
    case 1: return sort_variant_name_u64(true, v, count);
    case 2: return sort_variant_name_u128(false, v, count);
    case 3: return sort_variant_name_u128(true, v, count);
    case 4:
    case 5: {
      // the local sort's ranking methods (same order as local_rank_method);
      // 3-5: the same with the node records' local sort in its wide form
      static const char *const names[] = {"local match", "local atomic", "local ballot",
                                          "local match wide", "local atomic wide", "local ballot wide"};
      *count = 6;
      return v < 6 ? names[v] : nullptr;
    }
    default: return nullptr;
  }
}

uint32_t dbg_sort_variant_count(uint32_t kind) {
  uint32_t c = 0;
  variant_name_of(kind, 0, &c);
  return c;
}

const char *dbg_sort_variant_name(uint32_t kind, uint32_t variant) {
  uint32_t c = 0;
  return variant_name_of(kind, variant, &c);
}

dbg_status dbg_sort_variant_set(dbg_ctx *ctx, uint32_t kind, uint32_t variant) {
  if (!ctx || kind > 5 || variant >= dbg_sort_variant_count(kind)) {
    set_error("bad sort variant %u of kind %u", variant, kind);
    return DBG_EINVAL;
  }
  ctx->sort_variant[kind] = (int)variant;
  return DBG_OK;
}

int32_t dbg_sort_variant_get(const dbg_ctx *ctx, uint32_t kind) {
  return (ctx && kind <= 5) ? ctx->sort_variant[kind] : -1;
}

dbg_status dbg_sort_hybrid_set(dbg_ctx *ctx, int on) {
  if (!ctx) {
    set_error("null context");
    return DBG_EINVAL;
  }
  ctx->hybrid_sort = on ? 1 : 0;
  return DBG_OK;
}

dbg_status dbg_sort_count_first_set(dbg_ctx *ctx, int on) {
  if (!ctx) {
    set_error("null context");
    return DBG_EINVAL;
  }
  ctx->count_first = on ? 1 : 0;
  return DBG_OK;
}

uint64_t dbg_sort_fallbacks(const dbg_ctx *ctx) { return ctx ? ctx->local_sort_fallbacks : 0; }

uint64_t dbg_sort_count_overflows(const dbg_ctx *ctx) { return ctx ? ctx->count_overflow_tiles : 0; }

uint64_t dbg_sort_rank_fallbacks(const dbg_ctx *ctx) { return ctx ? ctx->rank_fallback_tiles : 0; }

dbg_status dbg_copy_streams_set(dbg_ctx *ctx, int n) {
  if (!ctx || n < 1 || n > kCopyStreams) {
    set_error("copy streams: null context or %d not in 1..%d", n, kCopyStreams);
    return DBG_EINVAL;
  }
  ctx->copy_streams = n;
  return DBG_OK;
}

dbg_status dbg_compact_mode_set(dbg_ctx *ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) {
    set_error("compact mode: null context or mode %d not in 0..2", mode);
    return DBG_EINVAL;
  }
  ctx->compact_mode = mode;
  return DBG_OK;
}

dbg_status dbg_node_mult_set(dbg_ctx *ctx, int on) {
  if (!ctx) {
    set_error("null context");
    return DBG_EINVAL;
  }
  ctx->node_mult = on ? 1 : 0;
  return DBG_OK;
}

dbg_status dbg_node_reads_set(dbg_ctx *ctx, int on) {
  if (!ctx) {
    set_error("null context");
    return DBG_EINVAL;
  }
  ctx->node_reads = on ? 1 : 0;
  return DBG_OK;
}

dbg_status dbg_graph_node_reads(const dbg_graph *g, uint32_t *reads) {
  if (!g) return DBG_EINVAL;
  if (!g->node_reads.p) {
    set_error("read counts were not counted for this graph (dbg_node_reads_set before dbg_build)");
    return DBG_EINVAL;
  }
  if (g->num_nodes && !reads) return DBG_EINVAL;
  return copy_plain(g->device, reads, g->node_reads.p, g->num_nodes * sizeof(uint32_t));
}

dbg_status dbg_roadmap_nodes(dbg_ctx *ctx, const dbg_graph *g, uint32_t min_reads, uint32_t *ids,
                             uint64_t *count) {
  if (!ctx || !g || !count) {
    set_error("ctx, graph or count is NULL");
    return DBG_EINVAL;
  }
  if (!g->node_reads.p) {
    set_error("read counts were not counted for this graph (dbg_node_reads_set before dbg_build)");
    return DBG_EINVAL;
  }
  DeviceScope scope(ctx->device);
  DevBuf tmp;
  uint32_t *d_ids = nullptr;
  if (ids) {
    if (is_device_ptr(ids)) {
      d_ids = ids;
    } else {
      DBG_TRY(alloc_buf(ctx, tmp, std::max<uint64_t>(1, g->num_nodes) * 4));
      d_ids = tmp.as<uint32_t>();
    }
  }
  dbg_status st = roadmap_nodes(ctx, g, min_reads, d_ids, count);
  if (st == DBG_OK && ids && d_ids != ids && *count)
    st = copy_plain(ctx->device, ids, d_ids, *count * sizeof(uint32_t));
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  return st;
}

dbg_status dbg_sort_partition_first_set(dbg_ctx *ctx, int on) {
  if (!ctx) {
    set_error("null context");
    return DBG_EINVAL;
  }
  ctx->partition_first = on ? 1 : 0;
  return DBG_OK;
}

dbg_status dbg_sort_local_rank_set(dbg_ctx *ctx, int on) {
  if (!ctx) {
    set_error("null context");
    return DBG_EINVAL;
  }
  ctx->seg_rank = on ? 1 : 0;
  return DBG_OK;
}

// cache line format: "<gpu name>|<SMs>" v0 v1 v2 v3
static std::string tune_cache_key(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string name = prop.name;
  for (char &c : name)
    if (c == ' ') c = '_';
  return name + "|" + std::to_string(prop.multiProcessorCount);
}

static bool tune_cache_load(const char *path, const std::string &key, int out[4]) {
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    char k[400];
    int v[4];
    if (std::sscanf(line, "%399s %d %d %d %d", k, &v[0], &v[1], &v[2], &v[3]) == 5 && key == k) {
      for (int i = 0; i < 4; i++) out[i] = v[i];
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

static void tune_cache_store(const char *path, const std::string &key, const int v[4]) {
  FILE *f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], v[3]);
  std::fclose(f);
}

dbg_status dbg_autotune(dbg_ctx *ctx, uint64_t n, const char *cache_path, double *ms_out) {
  if (!ctx) return DBG_EINVAL;
  DeviceScope scope(ctx->device);
  const std::string key = tune_cache_key(ctx->device);
  int cached[4];
  if (cache_path && tune_cache_load(cache_path, key, cached)) {
    bool ok = true;
    for (uint32_t kd = 0; kd < 4; kd++) ok = ok && cached[kd] >= 0 && (uint32_t)cached[kd] < dbg_sort_variant_count(kd);
    if (ok) {
      for (int kd = 0; kd < 4; kd++) ctx->sort_variant[kd] = cached[kd];
      return DBG_OK;
    }
  }
  if (n == 0) n = 1ull << 25;
  double *m = ms_out;
  constexpr int W = DBG_MAX_SORT_VARIANTS;
  for (uint32_t kd = 0; kd < 4; kd++)
    if (dbg_sort_variant_count(kd) > (uint32_t)W) {
      set_error("sort kind %u has more than %d variants", kd, W);
      return DBG_EINVAL;
    }
  dbg_status st = autotune_u64(ctx, n, m ? m : nullptr, m ? m + W : nullptr);
  if (st == DBG_OK) st = autotune_u128(ctx, n / 2, m ? m + 2 * W : nullptr, m ? m + 3 * W : nullptr);
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  if (st != DBG_OK) return st;
  if (cache_path) tune_cache_store(cache_path, key, ctx->sort_variant);
  return DBG_OK;
}

}  // extern "C"

// dbg_internal.h -- host-side state shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dbg.h"

namespace dbg {

void set_error(const char *fmt, ...);

// Stream-ordered device memory through the context's hooks.
struct Allocator {
  dbg_alloc_fn alloc = nullptr;
  dbg_free_fn free = nullptr;
  void *user = nullptr;
  cudaStream_t stream = nullptr;
  void *get(size_t bytes);
  void put(void *p, size_t bytes);
};

// One device buffer; released in stream order when it goes out of scope.
struct DevBuf {
  Allocator *al = nullptr;
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept { *this = std::move(o); }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) {
      release();
      al = o.al; p = o.p; bytes = o.bytes;
      o.p = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p && al) al->put(p, bytes);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T *as() const { return static_cast<T *>(p); }
};

enum Stage {
  ST_OFFSETS, ST_PACK, ST_EMIT, ST_SORT_EDGES, ST_RLE, ST_ENDPOINTS, ST_SORT_NODES, ST_NODE_IDS,
  ST_ADJACENCY, ST_COPIES, ST_COMPACT_LINKS, ST_COMPACT_RANK, ST_COMPACT_CYCLES, ST_COMPACT_OUTPUT,
  ST_LOCAL_SORT_EDGES, ST_LOCAL_SORT_NODES, ST_PARTITION_EDGES, ST_NODE_MULT, ST_COUNT
};
extern const char *const kStageNames[ST_COUNT];

struct ProfRecord {
  int stage;
  cudaEvent_t a, b;
  double bytes;
  uint32_t launches;
};

}  // namespace dbg

struct dbg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  dbg::Allocator al;
  uint64_t mem_budget = 0;
  uint32_t spin_limit = 1u << 22;
  // per sort kind: onesweep passes over 0: u64, 1: u64+payload, 2: u128,
  // 3: u128+payload keys; the local sort's ranking for 4: u64, 5: u128 keys
  int sort_variant[6] = {0, 0, 0, 0, 0, 0};
  int hybrid_sort = 1;                 // high digits globally + local sort of group-aligned tiles
  int count_first = 1;                 // local pass of the edge keys counts copies before sorting
  int partition_first = 1;             // first global pass of keys without payload: unordered partition
  int seg_rank = 1;                    // local passes rank within groups instead of digit passes
  int compact_mode = 0;                // 0 auto, 1 walks with 64-bit words, 2 pointer jumping only
  int copy_streams = 1;                // streams a graph's or unitigs' read-back is spread over
  int node_mult = 0;                   // dbg_build also counts every node's k-mer occurrences
  int node_reads = 0;                  // dbg_build also counts the distinct reads holding every node
  uint64_t count_overflow_tiles = 0;  // count-first tiles whose keys did not fit the hash table
  uint64_t local_sort_fallbacks = 0;   // local sorts that met a group longer than their window
  uint64_t rank_fallback_tiles = 0;    // tiles with a group too long to rank, sorted by digit passes
  int num_sms = 0;
  // persistent scratch: the look-back status words of every scan and sort
  // pass, tagged by epoch so they never need clearing between uses
  uint64_t *d_status = nullptr;
  size_t status_words = 0;
  uint32_t epoch = 1;
  uint32_t *d_err = nullptr;       // device error word
  uint32_t *d_counters = nullptr;  // small per-call counters (tile tickets, totals)
  uint32_t *h_pinned = nullptr;    // pinned host mirror for small read-backs
  cudaEvent_t ev = nullptr;
  cudaStream_t copy_stream = nullptr;  // host-to-device copies that overlap the build's stream
  // profiling
  bool prof = false;
  uint64_t launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<dbg::ProfRecord> pending;
  dbg_stage_stat stats[dbg::ST_COUNT] = {};
};

namespace dbg {
// Device bytes charged to a request server's budget.  A graph a server
// built keeps its bytes charged, through its own reference to this record,
// until dbg_graph_free, which may come after the server is gone.
struct BudgetShare {
  std::mutex mu;
  std::condition_variable cv;  // signalled whenever bytes are released
  uint64_t in_use = 0;
  void release(uint64_t bytes) {
    {
      std::lock_guard<std::mutex> lk(mu);
      in_use -= std::min(in_use, bytes);
    }
    cv.notify_all();
  }
};
}  // namespace dbg

namespace dbg {
constexpr int kCopyStreams = 8;  // most streams a result read-back is spread over
}  // namespace dbg

struct dbg_graph {
  uint32_t k = 0, key_words = 1;
  uint64_t num_nodes = 0, num_edges = 0, num_instances = 0;
  dbg::Allocator al;  // copy of the creating context's allocator
  int device = 0;
  uint32_t edge_buckets = 1, node_buckets = 1;  // key ranges used (bucket path)
  dbg::DevBuf node_keys, edge_keys, src, dst, orient, mult, row_ptr, adj_nbr, adj_edge, adj_role;
  dbg::DevBuf adj_side;    // per adjacency slot: its end's side | the far end's side << 1 (when built)
  dbg::DevBuf node_mult;   // k-mer occurrences per node, when the build counted them
  dbg::DevBuf node_reads;  // distinct reads per node, when the build counted them
  cudaStream_t copy_streams[dbg::kCopyStreams] = {};  // read-backs started by dbg_graph_*_async
  int copy_next = 0;                                   // the stream that takes the next chunk
  int n_copy = 1;                                      // streams in use (the context's setting)
  std::shared_ptr<dbg::BudgetShare> budget;  // the server budget this graph is charged to, if any
  uint64_t charged = 0;
  // device bytes of the graph's arrays
  uint64_t device_bytes() const {
    uint64_t b = 0;
    for (const dbg::DevBuf *x : {&node_keys, &edge_keys, &src, &dst, &orient, &mult, &row_ptr, &adj_nbr,
                                 &adj_edge, &adj_role, &adj_side, &node_mult, &node_reads})
      b += x->bytes;
    return b;
  }
};

struct dbg_unitigs {
  uint64_t count = 0, num_nodes = 0, total_bases = 0;
  dbg::Allocator al;
  int device = 0;
  int n_copy = 1;  // streams its read-back is spread over (the context's setting)
  dbg::DevBuf node_off, nodes, seq_off, seq, circular;
};

// The simplified graph: units (as unitigs) and the relabelled edges.
struct dbg_simple {
  dbg_unitigs units;
  uint64_t num_edges = 0, removed = 0;
  dbg::DevBuf unit_a, unit_b, side_a, side_b, edge;
};

namespace dbg {

#define DBG_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t e__ = (expr);                                                           \
    if (e__ != cudaSuccess) {                                                           \
      ::dbg::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e__), __FILE__, \
                       __LINE__);                                                       \
      return DBG_ECUDA;                                                                 \
    }                                                                                   \
  } while (0)

#define DBG_TRY(expr)                  \
  do {                                 \
    dbg_status s__ = (expr);           \
    if (s__ != DBG_OK) return s__;     \
  } while (0)

dbg_status alloc_buf(dbg_ctx *ctx, DevBuf &b, size_t bytes);
// grows the persistent look-back status array to at least `words` words
dbg_status ensure_status(dbg_ctx *ctx, size_t words);
// creates the context's copy stream on first use
dbg_status ensure_copy_stream(dbg_ctx *ctx);

// Copies of one array spread over several streams in chunks, so that the
// copy engines run side by side (one engine alone does not fill the
// host link); *next is the stream that takes the next chunk.
dbg_status copy_spread(cudaStream_t *streams, int n_streams, int *next, void *dst, const void *src, size_t bytes);

// events owned for one call, destroyed when it returns
struct EventSet {
  std::vector<cudaEvent_t> e;
  dbg_status create(size_t count) {
    e.assign(count, nullptr);
    for (cudaEvent_t &x : e)
      if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) {
        x = nullptr;
        set_error("cudaEventCreate failed");
        return DBG_ECUDA;
      }
    return DBG_OK;
  }
  ~EventSet() {
    for (cudaEvent_t x : e)
      if (x) cudaEventDestroy(x);
  }
};
// next epoch for a look-back scan; clears the status array when it wraps
dbg_status next_epoch(dbg_ctx *ctx, uint32_t *epoch);
// reads the device error word and maps it to a status (and clears it)
dbg_status check_device_error(dbg_ctx *ctx);

// Reads a few bytes of device memory through the pinned mirror (synchronizes).
dbg_status read_small(dbg_ctx *ctx, const void *d_src, size_t bytes, void *h_dst);

// Host copy of n words from device or host memory (synchronous on ctx stream).
dbg_status copy_out(dbg_ctx *ctx, void *dst, const void *src, size_t bytes);

// Brackets the kernels launched in its scope: counts them and, when the
// context profiles, records CUDA events around them.
struct Span {
  dbg_ctx *ctx;
  int stage;
  double bytes;
  uint32_t launches;
  cudaEvent_t a = nullptr;
  Span(dbg_ctx *c, int st, double algo_bytes, uint32_t n_launches = 1);
  ~Span();
};
// Launches one kernel (or a few statements) inside its own Span.
#define DBG_LAUNCH(ctx, stage, bytes, ...)        \
  do {                                            \
    ::dbg::Span dbg_span__((ctx), (stage), (bytes)); \
    __VA_ARGS__;                                  \
  } while (0)

// folds finished event pairs into the per-stage statistics (after a sync)
void prof_resolve(dbg_ctx *ctx);

// The build pipeline for one key width (k <= 31: uint64_t, else 128-bit).
struct BuildInput {
  const uint8_t *reads;       // ASCII, on the device or (h_reads) in host memory
  const uint32_t *d_lengths;  // device
  uint64_t n;
  bool h_reads;               // reads are in host memory: streamed in by chunks
  uint32_t k;
};

// Input of the bucket path (dbg_build_bucketed).
struct BucketInput {
  const char *reads;  // host or device
  bool reads_on_device;
  const uint32_t *d_lengths;
  uint64_t n;
  uint32_t k;
};
dbg_status build_bucketed_u64(dbg_ctx *ctx, const BucketInput &in, uint64_t budget, dbg_graph *g, uint32_t *eb,
                              uint32_t *nb);
dbg_status build_bucketed_u128(dbg_ctx *ctx, const BucketInput &in, uint64_t budget, dbg_graph *g, uint32_t *eb,
                               uint32_t *nb);
// Worst-case peak device bytes of one in-memory build of n reads holding
// `bases` bases and N edge instances (I reads of length exactly k).
uint64_t build_footprint(uint64_t n, uint64_t bases, uint64_t N, uint64_t I, uint32_t k, bool reads_on_host,
                         bool lengths_on_host);

dbg_status build_graph_u64(dbg_ctx *ctx, const BuildInput &in, dbg_graph *g);
// The chains of g into u: the unitigs (literal = false) or the chains of
// Section 6.1's candidate edges (literal = true).
dbg_status compact_chains(dbg_ctx *ctx, const dbg_graph *g, dbg_unitigs *u, bool literal);
// IDs of the nodes held by at least t distinct reads (device buffer of
// num_nodes entries, or NULL for the count only)
dbg_status roadmap_nodes(dbg_ctx *ctx, const dbg_graph *g, uint32_t t, uint32_t *d_ids, uint64_t *count);
dbg_status autotune_u64(dbg_ctx *ctx, uint64_t n, double *ms_keys, double *ms_pairs);
dbg_status autotune_u128(dbg_ctx *ctx, uint64_t n, double *ms_keys, double *ms_pairs);
const char *sort_variant_name_u64(bool pairs, uint32_t v, uint32_t *count);
const char *sort_variant_name_u128(bool pairs, uint32_t v, uint32_t *count);
dbg_status build_graph_u128(dbg_ctx *ctx, const BuildInput &in, dbg_graph *g);

}  // namespace dbg

// simplify.cu -- the simplified bi-directed graph (Section 6, with the
// literal compaction of Section 6.1).
//
// Section 6.1 merges the chains formed by its candidate edges, those
// "adjacent on nodes with exactly one in and out degree": here an edge whose
// two ends lie on distinct nodes that each carry exactly one edge end on
// each side (a walk enters a node by one side and leaves by the other, so a
// node's in- and out-degree are its two side degrees).  The chains come from
// the same list ranking as the unitigs with that rule (compact_chains with
// literal = true).  Only chains of at least min_nodes nodes are reported
// (the paper: three); every node of a shorter chain stays a unit of its own.
// Section 6 then relabels the remaining edges to the merged nodes: an edge
// end at a unit's first node on that node's entry side is the unit's left
// side, one at its last node on the exit side its right side, and any other
// end no longer fits the unit's label -- its edge is inconsistent and
// removed (counted).  With chains of nodes that have one edge end per side
// no such end exists; the count checks it.
//
// Layout: units as unitigs (node lists and spelled strings, ordered by
// first node ID); edges in graph edge order as (unit, side) pairs for the
// src and dst ends plus the graph edge ID.
#include <initializer_list>
#include <new>
#include <utility>

#include "k_build.cuh"

namespace dbg {
namespace {

unsigned grid_n(uint64_t n) {
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, 152ull * 64));
}

// exclusive scan of n flags into n + 1 positions; returns the total
dbg_status scan_flags_u32(dbg_ctx *ctx, const uint32_t *in, uint64_t n, uint64_t *out, uint64_t *total) {
  cudaStream_t s = ctx->stream;
  if (n == 0) {
    DBG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    *total = 0;
    return DBG_OK;
  }
  const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  DBG_TRY(ensure_status(ctx, tiles));
  uint32_t epoch;
  DBG_TRY(next_epoch(ctx, &epoch));
  DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, 2 * sizeof(uint32_t), s));
  DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 12.0 * n,
             k_scan_excl<<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, n, out, ctx->d_status, ctx->d_counters, epoch,
                                                                ctx->spin_limit, ctx->d_err, ctx->d_counters + 1));
  DBG_CUDA_TRY(cudaGetLastError());
  return read_small(ctx, out + n, sizeof(uint64_t), total);
}

// Per entry p of the chains' node list: the unit its node belongs to (by
// the unit's first node), its position and strand there.  A chain of at
// least min_nodes nodes is one unit; the nodes of a shorter one are units
// of their own, on the positive strand.  The first node of each unit also
// gets the start flag, the unit's length and its circular flag.
__global__ void k_simple_nodes(const uint64_t *__restrict__ node_off, const uint64_t *__restrict__ nodes,
                               const uint8_t *__restrict__ circular, uint64_t C, uint64_t V, uint32_t min_nodes,
                               uint32_t *__restrict__ unit_head, uint32_t *__restrict__ upos,
                               uint8_t *__restrict__ ustrand, uint32_t *__restrict__ ustart,
                               uint32_t *__restrict__ ulen, uint8_t *__restrict__ ucirc) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < V; p += (uint64_t)gridDim.x * blockDim.x) {
    // the chain holding entry p: the last c with node_off[c] <= p
    uint64_t lo = 0, hi = C;
    while (hi - lo > 1) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (node_off[mid] <= p) lo = mid; else hi = mid;
    }
    const uint64_t c = lo, c0 = node_off[c], m = node_off[c + 1] - c0;
    const uint64_t x = nodes[p];
    const uint32_t v = (uint32_t)(x >> 1);
    const bool whole = m >= min_nodes;
    const uint32_t h = whole ? (uint32_t)(nodes[c0] >> 1) : v;
    const uint32_t pos = whole ? (uint32_t)(p - c0) : 0u;
    unit_head[v] = h;
    upos[v] = pos;
    ustrand[v] = whole ? (uint8_t)(x & 1) : 0;
    if (pos == 0) {
      ustart[v] = 1;
      ulen[v] = whole ? (uint32_t)m : 1u;
      ucirc[v] = whole ? circular[c] : 0;
    }
  }
}

// Per unit (at its first node h): its offsets and flag.
__global__ void k_simple_heads(const uint32_t *__restrict__ ustart, const uint64_t *__restrict__ uidx,
                               const uint64_t *__restrict__ uoff, const uint8_t *__restrict__ ucirc, uint64_t V,
                               uint64_t U, int k, uint64_t *__restrict__ node_off, uint64_t *__restrict__ seq_off,
                               uint8_t *__restrict__ circular) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= V; v += (uint64_t)gridDim.x * blockDim.x) {
    if (v == V) {
      node_off[U] = V;
      seq_off[U] = V + U * (uint64_t)(k - 1);
      continue;
    }
    if (!ustart[v]) continue;
    const uint64_t u = uidx[v];
    node_off[u] = uoff[v];
    seq_off[u] = uoff[v] + u * (uint64_t)(k - 1);
    circular[u] = ucirc[v];
  }
}

// Per node: its entry in its unit's node list and its bases of the unit's
// string (the whole k-mer for the first node, else the last base of its
// k-mer on its strand in the unit).
template <class K>
__global__ void k_simple_write(const uint32_t *__restrict__ unit_head, const uint32_t *__restrict__ upos,
                               const uint8_t *__restrict__ ustrand, const uint64_t *__restrict__ uidx,
                               const uint64_t *__restrict__ uoff, const uint64_t *__restrict__ node_keys, uint64_t V,
                               int k, uint64_t *__restrict__ nodes_out, char *__restrict__ seq) {
  const char *acgt = "ACGT";
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t h = unit_head[v], pos = upos[v], st = ustrand[v];
    const uint64_t u = uidx[h], off = uoff[h], so = off + u * (uint64_t)(k - 1);
    nodes_out[off + pos] = (v << 1) | st;
    K km;
    if constexpr (sizeof(K) == 8) {
      km = node_keys[v];
    } else {
      km = Key128{node_keys[2 * v], node_keys[2 * v + 1]};
    }
    if (st) km = revcomp(km, k);
    if (pos == 0) {
      for (int i = 0; i < k; i++) seq[so + i] = acgt[KeyOps<K>::digit(km, 2 * (k - 1 - i), 2)];
    } else {
      seq[so + k - 1 + pos] = acgt[KeyOps<K>::low2(km)];
    }
  }
}

// side of an edge end: 0 = left, 1 = right (the src end of (u, v, o1, o2)
// is on u's right side when o1 = 0; the dst end on v's left side when o2 = 0)
__device__ __forceinline__ uint32_t end_side_of(uint8_t orient, int role) {
  return role == 0 ? ((orient >> 1) ? 0u : 1u) : ((orient & 1) ? 1u : 0u);
}

// Side degrees: deg[2v + side] = edge ends on that side of v.
__global__ void k_simple_degrees(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                                 const uint8_t *__restrict__ orient, uint64_t E, uint32_t *__restrict__ deg) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t o = orient[e];
    atomicAdd(&deg[2 * (uint64_t)src[e] + end_side_of(o, 0)], 1u);
    atomicAdd(&deg[2 * (uint64_t)dst[e] + end_side_of(o, 1)], 1u);
  }
}

// The (unit, side) of an edge end at node x on node side sd, or false when
// the end does not lie at a free end of its unit (inconsistent).
__device__ __forceinline__ bool unit_end(uint32_t x, uint32_t sd, const uint32_t *unit_head, const uint32_t *upos,
                                         const uint8_t *ustrand, const uint32_t *ulen, const uint8_t *ucirc,
                                         uint32_t *head, uint32_t *side) {
  const uint32_t h = unit_head[x], pos = upos[x], st = ustrand[x];
  if (ucirc[h]) return false;
  const uint32_t entry = st ? 1u : 0u, exit_ = st ? 0u : 1u;
  *head = h;
  if (pos == 0 && sd == entry) {
    *side = 0;
    return true;
  }
  if (pos == ulen[h] - 1 && sd == exit_) {
    *side = 1;
    return true;
  }
  return false;
}

// keep[e] = 1 for an edge that is neither inside a reported chain nor
// inconsistent; inconsistent edges are counted.
__global__ void k_simple_edge_flags(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                                    const uint8_t *__restrict__ orient, uint64_t E, const uint32_t *__restrict__ deg,
                                    const uint32_t *__restrict__ unit_head, const uint32_t *__restrict__ upos,
                                    const uint8_t *__restrict__ ustrand, const uint32_t *__restrict__ ulen,
                                    const uint8_t *__restrict__ ucirc, uint32_t *__restrict__ keep,
                                    unsigned long long *removed) {
  unsigned long long bad = 0;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t a = src[e], b = dst[e];
    const uint8_t o = orient[e];
    const bool simple_a = deg[2 * (uint64_t)a] == 1 && deg[2 * (uint64_t)a + 1] == 1;
    const bool simple_b = deg[2 * (uint64_t)b] == 1 && deg[2 * (uint64_t)b + 1] == 1;
    // a candidate edge joins two nodes of one chain; a reported chain swallows it
    if (a != b && simple_a && simple_b && ulen[unit_head[a]] > 1) {
      keep[e] = 0;
      continue;
    }
    uint32_t h, sd;
    const bool ok = unit_end(a, end_side_of(o, 0), unit_head, upos, ustrand, ulen, ucirc, &h, &sd) &&
                    unit_end(b, end_side_of(o, 1), unit_head, upos, ustrand, ulen, ucirc, &h, &sd);
    keep[e] = ok ? 1u : 0u;
    bad += ok ? 0 : 1;
  }
  bad = __reduce_add_sync(0xffffffffu, (unsigned)bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(removed, bad);
}

// The kept edges at their scanned positions, relabelled to (unit, side).
__global__ void k_simple_edge_write(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                                    const uint8_t *__restrict__ orient, uint64_t E,
                                    const uint32_t *__restrict__ keep, const uint64_t *__restrict__ pos,
                                    const uint32_t *__restrict__ unit_head, const uint32_t *__restrict__ upos,
                                    const uint8_t *__restrict__ ustrand, const uint32_t *__restrict__ ulen,
                                    const uint8_t *__restrict__ ucirc, const uint64_t *__restrict__ uidx,
                                    uint32_t *__restrict__ unit_a, uint8_t *__restrict__ side_a,
                                    uint32_t *__restrict__ unit_b, uint8_t *__restrict__ side_b,
                                    uint32_t *__restrict__ edge) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    if (!keep[e]) continue;
    const uint8_t o = orient[e];
    uint32_t ha = 0, sa = 0, hb = 0, sb = 0;
    unit_end(src[e], end_side_of(o, 0), unit_head, upos, ustrand, ulen, ucirc, &ha, &sa);
    unit_end(dst[e], end_side_of(o, 1), unit_head, upos, ustrand, ulen, ucirc, &hb, &sb);
    const uint64_t i = pos[e];
    unit_a[i] = (uint32_t)uidx[ha];
    side_a[i] = (uint8_t)sa;
    unit_b[i] = (uint32_t)uidx[hb];
    side_b[i] = (uint8_t)sb;
    edge[i] = (uint32_t)e;
  }
}

}  // namespace
}  // namespace dbg

namespace dbg {

template <class K>
static dbg_status simplify_impl(dbg_ctx *ctx, const dbg_graph *g, uint32_t min_nodes, dbg_simple *out) {
  cudaStream_t s = ctx->stream;
  const uint64_t V = g->num_nodes, E = g->num_edges, V1 = std::max<uint64_t>(1, V);
  const int k = (int)g->k;
  dbg_unitigs &un = out->units;
  un.num_nodes = V;
  // the chains of the candidate edges
  dbg_unitigs ch;
  ch.al = ctx->al;
  DBG_TRY(compact_chains(ctx, g, &ch, true));
  for (DevBuf *b : {&ch.node_off, &ch.nodes, &ch.seq_off, &ch.seq, &ch.circular}) b->al = &ch.al;
  DevBuf unit_head, upos, ustrand, ustart, ulen, ucirc, uidx, uoff;
  DBG_TRY(alloc_buf(ctx, unit_head, V1 * 4));
  DBG_TRY(alloc_buf(ctx, upos, V1 * 4));
  DBG_TRY(alloc_buf(ctx, ustrand, V1));
  DBG_TRY(alloc_buf(ctx, ustart, V1 * 4));
  DBG_TRY(alloc_buf(ctx, ulen, V1 * 4));
  DBG_TRY(alloc_buf(ctx, ucirc, V1));
  DBG_TRY(alloc_buf(ctx, uidx, (V + 1) * 8));
  DBG_TRY(alloc_buf(ctx, uoff, (V + 1) * 8));
  DBG_CUDA_TRY(cudaMemsetAsync(ustart.p, 0, V1 * 4, s));
  DBG_CUDA_TRY(cudaMemsetAsync(ulen.p, 0, V1 * 4, s));
  uint64_t U = 0, total = 0;
  if (V > 0) {
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 24.0 * V,
               k_simple_nodes<<<grid_n(V), 256, 0, s>>>(ch.node_off.as<uint64_t>(), ch.nodes.as<uint64_t>(),
                                                        ch.circular.as<uint8_t>(), ch.count, V, min_nodes,
                                                        unit_head.as<uint32_t>(), upos.as<uint32_t>(),
                                                        ustrand.as<uint8_t>(), ustart.as<uint32_t>(),
                                                        ulen.as<uint32_t>(), ucirc.as<uint8_t>()));
    DBG_CUDA_TRY(cudaGetLastError());
  }
  DBG_TRY(scan_flags_u32(ctx, ustart.as<uint32_t>(), V, uidx.as<uint64_t>(), &U));
  DBG_TRY(scan_flags_u32(ctx, ulen.as<uint32_t>(), V, uoff.as<uint64_t>(), &total));
  if (total != V) {
    set_error("units hold %llu nodes, expected %llu", (unsigned long long)total, (unsigned long long)V);
    return DBG_EINTERNAL;
  }
  un.count = U;
  un.total_bases = V + U * (uint64_t)(k - 1);
  DBG_TRY(alloc_buf(ctx, un.node_off, (U + 1) * 8));
  DBG_TRY(alloc_buf(ctx, un.seq_off, (U + 1) * 8));
  DBG_TRY(alloc_buf(ctx, un.circular, std::max<uint64_t>(1, U)));
  DBG_TRY(alloc_buf(ctx, un.nodes, V1 * 8));
  DBG_TRY(alloc_buf(ctx, un.seq, std::max<uint64_t>(1, un.total_bases)));
  DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 13.0 * V + 17.0 * U,
             k_simple_heads<<<grid_n(V + 1), 256, 0, s>>>(ustart.as<uint32_t>(), uidx.as<uint64_t>(),
                                                          uoff.as<uint64_t>(), ucirc.as<uint8_t>(), V, U, k,
                                                          un.node_off.as<uint64_t>(), un.seq_off.as<uint64_t>(),
                                                          un.circular.as<uint8_t>()));
  if (V > 0)
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, (double)V * (4 + 4 + 1 + 16 + 8 * g->key_words + 8 + 1) + (double)U * k,
               k_simple_write<K><<<grid_n(V), 256, 0, s>>>(unit_head.as<uint32_t>(), upos.as<uint32_t>(),
                                                           ustrand.as<uint8_t>(), uidx.as<uint64_t>(),
                                                           uoff.as<uint64_t>(), g->node_keys.as<uint64_t>(), V, k,
                                                           un.nodes.as<uint64_t>(), un.seq.as<char>()));
  DBG_CUDA_TRY(cudaGetLastError());
  // the edges: inside reported chains dropped, inconsistent ones counted,
  // the rest relabelled in edge order
  const uint64_t E1 = std::max<uint64_t>(1, E);
  DevBuf deg, keep, pos, removed;
  DBG_TRY(alloc_buf(ctx, deg, 2 * V1 * 4));
  DBG_TRY(alloc_buf(ctx, keep, E1 * 4));
  DBG_TRY(alloc_buf(ctx, pos, (E + 1) * 8));
  DBG_TRY(alloc_buf(ctx, removed, 8));
  DBG_CUDA_TRY(cudaMemsetAsync(deg.p, 0, 2 * V1 * 4, s));
  DBG_CUDA_TRY(cudaMemsetAsync(removed.p, 0, 8, s));
  uint64_t M = 0;
  if (E > 0) {
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 9.0 * E,
               k_simple_degrees<<<grid_n(E), 256, 0, s>>>(g->src.as<uint32_t>(), g->dst.as<uint32_t>(),
                                                          g->orient.as<uint8_t>(), E, deg.as<uint32_t>()));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 13.0 * E + 40.0 * E,
               k_simple_edge_flags<<<grid_n(E), 256, 0, s>>>(
                   g->src.as<uint32_t>(), g->dst.as<uint32_t>(), g->orient.as<uint8_t>(), E, deg.as<uint32_t>(),
                   unit_head.as<uint32_t>(), upos.as<uint32_t>(), ustrand.as<uint8_t>(), ulen.as<uint32_t>(),
                   ucirc.as<uint8_t>(), keep.as<uint32_t>(), removed.as<unsigned long long>()));
    DBG_CUDA_TRY(cudaGetLastError());
  }
  DBG_TRY(scan_flags_u32(ctx, keep.as<uint32_t>(), E, pos.as<uint64_t>(), &M));
  DBG_TRY(read_small(ctx, removed.p, 8, &out->removed));
  out->num_edges = M;
  const uint64_t M1 = std::max<uint64_t>(1, M);
  DBG_TRY(alloc_buf(ctx, out->unit_a, M1 * 4));
  DBG_TRY(alloc_buf(ctx, out->unit_b, M1 * 4));
  DBG_TRY(alloc_buf(ctx, out->side_a, M1));
  DBG_TRY(alloc_buf(ctx, out->side_b, M1));
  DBG_TRY(alloc_buf(ctx, out->edge, M1 * 4));
  if (M > 0)
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 13.0 * E + 60.0 * M,
               k_simple_edge_write<<<grid_n(E), 256, 0, s>>>(
                   g->src.as<uint32_t>(), g->dst.as<uint32_t>(), g->orient.as<uint8_t>(), E, keep.as<uint32_t>(),
                   pos.as<uint64_t>(), unit_head.as<uint32_t>(), upos.as<uint32_t>(), ustrand.as<uint8_t>(),
                   ulen.as<uint32_t>(), ucirc.as<uint8_t>(), uidx.as<uint64_t>(), out->unit_a.as<uint32_t>(),
                   out->side_a.as<uint8_t>(), out->unit_b.as<uint32_t>(), out->side_b.as<uint8_t>(),
                   out->edge.as<uint32_t>()));
  DBG_CUDA_TRY(cudaGetLastError());
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(ctx);
}

}  // namespace dbg

using namespace dbg;

namespace {
// copies of the simple graph's arrays into caller buffers (host or device)
dbg_status copy_items(int device, std::initializer_list<std::pair<void *, std::pair<const void *, size_t>>> items) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  dbg_status st = DBG_OK;
  for (const auto &it : items) {
    if (!it.first || !it.second.second) continue;
    const cudaError_t e = cudaMemcpy(it.first, it.second.first, it.second.second, cudaMemcpyDefault);
    if (e != cudaSuccess) {
      set_error("cudaMemcpy failed: %s", cudaGetErrorString(e));
      st = DBG_ECUDA;
      break;
    }
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return st;
}
}  // namespace

extern "C" {

dbg_status dbg_simplify(dbg_ctx *ctx, const dbg_graph *g, uint32_t min_nodes, dbg_simple **out) {
  if (!out) return DBG_EINVAL;
  *out = nullptr;
  if (!ctx || !g) {
    set_error("ctx or graph is NULL");
    return DBG_EINVAL;
  }
  if (g->num_nodes >= 0x7fffffffull) {
    set_error("simplification handles fewer than 2^31 nodes");
    return DBG_EOVERFLOW;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  dbg_simple *sg = new (std::nothrow) dbg_simple();
  if (!sg) return DBG_ENOMEM;
  sg->units.al = ctx->al;
  sg->units.device = ctx->device;
  dbg_status st = g->key_words == 1 ? simplify_impl<uint64_t>(ctx, g, min_nodes, sg)
                                    : simplify_impl<Key128>(ctx, g, min_nodes, sg);
  for (DevBuf *b : {&sg->units.node_off, &sg->units.nodes, &sg->units.seq_off, &sg->units.seq,
                    &sg->units.circular, &sg->unit_a, &sg->unit_b, &sg->side_a, &sg->side_b, &sg->edge})
    b->al = &sg->units.al;
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  if (st != DBG_OK) {
    cudaGetLastError();
    cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream);
    delete sg;
  } else {
    *out = sg;
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return st;
}

uint64_t dbg_simple_num_units(const dbg_simple *s) { return s ? s->units.count : 0; }
uint64_t dbg_simple_num_edges(const dbg_simple *s) { return s ? s->num_edges : 0; }
uint64_t dbg_simple_removed_edges(const dbg_simple *s) { return s ? s->removed : 0; }
uint64_t dbg_simple_total_bases(const dbg_simple *s) { return s ? s->units.total_bases : 0; }

dbg_status dbg_simple_units(const dbg_simple *s, uint64_t *node_off, uint64_t *nodes, uint64_t *seq_off, char *seq,
                            uint8_t *circular) {
  if (!s) return DBG_EINVAL;
  return dbg_unitigs_get(&s->units, node_off, nodes, seq_off, seq, circular);
}

dbg_status dbg_simple_edges(const dbg_simple *s, uint32_t *unit_a, uint8_t *side_a, uint32_t *unit_b, uint8_t *side_b,
                            uint32_t *edge) {
  if (!s) return DBG_EINVAL;
  const size_t M = s->num_edges;
  return copy_items(s->units.device, {{unit_a, {s->unit_a.p, M * 4}},
                                      {side_a, {s->side_a.p, M}},
                                      {unit_b, {s->unit_b.p, M * 4}},
                                      {side_b, {s->side_b.p, M}},
                                      {edge, {s->edge.p, M * 4}}});
}

void dbg_simple_free(dbg_simple *s) {
  if (!s) return;
  int prev = -1, dev = s->units.device;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  delete s;
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

}  // extern "C"

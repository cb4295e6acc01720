// compact.cu -- bi-directed chain compaction (Section 6) as list ranking on
// the GPU.
//
// ListRankingTransform: node v becomes two strand-nodes, x = 2v (v read on
// its positive strand: entered by the left side, left by the right side) and
// x = 2v + 1 (read as reverse complement: entered right, left left).  A
// mergeable edge -- ends on two distinct nodes, each end alone on its side --
// gives the arc v^a -> w^b and its mirror w^(1-b) -> v^(1-a), so every
// strand-node has at most one successor and one predecessor, and each
// unitig appears as two mirrored lists (Lemma 1: bi-directed walks are
// preserved).  Wyllie pointer jumping ranks every strand-node in its list;
// strand-nodes that never reach a list head lie on cycles, which are broken
// at their smallest strand-node (Section 6.2: "identify the cycles on the
// fly and break them").  Of each mirrored pair the copy with the smaller
// spelled string is kept (Section 6.1: canonicalize and remove duplicates).
#include <algorithm>
#include <cstring>

#include "k_build.cuh"

namespace dbg {

constexpr uint32_t NONE32 = 0xffffffffu;

template <class K>
__device__ __forceinline__ K load_node_key(const uint64_t *keys, uint64_t v);
template <>
__device__ __forceinline__ uint64_t load_node_key<uint64_t>(const uint64_t *keys, uint64_t v) {
  return keys[v];
}
template <>
__device__ __forceinline__ Key128 load_node_key<Key128>(const uint64_t *keys, uint64_t v) {
  return Key128{keys[2 * v], keys[2 * v + 1]};
}

// side of an edge end: 0 = left, 1 = right
__device__ __forceinline__ uint32_t end_side(uint8_t orient, uint32_t role) {
  const uint32_t o1 = orient >> 1, o2 = orient & 1u;
  return role == 0 ? (o1 ? 0u : 1u) : (o2 ? 1u : 0u);
}

// Per node: the single edge on each side, or NONE when the side has 0 or
// >= 2 edge ends.  link[2v + side].
__global__ void k_side_links(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ adj_edge,
                             const uint8_t *__restrict__ adj_role, const uint8_t *__restrict__ orient,
                             uint64_t V, uint32_t *__restrict__ link) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t cnt[2] = {0, 0}, e_at[2] = {NONE32, NONE32};
    for (uint64_t p = row_ptr[v]; p < row_ptr[v + 1]; p++) {
      const uint32_t e = adj_edge[p];
      const uint32_t sd = end_side(orient[e], adj_role[p]);
      cnt[sd]++;
      e_at[sd] = e;
    }
    link[2 * v] = cnt[0] == 1 ? e_at[0] : NONE32;
    link[2 * v + 1] = cnt[1] == 1 ? e_at[1] : NONE32;
  }
}

// succ of strand-node x = 2v + s: leave v by its right side (s = 0) or left
// side (s = 1); the far end w must have that edge alone on its side.
__global__ void k_successors(const uint32_t *__restrict__ link, const uint32_t *__restrict__ src,
                             const uint32_t *__restrict__ dst, const uint8_t *__restrict__ orient, uint64_t V,
                             uint32_t *__restrict__ succ, uint32_t *__restrict__ pred) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < 2 * V; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = x >> 1;
    const uint32_t s = (uint32_t)(x & 1);
    const uint32_t leave_side = s ? 0u : 1u;
    const uint32_t e = link[2 * v + leave_side];
    uint32_t out = NONE32;
    if (e != NONE32) {
      const uint32_t a = src[e], b = dst[e];
      if (a != b) {
        const uint32_t w = a == v ? b : a;
        const uint32_t wrole = a == v ? 1u : 0u;
        const uint32_t wside = end_side(orient[e], wrole);
        if (link[2 * (uint64_t)w + wside] == e) out = 2 * w + (wside == 0 ? 0u : 1u);
      }
    }
    succ[x] = out;
    if (out != NONE32) pred[out] = (uint32_t)x;
  }
}

// pointer-jumping state: P = current ancestor (itself for a list head),
// D = distance to it
__global__ void k_rank_init(const uint32_t *__restrict__ pred, uint64_t n, uint32_t *__restrict__ P,
                            uint32_t *__restrict__ D) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = pred[x];
    P[x] = p == NONE32 ? (uint32_t)x : p;
    D[x] = p == NONE32 ? 0u : 1u;
  }
}

// A list head points to itself at distance 0.  A strand-node on a cycle
// can also come to point to itself (when the cycle length divides 2^r), but
// always at a distance > 0, so (P == x, D == 0) identifies heads.
__device__ __forceinline__ bool is_root(const uint32_t *P, const uint32_t *D, uint32_t x) {
  return P[x] == x && D[x] == 0;
}

// One Wyllie round over all strand-nodes (or only those flagged in `only`).
// Counts the strand-nodes whose ancestor is not yet a list head.  Distances
// saturate, so on a cycle they never wrap back to 0.
__global__ void k_rank_jump(const uint32_t *__restrict__ Pin, const uint32_t *__restrict__ Din, uint64_t n,
                            uint32_t *__restrict__ Pout, uint32_t *__restrict__ Dout,
                            const uint8_t *__restrict__ only, uint32_t *unfinished) {
  uint32_t local = 0;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = Pin[x];
    uint32_t d = Din[x];
    uint32_t np = p;
    if (!(p == (uint32_t)x && d == 0) && (!only || only[x]) && !is_root(Pin, Din, p)) {
      d = (uint32_t)min((uint64_t)d + Din[p], (uint64_t)0x7fffffffu);
      np = Pin[p];
      local++;
    }
    Pout[x] = np;
    Dout[x] = d;
  }
  local = __reduce_add_sync(0xffffffffu, local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(unfinished, local);
}

// Strand-nodes whose ancestor is not a list head after convergence lie on
// cycles.  Marks them and seeds the min-label propagation.
__global__ void k_cycle_mark(const uint32_t *__restrict__ P, const uint32_t *__restrict__ D, uint64_t n,
                             uint8_t *__restrict__ on_cycle, uint32_t *__restrict__ label, uint32_t *count) {
  uint32_t local = 0;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    const bool c = !is_root(P, D, P[x]);
    on_cycle[x] = c;
    label[x] = (uint32_t)x;
    local += c;
  }
  local = __reduce_add_sync(0xffffffffu, local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

// One round of min-label propagation around cycles: M = min over 2^r preds.
__global__ void k_cycle_min(const uint32_t *__restrict__ Qin, const uint32_t *__restrict__ Min, uint64_t n,
                            const uint8_t *__restrict__ on_cycle, uint32_t *__restrict__ Qout,
                            uint32_t *__restrict__ Mout) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t q = Qin[x], m = Min[x];
    if (on_cycle[x]) {
      m = min(m, Min[q]);
      q = Qin[q];
    }
    Qout[x] = q;
    Mout[x] = m;
  }
}

// A cycle whose smallest strand-node is 2v (positive strand) is the copy
// kept; it is opened at that strand-node.  cyc: 0 path, 1 kept cycle, 2
// mirror of a kept cycle.
__global__ void k_cycle_break(const uint32_t *__restrict__ pred, const uint32_t *__restrict__ M,
                              const uint8_t *__restrict__ on_cycle, uint64_t n, uint8_t *__restrict__ cyc,
                              uint32_t *__restrict__ P, uint32_t *__restrict__ D) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    if (!on_cycle[x]) {
      cyc[x] = 0;
      continue;
    }
    const uint32_t m = M[x];
    cyc[x] = (m & 1u) ? 2 : 1;
    if (m == (uint32_t)x) {
      P[x] = (uint32_t)x;
      D[x] = 0;
    } else {
      P[x] = pred[x];
      D[x] = 1;
    }
  }
}

// Per node: the strand kept (canonical copy), its unitig's first node and
// its rank there.
template <class K>
__global__ void k_select(const uint32_t *__restrict__ P, const uint32_t *__restrict__ D,
                         const uint8_t *__restrict__ cyc, const uint64_t *__restrict__ node_keys, uint64_t V,
                         int k, uint8_t *__restrict__ strand, uint32_t *__restrict__ head,
                         uint32_t *__restrict__ rank, uint32_t *__restrict__ is_head) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x0 = 2 * v, x1 = 2 * v + 1;
    uint32_t s;
    if (cyc[x0] || cyc[x1]) {
      s = cyc[x0] == 1 ? 0u : 1u;
    } else {
      const uint32_t h0 = P[x0], h1 = P[x1];
      K a = load_node_key<K>(node_keys, h0 >> 1), b = load_node_key<K>(node_keys, h1 >> 1);
      if (h0 & 1u) a = revcomp(a, k);
      if (h1 & 1u) b = revcomp(b, k);
      s = KeyOps<K>::less(a, b) ? 0u : 1u;
    }
    const uint64_t x = 2 * v + s;
    const uint32_t h = P[x] >> 1;
    strand[v] = (uint8_t)s;
    head[v] = h;
    rank[v] = D[x];
    is_head[v] = h == (uint32_t)v ? 1u : 0u;
  }
}

// Exclusive scan of u32 values with decoupled look-back; out is 64-bit.
// The last tile writes out[n] = total and *total.
__global__ __launch_bounds__(SCAN_BLOCK) void k_scan_excl(const uint32_t *__restrict__ in, uint64_t n,
                                                          uint64_t *__restrict__ out, uint64_t *status,
                                                          uint32_t *ticket, uint32_t epoch, uint32_t spin_limit,
                                                          uint32_t *err, uint32_t *total) {
  constexpr int WARPS = SCAN_BLOCK / 32;
  __shared__ uint32_t s_w[WARPS * SCAN_ITEMS + 1];
  __shared__ uint32_t s_tile, s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  // blocked per thread: thread t owns [base + t*ITEMS, +ITEMS)
  const uint64_t base = (uint64_t)tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    v[i] = base + i < n ? in[base + i] : 0u;
    sum += v[i];
  }
  const uint32_t incl = warp_incl_scan(sum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint32_t wadd = 0, tile_total = 0;
  for (int w = 0; w < WARPS; w++) {
    if (w < warp) wadd += s_w[w];
    tile_total += s_w[w];
  }
  const uint32_t excl_tile = tile_prefix(status, tile, tile_total, epoch, spin_limit, err, &s_excl);
  uint64_t run = (uint64_t)excl_tile + wadd + incl - sum;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if ((uint64_t)(tile + 1) * SCAN_TILE >= n && threadIdx.x == 0) {
    out[n] = (uint64_t)excl_tile + tile_total;
    *total = excl_tile + tile_total;
  }
}

__global__ void k_unitig_len(const uint32_t *__restrict__ head, const uint64_t *__restrict__ uidx, uint64_t V,
                             uint64_t U, uint32_t *__restrict__ len, uint8_t *__restrict__ circ,
                             const uint8_t *__restrict__ cyc, const uint8_t *__restrict__ strand, uint32_t *err) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t u = uidx[head[v]];
    if (u >= U) {
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    atomicAdd(len + u, 1u);
    if (head[v] == (uint32_t)v) circ[u] = cyc[2 * v + strand[v]] == 1 ? 1 : 0;
  }
}

template <class K>
__global__ void k_unitig_write(const uint32_t *__restrict__ head, const uint32_t *__restrict__ rank,
                               const uint8_t *__restrict__ strand, const uint64_t *__restrict__ uidx,
                               const uint64_t *__restrict__ node_off, const uint64_t *__restrict__ node_keys,
                               uint64_t V, int k, uint64_t *__restrict__ nodes_out, char *__restrict__ seq,
                               uint32_t *err) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t u = uidx[head[v]];
    const uint64_t r = rank[v];
    const uint32_t s = strand[v];
    if (node_off[u] + r >= node_off[u + 1]) {  // ranks must fit their unitig
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    nodes_out[node_off[u] + r] = (v << 1) | s;
    K km = load_node_key<K>(node_keys, v);
    if (s) km = revcomp(km, k);
    const uint64_t so = node_off[u] + u * (uint64_t)(k - 1);
    const char *acgt = "ACGT";
    if (r == 0) {
      for (int i = 0; i < k; i++)
        seq[so + i] = acgt[KeyOps<K>::digit(km, 2 * (k - 1 - i), 2)];
    } else {
      seq[so + k - 1 + r] = acgt[KeyOps<K>::low2(km)];
    }
  }
}

__global__ void k_seq_off(const uint64_t *__restrict__ node_off, uint64_t U, int k, uint64_t *__restrict__ seq_off) {
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= U; u += (uint64_t)gridDim.x * blockDim.x)
    seq_off[u] = node_off[u] + u * (uint64_t)(k - 1);
}

static unsigned grid_of(uint64_t n) {
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, 152ull * 64));
}

static dbg_status scan_excl(dbg_ctx *ctx, const uint32_t *in, uint64_t n, uint64_t *out, uint32_t *total) {
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
  return read_small(ctx, ctx->d_counters + 1, sizeof(uint32_t), total);
}

// Runs pointer jumping until every strand-node that can reach a list head
// has done so.  P/D hold the result on return (buffers may be swapped).
static dbg_status rank_lists(dbg_ctx *ctx, uint32_t **P, uint32_t **D, uint32_t **P2, uint32_t **D2, uint64_t n,
                             const uint8_t *only, int *rounds) {
  cudaStream_t s = ctx->stream;
  uint32_t prev = 0xffffffffu;
  for (int r = 0; r < 64; r++) {
    DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 3, 0, sizeof(uint32_t), s));
    DBG_LAUNCH(ctx, ST_COMPACT_RANK, 24.0 * n,
               k_rank_jump<<<grid_of(n), 256, 0, s>>>(*P, *D, n, *P2, *D2, only, ctx->d_counters + 3));
    DBG_CUDA_TRY(cudaGetLastError());
    std::swap(*P, *P2);
    std::swap(*D, *D2);
    uint32_t unfinished;
    DBG_TRY(read_small(ctx, ctx->d_counters + 3, sizeof(uint32_t), &unfinished));
    ++*rounds;
    // no progress in a round: what is left lies on cycles (a list has a
    // strand-node at every distance up to its length, so a longer list
    // would still have shrunk the count)
    if (unfinished == 0 || unfinished == prev) return DBG_OK;
    prev = unfinished;
  }
  set_error("list ranking did not converge");
  return DBG_ETIMEOUT;
}

template <class K>
static dbg_status compact_impl(dbg_ctx *ctx, const dbg_graph *g, dbg_unitigs *u) {
  cudaStream_t s = ctx->stream;
  const uint64_t V = g->num_nodes, n = 2 * V, E2 = 2 * g->num_edges;
  const int k = (int)g->k;
  u->num_nodes = V;
  DevBuf link, succ, pred, P, D, P2, D2, oncyc, cyc, label, strand, head, rank, is_head, uidx, len;
  const uint64_t V1 = std::max<uint64_t>(1, V), n1 = std::max<uint64_t>(1, n);
  DBG_TRY(alloc_buf(ctx, link, n1 * 4));
  DBG_TRY(alloc_buf(ctx, succ, n1 * 4));
  DBG_TRY(alloc_buf(ctx, pred, n1 * 4));
  DBG_TRY(alloc_buf(ctx, P, n1 * 4));
  DBG_TRY(alloc_buf(ctx, D, n1 * 4));
  DBG_TRY(alloc_buf(ctx, P2, n1 * 4));
  DBG_TRY(alloc_buf(ctx, D2, n1 * 4));
  DBG_TRY(alloc_buf(ctx, oncyc, n1));
  DBG_TRY(alloc_buf(ctx, cyc, n1));
  uint64_t U = 0;
  if (V > 0) {
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, (double)V * 8 + 4.0 * E2 * 5 + 8.0 * V,
               k_side_links<<<grid_of(V), 256, 0, s>>>(g->row_ptr.as<uint64_t>(), g->adj_edge.as<uint32_t>(),
                                            g->adj_role.as<uint8_t>(), g->orient.as<uint8_t>(), V,
                                            link.as<uint32_t>()));
    DBG_CUDA_TRY(cudaMemsetAsync(pred.p, 0xff, n * 4, s));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 8.0 * n + 2.0 * n * (4 + 4 + 1 + 4) + 8.0 * n,
               k_successors<<<grid_of(n), 256, 0, s>>>(link.as<uint32_t>(), g->src.as<uint32_t>(), g->dst.as<uint32_t>(),
                                            g->orient.as<uint8_t>(), V, succ.as<uint32_t>(), pred.as<uint32_t>()));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 12.0 * n,
               k_rank_init<<<grid_of(n), 256, 0, s>>>(pred.as<uint32_t>(), n, P.as<uint32_t>(), D.as<uint32_t>()));
    DBG_CUDA_TRY(cudaGetLastError());
    uint32_t *p = P.as<uint32_t>(), *d = D.as<uint32_t>(), *p2 = P2.as<uint32_t>(), *d2 = D2.as<uint32_t>();
    int rounds = 0;
    DBG_TRY(rank_lists(ctx, &p, &d, &p2, &d2, n, nullptr, &rounds));
    // cycles
    DBG_TRY(alloc_buf(ctx, label, n1 * 4));
    DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 4, 0, sizeof(uint32_t), s));
    DBG_LAUNCH(ctx, ST_COMPACT_CYCLES, 13.0 * n,
               k_cycle_mark<<<grid_of(n), 256, 0, s>>>(p, d, n, oncyc.as<uint8_t>(), label.as<uint32_t>(), ctx->d_counters + 4));
    uint32_t ncyc;
    DBG_TRY(read_small(ctx, ctx->d_counters + 4, sizeof(uint32_t), &ncyc));
    if (ncyc > 0) {
      // min label over each cycle: ceil(log2(ncyc)) + 1 doubling rounds
      uint32_t *q = p2, *m = label.as<uint32_t>(), *q2 = d2;
      DevBuf m2buf;
      DBG_TRY(alloc_buf(ctx, m2buf, n1 * 4));
      uint32_t *m2 = m2buf.as<uint32_t>();
      DBG_CUDA_TRY(cudaMemcpyAsync(q, pred.p, n * 4, cudaMemcpyDeviceToDevice, s));
      int R = 1;
      while ((1ull << (R - 1)) < ncyc) R++;
      for (int r = 0; r < R; r++) {
        DBG_LAUNCH(ctx, ST_COMPACT_CYCLES, 25.0 * n,
                   k_cycle_min<<<grid_of(n), 256, 0, s>>>(q, m, n, oncyc.as<uint8_t>(), q2, m2));
        std::swap(q, q2);
        std::swap(m, m2);
      }
      DBG_LAUNCH(ctx, ST_COMPACT_CYCLES, 18.0 * n,
                 k_cycle_break<<<grid_of(n), 256, 0, s>>>(pred.as<uint32_t>(), m, oncyc.as<uint8_t>(), n, cyc.as<uint8_t>(), p,
                                               d));
      DBG_CUDA_TRY(cudaGetLastError());
      // rank the opened cycles (the other strand-nodes are already final)
      DBG_TRY(rank_lists(ctx, &p, &d, &p2, &d2, n, oncyc.as<uint8_t>(), &rounds));
    } else {
      DBG_CUDA_TRY(cudaMemsetAsync(cyc.p, 0, n, s));
    }
    label.release();
    DBG_TRY(alloc_buf(ctx, strand, V1));
    DBG_TRY(alloc_buf(ctx, head, V1 * 4));
    DBG_TRY(alloc_buf(ctx, rank, V1 * 4));
    DBG_TRY(alloc_buf(ctx, is_head, V1 * 4));
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 16.0 * n + 13.0 * V,
               k_select<K><<<grid_of(V), 256, 0, s>>>(p, d, cyc.as<uint8_t>(), g->node_keys.as<uint64_t>(), V, k,
                                           strand.as<uint8_t>(), head.as<uint32_t>(), rank.as<uint32_t>(),
                                           is_head.as<uint32_t>()));
    DBG_CUDA_TRY(cudaGetLastError());
    DBG_TRY(alloc_buf(ctx, uidx, (V + 1) * 8));
    uint32_t U32;
    DBG_TRY(scan_excl(ctx, is_head.as<uint32_t>(), V, uidx.as<uint64_t>(), &U32));
    U = U32;
  }
  u->count = U;
  const uint64_t U1 = std::max<uint64_t>(1, U);
  DBG_TRY(alloc_buf(ctx, u->node_off, (U + 1) * 8));
  DBG_TRY(alloc_buf(ctx, u->seq_off, (U + 1) * 8));
  DBG_TRY(alloc_buf(ctx, u->circular, U1));
  DBG_TRY(alloc_buf(ctx, u->nodes, V1 * 8));
  u->total_bases = V + U * (uint64_t)(k - 1);
  DBG_TRY(alloc_buf(ctx, u->seq, std::max<uint64_t>(1, u->total_bases)));
  if (V > 0) {
    DBG_TRY(alloc_buf(ctx, len, U1 * 4));
    DBG_CUDA_TRY(cudaMemsetAsync(len.p, 0, U1 * 4, s));
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 13.0 * V,
               k_unitig_len<<<grid_of(V), 256, 0, s>>>(head.as<uint32_t>(), uidx.as<uint64_t>(), V, U, len.as<uint32_t>(),
                                            u->circular.as<uint8_t>(), cyc.as<uint8_t>(), strand.as<uint8_t>(),
                                            ctx->d_err));
    uint32_t tot;
    DBG_TRY(scan_excl(ctx, len.as<uint32_t>(), U, u->node_off.as<uint64_t>(), &tot));
    if (tot != V) {
      set_error("unitigs hold %u nodes, expected %llu", tot, (unsigned long long)V);
      return DBG_ECUDA;
    }
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 16.0 * U,
               k_seq_off<<<grid_of(U + 1), 256, 0, s>>>(u->node_off.as<uint64_t>(), U, k, u->seq_off.as<uint64_t>()));
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, (double)V * (4 + 4 + 1 + 8 + 8 + 8 * g->key_words + 8 + 1) + (double)U * k,
               k_unitig_write<K><<<grid_of(V), 256, 0, s>>>(head.as<uint32_t>(), rank.as<uint32_t>(), strand.as<uint8_t>(),
                                                 uidx.as<uint64_t>(), u->node_off.as<uint64_t>(),
                                                 g->node_keys.as<uint64_t>(), V, k, u->nodes.as<uint64_t>(),
                                                 u->seq.as<char>(), ctx->d_err));
    DBG_CUDA_TRY(cudaGetLastError());
  } else {
    DBG_CUDA_TRY(cudaMemsetAsync(u->node_off.p, 0, 8, s));
    DBG_CUDA_TRY(cudaMemsetAsync(u->seq_off.p, 0, 8, s));
  }
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(ctx);
}

}  // namespace dbg

using namespace dbg;

extern "C" {

dbg_status dbg_compact(dbg_ctx *ctx, const dbg_graph *g, dbg_unitigs **out) {
  if (!out) return DBG_EINVAL;
  *out = nullptr;
  if (!ctx || !g) {
    set_error("ctx or graph is NULL");
    return DBG_EINVAL;
  }
  if (g->num_nodes >= 0x7fffffffull) {
    set_error("compaction handles fewer than 2^31 nodes");
    return DBG_EOVERFLOW;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  dbg_unitigs *u = new (std::nothrow) dbg_unitigs();
  if (!u) return DBG_ENOMEM;
  u->al = ctx->al;
  u->device = ctx->device;
  dbg_status st = g->key_words == 1 ? compact_impl<uint64_t>(ctx, g, u) : compact_impl<Key128>(ctx, g, u);
  for (DevBuf *b : {&u->node_off, &u->nodes, &u->seq_off, &u->seq, &u->circular}) b->al = &u->al;
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  if (st != DBG_OK) {
    cudaGetLastError();
    cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), ctx->stream);
    delete u;
  } else {
    *out = u;
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  return st;
}

uint64_t dbg_unitigs_count(const dbg_unitigs *u) { return u ? u->count : 0; }
uint64_t dbg_unitigs_total_bases(const dbg_unitigs *u) { return u ? u->total_bases : 0; }

dbg_status dbg_unitigs_get(const dbg_unitigs *u, uint64_t *node_off, uint64_t *nodes, uint64_t *seq_off, char *seq,
                           uint8_t *circular) {
  if (!u) return DBG_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != u->device) cudaSetDevice(u->device);
  struct Item { void *dst; const void *src; size_t bytes; } items[] = {
      {node_off, u->node_off.p, (u->count + 1) * 8}, {nodes, u->nodes.p, u->num_nodes * 8},
      {seq_off, u->seq_off.p, (u->count + 1) * 8},   {seq, u->seq.p, u->total_bases},
      {circular, u->circular.p, u->count}};
  dbg_status st = DBG_OK;
  for (auto &it : items) {
    if (!it.dst || !it.bytes) continue;
    cudaError_t e = cudaMemcpy(it.dst, it.src, it.bytes, cudaMemcpyDefault);
    if (e != cudaSuccess) {
      set_error("cudaMemcpy failed: %s", cudaGetErrorString(e));
      st = DBG_ECUDA;
      break;
    }
  }
  if (prev >= 0 && prev != u->device) cudaSetDevice(prev);
  return st;
}

void dbg_unitigs_free(dbg_unitigs *u) {
  if (!u) return;
  int prev = -1, dev = u->device;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  delete u;
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
}

}  // extern "C"

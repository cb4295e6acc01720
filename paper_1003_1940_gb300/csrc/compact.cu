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
#include <vector>
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

// Per node and side: the edge end alone on that side, if exactly one is
// (with `literal`, only at nodes whose two sides each carry one end).
// link_node[2v + side] = (w << 1) | side_at_w of the edge's other end, and
// link_edge[2v + side] = the edge | (entry base << 32), the edge being NONE
// when the side has 0 or >= 2 ends.  The entry base is the last base of v's
// k-mer read as a walk that enters v by that side reads it (forward when
// entering by the left side, reversed by the right), i.e. the base a walk
// appends on arriving at v that way.  The neighbour comes from the
// adjacency row, so only orient is gathered.
template <class K>
__global__ void k_side_links(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ adj_nbr,
                             const uint32_t *__restrict__ adj_edge, const uint8_t *__restrict__ adj_role,
                             const uint8_t *__restrict__ orient, const uint64_t *__restrict__ node_keys, uint64_t V,
                             int k, bool literal, uint32_t *__restrict__ link_node,
                             uint64_t *__restrict__ link_edge) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t cnt[2] = {0, 0}, e_at[2] = {NONE32, NONE32}, far[2] = {NONE32, NONE32};
    const uint64_t p0 = row_ptr[v], p1 = row_ptr[v + 1];
    for (uint64_t p = p0; p < p1; p++) {
      const uint32_t e = adj_edge[p], role = adj_role[p];
      const uint8_t o = orient[e];
      const uint32_t sd = end_side(o, role);
      cnt[sd]++;
      e_at[sd] = e;
      far[sd] = (adj_nbr[p] << 1) | end_side(o, 1u - role);
    }
    const K kv = load_node_key<K>(node_keys, v);
    const uint64_t entry[2] = {KeyOps<K>::low2(kv), 3u - KeyOps<K>::digit(kv, 2 * (k - 1), 2)};
    // the literal rule (Section 6.1) links only nodes with one end per side
    const bool ok = !literal || (cnt[0] == 1 && cnt[1] == 1);
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const bool one = ok && cnt[sd] == 1;
      link_node[2 * v + sd] = one ? far[sd] : NONE32;
      link_edge[2 * v + sd] = (entry[sd] << 32) | (one ? e_at[sd] : NONE32);
    }
  }
}

// A meeting walk's word per strand-node: its successor (or "tail") and its
// entry base -- the base a walk appends on arriving at it, the last base of
// its k-mer on its strand -- or a mark (the head of the walker that took
// the node on the other strand).  32-bit words for up to 2^29 - 1
// strand-nodes (successor in bits 0-28, all ones for a tail; base in bits
// 29-30; mark in bit 31), 64-bit words above (successor in the low word,
// all ones for a tail; base in bits 32-33; a mark as 2^62 | head).
template <class W>
struct WalkWord;
template <>
struct WalkWord<uint32_t> {
  static constexpr uint64_t MAX_N = (1ull << 29) - 1;
  __host__ __device__ static uint32_t make(uint32_t next, uint32_t base) {
    return ((base & 3u) << 29) | (next == NONE32 ? 0x1fffffffu : next);
  }
  __device__ static bool marked(uint32_t w) { return (w >> 31) != 0; }
  __device__ static uint32_t mark(uint32_t head) { return 0x80000000u | head; }
  __device__ static uint32_t head(uint32_t w) { return w & 0x7fffffffu; }
  __device__ static bool tail(uint32_t w) { return (w & 0x1fffffffu) == 0x1fffffffu; }
  __device__ static uint32_t next(uint32_t w) { return w & 0x1fffffffu; }
  __device__ static uint32_t base(uint32_t w) { return (w >> 29) & 3u; }
};
template <>
struct WalkWord<uint64_t> {
  static constexpr uint64_t MAX_N = 1ull << 30;  // a staged entry holds the strand-node in 30 bits
  __host__ __device__ static uint64_t make(uint32_t next, uint32_t base) {
    return ((uint64_t)(base & 3u) << 32) | next;
  }
  __device__ static bool marked(uint64_t w) { return (w >> 62) == 1ull; }
  __device__ static uint64_t mark(uint32_t head) { return (1ull << 62) | head; }
  __device__ static uint32_t head(uint64_t w) { return (uint32_t)w; }
  __device__ static bool tail(uint64_t w) { return (uint32_t)w == NONE32; }
  __device__ static uint32_t next(uint64_t w) { return (uint32_t)w; }
  __device__ static uint32_t base(uint64_t w) { return (uint32_t)(w >> 32) & 3u; }
};

// ListRankingTransform arcs.  Strand-node x = 2v + s leaves v by its right
// side (s = 0) or its left side (s = 1); the arc exists when the edge there
// joins two distinct nodes and is alone on the far node's side too.  It
// enters w on side sw: strand 0 when that is w's left side, 1 otherwise.
// succ[x] = the successor or NONE; mk, when given, receives x's walk word
// (the meeting walks' working copy, which they mark), with x's entry base
// (entering v by side s).
template <class W>
__global__ void k_successors(const uint32_t *__restrict__ link_node, const uint64_t *__restrict__ link_edge,
                             uint64_t V, uint32_t *__restrict__ succ, W *__restrict__ mk) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < 2 * V; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = x >> 1;
    const uint32_t leave = (x & 1) ? 0u : 1u;
    const uint32_t ln = link_node[2 * v + leave];
    uint32_t out = NONE32;
    uint64_t far = 0;
    if (ln != NONE32) {
      const uint32_t w = ln >> 1, sw = ln & 1u;
      far = link_edge[2 * (uint64_t)w + sw];
      if (w != (uint32_t)v && (uint32_t)far == (uint32_t)link_edge[2 * v + leave]) out = 2 * w + (sw == 0 ? 0u : 1u);
    }
    succ[x] = out;
    if (mk) mk[x] = WalkWord<W>::make(out, (uint32_t)(link_edge[2 * v + (x & 1)] >> 32));
  }
}

// The same arcs, for up to 2^29 - 1 strand-nodes, through a bitmap small
// enough for L2 instead of a random load of the far node's link.  Per node
// v (warps on 32 consecutive nodes): the lone end of each side as in
// k_side_links (each slot's side and its far end's side from adj_side, the
// build's byte per slot, when it has one, else from the edge's orient);
// bit 2v + sd of `lone` set when side sd holds exactly one
// end (and, with `literal`, each side of v holds one); and for x = 2v + s
// the candidate word (its would-be successor, entering the far node w by
// the far end's side, unless that is v itself, with x's entry base).
// Bit 2w + sw is the bit of that successor itself, so k_succ_lone keeps a
// candidate when the bit of its successor is set.
template <class K>
__global__ void k_side_cand(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ adj_nbr,
                            const uint32_t *__restrict__ adj_edge, const uint8_t *__restrict__ adj_role,
                            const uint8_t *__restrict__ orient, const uint8_t *__restrict__ adj_side,
                            const uint64_t *__restrict__ node_keys, uint64_t V, int k, bool literal,
                            uint32_t *__restrict__ cand, uint32_t *__restrict__ lone) {
  const int lane = threadIdx.x & 31;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g < V;
       g += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = g + lane;
    uint32_t pair = 0;
    if (v < V) {
      uint32_t cnt[2] = {0, 0}, far[2] = {NONE32, NONE32};
      const uint64_t p0 = row_ptr[v], p1 = row_ptr[v + 1];
      for (uint64_t p = p0; p < p1; p++) {
        uint32_t sd, fsd;
        if (adj_side) {  // the build's per-slot sides: no gather of the edge's orient
          const uint32_t b = adj_side[p];
          sd = b & 1u;
          fsd = b >> 1;
        } else {
          const uint32_t e = adj_edge[p], role = adj_role[p];
          const uint8_t o = orient[e];
          sd = end_side(o, role);
          fsd = end_side(o, 1u - role);
        }
        cnt[sd]++;
        far[sd] = (adj_nbr[p] << 1) | fsd;
      }
      const K kv = load_node_key<K>(node_keys, v);
      const uint32_t entry[2] = {(uint32_t)KeyOps<K>::low2(kv), 3u - KeyOps<K>::digit(kv, 2 * (k - 1), 2)};
      const bool ok = !literal || (cnt[0] == 1 && cnt[1] == 1);
      const bool one[2] = {ok && cnt[0] == 1, ok && cnt[1] == 1};
#pragma unroll
      for (int s = 0; s < 2; s++) {
        const int leave = 1 - s;
        uint32_t next = NONE32;
        if (one[leave] && (far[leave] >> 1) != (uint32_t)v) next = far[leave];  // = 2w + sw
        cand[2 * v + s] = WalkWord<uint32_t>::make(next, entry[s]);
      }
      pair = (one[0] ? 1u : 0u) | (one[1] ? 2u : 0u);
    }
    const uint32_t lo = __reduce_or_sync(0xffffffffu, lane < 16 ? pair << (2 * lane) : 0u);
    const uint32_t hi = __reduce_or_sync(0xffffffffu, lane >= 16 ? pair << (2 * (lane - 16)) : 0u);
    if (lane == 0) {
      lone[g / 16] = lo;
      if (g + 16 < V) lone[g / 16 + 1] = hi;
    }
  }
}

// Keeps the candidates whose successor's side is lone too: mk[x] (in
// place) and succ[x].  Each thread takes SL_U strand-nodes a grid stride
// apart, their candidate loads and then their bitmap lookups (L2 hits at
// random) in flight together.
constexpr int SL_U = 4;

__global__ void k_succ_lone(uint32_t *__restrict__ mk, const uint32_t *__restrict__ lone, uint64_t n,
                            uint32_t *__restrict__ succ) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x0 < n; x0 += stride * SL_U) {
    uint32_t c[SL_U], bits[SL_U];
#pragma unroll
    for (int u = 0; u < SL_U; u++) {
      const uint64_t x = x0 + (uint64_t)u * stride;
      c[u] = x < n ? mk[x] : 0u;
    }
#pragma unroll
    for (int u = 0; u < SL_U; u++) {
      const uint64_t x = x0 + (uint64_t)u * stride;
      bits[u] = 0;
      if (x < n && !WalkWord<uint32_t>::tail(c[u])) {
        const uint32_t y = WalkWord<uint32_t>::next(c[u]);
        bits[u] = __ldg(lone + (y >> 5)) >> (y & 31);
      }
    }
#pragma unroll
    for (int u = 0; u < SL_U; u++) {
      const uint64_t x = x0 + (uint64_t)u * stride;
      if (x >= n) break;
      uint32_t out = NONE32;
      if (!WalkWord<uint32_t>::tail(c[u])) {
        if (bits[u] & 1u) out = WalkWord<uint32_t>::next(c[u]);
        else c[u] = WalkWord<uint32_t>::make(NONE32, WalkWord<uint32_t>::base(c[u]));
      }
      mk[x] = c[u];
      succ[x] = out;
    }
  }
}

// The predecessor of a strand-node, from the mirror symmetry of the
// transform: an arc y -> x exists exactly when x^1 -> y^1 does.
__device__ __forceinline__ uint32_t pred_of(const uint32_t *__restrict__ succ, uint64_t x) {
  const uint32_t m = succ[x ^ 1];
  return m == NONE32 ? NONE32 : (m ^ 1u);
}

// Ranking state of a strand-node, one 64-bit word: (ancestor << 32) |
// distance.  A list head is (itself, 0).  Words are read and written whole,
// so a thread that reads a neighbour mid-update sees either its old or its
// new (ancestor, distance) pair, both valid.
__host__ __device__ __forceinline__ uint64_t pk(uint32_t a, uint32_t d) { return ((uint64_t)a << 32) | d; }
__host__ __device__ __forceinline__ uint32_t pk_a(uint64_t w) { return (uint32_t)(w >> 32); }
__host__ __device__ __forceinline__ uint32_t pk_d(uint64_t w) { return (uint32_t)w; }
__device__ __forceinline__ bool pk_root(uint64_t w, uint32_t x) { return pk_a(w) == x && pk_d(w) == 0; }
constexpr uint64_t UNSET64 = ~0ull;

// Every list head walks its list, writing (head, rank), for at most `cap`
// strand-nodes; the rest of a longer list and all cycles stay UNSET.
__global__ void k_walk_lists(const uint32_t *__restrict__ succ, uint64_t n, uint32_t cap, uint64_t *__restrict__ word) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    if (succ[x ^ 1] != NONE32) continue;  // not a list head
    uint32_t y = (uint32_t)x;
    for (uint32_t i = 0; i < cap; i++) {
      word[y] = pk((uint32_t)x, i);
      const uint32_t ny = succ[y];
      if (ny == NONE32) break;
      y = ny;
    }
  }
}

// Strand-nodes the walks did not reach go on an active list, pointing to
// their predecessor at distance 1.
__global__ void k_collect_active(const uint32_t *__restrict__ succ, uint64_t n, uint64_t *__restrict__ word,
                                 uint32_t *__restrict__ active, uint32_t *count) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    if (word[x] != UNSET64) continue;
    const uint32_t p = pred_of(succ, x);
    word[x] = p == NONE32 ? pk((uint32_t)x, 0) : pk(p, 1);
    active[atomicAdd(count, 1u)] = (uint32_t)x;
  }
}

// One round of pointer jumping, in place, over the active strand-nodes.
// Counts those whose ancestor was not yet a list head.  Distances saturate,
// so on a cycle they never return to 0.
__global__ void k_jump_active(const uint32_t *__restrict__ active, uint32_t A, uint64_t *word,
                              uint32_t *jumped) {
  uint32_t local = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < A; i += gridDim.x * blockDim.x) {
    const uint32_t x = active[i];
    const uint64_t w = word[x];
    if (pk_root(w, x)) continue;
    const uint32_t p = pk_a(w);
    const uint64_t wp = word[p];
    if (pk_root(wp, p)) continue;
    word[x] = pk(pk_a(wp), (uint32_t)min((uint64_t)pk_d(w) + pk_d(wp), (uint64_t)0x7fffffffu));
    local++;
  }
  local = __reduce_add_sync(0xffffffffu, local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(jumped, local);
}

// Active strand-nodes that never reached a head lie on cycles: list them and
// seed (predecessor, own index) words for the min-label propagation.
__global__ void k_collect_cycles(const uint32_t *__restrict__ active, uint32_t A, const uint64_t *__restrict__ word,
                                 const uint32_t *__restrict__ succ, uint32_t *__restrict__ cyc_list,
                                 uint64_t *__restrict__ lab, uint32_t *count) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < A; i += gridDim.x * blockDim.x) {
    const uint32_t x = active[i];
    const uint64_t w = word[x];
    if (pk_root(w, x) || pk_root(word[pk_a(w)], pk_a(w))) continue;
    cyc_list[atomicAdd(count, 1u)] = x;
    lab[x] = pk(pred_of(succ, x), x);
  }
}

// Min-label propagation around the cycles, in place: lab[x] = (q, m) with m
// the smallest strand-node index in the cycle stretch (q, x].
__global__ void k_cycle_min(const uint32_t *__restrict__ cyc_list, uint32_t C, uint64_t *lab) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    const uint32_t x = cyc_list[i];
    const uint64_t w = lab[x];
    const uint64_t wq = lab[pk_a(w)];
    lab[x] = pk(pk_a(wq), min(pk_d(w), pk_d(wq)));
  }
}

// A cycle whose smallest strand-node is 2v (positive strand) is the copy
// kept (cyc = 1); its mirror is cyc = 2.  Both are opened at their smallest
// strand-node and ranked again as lists.
__global__ void k_cycle_break(const uint32_t *__restrict__ cyc_list, uint32_t C, const uint64_t *__restrict__ lab,
                              const uint32_t *__restrict__ succ, uint8_t *__restrict__ cyc,
                              uint64_t *__restrict__ word) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
    const uint32_t x = cyc_list[i];
    const uint32_t m = pk_d(lab[x]);
    cyc[x] = (m & 1u) ? 2 : 1;
    word[x] = m == x ? pk(x, 0) : pk(pred_of(succ, x), 1);
  }
}

// Per node: the strand kept (canonical copy), its unitig's first node, its
// rank there; the last node of the kept copy records the unitig length at
// the first node's slot.
template <class K>
__global__ void k_select(const uint64_t *__restrict__ word, const uint32_t *__restrict__ succ,
                         const uint8_t *__restrict__ cyc, const uint64_t *__restrict__ node_keys, uint64_t V,
                         int k, uint8_t *__restrict__ strand, uint32_t *__restrict__ head,
                         uint32_t *__restrict__ rank, uint32_t *__restrict__ is_head,
                         uint32_t *__restrict__ len_at_head) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x0 = 2 * v, x1 = 2 * v + 1;
    const uint64_t w0 = word[x0], w1 = word[x1];
    uint32_t s;
    const uint8_t c0 = cyc ? cyc[x0] : 0, c1 = cyc ? cyc[x1] : 0;
    if (c0 || c1) {
      s = c0 == 1 ? 0u : 1u;
    } else {
      const uint32_t h0 = pk_a(w0), h1 = pk_a(w1);
      K a = load_node_key<K>(node_keys, h0 >> 1), b = load_node_key<K>(node_keys, h1 >> 1);
      if (h0 & 1u) a = revcomp(a, k);
      if (h1 & 1u) b = revcomp(b, k);
      s = KeyOps<K>::less(a, b) ? 0u : 1u;
    }
    const uint64_t w = s ? w1 : w0;
    const uint32_t hx = pk_a(w), r = pk_d(w), h = hx >> 1;
    strand[v] = (uint8_t)s;
    head[v] = h;
    rank[v] = r;
    is_head[v] = h == (uint32_t)v ? 1u : 0u;
    const uint32_t nx = succ[2 * v + s];
    if (nx == NONE32 || nx == hx) len_at_head[h] = r + 1;
  }
}

// Unitig tables, one thread per node; the first node of each unitig writes
// its entries.  off_by_v[h] = first output slot of the unitig headed by h.
__global__ void k_unitig_offsets(const uint32_t *__restrict__ is_head, const uint64_t *__restrict__ uidx,
                                 const uint64_t *__restrict__ off_by_v, const uint32_t *__restrict__ len_at_head,
                                 const uint8_t *__restrict__ cyc, const uint8_t *__restrict__ strand, uint64_t V,
                                 uint64_t U, int k, uint64_t *__restrict__ node_off, uint64_t *__restrict__ seq_off,
                                 uint8_t *__restrict__ circular, uint4 *__restrict__ hinfo) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= V; v += (uint64_t)gridDim.x * blockDim.x) {
    if (v == V) {
      node_off[U] = V;
      seq_off[U] = V + U * (uint64_t)(k - 1);
      continue;
    }
    if (!is_head[v]) continue;
    const uint64_t u = uidx[v];
    node_off[u] = off_by_v[v];
    seq_off[u] = off_by_v[v] + u * (uint64_t)(k - 1);
    circular[u] = cyc && cyc[2 * v + strand[v]] == 1 ? 1 : 0;
    // everything a node of this unitig needs, in one 16-byte gather
    hinfo[v] = make_uint4((uint32_t)off_by_v[v], (uint32_t)u, len_at_head[v], 0u);
  }
}

// Node list and spelled string of every unitig: the node at rank r writes
// its (ID, strand) entry and, for r = 0, the first k-mer, else the last base
// of its k-mer as read on the kept strand.
template <class K>
__global__ void k_unitig_write(const uint32_t *__restrict__ head, const uint32_t *__restrict__ rank,
                               const uint8_t *__restrict__ strand, const uint4 *__restrict__ hinfo,
                               const uint64_t *__restrict__ node_keys, uint64_t V, int k,
                               uint64_t *__restrict__ nodes_out, char *__restrict__ seq, uint32_t *err) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t h = head[v];
    const uint64_t r = rank[v];
    const uint4 hi = hinfo[h];  // (first slot, unitig index, length, -)
    if (r >= hi.z) {  // a rank must fall inside its unitig
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    const uint64_t u = hi.y;
    const uint32_t s = strand[v];
    nodes_out[hi.x + r] = (v << 1) | s;
    K km = load_node_key<K>(node_keys, v);
    if (s) km = revcomp(km, k);
    const uint64_t so = hi.x + u * (uint64_t)(k - 1);
    const char *acgt = "ACGT";
    if (r == 0) {
      for (int i = 0; i < k; i++) seq[so + i] = acgt[KeyOps<K>::digit(km, 2 * (k - 1 - i), 2)];
    } else {
      seq[so + k - 1 + r] = acgt[KeyOps<K>::low2(km)];
    }
  }
}

// ---------------------------------------------------------------------------
// Fast path, for graphs whose lists are all at most `cap` strand-nodes long
// and acyclic (the usual case): the two walkers of each unitig (its two list
// heads, one per mirrored copy) walk towards each other, meet half way, and
// stage the strand-nodes they take in walk order; per pair of walkers the
// unitig's length and kept copy follow, and one copy pass writes each kept
// unitig's nodes and bases from the two staged halves.  Every strand-node's
// successor word is loaded once; no per-strand-node ranking state is written.
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ K strand_kmer(const uint64_t *node_keys, uint32_t x, int k) {
  K km = load_node_key<K>(node_keys, x >> 1);
  return (x & 1u) ? revcomp(km, k) : km;
}

// Walk scheduling: each warp takes a chunk of WALK_CHUNK indices, queues the
// list heads it finds there in shared memory (ballots), and its lanes then
// take heads from the queue one at a time, so no lane idles while another
// finishes a long list.
constexpr int WALK_BLOCK = 256, WALK_WARPS = WALK_BLOCK / 32, WALK_CHUNK = 1024;

template <class IsHead>
__device__ __forceinline__ uint32_t queue_heads(uint64_t base, uint64_t n, uint32_t *q, IsHead is_head) {
  const int lane = threadIdx.x & 31;
  uint32_t cnt = 0;
  for (int r = 0; r < WALK_CHUNK / 32; r++) {
    const uint64_t x = base + r * 32 + lane;
    const bool h = x < n && is_head(x);
    const unsigned b = __ballot_sync(0xffffffffu, h);
    if (h) q[cnt + __popc(b & ((1u << lane) - 1u))] = (uint32_t)x;
    cnt += __popc(b);
  }
  __syncwarp();
  return cnt;
}

// The meeting walks.  A walker at strand-node y loads y's word from mk, the
// working copy of the successor words; if the other walker has marked it
// (with the other walker's head) the node is the other's and the walk
// stops; else the walker marks the word the other walker would load at
// this node, mk[y ^ 1], takes y and goes on.  Plain loads and stores: two
// walkers arriving together may both take a few nodes, which the pairing
// step measures.  hrec[x] = (nodes walker x took, its last strand-node, the
// other walker's head, the index of its first staged entry); the walker
// with the smaller head of each pair appends that head to `pairs`.
//
// Staging: each lane stages the strand-nodes its walks take, in walk order,
// as entries (y << 2) | y's entry base (the base the arc into y appends), at
// consecutive indices of lane-private pages of STAGE_PAGE entries taken
// from a global cursor; page_next[page] is the page the lane went on to.
// The entries pass through eight registers and are stored eight at a time,
// one whole 32-byte sector per store pair (entries stored one by one left
// sectors half written in L2 under the walks' random traffic).  If the
// staging area runs out, *overflow is set and the walks only measure.
constexpr uint32_t STAGE_PAGE = 256;

struct StageLane {
  uint32_t b[8];
  uint32_t nb = 0;         // entries held in b
  uint64_t idx = 0, end = 0;  // the next entry's index; the current page's end
  bool full = false;
};

// The entry at lane.idx; a fresh page when the current one is used up.
__device__ __forceinline__ void stage_push(StageLane &ln, uint32_t e, uint32_t *__restrict__ stage,
                                           uint32_t *__restrict__ page_next, unsigned long long *cursor,
                                           uint64_t stage_cap, uint32_t *overflow) {
  if (ln.full) return;
  if (ln.idx == ln.end) {  // (the buffer is empty here: pages hold whole groups of eight)
    const uint64_t np = atomicAdd(cursor, (unsigned long long)STAGE_PAGE);
    if (np + STAGE_PAGE > stage_cap) {
      ln.full = true;
      atomicOr(overflow, 1u);
      return;
    }
    if (ln.end) page_next[ln.end / STAGE_PAGE - 1] = (uint32_t)(np / STAGE_PAGE);
    ln.idx = np;
    ln.end = np + STAGE_PAGE;
  }
#pragma unroll
  for (int j = 0; j < 8; j++)
    if (ln.nb == (uint32_t)j) ln.b[j] = e;
  ln.nb++;
  ln.idx++;
  if (ln.nb == 8) {
    uint4 *dst = reinterpret_cast<uint4 *>(stage + (ln.idx - 8));
    dst[0] = make_uint4(ln.b[0], ln.b[1], ln.b[2], ln.b[3]);
    dst[1] = make_uint4(ln.b[4], ln.b[5], ln.b[6], ln.b[7]);
    ln.nb = 0;
  }
}

template <class W>
__global__ __launch_bounds__(WALK_BLOCK, 6) void k_mark_stage(W *__restrict__ mk,
                                                           const uint32_t *__restrict__ succ, uint64_t n,
                                                           uint32_t cap, uint4 *__restrict__ hrec,
                                                           uint32_t *__restrict__ stage,
                                                           uint32_t *__restrict__ page_next,
                                                           unsigned long long *__restrict__ cursor,
                                                           uint64_t stage_cap, uint32_t *too_long,
                                                           uint32_t *overflow, uint32_t *__restrict__ pairs,
                                                           uint32_t *pair_count) {
  __shared__ uint32_t s_q[WALK_WARPS][WALK_CHUNK];
  __shared__ uint32_t s_next[WALK_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t chunks = (n + WALK_CHUNK - 1) / WALK_CHUNK;
  uint32_t lng = 0;
  StageLane ln;
  for (uint64_t c = (uint64_t)blockIdx.x * WALK_WARPS + w; c < chunks; c += (uint64_t)gridDim.x * WALK_WARPS) {
    const uint32_t cnt = queue_heads(c * WALK_CHUNK, n, s_q[w], [&](uint64_t x) { return succ[x ^ 1] == NONE32; });
    if (lane == 0) s_next[w] = 0;
    __syncwarp();
    for (;;) {
      const uint32_t qi = atomicAdd(&s_next[w], 1u);
      if (qi >= cnt) break;
      const uint32_t x = s_q[w][qi];
      uint32_t y = x, d = 0, last = NONE32, partner = NONE32, first = NONE32;
      for (;;) {
        const W wd = __ldcg(mk + y);  // from L2: another SM's mark may be there
        if (WalkWord<W>::marked(wd)) {
          partner = WalkWord<W>::head(wd);
          break;
        }
        __stcg(mk + (y ^ 1u), WalkWord<W>::mark(x));
        stage_push(ln, (y << 2) | WalkWord<W>::base(wd), stage, page_next, cursor, stage_cap, overflow);
        if (first == NONE32 && !ln.full) first = (uint32_t)(ln.idx - 1);
        d++;
        last = y;
        if (WalkWord<W>::tail(wd)) {
          partner = y ^ 1u;
          break;
        }
        if (d >= cap) {
          lng++;
          break;
        }
        y = WalkWord<W>::next(wd);
      }
      hrec[x] = make_uint4(d, last, partner, first);
      // append x when it is its pair's smaller head (one atomic per warp
      // for the lanes here now)
      const bool smaller = partner != NONE32 && partner > x;
      const unsigned act = __activemask();
      const unsigned want = __ballot_sync(act, smaller);
      if (want) {
        const int leader = __ffs(act) - 1;
        uint32_t at = 0;
        if (lane == leader) at = atomicAdd(pair_count, (uint32_t)__popc(want));
        at = __shfl_sync(act, at, leader);
        if (smaller) pairs[at + __popc(want & ((1u << lane) - 1u))] = x;
      }
    }
    __syncwarp();
  }
  // the last, partly filled group
  if (!ln.full)
    for (uint32_t j = 0; j < ln.nb; j++) {
      uint32_t v = ln.b[0];
#pragma unroll
      for (int t = 1; t < 8; t++)
        if (j == (uint32_t)t) v = ln.b[t];
      stage[ln.idx - ln.nb + j] = v;
    }
  lng = __reduce_add_sync(0xffffffffu, lng);
  if (lane == 0 && lng) atomicAdd(too_long, lng);
}

// Per pair of walkers (listed by the smaller head): the unitig's length
// L = d_a + d_b - o, o the nodes both took (found by stepping from the
// second walker's last node, read on the first walker's strands, to the
// first walker's last node); the copy kept (the one whose first k-mer is
// smaller) and its first node's tables: its bit in the bitmap of unitig
// heads, and the unitig's length << 1 | the kept copy's strand (one word,
// one random store).
template <class K>
__global__ void k_mark_pair(const uint32_t *__restrict__ pairs, const uint32_t *__restrict__ pair_count,
                            const uint32_t *__restrict__ succ, uint64_t n, const uint4 *__restrict__ hrec,
                            const uint64_t *__restrict__ node_keys, int k, uint32_t cap,
                            uint32_t *__restrict__ head_bits, uint32_t *__restrict__ len_at_head,
                            unsigned long long *covered, uint32_t *err) {
  unsigned long long cov = 0;
  const uint32_t np = *pair_count;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = pairs[i];
    const uint4 ra = hrec[x];
    const uint32_t p = ra.z;
    if (p >= n || p <= x) {
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    const uint4 rb = hrec[p];
    if (rb.z != x) {
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    uint32_t o = 0;
    if (ra.x > 0 && rb.x > 0 && succ[ra.y] != (rb.y ^ 1u)) {
      // the walks overlap: step from b's last node (on a's strands) to a's last
      uint32_t y = rb.y ^ 1u, steps = 0;
      while (y != ra.y && steps <= cap) {
        y = succ[y];
        steps++;
      }
      if (y != ra.y) {
        atomicOr(err, ERR_INTERNAL);
        continue;
      }
      o = steps + 1;
    }
    const uint32_t L = ra.x + rb.x - o;
    const uint32_t kept = KeyOps<K>::less(strand_kmer<K>(node_keys, p, k), strand_kmer<K>(node_keys, x, k)) ? p : x;
    const uint32_t h = kept >> 1;
    atomicOr(head_bits + (h >> 5), 1u << (h & 31u));
    len_at_head[h] = L << 1 | (kept & 1u);
    cov += L;
  }
  cov = __reduce_add_sync(0xffffffffu, (unsigned)cov);
  if ((threadIdx.x & 31) == 0 && cov) atomicAdd(covered, cov);
}

// Bits set in each 32-node word of the head bitmap.
__global__ void k_head_popc(const uint32_t *__restrict__ head_bits, uint64_t nw, uint32_t *__restrict__ cnt) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (uint64_t)gridDim.x * blockDim.x)
    cnt[i] = __popc(head_bits[i]);
}

// The unitigs in the order of their first nodes: unitig u = the u-th set bit
// of the head bitmap (wpre = the exclusive scan of the words' bit counts),
// with its first strand-node uy[u] = 2v + the kept strand and its length
// (from the head's word, length << 1 | strand).
__global__ void k_head_list(const uint32_t *__restrict__ head_bits, uint64_t nw, const uint64_t *__restrict__ wpre,
                            const uint32_t *__restrict__ len_at_head, uint32_t *__restrict__ uy,
                            uint32_t *__restrict__ ulen) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t b = head_bits[i];
    uint64_t u = wpre[i];
    while (b) {
      const uint32_t v = (uint32_t)(i * 32) + (uint32_t)(__ffs(b) - 1);
      const uint32_t w = len_at_head[v];
      uy[u] = 2 * v + (w & 1u);
      ulen[u] = w >> 1;
      u++;
      b &= b - 1u;
    }
  }
}

// The index s entries after index q of the same walk (following the lanes'
// page links).
__device__ __forceinline__ uint64_t stage_advance(const uint32_t *__restrict__ page_next, uint64_t q, uint32_t s) {
  while (s > 0) {
    const uint32_t room = STAGE_PAGE - (uint32_t)(q % STAGE_PAGE);
    if (s < room) return q + s;
    s -= room;
    q = (uint64_t)page_next[q / STAGE_PAGE] * STAGE_PAGE;
  }
  return q;
}

// 'A', 'C', 'G', 'T' for 2-bit codes 0..3
__device__ __forceinline__ char base_char(uint32_t b) { return (char)((0x54474341u >> (8 * (b & 3u))) & 0xffu); }

// Every kept unitig from its two staged halves.  With the kept walker's
// head y (the unitig's first strand-node), a nodes taken by it and L in
// all, the first a nodes are its entries in order; the other L - a are the
// first L - a entries of the other walker, read backwards on the other
// strand.  The string S (k + L - 1 bases) starts with y's k-mer, then the
// bases the kept walker's arcs appended; the rest is the reverse complement
// of the first L - a characters of the other walker's string T (its head's
// k-mer, then its arcs' bases): S[k - 2 + L - m] is the complement of T[m].
// Groups of CG lanes take the unitigs of their warp's chunk of the head
// list in turn, and each group writes a unitig's nodes and bases CG at a
// time, so that every store of the group covers consecutive addresses.
constexpr int CG = 8;
constexpr int COPY_CHUNK = 64;  // unitigs per warp chunk (about as many nodes as a walk chunk)

template <class K>
__global__ __launch_bounds__(WALK_BLOCK, 6) void k_stage_copy(
    const uint32_t *__restrict__ uy, const uint32_t *__restrict__ ulen, const uint64_t *__restrict__ uoff,
    const uint4 *__restrict__ hrec, const uint32_t *__restrict__ stage, const uint32_t *__restrict__ page_next,
    const uint64_t *__restrict__ node_keys, uint64_t V, uint64_t U, int k, uint64_t *__restrict__ nodes_out,
    char *__restrict__ seq, uint64_t *__restrict__ node_off, uint64_t *__restrict__ seq_off,
    uint8_t *__restrict__ circular) {
  __shared__ uint32_t s_next[WALK_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, gl = lane % CG;
  const unsigned gmask = ((1u << CG) - 1u) << (lane - gl);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    node_off[U] = V;
    seq_off[U] = V + U * (uint64_t)(k - 1);
  }
  const uint64_t chunks = (U + COPY_CHUNK - 1) / COPY_CHUNK;
  for (uint64_t c = (uint64_t)blockIdx.x * WALK_WARPS + w; c < chunks; c += (uint64_t)gridDim.x * WALK_WARPS) {
    const uint64_t u0 = c * COPY_CHUNK;
    const uint32_t cnt = U - u0 < (uint64_t)COPY_CHUNK ? (uint32_t)(U - u0) : (uint32_t)COPY_CHUNK;
    if (lane == 0) s_next[w] = 0;
    __syncwarp();
    for (;;) {
      uint32_t qi = 0;
      if (gl == 0) qi = atomicAdd(&s_next[w], 1u);
      qi = __shfl_sync(gmask, qi, 0, CG);
      if (qi >= cnt) break;
      const uint64_t u = u0 + qi;
      const uint32_t y = uy[u];
      const uint4 ra = hrec[y];
      const uint32_t L = ulen[u], a = ra.x, bp = L - a;
      const uint64_t off = uoff[u], so = off + u * (uint64_t)(k - 1);
      if (gl == 0) {
        node_off[u] = off;
        seq_off[u] = so;
        circular[u] = 0;
      }
      const K km = strand_kmer<K>(node_keys, y, k);
      for (int j = gl; j < k; j += CG) seq[so + j] = base_char(KeyOps<K>::digit(km, 2 * (k - 1 - j), 2));
      // (a lane follows a walk's entries only while it has one to read: a
      // walk that took no node has no first entry)
      uint64_t q = (uint32_t)gl < a ? stage_advance(page_next, ra.w, (uint32_t)gl) : 0;
      for (uint32_t e = gl; e < a; e += CG) {
        const uint32_t t = stage[q];
        nodes_out[off + e] = t >> 2;
        if (e > 0) seq[so + k - 1 + e] = base_char(t);
        if (e + CG < a) q = stage_advance(page_next, q, CG);
      }
      if (bp > 0) {
        const uint32_t zb = ra.z;
        const K kb = strand_kmer<K>(node_keys, zb, k);
        const uint32_t mk_end = min((uint32_t)k, bp);
        for (uint32_t m = gl; m < mk_end; m += CG)
          seq[so + k - 2 + L - m] = base_char(3u - KeyOps<K>::digit(kb, 2 * (k - 1 - (int)m), 2));
        q = (uint32_t)gl < bp ? stage_advance(page_next, hrec[zb].w, (uint32_t)gl) : 0;
        for (uint32_t e = gl; e < bp; e += CG) {
          const uint32_t t = stage[q];
          nodes_out[off + L - 1 - e] = (t >> 2) ^ 1u;
          if (e >= 1 && e + (uint32_t)k - 1 < bp) seq[so + L - 1 - e] = base_char(3u - t);
          if (e + CG < bp) q = stage_advance(page_next, q, CG);
        }
      }
    }
    __syncwarp();
  }
}

// enough warps to fill the device in one wave (a block beyond the resident
// ones would start its fixed share of chunks only when another ends), at
// most one per chunk
template <class F>
static unsigned walk_grid(const dbg_ctx *ctx, uint64_t n, F kern, uint64_t chunk = WALK_CHUNK) {
  const uint64_t chunks = (n + chunk - 1) / chunk;
  const uint64_t blocks = (chunks + WALK_WARPS - 1) / WALK_WARPS;
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WALK_BLOCK, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (unsigned)std::max<uint64_t>(
      1, std::min<uint64_t>(blocks, (uint64_t)std::max(1, ctx->num_sms) * (uint64_t)per_sm));
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

// Pointer jumping over a list of strand-nodes until every one that can
// reach a list head has (a round without progress leaves only cycles: a list
// always has one strand-node that finishes per round).
static dbg_status jump_until_stable(dbg_ctx *ctx, const uint32_t *list, uint32_t A, uint64_t *word,
                                    uint32_t *remaining) {
  cudaStream_t s = ctx->stream;
  uint32_t prev = 0xffffffffu, jumped = 0;
  for (int r = 0; r < 96; r++) {
    DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 3, 0, sizeof(uint32_t), s));
    DBG_LAUNCH(ctx, ST_COMPACT_RANK, 24.0 * A,
               k_jump_active<<<grid_of(A), 256, 0, s>>>(list, A, word, ctx->d_counters + 3));
    DBG_CUDA_TRY(cudaGetLastError());
    DBG_TRY(read_small(ctx, ctx->d_counters + 3, sizeof(uint32_t), &jumped));
    if (jumped == 0 || jumped == prev) {
      *remaining = jumped;
      return DBG_OK;
    }
    prev = jumped;
  }
  set_error("list ranking did not converge");
  return DBG_ETIMEOUT;
}

// The general path's ending, from the ranking words (word[x] = (list head,
// rank) of every strand-node), the successors and the cycle marks: the kept
// copy of every unitig, its tables, node list and string.  Also the empty
// graph's (V = 0) tables.
template <class K>
static dbg_status finish_from_words(dbg_ctx *ctx, const dbg_graph *g, dbg_unitigs *u, DevBuf &word, DevBuf &succ,
                                    DevBuf &cyc, bool have_cycles) {
  cudaStream_t s = ctx->stream;
  const uint64_t V = g->num_nodes, n = 2 * V;
  const int k = (int)g->k;
  u->num_nodes = V;
  const uint64_t V1 = std::max<uint64_t>(1, V);
  DevBuf strand, head, rank, is_head, len_at_head, uidx, off_by_v;
  uint64_t U = 0;
  if (V > 0) {
    DBG_TRY(alloc_buf(ctx, strand, V1));
    DBG_TRY(alloc_buf(ctx, head, V1 * 4));
    DBG_TRY(alloc_buf(ctx, rank, V1 * 4));
    DBG_TRY(alloc_buf(ctx, is_head, V1 * 4));
    DBG_TRY(alloc_buf(ctx, len_at_head, V1 * 4));
    DBG_CUDA_TRY(cudaMemsetAsync(len_at_head.p, 0, V1 * 4, s));
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 16.0 * n + 8.0 * V + 17.0 * V,
               k_select<K><<<grid_of(V), 256, 0, s>>>(word.as<uint64_t>(), succ.as<uint32_t>(),
                                                      have_cycles ? cyc.as<uint8_t>() : nullptr,
                                                      g->node_keys.as<uint64_t>(), V, k, strand.as<uint8_t>(),
                                                      head.as<uint32_t>(), rank.as<uint32_t>(),
                                                      is_head.as<uint32_t>(), len_at_head.as<uint32_t>()));
    DBG_CUDA_TRY(cudaGetLastError());
    word.release();
    succ.release();
    DBG_TRY(alloc_buf(ctx, uidx, (V + 1) * 8));
    DBG_TRY(alloc_buf(ctx, off_by_v, (V + 1) * 8));
    uint32_t U32 = 0, total = 0;
    DBG_TRY(scan_excl(ctx, is_head.as<uint32_t>(), V, uidx.as<uint64_t>(), &U32));
    DBG_TRY(scan_excl(ctx, len_at_head.as<uint32_t>(), V, off_by_v.as<uint64_t>(), &total));
    if (total != V) {
      set_error("unitigs hold %u nodes, expected %llu", total, (unsigned long long)V);
      return DBG_EINTERNAL;
    }
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
    DevBuf hinfo;
    DBG_TRY(alloc_buf(ctx, hinfo, V1 * sizeof(uint4)));
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 4.0 * V + 16.0 * U * 5,
               k_unitig_offsets<<<grid_of(V + 1), 256, 0, s>>>(
                   is_head.as<uint32_t>(), uidx.as<uint64_t>(), off_by_v.as<uint64_t>(), len_at_head.as<uint32_t>(),
                   have_cycles ? cyc.as<uint8_t>() : nullptr, strand.as<uint8_t>(), V, U, k,
                   u->node_off.as<uint64_t>(), u->seq_off.as<uint64_t>(), u->circular.as<uint8_t>(),
                   hinfo.as<uint4>()));
    DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT,
               (double)V * (4 + 4 + 1 + 16 + 8 * g->key_words + 8 + 1) + (double)U * k,
               k_unitig_write<K><<<grid_of(V), 256, 0, s>>>(head.as<uint32_t>(), rank.as<uint32_t>(),
                                                            strand.as<uint8_t>(), hinfo.as<uint4>(),
                                                            g->node_keys.as<uint64_t>(), V, k,
                                                            u->nodes.as<uint64_t>(), u->seq.as<char>(), ctx->d_err));
    DBG_CUDA_TRY(cudaGetLastError());
  } else {
    DBG_CUDA_TRY(cudaMemsetAsync(u->node_off.p, 0, 8, s));
    DBG_CUDA_TRY(cudaMemsetAsync(u->seq_off.p, 0, 8, s));
  }
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  return check_device_error(ctx);
}


// Lists of up to this many strand-nodes are ranked by one walking thread.
constexpr uint32_t kWalkCap = 2048;

template <class K>
static dbg_status compact_impl(dbg_ctx *ctx, const dbg_graph *g, dbg_unitigs *u, bool literal = false) {
  cudaStream_t s = ctx->stream;
  const uint64_t V = g->num_nodes, n = 2 * V, E2 = 2 * g->num_edges;
  const int k = (int)g->k;
  u->num_nodes = V;
  const uint64_t V1 = std::max<uint64_t>(1, V), n1 = std::max<uint64_t>(1, n);
  DevBuf link_node, link_edge, succ, word, active, cycl, lab, cyc;
  bool have_cycles = false;
  if (V > 0) {
    // the meeting walks' words: 32-bit up to 2^29 - 1 strand-nodes, 64-bit
    // up to 2^30 (their staged entries hold a strand-node in 30 bits)
    const bool fast = ctx->compact_mode != 2 && n <= WalkWord<uint64_t>::MAX_N;
    const bool w32 = fast && ctx->compact_mode == 0 && n <= WalkWord<uint32_t>::MAX_N;
    DevBuf mk;
    DBG_TRY(alloc_buf(ctx, succ, n1 * 4));
    if (fast) DBG_TRY(alloc_buf(ctx, mk, n1 * (w32 ? 4 : 8)));
    if (w32) {
      // per side the lone end, a bitmap of the lone sides, the candidate
      // words; then the arcs whose far side is lone too
      DevBuf lone;
      DBG_TRY(alloc_buf(ctx, lone, (V / 16 + 2) * 4));
      DBG_LAUNCH(ctx, ST_COMPACT_LINKS,
                 16.0 * V + (double)E2 * (g->adj_side.p ? 5 : 10) + 8.0 * V * g->key_words + 8.0 * V + V / 4.0,
                 k_side_cand<K><<<grid_of(V), 256, 0, s>>>(g->row_ptr.as<uint64_t>(), g->adj_nbr.as<uint32_t>(),
                                                           g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(),
                                                           g->orient.as<uint8_t>(), g->adj_side.as<uint8_t>(),
                                                           g->node_keys.as<uint64_t>(), V, k, literal,
                                                           mk.as<uint32_t>(), lone.as<uint32_t>()));
      DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 12.0 * n,
                 k_succ_lone<<<grid_of(n), 256, 0, s>>>(mk.as<uint32_t>(), lone.as<uint32_t>(), n,
                                                        succ.as<uint32_t>()));
    } else {
      DBG_TRY(alloc_buf(ctx, link_node, n1 * 4));
      DBG_TRY(alloc_buf(ctx, link_edge, n1 * 8));
      DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 16.0 * V + (double)E2 * 10 + 8.0 * V * g->key_words + 12.0 * n,
                 k_side_links<K><<<grid_of(V), 256, 0, s>>>(g->row_ptr.as<uint64_t>(), g->adj_nbr.as<uint32_t>(),
                                                            g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(),
                                                            g->orient.as<uint8_t>(), g->node_keys.as<uint64_t>(), V,
                                                            k, literal, link_node.as<uint32_t>(),
                                                            link_edge.as<uint64_t>()));
      DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 12.0 * n + 8.0 * n + (fast ? 12.0 : 4.0) * n,
                 k_successors<uint64_t><<<grid_of(n), 256, 0, s>>>(link_node.as<uint32_t>(), link_edge.as<uint64_t>(),
                                                                   V, succ.as<uint32_t>(),
                                                                   fast ? mk.as<uint64_t>() : nullptr));
      link_node.release();
      link_edge.release();
    }
    // ---- fast path: short acyclic lists only ----
    if (fast) {
      // the heads of the unitigs as a bitmap over the nodes; their lengths
      // and kept strands at the head nodes only
      DevBuf f_bits, f_len, hrec, stage, page_next;
      const uint64_t nw = (V + 31) / 32, nw1 = std::max<uint64_t>(1, nw);
      DBG_TRY(alloc_buf(ctx, f_bits, nw1 * 4));
      DBG_TRY(alloc_buf(ctx, f_len, V1 * 4));
      DBG_CUDA_TRY(cudaMemsetAsync(f_bits.p, 0, nw1 * 4, s));
      // the two walkers of each unitig meet half way and stage what they
      // take (k_mark_stage); each pair gives its unitig's length and kept
      // copy (k_mark_pair).  Staging room: every node once (the few that
      // both walkers of a pair take within the margin), plus two partly
      // used pages per lane.
      const unsigned wgrid = w32 ? walk_grid(ctx, n, k_mark_stage<uint32_t>) : walk_grid(ctx, n, k_mark_stage<uint64_t>);
      const uint64_t lanes = (uint64_t)wgrid * WALK_BLOCK;
      const uint64_t stage_cap = ((V + V / 4 + 2 * lanes * STAGE_PAGE) / STAGE_PAGE + 1) * STAGE_PAGE;
      DBG_TRY(alloc_buf(ctx, hrec, n1 * sizeof(uint4)));
      DBG_TRY(alloc_buf(ctx, stage, stage_cap * 4));
      DBG_TRY(alloc_buf(ctx, page_next, stage_cap / STAGE_PAGE * 4));
      // counters: 11 too_long, 12-13 covered, 14-15 page cursor, 16 overflow,
      // 17 pairs listed
      DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 10, 0, 8 * sizeof(uint32_t), s));
      DevBuf pairs;
      DBG_TRY(alloc_buf(ctx, pairs, V1 * 4));
      unsigned long long *cursor = reinterpret_cast<unsigned long long *>(ctx->d_counters + 14);
      if (w32)
        DBG_LAUNCH(ctx, ST_COMPACT_RANK, 8.0 * n + 16.0 * V + 4.0 * V,
                   k_mark_stage<uint32_t><<<wgrid, WALK_BLOCK, 0, s>>>(
                       mk.as<uint32_t>(), succ.as<uint32_t>(), n, kWalkCap, hrec.as<uint4>(), stage.as<uint32_t>(),
                       page_next.as<uint32_t>(), cursor, stage_cap, ctx->d_counters + 11, ctx->d_counters + 16,
                       pairs.as<uint32_t>(), ctx->d_counters + 17));
      else
        DBG_LAUNCH(ctx, ST_COMPACT_RANK, 8.0 * n + 24.0 * V + 4.0 * V,
                   k_mark_stage<uint64_t><<<wgrid, WALK_BLOCK, 0, s>>>(
                       mk.as<uint64_t>(), succ.as<uint32_t>(), n, kWalkCap, hrec.as<uint4>(), stage.as<uint32_t>(),
                       page_next.as<uint32_t>(), cursor, stage_cap, ctx->d_counters + 11, ctx->d_counters + 16,
                       pairs.as<uint32_t>(), ctx->d_counters + 17));
      DBG_CUDA_TRY(cudaGetLastError());
      uint32_t flags[6] = {0, 0, 0, 0, 0, 0};  // counters 11..16
      DBG_TRY(read_small(ctx, ctx->d_counters + 11, sizeof(flags), flags));
      const uint32_t too_long = flags[0], overflow = flags[5];
      mk.release();
      uint64_t covered = 0;
      if (too_long == 0 && overflow == 0) {
        DBG_LAUNCH(ctx, ST_COMPACT_RANK, 8.0 * n + 32.0 * V,
                   k_mark_pair<K><<<grid_of(V), 256, 0, s>>>(pairs.as<uint32_t>(), ctx->d_counters + 17,
                                                             succ.as<uint32_t>(), n, hrec.as<uint4>(),
                                                             g->node_keys.as<uint64_t>(), k, kWalkCap,
                                                             f_bits.as<uint32_t>(), f_len.as<uint32_t>(),
                                                             reinterpret_cast<unsigned long long *>(ctx->d_counters + 12),
                                                             ctx->d_err));
        DBG_CUDA_TRY(cudaGetLastError());
        DBG_TRY(read_small(ctx, ctx->d_counters + 12, sizeof(uint64_t), &covered));
        DBG_TRY(check_device_error(ctx));
      }
      if (too_long == 0 && overflow == 0 && covered == V) {
        // the unitigs in the order of their first nodes: a scan over the
        // bitmap words, the list of heads, a scan over the unitigs' lengths
        DevBuf wcnt, wpre, uy, ulen, uoff;
        DBG_TRY(alloc_buf(ctx, wcnt, nw1 * 4));
        DBG_TRY(alloc_buf(ctx, wpre, (nw + 1) * 8));
        DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 8.0 * nw,
                   k_head_popc<<<grid_of(nw), 256, 0, s>>>(f_bits.as<uint32_t>(), nw, wcnt.as<uint32_t>()));
        uint32_t U32 = 0, total = 0;
        DBG_TRY(scan_excl(ctx, wcnt.as<uint32_t>(), nw, wpre.as<uint64_t>(), &U32));
        const uint64_t Uf = U32;
        DBG_TRY(alloc_buf(ctx, uy, std::max<uint64_t>(1, Uf) * 4));
        DBG_TRY(alloc_buf(ctx, ulen, std::max<uint64_t>(1, Uf) * 4));
        DBG_TRY(alloc_buf(ctx, uoff, (Uf + 1) * 8));
        DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, 12.0 * nw + (double)Uf * (4 + 4 + 4),
                   k_head_list<<<grid_of(nw), 256, 0, s>>>(f_bits.as<uint32_t>(), nw, wpre.as<uint64_t>(),
                                                           f_len.as<uint32_t>(), uy.as<uint32_t>(),
                                                           ulen.as<uint32_t>()));
        DBG_TRY(scan_excl(ctx, ulen.as<uint32_t>(), Uf, uoff.as<uint64_t>(), &total));
        if (total != V) {
          set_error("unitigs hold %u nodes, expected %llu", total, (unsigned long long)V);
          return DBG_EINTERNAL;
        }
        u->count = Uf;
        DBG_TRY(alloc_buf(ctx, u->node_off, (Uf + 1) * 8));
        DBG_TRY(alloc_buf(ctx, u->seq_off, (Uf + 1) * 8));
        DBG_TRY(alloc_buf(ctx, u->circular, std::max<uint64_t>(1, Uf)));
        DBG_TRY(alloc_buf(ctx, u->nodes, V1 * 8));
        u->total_bases = V + Uf * (uint64_t)(k - 1);
        DBG_TRY(alloc_buf(ctx, u->seq, std::max<uint64_t>(1, u->total_bases)));
        DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT,
                   (double)V * (4 + 8 + 1) + (double)Uf * (4 + 4 + 8 + 32 + 8 * g->key_words * 2 + 16 + k),
                   k_stage_copy<K><<<walk_grid(ctx, Uf, k_stage_copy<K>, COPY_CHUNK), WALK_BLOCK, 0, s>>>(
                       uy.as<uint32_t>(), ulen.as<uint32_t>(), uoff.as<uint64_t>(), hrec.as<uint4>(),
                       stage.as<uint32_t>(), page_next.as<uint32_t>(), g->node_keys.as<uint64_t>(), V, Uf, k,
                       u->nodes.as<uint64_t>(), u->seq.as<char>(), u->node_off.as<uint64_t>(),
                       u->seq_off.as<uint64_t>(), u->circular.as<uint8_t>()));
        DBG_CUDA_TRY(cudaGetLastError());
        DBG_CUDA_TRY(cudaStreamSynchronize(s));
        return check_device_error(ctx);
      }
    }
    // ---- general path: long lists or cycles present ----
    mk.release();
    DBG_TRY(alloc_buf(ctx, word, n1 * 8));
    DBG_CUDA_TRY(cudaMemsetAsync(word.p, 0xff, n * 8, s));
    DBG_LAUNCH(ctx, ST_COMPACT_RANK, 4.0 * n + 12.0 * n,
               k_walk_lists<<<grid_of(n), 256, 0, s>>>(succ.as<uint32_t>(), n, kWalkCap,
                                                       word.as<uint64_t>()));
    DBG_CUDA_TRY(cudaGetLastError());
    // what the walks left: tails of very long lists, and cycles
    DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 4, 0, sizeof(uint32_t), s));
    DBG_TRY(alloc_buf(ctx, active, n1 * 4));
    DBG_LAUNCH(ctx, ST_COMPACT_RANK, 16.0 * n,
               k_collect_active<<<grid_of(n), 256, 0, s>>>(succ.as<uint32_t>(), n, word.as<uint64_t>(),
                                                           active.as<uint32_t>(), ctx->d_counters + 4));
    uint32_t A = 0;
    DBG_TRY(read_small(ctx, ctx->d_counters + 4, sizeof(uint32_t), &A));
    if (A > 0) {
      uint32_t left = 0;
      DBG_TRY(jump_until_stable(ctx, active.as<uint32_t>(), A, word.as<uint64_t>(), &left));
      if (left > 0) {
        have_cycles = true;
        DBG_TRY(alloc_buf(ctx, cycl, (uint64_t)A * 4));
        DBG_TRY(alloc_buf(ctx, lab, n1 * 8));
        DBG_TRY(alloc_buf(ctx, cyc, n1));
        DBG_CUDA_TRY(cudaMemsetAsync(cyc.p, 0, n, s));
        DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 5, 0, sizeof(uint32_t), s));
        DBG_LAUNCH(ctx, ST_COMPACT_CYCLES, 24.0 * A,
                   k_collect_cycles<<<grid_of(A), 256, 0, s>>>(active.as<uint32_t>(), A, word.as<uint64_t>(),
                                                               succ.as<uint32_t>(), cycl.as<uint32_t>(),
                                                               lab.as<uint64_t>(), ctx->d_counters + 5));
        uint32_t C = 0;
        DBG_TRY(read_small(ctx, ctx->d_counters + 5, sizeof(uint32_t), &C));
        int R = 2;
        while ((1ull << (R - 2)) < C) R++;
        for (int r = 0; r < R; r++)
          DBG_LAUNCH(ctx, ST_COMPACT_CYCLES, 20.0 * C,
                     k_cycle_min<<<grid_of(C), 256, 0, s>>>(cycl.as<uint32_t>(), C, lab.as<uint64_t>()));
        DBG_LAUNCH(ctx, ST_COMPACT_CYCLES, 25.0 * C,
                   k_cycle_break<<<grid_of(C), 256, 0, s>>>(cycl.as<uint32_t>(), C, lab.as<uint64_t>(),
                                                            succ.as<uint32_t>(), cyc.as<uint8_t>(),
                                                            word.as<uint64_t>()));
        DBG_CUDA_TRY(cudaGetLastError());
        uint32_t still = 0;
        DBG_TRY(jump_until_stable(ctx, cycl.as<uint32_t>(), C, word.as<uint64_t>(), &still));
        if (still != 0) {
          set_error("%u strand-nodes stayed on cycles after they were opened", still);
          return DBG_EINTERNAL;
        }
      }
    }
    active.release();
    cycl.release();
    lab.release();
  }
  return finish_from_words<K>(ctx, g, u, word, succ, cyc, have_cycles);
}

// ---------------------------------------------------------------------------
// Out-of-core ranking (Section 6.2): list ranking as rounds of sort-join over
// key ranges.  The ranking word of every strand-node, W[x] = (ancestor,
// distance), lives in host memory.  A round takes every unresolved x, sorts
// its request -- the word W[x], whose ancestor is the join key -- by the
// ancestor's key range, and for each range brings the words of that range
// (the other side of the join, sorted by their own index) to the device
// with the range's requests, in batches that fit the memory budget; the
// device combines each request with its ancestor's word, and the results
// replace the words once the round is over (pointer jumping, synchronous).
// A strand-node whose ancestor is a list head does not jump and leaves the
// unresolved set.  When a round jumps as many strand-nodes as the one
// before, only cycles remain; they are labelled by their smallest
// strand-node with the same rounds (min-label doubling), opened there and
// ranked again.  The paper's join of the successor tuples (x, y) with the
// tuples (y, y') becomes the join of W[x] with W[ancestor of x].
// ---------------------------------------------------------------------------

// One synchronous round, for requests whose ancestor lies in the slice
// [lo, lo + m) of the words: mode 0 jumps (unless the ancestor is a list
// head), mode 1 takes the smaller label.  jumped counts the jumps.
__global__ void k_join_round(const uint64_t *__restrict__ req, uint64_t R, const uint64_t *__restrict__ slice,
                             uint32_t lo, int mode, uint64_t *__restrict__ out, uint8_t *__restrict__ moved,
                             uint32_t *jumped) {
  uint32_t local = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t w = req[i];
    const uint32_t t = pk_a(w);
    const uint64_t wt = slice[t - lo];
    if (mode == 0) {
      const bool stay = pk_root(wt, t);
      out[i] = stay ? w : pk(pk_a(wt), (uint32_t)min((uint64_t)pk_d(w) + pk_d(wt), (uint64_t)0x7fffffffu));
      moved[i] = stay ? 0 : 1;
      local += stay ? 0u : 1u;
    } else {
      out[i] = pk(pk_a(wt), min(pk_d(w), pk_d(wt)));
      moved[i] = 1;
    }
  }
  local = __reduce_add_sync(0xffffffffu, local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(jumped, local);
}

namespace {
struct PinnedBuf {
  void *p = nullptr;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf &) = delete;
  PinnedBuf &operator=(const PinnedBuf &) = delete;
  ~PinnedBuf() {
    if (p) cudaFreeHost(p);
  }
  dbg_status alloc(size_t bytes) {
    if (cudaMallocHost(&p, std::max<size_t>(bytes, 8)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error("cudaMallocHost of %zu bytes failed", bytes);
      return DBG_ENOMEM;
    }
    return DBG_OK;
  }
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// device buffers of one batch of a round
struct JoinBufs {
  DevBuf req, out, moved, slice;
  uint64_t batch = 0, slice_len = 0;
};
}  // namespace

// One round over the strand-nodes in act (words in W, n of them): the
// requests grouped by their ancestor's slice, each slice's requests joined
// on the device in batches; then the words replaced.  act keeps the nodes
// that moved (mode 0: jumped; mode 1: all).  Returns the jumps.
static dbg_status join_round(dbg_ctx *ctx, std::vector<uint32_t> &act, uint64_t *W, uint64_t n, int mode,
                             JoinBufs &jb, PinnedBuf &h_req, PinnedBuf &h_out, PinnedBuf &h_moved,
                             uint64_t *jumped) {
  cudaStream_t s = ctx->stream;
  const uint64_t A = act.size(), S = jb.slice_len;
  const uint64_t nb = (n + S - 1) / S;
  std::vector<uint64_t> start(nb + 1, 0);
  for (uint32_t x : act) start[pk_a(W[x]) / S + 1]++;
  for (uint64_t b = 0; b < nb; b++) start[b + 1] += start[b];
  std::vector<uint32_t> order(A);
  {
    std::vector<uint64_t> fill(start.begin(), start.end() - 1);
    uint64_t *req = h_req.as<uint64_t>();
    for (uint32_t x : act) {
      const uint64_t w = W[x];
      const uint64_t q = fill[pk_a(w) / S]++;
      order[q] = x;
      req[q] = w;
    }
  }
  DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 12, 0, sizeof(uint32_t), s));
  for (uint64_t b = 0; b < nb; b++) {
    const uint64_t r0 = start[b], r1 = start[b + 1];
    if (r0 == r1) continue;
    const uint64_t lo = b * S, m = std::min(S, n - lo);
    DBG_CUDA_TRY(cudaMemcpyAsync(jb.slice.p, W + lo, m * 8, cudaMemcpyHostToDevice, s));
    for (uint64_t r = r0; r < r1; r += jb.batch) {
      const uint64_t R = std::min(jb.batch, r1 - r);
      DBG_CUDA_TRY(cudaMemcpyAsync(jb.req.p, h_req.as<uint64_t>() + r, R * 8, cudaMemcpyHostToDevice, s));
      DBG_LAUNCH(ctx, ST_COMPACT_RANK, 25.0 * R,
                 k_join_round<<<grid_of(R), 256, 0, s>>>(jb.req.as<uint64_t>(), R, jb.slice.as<uint64_t>(),
                                                         (uint32_t)lo, mode, jb.out.as<uint64_t>(),
                                                         jb.moved.as<uint8_t>(), ctx->d_counters + 12));
      DBG_CUDA_TRY(cudaMemcpyAsync(h_out.as<uint64_t>() + r, jb.out.p, R * 8, cudaMemcpyDeviceToHost, s));
      DBG_CUDA_TRY(cudaMemcpyAsync(h_moved.as<uint8_t>() + r, jb.moved.p, R, cudaMemcpyDeviceToHost, s));
    }
  }
  DBG_CUDA_TRY(cudaGetLastError());
  uint32_t j = 0;
  DBG_TRY(read_small(ctx, ctx->d_counters + 12, sizeof(uint32_t), &j));  // synchronizes the stream
  *jumped = j;
  // every slice has been read: the new words replace the old ones
  const uint64_t *out = h_out.as<uint64_t>();
  const uint8_t *moved = h_moved.as<uint8_t>();
  act.clear();
  for (uint64_t q = 0; q < A; q++) {
    W[order[q]] = out[q];
    if (moved[q]) act.push_back(order[q]);
  }
  std::sort(act.begin(), act.end());
  return DBG_OK;
}

// Rounds of jumping over act until no strand-node jumps or the jumps stop
// shrinking (only cycles left); returns those left.
static dbg_status jump_rounds(dbg_ctx *ctx, std::vector<uint32_t> &act, uint64_t *W, uint64_t n, JoinBufs &jb,
                              PinnedBuf &h_req, PinnedBuf &h_out, PinnedBuf &h_moved, uint64_t *left) {
  uint64_t prev = ~0ull, jumped = 0;
  for (int r = 0; r < 96 && !act.empty(); r++) {
    DBG_TRY(join_round(ctx, act, W, n, 0, jb, h_req, h_out, h_moved, &jumped));
    if (jumped == 0 || jumped == prev) {
      *left = jumped;
      return DBG_OK;
    }
    prev = jumped;
  }
  *left = act.empty() ? 0 : jumped;
  if (!act.empty() && jumped != prev) {
    set_error("list ranking did not converge");
    return DBG_ETIMEOUT;
  }
  return DBG_OK;
}

template <class K>
static dbg_status compact_bucketed_impl(dbg_ctx *ctx, const dbg_graph *g, uint64_t budget, dbg_unitigs *u,
                                        uint32_t *rounds) {
  cudaStream_t s = ctx->stream;
  const uint64_t V = g->num_nodes, n = 2 * V;
  const int k = (int)g->k;
  DevBuf succ, word, cyc;
  if (V == 0) return finish_from_words<K>(ctx, g, u, word, succ, cyc, false);
  // successors on the device (the graph is there), then to host memory
  {
    DevBuf link_node, link_edge;
    DBG_TRY(alloc_buf(ctx, link_node, n * 4));
    DBG_TRY(alloc_buf(ctx, link_edge, n * 8));
    DBG_TRY(alloc_buf(ctx, succ, n * 4));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 16.0 * V + 20.0 * g->num_edges + 8.0 * V * g->key_words + 12.0 * n,
               k_side_links<K><<<grid_of(V), 256, 0, s>>>(g->row_ptr.as<uint64_t>(), g->adj_nbr.as<uint32_t>(),
                                                          g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(),
                                                          g->orient.as<uint8_t>(), g->node_keys.as<uint64_t>(), V, k,
                                                          false, link_node.as<uint32_t>(), link_edge.as<uint64_t>()));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 24.0 * n,
               k_successors<uint64_t><<<grid_of(n), 256, 0, s>>>(link_node.as<uint32_t>(), link_edge.as<uint64_t>(),
                                                                 V, succ.as<uint32_t>(), nullptr));
    DBG_CUDA_TRY(cudaGetLastError());
  }
  PinnedBuf h_succ, h_W, h_lab, h_req, h_out, h_moved;
  DBG_TRY(h_succ.alloc(n * 4));
  DBG_TRY(h_W.alloc(n * 8));
  DBG_TRY(h_req.alloc(n * 8));
  DBG_TRY(h_out.alloc(n * 8));
  DBG_TRY(h_moved.alloc(n));
  DBG_CUDA_TRY(cudaMemcpyAsync(h_succ.p, succ.p, n * 4, cudaMemcpyDeviceToHost, s));
  DBG_CUDA_TRY(cudaStreamSynchronize(s));
  const uint32_t *sc = h_succ.as<uint32_t>();
  uint64_t *W = h_W.as<uint64_t>();
  auto pred = [&](uint64_t x) -> uint32_t {
    const uint32_t m = sc[x ^ 1];
    return m == NONE32 ? NONE32 : (m ^ 1u);
  };
  // the device side of a round within the budget: a slice of words and a
  // batch of requests, results and flags (8 + 8 + 8 + 1 bytes per entry)
  JoinBufs jb;
  const uint64_t per = std::max<uint64_t>(1u << 12, budget / 25);
  jb.slice_len = std::min<uint64_t>(n, per);
  jb.batch = std::min<uint64_t>(n, per);
  DBG_TRY(alloc_buf(ctx, jb.slice, jb.slice_len * 8));
  DBG_TRY(alloc_buf(ctx, jb.req, jb.batch * 8));
  DBG_TRY(alloc_buf(ctx, jb.out, jb.batch * 8));
  DBG_TRY(alloc_buf(ctx, jb.moved, jb.batch));
  // initial words: a list head is its own root; every other strand-node
  // points at its predecessor at distance 1
  std::vector<uint32_t> act;
  for (uint64_t x = 0; x < n; x++) {
    const uint32_t p = pred(x);
    W[x] = p == NONE32 ? pk((uint32_t)x, 0) : pk(p, 1);
    if (p != NONE32) act.push_back((uint32_t)x);
  }
  uint64_t left = 0;
  const uint64_t r0 = ctx->launches;
  DBG_TRY(jump_rounds(ctx, act, W, n, jb, h_req, h_out, h_moved, &left));
  bool have_cycles = false;
  std::vector<uint8_t> h_cyc;
  if (left > 0) {
    // cycles: min-label doubling over their strand-nodes, then opened at the
    // smallest and ranked again
    have_cycles = true;
    std::vector<uint32_t> cyc_nodes = act;
    DBG_TRY(h_lab.alloc(n * 8));
    uint64_t *lab = h_lab.as<uint64_t>();
    for (uint32_t x : cyc_nodes) lab[x] = pk(pred(x), x);
    int R = 2;
    while ((1ull << (R - 2)) < cyc_nodes.size()) R++;
    for (int r = 0; r < R; r++) {
      std::vector<uint32_t> all = cyc_nodes;
      uint64_t dummy = 0;
      DBG_TRY(join_round(ctx, all, lab, n, 1, jb, h_req, h_out, h_moved, &dummy));
    }
    h_cyc.assign(n, 0);
    act.clear();
    for (uint32_t x : cyc_nodes) {
      const uint32_t m = pk_d(lab[x]);
      h_cyc[x] = (m & 1u) ? 2 : 1;
      W[x] = m == x ? pk(x, 0) : pk(pred(x), 1);
      if (m != x) act.push_back(x);
    }
    uint64_t still = 0;
    DBG_TRY(jump_rounds(ctx, act, W, n, jb, h_req, h_out, h_moved, &still));
    if (still != 0) {
      set_error("%llu strand-nodes stayed on cycles after they were opened", (unsigned long long)still);
      return DBG_EINTERNAL;
    }
  }
  *rounds = (uint32_t)(ctx->launches - r0);
  jb = JoinBufs();
  // the ranking words back on the device for the rest of the general path
  DBG_TRY(alloc_buf(ctx, word, n * 8));
  DBG_CUDA_TRY(cudaMemcpyAsync(word.p, W, n * 8, cudaMemcpyHostToDevice, s));
  if (have_cycles) {
    DBG_TRY(alloc_buf(ctx, cyc, n));
    DBG_CUDA_TRY(cudaMemcpyAsync(cyc.p, h_cyc.data(), n, cudaMemcpyHostToDevice, s));
  }
  DBG_CUDA_TRY(cudaStreamSynchronize(s));  // the host words may go
  return finish_from_words<K>(ctx, g, u, word, succ, cyc, have_cycles);
}

dbg_status compact_chains(dbg_ctx *ctx, const dbg_graph *g, dbg_unitigs *u, bool literal) {
  return g->key_words == 1 ? compact_impl<uint64_t>(ctx, g, u, literal) : compact_impl<Key128>(ctx, g, u, literal);
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
  u->n_copy = ctx->copy_streams;
  dbg_status st = compact_chains(ctx, g, u, false);
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

dbg_status dbg_compact_bucketed(dbg_ctx *ctx, const dbg_graph *g, uint64_t mem_budget, dbg_unitigs **out,
                                uint32_t *join_launches) {
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
  if (mem_budget == 0) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    mem_budget = free_b / 2;
  }
  dbg_unitigs *u = new (std::nothrow) dbg_unitigs();
  if (!u) return DBG_ENOMEM;
  u->al = ctx->al;
  u->device = ctx->device;
  u->n_copy = ctx->copy_streams;
  uint32_t launches = 0;
  dbg_status st = g->key_words == 1 ? compact_bucketed_impl<uint64_t>(ctx, g, mem_budget, u, &launches)
                                    : compact_bucketed_impl<Key128>(ctx, g, mem_budget, u, &launches);
  for (DevBuf *b : {&u->node_off, &u->nodes, &u->seq_off, &u->seq, &u->circular}) b->al = &u->al;
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  if (join_launches) *join_launches = launches;
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
  // the arrays in chunks over several streams (the copy engines side by side)
  dbg_status st = DBG_OK;
  cudaStream_t streams[kCopyStreams] = {};
  const int ns = std::max(1, std::min(u->n_copy, kCopyStreams));
  for (int i = 0; i < ns; i++)
    if (st == DBG_OK && cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaStreamCreate failed");
      st = DBG_ECUDA;
    }
  int next = 0;
  for (auto &it : items)
    if (st == DBG_OK && it.dst && it.bytes) st = copy_spread(streams, ns, &next, it.dst, it.src, it.bytes);
  for (cudaStream_t cs : streams) {
    if (!cs) continue;
    const cudaError_t e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess && st == DBG_OK) {
      set_error("copy failed: %s", cudaGetErrorString(e));
      st = DBG_ECUDA;
    }
    cudaStreamDestroy(cs);
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

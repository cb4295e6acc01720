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

// side of an edge end: 0 = left, 1 = right
__device__ __forceinline__ uint32_t end_side(uint8_t orient, uint32_t role) {
  const uint32_t o1 = orient >> 1, o2 = orient & 1u;
  return role == 0 ? (o1 ? 0u : 1u) : (o2 ? 1u : 0u);
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

// ListRankingTransform arcs.  Strand-node x = 2v + s leaves v by its right
// side (s = 0) or its left side (s = 1); the arc exists when the edge there
// joins two distinct nodes and is alone on the far node's side too.  It
// enters w on side sw: strand 0 when that is w's left side, 1 otherwise.
// succ_base[x] = succ[x] | (the base appended on that arc) << 32, or all
// ones, for the walks that write the unitigs' strings.
__global__ void k_successors(const uint32_t *__restrict__ link_node, const uint64_t *__restrict__ link_edge,
                             uint64_t V, uint32_t *__restrict__ succ, uint64_t *__restrict__ succ_base) {
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
    succ_base[x] = out == NONE32 ? ~0ull : ((far >> 32) << 32) | out;
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
// and acyclic (the usual case): one walk per list head measures the list
// and picks the copy to keep; a second walk writes each kept unitig's nodes
// and bases in order.  No per-strand-node ranking state is written.
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

template <class K>
__global__ __launch_bounds__(WALK_BLOCK) void k_fast_measure(const uint32_t *__restrict__ succ, uint64_t n,
                                                             const uint64_t *__restrict__ node_keys, int k,
                                                             uint32_t cap, uint32_t *__restrict__ is_head,
                                                             uint32_t *__restrict__ len_at_head,
                                                             uint8_t *__restrict__ hstrand, uint32_t *covered,
                                                             uint32_t *too_long) {
  __shared__ uint32_t s_q[WALK_WARPS][WALK_CHUNK];
  __shared__ uint32_t s_next[WALK_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t chunks = (n + WALK_CHUNK - 1) / WALK_CHUNK;
  uint32_t cov = 0, lng = 0;
  for (uint64_t c = (uint64_t)blockIdx.x * WALK_WARPS + w; c < chunks; c += (uint64_t)gridDim.x * WALK_WARPS) {
    const uint32_t cnt = queue_heads(c * WALK_CHUNK, n, s_q[w], [&](uint64_t x) { return succ[x ^ 1] == NONE32; });
    if (lane == 0) s_next[w] = 0;
    __syncwarp();
    uint32_t head = NONE32, y = 0, L = 0;
    for (;;) {
      if (head == NONE32) {
        const uint32_t qi = atomicAdd(&s_next[w], 1u);
        if (qi >= cnt) break;
        head = s_q[w][qi];
        y = head;
        L = 1;
      }
      const uint32_t ny = succ[y];
      if (ny != NONE32 && L < cap) {
        y = ny;
        L++;
        continue;
      }
      if (ny != NONE32) {
        lng++;
      } else if (KeyOps<K>::less(strand_kmer<K>(node_keys, head, k), strand_kmer<K>(node_keys, y ^ 1u, k))) {
        // the mirror copy starts at the tail on the other strand; the copy
        // whose first k-mer is smaller spells the smaller string
        const uint32_t v = head >> 1;
        is_head[v] = 1;
        len_at_head[v] = L;
        hstrand[v] = (uint8_t)(head & 1u);
        cov += 2 * L;
      }
      head = NONE32;
    }
    __syncwarp();
  }
  cov = __reduce_add_sync(0xffffffffu, cov);
  lng = __reduce_add_sync(0xffffffffu, lng);
  if (lane == 0) {
    if (cov) atomicAdd(covered, cov);
    if (lng) atomicAdd(too_long, lng);
  }
}

// Measuring with half the walking: both walkers of a unitig (its two list
// heads, one per mirrored copy) walk towards each other and stop where they
// meet.  A walker at strand-node y loads its successor word succ[y]; if the
// other walker has marked it (bit 31, with the other walker's head in the
// low bits) the node is the other's and the walk stops; else the walker
// marks the word the other walker would load at this node, succ[y ^ 1], and
// goes on.  Plain loads and stores: two walkers arriving together may both
// take a few nodes, which the pairing step measures.  hrec[x] = (nodes
// walker x took, its last strand-node, the other walker's head).  The
// successor words are spoiled for anything but this walk (the list heads are
// read from succ_base, which stays intact).
constexpr uint32_t MARK = 0x80000000u;

__global__ __launch_bounds__(WALK_BLOCK) void k_mark_measure(uint32_t *__restrict__ succ,
                                                             const uint64_t *__restrict__ succ_base, uint64_t n,
                                                             uint32_t cap, uint4 *__restrict__ hrec,
                                                             uint32_t *too_long) {
  __shared__ uint32_t s_q[WALK_WARPS][WALK_CHUNK];
  __shared__ uint32_t s_next[WALK_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t chunks = (n + WALK_CHUNK - 1) / WALK_CHUNK;
  uint32_t lng = 0;
  for (uint64_t c = (uint64_t)blockIdx.x * WALK_WARPS + w; c < chunks; c += (uint64_t)gridDim.x * WALK_WARPS) {
    const uint32_t cnt =
        queue_heads(c * WALK_CHUNK, n, s_q[w], [&](uint64_t x) { return succ_base[x ^ 1] == ~0ull; });
    if (lane == 0) s_next[w] = 0;
    __syncwarp();
    for (;;) {
      const uint32_t qi = atomicAdd(&s_next[w], 1u);
      if (qi >= cnt) break;
      const uint32_t x = s_q[w][qi];
      uint32_t y = x, d = 0, last = NONE32, partner = NONE32;
      for (;;) {
        const uint32_t nx = __ldcg(succ + y);  // from L2: another SM's mark may be there
        if (nx != NONE32 && (nx & MARK)) {
          partner = nx & ~MARK;
          break;
        }
        __stcg(succ + (y ^ 1u), MARK | x);
        d++;
        last = y;
        if (nx == NONE32) {
          partner = y ^ 1u;
          break;
        }
        if (d >= cap) {
          lng++;
          break;
        }
        y = nx;
      }
      hrec[x] = make_uint4(d, last, partner, 0u);
    }
    __syncwarp();
  }
  lng = __reduce_add_sync(0xffffffffu, lng);
  if (lane == 0 && lng) atomicAdd(too_long, lng);
}

// Per pair of walkers (handled by the smaller head): the unitig's length
// L = d_a + d_b - o, o the nodes both took (found by stepping from the
// second walker's last node, read on the first walker's strands, to the
// first walker's last node); the copy kept (the one whose first k-mer is
// smaller) and its first node's tables, as k_fast_measure writes them.
template <class K>
__global__ void k_mark_pair(const uint64_t *__restrict__ succ_base, uint64_t n, const uint4 *__restrict__ hrec,
                            const uint64_t *__restrict__ node_keys, int k, uint32_t cap,
                            uint32_t *__restrict__ is_head, uint32_t *__restrict__ len_at_head,
                            uint8_t *__restrict__ hstrand, unsigned long long *covered, uint32_t *err) {
  unsigned long long cov = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (succ_base[i ^ 1] != ~0ull) continue;  // not a list head
    const uint32_t x = (uint32_t)i;
    const uint4 ra = hrec[x];
    const uint32_t p = ra.z;
    if (p >= n || p == x) {
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    if (x > p) continue;
    const uint4 rb = hrec[p];
    if (rb.z != x) {
      atomicOr(err, ERR_INTERNAL);
      continue;
    }
    uint32_t o = 0;
    if (ra.x > 0 && rb.x > 0 && (uint32_t)succ_base[ra.y] != (rb.y ^ 1u)) {
      // the walks overlap: step from b's last node (on a's strands) to a's last
      uint32_t y = rb.y ^ 1u, steps = 0;
      while (y != ra.y && steps <= cap) {
        y = (uint32_t)succ_base[y];
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
    is_head[h] = 1;
    len_at_head[h] = L;
    hstrand[h] = (uint8_t)(kept & 1u);
    cov += L;
  }
  cov = __reduce_add_sync(0xffffffffu, (unsigned)cov);
  if ((threadIdx.x & 31) == 0 && cov) atomicAdd(covered, cov);
}

// The successor words again, from succ_base (after a measuring walk spoiled them).
__global__ void k_restore_succ(const uint64_t *__restrict__ succ_base, uint64_t n, uint32_t *__restrict__ succ) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = succ_base[x];
    succ[x] = b == ~0ull ? NONE32 : (uint32_t)b;
  }
}

// The first node of every kept unitig: its tables, node entry and first
// k-mer, and where its walk continues (walk[u] = succ_base of the first
// strand-node: the second one and the base it appends, or all ones).
template <class K>
__global__ void k_fast_heads(const uint64_t *__restrict__ succ_base, const uint32_t *__restrict__ is_head,
                             const uint8_t *__restrict__ hstrand, const uint64_t *__restrict__ uidx,
                             const uint64_t *__restrict__ off_by_v, const uint64_t *__restrict__ node_keys,
                             uint64_t V, uint64_t U, int k, uint64_t *__restrict__ nodes_out, char *__restrict__ seq,
                             uint64_t *__restrict__ node_off, uint64_t *__restrict__ seq_off,
                             uint8_t *__restrict__ circular, uint64_t *__restrict__ walk) {
  const char *acgt = "ACGT";
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= V; v += (uint64_t)gridDim.x * blockDim.x) {
    if (v == V) {
      node_off[U] = V;
      seq_off[U] = V + U * (uint64_t)(k - 1);
      continue;
    }
    if (!is_head[v]) continue;
    const uint64_t u = uidx[v], off = off_by_v[v], so = off + u * (uint64_t)(k - 1);
    const uint32_t y = 2 * (uint32_t)v + hstrand[v];
    node_off[u] = off;
    seq_off[u] = so;
    circular[u] = 0;
    nodes_out[off] = y;  // (node ID << 1) | strand
    const K km = strand_kmer<K>(node_keys, y, k);
    for (int j = 0; j < k; j++) seq[so + j] = acgt[KeyOps<K>::digit(km, 2 * (k - 1 - j), 2)];
    walk[u] = succ_base[y];
  }
}

// The rest of every kept unitig: lanes take unitigs in turn (per-warp
// chunks, a shared-memory counter) and walk them, writing each node's entry
// and the base its arc appends; only the successor words are loaded at random.
__global__ __launch_bounds__(WALK_BLOCK) void k_fast_walk(const uint64_t *__restrict__ succ_base,
                                                          const uint64_t *__restrict__ walk,
                                                          const uint64_t *__restrict__ node_off,
                                                          const uint64_t *__restrict__ seq_off, uint64_t U, int k,
                                                          uint64_t *__restrict__ nodes_out, char *__restrict__ seq) {
  __shared__ uint32_t s_next[WALK_WARPS];
  const char *acgt = "ACGT";
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t chunks = (U + WALK_CHUNK - 1) / WALK_CHUNK;
  for (uint64_t c = (uint64_t)blockIdx.x * WALK_WARPS + w; c < chunks; c += (uint64_t)gridDim.x * WALK_WARPS) {
    const uint64_t u0 = c * WALK_CHUNK;
    const uint32_t cnt = (uint32_t)min((uint64_t)WALK_CHUNK, U - u0);
    if (lane == 0) s_next[w] = 0;
    __syncwarp();
    bool busy = false;
    uint64_t nb = 0, pos = 0, spos = 0;
    for (;;) {
      if (!busy) {
        const uint32_t qi = atomicAdd(&s_next[w], 1u);
        if (qi >= cnt) break;
        const uint64_t u = u0 + qi;
        nb = walk[u];
        if (nb == ~0ull) continue;  // a single node
        pos = node_off[u] + 1;
        spos = seq_off[u] + k;
        busy = true;
      }
      const uint32_t y = (uint32_t)nb;
      nodes_out[pos++] = y;
      seq[spos++] = acgt[nb >> 32];
      nb = succ_base[y];
      busy = nb != ~0ull;
    }
    __syncwarp();
  }
}

// enough warps to fill the device, at most one per chunk
static unsigned walk_grid(const dbg_ctx *ctx, uint64_t n) {
  const uint64_t chunks = (n + WALK_CHUNK - 1) / WALK_CHUNK;
  const uint64_t blocks = (chunks + WALK_WARPS - 1) / WALK_WARPS;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)std::max(1, ctx->num_sms) * 6));
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
    DBG_TRY(alloc_buf(ctx, link_node, n1 * 4));
    DBG_TRY(alloc_buf(ctx, link_edge, n1 * 8));
    DBG_TRY(alloc_buf(ctx, succ, n1 * 4));
    DBG_TRY(alloc_buf(ctx, word, n1 * 8));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 16.0 * V + (double)E2 * 10 + 8.0 * V * g->key_words + 12.0 * n,
               k_side_links<K><<<grid_of(V), 256, 0, s>>>(g->row_ptr.as<uint64_t>(), g->adj_nbr.as<uint32_t>(),
                                                          g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(),
                                                          g->orient.as<uint8_t>(), g->node_keys.as<uint64_t>(), V, k,
                                                          literal, link_node.as<uint32_t>(), link_edge.as<uint64_t>()));
    // succ_base goes to the ranking words' buffer (free until the general path)
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 12.0 * n + 8.0 * n + 12.0 * n,
               k_successors<<<grid_of(n), 256, 0, s>>>(link_node.as<uint32_t>(), link_edge.as<uint64_t>(), V,
                                                       succ.as<uint32_t>(), word.as<uint64_t>()));
    link_node.release();
    link_edge.release();
    // ---- fast path: short acyclic lists only ----
    {
      DevBuf f_is_head, f_len, f_strand, f_uidx, f_off;
      DBG_TRY(alloc_buf(ctx, f_is_head, V1 * 4));
      DBG_TRY(alloc_buf(ctx, f_len, V1 * 4));
      DBG_TRY(alloc_buf(ctx, f_strand, V1));
      DBG_CUDA_TRY(cudaMemsetAsync(f_is_head.p, 0, V1 * 4, s));
      DBG_CUDA_TRY(cudaMemsetAsync(f_len.p, 0, V1 * 4, s));
      // the two walkers of each unitig meet half way (k_mark_measure), then
      // each pair gives its unitig's length and kept copy (k_mark_pair)
      DevBuf hrec;
      DBG_TRY(alloc_buf(ctx, hrec, n1 * sizeof(uint4)));
      DBG_CUDA_TRY(cudaMemsetAsync(ctx->d_counters + 10, 0, 4 * sizeof(uint32_t), s));
      DBG_LAUNCH(ctx, ST_COMPACT_RANK, 4.0 * n + 24.0 * V,
                 k_mark_measure<<<walk_grid(ctx, n), WALK_BLOCK, 0, s>>>(succ.as<uint32_t>(), word.as<uint64_t>(),
                                                                         n, kWalkCap, hrec.as<uint4>(),
                                                                         ctx->d_counters + 11));
      DBG_CUDA_TRY(cudaGetLastError());
      uint32_t too_long = 0;
      DBG_TRY(read_small(ctx, ctx->d_counters + 11, sizeof(uint32_t), &too_long));
      uint64_t covered = 0;
      if (too_long == 0) {
        DBG_LAUNCH(ctx, ST_COMPACT_RANK, 8.0 * n + 32.0 * V,
                   k_mark_pair<K><<<grid_of(n), 256, 0, s>>>(word.as<uint64_t>(), n, hrec.as<uint4>(),
                                                             g->node_keys.as<uint64_t>(), k, kWalkCap,
                                                             f_is_head.as<uint32_t>(), f_len.as<uint32_t>(),
                                                             f_strand.as<uint8_t>(),
                                                             reinterpret_cast<unsigned long long *>(ctx->d_counters + 12),
                                                             ctx->d_err));
        DBG_CUDA_TRY(cudaGetLastError());
        DBG_TRY(read_small(ctx, ctx->d_counters + 12, sizeof(uint64_t), &covered));
        DBG_TRY(check_device_error(ctx));
      }
      hrec.release();
      if (too_long == 0 && covered == V) {
        DBG_TRY(alloc_buf(ctx, f_uidx, (V + 1) * 8));
        DBG_TRY(alloc_buf(ctx, f_off, (V + 1) * 8));
        uint32_t U32 = 0, total = 0;
        DBG_TRY(scan_excl(ctx, f_is_head.as<uint32_t>(), V, f_uidx.as<uint64_t>(), &U32));
        DBG_TRY(scan_excl(ctx, f_len.as<uint32_t>(), V, f_off.as<uint64_t>(), &total));
        if (total != V) {
          set_error("unitigs hold %u nodes, expected %llu", total, (unsigned long long)V);
          return DBG_EINTERNAL;
        }
        const uint64_t Uf = U32;
        u->count = Uf;
        DBG_TRY(alloc_buf(ctx, u->node_off, (Uf + 1) * 8));
        DBG_TRY(alloc_buf(ctx, u->seq_off, (Uf + 1) * 8));
        DBG_TRY(alloc_buf(ctx, u->circular, std::max<uint64_t>(1, Uf)));
        DBG_TRY(alloc_buf(ctx, u->nodes, V1 * 8));
        u->total_bases = V + Uf * (uint64_t)(k - 1);
        DBG_TRY(alloc_buf(ctx, u->seq, std::max<uint64_t>(1, u->total_bases)));
        DevBuf walk;
        DBG_TRY(alloc_buf(ctx, walk, std::max<uint64_t>(1, Uf) * 8));
        DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, (double)V * (4 + 1) + (double)Uf * (16 + 8 + 8 * g->key_words + 8 + 25 + k),
                   k_fast_heads<K><<<grid_of(V + 1), 256, 0, s>>>(
                       word.as<uint64_t>(), f_is_head.as<uint32_t>(), f_strand.as<uint8_t>(), f_uidx.as<uint64_t>(),
                       f_off.as<uint64_t>(), g->node_keys.as<uint64_t>(), V, Uf, k, u->nodes.as<uint64_t>(),
                       u->seq.as<char>(), u->node_off.as<uint64_t>(), u->seq_off.as<uint64_t>(),
                       u->circular.as<uint8_t>(), walk.as<uint64_t>()));
        if (Uf > 0)
          DBG_LAUNCH(ctx, ST_COMPACT_OUTPUT, (double)(V - Uf) * (8 + 8 + 1) + (double)Uf * 24,
                     k_fast_walk<<<walk_grid(ctx, Uf), WALK_BLOCK, 0, s>>>(
                         word.as<uint64_t>(), walk.as<uint64_t>(), u->node_off.as<uint64_t>(),
                         u->seq_off.as<uint64_t>(), Uf, k, u->nodes.as<uint64_t>(), u->seq.as<char>()));
        DBG_CUDA_TRY(cudaGetLastError());
        DBG_CUDA_TRY(cudaStreamSynchronize(s));
        return check_device_error(ctx);
      }
    }
    // ---- general path: long lists or cycles present ----
    // (the measuring walk marked the successor words: rebuild them)
    DBG_LAUNCH(ctx, ST_COMPACT_RANK, 12.0 * n,
               k_restore_succ<<<grid_of(n), 256, 0, s>>>(word.as<uint64_t>(), n, succ.as<uint32_t>()));
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
    DBG_TRY(alloc_buf(ctx, word, n * 8));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 16.0 * V + 20.0 * g->num_edges + 8.0 * V * g->key_words + 12.0 * n,
               k_side_links<K><<<grid_of(V), 256, 0, s>>>(g->row_ptr.as<uint64_t>(), g->adj_nbr.as<uint32_t>(),
                                                          g->adj_edge.as<uint32_t>(), g->adj_role.as<uint8_t>(),
                                                          g->orient.as<uint8_t>(), g->node_keys.as<uint64_t>(), V, k,
                                                          false, link_node.as<uint32_t>(), link_edge.as<uint64_t>()));
    DBG_LAUNCH(ctx, ST_COMPACT_LINKS, 32.0 * n,
               k_successors<<<grid_of(n), 256, 0, s>>>(link_node.as<uint32_t>(), link_edge.as<uint64_t>(), V,
                                                       succ.as<uint32_t>(), word.as<uint64_t>()));
    DBG_CUDA_TRY(cudaGetLastError());
  }
  word.release();
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

/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU restatement of the bi-directed de Bruijn graph of
 * Kundeti et al., "Efficient Parallel and Out of Core Algorithms for
 * Constructing Large Bi-directed de Bruijn Graphs" (arXiv 1003.1940).
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library; the GPU library never does,
 * and this file shares no code, header or table with it.
 *
 * What it computes is the DEFINITION, not the paper's sort-based method:
 *
 *   nodes  (Section 2, "Preliminaries"): every k-molecule of the reads, named
 *          by its canonical k-mer, the smaller of a k-mer and its reverse
 *          complement in the order A < C < G < T.
 *   edges  (Section 2): for every pair of consecutive k-mers x, y of a read,
 *          one bi-directed edge between the molecules of x and y; the arrow
 *          head at a molecule is "positive" (o = 0) when the k-mer read there
 *          is the canonical one and "negative" (o = 1) otherwise.  The same
 *          edge read from the other end is (y^, x^, not o2, not o1); the
 *          oracle names each edge by the smaller of those two tuples and
 *          counts how often it occurs over the forward reads.
 *   adjacency (Section 3, STEP-4): per node, its edge ends in edge order.
 *   unitigs (Section 6): maximal chains of edges whose two end sides both
 *          have exactly one edge end, traced by walking the chain.
 *
 * Readings taken where the paper is silent or inconsistent:
 *   - multiplicities count the forward reads only (counting R* = R u rev(R)
 *     of Section 3 would double every count);
 *   - the alphabet order is A < C < G < T (Fig. 2 names GGA, not TCC, as the
 *     positive strand of its molecule);
 *   - a read of length exactly k contributes its node but no edge;
 *   - unitigs include singletons and two-node chains; the "at least three
 *     nodes" filter of Section 6.1 is not applied;
 *   - a circular chain starts at its smallest node, positive strand.
 *
 * Encoding: base codes A=0 C=1 G=2 T=3; an m-mer is the integer whose most
 * significant 2-bit digit is its first base, held in an unsigned __int128.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EINTERNAL = 3 };

/* ------------------------------------------------------------------ */
/* strings of bases (Section 2)                                        */
/* ------------------------------------------------------------------ */

static int base_code(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
  }
}

static const char BASE_CHAR[4] = {'A', 'C', 'G', 'T'};

/* integer value of the m-mer s[0..m), first base most significant */
static u128 mer_value(const char *s, int m) {
  u128 v = 0;
  for (int i = 0; i < m; i++) v = (v << 2) | (u128)base_code(s[i]);
  return v;
}

/* base i (0 = first) of an m-mer value */
static int mer_base(u128 v, int m, int i) { return (int)((v >> (2 * (m - 1 - i))) & 3); }

/* reverse complement (Section 2: AAGTA -> TACTT): reverse the string, then
 * replace every base by its complement A<->T, C<->G (code c -> 3 - c). */
static u128 mer_revcomp(u128 v, int m) {
  u128 r = 0;
  for (int i = m - 1; i >= 0; i--) r = (r << 2) | (u128)(3 - mer_base(v, m, i));
  return r;
}

/* canonical k-mer (Section 2): the lexicographically smaller of s and its
 * reverse complement; for equal-length strings over A<C<G<T the
 * lexicographic order is the integer order of the values. */
static u128 mer_canonical(u128 v, int m) {
  u128 r = mer_revcomp(v, m);
  return r < v ? r : v;
}

static void mer_spell(u128 v, int m, char *out) {
  for (int i = 0; i < m; i++) out[i] = BASE_CHAR[mer_base(v, m, i)];
}

/* ------------------------------------------------------------------ */
/* a plain open-addressing table: key (two 128-bit values + 2 bits)    */
/* ------------------------------------------------------------------ */

typedef struct {
  u128 a, b;       /* node keys, or (k+1)-mer in a with b = 0 */
  uint8_t tag;     /* orientation bits, 0..3 */
  uint8_t used;
  uint64_t count;
} slot_t;

typedef struct {
  slot_t *slots;
  uint64_t cap, size;
} table_t;

static uint64_t mix64(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}

static uint64_t slot_hash(u128 a, u128 b, uint8_t tag) {
  uint64_t h = mix64((uint64_t)a ^ 0x9e3779b97f4a7c15ULL);
  h = mix64(h ^ (uint64_t)(a >> 64));
  h = mix64(h ^ (uint64_t)b);
  h = mix64(h ^ (uint64_t)(b >> 64));
  return mix64(h ^ tag);
}

static int table_init(table_t *t, uint64_t expect) {
  uint64_t cap = 64;
  while (cap < 2 * expect + 64) cap <<= 1;
  t->slots = (slot_t *)calloc(cap, sizeof(slot_t));
  t->cap = cap;
  t->size = 0;
  return t->slots ? ORC_OK : ORC_ENOMEM;
}

static int table_grow(table_t *t);

/* returns the slot holding (a, b, tag), inserting it with count 0 */
static slot_t *table_find(table_t *t, u128 a, u128 b, uint8_t tag, int insert) {
  if (insert && 2 * (t->size + 1) > t->cap && table_grow(t) != ORC_OK) return NULL;
  uint64_t i = slot_hash(a, b, tag) & (t->cap - 1);
  for (;;) {
    slot_t *s = &t->slots[i];
    if (!s->used) {
      if (!insert) return NULL;
      s->used = 1; s->a = a; s->b = b; s->tag = tag; s->count = 0;
      t->size++;
      return s;
    }
    if (s->a == a && s->b == b && s->tag == tag) return s;
    i = (i + 1) & (t->cap - 1);
  }
}

static int table_grow(table_t *t) {
  table_t bigger;
  if (table_init(&bigger, t->cap) != ORC_OK) return ORC_ENOMEM;
  for (uint64_t i = 0; i < t->cap; i++) {
    slot_t *s = &t->slots[i];
    if (!s->used) continue;
    slot_t *d = table_find(&bigger, s->a, s->b, s->tag, 1);
    d->count = s->count;
  }
  free(t->slots);
  *t = bigger;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* graph construction by the definition (Section 2)                    */
/* ------------------------------------------------------------------ */

typedef struct {
  uint32_t k;
  uint64_t n_nodes, n_edges;
  uint64_t *node_keys;  /* 2 words per node: high, low 64 bits of the canonical k-mer */
  uint64_t *edge_keys;  /* 2 words per edge: canonical (k+1)-mer spelled by the edge */
  uint32_t *src, *dst;  /* node IDs (rank of the node key), src <= dst */
  uint8_t *orient;      /* (o1 << 1) | o2, o = 1 for the negative strand */
  uint32_t *mult;       /* occurrences over the forward reads (saturating) */
  uint64_t *row_ptr;    /* n_nodes + 1 */
  uint32_t *adj_nbr, *adj_edge;
  uint8_t *adj_role;    /* 0: this node is the edge's src end, 1: its dst end */
  uint32_t flags;       /* bit 0: some multiplicity saturated at 2^32 - 1 */
} orc_graph;

typedef struct { u128 src, dst; uint8_t o1, o2; uint64_t count; u128 key; } edge_rec;

static int cmp_u128(u128 a, u128 b) { return a < b ? -1 : (a > b ? 1 : 0); }

static int cmp_node(const void *pa, const void *pb) {
  return cmp_u128(*(const u128 *)pa, *(const u128 *)pb);
}

static int cmp_edge_by_key(const void *pa, const void *pb) {
  return cmp_u128(((const edge_rec *)pa)->key, ((const edge_rec *)pb)->key);
}

/* lexicographic order of edge tuples (src, dst, o1, o2) */
static int tuple_less(u128 s1, u128 d1, int a1, int b1, u128 s2, u128 d2, int a2, int b2) {
  if (s1 != s2) return s1 < s2;
  if (d1 != d2) return d1 < d2;
  if (a1 != a2) return a1 < a2;
  return b1 < b2;
}

static int64_t node_rank(const u128 *nodes, uint64_t n, u128 key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (nodes[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && nodes[lo] == key) ? (int64_t)lo : -1;
}

void orc_graph_free(orc_graph *g) {
  if (!g) return;
  free(g->node_keys); free(g->edge_keys); free(g->src); free(g->dst);
  free(g->orient); free(g->mult); free(g->row_ptr);
  free(g->adj_nbr); free(g->adj_edge); free(g->adj_role);
  free(g);
}

int orc_build(const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k, orc_graph **out) {
  if (!out) return ORC_EINVAL;
  *out = NULL;
  if (k < 1 || k > 63 || (k % 2) == 0) return ORC_EINVAL;  /* k odd (Section 2) */
  if (n > 0 && (!reads || !lengths)) return ORC_EINVAL;

  uint64_t total = 0;
  for (uint64_t r = 0; r < n; r++) total += lengths[r];
  for (uint64_t i = 0; i < total; i++)
    if (base_code(reads[i]) < 0) return ORC_EINVAL;  /* alphabet {A,C,G,T} */

  table_t nodes_t, edges_t;
  if (table_init(&nodes_t, 1024) != ORC_OK) return ORC_ENOMEM;
  if (table_init(&edges_t, 1024) != ORC_OK) { free(nodes_t.slots); return ORC_ENOMEM; }
  int K = (int)k;
  int rc = ORC_OK;

  const char *read = reads;
  for (uint64_t r = 0; r < n && rc == ORC_OK; r++) {
    int64_t L = lengths[r];
    /* every k-mer of the read is a node (k-spectrum, Section 2) */
    for (int64_t j = 0; j + K <= L; j++) {
      u128 x = mer_canonical(mer_value(read + j, K), K);
      if (!table_find(&nodes_t, x, 0, 0, 1)) { rc = ORC_ENOMEM; break; }
    }
    /* every two consecutive k-mers give one bi-directed edge */
    for (int64_t j = 0; j + K + 1 <= L && rc == ORC_OK; j++) {
      u128 x = mer_value(read + j, K);
      u128 y = mer_value(read + j + 1, K);
      u128 xh = mer_canonical(x, K), yh = mer_canonical(y, K);
      int o1 = (x != xh), o2 = (y != yh);
      /* the same edge seen from its other end: (y^, x^, not o2, not o1) */
      u128 s = xh, d = yh;
      int a = o1, b = o2;
      if (tuple_less(yh, xh, !o2, !o1, xh, yh, o1, o2)) { s = yh; d = xh; a = !o2; b = !o1; }
      slot_t *e = table_find(&edges_t, s, d, (uint8_t)((a << 1) | b), 1);
      if (!e) { rc = ORC_ENOMEM; break; }
      e->count++;
    }
    read += L;
  }

  orc_graph *g = NULL;
  u128 *nodes = NULL;
  edge_rec *edges = NULL;
  if (rc == ORC_OK) {
    g = (orc_graph *)calloc(1, sizeof(orc_graph));
    nodes = (u128 *)malloc((nodes_t.size + 1) * sizeof(u128));
    edges = (edge_rec *)malloc((edges_t.size + 1) * sizeof(edge_rec));
    if (!g || !nodes || !edges) rc = ORC_ENOMEM;
  }
  if (rc == ORC_OK) {
    g->k = k;
    uint64_t nv = 0, ne = 0;
    for (uint64_t i = 0; i < nodes_t.cap; i++)
      if (nodes_t.slots[i].used) nodes[nv++] = nodes_t.slots[i].a;
    for (uint64_t i = 0; i < edges_t.cap; i++) {
      slot_t *s = &edges_t.slots[i];
      if (!s->used) continue;
      edge_rec *e = &edges[ne++];
      e->src = s->a; e->dst = s->b; e->o1 = s->tag >> 1; e->o2 = s->tag & 1; e->count = s->count;
      /* the edge spells the (k+1)-mer z = x o last(y) with x, y the k-mers
       * read at its ends; edges are listed by min(z, revcomp z) */
      u128 x = e->o1 ? mer_revcomp(e->src, K) : e->src;
      u128 y = e->o2 ? mer_revcomp(e->dst, K) : e->dst;
      if ((x & ((((u128)1) << (2 * (K - 1))) - 1)) != (y >> 2)) { rc = ORC_EINTERNAL; break; }
      u128 z = (x << 2) | (y & 3);
      e->key = mer_canonical(z, K + 1);
    }
    g->n_nodes = nv;
    g->n_edges = ne;
  }
  free(nodes_t.slots);
  free(edges_t.slots);

  if (rc == ORC_OK) {
    uint64_t nv = g->n_nodes, ne = g->n_edges;
    qsort(nodes, nv, sizeof(u128), cmp_node);
    qsort(edges, ne, sizeof(edge_rec), cmp_edge_by_key);
    g->node_keys = (uint64_t *)malloc((2 * nv + 1) * sizeof(uint64_t));
    g->edge_keys = (uint64_t *)malloc((2 * ne + 1) * sizeof(uint64_t));
    g->src = (uint32_t *)malloc((ne + 1) * sizeof(uint32_t));
    g->dst = (uint32_t *)malloc((ne + 1) * sizeof(uint32_t));
    g->orient = (uint8_t *)malloc(ne + 1);
    g->mult = (uint32_t *)malloc((ne + 1) * sizeof(uint32_t));
    g->row_ptr = (uint64_t *)calloc(nv + 1, sizeof(uint64_t));
    g->adj_nbr = (uint32_t *)malloc((2 * ne + 1) * sizeof(uint32_t));
    g->adj_edge = (uint32_t *)malloc((2 * ne + 1) * sizeof(uint32_t));
    g->adj_role = (uint8_t *)malloc(2 * ne + 1);
    if (!g->node_keys || !g->edge_keys || !g->src || !g->dst || !g->orient || !g->mult ||
        !g->row_ptr || !g->adj_nbr || !g->adj_edge || !g->adj_role)
      rc = ORC_ENOMEM;
  }
  if (rc == ORC_OK) {
    uint64_t nv = g->n_nodes, ne = g->n_edges;
    for (uint64_t v = 0; v < nv; v++) {
      g->node_keys[2 * v] = (uint64_t)(nodes[v] >> 64);
      g->node_keys[2 * v + 1] = (uint64_t)nodes[v];
    }
    for (uint64_t i = 0; i < ne && rc == ORC_OK; i++) {
      edge_rec *e = &edges[i];
      int64_t s = node_rank(nodes, nv, e->src), d = node_rank(nodes, nv, e->dst);
      if (s < 0 || d < 0) { rc = ORC_EINTERNAL; break; }
      g->edge_keys[2 * i] = (uint64_t)(e->key >> 64);
      g->edge_keys[2 * i + 1] = (uint64_t)e->key;
      g->src[i] = (uint32_t)s;
      g->dst[i] = (uint32_t)d;
      g->orient[i] = (uint8_t)((e->o1 << 1) | e->o2);
      if (e->count > 0xffffffffULL) { g->mult[i] = 0xffffffffU; g->flags |= 1; }
      else g->mult[i] = (uint32_t)e->count;
      g->row_ptr[s + 1]++;
      g->row_ptr[d + 1]++;
    }
    /* adjacency (STEP-4): each node's row lists its edge ends in edge order */
    for (uint64_t v = 0; v < nv; v++) g->row_ptr[v + 1] += g->row_ptr[v];
    uint64_t *fill = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
    if (!fill) rc = ORC_ENOMEM;
    for (uint64_t v = 0; rc == ORC_OK && v < nv; v++) fill[v] = g->row_ptr[v];
    for (uint64_t i = 0; rc == ORC_OK && i < ne; i++) {
      uint32_t s = g->src[i], d = g->dst[i];
      uint64_t p = fill[s]++;
      g->adj_nbr[p] = d; g->adj_edge[p] = (uint32_t)i; g->adj_role[p] = 0;
      p = fill[d]++;
      g->adj_nbr[p] = s; g->adj_edge[p] = (uint32_t)i; g->adj_role[p] = 1;
    }
    free(fill);
  }
  free(nodes);
  free(edges);
  if (rc != ORC_OK) { orc_graph_free(g); return rc; }
  *out = g;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* sampled multiplicities for inputs too large to build in full        */
/* ------------------------------------------------------------------ */

/* For each query (k+1)-mer, counts the positions of the forward reads whose
 * (k+1)-mer is the query or its reverse complement: the multiplicity of the
 * bi-directed edge that the query spells (Section 2).  Queries are given as
 * k+1 characters each, back to back. */
int orc_count_kplus1(const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k,
                     const char *queries, uint64_t nq, uint64_t *counts) {
  if (k < 1 || k > 63 || (k % 2) == 0 || (nq > 0 && (!queries || !counts))) return ORC_EINVAL;
  int M = (int)k + 1;
  table_t t;
  if (table_init(&t, nq) != ORC_OK) return ORC_ENOMEM;
  for (uint64_t q = 0; q < nq; q++) {
    for (int i = 0; i < M; i++)
      if (base_code(queries[q * M + i]) < 0) { free(t.slots); return ORC_EINVAL; }
    u128 z = mer_canonical(mer_value(queries + q * M, M), M);
    if (!table_find(&t, z, 0, 0, 1)) { free(t.slots); return ORC_ENOMEM; }
  }
  /* slide a (k+1)-base window along each read, keeping the window and its
   * reverse complement up to date one base at a time */
  u128 mask = (M == 64) ? ~(u128)0 : ((((u128)1) << (2 * M)) - 1);
  const char *read = reads;
  for (uint64_t r = 0; r < n; r++) {
    int64_t L = lengths[r];
    u128 fwd = 0, rev = 0;
    for (int64_t j = 0; j < L; j++) {
      int c = base_code(read[j]);
      if (c < 0) { free(t.slots); return ORC_EINVAL; }
      fwd = ((fwd << 2) | (u128)c) & mask;
      rev = (rev >> 2) | ((u128)(3 - c) << (2 * (M - 1)));
      if (j + 1 < M) continue;
      u128 z = rev < fwd ? rev : fwd;
      slot_t *s = table_find(&t, z, 0, 0, 0);
      if (s) s->count++;
    }
    read += L;
  }
  for (uint64_t q = 0; q < nq; q++) {
    u128 z = mer_canonical(mer_value(queries + q * M, M), M);
    counts[q] = table_find(&t, z, 0, 0, 0)->count;
  }
  free(t.slots);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* node multiplicities                                                   */
/* ------------------------------------------------------------------ */

static int cmp_slot_key(const void *pa, const void *pb) {
  return cmp_u128(((const slot_t *)pa)->a, ((const slot_t *)pb)->a);
}

/* For every node of orc_build -- the canonical k-mers of the forward reads
 * of length >= k (Section 2) -- the number of positions of the forward
 * reads whose k-mer is it or its reverse complement: STEP-2's counting
 * (Section 3) applied to k-mers, the table of k-mer occurrences that
 * VELVET's roadmap is drawn from (Section 7).  *keys receives 2 words
 * (high, low) per node in ascending order, *counts one count per node;
 * both are allocated here (free them with orc_free). */
int orc_node_mult(const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k, uint64_t *n_nodes,
                  uint64_t **keys, uint64_t **counts) {
  if (k < 1 || k > 63 || (k % 2) == 0 || !n_nodes || !keys || !counts) return ORC_EINVAL;
  const int K = (int)k;
  table_t t;
  if (table_init(&t, 1024) != ORC_OK) return ORC_ENOMEM;
  /* slide a k-base window along each read */
  u128 mask = (K == 64) ? ~(u128)0 : ((((u128)1) << (2 * K)) - 1);
  const char *read = reads;
  for (uint64_t r = 0; r < n; r++) {
    int64_t L = lengths[r];
    u128 fwd = 0, rev = 0;
    for (int64_t j = 0; j < L; j++) {
      int c = base_code(read[j]);
      if (c < 0) { free(t.slots); return ORC_EINVAL; }
      fwd = ((fwd << 2) | (u128)c) & mask;
      rev = (rev >> 2) | ((u128)(3 - c) << (2 * (K - 1)));
      if (j + 1 < K) continue;
      slot_t *sl = table_find(&t, rev < fwd ? rev : fwd, 0, 0, 1);
      if (!sl) { free(t.slots); return ORC_ENOMEM; }
      sl->count++;
    }
    read += L;
  }
  /* the occupied slots, in key order */
  uint64_t m = 0;
  for (uint64_t i = 0; i < t.cap; i++)
    if (t.slots[i].used) t.slots[m++] = t.slots[i];
  qsort(t.slots, m, sizeof(slot_t), cmp_slot_key);
  *keys = (uint64_t *)malloc((m ? m : 1) * 2 * sizeof(uint64_t));
  *counts = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
  if (!*keys || !*counts) {
    free(*keys); free(*counts); free(t.slots);
    return ORC_ENOMEM;
  }
  for (uint64_t i = 0; i < m; i++) {
    (*keys)[2 * i] = (uint64_t)(t.slots[i].a >> 64);
    (*keys)[2 * i + 1] = (uint64_t)t.slots[i].a;
    (*counts)[i] = t.slots[i].count;
  }
  *n_nodes = m;
  free(t.slots);
  return ORC_OK;
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------ */
/* the roadmap counts: distinct reads per node                          */
/* ------------------------------------------------------------------ */

/* For every node of orc_build (canonical k-mers of the forward reads of
 * length >= k, Section 2), the number of distinct reads that contain it on
 * either strand.  VELVET keeps the k-mers present in at least 2 reads, its
 * "roadmap" (Section 7).  Each read's canonical k-mers are collected,
 * sorted and deduplicated, and every distinct one counts the read once.
 * Outputs as orc_node_mult (free them with orc_free). */
int orc_node_reads(const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k, uint64_t *n_nodes,
                   uint64_t **keys, uint64_t **counts) {
  if (k < 1 || k > 63 || (k % 2) == 0 || !n_nodes || !keys || !counts) return ORC_EINVAL;
  const int K = (int)k;
  table_t t;
  if (table_init(&t, 1024) != ORC_OK) return ORC_ENOMEM;
  uint64_t cap = 0;
  u128 *mine = NULL;
  const char *read = reads;
  int rc = ORC_OK;
  for (uint64_t r = 0; r < n && rc == ORC_OK; r++) {
    int64_t L = lengths[r];
    uint64_t m = 0;
    if (L >= K) {
      if ((uint64_t)(L - K + 1) > cap) {
        cap = (uint64_t)(L - K + 1);
        free(mine);
        mine = (u128 *)malloc(cap * sizeof(u128));
        if (!mine) { rc = ORC_ENOMEM; break; }
      }
      for (int64_t j = 0; j + K <= L; j++) {
        for (int i = 0; i < K; i++)
          if (base_code(read[j + i]) < 0) { rc = ORC_EINVAL; break; }
        if (rc != ORC_OK) break;
        mine[m++] = mer_canonical(mer_value(read + j, K), K);
      }
    }
    if (rc != ORC_OK) break;
    /* the read's distinct canonical k-mers count it once each */
    qsort(mine, m, sizeof(u128), cmp_node);
    for (uint64_t i = 0; i < m; i++) {
      if (i > 0 && mine[i] == mine[i - 1]) continue;
      slot_t *sl = table_find(&t, mine[i], 0, 0, 1);
      if (!sl) { rc = ORC_ENOMEM; break; }
      sl->count++;
    }
    read += L;
  }
  free(mine);
  if (rc != ORC_OK) { free(t.slots); return rc; }
  uint64_t m = 0;
  for (uint64_t i = 0; i < t.cap; i++)
    if (t.slots[i].used) t.slots[m++] = t.slots[i];
  qsort(t.slots, m, sizeof(slot_t), cmp_slot_key);
  *keys = (uint64_t *)malloc((m ? m : 1) * 2 * sizeof(uint64_t));
  *counts = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
  if (!*keys || !*counts) {
    free(*keys); free(*counts); free(t.slots);
    return ORC_ENOMEM;
  }
  for (uint64_t i = 0; i < m; i++) {
    (*keys)[2 * i] = (uint64_t)(t.slots[i].a >> 64);
    (*keys)[2 * i + 1] = (uint64_t)t.slots[i].a;
    (*counts)[i] = t.slots[i].count;
  }
  *n_nodes = m;
  free(t.slots);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* one partition of the edges, for the multi-core CPU baseline          */
/* ------------------------------------------------------------------ */

/* The edges of orc_build (Section 2 definition) whose canonical (k+1)-mer
 * falls in partition `part` of `parts` (partitioned by a hash of that key),
 * counted over all reads: *distinct edges and their *instances.  Each of
 * `parts` processes scans every read and keeps only its own edges, so the
 * parts together do the edge counting of orc_build once. */
int orc_edges_in_partition(const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k, uint32_t part,
                           uint32_t parts, uint64_t *distinct, uint64_t *instances) {
  if (k < 1 || k > 63 || (k % 2) == 0 || parts == 0 || part >= parts || !distinct || !instances) return ORC_EINVAL;
  int K = (int)k, M = K + 1;
  table_t t;
  if (table_init(&t, 1024) != ORC_OK) return ORC_ENOMEM;
  u128 mask = (M == 64) ? ~(u128)0 : ((((u128)1) << (2 * M)) - 1);
  uint64_t inst = 0;
  const char *read = reads;
  for (uint64_t r = 0; r < n; r++) {
    int64_t L = lengths[r];
    u128 fwd = 0, rev = 0;
    for (int64_t j = 0; j < L; j++) {
      int c = base_code(read[j]);
      if (c < 0) { free(t.slots); return ORC_EINVAL; }
      fwd = ((fwd << 2) | (u128)c) & mask;
      rev = (rev >> 2) | ((u128)(3 - c) << (2 * (M - 1)));
      if (j + 1 < M) continue;
      u128 z = rev < fwd ? rev : fwd;
      if (mix64((uint64_t)z ^ mix64((uint64_t)(z >> 64))) % parts != part) continue;
      /* the edge of the k-mer pair ending at j, named as in orc_build */
      const int64_t j0 = j + 1 - M;
      u128 x = mer_value(read + j0, K), y = mer_value(read + j0 + 1, K);
      u128 xh = mer_canonical(x, K), yh = mer_canonical(y, K);
      int o1 = (x != xh), o2 = (y != yh);
      u128 s = xh, d = yh;
      int a = o1, b = o2;
      if (tuple_less(yh, xh, !o2, !o1, xh, yh, o1, o2)) { s = yh; d = xh; a = !o2; b = !o1; }
      slot_t *e = table_find(&t, s, d, (uint8_t)((a << 1) | b), 1);
      if (!e) { free(t.slots); return ORC_ENOMEM; }
      e->count++;
      inst++;
    }
    read += L;
  }
  *distinct = t.size;
  *instances = inst;
  free(t.slots);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* one key range of the graph, for inputs too large to build at once    */
/* ------------------------------------------------------------------ */

/* The slice of orc_build's graph whose keys lie in given ranges: the edges
 * (Section 2, named and counted exactly as orc_build does) whose canonical
 * (k+1)-mer key z satisfies elo <= z <= ehi, and the nodes (canonical k-mers
 * of the forward reads, Section 2) whose key x satisfies nlo <= x <= nhi.
 * Bounds are inclusive (high, low) word pairs.  An edge is listed with the
 * keys of its two end nodes instead of their IDs (a node's ID is its rank
 * among ALL nodes, which one slice does not see).  Edges come out by
 * ascending key, nodes ascending, so cutting the key spaces into ranges and
 * concatenating the slices in range order gives orc_build's node and edge
 * lists.  Every read is scanned; only keys in range are kept. */
typedef struct {
  uint64_t n_edges, n_nodes;
  uint64_t *edge_keys;  /* 2 words per edge: canonical (k+1)-mer */
  uint64_t *src_keys;   /* 2 words per edge: node key at the src end */
  uint64_t *dst_keys;   /* 2 words per edge: node key at the dst end */
  uint8_t *orient;      /* (o1 << 1) | o2 */
  uint64_t *mult;       /* occurrences over the forward reads */
  uint64_t *node_keys;  /* 2 words per node */
} orc_range;

void orc_range_free(orc_range *r) {
  if (!r) return;
  free(r->edge_keys); free(r->src_keys); free(r->dst_keys);
  free(r->orient); free(r->mult); free(r->node_keys);
  free(r);
}

static u128 words_u128(const uint64_t *w) { return ((u128)w[0] << 64) | w[1]; }

int orc_graph_range(const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k, const uint64_t *elo,
                    const uint64_t *ehi, const uint64_t *nlo, const uint64_t *nhi, orc_range **out) {
  if (!out || !elo || !ehi || !nlo || !nhi) return ORC_EINVAL;
  *out = NULL;
  if (k < 1 || k > 63 || (k % 2) == 0) return ORC_EINVAL;
  if (n > 0 && (!reads || !lengths)) return ORC_EINVAL;
  const int K = (int)k, M = K + 1;
  const u128 e0 = words_u128(elo), e1 = words_u128(ehi), n0 = words_u128(nlo), n1 = words_u128(nhi);
  table_t nodes_t, edges_t;
  if (table_init(&nodes_t, 1024) != ORC_OK) return ORC_ENOMEM;
  if (table_init(&edges_t, 1024) != ORC_OK) { free(nodes_t.slots); return ORC_ENOMEM; }
  int rc = ORC_OK;
  /* the k-base and (k+1)-base windows ending at base j, and their reverse
   * complements, updated one base at a time */
  const u128 kmask = ((((u128)1) << (2 * K)) - 1);
  const u128 mmask = (M == 64) ? ~(u128)0 : ((((u128)1) << (2 * M)) - 1);
  const char *read = reads;
  for (uint64_t r = 0; r < n && rc == ORC_OK; r++) {
    int64_t L = lengths[r];
    u128 kf = 0, kr = 0, mf = 0, mr = 0;
    for (int64_t j = 0; j < L; j++) {
      int c = base_code(read[j]);
      if (c < 0) { rc = ORC_EINVAL; break; }
      kf = ((kf << 2) | (u128)c) & kmask;
      kr = (kr >> 2) | ((u128)(3 - c) << (2 * (K - 1)));
      mf = ((mf << 2) | (u128)c) & mmask;
      mr = (mr >> 2) | ((u128)(3 - c) << (2 * (M - 1)));
      if (j + 1 >= K) {
        /* node: the canonical k-mer read[j-K+1 .. j] */
        u128 x = kr < kf ? kr : kf;
        if (x >= n0 && x <= n1 && !table_find(&nodes_t, x, 0, 0, 1)) { rc = ORC_ENOMEM; break; }
      }
      if (j + 1 >= M) {
        /* edge: the k-mer pair read[j-K .. j-1], read[j-K+1 .. j] */
        u128 z = mr < mf ? mr : mf;
        if (z < e0 || z > e1) continue;
        const int64_t j0 = j + 1 - M;
        u128 x = mer_value(read + j0, K), y = mer_value(read + j0 + 1, K);
        u128 xh = mer_canonical(x, K), yh = mer_canonical(y, K);
        int o1 = (x != xh), o2 = (y != yh);
        u128 s = xh, d = yh;
        int a = o1, b = o2;
        if (tuple_less(yh, xh, !o2, !o1, xh, yh, o1, o2)) { s = yh; d = xh; a = !o2; b = !o1; }
        slot_t *e = table_find(&edges_t, s, d, (uint8_t)((a << 1) | b), 1);
        if (!e) { rc = ORC_ENOMEM; break; }
        e->count++;
      }
    }
    read += L;
  }
  orc_range *res = NULL;
  edge_rec *edges = NULL;
  u128 *nodes = NULL;
  if (rc == ORC_OK) {
    res = (orc_range *)calloc(1, sizeof(orc_range));
    edges = (edge_rec *)malloc((edges_t.size + 1) * sizeof(edge_rec));
    nodes = (u128 *)malloc((nodes_t.size + 1) * sizeof(u128));
    if (!res || !edges || !nodes) rc = ORC_ENOMEM;
  }
  if (rc == ORC_OK) {
    uint64_t ne = 0, nv = 0;
    for (uint64_t i = 0; i < edges_t.cap && rc == ORC_OK; i++) {
      slot_t *s = &edges_t.slots[i];
      if (!s->used) continue;
      edge_rec *e = &edges[ne++];
      e->src = s->a; e->dst = s->b; e->o1 = s->tag >> 1; e->o2 = s->tag & 1; e->count = s->count;
      /* the key is the canonical form of the (k+1)-mer the edge spells */
      u128 x = e->o1 ? mer_revcomp(e->src, K) : e->src;
      u128 y = e->o2 ? mer_revcomp(e->dst, K) : e->dst;
      if ((x & ((((u128)1) << (2 * (K - 1))) - 1)) != (y >> 2)) { rc = ORC_EINTERNAL; break; }
      e->key = mer_canonical((x << 2) | (y & 3), M);
    }
    for (uint64_t i = 0; i < nodes_t.cap; i++)
      if (nodes_t.slots[i].used) nodes[nv++] = nodes_t.slots[i].a;
    res->n_edges = ne;
    res->n_nodes = nv;
  }
  free(nodes_t.slots);
  free(edges_t.slots);
  if (rc == ORC_OK) {
    uint64_t ne = res->n_edges, nv = res->n_nodes;
    qsort(edges, ne, sizeof(edge_rec), cmp_edge_by_key);
    qsort(nodes, nv, sizeof(u128), cmp_node);
    res->edge_keys = (uint64_t *)malloc((2 * ne + 1) * sizeof(uint64_t));
    res->src_keys = (uint64_t *)malloc((2 * ne + 1) * sizeof(uint64_t));
    res->dst_keys = (uint64_t *)malloc((2 * ne + 1) * sizeof(uint64_t));
    res->orient = (uint8_t *)malloc(ne + 1);
    res->mult = (uint64_t *)malloc((ne + 1) * sizeof(uint64_t));
    res->node_keys = (uint64_t *)malloc((2 * nv + 1) * sizeof(uint64_t));
    if (!res->edge_keys || !res->src_keys || !res->dst_keys || !res->orient || !res->mult || !res->node_keys)
      rc = ORC_ENOMEM;
    for (uint64_t i = 0; rc == ORC_OK && i < ne; i++) {
      const edge_rec *e = &edges[i];
      res->edge_keys[2 * i] = (uint64_t)(e->key >> 64); res->edge_keys[2 * i + 1] = (uint64_t)e->key;
      res->src_keys[2 * i] = (uint64_t)(e->src >> 64); res->src_keys[2 * i + 1] = (uint64_t)e->src;
      res->dst_keys[2 * i] = (uint64_t)(e->dst >> 64); res->dst_keys[2 * i + 1] = (uint64_t)e->dst;
      res->orient[i] = (uint8_t)((e->o1 << 1) | e->o2);
      res->mult[i] = e->count;
    }
    for (uint64_t v = 0; rc == ORC_OK && v < nv; v++) {
      res->node_keys[2 * v] = (uint64_t)(nodes[v] >> 64);
      res->node_keys[2 * v + 1] = (uint64_t)nodes[v];
    }
  }
  free(edges);
  free(nodes);
  if (rc != ORC_OK) { orc_range_free(res); return rc; }
  *out = res;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* chain compaction by walking the chains (Section 6)                   */
/* ------------------------------------------------------------------ */

/* Each node has two sides.  An edge end whose k-mer is read on the positive
 * strand and continues to the right of it sits on the node's right side:
 * the src end of (u, v, o1, o2) is on u's right side when o1 = 0 and on its
 * left side when o1 = 1; the dst end is on v's left side when o2 = 0 and on
 * its right side when o2 = 1.  An edge can be merged into a chain when its
 * two ends are on distinct nodes and each end's side carries no other edge
 * end; a walk through a node then enters by one side and leaves by the
 * other, which is the validity rule for bi-directed walks of Section 2. */
enum { SIDE_L = 0, SIDE_R = 1 };

typedef struct {
  uint64_t count;
  uint64_t *node_off;  /* count + 1 */
  uint64_t *nodes;     /* (node ID << 1) | strand, strand 1 = read as reverse complement */
  uint64_t *seq_off;   /* count + 1 */
  char *seq;           /* spelled chains, m + k - 1 bases each, no separators */
  uint8_t *circular;   /* 1 for a chain that closes on itself */
} orc_unitigs;

void orc_unitigs_free(orc_unitigs *u) {
  if (!u) return;
  free(u->node_off); free(u->nodes); free(u->seq_off); free(u->seq); free(u->circular);
  free(u);
}

typedef struct { int64_t node; int side; } link_t;  /* node -1: none */

typedef struct { uint64_t head, first, len, circ; } chain_t;

static u128 graph_node(const orc_graph *g, uint64_t v) {
  return ((u128)g->node_keys[2 * v] << 64) | g->node_keys[2 * v + 1];
}

/* the k-mer read at node v on strand s */
static u128 strand_kmer(const orc_graph *g, uint64_t v, int s) {
  u128 key = graph_node(g, v);
  return s ? mer_revcomp(key, (int)g->k) : key;
}

static int cmp_chain_head(const void *pa, const void *pb) {
  uint64_t a = ((const chain_t *)pa)->head, b = ((const chain_t *)pb)->head;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* spells a chain of strand-nodes; returns 0 when consecutive k-mers fail to overlap */
static int spell_chain(const orc_graph *g, const uint64_t *list, uint64_t m, char *out) {
  int K = (int)g->k;
  u128 prev = strand_kmer(g, list[0] >> 1, (int)(list[0] & 1));
  mer_spell(prev, K, out);
  u128 low = (((u128)1) << (2 * (K - 1))) - 1;
  for (uint64_t i = 1; i < m; i++) {
    u128 cur = strand_kmer(g, list[i] >> 1, (int)(list[i] & 1));
    if ((prev & low) != (cur >> 2)) return 0;
    out[K - 1 + i] = BASE_CHAR[cur & 3];
    prev = cur;
  }
  return 1;
}

/* The chains of the graph under one of two merging rules:
 *   literal = 0: an edge is merged when its ends are on distinct nodes and
 *                each end's side carries no other edge end (the unitigs);
 *   literal = 1: Section 6.1's candidate edges, "adjacent on nodes with
 *                exactly one in and out degree": an edge is merged when its
 *                ends are on distinct nodes that both have exactly one edge
 *                end on each side (a walk enters a node by one side and
 *                leaves by the other, so a node's in- and out-degree are its
 *                two side degrees).
 * Every node lies in exactly one chain (singletons included). */
static int compact_rule(const orc_graph *g, int literal, orc_unitigs **out) {
  if (!g || !out) return ORC_EINVAL;
  *out = NULL;
  uint64_t nv = g->n_nodes, ne = g->n_edges;
  int K = (int)g->k;
  int rc = ORC_OK;

  uint64_t *deg = (uint64_t *)calloc(2 * nv + 1, sizeof(uint64_t));
  link_t *link = (link_t *)malloc((2 * nv + 1) * sizeof(link_t));
  uint8_t *seen = (uint8_t *)calloc(nv + 1, 1);
  uint64_t *walk = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
  uint64_t *mirror = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
  chain_t *chains = (chain_t *)malloc((nv + 1) * sizeof(chain_t));
  uint64_t *order = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
  char *sa = (char *)malloc(nv + (uint64_t)K + 1), *sb = (char *)malloc(nv + (uint64_t)K + 1);
  orc_unitigs *u = (orc_unitigs *)calloc(1, sizeof(orc_unitigs));
  if (!deg || !link || !seen || !walk || !mirror || !chains || !order || !sa || !sb || !u)
    rc = ORC_ENOMEM;

  /* side degrees */
  for (uint64_t i = 0; rc == ORC_OK && i < ne; i++) {
    int o1 = g->orient[i] >> 1, o2 = g->orient[i] & 1;
    deg[2 * (uint64_t)g->src[i] + (o1 ? SIDE_L : SIDE_R)]++;
    deg[2 * (uint64_t)g->dst[i] + (o2 ? SIDE_R : SIDE_L)]++;
  }
  for (uint64_t i = 0; rc == ORC_OK && i < 2 * nv; i++) link[i].node = -1;
  for (uint64_t i = 0; rc == ORC_OK && i < ne; i++) {
    uint64_t a = g->src[i], b = g->dst[i];
    int o1 = g->orient[i] >> 1, o2 = g->orient[i] & 1;
    int sa_ = o1 ? SIDE_L : SIDE_R, sb_ = o2 ? SIDE_R : SIDE_L;
    if (a == b || deg[2 * a + sa_] != 1 || deg[2 * b + sb_] != 1) continue;
    if (literal && !(deg[2 * a + SIDE_L] == 1 && deg[2 * a + SIDE_R] == 1 && deg[2 * b + SIDE_L] == 1 &&
                     deg[2 * b + SIDE_R] == 1))
      continue;
    link[2 * a + sa_].node = (int64_t)b; link[2 * a + sa_].side = sb_;
    link[2 * b + sb_].node = (int64_t)a; link[2 * b + sb_].side = sa_;
  }

  /* collect chains: first the open ones from their ends, then the cycles */
  uint64_t nchains = 0, used = 0;
  for (int pass = 0; rc == ORC_OK && pass < 2; pass++) {
    for (uint64_t v = 0; rc == ORC_OK && v < nv; v++) {
      if (seen[v]) continue;
      int open_l = link[2 * v + SIDE_L].node < 0, open_r = link[2 * v + SIDE_R].node < 0;
      if (pass == 0 && !open_l && !open_r) continue;
      /* strand 0 enters by the left side and leaves by the right */
      int strand = (pass == 0 && !open_l) ? 1 : 0;
      uint64_t m = 0, cur = v;
      int s = strand;
      for (;;) {
        seen[cur] = 1;
        walk[m++] = (cur << 1) | (uint64_t)s;
        link_t nx = link[2 * cur + (s ? SIDE_L : SIDE_R)];
        if (nx.node < 0 || (uint64_t)nx.node == v) break;
        if (seen[nx.node]) { rc = ORC_EINTERNAL; break; }
        cur = (uint64_t)nx.node;
        s = (nx.side == SIDE_L) ? 0 : 1;
      }
      if (rc != ORC_OK) break;
      uint64_t *pick = walk;
      if (pass == 0) {
        /* the mirror copy reads the chain backwards on the other strands;
         * keep the copy whose spelled string is lexicographically smaller */
        for (uint64_t i = 0; i < m; i++) mirror[i] = walk[m - 1 - i] ^ 1;
        if (!spell_chain(g, walk, m, sa) || !spell_chain(g, mirror, m, sb)) { rc = ORC_EINTERNAL; break; }
        if (memcmp(sb, sa, m + K - 1) < 0) pick = mirror;
      }
      memcpy(order + used, pick, m * sizeof(uint64_t));
      chains[nchains].head = pick[0] >> 1;
      chains[nchains].first = used;
      chains[nchains].len = m;
      chains[nchains].circ = (uint64_t)pass;
      nchains++;
      used += m;
    }
  }
  if (rc == ORC_OK && used != nv) rc = ORC_EINTERNAL;

  if (rc == ORC_OK) {
    qsort(chains, nchains, sizeof(chain_t), cmp_chain_head);
    u->count = nchains;
    u->node_off = (uint64_t *)malloc((nchains + 1) * sizeof(uint64_t));
    u->seq_off = (uint64_t *)malloc((nchains + 1) * sizeof(uint64_t));
    u->nodes = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
    u->circular = (uint8_t *)malloc(nchains + 1);
    u->seq = (char *)malloc(nv + nchains * (uint64_t)(K - 1) + 1);
    if (!u->node_off || !u->seq_off || !u->nodes || !u->circular || !u->seq) rc = ORC_ENOMEM;
  }
  if (rc == ORC_OK) {
    uint64_t no = 0, so = 0;
    for (uint64_t c = 0; c < nchains && rc == ORC_OK; c++) {
      u->node_off[c] = no;
      u->seq_off[c] = so;
      u->circular[c] = (uint8_t)chains[c].circ;
      memcpy(u->nodes + no, order + chains[c].first, chains[c].len * sizeof(uint64_t));
      if (!spell_chain(g, u->nodes + no, chains[c].len, u->seq + so)) rc = ORC_EINTERNAL;
      no += chains[c].len;
      so += chains[c].len + (uint64_t)K - 1;
    }
    u->node_off[nchains] = no;
    u->seq_off[nchains] = so;
  }

  free(deg); free(link); free(seen); free(walk); free(mirror); free(chains); free(order);
  free(sa); free(sb);
  if (rc != ORC_OK) { orc_unitigs_free(u); return rc; }
  *out = u;
  return ORC_OK;
}

int orc_compact(const orc_graph *g, orc_unitigs **out) { return compact_rule(g, 0, out); }

/* ------------------------------------------------------------------ */
/* the simplified graph: the literal compaction of Section 6.1          */
/* ------------------------------------------------------------------ */

/* Section 6.1 merges the chains of candidate edges (compact_rule, literal
 * = 1) and reports "only the chains which are resultant of compaction of at
 * least three bi-directed nodes"; Section 6 describes the compacted graph:
 * a merged chain is one node labelled with its spelled string, and an edge
 * that touches a chain anywhere but at its two free ends no longer fits the
 * label and is removed as inconsistent.  Here:
 *   - units: every chain of at least min_nodes nodes (its nodes, string and
 *     circular flag as a unitig), and every node of a shorter chain on its
 *     own (positive strand, its k-mer), ordered by their first node's ID;
 *   - edges: every edge not inside a reported chain, in edge-ID order, each
 *     end relabelled to (unit, side): the end at a unit's first node on that
 *     node's entry side is the unit's left side (0), the end at its last
 *     node on the exit side its right side (1) -- a node on strand 0 is
 *     entered by its left side and left by its right, on strand 1 the other
 *     way round; any other end is inconsistent, and its edge is removed and
 *     counted in `removed`. */
typedef struct {
  uint64_t n_units, n_edges, removed;
  uint64_t *node_off;  /* n_units + 1 */
  uint64_t *nodes;     /* (node ID << 1) | strand */
  uint64_t *seq_off;   /* n_units + 1 */
  char *seq;
  uint8_t *circular;
  uint32_t *unit_a, *unit_b;  /* per edge: the units of its src and dst ends */
  uint8_t *side_a, *side_b;   /* 0 left, 1 right */
  uint32_t *edge;             /* the edge's ID in the graph */
} orc_simple;

void orc_simple_free(orc_simple *s) {
  if (!s) return;
  free(s->node_off); free(s->nodes); free(s->seq_off); free(s->seq); free(s->circular);
  free(s->unit_a); free(s->unit_b); free(s->side_a); free(s->side_b); free(s->edge);
  free(s);
}

typedef struct { uint64_t first_node, chain, node; int whole; } unit_ref;

static int cmp_unit_ref(const void *pa, const void *pb) {
  uint64_t a = ((const unit_ref *)pa)->first_node, b = ((const unit_ref *)pb)->first_node;
  return a < b ? -1 : (a > b ? 1 : 0);
}

int orc_simplify(const orc_graph *g, uint32_t min_nodes, orc_simple **out) {
  if (!g || !out) return ORC_EINVAL;
  *out = NULL;
  orc_unitigs *ch = NULL;
  int rc = compact_rule(g, 1, &ch);
  if (rc != ORC_OK) return rc;
  const uint64_t nv = g->n_nodes, ne = g->n_edges;
  const int K = (int)g->k;
  orc_simple *s = (orc_simple *)calloc(1, sizeof(orc_simple));
  unit_ref *refs = (unit_ref *)malloc((nv + 1) * sizeof(unit_ref));
  uint64_t *unit_of = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
  uint64_t *pos_of = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
  uint8_t *strand_of = (uint8_t *)malloc(nv + 1);
  uint64_t *deg = (uint64_t *)calloc(2 * nv + 1, sizeof(uint64_t));
  uint64_t *ulen = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
  if (!s || !refs || !unit_of || !pos_of || !strand_of || !deg || !ulen) rc = ORC_ENOMEM;

  /* units: reported chains whole, the nodes of the others one by one */
  uint64_t nu = 0;
  for (uint64_t c = 0; rc == ORC_OK && c < ch->count; c++) {
    const uint64_t m = ch->node_off[c + 1] - ch->node_off[c];
    if (m >= min_nodes) {
      refs[nu].first_node = ch->nodes[ch->node_off[c]] >> 1;
      refs[nu].chain = c; refs[nu].whole = 1; nu++;
    } else {
      for (uint64_t i = 0; i < m; i++) {
        refs[nu].first_node = ch->nodes[ch->node_off[c] + i] >> 1;
        refs[nu].node = refs[nu].first_node; refs[nu].whole = 0; nu++;
      }
    }
  }
  if (rc == ORC_OK) {
    qsort(refs, nu, sizeof(unit_ref), cmp_unit_ref);
    s->n_units = nu;
    s->node_off = (uint64_t *)malloc((nu + 1) * sizeof(uint64_t));
    s->seq_off = (uint64_t *)malloc((nu + 1) * sizeof(uint64_t));
    s->nodes = (uint64_t *)malloc((nv + 1) * sizeof(uint64_t));
    s->circular = (uint8_t *)malloc(nu + 1);
    s->seq = (char *)malloc(nv + nu * (uint64_t)(K - 1) + 1);
    if (!s->node_off || !s->seq_off || !s->nodes || !s->circular || !s->seq) rc = ORC_ENOMEM;
  }
  uint64_t no = 0, so = 0;
  for (uint64_t u = 0; rc == ORC_OK && u < nu; u++) {
    s->node_off[u] = no;
    s->seq_off[u] = so;
    if (refs[u].whole) {
      const uint64_t c = refs[u].chain, m = ch->node_off[c + 1] - ch->node_off[c];
      memcpy(s->nodes + no, ch->nodes + ch->node_off[c], m * sizeof(uint64_t));
      memcpy(s->seq + so, ch->seq + ch->seq_off[c], m + (uint64_t)K - 1);
      s->circular[u] = ch->circular[c];
      ulen[u] = m;
    } else {
      s->nodes[no] = refs[u].node << 1;
      mer_spell(graph_node(g, refs[u].node), K, s->seq + so);
      s->circular[u] = 0;
      ulen[u] = 1;
    }
    for (uint64_t i = 0; i < ulen[u]; i++) {
      const uint64_t x = s->nodes[no + i];
      unit_of[x >> 1] = u; pos_of[x >> 1] = i; strand_of[x >> 1] = (uint8_t)(x & 1);
    }
    no += ulen[u];
    so += ulen[u] + (uint64_t)K - 1;
  }
  if (rc == ORC_OK) {
    s->node_off[nu] = no;
    s->seq_off[nu] = so;
    if (no != nv) rc = ORC_EINTERNAL;
  }

  /* edges: drop those inside reported chains, relabel the others' ends */
  for (uint64_t i = 0; rc == ORC_OK && i < ne; i++) {
    deg[2 * (uint64_t)g->src[i] + ((g->orient[i] >> 1) ? SIDE_L : SIDE_R)]++;
    deg[2 * (uint64_t)g->dst[i] + ((g->orient[i] & 1) ? SIDE_R : SIDE_L)]++;
  }
  if (rc == ORC_OK) {
    s->unit_a = (uint32_t *)malloc((ne + 1) * sizeof(uint32_t));
    s->unit_b = (uint32_t *)malloc((ne + 1) * sizeof(uint32_t));
    s->side_a = (uint8_t *)malloc(ne + 1);
    s->side_b = (uint8_t *)malloc(ne + 1);
    s->edge = (uint32_t *)malloc((ne + 1) * sizeof(uint32_t));
    if (!s->unit_a || !s->unit_b || !s->side_a || !s->side_b || !s->edge) rc = ORC_ENOMEM;
  }
  uint64_t kept = 0;
  for (uint64_t i = 0; rc == ORC_OK && i < ne; i++) {
    const uint64_t a = g->src[i], b = g->dst[i];
    const int sa = (g->orient[i] >> 1) ? SIDE_L : SIDE_R, sb = (g->orient[i] & 1) ? SIDE_R : SIDE_L;
    const int simple_a = deg[2 * a + SIDE_L] == 1 && deg[2 * a + SIDE_R] == 1;
    const int simple_b = deg[2 * b + SIDE_L] == 1 && deg[2 * b + SIDE_R] == 1;
    /* a candidate edge lies inside its chain; reported chains swallow it */
    if (a != b && simple_a && simple_b && ulen[unit_of[a]] > 1) continue;
    const uint64_t ends[2] = {a, b};
    const int sides[2] = {sa, sb};
    int unit_side[2] = {-1, -1};
    for (int j = 0; j < 2; j++) {
      const uint64_t x = ends[j], u = unit_of[x];
      const int st = strand_of[x];
      const int entry = st ? SIDE_R : SIDE_L, exit_ = st ? SIDE_L : SIDE_R;
      if (!s->circular[u] && pos_of[x] == 0 && sides[j] == entry) unit_side[j] = 0;
      else if (!s->circular[u] && pos_of[x] == ulen[u] - 1 && sides[j] == exit_) unit_side[j] = 1;
    }
    if (unit_side[0] < 0 || unit_side[1] < 0) { s->removed++; continue; }
    s->unit_a[kept] = (uint32_t)unit_of[a]; s->side_a[kept] = (uint8_t)unit_side[0];
    s->unit_b[kept] = (uint32_t)unit_of[b]; s->side_b[kept] = (uint8_t)unit_side[1];
    s->edge[kept] = (uint32_t)i;
    kept++;
  }
  if (rc == ORC_OK) s->n_edges = kept;
  free(refs); free(unit_of); free(pos_of); free(strand_of); free(deg); free(ulen);
  orc_unitigs_free(ch);
  if (rc != ORC_OK) { orc_simple_free(s); return rc; }
  *out = s;
  return ORC_OK;
}

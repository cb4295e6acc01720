/*
 * dbg.h -- C ABI of the GB300 bi-directed de Bruijn graph builder.
 *
 * The library builds the bi-directed de Bruijn graph of a set of DNA reads
 * by the sort-based method of Kundeti, Rajasekaran, Dinh, Vaughn and Thapar,
 * "Efficient Parallel and Out of Core Algorithms for Constructing Large
 * Bi-directed de Bruijn Graphs" (arXiv 1003.1940), on one GPU, and compacts
 * its chains into unitigs.
 *
 * Problem statement (Section 3): given reads R_f = {r_1..r_n} over
 * {A,C,G,T} and an odd k, produce the node list V (canonical k-mers), the
 * edge list E (canonical bi-directed edges with multiplicities) and the
 * adjacency lists.  Compaction (Section 6) merges chains of nodes joined by
 * a valid bi-directed walk into unitigs.
 *
 * Conventions for every call
 *   - The status code is the only error channel.  On error, *out is NULL and
 *     no partial result is returned.
 *   - Inputs are borrowed for the duration of the call only.  Pointers to
 *     caller data may be host pointers or device pointers of the context's
 *     device; the library tells them apart with cudaPointerGetAttributes.
 *   - Results (dbg_graph, dbg_unitigs) are owned by the library until the
 *     matching *_free call; accessors copy into caller buffers (host or
 *     device) and return when the copy is complete.
 *   - Calls on one dbg_ctx are not thread-safe; use one context per host
 *     thread, or the dbg_submit/dbg_poll serving calls.
 *
 * Encoding (all integer, bit-exact)
 *   - Bases A=0 C=1 G=2 T=3.  An m-mer is stored most-significant-base
 *     first, so integer order equals lexicographic order with A<C<G<T.
 *   - Keys of k <= 31 are one uint64_t; keys of 33 <= k <= 63 are two
 *     uint64_t words (high word first).  "key words" W below is 1 or 2.
 *     A node key holds k bases, an edge key k+1 bases.
 *   - orient = (o1 << 1) | o2, o = 1 when the k-mer read at that end of the
 *     edge is the negative strand (the reverse complement of the node key).
 *
 * Output orders (defined so that results are reproducible bit for bit)
 *   - nodes: ascending canonical k-mer; node ID = rank.
 *   - edges: ascending canonical (k+1)-mer; edge ID = rank; src <= dst.
 *   - adjacency row of a node: its edge ends by ascending (edge ID, role).
 *   - unitigs: ascending ID of their first node.
 */
#ifndef DBG_H
#define DBG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dbg_status {
  DBG_OK = 0,
  DBG_EINVAL = 1,      /* bad argument: k even or outside [1, 63], NULL, a byte outside {A,C,G,T} */
  DBG_ENOMEM = 2,      /* device or host allocation failed, or over the memory budget */
  DBG_ECUDA = 3,       /* a CUDA runtime call failed */
  DBG_ETIMEOUT = 4,    /* a bounded device-side wait reached its limit */
  DBG_ECANCELLED = 5,  /* request cancelled (serving) */
  DBG_EOVERFLOW = 6,   /* more than 2^32 - 1 edge instances, edges or nodes in one build */
  DBG_EAGAIN = 7,      /* dbg_poll without waiting: the request has not finished */
  DBG_EINTERNAL = 8    /* an internal consistency check failed (a library defect); no result */
} dbg_status;

typedef struct dbg_ctx dbg_ctx;
typedef struct dbg_graph dbg_graph;
typedef struct dbg_unitigs dbg_unitigs;

/* Optional device-memory hooks.  alloc returns device memory usable on
 * `stream` (NULL on failure); free releases it in stream order. */
typedef void *(*dbg_alloc_fn)(void *user, size_t bytes, void *stream);
typedef void (*dbg_free_fn)(void *user, void *ptr, size_t bytes, void *stream);

typedef struct dbg_options {
  uint32_t struct_size;    /* sizeof(dbg_options) */
  int32_t device;          /* CUDA device ordinal; -1 = the current device */
  void *stream;            /* cudaStream_t for all work; NULL = a stream the context creates */
  dbg_alloc_fn alloc;      /* NULL = stream-ordered cudaMallocAsync from the device pool */
  dbg_free_fn free;
  void *alloc_user;
  uint64_t mem_budget;     /* bytes a request may hold on the device; 0 = no limit */
  uint32_t spin_limit;     /* iterations a device wait may spin before DBG_ETIMEOUT; 0 = default */
  uint32_t reserved0;      /* must be 0 */
  uint32_t reserved1;      /* must be 0 */
  uint32_t reserved[8];
} dbg_options;

/* Fills *opt with defaults. */
void dbg_options_init(dbg_options *opt);

/* Creates a context on the device named by opt (NULL = defaults). */
dbg_status dbg_create(dbg_ctx **ctx, const dbg_options *opt);
void dbg_destroy(dbg_ctx *ctx);

/* Message for the last error of this host thread ("" if none). */
const char *dbg_last_error(void);

/* ----------------------------------------------------------------------
 * dbg_build -- the sort-based construction of Section 3 (BiConstruct):
 *   STEP-1: one canonical (k+1)-mer key per consecutive k-mer pair of every
 *           read (its canonical edge), STEP-2: radix sort + run-length
 *           reduce (edges with multiplicities), STEP-3: sort of the edge
 *           ends (nodes), STEP-4: adjacency lists.
 *   reads    all reads back to back, ASCII 'A','C','G','T' (no separators);
 *            device or host memory (host reads are streamed to the device
 *            in 256 MB pieces; pinned host memory copies fastest)
 *   lengths  n read lengths (bases), device or host memory
 *   n        number of reads; n = 0 gives an empty graph
 *   k        odd, 1 <= k <= 63 (Section 2: k odd, so no k-mer is its own
 *            reverse complement)
 *   out      receives the graph (library-owned; release with dbg_graph_free)
 * Multiplicities count the forward reads (sum of multiplicities =
 * sum over reads of max(0, L - k)).  A read of length exactly k adds its
 * k-mer as a node without edges (Section 2 takes every k-mer of the reads as
 * a node; STEP-3 alone would collect only edge ends); a shorter read adds
 * nothing.
 * Errors: DBG_EINVAL (k, NULL, non-ACGT byte), DBG_EOVERFLOW (>= 2^32
 * edge instances), DBG_ENOMEM, DBG_ECUDA, DBG_ETIMEOUT.
 * -------------------------------------------------------------------- */
dbg_status dbg_build(dbg_ctx *ctx, const char *reads, const uint32_t *lengths, uint64_t n,
                     uint32_t k, dbg_graph **out);

uint32_t dbg_graph_k(const dbg_graph *g);
uint32_t dbg_graph_key_words(const dbg_graph *g);  /* W: 1 for k <= 31, 2 above */
uint64_t dbg_graph_num_nodes(const dbg_graph *g);
uint64_t dbg_graph_num_edges(const dbg_graph *g);
uint64_t dbg_graph_num_instances(const dbg_graph *g);  /* sum over reads of max(0, L - k) */

/* Node keys: W words per node, ascending.  Buffer: num_nodes * W uint64_t. */
dbg_status dbg_graph_nodes(const dbg_graph *g, uint64_t *keys);

/* Edges by ascending canonical (k+1)-mer.  Any pointer may be NULL to skip
 * that array.  keys: num_edges * W words; src, dst: node IDs; orient as
 * above; mult: multiplicity. */
dbg_status dbg_graph_edges(const dbg_graph *g, uint64_t *keys, uint32_t *src, uint32_t *dst,
                           uint8_t *orient, uint32_t *mult);

/* Node multiplicities: for every node (ascending key order, as
 * dbg_graph_nodes), the number of positions of the forward reads whose
 * k-mer is the node's k-mer or its reverse complement -- STEP-2's counting
 * applied to k-mers, the k-mer occurrence table from which VELVET's roadmap
 * is drawn (Section 7).  They are counted by dbg_build when the context's
 * switch is on (dbg_node_mult_set; off by default: an extra k-mer sort),
 * not by dbg_build_bucketed.  mult: num_nodes uint32_t.  DBG_EINVAL if the
 * graph was built without them. */
dbg_status dbg_node_mult_set(dbg_ctx *ctx, int on);
dbg_status dbg_graph_node_mult(const dbg_graph *g, uint32_t *mult);

/* Roadmap counts (Section 7: VELVET builds its graph from the k-mers present
 * in at least 2 reads, its "roadmap"): for every node, the number of
 * distinct reads that hold its k-mer on either strand.  Counted by dbg_build
 * when the context's switch is on (dbg_node_reads_set; off by default: a
 * sort of (k-mer, read) records), not by dbg_build_bucketed.  reads:
 * num_nodes uint32_t.  DBG_EINVAL if the graph was built without them.
 * dbg_roadmap_nodes writes the IDs of the nodes held by at least min_reads
 * distinct reads, ascending, to ids (host or device, room for num_nodes
 * entries; NULL to count only) and their number to *count. */
dbg_status dbg_node_reads_set(dbg_ctx *ctx, int on);
dbg_status dbg_graph_node_reads(const dbg_graph *g, uint32_t *reads);
dbg_status dbg_roadmap_nodes(dbg_ctx *ctx, const dbg_graph *g, uint32_t min_reads, uint32_t *ids,
                             uint64_t *count);

/* The same copies, started on a stream of the graph's own and returned from
 * at once, so that they overlap later work on the GPU (e.g. dbg_compact of
 * the same graph, which only reads it).  Host buffers should be pinned for
 * the copies to run asynchronously; they must stay valid, and be left
 * unread, until dbg_graph_wait returns.  dbg_graph_wait blocks until every
 * copy started on the graph is done (DBG_OK at once if none was);
 * dbg_graph_free waits for them too.  Errors of the copies are reported by
 * the call that starts them or by dbg_graph_wait. */
dbg_status dbg_graph_edges_async(dbg_graph *g, uint64_t *keys, uint32_t *src, uint32_t *dst,
                                 uint8_t *orient, uint32_t *mult);
/* The node keys and the adjacency (as dbg_graph_nodes / dbg_graph_csr), the
 * same way. */
dbg_status dbg_graph_nodes_async(dbg_graph *g, uint64_t *keys);
dbg_status dbg_graph_csr_async(dbg_graph *g, uint64_t *row_ptr, uint32_t *nbr, uint32_t *edge, uint8_t *role);
dbg_status dbg_graph_wait(dbg_graph *g);

/* Adjacency (STEP-4) in CSR form: row_ptr has num_nodes + 1 entries; entry
 * p of a row holds the neighbour node ID, the edge ID and the role (0: the
 * row's node is the edge's src end, 1: its dst end).  A self-loop appears
 * twice in its node's row.  Any pointer may be NULL. */
dbg_status dbg_graph_csr(const dbg_graph *g, uint64_t *row_ptr, uint32_t *nbr, uint32_t *edge,
                         uint8_t *role);

/* Device pointers to the graph's arrays, valid until dbg_graph_free. */
typedef struct dbg_graph_view {
  uint32_t k, key_words;
  uint64_t num_nodes, num_edges, num_instances;
  const uint64_t *node_keys, *edge_keys, *row_ptr;
  const uint32_t *src, *dst, *mult, *adj_nbr, *adj_edge;
  const uint8_t *orient, *adj_role;
} dbg_graph_view;
dbg_status dbg_graph_device_view(const dbg_graph *g, dbg_graph_view *view);

void dbg_graph_free(dbg_graph *g);

/* ----------------------------------------------------------------------
 * dbg_compact -- bi-directed chain compaction (Section 6).
 * Each node has a left and a right side; the src end of (u, v, o1, o2) sits
 * on u's right side if o1 = 0, else its left; the dst end on v's left side
 * if o2 = 0, else its right.  An edge is merged when u != v and both of its
 * sides carry exactly one edge end.  The nodes split into unitigs: maximal
 * chains of merged edges (open or circular), singletons included.  The
 * chains are found by list ranking over the 2|V| strands of the
 * ListRankingTransform (each node v becomes v+ and v-).
 * Each open unitig is reported as the copy whose spelled string is
 * lexicographically smaller; a circular one starts at its smallest node,
 * positive strand.  Spelled length = nodes + k - 1.
 * -------------------------------------------------------------------- */
dbg_status dbg_compact(dbg_ctx *ctx, const dbg_graph *g, dbg_unitigs **out);

/* How dbg_compact ranks the lists.  0 (the default): the meeting walks
 * with staged halves when every list is short and acyclic, with 32-bit walk
 * words up to 2^29 - 1 strand-nodes and 64-bit words up to 2^30, else
 * pointer jumping with cycle breaking; 1: the walks with 64-bit words at
 * any size they allow; 2: pointer jumping only.  The unitigs are the same
 * either way.  DBG_EINVAL for another mode. */
dbg_status dbg_compact_mode_set(dbg_ctx *ctx, int mode);

/* Streams over which the read-back of a graph (dbg_graph_*_async) or of
 * unitigs (dbg_unitigs_get) built with this context is spread, in chunks
 * of at least 32 MB: 1 (the default) to 8.  DBG_EINVAL outside. */
dbg_status dbg_copy_streams_set(dbg_ctx *ctx, int n);

/* ----------------------------------------------------------------------
 * dbg_compact_bucketed -- dbg_compact with the out-of-core list ranking of
 * Section 6.2: the ranking words of the 2|V| strand-nodes (list head,
 * distance) live in host memory, and each round of pointer jumping is a
 * join of every unresolved strand-node's word with its ancestor's word,
 * sorted by the ancestor's key range and processed range by range on the
 * device in pieces that fit mem_budget bytes (0 = half the free device
 * memory).  Cycles are found when the rounds stop shrinking, labelled by
 * their smallest strand-node with the same joins, opened there and ranked
 * again.  The graph itself, the successors and the final selection and
 * output stay on the device.  The unitigs are identical to dbg_compact's.
 * join_launches (may be NULL) receives the number of join launches.
 * -------------------------------------------------------------------- */
dbg_status dbg_compact_bucketed(dbg_ctx *ctx, const dbg_graph *g, uint64_t mem_budget, dbg_unitigs **out,
                                uint32_t *join_launches);

uint64_t dbg_unitigs_count(const dbg_unitigs *u);
uint64_t dbg_unitigs_total_bases(const dbg_unitigs *u);
/* node_off, seq_off: count + 1 entries; nodes: num_nodes entries, each
 * (node ID << 1) | strand with strand 1 = read as reverse complement;
 * seq: ASCII, unitigs back to back; circular: count entries of 0/1.
 * Any pointer may be NULL. */
dbg_status dbg_unitigs_get(const dbg_unitigs *u, uint64_t *node_off, uint64_t *nodes,
                           uint64_t *seq_off, char *seq, uint8_t *circular);
void dbg_unitigs_free(dbg_unitigs *u);

/* ----------------------------------------------------------------------
 * dbg_simplify -- the simplified bi-directed graph (Section 6) with the
 * literal chain compaction of Section 6.1.
 * Candidate edges are those "adjacent on nodes with exactly one in and out
 * degree": an edge whose ends lie on two distinct nodes that each carry
 * exactly one edge end on each side (a walk enters a node by one side and
 * leaves by the other).  Their chains (paths or cycles, found by the list
 * ranking of dbg_compact) of at least min_nodes nodes are merged into one
 * unit each (Section 6.1 reports chains of at least 3); every other node is
 * a unit of its own, on its positive strand.  Units are listed like
 * unitigs (dbg_simple_units: node lists, spelled strings, circular flags),
 * ascending by first node ID.  Every edge not inside a merged chain is kept
 * in graph edge order with its ends relabelled to (unit, side): side 0 is
 * the unit's left side (its first node's entry side), 1 its right side (its
 * last node's exit side).  An edge with an end anywhere else on a unit no
 * longer fits the unit's label (Section 6); it is removed and counted in
 * dbg_simple_removed_edges (none exist under this candidate rule).
 *   unit_a, side_a: the src end; unit_b, side_b: the dst end; edge: its ID
 *   in g.  Any pointer may be NULL.  Host or device buffers.
 * -------------------------------------------------------------------- */
typedef struct dbg_simple dbg_simple;
dbg_status dbg_simplify(dbg_ctx *ctx, const dbg_graph *g, uint32_t min_nodes, dbg_simple **out);
uint64_t dbg_simple_num_units(const dbg_simple *s);
uint64_t dbg_simple_num_edges(const dbg_simple *s);
uint64_t dbg_simple_removed_edges(const dbg_simple *s);
uint64_t dbg_simple_total_bases(const dbg_simple *s);
dbg_status dbg_simple_units(const dbg_simple *s, uint64_t *node_off, uint64_t *nodes, uint64_t *seq_off, char *seq,
                            uint8_t *circular);
dbg_status dbg_simple_edges(const dbg_simple *s, uint32_t *unit_a, uint8_t *side_a, uint32_t *unit_b,
                            uint8_t *side_b, uint32_t *edge);
void dbg_simple_free(dbg_simple *s);

/* ----------------------------------------------------------------------
 * Many constructions at once (batched builds and a request server).
 *
 * A read set as dbg_build takes it.  The buffers are borrowed until the
 * request has finished (dbg_poll returned it, or dbg_build_batch returned).
 * flags: DBG_REQ_BUCKETED forces the key-range bucket path.
 * -------------------------------------------------------------------- */
typedef struct dbg_readset {
  const char *reads;
  const uint32_t *lengths;
  uint64_t n;
  uint32_t k;
  uint32_t flags;
} dbg_readset;
enum { DBG_REQ_BUCKETED = 1u };

typedef struct dbg_server dbg_server;

typedef struct dbg_server_options {
  uint32_t struct_size;     /* sizeof(dbg_server_options) */
  int32_t device;           /* -1 = the current device */
  uint32_t workers;         /* concurrent builds (each its own stream), 1..64; default 4 */
  uint32_t spin_limit;      /* as in dbg_options; 0 = default */
  uint64_t mem_budget;      /* device bytes running requests and unfreed results may hold; 0 = 80 % of free memory */
  uint32_t sort_variant[4]; /* radix sort variant per key kind (see dbg_sort_variant_set) */
  uint32_t reserved[8];
} dbg_server_options;

typedef struct dbg_request_stats {
  double queue_s;      /* submission to start */
  double run_s;        /* start to finish */
  double latency_s;    /* submission to finish */
  uint64_t footprint;  /* worst-case device bytes of the in-memory build */
  uint32_t bucketed;   /* 1 if built by the key-range bucket path */
  uint32_t retries;    /* times the build ran out of device memory and waited to run again */
  uint64_t charged;    /* bytes charged while it ran (bucket path: its key-range budget) */
} dbg_request_stats;

void dbg_server_options_init(dbg_server_options *opt);

/* Starts `workers` worker threads, each with its own context and stream.
 * Admission (continuous: a request that arrives while others run starts as
 * soon as it is admitted; their kernels overlap on the device):
 *   - a request's footprint is the worst-case peak of its in-memory build
 *     (every edge instance a distinct edge, every local-sort group oversize),
 *     computed at submission from the read lengths (device-resident lengths
 *     are copied to the host for it);
 *   - the first queued request whose footprint fits the budget next to what
 *     is charged runs when a worker is free (any request may run when none
 *     runs); it is charged its footprint while it runs;
 *   - a finished graph stays charged at its real size until dbg_graph_free
 *     (polled or not), so results count against the budget too;
 *   - a request whose footprint exceeds the whole budget runs on the bucket
 *     path with the part of the budget that is free when it starts (at least
 *     a quarter of what it asks, or whatever is free when it runs alone);
 *   - a build that still runs out of device memory (taken outside the
 *     budget) is queued again until another request finishes; alone, it
 *     fails with DBG_ENOMEM.
 * Results are the same graphs dbg_build returns for the same read set. */
dbg_status dbg_server_create(dbg_server **srv, const dbg_server_options *opt);
/* Waits for running requests; frees results nobody polled. */
void dbg_server_destroy(dbg_server *srv);
uint64_t dbg_server_budget(const dbg_server *srv);
/* Bytes charged to the budget now: running requests and unfreed results. */
uint64_t dbg_server_charged(const dbg_server *srv);
typedef struct dbg_server_counters {
  uint64_t charged;       /* as dbg_server_charged */
  uint64_t peak_charged;  /* the most charged right after an admission */
  uint64_t finished;      /* requests finished (successfully or not) */
  uint32_t running;       /* requests running now */
  uint32_t peak_running;  /* the most that ran at once */
  uint32_t queued;        /* requests waiting for admission */
  uint32_t reserved;
} dbg_server_counters;
dbg_status dbg_server_stats(const dbg_server *srv, dbg_server_counters *out);
dbg_status dbg_submit(dbg_server *srv, const dbg_readset *req, uint64_t *ticket);
/* wait != 0 blocks until the request has finished; otherwise returns
 * DBG_EAGAIN while it runs.  On success *out is the graph (the caller frees
 * it, before destroying the server) and the ticket is retired; an error
 * status of the build is returned here.  stats may be NULL. */
dbg_status dbg_poll(dbg_server *srv, uint64_t ticket, int wait, dbg_graph **out, dbg_request_stats *stats);

/* Builds nsets read sets concurrently (a transient server with `workers`
 * workers, 0 = 4) and returns one graph per set in outs; identical to
 * calling dbg_build on each.  On error every outs[i] is NULL. */
dbg_status dbg_build_batch(dbg_ctx *ctx, const dbg_readset *sets, uint32_t nsets, uint32_t workers,
                           dbg_graph **outs);

/* ----------------------------------------------------------------------
 * dbg_build_bucketed -- dbg_build for inputs whose edge keys do not fit the
 * device: the out-of-core construction of Section 5, with the external
 * R-way merge replaced by key-range partitioning.  The reads are packed
 * once on the device (host reads are streamed in chunks); the canonical
 * (k+1)-mer key space is cut into ranges that each fit mem_budget, and for
 * each range in ascending order only its keys are emitted, sorted and
 * reduced, so the concatenated results are the sorted edge list.  Nodes are
 * handled the same way over node-key ranges.  The result is bit-identical
 * to dbg_build's.  Packed reads, per-read offsets and the final graph must
 * fit on the device.  mem_budget = 0 uses half the free device memory.
 * -------------------------------------------------------------------- */
dbg_status dbg_build_bucketed(dbg_ctx *ctx, const char *reads, const uint32_t *lengths, uint64_t n, uint32_t k,
                              uint64_t mem_budget, dbg_graph **out);
/* Key ranges the build used (1 and 1 for dbg_build). */
void dbg_graph_buckets(const dbg_graph *g, uint32_t *edge_ranges, uint32_t *node_ranges);

/* ----------------------------------------------------------------------
 * dbg_rle_u64_noalloc -- STEP-2's run-length reduce over sorted 64-bit keys
 * (the distinct keys and where each run starts), as a call that allocates no
 * memory at all.  It runs a single-pass reduce with decoupled look-back that
 * dbg_build itself does not use (the build counts copies inside its local
 * sort pass); both give the same distinct keys and multiplicities.  The
 * paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at call
 * time -- a host program whose memory manager reserved the whole GPU up
 * front, a plugin whose host framework forbids allocation after start-up,
 * or a real-time loop that cannot take cudaMalloc's implicit device
 * synchronisation.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   keys       device, n keys in ascending order
 *   n          0 <= n <= 2^26 (67,108,864); larger n returns DBG_EINVAL
 *   uniq       device, room for n keys: the distinct keys, ascending
 *   run_start  device, room for n + 1 entries (never NULL, also for n = 0):
 *              index in `keys` of each distinct key's first occurrence, then
 *              n; the multiplicity of uniq[i] is run_start[i + 1] -
 *              run_start[i]
 *   count      host: receives the number of distinct keys
 *   stream     cudaStream_t to run on (NULL = the legacy default stream);
 *              the call returns after the stream has finished its work
 * Its scratch (per-tile look-back words, counters, error word: 128 KiB) is
 * a fixed array in the library's device memory, which every GPU that loads
 * the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the one array and
 * clear it at their start, so calls that overlap on the GPU (other streams,
 * other host threads) race: serialise them.
 * -------------------------------------------------------------------- */
dbg_status dbg_rle_u64_noalloc(const uint64_t *keys, uint64_t n, uint64_t *uniq, uint32_t *run_start,
                               uint64_t *count, void *stream);

/* ----------------------------------------------------------------------
 * Radix sort variants and the autotuner.  The onesweep sort of STEP-2/3 is
 * compiled in several configurations per key kind (tile shape, TMA or
 * register loads, ballot / atomicOr / match.any ranking); all sort
 * identically.  Kinds: 0 = 64-bit keys, 1 = 64-bit keys + 32-bit payload,
 * 2 = 128-bit keys, 3 = 128-bit keys + payload; kinds 4 (64-bit keys) and
 * 5 (128-bit keys) select the ranking method of the hybrid sort's local
 * pass (0 = match.any, 1 = shared-memory atomicOr, 2 = ballots).  A context
 * starts with variant 0 of every kind.
 * dbg_autotune times one digit pass of every variant on n synthetic keys
 * (0 = 2^25; 128-bit kinds use n / 2) and keeps the fastest of kinds 0-3 in
 * the context.  cache_path (may be NULL) names a text file of choices keyed
 * by GPU name and SM count: a matching line is used instead of timing, and
 * a new result is appended.  ms_out (may be NULL) receives 4 x
 * DBG_MAX_SORT_VARIANTS pass times in ms (kind-major; variant v of kind k at
 * k * DBG_MAX_SORT_VARIANTS + v).
 * -------------------------------------------------------------------- */
#define DBG_MAX_SORT_VARIANTS 64 /* per kind */
uint32_t dbg_sort_variant_count(uint32_t kind);
const char *dbg_sort_variant_name(uint32_t kind, uint32_t variant);
dbg_status dbg_sort_variant_set(dbg_ctx *ctx, uint32_t kind, uint32_t variant);
int32_t dbg_sort_variant_get(const dbg_ctx *ctx, uint32_t kind);
dbg_status dbg_autotune(dbg_ctx *ctx, uint64_t n, const char *cache_path, double *ms_out);

/* ----------------------------------------------------------------------
 * Hybrid sort switch.  With it on (the default) the sorts of STEP-2 and
 * STEP-3 run the onesweep passes only over the high digits, which groups
 * keys with equal high bits, and finish each run of whole groups in shared
 * memory (for the edge keys fused with STEP-2's duplicate removal).  Runs
 * longer than shared memory holds (6144 keys for k <= 31, 3072 above; e.g.
 * the (k+1)-mers of a tandem repeat) are gathered and sorted over every
 * digit globally instead; the result is the same either way.
 * dbg_sort_fallbacks counts the sorts of the context that had such runs.
 * on = 0 sorts every digit globally.
 * -------------------------------------------------------------------- */
dbg_status dbg_sort_hybrid_set(dbg_ctx *ctx, int on);
uint64_t dbg_sort_fallbacks(const dbg_ctx *ctx);

/* ----------------------------------------------------------------------
 * Count-first switch.  With it on (the default) the local pass
 * of the hybrid edge-key sort counts each tile's copies of every key in a
 * shared-memory hash table of 2048 slots and sorts only the distinct keys,
 * which at read coverage c are about 1/c of them; a tile whose distinct
 * keys do not fit (about 1500 and up) is sorted copy by copy instead, and
 * dbg_sort_count_overflows counts such tiles over the context's builds.
 * Off, every tile is sorted copy by copy.  The edge list is the same
 * either way.
 * -------------------------------------------------------------------- */
dbg_status dbg_sort_count_first_set(dbg_ctx *ctx, int on);
uint64_t dbg_sort_count_overflows(const dbg_ctx *ctx);

/* ----------------------------------------------------------------------
 * Partition-first switch.  With it on (the default) the first global
 * radix pass over the edge keys (which carry no payload) is an unordered
 * partition by that digit: keys of one digit keep no particular order,
 * which no later step depends on (the later passes are stable and equal
 * keys are identical), and no tile waits for another.  Off, it is a
 * stable onesweep pass like the others.  The graph is the same either
 * way.  Node records, whose payload order matters, always sort stably.
 * -------------------------------------------------------------------- */
dbg_status dbg_sort_partition_first_set(dbg_ctx *ctx, int on);

/* ----------------------------------------------------------------------
 * Group-ranking switch for the local passes of the hybrid sort.  The
 * global passes leave keys with equal high bits (a group) contiguous; with
 * the switch on (the default) a local pass places each key at its group's
 * start plus the number of the group's keys that precede it (for the
 * count-first edge pass, the distinct keys below it; for 64-bit node
 * records, the records with smaller low bits or an equal key and an
 * earlier position, which keeps the sort stable).  Tiles holding a group
 * too long for that (over 256 distinct edge keys or 512 records) take the
 * shared-memory digit passes, as every tile does with the switch off.
 * The graph is the same either way.
 * -------------------------------------------------------------------- */
dbg_status dbg_sort_local_rank_set(dbg_ctx *ctx, int on);
/* Tiles that met such a group, over the context's builds. */
uint64_t dbg_sort_rank_fallbacks(const dbg_ctx *ctx);

/* ----------------------------------------------------------------------
 * Failure detection.  Every device-side wait of the library (decoupled
 * look-back, TMA completion) spins at most spin_limit times, then records
 * DBG_ETIMEOUT in the context's device error word and returns; the call
 * reports it and the context stays usable.  dbg_selftest_wait runs one such
 * wait on a status word that nothing writes, with the given limit
 * (1..2^20), so the path can be tested: it returns DBG_ETIMEOUT.
 * -------------------------------------------------------------------- */
dbg_status dbg_selftest_wait(dbg_ctx *ctx, uint32_t spin_limit);

/* ----------------------------------------------------------------------
 * Profiling (tracing).  When enabled, the context brackets every kernel it
 * launches with CUDA events on its stream and accumulates, per stage, the
 * launches, device time and algorithmic bytes (the bytes the stage must
 * read and write by its definition, not measured traffic).  Stage names:
 * offsets, pack, emit, sort_edges, rle, endpoints, sort_nodes, node_ids,
 * adjacency, copies, compact_links, compact_rank, compact_cycles,
 * compact_output, local_sort_edges, local_sort_nodes, partition_edges
 * (the edge keys' first global pass when it is a partition; sort_edges
 * then holds their stable onesweep passes), node_mult (the k-mer counting
 * for node multiplicities, whose sort passes count under the edge-key
 * sort stages).
 * -------------------------------------------------------------------- */
typedef struct dbg_stage_stat {
  char name[24];
  uint64_t launches;   /* kernel launches of the stage */
  double ms;           /* summed device time of those launches */
  double bytes;        /* summed algorithmic bytes */
} dbg_stage_stat;

/* on != 0 enables timing; any call resets the statistics. */
dbg_status dbg_profile_enable(dbg_ctx *ctx, int on);
/* Copies up to cap stage records; returns the number of stages. */
uint32_t dbg_profile_read(dbg_ctx *ctx, dbg_stage_stat *out, uint32_t cap);
/* Kernels launched by this context since it was created. */
uint64_t dbg_launch_count(const dbg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DBG_H */

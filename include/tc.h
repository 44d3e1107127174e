/*
 * tc.h — C ABI of libtc: cover-edge triangle counting on one GB300 (sm_103a).
 *
 * Method: D. A. Bader et al., "Cover Edge-Based Novel Triangle Counting"
 * (arXiv 2403.02997).  The count follows Algorithm CETC-Seq (Section "Cover-Edge
 * Triangle Counting"), computed in the data-parallel shape of Algorithm CETC-SM:
 *
 *   1. BFS levels L(v) from a root (Definition "BFS-Edge"); vertices the root does
 *      not reach get levels from further searches started, in ascending id order,
 *      at every still-unvisited vertex (the restart loop of Algorithm CETC-Seq);
 *   2. the cover-edge set S = { {u, v} : L(u) == L(v) }, the horizontal edges,
 *      which holds an edge of every triangle (Lemma "H-E", Theorem "Cover-Edge Set
 *      Generation");
 *   3. for each {u, v} in S with u < v, the common neighbours w of u and v are
 *      counted when L(w) != L(u), or when L(w) == L(u) and v < w (Theorem
 *      "Correctness": every triangle is counted exactly once).
 *
 * Every step runs in CUDA kernels on the device; there is no CPU path.
 *
 * Conventions for every call:
 *   - vertex ids are uint32 in [0, n) and n < 2^31;
 *   - pointers named host_* are host memory; `src`/`dst` are host or device
 *     memory as `edges_on_device` says; everything else the library owns;
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream); work is ordered on it;
 *   - calls on one graph handle must not run concurrently from several host
 *     threads; different handles are independent;
 *   - a call that fails with a status other than TC_ERR_CUDA leaves the handle
 *     valid; after TC_ERR_CUDA the CUDA context may be unusable.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_graph tc_graph; /* opaque: device CSR, level array, scratch */

typedef enum tc_status {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = 1,  /* NULL pointer, root >= n, n >= 2^31, ... */
  TC_ERR_VERTEX_RANGE = 2, /* an edge endpoint is >= num_vertices */
  TC_ERR_OOM = 3,          /* device allocation failed */
  TC_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
  TC_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
  TC_ERR_OVERFLOW = 6      /* sizes beyond what the library supports */
} tc_status;

/*
 * Build a graph from an edge list (Section "Notations and Definitions": an
 * undirected graph G = (V, E) with neighbour sets N(v)).
 *
 * src[i], dst[i] (i < num_edges) is one undirected edge.  Self-loops are
 * dropped and repeated pairs (in either orientation) collapse to one edge; the
 * stored form is a CSR with every row sorted ascending and each edge in both
 * rows.  If edges_on_device != 0 the arrays are device pointers, else host
 * pointers.  The arrays are copied: the caller may free them when the call
 * returns.  Work runs on `stream`, which is synchronised before return.
 *
 * Errors: TC_ERR_INVALID_ARG (out == NULL, or num_edges > 0 with a NULL array,
 * or num_vertices >= 2^31), TC_ERR_VERTEX_RANGE (an id >= num_vertices; *out
 * stays NULL), TC_ERR_OOM, TC_ERR_CUDA.  num_vertices == 0 or num_edges == 0 is
 * valid and gives an edgeless graph.  The handle owns all its device memory,
 * taken stream-ordered from the library's memory pool (see tc_pool_trim).
 */
tc_status tc_graph_create(const uint32_t* src, const uint32_t* dst, uint64_t num_edges,
                          uint32_t num_vertices, int edges_on_device, void* stream,
                          tc_graph** out);

/*
 * Degree ordering, the pre-processing of Algorithms CETC-Seq-D and CETC-Seq-SD
 * (Section "Experimental Results"; the reordering "in decreasing order of their
 * degrees" of Section "Related Work"): a new graph whose vertex i is the old
 * vertex host_old_of_new[i], the vertices taken by decreasing degree, ties by
 * increasing id (so the new vertex 0 has the largest degree).  tc_count on the
 * new handle is Algorithm CETC-Seq-D and tc_count_split is CETC-Seq-SD; the
 * count equals the original graph's, while levels and cover edges are those of
 * the relabelled graph.  host_old_of_new (n entries) may be NULL.  The new
 * handle copies g's tunables and is independent of g (destroy both).  Errors:
 * TC_ERR_INVALID_ARG (g or out NULL), TC_ERR_OOM, TC_ERR_CUDA.
 */
tc_status tc_graph_relabel_degree(const tc_graph* g, void* stream, tc_graph** out,
                                  uint32_t* host_old_of_new);

/*
 * Free the handle and all device memory it owns.  NULL is accepted.  Every
 * call on a handle has finished its device work when it returns (each
 * synchronises its own stream), so destroy adds no synchronisation of its own.
 * The memory goes back to the library's pool (reserved for the next handle
 * until tc_pool_trim).
 */
tc_status tc_graph_destroy(tc_graph* g);

/*
 * Sizes: n, m = number of undirected edges after canonicalising, and the
 * largest degree d_max (Section "Notations and Definitions").  Any out pointer
 * may be NULL.
 */
tc_status tc_graph_info(const tc_graph* g, uint32_t* n, uint64_t* m, uint32_t* d_max);

/*
 * Count the triangles of the graph by the cover-edge method with BFS root
 * `root` (Algorithm CETC-Seq; any root gives the same count, the levels and
 * the cover set depend on it).  Enqueues the whole path on `stream`, waits for
 * it and writes the count to *count (host).
 *
 * Errors: TC_ERR_INVALID_ARG (root >= n while n > 0, or count == NULL),
 * TC_ERR_TIMEOUT, TC_ERR_CUDA.  For n == 0 the count is 0.
 */
tc_status tc_count(tc_graph* g, uint32_t root, void* stream, uint64_t* count);

/*
 * Triangle listing and per-vertex triangle counts from the cover-edge count
 * (the Introduction names k-truss and clustering coefficients as their users).
 * The count runs as tc_count with root `root`; every triangle, found once at
 * its cover edge {u, v} (u < v, L(u) == L(v)) with apex w under Algorithm
 * CETC-Seq's rule, is also
 *   - written to `triangles` (device, 3 x capacity uint32) as (u, v, w), in an
 *     unspecified order, while fewer than `capacity` have been written;
 *   - counted in vertex_counts[u], [v] and [w] (device, n uint64, zeroed by the
 *     call; the number of triangles through each vertex).
 * Either output may be NULL.  *count = all triangles; *written = the triples
 * stored (min(count, capacity); may be NULL).  A count larger than capacity is
 * not an error: call again with capacity >= count for the full list.  Levels,
 * cover edges and statistics read as after tc_count.  Errors as tc_count.
 */
tc_status tc_list_triangles(tc_graph* g, uint32_t root, void* stream, uint32_t* triangles,
                            uint64_t capacity, uint64_t* vertex_counts, uint64_t* count,
                            uint64_t* written);

/*
 * Algorithm CETC-Seq-S (Section "CETC Split Triangle Counting").  BFS levels
 * from `root` as in tc_count; the edges then split into G0, the horizontal
 * edges, and G1, the edges between levels.  T0 = the triangles of G0 by
 * Algorithm forward-hashed (Section "Related Work"; the vertices ranked by
 * their G0 degree), T1 = the sum over horizontal edges {u, v} of
 * |N_G1(u) ∩ N_G1(v)|.  *count = T0 + T1, the same count as tc_count's;
 * tc_get_stats gives c1 = T1 and c2 = 3 T0 (Algorithm CETC-SM's split), and
 * levels and cover edges can be read as after tc_count.  The first call
 * allocates the handle's oriented adjacency (n + 1 offsets and m ids).
 * Errors as tc_count, plus TC_ERR_OOM.
 */
tc_status tc_count_split(tc_graph* g, uint32_t root, void* stream, uint64_t* count);

/*
 * Algorithm Forward with hashed intersections (Section "Related Work"), the
 * vertices ranked by (degree, id) as in the paper's reordering by degree:
 * every edge is oriented towards its endpoint of higher rank, A+(x) holds the
 * ends of x's outgoing edges, and each oriented edge (x, w) adds
 * |A+(x) ∩ A+(w)|.  No BFS: tc_get_levels and tc_get_cover_edges refuse
 * (TC_ERR_INVALID_ARG) until the next tc_count.  Allocates as tc_count_split.
 * Errors: TC_ERR_INVALID_ARG (count == NULL), TC_ERR_OOM, TC_ERR_CUDA.
 */
tc_status tc_count_forward(tc_graph* g, void* stream, uint64_t* count);

/*
 * Algorithm CETC-Seq-FE (Section "CETC Forward Exchanging Triangle Counting"):
 * BFS from `root`, then the covering ratio c = |S| / m; when c < threshold the
 * count goes on as tc_count (Algorithm CETC-Seq), otherwise as
 * tc_count_forward.  The paper's experiments use threshold 0.7.
 * *used_forward (may be NULL) receives 1 when the forward count ran.  After a
 * forward count the levels and cover edges are not available.  Errors as
 * tc_count, plus TC_ERR_INVALID_ARG for a negative or NaN threshold.
 */
tc_status tc_count_fe(tc_graph* g, uint32_t root, float threshold, void* stream, uint64_t* count,
                      int* used_forward);

/*
 * Count k graphs (roots[i] for gs[i]) together (the batched form of the
 * data-parallel Algorithm CETC-SM): the graphs are concatenated into one CSR
 * with per-graph vertex and entry offsets, and every phase runs as one sequence
 * of launches over all of them -- a multi-source BFS from the k roots, one
 * cover-edge pass, one owner-hash pass -- with each hit added to its graph's
 * counter.  counts (host, k entries) receives one count per graph, equal to
 * what tc_count gives for that graph and root.  gs[i] must be pairwise
 * distinct; the tunables are those of gs[0].  Builds a temporary batch (see
 * tc_batch_create) and frees it before returning.  Errors as tc_count and
 * tc_batch_create; on error no count is written.
 */
tc_status tc_count_many(tc_graph* const* gs, const uint32_t* roots, size_t k, void* stream,
                        uint64_t* counts);

/*
 * Introspection of the last tc_count on this handle, for parity checks (a
 * batched count reports through tc_batch_get_*).  Each call synchronises the
 * device.
 */

/* host_levels[n] receives L(v) (int32, every vertex >= 0 after a count). */
tc_status tc_get_levels(const tc_graph* g, int32_t* host_levels);

/*
 * The cover-edge set S (Theorem "Cover-Edge Set Generation"): *num_cover = |S|;
 * if host_u and host_v are both non-NULL they receive the |S| pairs u < v in
 * an unspecified order.  Pass NULL arrays to query the size first.
 */
tc_status tc_get_cover_edges(const tc_graph* g, uint64_t* num_cover, uint32_t* host_u,
                             uint32_t* host_v);

/* The CSR: host_row_ptr[n+1] (uint64 offsets), host_col[2m]. */
tc_status tc_get_csr(const tc_graph* g, uint64_t* host_row_ptr, uint32_t* host_col);

/* Statistics of the last count. */
typedef struct tc_stats {
  uint64_t triangles;   /* T */
  uint64_t c1;          /* common neighbours on another level (Algorithm CETC-SM) */
  uint64_t c2;          /* common neighbours on the same level; T == c1 + c2 / 3 */
  uint64_t num_cover;   /* |S| */
  uint64_t m;           /* undirected edges */
  uint32_t num_levels;  /* 1 + largest level reached from the root */
  uint32_t bfs_steps;   /* level-synchronous steps run, restarts included */
  uint32_t bottom_up_steps;
  uint32_t restarted;   /* 1 if vertices outside the root's component existed */
  float ms_bfs;         /* phase times (CUDA events), ms */
  float ms_cover;
  float ms_intersect;
  float ms_total;
  float ms_hash;        /* the owner-hash intersection kernel alone */
  uint32_t launches;    /* kernels launched by the count */
  uint64_t hash_items;  /* owner-hash work items */
  uint64_t hash_edges;  /* cover edges on the owner-hash path */
} tc_stats;

tc_status tc_get_stats(const tc_graph* g, tc_stats* out);

/* Smallest id among the vertices of largest degree (0 when n == 0). */
tc_status tc_max_degree_vertex(const tc_graph* g, uint32_t* v);

/*
 * Tunables of the count (all have defaults; see tc_params_default).  They
 * change speed only, never results.
 */
typedef struct tc_params {
  uint32_t small_max_degree; /* cover edges with both degrees <= this use the direct merge */
  uint32_t hash_chunk;       /* owner-row entries per shared-memory hash chunk (multiple of 32,
                                32..16384) */
  uint32_t edges_per_item;   /* cover edges per hash work item: 1..1024 with hash_block 512,
                                1..4096 with 1024; on graphs of 2^32 or more adjacency entries
                                it is clamped to hash_block */
  uint32_t bfs_alpha;        /* top-down -> bottom-up when frontier edges > unexplored / alpha */
  uint32_t bfs_beta;         /* bottom-up -> top-down when frontier < n / beta */
  uint32_t sorted_lookup;    /* 1: look ids up by binary search in the sorted chunk instead of
                                the cuckoo table (the automatic fallback if a build fails) */
  uint32_t persistent_bfs;   /* 1 (default): runs of small frontiers go to one persistent
                                cooperative kernel with a device-side grid barrier */
  uint32_t barrier_timeout_ms; /* bound on each device-side barrier wait (default 2000); past it
                                  the count fails with TC_ERR_TIMEOUT and the handle stays usable */
  uint32_t test_barrier_skip;  /* testing only: 1 makes one block leave the persistent kernel
                                  without arriving at a barrier, so the other blocks time out */
  uint32_t medium_max_degree;  /* cover edges above the small bin whose larger degree is <= this
                                  (at most 1024; 0 disables the bin) go to a warp merge: the
                                  longer row staged in shared memory, the shorter searched in it */
  uint32_t hash_block;       /* threads per owner-hash block: 512 (default) or 1024 (one block per
                                SM; allows hash_chunk 16384 with the SM's full warp count) */
  uint32_t cluster_bfs;      /* 1 (default, with persistent_bfs): runs of frontiers of at most 4096
                                vertices of degree <= 8 go to a search in one cluster of 8 blocks
                                (hardware cluster barrier between levels); 0: to the persistent
                                kernel */
} tc_params;

tc_status tc_params_default(tc_params* p);
/* Errors: TC_ERR_INVALID_ARG for a value out of range, or for a hash_chunk
 * whose tables exceed the device's shared memory per block. */
tc_status tc_set_params(tc_graph* g, const tc_params* p);

/*
 * A reusable batch of graphs (for repeated counts, e.g. a serving loop).
 * tc_batch_create copies the k graphs' CSRs into one concatenated device CSR
 * (the handles stay owned by the caller and may be destroyed afterwards) and
 * sizes the per-count state for the union.  Errors: TC_ERR_INVALID_ARG (k == 0,
 * NULL or repeated handles), TC_ERR_OVERFLOW (more than 2^31 - 1 vertices in
 * total), TC_ERR_OOM, TC_ERR_CUDA.
 */
typedef struct tc_batch tc_batch;
tc_status tc_batch_create(tc_graph* const* gs, size_t k, void* stream, tc_batch** out);
/*
 * A batch straight from k graphs' edge lists, without per-graph handles: the
 * edges of graph i are src[j], dst[j] for edge_offsets[i] <= j < edge_offsets[i+1]
 * (edge_offsets: host, k+1 entries, edge_offsets[0] == 0), with local ids below
 * num_vertices[i] (host, k entries).  src/dst are device arrays if
 * edges_on_device != 0, else host arrays; they are copied.  One radix sort
 * canonicalises every graph at once (self-loops dropped, repeats collapsed,
 * rows sorted), exactly as tc_graph_create does per graph.  Errors as
 * tc_batch_create, plus TC_ERR_VERTEX_RANGE when an id is >= its own graph's
 * vertex count.
 *
 * Memory: everything this batch uses on the device, the build's sort buffers
 * included, is taken in stream order on `stream` from the library's memory
 * pool for the current device, and tc_batch_destroy returns it in stream
 * order on a library-owned stream.  So building one batch and destroying
 * another never synchronises the device (a serving loop builds on one stream
 * while it counts on another).  The pool keeps freed memory reserved for the
 * next build; tc_pool_trim returns it to the driver.  Pass pinned host arrays
 * for the copies to run asynchronously.
 */
tc_status tc_batch_create_from_edges(const uint32_t* src, const uint32_t* dst,
                                     const uint64_t* edge_offsets, const uint32_t* num_vertices,
                                     size_t k, int edges_on_device, void* stream, tc_batch** out);
/* host_roots[i] = smallest local id of largest degree in graph i (0 if empty). */
tc_status tc_batch_max_degree_vertices(tc_batch* b, void* stream, uint32_t* host_roots);
/* roots[i] < n_i of graph i (ignored for empty graphs); counts: host, k entries. */
tc_status tc_batch_count(tc_batch* b, const uint32_t* roots, void* stream, uint64_t* counts);
/*
 * The same counts (and levels, for tc_batch_get_levels) from ONE persistent
 * launch: each block takes whole graphs from a device work queue, largest
 * first, and runs the path for a graph inside the block -- BFS from its root
 * and the restart rule of Algorithm CETC-Seq, the cover edges (Theorem
 * "Cover-Edge Set Generation") and their intersections under the counting
 * rule of Algorithm CETC-Seq.  Meant for batches of many small graphs (a few
 * million edges each at most: a graph is one block's work).  The first call on
 * a batch also sorts its graphs by size (one extra launch and synchronisation).
 * Statistics: ms_total, the batch's triangles, c1, c2 and cover edges.
 * Errors as tc_batch_count.
 */
tc_status tc_batch_count_persistent(tc_batch* b, const uint32_t* roots, void* stream,
                                    uint64_t* counts);
tc_status tc_batch_set_params(tc_batch* b, const tc_params* p);
/* Statistics of the last tc_batch_count, summed over the batch. */
tc_status tc_batch_get_stats(const tc_batch* b, tc_stats* out);
/* Levels of graph i after tc_batch_count: host_levels[n_i]. */
tc_status tc_batch_get_levels(const tc_batch* b, size_t i, int32_t* host_levels);
/* Free a batch (NULL is accepted); no device-wide synchronisation for batches
 * from tc_batch_create_from_edges (see there). */
tc_status tc_batch_destroy(tc_batch* b);

/*
 * The library's memory pool on the current device (stream-ordered memory of
 * the graphs from tc_graph_create and the batches built from edge lists).  tc_pool_trim releases reserved but
 * unused memory until at most keep_bytes stay reserved (it synchronises the
 * library's free stream first); tc_pool_reserved reports the bytes the pool
 * holds from the driver now.  Errors: TC_ERR_INVALID_ARG (NULL), TC_ERR_CUDA.
 */
tc_status tc_pool_trim(uint64_t keep_bytes);
tc_status tc_pool_reserved(uint64_t* bytes);

/*
 * BFS levels of a caller-owned device graph, allocating no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- applications that own all device memory through their own
 * pool or a fixed budget, and services that must not allocate once running.
 *
 * row_ptr (device, n+1 uint64 offsets) and col (device, row_ptr[n] uint32 ids)
 * are an undirected graph in CSR form: every edge in both rows, no self-loops;
 * rows need not be sorted (tc_get_csr's output qualifies).  levels (device, n
 * int32) receives L(v): the BFS distance from root, and for vertices the root
 * does not reach, the distance from the smallest id of their connected
 * component, so every entry ends >= 0.  The caller
 * owns all three arrays; nothing is retained after the call returns.  Work is
 * ordered on `stream`, which the call synchronises once per BFS level.
 *
 * Scratch: one fixed __device__ array of 12 MiB + 256 B (queues and union-find
 * parents for up to 2^20 vertices), held by every GPU that loads the library
 * until the process exits.  The first call on a device looks up its address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call on a device shares the array and
 * leaves its contents behind; the call clears what it needs.  Calls whose
 * device work overlaps (other streams or host threads at the same time) race
 * on the shared array: serialise them.
 *
 * Errors: TC_ERR_OVERFLOW if n > 2^20 (nothing is written); TC_ERR_INVALID_ARG
 * for a NULL pointer or root >= n; TC_ERR_CUDA.  n == 0 returns TC_OK at once.
 */
tc_status tc_bfs_levels_noalloc(const uint64_t* row_ptr, const uint32_t* col, uint32_t n,
                                uint32_t root, int32_t* levels, void* stream);

/* Human-readable name of a status. */
const char* tc_status_string(tc_status s);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */

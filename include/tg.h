/*
 * tg.h -- exact typed-graphlet counting on one GPU (C ABI).
 *
 * Computes, for an undirected simple graph whose nodes carry one of L types,
 * the two problems of "Heterogeneous Graphlets" (Rossi et al., TKDD 2020):
 *
 *   Problem 1 (Sec. 4, "local typed graphlet counting"): for every edge
 *     (i,j), the count of every typed 3- and 4-node graphlet orbit that
 *     contains the edge.
 *   Problem 2 (Sec. 6, "global typed graphlet counting"): the total count of
 *     every typed 2-, 3- and 4-node graphlet, C_H = (1/|E(H)|) x^T e.
 *
 * Every count is an exact integer.  Node types only (Alg. 1-3 use node
 * types; the edge types of Def. 1 are not part of this library).
 *
 * ------------------------------------------------------------------------
 * Conventions
 *
 * Graph input: a symmetric CSR.  row_ptr (int64, n+1 entries, row_ptr[0] =
 *   0, non-decreasing, row_ptr[n] = nnz), col (int32, nnz entries, each in
 *   [0,n)), node_types (uint8, n entries, each in [0,L)).  Every undirected
 *   edge {u,v} appears once in row u and once in row v; rows may be
 *   unsorted.  Self-loops, repeated entries and one-sided entries make the
 *   graph invalid.  1 <= L <= TG_MAX_TYPES.
 *
 * Pointers: any pointer argument that carries graph data or results may be
 *   host memory (pageable or pinned) or device memory of the current device;
 *   the library inspects each one.  Host inputs are copied in on the given
 *   stream; host outputs are copied out and the call then synchronises the
 *   stream.  The library never frees or keeps caller memory.
 *
 * Streams: every call that takes `stream` (a cudaStream_t, NULL = legacy
 *   default stream) is stream-ordered.  Device outputs are complete when the
 *   stream reaches the call's end.
 *
 * Edge ids: the edges {u,v}, u < v in the caller's node ids, numbered
 *   0..m-1 in lexicographic order of (u,v).  For a batch (tg_build_batch)
 *   the node id ranges of the graphs follow each other, so graph g's edges
 *   form the id range [edge_off[g], edge_off[g+1]).
 *
 * Per-edge output (Problem 1): uint32 rows of S(L) slots, row e = edge e.
 *   P = L(L+1)/2 unordered type pairs; pair(t,t') for t <= t' is the position
 *   of (t,t') in the lexicographic list (0,0),(0,1),...,(0,L-1),(1,1),...
 *     slot t          (0 <= t < L): typed 3-paths through the edge whose
 *                     third node has type t: |S_i^t| + |S_j^t| (Cor. 3)
 *     slot L + t:     typed triangles, |T_ij^t| (Cor. 1)
 *     slot 2L + (o-3)P + pair(t,t'), o = 3..12: orbit g_o (Table 3) with the
 *                     two other nodes of types {t,t'}.  Orbits: g3 4-path
 *                     end edge, g4 4-path centre edge, g5 4-star, g6 4-cycle,
 *                     g7 tailed-triangle tail, g8 tailed-triangle edge
 *                     opposite the degree-3 node, g9 tailed-triangle edge at
 *                     the degree-3 node, g10 chordal-cycle outer edge, g11
 *                     chordal-cycle chord, g12 4-clique.
 *   S(L) = 2L + 10P for k = 4; S(L) = 2L for k = 3 (3-node slots only).
 *   A count above 2^32-1 is stored as 2^32-1 and raises TG_ERR_OVERFLOW
 *   in the status word; global totals are always exact.
 *
 * Global output (Problem 2): int64, G(L) slots per graph, in blocks
 *     block 0  typed edges           C(L+1,2) type multisets of size 2
 *     block 1  typed 3-paths         C(L+2,3) multisets of size 3
 *     block 2  typed triangles       C(L+2,3)
 *     blocks 3..8 typed 4-paths, 4-stars, 4-cycles, tailed-triangles,
 *              chordal-cycles, 4-cliques   C(L+3,4) multisets of size 4 each
 *   (k = 3: blocks 0..2 only).  Inside a block, slot = position of the
 *   sorted type multiset in the lexicographic list of sorted multisets.
 *   The block sizes are Table 2's ((L multichoose K)).
 *
 * Errors: host-detectable errors are returned at once and change nothing.
 *   Errors found on the device (invalid graph, overflow, a bounded wait that
 *   ran out, an internal consistency check) are OR-ed into the graph's
 *   device status word, which tg_query_status returns.  No call traps,
 *   aborts or exits.
 * ------------------------------------------------------------------------
 */
#ifndef TG_H_
#define TG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TG_MAX_TYPES 8
#define TG_ABI_VERSION 1

typedef enum {
    TG_OK = 0,
    TG_ERR_INVALID_ARG = 1,     /* bad argument (size, k, NULL where required) */
    TG_ERR_INVALID_GRAPH = 2,   /* not a simple symmetric CSR, or a type >= L */
    TG_ERR_TOO_MANY_TYPES = 3,  /* L < 1 or L > TG_MAX_TYPES */
    TG_ERR_OOM = 4,             /* device memory exhausted */
    TG_ERR_OVERFLOW = 5,        /* a per-edge count exceeded 2^32-1 (saturated) */
    TG_ERR_TIMEOUT = 6,         /* a bounded device wait ran out */
    TG_ERR_CUDA = 7,            /* a CUDA runtime call failed */
    TG_ERR_INTERNAL = 8,        /* an internal consistency check failed */
    TG_ERR_TOO_LARGE = 9        /* graph exceeds an index-width limit */
} tg_status;

typedef struct tg_graph tg_graph;   /* opaque; owns device copies of the graph */

/* Slot layout for (L, k).  Pure host function. */
typedef struct {
    int32_t L, k;
    int64_t pairs;               /* P = L(L+1)/2 */
    int64_t per_edge_slots;      /* S(L) */
    int64_t global_slots;        /* G(L) */
    int64_t orbit_offset[13];    /* per-edge slot of orbit o's first pair; o = 1 (3-path), 2 (triangle),
                                    3..12; entry 0 unused */
    int64_t global_block_offset[9];
    int64_t global_block_size[9];
    int32_t graphlet_edges[9];   /* |E(H)| of each global block: 1,2,3,3,3,4,4,5,6 */
} tg_layout_t;

/* Tuning knobs (0 = library default).  Results never depend on them. */
typedef struct {
    int32_t light_edge_max_degree;    /* edges whose triangle set T has at most max(this, 32) nodes:
                                         warp per edge in the 4-clique pass (CTA per edge above) */
    int32_t light_anchor_max_wedges;  /* wedge anchors with at most this many wedges: warp per anchor
                                         (at most 2048, and what one CTA's shared memory holds for L) */
    int32_t anchor_table_budget_mb;   /* device memory for the dense node tables of heavy anchors with
                                         too many wedges for shared memory, one per CTA that takes them
                                         (default 12,288; at most two CTAs per SM get one) */
    int32_t ctas_per_sm;              /* resident CTAs per SM for the per-edge kernels */
    int32_t cycle_budget_mb;          /* device memory for the per-slot 4-cycle array; a batch whose
                                         array would exceed it is counted in chunks of whole graphs */
    int32_t hub_min_wedges;           /* anchors with more wedges than this are hubs: each is counted
                                         by the whole GPU against one node table shared by all CTAs */
    int32_t hub_l2_mb;                /* MB of hub node tables of the persistent hub pass: one group
                                         of hubs fills at most half of it (about the L2 size) */
    int32_t isect_modes;              /* typed set intersection per bucket of the shorter segment's
                                         length (buckets [1,32) [32,128) [128,512) [512,inf), two bits
                                         each from bit 0): 0 default = 1, 1 binary search of each
                                         shorter entry in the longer segment, 2 warp-wide merge of
                                         both segments, 3 whichever a dependent-load count favours */
} tg_options;

/* ---- layout ---------------------------------------------------------- */

/* Fills *out for L types and k in {3,4}.  Errors: TG_ERR_TOO_MANY_TYPES,
 * TG_ERR_INVALID_ARG. */
tg_status tg_layout(int32_t L, int32_t k, tg_layout_t *out);

/* Default tuning knobs. */
void tg_default_options(tg_options *opt);

/* ---- graph handles --------------------------------------------------- */

/* Builds a device handle for one graph (Sec. 4.1, Def. 6-7: typed
 * neighbourhoods).  The library copies what it needs; the caller may free
 * its inputs when the stream reaches the end of the call.  On the device it
 * validates the graph, orders nodes by (degree, id), sorts every adjacency
 * list by (type, id) with per-type offsets (typed neighbourhoods Gamma_i^t
 * and typed degrees d_i^t), numbers the edges and precomputes per-node
 * typed degree sums.  opt may be NULL.  Synchronises `stream` once (to size
 * work lists).  Errors: TG_ERR_INVALID_ARG, TG_ERR_TOO_MANY_TYPES,
 * TG_ERR_INVALID_GRAPH, TG_ERR_OOM, TG_ERR_TOO_LARGE, TG_ERR_CUDA; on error
 * *out is NULL. */
tg_status tg_build(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                   const uint8_t *node_types, int32_t L, const tg_options *opt,
                   void *stream, tg_graph **out);

/* Builds one handle for `ngraphs` independent graphs given as one
 * block-diagonal CSR: graph g owns nodes [node_off[g], node_off[g+1]) (host
 * array of ngraphs+1 int64, node_off[0] = 0, node_off[ngraphs] = n) and no
 * edge joins two graphs.  Counting the handle counts every graph at once
 * (pattern: batched small graphs) and writes per-graph global totals.
 * Errors as tg_build. */
tg_status tg_build_batch(int32_t ngraphs, const int64_t *node_off, int64_t n, int64_t nnz,
                         const int64_t *row_ptr, const int32_t *col, const uint8_t *node_types,
                         int32_t L, const tg_options *opt, void *stream, tg_graph **out);

/* Releases everything the handle owns (after synchronising its stream). */
void tg_free(tg_graph *g);

int64_t tg_num_nodes(const tg_graph *g);
int64_t tg_num_edges(const tg_graph *g);
int32_t tg_num_graphs(const tg_graph *g);
int32_t tg_num_types(const tg_graph *g);
/* Device memory the handle holds now, in bytes. */
int64_t tg_device_bytes(const tg_graph *g);

/* Edge id -> endpoints in the caller's node ids: src[e] < dst[e], int32,
 * m entries each (host or device).  Stream-ordered on the build stream. */
tg_status tg_edge_endpoints(const tg_graph *g, int32_t *src, int32_t *dst);

/* Per-graph first edge ids: out[ngraphs+1] (host). */
tg_status tg_edge_offsets(const tg_graph *g, int64_t *out);

/* ---- counting -------------------------------------------------------- */

/* Problem 1 + Problem 2 for every graph of the handle.
 *   k = 3: typed triangles and 3-paths (Cor. 1-3).
 *   k = 4: additionally the ten typed 4-node orbits (Alg. 1-3, Lemmas 1-4,
 *          Table 3) and the six typed 4-node graphlets (Sec. 4.4).
 * per_edge_out: uint32 [m][S(L)] or NULL (global totals only).
 * global_out:   int64 [ngraphs][G(L)] or NULL.
 * Working memory is allocated on the first call and kept by the handle.
 * Errors: TG_ERR_INVALID_ARG, TG_ERR_OOM, TG_ERR_CUDA (device-detected
 * errors go to the status word). */
tg_status tg_count(tg_graph *g, int32_t k, uint32_t *per_edge_out, int64_t *global_out,
                   void *stream);

/* As tg_count for the edge id range [e_begin, e_end) only (chunked or
 * sharded runs; edges are independent given the graph, Sec. 4.7).
 * per_edge_out row 0 is edge e_begin.  global_accum (int64 [ngraphs][G],
 * may be NULL) receives, added to its contents, the raw per-edge sums
 * sum_e x_e of the range -- not yet divided by |E(H)|; tg_finalize_global
 * turns the sum over all ranges into totals.  The per-graph preparation
 * (typed triangle counts, wedge tables) runs once per handle and k. */
tg_status tg_count_range(tg_graph *g, int32_t k, int64_t e_begin, int64_t e_end,
                         uint32_t *per_edge_out, int64_t *global_accum, void *stream);

/* Divides raw per-graphlet edge sums by |E(H)| (Sec. 6).  Host arrays of
 * ngraphs*G(L) int64.  Returns TG_ERR_INTERNAL if a sum is not a multiple. */
tg_status tg_finalize_global(int32_t L, int32_t k, int32_t ngraphs, const int64_t *raw,
                             int64_t *out);

/* Problem 1 in the sparse form of Sec. 4.6 (X_ij: only the nonzero counts
 * of each edge).  Edge e's pairs are entries row_off[e] .. row_off[e+1]-1
 * of slot / value: slot = its per-edge slot in the dense layout of
 * tg_layout (increasing), value = the count.  row_off: int64 [m+1]; slot:
 * uint16, value: uint32, `cap` entries each; all three DEVICE memory owned
 * by the caller (row_off may be NULL).  *nnz (host) receives the number of
 * pairs.  With slot = value = NULL the call only sizes: it fills row_off and
 * *nnz and returns TG_OK.  If the pairs exceed cap, the ones that fit whole
 * windows may have been written, *nnz is the capacity needed and the call
 * returns TG_ERR_TOO_LARGE.  global_out as in tg_count (host or device, may
 * be NULL).  The edges are counted in windows whose dense rows take at most
 * 1 GB of library memory; synchronises `stream` once per window.  Errors:
 * TG_ERR_INVALID_ARG (k, NULL nnz, only one of slot/value, host arrays),
 * TG_ERR_TOO_LARGE, TG_ERR_OOM, TG_ERR_CUDA. */
tg_status tg_count_sparse(tg_graph *g, int32_t k, int64_t *row_off, uint16_t *slot, uint32_t *value,
                          int64_t cap, int64_t *nnz, int64_t *global_out, void *stream);

/* Typed-graphlet weighted graph, the first step of Alg. 5: for the typed
 * graphlet H = (block, rank) -- block as in tg_layout's global blocks (0
 * edge, 1 3-path, 2 triangle, 3 4-path, 4 4-star, 5 4-cycle, 6 tailed
 * triangle, 7 chordal cycle, 8 4-clique), rank = the lexicographic rank of
 * H's type multiset within the block -- weights[e] = the number of instances
 * of H that contain both endpoints of edge e, and (if degree != NULL)
 * degree[x] = sum of weights[e] over the edges e at node x (the
 * typed-graphlet degree D_xx).  per_edge_rows: this handle's rows from
 * tg_count with the same k (blocks 0-2 need k = 3 or 4, blocks 3-8 k = 4).
 * weights: int64 [m] in edge-id order; degree: int64 [n] in the caller's
 * node ids.  All three DEVICE memory owned by the caller.  Synchronises
 * `stream`.  Errors: TG_ERR_INVALID_ARG (k, block, rank, NULL, host
 * memory), TG_ERR_CUDA. */
tg_status tg_graphlet_weights(tg_graph *g, int32_t k, const uint32_t *per_edge_rows, int32_t block, int64_t rank,
                              int64_t *weights, int64_t *degree, void *stream);

/* ---- position-aware typed graphlets (Sec. 5, Def. 8) ------------------
 *
 * Def. 8 identifies two typed instances of one shape when an isomorphism
 * between them maps every node onto a node of the same type.  With the
 * shape's nodes numbered, a position-aware typed graphlet is a labelling
 * (types of nodes 0..k-1) up to the automorphisms of the numbered shape;
 * its global slot ranks it by its lexicographically smallest labelling
 * within the shape's block.  Numbered shapes (global blocks 0..8): 0 edge
 * 0-1; 1 3-path, 0 the centre; 2 triangle; 3 4-path 0-1-2-3; 4 4-star, 0
 * the centre; 5 4-cycle 0-1-2-3-0; 6 tailed triangle, 0 the degree-3 node, 1
 * the tail, 2-3 the triangle's other edge; 7 chordal cycle, 0-1 the chord;
 * 8 4-clique.  Block sizes are the numbers of labellings up to symmetry
 * (Burnside), e.g. (L^4 + L^2)/2 for the 4-path; L^K labellings in all.
 *
 * Per-edge rows (uint32, S_pa(L) = 3L + 9L^2 + 6P slots): edge e = {lo, hi},
 * lo < hi in the caller's ids; "side" 0 = lo, 1 = hi; an ordered type pair
 * (x, y) at x*L + y; an unordered pair at pair(t, t') as in the typed layout.
 * Blocks, in this order (block_offset[1..12]):
 *   O1  3-path: [side of the centre][type of the third node]          2L
 *   O2  triangle: [type of the third node]                             L
 *   O3  4-path, end edge: [side of the inner endpoint][type of its other
 *       neighbour][type of the far end]                                2L^2
 *   O4  4-path, centre edge: [type of lo's other neighbour][of hi's]   L^2
 *   O5  4-star: [side of the centre][pair of the other two leaves]     2P
 *   O6  4-cycle: [type of lo's other neighbour][of hi's]               L^2
 *   O7  tailed triangle, tail edge: [side of the degree-3 node][pair of
 *       the other two triangle nodes]                                  2P
 *   O8  tailed triangle, edge opposite the degree-3 node: [type of the
 *       degree-3 node][type of the tail]                               L^2
 *   O9  tailed triangle, triangle edge at the degree-3 node: [side of the
 *       degree-3 node][type of the third triangle node][type of the tail]
 *                                                                      2L^2
 *   O10 chordal cycle, outer edge: [side of the degree-3 endpoint][type of
 *       the other degree-3 node][type of the other degree-2 node]      2L^2
 *   O11 chordal cycle, chord: [pair of the two degree-2 nodes]         P
 *   O12 4-clique: [pair of the other two nodes]                        P
 * Summing the sides and the orderings of a row gives the typed row of
 * tg_count (k = 4).  A count above 2^32-1 saturates as in tg_count. */
typedef struct {
    int32_t L;
    int64_t per_edge_slots;           /* S_pa(L) */
    int64_t global_slots;             /* G_pa(L): sum of the block sizes */
    int64_t block_offset[13];         /* first per-edge slot of O1..O12; entry 0 unused */
    int64_t global_block_offset[9];
    int64_t global_block_size[9];
    int32_t graphlet_edges[9];        /* |E(H)| of each global block */
} tg_pa_layout_t;

/* Fills *out for L types.  Pure host function.  Errors:
 * TG_ERR_TOO_MANY_TYPES, TG_ERR_INVALID_ARG (NULL). */
tg_status tg_pa_layout(int32_t L, tg_pa_layout_t *out);

/* The smallest labelling of position-aware class `rank` of global block
 * `block`: types_out[0..k-1] (host, k = 2, 3 or 4 nodes of the numbered
 * shape).  Pure host function.  Errors: TG_ERR_TOO_MANY_TYPES,
 * TG_ERR_INVALID_ARG (block, rank, NULL). */
tg_status tg_pa_labelling(int32_t L, int32_t block, int64_t rank, int32_t *types_out);

/* The global slot (class) counted by per-edge slot `slot` of an edge whose
 * endpoints have types phi_lo (the smaller caller id) and phi_hi: the
 * position-aware typed graphlet of the instances that slot counts; slot =
 * S_pa(L) gives the class of the edge itself (block 0).  *class_out (host)
 * receives the global slot.  Pure host function.  Errors:
 * TG_ERR_TOO_MANY_TYPES, TG_ERR_INVALID_ARG (types, slot, NULL). */
tg_status tg_pa_slot_class(int32_t L, int32_t phi_lo, int32_t phi_hi, int64_t slot, int64_t *class_out);

/* Position-aware counts of every graph of the handle: per_edge_out uint32
 * [m][S_pa(L)] or NULL; global_out int64 [ngraphs][G_pa(L)] or NULL (each
 * class's instances: the per-edge sums divided by |E(H)|, Sec. 6).  Host
 * or device buffers.  The gathering passes are those of tg_count (k = 4);
 * only the per-edge epilogue differs.  Errors: TG_ERR_INVALID_ARG,
 * TG_ERR_OOM, TG_ERR_CUDA (device-detected errors go to the status word). */
tg_status tg_count_position_aware(tg_graph *g, uint32_t *per_edge_out, int64_t *global_out, void *stream);

/* Batched form: counts every graph of a batch handle with the whole
 * sequence of kernels captured once into a CUDA graph and replayed on later
 * calls with the same (k, per_edge_out, global_out, stream).  Results are
 * identical to tg_count. */
tg_status tg_count_batch(tg_graph *g, int32_t k, uint32_t *per_edge_out, int64_t *global_out,
                         void *stream);

/* The list form of the batched call (Problem 2 for several graphs the
 * caller already holds as handles): counts handles gs[0..ngraphs-1] (each a
 * single graph or a batch, any L) on one stream, global totals only, into
 * global_out int64 (host or device): handle h's totals, ngraphs_h *
 * global_slots(L_h, k) values, follow those of handles 0..h-1.  Per-edge
 * rows: call tg_count per handle.  Device-detected errors go to each
 * handle's status word (tg_query_status).  Errors: TG_ERR_INVALID_ARG
 * (NULL, k, ngraphs < 0), TG_ERR_OOM, TG_ERR_CUDA. */
tg_status tg_count_handles(tg_graph *const *gs, int32_t ngraphs, int32_t k, int64_t *global_out, void *stream);

/* Synchronises the handle's last stream and returns the first error
 * recorded in its device status word (TG_OK if none), then clears it. */
tg_status tg_query_status(tg_graph *g);

/* Static description of a status code. */
const char *tg_status_string(tg_status s);

/* Text of the calling host thread's most recent failed call into this
 * library: the failing step and, for TG_ERR_CUDA / TG_ERR_OOM, the CUDA
 * runtime's error string.  Thread-local storage owned by the library; valid
 * until the thread's next failed call; "" if none failed yet.  Diagnostic
 * only (the paper has no counterpart). */
const char *tg_last_error(void);

/* Number of this library's own kernel launches (not counting the CUB
 * primitives the build sorts with) issued by the last tg_build /
 * tg_build_batch, tg_count, tg_count_range or tg_count_batch call on this
 * handle (a CUDA-graph replay counts its kernels). */
int64_t tg_last_launch_count(const tg_graph *g);

/* Per-kernel timing.  While enabled, every kernel that tg_count or
 * tg_count_range launches is bracketed by a CUDA event pair recorded on the
 * launching stream, and the elapsed times are accumulated per kernel name.
 * (Not recorded inside tg_count_batch's captured graph.) */
tg_status tg_set_timing(tg_graph *g, int32_t on);

/* Synchronises the handle's stream and reports the accumulated timing:
 * up to `max` entries of kernel name (static string), total milliseconds and
 * launch count; *n receives the number of entries.  Then clears it. */
tg_status tg_get_timing(tg_graph *g, int32_t max, const char **names, double *ms, int64_t *launches,
                        int32_t *n);

/* ---------------------------------------------------------------------
 * Directed typed 3-node graphlets (Sec. 4.8: every typed set split into
 * typed out-neighbours Gamma^{t,+} and in-neighbours Gamma^{t,-}).
 *
 * Input: an oriented graph -- arcs u -> v as an out-neighbour CSR
 * (out_row_ptr int64 [n+1], out_col int32 [n_arcs], rows in any order),
 * node types uint8 [n] in [0, L).  The split is a partition, so a graph
 * with a reciprocal pair (u -> v and v -> u), a repeated arc or a
 * self-loop is rejected (TG_ERR_INVALID_GRAPH).  Host or device pointers;
 * the handle keeps its own copies.
 *
 * Edges are those of the underlying undirected graph, numbered like
 * tg_build's (lexicographic (u, v), u < v, caller ids).  For edge {i, j},
 * i < j, and each third node w, the sign of w at an endpoint is + when the
 * endpoint is the tail of the arc between them.  Per edge, 8L uint32 slots,
 * block b at b*L + t (t = type of w):
 *   0 S_i^{t,+}  1 S_i^{t,-}  2 S_j^{t,+}  3 S_j^{t,-}
 *   4 T^t(+,+)   5 T^t(+,-)   6 T^t(-,+)   7 T^t(-,-)   (sign at i, sign at j)
 * (S_i excludes j, S_j excludes i, as for the undirected counts.)
 * Global, int64: block 0, directed typed edges, L*L slots at
 * tail_type*L + head_type; block 1, one slot per connected directed typed
 * 3-node graphlet (isomorphism class).  A configuration on nodes 0, 1, 2 is
 * the code (t0, t1, t2, a01, a02, a12), a_xy = 0 no arc, 1 x -> y, 2 y -> x,
 * read as one integer in mixed radix (L, L, L, 3, 3, 3); a class is
 * represented by the smallest code over the 6 renumberings of the nodes,
 * and classes are ranked by that code.  Their number is
 * (20 L^3 + 6 L^2 + 4 L) / 6 (Burnside). */
typedef struct {
    int32_t L;
    int64_t per_edge_slots;           /* 8L */
    int64_t global_slots;             /* L*L + classes */
    int64_t classes;                  /* connected directed typed 3-node graphlets */
} tg_directed_layout_t;

/* Pure host function.  Errors: TG_ERR_TOO_MANY_TYPES, TG_ERR_INVALID_ARG. */
tg_status tg_directed_layout(int32_t L, tg_directed_layout_t *out);

/* Representative configuration of class `rank`: types3[3] and arcs3[3]
 * (host; arc states of pairs (0,1), (0,2), (1,2)).  Pure host function.
 * Errors: TG_ERR_TOO_MANY_TYPES, TG_ERR_INVALID_ARG (rank, NULL). */
tg_status tg_directed_class_code(int32_t L, int64_t rank, int32_t *types3, int32_t *arcs3);

/* Builds a handle for directed counting from an oriented graph (above).
 * Stream-ordered; synchronises to validate.  Errors: TG_ERR_INVALID_ARG,
 * TG_ERR_TOO_MANY_TYPES, TG_ERR_INVALID_GRAPH, TG_ERR_TOO_LARGE,
 * TG_ERR_OOM, TG_ERR_CUDA.  The handle also serves tg_count and the other
 * undirected calls, on the underlying undirected graph. */
tg_status tg_build_directed(int64_t n, int64_t n_arcs, const int64_t *out_row_ptr, const int32_t *out_col,
                            const uint8_t *node_types, int32_t L, const tg_options *opt, void *stream,
                            tg_graph **out);

/* Directed typed 3-node counts of a tg_build_directed handle: per_edge_out
 * uint32 [m][8L] (may be NULL), global_out int64 [global_slots] (may be
 * NULL); host or device.  Device-detected errors through tg_query_status.
 * Errors: TG_ERR_INVALID_ARG (not a directed handle), TG_ERR_OOM,
 * TG_ERR_CUDA. */
tg_status tg_count_directed3(tg_graph *g, uint32_t *per_edge_out, int64_t *global_out, void *stream);

/* ---------------------------------------------------------------------
 * Edge-typed typed 3-node graphlets (Def. 1's edge types xi; Defs. 4-5: the
 * class of a typed graphlet is its shape with the multisets of its node
 * types and of its edge types).
 *
 * Input: the symmetric CSR of tg_build plus edge_types (uint8, one per
 * entry of col, in [0, X)); the two entries of an edge must carry the same
 * type.  1 <= X <= TG_MAX_EDGE_TYPES.  Host or device pointers.
 *
 * Edges are numbered like tg_build's.  For edge {i, j} and each third node
 * w of type t, per edge uint32 slots:
 *   [0, L*X)       3-paths: slot t*X + x, x the type of w's edge to i (w in
 *                  S_i) or to j (w in S_j) -- the path's class is the same;
 *   [L*X, S)       triangles: slot L*X + t*P + rank(x, y), P = X(X+1)/2,
 *                  {x, y} the types of w's edges to i and j, ranked as a
 *                  sorted pair over [0, X) in lexicographic order.
 * Global, int64, three blocks: edges (multisets of 2 node types x X edge
 * types: rank2*X + xi), 3-paths (multisets of 3 node types x multisets of
 * 2 edge types: rank3*C(X+1,2) + rank2), triangles (multisets of 3 node
 * types x multisets of 3 edge types: rank3*C(X+2,3) + rank3); multisets
 * sorted and ranked lexicographically; each instance counted once. */
#define TG_MAX_EDGE_TYPES 4

typedef struct {
    int32_t L, X;
    int64_t per_edge_slots;           /* L*X + L*X*(X+1)/2 */
    int64_t triangle_offset;          /* L*X */
    int64_t global_slots;
    int64_t global_block_offset[3];   /* edges, 3-paths, triangles */
    int64_t global_block_size[3];
} tg_edge_typed_layout_t;

/* Pure host function.  Errors: TG_ERR_TOO_MANY_TYPES (L or X), TG_ERR_INVALID_ARG. */
tg_status tg_edge_typed_layout(int32_t L, int32_t X, tg_edge_typed_layout_t *out);

/* Builds a handle for edge-typed counting (above).  Stream-ordered;
 * synchronises to validate.  Errors: TG_ERR_INVALID_ARG,
 * TG_ERR_TOO_MANY_TYPES, TG_ERR_INVALID_GRAPH (tg_build's checks, an edge
 * type out of range or different on an edge's two entries),
 * TG_ERR_TOO_LARGE, TG_ERR_OOM, TG_ERR_CUDA.  The handle also serves
 * tg_count and the other node-typed calls. */
tg_status tg_build_edge_typed(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                              const uint8_t *node_types, const uint8_t *edge_types, int32_t L, int32_t X,
                              const tg_options *opt, void *stream, tg_graph **out);

/* Edge-typed 3-node counts of a tg_build_edge_typed handle: per_edge_out
 * uint32 [m][per_edge_slots] (may be NULL), global_out int64
 * [global_slots] (may be NULL); host or device.  Device-detected errors
 * through tg_query_status.  Errors: TG_ERR_INVALID_ARG (not an edge-typed
 * handle), TG_ERR_OOM, TG_ERR_CUDA. */
tg_status tg_count_edge_typed3(tg_graph *g, uint32_t *per_edge_out, int64_t *global_out, void *stream);

/* Work counters (diagnostics for the benchmark's roofline; no effect on the
 * counts).  While enabled, the counting kernels add the units of work they
 * did to per-handle counters, slot TG_WORK_*: the set-of-T lookups of the
 * 4-clique scans (one per entry of N+(w) for every member w of T, Alg. 3's
 * 4-clique branch) by the warp-per-edge and CTA-per-edge kernels, the pair
 * searches of edges with few pairs, and the SM clock cycles the CTAs of the
 * hub wedge pass spent waiting for their tickets' dependencies and working
 * on tickets of each kind (fill the counter tables, read them, clear them
 * by walking the wedges, clear them by zeroing), the wedges of the hub
 * anchors and the nonzero 4-cycle slot updates the hub pass made (one per
 * wedge (v, w) and type t of the fourth node with a nonzero count, and one
 * per (hub, v, type) sum).  Off by default. */
#define TG_WORK_CLIQUE_PROBES 0
#define TG_WORK_CLIQUE_SEARCHES 1
#define TG_WORK_CLIQUE_BIG_PROBES 2
#define TG_WORK_HUB_WAIT_CYCLES 3
#define TG_WORK_HUB_FILL_CYCLES 4
#define TG_WORK_HUB_READ_CYCLES 5
#define TG_WORK_HUB_WALK_CLEAR_CYCLES 6
#define TG_WORK_HUB_ZERO_CLEAR_CYCLES 7
#define TG_WORK_HUB_WEDGES 8            /* wedges of the hub anchors (fill tickets) */
#define TG_WORK_HUB_SLOT_UPDATES 9      /* nonzero 4-cycle slot updates of the hub pass */
#define TG_WORK_SLOTS 16
tg_status tg_set_work_counting(tg_graph *g, int32_t on);

/* Synchronises the handle's stream, copies min(n, TG_WORK_SLOTS) counters
 * to out (host, int64; zeros beyond) and clears them. */
tg_status tg_get_work(tg_graph *g, int64_t *out, int32_t n);

/* Typed 3-node counts without any allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- services whose device memory is all owned by their own pool,
 * code running while a CUDA graph is captured (plain cudaMalloc/cudaFree
 * cannot be captured), loops that cannot afford cudaFree's implicit device
 * synchronisation.  It computes what tg_count(k = 3) computes (per-edge rows
 * of 2L uint32: typed 3-paths then typed triangles; global typed edge,
 * 3-path and triangle totals, G(L, 3) int64) straight from a caller CSR, no
 * tg_graph handle.  Arguments: device pointers only (TG_ERR_INVALID_ARG
 * otherwise); rows must be sorted by neighbour id and symmetric (each edge
 * in both rows); per_edge_out, global_out and device_status may be NULL;
 * device_status receives the device-detected error bits OR-ed in, in stream
 * order: non-zero for an invalid graph (unsorted, one-sided or duplicate
 * entries, self-loops, ids or types out of range -- the per-edge rows are
 * then left unwritten) or an internal error.
 * Working memory: one file-scope device array of about 8 MB that every GPU
 * which loads the library keeps until the process exits, shared by all
 * calls; at most 1,048,576 nodes per call (TG_ERR_TOO_LARGE beyond).  The
 * first call on a device looks up that array's device address (set-up); make
 * it before any stream capture.  Calls that overlap on the GPU (other
 * streams, other host threads) race on the shared array: serialise them. */
tg_status tg_count3_static(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                           const uint8_t *node_types, int32_t L, uint32_t *per_edge_out, int64_t *global_out,
                           uint32_t *device_status, void *stream);

/* Library ABI version (TG_ABI_VERSION). */
int32_t tg_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TG_H_ */

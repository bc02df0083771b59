// tg_internal.cuh -- types and helpers shared by the CUDA sources of libtg.
//
// Internal graph layout (all device arrays, built by tg_build):
//   nodes are renumbered by (graph, degree, id) ascending ("priority order"):
//   inside a graph, a larger internal id means a higher degree.  Every
//   adjacency row lists the neighbours sorted by (type, internal id), so the
//   typed neighbourhood Gamma_x^t (Def. 6) is the contiguous segment
//   adj[rp[x] + toff[x*(L+1)+t] .. rp[x] + toff[x*(L+1)+t+1]) and its length
//   is the typed degree d_x^t (Def. 7).
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#include "tg.h"

namespace tg {

// Device status word bits (OR-ed by kernels, read by tg_query_status).
enum : uint32_t {
    ST_INVALID_GRAPH = 1u << 0,
    ST_OVERFLOW = 1u << 1,
    ST_TIMEOUT = 1u << 2,
    ST_INTERNAL = 1u << 3,
    ST_TOO_LARGE = 1u << 4,
};

constexpr int kMaxL = TG_MAX_TYPES;
constexpr int kWarp = 32;
constexpr int kTypeShift = 29;                     // packed (type << 29 | id) sort keys
constexpr int32_t kIdMask = (1 << kTypeShift) - 1;
constexpr int kHeavyCap = 4096;                    // shared-memory hash rows of a heavy anchor
// slots of the optional work counters (tg_set_work_counting; TG_WORK_*)
enum : int { kWorkCliqueProbes = 0, kWorkCliqueSearches = 1, kWorkCliqueBigProbes = 2, kWorkHubWait = 3,
             kWorkHubKind = 4 /* + ticket kind 0..3 */, kWorkHubWedges = 8, kWorkHubSlotUpdates = 9,
             kWorkSlots = 16 };
constexpr int kHeavyFit = kHeavyCap / 4 * 3;       // its load limit (distinct wedge ends)

// Persistent hub pass (tg_count.cu): a group of hubs whose counter tables
// share one table buffer, and the ticket queue as runs of tickets of one
// (group, kind) in queue order; kinds 0 fill, 1 read, 2 clear by walking the
// wedges, 3 clear by zeroing the group's table words.
struct HubGroup {
    int64_t i0, i1;             // items
    int64_t w0, w1;             // wedges
    int64_t tw;                 // wedges per fill / read / walk-clear ticket
    int64_t zwords;             // table words of the group (zeroing tickets: kHubTicketWords each)
    int32_t h0, buf;            // first hub, table buffer
};
struct HubSegment {
    int64_t t0;                 // first ticket of the run
    int32_t group, kind;
};
constexpr int64_t kHubTicketWords = 1 << 16;

// Read-only view of a built graph, passed to kernels by value.
struct GraphView {
    int32_t ngraphs;
    int32_t L;
    int32_t isect_modes;       // tg_options::isect_modes
    int64_t n, nnz, m;
    const int64_t *node_off;   // [ngraphs+1] internal node id ranges per graph
    const int64_t *edge_off;   // [ngraphs+1] edge id ranges per graph
    const int64_t *rp;         // [n+1]
    const int32_t *adj;        // [nnz] internal ids, rows sorted by (type, id)
    const int32_t *toff;       // [n*(L+1)] type segment starts, relative to rp[x]
    const int32_t *pivot;      // [n*L] first slot of segment (x,t) with id > x, relative to rp[x]
    const int32_t *nplus;      // [n] neighbours of higher priority (id > x)
    const uint8_t *ty;         // [n] node type by internal id
    const int32_t *slot_eid;   // [nnz] edge id of each adjacency slot
    const int32_t *e_lo;       // [m] internal endpoint with the smaller id
    const int32_t *e_hi;       // [m] internal endpoint with the larger id
    const int64_t *e_slot_lo;  // [m] slot of e_hi inside row e_lo
    const int64_t *e_slot_hi;  // [m] slot of e_lo inside row e_hi
    const int64_t *delta;      // [n*L*L] sum_{w in Gamma_x^t} d_w^t'
    const int64_t *plus_off;   // [n+1] start of x's higher-priority neighbours in plus_adj
    const int32_t *plus_adj;   // [m] higher-priority neighbours of each node, (type << 29 | id),
                               // grouped by type in (type, id) order
};

// Per-count working arrays.
struct CountView {
    uint32_t *C;                // [m*L]   typed triangle counts c_e^t
    int64_t *tau;               // [n*L*L] ordered typed edges inside Gamma_x
    uint32_t *A;                // [L*L][a_stride] 4-cycle contributions per slot of the current chunk
    int64_t a_base;             // first adjacency slot of the current chunk
    int64_t a_stride;           // slots per type-pair row of A
    int64_t e_base;             // first edge of the current range (per-edge arrays are relative to it)
    int64_t *toffs;             // [edges + 1] T list offsets of the range
    int32_t *tlist;             // T lists of the range, each sorted by (type, id)
    unsigned long long *tsum;   // [edges][3][L*L] TCi, TCj, DT
    unsigned long long *kmat;   // [edges][L*L] adjacent pairs inside T, (smaller id type, larger id type)
    uint32_t *tables;           // dense per-CTA wedge tables
    int64_t table_stride;       // entries (uint32) per CTA table
    unsigned long long *gacc;   // [ngraphs*G] raw per-graphlet edge sums
    uint32_t *status;           // device status word
    unsigned long long *work;   // [kWorkSlots] work counters, or nullptr (counting off)
};

__host__ __device__ inline int64_t npairs(int L) { return (int64_t)L * (L + 1) / 2; }

__host__ __device__ inline int64_t binom_small(int64_t a, int64_t b) {
    if (b < 0 || a < b) return 0;
    int64_t r = 1;
    for (int64_t k = 1; k <= b; ++k) r = r * (a - b + k) / k;
    return r;
}

__host__ __device__ inline int64_t per_edge_slots(int L, int k) {
    return k == 3 ? 2 * (int64_t)L : 2 * (int64_t)L + 10 * npairs(L);
}

__host__ __device__ inline int64_t global_slots(int L, int k) {
    int64_t g = binom_small(L + 1, 2) + 2 * binom_small(L + 2, 3);
    if (k == 4) g += 6 * binom_small(L + 3, 4);
    return g;
}

// first index in [lo, hi) with a[idx] >= key (a sorted ascending)
// First position in a[lo, hi) (sorted) whose value is >= key, else hi.
// Branch-free halving of a 32-bit length (ceil(log2(hi - lo)) steps, the
// same for every lane searching a segment of the same length).
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *__restrict__ a, int64_t lo, int64_t hi,
                                                   int32_t key) {
    if (hi <= lo) return lo;
    const int32_t *base = a + lo;
    uint32_t n = (uint32_t)(hi - lo);
    while (n > 1) {
        const uint32_t half = n >> 1;
        base = __ldg(base + half) < key ? base + half : base;
        n -= half;
    }
    return (base - a) + (__ldg(base) < key ? 1 : 0);
}

// Typed set intersection of two sorted, duplicate-free segments A =
// adj[sa, ea) and B = adj[sb, eb), |A| <= |B|, by one warp.  fn(found, s,
// r, w) is called by every lane once per round (warp-uniform): lane s's
// entry w = adj[s] of A, found in B at r when `found`.  Rounds visit A's
// entries in order, so the found entries come out sorted.
//   binary: 32 entries of A per round, each searched in B (ceil(log2 |B|)
//           dependent loads);
//   merge:  a window of 32 entries of A against a window of 32 of B per
//           round (both loads coalesced), each A entry searched in the B
//           window by shuffles; the window with the smaller last entry
//           moves on (both when equal), so an equal pair always meets.
// isect_use_merge picks per bucket of |A| (tg_options::isect_modes); binary
// search unless a bucket asks for merge or for the dependent-load count.
__device__ __forceinline__ bool isect_use_merge(int32_t modes, int64_t a, int64_t b) {
    const int bucket = a < 32 ? 0 : (a < 128 ? 1 : (a < 512 ? 2 : 3));
    const int mode = (modes >> (2 * bucket)) & 3;
    if (mode != 3) return mode == 2;                        // 0 (default) and 1: binary search
    const int64_t lg = 64 - __clzll((unsigned long long)(b > 2 ? b - 1 : 1));   // ceil(log2 b)
    return (a + b + 31) / 32 < ((a + 31) / 32) * lg;                            // dependent-load rounds
}

template <class F>
__device__ __forceinline__ void isect_merge(const int32_t *__restrict__ adj, int64_t sa, int64_t ea, int64_t sb,
                                            int64_t eb, int lane, F fn) {
    int64_t pa = sa, pb = sb;
    while (pa < ea && pb < eb) {                            // warp-uniform
        const int64_t ia = pa + lane, ib = pb + lane;
        const int32_t av = ia < ea ? __ldg(adj + ia) : INT32_MAX;
        const int32_t bv = ib < eb ? __ldg(adj + ib) : INT32_MAX;
        const int na = (int)(ea - pa < 32 ? ea - pa : 32), nb = (int)(eb - pb < 32 ? eb - pb : 32);
        const int32_t alast = __shfl_sync(0xffffffffu, av, na - 1);
        const int32_t blast = __shfl_sync(0xffffffffu, bv, nb - 1);
        int k = 0;                                          // last B entry <= av (B window in registers)
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int32_t c = __shfl_sync(0xffffffffu, bv, k + st);
            if (c <= av) k += st;
        }
        const int32_t bk = __shfl_sync(0xffffffffu, bv, k);
        fn(ia < ea && bk == av, ia, pb + k, av);
        if (alast <= blast) pa += 32;
        if (blast <= alast) pb += 32;
    }
}

template <class F>
__device__ __forceinline__ void isect_binary(const int32_t *__restrict__ adj, int64_t sa, int64_t ea, int64_t sb,
                                             int64_t eb, int lane, F fn) {
    for (int64_t r0 = sa; r0 < ea; r0 += 32) {
        const int64_t s = r0 + lane;
        bool found = false;
        int64_t r = 0;
        int32_t w = 0;
        if (s < ea) {
            w = adj[s];
            r = lower_bound_i32(adj, sb, eb, w);
            found = r < eb && adj[r] == w;
        }
        fn(found, s, r, w);
    }
}

// kMerge: the kernel was instantiated for options that may ask for merge
// (isect_any_merge); without it only binary search is compiled in.
template <bool kMerge, class F>
__device__ __forceinline__ void isect(const int32_t *__restrict__ adj, int32_t modes, int64_t sa, int64_t ea,
                                      int64_t sb, int64_t eb, int lane, F fn) {
    if (kMerge && isect_use_merge(modes, ea - sa, eb - sb)) isect_merge(adj, sa, ea, sb, eb, lane, fn);
    else isect_binary(adj, sa, ea, sb, eb, lane, fn);
}

__host__ __device__ inline bool isect_any_merge(int32_t modes) {
    for (int b = 0; b < 4; ++b)
        if (((modes >> (2 * b)) & 3) >= 2) return true;
    return false;
}

__device__ __forceinline__ int64_t seg_begin(const GraphView &g, int64_t x, int t) {
    return g.rp[x] + g.toff[x * (g.L + 1) + t];
}

__device__ __forceinline__ int64_t seg_end(const GraphView &g, int64_t x, int t) {
    return g.rp[x] + g.toff[x * (g.L + 1) + t + 1];
}

__device__ __forceinline__ int32_t typed_degree(const GraphView &g, int64_t x, int t) {
    const int32_t *o = g.toff + x * (g.L + 1);
    return o[t + 1] - o[t];
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bits) {
    atomicOr(status, bits);
}

// graph index of an internal node id (binary search over node_off)
__device__ __forceinline__ int graph_of_node(const GraphView &g, int64_t x) {
    int lo = 0, hi = g.ngraphs;          // node_off[lo] <= x < node_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (g.node_off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int graph_of_edge(const GraphView &g, int64_t e) {
    int lo = 0, hi = g.ngraphs;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (g.edge_off[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace tg

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
enum : int { kWorkCliqueProbes = 0, kWorkCliqueSearches = 1, kWorkCliqueBigProbes = 2, kWorkSlots = 8 };
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

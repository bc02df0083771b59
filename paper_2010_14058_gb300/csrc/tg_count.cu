// tg_count.cu -- per-edge typed 3- and 4-node graphlet counts and global totals.
//
// The GPU path computes, for every edge e = (i,j) (i the endpoint with the
// smaller internal id, types p = phi_i, q = phi_j), the same numbers as
// Alg. 1-3 + Lemmas 1-4 of the paper, but it never scans Gamma_w for every
// w in T u S_i u S_j (that scan costs sum_e sum_{w in U_e} d_w, far too much
// on hub-heavy graphs).  Instead it gathers these typed quantities
// (t = type of the first node, t' = type of the second):
//
//   c[t]        |T_ij^t| (Cor. 1), by typed set intersection       (k_tri)
//   TCi[t][t']  sum_{w in T^t} c_{iw}^{t'}                         (k_tsum)
//   TCj[t][t']  sum_{w in T^t} c_{jw}^{t'}                         (k_tsum)
//   DT[t][t']   sum_{w in T^t} d_w^{t'}                            (k_tsum)
//   K[t][t']    ordered adjacent pairs (w,x) in T^t x T^t' (each pair is found
//               once, from its smaller id, by k_clique / k_clique_big; the
//               epilogue adds the transpose)
//   P[t][t']    3-paths j - w - r - i, w of type t, r of type t'   (k_wedge*)
//   tau_x[t][t'] ordered adjacent pairs inside Gamma_x              (k_tau)
//   delta_x[t][t'] sum_{w in Gamma_x^t} d_w^{t'}                    (build)
//
// and obtains every orbit of Table 3 by the inclusion-exclusion of Thm. 1
// (the sets T, S_i, S_j, I of Cor. 1-2 and Eq. indep-node-set partition
// each neighbourhood):
//   CTi = TCi - K - [t'=q] c_t          (w in T, r in S_i, adjacent)
//   CTj = TCj - K - [t'=p] c_t          (w in T, r in S_j, adjacent)
//   Wi  = tau_i - CTi - CTi^T - K - [t=q] c_t' - [t'=q] c_t   (pairs in S_i)
//   Wj  = tau_j - CTj - CTj^T - K - [t=p] c_t' - [t'=p] c_t   (pairs in S_j)
//   Q   = P - CTj^T - CTi - K           (w in S_j, r in S_i: 4-cycles)
//   Ri  = delta_i - DT - [t=q] d_j^t' - [t'=p] a_t - Wi - CTi^T - Q^T   (S_i to I)
//   Rj  = delta_j - DT - [t=p] d_i^t' - [t'=q] b_t - Wj - CTj^T - Q     (S_j to I)
//   G8  = DT - ([t'=p]+[t'=q]) c_t - K - CTi - CTj                      (T to I)
// then, for t <= t' (X^T is the transpose):
//   g3 = R(+sym), g6 = Q(+sym), g7 = W/2 on the diagonal, g8 = G8(+sym),
//   g10 = CT(+sym), g12 = K/2 on the diagonal; g4, g5, g9, g11 by
//   Lemmas 1-4; global totals by Sec. 4.4 and Sec. 6.
//
// P uses degree-priority wedges: each 4-cycle is found once, from its node
// of highest (degree, id) priority u, as two wedges u - v - w and u - x - w
// with v, w, x all of lower priority; the wedge work is
// sum_{(u,v) in E} min(d_u, d_v).
#include <algorithm>
#include <vector>

#include <cub/device/device_scan.cuh>

#include <mutex>

#include "tg_host.hpp"

namespace tg {

namespace {

constexpr int kAnchorThreads = 512;         // k_wedge_heavy: one anchor per CTA
constexpr int kLightAnchorWarps = 4;        // k_wedge_light: one anchor per warp
constexpr int kTile = 2048;                 // most edges per tile of k_epi4 and k_edge3 (tile_edges)

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// lexicographic rank of a sorted K-multiset over [0,L): the number of
// non-decreasing K-tuples that precede it, counted position by position.
__device__ __forceinline__ int multichoose(int n, int r) {   // C(n + r - 1, r), n >= 1
    int64_t v = 1;
    for (int k = 1; k <= r; ++k) v = v * (n + k - 1) / k;
    return (int)v;
}
__device__ int multiset_rank_dev(int L, int K, const int *s) {
    int r = 0, prev = 0;
    for (int k = 0; k < K; ++k) {
        for (int v = prev; v < s[k]; ++v) r += multichoose(L - v, K - k - 1);
        prev = s[k];
    }
    return r;
}
__device__ __forceinline__ void sort4(int *s) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 3 - a; ++b)
            if (s[b] > s[b + 1]) { int x = s[b]; s[b] = s[b + 1]; s[b + 1] = x; }
}
__device__ __forceinline__ void sort3(int *s) {
    if (s[0] > s[1]) { int x = s[0]; s[0] = s[1]; s[1] = x; }
    if (s[1] > s[2]) { int x = s[1]; s[1] = s[2]; s[2] = x; }
    if (s[0] > s[1]) { int x = s[0]; s[0] = s[1]; s[1] = x; }
}

// global block offsets (block 0 edges, 1 3-path, 2 triangle, 3..8 four-node)
__device__ __forceinline__ int gblock_off(int L, int b) {
    int c2 = multichoose(L, 2), c3 = multichoose(L, 3), c4 = multichoose(L, 4);
    if (b == 0) return 0;
    if (b <= 2) return c2 + (b - 1) * c3;
    return c2 + 2 * c3 + (b - 3) * c4;
}

__device__ __forceinline__ int pair_idx(int L, int t, int u) {   // t <= u
    return t * L - t * (t - 1) / 2 + (u - t);
}

// ------------------------------------------------------------------ k_tri
// Warp per edge: c_e^t = |Gamma_i^t cap Gamma_j^t| (Cor. 1; Thm. 2's O(Delta)).
// Binary search form: the shorter side of every typed pair, concatenated
// over t, is one list of sum_t min(d_i^t, d_j^t) entries that the lanes
// stride over (so the lanes are busy across type boundaries); each entry is
// searched in the other side's segment of its type.  Lane q < L holds type
// q's segments; per round every lane finds its entry's type from the
// prefix ends (in registers) and the segments by shuffles.  Hits are
// counted by type in the 8-bit fields of one register per lane (emptied
// every 255 rounds).  Merge form (isect): one typed pair at a time.
struct TypedPairs {
    int64_t sa, sb;             // lane q < L: start of the shorter / longer type-q segment
    int32_t nb;                 // length of the longer one
    int32_t excl;               // entries of the shorter segments of types < q
    int32_t incl[kMaxL];        // every lane: entries of types <= q, for each q
    int32_t total;              // entries of all shorter segments
};

// the typed pairs of edge (i, j), each side's segment of type q on lane q
__device__ __forceinline__ void typed_pairs(const GraphView &g, int32_t i, int32_t j, int lane, TypedPairs &tp) {
    const int L = g.L;
    int64_t si = 0, sj = 0;
    int32_t di = 0, dj = 0;
    if (lane < L) {
        const int32_t *oi = g.toff + (int64_t)i * (L + 1), *oj = g.toff + (int64_t)j * (L + 1);
        const int32_t a0 = oi[lane], b0 = oj[lane];
        si = g.rp[i] + a0;
        sj = g.rp[j] + b0;
        di = oi[lane + 1] - a0;
        dj = oj[lane + 1] - b0;
    }
    const bool sw = di > dj;
    tp.sa = sw ? sj : si;
    tp.sb = sw ? si : sj;
    const int32_t na = sw ? dj : di;
    tp.nb = sw ? di : dj;
    int32_t inc = na;
#pragma unroll
    for (int s = 1; s < kMaxL; s <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, s);
        if (lane >= s) inc += y;
    }
    tp.excl = inc - na;
#pragma unroll
    for (int q = 0; q < kMaxL; ++q) tp.incl[q] = __shfl_sync(0xffffffffu, inc, q);   // = total for q >= L
    tp.total = tp.incl[kMaxL - 1];
}

template <bool kMerge>
__global__ void __launch_bounds__(256) k_tri(GraphView g, CountView cv) {
    const int lane = threadIdx.x & 31;
    const int L = g.L;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < g.m; e += nw) {
        const int32_t i = g.e_lo[e], j = g.e_hi[e];
        if (kMerge) {
            for (int t = 0; t < L; ++t) {
                int64_t bi = seg_begin(g, i, t), ei = seg_end(g, i, t);
                int64_t bj = seg_begin(g, j, t), ej = seg_end(g, j, t);
                if (ei == bi || ej == bj) {                 // an empty typed segment (warp-uniform)
                    if (lane == 0) cv.C[e * L + t] = 0;
                    continue;
                }
                if (ei - bi > ej - bj) {
                    int64_t x = bi; bi = bj; bj = x;
                    x = ei; ei = ej; ej = x;
                }
                unsigned cnt = 0;
                isect<true>(g.adj, g.isect_modes, bi, ei, bj, ej, lane,
                            [&](bool found, int64_t, int64_t, int32_t) { cnt += found ? 1u : 0u; });
                cnt = warp_sum_u32(cnt);
                if (lane == 0) cv.C[e * L + t] = cnt;
            }
            continue;
        }
        TypedPairs tp;
        typed_pairs(g, i, j, lane, tp);
        unsigned long long acc = 0, kreg = 0;
        int since = 0;
        for (int32_t p0 = 0; p0 < tp.total; p0 += 32) {
            const int32_t p = p0 + lane;
            int t = 0;
#pragma unroll
            for (int q = 0; q < kMaxL - 1; ++q) t += tp.incl[q] <= p ? 1 : 0;
            const int64_t sa = __shfl_sync(0xffffffffu, tp.sa, t);
            const int64_t sb = __shfl_sync(0xffffffffu, tp.sb, t);
            const int32_t nb = __shfl_sync(0xffffffffu, tp.nb, t);
            const int32_t ex = __shfl_sync(0xffffffffu, tp.excl, t);
            if (p < tp.total) {
                const int32_t w = g.adj[sa + (p - ex)];
                const int64_t r = lower_bound_i32(g.adj, sb, sb + nb, w);
                acc += (unsigned long long)(r < sb + nb && g.adj[r] == w) << (8 * t);
            }
            if (++since == 255) {
                for (int q = 0; q < L; ++q) {
                    const unsigned v = __reduce_add_sync(0xffffffffu, (unsigned)(acc >> (8 * q)) & 0xffu);
                    kreg += lane == q ? v : 0u;
                }
                acc = 0;
                since = 0;
            }
        }
        for (int q = 0; q < L; ++q) {
            const unsigned v = __reduce_add_sync(0xffffffffu, (unsigned)(acc >> (8 * q)) & 0xffu);
            kreg += lane == q ? v : 0u;
        }
        if (lane < L) cv.C[e * L + lane] = (uint32_t)kreg;
    }
}

// ------------------------------------------------------------------ k_tau
// Warp per node x: tau_x[t][t'] = sum_{w in Gamma_x^t} c_{xw}^{t'}, the
// ordered adjacent pairs inside Gamma_x by type.
__global__ void __launch_bounds__(256) k_tau(GraphView g, CountView cv) {
    const int lane = threadIdx.x & 31;
    const int L = g.L;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; x < g.n; x += nw) {
        for (int t = 0; t < L; ++t) {
            unsigned long long acc[kMaxL];
#pragma unroll
            for (int q = 0; q < kMaxL; ++q) acc[q] = 0;
            for (int64_t s = seg_begin(g, x, t) + lane; s < seg_end(g, x, t); s += 32) {
                const uint32_t *c = cv.C + (int64_t)g.slot_eid[s] * L;
#pragma unroll
                for (int q = 0; q < kMaxL; ++q)
                    if (q < L) acc[q] += c[q];
            }
#pragma unroll
            for (int q = 0; q < kMaxL; ++q) {
                if (q >= L) break;
                unsigned long long v = warp_sum_u64(acc[q]);
                if (lane == 0) cv.tau[(x * L + t) * L + q] = (int64_t)v;
            }
        }
    }
}

// ------------------------------------------------------------ wedge kernels
// For an anchor u, V_u = {v in Gamma_u : v < u} and, for v in V_u, the
// wedge ends {w in Gamma_v : w < u}.  Phase 1 counts, per wedge end w and
// per type t of the middle node, the wedges u - v - w (table H_u[w][t]).
// Phase 2 revisits every wedge u - v - w: the other middles x of (u,w) of
// type t number cnt_t = H_u[w][t] - [phi_v = t]; each closes the 4-cycle
// u - v - w - x - u, which is recorded on
//   slot (v -> w): A[phi_u][t]   (v's other cycle neighbour u, w's is x)
//   slot (u -> v): A[t][phi_w]   (u's other cycle neighbour x, v's is w).
// A[s][t] of a slot (a -> b) counts 4-cycles a - b - y - z - a with
// phi_z = s (a's other neighbour) and phi_y = t (b's other neighbour).

// cut of typed segment (x, t) at id < bound
__device__ __forceinline__ void seg_prefix(const GraphView &g, int64_t x, int t, int32_t bound, int64_t &b,
                                           int64_t &cut) {
    b = seg_begin(g, x, t);
    cut = lower_bound_i32(g.adj, b, seg_end(g, x, t), bound);
}

__device__ __forceinline__ int hash_slot(int32_t w, int cap) {
    return (int)(((uint32_t)w * 2654435761u) & (uint32_t)(cap - 1));
}

// open addressing in shared memory; returns the slot or -1 when full
__device__ int hash_insert(int32_t *keys, int cap, int32_t w) {
    int h = hash_slot(w, cap);
    for (int probe = 0; probe < cap; ++probe) {
        int32_t k = keys[h];
        if (k == w) return h;
        if (k == -1) {
            int32_t old = atomicCAS(&keys[h], -1, w);
            if (old == -1 || old == w) return h;
        }
        h = (h + 1) & (cap - 1);
    }
    return -1;
}
__device__ int hash_find(const int32_t *keys, int cap, int32_t w) {
    int h = hash_slot(w, cap);
    for (int probe = 0; probe < cap; ++probe) {
        int32_t k = keys[h];
        if (k == w) return h;
        if (k == -1) return -1;
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

// ------------------------------------------------------------ wedges of one v
// The wedges u - v - w (v, w below the anchor u) of one neighbour v, all
// types of w flattened: lane t < L finds the part of v's type-t segment
// below u (one binary search per lane, in parallel) and its exclusive
// offset; wedge p of v then has type tw = the last lane t whose offset is
// <= p, and lanes take 32 wedges at a time whatever their types.
struct VRuns {
    int64_t b;          // lane t < L: first slot of type t in v's row
    int32_t off;        // lane t < L: wedges of types < t (total on lanes >= L)
    int32_t total;      // wedges of v
};

__device__ __forceinline__ VRuns v_runs(const GraphView &g, int32_t v, int32_t u, int lane) {
    VRuns r;
    r.b = 0;
    int32_t n = 0;
    if (lane < g.L) {
        int64_t cut;
        seg_prefix(g, v, lane, u, r.b, cut);
        n = (int32_t)(cut - r.b);
    }
    int32_t inc = n;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    r.off = inc - n;
    r.total = __shfl_sync(0xffffffffu, inc, kMaxL - 1);
    return r;
}

// per-(v, type of w) sums of phase 1 over the lanes (runs of equal tw are
// contiguous): tail lanes add them to the 4-cycle slot of (u, v)
__device__ __forceinline__ void flush_runs(uint32_t *A, int64_t nnz, int L, const uint32_t *c, int key, int tw,
                                           int64_t sv, int lane) {
    unsigned same = 0;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int kk = __shfl_up_sync(0xffffffffu, key, 1 << s);
        if (lane >= (1 << s) && kk == key) same |= 1u << s;
    }
    const int knext = __shfl_down_sync(0xffffffffu, key, 1);
    const bool tail = key >= 0 && (lane == 31 || knext != key);
#pragma unroll
    for (int t = 0; t < kMaxL; ++t) {
        if (t >= L) break;
        uint32_t v = c[t];
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, 1 << s);
            if (same & (1u << s)) v += y;
        }
        if (tail && v) atomicAdd(&A[(int64_t)(t * L + tw) * nnz + sv], v);
    }
}

// One phase of the wedges of v for one warp.  rows(w, insert) gives w's
// counter row (L entries): phase 0 inserts and adds 1 at t_v; phase 1 adds
// h[w][t] - [t = t_v] to the slot of (v, w) and the per-type sums to the
// slot of (u, v); phase 2 clears the row (dense tables only).
template <class Rows>
__device__ __forceinline__ void wedge_v(const GraphView &g, uint32_t *A, int64_t nnz, int32_t u, int tu, int32_t v,
                                        int tv, int64_t sv, int phase, int lane, Rows rows) {
    const int L = g.L;
    const VRuns r = v_runs(g, v, u, lane);
    for (int32_t p0 = 0; p0 < r.total; p0 += 32) {
        const int32_t p = p0 + lane;
        int tw = 0;
#pragma unroll
        for (int st = kMaxL / 2; st > 0; st >>= 1) {
            const int32_t c = __shfl_sync(0xffffffffu, r.off, tw + st);
            if (c <= p) tw += st;
        }
        const int64_t k = __shfl_sync(0xffffffffu, r.b, tw) + (p - __shfl_sync(0xffffffffu, r.off, tw));
        const bool act = p < r.total;
        uint32_t c[kMaxL];
#pragma unroll
        for (int t = 0; t < kMaxL; ++t) c[t] = 0;
        if (act) {
            const int32_t w = g.adj[k];
            uint32_t *row = rows(w, phase == 0);
            if (row) {
                if (phase == 0) {
                    atomicAdd(row + tv, 1u);
                } else if (phase == 1) {
#pragma unroll
                    for (int t = 0; t < kMaxL; ++t) {
                        if (t >= L) break;
                        const uint32_t x = row[t] - (t == tv ? 1u : 0u);
                        c[t] = x;
                        if (x) atomicAdd(&A[(int64_t)(tu * L + t) * nnz + k], x);
                    }
                } else {
                    for (int t = 0; t < L; ++t) row[t] = 0;
                }
            }
        }
        if (phase == 1) flush_runs(A, nnz, L, c, act ? tw : -1, tw, sv, lane);
    }
}

// lower-priority neighbours of u by type: lane t < L gets the first slot
// of type t and the exclusive offset of its part; returns their number
__device__ __forceinline__ int32_t u_runs(const GraphView &g, int32_t u, int lane, int64_t &ub, int32_t &uoff) {
    int32_t n = 0;
    ub = 0;
    if (lane < g.L) {
        int64_t cut;
        seg_prefix(g, u, lane, u, ub, cut);
        n = (int32_t)(cut - ub);
    }
    int32_t inc = n;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    uoff = inc - n;
    return __shfl_sync(0xffffffffu, inc, kMaxL - 1);
}

// neighbour number kv of u's lower-priority neighbours -> (slot, type)
__device__ __forceinline__ int64_t u_slot(int64_t ub, int32_t uoff, int32_t kv, int &tv) {
    tv = 0;
#pragma unroll
    for (int st = kMaxL / 2; st > 0; st >>= 1) {
        const int32_t c = __shfl_sync(0xffffffffu, uoff, tv + st);
        if (c <= kv) tv += st;
    }
    return __shfl_sync(0xffffffffu, ub, tv) + (kv - __shfl_sync(0xffffffffu, uoff, tv));
}

// Light anchors (few wedges): one warp per anchor, table in shared memory
// (a hash of capacity `cap` >= 2 x the anchor's wedges).
__global__ void __launch_bounds__(kLightAnchorWarps * 32) k_wedge_light(GraphView g, CountView cv,
                                                                        const int32_t *__restrict__ anchors,
                                                                        int64_t n_anchors, int cap, int64_t n0,
                                                                        int64_t n1) {
    extern __shared__ int32_t smem[];
    const int L = g.L;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *keys = smem + wid * cap * (1 + L);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(keys + cap);
    for (int k = lane; k < cap; k += 32) keys[k] = -1;
    for (int k = lane; k < cap * L; k += 32) cnt[k] = 0;
    __syncwarp();
    const int64_t nw = (int64_t)gridDim.x * kLightAnchorWarps;
    const int64_t nnz = cv.a_stride;
    uint32_t *A = cv.A - cv.a_base;                          // indexed by absolute slot
    auto rows = [&](int32_t w, bool insert) -> uint32_t * {
        const int h = insert ? hash_insert(keys, cap, w) : hash_find(keys, cap, w);
        if (h < 0) {
            if (insert) set_status(cv.status, ST_INTERNAL);
            return nullptr;
        }
        return cnt + h * L;
    };
    for (int64_t a = (int64_t)blockIdx.x * kLightAnchorWarps + wid; a < n_anchors; a += nw) {
        const int32_t u = anchors[a];
        if (u < n0 || u >= n1) continue;                    // anchor outside this chunk
        const int tu = g.ty[u];
        int64_t ub;
        int32_t uoff;
        const int32_t nV = u_runs(g, u, lane, ub, uoff);
        for (int phase = 0; phase < 2; ++phase) {
            for (int32_t kv = 0; kv < nV; ++kv) {
                int tv;
                const int64_t sv = u_slot(ub, uoff, kv, tv);
                wedge_v(g, A, nnz, u, tu, g.adj[sv], tv, sv, phase, lane, rows);
            }
            __syncwarp();
        }
        for (int k = lane; k < cap; k += 32) keys[k] = -1;
        for (int k = lane; k < cap * L; k += 32) cnt[k] = 0;
        __syncwarp();
    }
}

// Heavy anchors: one CTA per anchor, warps over the anchor's lower-priority
// neighbours v.  The rows h[w][.] live in a shared-memory hash of kHeavyCap
// entries.  Anchors with more wedges than 3/4 of it go to a dense node table
// in global memory (cleared again by phase 2): on power-law graphs their
// wedge ends are almost all distinct.  Only the first n_tables CTAs own a
// table (the budget of anchor_table_budget_mb); the grid may be larger, and
// the CTAs without a table take hash anchors only.

__device__ int hash_insert_bounded(int32_t *keys, int cap, int32_t w, int *fill, int limit) {
    int h = hash_slot(w, cap);
    for (int probe = 0; probe < cap; ++probe) {
        int32_t k = keys[h];
        if (k == w) return h;
        if (k == -1) {
            if (atomicAdd(fill, 1) >= limit) return -1;     // over the load limit
            const int32_t old = atomicCAS(&keys[h], -1, w);
            if (old == -1) return h;
            atomicSub(fill, 1);
            if (old == w) return h;
        }
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

__global__ void __launch_bounds__(kAnchorThreads, 2) k_wedge_heavy(GraphView g, CountView cv,
                                                               const int32_t *__restrict__ anchors,
                                                               int64_t n_anchors, int64_t n_dense, int64_t n_tables,
                                                               int64_t n0, int64_t n1) {
    extern __shared__ int32_t hsm[];
    __shared__ int s_fill, s_over;
    const int L = g.L;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    int32_t *keys = hsm;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(hsm + kHeavyCap);
    const bool has_table = blockIdx.x < n_tables;
    uint32_t *tbl = cv.tables + (int64_t)(has_table ? blockIdx.x : 0) * cv.table_stride;
    // a CTA without a dense table never falls back to one: its hash anchors
    // have at most kHeavyFit distinct wedge ends, and with the limit at the
    // capacity the fill count (distinct ends plus at most one in-flight
    // insert per thread) cannot reach it
    const int limit = has_table ? kHeavyFit : kHeavyCap - 1;
    const int64_t nnz = cv.a_stride;
    uint32_t *A = cv.A - cv.a_base;                          // indexed by absolute slot
    // pass 0: the first n_dense anchors (more wedges than the hash's load
    // limit, sorted first) against the dense tables, by the CTAs that own
    // one; pass 1: the other anchors against the shared-memory hash, by all
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t a_end = pass == 0 ? (has_table ? n_dense : 0) : n_anchors;
        const int64_t a_step = pass == 0 ? n_tables : gridDim.x;
        for (int64_t a = (pass == 0 ? 0 : n_dense) + blockIdx.x; a < a_end; a += a_step) {
            const int32_t u = anchors[a];
            if (u < n0 || u >= n1) continue;                // anchor outside this chunk (uniform per CTA)
            const int tu = g.ty[u];
            const int64_t base = g.node_off[graph_of_node(g, u)];
            const bool pre_dense = pass == 0;
            if (!pre_dense) {
                for (int k = threadIdx.x; k < kHeavyCap; k += blockDim.x) keys[k] = -1;
                for (int k = threadIdx.x; k < kHeavyCap * L; k += blockDim.x) cnt[k] = 0;
            }
            if (threadIdx.x == 0) { s_fill = 0; s_over = pre_dense ? 1 : 0; }
            __syncthreads();
            int64_t ub;
            int32_t uoff;
            const int32_t nV = u_runs(g, u, lane, ub, uoff);
            auto hash_rows = [&](int32_t w, bool insert) -> uint32_t * {
                int h;
                if (insert) {
                    h = hash_insert_bounded(keys, kHeavyCap, w, &s_fill, limit);
                    if (h < 0) { s_over = 1; return nullptr; }
                } else {
                    h = hash_find(keys, kHeavyCap, w);
                    if (h < 0) return nullptr;
                }
                return cnt + h * L;
            };
            auto dense_rows = [&](int32_t w, bool) -> uint32_t * { return tbl + (int64_t)(w - base) * L; };
            if (!pre_dense) {
                for (int32_t kv = wid; kv < nV; kv += nwarp) {
                    int tv;
                    const int64_t sv = u_slot(ub, uoff, kv, tv);
                    wedge_v(g, A, nnz, u, tu, g.adj[sv], tv, sv, 0, lane, hash_rows);
                }
                __syncthreads();
            }
            const bool dense = s_over != 0;                 // uniform after the barrier
            if (dense && !has_table) {                      // excluded above; reported, never miscounted
                if (threadIdx.x == 0) set_status(cv.status, ST_INTERNAL);
                __syncthreads();
                continue;
            }
            if (dense)
                for (int32_t kv = wid; kv < nV; kv += nwarp) {
                    int tv;
                    const int64_t sv = u_slot(ub, uoff, kv, tv);
                    wedge_v(g, A, nnz, u, tu, g.adj[sv], tv, sv, 0, lane, dense_rows);
                }
            __syncthreads();
            for (int phase = 1; phase < (dense ? 3 : 2); ++phase) {
                for (int32_t kv = wid; kv < nV; kv += nwarp) {
                    int tv;
                    const int64_t sv = u_slot(ub, uoff, kv, tv);
                    if (dense) wedge_v(g, A, nnz, u, tu, g.adj[sv], tv, sv, phase, lane, dense_rows);
                    else wedge_v(g, A, nnz, u, tu, g.adj[sv], tv, sv, phase, lane, hash_rows);
                }
                __syncthreads();
            }
        }
    }
}

// ------------------------------------------------------------ hub anchors
// An anchor u with very many wedges (a hub) is counted by the whole GPU at
// once: every CTA works on the wedges of the same few hubs, against one node
// table per hub that all CTAs share, so the tables stay in L2 instead of one
// dense table per CTA streaming through HBM.  The wedges u - v - w (v, w of
// lower priority than u) of every hub are flattened into items, one per
// (hub, v, type of w) with at least one wedge; item_woff is the exclusive
// prefix of the items' wedge counts, so wedge x of the flattened order is
// w = adj[item_vb[it] + x - item_woff[it]] for the item it containing x.
// The counts are the same as k_wedge_heavy's: phase 0 fills h_u[w][t] (the
// number of type-t neighbours v of u below u that are adjacent to w),
// phase 1 adds h_u[w][t] - [t = t_v] to the 4-cycle slot of (v, w) and the
// per-(v, type of w) sums to the slot of (u, v), phase 2 clears the rows.
// All hubs of a chunk run in one persistent launch (k_wedge_hub below):
// hubs in groups, every (group, phase) cut into tickets, ticket waits on the
// phases it depends on.

struct HubView {
    const int32_t *hubs;        // hub node ids
    const int64_t *hub_base;    // first node of each hub's graph (read when batched)
    const int64_t *woff;        // [n_items + 1] first wedge of each item
    const int4 *item;           // per item: adj position of its first w, adj position of v in the
                                // hub's row, hub index, type of u << 8 | type of v << 4 | type of w
    bool batched;               // several graphs: tables are indexed from each hub's graph's first node
};

constexpr int kHubThreads = 256;

__global__ void k_hub_nv(GraphView g, const int32_t *__restrict__ hubs, int64_t n_hubs, int64_t *nv,
                         int64_t *hub_base) {
    const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h > n_hubs) return;
    if (h == n_hubs) { nv[h] = 0; return; }
    const int32_t u = hubs[h];
    int64_t acc = 0;
    for (int t = 0; t < g.L; ++t) {
        int64_t b, cut;
        seg_prefix(g, u, t, u, b, cut);
        acc += cut - b;
    }
    nv[h] = acc;
    hub_base[h] = g.node_off[graph_of_node(g, u)];
}

// CTA per hub: wedge count of every (v, type of w) of the hub
__global__ void __launch_bounds__(256) k_hub_cnt(GraphView g, const int32_t *__restrict__ hubs, int64_t n_hubs,
                                                 const int64_t *__restrict__ vbase, int32_t *cnt, int64_t *flag,
                                                 int32_t *sv_of, int32_t *hub_of) {
    __shared__ int64_t s_b[kMaxL + 1], s_cnt[kMaxL + 1];
    const int L = g.L;
    for (int64_t h = blockIdx.x; h < n_hubs; h += gridDim.x) {
        const int32_t u = hubs[h];
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t acc = 0;
            for (int t = 0; t < L; ++t) {
                int64_t b, cut;
                seg_prefix(g, u, t, u, b, cut);
                s_b[t] = b;
                s_cnt[t] = acc;
                acc += cut - b;
            }
            s_cnt[L] = acc;
        }
        __syncthreads();
        const int64_t nV = s_cnt[L], base = vbase[h];
        for (int64_t kv = threadIdx.x; kv < nV; kv += blockDim.x) {
            int tv = 0;
            while (tv + 1 < L && s_cnt[tv + 1] <= kv) ++tv;
            const int64_t sv = s_b[tv] + (kv - s_cnt[tv]);
            const int32_t v = g.adj[sv];
            sv_of[base + kv] = (int32_t)sv;
            hub_of[base + kv] = (int32_t)h;
            for (int tw = 0; tw < L; ++tw) {
                int64_t vb, vcut;
                seg_prefix(g, v, tw, u, vb, vcut);
                const int64_t idx = (base + kv) * L + tw;
                cnt[idx] = (int32_t)(vcut - vb);
                flag[idx] = vcut > vb ? 1 : 0;
            }
        }
    }
}

__global__ void k_hub_items(GraphView g, int64_t ni, const int32_t *__restrict__ cnt, const int64_t *__restrict__ pos,
                            const int32_t *__restrict__ sv_of, const int32_t *__restrict__ hub_of,
                            const int32_t *__restrict__ hubs, int4 *item, int64_t *icnt) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= ni) return;
    const int32_t c = cnt[idx];
    if (c == 0) return;
    const int64_t j = pos[idx], kv = idx / g.L;
    const int tw = (int)(idx - kv * g.L);
    const int32_t s = sv_of[kv];
    const int32_t v = g.adj[s];
    const int32_t h = hub_of[kv];
    item[j] = make_int4((int32_t)seg_begin(g, v, tw), s, h, (g.ty[hubs[h]] << 8) | (g.ty[v] << 4) | tw);
    icnt[j] = c;
}

__global__ void k_hub_bounds(int64_t n_hubs, int L, const int64_t *__restrict__ vbase, const int64_t *__restrict__ pos,
                             const int64_t *__restrict__ woff, int64_t *first_item, int64_t *first_wedge) {
    const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h > n_hubs) return;
    const int64_t it = pos[vbase[h] * L];
    first_item[h] = it;
    first_wedge[h] = woff[it];
}

// largest j in [lo, hi) with woff[j] <= x, given woff[lo] <= x < woff[hi];
// a 32-way search by the whole warp
__device__ __forceinline__ int64_t hub_find_item(const int64_t *__restrict__ woff, int64_t lo, int64_t hi, int64_t x,
                                                 int lane) {
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t p = lo + lane * step;
        const unsigned b = __ballot_sync(0xffffffffu, p < hi && woff[p] <= x);
        lo += (int64_t)(31 - __clz(b)) * step;
        hi = min(hi, lo + step);
    }
    const int64_t p = lo + lane;
    const unsigned b = __ballot_sync(0xffffffffu, p < hi && woff[p] <= x);
    return lo + (31 - __clz(b));
}

// One phase of the hub wedge pass over the wedges [x0r, x1r) of one group of
// hubs (items [i0, i1), first hub h0; hub h's table at tbl + (h - h0) *
// stride).  Warp wi of nwi takes one contiguous run of the range, 32 wedges
// at a time, one wedge per lane; the item window of the next 32 wedges is
// loaded while the current ones are worked on.  Counters: kPacked = two
// 16-bit counters per 32-bit word (types 2k and 2k+1; every count is at
// most the hub's degree, below 2^16 when this layout is chosen), else one
// 32-bit counter per type.  The tables are read and cleared at L2
// (ld/st.cg): other CTAs of the same launch update them, so no L1 copy may
// be trusted.
template <bool kPacked, bool kCount>
__device__ void hub_wedges(const GraphView &g, const CountView &cv, const HubView &hv, int64_t i0, int64_t i1,
                           int64_t x0r, int64_t x1r, int32_t h0, uint32_t *tbl, int64_t stride, int phase, int wi,
                           int nwi, int lane) {
    const int L = g.L;
    const int RW = kPacked ? (L + 1) / 2 : L;               // words per table row
    const int64_t per = (((x1r - x0r) + nwi - 1) / nwi + 31) & ~(int64_t)31;
    int64_t x0 = x0r + wi * per;
    const int64_t xe = min(x1r, x0 + per);
    if (x0 >= xe) return;                                   // warp-uniform
    if (kCount && phase == 0 && lane == 0) atomicAdd(&cv.work[kWorkHubWedges], (unsigned long long)(xe - x0));
    const int64_t nnz = cv.a_stride;
    uint32_t *A = cv.A - cv.a_base;                         // indexed by absolute slot
    int64_t j = hub_find_item(hv.woff, i0, i1, x0, lane);
    int64_t wo = j + lane < i1 ? hv.woff[j + lane] : INT64_MAX;
    unsigned long long nupd_run = 0;                        // (work counting) the warp's slot updates
    for (; x0 < xe; x0 += 32) {
        // the wedges x0 .. x0+31 lie in items j .. j+31 (every item is non-empty)
        const int64_t x = x0 + lane;
        const bool act = x < xe;
        int k = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int64_t c = __shfl_sync(0xffffffffu, wo, k + st);
            if (c <= x) k += st;
        }
        const int64_t it = j + k;
        const int64_t wstart = __shfl_sync(0xffffffffu, wo, k);
        const int k31 = __shfl_sync(0xffffffffu, k, 31);
        const int64_t wnext = k31 < 31 ? __shfl_sync(0xffffffffu, wo, k31 < 31 ? k31 + 1 : 31)
                                       : (j + 32 < i1 ? hv.woff[j + 32] : INT64_MAX);
        // first item of the next 32 wedges (the item of x0 + 32), and its window
        const int64_t jn = (wnext <= x0 + 32) ? j + k31 + 1 : j + k31;
        const int64_t won = x0 + 32 < xe && jn + lane < i1 ? hv.woff[jn + lane] : INT64_MAX;
        int32_t svp = 0;
        int tw = 0;
        uint32_t c[kMaxL];
#pragma unroll
        for (int t = 0; t < kMaxL; ++t) c[t] = 0;
        if (act) {
            const int4 rec = hv.item[it];
            const int32_t hh = rec.z;
            const int tv = (rec.w >> 4) & 15;
            tw = rec.w & 15;
            svp = rec.y;
            const int64_t pos = (int64_t)rec.x + (x - wstart);
            const int32_t w = g.adj[pos];
            const int64_t base = hv.batched ? hv.hub_base[hh] : 0;
            uint32_t *row = tbl + (int64_t)(hh - h0) * stride + (w - base) * RW;
            if (phase == 0) {
                if (kPacked) atomicAdd(row + (tv >> 1), 1u << (16 * (tv & 1)));
                else atomicAdd(row + tv, 1u);
            } else if (phase == 1) {
                const int tu = rec.w >> 8;
                uint32_t words[kMaxL];
#pragma unroll
                for (int q = 0; q < kMaxL; ++q) words[q] = q < RW ? __ldcg(row + q) : 0u;
#pragma unroll
                for (int t = 0; t < kMaxL; ++t) {
                    if (t >= L) break;
                    const uint32_t h = kPacked ? (words[t >> 1] >> (16 * (t & 1))) & 0xffffu : words[t];
                    const uint32_t v = h - (t == tv ? 1u : 0u);
                    c[t] = v;
                    if (v) atomicAdd(&A[(int64_t)(tu * L + t) * nnz + pos], v);
                }
            } else {
                for (int q = 0; q < RW; ++q) __stcg(row + q, 0u);
            }
        }
        if (phase == 1) {
            // (work counting) the round's nonzero slot updates: per wedge, then per item sum
            unsigned nupd = 0;                              // (work counting) these 32 wedges' updates, warp-wide
            if (kCount) {
#pragma unroll
                for (int t = 0; t < kMaxL; ++t) nupd += t < L && c[t] ? 1u : 0u;
                nupd = __reduce_add_sync(0xffffffffu, nupd);
            }
            // per-item sums over the lanes of each item (items are contiguous runs of lanes)
            const int64_t key = act ? it : -1;
            const int64_t key0 = __shfl_sync(0xffffffffu, key, 0);
            if (__all_sync(0xffffffffu, !act || key == key0)) {
                // one item: warp sums, added by lane 0 (always active here)
#pragma unroll
                for (int t = 0; t < kMaxL; ++t) {
                    if (t >= L) break;
                    const uint32_t v = __reduce_add_sync(0xffffffffu, c[t]);
                    if (lane == 0 && v) atomicAdd(&A[(int64_t)(t * L + tw) * nnz + svp], v);
                    if (kCount) nupd += v ? 1u : 0u;       // (warp-uniform)
                }
            } else {
                unsigned same = 0;
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    const int64_t kk = __shfl_up_sync(0xffffffffu, key, 1 << s);
                    if (lane >= (1 << s) && kk == key) same |= 1u << s;
                }
                const int64_t knext = __shfl_down_sync(0xffffffffu, key, 1);
                const bool tail = act && (lane == 31 || knext != key);
#pragma unroll
                for (int t = 0; t < kMaxL; ++t) {
                    if (t >= L) break;
                    uint32_t v = c[t];
#pragma unroll
                    for (int s = 0; s < 5; ++s) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, v, 1 << s);
                        if (same & (1u << s)) v += y;
                    }
                    if (tail && v) atomicAdd(&A[(int64_t)(t * L + tw) * nnz + svp], v);
                    if (kCount) nupd += __popc(__ballot_sync(0xffffffffu, tail && v));
                }
            }
            if (kCount) nupd_run += nupd;
        }
        j = jn;
        wo = won;
    }
    if (kCount && lane == 0 && nupd_run) atomicAdd(&cv.work[kWorkHubSlotUpdates], nupd_run);
}

// The hub pass as one persistent launch over a ticket queue.  The hubs are
// cut into groups whose tables fit one of kHubBuffers table buffers; every
// group has four kinds of tickets, each a range of its wedges or table
// words: 0 fill the counters, 1 read them (4-cycle slot updates), 2 clear
// them by walking the wedges again or 3 by zeroing the group's table words.
// A CTA takes the next ticket from a device counter and, before working on
// it, waits until the tickets it needs are done: reading needs the group's
// fills, clearing its reads, and filling the clears of the group that used
// the same buffer before (kHubBuffers groups back).  Tickets are queued so
// that those are a few groups earlier, and a ticket is taken only by a
// running CTA, so every wait ends; each wait is bounded all the same and
// reports TG_ERR_TIMEOUT (the ticket is then skipped but still marked done,
// so no other wait depends on it forever).

constexpr int kHubBuffers = 3;
constexpr int kHubKinds = 4;
constexpr long long kSpinLimit = 1ll << 24;                // polls of 256 ns and more: several seconds

// range of ticket `local` of a (group, kind) run: wedges for kinds 0-2,
// table words of the group's buffer for kind 3
__device__ __forceinline__ void hub_ticket_range(const HubGroup &gr, int kind, int64_t local, int64_t &x0, int64_t &x1) {
    if (kind == 3) {
        x0 = local * kHubTicketWords;
        x1 = min(gr.zwords, x0 + kHubTicketWords);
    } else {
        x0 = gr.w0 + local * gr.tw;
        x1 = min(gr.w1, x0 + gr.tw);
    }
}

__device__ bool wait_done(const unsigned long long *ctr, unsigned long long target, uint32_t *status) {
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (*(volatile const unsigned long long *)ctr >= target) return true;
        if (*(volatile const uint32_t *)status & ST_TIMEOUT) return false;   // another wait ran out: drain
        __nanosleep(256);
    }
    set_status(status, ST_TIMEOUT);
    return false;
}

template <bool kPacked, bool kCount>
__global__ void __launch_bounds__(kHubThreads, 5) k_wedge_hub(GraphView g, CountView cv, HubView hv,
                                                           const HubSegment *__restrict__ segs, int64_t n_segs,
                                                           int64_t n_tickets, const HubGroup *__restrict__ groups,
                                                           const int64_t *__restrict__ ntick,
                                                           unsigned long long *ctr, uint32_t *tables, int64_t buf_words,
                                                           int64_t stride) {
    __shared__ int64_t s_t, s_x0, s_x1;
    __shared__ int s_ok, s_group, s_kind;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned long long *next = ctr;                         // ticket counter
    unsigned long long *done = ctr + 1;                     // [group][kind] tickets done
    long long c0 = 0;                                       // work counting: clock at the ticket's start
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t t = (int64_t)atomicAdd(next, 1ull);
            if (cv.work) c0 = clock64();
            bool ok = true;
            if (t < n_tickets) {
                int64_t lo = 0, hi = n_segs;                // the run holding ticket t: segs[lo].t0 <= t
                while (hi - lo > 1) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (segs[mid].t0 <= t) lo = mid; else hi = mid;
                }
                const HubSegment sg = segs[lo];
                int64_t x0, x1;
                hub_ticket_range(groups[sg.group], sg.kind, t - sg.t0, x0, x1);
                s_x0 = x0;
                s_x1 = x1;
                s_group = sg.group;
                s_kind = sg.kind;
                const int64_t q = sg.group;
                if (sg.kind == 1) {
                    ok = wait_done(&done[q * kHubKinds + 0], (unsigned long long)ntick[q * kHubKinds + 0], cv.status);
                } else if (sg.kind >= 2) {
                    ok = wait_done(&done[q * kHubKinds + 1], (unsigned long long)ntick[q * kHubKinds + 1], cv.status);
                } else if (q >= kHubBuffers) {
                    const int64_t p = q - kHubBuffers;
                    ok = wait_done(&done[p * kHubKinds + 2], (unsigned long long)ntick[p * kHubKinds + 2], cv.status) &&
                         wait_done(&done[p * kHubKinds + 3], (unsigned long long)ntick[p * kHubKinds + 3], cv.status);
                }
                __threadfence();
            }
            if (cv.work) {
                const long long c1 = clock64();
                atomicAdd(&cv.work[kWorkHubWait], (unsigned long long)(c1 - c0));
                c0 = c1;
            }
            s_t = t;
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        const int64_t t = s_t;
        if (t >= n_tickets) break;                          // CTA-uniform
        const int group = s_group, kind = s_kind;
        const int64_t x0 = s_x0, x1 = s_x1;
        const HubGroup gr = groups[group];
        uint32_t *tbl = tables + (int64_t)gr.buf * buf_words;
        if (s_ok) {
            if (kind == 3) {
                for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) __stcg(tbl + x, 0u);
            } else {
                hub_wedges<kPacked, kCount>(g, cv, hv, gr.i0, gr.i1, x0, x1, gr.h0, tbl, stride, kind, wid, nwarp,
                                            lane);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&done[(int64_t)group * kHubKinds + kind], 1ull);
            if (cv.work) atomicAdd(&cv.work[kWorkHubKind + kind], (unsigned long long)(clock64() - c0));
        }
    }
}

// ------------------------------------------------------------ per-edge 4-node
// The per-edge stage runs as three lean warp-per-edge kernels with the
// per-edge intermediates in HBM (all indexed relative to the chunk's first
// edge e_base):
//   k_tsum    T list of the edge (sorted by (type, id)) and the sums TCi, TCj,
//             DT over its triangle nodes;
//   k_clique  K: adjacent pairs inside T (warp per edge; CTA per edge for
//             the edges with |T| above a threshold, collected on the device);
//   k_epi4    every orbit of Table 3 from the gathered sums, one warp per
//             edge with the L x L matrices held one entry per lane and
//             transposed by shuffles; writes the row and the CTA histogram.

__device__ __forceinline__ uint32_t sat32(int64_t v, uint32_t *status) {
    if (v > 0xffffffffll) {
        set_status(status, ST_OVERFLOW);
        return 0xffffffffu;
    }
    return (uint32_t)v;
}

// orbit o (3..12) -> global block of its graphlet (Sec. 4.4)
__device__ __forceinline__ int graphlet_block(int o) {
    switch (o) {
        case 3: case 4: return 3;
        case 5: return 4;
        case 6: return 5;
        case 7: case 8: case 9: return 6;
        case 10: case 11: return 7;
        default: return 8;
    }
}

__device__ void flush_hist(unsigned long long *hist, int G, unsigned long long *gacc, int graph, int gsize, int gr) {
    for (int s = gr; s < G; s += gsize) {
        unsigned long long v = hist[s];
        if (v) atomicAdd(&gacc[(int64_t)graph * G + s], v);
        hist[s] = 0;
    }
}

// the sum of `copies` histograms of one graph into gacc; clears them
__device__ void flush_hist_copies(unsigned long long *hist, int hw, int copies, int G, unsigned long long *gacc,
                                  int graph, int gsize, int gr) {
    for (int s = gr; s < G; s += gsize) {
        unsigned long long v = 0;
        for (int c = 0; c < copies; ++c) {
            v += hist[c * hw + s];
            hist[c * hw + s] = 0;
        }
        if (v) atomicAdd(&gacc[(int64_t)graph * G + s], v);
    }
}

struct Tile {
    int64_t begin, end;
    int32_t graph, pad;
};

__device__ __forceinline__ unsigned long long warp_allsum_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// |T_e| per edge of the chunk (input of the offset scan), and the device
// list of edges whose T is too large for one warp's 4-clique pass.
__global__ void k_tcount(GraphView g, CountView cv, int64_t e0, int64_t e1, int64_t big_t, int64_t *tcount,
                         int32_t *big_list, unsigned long long *big_count) {
    const int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e > e1) return;
    if (e == e1) { tcount[e1 - e0] = 0; return; }
    int64_t c = 0;
    for (int t = 0; t < g.L; ++t) c += cv.C[e * g.L + t];
    tcount[e - e0] = c;
    if (c > big_t) {
        const unsigned long long k = atomicAdd(big_count, 1ull);
        big_list[k] = (int32_t)e;
    }
}

// Warp per edge: T list and the triangle-node sums (Cor. 1; gathers of the
// typed triangle counts of the edges (i,w), (j,w) and of d_w^t').  The
// sums of one type t are held by lane t' (three registers per lane); each
// round of 32 candidates adds the found nodes' terms with one warp
// reduction per (sum, t').  Acc = uint32_t when the maximum degree is below
// 2^16 (every sum here is then below 2^32 and a warp reduction of 32 terms
// below 2^21), else unsigned long long (terms split into 16-bit halves for
// the 32-bit reductions).
__device__ __forceinline__ unsigned long long warp_total(uint32_t v, uint32_t) {
    return __reduce_add_sync(0xffffffffu, v);
}
__device__ __forceinline__ unsigned long long warp_total(uint32_t v, unsigned long long) {
    const unsigned long long lo = __reduce_add_sync(0xffffffffu, v & 0xffffu);
    const unsigned long long hi = __reduce_add_sync(0xffffffffu, v >> 16);
    return lo + (hi << 16);
}

template <class Acc, bool kMerge>
__global__ void __launch_bounds__(256, sizeof(Acc) == 4 ? 6 : 4) k_tsum(GraphView g, CountView cv, int64_t e0,
                                                                        int64_t e1) {
    const int L = g.L, LL = L * L;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = e0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); e < e1; e += nw) {
        const int64_t er = e - e0;
        const int32_t i = g.e_lo[e], j = g.e_hi[e];
        int32_t *tl = cv.tlist + cv.toffs[er];
        unsigned long long *sum = cv.tsum + er * 3 * LL;
        int32_t pos = 0;
        for (int t = 0; t < L; ++t) {
            Acc s1 = 0, s2 = 0, s3 = 0;                     // lane q < L: the sums over T^t for type q
            if (cv.C[e * L + t] != 0) {
                int64_t bi = seg_begin(g, i, t), ei = seg_end(g, i, t);
                int64_t bj = seg_begin(g, j, t), ej = seg_end(g, j, t);
                bool swapped = false;
                if (ei - bi > ej - bj) {
                    int64_t x = bi; bi = bj; bj = x;
                    x = ei; ei = ej; ej = x;
                    swapped = true;
                }
                isect<kMerge>(g.adj, g.isect_modes, bi, ei, bj, ej, lane, [&](bool found, int64_t s, int64_t r,
                                                                                 int32_t w) {
                    const unsigned bal = __ballot_sync(0xffffffffu, found);
                    if (bal == 0) return;                   // warp-uniform
                    const uint32_t *ci = cv.C, *cj = cv.C;
                    const int32_t *o = g.toff;
                    if (found) {
                        tl[pos + __popc(bal & ((1u << lane) - 1u))] = w;
                        ci = cv.C + (int64_t)g.slot_eid[swapped ? r : s] * L;
                        cj = cv.C + (int64_t)g.slot_eid[swapped ? s : r] * L;
                        o = g.toff + (int64_t)w * (L + 1);
                    }
                    pos += __popc(bal);
                    for (int q = 0; q < L; ++q) {
                        const uint32_t v1 = found ? ci[q] : 0u;
                        const uint32_t v2 = found ? cj[q] : 0u;
                        const uint32_t v3 = found ? (uint32_t)(o[q + 1] - o[q]) : 0u;
                        const unsigned long long t1 = warp_total(v1, Acc()), t2 = warp_total(v2, Acc());
                        const unsigned long long t3 = warp_total(v3, Acc());
                        if (lane == q) {
                            s1 += (Acc)t1;
                            s2 += (Acc)t2;
                            s3 += (Acc)t3;
                        }
                    }
                });
            }
            if (lane < L) {
                sum[t * L + lane] = (unsigned long long)s1;
                sum[LL + t * L + lane] = (unsigned long long)s2;
                sum[2 * LL + t * L + lane] = (unsigned long long)s3;
            }
        }
    }
}

// type boundaries of an edge's T list, from its typed triangle counts
// (indices unrolled, so ts[] stays in registers)
__device__ __forceinline__ void t_bounds(const CountView &cv, int L, int64_t e, int32_t *ts) {
    int32_t acc = 0;
#pragma unroll
    for (int q = 0; q <= kMaxL; ++q) {
        ts[q] = acc;
        if (q < L) acc += (int32_t)cv.C[e * L + q];
    }
}

// type of T's member k (0 <= k < |T|): ts[q] = |T| > k for q >= L
__device__ __forceinline__ int type_of_index(const int32_t *ts, int32_t k) {
    int t = 0;
#pragma unroll
    for (int q = 1; q < kMaxL; ++q) t += ts[q] <= k ? 1 : 0;
    return t;
}

// ------------------------------------------------------------- 4-cliques
// K[t][t'] of an edge counts the adjacent pairs (w, x) inside T, w of type
// t and x of type t', each pair once, from its lower-priority node w: x is
// then one of w's higher-priority neighbours N+(w) (a contiguous list of
// (type << 29 | id) entries grouped by type, built once per graph).  So
// every member w of T scans N+(w) and looks each entry up in a set of T:
// sum_{w in T} |N+(w)| lookups.
//
// The set.  Ids are degree ranks, and on power-law graphs the members of T
// and the entries of their N+ lists crowd at the top of the id range: the
// members within B below the largest member tmax (B = 2^13 for a warp's
// edge, 2^15 for a CTA's) take over 98% of the lookups on the graphs
// measured.  When at least 3/4 of the members lie in that window, they are
// a bitmap indexed by tmax - x (one 32-bit shared-memory load per lookup)
// and the members below it a hash set, looked up only by entries between
// the smallest member and the window.  Otherwise all members are in the
// hash set.  The hash set: buckets of 4 slots (one 16-byte load per
// lookup), slots taken in order by atomicCAS, -1 when empty, so a bucket
// whose last slot is empty is not full and a lookup stops there; with at
// least 4 slots per member almost every lookup reads one bucket.  The
// bitmap is all zero between edges: the words of an edge's members are
// cleared after its scan.
// The scan: one whole warp per member, lanes striding over N+(w) (coalesced
// loads, 4 in flight per lane) -- the lists behind almost all lookups are
// tens to thousands of entries long.  A window lookup has no branch; the
// hash lookups (entries between the smallest member and the window, and
// every entry within T's range in the hash form) are taken by the lanes
// that need them, once per round of four, when any lane of the warp
// does.  Only members below the window check for them: N+(w) holds ids
// above w, so a member in the window meets no member below it.  Each lane
// counts its hits by
// type of x in the fields of one register (no warp-wide step inside the
// scan, so a lane's four lookups overlap); the warp sums the fields with
// __reduce_add_sync before any can overflow and when the member type t
// changes (T is sorted by type), and lane q adds the count for x of type q
// to K[t][q].

__device__ __forceinline__ uint32_t t_hash(int32_t x, int lgnb) {      // lgnb >= 1
    return ((uint32_t)x * 2654435761u) >> (32 - lgnb);
}

__device__ __forceinline__ void group_sync(int gsize) {
    if (gsize > 32) __syncthreads(); else __syncwarp();
}

// the members x <= xmax of T (nT distinct ids) in 2^lgnb buckets, built by the group
__device__ void tset_build(const int32_t *T, int32_t nT, int4 *set, int lgnb, int gsize, int gr, int32_t xmax) {
    const int nb = 1 << lgnb;
    int32_t *slot = reinterpret_cast<int32_t *>(set);
    for (int k = gr; k < 4 * nb; k += gsize) slot[k] = -1;
    group_sync(gsize);
    for (int32_t k = gr; k < nT; k += gsize) {
        const int32_t x = T[k];
        if (x > xmax) continue;
        uint32_t b = t_hash(x, lgnb);
        bool done = false;
        for (int probe = 0; probe < nb && !done; ++probe) {   // 4 nb >= 2 nT: a free slot exists
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (!done) done = atomicCAS(&slot[4 * b + q], -1, x) == -1;
            b = (b + 1) & (nb - 1);
        }
    }
    group_sync(gsize);
}

__device__ __forceinline__ bool bucket_has(const int4 &k, int32_t x) {
    return (k.x == x) | (k.y == x) | (k.z == x) | (k.w == x);
}

__device__ __forceinline__ bool tset_has(const int4 *set, int lgnb, int32_t x) {
    uint32_t b = t_hash(x, lgnb);
    int4 k = set[b];
    if (bucket_has(k, x)) return true;
    if (k.w == -1) return false;                            // the bucket is not full
    const int nb = 1 << lgnb;                               // rare: continue in the next buckets
    for (int probe = 1; probe < nb; ++probe) {
        b = (b + 1) & (nb - 1);
        k = set[b];
        if (bucket_has(k, x)) return true;
        if (k.w == -1) return false;
    }
    return false;
}

// buckets for nT members: 4 slots per member when they fit max_slots, else
// 2 (2^lgnb buckets of 4 slots); -1 when even that exceeds max_slots
__device__ __forceinline__ int tset_lgnb(int32_t nT, int max_slots) {
    int lg = 1;
    while ((4 << lg) < 4 * nT) ++lg;
    if ((4 << lg) <= max_slots) return lg;
    lg = 1;
    while ((4 << lg) < 2 * nT) ++lg;
    return (4 << lg) <= max_slots ? lg : -1;
}

// T of one edge: the window bitmap and the hash set
struct TWin {
    const uint32_t *bm;         // bit d: member tmax - d, for d < wbits; word wbits / 32 is zero
    const int4 *set;            // the members below the window (all of them in the hash form)
    int32_t tmax, tmin, lowmax; // lowmax: the largest id the hash set may hold, else -1
    uint32_t wbits;             // the window's width: B, or 0 in the hash form
    uint32_t lowspan;           // ids tmin .. tmin + lowspan - 1 are looked up in the hash set
    int lgnb;
};

// smallest and largest member of T (each type's run is in increasing id order)
__device__ __forceinline__ void t_range(const int32_t *T, const int32_t *ts, int L, int32_t &tmin, int32_t &tmax) {
    tmin = INT32_MAX;
    tmax = -1;
#pragma unroll
    for (int q = 0; q < kMaxL; ++q) {
        if (q < L && ts[q + 1] > ts[q]) {
            tmin = min(tmin, T[ts[q]]);
            tmax = max(tmax, T[ts[q + 1] - 1]);
        }
    }
}

// members of the group (strided by gsize from gr) below the window of B
template <int B>
__device__ __forceinline__ int32_t twin_below(const int32_t *T, int32_t nT, int32_t tmax, int gsize, int gr) {
    int32_t low = 0;
    for (int32_t k = gr; k < nT; k += gsize) low += (uint32_t)(tmax - T[k]) >= (uint32_t)B ? 1 : 0;
    return low;
}

// sets (or, set = false, clears the words of) the window bits of the group's members
template <int B>
__device__ __forceinline__ void twin_bits(const int32_t *T, int32_t nT, int32_t tmax, uint32_t *bm, int gsize, int gr,
                                          bool set) {
    for (int32_t k = gr; k < nT; k += gsize) {
        const uint32_t d = (uint32_t)(tmax - T[k]);
        if (d < (uint32_t)B) {
            if (set) atomicOr(&bm[d >> 5], 1u << (d & 31u));
            else bm[d >> 5] = 0u;
        }
    }
}

// Per-lane hit counters of one warp: field q (F bits of `acc`) counts the
// lane's hits on entries of type q; `since` counts scan rounds (at most 4
// hits per field each) since the fields were last emptied into `kreg`,
// where lane q holds the warp's count for type q.  Two layouts: 6-bit
// fields in 32 bits for L <= 5 (emptied every 15 rounds), 8-bit fields in
// 64 bits otherwise (every 63).  Warp-uniform control flow.
template <class A>
struct CliqueAcc {
    static constexpr int F = sizeof(A) == 4 ? 6 : 8;
    static constexpr int R = ((1 << F) - 1) / 4;
    A acc = 0;
    unsigned long long kreg = 0;
    int since = 0;
    __device__ __forceinline__ void add(bool hit, uint32_t ent) {
        acc += (A)hit << (F * (ent >> kTypeShift));
    }
    __device__ __forceinline__ void add_bit(uint32_t bit, uint32_t ent) {   // bit: 0 or 1
        acc += (A)bit << (F * (ent >> kTypeShift));
    }
    __device__ __forceinline__ void drain(int L) {
        for (int q = 0; q < L; ++q) {
            const unsigned v = __reduce_add_sync(0xffffffffu, (unsigned)(acc >> (F * q)) & ((1u << F) - 1u));
            kreg += (threadIdx.x & 31) == (unsigned)q ? (unsigned long long)v : 0ull;
        }
        acc = 0;
        since = 0;
    }
};

// lanes q < L add the warp's counts to K[tw][q]
template <class A>
__device__ __forceinline__ void flush_k(CliqueAcc<A> &a, int tw, unsigned long long *K, int L, int lane, bool shared_k) {
    a.drain(L);
    if (tw >= 0 && lane < L && a.kreg) {
        if (shared_k) atomicAdd(&K[tw * kMaxL + lane], a.kreg);
        else K[tw * kMaxL + lane] += a.kreg;
    }
    a.kreg = 0;
}

// one lookup of entry `ent` (slot u of a round): the window bit (d is
// clamped to wbits, whose word and bit are always zero) counted at once,
// and bit u of `slow` set when the entry falls in the hash set's range
template <bool kSlow, class A>
__device__ __forceinline__ void look(const TWin &tw, uint32_t ent, CliqueAcc<A> &a, unsigned &slow, int u) {
    const int32_t x = (int32_t)(ent & (uint32_t)kIdMask);
    const uint32_t d = min((uint32_t)(tw.tmax - x), tw.wbits);
    const uint32_t word = tw.bm[d >> 5];
    a.add_bit(__funnelshift_r(word, 0u, d) & 1u, ent);       // bit d % 32 of the word
    if (kSlow) slow |= ((uint32_t)(x - tw.tmin) < tw.lowspan ? 1u : 0u) << u;
}

// the hash lookups of the round's slow entries, when any lane has one
template <bool kSlow, class A>
__device__ __forceinline__ void look_slow(const TWin &tw, const uint32_t *ent, CliqueAcc<A> &a, unsigned slow) {
    if (kSlow && __any_sync(0xffffffffu, slow != 0u)) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if ((slow >> u) & 1u) a.add(tset_has(tw.set, tw.lgnb, (int32_t)(ent[u] & (uint32_t)kIdMask)), ent[u]);
    }
}

// member w of T: the whole warp scans N+(w), 128 entries a round (full
// rounds without bounds checks, then the partial one); returns |N+(w)|.
// kSlow: w may have hash-set members in N+(w), i.e. w <= lowmax (N+(w)
// holds ids above w only, so a member in the window meets window members
// only).
template <bool kSlow, class A>
__device__ __forceinline__ int32_t scan_list(const GraphView &g, int32_t w, const TWin &tw, CliqueAcc<A> &a,
                                             int lane) {
    const int64_t pb = g.plus_off[w];
    const int32_t np = (int32_t)(g.plus_off[w + 1] - pb);
    const int32_t *p = g.plus_adj + pb + lane;
    int32_t r0 = 0;
    for (; r0 + 128 <= np; r0 += 128, p += 128) {
        uint32_t ent[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ent[u] = (uint32_t)__ldg(p + 32 * u);
        unsigned slow = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) look<kSlow>(tw, ent[u], a, slow, u);
        look_slow<kSlow>(tw, ent, a, slow);
        if (++a.since == CliqueAcc<A>::R) a.drain(g.L);
    }
    if (r0 < np) {
        // entries past the list are looked up as id kIdMask of type 0, above
        // every member: no hit, and not in the hash set's range
        uint32_t ent[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ent[u] = r0 + 32 * u + lane < np ? (uint32_t)__ldg(p + 32 * u) : 0u;
        unsigned slow = 0, valid = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const bool v = r0 + 32 * u + lane < np;
            valid |= (v ? 1u : 0u) << u;
            uint32_t e = v ? ent[u] : (uint32_t)kIdMask;    // an id above every member: no hit, not slow
            look<kSlow>(tw, e, a, slow, u);
        }
        look_slow<kSlow>(tw, ent, a, slow & valid);
        if (++a.since == CliqueAcc<A>::R) a.drain(g.L);
    }
    return np;
}

template <class A>
__device__ __forceinline__ int32_t scan_member(const GraphView &g, int32_t w, const TWin &tw, CliqueAcc<A> &a,
                                               int lane) {
    return w <= tw.lowmax ? scan_list<true>(g, w, tw, a, lane) : scan_list<false>(g, w, tw, a, lane);
}

// the members of T, warp-serially, into K (sK) by member type
template <class A>
__device__ __forceinline__ unsigned long long scan_members_warp(const GraphView &g, const int32_t *T, int32_t nT,
                                                                const int32_t *ts, const TWin &tw,
                                                                unsigned long long *sK, int lane) {
    CliqueAcc<A> acc;
    unsigned long long probes = 0;
    int t = -1;
    for (int32_t k = 0; k < nT; ++k) {
        const int tk = type_of_index(ts, k);
        if (tk != t) {
            flush_k(acc, t, sK, g.L, lane, false);
            t = tk;
        }
        probes += (unsigned long long)scan_member(g, T[k], tw, acc, lane);
    }
    flush_k(acc, t, sK, g.L, lane, false);
    return probes;
}

// few pairs: every pair (a, b) of T checked by a binary search in the
// smaller id's typed row; K by (type of smaller, type of larger)
__device__ void clique_pairs_search(const GraphView &g, const int32_t *T, int32_t nT, const int32_t *ts,
                                    unsigned long long *sK, int gsize, int gr) {
    const long long npair = (long long)nT * (nT - 1) / 2;
    for (long long pk = gr; pk < npair; pk += gsize) {
        int32_t a = 0;
        long long rem = pk;
        while (rem >= nT - 1 - a) { rem -= nT - 1 - a; ++a; }
        const int32_t b = a + 1 + (int32_t)rem;
        int32_t w = T[a], x = T[b];
        int tw = type_of_index(ts, a), tx = type_of_index(ts, b);
        if (x < w) { int32_t y = w; w = x; x = y; int ty = tw; tw = tx; tx = ty; }
        const int64_t sb = seg_begin(g, w, tx), se = seg_end(g, w, tx);
        const int64_t r = lower_bound_i32(g.adj, sb, se, x);
        if (r < se && g.adj[r] == x) atomicAdd(&sK[tw * kMaxL + tx], 1ull);
    }
}

// optional diagnostic work counters (bench): lookups of the scans, pair searches
__device__ __forceinline__ void add_work(unsigned long long *work, int slot, unsigned long long v, int lane) {
    if (work && lane == 0 && v) atomicAdd(&work[slot], v);
}

// the window form when at least 3/4 of the members lie in the window
__device__ __forceinline__ bool use_window(int32_t nlow, int32_t nT) { return 4 * nlow <= nT; }

// Warp per edge (edges with |T| <= big_t): K into kmat.  A = the counter
// register type (uint32_t for L <= 5).
constexpr int kCliqueWarpSlots = 1024;       // per-warp set: 4 slots per member up to |T| = 256
constexpr int kCliqueWarpWin = 1 << 13;      // per-warp window bits (1 KB)
template <class A>
__global__ void __launch_bounds__(256, 5) k_clique(GraphView g, CountView cv, int64_t e0, int64_t e1, int64_t big_t) {
    __shared__ unsigned long long sKw[8][kMaxL * kMaxL];
    __shared__ int4 setw[8][kCliqueWarpSlots / 4];
    __shared__ uint32_t bmw[8][kCliqueWarpWin / 32 + 1];   // + the zero word of clamped lookups
    const int L = g.L, LL = L * L;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long *sK = sKw[wid];
    uint32_t *bm = bmw[wid];
    for (int k = lane; k <= kCliqueWarpWin / 32; k += 32) bm[k] = 0u;
    __syncwarp();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = e0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); e < e1; e += nw) {
        const int64_t er = e - e0;
        const int32_t nT = (int32_t)(cv.toffs[er + 1] - cv.toffs[er]);
        if (nT > big_t) continue;                           // done by k_clique_big
        unsigned long long *km = cv.kmat + er * LL;
        if (nT < 2) {
            for (int k = lane; k < LL; k += 32) km[k] = 0;
            continue;
        }
        for (int k = lane; k < kMaxL * kMaxL; k += 32) sK[k] = 0;
        __syncwarp();
        int32_t ts[kMaxL + 1];
        t_bounds(cv, L, e, ts);
        const int32_t *T = cv.tlist + cv.toffs[er];
        const long long npair = (long long)nT * (nT - 1) / 2;
        if (npair <= 64) {
            clique_pairs_search(g, T, nT, ts, sK, 32, lane);
            add_work(cv.work, kWorkCliqueSearches, (unsigned long long)npair, lane);
        } else {
            TWin tw;
            t_range(T, ts, L, tw.tmin, tw.tmax);
            const int32_t nlow = (int32_t)__reduce_add_sync(
                0xffffffffu, (unsigned)twin_below<kCliqueWarpWin>(T, nT, tw.tmax, 32, lane));
            const bool win = use_window(nlow, nT);
            const int32_t nset = win ? nlow : nT;           // members in the hash set
            tw.bm = bm;
            tw.set = setw[wid];
            tw.wbits = win ? kCliqueWarpWin : 0u;
            tw.lowmax = !win ? tw.tmax : nlow > 0 ? tw.tmax - kCliqueWarpWin : -1;
            tw.lowspan = tw.lowmax >= tw.tmin ? (uint32_t)(tw.lowmax - tw.tmin) + 1u : 0u;
            tw.lgnb = nset > 0 ? tset_lgnb(nset, kCliqueWarpSlots) : 1;   // nset <= 256: 4 slots per member
            if (tw.lgnb < 0) {                              // the options clamp big_t to 256
                if (lane == 0) set_status(cv.status, ST_INTERNAL);
                continue;
            }
            if (win) twin_bits<kCliqueWarpWin>(T, nT, tw.tmax, bm, 32, lane, true);
            if (nset > 0) tset_build(T, nT, setw[wid], tw.lgnb, 32, lane, tw.lowmax);
            else __syncwarp();                              // (tset_build ends with __syncwarp)
            const unsigned long long probes = scan_members_warp<A>(g, T, nT, ts, tw, sK, lane);
            add_work(cv.work, kWorkCliqueProbes, probes, lane);
            __syncwarp();
            if (win) twin_bits<kCliqueWarpWin>(T, nT, tw.tmax, bm, 32, lane, false);
        }
        __syncwarp();
        for (int k = lane; k < LL; k += 32) km[k] = sK[(k / L) * kMaxL + (k % L)];
        __syncwarp();
    }
}

// the members of T taken by the CTA's warps from a shared counter (in
// order, so each warp's member types only rise)
template <class A>
__device__ __forceinline__ unsigned long long big_members(const GraphView &g, const int32_t *T, int32_t nT,
                                                          const int32_t *ts, const TWin &tw, unsigned long long *sK,
                                                          int *next, int lane) {
    CliqueAcc<A> acc;
    unsigned long long probes = 0;
    int t = -1;
    for (;;) {
        int32_t m = 0;
        if (lane == 0) m = atomicAdd(next, 1);
        m = __shfl_sync(0xffffffffu, m, 0);
        if (m >= nT) break;
        const int tm = type_of_index(ts, m);
        if (tm != t) {
            flush_k(acc, t, sK, g.L, lane, true);
            t = tm;
        }
        probes += (unsigned long long)scan_member(g, T[m], tw, acc, lane);
    }
    flush_k(acc, t, sK, g.L, lane, true);
    return probes;
}

// CTA per edge for the listed edges with a large T; the hash set lives in
// shared memory up to kBigSetSmem slots, else in this CTA's global slice
// (2 slots per member).
constexpr int kBigSetSmem = 1 << 13;
constexpr int kBigThreads = 256;
constexpr int kBigWin = 1 << 15;             // window bits (4 KB)
template <class A>
__global__ void __launch_bounds__(kBigThreads, 5) k_clique_big(GraphView g, CountView cv, int64_t e0,
                                                          const int32_t *__restrict__ big_list,
                                                          const unsigned long long *__restrict__ big_count,
                                                          int32_t *set_scratch, int64_t set_stride) {
    __shared__ unsigned long long sK[kMaxL * kMaxL];
    __shared__ uint32_t bm[kBigWin / 32 + 1];            // + the zero word of clamped lookups
    __shared__ int s_next, s_low;
    extern __shared__ int4 set_smem[];
    const int L = g.L, LL = L * L;
    const int lane = threadIdx.x & 31;
    const int64_t nb = (int64_t)*big_count;
    unsigned long long probes = 0;
    for (int x = threadIdx.x; x <= kBigWin / 32; x += blockDim.x) bm[x] = 0u;
    for (int64_t k = blockIdx.x; k < nb; k += gridDim.x) {
        const int64_t e = big_list[k];
        const int64_t er = e - e0;
        const int32_t nT = (int32_t)(cv.toffs[er + 1] - cv.toffs[er]);
        for (int x = threadIdx.x; x < kMaxL * kMaxL; x += blockDim.x) sK[x] = 0;
        if (threadIdx.x == 0) {
            s_next = 0;
            s_low = 0;
        }
        int32_t ts[kMaxL + 1];
        t_bounds(cv, L, e, ts);
        const int32_t *T = cv.tlist + cv.toffs[er];
        TWin tw;
        t_range(T, ts, L, tw.tmin, tw.tmax);
        __syncthreads();                                    // s_low zero, the previous edge done
        const unsigned low = __reduce_add_sync(0xffffffffu,
                                               (unsigned)twin_below<kBigWin>(T, nT, tw.tmax, blockDim.x, threadIdx.x));
        if (lane == 0 && low) atomicAdd(&s_low, (int)low);
        __syncthreads();
        const int32_t nlow = s_low;
        const bool win = use_window(nlow, nT);              // CTA-uniform
        const int32_t nset = win ? nlow : nT;
        tw.bm = bm;
        tw.wbits = win ? kBigWin : 0u;
        tw.lowmax = !win ? tw.tmax : nlow > 0 ? tw.tmax - kBigWin : -1;
        tw.lowspan = tw.lowmax >= tw.tmin ? (uint32_t)(tw.lowmax - tw.tmin) + 1u : 0u;
        const int32_t xmax = tw.lowmax;
        if (win) twin_bits<kBigWin>(T, nT, tw.tmax, bm, blockDim.x, threadIdx.x, true);
        const int lgs = nset > 0 ? tset_lgnb(nset, kBigSetSmem) : 1;
        if (lgs >= 0) {
            tw.set = set_smem;
            tw.lgnb = lgs;
            if (nset > 0) tset_build(T, nT, set_smem, lgs, blockDim.x, threadIdx.x, xmax);   // ends with a barrier
            else __syncthreads();
        } else {                                            // global slice: 2^lg >= 2 nset slots
            int lg = 1;
            while ((4 << lg) < 2 * nset) ++lg;
            int4 *set = reinterpret_cast<int4 *>(set_scratch + (int64_t)blockIdx.x * set_stride);
            tw.set = set;
            tw.lgnb = lg;
            tset_build(T, nT, set, lg, blockDim.x, threadIdx.x, xmax);
        }
        probes += big_members<A>(g, T, nT, ts, tw, sK, &s_next, lane);
        __syncthreads();
        for (int x = threadIdx.x; x < LL; x += blockDim.x) cv.kmat[er * LL + x] = sK[(x / L) * kMaxL + (x % L)];
        if (win) twin_bits<kBigWin>(T, nT, tw.tmax, bm, blockDim.x, threadIdx.x, false);
        __syncthreads();
    }
    add_work(cv.work, kWorkCliqueBigProbes, probes, lane);
}

// value of matrix entry k (0 <= k < L*L) held as (r0 on lane k, or r1 on lane k-32)
__device__ __forceinline__ long long mat_get(long long r0, long long r1, int k) {
    const long long v0 = __shfl_sync(0xffffffffu, r0, k & 31);
    const long long v1 = __shfl_sync(0xffffffffu, r1, k & 31);
    return k < 32 ? v0 : v1;
}
__device__ __forceinline__ long long lane_get(long long v, int t) { return __shfl_sync(0xffffffffu, v, t); }

// Warp per edge: all orbits of Table 3 from the gathered sums (the
// inclusion-exclusion of Thm. 1 over S_i, S_j, T, I; then Lemmas 1-4).
// Lane l holds entry k = l (and k = l + 32 when L*L > 32) of each L x L
// matrix, (x, y) = (k / L, k % L); transposed entries come by shuffle.
// Shared memory of k_epi4: `copies` histograms of G(L) u64 (warp w adds into
// copy w % copies, so fewer warps contend per entry), then the multiset
// rank tables: rank2[p][q], rank3[p][q][t], rank4[p][q][pair] (uint16).
__host__ __device__ __forceinline__ size_t epi4_hist_words(int L) { return (size_t)((global_slots(L, 4) + 1) & ~1); }
__host__ __device__ __forceinline__ size_t epi4_smem_bytes(int L, int copies) {
    const int P = L * (L + 1) / 2;
    return epi4_hist_words(L) * copies * sizeof(unsigned long long) +
           (size_t)(L * L + L * L * L + L * L * P + 1) * sizeof(uint16_t);
}

__global__ void __launch_bounds__(256, 3) k_epi4(GraphView g, CountView cv, const Tile *__restrict__ tiles,
                                             int64_t n_tiles, int64_t row_base, uint32_t *per_edge_out,
                                             unsigned long long *gacc, int copies) {
    extern __shared__ unsigned long long hist_all[];
    const int L = g.L, LL = L * L, P = L * (L + 1) / 2;
    const int G = (int)global_slots(L, 4);
    const int S = (int)per_edge_slots(L, 4);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int HW = (int)epi4_hist_words(L);
    unsigned long long *hist = hist_all + (wid % copies) * HW;
    uint16_t *rank2 = reinterpret_cast<uint16_t *>(hist_all + (size_t)copies * HW);
    uint16_t *rank3 = rank2 + LL;
    uint16_t *rank4 = rank3 + LL * L;
    for (int s = threadIdx.x; s < copies * HW; s += blockDim.x) hist_all[s] = 0;
    for (int k = threadIdx.x; k < LL * P; k += blockDim.x) {
        const int pq = k / P, pi = k % P;
        int t = 0;
        while (pair_idx(L, t, L - 1) < pi) ++t;
        int ms[4] = {pq / L, pq % L, t, t + (pi - pair_idx(L, t, t))};
        sort4(ms);
        rank4[k] = (uint16_t)multiset_rank_dev(L, 4, ms);
    }
    for (int k = threadIdx.x; k < LL * L; k += blockDim.x) {
        int ms[3] = {k / LL, (k / L) % L, k % L};
        sort3(ms);
        rank3[k] = (uint16_t)multiset_rank_dev(L, 3, ms);
    }
    for (int k = threadIdx.x; k < LL; k += blockDim.x) {
        int ms[2] = {k / L < k % L ? k / L : k % L, k / L < k % L ? k % L : k / L};
        rank2[k] = (uint16_t)multiset_rank_dev(L, 2, ms);
    }
    const int off1 = gblock_off(L, 1), off2 = gblock_off(L, 2), off4 = gblock_off(L, 3), c4 = multichoose(L, 4);
    __syncthreads();
    int cur_graph = -1;
    const int kA = lane, kB = lane + 32;                     // this lane's matrix entries
    const int xA = kA / L, yA = kA % L, xB = kB / L, yB = kB % L;
    const bool hasA = kA < LL, hasB = kB < LL;
    const int tA = yA * L + xA, tB = yB * L + xB;            // transposed entries
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const Tile tile = tiles[ti];
        if (tile.graph != cur_graph) {
            __syncthreads();
            if (cur_graph >= 0) flush_hist_copies(hist_all, HW, copies, G, gacc, cur_graph, blockDim.x, threadIdx.x);
            __syncthreads();
            cur_graph = tile.graph;
        }
        for (int64_t e = tile.begin + wid; e < tile.end; e += nwarp) {
            const int64_t er = e - cv.e_base;
            const int32_t i = g.e_lo[e], j = g.e_hi[e];
            const int p = g.ty[i], q = g.ty[j];
            // per-type scalars, lane t < L
            long long c = 0, di = 0, dj = 0;
            if (lane < L) {
                c = cv.C[e * L + lane];
                di = typed_degree(g, i, lane);
                dj = typed_degree(g, j, lane);
            }
            const long long a = di - c - (q == lane ? 1 : 0);  // |S_i^t|
            const long long b = dj - c - (p == lane ? 1 : 0);  // |S_j^t|
            // gathered matrices
            const unsigned long long *sum = cv.tsum + er * 3 * LL;
            const unsigned long long *km = cv.kmat + er * LL;
            const int64_t *tau_i = cv.tau + (int64_t)i * LL, *tau_j = cv.tau + (int64_t)j * LL;
            const int64_t *del_i = g.delta + (int64_t)i * LL, *del_j = g.delta + (int64_t)j * LL;
            const uint32_t *A = cv.A - cv.a_base;
            const int64_t sij = g.e_slot_lo[e], sji = g.e_slot_hi[e];
            long long TCi[2] = {0, 0}, TCj[2] = {0, 0}, DT[2] = {0, 0}, Kd[2] = {0, 0}, Pm[2] = {0, 0};
            long long ti_[2] = {0, 0}, tj_[2] = {0, 0}, dI[2] = {0, 0}, dJ[2] = {0, 0};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool has = h ? hasB : hasA;
                const int k = h ? kB : kA, x = h ? xB : xA, y = h ? yB : yA;
                if (has) {
                    TCi[h] = (long long)sum[k];
                    TCj[h] = (long long)sum[LL + k];
                    DT[h] = (long long)sum[2 * LL + k];
                    Kd[h] = (long long)km[k];
                    // P[x][y]: slot i->j holds [type next to i][type next to j], slot j->i the reverse
                    Pm[h] = (long long)A[(int64_t)(y * L + x) * cv.a_stride + sij] +
                            (long long)A[(int64_t)(x * L + y) * cv.a_stride + sji];
                    ti_[h] = tau_i[k];
                    tj_[h] = tau_j[k];
                    dI[h] = del_i[k];
                    dJ[h] = del_j[k];
                }
            }
            // Ks = K + K^T
            long long Ks[2];
            Ks[0] = Kd[0] + mat_get(Kd[0], Kd[1], hasA ? tA : 0);
            Ks[1] = Kd[1] + mat_get(Kd[0], Kd[1], hasB ? tB : 0);
            // CTi, CTj
            long long CTi[2], CTj[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = h ? xB : xA, y = h ? yB : yA;
                const long long cx = lane_get(c, x < L ? x : 0);
                CTi[h] = TCi[h] - Ks[h] - (y == q ? cx : 0);
                CTj[h] = TCj[h] - Ks[h] - (y == p ? cx : 0);
            }
            long long CTiT[2], CTjT[2];
            CTiT[0] = mat_get(CTi[0], CTi[1], hasA ? tA : 0);
            CTiT[1] = mat_get(CTi[0], CTi[1], hasB ? tB : 0);
            CTjT[0] = mat_get(CTj[0], CTj[1], hasA ? tA : 0);
            CTjT[1] = mat_get(CTj[0], CTj[1], hasB ? tB : 0);
            // W, Q
            long long Wi[2], Wj[2], Q[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = h ? xB : xA, y = h ? yB : yA;
                const long long cx = lane_get(c, x < L ? x : 0), cy = lane_get(c, y < L ? y : 0);
                Wi[h] = ti_[h] - CTi[h] - CTiT[h] - Ks[h] - (x == q ? cy : 0) - (y == q ? cx : 0);
                Wj[h] = tj_[h] - CTj[h] - CTjT[h] - Ks[h] - (x == p ? cy : 0) - (y == p ? cx : 0);
                Q[h] = Pm[h] - CTjT[h] - CTi[h] - Ks[h];
            }
            long long QT[2];
            QT[0] = mat_get(Q[0], Q[1], hasA ? tA : 0);
            QT[1] = mat_get(Q[0], Q[1], hasB ? tB : 0);
            // R = Ri + Rj, G8, W = Wi + Wj, CT = CTi + CTj
            long long R[2], G8[2], W[2], CT[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = h ? xB : xA, y = h ? yB : yA;
                const long long cx = lane_get(c, x < L ? x : 0);
                const long long ax = lane_get(a, x < L ? x : 0), bx = lane_get(b, x < L ? x : 0);
                const long long djy = lane_get(dj, y < L ? y : 0), diy = lane_get(di, y < L ? y : 0);
                const long long Ri = dI[h] - DT[h] - (x == q ? djy : 0) - (y == p ? ax : 0) - Wi[h] - CTiT[h] - QT[h];
                const long long Rj = dJ[h] - DT[h] - (x == p ? diy : 0) - (y == q ? bx : 0) - Wj[h] - CTjT[h] - Q[h];
                R[h] = Ri + Rj;
                G8[h] = DT[h] - ((y == p ? 1 : 0) + (y == q ? 1 : 0)) * cx - Ks[h] - CTi[h] - CTj[h];
                W[h] = Wi[h] + Wj[h];
                CT[h] = CTi[h] + CTj[h];
            }
            uint32_t *row = per_edge_out ? per_edge_out + (e - row_base) * S : nullptr;
            // 3-node slots, typed edge and 3-node global blocks
            if (lane < L) {
                const long long s3 = a + b;
                if (a < 0 || b < 0) set_status(cv.status, ST_INTERNAL);
                if (row) {
                    row[lane] = sat32(s3, cv.status);
                    row[L + lane] = sat32(c, cv.status);
                }
                const int r = rank3[(p * L + q) * L + lane];
                if (s3) atomicAdd(&hist[off1 + r], (unsigned long long)s3);
                if (c) atomicAdd(&hist[off2 + r], (unsigned long long)c);
            }
            if (lane == 0) atomicAdd(&hist[rank2[p * L + q]], 1ull);
            // orbits, one type pair (t <= u) per lane (two rounds when P > 32)
            for (int base = 0; base < P; base += 32) {
                const int pi = base + lane;
                int t = 0;
                if (pi < P)
                    while (pair_idx(L, t, L - 1) < pi) ++t;
                const int u = pi < P ? t + (pi - pair_idx(L, t, t)) : 0;
                const int ktu = t * L + u, kut = u * L + t;
                const long long Rtu = mat_get(R[0], R[1], ktu), Rut = mat_get(R[0], R[1], kut);
                const long long Qtu = mat_get(Q[0], Q[1], ktu), Qut = mat_get(Q[0], Q[1], kut);
                const long long Wtu = mat_get(W[0], W[1], ktu);
                const long long Gtu = mat_get(G8[0], G8[1], ktu), Gut = mat_get(G8[0], G8[1], kut);
                const long long CTtu = mat_get(CT[0], CT[1], ktu), CTut = mat_get(CT[0], CT[1], kut);
                const long long Ktu = mat_get(Ks[0], Ks[1], ktu);
                const long long at = lane_get(a, t), au = lane_get(a, u), bt = lane_get(b, t), bu = lane_get(b, u);
                const long long ct = lane_get(c, t), cu = lane_get(c, u);
                if (pi >= P) continue;
                long long gv[10];
                bool ok = true;
                if (t != u) {
                    gv[0] = Rtu + Rut;                                 // g3
                    gv[3] = Qtu + Qut;                                 // g6
                    gv[4] = Wtu;                                       // g7
                    gv[5] = Gtu + Gut;                                 // g8
                    gv[7] = CTtu + CTut;                               // g10
                    gv[9] = Ktu;                                       // g12
                    gv[1] = at * bu + au * bt - gv[3];                 // Lemma 1
                    gv[2] = at * au + bt * bu - gv[4];                 // Lemma 2
                    gv[6] = ct * (au + bu) + cu * (at + bt) - gv[7];   // Lemma 3
                    gv[8] = ct * cu - gv[9];                           // Lemma 4
                } else {
                    ok = !(Wtu & 1) && !(Ktu & 1);
                    gv[0] = Rtu;
                    gv[3] = Qtu;
                    gv[4] = Wtu / 2;
                    gv[5] = Gtu;
                    gv[7] = CTtu;
                    gv[9] = Ktu / 2;
                    gv[1] = at * bt - gv[3];
                    gv[2] = at * (at - 1) / 2 + bt * (bt - 1) / 2 - gv[4];
                    gv[6] = ct * (at + bt) - gv[7];
                    gv[8] = ct * (ct - 1) / 2 - gv[9];
                }
                const int r = rank4[(p * L + q) * P + pi];
#pragma unroll
                for (int o = 3; o <= 12; ++o) {
                    const long long v = gv[o - 3];
                    ok = ok && v >= 0;
                    if (row) row[2 * L + (o - 3) * P + pi] = sat32(v, cv.status);
                    if (v > 0) atomicAdd(&hist[off4 + (graphlet_block(o) - 3) * c4 + r], (unsigned long long)v);
                }
                if (!ok) set_status(cv.status, ST_INTERNAL);
            }
        }
    }
    __syncthreads();
    if (cur_graph >= 0) flush_hist_copies(hist_all, HW, copies, G, gacc, cur_graph, blockDim.x, threadIdx.x);
}

// k = 3: 3-node slots and global blocks 0..2 only (warp per edge)
__global__ void __launch_bounds__(256) k_edge3(GraphView g, CountView cv, const Tile *__restrict__ tiles, int64_t n_tiles,
                                               int64_t e_begin, uint32_t *per_edge_out, unsigned long long *gacc) {
    extern __shared__ unsigned long long hist[];
    const int L = g.L;
    const int G = (int)global_slots(L, 3);
    const int S = 2 * L;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int s = threadIdx.x; s < G; s += blockDim.x) hist[s] = 0;
    __syncthreads();
    int cur_graph = -1;
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const Tile tile = tiles[ti];
        if (tile.graph != cur_graph) {
            if (cur_graph >= 0) flush_hist(hist, G, gacc, cur_graph, blockDim.x, threadIdx.x);
            __syncthreads();
            cur_graph = tile.graph;
        }
        for (int64_t e = tile.begin + wid; e < tile.end; e += nwarp) {
            const int32_t i = g.e_lo[e], j = g.e_hi[e];
            const int p = g.ty[i], q = g.ty[j];
            for (int t = lane; t < L; t += 32) {
                const int64_t c = cv.C[e * L + t];
                const int64_t a = typed_degree(g, i, t) - c - (q == t ? 1 : 0);
                const int64_t b = typed_degree(g, j, t) - c - (p == t ? 1 : 0);
                if (per_edge_out) {
                    uint32_t *row = per_edge_out + (e - e_begin) * S;
                    row[t] = sat32(a + b, cv.status);
                    row[L + t] = sat32(c, cv.status);
                }
                int ms[3] = {p, q, t};
                sort3(ms);
                const int r = multiset_rank_dev(L, 3, ms);
                if (a + b) atomicAdd(&hist[gblock_off(L, 1) + r], (unsigned long long)(a + b));
                if (c) atomicAdd(&hist[gblock_off(L, 2) + r], (unsigned long long)c);
            }
            if (lane == 0) {
                int ms[2] = {p < q ? p : q, p < q ? q : p};
                atomicAdd(&hist[multiset_rank_dev(L, 2, ms)], 1ull);
            }
        }
        __syncthreads();
    }
    if (cur_graph >= 0) flush_hist(hist, G, gacc, cur_graph, blockDim.x, threadIdx.x);
}

// ------------------------------------------------- position-aware epilogue
// Sec. 5 (Def. 8): before k_epi4 folds them into unordered type pairs, its
// matrices already keep the positions of an instance apart: Ri / Rj (4-path
// end edges with inner endpoint i / j: w the inner endpoint's other
// neighbour, r the far end), Q (4-cycles; first index the type of j's
// neighbour), Wi / Wj (adjacent pairs inside S_i / S_j), CTi / CTj (a
// triangle node and an adjacent node of S_i / S_j), G8 (a triangle node and
// its tail in I) and K (adjacent pairs inside T).  k_epi4_pa writes them by
// position -- the row layout of tg_pa.cu, sides named by caller ids (lo =
// the smaller) -- and adds every count to the class that the slot and the
// endpoint types fix (host table).  One warp per edge, as k_epi4; the gather
// and the matrices Ks, CTi, CTj, Wi, Wj, Q below repeat k_epi4's line for
// line, and the two kernels must change together.
struct PaView {
    const int32_t *cls;       // [L*L][S+1] class of (phi_lo, phi_hi, slot); slot S: the edge itself
    const int32_t *old_of;    // [n] caller id of each internal node
    int32_t S;                // per-edge slots
    int32_t G;                // classes (global slots) per graph
    int32_t off[13];          // first slot of blocks O1..O12
};

__host__ __device__ __forceinline__ size_t epi4_pa_hist_words(int G) { return (size_t)((G + 1) & ~1); }

__global__ void __launch_bounds__(256) k_epi4_pa(GraphView g, CountView cv, PaView pv, const Tile *__restrict__ tiles,
                                                 int64_t n_tiles, int64_t row_base, uint32_t *per_edge_out,
                                                 unsigned long long *gacc, int copies) {
    extern __shared__ unsigned long long hist_all[];
    const int L = g.L, LL = L * L, P = L * (L + 1) / 2;
    const int S = pv.S, G = pv.G;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int HW = (int)epi4_pa_hist_words(G);
    unsigned long long *hist = hist_all + (wid % copies) * HW;
    for (int s = threadIdx.x; s < copies * HW; s += blockDim.x) hist_all[s] = 0;
    __syncthreads();
    int cur_graph = -1;
    const int kA = lane, kB = lane + 32;                     // this lane's matrix entries
    const int xA = kA / L, yA = kA % L, xB = kB / L, yB = kB % L;
    const bool hasA = kA < LL, hasB = kB < LL;
    const int tA = yA * L + xA, tB = yB * L + xB;            // transposed entries
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const Tile tile = tiles[ti];
        if (tile.graph != cur_graph) {
            __syncthreads();
            if (cur_graph >= 0) flush_hist_copies(hist_all, HW, copies, G, gacc, cur_graph, blockDim.x, threadIdx.x);
            __syncthreads();
            cur_graph = tile.graph;
        }
        for (int64_t e = tile.begin + wid; e < tile.end; e += nwarp) {
            const int64_t er = e - cv.e_base;
            const int32_t i = g.e_lo[e], j = g.e_hi[e];
            const int p = g.ty[i], q = g.ty[j];
            long long c = 0, di = 0, dj = 0;
            if (lane < L) {
                c = cv.C[e * L + lane];
                di = typed_degree(g, i, lane);
                dj = typed_degree(g, j, lane);
            }
            const long long a = di - c - (q == lane ? 1 : 0);  // |S_i^t|
            const long long b = dj - c - (p == lane ? 1 : 0);  // |S_j^t|
            const unsigned long long *sum = cv.tsum + er * 3 * LL;
            const unsigned long long *km = cv.kmat + er * LL;
            const int64_t *tau_i = cv.tau + (int64_t)i * LL, *tau_j = cv.tau + (int64_t)j * LL;
            const int64_t *del_i = g.delta + (int64_t)i * LL, *del_j = g.delta + (int64_t)j * LL;
            const uint32_t *A = cv.A - cv.a_base;
            const int64_t sij = g.e_slot_lo[e], sji = g.e_slot_hi[e];
            long long TCi[2] = {0, 0}, TCj[2] = {0, 0}, DT[2] = {0, 0}, Kd[2] = {0, 0}, Pm[2] = {0, 0};
            long long ti_[2] = {0, 0}, tj_[2] = {0, 0}, dI[2] = {0, 0}, dJ[2] = {0, 0};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool has = h ? hasB : hasA;
                const int k = h ? kB : kA, x = h ? xB : xA, y = h ? yB : yA;
                if (has) {
                    TCi[h] = (long long)sum[k];
                    TCj[h] = (long long)sum[LL + k];
                    DT[h] = (long long)sum[2 * LL + k];
                    Kd[h] = (long long)km[k];
                    Pm[h] = (long long)A[(int64_t)(y * L + x) * cv.a_stride + sij] +
                            (long long)A[(int64_t)(x * L + y) * cv.a_stride + sji];
                    ti_[h] = tau_i[k];
                    tj_[h] = tau_j[k];
                    dI[h] = del_i[k];
                    dJ[h] = del_j[k];
                }
            }
            long long Ks[2];
            Ks[0] = Kd[0] + mat_get(Kd[0], Kd[1], hasA ? tA : 0);
            Ks[1] = Kd[1] + mat_get(Kd[0], Kd[1], hasB ? tB : 0);
            long long CTi[2], CTj[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = h ? xB : xA, y = h ? yB : yA;
                const long long cx = lane_get(c, x < L ? x : 0);
                CTi[h] = TCi[h] - Ks[h] - (y == q ? cx : 0);
                CTj[h] = TCj[h] - Ks[h] - (y == p ? cx : 0);
            }
            long long CTiT[2], CTjT[2];
            CTiT[0] = mat_get(CTi[0], CTi[1], hasA ? tA : 0);
            CTiT[1] = mat_get(CTi[0], CTi[1], hasB ? tB : 0);
            CTjT[0] = mat_get(CTj[0], CTj[1], hasA ? tA : 0);
            CTjT[1] = mat_get(CTj[0], CTj[1], hasB ? tB : 0);
            long long Wi[2], Wj[2], Q[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int x = h ? xB : xA, y = h ? yB : yA;
                const long long cx = lane_get(c, x < L ? x : 0), cy = lane_get(c, y < L ? y : 0);
                Wi[h] = ti_[h] - CTi[h] - CTiT[h] - Ks[h] - (x == q ? cy : 0) - (y == q ? cx : 0);
                Wj[h] = tj_[h] - CTj[h] - CTjT[h] - Ks[h] - (x == p ? cy : 0) - (y == p ? cx : 0);
                Q[h] = Pm[h] - CTjT[h] - CTi[h] - Ks[h];
            }
            long long QT[2];
            QT[0] = mat_get(Q[0], Q[1], hasA ? tA : 0);
            QT[1] = mat_get(Q[0], Q[1], hasB ? tB : 0);
            // orientation: side 0 is the endpoint with the smaller caller id
            const bool lo_is_i = pv.old_of[i] < pv.old_of[j];
            const int sI = lo_is_i ? 0 : 1, sJ = 1 - sI;
            const int pl = lo_is_i ? p : q, ph = lo_is_i ? q : p;
            const int32_t *cls = pv.cls + (int64_t)(pl * L + ph) * (S + 1);
            uint32_t *row = per_edge_out ? per_edge_out + (e - row_base) * S : nullptr;
            bool ok = true;
            auto emit = [&](int slot, long long v) {
                ok = ok && v >= 0;
                if (row) row[slot] = sat32(v, cv.status);
                if (v > 0) atomicAdd(&hist[cls[slot]], (unsigned long long)v);
            };
            if (lane == 0) atomicAdd(&hist[cls[S]], 1ull);            // the edge itself
            if (lane < L) {
                if (a < 0 || b < 0) set_status(cv.status, ST_INTERNAL);
                emit(pv.off[1] + sI * L + lane, a);                  // 3-path centred at i
                emit(pv.off[1] + sJ * L + lane, b);                  // centred at j
                emit(pv.off[2] + lane, c);
            }
            // ordered blocks: entry (x, y) of each matrix on this lane
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool has = h ? hasB : hasA;
                const int k = h ? kB : kA, x = h ? xB : xA, y = h ? yB : yA;
                const int kt = h ? tB : tA;                          // (y, x)
                const long long cx = lane_get(c, x < L ? x : 0);
                const long long ax = lane_get(a, x < L ? x : 0), ay = lane_get(a, y < L ? y : 0);
                const long long bx = lane_get(b, x < L ? x : 0), by = lane_get(b, y < L ? y : 0);
                const long long djy = lane_get(dj, y < L ? y : 0), diy = lane_get(di, y < L ? y : 0);
                if (!has) continue;
                const long long Ri = dI[h] - DT[h] - (x == q ? djy : 0) - (y == p ? ax : 0) - Wi[h] - CTiT[h] - QT[h];
                const long long Rj = dJ[h] - DT[h] - (x == p ? diy : 0) - (y == q ? bx : 0) - Wj[h] - CTjT[h] - Q[h];
                const long long G8 = DT[h] - ((y == p ? 1 : 0) + (y == q ? 1 : 0)) * cx - Ks[h] - CTi[h] - CTj[h];
                emit(pv.off[3] + sI * LL + k, Ri);                   // inner endpoint i: near x, far y
                emit(pv.off[3] + sJ * LL + k, Rj);
                emit(pv.off[4] + (lo_is_i ? k : kt), ax * by - QT[h]);   // i's neighbour x, j's y (Lemma 1)
                emit(pv.off[6] + (lo_is_i ? k : kt), QT[h]);         // 4-cycle: i's neighbour x, j's y
                emit(pv.off[8] + k, G8);                             // triangle node x, tail y
                emit(pv.off[9] + sI * LL + k, cx * ay - CTi[h]);     // Lemma 3, degree-3 node i
                emit(pv.off[9] + sJ * LL + k, cx * by - CTj[h]);
                emit(pv.off[10] + sI * LL + k, CTi[h]);              // chordal outer edge, degree-3 node i
                emit(pv.off[10] + sJ * LL + k, CTj[h]);
            }
            // unordered pairs (t <= u), one per lane
            for (int base = 0; base < P; base += 32) {
                const int pi = base + lane;
                int t = 0;
                if (pi < P)
                    while (pair_idx(L, t, L - 1) < pi) ++t;
                const int u = pi < P ? t + (pi - pair_idx(L, t, t)) : 0;
                const int ktu = t * L + u;
                const long long Witu = mat_get(Wi[0], Wi[1], ktu), Wjtu = mat_get(Wj[0], Wj[1], ktu);
                const long long Ktu = mat_get(Ks[0], Ks[1], ktu);
                const long long at = lane_get(a, t), au = lane_get(a, u), bt = lane_get(b, t), bu = lane_get(b, u);
                const long long ct = lane_get(c, t), cu = lane_get(c, u);
                if (pi >= P) continue;
                long long star_i, star_j, tail_i, tail_j, chord, clique;
                if (t != u) {
                    star_i = at * au - Witu;                         // Lemma 2, centre i
                    star_j = bt * bu - Wjtu;
                    tail_i = Witu;
                    tail_j = Wjtu;
                    chord = ct * cu - Ktu;                           // Lemma 4
                    clique = Ktu;
                } else {
                    ok = ok && !(Witu & 1) && !(Wjtu & 1) && !(Ktu & 1);
                    star_i = at * (at - 1) / 2 - Witu / 2;
                    star_j = bt * (bt - 1) / 2 - Wjtu / 2;
                    tail_i = Witu / 2;
                    tail_j = Wjtu / 2;
                    chord = ct * (ct - 1) / 2 - Ktu / 2;
                    clique = Ktu / 2;
                }
                emit(pv.off[5] + sI * P + pi, star_i);
                emit(pv.off[5] + sJ * P + pi, star_j);
                emit(pv.off[7] + sI * P + pi, tail_i);
                emit(pv.off[7] + sJ * P + pi, tail_j);
                emit(pv.off[11] + pi, chord);
                emit(pv.off[12] + pi, clique);
            }
            if (!ok) set_status(cv.status, ST_INTERNAL);
        }
    }
    __syncthreads();
    if (cur_graph >= 0) flush_hist_copies(hist_all, HW, copies, G, gacc, cur_graph, blockDim.x, threadIdx.x);
}

// global totals: C_H = (1/|E(H)|) * sum_e x_e (Sec. 6), exact division
__global__ void k_finalize(int ngraphs, int L, int k, const unsigned long long *__restrict__ gacc, int64_t *out,
                           uint32_t *status) {
    const int G = (int)global_slots(L, k);
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ngraphs * G) return;
    const int s = (int)(idx % G);
    const int nb = k == 4 ? 9 : 3;
    int b = 0;
    while (b + 1 < nb && gblock_off(L, b + 1) <= s) ++b;
    const int edges_of[9] = {1, 2, 3, 3, 3, 4, 4, 5, 6};
    const unsigned long long v = gacc[idx];
    if (v % edges_of[b]) set_status(status, ST_INTERNAL);
    out[idx] = (int64_t)(v / edges_of[b]);
}

int grid_for(int64_t items, int per_block, int cap) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

// Edges per tile: kTile, or fewer for a small handle so that its tiles
// still fill the GPU (at least about 12 tiles per SM, 64 edges or more each).
static int64_t tile_edges(const Graph &G) {
    const int64_t want = (G.m + (int64_t)sm_count() * 12 - 1) / ((int64_t)sm_count() * 12);
    int64_t t = 64;
    while (t < want && t < kTile) t <<= 1;
    return t;
}

static std::vector<Tile> make_tiles(const Graph &G, int64_t e_begin, int64_t e_end) {
    std::vector<Tile> tiles;
    const int64_t te = tile_edges(G);
    for (int gi = 0; gi < G.ngraphs; ++gi) {
        int64_t b = std::max(e_begin, G.h_edge_off[gi]), e = std::min(e_end, G.h_edge_off[gi + 1]);
        for (int64_t x = b; x < e; x += te) tiles.push_back(Tile{x, std::min(e, x + te), gi, 0});
    }
    return tiles;
}

// Splits the graphs into consecutive chunks whose adjacency slots fit the
// 4-cycle array budget (a single graph larger than the budget is a chunk of
// its own), and sizes the array for the largest chunk.
static void plan_chunks(Graph &G) {
    G.chunks.clear();
    // working bytes of a chunk: the 4-cycle array (4 L^2 per slot) and the
    // per-edge sums, K and offsets (32 L^2 + 28 per edge)
    const int64_t LL = (int64_t)G.L * G.L;
    const int64_t budget = std::max<int64_t>((int64_t)G.opt.cycle_budget_mb << 20, 1);
    auto bytes_of = [&](int a, int b) {
        return (G.h_slot_off[b] - G.h_slot_off[a]) * 4 * LL + (G.h_edge_off[b] - G.h_edge_off[a]) * (32 * LL + 28);
    };
    // tile index ranges follow graph boundaries (make_tiles emits graph after graph)
    std::vector<int64_t> tile_off(G.ngraphs + 1, 0);
    const int64_t te = tile_edges(G);
    for (int gi = 0; gi < G.ngraphs; ++gi)
        tile_off[gi + 1] = tile_off[gi] + (G.h_edge_off[gi + 1] - G.h_edge_off[gi] + te - 1) / te;
    int g0 = 0;
    int64_t widest = 0;
    while (g0 < G.ngraphs) {
        int g1 = g0 + 1;
        while (g1 < G.ngraphs && bytes_of(g0, g1 + 1) <= budget) ++g1;
        Graph::Chunk c;
        c.g0 = g0; c.g1 = g1;
        c.n0 = G.h_node_off[g0]; c.n1 = G.h_node_off[g1];
        c.s0 = G.h_slot_off[g0]; c.s1 = G.h_slot_off[g1];
        c.e0 = G.h_edge_off[g0]; c.e1 = G.h_edge_off[g1];
        c.t0 = tile_off[g0]; c.t1 = tile_off[g1];
        widest = std::max(widest, c.s1 - c.s0);
        G.max_chunk_edges = std::max(G.max_chunk_edges, c.e1 - c.e0);
        G.chunks.push_back(c);
        g0 = g1;
    }
    G.a_stride = std::max<int64_t>(widest, 1);
}

static size_t hist_bytes(int L, int k) { return (size_t)((global_slots(L, k) + 1) & ~1) * sizeof(unsigned long long); }

// Device tile list of [e_begin, e_end); the full range is cached by the
// handle (so that a captured CUDA graph never copies from host memory).
static const Tile *tiles_for(Graph &G, int64_t e_begin, int64_t e_end, int64_t &n_tiles, DBuf &tmp, cudaStream_t s) {
    const bool full = e_begin == 0 && e_end == G.m;
    if (full && G.tiles_full.p) {
        n_tiles = G.n_tiles_full;
        return G.tiles_full.as<Tile>();
    }
    std::vector<Tile> tiles = make_tiles(G, e_begin, e_end);
    n_tiles = (int64_t)tiles.size();
    DBuf &dst = full ? G.tiles_full : tmp;
    dst.alloc(sizeof(Tile) * std::max<size_t>(tiles.size(), 1));
    if (!tiles.empty()) {
        TG_CK(cudaMemcpyAsync(dst.p, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, s));
        TG_CK(cudaStreamSynchronize(s));   // the host vector goes out of scope
    }
    if (full) G.n_tiles_full = n_tiles;
    return dst.as<Tile>();
}

// |T_e| summed over the edges of each chunk (from c_e^t)
__global__ void k_chunk_t(GraphView g, CountView cv, int64_t e0, int64_t e1, unsigned long long *out) {
    unsigned long long acc = 0;
    for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1; e += (int64_t)gridDim.x * blockDim.x)
        for (int t = 0; t < g.L; ++t) acc += cv.C[e * g.L + t];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

int light_anchor_limit(int L) {
    int dev = 0, optin = 0;
    TG_CK(cudaGetDevice(&dev));
    TG_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int cap = 1;                                              // per-warp hash of k_wedge_light
    while ((size_t)kLightAnchorWarps * (cap * 2) * (1 + L) * sizeof(int32_t) <= (size_t)optin) cap *= 2;
    return cap / 2;                                           // capacity >= 2 x wedges
}

void raise_smem_limit(const void *func, size_t bytes) {
    struct Limit { const void *func; int dev; size_t bytes; };
    static std::mutex mu;
    static std::vector<Limit> set;
    int dev = 0;
    TG_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    Limit *hit = nullptr;
    for (auto &l : set)
        if (l.func == func && l.dev == dev) hit = &l;
    if (hit && hit->bytes >= bytes) return;
    TG_CK(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    if (hit) hit->bytes = bytes;
    else set.push_back({func, dev, bytes});
}

// Allocations and kernel attributes of the per-edge stage (done before any
// capture).
// histogram copies of k_epi4: one per warp while they fit in 64 KB
static int epi4_copies(int L) {
    int c = 8;
    while (c > 1 && epi4_hist_words(L) * c * sizeof(unsigned long long) > (64u << 10)) c >>= 1;
    return c;
}

// histogram copies of k_epi4_pa: as many as fit 64 KB (at least one)
static int epi4_pa_copies(int G) {
    int c = 8;
    while (c > 1 && epi4_pa_hist_words(G) * c * sizeof(unsigned long long) > (64u << 10)) c >>= 1;
    return c;
}

void prepare_epi4_pa(Graph &G) {
    raise_smem_limit((const void *)k_epi4_pa,
                     epi4_pa_hist_words((int)G.pa.G) * epi4_pa_copies((int)G.pa.G) * sizeof(unsigned long long));
}

static PaView pa_view(const Graph &G) {
    PaView v;
    v.cls = G.pa_cls.as<int32_t>();
    v.old_of = G.old_of.as<int32_t>();
    v.S = G.pa.S;
    v.G = (int32_t)G.pa.G;
    for (int o = 0; o < 13; ++o) v.off[o] = G.pa.off[o];
    return v;
}

void prepare_edges(Graph &G, int k, cudaStream_t s) {
    raise_smem_limit((const void *)k_edge3, hist_bytes(G.L, 3));
    raise_smem_limit((const void *)k_epi4, epi4_smem_bytes(G.L, epi4_copies(G.L)));
    raise_smem_limit((const void *)k_clique_big<uint32_t>, kBigSetSmem * sizeof(int32_t));
    raise_smem_limit((const void *)k_clique_big<unsigned long long>, kBigSetSmem * sizeof(int32_t));
    raise_smem_limit((const void *)k_wedge_heavy, (size_t)kHeavyCap * (1 + G.L) * sizeof(int32_t));
    if (k == 4 && !G.set_scratch.p) {
        // a set of capacity >= 2 max degree per CTA, for edges whose T exceeds shared memory
        int64_t cap = 1;
        while (cap < 2 * std::max<int64_t>(G.max_degree, 1)) cap <<= 1;
        G.big_blocks = sm_count() * 5;
        G.set_stride = cap > kBigSetSmem ? cap : 1;
        G.set_scratch.alloc(sizeof(int32_t) * (size_t)(G.set_stride * G.big_blocks));
    }
    DBuf unused;
    unused.owner = &G.stream;
    int64_t nt = 0;
    tiles_for(G, 0, G.m, nt, unused, s);
    if (k == 4 && G.n_anchors_light > 0) {
        int cap = 1;
        while (cap < 2 * G.opt.light_anchor_max_wedges) cap <<= 1;
        const size_t smem = (size_t)kLightAnchorWarps * cap * (1 + G.L) * sizeof(int32_t);
        raise_smem_limit((const void *)k_wedge_light, smem);
    }
}

// typed triangles per edge and per-node typed triangle sums: whole graph
static int64_t launch_triangles(Graph &G, cudaStream_t s) {
    const GraphView gv = G.view();
    const CountView cv = G.cview();
    const int sms = sm_count();
    int64_t launches = 0;
    if (G.m > 0) {
        KernelTimer kt(G, s, "k_tri");
        if (isect_any_merge(G.opt.isect_modes)) k_tri<true><<<grid_for(G.m, 8, sms * 16), 256, 0, s>>>(gv, cv);
        else k_tri<false><<<grid_for(G.m, 8, sms * 16), 256, 0, s>>>(gv, cv);
        ++launches;
    }
    if (G.n > 0) {
        KernelTimer kt(G, s, "k_tau");
        k_tau<<<grid_for(G.n, 8, sms * 16), 256, 0, s>>>(gv, cv);
        ++launches;
    }
    TG_CK(cudaGetLastError());
    return launches;
}

// Triangle-node entries of every chunk (a graph invariant, computed once
// after the first k_tri; synchronises) and the T list buffer sized for the
// largest chunk.
static void ensure_t_sizes(Graph &G, cudaStream_t s) {
    if (!G.chunk_t.empty()) return;
    TBuf cnt(sizeof(unsigned long long) * G.chunks.size(), s);
    TG_CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * G.chunks.size(), s));
    const GraphView gv = G.view();
    const CountView cv = G.cview();
    for (size_t x = 0; x < G.chunks.size(); ++x) {
        const Graph::Chunk &c = G.chunks[x];
        if (c.e1 > c.e0)
            k_chunk_t<<<grid_for(c.e1 - c.e0, 256, sm_count() * 8), 256, 0, s>>>(gv, cv, c.e0, c.e1,
                                                                               cnt.as<unsigned long long>() + x);
    }
    TG_CK(cudaGetLastError());
    std::vector<unsigned long long> h(G.chunks.size());
    TG_CK(cudaMemcpyAsync(h.data(), cnt.p, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    G.chunk_t.assign(h.begin(), h.end());
    const int64_t cap = std::max<int64_t>(*std::max_element(G.chunk_t.begin(), G.chunk_t.end()), 1);
    if (G.tlist_cap < cap) {
        G.tlist.alloc(sizeof(int32_t) * (size_t)cap);
        G.tlist_cap = cap;
    }
}

// words of one hub's counter table (one row of L counters per node of its graph)
static int64_t hub_words_per_table(const Graph &G) {
    const int64_t rw = G.hub_packed ? (G.L + 1) / 2 : G.L;
    return std::max<int64_t>(G.max_graph_nodes, 1) * rw;
}

// hubs of one group: their tables fill at most half of hub_l2_mb (the
// persistent pass fills one group's tables while it reads the previous one's)
static int64_t hub_group_max(const Graph &G) {
    const int64_t per = hub_words_per_table(G) * (int64_t)sizeof(uint32_t);
    return std::max<int64_t>(((int64_t)G.opt.hub_l2_mb << 20) / 2 / per, 1);
}

constexpr int kHubCtasPerSm = 5;                            // k_wedge_hub's launch bounds

template <class T>
static void exclusive_sum(const T *in, T *out, int64_t n, cudaStream_t s) {
    size_t tb = 0;
    TG_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, n, s));
    TBuf tmp(std::max<size_t>(tb, 16), s);
    TG_CK(cub::DeviceScan::ExclusiveSum(tmp.p, tb, in, out, n, s));
}

static HubView hub_view(const Graph &G) {
    HubView h;
    h.hubs = G.hubs.as<int32_t>();
    h.hub_base = G.hub_base.as<int64_t>();
    h.woff = G.item_woff.as<int64_t>();
    h.item = G.item_rec.as<int4>();
    h.batched = G.ngraphs > 1;
    return h;
}

// Wedge items of the hub anchors (graph invariant, built at the first count).
static void prepare_hubs(Graph &G, cudaStream_t s) {
    const int L = G.L;
    const int64_t nh = G.n_hubs;
    const GraphView gv = G.view();
    TBuf nv(sizeof(int64_t) * (nh + 1), s), vbase(sizeof(int64_t) * (nh + 1), s);
    G.hub_base.alloc(sizeof(int64_t) * nh);
    k_hub_nv<<<grid_for(nh + 1, 256, 1 << 20), 256, 0, s>>>(gv, G.hubs.as<int32_t>(), nh, nv.as<int64_t>(),
                                                            G.hub_base.as<int64_t>());
    TG_CK(cudaGetLastError());
    exclusive_sum(nv.as<int64_t>(), vbase.as<int64_t>(), nh + 1, s);
    int64_t NV = 0;
    TG_CK(cudaMemcpyAsync(&NV, vbase.as<int64_t>() + nh, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    const int64_t NI = NV * L;
    TBuf cnt(sizeof(int32_t) * std::max<int64_t>(NI, 1), s), flag(sizeof(int64_t) * (NI + 1), s);
    TBuf pos(sizeof(int64_t) * (NI + 1), s);
    TBuf sv_of(sizeof(int32_t) * std::max<int64_t>(NV, 1), s), hub_of(sizeof(int32_t) * std::max<int64_t>(NV, 1), s);
    TG_CK(cudaMemsetAsync(flag.p, 0, sizeof(int64_t) * (NI + 1), s));
    k_hub_cnt<<<grid_for(nh, 1, sm_count() * 8), 256, 0, s>>>(gv, G.hubs.as<int32_t>(), nh, vbase.as<int64_t>(),
                                                               cnt.as<int32_t>(), flag.as<int64_t>(),
                                                               sv_of.as<int32_t>(), hub_of.as<int32_t>());
    TG_CK(cudaGetLastError());
    exclusive_sum(flag.as<int64_t>(), pos.as<int64_t>(), NI + 1, s);
    TG_CK(cudaMemcpyAsync(&G.n_items, pos.as<int64_t>() + NI, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    const int64_t ni = std::max<int64_t>(G.n_items, 1);
    G.item_rec.alloc(sizeof(int4) * ni);
    G.item_woff.alloc(sizeof(int64_t) * (G.n_items + 1));
    TBuf icnt(sizeof(int64_t) * (G.n_items + 1), s);
    TG_CK(cudaMemsetAsync(icnt.p, 0, sizeof(int64_t) * (G.n_items + 1), s));
    if (NI > 0) {
        k_hub_items<<<grid_for(NI, 256, 1 << 30), 256, 0, s>>>(gv, NI, cnt.as<int32_t>(), pos.as<int64_t>(),
                                                               sv_of.as<int32_t>(), hub_of.as<int32_t>(),
                                                               G.hubs.as<int32_t>(), G.item_rec.as<int4>(),
                                                               icnt.as<int64_t>());
        TG_CK(cudaGetLastError());
    }
    exclusive_sum(icnt.as<int64_t>(), G.item_woff.as<int64_t>(), G.n_items + 1, s);
    TBuf fi(sizeof(int64_t) * (nh + 1), s), fw(sizeof(int64_t) * (nh + 1), s);
    k_hub_bounds<<<grid_for(nh + 1, 256, 1 << 20), 256, 0, s>>>(nh, L, vbase.as<int64_t>(), pos.as<int64_t>(),
                                                                G.item_woff.as<int64_t>(), fi.as<int64_t>(),
                                                                fw.as<int64_t>());
    TG_CK(cudaGetLastError());
    G.h_hub_item.assign(nh + 1, 0);
    G.h_hub_woff.assign(nh + 1, 0);
    TG_CK(cudaMemcpyAsync(G.h_hub_item.data(), fi.p, sizeof(int64_t) * (nh + 1), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaMemcpyAsync(G.h_hub_woff.data(), fw.p, sizeof(int64_t) * (nh + 1), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    for (int64_t h = 0; h < nh; ++h)   // the items hold exactly the wedges the build counted
        if (G.h_hub_woff[h + 1] - G.h_hub_woff[h] != G.h_hub_wedges[h]) throw Error{TG_ERR_INTERNAL, "hub wedges"};
    G.hubs_ready = true;
}

// Ticket queues of the persistent hub pass, one per chunk (graph invariant,
// built before any capture): hubs in groups of at most hub_group_max tables
// and about 2^22 wedges; per group, fill and read tickets of at least 2 per
// CTA of the launch (1,024 to 8,192 wedges each) and clear tickets (zeroing
// the group's table words when that is cheaper than walking its wedges
// again).  Queue order: the clears of group s - 2, the reads of group s - 1,
// the fills of group s, for s = 0, 1, ...: every ticket waits on tickets at
// least one phase of another group earlier in the queue.
static void plan_hubs(Graph &G, cudaStream_t s) {
    const int64_t ctas = (int64_t)sm_count() * kHubCtasPerSm;
    G.hub_packed = G.max_degree < 65536;
    G.hub_stride = hub_words_per_table(G);
    // no more tables per buffer than there are hubs (a small graph's budget
    // would otherwise reserve hub_l2_mb for a few hubs)
    const int64_t gmax = std::min<int64_t>(hub_group_max(G), std::max<int64_t>(G.n_hubs, 1));
    G.hub_buf_words = gmax * G.hub_stride;
    const size_t tbytes = sizeof(uint32_t) * (size_t)(kHubBuffers * G.hub_buf_words);
    G.hub_tables.alloc(tbytes);
    TG_CK(cudaMemsetAsync(G.hub_tables.p, 0, tbytes, s));
    G.hub_plans.clear();
    for (const Graph::Chunk &c : G.chunks) {
        auto plan = std::make_unique<Graph::HubPlan>();
        for (DBuf *d : {&plan->segs, &plan->groups, &plan->ntick, &plan->ctr}) d->owner = &G.stream;
        const int64_t hb0 = std::lower_bound(G.h_hub_id.begin(), G.h_hub_id.end(), (int32_t)c.n0) - G.h_hub_id.begin();
        const int64_t hb1 = std::lower_bound(G.h_hub_id.begin(), G.h_hub_id.end(),
                                             (int32_t)std::min<int64_t>(c.n1, INT32_MAX)) - G.h_hub_id.begin();
        std::vector<HubGroup> &groups = plan->h_groups;
        std::vector<int64_t> &ntick = plan->h_ntick;
        for (int64_t h = hb0; h < hb1;) {
            int64_t h1 = h, wsum = 0;
            while (h1 < hb1 && h1 - h < gmax && wsum < ((int64_t)1 << 22)) wsum += G.h_hub_wedges[h1++];
            const int64_t w0 = G.h_hub_woff[h], w1 = G.h_hub_woff[h1];
            if (w1 > w0) {
                HubGroup gr;
                gr.i0 = G.h_hub_item[h];
                gr.i1 = G.h_hub_item[h1];
                gr.w0 = w0;
                gr.w1 = w1;
                gr.tw = std::min<int64_t>(std::max<int64_t>((wsum / (2 * ctas) + 255) & ~(int64_t)255, 1024), 8192);
                gr.zwords = (h1 - h) * G.hub_stride;
                gr.h0 = (int32_t)h;
                gr.buf = (int32_t)(groups.size() % kHubBuffers);
                const int64_t nw = (w1 - w0 + gr.tw - 1) / gr.tw;
                const bool zero = gr.zwords * (int64_t)sizeof(uint32_t) <= 32 * wsum;
                ntick.push_back(nw);                                                     // fill
                ntick.push_back(nw);                                                     // read
                ntick.push_back(zero ? 0 : nw);                                          // clear by walking
                ntick.push_back(zero ? (gr.zwords + kHubTicketWords - 1) / kHubTicketWords : 0);   // clear by zeroing
                groups.push_back(gr);
            }
            h = h1;
        }
        const int64_t ng = (int64_t)groups.size();
        std::vector<HubSegment> &segs = plan->h_segs;
        int64_t nt = 0;
        for (int64_t st = 0; st < ng + 2; ++st) {
            auto emit = [&](int64_t q, int kind) {
                if (q < 0 || q >= ng || ntick[q * kHubKinds + kind] == 0) return;
                segs.push_back(HubSegment{nt, (int32_t)q, kind});
                nt += ntick[q * kHubKinds + kind];
            };
            emit(st - 2, 2);
            emit(st - 2, 3);
            emit(st - 1, 1);
            emit(st, 0);
        }
        // every run waits only on runs queued before it (so each wait ends:
        // those tickets were taken by running CTAs)
        {
            std::vector<int64_t> pos((size_t)std::max<int64_t>(ng * kHubKinds, 1), -1);
            for (int64_t k = 0; k < (int64_t)segs.size(); ++k) pos[(size_t)(segs[k].group * kHubKinds + segs[k].kind)] = k;
            for (int64_t k = 0; k < (int64_t)segs.size(); ++k) {
                const int64_t q = segs[k].group;
                const int kind = segs[k].kind;
                int64_t dep[2] = {-1, -1};
                if (kind == 1) dep[0] = q * kHubKinds;
                else if (kind >= 2) dep[0] = q * kHubKinds + 1;
                else if (q >= kHubBuffers) { dep[0] = (q - kHubBuffers) * kHubKinds + 2; dep[1] = dep[0] + 1; }
                for (int64_t d : dep)
                    if (d >= 0 && pos[(size_t)d] >= k) throw Error{TG_ERR_INTERNAL, "hub ticket order"};
            }
        }
        plan->n_groups = ng;
        plan->n_segs = (int64_t)segs.size();
        plan->n_tickets = nt;
        if (ng > 0) {
            plan->segs.alloc(sizeof(HubSegment) * segs.size());
            plan->groups.alloc(sizeof(HubGroup) * groups.size());
            plan->ntick.alloc(sizeof(int64_t) * ntick.size());
            plan->ctr.alloc(sizeof(unsigned long long) * (size_t)(1 + ng * kHubKinds));
            TG_CK(cudaMemcpyAsync(plan->segs.p, segs.data(), sizeof(HubSegment) * segs.size(), cudaMemcpyHostToDevice, s));
            TG_CK(cudaMemcpyAsync(plan->groups.p, groups.data(), sizeof(HubGroup) * groups.size(),
                                  cudaMemcpyHostToDevice, s));
            TG_CK(cudaMemcpyAsync(plan->ntick.p, ntick.data(), sizeof(int64_t) * ntick.size(), cudaMemcpyHostToDevice,
                                  s));
        }
        G.hub_plans.push_back(std::move(plan));
    }
}

// The hubs of chunk ci: one persistent launch over the chunk's tickets.
static int64_t launch_hubs(Graph &G, size_t ci, cudaStream_t s) {
    Graph::HubPlan &P = *G.hub_plans[ci];
    if (P.n_tickets == 0) return 0;
    TG_CK(cudaMemsetAsync(P.ctr.p, 0, sizeof(unsigned long long) * (size_t)(1 + P.n_groups * kHubKinds), s));
    const GraphView gv = G.view();
    const CountView cv = G.cview();
    const HubView hv = hub_view(G);
    const int grid = sm_count() * kHubCtasPerSm;
    KernelTimer kt(G, s, "k_wedge_hub");
    auto launch = [&](auto kern) {
        kern<<<grid, kHubThreads, 0, s>>>(gv, cv, hv, P.segs.as<HubSegment>(), P.n_segs, P.n_tickets,
                                          P.groups.as<HubGroup>(), P.ntick.as<int64_t>(), P.ctr.as<unsigned long long>(),
                                          G.hub_tables.as<uint32_t>(), G.hub_buf_words, G.hub_stride);
    };
    const bool count = cv.work != nullptr;                  // the work-counting form (diagnostics)
    if (G.hub_packed) {
        if (count) launch(k_wedge_hub<true, true>);
        else launch(k_wedge_hub<true, false>);
    } else {
        if (count) launch(k_wedge_hub<false, true>);
        else launch(k_wedge_hub<false, false>);
    }
    TG_CK(cudaGetLastError());
    return 1;
}

static int64_t launch_wedges(Graph &G, const Graph::Chunk &c, cudaStream_t s) {
    G.a_base = c.s0;
    const GraphView gv = G.view();
    const CountView cv = G.cview();
    const int sms = sm_count();
    int64_t launches = 0;
    const int L = G.L;
    if (c.s1 > c.s0)
        TG_CK(cudaMemset2DAsync(G.A.p, (size_t)G.a_stride * sizeof(uint32_t), 0, (size_t)(c.s1 - c.s0) * sizeof(uint32_t),
                                (size_t)L * L, s));
    if (G.n_anchors_light > 0) {
        int cap = 1;
        while (cap < 2 * G.opt.light_anchor_max_wedges) cap <<= 1;
        const size_t smem = (size_t)kLightAnchorWarps * cap * (1 + L) * sizeof(int32_t);
        KernelTimer kt(G, s, "k_wedge_light");
        k_wedge_light<<<grid_for(G.n_anchors_light, kLightAnchorWarps, sms * 8), kLightAnchorWarps * 32, smem, s>>>(
            gv, cv, G.anchors_light.as<int32_t>(), G.n_anchors_light, cap, c.n0, c.n1);
        ++launches;
    }
    if (G.n_hubs > 0) launches += launch_hubs(G, (size_t)(&c - G.chunks.data()), s);
    if (G.n_anchors_heavy > 0) {
        KernelTimer kt(G, s, "k_wedge_heavy");
        const int grid = (int)std::min<int64_t>(std::max<int64_t>(G.n_tables, 2 * sms), G.n_anchors_heavy);
        k_wedge_heavy<<<std::max(grid, G.n_tables), kAnchorThreads, (size_t)kHeavyCap * (1 + L) * sizeof(int32_t), s>>>(
            gv, cv, G.anchors_heavy.as<int32_t>(), G.n_anchors_heavy, G.n_heavy_dense, G.n_tables, c.n0, c.n1);
        ++launches;
    }
    TG_CK(cudaGetLastError());
    return launches;
}

// per-edge 4-node stage of edges [b, e) (inside one chunk, whose wedge pass
// is in A): T offsets, T lists and sums, K, orbits
static int64_t launch_edges4(Graph &G, int64_t b, int64_t e, const Tile *tiles, int64_t n_tiles, int64_t row_base,
                             uint32_t *per_edge_out, unsigned long long *gacc, cudaStream_t s) {
    if (e <= b) return 0;
    G.e_base = b;
    const GraphView gv = G.view();
    const CountView cv = G.cview();
    const int sms = sm_count();
    const int64_t ne = e - b;
    const int64_t big_t = std::max<int64_t>(G.opt.light_edge_max_degree, 32);
    int64_t launches = 0;
    TG_CK(cudaMemsetAsync(G.big_count.p, 0, sizeof(unsigned long long), s));
    {
        KernelTimer kt(G, s, "k_tcount");
        k_tcount<<<grid_for(ne + 1, 256, 1 << 30), 256, 0, s>>>(gv, cv, b, e, big_t, G.tcount.as<int64_t>(),
                                                                G.big_list.as<int32_t>(),
                                                                G.big_count.as<unsigned long long>());
        ++launches;
    }
    size_t tmp_bytes = G.scan_tmp_bytes;
    TG_CK(cub::DeviceScan::ExclusiveSum(G.scan_tmp.p, tmp_bytes, G.tcount.as<int64_t>(), G.toffs.as<int64_t>(),
                                        ne + 1, s));
    {
        KernelTimer kt(G, s, "k_tsum");
        const unsigned grid = (unsigned)grid_for(ne, 8, sms * 32);
        const bool merge = isect_any_merge(G.opt.isect_modes);
        if (G.max_degree < (1 << 16)) {
            if (merge) k_tsum<uint32_t, true><<<grid, 256, 0, s>>>(gv, cv, b, e);
            else k_tsum<uint32_t, false><<<grid, 256, 0, s>>>(gv, cv, b, e);
        } else {
            if (merge) k_tsum<unsigned long long, true><<<grid, 256, 0, s>>>(gv, cv, b, e);
            else k_tsum<unsigned long long, false><<<grid, 256, 0, s>>>(gv, cv, b, e);
        }
        ++launches;
    }
    {
        KernelTimer kt(G, s, "k_clique");
        if (G.L <= 5) k_clique<uint32_t><<<grid_for(ne, 8, sms * 32), 256, 0, s>>>(gv, cv, b, e, big_t);
        else k_clique<unsigned long long><<<grid_for(ne, 8, sms * 32), 256, 0, s>>>(gv, cv, b, e, big_t);
        ++launches;
    }
    {
        KernelTimer kt(G, s, "k_clique_big");
        if (G.L <= 5)
            k_clique_big<uint32_t><<<G.big_blocks, 256, kBigSetSmem * sizeof(int32_t), s>>>(
                gv, cv, b, G.big_list.as<int32_t>(), G.big_count.as<unsigned long long>(), G.set_scratch.as<int32_t>(),
                G.set_stride);
        else
            k_clique_big<unsigned long long><<<G.big_blocks, 256, kBigSetSmem * sizeof(int32_t), s>>>(
                gv, cv, b, G.big_list.as<int32_t>(), G.big_count.as<unsigned long long>(), G.set_scratch.as<int32_t>(),
                G.set_stride);
        ++launches;
    }
    if (n_tiles > 0 && G.pa_active) {
        KernelTimer kt(G, s, "k_epi4_pa");
        const int copies = epi4_pa_copies((int)G.pa.G);
        k_epi4_pa<<<grid_for(n_tiles, 1, sms * G.opt.ctas_per_sm), 256,
                    epi4_pa_hist_words((int)G.pa.G) * copies * sizeof(unsigned long long), s>>>(
            gv, cv, pa_view(G), tiles, n_tiles, row_base, per_edge_out, gacc, copies);
        ++launches;
    } else if (n_tiles > 0) {
        KernelTimer kt(G, s, "k_epi4");
        const int copies = epi4_copies(G.L);
        k_epi4<<<grid_for(n_tiles, 1, sms * G.opt.ctas_per_sm), 256, epi4_smem_bytes(G.L, copies), s>>>(
            gv, cv, tiles, n_tiles, row_base, per_edge_out, gacc, copies);
        ++launches;
    }
    TG_CK(cudaGetLastError());
    return launches;
}


// Allocates the working arrays of a count with this k (kept by the handle).
void prepare_counting(Graph &G, int k, cudaStream_t s) {
    const int L = G.L;
    const size_t m = (size_t)std::max<int64_t>(G.m, 1), n = (size_t)std::max<int64_t>(G.n, 1);
    if (G.C.bytes < m * L * sizeof(uint32_t)) G.C.alloc(m * L * sizeof(uint32_t));
    if (G.tau.bytes < n * L * L * sizeof(int64_t)) G.tau.alloc(n * L * L * sizeof(int64_t));
    const size_t gbytes = (size_t)G.ngraphs * global_slots(L, 4) * sizeof(unsigned long long);
    if (G.gacc.bytes < gbytes) G.gacc.alloc(gbytes);
    if (k == 4) {
        if (G.chunks.empty()) plan_chunks(G);
        const size_t ab = (size_t)G.a_stride * L * L * sizeof(uint32_t);
        if (G.A.bytes < ab) G.A.alloc(ab);
        const size_t me = (size_t)std::max<int64_t>(G.max_chunk_edges, 1);
        if (G.tcount.bytes < (me + 1) * sizeof(int64_t)) {
            G.tcount.alloc((me + 1) * sizeof(int64_t));
            G.toffs.alloc((me + 1) * sizeof(int64_t));
            G.tsum.alloc(me * 3 * L * L * sizeof(unsigned long long));
            G.kmat.alloc(me * L * L * sizeof(unsigned long long));
            G.big_list.alloc(me * sizeof(int32_t));
            G.big_count.alloc(sizeof(unsigned long long));
            size_t tb = 0;
            TG_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, G.tcount.as<int64_t>(), G.toffs.as<int64_t>(),
                                                (int64_t)me + 1, s));
            G.scan_tmp.alloc(tb);
            G.scan_tmp_bytes = tb;
        }
        if (G.n_hubs > 0 && !G.hubs_ready) prepare_hubs(G, s);
        if (G.n_hubs > 0 && G.hub_plans.empty()) plan_hubs(G, s);
        if (G.n_anchors_heavy > 0 && G.n_tables == 0) {
            const int64_t stride = std::max<int64_t>(G.max_graph_nodes, 1) * L;
            const int64_t per = stride * (int64_t)sizeof(uint32_t);
            int64_t budget = (int64_t)G.opt.anchor_table_budget_mb << 20;
            const int64_t need = G.n_anchors_heavy;
            int64_t nt = std::min<int64_t>({(int64_t)2 * sm_count(), need, std::max<int64_t>(budget / per, 1)});
            G.tables.alloc((size_t)(nt * per));
            TG_CK(cudaMemsetAsync(G.tables.p, 0, (size_t)(nt * per), s));
            G.table_stride = stride;
            G.n_tables = (int32_t)nt;
        }
    }
}

// For a captured count: the T list size needs one k_tri before capture.
void prepare_capture(Graph &G, int k, cudaStream_t s) {
    if (k == 4 && G.chunk_t.empty()) {
        launch_triangles(G, s);
        ensure_t_sizes(G, s);
    }
}

int64_t run_count(Graph &G, int k, int64_t e_begin, int64_t e_end, uint32_t *per_edge_out, unsigned long long *gacc,
                  bool full, cudaStream_t s) {
    int64_t launches = 0;
    if (full || G.prepared_k < 3) {
        launches += launch_triangles(G, s);
        G.prepared_k = std::max(G.prepared_k, 3);
    }
    DBuf tmp;                                                // tiles of a range, stream-ordered
    tmp.owner = &G.stream;
    int64_t n_tiles = 0;
    const Tile *tiles = tiles_for(G, e_begin, e_end, n_tiles, tmp, s);
    if (k == 3) {
        if (n_tiles > 0) {
            const GraphView gv = G.view();
            const CountView cv = G.cview();
            KernelTimer kt(G, s, "k_edge3");
            k_edge3<<<grid_for(n_tiles, 1, sm_count() * 8), 256, hist_bytes(G.L, 3), s>>>(gv, cv, tiles, n_tiles, e_begin,
                                                                                       per_edge_out, gacc);
            ++launches;
            TG_CK(cudaGetLastError());
        }
    } else {
        ensure_t_sizes(G, s);
        const bool whole = e_begin == 0 && e_end == G.m;
        std::vector<Tile> host;
        if (!whole) host = make_tiles(G, e_begin, e_end);
        for (const Graph::Chunk &c : G.chunks) {
            const int64_t b = std::max(e_begin, c.e0), e = std::min(e_end, c.e1);
            if (b >= e) continue;
            // the wedge pass of a single-chunk handle is reused by later range calls
            if (full || G.chunks.size() > 1 || G.prepared_k != 4) {
                launches += launch_wedges(G, c, s);
                if (G.chunks.size() == 1) G.prepared_k = 4;
            }
            G.a_base = c.s0;
            const Tile *ct = tiles;
            int64_t nct = n_tiles;
            if (whole) {
                ct = tiles + c.t0;
                nct = c.t1 - c.t0;
            } else {
                int64_t a = 0;
                while (a < n_tiles && host[a].end <= b) ++a;
                int64_t y = a;
                while (y < n_tiles && host[y].begin < e) ++y;
                ct = tiles + a;
                nct = y - a;
            }
            launches += launch_edges4(G, b, e, ct, nct, e_begin, per_edge_out, gacc, s);
        }
    }
    if (tmp.p) TG_CK(cudaStreamSynchronize(s));
    return launches;
}

int64_t launch_finalize(Graph &G, int k, int64_t *global_out, cudaStream_t s) {
    const int64_t total = (int64_t)G.ngraphs * global_slots(G.L, k);
    KernelTimer kt(G, s, "k_finalize");
    k_finalize<<<grid_for(total, 256, 1 << 20), 256, 0, s>>>(G.ngraphs, G.L, k, G.gacc.as<unsigned long long>(), global_out,
                                                              G.status.as<uint32_t>());
    TG_CK(cudaGetLastError());
    return 1;
}

}  // namespace tg

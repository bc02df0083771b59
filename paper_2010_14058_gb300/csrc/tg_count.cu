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
//   TCi[t][t']  sum_{w in T^t} c_{iw}^{t'}                         (k_edge4)
//   TCj[t][t']  sum_{w in T^t} c_{jw}^{t'}                         (k_edge4)
//   DT[t][t']   sum_{w in T^t} d_w^{t'}                            (k_edge4)
//   K[t][t']    ordered adjacent pairs (w,x) in T^t x T^t'         (k_edge4)
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

#include "tg_host.hpp"

namespace tg {

namespace {

constexpr int kEdgeThreads = 256;           // k_edge4_light: 8 warps, one edge each
constexpr int kHeavyThreads = 512;          // k_edge4_heavy: one edge per CTA
constexpr int kAnchorThreads = 512;         // k_wedge_heavy: one anchor per CTA
constexpr int kLightAnchorWarps = 4;        // k_wedge_light: one anchor per warp
constexpr int kTCapWarp = 256;              // T list capacity of a warp (light edges: |T| <= 256)
constexpr int kTCapSmemHeavy = 8192;        // T list capacity in shared memory for a heavy edge
constexpr int kTile = 2048;                 // edges per tile of k_edge4_light

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
// Warp per edge: c_e^t = |Gamma_i^t cap Gamma_j^t| by searching each element
// of the shorter typed segment in the longer one (Cor. 1; Thm. 2's O(Delta)).
__global__ void __launch_bounds__(256) k_tri(GraphView g, CountView cv) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < g.m; e += nw) {
        const int32_t i = g.e_lo[e], j = g.e_hi[e];
        for (int t = 0; t < g.L; ++t) {
            int64_t bi = seg_begin(g, i, t), ei = seg_end(g, i, t);
            int64_t bj = seg_begin(g, j, t), ej = seg_end(g, j, t);
            if (ei - bi > ej - bj) {
                int64_t x = bi; bi = bj; bj = x;
                x = ei; ei = ej; ej = x;
            }
            unsigned cnt = 0;
            for (int64_t s = bi + lane; s < ei; s += 32) {
                int32_t w = g.adj[s];
                int64_t r = lower_bound_i32(g.adj, bj, ej, w);
                cnt += (r < ej && g.adj[r] == w) ? 1u : 0u;
            }
            cnt = warp_sum_u32(cnt);
            if (lane == 0) cv.C[e * g.L + t] = cnt;
        }
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

// Light anchors (few wedges): one warp per anchor, table in shared memory.
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
    for (int64_t a = (int64_t)blockIdx.x * kLightAnchorWarps + wid; a < n_anchors; a += nw) {
        const int32_t u = anchors[a];
        if (u < n0 || u >= n1) continue;                    // anchor outside this chunk
        const int tu = g.ty[u];
        // phase 1
        for (int tv = 0; tv < L; ++tv) {
            int64_t ub, ucut;
            seg_prefix(g, u, tv, u, ub, ucut);
            for (int64_t sv = ub; sv < ucut; ++sv) {
                const int32_t v = g.adj[sv];
                for (int tw = 0; tw < L; ++tw) {
                    int64_t vb, vcut;
                    seg_prefix(g, v, tw, u, vb, vcut);
                    for (int64_t k = vb + lane; k < vcut; k += 32) {
                        int h = hash_insert(keys, cap, g.adj[k]);
                        if (h >= 0) atomicAdd(&cnt[h * L + tv], 1u);
                        else set_status(cv.status, ST_INTERNAL);
                    }
                }
            }
        }
        __syncwarp();
        // phase 2
        for (int tv = 0; tv < L; ++tv) {
            int64_t ub, ucut;
            seg_prefix(g, u, tv, u, ub, ucut);
            for (int64_t sv = ub; sv < ucut; ++sv) {
                const int32_t v = g.adj[sv];
                for (int tw = 0; tw < L; ++tw) {
                    int64_t vb, vcut;
                    seg_prefix(g, v, tw, u, vb, vcut);
                    unsigned acc[kMaxL];
#pragma unroll
                    for (int t = 0; t < kMaxL; ++t) acc[t] = 0;
                    for (int64_t k = vb + lane; k < vcut; k += 32) {
                        int h = hash_find(keys, cap, g.adj[k]);
                        if (h < 0) continue;
#pragma unroll
                        for (int t = 0; t < kMaxL; ++t) {
                            if (t >= L) break;
                            unsigned c = cnt[h * L + t] - (t == tv ? 1u : 0u);
                            if (c) {
                                atomicAdd(&A[(int64_t)(tu * L + t) * nnz + k], c);
                                acc[t] += c;
                            }
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kMaxL; ++t) {
                        if (t >= L) break;
                        unsigned r = warp_sum_u32(acc[t]);
                        if (lane == 0 && r) atomicAdd(&A[(int64_t)(t * L + tw) * nnz + sv], r);
                    }
                }
            }
        }
        __syncwarp();
        for (int k = lane; k < cap; k += 32) keys[k] = -1;
        for (int k = lane; k < cap * L; k += 32) cnt[k] = 0;
        __syncwarp();
    }
}

// Heavy anchors: one CTA per anchor, dense table in this CTA's global slice
// indexed by (w - first node of u's graph).  Warps take the v in V_u.
__global__ void __launch_bounds__(kAnchorThreads) k_wedge_heavy(GraphView g, CountView cv,
                                                               const int32_t *__restrict__ anchors,
                                                               int64_t n_anchors, int64_t n0, int64_t n1) {
    __shared__ int64_t s_b[kMaxL + 1], s_cnt[kMaxL + 1];
    const int L = g.L;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    uint32_t *tbl = cv.tables + (int64_t)blockIdx.x * cv.table_stride;
    const int64_t nnz = cv.a_stride;
    uint32_t *A = cv.A - cv.a_base;                          // indexed by absolute slot
    for (int64_t a = blockIdx.x; a < n_anchors; a += gridDim.x) {
        const int32_t u = anchors[a];
        if (u < n0 || u >= n1) continue;                    // anchor outside this chunk (uniform per CTA)
        const int tu = g.ty[u];
        const int64_t base = g.node_off[graph_of_node(g, u)];
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
        const int64_t nV = s_cnt[L];
        for (int phase = 0; phase < 3; ++phase) {
            for (int64_t kv = wid; kv < nV; kv += nwarp) {
                int tv = 0;
                while (tv + 1 < L && s_cnt[tv + 1] <= kv) ++tv;
                const int64_t sv = s_b[tv] + (kv - s_cnt[tv]);
                const int32_t v = g.adj[sv];
                for (int tw = 0; tw < L; ++tw) {
                    int64_t vb, vcut;
                    seg_prefix(g, v, tw, u, vb, vcut);
                    if (phase == 0) {
                        for (int64_t k = vb + lane; k < vcut; k += 32)
                            atomicAdd(&tbl[(g.adj[k] - base) * L + tv], 1u);
                    } else if (phase == 1) {
                        unsigned acc[kMaxL];
#pragma unroll
                        for (int t = 0; t < kMaxL; ++t) acc[t] = 0;
                        for (int64_t k = vb + lane; k < vcut; k += 32) {
                            const uint32_t *h = tbl + (g.adj[k] - base) * L;
#pragma unroll
                            for (int t = 0; t < kMaxL; ++t) {
                                if (t >= L) break;
                                unsigned c = h[t] - (t == tv ? 1u : 0u);
                                if (c) {
                                    atomicAdd(&A[(int64_t)(tu * L + t) * nnz + k], c);
                                    acc[t] += c;
                                }
                            }
                        }
#pragma unroll
                        for (int t = 0; t < kMaxL; ++t) {
                            if (t >= L) break;
                            unsigned r = warp_sum_u32(acc[t]);
                            if (lane == 0 && r) atomicAdd(&A[(int64_t)(t * L + tw) * nnz + sv], r);
                        }
                    } else {
                        for (int64_t k = vb + lane; k < vcut; k += 32) {
                            uint32_t *h = tbl + (g.adj[k] - base) * L;
                            for (int t = 0; t < L; ++t) h[t] = 0;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ per-edge 4-node
// Shared workspace of one edge.
struct EdgeWs {
    unsigned long long TCi[kMaxL * kMaxL], TCj[kMaxL * kMaxL], DT[kMaxL * kMaxL], K[kMaxL * kMaxL];
    int64_t Pm[kMaxL * kMaxL];                  // 3-paths j - w - r - i by (type w, type r); then Q
    int64_t Ks[kMaxL * kMaxL];                  // ordered adjacent pairs in T (K + K^T)
    int64_t taui[kMaxL * kMaxL], tauj[kMaxL * kMaxL], deli[kMaxL * kMaxL], delj[kMaxL * kMaxL];
    int64_t c[kMaxL], a[kMaxL], b[kMaxL], di[kMaxL], dj[kMaxL];
    int32_t tstart[kMaxL + 1];   // T list offsets per type
    int32_t nT;
    int32_t p, q;                // types of the endpoints
    int32_t wcount[32];          // per-warp compaction counts (CTA variant)
};

// Enumerates T_ij (typed intersection), appends it to Tlist in (type, id)
// order and accumulates TCi, TCj, DT.  `gsize` threads of the group, thread
// rank `gr`; the group has gsize/32 warps.  bar() is the group barrier.
template <class Bar>
__device__ void enumerate_T(const GraphView &g, const CountView &cv, int64_t e, int32_t i, int32_t j, EdgeWs &ws,
                            int32_t *Tlist, int64_t Tcap, int gsize, int gr, Bar bar) {
    const int L = g.L;
    const int lane = gr & 31, wid = gr >> 5, nwarp = gsize >> 5;
    int32_t base = 0;
    for (int t = 0; t < L; ++t) {
        if (gr == 0) ws.tstart[t] = base;
        const uint32_t ct = cv.C[e * L + t];      // |T_ij^t| from k_tri: nothing to find when 0
        if (ct == 0) continue;
        int64_t bi = seg_begin(g, i, t), ei = seg_end(g, i, t);
        int64_t bj = seg_begin(g, j, t), ej = seg_end(g, j, t);
        bool swapped = false;
        if (ei - bi > ej - bj) {
            int64_t x = bi; bi = bj; bj = x;
            x = ei; ei = ej; ej = x;
            swapped = true;
        }
        // per-thread sums over this type segment, reduced per warp at its end
        unsigned long long a_ci[kMaxL], a_cj[kMaxL], a_dt[kMaxL];
#pragma unroll
        for (int q = 0; q < kMaxL; ++q) { a_ci[q] = 0; a_cj[q] = 0; a_dt[q] = 0; }
        for (int64_t r0 = bi; r0 < ei; r0 += gsize) {
            const int64_t s = r0 + gr;
            bool found = false;
            int64_t r = -1;
            int32_t w = 0;
            if (s < ei) {
                w = g.adj[s];
                r = lower_bound_i32(g.adj, bj, ej, w);
                found = r < ej && g.adj[r] == w;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, found);
            if (nwarp > 1) {
                if (lane == 0) ws.wcount[wid] = __popc(bal);
                bar();
            }
            int32_t off = base;
            int32_t total = __popc(bal);
            if (nwarp > 1) {
                total = 0;
                for (int q = 0; q < nwarp; ++q) {
                    if (q < wid) off += ws.wcount[q];
                    total += ws.wcount[q];
                }
            }
            if (found) {
                const int32_t pos = off + __popc(bal & ((1u << lane) - 1u));
                if (pos < Tcap) Tlist[pos] = w;
                else set_status(cv.status, ST_INTERNAL);
                const int64_t si = swapped ? r : s, sj = swapped ? s : r;   // slots of w in rows i and j
                const uint32_t *ci = cv.C + (int64_t)g.slot_eid[si] * L;
                const uint32_t *cj = cv.C + (int64_t)g.slot_eid[sj] * L;
                const int32_t *o = g.toff + (int64_t)w * (L + 1);
#pragma unroll
                for (int q = 0; q < kMaxL; ++q) {
                    if (q < L) {
                        a_ci[q] += ci[q];
                        a_cj[q] += cj[q];
                        a_dt[q] += (unsigned)(o[q + 1] - o[q]);
                    }
                }
            }
            base += total;
            if (nwarp > 1) bar();
        }
        if (bi < ei) {
#pragma unroll
            for (int q = 0; q < kMaxL; ++q) {
                if (q >= L) break;
                const unsigned long long x1 = warp_sum_u64(a_ci[q]), x2 = warp_sum_u64(a_cj[q]), x3 = warp_sum_u64(a_dt[q]);
                if (lane == 0) {
                    if (x1) atomicAdd(&ws.TCi[t * kMaxL + q], x1);
                    if (x2) atomicAdd(&ws.TCj[t * kMaxL + q], x2);
                    if (x3) atomicAdd(&ws.DT[t * kMaxL + q], x3);
                }
            }
        }
    }
    if (gr == 0) {
        ws.tstart[L] = base;
        ws.nT = base;
    }
    bar();
}

// K: adjacent pairs (w, x) of T with w < x, by type.  For each w, either
// scan N+(w) = {x in Gamma_w : x > w} (all types, flattened over the warp's
// lanes, each x looked up in T's sorted segment of its type), or take each
// x > w of T and look it up in Gamma_w -- whichever touches fewer entries.
template <class Bar>
__device__ void count_K(const GraphView &g, EdgeWs &ws, const int32_t *Tlist, int gsize, int gr, Bar bar) {
    const int L = g.L;
    const int lane = gr & 31, wid = gr >> 5, nwarp = gsize >> 5;
    const int32_t nT = ws.nT;
    if (nT < 2) {
        bar();
        return;
    }
    int32_t ts[kMaxL + 1];
#pragma unroll
    for (int q = 0; q <= kMaxL; ++q) ts[q] = q <= L ? ws.tstart[q] : nT;
    const int32_t npair = nT * (nT - 1) / 2;
    if (npair <= 2 * gsize) {
        // few pairs: one pair {T[a], T[b]} per thread, adjacency by binary search
        // of the larger id in the smaller id's typed segment; each adjacent pair
        // is counted once, as (smaller id, larger id)
        for (int32_t pk = gr; pk < npair; pk += gsize) {
            int32_t a = 0, rem = pk;
            while (rem >= nT - 1 - a) { rem -= nT - 1 - a; ++a; }
            const int32_t b = a + 1 + rem;
            int ta = 0, tb = 0;
#pragma unroll
            for (int qq = 1; qq < kMaxL; ++qq) {
                ta += (qq < L && ts[qq] <= a) ? 1 : 0;
                tb += (qq < L && ts[qq] <= b) ? 1 : 0;
            }
            int32_t w = Tlist[a], x = Tlist[b];
            int tw = ta, tx = tb;
            if (x < w) { int32_t y = w; w = x; x = y; int ty = tw; tw = tx; tx = ty; }
            const int64_t sb = seg_begin(g, w, tx), se = seg_end(g, w, tx);
            const int64_t r = lower_bound_i32(g.adj, sb, se, x);
            if (r < se && g.adj[r] == x) atomicAdd(&ws.K[tw * kMaxL + tx], 1ull);
        }
        bar();
        return;
    }
    for (int32_t kw = wid; kw < nT; kw += nwarp) {
        const int32_t w = Tlist[kw];
        int tw = 0;
#pragma unroll
        for (int q = 1; q < kMaxL; ++q) tw += (q < L && ts[q] <= kw) ? 1 : 0;
        // N+(w) per type: [pb_q, pb_q + cnt_q)
        int64_t pb = 0;
        int32_t cnt = 0;
        const int64_t rw = g.rp[w];
        if (lane < L) {
            pb = rw + g.pivot[(int64_t)w * L + lane];
            cnt = (int32_t)(rw + g.toff[(int64_t)w * (L + 1) + lane + 1] - pb);
        }
        int32_t pre = cnt;                                   // inclusive prefix over lanes < L
#pragma unroll
        for (int o = 1; o < kMaxL; o <<= 1) {
            int32_t v = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += v;
        }
        int64_t pbq[kMaxL];
        int32_t preq[kMaxL];
#pragma unroll
        for (int q = 0; q < kMaxL; ++q) {
            pbq[q] = __shfl_sync(0xffffffffu, pb, q);
            preq[q] = q < L ? __shfl_sync(0xffffffffu, pre, q) : 0x7fffffff;
        }
        const int32_t dplus = preq[L - 1];
        if (dplus == 0) continue;
        unsigned cq[kMaxL];
#pragma unroll
        for (int q = 0; q < kMaxL; ++q) cq[q] = 0;
        int lgT = 1;
        while ((1 << lgT) < nT + 1) ++lgT;
        const int64_t dw = g.rp[w + 1] - rw;
        int lgd = 1;
        while ((1ll << lgd) < dw + 1) ++lgd;
        // members of T above w, per type: [tg_q, ts_{q+1}) (each T segment is id-sorted)
        int32_t tgt = 0;
        if (lane < L) {
            int32_t lo = ts[0], hi = ts[0];
#pragma unroll
            for (int qq = 0; qq < kMaxL; ++qq)
                if (qq == lane) { lo = ts[qq]; hi = ts[qq + 1]; }
            while (lo < hi) {
                int32_t mid = (lo + hi) >> 1;
                if (Tlist[mid] <= w) lo = mid + 1; else hi = mid;
            }
            tgt = lo;
        }
        int32_t above = 0;
        if (lane < L) {
            int32_t te = 0;
#pragma unroll
            for (int qq = 0; qq < kMaxL; ++qq)
                if (qq == lane) te = ts[qq + 1];
            above = te - tgt;
        }
        int32_t nabove = above;
        for (int o = 16; o > 0; o >>= 1) nabove += __shfl_xor_sync(0xffffffffu, nabove, o);
        if (nabove == 0) continue;
        if ((int64_t)dplus * lgT <= (int64_t)nabove * lgd) {
            for (int32_t f = lane; f < dplus; f += 32) {
                int q = 0;
#pragma unroll
                for (int qq = 0; qq < kMaxL - 1; ++qq) q += (f >= preq[qq]) ? 1 : 0;
                int64_t slot = 0;
#pragma unroll
                for (int qq = 0; qq < kMaxL; ++qq)
                    if (qq == q) slot = pbq[qq] + (f - (qq ? preq[qq - 1] : 0));
                const int32_t x = g.adj[slot];
                int32_t lo = 0, hi = 0;
#pragma unroll
                for (int qq = 0; qq < kMaxL; ++qq)
                    if (qq == q) { lo = ts[qq]; hi = ts[qq + 1]; }
                const int32_t te = hi;
                while (lo < hi) {
                    int32_t mid = (lo + hi) >> 1;
                    if (Tlist[mid] < x) lo = mid + 1; else hi = mid;
                }
                if (lo < te && Tlist[lo] == x) {
#pragma unroll
                    for (int qq = 0; qq < kMaxL; ++qq) cq[qq] += (qq == q) ? 1u : 0u;
                }
            }
        } else {
            for (int q = 0; q < L; ++q) {
                const int32_t kb = __shfl_sync(0xffffffffu, tgt, q);
                const int32_t ke = ts[q + 1 <= kMaxL ? q + 1 : kMaxL];
                if (kb >= ke) continue;
                const int64_t b = seg_begin(g, w, q), e = seg_end(g, w, q);
                if (b == e) continue;
                unsigned c = 0;
                for (int32_t k = kb + lane; k < ke; k += 32) {
                    const int32_t x = Tlist[k];
                    const int64_t r = lower_bound_i32(g.adj, b, e, x);
                    c += (r < e && g.adj[r] == x) ? 1u : 0u;
                }
#pragma unroll
                for (int qq = 0; qq < kMaxL; ++qq) cq[qq] += (qq == q) ? c : 0u;
            }
        }
#pragma unroll
        for (int q = 0; q < kMaxL; ++q) {
            if (q >= L) break;
            unsigned v = warp_sum_u32(cq[q]);
            if (lane == 0 && v) atomicAdd(&ws.K[tw * kMaxL + q], (unsigned long long)v);
        }
    }
    bar();
}

// Derived typed counts of one edge, each matrix entry computed once, in
// place, in dependency order (x, y index types; z = x * kMaxL + y):
//   Ks  = K + K^T                       ordered adjacent pairs in T
//   TCi -> CTi = TCi - Ks - [y=q] c_x   (w in T^x, r in S_i^y adjacent)
//   TCj -> CTj = TCj - Ks - [y=p] c_x
//   taui -> Wi = tau_i - CTi - CTi^T - Ks - [x=q] c_y - [y=q] c_x
//   tauj -> Wj = tau_j - CTj - CTj^T - Ks - [x=p] c_y - [y=p] c_x
//   Pm  -> Q   = P - CTj^T - CTi - Ks  (w in S_j^x, r in S_i^y: 4-cycles)
//   deli -> Ri = delta_i - DT - [x=q] d_j^y - [y=p] a_x - Wi - CTi^T - Q^T
//   delj -> Rj = delta_j - DT - [x=p] d_i^y - [y=q] b_x - Wj - CTj^T - Q
//   DT  -> G8  = DT - ([y=p]+[y=q]) c_x - Ks - CTi - CTj
template <class Bar>
__device__ void derive_matrices(EdgeWs &ws, int L, int gsize, int gr, Bar bar) {
    const int p = ws.p, q = ws.q;
    const int n2 = L * L;
    for (int k = gr; k < n2; k += gsize) {
        const int x = k / L, y = k % L, z = x * kMaxL + y, zt = y * kMaxL + x;
        ws.Ks[z] = (int64_t)ws.K[z] + (int64_t)ws.K[zt];
    }
    bar();
    for (int k = gr; k < n2; k += gsize) {
        const int x = k / L, y = k % L, z = x * kMaxL + y;
        ws.TCi[z] = (unsigned long long)((int64_t)ws.TCi[z] - ws.Ks[z] - (y == q ? ws.c[x] : 0));
        ws.TCj[z] = (unsigned long long)((int64_t)ws.TCj[z] - ws.Ks[z] - (y == p ? ws.c[x] : 0));
    }
    bar();
    const long long *CTi = reinterpret_cast<const long long *>(ws.TCi);
    const long long *CTj = reinterpret_cast<const long long *>(ws.TCj);
    for (int k = gr; k < n2; k += gsize) {
        const int x = k / L, y = k % L, z = x * kMaxL + y, zt = y * kMaxL + x;
        ws.taui[z] = ws.taui[z] - CTi[z] - CTi[zt] - ws.Ks[z] - (x == q ? ws.c[y] : 0) - (y == q ? ws.c[x] : 0);
        ws.tauj[z] = ws.tauj[z] - CTj[z] - CTj[zt] - ws.Ks[z] - (x == p ? ws.c[y] : 0) - (y == p ? ws.c[x] : 0);
        ws.Pm[z] = ws.Pm[z] - CTj[zt] - CTi[z] - ws.Ks[z];
    }
    bar();
    for (int k = gr; k < n2; k += gsize) {
        const int x = k / L, y = k % L, z = x * kMaxL + y, zt = y * kMaxL + x;
        const int64_t dt = (int64_t)ws.DT[z];
        ws.deli[z] = ws.deli[z] - dt - (x == q ? ws.dj[y] : 0) - (y == p ? ws.a[x] : 0) - ws.taui[z] - CTi[zt] - ws.Pm[zt];
        ws.delj[z] = ws.delj[z] - dt - (x == p ? ws.di[y] : 0) - (y == q ? ws.b[x] : 0) - ws.tauj[z] - CTj[zt] - ws.Pm[z];
    }
    bar();
    for (int k = gr; k < n2; k += gsize) {
        const int x = k / L, y = k % L, z = x * kMaxL + y;
        ws.DT[z] = (unsigned long long)((int64_t)ws.DT[z] - ((y == p ? 1 : 0) + (y == q ? 1 : 0)) * ws.c[x] - ws.Ks[z] -
                                        CTi[z] - CTj[z]);
    }
    bar();
}

// Orbit values of one type pair (t <= u) from the derived matrices;
// returns false if an internal identity fails (negative count, odd diagonal).
__device__ __noinline__ bool orbit_values(const EdgeWs &ws, int t, int u, int64_t *gv /*[10]: g3..g12*/) {
    const long long *CTi = reinterpret_cast<const long long *>(ws.TCi);
    const long long *CTj = reinterpret_cast<const long long *>(ws.TCj);
    const long long *G8 = reinterpret_cast<const long long *>(ws.DT);
    const int tu = t * kMaxL + u, ut = u * kMaxL + t, tt = t * kMaxL + t;
    bool ok = true;
    int64_t g3, g6, g7, g8, g10, g12;
    if (t != u) {
        g3 = ws.deli[tu] + ws.delj[tu] + ws.deli[ut] + ws.delj[ut];   // Ri + Rj, both orders
        g6 = ws.Pm[tu] + ws.Pm[ut];                                   // Q
        g7 = ws.taui[tu] + ws.tauj[tu];                               // Wi + Wj
        g8 = G8[tu] + G8[ut];
        g10 = CTi[tu] + CTj[tu] + CTi[ut] + CTj[ut];
        g12 = ws.Ks[tu];
    } else {
        g3 = ws.deli[tt] + ws.delj[tt];
        g6 = ws.Pm[tt];
        const int64_t w2 = ws.taui[tt] + ws.tauj[tt], k2 = ws.Ks[tt];
        ok = !(w2 & 1) && !(k2 & 1);
        g7 = w2 / 2;
        g8 = G8[tt];
        g10 = CTi[tt] + CTj[tt];
        g12 = k2 / 2;
    }
    const int64_t at = ws.a[t], au = ws.a[u], bt = ws.b[t], bu = ws.b[u], ct = ws.c[t], cu = ws.c[u];
    int64_t g4, g5, g9, g11;
    if (t == u) {
        g4 = at * bt - g6;                                   // Lemma 1
        g5 = at * (at - 1) / 2 + bt * (bt - 1) / 2 - g7;     // Lemma 2
        g9 = ct * (at + bt) - g10;                           // Lemma 3
        g11 = ct * (ct - 1) / 2 - g12;                       // Lemma 4
    } else {
        g4 = at * bu + au * bt - g6;
        g5 = at * au + bt * bu - g7;
        g9 = ct * (au + bu) + cu * (at + bt) - g10;
        g11 = ct * cu - g12;
    }
    gv[0] = g3; gv[1] = g4; gv[2] = g5; gv[3] = g6; gv[4] = g7;
    gv[5] = g8; gv[6] = g9; gv[7] = g10; gv[8] = g11; gv[9] = g12;
    for (int k = 0; k < 10; ++k) ok = ok && gv[k] >= 0;
    return ok;
}

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

// Epilogue of one edge: stages the per-edge inputs in shared memory, then
// writes the row and adds to the CTA histogram.
template <class Bar>
__device__ void edge_epilogue(const GraphView &g, const CountView &cv, int64_t e, int32_t i, int32_t j, EdgeWs &ws,
                              uint32_t *row, unsigned long long *hist, int gsize, int gr, Bar bar) {
    const int L = g.L;
    const int p = g.ty[i], q = g.ty[j];
    if (gr == 0) { ws.p = p; ws.q = q; }
    for (int t = gr; t < L; t += gsize) {
        const int64_t c = cv.C[e * L + t];
        const int64_t di = typed_degree(g, i, t), dj = typed_degree(g, j, t);
        ws.c[t] = c;
        ws.di[t] = di;
        ws.dj[t] = dj;
        ws.a[t] = di - c - (q == t ? 1 : 0);
        ws.b[t] = dj - c - (p == t ? 1 : 0);
    }
    const int64_t slot_ij = g.e_slot_lo[e], slot_ji = g.e_slot_hi[e];
    const int64_t *tau_i = cv.tau + (int64_t)i * L * L, *tau_j = cv.tau + (int64_t)j * L * L;
    const int64_t *del_i = g.delta + (int64_t)i * L * L, *del_j = g.delta + (int64_t)j * L * L;
    for (int k = gr; k < L * L; k += gsize) {
        const int x = k / L, y = k % L;
        const int z = x * kMaxL + y;
        // P[x][y]: 3-paths j - w - r - i with phi_w = x, phi_r = y (slot i->j holds
        // [type next to i][type next to j], slot j->i the reverse)
        const uint32_t *A = cv.A - cv.a_base;
        ws.Pm[z] = (int64_t)A[(int64_t)(y * L + x) * cv.a_stride + slot_ij] + (int64_t)A[(int64_t)(x * L + y) * cv.a_stride + slot_ji];
        ws.taui[z] = tau_i[k];
        ws.tauj[z] = tau_j[k];
        ws.deli[z] = del_i[k];
        ws.delj[z] = del_j[k];
    }
    bar();
    derive_matrices(ws, L, gsize, gr, bar);
    const int P = L * (L + 1) / 2;
    // 3-node slots and 2-node / 3-node global blocks
    for (int t = gr; t < L; t += gsize) {
        const int64_t s3 = ws.a[t] + ws.b[t];
        if (ws.a[t] < 0 || ws.b[t] < 0) set_status(cv.status, ST_INTERNAL);
        if (row) {
            row[t] = sat32(s3, cv.status);
            row[L + t] = sat32(ws.c[t], cv.status);
        }
        int ms[3] = {p, q, t};
        sort3(ms);
        const int r = multiset_rank_dev(L, 3, ms);
        if (s3) atomicAdd(&hist[gblock_off(L, 1) + r], (unsigned long long)s3);
        if (ws.c[t]) atomicAdd(&hist[gblock_off(L, 2) + r], (unsigned long long)ws.c[t]);
    }
    if (gr == 0) {
        int ms[2] = {p < q ? p : q, p < q ? q : p};
        atomicAdd(&hist[multiset_rank_dev(L, 2, ms)], 1ull);
    }
    for (int pi = gr; pi < P; pi += gsize) {
        int t = 0;
        while (pair_idx(L, t, L - 1) < pi) ++t;
        const int u = t + (pi - pair_idx(L, t, t));
        int64_t gv[10];
        if (!orbit_values(ws, t, u, gv)) set_status(cv.status, ST_INTERNAL);
        int ms[4] = {p, q, t, u};
        sort4(ms);
        const int r = multiset_rank_dev(L, 4, ms);
        for (int o = 3; o <= 12; ++o) {
            const int64_t v = gv[o - 3];
            if (row) row[2 * L + (o - 3) * P + pi] = sat32(v, cv.status);
            if (v > 0) atomicAdd(&hist[gblock_off(L, graphlet_block(o)) + r], (unsigned long long)v);
        }
    }
    bar();
}

__device__ void clear_ws(EdgeWs &ws, int gsize, int gr) {
    for (int k = gr; k < kMaxL * kMaxL; k += gsize) {
        ws.TCi[k] = 0; ws.TCj[k] = 0; ws.DT[k] = 0; ws.K[k] = 0;
    }
}

__device__ void flush_hist(unsigned long long *hist, int G, unsigned long long *gacc, int graph, int gsize, int gr) {
    for (int s = gr; s < G; s += gsize) {
        unsigned long long v = hist[s];
        if (v) atomicAdd(&gacc[(int64_t)graph * G + s], v);
        hist[s] = 0;
    }
}

struct Tile {
    int64_t begin, end;
    int32_t graph, pad;
};

// Light edges (min(d_i, d_j) <= light_max): one warp per edge, tiles of edge
// ids that never cross a graph, a per-CTA histogram for global sums.
// Dynamic shared memory: [histogram G u64][EdgeWs per warp][T list per warp].
__global__ void __launch_bounds__(kEdgeThreads, 4) k_edge4_light(GraphView g, CountView cv, const Tile *__restrict__ tiles,
                                                             int64_t n_tiles, int64_t light_max, int64_t e_begin,
                                                             uint32_t *per_edge_out, unsigned long long *gacc) {
    extern __shared__ unsigned long long dsm[];
    const int L = g.L;
    const int G = (int)global_slots(L, 4);
    const int S = (int)per_edge_slots(L, 4);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long *hist = dsm;
    EdgeWs *wsa = reinterpret_cast<EdgeWs *>(dsm + ((G + 1) & ~1));
    int32_t *tl = reinterpret_cast<int32_t *>(wsa + kEdgeThreads / 32) + wid * kTCapWarp;
    EdgeWs &ws = wsa[wid];
    for (int s = threadIdx.x; s < G; s += blockDim.x) hist[s] = 0;
    __syncthreads();
    int cur_graph = -1;
    auto wbar = []() { __syncwarp(); };
    for (int64_t ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
        const Tile tile = tiles[ti];
        if (tile.graph != cur_graph) {
            if (cur_graph >= 0) flush_hist(hist, G, gacc, cur_graph, blockDim.x, threadIdx.x);
            __syncthreads();
            cur_graph = tile.graph;
        }
        for (int64_t e = tile.begin + wid; e < tile.end; e += kEdgeThreads / 32) {
            const int32_t i = g.e_lo[e], j = g.e_hi[e];
            const int64_t di = g.rp[i + 1] - g.rp[i], dj = g.rp[j + 1] - g.rp[j];
            if ((di < dj ? di : dj) > light_max) continue;
            clear_ws(ws, 32, lane);
            __syncwarp();
            enumerate_T(g, cv, e, i, j, ws, tl, kTCapWarp, 32, lane, wbar);
            count_K(g, ws, tl, 32, lane, wbar);
            uint32_t *row = per_edge_out ? per_edge_out + (e - e_begin) * S : nullptr;
            edge_epilogue(g, cv, e, i, j, ws, row, hist, 32, lane, wbar);
        }
        __syncthreads();
    }
    if (cur_graph >= 0) flush_hist(hist, G, gacc, cur_graph, blockDim.x, threadIdx.x);
}

// Heavy edges: one CTA per edge (the list is sorted by cost, largest first).
// T lives in shared memory when it fits, else in this CTA's global slice.
__global__ void __launch_bounds__(kHeavyThreads, 2) k_edge4_heavy(GraphView g, CountView cv, const int32_t *__restrict__ list,
                                                              int64_t n_list, int64_t e_begin, int64_t e_end,
                                                              int64_t row_base, uint32_t *per_edge_out,
                                                              unsigned long long *gacc, int32_t *tscratch,
                                                              int64_t tscratch_stride) {
    extern __shared__ unsigned long long dsm[];
    const int L = g.L;
    const int G = (int)global_slots(L, 4);
    const int S = (int)per_edge_slots(L, 4);
    unsigned long long *hist = dsm;
    EdgeWs &ws = *reinterpret_cast<EdgeWs *>(dsm + ((G + 1) & ~1));
    int32_t *tl_smem = reinterpret_cast<int32_t *>(&ws + 1);
    for (int s = threadIdx.x; s < G; s += blockDim.x) hist[s] = 0;
    __syncthreads();
    auto bbar = []() { __syncthreads(); };
    int cur_graph = -1;
    for (int64_t k = blockIdx.x; k < n_list; k += gridDim.x) {
        const int64_t e = list[k];
        if (e < e_begin || e >= e_end) continue;
        const int graph = graph_of_edge(g, e);
        if (graph != cur_graph) {
            if (cur_graph >= 0) flush_hist(hist, G, gacc, cur_graph, blockDim.x, threadIdx.x);
            __syncthreads();
            cur_graph = graph;
        }
        const int32_t i = g.e_lo[e], j = g.e_hi[e];
        const int64_t di = g.rp[i + 1] - g.rp[i], dj = g.rp[j + 1] - g.rp[j];
        const int64_t cap = di < dj ? di : dj;
        int32_t *tl = cap <= kTCapSmemHeavy ? tl_smem : tscratch + (int64_t)blockIdx.x * tscratch_stride;
        clear_ws(ws, blockDim.x, threadIdx.x);
        __syncthreads();
        enumerate_T(g, cv, e, i, j, ws, tl, cap, blockDim.x, threadIdx.x, bbar);
        count_K(g, ws, tl, blockDim.x, threadIdx.x, bbar);
        uint32_t *row = per_edge_out ? per_edge_out + (e - row_base) * S : nullptr;
        edge_epilogue(g, cv, e, i, j, ws, row, hist, blockDim.x, threadIdx.x, bbar);
    }
    __syncthreads();
    if (cur_graph >= 0) flush_hist(hist, G, gacc, cur_graph, blockDim.x, threadIdx.x);
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

static std::vector<Tile> make_tiles(const Graph &G, int64_t e_begin, int64_t e_end) {
    std::vector<Tile> tiles;
    for (int gi = 0; gi < G.ngraphs; ++gi) {
        int64_t b = std::max(e_begin, G.h_edge_off[gi]), e = std::min(e_end, G.h_edge_off[gi + 1]);
        for (int64_t x = b; x < e; x += kTile) tiles.push_back(Tile{x, std::min(e, x + kTile), gi, 0});
    }
    return tiles;
}

// Splits the graphs into consecutive chunks whose adjacency slots fit the
// 4-cycle array budget (a single graph larger than the budget is a chunk of
// its own), and sizes the array for the largest chunk.
static void plan_chunks(Graph &G) {
    G.chunks.clear();
    const int64_t per_slot = (int64_t)G.L * G.L * (int64_t)sizeof(uint32_t);
    const int64_t max_slots = std::max<int64_t>(((int64_t)G.opt.cycle_budget_mb << 20) / per_slot, 1);
    // tile index ranges follow graph boundaries (make_tiles emits graph after graph)
    std::vector<int64_t> tile_off(G.ngraphs + 1, 0);
    for (int gi = 0; gi < G.ngraphs; ++gi)
        tile_off[gi + 1] = tile_off[gi] + (G.h_edge_off[gi + 1] - G.h_edge_off[gi] + kTile - 1) / kTile;
    int g0 = 0;
    int64_t widest = 0;
    while (g0 < G.ngraphs) {
        int g1 = g0 + 1;
        while (g1 < G.ngraphs && G.h_slot_off[g1 + 1] - G.h_slot_off[g0] <= max_slots) ++g1;
        Graph::Chunk c;
        c.g0 = g0; c.g1 = g1;
        c.n0 = G.h_node_off[g0]; c.n1 = G.h_node_off[g1];
        c.s0 = G.h_slot_off[g0]; c.s1 = G.h_slot_off[g1];
        c.e0 = G.h_edge_off[g0]; c.e1 = G.h_edge_off[g1];
        c.t0 = tile_off[g0]; c.t1 = tile_off[g1];
        widest = std::max(widest, c.s1 - c.s0);
        G.chunks.push_back(c);
        g0 = g1;
    }
    G.a_stride = std::max<int64_t>(widest, 1);
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
        if (G.n_anchors_heavy > 0 && G.n_tables == 0) {
            const int64_t stride = std::max<int64_t>(G.max_graph_nodes, 1) * L;
            const int64_t per = stride * (int64_t)sizeof(uint32_t);
            int64_t budget = (int64_t)G.opt.anchor_table_budget_mb << 20;
            int64_t nt = std::min<int64_t>({(int64_t)2 * sm_count(), G.n_anchors_heavy, std::max<int64_t>(budget / per, 1)});
            G.tables.alloc((size_t)(nt * per));
            TG_CK(cudaMemsetAsync(G.tables.p, 0, (size_t)(nt * per), s));
            G.table_stride = stride;
            G.n_tables = (int32_t)nt;
        }
    }
}

static size_t hist_bytes(int L, int k) { return (size_t)((global_slots(L, k) + 1) & ~1) * sizeof(unsigned long long); }
static size_t light_smem(int L) {
    return hist_bytes(L, 4) + (kEdgeThreads / 32) * (sizeof(EdgeWs) + kTCapWarp * sizeof(int32_t));
}
static size_t heavy_smem(int L) { return hist_bytes(L, 4) + sizeof(EdgeWs) + kTCapSmemHeavy * sizeof(int32_t); }

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

// Allocations and kernel attributes of the per-edge stage (done before any
// capture).
void prepare_edges(Graph &G, int k, cudaStream_t s) {
    TG_CK(cudaFuncSetAttribute(k_edge3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hist_bytes(G.L, 3)));
    TG_CK(cudaFuncSetAttribute(k_edge4_light, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)light_smem(G.L)));
    TG_CK(cudaFuncSetAttribute(k_edge4_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)heavy_smem(G.L)));
    if (k == 4 && G.n_edges_heavy > 0 && !G.tscratch.p) {
        const int64_t nblk = std::min<int64_t>(G.n_edges_heavy, (int64_t)sm_count() * 2);
        const int64_t stride = std::max<int64_t>(G.max_degree, 1);
        G.tscratch.alloc(sizeof(int32_t) * (size_t)(stride * nblk));
        G.tscratch_stride = stride;
        G.tscratch_blocks = (int32_t)nblk;
    }
    DBuf unused;
    int64_t nt = 0;
    tiles_for(G, 0, G.m, nt, unused, s);
    if (k == 4 && G.n_anchors_light > 0) {
        int cap = 1;
        while (cap < 2 * G.opt.light_anchor_max_wedges) cap <<= 1;
        const size_t smem = (size_t)kLightAnchorWarps * cap * (1 + G.L) * sizeof(int32_t);
        TG_CK(cudaFuncSetAttribute(k_wedge_light, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
        k_tri<<<grid_for(G.m, 8, sms * 16), 256, 0, s>>>(gv, cv);
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

// degree-priority wedges of the anchors of one chunk into A
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
    if (G.n_anchors_heavy > 0) {
        KernelTimer kt(G, s, "k_wedge_heavy");
        k_wedge_heavy<<<G.n_tables, kAnchorThreads, 0, s>>>(gv, cv, G.anchors_heavy.as<int32_t>(), G.n_anchors_heavy,
                                                             c.n0, c.n1);
        ++launches;
    }
    TG_CK(cudaGetLastError());
    return launches;
}

// per-edge stage of edges [e_begin, e_end) given as tiles (inside one chunk for k = 4)
static int64_t launch_edge_tiles(Graph &G, int k, const Tile *tiles, int64_t n_tiles, int64_t e_begin, int64_t e_end,
                                 int64_t row_base, uint32_t *per_edge_out, unsigned long long *gacc, cudaStream_t s) {
    if (n_tiles <= 0) return 0;
    const GraphView gv = G.view();
    const CountView cv = G.cview();
    const int sms = sm_count();
    int64_t launches = 0;
    if (k == 3) {
        KernelTimer kt(G, s, "k_edge3");
        k_edge3<<<grid_for(n_tiles, 1, sms * 8), 256, hist_bytes(G.L, 3), s>>>(gv, cv, tiles, n_tiles, row_base,
                                                                                per_edge_out, gacc);
        ++launches;
    } else {
        {
            KernelTimer kt(G, s, "k_edge4_light");
            k_edge4_light<<<grid_for(n_tiles, 1, sms * G.opt.ctas_per_sm), kEdgeThreads, light_smem(G.L), s>>>(
                gv, cv, tiles, n_tiles, G.opt.light_edge_max_degree, row_base, per_edge_out, gacc);
            ++launches;
        }
        if (G.n_edges_heavy > 0) {
            KernelTimer kt(G, s, "k_edge4_heavy");
            k_edge4_heavy<<<G.tscratch_blocks, kHeavyThreads, heavy_smem(G.L), s>>>(
                gv, cv, G.edges_heavy.as<int32_t>(), G.n_edges_heavy, e_begin, e_end, row_base, per_edge_out, gacc,
                G.tscratch.as<int32_t>(), G.tscratch_stride);
            ++launches;
        }
    }
    TG_CK(cudaGetLastError());
    return launches;
}

int64_t run_count(Graph &G, int k, int64_t e_begin, int64_t e_end, uint32_t *per_edge_out, unsigned long long *gacc,
                  bool full, cudaStream_t s) {
    int64_t launches = 0;
    if (full || G.prepared_k < 3) {
        launches += launch_triangles(G, s);
        G.prepared_k = 3;
    }
    DBuf tmp;
    int64_t n_tiles = 0;
    const Tile *tiles = tiles_for(G, e_begin, e_end, n_tiles, tmp, s);
    if (k == 3) {
        launches += launch_edge_tiles(G, 3, tiles, n_tiles, e_begin, e_end, e_begin, per_edge_out, gacc, s);
    } else {
        const bool whole = e_begin == 0 && e_end == G.m;
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
                // tiles of an arbitrary range: the kernel skips none; pick this chunk's part
                int64_t a = 0, z = n_tiles;
                std::vector<Tile> host = make_tiles(G, e_begin, e_end);
                while (a < z && host[a].end <= b) ++a;
                int64_t y = a;
                while (y < z && host[y].begin < e) ++y;
                ct = tiles + a;
                nct = y - a;
            }
            launches += launch_edge_tiles(G, 4, ct, nct, b, e, e_begin, per_edge_out, gacc, s);
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

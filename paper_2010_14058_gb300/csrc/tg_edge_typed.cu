// tg_edge_typed.cu -- typed 3-node graphlets of a graph whose edges carry
// types too (Def. 1's edge types xi; Defs. 4-5: the class of a typed
// graphlet is its shape with the multisets of its node types and of its
// edge types).
//
// The handle is the ordinary tg_build layout (rows by (type, id), per-type
// segments) plus one edge type per adjacency slot and, per node x, node type
// t and edge type q, the number d_x^{t,q} of x's type-t neighbours joined to
// x by an edge of type q.  Per edge {i, j}, one warp intersects the typed
// segments of i and j (binary search or merge, isect); each triangle node w
// of type t adds 1 to the warp's cell (t, type of {i,w}, type of {j,w}).
// The sets S_i, S_j follow by Cor. 1-2, split by edge type:
//   |S_i^{t,x}| = d_i^{t,x} - |{w in T^t : xi_iw = x}| - [phi_j = t, xi_ij = x]
// and likewise for S_j.  A 3-path's slot is (t, x) whichever endpoint is its
// centre (its class ({phi_i, phi_j, t}, {xi_ij, x}) is the same), a
// triangle's slot (t, {xi_iw, xi_jw}).  Per-edge layout and class ranks:
// include/tg.h.
#include <algorithm>

#include "tg_host.hpp"

namespace tg {

namespace {

constexpr int kMaxX = TG_MAX_EDGE_TYPES;

// multisets of size r from n symbols, C(n + r - 1, r)
__host__ __device__ inline int64_t mchoose(int n, int r) {
    int64_t c = 1;
    for (int k = 1; k <= r; ++k) c = c * (n + k - 1) / k;
    return c;
}

// rank of the non-decreasing K-tuple s over [0, A) among all of them in
// lexicographic order: for each position, the tuples that agree before it
// and hold a smaller value there
__host__ __device__ inline int64_t ms_rank(int A, int K, const int *s) {
    int64_t r = 0;
    int prev = 0;
    for (int k = 0; k < K; ++k) {
        for (int v = prev; v < s[k]; ++v) r += mchoose(A - v, K - k - 1);
        prev = s[k];
    }
    return r;
}

__host__ __device__ inline void sort2(int *a) {
    if (a[1] < a[0]) { const int x = a[0]; a[0] = a[1]; a[1] = x; }
}
__host__ __device__ inline void sort3v(int *a) {
    if (a[1] < a[0]) { const int x = a[0]; a[0] = a[1]; a[1] = x; }
    if (a[2] < a[1]) { const int x = a[1]; a[1] = a[2]; a[2] = x; }
    if (a[1] < a[0]) { const int x = a[0]; a[0] = a[1]; a[1] = x; }
}

// ---------------------------------------------------------------- build
__global__ void k_et_new_of(int64_t n, const int32_t *__restrict__ old_of, int32_t *new_of) {
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x < n) new_of[old_of[x]] = (int32_t)x;
}

// slot of internal node y in the typed segment of row x, or -1
__device__ __forceinline__ int64_t et_slot(const GraphView &g, int32_t x, int32_t y) {
    const int64_t b = seg_begin(g, x, g.ty[y]), e = seg_end(g, x, g.ty[y]);
    const int64_t r = lower_bound_i32(g.adj, b, e, y);
    return (r < e && g.adj[r] == y) ? r : -1;
}

// the caller's entry k (row found by binary search over its row pointers)
// gives its edge type to the slot of that entry
__global__ void k_et_fill(GraphView g, int64_t nnz, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                          const uint8_t *__restrict__ xi, int X, const int32_t *__restrict__ new_of, uint8_t *etype,
                          uint32_t *status) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    int64_t lo = 0, hi = g.n;                               // rp[lo] <= k < rp[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (rp[mid] <= k) lo = mid; else hi = mid;
    }
    const uint8_t t = xi[k];
    if (t >= X) {
        set_status(status, ST_INVALID_GRAPH);
        return;
    }
    const int64_t s = et_slot(g, new_of[lo], new_of[col[k]]);
    if (s < 0) {
        set_status(status, ST_INTERNAL);
        return;
    }
    etype[s] = t;
}

// both slots of every edge hold the same type
__global__ void k_et_check(GraphView g, const uint8_t *__restrict__ etype, uint32_t *status) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= g.m) return;
    const uint8_t a = etype[g.e_slot_lo[e]], b = etype[g.e_slot_hi[e]];
    if (a == 0xff || a != b) set_status(status, ST_INVALID_GRAPH);
}

// d_x^{t,q}: warp per node, one warp sum per (type, edge type)
__global__ void __launch_bounds__(256) k_et_degree(GraphView g, const uint8_t *__restrict__ etype, int X,
                                                   int32_t *etdeg) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; x < g.n; x += nw) {
        for (int t = 0; t < g.L; ++t) {
            unsigned c[kMaxX];
#pragma unroll
            for (int q = 0; q < kMaxX; ++q) c[q] = 0;
            for (int64_t s = seg_begin(g, x, t) + lane; s < seg_end(g, x, t); s += 32) {
                const int q = etype[s];
#pragma unroll
                for (int r = 0; r < kMaxX; ++r) c[r] += q == r ? 1u : 0u;
            }
#pragma unroll
            for (int q = 0; q < kMaxX; ++q) {
                if (q >= X) break;
                const unsigned v = __reduce_add_sync(0xffffffffu, c[q]);
                if (lane == 0) etdeg[(x * g.L + t) * X + q] = (int32_t)v;
            }
        }
    }
}

// ---------------------------------------------------------------- count
// Warp per edge {i, j}: the triangle cells in the warp's shared-memory
// histogram, then per lane the path and triangle slots, the row, and the
// per-CTA class histogram (block 0 edges, block 1 3-paths, block 2
// triangles).
template <bool kMerge>
__global__ void __launch_bounds__(256) k_edge_typed3(GraphView g, const uint8_t *__restrict__ etype,
                                                     const int32_t *__restrict__ etdeg, int X, int G,
                                                     uint32_t *per_edge_out, unsigned long long *gacc,
                                                     uint32_t *status) {
    extern __shared__ unsigned long long ehist[];
    __shared__ uint32_t wh_all[8][kMaxL * kMaxX * kMaxX];
    const int L = g.L;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *wh = wh_all[wid];
    const int XX = X * X, P = X * (X + 1) / 2;
    const int64_t S = (int64_t)L * X + (int64_t)L * P;
    const int64_t off1 = mchoose(L, 2) * X, off2 = off1 + mchoose(L, 3) * mchoose(X, 2);
    const int64_t w2 = mchoose(X, 2), w3 = mchoose(X, 3);
    for (int s = threadIdx.x; s < G; s += blockDim.x) ehist[s] = 0;
    __syncthreads();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < g.m; e += nw) {
        const int32_t i = g.e_lo[e], j = g.e_hi[e];
        const int pi = g.ty[i], pj = g.ty[j];
        const int xij = etype[g.e_slot_lo[e]];
        for (int k = lane; k < L * XX; k += 32) wh[k] = 0;
        __syncwarp();
        for (int t = 0; t < L; ++t) {
            const int64_t bi = seg_begin(g, i, t), ei = seg_end(g, i, t);
            const int64_t bj = seg_begin(g, j, t), ej = seg_end(g, j, t);
            if (ei == bi || ej == bj) continue;                          // warp-uniform
            const bool i_short = ei - bi <= ej - bj;
            const int64_t sb = i_short ? bi : bj, se = i_short ? ei : ej;
            const int64_t lb = i_short ? bj : bi, le = i_short ? ej : ei;
            isect<kMerge>(g.adj, g.isect_modes, sb, se, lb, le, lane, [&](bool found, int64_t s, int64_t r, int32_t) {
                if (found) {
                    const int xa = etype[i_short ? s : r], xb = etype[i_short ? r : s];   // edges {i,w}, {j,w}
                    atomicAdd(&wh[(t * X + xa) * X + xb], 1u);
                }
            });
        }
        __syncwarp();
        uint32_t *row = per_edge_out ? per_edge_out + e * S : nullptr;
        for (int p = lane; p < L * X; p += 32) {                        // 3-paths (t, x)
            const int t = p / X, x = p - t * X;
            int64_t ti = 0, tj = 0;
            for (int y = 0; y < X; ++y) {
                ti += wh[(t * X + x) * X + y];
                tj += wh[(t * X + y) * X + x];
            }
            const int64_t a = etdeg[((int64_t)i * L + t) * X + x] - ti - ((pj == t && xij == x) ? 1 : 0);
            const int64_t b = etdeg[((int64_t)j * L + t) * X + x] - tj - ((pi == t && xij == x) ? 1 : 0);
            if (a < 0 || b < 0) set_status(status, ST_INTERNAL);
            const int64_t v = (a < 0 ? 0 : a) + (b < 0 ? 0 : b);
            if (row) row[p] = (uint32_t)v;
            if (v) {
                int n3[3] = {pi, pj, t}, e2[2] = {xij, x};
                sort3v(n3);
                sort2(e2);
                atomicAdd(&ehist[off1 + ms_rank(L, 3, n3) * w2 + ms_rank(X, 2, e2)], (unsigned long long)v);
            }
        }
        for (int q = lane; q < L * P; q += 32) {                        // triangles (t, {x, y})
            const int t = q / P;
            int r = q - t * P, x = 0;
            while (r >= X - x) { r -= X - x; ++x; }
            const int y = x + r;
            const uint32_t v = wh[(t * X + x) * X + y] + (x != y ? wh[(t * X + y) * X + x] : 0u);
            if (row) row[(int64_t)L * X + q] = v;
            if (v) {
                int n3[3] = {pi, pj, t}, e3[3] = {xij, x, y};
                sort3v(n3);
                sort3v(e3);
                atomicAdd(&ehist[off2 + ms_rank(L, 3, n3) * w3 + ms_rank(X, 3, e3)], (unsigned long long)v);
            }
        }
        if (lane == 0) {
            int n2[2] = {pi, pj};
            sort2(n2);
            atomicAdd(&ehist[ms_rank(L, 2, n2) * X + xij], 1ull);
        }
        __syncwarp();                                                   // the cells are cleared next
    }
    __syncthreads();
    for (int s = threadIdx.x; s < G; s += blockDim.x)
        if (ehist[s]) atomicAdd(&gacc[s], ehist[s]);
}

// totals (Sec. 6): each 3-path was seen from its 2 edges, each triangle
// from its 3
__global__ void k_et_finalize(int G, int64_t off1, int64_t off2, const unsigned long long *__restrict__ gacc,
                              int64_t *global_out, uint32_t *status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= G) return;
    const unsigned long long d = s < off1 ? 1ull : (s < off2 ? 2ull : 3ull);
    if (gacc[s] % d) set_status(status, ST_INTERNAL);
    global_out[s] = (int64_t)(gacc[s] / d);
}

}  // namespace

int64_t edge_typed_global_slots(int L, int X) {
    return mchoose(L, 2) * X + mchoose(L, 3) * mchoose(X, 2) + mchoose(L, 3) * mchoose(X, 3);
}

// Edge types of the slots (from the caller's CSR positions, device arrays)
// and the per-node counts by (node type, edge type); throws
// TG_ERR_INVALID_GRAPH for a type out of range or different on the two
// entries of an edge.
void prepare_edge_typed(Graph &G, int X, const int64_t *row_ptr, const int32_t *col, const uint8_t *edge_types,
                        cudaStream_t s) {
    const GraphView gv = G.view();
    G.etype.alloc(std::max<int64_t>(G.nnz, 1));
    G.etdeg.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(G.n * G.L * X, 1));
    TG_CK(cudaMemsetAsync(G.etype.p, 0xff, std::max<int64_t>(G.nnz, 1), s));
    TG_CK(cudaMemsetAsync(G.status.p, 0, sizeof(uint32_t), s));
    TBuf new_of(sizeof(int32_t) * std::max<int64_t>(G.n, 1), s);
    if (G.n > 0)
        k_et_new_of<<<(unsigned)((G.n + 255) / 256), 256, 0, s>>>(G.n, G.old_of.as<int32_t>(), new_of.as<int32_t>());
    if (G.nnz > 0)
        k_et_fill<<<(unsigned)((G.nnz + 255) / 256), 256, 0, s>>>(gv, G.nnz, row_ptr, col, edge_types, X,
                                                                   new_of.as<int32_t>(), G.etype.as<uint8_t>(),
                                                                   G.status.as<uint32_t>());
    if (G.m > 0)
        k_et_check<<<(unsigned)((G.m + 255) / 256), 256, 0, s>>>(gv, G.etype.as<uint8_t>(), G.status.as<uint32_t>());
    TG_CK(cudaGetLastError());
    uint32_t st = 0;
    TG_CK(cudaMemcpyAsync(&st, G.status.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    if (st & ST_INVALID_GRAPH) throw Error{TG_ERR_INVALID_GRAPH, "edge types out of range or unequal on an edge's entries"};
    if (st) throw Error{TG_ERR_INTERNAL, "edge type slots"};
    if (G.n > 0)
        k_et_degree<<<(unsigned)std::min<int64_t>((G.n + 7) / 8, (int64_t)sm_count() * 16), 256, 0, s>>>(
            gv, G.etype.as<uint8_t>(), X, G.etdeg.as<int32_t>());
    TG_CK(cudaGetLastError());
    G.et_X = X;
    G.et_global = edge_typed_global_slots(G.L, X);
    G.etgacc.alloc(sizeof(unsigned long long) * (size_t)G.et_global);
    G.edge_typed = true;
}

int64_t run_edge_typed3(Graph &G, uint32_t *per_edge_out, int64_t *global_out, cudaStream_t s) {
    const int Gs = (int)G.et_global, X = G.et_X, L = G.L;
    TG_CK(cudaMemsetAsync(G.etgacc.p, 0, sizeof(unsigned long long) * (size_t)Gs, s));
    const size_t smem = sizeof(unsigned long long) * (size_t)Gs;
    const bool merge = isect_any_merge(G.opt.isect_modes);
    const void *fn = merge ? (const void *)k_edge_typed3<true> : (const void *)k_edge_typed3<false>;
    raise_smem_limit(fn, smem);
    int64_t launches = 0;
    if (G.m > 0) {
        KernelTimer kt(G, s, "k_edge_typed3");
        const unsigned grid = (unsigned)std::min<int64_t>((G.m + 7) / 8, (int64_t)sm_count() * 16);
        if (merge)
            k_edge_typed3<true><<<grid, 256, smem, s>>>(G.view(), G.etype.as<uint8_t>(), G.etdeg.as<int32_t>(), X, Gs,
                                                         per_edge_out, G.etgacc.as<unsigned long long>(),
                                                         G.status.as<uint32_t>());
        else
            k_edge_typed3<false><<<grid, 256, smem, s>>>(G.view(), G.etype.as<uint8_t>(), G.etdeg.as<int32_t>(), X, Gs,
                                                          per_edge_out, G.etgacc.as<unsigned long long>(),
                                                          G.status.as<uint32_t>());
        ++launches;
    }
    if (global_out) {
        const int64_t off1 = mchoose(L, 2) * X, off2 = off1 + mchoose(L, 3) * mchoose(X, 2);
        k_et_finalize<<<(unsigned)((Gs + 255) / 256), 256, 0, s>>>(Gs, off1, off2, G.etgacc.as<unsigned long long>(),
                                                                  global_out, G.status.as<uint32_t>());
        ++launches;
    }
    TG_CK(cudaGetLastError());
    return launches;
}

}  // namespace tg

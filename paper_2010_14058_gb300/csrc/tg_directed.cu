// tg_directed.cu -- directed typed 3-node graphlets (Sec. 4.8).
//
// Sec. 4.8 splits every typed neighbourhood Gamma_i^t into the typed
// out-neighbours Gamma_i^{t,+} and in-neighbours Gamma_i^{t,-}, and the sets
// T_ij^t, S_i^t, S_j^t of Alg. 1 with it.  On the GPU an oriented graph is
// held as its underlying undirected graph (the ordinary tg_build layout:
// rows by (type, id), per-type segments) plus one sign per adjacency slot
// (+1 when the row's node is the arc's tail) and the typed out-degrees of
// every node.  Per edge {i, j}, one warp intersects the typed segments of i
// and j (binary search or merge, isect); each triangle node w falls into
// T^t(sign at i, sign at j), counted with ballots; the S sets follow from the typed out- and in-degrees by
// Cor. 1-2: |S_i^{t,+}| = d_i^{t,+} - |T^t(+,.)| - [phi_j = t, i -> j] and
// so on.  Per-edge layout and class ranks: include/tg.h.
#include <algorithm>
#include <mutex>
#include <vector>

#include <cub/device/device_scan.cuh>

#include "tg_host.hpp"

namespace tg {

namespace {

// ---------------------------------------------------------------- classes
// configuration code of nodes 0, 1, 2: (t0, t1, t2, a01, a02, a12) in mixed
// radix (L, L, L, 3, 3, 3); a_xy = 0 no arc, 1 x -> y, 2 y -> x
int64_t conf_code(int L, const int *t, const int *a) {
    return ((((int64_t)(t[0] * L + t[1]) * L + t[2]) * 3 + a[0]) * 3 + a[1]) * 3 + a[2];
}

// arc state of the ordered pair (x, y): 0 none, 1 x -> y, 2 y -> x
int pair_state(const int *a, int x, int y) {
    const int lo = std::min(x, y), hi = std::max(x, y);
    const int st = a[lo == 0 ? hi - 1 : 2];                   // pairs (0,1) (0,2) (1,2)
    return (st == 0 || x == lo) ? st : 3 - st;
}

// smallest code over the renumberings (new node k = old node p[k])
int64_t smallest_code(int L, const int *t, const int *a) {
    int p[3] = {0, 1, 2};
    int64_t best = INT64_MAX;
    do {
        const int tt[3] = {t[p[0]], t[p[1]], t[p[2]]};
        const int aa[3] = {pair_state(a, p[0], p[1]), pair_state(a, p[0], p[2]), pair_state(a, p[1], p[2])};
        best = std::min(best, conf_code(L, tt, aa));
    } while (std::next_permutation(p, p + 3));
    return best;
}

struct DirectedTables {
    std::vector<int64_t> codes;       // class representatives, ascending
    std::vector<int32_t> slot_class;  // [(phi_i*L + phi_j)*2 + o][8L] class of a per-edge slot
    std::vector<uint8_t> arcs;        // arcs of each class (2: path, 3: triangle)
};

const DirectedTables &directed_tables(int L) {
    static std::mutex mu;
    static DirectedTables tables[TG_MAX_TYPES + 1];
    std::lock_guard<std::mutex> lock(mu);
    DirectedTables &D = tables[L];
    if (!D.codes.empty()) return D;
    for (int t0 = 0; t0 < L; ++t0)
        for (int t1 = 0; t1 < L; ++t1)
            for (int t2 = 0; t2 < L; ++t2)
                for (int a0 = 0; a0 < 3; ++a0)
                    for (int a1 = 0; a1 < 3; ++a1)
                        for (int a2 = 0; a2 < 3; ++a2) {
                            const int t[3] = {t0, t1, t2}, a[3] = {a0, a1, a2};
                            const int na = (a0 != 0) + (a1 != 0) + (a2 != 0);
                            if (na >= 2 && smallest_code(L, t, a) == conf_code(L, t, a)) {
                                D.codes.push_back(conf_code(L, t, a));
                                D.arcs.push_back((uint8_t)na);
                            }
                        }
    D.slot_class.assign((size_t)L * L * 2 * 8 * L, -1);
    for (int pi = 0; pi < L; ++pi)
        for (int pj = 0; pj < L; ++pj)
            for (int o = 0; o < 2; ++o)
                for (int b = 0; b < 8; ++b)
                    for (int t = 0; t < L; ++t) {
                        // node 0 = i, 1 = j, 2 = w; o = 0: i -> j
                        const int si = b < 2 ? (b == 0 ? 1 : -1) : (b < 4 ? 0 : (b < 6 ? 1 : -1));
                        const int sj = b < 2 ? 0 : (b < 4 ? (b == 2 ? 1 : -1) : ((b & 1) ? -1 : 1));
                        const int tt[3] = {pi, pj, t};
                        const int a[3] = {o == 0 ? 1 : 2, si == 0 ? 0 : (si > 0 ? 1 : 2), sj == 0 ? 0 : (sj > 0 ? 1 : 2)};
                        const int64_t c = smallest_code(L, tt, a);
                        const auto it = std::lower_bound(D.codes.begin(), D.codes.end(), c);
                        D.slot_class[(((size_t)pi * L + pj) * 2 + o) * 8 * L + b * L + t] =
                            (int32_t)(it - D.codes.begin());
                    }
    return D;
}

// ---------------------------------------------------------------- build
// arc k = u -> v: u from the row pointers, degrees of the symmetric rows
__global__ void k_arc_ends(int64_t n, int64_t na, const int64_t *__restrict__ orp, const int32_t *__restrict__ ocol,
                           int32_t *src, unsigned long long *deg, uint32_t *status) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= na) return;
    int64_t lo = 0, hi = n;                                 // orp[lo] <= k < orp[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (orp[mid] <= k) lo = mid; else hi = mid;
    }
    const int32_t v = ocol[k];
    src[k] = (int32_t)lo;
    if (v < 0 || v >= n) {
        set_status(status, ST_INVALID_GRAPH);
        return;
    }
    atomicAdd(&deg[lo], 1ull);
    atomicAdd(&deg[v], 1ull);
}

__global__ void k_arc_fill(int64_t na, const int32_t *__restrict__ src, const int32_t *__restrict__ ocol,
                           const int64_t *__restrict__ srp, unsigned long long *fill, int32_t *scol) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= na) return;
    const int32_t u = src[k], v = ocol[k];
    scol[srp[u] + (int64_t)atomicAdd(&fill[u], 1ull)] = v;
    scol[srp[v] + (int64_t)atomicAdd(&fill[v], 1ull)] = u;
}

__global__ void k_new_of(int64_t n, const int32_t *__restrict__ old_of, int32_t *new_of) {
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x < n) new_of[old_of[x]] = (int32_t)x;
}

// slot of internal node y in the typed segment of row x, or -1
__device__ __forceinline__ int64_t slot_of(const GraphView &g, int32_t x, int32_t y) {
    const int64_t b = seg_begin(g, x, g.ty[y]), e = seg_end(g, x, g.ty[y]);
    const int64_t r = lower_bound_i32(g.adj, b, e, y);
    return (r < e && g.adj[r] == y) ? r : -1;
}

// signs of both slots of every arc
__global__ void k_arc_sign(GraphView g, int64_t na, const int32_t *__restrict__ src, const int32_t *__restrict__ ocol,
                           const int32_t *__restrict__ new_of, int8_t *sign, uint32_t *status) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= na) return;
    const int32_t x = new_of[src[k]], y = new_of[ocol[k]];
    const int64_t s1 = slot_of(g, x, y), s2 = slot_of(g, y, x);
    if (s1 < 0 || s2 < 0) {
        set_status(status, ST_INTERNAL);
        return;
    }
    sign[s1] = 1;
    sign[s2] = -1;
}

// typed out-degrees d_x^{t,+}, warp per node
__global__ void __launch_bounds__(256) k_out_degree(GraphView g, const int8_t *__restrict__ sign, int32_t *outdeg,
                                                    uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; x < g.n; x += nw) {
        for (int t = 0; t < g.L; ++t) {
            unsigned c = 0;
            for (int64_t s = seg_begin(g, x, t) + lane; s < seg_end(g, x, t); s += 32) {
                const int8_t v = sign[s];
                if (v == 0) set_status(status, ST_INTERNAL);            // a slot no arc reached
                c += v > 0 ? 1u : 0u;
            }
            c = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0) outdeg[x * g.L + t] = (int32_t)c;
        }
    }
}

// ---------------------------------------------------------------- count
// Warp per edge {i, j} (i the smaller caller id): T^t by signs at i and j
// with ballots (lane t keeps type t's four counts), then S^t from the
// typed out- and in-degrees, the row, and the per-CTA class histogram.
template <bool kMerge>
__global__ void __launch_bounds__(256) k_directed3(GraphView g, const int8_t *__restrict__ sign,
                                                   const int32_t *__restrict__ outdeg,
                                                   const int32_t *__restrict__ old_of,
                                                   const int32_t *__restrict__ slot_class, int G,
                                                   uint32_t *per_edge_out, unsigned long long *gacc,
                                                   uint32_t *status) {
    extern __shared__ unsigned long long dhist[];
    const int L = g.L, LL = L * L;
    const int lane = threadIdx.x & 31;
    for (int s = threadIdx.x; s < G; s += blockDim.x) dhist[s] = 0;
    __syncthreads();
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < g.m; e += nw) {
        const int32_t a = g.e_lo[e], b = g.e_hi[e];
        const bool swap = old_of[a] > old_of[b];
        const int32_t i = swap ? b : a, j = swap ? a : b;
        const int64_t sij = swap ? g.e_slot_hi[e] : g.e_slot_lo[e];     // slot of j in row i
        const int o = sign[sij] > 0 ? 0 : 1;                             // 0: i -> j
        const int pi = g.ty[i], pj = g.ty[j];
        unsigned c0 = 0, c1 = 0, c2 = 0, c3 = 0;                         // lane t: T^t(++ +- -+ --)
        for (int t = 0; t < L; ++t) {
            int64_t bi = seg_begin(g, i, t), ei = seg_end(g, i, t);
            int64_t bj = seg_begin(g, j, t), ej = seg_end(g, j, t);
            if (ei == bi || ej == bj) continue;                          // warp-uniform
            const bool i_short = ei - bi <= ej - bj;
            const int64_t sb = i_short ? bi : bj, se = i_short ? ei : ej;
            const int64_t lb = i_short ? bj : bi, le = i_short ? ej : ei;
            isect<kMerge>(g.adj, g.isect_modes, sb, se, lb, le, lane, [&](bool found, int64_t s, int64_t r, int32_t) {
                int q = -1;
                if (found) {
                    const int8_t at_i = sign[i_short ? s : r], at_j = sign[i_short ? r : s];
                    q = (at_i > 0 ? 0 : 2) + (at_j > 0 ? 0 : 1);
                }
                const unsigned n0 = __popc(__ballot_sync(0xffffffffu, q == 0));
                const unsigned n1 = __popc(__ballot_sync(0xffffffffu, q == 1));
                const unsigned n2 = __popc(__ballot_sync(0xffffffffu, q == 2));
                const unsigned n3 = __popc(__ballot_sync(0xffffffffu, q == 3));
                if (lane == t) { c0 += n0; c1 += n1; c2 += n2; c3 += n3; }
            });
        }
        if (lane < L) {
            const int t = lane;
            const int64_t di = typed_degree(g, i, t), dj = typed_degree(g, j, t);
            const int64_t oi = outdeg[(int64_t)i * L + t], oj = outdeg[(int64_t)j * L + t];
            const int64_t v[8] = {
                oi - c0 - c1 - ((pj == t && o == 0) ? 1 : 0),                   // S_i^{t,+}
                (di - oi) - c2 - c3 - ((pj == t && o == 1) ? 1 : 0),            // S_i^{t,-}
                oj - c0 - c2 - ((pi == t && o == 1) ? 1 : 0),                   // S_j^{t,+}
                (dj - oj) - c1 - c3 - ((pi == t && o == 0) ? 1 : 0),            // S_j^{t,-}
                c0, c1, c2, c3};
            const int32_t *cls = slot_class + (((int64_t)pi * L + pj) * 2 + o) * 8 * L;
            uint32_t *row = per_edge_out ? per_edge_out + e * 8 * L : nullptr;
            for (int k = 0; k < 8; ++k) {
                if (v[k] < 0) set_status(status, ST_INTERNAL);
                if (row) row[k * L + t] = (uint32_t)(v[k] < 0 ? 0 : v[k]);
                if (v[k] > 0) atomicAdd(&dhist[LL + cls[k * L + t]], (unsigned long long)v[k]);
            }
        }
        if (lane == 0) atomicAdd(&dhist[o == 0 ? pi * L + pj : pj * L + pi], 1ull);   // (tail type, head type)
    }
    __syncthreads();
    for (int s = threadIdx.x; s < G; s += blockDim.x)
        if (dhist[s]) atomicAdd(&gacc[s], dhist[s]);
}

// totals: each 3-node instance was seen from each of its arcs
__global__ void k_directed_finalize(int G, int LL, const unsigned long long *__restrict__ gacc,
                                    const uint8_t *__restrict__ arcs, int64_t *global_out, uint32_t *status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= G) return;
    const unsigned long long d = s < LL ? 1ull : (unsigned long long)arcs[s - LL];
    if (gacc[s] % d) set_status(status, ST_INTERNAL);
    global_out[s] = (int64_t)(gacc[s] / d);
}

}  // namespace

int64_t directed_classes(int L) { return (int64_t)directed_tables(L).codes.size(); }

bool directed_class_code(int L, int64_t rank, int32_t *types3, int32_t *arcs3) {
    const DirectedTables &D = directed_tables(L);
    if (rank < 0 || rank >= (int64_t)D.codes.size()) return false;
    int64_t c = D.codes[(size_t)rank];
    arcs3[2] = (int32_t)(c % 3); c /= 3;
    arcs3[1] = (int32_t)(c % 3); c /= 3;
    arcs3[0] = (int32_t)(c % 3); c /= 3;
    types3[2] = (int32_t)(c % L); c /= L;
    types3[1] = (int32_t)(c % L); c /= L;
    types3[0] = (int32_t)c;
    return true;
}

// The symmetric CSR of an oriented graph's arcs (device arrays owned by the
// caller's TBufs); throws TG_ERR_INVALID_GRAPH for ids out of range.
void symmetrize_arcs(int64_t n, int64_t na, const int64_t *orp, const int32_t *ocol, int64_t *srp, int32_t *scol,
                     int32_t *src, cudaStream_t s) {
    TBuf deg(sizeof(unsigned long long) * (n + 1), s), fill(sizeof(unsigned long long) * std::max<int64_t>(n, 1), s),
        st(sizeof(uint32_t), s);
    TG_CK(cudaMemsetAsync(deg.p, 0, sizeof(unsigned long long) * (n + 1), s));
    TG_CK(cudaMemsetAsync(fill.p, 0, sizeof(unsigned long long) * std::max<int64_t>(n, 1), s));
    TG_CK(cudaMemsetAsync(st.p, 0, sizeof(uint32_t), s));
    if (na > 0)
        k_arc_ends<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(n, na, orp, ocol, src, deg.as<unsigned long long>(),
                                                                 st.as<uint32_t>());
    TG_CK(cudaGetLastError());
    uint32_t bad = 0;
    TG_CK(cudaMemcpyAsync(&bad, st.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    if (bad) throw Error{TG_ERR_INVALID_GRAPH, "arc head out of range"};
    size_t tb = 0;
    const int64_t *din = reinterpret_cast<const int64_t *>(deg.p);
    TG_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, din, srp, n + 1, s));
    TBuf tmp(std::max<size_t>(tb, 16), s);
    TG_CK(cub::DeviceScan::ExclusiveSum(tmp.p, tb, din, srp, n + 1, s));
    if (na > 0)
        k_arc_fill<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(na, src, ocol, srp, fill.as<unsigned long long>(), scol);
    TG_CK(cudaGetLastError());
}

// Signs of the slots and typed out-degrees of a handle built from the
// symmetric CSR of these arcs; the class tables of L on the device.
void prepare_directed(Graph &G, int64_t na, const int32_t *src, const int32_t *ocol, cudaStream_t s) {
    const GraphView gv = G.view();
    G.dsign.alloc(std::max<int64_t>(G.nnz, 1));
    G.doutdeg.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(G.n * G.L, 1));
    TG_CK(cudaMemsetAsync(G.dsign.p, 0, std::max<int64_t>(G.nnz, 1), s));
    TBuf new_of(sizeof(int32_t) * std::max<int64_t>(G.n, 1), s);
    if (G.n > 0)
        k_new_of<<<(unsigned)((G.n + 255) / 256), 256, 0, s>>>(G.n, G.old_of.as<int32_t>(), new_of.as<int32_t>());
    if (na > 0)
        k_arc_sign<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(gv, na, src, ocol, new_of.as<int32_t>(),
                                                                 G.dsign.as<int8_t>(), G.status.as<uint32_t>());
    if (G.n > 0)
        k_out_degree<<<(unsigned)std::min<int64_t>((G.n + 7) / 8, (int64_t)sm_count() * 16), 256, 0, s>>>(
            gv, G.dsign.as<int8_t>(), G.doutdeg.as<int32_t>(), G.status.as<uint32_t>());
    TG_CK(cudaGetLastError());
    const DirectedTables &D = directed_tables(G.L);
    G.dcls.alloc(sizeof(int32_t) * D.slot_class.size());
    G.darcs.alloc(std::max<size_t>(D.arcs.size(), 1));
    TG_CK(cudaMemcpyAsync(G.dcls.p, D.slot_class.data(), sizeof(int32_t) * D.slot_class.size(), cudaMemcpyHostToDevice,
                          s));
    if (!D.arcs.empty())
        TG_CK(cudaMemcpyAsync(G.darcs.p, D.arcs.data(), D.arcs.size(), cudaMemcpyHostToDevice, s));
    G.d_global = G.L * G.L + (int64_t)D.codes.size();
    G.dgacc.alloc(sizeof(unsigned long long) * (size_t)G.d_global);
    G.directed = true;
}

int64_t run_directed3(Graph &G, uint32_t *per_edge_out, int64_t *global_out, cudaStream_t s) {
    const int Gs = (int)G.d_global;
    TG_CK(cudaMemsetAsync(G.dgacc.p, 0, sizeof(unsigned long long) * (size_t)Gs, s));
    const size_t smem = sizeof(unsigned long long) * (size_t)Gs;
    const bool merge = isect_any_merge(G.opt.isect_modes);
    const void *fn = merge ? (const void *)k_directed3<true> : (const void *)k_directed3<false>;
    raise_smem_limit(fn, smem);
    int64_t launches = 0;
    if (G.m > 0) {
        KernelTimer kt(G, s, "k_directed3");
        const unsigned grid = (unsigned)std::min<int64_t>((G.m + 7) / 8, (int64_t)sm_count() * 16);
        if (merge)
            k_directed3<true><<<grid, 256, smem, s>>>(G.view(), G.dsign.as<int8_t>(), G.doutdeg.as<int32_t>(),
                                                       G.old_of.as<int32_t>(), G.dcls.as<int32_t>(), Gs, per_edge_out,
                                                       G.dgacc.as<unsigned long long>(), G.status.as<uint32_t>());
        else
            k_directed3<false><<<grid, 256, smem, s>>>(G.view(), G.dsign.as<int8_t>(), G.doutdeg.as<int32_t>(),
                                                        G.old_of.as<int32_t>(), G.dcls.as<int32_t>(), Gs, per_edge_out,
                                                        G.dgacc.as<unsigned long long>(), G.status.as<uint32_t>());
        ++launches;
    }
    if (global_out) {
        k_directed_finalize<<<(unsigned)((Gs + 255) / 256), 256, 0, s>>>(Gs, G.L * G.L, G.dgacc.as<unsigned long long>(),
                                                                        G.darcs.as<uint8_t>(), global_out,
                                                                        G.status.as<uint32_t>());
        ++launches;
    }
    TG_CK(cudaGetLastError());
    return launches;
}

}  // namespace tg

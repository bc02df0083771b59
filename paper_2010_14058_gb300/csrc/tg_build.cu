// tg_build.cu -- device preprocessing of a typed graph (tg_build).
//
// From a caller CSR it builds, on the GPU:
//   * validation: row pointers, ranges, types < L, no self-loops, no repeated
//     entries, symmetric rows, no edge between two graphs of a batch;
//   * a node order by (graph, degree, id): the internal id of a node is its
//     rank, so comparisons of internal ids compare priorities;
//   * adjacency rows sorted by (type, internal id) with per-type offsets:
//     the typed neighbourhoods Gamma_x^t and typed degrees d_x^t of Def. 6-7;
//   * edge ids in the caller's lexicographic (u < v) order, the two slots of
//     each edge and the edge id of every slot;
//   * per-node typed degree sums delta_x[t][t'] = sum_{w in Gamma_x^t} d_w^t';
//   * work lists: wedge anchors by wedge count, edges by min endpoint degree.
// Sorting and compaction use CUB device primitives.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include "tg_host.hpp"

namespace tg {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t items, int per_block) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > (1ll << 30)) b = 1ll << 30;
    return (int)b;
}

__global__ void k_check_rows(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                             const uint8_t *__restrict__ types, int L, uint32_t *status) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v > n) return;
    int64_t a = rp[v];
    bool bad = a < 0 || a > nnz;
    if (v == 0 && a != 0) bad = true;
    if (v == n && a != nnz) bad = true;
    if (v < n) {
        if (rp[v + 1] < a) bad = true;
        if (types[v] >= L) bad = true;
    }
    if (bad) set_status(status, ST_INVALID_GRAPH);
}

__global__ void k_check_cols(int64_t nnz, int64_t n, const int32_t *__restrict__ col, uint32_t *status) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nnz) return;
    int32_t v = col[s];
    if (v < 0 || v >= n) set_status(status, ST_INVALID_GRAPH);
}

__global__ void k_degree_keys(int64_t n, const int64_t *__restrict__ rp, const int64_t *__restrict__ node_off,
                              int ngraphs, unsigned long long *keys, int32_t *vals) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    int lo = 0, hi = ngraphs;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (node_off[mid] <= v) lo = mid; else hi = mid;
    }
    unsigned long long d = (unsigned long long)(rp[v + 1] - rp[v]);
    keys[v] = ((unsigned long long)lo << 32) | d;
    vals[v] = (int32_t)v;
}

__global__ void k_inverse(int64_t n, const int32_t *__restrict__ old_of, const int64_t *__restrict__ rp,
                          int32_t *new_of, int64_t *ndeg) {
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x > n) return;
    if (x == n) { ndeg[n] = 0; return; }
    int32_t u = old_of[x];
    new_of[u] = (int32_t)x;
    ndeg[x] = rp[u + 1] - rp[u];
}

// warp per caller node u: packed keys (row << 32 | type << 29 | neighbour)
__global__ void k_fill_keys(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const uint8_t *__restrict__ types, const int32_t *__restrict__ new_of,
                            const int64_t *__restrict__ rp_new, const int64_t *__restrict__ node_off, int ngraphs,
                            unsigned long long *keys, uint32_t *status) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & (kWarp - 1);
    if (warp >= n) return;
    int64_t u = warp;
    int32_t x = new_of[u];
    int64_t b = rp[u], e = rp[u + 1], base = rp_new[x];
    int64_t glo = 0, ghi = 0;
    if (ngraphs > 1) {
        int lo = 0, hi = ngraphs;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (node_off[mid] <= u) lo = mid; else hi = mid;
        }
        glo = node_off[lo];
        ghi = node_off[lo + 1];
    }
    for (int64_t k = b + lane; k < e; k += kWarp) {
        int32_t v = col[k];
        if (ngraphs > 1 && (v < glo || v >= ghi)) set_status(status, ST_INVALID_GRAPH);
        uint32_t low = ((uint32_t)types[v] << kTypeShift) | (uint32_t)new_of[v];
        keys[base + (k - b)] = ((unsigned long long)(uint32_t)x << 32) | low;
    }
}

__global__ void k_gather_types(int64_t n, const int32_t *__restrict__ old_of, const uint8_t *__restrict__ ty,
                               uint8_t *out) {
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x < n) out[x] = ty[old_of[x]];
}

// warp per internal row x: adjacency ids, self-loop / repeat checks, type offsets
__global__ void k_rows(int64_t n, int L, const int64_t *__restrict__ rp, const unsigned long long *__restrict__ keys,
                       int32_t *adj, int32_t *toff, int32_t *pivot, int32_t *nplus, uint32_t *status) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & (kWarp - 1);
    if (warp >= n) return;
    int64_t x = warp;
    int64_t b = rp[x], e = rp[x + 1];
    for (int64_t s = b + lane; s < e; s += kWarp) {
        unsigned long long k = keys[s];
        uint32_t low = (uint32_t)k;
        int32_t y = (int32_t)(low & kIdMask);
        adj[s] = y;
        if ((int64_t)(k >> 32) != x || y == x) set_status(status, ST_INVALID_GRAPH);
        if (s > b && keys[s - 1] == k) set_status(status, ST_INVALID_GRAPH);
    }
    // type t < L starts at the first slot whose packed type is >= t; the
    // end sentinel (t = L) is the row length (L << 29 would not fit 32 bits
    // for L = 8)
    if (lane < L) {
        uint32_t key = (uint32_t)lane << kTypeShift;
        int64_t lo = b, hi = e;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((uint32_t)keys[mid] < key) lo = mid + 1; else hi = mid;
        }
        toff[x * (L + 1) + lane] = (int32_t)(lo - b);
    } else if (lane == L) {
        toff[x * (L + 1) + L] = (int32_t)(e - b);
    }
    // pivot: first slot of each type segment whose id exceeds x (the
    // neighbours of higher priority)
    __syncwarp();
    const int32_t sb = lane < L ? toff[x * (L + 1) + lane] : 0;
    const int32_t se = lane < L ? toff[x * (L + 1) + lane + 1] : 0;
    int32_t up = 0;                      // higher-priority neighbours of this type segment
    if (lane < L) {
        int64_t lo = b + sb, hi = b + se;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (adj[mid] < (int32_t)x + 1) lo = mid + 1; else hi = mid;
        }
        pivot[x * L + lane] = (int32_t)(lo - b);
        up = se - (int32_t)(lo - b);
    }
    for (int o = 16; o > 0; o >>= 1) up += __shfl_xor_sync(0xffffffffu, up, o);
    if (lane == 0) nplus[x] = up;
}

// warp per node x: its higher-priority neighbours (the part of each type
// segment past the pivot), packed (type << 29 | id), into one contiguous list
__global__ void k_plus_fill(GraphView g, int32_t *plus_adj) {
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
    const int lane = threadIdx.x & (kWarp - 1);
    if (warp >= g.n) return;
    const int64_t x = warp, r = g.rp[x];
    int64_t out = g.plus_off[x];
    for (int q = 0; q < g.L; ++q) {
        const int64_t b = r + g.pivot[x * g.L + q], e = r + g.toff[x * (g.L + 1) + q + 1];
        for (int64_t k = b + lane; k < e; k += kWarp)
            plus_adj[out + (k - b)] = (int32_t)(((uint32_t)q << kTypeShift) | (uint32_t)g.adj[k]);
        out += e - b;
    }
}

// warp per internal row x: forward slots (caller id of x < caller id of y) become edges
__global__ void k_edge_keys(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ adj,
                            const int32_t *__restrict__ old_of, int64_t m_expected,
                            unsigned long long *ekeys, int64_t *eslots, unsigned long long *counter,
                            uint32_t *status) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & (kWarp - 1);
    if (warp >= n) return;
    int64_t x = warp;
    uint32_t ox = (uint32_t)old_of[x];
    for (int64_t s = rp[x] + lane; s < rp[x + 1]; s += kWarp) {
        uint32_t oy = (uint32_t)old_of[adj[s]];
        if (ox < oy) {
            unsigned long long idx = atomicAdd(counter, 1ull);
            if ((int64_t)idx < m_expected) {
                ekeys[idx] = ((unsigned long long)ox << 32) | oy;
                eslots[idx] = s;
            } else {
                set_status(status, ST_INVALID_GRAPH);
            }
        }
    }
}

// thread per edge id: endpoints, both slots, slot -> edge id
__global__ void k_edges(int64_t m, const unsigned long long *__restrict__ ekeys, const int64_t *__restrict__ eslots,
                        GraphView g, const int32_t *__restrict__ new_of, int32_t *e_lo, int32_t *e_hi,
                        int64_t *e_slot_lo, int64_t *e_slot_hi, int32_t *slot_eid, uint32_t *status) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    unsigned long long k = ekeys[e];
    int32_t x = new_of[(uint32_t)(k >> 32)];
    int32_t y = new_of[(uint32_t)k];
    int64_t s = eslots[e];                      // slot of y in row x
    int tx = g.ty[x];
    int64_t b = seg_begin(g, y, tx), en = seg_end(g, y, tx);
    int64_t r = lower_bound_i32(g.adj, b, en, x);
    if (r >= en || g.adj[r] != x) {             // one-sided entry
        set_status(status, ST_INVALID_GRAPH);
        return;
    }
    slot_eid[s] = (int32_t)e;
    slot_eid[r] = (int32_t)e;
    if (x < y) {
        e_lo[e] = x; e_hi[e] = y; e_slot_lo[e] = s; e_slot_hi[e] = r;
    } else {
        e_lo[e] = y; e_hi[e] = x; e_slot_lo[e] = r; e_slot_hi[e] = s;
    }
}

// warp per row x: delta_x[t][t'] = sum over w in Gamma_x^t of d_w^t'
__global__ void k_delta(GraphView g, int64_t *delta) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & (kWarp - 1);
    if (warp >= g.n) return;
    int64_t x = warp;
    const int L = g.L;
    for (int t = 0; t < L; ++t) {
        int64_t acc[kMaxL];
#pragma unroll
        for (int q = 0; q < kMaxL; ++q) acc[q] = 0;
        for (int64_t s = seg_begin(g, x, t) + lane; s < seg_end(g, x, t); s += kWarp) {
            int32_t w = g.adj[s];
            const int32_t *o = g.toff + (int64_t)w * (L + 1);
#pragma unroll
            for (int q = 0; q < kMaxL; ++q)
                if (q < L) acc[q] += o[q + 1] - o[q];
        }
#pragma unroll
        for (int q = 0; q < kMaxL; ++q) {
            if (q >= L) break;
            int64_t v = acc[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) delta[(x * L + t) * L + q] = v;
        }
    }
}

// warp per anchor x: number of wedges x - v - w with v < x and w < x
__global__ void k_anchor_work(GraphView g, int64_t *work) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
    int lane = threadIdx.x & (kWarp - 1);
    if (warp >= g.n) return;
    int32_t x = (int32_t)warp;
    int64_t total = 0;
    for (int t = 0; t < g.L; ++t) {
        int64_t b = seg_begin(g, x, t), e = seg_end(g, x, t);
        int64_t cut = lower_bound_i32(g.adj, b, e, x);
        for (int64_t s = b + lane; s < cut; s += kWarp) {
            int32_t v = g.adj[s];
            for (int q = 0; q < g.L; ++q) {
                int64_t vb = seg_begin(g, v, q), ve = seg_end(g, v, q);
                total += lower_bound_i32(g.adj, vb, ve, x) - vb;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) total += __shfl_down_sync(0xffffffffu, total, off);
    if (lane == 0) work[x] = total;
}

__global__ void k_classify_anchors(int64_t n, const int64_t *__restrict__ work, int64_t light_max, int64_t hub_min,
                                   uint8_t *is_light, uint8_t *is_heavy, uint8_t *is_hub, int32_t *ids,
                                   unsigned long long *heavy_key) {
    int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= n) return;
    int64_t w = work[x];
    is_light[x] = (w > 0 && w <= light_max) ? 1 : 0;
    is_heavy[x] = (w > light_max && w <= hub_min) ? 1 : 0;
    is_hub[x] = (w > hub_min) ? 1 : 0;
    ids[x] = (int32_t)x;
    heavy_key[x] = (unsigned long long)w;
}

__global__ void k_classify_edges(int64_t m, GraphView g, int64_t light_max_deg, uint8_t *is_light,
                                 uint8_t *is_heavy, int32_t *ids, unsigned long long *cost) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    int32_t a = g.e_lo[e], b = g.e_hi[e];
    int64_t da = g.rp[a + 1] - g.rp[a], db = g.rp[b + 1] - g.rp[b];
    int64_t mn = da < db ? da : db;
    is_light[e] = mn <= light_max_deg ? 1 : 0;
    is_heavy[e] = mn > light_max_deg ? 1 : 0;
    ids[e] = (int32_t)e;
    cost[e] = (unsigned long long)(da + db);
}

template <class F>
void cub_call(F f, cudaStream_t s) {
    size_t bytes = 0;
    TG_CK(f(nullptr, bytes));
    TBuf tmp(bytes, s);
    TG_CK(f(tmp.p, bytes));
}

int bits_for(int64_t v) {
    int b = 1;
    while (b < 63 && (1ll << b) <= v) ++b;
    return b;
}

// Selects the flagged ids into a new device buffer; returns the count.
int64_t select_flagged(const int32_t *ids, const uint8_t *flags, int64_t n, DBuf &out, cudaStream_t s) {
    TBuf sel(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), s);
    TBuf cnt(sizeof(int64_t), s);
    cub_call([&](void *t, size_t &b) {
        return cub::DeviceSelect::Flagged(t, b, ids, flags, sel.as<int32_t>(), cnt.as<int64_t>(), n, s);
    }, s);
    int64_t c = 0;
    TG_CK(cudaMemcpyAsync(&c, cnt.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    out.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(c, 1));
    TG_CK(cudaMemcpyAsync(out.p, sel.p, sizeof(int32_t) * (size_t)c, cudaMemcpyDeviceToDevice, s));
    return c;
}

__global__ void k_widen(int64_t n, const int32_t *__restrict__ in, int64_t *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

__global__ void k_count_above(int64_t c, const int32_t *__restrict__ ids, const unsigned long long *__restrict__ key,
                              unsigned long long limit, unsigned long long *count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < c && key[ids[i]] > limit) atomicAdd(count, 1ull);
}

// Sorts `ids` (count c) by descending key (keys indexed by id).
__global__ void k_gather_keys(int64_t c, const int32_t *__restrict__ ids, const unsigned long long *__restrict__ key,
                              unsigned long long *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < c) out[i] = key[ids[i]];
}

void sort_desc_by_key(DBuf &ids, int64_t c, const unsigned long long *key, cudaStream_t s, int64_t &launches) {
    if (c <= 1) return;
    ++launches;
    TBuf k_in(sizeof(unsigned long long) * c, s), k_out(sizeof(unsigned long long) * c, s);
    TBuf v_out(sizeof(int32_t) * c, s);
    k_gather_keys<<<blocks_for(c, kThreads), kThreads, 0, s>>>(c, ids.as<int32_t>(), key, k_in.as<unsigned long long>());
    TG_CK(cudaGetLastError());
    cub_call([&](void *t, size_t &b) {
        return cub::DeviceRadixSort::SortPairsDescending(t, b, k_in.as<unsigned long long>(),
                                                         k_out.as<unsigned long long>(), ids.as<int32_t>(),
                                                         v_out.as<int32_t>(), c, 0, 64, s);
    }, s);
    TG_CK(cudaMemcpyAsync(ids.p, v_out.p, sizeof(int32_t) * c, cudaMemcpyDeviceToDevice, s));
}

uint32_t read_status(const DBuf &st, cudaStream_t s) {
    uint32_t v = 0;
    TG_CK(cudaMemcpyAsync(&v, st.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    return v;
}

}  // namespace

cudaMemPool_t device_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    TG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error{TG_ERR_INVALID_ARG, "device index"};
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        TG_CK(cudaMemPoolCreate(&pools[dev], &props));
        uint64_t keep = UINT64_MAX;
        TG_CK(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    return pools[dev];
}

int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0;
        TG_CK(cudaGetDevice(&dev));
        TG_CK(cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev));
    }
    return cached;
}

void build_graph(Graph &G, int32_t ngraphs, const int64_t *node_off_host, int64_t n, int64_t nnz,
                 const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int32_t L,
                 const tg_options &opt, cudaStream_t s) {
    G.stream = s;
    G.last_launches = 0;
    G.ngraphs = ngraphs;
    G.L = L;
    G.n = n;
    G.nnz = nnz;
    G.m = nnz / 2;
    G.opt = opt;
    TG_CK(cudaGetDevice(&G.device));
    G.h_node_off.assign(node_off_host, node_off_host + ngraphs + 1);
    G.max_graph_nodes = 0;
    for (int g = 0; g < ngraphs; ++g)
        G.max_graph_nodes = std::max(G.max_graph_nodes, G.h_node_off[g + 1] - G.h_node_off[g]);

    G.status.alloc(sizeof(uint32_t));
    TG_CK(cudaMemsetAsync(G.status.p, 0, sizeof(uint32_t), s));
    uint32_t *status = G.status.as<uint32_t>();

    // inputs on the device (copied in when the caller passed host memory)
    TBuf rp_in(sizeof(int64_t) * (n + 1), s), col_in(sizeof(int32_t) * std::max<int64_t>(nnz, 1), s),
        ty_in(std::max<int64_t>(n, 1), s);
    TG_CK(cudaMemcpyAsync(rp_in.p, row_ptr, sizeof(int64_t) * (n + 1),
                          is_device_pointer(row_ptr) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (nnz > 0)
        TG_CK(cudaMemcpyAsync(col_in.p, col, sizeof(int32_t) * nnz,
                              is_device_pointer(col) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (n > 0)
        TG_CK(cudaMemcpyAsync(ty_in.p, types, n,
                              is_device_pointer(types) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    G.node_off.alloc(sizeof(int64_t) * (ngraphs + 1));
    TG_CK(cudaMemcpyAsync(G.node_off.p, G.h_node_off.data(), sizeof(int64_t) * (ngraphs + 1),
                          cudaMemcpyHostToDevice, s));
    const int64_t *rp = rp_in.as<int64_t>();
    const int32_t *cl = col_in.as<int32_t>();
    const uint8_t *ty = ty_in.as<uint8_t>();

    // 1. ranges, row pointers, types
    ++G.last_launches;
    k_check_rows<<<blocks_for(n + 1, kThreads), kThreads, 0, s>>>(n, nnz, rp, ty, L, status);
    if (nnz > 0) ++G.last_launches;
    if (nnz > 0) k_check_cols<<<blocks_for(nnz, kThreads), kThreads, 0, s>>>(nnz, n, cl, status);
    TG_CK(cudaGetLastError());
    if (read_status(G.status, s) & ST_INVALID_GRAPH) throw Error{TG_ERR_INVALID_GRAPH, "row pointers, ids or types"};

    // 2. priority order: sort nodes by (graph, degree), stable in id
    G.old_of.alloc(sizeof(int32_t) * std::max<int64_t>(n, 1));
    G.rp.alloc(sizeof(int64_t) * (n + 1));
    TBuf new_of(sizeof(int32_t) * std::max<int64_t>(n, 1), s);
    {
        TBuf keys(sizeof(unsigned long long) * std::max<int64_t>(n, 1), s), keys2(sizeof(unsigned long long) * std::max<int64_t>(n, 1), s);
        TBuf vals(sizeof(int32_t) * std::max<int64_t>(n, 1), s);
        if (n > 0) {
            ++G.last_launches;
            k_degree_keys<<<blocks_for(n, kThreads), kThreads, 0, s>>>(n, rp, G.node_off.as<int64_t>(), ngraphs,
                                                                       keys.as<unsigned long long>(), vals.as<int32_t>());
            TG_CK(cudaGetLastError());
            int end_bit = 32 + bits_for(ngraphs);
            cub_call([&](void *t, size_t &b) {
                return cub::DeviceRadixSort::SortPairs(t, b, keys.as<unsigned long long>(), keys2.as<unsigned long long>(),
                                                       vals.as<int32_t>(), G.old_of.as<int32_t>(), n, 0, end_bit, s);
            }, s);
        }
        TBuf ndeg(sizeof(int64_t) * (n + 1), s);
        ++G.last_launches;
        k_inverse<<<blocks_for(n + 1, kThreads), kThreads, 0, s>>>(n, G.old_of.as<int32_t>(), rp, new_of.as<int32_t>(),
                                                                   ndeg.as<int64_t>());
        TG_CK(cudaGetLastError());
        cub_call([&](void *t, size_t &b) {
            return cub::DeviceScan::ExclusiveSum(t, b, ndeg.as<int64_t>(), G.rp.as<int64_t>(), n + 1, s);
        }, s);
    }

    // 3. rows sorted by (type, internal id)
    G.adj.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    G.toff.alloc(sizeof(int32_t) * std::max<int64_t>(n * (L + 1), 1));
    G.pivot.alloc(sizeof(int32_t) * std::max<int64_t>(n * L, 1));
    G.nplus.alloc(sizeof(int32_t) * std::max<int64_t>(n, 1));
    G.ty.alloc(std::max<int64_t>(n, 1));
    {
        TBuf keys(sizeof(unsigned long long) * std::max<int64_t>(nnz, 1), s), keys2(sizeof(unsigned long long) * std::max<int64_t>(nnz, 1), s);
        if (n > 0) {
            ++G.last_launches;
            k_fill_keys<<<blocks_for(n * kWarp, kThreads), kThreads, 0, s>>>(
                n, rp, cl, ty, new_of.as<int32_t>(), G.rp.as<int64_t>(), G.node_off.as<int64_t>(), ngraphs,
                keys.as<unsigned long long>(), status);
            TG_CK(cudaGetLastError());
        }
        if (nnz > 0) {
            int end_bit = 32 + bits_for(n);
            cub_call([&](void *t, size_t &b) {
                return cub::DeviceRadixSort::SortKeys(t, b, keys.as<unsigned long long>(), keys2.as<unsigned long long>(),
                                                      nnz, 0, end_bit, s);
            }, s);
        }
        if (n > 0) {
            ++G.last_launches;
            k_rows<<<blocks_for(n * kWarp, kThreads), kThreads, 0, s>>>(n, L, G.rp.as<int64_t>(), keys2.as<unsigned long long>(),
                                                                       G.adj.as<int32_t>(), G.toff.as<int32_t>(),
                                                                       G.pivot.as<int32_t>(), G.nplus.as<int32_t>(), status);
            TG_CK(cudaGetLastError());
        }
    }
    // types by internal id
    if (n > 0) {
        ++G.last_launches;
        k_gather_types<<<blocks_for(n, kThreads), kThreads, 0, s>>>(n, G.old_of.as<int32_t>(), ty, G.ty.as<uint8_t>());
        TG_CK(cudaGetLastError());
    }
    if (read_status(G.status, s) & ST_INVALID_GRAPH) throw Error{TG_ERR_INVALID_GRAPH, "self-loop, repeated entry or cross-graph edge"};

    // 4. edges in caller order
    const int64_t m = G.m;
    G.slot_eid.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1));
    G.e_lo.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1));
    G.e_hi.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1));
    G.e_slot_lo.alloc(sizeof(int64_t) * std::max<int64_t>(m, 1));
    G.e_slot_hi.alloc(sizeof(int64_t) * std::max<int64_t>(m, 1));
    {
        TBuf ekeys(sizeof(unsigned long long) * std::max<int64_t>(m, 1), s), ekeys2(sizeof(unsigned long long) * std::max<int64_t>(m, 1), s);
        TBuf eslots(sizeof(int64_t) * std::max<int64_t>(m, 1), s), eslots2(sizeof(int64_t) * std::max<int64_t>(m, 1), s);
        TBuf counter(sizeof(unsigned long long), s);
        TG_CK(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), s));
        if (n > 0) {
            ++G.last_launches;
            k_edge_keys<<<blocks_for(n * kWarp, kThreads), kThreads, 0, s>>>(
                n, G.rp.as<int64_t>(), G.adj.as<int32_t>(), G.old_of.as<int32_t>(), m, ekeys.as<unsigned long long>(),
                eslots.as<int64_t>(), counter.as<unsigned long long>(), status);
            TG_CK(cudaGetLastError());
        }
        unsigned long long cnt = 0;
        TG_CK(cudaMemcpyAsync(&cnt, counter.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
        TG_CK(cudaStreamSynchronize(s));
        if ((int64_t)cnt != m) throw Error{TG_ERR_INVALID_GRAPH, "asymmetric rows"};
        if (m > 0) {
            cub_call([&](void *t, size_t &b) {
                return cub::DeviceRadixSort::SortPairs(t, b, ekeys.as<unsigned long long>(), ekeys2.as<unsigned long long>(),
                                                       eslots.as<int64_t>(), eslots2.as<int64_t>(), m, 0, 64, s);
            }, s);
            ++G.last_launches;
            k_edges<<<blocks_for(m, kThreads), kThreads, 0, s>>>(
                m, ekeys2.as<unsigned long long>(), eslots2.as<int64_t>(), G.view(), new_of.as<int32_t>(),
                G.e_lo.as<int32_t>(), G.e_hi.as<int32_t>(), G.e_slot_lo.as<int64_t>(), G.e_slot_hi.as<int64_t>(),
                G.slot_eid.as<int32_t>(), status);
            TG_CK(cudaGetLastError());
        }
    }
    // per-graph edge ranges: edges of graph g are those whose smaller caller id lies in graph g;
    // with caller ids grouped by graph and lexicographic edge order they are contiguous.
    G.h_edge_off.assign(ngraphs + 1, 0);
    {
        std::vector<int64_t> h_rp(n + 1);
        TG_CK(cudaMemcpyAsync(h_rp.data(), rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
        TG_CK(cudaStreamSynchronize(s));
        // each graph holds half of its rows' entries
        for (int g = 0; g < ngraphs; ++g)
            G.h_edge_off[g + 1] = G.h_edge_off[g] + (h_rp[G.h_node_off[g + 1]] - h_rp[G.h_node_off[g]]) / 2;
        G.h_slot_off.assign(ngraphs + 1, 0);
        for (int g = 0; g <= ngraphs; ++g) G.h_slot_off[g] = h_rp[G.h_node_off[g]];
        G.max_degree = 0;
        for (int64_t v = 0; v < n; ++v) G.max_degree = std::max(G.max_degree, h_rp[v + 1] - h_rp[v]);
        if (G.h_edge_off[ngraphs] != m) throw Error{TG_ERR_INVALID_GRAPH, "edge count per graph"};
    }
    G.edge_off.alloc(sizeof(int64_t) * (ngraphs + 1));
    TG_CK(cudaMemcpyAsync(G.edge_off.p, G.h_edge_off.data(), sizeof(int64_t) * (ngraphs + 1), cudaMemcpyHostToDevice, s));

    // 5. per-node typed degree sums
    G.delta.alloc(sizeof(int64_t) * std::max<int64_t>(n * L * L, 1));
    if (n > 0) {
        ++G.last_launches;
        k_delta<<<blocks_for(n * kWarp, kThreads), kThreads, 0, s>>>(G.view(), G.delta.as<int64_t>());
        TG_CK(cudaGetLastError());
    }

    // 6. work lists
    {
        TBuf work(sizeof(int64_t) * std::max<int64_t>(n, 1), s);
        TBuf fl(std::max<int64_t>(n, 1), s), fh(std::max<int64_t>(n, 1), s), ids(sizeof(int32_t) * std::max<int64_t>(n, 1), s);
        TBuf key(sizeof(unsigned long long) * std::max<int64_t>(n, 1), s);
        TBuf fhub(std::max<int64_t>(n, 1), s);
        if (n > 0) {
            ++G.last_launches;
            k_anchor_work<<<blocks_for(n * kWarp, kThreads), kThreads, 0, s>>>(G.view(), work.as<int64_t>());
            ++G.last_launches;
            k_classify_anchors<<<blocks_for(n, kThreads), kThreads, 0, s>>>(
                n, work.as<int64_t>(), opt.light_anchor_max_wedges, opt.hub_min_wedges, fl.as<uint8_t>(),
                fh.as<uint8_t>(), fhub.as<uint8_t>(), ids.as<int32_t>(), key.as<unsigned long long>());
            TG_CK(cudaGetLastError());
        }
        G.n_anchors_light = select_flagged(ids.as<int32_t>(), fl.as<uint8_t>(), n, G.anchors_light, s);
        G.n_anchors_heavy = select_flagged(ids.as<int32_t>(), fh.as<uint8_t>(), n, G.anchors_heavy, s);
        sort_desc_by_key(G.anchors_heavy, G.n_anchors_heavy, key.as<unsigned long long>(), s, G.last_launches);
        {   // heavy anchors above the shared-memory hash's limit (they lead the sorted list)
            TBuf cnt(sizeof(unsigned long long), s);
            TG_CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
            if (G.n_anchors_heavy > 0) {
                ++G.last_launches;
                k_count_above<<<blocks_for(G.n_anchors_heavy, kThreads), kThreads, 0, s>>>(
                    G.n_anchors_heavy, G.anchors_heavy.as<int32_t>(), key.as<unsigned long long>(), kHeavyFit,
                    cnt.as<unsigned long long>());
                TG_CK(cudaGetLastError());
            }
            unsigned long long c = 0;
            TG_CK(cudaMemcpyAsync(&c, cnt.p, sizeof(c), cudaMemcpyDeviceToHost, s));
            TG_CK(cudaStreamSynchronize(s));
            G.n_heavy_dense = (int64_t)c;
        }
        G.n_hubs = select_flagged(ids.as<int32_t>(), fhub.as<uint8_t>(), n, G.hubs, s);
        G.h_hub_id.assign((size_t)G.n_hubs, 0);
        G.h_hub_wedges.assign((size_t)G.n_hubs, 0);
        if (G.n_hubs > 0) {
            TBuf wk(sizeof(unsigned long long) * (size_t)G.n_hubs, s);
            ++G.last_launches;
            k_gather_keys<<<blocks_for(G.n_hubs, kThreads), kThreads, 0, s>>>(
                G.n_hubs, G.hubs.as<int32_t>(), key.as<unsigned long long>(), wk.as<unsigned long long>());
            TG_CK(cudaGetLastError());
            TG_CK(cudaMemcpyAsync(G.h_hub_id.data(), G.hubs.p, sizeof(int32_t) * G.n_hubs, cudaMemcpyDeviceToHost, s));
            TG_CK(cudaMemcpyAsync(G.h_hub_wedges.data(), wk.p, sizeof(int64_t) * G.n_hubs, cudaMemcpyDeviceToHost, s));
            TG_CK(cudaStreamSynchronize(s));
        }
    }
    {
        TBuf fl(std::max<int64_t>(m, 1), s), fh(std::max<int64_t>(m, 1), s), ids(sizeof(int32_t) * std::max<int64_t>(m, 1), s);
        TBuf cost(sizeof(unsigned long long) * std::max<int64_t>(m, 1), s);
        if (m > 0) {
            ++G.last_launches;
            k_classify_edges<<<blocks_for(m, kThreads), kThreads, 0, s>>>(
                m, G.view(), opt.light_edge_max_degree, fl.as<uint8_t>(), fh.as<uint8_t>(), ids.as<int32_t>(),
                cost.as<unsigned long long>());
            TG_CK(cudaGetLastError());
        }
        G.n_edges_light = select_flagged(ids.as<int32_t>(), fl.as<uint8_t>(), m, G.edges_light, s);
        G.n_edges_heavy = select_flagged(ids.as<int32_t>(), fh.as<uint8_t>(), m, G.edges_heavy, s);
        sort_desc_by_key(G.edges_heavy, G.n_edges_heavy, cost.as<unsigned long long>(), s, G.last_launches);
    }
    if (read_status(G.status, s) & ST_INVALID_GRAPH) throw Error{TG_ERR_INVALID_GRAPH, "asymmetric rows"};

    // 7. higher-priority neighbour lists (4-clique pass); one per edge
    G.plus_off.alloc(sizeof(int64_t) * (n + 1));
    {
        TBuf np64(sizeof(int64_t) * (n + 1), s);
        TG_CK(cudaMemsetAsync(np64.p, 0, sizeof(int64_t) * (n + 1), s));
        if (n > 0) {
            ++G.last_launches;
            k_widen<<<blocks_for(n, kThreads), kThreads, 0, s>>>(n, G.nplus.as<int32_t>(), np64.as<int64_t>());
            TG_CK(cudaGetLastError());
        }
        cub_call([&](void *t, size_t &b) {
            return cub::DeviceScan::ExclusiveSum(t, b, np64.as<int64_t>(), G.plus_off.as<int64_t>(), n + 1, s);
        }, s);
    }
    int64_t nplus_total = 0;
    TG_CK(cudaMemcpyAsync(&nplus_total, G.plus_off.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TG_CK(cudaStreamSynchronize(s));
    if (nplus_total != m) throw Error{TG_ERR_INTERNAL, "higher-priority neighbours"};
    G.plus_adj.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1));
    if (n > 0) {
        ++G.last_launches;
        k_plus_fill<<<blocks_for(n * kWarp, kThreads), kThreads, 0, s>>>(G.view(), G.plus_adj.as<int32_t>());
        TG_CK(cudaGetLastError());
    }
}

}  // namespace tg

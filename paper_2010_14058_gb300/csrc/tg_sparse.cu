// tg_sparse.cu -- per-edge counts in the sparse form of Sec. 4.6 (X_ij):
// only the nonzero slots of each edge, as (slot, count) pairs.
//
// The edges are counted in windows whose dense rows fit a bounded scratch
// (the wedge and triangle passes run once, for the first window); for each
// window one kernel counts every row's nonzeros, a scan turns the counts
// into offsets after the running total, and a second kernel writes the pairs
// in slot order.  One host synchronisation per window reads the window's
// total, so the call can stop writing when the caller's capacity runs out
// and still report the capacity needed.
#include <algorithm>

#include <cub/device/device_scan.cuh>

#include "tg_host.hpp"

namespace tg {
namespace {

constexpr size_t kWindowBytes = size_t(1) << 30;   // dense rows of one window

// warp per edge: nonzero slots of its dense row
__global__ void k_sparse_nnz(const uint32_t *__restrict__ rows, int S, int64_t ne, int64_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e <= ne; e += nw) {
        if (e == ne) {
            if (lane == 0) cnt[ne] = 0;
            continue;
        }
        const uint32_t *r = rows + e * S;
        int c = 0;
        for (int s = lane; s < S; s += 32) c += r[s] != 0 ? 1 : 0;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[e] = c;
    }
}

// row offsets of the window: base + exclusive prefix
__global__ void k_sparse_offsets(const int64_t *__restrict__ local, int64_t ne, int64_t base, int64_t *row_off) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < ne) row_off[e] = base + local[e];
}

// warp per edge: its nonzero (slot, count) pairs in slot order
__global__ void k_sparse_fill(const uint32_t *__restrict__ rows, int S, int64_t ne, const int64_t *__restrict__ local,
                              int64_t base, uint16_t *slot, uint32_t *value) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < ne; e += nw) {
        const uint32_t *r = rows + e * S;
        int64_t out = base + local[e];
        for (int s0 = 0; s0 < S; s0 += 32) {
            const int s = s0 + lane;
            const uint32_t v = s < S ? r[s] : 0u;
            const unsigned nz = __ballot_sync(0xffffffffu, v != 0);
            if (v != 0) {
                const int64_t x = out + __popc(nz & ((1u << lane) - 1u));
                slot[x] = (uint16_t)s;
                value[x] = v;
            }
            out += __popc(nz);
        }
    }
}

int grid_warps(int64_t items) {
    const int64_t b = (items * 32 + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 32));
}

}  // namespace

int64_t count_sparse(Graph &G, int k, int64_t *row_off, uint16_t *slot, uint32_t *value, int64_t cap, bool &fits,
                     cudaStream_t s) {
    const int S = (int)per_edge_slots(G.L, k);
    const int64_t m = G.m;
    const int64_t window = std::max<int64_t>(1, std::min<int64_t>(m, (int64_t)(kWindowBytes / (S * sizeof(uint32_t)))));
    DBuf dense, cnt, local;
    dense.owner = cnt.owner = local.owner = &G.stream;
    dense.alloc((size_t)window * S * sizeof(uint32_t));
    cnt.alloc((size_t)(window + 1) * sizeof(int64_t));
    local.alloc((size_t)(window + 1) * sizeof(int64_t));
    size_t tb = 0;
    TG_CK(cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt.as<int64_t>(), local.as<int64_t>(), window + 1, s));
    DBuf tmp;
    tmp.owner = &G.stream;
    tmp.alloc(std::max<size_t>(tb, 16));
    G.prepared_k = 0;                                     // fresh triangle and wedge passes
    int64_t base = 0;
    fits = true;
    for (int64_t b = 0; b < m; b += window) {
        const int64_t e = std::min(m, b + window), ne = e - b;
        run_count(G, k, b, e, dense.as<uint32_t>(), G.gacc.as<unsigned long long>(), false, s);
        k_sparse_nnz<<<grid_warps(ne + 1), 256, 0, s>>>(dense.as<uint32_t>(), S, ne, cnt.as<int64_t>());
        TG_CK(cudaGetLastError());
        size_t tb2 = tb;
        TG_CK(cub::DeviceScan::ExclusiveSum(tmp.p, tb2, cnt.as<int64_t>(), local.as<int64_t>(), ne + 1, s));
        int64_t total = 0;
        TG_CK(cudaMemcpyAsync(&total, local.as<int64_t>() + ne, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TG_CK(cudaStreamSynchronize(s));
        if (row_off) {
            k_sparse_offsets<<<(int)((ne + 255) / 256), 256, 0, s>>>(local.as<int64_t>(), ne, base, row_off + b);
            TG_CK(cudaGetLastError());
        }
        if (slot && value && fits && base + total <= cap) {
            k_sparse_fill<<<grid_warps(ne), 256, 0, s>>>(dense.as<uint32_t>(), S, ne, local.as<int64_t>(), base, slot,
                                                         value);
            TG_CK(cudaGetLastError());
        } else {
            fits = false;
        }
        base += total;
    }
    if (row_off) TG_CK(cudaMemcpyAsync(row_off + m, &base, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    TG_CK(cudaStreamSynchronize(s));                       // `base` lives on this stack frame
    return base;
}

}  // namespace tg

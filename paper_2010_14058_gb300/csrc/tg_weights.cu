// tg_weights.cu -- the typed-graphlet weighted graph of Alg. 5 (its first
// step): for one typed graphlet H, W_ij = the number of instances of H that
// contain both endpoints of the edge (i, j), and the typed-graphlet degree
// D_ii = sum_j W_ij.
//
// An instance of H containing the edge (i, j) is counted in exactly one
// per-edge slot of the edge's row: the orbit of (i, j) in H's shape and the
// pair of types of the other nodes.  With the edge's types (p, q) fixed, the
// pair is the type multiset of H minus {p, q}, so each (p, q) selects at most
// one slot per orbit of the shape (three orbits at most).  The host builds
// that (p, q) -> slots table; a kernel sums the slots of every edge.
#include <algorithm>
#include <vector>

#include "tg_host.hpp"

namespace tg {
namespace {

constexpr int kMaxWeightSlots = 3;
constexpr int32_t kEdgeItself = -2;            // block 0: the edge is its own instance

int64_t multichoose_h(int n, int r) {         // C(n + r - 1, r)
    int64_t v = 1;
    for (int x = 1; x <= r; ++x) v = v * (n + x - 1) / x;
    return v;
}

int64_t rank_h(int L, std::vector<int> s) {   // lexicographic rank of a sorted multiset
    std::sort(s.begin(), s.end());
    const int K = (int)s.size();
    int64_t r = 0;
    int prev = 0;
    for (int k = 0; k < K; ++k) {
        for (int v = prev; v < s[k]; ++v) r += multichoose_h(L - v, K - k - 1);
        prev = s[k];
    }
    return r;
}

int block_of_orbit(int o) {
    switch (o) {
        case 3: case 4: return 3;
        case 5: return 4;
        case 6: return 5;
        case 7: case 8: case 9: return 6;
        case 10: case 11: return 7;
        default: return 8;
    }
}

__global__ void k_weights(GraphView g, const uint32_t *__restrict__ rows, int S, const int32_t *__restrict__ table,
                          const int32_t *__restrict__ old_of, int64_t *weights, unsigned long long *degree) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= g.m) return;
    const int32_t i = g.e_lo[e], j = g.e_hi[e];
    const int32_t *sl = table + (g.ty[i] * g.L + g.ty[j]) * kMaxWeightSlots;
    int64_t w = 0;
    for (int k = 0; k < kMaxWeightSlots; ++k) {
        const int32_t s = sl[k];
        if (s == kEdgeItself) w += 1;
        else if (s >= 0) w += rows[e * S + s];
    }
    weights[e] = w;
    if (degree && w) {
        atomicAdd(&degree[old_of[i]], (unsigned long long)w);
        atomicAdd(&degree[old_of[j]], (unsigned long long)w);
    }
}

}  // namespace

// (p, q) -> slots of the typed graphlet (block, rank); throws on a bad block
// or rank
std::vector<int32_t> weight_slots(int L, int k, int block, int64_t rank) {
    const int nb = k == 4 ? 9 : 3;
    if (block < 0 || block >= nb) throw Error{TG_ERR_INVALID_ARG, "block"};
    const int K = block == 0 ? 2 : block <= 2 ? 3 : 4;
    if (rank < 0 || rank >= multichoose_h(L, K)) throw Error{TG_ERR_INVALID_ARG, "rank"};
    const int P = L * (L + 1) / 2;
    std::vector<int32_t> table((size_t)L * L * kMaxWeightSlots, -1);
    for (int p = 0; p < L; ++p)
        for (int q = 0; q < L; ++q) {
            int32_t *sl = &table[((size_t)p * L + q) * kMaxWeightSlots];
            int n = 0;
            auto add = [&](int32_t slot) {
                if (n == kMaxWeightSlots) throw Error{TG_ERR_INTERNAL, "weight slots"};
                sl[n++] = slot;
            };
            if (block == 0) {
                if (rank_h(L, {p, q}) == rank) add(kEdgeItself);
            } else if (block <= 2) {
                for (int t = 0; t < L; ++t)
                    if (rank_h(L, {p, q, t}) == rank) add((block == 1 ? 0 : L) + t);
            } else {
                for (int o = 3; o <= 12; ++o) {
                    if (block_of_orbit(o) != block) continue;
                    int pi = 0;
                    for (int t = 0; t < L; ++t)
                        for (int u = t; u < L; ++u, ++pi)
                            if (rank_h(L, {p, q, t, u}) == rank) add(2 * L + (o - 3) * P + pi);
                }
            }
        }
    return table;
}

void launch_weights(Graph &G, int k, const uint32_t *rows, int block, int64_t rank, int64_t *weights,
                    int64_t *degree, cudaStream_t s) {
    const std::vector<int32_t> table = weight_slots(G.L, k, block, rank);
    TBuf dt(sizeof(int32_t) * table.size(), s);
    TG_CK(cudaMemcpyAsync(dt.p, table.data(), sizeof(int32_t) * table.size(), cudaMemcpyHostToDevice, s));
    if (degree) TG_CK(cudaMemsetAsync(degree, 0, sizeof(int64_t) * (size_t)G.n, s));
    if (G.m > 0) {
        k_weights<<<(unsigned)((G.m + 255) / 256), 256, 0, s>>>(G.view(), rows, (int)per_edge_slots(G.L, k),
                                                               dt.as<int32_t>(), G.old_of.as<int32_t>(), weights,
                                                               reinterpret_cast<unsigned long long *>(degree));
        TG_CK(cudaGetLastError());
    }
    TG_CK(cudaStreamSynchronize(s));                   // the table lives on this stack frame
}

}  // namespace tg

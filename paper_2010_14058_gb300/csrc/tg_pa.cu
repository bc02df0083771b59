// tg_pa.cu -- position-aware typed graphlets (Sec. 5, Def. 8): layout, class
// tables and the global finalisation.
//
// Def. 8 identifies two typed instances of one shape when an isomorphism
// between them maps every node onto a node of the same type.  With the
// shape's nodes numbered, a position-aware typed graphlet is a labelling
// (types of nodes 0..k-1) up to the automorphisms of the numbered shape; a
// class is represented by its lexicographically smallest labelling and the
// classes of a shape are ranked in the order of those representatives.
// Numbered shapes, one per global block:
//   0 edge 0-1          1 3-path, 0 the centre       2 triangle
//   3 4-path 0-1-2-3    4 4-star, 0 the centre       5 4-cycle 0-1-2-3-0
//   6 tailed triangle, 0 the degree-3 node, 1 the tail, 2-3 the triangle's
//     other edge         7 chordal cycle, 0-1 the chord      8 4-clique
//
// Per-edge rows (k_epi4_pa): blocks O1..O12 of the edge e = {lo, hi} (caller
// ids, lo < hi), side 0 = lo, 1 = hi, ordered pairs (x, y) at x*L + y:
//   O1  3-path, [side of the centre][type of the third node]
//   O2  triangle, [type of the third node]
//   O3  4-path end edge, [side of the inner endpoint][its other neighbour][far end]
//   O4  4-path centre edge, [lo's other neighbour][hi's other neighbour]
//   O5  4-star, [side of the centre][pair of the other leaves]
//   O6  4-cycle, [lo's other neighbour][hi's other neighbour]
//   O7  tailed-triangle tail edge, [side of the degree-3 node][pair of the other triangle nodes]
//   O8  tailed-triangle edge opposite the degree-3 node, [degree-3 node][tail]
//   O9  tailed-triangle edge at the degree-3 node, [its side][third triangle node][tail]
//   O10 chordal-cycle outer edge, [side of the degree-3 endpoint][other degree-3 node][other degree-2 node]
//   O11 chordal-cycle chord, [pair of the degree-2 nodes]
//   O12 4-clique, [pair of the other nodes]
// A slot and the endpoint types (phi_lo, phi_hi) fix the instance's
// labelling, hence its class: the host tabulates that map once per handle.
#include <algorithm>
#include <array>
#include <numeric>
#include <vector>

#include "tg_host.hpp"

namespace tg {
namespace {

constexpr int kShapeNodes[9] = {2, 3, 3, 4, 4, 4, 4, 4, 4};
constexpr int kShapeEdges[9] = {1, 2, 3, 3, 3, 4, 4, 5, 6};   // |E(H)| (Table 3)

bool shape_adjacent(int b, int u, int v) {
    auto has = [&](int a, int c) { return (u == a && v == c) || (u == c && v == a); };
    switch (b) {
        case 0: return has(0, 1);
        case 1: return has(0, 1) || has(0, 2);
        case 2: case 8: return u != v;
        case 3: return has(0, 1) || has(1, 2) || has(2, 3);
        case 4: return has(0, 1) || has(0, 2) || has(0, 3);
        case 5: return has(0, 1) || has(1, 2) || has(2, 3) || has(3, 0);
        case 6: return has(0, 1) || has(0, 2) || has(0, 3) || has(2, 3);
        default: return u != v && !has(2, 3);                  // chordal cycle: K4 less 2-3
    }
}

// class rank of every labelling code (code = sum lab[a] L^(k-1-a)) of shape b
std::vector<int32_t> shape_classes(int L, int b, int32_t &nclass) {
    const int k = kShapeNodes[b];
    std::array<int, 4> perm{0, 1, 2, 3};
    std::vector<std::array<int, 4>> aut;
    do {
        bool ok = true;
        for (int u = 0; u < k && ok; ++u)
            for (int v = 0; v < k && ok; ++v)
                ok = shape_adjacent(b, u, v) == shape_adjacent(b, perm[u], perm[v]);
        if (ok) aut.push_back(perm);
    } while (std::next_permutation(perm.begin(), perm.begin() + k));
    int ncodes = 1;
    for (int a = 0; a < k; ++a) ncodes *= L;
    std::vector<int32_t> cls(ncodes);
    nclass = 0;
    for (int code = 0; code < ncodes; ++code) {
        int lab[4] = {0, 0, 0, 0};
        for (int a = k - 1, x = code; a >= 0; --a, x /= L) lab[a] = x % L;
        int smallest = code;
        for (const auto &p : aut) {
            int img = 0;
            for (int a = 0; a < k; ++a) img = img * L + lab[p[a]];
            smallest = std::min(smallest, img);
        }
        // codes rise with the lexicographic order, so a class's smallest
        // member is met before the rest of it
        cls[code] = smallest == code ? nclass++ : cls[smallest];
    }
    return cls;
}

int pa_pair_index(int L, int t, int u) {                      // t <= u, lexicographic
    return t * L - t * (t - 1) / 2 + (u - t);
}

void pair_of_index(int L, int r, int &t, int &u) {
    t = 0;
    while (pa_pair_index(L, t, L - 1) < r) ++t;
    u = t + (r - pa_pair_index(L, t, t));
}

}  // namespace

PaLayout pa_layout(int L) {
    PaLayout Y;
    Y.L = L;
    const int LL = L * L, P = L * (L + 1) / 2;
    const int size[13] = {0, 2 * L, L, 2 * LL, LL, 2 * P, LL, 2 * P, LL, 2 * LL, 2 * LL, P, P};
    Y.off[0] = 0;
    int s = 0;
    for (int o = 1; o <= 12; ++o) {
        Y.off[o] = s;
        s += size[o];
    }
    Y.S = s;
    int64_t g = 0;
    for (int b = 0; b < 9; ++b) {
        int32_t nc = 0;
        shape_classes(L, b, nc);
        Y.boff[b] = g;
        Y.bsize[b] = nc;
        g += nc;
    }
    Y.boff[9] = g;
    Y.G = g;
    return Y;
}

// canonical labelling of class `rank` of block b
bool pa_labelling(int L, int b, int64_t rank, int32_t *lab) {
    int32_t nc = 0;
    const std::vector<int32_t> cls = shape_classes(L, b, nc);
    if (rank < 0 || rank >= nc) return false;
    const int k = kShapeNodes[b];
    for (int code = 0; code < (int)cls.size(); ++code)
        if (cls[code] == rank) {
            for (int a = k - 1, x = code; a >= 0; --a, x /= L) lab[a] = x % L;
            return true;
        }
    return false;
}

// global class slot of (phi_lo, phi_hi, slot); slot == S: the edge itself
std::vector<int32_t> pa_class_table(const PaLayout &Y) {
    const int L = Y.L, LL = L * L, P = L * (L + 1) / 2, S = Y.S;
    std::vector<std::vector<int32_t>> cls(9);
    for (int b = 0; b < 9; ++b) {
        int32_t nc = 0;
        cls[b] = shape_classes(L, b, nc);
    }
    std::vector<int32_t> table((size_t)LL * (S + 1));
    for (int pl = 0; pl < L; ++pl)
        for (int ph = 0; ph < L; ++ph) {
            int32_t *row = &table[(size_t)(pl * L + ph) * (S + 1)];
            auto put = [&](int slot, int b, int l0, int l1, int l2, int l3) {
                const int lab[4] = {l0, l1, l2, l3};
                int code = 0;
                for (int a = 0; a < kShapeNodes[b]; ++a) code = code * L + lab[a];
                row[slot] = (int32_t)(Y.boff[b] + cls[b][code]);
            };
            put(S, 0, pl, ph, 0, 0);
            for (int slot = 0; slot < S; ++slot) {
                int o = 12;
                while (Y.off[o] > slot) --o;
                const int r = slot - Y.off[o];
                const int side = (o == 5 || o == 7) ? r / P : (o == 1 ? r / L : r / LL);
                const int me = side == 0 ? pl : ph, other = side == 0 ? ph : pl;
                const int x = (r % LL) / L, y = r % L;
                int t = 0, u = 0;
                pair_of_index(L, r % P, t, u);
                switch (o) {
                    case 1: put(slot, 1, me, other, r % L, 0); break;
                    case 2: put(slot, 2, pl, ph, r, 0); break;
                    case 3: put(slot, 3, y, x, me, other); break;
                    case 4: put(slot, 3, x, pl, ph, y); break;
                    case 5: put(slot, 4, me, other, t, u); break;
                    case 6: put(slot, 5, pl, ph, y, x); break;
                    case 7: put(slot, 6, me, other, t, u); break;
                    case 8: put(slot, 6, x, y, pl, ph); break;
                    case 9: put(slot, 6, me, y, other, x); break;
                    case 10: put(slot, 7, me, x, other, y); break;
                    case 11: put(slot, 7, pl, ph, t, u); break;
                    default: put(slot, 8, pl, ph, t, u); break;
                }
            }
        }
    return table;
}

namespace {

struct PaBlocks {
    int64_t boff[10];                  // first class of each block
    int32_t edges[9];                  // |E(H)| of each block
};

// position-aware totals: the raw per-class edge sums divided by |E(H)|
// (Sec. 6), exact
__global__ void k_finalize_pa(int ngraphs, int64_t G, PaBlocks pb, const unsigned long long *__restrict__ gacc,
                              int64_t *out, uint32_t *status) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ngraphs * G) return;
    const int64_t s = idx % G;
    int b = 0;
    while (b < 8 && pb.boff[b + 1] <= s) ++b;
    const unsigned long long v = gacc[idx], d = (unsigned long long)pb.edges[b];
    if (v % d) set_status(status, ST_INTERNAL);
    out[idx] = (int64_t)(v / d);
}

}  // namespace

void prepare_position_aware(Graph &G, cudaStream_t s) {
    if (!G.pa_cls.p) {
        const PaLayout Y = pa_layout(G.L);
        const std::vector<int32_t> table = pa_class_table(Y);
        G.pa = Y;
        G.pa_cls.alloc(table.size() * sizeof(int32_t));
        TG_CK(cudaMemcpyAsync(G.pa_cls.p, table.data(), table.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        TG_CK(cudaStreamSynchronize(s));                   // the table lives on this stack frame
    }
    const size_t gbytes = (size_t)G.ngraphs * G.pa.G * sizeof(unsigned long long);
    if (G.pa_gacc.bytes < gbytes) G.pa_gacc.alloc(gbytes);
    prepare_epi4_pa(G);
}

int64_t launch_finalize_pa(Graph &G, int64_t *global_out, cudaStream_t s) {
    const int64_t total = (int64_t)G.ngraphs * G.pa.G;
    PaBlocks pb;
    for (int b = 0; b < 10; ++b) pb.boff[b] = G.pa.boff[b];
    for (int b = 0; b < 9; ++b) pb.edges[b] = kShapeEdges[b];
    KernelTimer kt(G, s, "k_finalize_pa");
    k_finalize_pa<<<(unsigned)std::max<int64_t>(1, (total + 255) / 256), 256, 0, s>>>(
        G.ngraphs, G.pa.G, pb, G.pa_gacc.as<unsigned long long>(), global_out, G.status.as<uint32_t>());
    TG_CK(cudaGetLastError());
    return 1;
}

}  // namespace tg

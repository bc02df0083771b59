/*
 * graphgen.c -- seeded synthetic typed graphs (inputs only).
 *
 * This file holds no part of the counting method: it draws random simple
 * undirected graphs and node types, and turns an edge list into a symmetric
 * CSR.  Both the CPU oracle and the GPU path read graphs made here, so that
 * they see identical inputs.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) expands a 64-bit seed into
 * the state of xoshiro256** (Blackman, Vigna, "Scrambled linear pseudorandom
 * number generators", ACM TOMS 2021), which draws every variate.
 *
 * Models (the paper's synthetic graph families, Sec. 8.1 and 8.5):
 *   - Erdos-Renyi G(n, m): m distinct pairs uniform over all C(n,2) pairs.
 *   - Chung-Lu: expected-degree weights w_i = C (i + i0)^(-1/(gamma-1)),
 *     endpoints drawn in proportion to w, self-loops and repeats rejected
 *     until exactly m edges exist.
 *   - Stochastic block model: exact edge counts per block pair, uniform
 *     distinct pairs inside each block pair, node ids shuffled.
 *   - Ego networks: breadth-first balls around degree-proportional seeds
 *     of a parent graph, induced subgraphs, renumbered densely.
 *
 * Portable C99 (+ unsigned __int128, which gcc provides on x86_64 and
 * aarch64).  No architecture-specific code.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG */

typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int k = 0; k < 4; ++k) r->s[k] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(gg_rng *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform integer in [0, n) by the multiply-high method */
static inline uint64_t rng_below(gg_rng *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unit(gg_rng *r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* --------------------------------------------------------- pair hash set */

typedef struct { uint64_t *slot; uint64_t mask; } pairset;

#define PAIR_EMPTY 0xFFFFFFFFFFFFFFFFull

static int pairset_init(pairset *ps, int64_t expected) {
    uint64_t cap = 16;
    while (cap < (uint64_t)expected * 2 + 16) cap <<= 1;
    ps->slot = (uint64_t *)malloc(cap * sizeof(uint64_t));
    if (!ps->slot) return -1;
    memset(ps->slot, 0xFF, cap * sizeof(uint64_t));
    ps->mask = cap - 1;
    return 0;
}

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdull;
    z = (z ^ (z >> 33)) * 0xc4ceb9fe1a85ec53ull;
    return z ^ (z >> 33);
}

/* returns 1 if inserted, 0 if already present */
static int pairset_insert(pairset *ps, uint64_t key) {
    uint64_t h = mix64(key) & ps->mask;
    for (;;) {
        uint64_t v = ps->slot[h];
        if (v == PAIR_EMPTY) { ps->slot[h] = key; return 1; }
        if (v == key) return 0;
        h = (h + 1) & ps->mask;
    }
}

static void pairset_free(pairset *ps) { free(ps->slot); ps->slot = NULL; }

static inline uint64_t pair_key(int64_t u, int64_t v) {
    if (u > v) { int64_t t = u; u = v; v = t; }
    return ((uint64_t)u << 32) | (uint64_t)v;
}

/* ---------------------------------------------------------- node types */

int gg_types_uniform(int64_t n, int32_t L, uint64_t seed, uint8_t *types) {
    if (n < 0 || L < 1 || L > 255) return -1;
    gg_rng r; rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) types[i] = (uint8_t)rng_below(&r, (uint64_t)L);
    return 0;
}

/* P(t) proportional to (t+1)^(-s), t = 0..L-1, independent per node */
int gg_types_zipf(int64_t n, int32_t L, double s, uint64_t seed, uint8_t *types) {
    if (n < 0 || L < 1 || L > 255) return -1;
    double cdf[256], tot = 0.0;
    for (int t = 0; t < L; ++t) { tot += pow((double)(t + 1), -s); cdf[t] = tot; }
    for (int t = 0; t < L; ++t) cdf[t] /= tot;
    cdf[L - 1] = 1.0;
    gg_rng r; rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) {
        double u = rng_unit(&r);
        int t = 0;
        while (t < L - 1 && u >= cdf[t]) ++t;
        types[i] = (uint8_t)t;
    }
    return 0;
}

/* ------------------------------------------------------------ Erdos-Renyi */

int gg_er_edges(int64_t n, int64_t m, uint64_t seed, int32_t *eu, int32_t *ev) {
    if (n < 2 || m < 0 || (double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
    if (n > 0x7fffffff) return -1;
    pairset ps;
    if (pairset_init(&ps, m)) return -2;
    gg_rng r; rng_seed(&r, seed);
    int64_t k = 0;
    while (k < m) {
        int64_t u = (int64_t)rng_below(&r, (uint64_t)n);
        int64_t v = (int64_t)rng_below(&r, (uint64_t)n);
        if (u == v) continue;
        if (!pairset_insert(&ps, pair_key(u, v))) continue;
        eu[k] = (int32_t)(u < v ? u : v);
        ev[k] = (int32_t)(u < v ? v : u);
        ++k;
    }
    pairset_free(&ps);
    return 0;
}

/* ---------------------------------------------------------------- Chung-Lu */

/* Vose alias table over n weights */
typedef struct { double *prob; int32_t *alias; int64_t n; } alias_tab;

static int alias_build(alias_tab *a, const double *w, int64_t n) {
    a->n = n;
    a->prob = (double *)malloc((size_t)n * sizeof(double));
    a->alias = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *small = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *large = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!a->prob || !a->alias || !small || !large) return -1;
    double tot = 0.0;
    for (int64_t i = 0; i < n; ++i) tot += w[i];
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        a->prob[i] = w[i] * (double)n / tot;
        a->alias[i] = (int32_t)i;
        if (a->prob[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
    }
    while (ns > 0 && nl > 0) {
        int32_t s = small[--ns], l = large[--nl];
        a->alias[s] = l;
        a->prob[l] = (a->prob[l] + a->prob[s]) - 1.0;
        if (a->prob[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) a->prob[large[--nl]] = 1.0;
    while (ns > 0) a->prob[small[--ns]] = 1.0;
    free(small); free(large);
    return 0;
}

static inline int64_t alias_draw(const alias_tab *a, gg_rng *r) {
    int64_t i = (int64_t)rng_below(r, (uint64_t)a->n);
    return rng_unit(r) < a->prob[i] ? i : a->alias[i];
}

static void alias_free(alias_tab *a) { free(a->prob); free(a->alias); }

/* Weights w_i = C (i + i0)^(-1/(gamma-1)), i = 0..n-1, with C and i0 chosen
 * so that w_0 = wmax and sum_i w_i = wsum.  Written into w[]. */
int gg_chung_lu_weights(int64_t n, double gamma, double wmax, double wsum, double *w) {
    if (n < 2 || gamma <= 1.0 || wmax <= 0 || wsum <= wmax) return -1;
    double alpha = 1.0 / (gamma - 1.0);
    /* S(i0) = sum_i wmax * (i0 / (i + i0))^alpha grows with i0 */
    double lo = 1e-9, hi = 1.0;
    for (;;) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += wmax * pow(hi / ((double)i + hi), alpha);
        if (s >= wsum) break;
        hi *= 2.0;
        if (hi > 1e15) return -2;
    }
    for (int it = 0; it < 60; ++it) {
        double mid = 0.5 * (lo + hi), s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += wmax * pow(mid / ((double)i + mid), alpha);
        if (s < wsum) lo = mid; else hi = mid;
    }
    double i0 = 0.5 * (lo + hi);
    for (int64_t i = 0; i < n; ++i) w[i] = wmax * pow(i0 / ((double)i + i0), alpha);
    return 0;
}

int gg_chung_lu_edges(int64_t n, int64_t m, double gamma, double wmax, uint64_t seed,
                      int32_t *eu, int32_t *ev) {
    if (n < 2 || m < 0 || n > 0x7fffffff) return -1;
    double *w = (double *)malloc((size_t)n * sizeof(double));
    if (!w) return -2;
    int rc = gg_chung_lu_weights(n, gamma, wmax, 2.0 * (double)m, w);
    if (rc) { free(w); return rc; }
    alias_tab a;
    if (alias_build(&a, w, n)) { free(w); return -2; }
    free(w);
    pairset ps;
    if (pairset_init(&ps, m)) { alias_free(&a); return -2; }
    gg_rng r; rng_seed(&r, seed);
    int64_t k = 0, tries = 0, max_tries = 64 * m + 1000000;
    while (k < m) {
        if (++tries > max_tries) { pairset_free(&ps); alias_free(&a); return -3; }
        int64_t u = alias_draw(&a, &r), v = alias_draw(&a, &r);
        if (u == v) continue;
        if (!pairset_insert(&ps, pair_key(u, v))) continue;
        eu[k] = (int32_t)(u < v ? u : v);
        ev[k] = (int32_t)(u < v ? v : u);
        ++k;
    }
    pairset_free(&ps);
    alias_free(&a);
    return 0;
}

/* ---------------------------------------------------- stochastic block model */

/* Blocks b = 0..B-1 of the given sizes; block b is node type b.  The
 * expected edge mass of block pair (a,b) is sizes[a]*sizes[b]*aff[a*B+b] for
 * a != b and C(sizes[a],2)*aff[a*B+a] within a block; the m edges are split
 * over block pairs in proportion (largest remainder), then drawn as distinct
 * uniform pairs inside each block pair.  Node ids are a random permutation of
 * the block layout.  Writes eu/ev (m entries) and types (sum of sizes). */
int gg_sbm_edges(int32_t B, const int64_t *sizes, const double *aff, int64_t m, uint64_t seed,
                 int32_t *eu, int32_t *ev, uint8_t *types) {
    if (B < 1 || B > 255 || m < 0) return -1;
    int64_t n = 0;
    int64_t start[256];
    for (int b = 0; b < B; ++b) { start[b] = n; n += sizes[b]; }
    if (n > 0x7fffffff) return -1;
    int np = B * (B + 1) / 2;
    double *mass = (double *)calloc((size_t)np, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)np, sizeof(int64_t));
    double *frac = (double *)calloc((size_t)np, sizeof(double));
    if (!mass || !cnt || !frac) return -2;
    double tot = 0.0;
    int p = 0;
    for (int a = 0; a < B; ++a)
        for (int b = a; b < B; ++b, ++p) {
            double pairs = (a == b) ? 0.5 * (double)sizes[a] * (double)(sizes[a] - 1)
                                    : (double)sizes[a] * (double)sizes[b];
            mass[p] = pairs * aff[a * B + b];
            tot += mass[p];
        }
    int64_t assigned = 0;
    for (p = 0; p < np; ++p) {
        double x = (double)m * mass[p] / tot;
        cnt[p] = (int64_t)floor(x);
        frac[p] = x - (double)cnt[p];
        assigned += cnt[p];
    }
    while (assigned < m) {           /* largest remainder, ties to lowest index */
        int best = 0;
        for (p = 1; p < np; ++p) if (frac[p] > frac[best]) best = p;
        cnt[best] += 1; frac[best] = -1.0; ++assigned;
    }
    /* node id permutation (Fisher-Yates) */
    int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!perm) return -2;
    gg_rng r; rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)rng_below(&r, (uint64_t)(i + 1));
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (int b = 0; b < B; ++b)
        for (int64_t i = 0; i < sizes[b]; ++i) types[perm[start[b] + i]] = (uint8_t)b;
    pairset ps;
    if (pairset_init(&ps, m)) return -2;
    int64_t k = 0;
    p = 0;
    for (int a = 0; a < B; ++a)
        for (int b = a; b < B; ++b, ++p) {
            double pairs = (a == b) ? 0.5 * (double)sizes[a] * (double)(sizes[a] - 1)
                                    : (double)sizes[a] * (double)sizes[b];
            if ((double)cnt[p] > pairs) { pairset_free(&ps); return -4; }
            int64_t got = 0;
            while (got < cnt[p]) {
                int64_t u = start[a] + (int64_t)rng_below(&r, (uint64_t)sizes[a]);
                int64_t v = start[b] + (int64_t)rng_below(&r, (uint64_t)sizes[b]);
                if (u == v) continue;
                int64_t pu = perm[u], pv = perm[v];
                if (!pairset_insert(&ps, pair_key(pu, pv))) continue;
                eu[k] = (int32_t)(pu < pv ? pu : pv);
                ev[k] = (int32_t)(pu < pv ? pv : pu);
                ++k; ++got;
            }
        }
    pairset_free(&ps);
    free(perm); free(mass); free(cnt); free(frac);
    return 0;
}

/* ------------------------------------------------------------------- CSR */

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Symmetric CSR from an undirected edge list: each edge {u,v} appears in
 * row u and row v; every row sorted by neighbour id. */
int gg_edges_to_csr(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                    int64_t *row_ptr, int32_t *col) {
    if (n < 0 || m < 0) return -1;
    memset(row_ptr, 0, (size_t)(n + 1) * sizeof(int64_t));
    for (int64_t k = 0; k < m; ++k) {
        if (eu[k] < 0 || eu[k] >= n || ev[k] < 0 || ev[k] >= n) return -1;
        row_ptr[eu[k] + 1]++;
        row_ptr[ev[k] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!fill) return -2;
    memcpy(fill, row_ptr, (size_t)n * sizeof(int64_t));
    for (int64_t k = 0; k < m; ++k) {
        col[fill[eu[k]]++] = ev[k];
        col[fill[ev[k]]++] = eu[k];
    }
    free(fill);
    for (int64_t i = 0; i < n; ++i)
        qsort(col + row_ptr[i], (size_t)(row_ptr[i + 1] - row_ptr[i]), sizeof(int32_t), cmp_i32);
    return 0;
}

/* ------------------------------------------------------------ ego networks */

/* One ego network of a parent CSR graph: a breadth-first ball around `seed`
 * (neighbours visited in CSR order) truncated to at most `n_target` nodes,
 * then the induced subgraph.  The ball's nodes are renumbered 0..n_g-1 in
 * visit order.  `mark` is caller scratch of n_parent int32 entries holding
 * -1 on entry and on return.  If more than `m_cap` edges are induced, edges
 * are kept by a uniform random subset (partial Fisher-Yates).  Output
 * buffers: nodes[n_target], eu/ev[cap_edges].  Returns the edge count, or a
 * negative value on error (cap_edges too small). */
int64_t gg_ego_network(int64_t n_parent, const int64_t *row_ptr, const int32_t *col,
                       int32_t seed_node, int64_t n_target, int64_t m_cap, uint64_t seed,
                       int32_t *mark, int32_t *nodes, int64_t *n_out,
                       int32_t *eu, int32_t *ev, int64_t cap_edges) {
    if (seed_node < 0 || seed_node >= n_parent || n_target < 1) return -1;
    int64_t nn = 0, head = 0;
    nodes[nn] = seed_node; mark[seed_node] = (int32_t)nn; ++nn;
    while (head < nn && nn < n_target) {
        int32_t v = nodes[head++];
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1] && nn < n_target; ++k) {
            int32_t w = col[k];
            if (mark[w] < 0) { mark[w] = (int32_t)nn; nodes[nn++] = w; }
        }
    }
    int64_t me = 0;
    for (int64_t a = 0; a < nn; ++a) {
        int32_t v = nodes[a];
        for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            int32_t b = mark[col[k]];
            if (b > a) {
                if (me >= cap_edges) { for (int64_t q = 0; q < nn; ++q) mark[nodes[q]] = -1; return -2; }
                eu[me] = (int32_t)a; ev[me] = b; ++me;
            }
        }
    }
    for (int64_t q = 0; q < nn; ++q) mark[nodes[q]] = -1;
    if (me > m_cap) {
        gg_rng r; rng_seed(&r, seed);
        for (int64_t k = 0; k < m_cap; ++k) {
            int64_t j = k + (int64_t)rng_below(&r, (uint64_t)(me - k));
            int32_t tu = eu[k], tv = ev[k];
            eu[k] = eu[j]; ev[k] = ev[j]; eu[j] = tu; ev[j] = tv;
        }
        me = m_cap;
    }
    *n_out = nn;
    return me;
}

/* degree-proportional node draw: pick a uniform adjacency entry, return its row */
int32_t gg_degree_proportional_node(int64_t n, const int64_t *row_ptr, uint64_t seed) {
    gg_rng r; rng_seed(&r, seed);
    int64_t nnz = row_ptr[n];
    if (nnz <= 0) return (int32_t)rng_below(&r, (uint64_t)n);
    int64_t k = (int64_t)rng_below(&r, (uint64_t)nnz);
    int64_t lo = 0, hi = n;              /* largest i with row_ptr[i] <= k */
    while (hi - lo > 1) { int64_t mid = (lo + hi) / 2; if (row_ptr[mid] <= k) lo = mid; else hi = mid; }
    return (int32_t)lo;
}

/* uniform double in [0,1) from a seed (for callers that need one draw) */
double gg_unit_from_seed(uint64_t seed) { gg_rng r; rng_seed(&r, seed); return rng_unit(&r); }

/* ------------------------------------------------------- ego-network batch */

/* Ego network g of a parent CSR with an edge target: a breadth-first ball
 * around `seed_node` (neighbours in CSR order) grows one node at a time until
 * the induced subgraph holds at least m_target edges or n_max nodes.  Writes
 * the ball's parent ids in visit order to nodes[] (capacity n_max) and
 * returns the node count; *m_out receives the induced edge count.  `mark`
 * (n_parent int32, all -1) is restored before return. */
static int64_t ego_ball(const int64_t *rp, const int32_t *col, int32_t seed_node, int64_t m_target, int64_t n_max,
                        int32_t *mark, int32_t *nodes, int64_t *m_out) {
    int64_t nn = 0, head = 0, me = 0;
    nodes[nn] = seed_node; mark[seed_node] = (int32_t)nn; ++nn;
    while (head < nn && nn < n_max && me < m_target) {
        int32_t v = nodes[head++];
        for (int64_t k = rp[v]; k < rp[v + 1] && nn < n_max && me < m_target; ++k) {
            int32_t w = col[k];
            if (mark[w] >= 0) continue;
            int64_t add = 0;                           /* edges from w into the ball */
            for (int64_t q = rp[w]; q < rp[w + 1]; ++q) add += mark[col[q]] >= 0;
            mark[w] = (int32_t)nn; nodes[nn++] = w; me += add;
        }
    }
    *m_out = me;
    return nn;
}

/* Sizes pass of a batch: for graph g (seed seed + g), u ~ U(0,1), edge target
 * round(m_min * (m_max/m_min)^u), seed node drawn in proportion to degree.
 * n_out[g], m_out[g] receive the ball's sizes.  OpenMP over graphs. */
int gg_ego_batch_sizes(int64_t n_parent, const int64_t *rp, const int32_t *col, int64_t count, int64_t m_min,
                       int64_t m_max, int64_t n_max, uint64_t seed, int64_t *n_out, int64_t *m_out) {
    int bad = 0;
#pragma omp parallel reduction(|:bad)
    {
        int32_t *mark = (int32_t *)malloc((size_t)n_parent * sizeof(int32_t));
        int32_t *nodes = (int32_t *)malloc((size_t)n_max * sizeof(int32_t));
        if (!mark || !nodes) bad = 1;
        else {
            for (int64_t v = 0; v < n_parent; ++v) mark[v] = -1;
#pragma omp for schedule(dynamic, 4)
            for (int64_t g = 0; g < count; ++g) {
                uint64_t s = seed + (uint64_t)g;
                double u = gg_unit_from_seed(s);
                int64_t mt = (int64_t)llround((double)m_min * pow((double)m_max / (double)m_min, u));
                int32_t sn = gg_degree_proportional_node(n_parent, rp, s ^ 0x5EEDull);
                int64_t me = 0;
                int64_t nn = ego_ball(rp, col, sn, mt, n_max, mark, nodes, &me);
                for (int64_t q = 0; q < nn; ++q) mark[nodes[q]] = -1;
                n_out[g] = nn; m_out[g] = me;
            }
        }
        free(mark); free(nodes);
    }
    return bad ? -2 : 0;
}

/* Fill pass: the union CSR of the batch.  node_off[g] / nnz_off[g] are the
 * prefix sums of n_out and 2*m_out.  Graph g's nodes are numbered
 * node_off[g] + visit order; rows are sorted by neighbour id; types uniform
 * over L from seed + g.  OpenMP over graphs. */
int gg_ego_batch_fill(int64_t n_parent, const int64_t *rp, const int32_t *col, int64_t count, int64_t m_min,
                      int64_t m_max, int64_t n_max, uint64_t seed, int32_t L, const int64_t *node_off,
                      const int64_t *nnz_off, int64_t *u_rp, int32_t *u_col, uint8_t *u_ty) {
    int bad = 0;
#pragma omp parallel reduction(|:bad)
    {
        int32_t *mark = (int32_t *)malloc((size_t)n_parent * sizeof(int32_t));
        int32_t *nodes = (int32_t *)malloc((size_t)n_max * sizeof(int32_t));
        if (!mark || !nodes) bad = 1;
        else {
            for (int64_t v = 0; v < n_parent; ++v) mark[v] = -1;
#pragma omp for schedule(dynamic, 4)
            for (int64_t g = 0; g < count; ++g) {
                uint64_t s = seed + (uint64_t)g;
                double u = gg_unit_from_seed(s);
                int64_t mt = (int64_t)llround((double)m_min * pow((double)m_max / (double)m_min, u));
                int32_t sn = gg_degree_proportional_node(n_parent, rp, s ^ 0x5EEDull);
                int64_t me = 0;
                int64_t nn = ego_ball(rp, col, sn, mt, n_max, mark, nodes, &me);
                if (nn != node_off[g + 1] - node_off[g] || 2 * me != nnz_off[g + 1] - nnz_off[g]) { bad = 1; }
                else {
                    /* rows: local ids in visit order, neighbours inside the ball */
                    int64_t pos = nnz_off[g];
                    for (int64_t a = 0; a < nn; ++a) {
                        int32_t v = nodes[a];
                        u_rp[node_off[g] + a] = pos;
                        int64_t b0 = pos;
                        for (int64_t k = rp[v]; k < rp[v + 1]; ++k) {
                            int32_t b = mark[col[k]];
                            if (b >= 0) u_col[pos++] = (int32_t)(node_off[g] + b);
                        }
                        qsort(u_col + b0, (size_t)(pos - b0), sizeof(int32_t), cmp_i32);
                    }
                    gg_rng r; rng_seed(&r, s ^ 0x7E57ull);
                    for (int64_t a = 0; a < nn; ++a) u_ty[node_off[g] + a] = (uint8_t)rng_below(&r, (uint64_t)L);
                }
                for (int64_t q = 0; q < nn; ++q) mark[nodes[q]] = -1;
            }
        }
        free(mark); free(nodes);
    }
    return bad ? -2 : 0;
}

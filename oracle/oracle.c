/*
 * oracle.c -- plain, slow CPU reference for typed-graphlet counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library never
 * links it, shares no code, header, table or helper with it, and must fail
 * loudly rather than fall back to it.
 *
 * What it computes (Heterogeneous Graphlets, Rossi et al., TKDD 2020):
 *   Problem 1 (Sec. 4): for every edge (i,j) of an undirected simple graph
 *   with node types phi in [0,L), the counts of every typed 3- and 4-node
 *   graphlet orbit that contains the edge.  Problem 2 (Sec. 6): the global
 *   count of every typed {2,3,4}-node graphlet.
 *
 * Three independent routes, which the tests require to agree:
 *   oracle_paper   -- Alg. 1 (typed sets T, S_i, S_j, Cor. 1-3), Alg. 2
 *                     (path-based orbits g3, g6, g7), Alg. 3 (triangle-based
 *                     orbits g8, g10, g12), then Lemmas 1-4 (g4, g5, g9, g11)
 *                     for every type pair t <= t', then Sec. 4.4 / Sec. 6.
 *   oracle_table3  -- every orbit straight from its set-builder definition in
 *                     Table 3, enumerating node pairs (w_k, w_r) over the sets
 *                     T, S_i, S_j and I; no lemma is used.
 *   oracle_brute   -- every 3- and 4-node subset of V, its induced subgraph
 *                     classified by edge count and induced degrees; no typed
 *                     set is used.  Small graphs only.
 *
 * Alg. 5 (first two steps): oracle_weights gives the typed-graphlet weighted
 * graph W (instances of each typed graphlet containing an edge's endpoints)
 * and its degree D, by direct enumeration of the node sets that contain the
 * edge.  Small graphs only.
 *
 * Output layout (shared by specification with the GPU library, written
 * independently on each side):
 *   per edge (row stride S(L) = 2L + 10P, P = L(L+1)/2, int64 here):
 *     [t]                      g1: typed 3-paths, third node of type t
 *                              (= |S_i^t| + |S_j^t|, Cor. 3)
 *     [L + t]                  g2: typed triangles, |T_ij^t| (Cor. 1)
 *     [2L + (o-3)P + pair(t,t')]  orbit g_o, o = 3..12, the two other nodes
 *                              of types {t, t'}, t <= t'
 *     pair(t,t') = position of (t,t') in the lexicographic list of pairs
 *     t <= t'.  With k = 3 only the first 2L slots exist (stride 2L).
 *   global (int64): block 0 typed edges (C(L+1,2) multisets of 2 types),
 *     block 1 typed 3-paths, block 2 typed triangles (C(L+2,3) each), blocks
 *     3..8 typed 4-path, 4-star, 4-cycle, tailed-triangle, chordal-cycle,
 *     4-clique (C(L+3,4) each); inside a block, the position of the sorted
 *     type multiset in the lexicographic list of sorted multisets.
 *   Edge ids: edges {u,v}, u < v, numbered in lexicographic order of (u,v).
 *
 * Readings of the paper (where it is ambiguous), followed here:
 *   - S_i^t excludes j and S_j^t excludes i (Cor. 2's set equation; Alg. 1's
 *     shorthand Gamma_i^t \ T_ij^t would keep j).
 *   - T_ij^t is an intersection (Cor. 1), also where Sec. 4.2 writes a union.
 *   - The tie-break "w_r <= w_k" of Alg. 2/3 is taken as w_r < w_k on node
 *     ids (w_r = w_k is impossible in a simple graph).
 *   - A per-edge typed graphlet is keyed by the orbit and the unordered pair
 *     of the two other nodes' types: with phi_i, phi_j fixed, merging all
 *     orderings of the type vector (Sec. 4.5) leaves exactly that.
 *   - The 3-node graphlets are numbered g1/h1 = 3-path, g2/h2 = triangle.
 *   - Node types only; the edge types of Def. 1 are not used by Alg. 1-3.
 *
 * Plain C99 + optional OpenMP (the paper's own edge-parallel scheme, Sec.
 * 4.7: every edge is independent, rows written by edge id without locks).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_L 16

/* Planted mistakes for the pin tests: a test compiles a separate copy of
 * this file with -DORACLE_MUTANT=k (k = 1..10) and checks that the pins fail.
 * The default build (ORACLE_MUTANT undefined) contains none of them. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(k) (ORACLE_MUTANT == (k))

enum { OK = 0, ERR_ARG = 1, ERR_GRAPH = 2, ERR_MEM = 3, ERR_REMAINDER = 4 };

/* ------------------------------------------------------------- layout */

static int64_t binom(int64_t a, int64_t b) {
    if (b < 0 || a < b) return 0;
    int64_t r = 1;
    for (int64_t k = 1; k <= b; ++k) r = r * (a - b + k) / k;
    return r;
}

/* number of type pairs t <= t' */
static int64_t npairs(int L) { return (int64_t)L * (L + 1) / 2; }

/* position of (t,t'), t <= t', in the lexicographic list of such pairs,
 * found by walking the list */
static int64_t pair_index(int L, int t, int tp) {
    if (t > tp) { int x = t; t = tp; tp = x; }
    int64_t k = 0;
    for (int a = 0; a < L; ++a)
        for (int b = a; b < L; ++b, ++k)
            if (a == t && b == tp) return k;
    return -1;
}

/* position of the sorted multiset (types of length K) in the lexicographic
 * list of non-decreasing K-tuples over [0,L), found by walking the list */
static int64_t multiset_rank(int L, int K, const int *types_in) {
    int s[4];
    for (int a = 0; a < K; ++a) s[a] = types_in[a];
    for (int a = 0; a < K; ++a)           /* insertion sort */
        for (int b = a + 1; b < K; ++b)
            if (s[b] < s[a] && !MUTANT(6)) { int x = s[a]; s[a] = s[b]; s[b] = x; }
    int cur[4] = {0, 0, 0, 0};
    int64_t r = 0;
    for (;;) {
        int eq = 1;
        for (int a = 0; a < K; ++a) if (cur[a] != s[a]) { eq = 0; break; }
        if (eq) return r;
        ++r;
        int p = K - 1;                     /* next non-decreasing tuple */
        while (p >= 0 && cur[p] == L - 1) --p;
        if (p < 0) return -1;
        cur[p]++;
        for (int a = p + 1; a < K; ++a) cur[a] = cur[p];
    }
}

int64_t oracle_per_edge_slots(int L, int k) {
    return k == 3 ? 2 * (int64_t)L : 2 * (int64_t)L + 10 * npairs(L);
}

int64_t oracle_global_slots(int L, int k) {
    int64_t g = binom(L + 1, 2) + 2 * binom(L + 2, 3);
    if (k == 4) g += 6 * binom(L + 3, 4);
    return g;
}

/* offset of global block b (0 = edges, 1 = 3-path, 2 = triangle,
 * 3..8 = 4-path, 4-star, 4-cycle, tailed-triangle, chordal-cycle, 4-clique) */
static int64_t global_block_offset(int L, int b) {
    int64_t off = 0;
    for (int x = 0; x < b; ++x) off += (x == 0) ? binom(L + 1, 2) : (x <= 2 ? binom(L + 2, 3) : binom(L + 3, 4));
    return off;
}

int64_t oracle_pair_index(int L, int t, int tp) { return pair_index(L, t, tp); }
int64_t oracle_multiset_rank(int L, int K, const int32_t *types) {
    int s[4];
    for (int a = 0; a < K; ++a) s[a] = types[a];
    return multiset_rank(L, K, s);
}

/* adds v to slot `rank` of global block `block`; a rank outside the block
 * (which a correct rank function never returns) is reported, not written */
static int global_add(int64_t *acc, int L, int block, int64_t rank, int64_t v) {
    int64_t len = block == 0 ? binom(L + 1, 2) : (block <= 2 ? binom(L + 2, 3) : binom(L + 3, 4));
    if (rank < 0 || rank >= len) return 1;
    acc[global_block_offset(L, block) + rank] += v;
    return 0;
}

/* number of edges |E(H)| of each graphlet, h1..h8 (Table 3) */
static const int64_t EDGES_OF_GRAPHLET[9] = {1, 2, 3, 3, 3, 4, 4, 5, 6};

/* graphlet h of a 4-node orbit g (Sec. 4.4): h3 = g3+g4, h4 = g5, h5 = g6,
 * h6 = g7+g8+g9, h7 = g10+g11, h8 = g12 */
static int graphlet_of_orbit(int g) {
    switch (g) {
        case 3: case 4: return 3;
        case 5: return 4;
        case 6: return 5;
        case 7: case 8: case 9: return 6;
        case 10: case 11: return 7;
        case 12: return 8;
    }
    return -1;
}

/* --------------------------------------------------------------- graph */

typedef struct {
    int64_t n, m;
    const int64_t *rp;     /* row_ptr, as given */
    int32_t *adj;          /* private copy, every row sorted by id */
    const uint8_t *phi;
    int L;
    int64_t *eu, *ev;      /* edge id -> (u, v), u < v */
} graph_t;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int is_adjacent(const graph_t *G, int64_t u, int64_t v) {
    int64_t lo = G->rp[u], hi = G->rp[u + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (G->adj[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < G->rp[u + 1] && G->adj[lo] == v;
}

/* copies and sorts the rows, checks a simple symmetric graph, numbers the
 * edges */
static int graph_open(graph_t *G, int64_t n, const int64_t *rp, const int32_t *col,
                      const uint8_t *phi, int L) {
    memset(G, 0, sizeof(*G));
    if (n < 0 || L < 1 || L > OR_MAX_L) return ERR_ARG;
    int64_t nnz = rp[n];
    if (rp[0] != 0 || nnz < 0 || (nnz & 1)) return ERR_GRAPH;
    for (int64_t v = 0; v < n; ++v) if (rp[v + 1] < rp[v]) return ERR_GRAPH;
    for (int64_t v = 0; v < n; ++v) if (phi[v] >= L) return ERR_GRAPH;
    G->n = n; G->m = nnz / 2; G->rp = rp; G->phi = phi; G->L = L;
    G->adj = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    G->eu = (int64_t *)malloc((size_t)(G->m > 0 ? G->m : 1) * sizeof(int64_t));
    G->ev = (int64_t *)malloc((size_t)(G->m > 0 ? G->m : 1) * sizeof(int64_t));
    if (!G->adj || !G->eu || !G->ev) return ERR_MEM;
    memcpy(G->adj, col, (size_t)nnz * sizeof(int32_t));
    for (int64_t v = 0; v < n; ++v)
        qsort(G->adj + rp[v], (size_t)(rp[v + 1] - rp[v]), sizeof(int32_t), cmp_i32);
    int64_t e = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = rp[u]; k < rp[u + 1]; ++k) {
            int64_t v = G->adj[k];
            if (v < 0 || v >= n || v == u) return ERR_GRAPH;                   /* range, self-loop */
            if (k > rp[u] && G->adj[k - 1] == v) return ERR_GRAPH;              /* duplicate */
            if (!is_adjacent(G, v, u)) return ERR_GRAPH;                        /* asymmetric */
            if (u < v) {
                if (e >= G->m) return ERR_GRAPH;
                G->eu[e] = u; G->ev[e] = v; ++e;
            }
        }
    if (e != G->m) return ERR_GRAPH;
    return OK;
}

static void graph_close(graph_t *G) { free(G->adj); free(G->eu); free(G->ev); }

/* ----------------------------------------------- Alg. 1-3 + Lemmas 1-4 */

/* relation of a node to the current edge (the hash Psi of Table 1):
 * 0 = neither (the set I, or i/j themselves), 1 = S_i, 2 = S_j, 3 = T */
enum { REL_NONE = 0, REL_SI = 1, REL_SJ = 2, REL_T = 3 };

typedef struct {
    int64_t x3[OR_MAX_L * 2];                   /* g1, g2 by type */
    int64_t x4[13][OR_MAX_L * (OR_MAX_L + 1) / 2]; /* g3..g12 by type pair */
} counts_t;

/* Update (Alg. 4): the dense slot of (orbit g, types of w_k and w_r) plays
 * the role of the typed-graphlet hash; incrementing it is the update. */
static void update(counts_t *x, int L, int g, int tk, int tr) {
    x->x4[g][pair_index(L, tk, tr)] += 1;
}

/* Alg. 1 body for one edge (i,j); psi is an n-sized scratch of REL_NONE */
static void paper_edge(const graph_t *G, int64_t i, int64_t j, uint8_t *psi, counts_t *x) {
    const int L = G->L;
    const uint8_t *phi = G->phi;
    const int64_t *rp = G->rp;
    const int32_t *adj = G->adj;
    memset(x, 0, sizeof(*x));
    int64_t nT[OR_MAX_L] = {0}, nSi[OR_MAX_L] = {0}, nSj[OR_MAX_L] = {0};

    /* Psi: mark Gamma_i \ {j} as S_i, then Gamma_j \ {i}: a node already
     * marked becomes T (Cor. 1), otherwise S_j (Cor. 2). */
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) if (adj[k] != j) psi[adj[k]] = REL_SI;
    for (int64_t k = rp[j]; k < rp[j + 1]; ++k) {
        int64_t w = adj[k];
        if (w == i) continue;
        psi[w] = (psi[w] == REL_SI) ? REL_T : REL_SJ;
    }
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        int64_t w = adj[k];
        if (w == j) continue;
        if (psi[w] == REL_T) nT[phi[w]]++; else nSi[phi[w]]++;
    }
    for (int64_t k = rp[j]; k < rp[j + 1]; ++k) {
        int64_t w = adj[k];
        if (w == i) continue;
        if (psi[w] == REL_SJ) nSj[phi[w]]++;
    }
    /* 3-node typed graphlets: |S_ij^t| = |S_i^t| + |S_j^t| (Cor. 3), |T_ij^t| */
    if (MUTANT(3)) nSi[phi[j]]++;                 /* planted: j left inside S_i */
    for (int t = 0; t < L; ++t) {
        x->x3[t] = nSi[t] + nSj[t];
        x->x3[L + t] = nT[t];
    }

    /* Alg. 2: path-based orbits, first over S_i, then over S_j */
    for (int pass = 0; pass < 2; ++pass) {
        int64_t c = pass == 0 ? i : j;
        uint8_t own = pass == 0 ? REL_SI : REL_SJ;
        for (int64_t k = rp[c]; k < rp[c + 1]; ++k) {
            int64_t wk = adj[k];
            if (wk == i || wk == j || psi[wk] != own) continue;      /* w_k in S_c */
            for (int64_t q = rp[wk]; q < rp[wk + 1]; ++q) {
                int64_t wr = adj[q];
                if ((wr == i || wr == j) && !MUTANT(8)) continue;   /* Gamma_{w_k} \ {i,j} */
                if (psi[wr] == REL_NONE) {                          /* w_r not in Gamma_i u Gamma_j */
                    update(x, L, 3, phi[wk], phi[wr]);              /* 4-path, edge orbit */
                } else if (psi[wr] == own && (wr < wk || MUTANT(2))) {
                    update(x, L, 7, phi[wk], phi[wr]);              /* tailed-triangle, tail */
                } else if (pass == 1 && psi[wr] == REL_SI) {
                    update(x, L, 6, phi[wk], phi[wr]);              /* 4-cycle */
                }
            }
        }
    }

    /* Alg. 3: triangle-based orbits over T */
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        int64_t wk = adj[k];
        if (wk == j || psi[wk] != REL_T) continue;
        for (int64_t q = rp[wk]; q < rp[wk + 1]; ++q) {
            int64_t wr = adj[q];
            if (wr == i || wr == j) continue;
            if (psi[wr] == REL_T) {
                if (wr < wk) update(x, L, 12, phi[wk], phi[wr]);    /* 4-clique */
            } else if (psi[wr] == REL_SI || psi[wr] == REL_SJ) {
                update(x, L, MUTANT(5) ? 8 : 10, phi[wk], phi[wr]); /* chordal-cycle, edge */
            } else {
                update(x, L, 8, phi[wk], phi[wr]);                  /* tailed-triangle, centre */
            }
        }
    }

    /* Alg. 1, type-pair loop: the remaining orbits in O(1) per pair */
    for (int t = 0; t < L; ++t)
        for (int tp = t; tp < L; ++tp) {
            int64_t p = pair_index(L, t, tp);
            int64_t a = nSi[t], ap = nSi[tp];     /* |S_i^t|, |S_i^t'| */
            int64_t b = nSj[t], bp = nSj[tp];     /* |S_j^t|, |S_j^t'| */
            int64_t c = nT[t], cp = nT[tp];       /* |T_ij^t|, |T_ij^t'| */
            if (t == tp) {
                x->x4[4][p]  = a * b - (MUTANT(1) ? 0 : x->x4[6][p]);                /* Lemma 1 */
                x->x4[5][p]  = a * (a - 1) / (MUTANT(7) ? 1 : 2) + b * (b - 1) / 2
                               - x->x4[7][p];                                        /* Lemma 2 */
                x->x4[9][p]  = c * (a + b) - x->x4[10][p];                           /* Lemma 3 */
                x->x4[11][p] = c * (c - 1) / 2 - x->x4[12][p];                       /* Lemma 4 */
            } else {
                x->x4[4][p]  = a * bp + ap * b - x->x4[6][p];
                x->x4[5][p]  = a * ap + b * bp - x->x4[7][p];
                x->x4[9][p]  = MUTANT(4) ? c * (a + b) + cp * (ap + bp) - x->x4[10][p]
                                         : c * (ap + bp) + cp * (a + b) - x->x4[10][p];
                x->x4[11][p] = c * cp - x->x4[12][p];
            }
        }

    /* clear Psi */
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) psi[adj[k]] = REL_NONE;
    for (int64_t k = rp[j]; k < rp[j + 1]; ++k) psi[adj[k]] = REL_NONE;
}

/* ------------------------------------------------ Table 3, term by term */

/* Every 4-node orbit from its set-builder definition.  Pairs (w_k, w_r)
 * range over the typed sets; sets built by plain membership tests. */
static void table3_edge(const graph_t *G, int64_t i, int64_t j, counts_t *x) {
    const int L = G->L;
    const uint8_t *phi = G->phi;
    memset(x, 0, sizeof(*x));
    /* U = Gamma_i u Gamma_j \ {i,j}, each node with its set */
    int64_t du = (G->rp[i + 1] - G->rp[i]) + (G->rp[j + 1] - G->rp[j]);
    int64_t *U = (int64_t *)malloc((size_t)(du > 0 ? du : 1) * sizeof(int64_t));
    int *cls = (int *)malloc((size_t)(du > 0 ? du : 1) * sizeof(int));
    int64_t nu = 0;
    for (int64_t k = G->rp[i]; k < G->rp[i + 1]; ++k) {
        int64_t w = G->adj[k];
        if (w == j) continue;
        U[nu] = w; cls[nu] = is_adjacent(G, j, w) ? REL_T : REL_SI; ++nu;
    }
    for (int64_t k = G->rp[j]; k < G->rp[j + 1]; ++k) {
        int64_t w = G->adj[k];
        if (w == i || is_adjacent(G, i, w)) continue;
        U[nu] = w; cls[nu] = REL_SJ; ++nu;
    }
    for (int64_t a = 0; a < nu; ++a) {
        int t = phi[U[a]];
        if (cls[a] == REL_T) x->x3[L + t]++; else x->x3[t]++;
    }
    /* pairs inside U: orbits 4,5,6,7,9,10,11,12 */
    for (int64_t a = 0; a < nu; ++a)
        for (int64_t b = 0; b < nu; ++b) {
            if (a == b) continue;
            int64_t wk = U[a], wr = U[b];
            int ck = cls[a], cr = cls[b];
            int e = is_adjacent(G, wk, wr);
            int tk = phi[wk], tr = phi[wr];
            /* ordered pairs (a,b) and (b,a) describe the same 4-node set;
             * conditions that are symmetric in (w_k, w_r) are counted on
             * a < b only */
            if (a < b) {
                if (((ck == REL_SI && cr == REL_SI) || (ck == REL_SJ && cr == REL_SJ)) && !e) update(x, L, 5, tk, tr);
                if (((ck == REL_SI && cr == REL_SI) || (ck == REL_SJ && cr == REL_SJ)) && e) update(x, L, 7, tk, tr);
                if (ck == REL_T && cr == REL_T && !e) update(x, L, 11, tk, tr);
                if (ck == REL_T && cr == REL_T && e) update(x, L, 12, tk, tr);
            }
            if (ck == REL_SJ && cr == REL_SI && !e) update(x, L, 4, tk, tr);
            if (ck == REL_SJ && cr == REL_SI && e) update(x, L, 6, tk, tr);
            if (ck == REL_T && (cr == REL_SI || cr == REL_SJ) && !e) update(x, L, 9, tk, tr);
            if (ck == REL_T && (cr == REL_SI || cr == REL_SJ) && e) update(x, L, 10, tk, tr);
        }
    /* pairs with w_r in I (adjacent to w_k, not to i or j): orbits 3, 8 */
    for (int64_t a = 0; a < nu; ++a) {
        int64_t wk = U[a];
        for (int64_t q = G->rp[wk]; q < G->rp[wk + 1]; ++q) {
            int64_t wr = G->adj[q];
            if (wr == i || wr == j || is_adjacent(G, i, wr) || is_adjacent(G, j, wr)) continue;
            if (cls[a] == REL_SI || cls[a] == REL_SJ) update(x, L, 3, phi[wk], phi[wr]);
            else update(x, L, 8, phi[wk], phi[wr]);
        }
    }
    free(U); free(cls);
}

/* ----------------------------------------------------------- emit rows */

/* writes the edge's counts into row (if not NULL) and adds them to the
 * global accumulator (if not NULL); returns 1 if a count is negative */
static int emit_row(const graph_t *G, int k, const counts_t *x, int64_t e, int64_t *row,
                    int64_t *gacc) {
    const int L = G->L;
    int64_t P = npairs(L);
    int64_t i = G->eu[e], j = G->ev[e];
    int pi = G->phi[i], pj = G->phi[j];
    int bad = 0;
    for (int t = 0; t < L; ++t) {
        if (row) { row[t] = x->x3[t]; row[L + t] = x->x3[L + t]; }
        if (x->x3[t] < 0 || x->x3[L + t] < 0) bad = 1;
        if (gacc) {
            int ty[3] = {pi, pj, t};
            bad |= global_add(gacc, L, 1, multiset_rank(L, 3, ty), x->x3[t]);
            bad |= global_add(gacc, L, 2, multiset_rank(L, 3, ty), x->x3[L + t]);
        }
    }
    if (gacc) { int ty[2] = {pi, pj}; bad |= global_add(gacc, L, 0, multiset_rank(L, 2, ty), 1); }
    if (k == 4)
        for (int g = 3; g <= 12; ++g)
            for (int t = 0; t < L; ++t)
                for (int tp = t; tp < L; ++tp) {
                    int64_t p = pair_index(L, t, tp);
                    int64_t v = x->x4[g][p];
                    if (v < 0) bad = 1;
                    if (row) row[2 * L + (g - 3) * P + p] = v;
                    if (gacc) {
                        int ty[4] = {pi, pj, t, tp};
                        bad |= global_add(gacc, L, graphlet_of_orbit(g), multiset_rank(L, 4, ty), v);
                    }
                }
    return bad;
}

/* Global counts (Sec. 6): C_H = (1/|E(H)|) * sum over edges; the sums must
 * divide exactly. */
static int finish_global(int L, int k, int64_t *gacc, int64_t *global_out) {
    int nb = k == 4 ? 9 : 3;
    for (int b = 0; b < nb; ++b) {
        int64_t off = global_block_offset(L, b);
        int64_t len = b == 0 ? binom(L + 1, 2) : (b <= 2 ? binom(L + 2, 3) : binom(L + 3, 4));
        for (int64_t s = 0; s < len; ++s) {
            if (gacc[off + s] % EDGES_OF_GRAPHLET[b] != 0) return ERR_REMAINDER;
            global_out[off + s] = gacc[off + s] / EDGES_OF_GRAPHLET[b];
        }
    }
    return OK;
}

typedef void (*edge_fn)(const graph_t *, int64_t, int64_t, uint8_t *, counts_t *);

static void table3_adapter(const graph_t *G, int64_t i, int64_t j, uint8_t *psi, counts_t *x) {
    (void)psi;
    table3_edge(G, i, j, x);
}

static int run_edges(const graph_t *G, int k, edge_fn fn, int64_t *per_edge, int64_t *global_out,
                     const int64_t *edge_ids, int64_t n_ids, int nthreads) {
    const int L = G->L;
    const int64_t Gs = oracle_global_slots(L, k), S = oracle_per_edge_slots(L, k);
    int64_t *gacc = global_out ? (int64_t *)calloc((size_t)Gs, sizeof(int64_t)) : NULL;
    if (global_out && !gacc) return ERR_MEM;
    int64_t count = edge_ids ? n_ids : G->m;
    int bad = 0, memfail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel reduction(|:bad, memfail)
    {
        uint8_t *psi = (uint8_t *)calloc((size_t)(G->n > 0 ? G->n : 1), 1);
        int64_t *lacc = gacc ? (int64_t *)calloc((size_t)Gs, sizeof(int64_t)) : NULL;
        counts_t *x = (counts_t *)malloc(sizeof(counts_t));
        if (!psi || !x || (gacc && !lacc)) {
            memfail = 1;
        } else {
            /* edges are independent: row q is written by one thread only */
#pragma omp for schedule(dynamic, 64)
            for (int64_t q = 0; q < count; ++q) {
                int64_t e = edge_ids ? edge_ids[q] : q;
                fn(G, G->eu[e], G->ev[e], psi, x);
                bad |= emit_row(G, k, x, e, per_edge ? per_edge + q * S : NULL, lacc);
            }
#pragma omp critical
            if (gacc) for (int64_t s = 0; s < Gs; ++s) gacc[s] += lacc[s];
        }
        free(psi); free(lacc); free(x);
    }
    int rc = OK;
    if (memfail) rc = ERR_MEM;
    else if (bad) rc = ERR_REMAINDER;
    else if (global_out && !edge_ids) rc = finish_global(L, k, gacc, global_out);
    else if (global_out) memcpy(global_out, gacc, (size_t)Gs * sizeof(int64_t)); /* raw sums of a sample */
    free(gacc);
    return rc;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Alg. 1-3 + Lemmas 1-4 on every edge.  per_edge_out: int64 [m][S] or NULL;
 * global_out: int64 [G] or NULL.  nthreads <= 0: OpenMP default. */
int oracle_paper(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                 int k, int64_t *per_edge_out, int64_t *global_out, int nthreads) {
    if (k != 3 && k != 4) return ERR_ARG;
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc == OK) rc = run_edges(&G, k, paper_edge, per_edge_out, global_out, NULL, 0, nthreads);
    graph_close(&G);
    return rc;
}

/* Alg. 1-3 + Lemmas on the listed edge ids only; row q of per_edge_out is
 * edge edge_ids[q].  global_out (optional) receives the raw per-edge sums
 * of the sample (not divided by |E(H)|). */
int oracle_paper_edges(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types,
                       int L, int k, const int64_t *edge_ids, int64_t n_ids, int64_t *per_edge_out,
                       int64_t *sample_sums, int nthreads) {
    if (k != 3 && k != 4) return ERR_ARG;
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc == OK)
        for (int64_t q = 0; q < n_ids; ++q)
            if (edge_ids[q] < 0 || edge_ids[q] >= G.m) { rc = ERR_ARG; break; }
    if (rc == OK) rc = run_edges(&G, k, paper_edge, per_edge_out, sample_sums, edge_ids, n_ids, nthreads);
    graph_close(&G);
    return rc;
}

/* Table 3 definitions on every edge (k = 4 layout). */
int oracle_table3(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                  int64_t *per_edge_out, int64_t *global_out) {
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc == OK) rc = run_edges(&G, 4, table3_adapter, per_edge_out, global_out, NULL, 0, 1);
    graph_close(&G);
    return rc;
}

/* Edge list in edge-id order: src[e] < dst[e]. */
int oracle_edges(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                 int64_t *src, int64_t *dst) {
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc == OK) {
        memcpy(src, G.eu, (size_t)G.m * sizeof(int64_t));
        memcpy(dst, G.ev, (size_t)G.m * sizeof(int64_t));
    }
    graph_close(&G);
    return rc;
}

/* Validation only: OK or ERR_GRAPH / ERR_ARG. */
int oracle_validate(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L) {
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    graph_close(&G);
    return rc;
}

/* ---------------------------------------------------------- brute force */

/* edge id of {u,v} by binary search over the sorted edge list */
static int64_t edge_id_of(const graph_t *G, int64_t u, int64_t v) {
    if (u > v) { int64_t x = u; u = v; v = x; }
    int64_t lo = 0, hi = G->m;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (G->eu[mid] < u || (G->eu[mid] == u && G->ev[mid] < v)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* All 3- and 4-node subsets.  For a connected induced subgraph: the
 * graphlet from its edge count and induced degrees, the orbit of each of
 * its edges from the induced degrees of the edge's endpoints; the edge's
 * slot is keyed by the types of the other nodes.  Global: each connected
 * subset counted once under its sorted type multiset. */
int oracle_brute(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                 int64_t *per_edge_out, int64_t *global_out) {
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc != OK) { graph_close(&G); return rc; }
    const int64_t S = oracle_per_edge_slots(L, 4), P = npairs(L);
    int64_t Gs = oracle_global_slots(L, 4);
    if (per_edge_out) memset(per_edge_out, 0, (size_t)(G.m * S) * sizeof(int64_t));
    if (global_out) memset(global_out, 0, (size_t)Gs * sizeof(int64_t));
    for (int64_t e = 0; e < G.m; ++e) {                       /* 2-node graphlets */
        int ty[2] = {types[G.eu[e]], types[G.ev[e]]};
        if (global_out && global_add(global_out, L, 0, multiset_rank(L, 2, ty), 1)) rc = ERR_REMAINDER;
    }
    /* 3-node subsets */
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b)
            for (int64_t c = b + 1; c < n; ++c) {
                int64_t v[3] = {a, b, c};
                int ne = 0, A[3][3] = {{0}};
                for (int x = 0; x < 3; ++x)
                    for (int y = x + 1; y < 3; ++y)
                        if (is_adjacent(&G, v[x], v[y])) { A[x][y] = A[y][x] = 1; ++ne; }
                if (ne < 2) continue;
                int g = ne == 2 ? 1 : 2;             /* 3-path or triangle */
                int ty[3] = {types[a], types[b], types[c]};
                if (global_out && global_add(global_out, L, g, multiset_rank(L, 3, ty), 1)) rc = ERR_REMAINDER;
                if (per_edge_out)
                    for (int x = 0; x < 3; ++x)
                        for (int y = x + 1; y < 3; ++y) {
                            if (!A[x][y]) continue;
                            int z = 3 - x - y;
                            int64_t e = edge_id_of(&G, v[x], v[y]);
                            per_edge_out[e * S + (g == 1 ? 0 : L) + types[v[z]]] += 1;
                        }
            }
    /* 4-node subsets */
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b)
            for (int64_t c = b + 1; c < n; ++c)
                for (int64_t d = c + 1; d < n; ++d) {
                    int64_t v[4] = {a, b, c, d};
                    int ne = 0, A[4][4] = {{0}}, deg[4] = {0};
                    for (int x = 0; x < 4; ++x)
                        for (int y = x + 1; y < 4; ++y)
                            if (is_adjacent(&G, v[x], v[y])) {
                                A[x][y] = A[y][x] = 1; ++ne; deg[x]++; deg[y]++;
                            }
                    if (ne < 3) continue;
                    int maxd = 0, mind = 4;
                    for (int x = 0; x < 4; ++x) { if (deg[x] > maxd) maxd = deg[x]; if (deg[x] < mind) mind = deg[x]; }
                    if (mind == 0) continue;                 /* triangle + isolated node */
                    int h;
                    if (ne == 3) h = maxd == 3 ? 4 : 3;       /* 4-star : 4-path */
                    else if (ne == 4) h = maxd == 3 ? 6 : 5;  /* tailed-triangle : 4-cycle */
                    else if (ne == 5) h = 7;                  /* chordal-cycle */
                    else h = 8;                               /* 4-clique */
                    int ty4[4] = {types[a], types[b], types[c], types[d]};
                    if (global_out && global_add(global_out, L, h, multiset_rank(L, 4, ty4), 1)) rc = ERR_REMAINDER;
                    if (!per_edge_out) continue;
                    for (int x = 0; x < 4; ++x)
                        for (int y = x + 1; y < 4; ++y) {
                            if (!A[x][y]) continue;
                            int dx = deg[x] < deg[y] ? deg[x] : deg[y];
                            int dy = deg[x] < deg[y] ? deg[y] : deg[x];
                            int g = 0;
                            switch (h) {
                                case 3: g = (dx == 1) ? 3 : 4; break;          /* end {1,2} / centre {2,2} */
                                case 4: g = 5; break;
                                case 5: g = 6; break;
                                case 6: g = (dx == 1) ? 7 : (dy == 2 ? 8 : 9); break; /* tail {1,3}, {2,2}, {2,3} */
                                case 7: g = (dx == 3) ? 11 : 10; break;        /* chord {3,3} / outer {2,3} */
                                case 8: g = 12; break;
                            }
                            int o[2], no = 0;
                            for (int z = 0; z < 4; ++z) if (z != x && z != y) o[no++] = z;
                            int64_t e = edge_id_of(&G, v[x], v[y]);
                            per_edge_out[e * S + 2 * L + (g - 3) * P + pair_index(L, types[v[o[0]]], types[v[o[1]]])] += 1;
                        }
                }
    graph_close(&G);
    return rc;
}

/* ------------------------------------ typed-graphlet weighted graph */

/* Alg. 5, first two steps, for every typed {2,3,4}-node graphlet H at once:
 * W[e][s] = the number of instances of H (global slot s) that contain both
 * endpoints of edge e, D[v][s] = sum over the edges e at v of W[e][s].  An
 * instance is a connected induced subgraph; since {i,j} is an edge it is an
 * edge of every instance counted.  Direct enumeration: the edge itself, every
 * third node x, every pair of other nodes x < y, each set classified by its
 * induced edge count and degrees.  Small graphs only (m n^2 / 2 sets).
 * w_out: int64 [m][G(L)]; d_out: int64 [n][G(L)] or NULL. */
int oracle_weights(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                   int64_t *w_out, int64_t *d_out) {
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc != OK) { graph_close(&G); return rc; }
    const int64_t Gs = oracle_global_slots(L, 4);
    memset(w_out, 0, (size_t)(G.m * Gs) * sizeof(int64_t));
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(|:bad)
    for (int64_t e = 0; e < G.m; ++e) {
        const int64_t i = G.eu[e], j = G.ev[e];
        int64_t *w = w_out + e * Gs;
        int t2[2] = {types[i], types[j]};
        bad |= global_add(w, L, 0, multiset_rank(L, 2, t2), 1);
        for (int64_t x = 0; x < n; ++x) {
            if (x == i || x == j) continue;
            const int ne = 1 + is_adjacent(&G, x, i) + is_adjacent(&G, x, j);
            if (ne < 2) continue;                                 /* x isolated from the edge */
            int t3[3] = {types[i], types[j], types[x]};
            bad |= global_add(w, L, ne == 2 ? 1 : 2, multiset_rank(L, 3, t3), 1);
        }
        for (int64_t x = 0; x < n; ++x) {
            if (x == i || x == j) continue;
            for (int64_t y = x + 1; y < n; ++y) {
                if (y == i || y == j) continue;
                const int64_t v[4] = {i, j, x, y};
                int ne = 0, deg[4] = {0, 0, 0, 0};
                for (int a = 0; a < 4; ++a)
                    for (int b = a + 1; b < 4; ++b)
                        if (is_adjacent(&G, v[a], v[b])) { ++ne; deg[a]++; deg[b]++; }
                int mind = 4, maxd = 0;
                for (int a = 0; a < 4; ++a) {
                    if (deg[a] < mind) mind = deg[a];
                    if (deg[a] > maxd) maxd = deg[a];
                }
                if (ne < 3 || mind == 0) continue;                /* not connected */
                int h;
                if (ne == 3) h = maxd == 3 ? 4 : 3;               /* 4-star : 4-path */
                else if (ne == 4) h = (maxd == 3 && !MUTANT(9)) ? 6 : 5;   /* tailed-triangle : 4-cycle */
                else h = ne == 5 ? 7 : 8;                         /* chordal-cycle : 4-clique */
                int t4[4] = {types[i], types[j], types[x], types[y]};
                bad |= global_add(w, L, h, multiset_rank(L, 4, t4), 1);
            }
        }
    }
    if (d_out) {
        memset(d_out, 0, (size_t)(n * Gs) * sizeof(int64_t));
        for (int64_t e = 0; e < G.m; ++e)
            for (int64_t s = 0; s < Gs; ++s) {
                d_out[G.eu[e] * Gs + s] += w_out[e * Gs + s];
                if (!MUTANT(10)) d_out[G.ev[e] * Gs + s] += w_out[e * Gs + s];
            }
    }
    graph_close(&G);
    return bad ? ERR_REMAINDER : OK;
}

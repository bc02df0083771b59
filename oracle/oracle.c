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
 * Sec. 5 (Def. 8): oracle_position_aware gives position-aware typed
 * counts per edge and globally, by visiting every connected node set that
 * contains an edge; oracle_position_aware_brute gives the global counts from
 * all node sets of the graph.
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
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_L 16

/* Planted mistakes for the pin tests: a test compiles a separate copy of
 * this file with -DORACLE_MUTANT=k (k = 1..16) and checks that the pins fail.
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

static double now_seconds(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* edge_seconds (optional, listed edges only): the time the thread spent on
 * each edge, for the benchmark's sampled timing; no effect on the counts. */
static int run_edges(const graph_t *G, int k, edge_fn fn, int64_t *per_edge, int64_t *global_out,
                     const int64_t *edge_ids, int64_t n_ids, int nthreads, double *edge_seconds) {
    const int L = G->L;
    const int64_t Gs = oracle_global_slots(L, k), S = oracle_per_edge_slots(L, k);
    int64_t *gacc = global_out ? (int64_t *)calloc((size_t)Gs, sizeof(int64_t)) : NULL;
    if (global_out && !gacc) return ERR_MEM;
    int64_t count = edge_ids ? n_ids : G->m;
    int bad = 0, memfail = 0;
#ifdef _OPENMP
    /* a per-call thread count that leaves the process default unchanged */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
#endif
#pragma omp parallel num_threads(nt) reduction(|:bad, memfail)
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
                double t0 = edge_seconds ? now_seconds() : 0.0;
                fn(G, G->eu[e], G->ev[e], psi, x);
                bad |= emit_row(G, k, x, e, per_edge ? per_edge + q * S : NULL, lacc);
                if (edge_seconds) edge_seconds[q] = now_seconds() - t0;
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
    if (rc == OK) rc = run_edges(&G, k, paper_edge, per_edge_out, global_out, NULL, 0, nthreads, NULL);
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
    if (rc == OK) rc = run_edges(&G, k, paper_edge, per_edge_out, sample_sums, edge_ids, n_ids, nthreads, NULL);
    graph_close(&G);
    return rc;
}

/* Table 3 definitions on every edge (k = 4 layout). */
/* An opened graph kept across calls: the validated, row-sorted copy that
 * every route above builds first (graph_open), so that a caller timing the
 * per-edge work of several edge samples opens the graph once.  The caller's
 * row_ptr and types arrays must outlive the handle (they are not copied). */
void *oracle_graph_open(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                        int32_t *status) {
    graph_t *G = (graph_t *)malloc(sizeof(graph_t));
    int rc = G ? graph_open(G, n, row_ptr, col, types, L) : ERR_MEM;
    if (status) *status = rc;
    if (rc != OK) {
        if (G) { graph_close(G); free(G); }
        return NULL;
    }
    return G;
}

void oracle_graph_close(void *h) {
    if (!h) return;
    graph_close((graph_t *)h);
    free(h);
}

/* oracle_paper_edges on an opened graph; edge_seconds (optional) receives
 * the time spent on each listed edge by the thread that counted it. */
int oracle_graph_paper_edges(void *h, int k, const int64_t *edge_ids, int64_t n_ids, int64_t *per_edge_out,
                             int64_t *sample_sums, double *edge_seconds, int nthreads) {
    const graph_t *G = (const graph_t *)h;
    if (!G || (k != 3 && k != 4) || n_ids < 0) return ERR_ARG;
    for (int64_t q = 0; q < n_ids; ++q)
        if (edge_ids[q] < 0 || edge_ids[q] >= G->m) return ERR_ARG;
    return run_edges(G, k, paper_edge, per_edge_out, sample_sums, edge_ids, n_ids, nthreads, edge_seconds);
}

int oracle_table3(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                  int64_t *per_edge_out, int64_t *global_out) {
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc == OK) rc = run_edges(&G, 4, table3_adapter, per_edge_out, global_out, NULL, 0, 1, NULL);
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

/* ------------------------------- position-aware typed graphlets (Sec. 5) */

/* Def. 8: two typed instances of one shape are the same position-aware
 * typed graphlet when an isomorphism between them maps every node onto a
 * node of the same type.  For a shape with its nodes numbered, a
 * position-aware typed graphlet is therefore a labelling (types of nodes
 * 0..k-1) up to the shape's automorphisms; its class is represented by the
 * lexicographically smallest labelling in it, and the classes of a shape
 * are numbered in the lexicographic order of those representatives.
 *
 * Numbered shapes (global blocks as for typed graphlets):
 *   0 edge 0-1; 1 3-path, 0 the centre; 2 triangle; 3 4-path 0-1-2-3;
 *   4 4-star, 0 the centre; 5 4-cycle 0-1-2-3-0; 6 tailed triangle, 0 the
 *   degree-3 node, 1 the tail, 2-3 the rest of the triangle; 7 chordal cycle,
 *   0-1 the chord; 8 4-clique.
 *
 * Per-edge rows, edge e = {lo, hi} (lo < hi, caller ids); "side" 0 = lo,
 * 1 = hi; ordered type pairs (x, y) at x*L + y; unordered pairs as
 * pair_index; blocks in this order:
 *   O1  3-path      [side of the centre][type of the third node]     2L
 *   O2  triangle    [type of the third node]                          L
 *   O3  4-path, end edge  [side of the inner endpoint][type of its other
 *                   neighbour][type of the far end]                   2L^2
 *   O4  4-path, centre edge [type of lo's other neighbour][of hi's]   L^2
 *   O5  4-star      [side of the centre][pair of the other leaves]    2P
 *   O6  4-cycle     [type of lo's other neighbour][of hi's]           L^2
 *   O7  tailed triangle, tail edge [side of the degree-3 node][pair of
 *                   the other triangle nodes]                         2P
 *   O8  tailed triangle, edge opposite the degree-3 node [type of the
 *                   degree-3 node][type of the tail]                  L^2
 *   O9  tailed triangle, triangle edge at the degree-3 node [side of the
 *                   degree-3 node][type of the third triangle node][type
 *                   of the tail]                                      2L^2
 *   O10 chordal cycle, outer edge [side of the degree-3 endpoint][type of
 *                   the other degree-3 node][type of the other
 *                   degree-2 node]                                    2L^2
 *   O11 chordal cycle, chord [pair of the degree-2 nodes]             P
 *   O12 4-clique    [pair of the other nodes]                         P
 * The per-edge keys fix which endpoint holds each position; merging the
 * two sides when phi_lo = phi_hi gives the instances of a (position-aware
 * typed graphlet, edge orbit).  Global counts: Sec. 6 applied per class. */

#define PA_MAX_CODES 4096               /* 8^4 labellings of a 4-node shape: L <= 8 here */

static const int PA_K[9] = {2, 3, 3, 4, 4, 4, 4, 4, 4};
static const int PA_EDGES[9][6][2] = {
    {{0, 1}},
    {{0, 1}, {0, 2}},
    {{0, 1}, {0, 2}, {1, 2}},
    {{0, 1}, {1, 2}, {2, 3}},
    {{0, 1}, {0, 2}, {0, 3}},
    {{0, 1}, {1, 2}, {2, 3}, {3, 0}},
    {{0, 1}, {0, 2}, {0, 3}, {2, 3}},
    {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}},
    {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}},
};
static const int PA_NEDGES[9] = {1, 2, 3, 3, 3, 4, 4, 5, 6};

static void pa_adjacency(int b, int A[4][4]) {
    memset(A, 0, sizeof(int) * 16);
    for (int x = 0; x < PA_NEDGES[b]; ++x) {
        A[PA_EDGES[b][x][0]][PA_EDGES[b][x][1]] = 1;
        A[PA_EDGES[b][x][1]][PA_EDGES[b][x][0]] = 1;
    }
}

/* all permutations of k <= 4 nodes, as arrays; returns their number */
static int all_perms(int k, int perms[24][4]) {
    int np = 0, p[4];
    for (p[0] = 0; p[0] < k; ++p[0])
        for (p[1] = 0; p[1] < k; ++p[1])
            for (p[2] = 0; p[2] < (k > 2 ? k : 1); ++p[2])
                for (p[3] = 0; p[3] < (k > 3 ? k : 1); ++p[3]) {
                    int used = 0, ok = 1;
                    for (int a = 0; a < k; ++a) {
                        if (used & (1 << p[a])) ok = 0;
                        used |= 1 << p[a];
                    }
                    if (!ok) continue;
                    for (int a = 0; a < 4; ++a) perms[np][a] = a < k ? p[a] : 0;
                    ++np;
                }
    return np;
}

/* automorphisms of numbered shape b: permutations keeping its adjacency */
static int pa_automorphisms(int b, int aut[24][4]) {
    int A[4][4], perms[24][4], k = PA_K[b], na = 0;
    pa_adjacency(b, A);
    int np = all_perms(k, perms);
    for (int x = 0; x < np; ++x) {
        int ok = 1;
        for (int u = 0; u < k && ok; ++u)
            for (int v = 0; v < k && ok; ++v)
                if (A[u][v] != A[perms[x][u]][perms[x][v]]) ok = 0;
        if (ok) { memcpy(aut[na], perms[x], sizeof(perms[x])); ++na; }
    }
    return na;
}

static int pa_code(int L, int k, const int *lab) {
    int c = 0;
    for (int a = 0; a < k; ++a) c = c * L + lab[a];
    return c;
}

/* class table of shape b: cls[code] = rank of the labelling's class;
 * returns the number of classes */
static int pa_class_table(int L, int b, int32_t *cls) {
    int aut[24][4];
    const int na = pa_automorphisms(b, aut), k = PA_K[b];
    int ncodes = 1;
    for (int a = 0; a < k; ++a) ncodes *= L;
    int nclass = 0;
    /* codes in increasing order are labellings in lexicographic order, so
     * a canonical labelling is met before every other member of its class */
    for (int code = 0; code < ncodes; ++code) {
        int lab[4], x = code;
        for (int a = k - 1; a >= 0; --a) { lab[a] = x % L; x /= L; }
        int best = code;
        for (int g = 0; g < na; ++g) {
            int img[4];
            for (int a = 0; a < k; ++a) img[a] = lab[aut[g][a]];
            int c = pa_code(L, k, img);
            if (c < best) best = c;
        }
        cls[code] = best == code ? nclass++ : cls[best];
    }
    return nclass;
}

static int64_t pa_block_size(int L, int b) {
    int32_t cls[PA_MAX_CODES];
    return pa_class_table(L, b, cls);
}

int64_t oracle_pa_per_edge_slots(int L) { return 3 * (int64_t)L + 9 * (int64_t)L * L + 6 * npairs(L); }

int64_t oracle_pa_block_size(int L, int b) {
    if (L < 1 || L > 8 || b < 0 || b > 8) return -1;
    return pa_block_size(L, b);
}

int64_t oracle_pa_global_slots(int L) {
    if (L < 1 || L > 8) return -1;
    int64_t s = 0;
    for (int b = 0; b < 9; ++b) s += pa_block_size(L, b);
    return s;
}

/* class rank of a labelling of numbered shape b (-1 on a bad argument) */
int64_t oracle_pa_class(int L, int b, const int32_t *lab) {
    if (L < 1 || L > 8 || b < 0 || b > 8) return -1;
    int32_t cls[PA_MAX_CODES];
    pa_class_table(L, b, cls);
    int l[4];
    for (int a = 0; a < PA_K[b]; ++a) {
        if (lab[a] < 0 || lab[a] >= L) return -1;
        l[a] = lab[a];
    }
    return cls[pa_code(L, PA_K[b], l)];
}

/* per-edge block offsets O1..O12 (index 1..12) */
static void pa_offsets(int L, int64_t off[13]) {
    const int64_t P = npairs(L), LL = (int64_t)L * L;
    const int64_t size[13] = {0, 2 * L, L, 2 * LL, LL, 2 * P, LL, 2 * P, LL, 2 * LL, 2 * LL, P, P};
    off[0] = 0;
    int64_t s = 0;
    for (int o = 1; o <= 12; ++o) { off[o] = s; s += size[o]; }
}

typedef struct {
    int L;
    int32_t cls[9][PA_MAX_CODES];
    int64_t block_off[9];
    int64_t off[13];
    int perms[24][4];                   /* all permutations of 4 nodes */
    int nperms;
    int shape[9][4][4];                 /* adjacency of each numbered shape */
} pa_tables_t;

static void pa_tables(int L, pa_tables_t *T) {
    T->L = L;
    int64_t s = 0;
    for (int b = 0; b < 9; ++b) {
        T->block_off[b] = s;
        s += pa_class_table(L, b, T->cls[b]);
        pa_adjacency(b, T->shape[b]);
    }
    pa_offsets(L, T->off);
    T->nperms = all_perms(4, T->perms);
}

/* global slot of the instance whose node x sits at numbered position
 * pos[x] of shape b (types phi of the instance's nodes v[]) */
static int64_t pa_global_slot(const pa_tables_t *T, int b, int k, const int64_t *v, const int *pos,
                              const uint8_t *phi) {
    int lab[4];
    for (int x = 0; x < k; ++x) lab[pos[x]] = phi[v[x]];
    return T->block_off[b] + T->cls[b][pa_code(T->L, PA_K[b], lab)];
}

/* positions of the k nodes of an instance in numbered shape b: the first
 * permutation (in the order all_perms lists them) that maps the instance's
 * adjacency onto the shape's; 0 if there is none */
static int pa_positions(const pa_tables_t *T, int b, int k, int A[4][4], int *pos) {
    int small[24][4], nsmall = 0;
    const int (*perms)[4] = T->perms;
    int np = T->nperms;
    if (k < 4) {                                     /* permutations of the first k nodes */
        nsmall = all_perms(k, small);
        perms = (const int (*)[4])small;
        np = nsmall;
    }
    const int (*S)[4] = T->shape[b];
    for (int x = 0; x < np; ++x) {
        int ok = 1;
        for (int u = 0; u < k && ok; ++u)
            for (int w = u + 1; w < k && ok; ++w)
                if (A[u][w] != S[perms[x][u]][perms[x][w]]) ok = 0;
        if (ok) { for (int u = 0; u < k; ++u) pos[u] = perms[x][u]; return 1; }
    }
    return 0;
}

/* Position-aware per-edge rows and global counts.  Every node set that
 * contains the edge and induces a connected subgraph is visited once: third
 * nodes x in U (the neighbours of lo or hi), and pairs {x, y} with x in U and
 * y in U after x or y a neighbour of x outside U.  The edge's slot follows from the induced
 * degrees (layout above); the instance's class from a numbering of its
 * nodes onto the shape.  Global: raw sums over edges divided by |E(H)|
 * (Sec. 6).  per_edge_out: int64 [m][S_pa] or NULL; global_out: int64
 * [G_pa] or NULL. */
int oracle_position_aware(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                          int64_t *per_edge_out, int64_t *global_out) {
    if (L < 1 || L > 8) return ERR_ARG;
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc != OK) { graph_close(&G); return rc; }
    pa_tables_t *T = (pa_tables_t *)malloc(sizeof(pa_tables_t));
    if (!T) { graph_close(&G); return ERR_MEM; }
    pa_tables(L, T);
    const int64_t S = oracle_pa_per_edge_slots(L), Gs = oracle_pa_global_slots(L), P = npairs(L);
    int64_t *raw = (int64_t *)calloc((size_t)Gs, sizeof(int64_t));
    if (!raw) { free(T); graph_close(&G); return ERR_MEM; }
    if (per_edge_out) memset(per_edge_out, 0, (size_t)(G.m * S) * sizeof(int64_t));
    const int64_t *O = T->off;
    int bad = 0, memfail = 0;
#pragma omp parallel reduction(|:bad, memfail)
    {
        int64_t *acc = (int64_t *)calloc((size_t)Gs, sizeof(int64_t));
        int64_t *row = (int64_t *)malloc((size_t)S * sizeof(int64_t));
        uint8_t *near = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);  /* bit 0: adjacent to lo, bit 1: to hi */
        int64_t *U = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        if (!acc || !row || !near || !U) memfail = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t e = 0; e < G.m; ++e) {
            if (memfail) continue;
            const int64_t lo = G.eu[e], hi = G.ev[e];
            memset(row, 0, (size_t)S * sizeof(int64_t));
            { int64_t v[2] = {lo, hi}; int pos[2] = {0, 1}; acc[pa_global_slot(T, 0, 2, v, pos, types)] += 1; }
            /* U = the nodes other than lo and hi adjacent to lo or hi */
            int64_t nu = 0;
            for (int side = 0; side < 2; ++side) {
                const int64_t a = side == 0 ? lo : hi, other = side == 0 ? hi : lo;
                for (int64_t k = G.rp[a]; k < G.rp[a + 1]; ++k) {
                    const int64_t x = G.adj[k];
                    if (x == other) continue;
                    if (!near[x]) U[nu++] = x;
                    near[x] |= (uint8_t)(1 << side);
                }
            }
            for (int64_t ux = 0; ux < nu; ++ux) {                   /* 3-node sets */
                const int64_t x = U[ux];
                int64_t v[3] = {lo, hi, x};
                if (near[x] == 3) {                                  /* triangle */
                    row[O[2] + types[x]] += 1;
                    int pos[3] = {0, 1, 2};
                    acc[pa_global_slot(T, 2, 3, v, pos, types)] += 1;
                } else {                                             /* 3-path, centre lo or hi */
                    const int al = near[x] & 1;
                    row[O[1] + (al ? 0 : 1) * L + types[x]] += 1;
                    int pos[3] = {al ? 0 : 1, al ? 1 : 0, 2};
                    acc[pa_global_slot(T, 1, 3, v, pos, types)] += 1;
                }
            }
            /* 4-node sets {lo, hi, x, y}: x in U, and y in U after x, or y
             * outside U (and not lo, hi) adjacent to x */
            for (int64_t ux = 0; ux < nu; ++ux) {
                const int64_t x = U[ux];
                for (int pass = 0; pass < 2; ++pass) {
                    const int64_t yb = pass == 0 ? ux + 1 : G.rp[x], ye = pass == 0 ? nu : G.rp[x + 1];
                    for (int64_t yi = yb; yi < ye; ++yi) {
                        const int64_t y = pass == 0 ? U[yi] : G.adj[yi];
                        if (pass == 1 && (near[y] || y == lo || y == hi)) continue;
                        const int64_t v[4] = {lo, hi, x, y};
                        int A[4][4] = {{0}}, deg[4] = {0, 0, 0, 0}, ne = 0;
                        const int xy = pass == 1 ? 1 : is_adjacent(&G, x, y);
                        const int adj4[6][3] = {{0, 1, 1}, {0, 2, near[x] & 1}, {0, 3, near[y] & 1},
                                                {1, 2, (near[x] >> 1) & 1}, {1, 3, (near[y] >> 1) & 1}, {2, 3, xy}};
                        for (int q = 0; q < 6; ++q)
                            if (adj4[q][2]) {
                                const int a = adj4[q][0], c = adj4[q][1];
                                A[a][c] = A[c][a] = 1; deg[a]++; deg[c]++; ++ne;
                            }
                        int mind = 4, maxd = 0;
                        for (int a = 0; a < 4; ++a) {
                            if (deg[a] < mind) mind = deg[a];
                            if (deg[a] > maxd) maxd = deg[a];
                        }
                        if (ne < 3 || mind == 0) continue;               /* not connected */
                        const int tx = types[x], ty = types[y];
                        /* the other-node index (2 = x, 3 = y) adjacent to endpoint a */
#define OTHER_AT(a) (A[a][2] ? 2 : 3)
                        int b;
                        if (ne == 3 && maxd == 2) {                      /* 4-path */
                            b = 3;
                            if (deg[0] == 2 && deg[1] == 2) {            /* centre edge */
                                const int nl = OTHER_AT(0), nh = OTHER_AT(1);
                                row[O[4] + types[v[nl]] * L + types[v[nh]]] += 1;
                            } else {                                     /* end edge */
                                const int s = deg[0] == 2 ? 0 : 1;
                                const int nr = OTHER_AT(s), fr = 5 - nr;
                                row[O[3] + s * L * L + types[v[nr]] * L + types[v[fr]]] += 1;
                            }
                        } else if (ne == 3) {                            /* 4-star, centre lo or hi */
                            b = 4;
                            const int s = deg[0] == 3 ? 0 : 1;
                            row[O[5] + s * P + pair_index(L, tx, ty)] += 1;
                        } else if (ne == 4 && maxd == 2) {               /* 4-cycle */
                            b = 5;
                            const int nl = OTHER_AT(0), nh = OTHER_AT(1);
                            if (MUTANT(11)) row[O[6] + types[v[nh]] * L + types[v[nl]]] += 1;
                            else row[O[6] + types[v[nl]] * L + types[v[nh]]] += 1;
                        } else if (ne == 4) {                            /* tailed triangle */
                            b = 6;
                            int a3 = 0, tail = 0;
                            for (int a = 0; a < 4; ++a) {
                                if (deg[a] == 3) a3 = a;
                                if (deg[a] == 1) tail = a;
                            }
                            if ((a3 == 0 && tail == 1) || (a3 == 1 && tail == 0)) {          /* tail edge */
                                row[O[7] + a3 * P + pair_index(L, tx, ty)] += 1;
                            } else if (a3 >= 2) {                                            /* opposite */
                                row[O[8] + types[v[a3]] * L + types[v[tail]]] += 1;
                            } else {                                                         /* at a3 */
                                const int s = MUTANT(12) ? 1 - a3 : a3;
                                const int third = 5 - tail;
                                row[O[9] + s * L * L + types[v[third]] * L + types[v[tail]]] += 1;
                            }
                        } else if (ne == 5) {                            /* chordal cycle */
                            b = 7;
                            if (deg[0] == 3 && deg[1] == 3) {            /* chord */
                                row[O[11] + pair_index(L, tx, ty)] += 1;
                            } else {                                     /* outer edge */
                                const int s = deg[0] == 3 ? 0 : 1;
                                const int b3 = deg[2] == 3 ? 2 : 3, d2 = 5 - b3;
                                row[O[10] + s * L * L + types[v[b3]] * L + types[v[d2]]] += 1;
                            }
                        } else {                                         /* 4-clique */
                            b = 8;
                            row[O[12] + pair_index(L, tx, ty)] += 1;
                        }
#undef OTHER_AT
                        int pos[4];
                        if (!pa_positions(T, b, 4, A, pos)) { bad = 1; continue; }
                        acc[pa_global_slot(T, b, 4, v, pos, types)] += 1;
                    }
                }
            }
            for (int64_t ux = 0; ux < nu; ++ux) near[U[ux]] = 0;
            if (per_edge_out) memcpy(per_edge_out + e * S, row, (size_t)S * sizeof(int64_t));
        }
#pragma omp critical
        if (acc) for (int64_t s = 0; s < Gs; ++s) raw[s] += acc[s];
        free(acc); free(row); free(near); free(U);
    }
    if (memfail) rc = ERR_MEM;
    else if (bad) rc = ERR_REMAINDER;
    if (rc == OK && global_out) {
        for (int b = 0; b < 9; ++b) {
            const int64_t end = b < 8 ? T->block_off[b + 1] : Gs;
            for (int64_t s = T->block_off[b]; s < end; ++s) {
                if (raw[s] % EDGES_OF_GRAPHLET[b]) rc = ERR_REMAINDER;
                global_out[s] = raw[s] / EDGES_OF_GRAPHLET[b];
            }
        }
    }
    free(raw); free(T);
    graph_close(&G);
    return rc;
}

/* Position-aware global counts by brute force over all 2-, 3- and 4-node
 * sets (no per-edge step): each connected set counted once in its class.
 * Small graphs only. */
int oracle_position_aware_brute(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int L,
                                int64_t *global_out) {
    if (L < 1 || L > 8) return ERR_ARG;
    graph_t G;
    int rc = graph_open(&G, n, row_ptr, col, types, L);
    if (rc != OK) { graph_close(&G); return rc; }
    pa_tables_t *T = (pa_tables_t *)malloc(sizeof(pa_tables_t));
    if (!T) { graph_close(&G); return ERR_MEM; }
    pa_tables(L, T);
    memset(global_out, 0, (size_t)oracle_pa_global_slots(L) * sizeof(int64_t));
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b) {
            const int64_t v2[2] = {a, b};
            int pos2[2] = {0, 1};
            if (is_adjacent(&G, a, b)) global_out[pa_global_slot(T, 0, 2, v2, pos2, types)] += 1;
            for (int64_t c = b + 1; c < n; ++c) {
                int64_t v3[3] = {a, b, c};
                int A[4][4] = {{0}}, ne = 0;
                for (int x = 0; x < 3; ++x)
                    for (int y = x + 1; y < 3; ++y)
                        if (is_adjacent(&G, v3[x], v3[y])) { A[x][y] = A[y][x] = 1; ++ne; }
                if (ne >= 2) {
                    int pos[3], sh = ne == 2 ? 1 : 2;
                    if (!pa_positions(T, sh, 3, A, pos)) rc = ERR_REMAINDER;
                    else global_out[pa_global_slot(T, sh, 3, v3, pos, types)] += 1;
                }
                for (int64_t d = c + 1; d < n; ++d) {
                    int64_t v4[4] = {a, b, c, d};
                    int B[4][4] = {{0}}, deg[4] = {0, 0, 0, 0}, m4 = 0;
                    for (int x = 0; x < 4; ++x)
                        for (int y = x + 1; y < 4; ++y)
                            if (is_adjacent(&G, v4[x], v4[y])) { B[x][y] = B[y][x] = 1; deg[x]++; deg[y]++; ++m4; }
                    int mind = 4;
                    for (int x = 0; x < 4; ++x) if (deg[x] < mind) mind = deg[x];
                    if (m4 < 3 || mind == 0) continue;
                    int pos[4], found = 0;
                    for (int sh = 3; sh <= 8 && !found; ++sh) {
                        if (PA_NEDGES[sh] != m4) continue;
                        if (pa_positions(T, sh, 4, B, pos)) {
                            global_out[pa_global_slot(T, sh, 4, v4, pos, types)] += 1;
                            found = 1;
                        }
                    }
                    if (!found) rc = ERR_REMAINDER;
                }
            }
        }
    free(T);
    graph_close(&G);
    return rc;
}

/* ------------------------------------------- directed typed 3-node graphlets
 *
 * Sec. 4.8: in a directed graph every typed neighbourhood Gamma_i^t splits
 * into the typed out-neighbours Gamma_i^{t,+} and in-neighbours
 * Gamma_i^{t,-}, and so do T_ij^t, S_i^t and S_j^t.  The split is a
 * partition, so the input is an oriented graph: arcs u -> v given as an
 * out-neighbour CSR, no self-loops, no repeated arcs and no reciprocal pair
 * (u -> v together with v -> u).
 *
 * Per edge {i, j} of the underlying undirected graph (edge ids as above:
 * i < j, lexicographic), 8L slots, block b at b*L + t (t = type of the
 * third node w; the sign is the direction of the arc between the endpoint
 * and w, + when the endpoint is its tail):
 *   0 S_i^{t,+}   1 S_i^{t,-}   2 S_j^{t,+}   3 S_j^{t,-}
 *   4 T^{t}(+,+)  5 T^{t}(+,-)  6 T^{t}(-,+)  7 T^{t}(-,-)   (sign at i, sign at j)
 * Global: block 0, directed typed edges (type of tail, type of head), L^2
 * slots at tail*L + head; block 1, the connected directed typed 3-node
 * graphlets, one slot per isomorphism class, ranked by canonical code.
 * A labelled configuration on nodes 0, 1, 2 is the code (t0, t1, t2, a01,
 * a02, a12) with a_xy = 0 (no arc), 1 (x -> y) or 2 (y -> x), read as one
 * integer in mixed radix (L, L, L, 3, 3, 3); its class is represented by the
 * smallest code over the 6 renumberings of the nodes. */

static int64_t dir_code(int L, const int t[3], const int a[3]) {
    return ((((int64_t)(t[0] * L + t[1]) * L + t[2]) * 3 + a[0]) * 3 + a[1]) * 3 + a[2];
}

/* arc state of pair (x, y), x != y, in a configuration: 0 none, 1 x -> y, 2 y -> x */
static int dir_arc(const int a[3], int x, int y) {
    int lo = x < y ? x : y, hi = x < y ? y : x;
    int k = lo == 0 ? (hi == 1 ? 0 : 1) : 2;          /* pairs (0,1) (0,2) (1,2) */
    int s = a[k];
    if (s == 0 || x == lo) return s;
    return 3 - s;
}

/* smallest code over the renumberings: new node q is old node p[q] */
static int64_t dir_canonical(int L, const int t[3], const int a[3]) {
    static const int P[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int64_t best = -1;
    for (int k = 0; k < 6; ++k) {
        const int *p = P[k];
        int tt[3] = {t[p[0]], t[p[1]], t[p[2]]};
        int aa[3] = {dir_arc(a, p[0], p[1]), dir_arc(a, p[0], p[2]), dir_arc(a, p[1], p[2])};
        int64_t c = dir_code(L, tt, aa);
        if (best < 0 || c < best) best = c;
    }
    return best;
}

/* sorted canonical codes of all connected classes (returns their number) */
static int64_t dir_class_codes(int L, int64_t *codes) {
    int64_t nc = 0;
    for (int t0 = 0; t0 < L; ++t0) for (int t1 = 0; t1 < L; ++t1) for (int t2 = 0; t2 < L; ++t2)
    for (int a0 = 0; a0 < 3; ++a0) for (int a1 = 0; a1 < 3; ++a1) for (int a2 = 0; a2 < 3; ++a2) {
        int arcs = (a0 != 0) + (a1 != 0) + (a2 != 0);
        if (arcs < 2) continue;                        /* 3 nodes are connected by 2 or 3 arcs */
        int t[3] = {t0, t1, t2}, a[3] = {a0, a1, a2};
        int64_t c = dir_code(L, t, a);
        if (dir_canonical(L, t, a) != c) continue;     /* codes rise in loop order */
        if (codes) codes[nc] = c;
        ++nc;
    }
    return nc;
}

int64_t oracle_directed_classes(int L) {
    if (L < 1 || L > OR_MAX_L) return -1;
    return dir_class_codes(L, NULL);
}

int64_t oracle_directed_global_slots(int L) {
    if (L < 1 || L > OR_MAX_L) return -1;
    return (int64_t)L * L + dir_class_codes(L, NULL);
}

/* rank of the class of a labelled configuration, -1 if disconnected */
static int64_t dir_rank(int L, const int64_t *codes, int64_t nc, const int t[3], const int a[3]) {
    if ((a[0] != 0) + (a[1] != 0) + (a[2] != 0) < 2) return -1;
    int64_t c = dir_canonical(L, t, a), lo = 0, hi = nc;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (codes[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo < nc && codes[lo] == c ? lo : -1;
}

int64_t oracle_directed_class(int L, const int32_t *t, const int32_t *a) {
    if (L < 1 || L > OR_MAX_L) return -1;
    int64_t nc = dir_class_codes(L, NULL);
    int64_t *codes = (int64_t *)malloc((size_t)nc * sizeof(int64_t));
    if (!codes) return -1;
    dir_class_codes(L, codes);
    int tt[3] = {t[0], t[1], t[2]}, aa[3] = {a[0], a[1], a[2]};
    int64_t r = dir_rank(L, codes, nc, tt, aa);
    free(codes);
    return r;
}

typedef struct {
    int64_t n, m;
    int L;
    const uint8_t *phi;
    int64_t *rp;                /* symmetric rows, sorted by neighbour id */
    int32_t *adj;
    int8_t *sg;                 /* +1: the row node is the arc's tail, -1: its head */
    int64_t *eu, *ev;           /* edges u < v, lexicographic */
    int8_t *eo;                 /* 0: arc eu -> ev, 1: arc ev -> eu */
} dgraph_t;

static void dgraph_close(dgraph_t *D) { free(D->rp); free(D->adj); free(D->sg); free(D->eu); free(D->ev); free(D->eo); }

typedef struct { int32_t v; int8_t s; } dent_t;
static int cmp_dent(const void *x, const void *y) {
    int32_t a = ((const dent_t *)x)->v, b = ((const dent_t *)y)->v;
    return (a > b) - (a < b);
}

static int dgraph_open(dgraph_t *D, int64_t n, const int64_t *orp, const int32_t *ocol, const uint8_t *phi, int L) {
    memset(D, 0, sizeof(*D));
    if (n < 0 || L < 1 || L > OR_MAX_L) return ERR_ARG;
    int64_t na = orp[n];
    if (orp[0] != 0 || na < 0) return ERR_GRAPH;
    for (int64_t v = 0; v < n; ++v) if (orp[v + 1] < orp[v] || phi[v] >= L) return ERR_GRAPH;
    for (int64_t k = 0; k < na; ++k) if (ocol[k] < 0 || ocol[k] >= n) return ERR_GRAPH;
    D->n = n; D->m = na; D->L = L; D->phi = phi;
    D->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    D->adj = (int32_t *)malloc((size_t)(2 * na > 0 ? 2 * na : 1) * sizeof(int32_t));
    D->sg = (int8_t *)malloc((size_t)(2 * na > 0 ? 2 * na : 1));
    D->eu = (int64_t *)malloc((size_t)(na > 0 ? na : 1) * sizeof(int64_t));
    D->ev = (int64_t *)malloc((size_t)(na > 0 ? na : 1) * sizeof(int64_t));
    D->eo = (int8_t *)malloc((size_t)(na > 0 ? na : 1));
    dent_t *tmp = (dent_t *)malloc((size_t)(2 * na > 0 ? 2 * na : 1) * sizeof(dent_t));
    int64_t *fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!D->rp || !D->adj || !D->sg || !D->eu || !D->ev || !D->eo || !tmp || !fill) { free(tmp); free(fill); return ERR_MEM; }
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = orp[u]; k < orp[u + 1]; ++k) { D->rp[u + 1]++; D->rp[ocol[k] + 1]++; }
    for (int64_t v = 0; v < n; ++v) D->rp[v + 1] += D->rp[v];
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = orp[u]; k < orp[u + 1]; ++k) {
            int64_t v = ocol[k];
            if (v == u) { free(tmp); free(fill); return ERR_GRAPH; }                 /* self-loop */
            tmp[D->rp[u] + fill[u]++] = (dent_t){(int32_t)v, 1};
            tmp[D->rp[v] + fill[v]++] = (dent_t){(int32_t)u, -1};
        }
    int rc = OK;
    int64_t e = 0;
    for (int64_t u = 0; u < n && rc == OK; ++u) {
        qsort(tmp + D->rp[u], (size_t)(D->rp[u + 1] - D->rp[u]), sizeof(dent_t), cmp_dent);
        for (int64_t k = D->rp[u]; k < D->rp[u + 1]; ++k) {
            if (k > D->rp[u] && tmp[k - 1].v == tmp[k].v) { rc = ERR_GRAPH; break; }  /* repeated or reciprocal */
            D->adj[k] = tmp[k].v;
            D->sg[k] = tmp[k].s;
            if (tmp[k].v > u) { D->eu[e] = u; D->ev[e] = tmp[k].v; D->eo[e] = tmp[k].s > 0 ? 0 : 1; ++e; }
        }
    }
    free(tmp); free(fill);
    if (rc == OK && e != na) rc = ERR_GRAPH;
    return rc;
}

/* configuration of (i = 0, j = 1, w = 2) for an edge of orientation o and
 * the third node's signs at i and j (0: not adjacent) */
static void dir_config(int o, int si, int sj, int a[3]) {
    a[0] = o == 0 ? 1 : 2;
    a[1] = si == 0 ? 0 : (si > 0 ? 1 : 2);            /* i -> w when i is the tail */
    a[2] = sj == 0 ? 0 : (sj > 0 ? 1 : 2);
}

/* per-edge slot block of a third node from its signs at i and j */
static int dir_block(int si, int sj) {
    if (si != 0 && sj != 0) return 4 + (si > 0 ? 0 : 2) + (sj > 0 ? 0 : 1);
    if (si != 0) return si > 0 ? 0 : 1;
    return sj > 0 ? 2 : 3;
}

/* Alg. 1 with the sets split by direction (Sec. 4.8): mark Gamma_i with
 * the signs at i, scan Gamma_j, then the rest of Gamma_i.  per_edge_out:
 * int64 [m][8L] or NULL; global_out: int64 [L^2 + classes] or NULL. */
int oracle_directed3(int64_t n, const int64_t *out_row_ptr, const int32_t *out_col, const uint8_t *types, int L,
                     int64_t *per_edge_out, int64_t *global_out) {
    dgraph_t D;
    int rc = dgraph_open(&D, n, out_row_ptr, out_col, types, L);
    if (rc != OK) { dgraph_close(&D); return rc; }
    const int64_t nc = dir_class_codes(L, NULL);
    int64_t *codes = (int64_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
    int8_t *psi = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *raw = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!codes || !psi || !raw) { free(codes); free(psi); free(raw); dgraph_close(&D); return ERR_MEM; }
    dir_class_codes(L, codes);
    const int64_t S = 8 * (int64_t)L;
    if (global_out) memset(global_out, 0, (size_t)(L * L + nc) * sizeof(int64_t));
    int64_t row[8 * OR_MAX_L];
    for (int64_t e = 0; e < D.m && rc == OK; ++e) {
        const int64_t i = D.eu[e], j = D.ev[e];
        const int o = D.eo[e];
        memset(row, 0, sizeof(row));
        for (int64_t k = D.rp[i]; k < D.rp[i + 1]; ++k) if (D.adj[k] != j) psi[D.adj[k]] = D.sg[k];
        for (int64_t k = D.rp[j]; k < D.rp[j + 1]; ++k) {                  /* T and S_j */
            int64_t w = D.adj[k];
            if (w == i) continue;
            int si = psi[w], sj = D.sg[k];
            if (MUTANT(13) && si == 0) sj = -sj;                            /* planted: S_j signs flipped */
            row[dir_block(si, sj) * L + types[w]] += 1;
        }
        for (int64_t k = D.rp[j]; k < D.rp[j + 1]; ++k) psi[D.adj[k]] = psi[D.adj[k]] ? 2 : 0;   /* 2: in T */
        for (int64_t k = D.rp[i]; k < D.rp[i + 1]; ++k) {                  /* S_i */
            int64_t w = D.adj[k];
            if (w == j || psi[w] == 2) continue;
            row[dir_block(D.sg[k], 0) * L + types[w]] += 1;
        }
        for (int64_t k = D.rp[i]; k < D.rp[i + 1]; ++k) psi[D.adj[k]] = 0;
        for (int64_t k = D.rp[j]; k < D.rp[j + 1]; ++k) psi[D.adj[k]] = 0;
        if (per_edge_out) memcpy(per_edge_out + e * S, row, (size_t)S * sizeof(int64_t));
        if (global_out) {
            const int tail = types[o == 0 ? i : j], head = types[o == 0 ? j : i];
            global_out[tail * L + head] += 1;
            for (int b = 0; b < 8; ++b)
                for (int t = 0; t < L; ++t) {
                    int64_t v = row[b * L + t];
                    if (!v) continue;
                    int si = b < 2 ? (b == 0 ? 1 : -1) : (b < 4 ? 0 : (b < 6 ? 1 : -1));
                    int sj = b < 2 ? 0 : (b < 4 ? (b == 2 ? 1 : -1) : ((b & 1) ? -1 : 1));
                    int a[3], tt[3] = {types[i], types[j], t};
                    dir_config(MUTANT(14) ? 0 : o, si, sj, a);                /* planted: orientation dropped */
                    int64_t r = dir_rank(L, codes, nc, tt, a);
                    if (r < 0) { rc = ERR_REMAINDER; break; }
                    raw[r] += v;
                }
        }
    }
    if (global_out && rc == OK)
        for (int64_t r = 0; r < nc; ++r) {
            /* a path is seen from its 2 arcs, a triangle from its 3 */
            int64_t c = codes[r];
            int a2 = (int)(c % 3), a1 = (int)(c / 3 % 3), a0 = (int)(c / 9 % 3);
            int arcs = (a0 != 0) + (a1 != 0) + (a2 != 0);
            if (raw[r] % arcs) { rc = ERR_REMAINDER; break; }
            global_out[L * L + r] = raw[r] / arcs;
        }
    free(codes); free(psi); free(raw);
    dgraph_close(&D);
    return rc;
}

/* Every 3-node subset: its induced arcs; a connected one adds 1 to its class
 * and, for each of its arcs, to the slot of that edge keyed by the third
 * node.  Small graphs only. */
int oracle_directed3_brute(int64_t n, const int64_t *out_row_ptr, const int32_t *out_col, const uint8_t *types, int L,
                           int64_t *per_edge_out, int64_t *global_out) {
    dgraph_t D;
    int rc = dgraph_open(&D, n, out_row_ptr, out_col, types, L);
    if (rc != OK) { dgraph_close(&D); return rc; }
    const int64_t nc = dir_class_codes(L, NULL);
    int64_t *codes = (int64_t *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int64_t));
    if (!codes) { dgraph_close(&D); return ERR_MEM; }
    dir_class_codes(L, codes);
    const int64_t S = 8 * (int64_t)L;
    if (per_edge_out) memset(per_edge_out, 0, (size_t)(D.m * S) * sizeof(int64_t));
    if (global_out) memset(global_out, 0, (size_t)(L * L + nc) * sizeof(int64_t));
    for (int64_t e = 0; e < D.m; ++e)
        if (global_out) {
            const int64_t i = D.eu[e], j = D.ev[e];
            const int tail = types[D.eo[e] == 0 ? i : j], head = types[D.eo[e] == 0 ? j : i];
            global_out[tail * L + head] += 1;
        }
    for (int64_t x = 0; x < n && rc == OK; ++x)
        for (int64_t y = x + 1; y < n && rc == OK; ++y)
            for (int64_t z = y + 1; z < n && rc == OK; ++z) {
                int64_t v[3] = {x, y, z};
                int s[3][3] = {{0}};
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q)
                        if (p != q) {
                            int64_t lo = D.rp[v[p]], hi = D.rp[v[p] + 1];
                            while (lo < hi) {
                                int64_t mid = (lo + hi) / 2;
                                if (D.adj[mid] < v[q]) lo = mid + 1; else hi = mid;
                            }
                            if (lo < D.rp[v[p] + 1] && D.adj[lo] == v[q]) s[p][q] = D.sg[lo];
                        }
                int t[3] = {types[x], types[y], types[z]};
                int a[3] = {s[0][1] == 0 ? 0 : (s[0][1] > 0 ? 1 : 2), s[0][2] == 0 ? 0 : (s[0][2] > 0 ? 1 : 2),
                            s[1][2] == 0 ? 0 : (s[1][2] > 0 ? 1 : 2)};
                int64_t r = dir_rank(L, codes, nc, t, a);
                if (r < 0) continue;                                      /* disconnected */
                if (global_out) global_out[L * L + r] += 1;
                if (!per_edge_out) continue;
                for (int p = 0; p < 3; ++p)
                    for (int q = p + 1; q < 3; ++q) {
                        if (!s[p][q]) continue;
                        int w = 3 - p - q;                                /* v[p] < v[q]: i = v[p], j = v[q] */
                        int64_t lo = 0, hi = D.m;
                        while (lo < hi) {
                            int64_t mid = (lo + hi) / 2;
                            if (D.eu[mid] < v[p] || (D.eu[mid] == v[p] && D.ev[mid] < v[q])) lo = mid + 1; else hi = mid;
                        }
                        per_edge_out[lo * S + dir_block(s[p][w], s[q][w]) * L + t[w]] += 1;
                    }
            }
    free(codes);
    dgraph_close(&D);
    return rc;
}

/* Edges of the underlying undirected graph in edge-id order (u < v) and
 * their orientation (0: u -> v, 1: v -> u). */
int oracle_directed_edges(int64_t n, const int64_t *out_row_ptr, const int32_t *out_col, const uint8_t *types, int L,
                          int64_t *src, int64_t *dst, int8_t *orient) {
    dgraph_t D;
    int rc = dgraph_open(&D, n, out_row_ptr, out_col, types, L);
    if (rc == OK) {
        memcpy(src, D.eu, (size_t)D.m * sizeof(int64_t));
        memcpy(dst, D.ev, (size_t)D.m * sizeof(int64_t));
        memcpy(orient, D.eo, (size_t)D.m);
    }
    dgraph_close(&D);
    return rc;
}

/* ======================================================================
 * Edge-typed 3-node graphlets (Def. 1's edge types xi; Defs. 4-5: the
 * class of a typed graphlet is its shape with the multisets of its node
 * types and of its edge types).
 *
 * Per edge e = (i, j), i < j in the caller's ids, every third node k of
 * type t adds 1 to one slot:
 *   k in S_i or S_j (a 3-path through e): slot (t, x) of the path block,
 *     x the type of k's edge to i (S_i) or to j (S_j) -- the path's class
 *     ({phi_i, phi_j, t}, {xi_ij, x}) is the same either way;
 *   k in T (a triangle): slot (t, {xi_ik, xi_jk}) of the triangle block.
 * Per-edge layout: [L][X] paths, then [L][X(X+1)/2] triangles, the pair of
 * edge types ranked as a sorted 2-multiset over [0, X).
 * Global layout: [edges: multisets of 2 node types x X edge types]
 * [3-paths: multisets of 3 node types x multisets of 2 edge types]
 * [triangles: multisets of 3 node types x multisets of 3 edge types],
 * the node-type multiset rank the major index.
 * ==================================================================== */

#define OR_MAX_X 8

int64_t oracle_et_per_edge_slots(int L, int X) { return (int64_t)L * X + (int64_t)L * npairs(X); }

int64_t oracle_et_global_slots(int L, int X) {
    return binom(L + 1, 2) * X + binom(L + 2, 3) * binom(X + 1, 2) + binom(L + 2, 3) * binom(X + 2, 3);
}

typedef struct { int32_t v; uint8_t x; } eent_t;
static int cmp_eent(const void *p, const void *q) {
    int32_t a = ((const eent_t *)p)->v, b = ((const eent_t *)q)->v;
    return (a > b) - (a < b);
}

typedef struct {
    int64_t n, m;
    int L, X;
    const int64_t *rp;
    int32_t *adj;              /* rows sorted by id */
    uint8_t *xi;               /* edge type of each entry */
    const uint8_t *phi;
    int64_t *eu, *ev;          /* edges u < v, lexicographic */
} egraph_t;

static void egraph_close(egraph_t *E) { free(E->adj); free(E->xi); free(E->eu); free(E->ev); }

/* edge type of {u, v}, or -1 when u and v are not adjacent */
static int egraph_type(const egraph_t *E, int64_t u, int64_t v) {
    int64_t lo = E->rp[u], hi = E->rp[u + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (E->adj[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (lo < E->rp[u + 1] && E->adj[lo] == v) ? E->xi[lo] : -1;
}

/* copies and sorts the rows with their edge types; a simple symmetric graph
 * whose two entries of every edge carry the same type below X */
static int egraph_open(egraph_t *E, int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *phi,
                       const uint8_t *xi, int L, int X) {
    memset(E, 0, sizeof(*E));
    if (n < 0 || L < 1 || L > OR_MAX_L || X < 1 || X > OR_MAX_X) return ERR_ARG;
    int64_t nnz = rp[n];
    if (rp[0] != 0 || nnz < 0 || (nnz & 1)) return ERR_GRAPH;
    for (int64_t v = 0; v < n; ++v) if (rp[v + 1] < rp[v] || phi[v] >= L) return ERR_GRAPH;
    for (int64_t k = 0; k < nnz; ++k) if (col[k] < 0 || col[k] >= n || xi[k] >= X) return ERR_GRAPH;
    E->n = n; E->m = nnz / 2; E->L = L; E->X = X; E->rp = rp; E->phi = phi;
    E->adj = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    E->xi = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    E->eu = (int64_t *)malloc((size_t)(E->m > 0 ? E->m : 1) * sizeof(int64_t));
    E->ev = (int64_t *)malloc((size_t)(E->m > 0 ? E->m : 1) * sizeof(int64_t));
    eent_t *tmp = (eent_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(eent_t));
    if (!E->adj || !E->xi || !E->eu || !E->ev || !tmp) { free(tmp); return ERR_MEM; }
    for (int64_t k = 0; k < nnz; ++k) tmp[k] = (eent_t){col[k], xi[k]};
    for (int64_t v = 0; v < n; ++v) qsort(tmp + rp[v], (size_t)(rp[v + 1] - rp[v]), sizeof(eent_t), cmp_eent);
    for (int64_t k = 0; k < nnz; ++k) { E->adj[k] = tmp[k].v; E->xi[k] = tmp[k].x; }
    free(tmp);
    int64_t e = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = rp[u]; k < rp[u + 1]; ++k) {
            int64_t v = E->adj[k];
            if (v == u) return ERR_GRAPH;                                        /* self-loop */
            if (k > rp[u] && E->adj[k - 1] == v) return ERR_GRAPH;               /* duplicate */
            if (egraph_type(E, v, u) != E->xi[k]) return ERR_GRAPH;              /* asymmetric, or types differ */
            if (u < v) {
                if (e >= E->m) return ERR_GRAPH;
                E->eu[e] = u; E->ev[e] = v; ++e;
            }
        }
    if (e != E->m) return ERR_GRAPH;
    return OK;
}

/* global slot of a class: block 0 (an edge), 1 (a 3-path), 2 (a triangle);
 * nt node types and nt - 1 (edge) or the shape's edge types */
static int64_t et_global_slot(int L, int X, int block, const int *nodes, const int *edges) {
    const int64_t rn = multiset_rank(L, block == 0 ? 2 : 3, nodes);
    const int64_t re = block == 0 ? edges[0] : multiset_rank(X, block == 1 ? 2 : 3, edges);
    if (rn < 0 || re < 0) return -1;                                   /* (a wrong rank is reported) */
    if (block == 0) return rn * X + re;
    const int64_t off1 = binom(L + 1, 2) * X, off2 = off1 + binom(L + 2, 3) * binom(X + 1, 2);
    if (block == 1) return off1 + rn * binom(X + 1, 2) + re;
    return off2 + rn * binom(X + 2, 3) + re;
}

/* Alg. 1 with the sets split by edge type: mark Gamma_i with the type of
 * each node's edge to i, scan Gamma_j (T and S_j), then the rest of Gamma_i
 * (S_i).  per_edge_out: int64 [m][oracle_et_per_edge_slots] or NULL;
 * global_out: int64 [oracle_et_global_slots] or NULL. */
int oracle_edge_typed3(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types,
                       const uint8_t *edge_types, int L, int X, int64_t *per_edge_out, int64_t *global_out) {
    egraph_t E;
    int rc = egraph_open(&E, n, row_ptr, col, types, edge_types, L, X);
    if (rc != OK) { egraph_close(&E); return rc; }
    const int64_t S = oracle_et_per_edge_slots(L, X), PX = npairs(X), Gs = oracle_et_global_slots(L, X);
    int16_t *mark = (int16_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int16_t));   /* 1 + type of the edge to i */
    int64_t *row = (int64_t *)malloc((size_t)S * sizeof(int64_t));
    int64_t *raw = (int64_t *)calloc((size_t)Gs, sizeof(int64_t));
    if (!mark || !row || !raw) { free(mark); free(row); free(raw); egraph_close(&E); return ERR_MEM; }
    for (int64_t e = 0; e < E.m && rc == OK; ++e) {
        const int64_t i = E.eu[e], j = E.ev[e];
        const int xij = egraph_type(&E, i, j);
        memset(row, 0, (size_t)S * sizeof(int64_t));
        for (int64_t k = E.rp[i]; k < E.rp[i + 1]; ++k) if (E.adj[k] != j) mark[E.adj[k]] = (int16_t)(1 + E.xi[k]);
        for (int64_t k = E.rp[j]; k < E.rp[j + 1]; ++k) {                  /* T and S_j */
            const int64_t w = E.adj[k];
            if (w == i) continue;
            const int t = types[w], xj = E.xi[k];
            if (mark[w] > 0) {
                const int xi_w = mark[w] - 1;
                const int pair[2] = {xi_w, MUTANT(16) ? xi_w : xj};           /* planted: j's edge dropped */
                const int64_t r = multiset_rank(X, 2, pair);
                if (r < 0) { rc = ERR_REMAINDER; break; }                  /* (a wrong rank is reported) */
                row[(int64_t)L * X + t * PX + r] += 1;
                mark[w] = -1;                                              /* in T */
            } else {
                row[t * X + (MUTANT(15) ? xij : xj)] += 1;                  /* planted: the edge's own type */
            }
        }
        for (int64_t k = E.rp[i]; k < E.rp[i + 1]; ++k) {                  /* S_i */
            const int64_t w = E.adj[k];
            if (w == j || mark[w] < 0) continue;
            row[types[w] * X + E.xi[k]] += 1;
        }
        for (int64_t k = E.rp[i]; k < E.rp[i + 1]; ++k) mark[E.adj[k]] = 0;
        if (per_edge_out) memcpy(per_edge_out + e * S, row, (size_t)S * sizeof(int64_t));
        if (global_out) {
            const int nodes2[2] = {types[i], types[j]}, edges1[1] = {xij};
            const int64_t g2 = et_global_slot(L, X, 0, nodes2, edges1);
            if (g2 < 0) rc = ERR_REMAINDER; else raw[g2] += 1;
            for (int t = 0; t < L; ++t) {
                const int nodes3[3] = {types[i], types[j], t};
                for (int x = 0; x < X; ++x) {
                    const int64_t v = row[t * X + x];
                    const int edges2[2] = {xij, x};
                    const int64_t gs = et_global_slot(L, X, 1, nodes3, edges2);
                    if (gs < 0) rc = ERR_REMAINDER;
                    else if (v) raw[gs] += v;
                }
                for (int x = 0; x < X; ++x)
                    for (int y = x; y < X; ++y) {
                        const int pair[2] = {x, y};
                        const int64_t r = multiset_rank(X, 2, pair);
                        const int edges3[3] = {xij, x, y};
                        const int64_t gs = et_global_slot(L, X, 2, nodes3, edges3);
                        if (r < 0 || gs < 0) { rc = ERR_REMAINDER; continue; }
                        const int64_t v = row[(int64_t)L * X + t * PX + r];
                        if (v) raw[gs] += v;
                    }
            }
        }
    }
    if (global_out && rc == OK) {
        /* Sec. 6: a 3-path is seen from its 2 edges, a triangle from its 3 */
        const int64_t off1 = binom(L + 1, 2) * X, off2 = off1 + binom(L + 2, 3) * binom(X + 1, 2);
        for (int64_t s = 0; s < Gs && rc == OK; ++s) {
            const int64_t d = s < off1 ? 1 : (s < off2 ? 2 : 3);
            if (raw[s] % d) rc = ERR_REMAINDER;
            global_out[s] = raw[s] / d;
        }
    }
    free(mark); free(row); free(raw);
    egraph_close(&E);
    return rc;
}

/* Every 3-node subset: its induced edges and their types; a connected one
 * adds 1 to its class and, for each of its edges, to that edge's slot keyed
 * by the third node.  Small graphs only. */
int oracle_edge_typed3_brute(int64_t n, const int64_t *row_ptr, const int32_t *col, const uint8_t *types,
                             const uint8_t *edge_types, int L, int X, int64_t *per_edge_out, int64_t *global_out) {
    egraph_t E;
    int rc = egraph_open(&E, n, row_ptr, col, types, edge_types, L, X);
    if (rc != OK) { egraph_close(&E); return rc; }
    const int64_t S = oracle_et_per_edge_slots(L, X), PX = npairs(X);
    if (per_edge_out) memset(per_edge_out, 0, (size_t)(E.m * S) * sizeof(int64_t));
    if (global_out) memset(global_out, 0, (size_t)oracle_et_global_slots(L, X) * sizeof(int64_t));
    for (int64_t e = 0; e < E.m; ++e)
        if (global_out) {
            const int nodes2[2] = {types[E.eu[e]], types[E.ev[e]]}, edges1[1] = {egraph_type(&E, E.eu[e], E.ev[e])};
            const int64_t g2 = et_global_slot(L, X, 0, nodes2, edges1);
            if (g2 < 0) rc = ERR_REMAINDER; else global_out[g2] += 1;
        }
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b)
            for (int64_t c = b + 1; c < n; ++c) {
                const int64_t v[3] = {a, b, c};
                int x[3][3], ne = 0, ed[3];
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q) x[p][q] = p == q ? -1 : egraph_type(&E, v[p], v[q]);
                for (int p = 0; p < 3; ++p)
                    for (int q = p + 1; q < 3; ++q)
                        if (x[p][q] >= 0) ed[ne++] = x[p][q];
                if (ne < 2) continue;                                      /* not connected */
                const int nodes3[3] = {types[a], types[b], types[c]};
                const int64_t gs = et_global_slot(L, X, ne == 2 ? 1 : 2, nodes3, ed);
                if (gs < 0) { rc = ERR_REMAINDER; continue; }
                if (global_out) global_out[gs] += 1;
                if (!per_edge_out) continue;
                for (int p = 0; p < 3; ++p)
                    for (int q = p + 1; q < 3; ++q) {
                        if (x[p][q] < 0) continue;
                        const int w = 3 - p - q;                           /* edge (v[p], v[q]), third node v[w] */
                        int64_t lo = 0, hi = E.m;
                        while (lo < hi) {
                            int64_t mid = (lo + hi) / 2;
                            if (E.eu[mid] < v[p] || (E.eu[mid] == v[p] && E.ev[mid] < v[q])) lo = mid + 1; else hi = mid;
                        }
                        const int t = types[v[w]];
                        if (ne == 3) {
                            const int pair[2] = {x[p][w], x[q][w]};
                            const int64_t r = multiset_rank(X, 2, pair);
                            if (r < 0) { rc = ERR_REMAINDER; continue; }
                            per_edge_out[lo * S + (int64_t)L * X + t * PX + r] += 1;
                        } else {
                            per_edge_out[lo * S + t * X + (x[p][w] >= 0 ? x[p][w] : x[q][w])] += 1;
                        }
                    }
            }
    egraph_close(&E);
    return rc;
}

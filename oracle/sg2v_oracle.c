/*
 * Exact CPU oracle for colour-coding tree counting
 * (SubGraph2Vec: Highly-Vectorized Tree-like Subgraph Counting, arXiv 2009.11665).
 *
 * TEST INFRASTRUCTURE ONLY.  This file builds a standalone shared library that
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * load through ctypes.  The CUDA product path never links, loads or calls it,
 * and the two share no code, header, table or constant generator.
 *
 * What it computes (Sec. 2.2.1-2.2.2, Alg. 1).  For a graph G given as a
 * symmetric CSR matrix, a tree template T (parent array, root rho) and a
 * colouring col : V -> {0..kc-1}:
 *
 *   per_vertex[v] = number of maps phi : V_T -> V that send every tree edge to
 *                   a graph edge, give the |V_T| template vertices pairwise
 *                   distinct colours, and send rho to v;
 *   total         = sum over v of per_vertex[v].
 *
 * With integer edge weights each map contributes the product of the weights
 * of the graph edges it uses instead of 1 (the weighted form; unweighted is
 * every weight equal to one).
 *
 * Three independent routes reach that number:
 *   oracle_dp(mode = ORACLE_DECOUPLED)  neighbour sums first, then products
 *                                       over colour-set splits (Alg. 3, Eq. 1);
 *   oracle_dp(mode = ORACLE_STANDARD)   products inside the neighbour loop
 *                                       (Alg. 2);
 *   oracle_brute                        depth-first enumeration of every map.
 * Sec. 6.7 states that the first two agree exactly in exact arithmetic.
 *
 * Template partitioning (Sec. 2.3.2): the sub-template rooted at x that keeps
 * children c_lo..c_{hi-1} of x is split by cutting the edge to one kept child
 * tau (the last kept child, or the first with ORACLE_CUT_FIRST); the part that
 * keeps x is the active child, the subtree of tau (rooted at tau) the passive
 * child.  Children of a vertex are ordered by vertex index in the tree
 * re-rooted at rho.  The counts do not depend on this choice.
 *
 * Colour sets are bitmasks.  Columns of a table for t-element sets are
 * numbered in lexicographic order of the sorted element tuples (the paper
 * leaves I_C unspecified, Table 1).
 *
 * Arithmetic: unsigned integers of NL 64-bit limbs (compile-time constant)
 * with a sticky overflow flag; callers rebuild/rerun with a wider NL when the
 * flag is raised.  No floating point is used anywhere in this file.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef NL
#define NL 2
#endif

#define ORACLE_DECOUPLED 0
#define ORACLE_STANDARD 1
#define ORACLE_CUT_LAST 0
#define ORACLE_CUT_FIRST 1

#define ORACLE_OK 0
#define ORACLE_OVERFLOW 1
#define ORACLE_BAD_INPUT (-1)
#define ORACLE_NO_MEMORY (-2)

#define MAXK 24

/* ---------------------------------------------------------------- big ints */

typedef struct {
    uint64_t w[NL];
} big;

static inline void big_zero(big *x) { memset(x, 0, sizeof *x); }

static inline void big_from_u64(big *x, uint64_t v) {
    big_zero(x);
    x->w[0] = v;
}

static inline int big_is_zero(const big *x) {
    for (int i = 0; i < NL; ++i)
        if (x->w[i]) return 0;
    return 1;
}

/* x += y; returns nonzero when the sum does not fit in NL limbs */
static inline int big_add(big *x, const big *y) {
    uint64_t carry = 0;
    for (int i = 0; i < NL; ++i) {
        unsigned __int128 s = (unsigned __int128)x->w[i] + y->w[i] + carry;
        x->w[i] = (uint64_t)s;
        carry = (uint64_t)(s >> 64);
    }
    return carry != 0;
}

/* r = x * y (schoolbook); returns nonzero when the product needs more limbs */
static inline int big_mul(big *r, const big *x, const big *y) {
    uint64_t t[2 * NL];
    memset(t, 0, sizeof t);
    for (int i = 0; i < NL; ++i) {
        if (!x->w[i]) continue;
        uint64_t carry = 0;
        for (int j = 0; j < NL; ++j) {
            unsigned __int128 p = (unsigned __int128)x->w[i] * y->w[j] + t[i + j] + carry;
            t[i + j] = (uint64_t)p;
            carry = (uint64_t)(p >> 64);
        }
        t[i + NL] = carry;
    }
    int ovf = 0;
    for (int i = NL; i < 2 * NL; ++i) ovf |= (t[i] != 0);
    memcpy(r->w, t, sizeof r->w);
    return ovf;
}

/* acc += x * y */
static inline int big_fma(big *acc, const big *x, const big *y) {
    if (big_is_zero(x) || big_is_zero(y)) return 0;
    big p;
    int o = big_mul(&p, x, y);
    o |= big_add(acc, &p);
    return o;
}

/* number of significant bits (0 for zero) */
static inline int big_bits(const big *x) {
    for (int i = NL - 1; i >= 0; --i)
        if (x->w[i]) return 64 * i + 64 - __builtin_clzll(x->w[i]);
    return 0;
}

/* ------------------------------------------------------------ the template */

typedef struct {
    int k;                   /* template vertices */
    int root;                /* rho */
    int par[MAXK];           /* parent in the tree re-rooted at rho, -1 at rho */
    int nchild[MAXK];
    int child[MAXK][MAXK];   /* children in increasing vertex index */
    int subsize[MAXK];       /* vertices in the subtree of each vertex */
} tree_t;

/* Reads a parent array (one -1 entry), checks that it describes a tree on k
 * vertices and re-roots it at `root`.  Returns 0 or ORACLE_BAD_INPUT. */
static int tree_build(int k, const int32_t *parent, int root, tree_t *T) {
    if (k < 1 || k > MAXK || root < 0 || root >= k) return ORACLE_BAD_INPUT;
    int adj[MAXK][MAXK], deg[MAXK];
    memset(deg, 0, sizeof deg);
    int roots = 0;
    for (int i = 0; i < k; ++i) {
        if (parent[i] == -1) {
            ++roots;
            continue;
        }
        if (parent[i] < 0 || parent[i] >= k || parent[i] == i) return ORACLE_BAD_INPUT;
        int p = parent[i];
        adj[i][deg[i]++] = p;
        adj[p][deg[p]++] = i;
    }
    if (roots != 1) return ORACLE_BAD_INPUT;
    /* k-1 edges; connected from rho means it is a tree */
    int seen[MAXK], queue[MAXK], head = 0, tail = 0;
    memset(seen, 0, sizeof seen);
    T->k = k;
    T->root = root;
    T->par[root] = -1;
    seen[root] = 1;
    queue[tail++] = root;
    for (int i = 0; i < k; ++i) T->nchild[i] = 0;
    while (head < tail) {
        int x = queue[head++];
        /* neighbours in increasing index give children in increasing index */
        int nb[MAXK], m = deg[x];
        memcpy(nb, adj[x], sizeof(int) * (size_t)m);
        for (int a = 1; a < m; ++a)
            for (int b = a; b > 0 && nb[b - 1] > nb[b]; --b) {
                int t = nb[b];
                nb[b] = nb[b - 1];
                nb[b - 1] = t;
            }
        for (int j = 0; j < m; ++j) {
            int y = nb[j];
            if (y == T->par[x]) continue;
            if (seen[y]) return ORACLE_BAD_INPUT; /* a cycle */
            seen[y] = 1;
            T->par[y] = x;
            T->child[x][T->nchild[x]++] = y;
            queue[tail++] = y;
        }
    }
    if (tail != k) return ORACLE_BAD_INPUT;
    for (int q = k - 1; q >= 0; --q) {
        int x = queue[q];
        T->subsize[x] = 1;
        for (int j = 0; j < T->nchild[x]; ++j) T->subsize[x] += T->subsize[T->child[x][j]];
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------ colour-set columns */

typedef struct {
    int kc;
    int32_t *index_of;       /* [2^kc] lexicographic column of a mask among sets of its size */
    uint32_t *masks[MAXK + 1]; /* masks[t][i] = the i-th t-set */
    int64_t count[MAXK + 1];
} colsets_t;

static void lex_fill(colsets_t *cs, int t, int start, int left, uint32_t mask, int64_t *next) {
    if (left == 0) {
        cs->masks[t][*next] = mask;
        cs->index_of[mask] = (int32_t)*next;
        ++*next;
        return;
    }
    for (int c = start; c <= cs->kc - left; ++c) lex_fill(cs, t, c + 1, left - 1, mask | (1u << c), next);
}

static int colsets_init(colsets_t *cs, int kc, int tmax) {
    memset(cs, 0, sizeof *cs);
    cs->kc = kc;
    cs->index_of = (int32_t *)malloc(sizeof(int32_t) << kc);
    if (!cs->index_of) return ORACLE_NO_MEMORY;
    for (int t = 1; t <= tmax; ++t) {
        int64_t c = 1;
        for (int i = 0; i < t; ++i) c = c * (kc - i) / (i + 1);
        cs->count[t] = c;
        cs->masks[t] = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)c);
        if (!cs->masks[t]) return ORACLE_NO_MEMORY;
        int64_t next = 0;
        lex_fill(cs, t, 0, t, 0u, &next);
    }
    return ORACLE_OK;
}

static void colsets_free(colsets_t *cs) {
    free(cs->index_of);
    for (int t = 0; t <= MAXK; ++t) free(cs->masks[t]);
}

/* ----------------------------------------------------------------- the DP */

typedef struct {
    int64_t n;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const uint64_t *wint;     /* integer arc weights, or NULL for all ones */
    const int8_t *colours;
    const tree_t *T;
    colsets_t cs;
    int mode, cut;
    int overflow;
    int max_bits;             /* over every table the DP builds */
} dp_t;

static int table_bits(const big *M, int64_t entries) {
    int mb = 0;
#pragma omp parallel for reduction(max : mb) schedule(static)
    for (int64_t i = 0; i < entries; ++i) {
        int b = big_bits(&M[i]);
        if (b > mb) mb = b;
    }
    return mb;
}

static inline void arc_weight(const dp_t *D, int64_t e, big *w) { big_from_u64(w, D->wint ? D->wint[e] : 1u); }

/* Table of the sub-template rooted at x that keeps children [lo, hi) of x.
 * Rows are vertices, columns are colour sets of the sub-template's size. */
static big *dp_table(dp_t *D, int x, int lo, int hi, int *size_out) {
    const tree_t *T = D->T;
    int64_t n = D->n;
    if (lo == hi) {
        /* single vertex: M(i, {col i}) = 1 (Alg. 2, bottom sub-template) */
        int64_t cols = D->cs.count[1];
        big *L = (big *)calloc((size_t)(n * cols), sizeof(big));
        if (!L) return NULL;
        for (int64_t i = 0; i < n; ++i) big_from_u64(&L[i * cols + D->cs.index_of[1u << D->colours[i]]], 1);
        *size_out = 1;
        if (1 > D->max_bits) D->max_bits = 1;
        return L;
    }
    int tau, alo = lo, ahi = hi;
    if (D->cut == ORACLE_CUT_FIRST) {
        tau = T->child[x][lo];
        alo = lo + 1;
    } else {
        tau = T->child[x][hi - 1];
        ahi = hi - 1;
    }
    int a, p;
    big *Ma = dp_table(D, x, alo, ahi, &a);
    if (!Ma) return NULL;
    big *Mp = dp_table(D, tau, 0, T->nchild[tau], &p);
    if (!Mp) {
        free(Ma);
        return NULL;
    }
    int t = a + p;
    int64_t ca = D->cs.count[a], cp = D->cs.count[p], ct = D->cs.count[t];
    big *Ms = (big *)calloc((size_t)(n * ct), sizeof(big));
    if (!Ms) {
        free(Ma);
        free(Mp);
        return NULL;
    }
    int ovf = 0;
    if (D->mode == ORACLE_DECOUPLED) {
        /* stage 1: B(i, P) = sum over neighbours j of w_ij * M_p(j, P) */
        big *B = (big *)calloc((size_t)(n * cp), sizeof(big));
        if (!B) {
            free(Ma);
            free(Mp);
            free(Ms);
            return NULL;
        }
#pragma omp parallel for reduction(| : ovf) schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            big *Bi = &B[i * cp];
            for (int64_t e = D->row_ptr[i]; e < D->row_ptr[i + 1]; ++e) {
                int64_t j = D->col_idx[e];
                big w;
                arc_weight(D, e, &w);
                const big *Mj = &Mp[j * cp];
                for (int64_t c = 0; c < cp; ++c) ovf |= big_fma(&Bi[c], &w, &Mj[c]);
            }
        }
        int bb = table_bits(B, n * cp);
        if (bb > D->max_bits) D->max_bits = bb;
        /* stage 2: M_s(i, S) = sum over splits S = A + P of M_a(i, A) * B(i, P) */
#pragma omp parallel for reduction(| : ovf) schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t s = 0; s < ct; ++s) {
                uint32_t S = D->cs.masks[t][s];
                big acc;
                big_zero(&acc);
                for (uint32_t A = S;; A = (A - 1) & S) {
                    if (__builtin_popcount(A) == a) {
                        uint32_t P = S ^ A;
                        ovf |= big_fma(&acc, &Ma[i * ca + D->cs.index_of[A]], &B[i * cp + D->cs.index_of[P]]);
                    }
                    if (A == 0) break;
                }
                Ms[i * ct + s] = acc;
            }
        }
        free(B);
    } else {
        /* Alg. 2: the neighbour loop sits inside the split loop */
#pragma omp parallel for reduction(| : ovf) schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t s = 0; s < ct; ++s) {
                uint32_t S = D->cs.masks[t][s];
                big acc;
                big_zero(&acc);
                for (uint32_t A = S;; A = (A - 1) & S) {
                    if (__builtin_popcount(A) == a) {
                        uint32_t P = S ^ A;
                        const big *ma = &Ma[i * ca + D->cs.index_of[A]];
                        for (int64_t e = D->row_ptr[i]; e < D->row_ptr[i + 1]; ++e) {
                            int64_t j = D->col_idx[e];
                            big w, wm;
                            arc_weight(D, e, &w);
                            ovf |= big_mul(&wm, &w, &Mp[j * cp + D->cs.index_of[P]]);
                            ovf |= big_fma(&acc, ma, &wm);
                        }
                    }
                    if (A == 0) break;
                }
                Ms[i * ct + s] = acc;
            }
        }
    }
    free(Ma);
    free(Mp);
    if (ovf) D->overflow = 1;
    int mb = table_bits(Ms, n * ct);
    if (mb > D->max_bits) D->max_bits = mb;
    *size_out = t;
    return Ms;
}

static int check_graph(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const int8_t *colours, int kc) {
    if (n < 0 || !row_ptr || (n > 0 && (!col_idx || !colours))) return ORACLE_BAD_INPUT;
    if (row_ptr[0] != 0) return ORACLE_BAD_INPUT;
    for (int64_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return ORACLE_BAD_INPUT;
        if (colours[i] < 0 || colours[i] >= kc) return ORACLE_BAD_INPUT;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (col_idx[e] < 0 || col_idx[e] >= n) return ORACLE_BAD_INPUT;
    }
    return ORACLE_OK;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/*
 * Colourful-embedding counts by dynamic programming over the template
 * partition.
 *   k, parent, root : template (parent array with one -1), root rho
 *   kc              : number of colours, k <= kc <= 20
 *   colours         : [n] values in [0, kc)
 *   wint            : [nnz] integer arc weights (symmetric), or NULL
 *   per_vertex      : [n][NL] limbs, little-endian (may be NULL)
 *   total           : [NL] limbs
 *   max_bits        : bits of the largest entry of any table built
 * Returns ORACLE_OK, ORACLE_OVERFLOW (results invalid), or a negative error.
 */
int oracle_dp(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *wint, int k,
              const int32_t *parent, int root, int kc, const int8_t *colours, int mode, int cut, uint64_t *per_vertex,
              uint64_t *total, int32_t *max_bits, int nthreads) {
    if (kc < k || kc > 20 || k < 1) return ORACLE_BAD_INPUT;
    if (check_graph(n, row_ptr, col_idx, colours, kc)) return ORACLE_BAD_INPUT;
    tree_t T;
    if (tree_build(k, parent, root, &T)) return ORACLE_BAD_INPUT;
    set_threads(nthreads);
    dp_t D;
    memset(&D, 0, sizeof D);
    D.n = n;
    D.row_ptr = row_ptr;
    D.col_idx = col_idx;
    D.wint = wint;
    D.colours = colours;
    D.T = &T;
    D.mode = mode;
    D.cut = cut;
    if (colsets_init(&D.cs, kc, k)) {
        colsets_free(&D.cs);
        return ORACLE_NO_MEMORY;
    }
    int t;
    big *M0 = dp_table(&D, root, 0, T.nchild[root], &t);
    if (!M0) {
        colsets_free(&D.cs);
        return ORACLE_NO_MEMORY;
    }
    /* per_vertex[i] = sum over the columns of the root table (one column when kc = k) */
    int64_t c0 = D.cs.count[k];
    big tot;
    big_zero(&tot);
    int ovf = D.overflow;
    for (int64_t i = 0; i < n; ++i) {
        big s;
        big_zero(&s);
        for (int64_t c = 0; c < c0; ++c) ovf |= big_add(&s, &M0[i * c0 + c]);
        if (per_vertex) memcpy(&per_vertex[i * NL], s.w, sizeof s.w);
        ovf |= big_add(&tot, &s);
    }
    memcpy(total, tot.w, sizeof tot.w);
    if (max_bits) *max_bits = D.max_bits;
    free(M0);
    colsets_free(&D.cs);
    return ovf ? ORACLE_OVERFLOW : ORACLE_OK;
}

/* ----------------------------------------------------------- brute force */

typedef struct {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const uint64_t *wint;
    const int8_t *colours;
    int k, injective_only;
    int ord_par[MAXK];        /* position (in BFS order) of each template vertex's parent */
    int overflow;
} brute_t;

static void brute_rec(brute_t *Bt, int q, int32_t *phi, uint32_t used, const big *weight, big *acc) {
    if (q == Bt->k) {
        Bt->overflow |= big_add(acc, weight);
        return;
    }
    int32_t x = phi[Bt->ord_par[q]];
    for (int64_t e = Bt->row_ptr[x]; e < Bt->row_ptr[x + 1]; ++e) {
        int32_t y = Bt->col_idx[e];
        uint32_t bit = 0;
        if (Bt->injective_only) {
            int clash = 0;
            for (int r = 0; r < q; ++r) clash |= (phi[r] == y);
            if (clash) continue;
        } else {
            bit = 1u << Bt->colours[y];
            if (used & bit) continue; /* distinct colours imply distinct vertices */
        }
        phi[q] = y;
        big w, nw;
        big_from_u64(&w, Bt->wint ? Bt->wint[e] : 1u);
        Bt->overflow |= big_mul(&nw, weight, &w);
        brute_rec(Bt, q + 1, phi, used | bit, &nw, acc);
    }
}

/*
 * Enumerates every map phi of the template into G (template vertices taken in
 * breadth-first order from rho, each mapped to a neighbour of its parent's
 * image).  injective_only = 0: colourful maps (distinct colours);
 * injective_only = 1: maps with distinct vertices, colours ignored (used for
 * emb(T, G) and, with G = T, for the automorphism count).
 */
int oracle_brute(int64_t n, const int64_t *row_ptr, const int32_t *col_idx, const uint64_t *wint, int k,
                 const int32_t *parent, int root, int kc, const int8_t *colours, int injective_only,
                 uint64_t *per_vertex, uint64_t *total, int nthreads) {
    if (kc < k || kc > 32 || k < 1) return ORACLE_BAD_INPUT;
    if (check_graph(n, row_ptr, col_idx, colours, kc)) return ORACLE_BAD_INPUT;
    tree_t T;
    if (tree_build(k, parent, root, &T)) return ORACLE_BAD_INPUT;
    set_threads(nthreads);
    brute_t Bt;
    memset(&Bt, 0, sizeof Bt);
    Bt.row_ptr = row_ptr;
    Bt.col_idx = col_idx;
    Bt.wint = wint;
    Bt.colours = colours;
    Bt.k = k;
    Bt.injective_only = injective_only;
    int ord[MAXK], pos[MAXK], head = 0, tail = 0;
    ord[tail++] = root;
    while (head < tail) {
        int x = ord[head++];
        for (int j = 0; j < T.nchild[x]; ++j) ord[tail++] = T.child[x][j];
    }
    for (int q = 0; q < k; ++q) pos[ord[q]] = q;
    Bt.ord_par[0] = -1;
    for (int q = 1; q < k; ++q) Bt.ord_par[q] = pos[T.par[ord[q]]];
    big tot;
    big_zero(&tot);
    int ovf = 0;
#pragma omp parallel
    {
        brute_t local = Bt;
        big mytot;
        big_zero(&mytot);
#pragma omp for schedule(dynamic, 1)
        for (int64_t v = 0; v < n; ++v) {
            int32_t phi[MAXK];
            phi[0] = (int32_t)v;
            big acc, one;
            big_zero(&acc);
            big_from_u64(&one, 1);
            uint32_t used = injective_only ? 0u : (1u << colours[v]);
            brute_rec(&local, 1, phi, used, &one, &acc);
            if (per_vertex) memcpy(&per_vertex[v * NL], acc.w, sizeof acc.w);
            local.overflow |= big_add(&mytot, &acc);
        }
#pragma omp critical
        {
            ovf |= local.overflow;
            ovf |= big_add(&tot, &mytot);
        }
    }
    memcpy(total, tot.w, sizeof tot.w);
    return ovf ? ORACLE_OVERFLOW : ORACLE_OK;
}

/* number of 64-bit limbs of this build */
int oracle_limbs(void) { return NL; }

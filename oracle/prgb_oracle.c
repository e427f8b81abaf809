/*
 * prgb_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * componentwise PageRank method of Engstrom & Silvestrov, "Graph partitioning
 * and a componentwise PageRank algorithm" (arXiv 1609.09068).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (every function cites the passage it follows):
 *   oracle_partition     SCC/CAC partition with levels: the modified Tarjan
 *                        DFS of Sec. 4.1 (Discover / Explore / Finish) with a
 *                        merge-find structure, then the canonical relabel.
 *   oracle_solve_cw      componentwise PageRank step of Sec. 4.3: levels from
 *                        the highest down; 1-vertex components copy W, CACs
 *                        use the CAC-PageRank BFS of Sec. 4.3.1, SCCs use the
 *                        power series of Sec. 4.3.2 (or dense LU below a size
 *                        threshold, Sec. 4.3 item 3), then the weight update
 *                        of Eq. (PR:levels).
 *   oracle_solve_global  the same power series on the whole graph (the
 *                        baseline method, end of Sec. 4.3.2).
 *   oracle_residual_l1   || u + c A^T (R/outdeg) - R ||_1, the defining system
 *                        (I - cA^T) R = W of Def. 3.5 / Sec. 4.3 item 3.
 *   oracle_dense_solve   Gaussian elimination with partial pivoting of the
 *                        same system (Sec. 4.3 item 3 names LU).
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *   - Self-loops are ignored everywhere (Sec. 4.1 first paragraph, Sec. 5.2
 *     "any loops in the graph where ignored"); they count neither in the
 *     partition nor in outdeg.  A_ij = 1/outdeg(i) for each edge i->j
 *     (Def. 3.4: rows of A sum to one); dangling rows are zero.
 *   - Levels are 0-based as in Def. 3.3 and Fig. 1; the DFS initialises
 *     v.level to 1, which is the same quantity plus one, so one is
 *     subtracted when the result is returned.
 *   - In Finish the merge flag m and the list are initialised once, before
 *     the loop over out-edges (the printed listing re-initialises them inside
 *     the loop, which would forget all but the last edge).
 *   - The CAC BFS enqueues the out-neighbour u whose in-degree reaches zero
 *     (the printed listing tests and enqueues w, the vertex being dequeued).
 *   - The labelling counter starts once before the loop over vertices.
 *   - The power series for SCCs applies c A^T (A row-normalised), i.e.
 *     P_{n+1,i} = sum_{j -> i} c P_{n,j} / outdeg(j); the listing writes cA
 *     and M*mr with M the transposed Google matrix.  Eq. (PR:levels) is read
 *     as the same transposed product.
 *   - Stopping rule: PR_NORM_LINF is the paper's "while max(mr) >= tol";
 *     PR_NORM_L1 stops after adding an increment P with ||P||_1 <= tau_C,
 *     where tau_C = tol * |C| / |V| (the paper is silent on how a global
 *     tolerance splits over components; this budget sums to tol).  At least
 *     one iteration is always done (do-while in Sec. 4.3.2).
 *   - Canonical component ids: sorted by level descending, then size
 *     descending (Sec. 4.2), then smallest vertex id ascending (the paper is
 *     silent on ties).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENOCONV 4

#define NORM_L1 0
#define NORM_LINF 1

#define TYPE_CAC 0
#define TYPE_SCC 1

/* ------------------------------------------------------------------------ */
/* Graph model: loop-free out-adjacency, out-degree, in-adjacency.           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n;
    int64_t m;          /* loop-free edge count */
    int64_t *optr;      /* [n+1] out-edges, targets ascending */
    int32_t *oidx;
    int64_t *iptr;      /* [n+1] in-edges, sources ascending */
    int32_t *iidx;
    int32_t *outdeg;    /* loop-free out-degree */
} graph_t;

static void graph_free(graph_t *g) {
    free(g->optr); free(g->oidx); free(g->iptr); free(g->iidx); free(g->outdeg);
    memset(g, 0, sizeof(*g));
}

/* Sec. 3 (simple digraph) and Sec. 4.1 / 5.2 (loops ignored). */
static int graph_build(int32_t n, const int32_t *rowptr, const int32_t *col, graph_t *g) {
    memset(g, 0, sizeof(*g));
    if (n < 0) return OR_EINVAL;
    g->n = n;
    if (n > 0 && rowptr[0] != 0) return OR_EINVAL;
    int64_t m = 0;
    for (int32_t i = 0; i < n; i++) {
        if (rowptr[i + 1] < rowptr[i]) return OR_EINVAL;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            if (col[e] < 0 || col[e] >= n) return OR_EINVAL;
            if (e > rowptr[i] && col[e] <= col[e - 1]) return OR_EINVAL;
            if (col[e] != i) m++;
        }
    }
    g->m = m;
    g->optr = calloc((size_t)n + 1, sizeof(int64_t));
    g->iptr = calloc((size_t)n + 1, sizeof(int64_t));
    g->oidx = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    g->iidx = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    g->outdeg = calloc((size_t)n + 1, sizeof(int32_t));
    if (!g->optr || !g->iptr || !g->oidx || !g->iidx || !g->outdeg) { graph_free(g); return OR_ENOMEM; }
    int64_t k = 0;
    for (int32_t i = 0; i < n; i++) {
        g->optr[i] = k;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++)
            if (col[e] != i) g->oidx[k++] = col[e];
        g->outdeg[i] = (int32_t)(k - g->optr[i]);
    }
    g->optr[n] = k;
    /* in-adjacency by counting sort over sources in ascending order */
    for (int64_t e = 0; e < m; e++) g->iptr[g->oidx[e] + 1]++;
    for (int32_t i = 0; i < n; i++) g->iptr[i + 1] += g->iptr[i];
    int64_t *fill = malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!fill) { graph_free(g); return OR_ENOMEM; }
    memcpy(fill, g->iptr, ((size_t)n + 1) * sizeof(int64_t));
    for (int32_t i = 0; i < n; i++)
        for (int64_t e = g->optr[i]; e < g->optr[i + 1]; e++)
            g->iidx[fill[g->oidx[e]]++] = i;
    free(fill);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1: component finding by a modified Tarjan DFS.                      */
/* ------------------------------------------------------------------------ */

/* merge-find on the .lowlink (parent) and .depth (rank) fields, Sec. 4.1.
 * The paper stores the parent in .lowlink once a vertex has left the stack;
 * here the parent gets its own array so that the Tarjan lowlink stays an
 * index throughout. */
static int32_t uf_find(int32_t *parent, int32_t x) {
    int32_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) { int32_t nx = parent[x]; parent[x] = r; x = nx; }
    return r;
}

static void uf_merge(int32_t *parent, int32_t *depth, int32_t a, int32_t b) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return;
    if (depth[a] < depth[b]) { int32_t t = a; a = b; b = t; }
    parent[b] = a;
    if (depth[a] == depth[b]) depth[a]++;
}

typedef struct { int32_t v; int64_t e; int returning; } frame_t;

/* Canonical relabel shared by both partition modes: components sorted by
 * level desc, size desc, smallest vertex asc (Sec. 4.2 + tie-break). */
typedef struct { int32_t level, size, minv, head; } ckey_t;

static int ckey_cmp(const void *pa, const void *pb) {
    const ckey_t *a = pa, *b = pb;
    if (a->level != b->level) return a->level > b->level ? -1 : 1;
    if (a->size != b->size) return a->size > b->size ? -1 : 1;
    return (a->minv < b->minv) ? -1 : (a->minv > b->minv);
}

/*
 * oracle_partition: Sec. 4.1 Discover / Explore / Finish, iterative (Sec. 5
 * says the implementation is iterative so deep graphs do not overflow).
 * merge = 0 gives the plain SCC partition with SCC-only levels (the vertex
 * labels of Fig. 1); merge = 1 gives the SCC/CAC partition of Theorem 3.1.
 * Outputs are canonical: comp[v] in [0, n_comp), type[v] (0 CAC, 1 SCC),
 * level[v] (0-based).
 */
int oracle_partition(int32_t n, const int32_t *rowptr, const int32_t *col, int merge,
                     int32_t *comp, uint8_t *type, int32_t *level,
                     int32_t *n_comp, int32_t *n_levels) {
    graph_t g;
    int rc = graph_build(n, rowptr, col, &g);
    if (rc) return rc;
    *n_comp = 0; *n_levels = 0;
    if (n == 0) { graph_free(&g); return OR_OK; }
    int32_t *index = malloc((size_t)n * sizeof(int32_t));
    int32_t *lowlink = malloc((size_t)n * sizeof(int32_t));
    int32_t *lvl = malloc((size_t)n * sizeof(int32_t));
    int32_t *depth = malloc((size_t)n * sizeof(int32_t));
    int32_t *parent = malloc((size_t)n * sizeof(int32_t));
    int8_t *vtype = malloc((size_t)n);         /* -1 = not yet in a component */
    int32_t *stack = malloc((size_t)n * sizeof(int32_t));
    frame_t *frames = malloc((size_t)n * sizeof(frame_t));
    int32_t *list = malloc((size_t)n * sizeof(int32_t));
    if (!index || !lowlink || !lvl || !depth || !parent || !vtype || !stack || !frames || !list) {
        rc = OR_ENOMEM; goto done;
    }
    for (int32_t i = 0; i < n; i++) { index[i] = -1; vtype[i] = -1; parent[i] = i; depth[i] = 1; }
    int32_t counter = 1, sp = 0, fp = 0;

    for (int32_t root = 0; root < n; root++) {
        if (index[root] >= 0) continue;
        /* Discover(root) */
        index[root] = lowlink[root] = counter++;
        lvl[root] = 1; depth[root] = 1;
        stack[sp++] = root;
        frames[fp].v = root; frames[fp].e = g.optr[root]; frames[fp].returning = 0; fp++;
        while (fp > 0) {
            frame_t *f = &frames[fp - 1];
            int32_t v = f->v;
            if (f->e < g.optr[v + 1]) {
                /* Explore(v): one out-edge (v, w) at a time */
                int32_t w = g.oidx[f->e];
                if (!f->returning && index[w] < 0) {
                    /* w not initialised: DFS(w) = Discover, Explore, Finish */
                    f->returning = 1;
                    index[w] = lowlink[w] = counter++;
                    lvl[w] = 1; depth[w] = 1;
                    stack[sp++] = w;
                    frames[fp].v = w; frames[fp].e = g.optr[w]; frames[fp].returning = 0; fp++;
                    continue;
                }
                /* w is in a component, or on the stack in v's SCC */
                if (vtype[w] >= 0) {
                    if (lvl[w] + 1 > lvl[v]) lvl[v] = lvl[w] + 1;
                } else {
                    if (lvl[w] > lvl[v]) lvl[v] = lvl[w];
                    if (lowlink[w] < lowlink[v]) lowlink[v] = lowlink[w];
                }
                f->returning = 0;
                f->e++;
                continue;
            }
            /* Finish(v) */
            if (lowlink[v] == index[v]) {
                int32_t size = 0, w;
                do {
                    w = stack[--sp];
                    parent[w] = v;          /* w.lowlink := v ; merge(w, v) */
                    lvl[w] = lvl[v];
                    vtype[w] = TYPE_SCC;
                    size++;
                } while (w != v);
                if (size > 1) depth[v] = 2;
                if (size == 1) {
                    vtype[v] = TYPE_CAC;
                    if (merge) {
                        /* check for merges with v as head (Theorem 3.1) */
                        int m = 0, nl = 0;
                        for (int64_t e = g.optr[v]; e < g.optr[v + 1]; e++) {
                            int32_t x = g.oidx[e];
                            if (vtype[x] == TYPE_SCC && lvl[x] == lvl[v] - 1) { m = 0; break; }
                            if (vtype[x] == TYPE_CAC && lvl[x] == lvl[v] - 1) { list[nl++] = x; m = 1; }
                        }
                        if (m) {
                            lvl[v] = lvl[v] - 1;
                            for (int i = 0; i < nl; i++) uf_merge(parent, depth, list[i], v);
                        }
                    }
                }
            }
            fp--;
        }
    }

    /* labelling by find (Sec. 4.1, last listing), then canonical order */
    {
        int32_t *headcomp = malloc((size_t)n * sizeof(int32_t));
        ckey_t *keys = malloc((size_t)n * sizeof(ckey_t));
        int32_t *rank = malloc((size_t)n * sizeof(int32_t));
        if (!headcomp || !keys || !rank) { free(headcomp); free(keys); free(rank); rc = OR_ENOMEM; goto done; }
        int32_t ind = 0;
        for (int32_t v = 0; v < n; v++) headcomp[v] = -1;
        for (int32_t v = 0; v < n; v++) {
            int32_t h = uf_find(parent, v);
            if (headcomp[h] < 0) {
                headcomp[h] = ind;
                keys[ind].level = lvl[h] - 1;   /* 0-based level */
                keys[ind].size = 0;
                keys[ind].minv = v;             /* first v seen is the smallest */
                keys[ind].head = ind;
                ind++;
            }
            comp[v] = headcomp[h];
            keys[comp[v]].size++;
        }
        qsort(keys, (size_t)ind, sizeof(ckey_t), ckey_cmp);
        for (int32_t k = 0; k < ind; k++) rank[keys[k].head] = k;
        int32_t maxl = -1;
        for (int32_t v = 0; v < n; v++) {
            int32_t h = uf_find(parent, v);
            comp[v] = rank[comp[v]];
            level[v] = lvl[h] - 1;
            type[v] = (uint8_t)vtype[v];
            if (level[v] > maxl) maxl = level[v];
        }
        *n_comp = ind;
        *n_levels = maxl + 1;
        free(headcomp); free(keys); free(rank);
    }
done:
    free(index); free(lowlink); free(lvl); free(depth); free(parent); free(vtype);
    free(stack); free(frames); free(list);
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Dense solve of (I - c A_C^T) R = W_C (Sec. 4.3 item 3: "LU factorization"). */
/* ------------------------------------------------------------------------ */

/* Solve M x = b in place (M row-major k x k) by Gaussian elimination with
 * partial pivoting; returns OR_EINVAL for a singular pivot. */
static int gauss_solve(int32_t k, double *M, double *b) {
    for (int32_t col = 0; col < k; col++) {
        int32_t piv = col;
        double best = fabs(M[(size_t)col * k + col]);
        for (int32_t r = col + 1; r < k; r++) {
            double a = fabs(M[(size_t)r * k + col]);
            if (a > best) { best = a; piv = r; }
        }
        if (best == 0.0) return OR_EINVAL;
        if (piv != col) {
            for (int32_t j = 0; j < k; j++) {
                double t = M[(size_t)col * k + j];
                M[(size_t)col * k + j] = M[(size_t)piv * k + j];
                M[(size_t)piv * k + j] = t;
            }
            double t = b[col]; b[col] = b[piv]; b[piv] = t;
        }
        for (int32_t r = col + 1; r < k; r++) {
            double f = M[(size_t)r * k + col] / M[(size_t)col * k + col];
            if (f == 0.0) continue;
            for (int32_t j = col; j < k; j++) M[(size_t)r * k + j] -= f * M[(size_t)col * k + j];
            b[r] -= f * b[col];
        }
    }
    for (int32_t r = k - 1; r >= 0; r--) {
        double s = b[r];
        for (int32_t j = r + 1; j < k; j++) s -= M[(size_t)r * k + j] * b[j];
        b[r] = s / M[(size_t)r * k + r];
    }
    return OR_OK;
}

/* Dense (I - cA^T) R = u on the whole graph (Def. 3.5 with W = u). */
int oracle_dense_solve(int32_t n, const int32_t *rowptr, const int32_t *col,
                       double c, const double *u, double *R) {
    graph_t g;
    int rc = graph_build(n, rowptr, col, &g);
    if (rc) return rc;
    double *M = calloc((size_t)n * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (!M) { graph_free(&g); return OR_ENOMEM; }
    for (int32_t i = 0; i < n; i++) M[(size_t)i * n + i] = 1.0;
    /* row i of (I - cA^T): -c A_ji = -c / outdeg(j) for each edge j -> i */
    for (int32_t j = 0; j < n; j++)
        for (int64_t e = g.optr[j]; e < g.optr[j + 1]; e++)
            M[(size_t)g.oidx[e] * n + j] -= c / (double)g.outdeg[j];
    for (int32_t i = 0; i < n; i++) R[i] = u[i];
    rc = gauss_solve(n, M, R);
    free(M);
    graph_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.3: PageRank step, level by level.                                   */
/* ------------------------------------------------------------------------ */

static double vec_norm(const double *p, int64_t k, int norm) {
    double s = 0.0;
    if (norm == NORM_LINF) {
        for (int64_t i = 0; i < k; i++) if (p[i] > s) s = p[i];
    } else {
        for (int64_t i = 0; i < k; i++) s += fabs(p[i]);
    }
    return s;
}

/* continue the series?  L_inf: the paper's "while max(mr) >= tol";
 * L1: continue while ||P||_1 > tau. */
static int keep_going(double s, double tau, int norm) {
    return norm == NORM_LINF ? (s >= tau) : (s > tau);
}

/*
 * oracle_solve_cw: Sec. 4.3 steps 1-4.  comp/type/level come from
 * oracle_partition (canonical ids, so components of one level are
 * consecutive and in size-descending order).  replay_iters, when non-NULL,
 * fixes the number of power-series iterations of each SCC component
 * (indexed by component id) instead of the stopping rule.
 */
int oracle_solve_cw(int32_t n, const int32_t *rowptr, const int32_t *col,
                    const int32_t *comp, const uint8_t *type, const int32_t *level,
                    int32_t n_comp, double c, const double *u, double tol, int norm,
                    int32_t max_iter, int32_t lu_threshold, const int32_t *replay_iters,
                    double *R, int32_t *comp_iters) {
    graph_t g;
    int rc = graph_build(n, rowptr, col, &g);
    if (rc) return rc;
    if (!(c > 0.0 && c < 1.0) || !(tol > 0.0)) { graph_free(&g); return OR_EINVAL; }
    int32_t *cstart = calloc((size_t)n_comp + 1, sizeof(int32_t));
    int32_t *members = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *local = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    double *W = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *P = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *Pn = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int32_t *deg = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *queue = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!cstart || !members || !local || !W || !P || !Pn || !deg || !queue) { rc = OR_ENOMEM; goto done; }

    /* members of each component in ascending vertex id */
    for (int32_t v = 0; v < n; v++) cstart[comp[v] + 1]++;
    for (int32_t k = 0; k < n_comp; k++) cstart[k + 1] += cstart[k];
    {
        int32_t *fill = malloc(((size_t)n_comp + 1) * sizeof(int32_t));
        if (!fill) { rc = OR_ENOMEM; goto done; }
        memcpy(fill, cstart, ((size_t)n_comp + 1) * sizeof(int32_t));
        for (int32_t v = 0; v < n; v++) members[fill[comp[v]]++] = v;
        free(fill);
    }
    for (int32_t v = 0; v < n; v++) { W[v] = u[v]; R[v] = 0.0; }
    for (int32_t k = 0; k < n_comp; k++) if (comp_iters) comp_iters[k] = 0;

    /* Step 1: L = max level.  Canonical ids run from the highest level down. */
    int32_t k0 = 0;
    while (k0 < n_comp) {
        int32_t L = level[members[cstart[k0]]];
        int32_t k1 = k0;
        while (k1 < n_comp && level[members[cstart[k1]]] == L) k1++;

        /* Step 2: each component of level L by its type and size */
        for (int32_t k = k0; k < k1; k++) {
            const int32_t *mem = members + cstart[k];
            int32_t sz = cstart[k + 1] - cstart[k];
            int32_t t = type[mem[0]];
            if (sz == 1) {
                /* collection of 1-vertex components: R = w (no loops) */
                R[mem[0]] = W[mem[0]];
            } else if (t == TYPE_CAC) {
                /* Sec. 4.3.1 CAC-PageRank: BFS that enqueues a vertex once all
                 * its incoming (internal) edges have been used. */
                for (int32_t i = 0; i < sz; i++) {
                    int32_t v = mem[i], d = 0;
                    for (int64_t e = g.iptr[v]; e < g.iptr[v + 1]; e++)
                        if (comp[g.iidx[e]] == k) d++;
                    deg[v] = d;
                    R[v] = W[v];              /* v.rank := w_v */
                }
                for (int32_t i = 0; i < sz; i++) {
                    int32_t v = mem[i];
                    if (deg[v] != 0) continue;
                    int32_t qh = 0, qt = 0;
                    queue[qt++] = v;
                    while (qt > qh) {
                        int32_t w = queue[qh++];
                        /* loop factor 1/(1 - W(w,w)) = 1: loops are ignored */
                        for (int64_t e = g.optr[w]; e < g.optr[w + 1]; e++) {
                            int32_t x = g.oidx[e];
                            if (comp[x] != k) continue;
                            R[x] = R[x] + R[w] * (c / (double)g.outdeg[w]);
                            deg[x] = deg[x] - 1;
                            if (deg[x] == 0) queue[qt++] = x;
                        }
                        deg[w] = deg[w] - 1;  /* never enqueue w again */
                    }
                }
            } else if (lu_threshold > 0 && sz < lu_threshold) {
                /* Sec. 4.3 item 3: small SCC, solve (I - cA_C^T) R = W_C */
                double *M = calloc((size_t)sz * sz, sizeof(double));
                double *b = malloc((size_t)sz * sizeof(double));
                if (!M || !b) { free(M); free(b); rc = OR_ENOMEM; goto done; }
                for (int32_t i = 0; i < sz; i++) { local[mem[i]] = i; M[(size_t)i * sz + i] = 1.0; b[i] = W[mem[i]]; }
                for (int32_t j = 0; j < sz; j++) {
                    int32_t vj = mem[j];
                    for (int64_t e = g.optr[vj]; e < g.optr[vj + 1]; e++) {
                        int32_t x = g.oidx[e];
                        if (comp[x] == k) M[(size_t)local[x] * sz + j] -= c / (double)g.outdeg[vj];
                    }
                }
                int r2 = gauss_solve(sz, M, b);
                for (int32_t i = 0; i < sz; i++) R[mem[i]] = b[i];
                free(M); free(b);
                if (r2) { rc = r2; goto done; }
            } else {
                /* Sec. 4.3.2: P_0 = W, P_{n+1} = c A^T P_n, R = sum_k P_k */
                double tau = (norm == NORM_LINF) ? tol : tol * (double)sz / (double)n;
                for (int32_t i = 0; i < sz; i++) { local[mem[i]] = i; P[i] = W[mem[i]]; R[mem[i]] = W[mem[i]]; }
                int32_t it = 0;
                int32_t fixed = replay_iters ? replay_iters[k] : -1;
                for (;;) {
                    for (int32_t i = 0; i < sz; i++) {
                        int32_t vi = mem[i];
                        double s = 0.0;
                        for (int64_t e = g.iptr[vi]; e < g.iptr[vi + 1]; e++) {
                            int32_t j = g.iidx[e];
                            if (comp[j] == k) s += P[local[j]] / (double)g.outdeg[j];
                        }
                        Pn[i] = c * s;
                    }
                    for (int32_t i = 0; i < sz; i++) { P[i] = Pn[i]; R[mem[i]] += P[i]; }
                    it++;
                    if (fixed >= 0) { if (it >= fixed) break; continue; }
                    if (!keep_going(vec_norm(P, sz, norm), tau, norm)) break;
                    if (it >= max_iter) { rc = OR_ENOCONV; break; }
                }
                if (comp_iters) comp_iters[k] = it;
            }
        }

        /* Step 3, Eq. (PR:levels): W_i += c R_j / outdeg(j) for every edge
         * j -> i from level L into a lower level. */
        for (int32_t k = k0; k < k1; k++) {
            for (int32_t q = cstart[k]; q < cstart[k + 1]; q++) {
                int32_t j = members[q];
                for (int64_t e = g.optr[j]; e < g.optr[j + 1]; e++) {
                    int32_t i = g.oidx[e];
                    if (level[i] < L) W[i] += c * R[j] / (double)g.outdeg[j];
                }
            }
        }
        /* Step 4: next level down */
        k0 = k1;
    }
done:
    free(cstart); free(members); free(local); free(W); free(P); free(Pn); free(deg); free(queue);
    graph_free(&g);
    return rc;
}

/* The baseline: the Sec. 4.3.2 series on the whole graph with tau = tol. */
int oracle_solve_global(int32_t n, const int32_t *rowptr, const int32_t *col,
                        double c, const double *u, double tol, int norm, int32_t max_iter,
                        int32_t replay_iters, double *R, int32_t *iters) {
    graph_t g;
    int rc = graph_build(n, rowptr, col, &g);
    if (rc) return rc;
    if (!(c > 0.0 && c < 1.0) || !(tol > 0.0)) { graph_free(&g); return OR_EINVAL; }
    double *P = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *Pn = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!P || !Pn) { free(P); free(Pn); graph_free(&g); return OR_ENOMEM; }
    for (int32_t i = 0; i < n; i++) { P[i] = u[i]; R[i] = u[i]; }
    int32_t it = 0;
    for (;;) {
        for (int32_t i = 0; i < n; i++) {
            double s = 0.0;
            for (int64_t e = g.iptr[i]; e < g.iptr[i + 1]; e++) {
                int32_t j = g.iidx[e];
                s += P[j] / (double)g.outdeg[j];
            }
            Pn[i] = c * s;
        }
        for (int32_t i = 0; i < n; i++) { P[i] = Pn[i]; R[i] += P[i]; }
        it++;
        if (replay_iters >= 0) { if (it >= replay_iters) break; continue; }
        if (!keep_going(vec_norm(P, n, norm), tol, norm)) break;
        if (it >= max_iter) { rc = OR_ENOCONV; break; }
    }
    *iters = it;
    free(P); free(Pn);
    graph_free(&g);
    return rc;
}

/* || u + c A^T (R / outdeg) - R ||_1 : the residual of (I - cA^T) R = u. */
double oracle_residual_l1(int32_t n, const int32_t *rowptr, const int32_t *col,
                          double c, const double *u, const double *R) {
    graph_t g;
    if (graph_build(n, rowptr, col, &g)) return -1.0;
    double tot = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t e = g.iptr[i]; e < g.iptr[i + 1]; e++) {
            int32_t j = g.iidx[e];
            s += R[j] / (double)g.outdeg[j];
        }
        tot += fabs(u[i] + c * s - R[i]);
    }
    graph_free(&g);
    return tot;
}

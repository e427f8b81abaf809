/*
 * prgb_cpu_parallel.c -- the multi-core CPU baseline: the componentwise
 * PageRank step (Sec. 4.3) and the global power series (Sec. 4.3.2 applied to
 * the whole graph), parallelised with OpenMP over the host's cores.
 *
 * It exists to be timed next to the GPU path, in the spirit of the paper's
 * own parallel implementation (Sec. 5.2, components of a level solved
 * concurrently on the CPU's cores).  It is neither the oracle nor part of the
 * GPU path: it takes the partition (component id, type, level per vertex,
 * canonical ids) as input and shares no code with either.
 *
 * Problem: R = u + c A^T R with A_ij = 1/outdeg(i) (self-loops ignored,
 * dangling rows zero).  z = c R / outdeg is the only gathered vector.
 *
 *   cw:     levels from the highest down (canonical ids put a level's
 *           components next to each other, size-descending).  Per level:
 *           W = u + (sum of z over external in-edges) for every vertex of the
 *           level, in parallel; then every component: a 1-vertex component
 *           takes R = W, a CAC one pass in topological order (Sec. 4.3.1), an
 *           SCC the series P_0 = W, P_{k+1} = c A_C^T P_k, R = sum P_k until
 *           ||P||_1 <= tol |C| / n (Sec. 4.3.2).  Components of at least
 *           `big` vertices run one at a time with their sweeps spread over
 *           all threads; the others are spread over the threads one
 *           component each (dynamic schedule, largest first).
 *   global: the same series on the whole graph until ||P||_1 <= tol, sweeps
 *           spread over all threads.
 *
 * Build: gcc -O3 -fopenmp -shared -fPIC.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { CPB_OK = 0, CPB_EINVAL = 1, CPB_ENOMEM = 2, CPB_ENOCONV = 3 };

typedef struct cpb_plan {
    int32_t n, n_comp, n_lev;
    double *inv;      /* [n] 1/outdeg by position (0 for dangling) */
    int32_t *perm;    /* [n] position -> vertex */
    int32_t *pos;     /* [n] vertex -> position */
    int32_t *c_off;   /* [n_comp+1] first position of each component */
    uint8_t *c_type;  /* [n_comp] 1 = SCC, 0 = CAC */
    int32_t *l_comp;  /* [n_lev+1] first component of each level (solve order) */
    int32_t *int_ptr, *int_idx;  /* internal in-edges by position (source positions) */
    int32_t *ext_ptr, *ext_idx;  /* external in-edges by position */
    int32_t *all_ptr, *all_idx;  /* all in-edges by position (global series) */
} cpb_plan;

void cpb_plan_destroy(cpb_plan *P) {
    if (!P) return;
    free(P->inv); free(P->perm); free(P->pos); free(P->c_off); free(P->c_type); free(P->l_comp);
    free(P->int_ptr); free(P->int_idx); free(P->ext_ptr); free(P->ext_idx);
    free(P->all_ptr); free(P->all_idx);
    free(P);
}

/* Layout (untimed): positions ordered by component id, a CAC's members in
 * topological order (Kahn over its internal edges), an SCC's by vertex id. */
int cpb_plan_create(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *comp,
                    const uint8_t *type, const int32_t *level, int32_t n_comp, cpb_plan **out) {
    if (!out || n < 0 || n_comp < 0 || (n > 0 && (!rowptr || !col || !comp || !type || !level)))
        return CPB_EINVAL;
    *out = NULL;
    cpb_plan *P = calloc(1, sizeof(cpb_plan));
    if (!P) return CPB_ENOMEM;
    P->n = n;
    P->n_comp = n_comp;
    const size_t n1 = (size_t)n + 1, nn = n > 0 ? (size_t)n : 1;
    const int64_t m = n > 0 ? rowptr[n] : 0;
    int32_t *outdeg = calloc(nn, sizeof(int32_t));
    int32_t *iptr = calloc(n1, sizeof(int32_t));
    int32_t *iidx = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t *fill = malloc(n1 * sizeof(int32_t));
    int32_t *cnt = calloc((size_t)n_comp + 1, sizeof(int32_t));
    int32_t *deg = malloc(nn * sizeof(int32_t));
    int32_t *queue = malloc(nn * sizeof(int32_t));
    int rc = CPB_OK;
    P->inv = malloc(nn * sizeof(double));
    P->perm = malloc(nn * sizeof(int32_t));
    P->pos = malloc(nn * sizeof(int32_t));
    P->c_off = calloc((size_t)n_comp + 1, sizeof(int32_t));
    P->c_type = calloc((size_t)(n_comp > 0 ? n_comp : 1), 1);
    P->l_comp = malloc(((size_t)n_comp + 1) * sizeof(int32_t));
    P->int_ptr = calloc(n1, sizeof(int32_t));
    P->ext_ptr = calloc(n1, sizeof(int32_t));
    P->all_ptr = calloc(n1, sizeof(int32_t));
    if (!outdeg || !iptr || !iidx || !fill || !cnt || !deg || !queue || !P->inv || !P->perm || !P->pos ||
        !P->c_off || !P->c_type || !P->l_comp || !P->int_ptr || !P->ext_ptr || !P->all_ptr) {
        rc = CPB_ENOMEM;
        goto done;
    }
    /* loop-free in-CSC of the graph */
    for (int32_t v = 0; v < n; v++)
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
            const int32_t w = col[e];
            if (w < 0 || w >= n) { rc = CPB_EINVAL; goto done; }
            if (w == v) continue;
            outdeg[v]++;
            iptr[w + 1]++;
        }
    for (int32_t v = 0; v < n; v++) iptr[v + 1] += iptr[v];
    memcpy(fill, iptr, n1 * sizeof(int32_t));
    for (int32_t v = 0; v < n; v++)
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++)
            if (col[e] != v) iidx[fill[col[e]]++] = v;
    /* components: sizes, offsets, levels (canonical ids: levels descending) */
    for (int32_t v = 0; v < n; v++) {
        if (comp[v] < 0 || comp[v] >= n_comp) { rc = CPB_EINVAL; goto done; }
        cnt[comp[v] + 1]++;
    }
    for (int32_t k = 0; k < n_comp; k++) cnt[k + 1] += cnt[k];
    memcpy(P->c_off, cnt, ((size_t)n_comp + 1) * sizeof(int32_t));
    P->n_lev = 0;
    {
        int32_t prev = -1;
        /* the level of component k is the level of any member */
        int32_t *klev = malloc(((size_t)n_comp + 1) * sizeof(int32_t));
        if (!klev) { rc = CPB_ENOMEM; goto done; }
        for (int32_t v = 0; v < n; v++) {
            klev[comp[v]] = level[v];
            P->c_type[comp[v]] = type[v];
        }
        for (int32_t k = 0; k < n_comp; k++) {
            if (k > 0 && klev[k] > klev[k - 1]) { free(klev); rc = CPB_EINVAL; goto done; }
            if (klev[k] != prev) {
                P->l_comp[P->n_lev++] = k;
                prev = klev[k];
            }
        }
        P->l_comp[P->n_lev] = n_comp;
        free(klev);
    }
    /* positions: members by component; CAC members in topological order */
    memcpy(fill, cnt, ((size_t)n_comp + 1) * sizeof(int32_t));
    for (int32_t v = 0; v < n; v++) P->perm[fill[comp[v]]++] = v;
    for (int32_t k = 0; k < n_comp; k++) {
        const int32_t a = P->c_off[k], b = P->c_off[k + 1];
        if (P->c_type[k] == 1 || b - a < 2) continue;
        for (int32_t q = a; q < b; q++) {
            const int32_t v = P->perm[q];
            int32_t d = 0;
            for (int32_t e = iptr[v]; e < iptr[v + 1]; e++) d += comp[iidx[e]] == k;
            deg[v] = d;
        }
        int32_t qh = 0, qt = 0;
        for (int32_t q = a; q < b; q++)
            if (deg[P->perm[q]] == 0) queue[qt++] = P->perm[q];
        while (qh < qt) {
            const int32_t w = queue[qh++];
            for (int64_t e = rowptr[w]; e < rowptr[w + 1]; e++) {
                const int32_t x = col[e];
                if (x == w || comp[x] != k) continue;
                if (--deg[x] == 0) queue[qt++] = x;
            }
        }
        if (qt != b - a) { rc = CPB_EINVAL; goto done; } /* a cycle: not acyclic */
        memcpy(P->perm + a, queue, (size_t)qt * sizeof(int32_t));
    }
    for (int32_t p = 0; p < n; p++) P->pos[P->perm[p]] = p;
    for (int32_t p = 0; p < n; p++) {
        const int32_t v = P->perm[p];
        P->inv[p] = outdeg[v] > 0 ? 1.0 / (double)outdeg[v] : 0.0;
        int32_t ni = 0, ne = 0;
        for (int32_t e = iptr[v]; e < iptr[v + 1]; e++) {
            if (comp[iidx[e]] == comp[v]) ni++;
            else ne++;
        }
        P->int_ptr[p + 1] = ni;
        P->ext_ptr[p + 1] = ne;
        P->all_ptr[p + 1] = ni + ne;
    }
    for (int32_t p = 0; p < n; p++) {
        P->int_ptr[p + 1] += P->int_ptr[p];
        P->ext_ptr[p + 1] += P->ext_ptr[p];
        P->all_ptr[p + 1] += P->all_ptr[p];
    }
    P->int_idx = malloc((size_t)(P->int_ptr[n] > 0 ? P->int_ptr[n] : 1) * sizeof(int32_t));
    P->ext_idx = malloc((size_t)(P->ext_ptr[n] > 0 ? P->ext_ptr[n] : 1) * sizeof(int32_t));
    P->all_idx = malloc((size_t)(P->all_ptr[n] > 0 ? P->all_ptr[n] : 1) * sizeof(int32_t));
    if (!P->int_idx || !P->ext_idx || !P->all_idx) { rc = CPB_ENOMEM; goto done; }
    for (int32_t p = 0; p < n; p++) {
        const int32_t v = P->perm[p];
        int32_t oi = P->int_ptr[p], oe = P->ext_ptr[p], oa = P->all_ptr[p];
        for (int32_t e = iptr[v]; e < iptr[v + 1]; e++) {
            const int32_t j = iidx[e], q = P->pos[j];
            if (comp[j] == comp[v]) P->int_idx[oi++] = q;
            else P->ext_idx[oe++] = q;
            P->all_idx[oa++] = q;
        }
    }
done:
    free(outdeg); free(iptr); free(iidx); free(fill); free(cnt); free(deg); free(queue);
    if (rc) { cpb_plan_destroy(P); return rc; }
    *out = P;
    return CPB_OK;
}

/* one SCC's series, serial: positions [a, b), W in R on entry */
static int32_t scc_serial(const cpb_plan *P, int32_t a, int32_t b, double c, double tau, int32_t max_iter,
                          double *R, double *z0, double *z1, int *noconv) {
    for (int32_t p = a; p < b; p++) z0[p] = c * R[p] * P->inv[p];
    double *zc = z0, *zn = z1;
    int32_t it = 0;
    for (;;) {
        double s = 0.0;
        for (int32_t p = a; p < b; p++) {
            double acc = 0.0;
            for (int32_t e = P->int_ptr[p]; e < P->int_ptr[p + 1]; e++) acc += zc[P->int_idx[e]];
            R[p] += acc;
            zn[p] = c * acc * P->inv[p];
            s += fabs(acc);
        }
        double *t = zc; zc = zn; zn = t;
        it++;
        if (!(s > tau)) break;
        if (it >= max_iter) { *noconv = 1; break; }
    }
    return it;
}

/* the same with the sweep spread over the threads */
static int32_t scc_parallel(const cpb_plan *P, int32_t a, int32_t b, double c, double tau, int32_t max_iter,
                            double *R, double *z0, double *z1, int *noconv) {
#pragma omp parallel for schedule(static)
    for (int32_t p = a; p < b; p++) z0[p] = c * R[p] * P->inv[p];
    double *zc = z0, *zn = z1;
    int32_t it = 0;
    for (;;) {
        double s = 0.0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : s)
        for (int32_t p = a; p < b; p++) {
            double acc = 0.0;
            for (int32_t e = P->int_ptr[p]; e < P->int_ptr[p + 1]; e++) acc += zc[P->int_idx[e]];
            R[p] += acc;
            zn[p] = c * acc * P->inv[p];
            s += fabs(acc);
        }
        double *t = zc; zc = zn; zn = t;
        it++;
        if (!(s > tau)) break;
        if (it >= max_iter) { *noconv = 1; break; }
    }
    return it;
}

/* one CAC's pass: positions in topological order, W in R on entry */
static void cac_pass(const cpb_plan *P, int32_t a, int32_t b, double c, double *R, double *zr) {
    for (int32_t p = a; p < b; p++) {
        double acc = 0.0;
        for (int32_t e = P->int_ptr[p]; e < P->int_ptr[p + 1]; e++) acc += zr[P->int_idx[e]];
        R[p] += acc;
        zr[p] = c * R[p] * P->inv[p];
    }
}

/* R (original vertex order) of the componentwise step; iters_max: the
 * largest number of sweeps of any SCC.  threads <= 0: OpenMP's default. */
int cpb_solve_cw(const cpb_plan *P, double c, const double *u, double tol, int32_t max_iter, int32_t threads,
                 int32_t big, double *R_out, int32_t *iters_max) {
    if (!P || !(c > 0.0 && c < 1.0) || !(tol > 0.0) || max_iter < 1 || (P->n > 0 && (!u || !R_out)))
        return CPB_EINVAL;
    if (threads > 0) omp_set_num_threads(threads);
    const int32_t n = P->n;
    const size_t nn = n > 0 ? (size_t)n : 1;
    double *R = malloc(nn * sizeof(double)), *zr = malloc(nn * sizeof(double));
    double *z0 = malloc(nn * sizeof(double)), *z1 = malloc(nn * sizeof(double));
    if (!R || !zr || !z0 || !z1) { free(R); free(zr); free(z0); free(z1); return CPB_ENOMEM; }
    int noconv = 0;
    int32_t imax = 0;
    for (int32_t l = 0; l < P->n_lev; l++) {
        const int32_t k0 = P->l_comp[l], k1 = P->l_comp[l + 1];
        const int32_t p0 = P->c_off[k0], p1 = P->c_off[k1];
        /* W = u + inflow from the levels already solved */
#pragma omp parallel for schedule(static)
        for (int32_t p = p0; p < p1; p++) {
            double acc = 0.0;
            for (int32_t e = P->ext_ptr[p]; e < P->ext_ptr[p + 1]; e++) acc += zr[P->ext_idx[e]];
            R[p] = u[P->perm[p]] + acc;
        }
        /* large components one at a time, all threads on each sweep */
        int32_t k = k0;
        for (; k < k1 && P->c_off[k + 1] - P->c_off[k] >= big; k++) {
            const int32_t a = P->c_off[k], b = P->c_off[k + 1];
            if (P->c_type[k] == 1) {
                const double tau = tol * (double)(b - a) / (double)n;
                const int32_t it = scc_parallel(P, a, b, c, tau, max_iter, R, z0, z1, &noconv);
                if (it > imax) imax = it;
#pragma omp parallel for schedule(static)
                for (int32_t p = a; p < b; p++) zr[p] = c * R[p] * P->inv[p];
            } else {
                cac_pass(P, a, b, c, R, zr);
            }
        }
        /* the rest: a component per thread, largest first */
        int32_t lmax = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : lmax)
        for (int32_t kk = k; kk < k1; kk++) {
            const int32_t a = P->c_off[kk], b = P->c_off[kk + 1];
            if (b - a == 1) {
                zr[a] = c * R[a] * P->inv[a];
            } else if (P->c_type[kk] == 1) {
                int nc = 0;
                const double tau = tol * (double)(b - a) / (double)n;
                const int32_t it = scc_serial(P, a, b, c, tau, max_iter, R, z0, z1, &nc);
                if (nc) {
#pragma omp atomic write
                    noconv = 1;
                }
                if (it > lmax) lmax = it;
                for (int32_t p = a; p < b; p++) zr[p] = c * R[p] * P->inv[p];
            } else {
                cac_pass(P, a, b, c, R, zr);
            }
        }
        if (lmax > imax) imax = lmax;
    }
#pragma omp parallel for schedule(static)
    for (int32_t p = 0; p < n; p++) R_out[P->perm[p]] = R[p];
    free(R); free(zr); free(z0); free(z1);
    if (iters_max) *iters_max = imax;
    return noconv ? CPB_ENOCONV : CPB_OK;
}

/* The global series on the whole graph: R (original order), iters. */
int cpb_solve_global(const cpb_plan *P, double c, const double *u, double tol, int32_t max_iter, int32_t threads,
                     double *R_out, int32_t *iters) {
    if (!P || !(c > 0.0 && c < 1.0) || !(tol > 0.0) || max_iter < 1 || (P->n > 0 && (!u || !R_out)))
        return CPB_EINVAL;
    if (threads > 0) omp_set_num_threads(threads);
    const int32_t n = P->n;
    const size_t nn = n > 0 ? (size_t)n : 1;
    double *R = malloc(nn * sizeof(double)), *z0 = malloc(nn * sizeof(double)), *z1 = malloc(nn * sizeof(double));
    if (!R || !z0 || !z1) { free(R); free(z0); free(z1); return CPB_ENOMEM; }
#pragma omp parallel for schedule(static)
    for (int32_t p = 0; p < n; p++) {
        R[p] = u[P->perm[p]];
        z0[p] = c * R[p] * P->inv[p];
    }
    double *zc = z0, *zn = z1;
    int32_t it = 0;
    int rc = CPB_OK;
    for (;;) {
        double s = 0.0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : s)
        for (int32_t p = 0; p < n; p++) {
            double acc = 0.0;
            for (int32_t e = P->all_ptr[p]; e < P->all_ptr[p + 1]; e++) acc += zc[P->all_idx[e]];
            R[p] += acc;
            zn[p] = c * acc * P->inv[p];
            s += fabs(acc);
        }
        double *t = zc; zc = zn; zn = t;
        it++;
        if (!(s > tol)) break;
        if (it >= max_iter) { rc = CPB_ENOCONV; break; }
    }
#pragma omp parallel for schedule(static)
    for (int32_t p = 0; p < n; p++) R_out[P->perm[p]] = R[p];
    free(R); free(z0); free(z1);
    if (iters) *iters = it;
    return rc;
}

int cpb_max_threads(void) { return omp_get_max_threads(); }

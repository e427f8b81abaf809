/*
 * prgb.h -- C ABI of the componentwise PageRank library for GB300 (sm_103a).
 *
 * The library computes the non-normalised PageRank R of Def. 3.5 of
 * Engstrom & Silvestrov, "Graph partitioning and a componentwise PageRank
 * algorithm" (arXiv 1609.09068): the solution of (I - c A^T) R = u, where
 * A_ij = 1/outdeg(i) for each edge i -> j, dangling rows of A are zero and
 * 0 < c < 1.  Self-loops are ignored (Sec. 4.1 and Sec. 5.2).
 *
 * It follows the paper's three steps (Sec. 4): component finding
 * (SCC/CAC partition with levels, Sec. 3 Theorem 3.1 and Sec. 4.1), an
 * intermediate layout step (Sec. 4.2) and the level-by-level PageRank step
 * (Sec. 4.3).  pr_partition_create performs the first two, pr_solve the
 * third.  Calls that read the graph take a prepared pr_graph handle made
 * once from the caller's CSR by pr_graph_create (validation, loop removal
 * and the in-adjacency are done once and shared by the partition, the
 * global series and the residual) rather than the CSR itself.
 * pr_partition_save and pr_partition_load keep a partition in a file and
 * rebuild it for the same graph without the component search.
 * pr_global_power is the paper's baseline (the power series on the whole
 * graph, Sec. 4.3.2) and pr_residual_l1 evaluates the residual of the
 * defining system.
 *
 * Conventions shared by every entry point
 *   - Graphs are CSR out-adjacency: rowptr[n+1] (int32, rowptr[0] = 0,
 *     non-decreasing, rowptr[n] = nnz) and col[nnz] (int32 in [0, n)),
 *     column indices strictly increasing inside each row (simple graph,
 *     Sec. 3).  A self-loop i -> i may be present; it is ignored.
 *   - Indices are int32, so n < 2^31 and nnz < 2^31.
 *   - Pointers are borrowed: the library never frees caller memory and
 *     keeps no pointer to it after a call returns.  "device" means memory
 *     the current CUDA device can address (cudaMalloc, cudaMallocAsync or
 *     torch CUDA tensors); "host" means ordinary or pinned host memory.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls that return host results
 *     synchronise that stream before returning.
 *   - Every call returns a pr_status.  PR_ECUDA means a CUDA runtime call
 *     failed (pr_last_cuda_error gives its code); PR_ETIMEOUT means a
 *     device-side wait reached its time limit (two seconds unless
 *     pr_set_wait_limit says otherwise) and the kernel returned early; the
 *     CUDA context stays usable after both.
 *   - The library allocates device memory with cudaMallocAsync on the
 *     caller's stream and releases it the same way.
 */
#ifndef PRGB_H
#define PRGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PR_OK = 0,
    PR_EINVAL = 1,     /* bad argument or malformed CSR */
    PR_ENOMEM = 2,     /* device allocation failed */
    PR_ECUDA = 3,      /* a CUDA runtime call failed */
    PR_ENOCONV = 4,    /* max_iter reached; R holds the partial sum */
    PR_ETIMEOUT = 5,   /* a bounded device-side wait expired */
    PR_EINTERNAL = 6   /* an internal consistency check failed */
} pr_status;

/* CSR out-adjacency of the graph (see conventions above). */
typedef struct pr_csr {
    int32_t n;             /* number of vertices, >= 0 */
    int64_t nnz;           /* number of stored edges (self-loops included) */
    const int32_t *rowptr; /* [n+1] */
    const int32_t *col;    /* [nnz] */
    int32_t on_host;       /* 0: rowptr/col are device pointers; 1: host
                              pointers, copied to the device inside the call */
} pr_csr;

/* Opaque prepared graph: the validated, loop-free out-adjacency plus the
 * in-adjacency (CSC) built once by pr_graph_create (the graph model of
 * Sec. 3 and Def. 3.4).  Owned by the library until pr_graph_destroy. */
typedef struct pr_graph_s pr_graph;

/* Opaque partition: the SCC/CAC components, their levels and the permuted
 * layout the solver streams.  Owned by the library until
 * pr_partition_destroy; it refers to its pr_graph, which must outlive it. */
typedef struct pr_partition_s pr_partition;

/* Opaque learned warm-start model (see pr_mpnn_create). */
typedef struct pr_mpnn_s pr_mpnn;

/* Component types (Sec. 3 Def. 3.1-3.2; 1-vertex components are CACs). */
#define PR_TYPE_CAC 0
#define PR_TYPE_SCC 1

/* Stopping norms for the SCC power series (Sec. 4.3.2). */
#define PR_NORM_L1 0   /* stop after adding P with ||P||_1 <= tol*|C|/n */
#define PR_NORM_LINF 1 /* the paper's rule: iterate while max(P) >= tol */

/* Arithmetic of the solve. */
#define PR_PREC_FP64 0  /* FP64, except that the SCC series of every
                           component outside the cluster class (SCCs of at
                           most 1,024 or more than 16,384 vertices) is summed
                           exactly in 128-bit fixed point (each row's sum and
                           R exact, each term rounded once: to a quantum of
                           about 2^-110 ||W_C||_1, or 2^-110 |C| max W_C for
                           the grid-wide ones, whose z may be gathered as the
                           nearest FP64 values), which is at least as
                           accurate */
#define PR_PREC_MIXED 1 /* pr_solve only, with PR_NORM_L1 and no replay: the
                           series of each SCC of the cluster class
                           (1,025-16,384 vertices) runs in FP32 (values,
                           z = P/outdeg and accumulation), then an FP64
                           residual r = W + cA^T(R/outdeg) - R of the
                           component is formed; while ||r||_1 > tol*|C|/n
                           the correction (I - cA^T)D = r is summed by the
                           same FP32 series and R += D in FP64.  The other
                           SCCs run the exact fixed-point series as in
                           PR_PREC_FP64 (faster there on this GPU); the
                           inflow gather, CACs and 1-vertex components stay
                           FP64.  Every SCC ends with a residual within its
                           budget, so the L1 residual of R is at most tol
                           (plus FP64 rounding of the gather) as in FP64
                           mode; R differs from the FP64 result by at most
                           2*tol/(1-c) in L1.  PR_ENOCONV when six
                           corrections do not meet the budget (tol below
                           ~1e-13 ||R||_1) or max_iter sweeps are reached. */

typedef struct pr_solve_opts {
    int32_t norm;                /* PR_NORM_L1 (default) or PR_NORM_LINF */
    int32_t max_iter;            /* per component; <= 0 selects 10000 */
    int32_t precision;           /* PR_PREC_FP64 (default) or PR_PREC_MIXED */
    int32_t io_on_host;          /* 1: u and R are host pointers (copied in
                                    and out inside the call) */
    const int32_t *replay_iters; /* optional HOST array [n_comp]: run exactly
                                    this many series iterations per SCC
                                    component instead of the stopping rule
                                    (index = canonical component id); for
                                    pr_global_power, element 0 is used */
    const struct pr_mpnn_s *warm_start; /* optional (pr_solve only, not with
                                    replay_iters): the network of
                                    pr_mpnn_create guesses each SCC's R from
                                    its vertices' degrees, size and weights W;
                                    the series then continues from the
                                    residual of the guess, so the result
                                    meets the same stopping rule and residual
                                    bound as a cold start */
    int32_t lu_threshold;        /* pr_solve only: SCC components of fewer
                                    than lu_threshold vertices (0 = none, at
                                    most 129) are solved directly,
                                    (I - cA_C^T)R_C = W_C by Gaussian
                                    elimination (Sec. 4.3 item 3: the paper
                                    suggests fewer than ~100); their
                                    iteration count is 0 */
} pr_solve_opts;

typedef struct pr_solve_stats {
    int32_t iters_max;    /* largest per-component (or global) iteration count */
    int32_t n_levels;     /* levels walked by the solve */
    int64_t edge_visits;  /* edges read by the gather, CAC and SpMV kernels */
    int64_t launches;     /* kernels launched by the call */
    int32_t *comp_iters;  /* optional caller-owned HOST array [n_comp];
                             filled with per-component iteration counts when
                             non-NULL (0 for CACs and 1-vertex components) */
    int32_t timing;       /* in: 1 = time the grid-wide power-series kernels
                             with CUDA events on the call's stream; 2 = also
                             record an event between the levels (level_ms;
                             a few microseconds a level) */
    float kernel_ms;      /* out (timing = 1): their summed device time */
    int64_t kernel_bytes; /* out (timing = 1): their algorithmic bytes
                             (the exact fixed-point series): per sweep 4 B
                             per edge (index) + 72 B per row (z gather and
                             write, R read and write, c/outdeg), plus 88 B
                             per row once per launch (the start and the end
                             of the series); 56 B and 80 B when z is
                             gathered as FP64 values (an SCC whose sweep does
                             not fit in half the L2) */
    int64_t kernel_launches; /* out (timing = 1): number of such launches */
    int32_t fp64_sweeps_max; /* PR_PREC_MIXED: the most FP64 residual sweeps
                                of any SCC (included in iters_max and
                                comp_iters, which count all sweeps) */
    int64_t fp64_edge_visits; /* PR_PREC_MIXED: edges read by FP64 residual
                                 sweeps (included in edge_visits) */
    float *level_ms;      /* optional caller-owned HOST array [n_levels]; with
                             timing = 2 (pr_solve only) each level's device
                             time in walk order (Eq. PR:levels gather through
                             the level's last component), from CUDA events
                             recorded between the levels */
    int32_t counts_off;   /* in: 1 = leave iters_max, edge_visits, fp64_* and
                             comp_iters unset: the call then reads back only
                             what timing needs (the grid-wide components'
                             sweep counts) */
} pr_solve_stats;

/*
 * pr_graph_create -- validate a CSR and prepare it (Sec. 3: simple digraph;
 * Sec. 4.1 / 5.2: self-loops ignored): loop-free out-degrees and
 * out-adjacency, and the in-adjacency with sources ascending in each column.
 *   csr    : the graph (device or host arrays, see pr_csr.on_host).
 *   stream : CUDA stream.
 *   out    : receives a new graph handle on PR_OK (NULL otherwise).
 * Errors: PR_EINVAL for n < 0, nnz < 0 or >= 2^31, NULL arrays with n > 0, or
 * a malformed CSR (rowptr[0] != 0, rowptr[n] != nnz, non-monotone rowptr,
 * column out of range, unsorted or duplicate columns in a row); PR_ENOMEM,
 * PR_ECUDA.  Synchronises the stream.
 */
pr_status pr_graph_create(const pr_csr *csr, void *stream, pr_graph **out);

/* Flags of pr_graph_create_ex. */
#define PR_CANONICALIZE 1u /* sort every row's columns and drop repeated ones
                              (one edge per ordered pair: the simple graph of
                              Sec. 3) instead of rejecting the CSR */

/*
 * pr_graph_create_ex -- pr_graph_create with flags: 0 behaves exactly like
 * pr_graph_create; PR_CANONICALIZE accepts rows with unsorted or repeated
 * columns and builds the graph of the distinct edges (on the device: two
 * stable radix sorts of the edges by column and by row, then a compaction).
 * Row offsets and column ranges must still be valid.
 * Errors: PR_EINVAL for an unknown flag, invalid offsets or a column out of
 * range; otherwise those of pr_graph_create.  Synchronises the stream.
 */
pr_status pr_graph_create_ex(const pr_csr *csr, uint32_t flags, void *stream, pr_graph **out);

/* Release a graph (asynchronously, on the stream it was created on, which
 * must still exist).  Partitions built on it must be destroyed first.  NULL is
 * accepted. */
void pr_graph_destroy(pr_graph *g);

/* Flags of pr_partition_create. */
#define PR_PARTITION_TIMING 1u /* record CUDA events between the phases, for
                                  pr_partition_timing_get */

/* Phase times of a partition built with PR_PARTITION_TIMING: device time
 * between CUDA events recorded on its stream (host gaps between launches
 * included), and what the frontier-wave kernels ran. */
typedef struct pr_partition_timing {
    float trim_ms;    /* peeling of vertices with no in- or out-edge (Sec. 3
                         remark on 1-vertex SCCs) */
    float giant_ms;   /* forward-backward search for the largest SCC */
    float colour_ms;  /* colouring rounds for the other SCCs (Def. 3.1) */
    float levels_ms;  /* levels and CAC merges (Def. 3.3, Theorem 3.1) */
    float layout_ms;  /* canonical ids and the solve's layout */
    float total_ms;   /* the whole call up to its final synchronisation */
    int32_t colour_rounds;
    /* waves per kernel, [k][0] run by the whole grid (one grid barrier each)
       and [k][1] by one block alone (small frontiers); k = 0 trim,
       1 colour propagation, 2 forward-backward reachability, 3 backward
       search from the colour roots, 4 Kahn level order */
    int32_t waves[5][2];
} pr_partition_timing;

/*
 * pr_partition_create -- component finding and intermediate step
 * (Sec. 4.1-4.2).
 *   g      : a prepared graph; it must outlive the partition.
 *   flags  : 0 or PR_PARTITION_TIMING.
 *   stream : CUDA stream.
 *   out    : receives a new partition handle on PR_OK (NULL otherwise).
 * The partition is the unique SCC/CAC partition of Theorem 3.1 with
 * 0-based levels (Def. 3.3).  Component ids are canonical: sorted by level
 * descending, size descending, smallest vertex id ascending.
 * Errors: PR_EINVAL for a NULL graph or output, or an unknown flag;
 * PR_ENOMEM, PR_ECUDA, PR_ETIMEOUT, PR_EINTERNAL.  Synchronises the stream
 * (component counts are read back).
 */
pr_status pr_partition_create(const pr_graph *g, uint32_t flags, void *stream, pr_partition **out);

/*
 * pr_partition_save -- write a partition to a host file, so that the same
 * graph can be partitioned again (pr_partition_load) without the component
 * search and level assignment of Sec. 4.1.
 *   part   : the partition (from pr_partition_create or pr_partition_load).
 *   path   : host file path, created or truncated.
 *   stream : CUDA stream; synchronised.
 * Format (little endian): a 64-byte header -- magic "PRGBPART", format
 * version 1 (uint32), header size 64 (uint32), n and the loop-free edge
 * count (int64 each), a 64-bit digest of the graph's loop-free edge set, a
 * 64-bit digest of the arrays below and the three counts that follow, the
 * component count, level count and largest sub-level wave (int32 each), 4
 * bytes of zero -- then for every
 * vertex in the graph's vertex order its component id, its level (Def. 3.3),
 * its sub-level wave (int32 arrays of n entries each; a wave orders the
 * vertices of a CAC topologically) and its type PR_TYPE_* (uint8 array):
 * 13 bytes per vertex.  The digests detect a different graph and accidental
 * damage, not deliberate tampering: a loaded file is trusted.
 * Errors: PR_EINVAL for NULL arguments or a file that cannot be written (a
 * partly written file is removed); PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_partition_save(const pr_partition *part, const char *path, void *stream);

/*
 * pr_partition_load -- the partition of g read from a file that
 * pr_partition_save wrote for the same graph (same n, same loop-free edge
 * set): the layout of Sec. 4.2 is rebuilt from it on the device.  The
 * result equals pr_partition_create(g): the same component ids, types and
 * levels, and solves with the same results.
 *   g      : a prepared graph; it must outlive the partition.
 *   path   : host file path.
 *   flags  : 0.
 *   stream : CUDA stream; synchronised.
 *   out    : receives a new partition handle on PR_OK (NULL otherwise).
 * Errors: PR_EINVAL for NULL arguments, a nonzero flag, or a file that
 * cannot be read, is not a partition file of format version 1, was written
 * for a graph with another n, edge count or edge set, is truncated or
 * longer than its header says, holds a value out of range or fails its
 * digest, or whose component ids the rebuilt layout does not reproduce;
 * PR_ENOMEM, PR_ECUDA, PR_ETIMEOUT, PR_EINTERNAL.
 */
pr_status pr_partition_load(const pr_graph *g, const char *path, uint32_t flags, void *stream,
                            pr_partition **out);

/*
 * pr_partition_timing_get -- the phase times and wave counts of a partition
 * created with PR_PARTITION_TIMING, copied to *out (host).
 * Errors: PR_EINVAL for NULL arguments or a partition created without the
 * flag.
 */
pr_status pr_partition_timing_get(const pr_partition *part, pr_partition_timing *out);

/*
 * pr_partition_query -- copy the partition out, one entry per vertex in the
 * caller's original vertex order.
 *   comp_id [n] int32 (device), type [n] uint8 PR_TYPE_* (device),
 *   level [n] int32 (device): any of them may be NULL to skip it.
 *   n_comp, n_levels: host int32 outputs, may be NULL.
 * Errors: PR_EINVAL for a NULL partition; PR_ECUDA.
 */
pr_status pr_partition_query(const pr_partition *part, int32_t *comp_id, uint8_t *type,
                             int32_t *level, int32_t *n_comp, int32_t *n_levels, void *stream);

/*
 * pr_partition_info -- host-side counts: n, loop-free edge count, number of
 * components, levels, SCC components, and vertices in SCC components.
 * Any output may be NULL.
 */
pr_status pr_partition_info(const pr_partition *part, int32_t *n, int64_t *m, int32_t *n_comp,
                            int32_t *n_levels, int32_t *n_scc, int32_t *n_scc_vertices);

/*
 * pr_partition_tune -- autotuner of the solve's launch shapes (the paper has
 * no counterpart: the level schedule of Sec. 4.3 on this GPU).  Times
 * pr_solve (FP64, L1, tol) on this partition for each candidate of
 *   - the size boundary between the one-CTA class and the 8-CTA cluster
 *     class (64, 128 or 256 vertices), and
 *   - the blocks per SM of the grid-wide power-series kernels (3 or 4),
 *   - then, for the best of those, whether the grid-wide sweeps share their
 *     short rows among warps by cost (in-degree + 8) or in strided groups,
 * keeps the fastest for this partition and makes it the default of
 * partitions created later in the process.  Results of pr_solve do not
 * depend on the choice beyond rounding order.
 *   u      : [n] float64 DEVICE weights for the timed solves.
 *   cta_max, coop_blocks, balance, best_ms : optional host outputs (the
 *            choice and its solve time).
 * Errors: PR_EINVAL, PR_ENOMEM, PR_ECUDA and the errors of pr_solve.
 * Synchronises the stream; about twenty-one solves' worth of time.
 */
pr_status pr_partition_tune(pr_partition *part, double c, const double *u, double tol, void *stream,
                            int32_t *cta_max, int32_t *coop_blocks, int32_t *balance, float *best_ms);

/* Set the tuner's parameters by hand for this partition: cta_max in
 * [32, 256], coop_blocks in [1, 8] (fewer if the kernels do not fit),
 * balance 0 or 1.  Errors: PR_EINVAL. */
pr_status pr_partition_set_shape(pr_partition *part, int32_t cta_max, int32_t coop_blocks, int32_t balance);

/* Release the partition's device memory (asynchronously, on the stream it
 * was created on, which must still exist). NULL is accepted. */
void pr_partition_destroy(pr_partition *part);

/*
 * pr_solve -- the PageRank step of Sec. 4.3 on a partition.
 *   part   : from pr_partition_create.
 *   c      : damping factor, 0 < c < 1 (Def. 3.4).
 *   u      : [n] float64 weight vector W of Def. 3.5, finite and >= 0, in the
 *            original vertex order (device, or host with io_on_host = 1).
 *   tol    : > 0.  With PR_NORM_L1 each SCC component C stops after adding a
 *            series term of L1 norm <= tol*|C|/n, which bounds the L1
 *            residual of the whole solve by c*tol; CACs and 1-vertex
 *            components are solved exactly (Sec. 4.3 items 1-2).
 *   opts   : NULL for defaults.
 *   R      : [n] float64 output in the original vertex order (device, or
 *            host with io_on_host = 1), caller-owned.
 *   stats  : optional host output.
 * Levels are solved from the highest down; all components of one level run
 * concurrently (Sec. 4.3, last paragraph).  Synchronises the stream.
 * Errors: PR_EINVAL (bad c, tol, u; NULL pointers; replay array with a
 * negative entry), PR_ENOCONV (R holds the partial sums, stats are valid),
 * PR_ENOMEM, PR_ECUDA, PR_ETIMEOUT.
 */
pr_status pr_solve(const pr_partition *part, double c, const double *u, double tol,
                   const pr_solve_opts *opts, double *R, pr_solve_stats *stats, void *stream);

/*
 * pr_global_power -- the baseline of Sec. 4.3.2 / Sec. 5.2 method 1: the
 * power series P_0 = u, P_{k+1} = c A^T P_k, R = sum_k P_k on the whole
 * graph, stopping after adding P with ||P||_1 <= tol (PR_NORM_L1) or when
 * max(P) < tol (PR_NORM_LINF).  Arguments as for pr_solve, on a prepared
 * graph.  Synchronises the stream.
 */
pr_status pr_global_power(const pr_graph *g, double c, const double *u, double tol,
                          const pr_solve_opts *opts, double *R, pr_solve_stats *stats,
                          void *stream);

/*
 * pr_residual_l1 -- || u + c A^T (R ./ outdeg) - R ||_1 in FP64, the residual
 * of the system of Def. 3.5 (dangling vertices contribute no inflow).
 *   g : prepared graph; c as above; u, R : [n] float64 DEVICE pointers in the
 *   original vertex order.
 *   out_host : receives the residual.
 * Deterministic: the same inputs give the same bits.  Synchronises the
 * stream.
 */
pr_status pr_residual_l1(const pr_graph *g, double c, const double *u, const double *R,
                         double *out_host, void *stream);

/* Number of kernels this library has launched in this process so far (all
 * entry points, all threads).  Lets a caller count the kernels of a region. */
int64_t pr_launch_count(void);

/*
 * pr_set_wait_limit -- the time limit of every bounded device-side wait (the
 * grid barriers of the persistent kernels), in microseconds, for the calls
 * that start after it (a solve's cached graph is rebuilt for a new limit);
 * 0 restores the default of two seconds.  When a wait reaches the limit the
 * kernel records PR_ETIMEOUT and returns, and the call returns PR_ETIMEOUT;
 * the CUDA context stays usable.  The paper has no counterpart: this is the
 * library's failure detection.  Process-wide; always returns PR_OK.
 */
pr_status pr_set_wait_limit(uint32_t microseconds);

/*
 * pr_residual_l1_static -- the same L1 residual as pr_residual_l1, for
 * callers that cannot allocate device memory (for example code running
 * inside another framework's memory manager, which owns all device memory,
 * or a latency-critical path where cudaMalloc / cudaFree would synchronise
 * the device).  The paper has no counterpart; this is a service of the
 * library.
 *   g        : CSR with DEVICE arrays (on_host must be 0), n <= PR_STATIC_MAX_N.
 *   c, u, R  : as for pr_residual_l1 (u, R device pointers, original order).
 *   out_host : receives the residual.
 * It allocates nothing: its scratch is a fixed array in the library's device
 * data segment (PR_STATIC_MAX_N doubles plus 8 KB), which every GPU that
 * loads the library holds until the process exits.  The first call on a
 * device looks up that array's device address; make that first call before
 * any stream capture.  Every call shares the array (each call clears what it
 * uses); calls that overlap on the GPU race on it, so serialise them.  The
 * in-flow is accumulated with atomic adds, so the last bits can differ from
 * pr_residual_l1 and from call to call.
 * Errors: PR_EINVAL for n > PR_STATIC_MAX_N, on_host = 1, NULL pointers, or a
 * malformed CSR as pr_graph_create defines it (rowptr[0] != 0,
 * rowptr[n] != nnz, a decreasing rowptr, a column out of range, unsorted or
 * duplicate columns in a row); PR_ECUDA.  Synchronises the stream.
 */
#define PR_STATIC_MAX_N 1048576
pr_status pr_residual_l1_static(const pr_csr *g, double c, const double *u, const double *R,
                                double *out_host, void *stream);

/*
 * Learned warm start.  The paper starts each SCC's power series from
 * P_0 = W (Sec. 4.3.2); these calls build, train and evaluate a network that
 * guesses the SCC's solution instead, so that pr_solve (opts.warm_start)
 * continues the series from the guess's residual.  The paper has no learned
 * component; the guess only changes where the series starts, never what it
 * converges to or when it stops.
 *
 * Model, per vertex i of an SCC C (d_i internal in-edges, W_i the
 * inflow-adjusted weight of Eq. PR:levels, n vertices in the graph):
 *   x_i  = [log1p(d_i), log1p(outdeg_i), log|C|, log(n W_i + 1e-3), 1, 0, 0, 0]
 *   h_i  = relu(A1 x_i + B1 mean_{j->i, j in C} x_j + b1)        (64)
 *   g_i  = relu(A2 h_i + B2 mean_{j->i, j in C} h_j + b2)        (64)
 *   yhat = v . g_i + b3;  guess R0_i = W_i exp(clamp(yhat, 0, 10)).
 * Parameters: one float32 vector of pr_mpnn_param_count() = 9409 entries,
 * A1[64][8], B1[64][8], b1[64], A2[64][64], B2[64][64], b2[64], v[64], b3
 * (row-major, output index first), rounded to bfloat16 (nearest, ties to
 * even) for every forward pass; sums in float32.  Training target
 * y_i = log(R_i / W_i) of a solved R (vertices with W_i = 0 excluded), loss
 * = mean (yhat_i - y_i)^2 over the SCC vertices, optimiser Adam (0.9, 0.999,
 * 1e-8) on the float32 weights.
 */
int64_t pr_mpnn_param_count(void);

/* New model with seeded weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in))
 * from splitmix64(seed), zero biases, b3 = 1.  Owned by the caller until
 * pr_mpnn_destroy.  Errors: PR_EINVAL (out NULL), PR_ENOMEM, PR_ECUDA.
 * Synchronises the stream. */
pr_status pr_mpnn_create(uint64_t seed, void *stream, pr_mpnn **out);
void pr_mpnn_destroy(pr_mpnn *m);

/* Copy the float32 weights out / in (host arrays of exactly
 * pr_mpnn_param_count() floats, else PR_EINVAL).  Setting them clears the
 * optimiser state.  Synchronise the model's stream. */
pr_status pr_mpnn_get_params(const pr_mpnn *m, float *host, int64_t count);
pr_status pr_mpnn_set_params(pr_mpnn *m, const float *host, int64_t count);

/*
 * pr_mpnn_predict -- forward pass on a solved graph.
 *   part : partition of the graph; c : damping factor;
 *   u, R : [n] float64 DEVICE arrays in the original vertex order: the
 *          weights and a solution (W is formed from them by Eq. PR:levels).
 *   yhat : [n] float32 DEVICE output, one entry per vertex in the original
 *          vertex order (0 outside SCCs); may be NULL when only the loss is
 *          wanted.
 *   loss : optional host output, the training loss against R.
 * Errors: PR_EINVAL, PR_ECUDA.  Synchronises the stream.
 */
pr_status pr_mpnn_predict(const pr_mpnn *m, const pr_partition *part, double c, const double *u,
                          const double *R, float *yhat, double *loss, void *stream);

/* Loss and gradient (float32, host array of pr_mpnn_param_count() floats, or
 * NULL) of the model on one solved graph, without updating it.  Arguments as
 * for pr_mpnn_predict.  Synchronises the stream. */
pr_status pr_mpnn_loss_grad(pr_mpnn *m, const pr_partition *part, double c, const double *u,
                            const double *R, float *grad_host, double *loss, void *stream);

/* One Adam step (learning rate lr > 0) on the full batch of one solved
 * graph's SCC vertices; loss (optional) receives the loss before the step.
 * Synchronises the stream. */
pr_status pr_mpnn_train_step(pr_mpnn *m, const pr_partition *part, double c, const double *u,
                             const double *R, float lr, double *loss, void *stream);

/* Human-readable name of a status code (static storage). */
const char *pr_status_str(pr_status s);

/* The cudaError_t of the most recent PR_ECUDA in this thread (0 if none). */
int pr_last_cuda_error(void);

/* The most recent non-OK status that a call of this library returned in
 * this thread -- a failed argument check, an allocation, a CUDA call, or a
 * device-side check or bounded wait (PR_EINTERNAL, PR_ETIMEOUT) -- and
 * PR_OK if none failed since the last read.  Reading clears it.  Every
 * call also returns its own status; this is for callers that check
 * after a batch of calls. */
pr_status pr_last_device_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PRGB_H */

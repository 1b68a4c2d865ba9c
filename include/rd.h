/*
 * rd.h -- resistance distance by Lanczos iteration on one GPU (sm_103a).
 *
 * C ABI of librd.so. Every call takes plain pointers and sizes; nothing here
 * depends on PyTorch or any other framework.
 *
 * The method (paper: Section 3, Algorithm 3 and Eq. (approx_formula)): for an
 * undirected connected graph with positive edge weights w_uv, degrees
 * d_u = sum_v w_uv, Ahat = D^{-1/2} W D^{-1/2} and
 * b = e_s/sqrt(d_s) - e_t/sqrt(d_t),
 *
 *     r(s,t) = (e_s - e_t)^T L^+ (e_s - e_t) = b^T (I - Ahat)^+ b
 *           ~= ||b||^2 e_1^T (I - T_k)^{-1} e_1,
 *
 * with T_k the tridiagonal matrix built by k steps of the Lanczos three-term
 * recurrence started from v_1 = b/||b|| (Eq. (lz_recurrence)). The
 * resistance distance itself is the Definition of RD in Section 2.1.
 *
 * Conventions shared by all calls:
 *  - Status: every call returns an rd_status; nothing throws across the ABI.
 *    rd_last_error() returns a human-readable detail for the calling thread.
 *  - Pointers marked "host or device" may be either; the library tells them
 *    apart with cudaPointerGetAttributes and stages host buffers itself.
 *    Device pointers must be device memory of the current CUDA device.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream). All device work of a call is ordered on that stream.
 *    rd_query, rd_edge_grad and rd_potential synchronize that stream before
 *    returning (they poll per-pair convergence), so their outputs are ready
 *    on return.
 *  - Ownership: the caller owns every pointer it passes. rd_graph owns only
 *    what it allocates (its device copy of the CSR, derived arrays and a
 *    grow-only workspace reused by later calls); rd_graph_destroy frees it.
 *  - Threads: an rd_graph may be used by one thread at a time.
 *  - Sizes: 1 <= n < 2^31, 0 <= nnz < 2^31.
 */
#ifndef RD_H
#define RD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RD_ABI_VERSION 1

typedef struct rd_graph rd_graph;

typedef enum {
    RD_OK = 0,
    RD_WARN_NOT_CONVERGED = 1, /* per pair: k_max reached before the tolerance */
    RD_ERR_INVALID_ARG = -1,   /* bad size, id out of range, bad CSR, NaN/negative weight */
    RD_ERR_ZERO_DEGREE = -2,   /* a vertex has no incident edge (degree 0) */
    RD_ERR_DISCONNECTED = -3,  /* per pair: s and t lie in different components (r = +inf) */
    RD_ERR_CUDA = -4,          /* a CUDA runtime call failed */
    RD_ERR_OOM = -5,           /* device allocation failed */
    RD_ERR_TIMEOUT = -6,       /* a bounded device loop gave up */
    RD_ERR_NUMERIC = -7,       /* per pair: I - T_k lost positive definiteness or a value is not finite */
    RD_ERR_UNSUPPORTED = -8    /* valid request the library does not implement */
} rd_status;

typedef enum {
    RD_MODE_FP64 = 0,        /* vectors, SpMV/SpMM and all scalars in FP64 */
    RD_MODE_FP32V_FP64S = 1, /* vectors and SpMM in FP32; alpha, beta, T_k, its solve and every
                                cross-thread reduction in FP64. Accuracy floor: the FP32 rounding of
                                the vectors limits the attainable relative error of r, and the
                                floor grows with the condition number kappa = 2/(1 - mu_2(Ahat)):
                                below 1e-7 at kappa ~ 10 (power-law graphs), about 5e-6 on a 64x64
                                grid (kappa ~ 3e3), about 2e-4 on a 4096x4096 road-like grid
                                (kappa ~ 1.4e7). Tolerances below the floor are not met there (the
                                iteration runs on, or stops on an estimate that is not a bound): use
                                RD_MODE_FP64 or RD_MODE_DF64 for large-kappa graphs */
    RD_MODE_DF64 = 2         /* rd_query only (the other calls run it as RD_MODE_FP64): vectors
                                stored as pairs of FP32 numbers (hi + lo, about 48 significant
                                bits) with the element arithmetic on the FP32 units by error-free
                                transformations; scalars as in RD_MODE_FP64. FP64-class accuracy
                                where FP64 arithmetic, not memory, bounds the step */
} rd_mode;

/* rd_graph_create / rd_graph_set_weights flags */
#define RD_INPUT_ON_DEVICE 1u   /* force: the CSR pointers are device pointers (else auto-detected) */
#define RD_CHECK_SYMMETRY 2u    /* verify that (v,u,w) is stored for every (u,v,w); error if not */
#define RD_LABEL_COMPONENTS 4u  /* label connected components so disconnected pairs get +inf */

/* rd_query_opts.flags */
#define RD_Q_FIXED_K 1u     /* ignore rel_tol/resid_tol: every pair runs exactly k_max steps
                               (or stops at breakdown) */
#define RD_Q_NO_DEFLATE 2u  /* do not remove the component along D^{1/2}1 from each new vector */
#define RD_Q_PLAIN 4u       /* answer the pairs one at a time with the single-vector SpMV path */
#define RD_Q_PROFILE 8u     /* time the dominant kernel with CUDA events (see rd_last_call_stats) */
#define RD_Q_NO_COMPACT 16u /* rd_query: keep every pair's column until the end instead of packing
                               the still-active pairs into a narrower block as pairs converge */
#define RD_Q_NO_ONCHIP 32u  /* rd_query: do not run small graphs (three vectors fit in one SM's
                               shared memory) as one whole-recurrence kernel with one block per pair */
#define RD_Q_NO_TUNE 64u    /* with rhs_tile, rows_per_warp and kernel all 0: pick the SpMM
                               configuration by a fixed rule instead of the autotuner (see
                               rd_autotune) */
#define RD_Q_EST_DELAYED 256u /* rel_tol test on the sum of the last 4 increments of
                               e_1^T (I-T_k)^{-1} e_1 (the error of the estimate 4 steps back)
                               instead of the default geometric tail estimate (see rel_tol) */
#define RD_Q_NO_GRAPH 128u  /* rd_query: launch every kernel of every step from the host instead
                               of replaying a captured CUDA graph of one step (the results are
                               bitwise the same; RD_Q_PROFILE also turns the graphs off) */
#define RD_Q_DENSE_FIRST 512u /* compute the first step's product D^{-1} A q_1 with the SpMM over
                               every row. By default, when the graph's rows are sorted by column
                               and its entries symmetric (checked by rd_graph_create and
                               rd_graph_set_weights), a kernel visits only the rows adjacent to s
                               and t, where q_1 (nonzero in rows s and t alone) makes it nonzero;
                               the two agree to rounding */
#define RD_Q_REPLAY_POTENTIAL 1024u /* rd_edge_grad / rd_potential / rd_flow: form the potential
                               sum_j ||b|| z_j q_j (z = (I - T_k)^{-1} e_1) by a second pass that
                               regenerates q_1..q_k from the stored coefficients (Algorithm 5),
                               instead of the default direct update during the forward steps
                               (p_i = q_i + (beta_i/delta_{i-1}) p_{i-1}, x += ||b|| (g_i/delta_i) p_i
                               from the LDL^T factors of I - T_i; one extra vector, no second pass);
                               the two agree to rounding */
#define RD_Q_NO_CLUSTER 2048u /* rd_query: run the whole-recurrence kernel of small graphs with one CTA
                               per pair. By default, when few pairs are asked (pairs x 2 x CTAs <= SMs),
                               each pair's recurrence runs on a thread-block cluster of up to 16 CTAs
                               (one per SM), each holding a slice of the three vectors in its shared
                               memory and reading the others' through distributed shared memory; the
                               two agree to rounding */
#define RD_Q_NO_DEVICE_LOOP 4096u /* rd_query: launch each step's CUDA graph from the host and poll
                               the active count between steps. By default the steps after the first
                               run in one graph whose conditional (while) node repeats the step on
                               the device until every pair has stopped, k_max is reached or a column
                               compaction is due; the host steps in only to pack the columns, with
                               the normalise pass of the step before the packing fused into it. Both
                               give bitwise the same results (the device loop may skip a packing
                               that the host-driven loop makes after the last pair has stopped) */

typedef struct {
    int32_t k_max;         /* step cap (>= 1) */
    double rel_tol;        /* stop when the estimated relative error of r is <= rel_tol (0 = off);
                              estimate (from step 4 on): with d_j the increments of
                              S_k = e_1^T (I-T_k)^{-1} e_1 and rho the largest of the last three
                              ratios d_j / d_{j-1} (at least 1/2), d_k * rho / (1 - rho)^2 / S_k,
                              the tail of a geometric series with a margin for slow decay; not
                              a bound (RD_Q_EST_DELAYED selects the delayed-sum estimate); with
                              RD_MODE_FP32V_FP64S on large-kappa graphs the FP32 floor (see rd_mode)
                              can exceed rel_tol, and the pair then stops with an error above it */
    double resid_tol;      /* stop when ||b - (I - Ahat) x_k|| / ||b|| <= resid_tol (0 = off) */
    int32_t mode;          /* rd_mode */
    int32_t rhs_tile;      /* right-hand-side columns per SpMM sweep; 0 = tuned */
    int32_t rows_per_warp; /* rows a warp works on at once; 0 = tuned */
    int32_t chunk_steps;   /* steps between synchronous host convergence polls where those are used
                              (rd_edge_grad, rd_potential, rd_query_noalloc); 0 = default (8).
                              rd_query polls every step, one step behind the device. */
    uint32_t flags;        /* RD_Q_* */
    int32_t kernel;        /* SpMM kernel: 0 = tuned, 1 = row-group (warp lanes split a row's
                              nonzeros), 2 = row-stream (row groups walk runs of consecutive rows),
                              3 = row-group visiting the rows by decreasing degree (the row groups
                              of a warp then hold rows of equal length), 4 = warp-per-task SpMV
                              (one column only: RD_Q_PLAIN or one pair; RD_ERR_UNSUPPORTED
                              otherwise), 5 = row-stream with asynchronous copies of the gathered
                              rows into a shared-memory ring (FP32 vectors and 16 to 128 columns per
                              slab only; RD_ERR_UNSUPPORTED otherwise; with one column it takes 4);
                              with one column the fixed rule (RD_Q_NO_TUNE) takes 4 */
} rd_query_opts;

/* Per-call statistics of the last rd_query / rd_edge_grad / rd_potential on g. */
typedef struct {
    int64_t launches;        /* kernels this library launched during the call */
    int64_t spmm_launches;   /* launches of the dominant SpMM/SpMV kernel */
    double spmm_ms;          /* summed CUDA-event time of those launches (RD_Q_PROFILE only, else 0) */
    int32_t steps;           /* Lanczos steps run (max over pairs) */
    int32_t rhs_tile;        /* configuration used */
    int32_t rows_per_warp;
    int32_t nnz_lanes;       /* lanes that share one row's nonzeros */
    int32_t kernel;          /* SpMM kernel used, numbered as rd_query_opts::kernel (1 .. 5) */
    int64_t ld;              /* padded number of right-hand-side columns (vector row stride) */
    double spmm_bytes;       /* algorithmic bytes of all SpMM launches of the call, each
                                4*nnz (+4*nnz weights) + 8*(n+1) + 3*ld*n*sizeof(element) with the
                                ld in force at that launch (it shrinks as converged pairs are packed) */
    int32_t compactions;     /* times the active pairs were packed into a narrower block */
    int32_t tuned;           /* 1 if the configuration came from the autotuner's table */
    int32_t row_order;       /* 1 if the row-group kernel visited rows by decreasing degree */
    int32_t sparse_first;    /* 1 if the first step visited only the rows adjacent to s and t
                                (see RD_Q_DENSE_FIRST) */
    int32_t onchip_ctas;     /* CTAs per pair of the whole-recurrence kernel (1: one CTA, 2..16: a
                                thread-block cluster; see RD_Q_NO_CLUSTER), 0 if it did not run */
    int32_t device_loop;     /* 1 if the steps after the first ran in the device-resident loop
                                (see RD_Q_NO_DEVICE_LOOP) */
} rd_call_stats;

/* Fill `opts` with defaults: k_max 1000, rel_tol 1e-7, resid_tol 0, FP32 vectors with FP64
 * scalars, tuned tiles and kernel, chunk 8, flags 0. */
void rd_query_opts_init(rd_query_opts* opts);

/* Build a device graph from symmetric CSR (Section 2.1: undirected graph; weighted
 * generalisation as stated there).
 *  n, nnz       : vertices and stored entries (each undirected edge is stored twice).
 *  row_ptr      : int64[n+1], host or device, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *  col_idx      : int32[nnz], host or device, values in [0, n).
 *  weights      : float[nnz] host or device, all > 0 and finite; NULL = unweighted (all 1).
 *  flags        : RD_INPUT_ON_DEVICE | RD_CHECK_SYMMETRY | RD_LABEL_COMPONENTS.
 * Self-loops are dropped (they cancel in L = D - W, so r is unchanged); duplicate entries
 * are summed. The arrays are copied; the caller may free them after return.
 * Errors: RD_ERR_INVALID_ARG (sizes, CSR shape, ids, weights, asymmetry when checked),
 * RD_ERR_ZERO_DEGREE (a vertex with no edge, n > 1), RD_ERR_OOM, RD_ERR_CUDA.
 * On error *out is NULL. */
rd_status rd_graph_create(rd_graph** out, int64_t n, int64_t nnz, const int64_t* row_ptr,
                          const int32_t* col_idx, const float* weights, uint32_t flags, void* stream);

/* Replace the edge weights (same structure, float[nnz] in the order given at create, before
 * self-loop removal), host or device; recomputes degrees. Same weight errors as create. */
rd_status rd_graph_set_weights(rd_graph* g, const float* weights, void* stream);

/* Free everything the graph owns. NULL is accepted. */
rd_status rd_graph_destroy(rd_graph* g);

/* Host outputs (any may be NULL): vertices, stored entries after self-loop removal, whether
 * weighted, number of components (0 if not labelled). */
rd_status rd_graph_info(const rd_graph* g, int64_t* n, int64_t* nnz, int32_t* weighted,
                        int32_t* ncomponents);

/* Resistance distances of npairs (s,t) pairs (Algorithm 3, batched: all pairs advance
 * together as one SpMM over an n x ld row-major block of vectors).
 *  s, t           : int32[npairs], host or device, ids in [0, n).
 *  opts           : NULL = rd_query_opts_init defaults.
 *  r_out          : double[npairs], host or device: ||b||^2 e_1^T (I - T_k)^{-1} e_1.
 *  iters_out      : int32[npairs] or NULL: k per pair.
 *  err_est_out    : double[npairs] or NULL: estimated relative error (rel_tol's estimate).
 *  pair_status_out: int32[npairs] or NULL: per-pair rd_status. s == t gives r = 0, RD_OK;
 *                   different components (when labelled) give r = +inf, RD_ERR_DISCONNECTED;
 *                   k_max reached gives the estimate so far and RD_WARN_NOT_CONVERGED;
 *                   loss of definiteness gives the last good estimate and RD_ERR_NUMERIC.
 * Per-pair problems do not fail the call. The call returns RD_OK, or RD_WARN_NOT_CONVERGED
 * if any pair did not converge, or an error for the whole call (RD_ERR_INVALID_ARG for an
 * id out of range or npairs < 0; RD_ERR_OOM; RD_ERR_CUDA). npairs == 0 returns RD_OK. */
rd_status rd_query(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs,
                   const rd_query_opts* opts, double* r_out, int32_t* iters_out, double* err_est_out,
                   int32_t* pair_status_out, void* stream);

/* Gradient of sum_p grad_r[p] * r(s_p, t_p) with respect to the stored edge weights.
 * For stored entry e = (u -> v): grad_w_out[e] = 1/2 * sum_p grad_r[p] * dr_p/dw_uv with
 * dr/dw_uv = -(phi(u) - phi(v))^2 and phi = sqrt(1/d_s+1/d_t) D^{-1/2} V_k (I-T_k)^{-1} e_1,
 * the Lanczos potential of Section 6.3 (the one Algorithm 5 starts from). Both stored copies of an
 * edge get the same value, so moving both copies by delta changes the objective by
 * delta * (sum of the two). phi is built during the forward steps from the LDL^T factors of
 * I - T_i (no basis V_k is kept and no second pass runs); RD_Q_REPLAY_POTENTIAL instead
 * rebuilds it by a second Lanczos pass that replays the stored alpha/beta.
 *  grad_r     : double[npairs] host or device, or NULL for all ones.
 *  grad_w_out : float[nnz_created] host or device (nnz as passed to create; entries that
 *               were self-loops get 0).
 *  r_out      : double[npairs] or NULL.
 * Errors as rd_query. */
rd_status rd_edge_grad(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs,
                       const double* grad_r, const rd_query_opts* opts, float* grad_w_out,
                       double* r_out, void* stream);

/* Lanczos potentials (Section 6.3, Definition electric_flow and Algorithm 5):
 * phi_out is float[npairs][n] (pair-major), host or device; phi_p is defined up to an
 * additive constant (the library's is orthogonal to the degree vector). Edge flows are
 * f(e) = phi(u) - phi(v). r_out as rd_query (nullable). Errors as rd_query. */
rd_status rd_potential(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs,
                       const rd_query_opts* opts, float* phi_out, double* r_out, void* stream);

/* Triangle-count edge weights for the weighted experiments (Section 6, Exp-2): for every stored
 * entry e = (u, v), w_out[e] = number of triangles containing edge uv, or 1 if there is none.
 * The graph's own weights are ignored; its rows must have strictly increasing columns
 * (RD_ERR_INVALID_ARG otherwise). w_out: float[nnz], host or device. Pass the result to
 * rd_graph_set_weights to run the weighted method. */
rd_status rd_triangle_weights(const rd_graph* g, float* w_out, void* stream);

/* Power Method (Section 2.2, Algorithm 1), batched over pairs on the same SpMM kernels: the
 * truncated lazy-walk series rbar_l = 1/2 sum_{i=0..l} (e_s-e_t)^T D^{-1} (I/2 + P/2)^i (e_s-e_t),
 * P = A D^{-1} (Eq. (er_laylor_expansion) truncated at l). A baseline for the Lanczos path.
 *  steps     : l >= 0 (l + 1 terms).
 *  mode      : rd_mode (vector precision; the sums are FP64).
 *  r_out     : double[npairs], host or device.
 *  r_hist_out: double[steps + 1][npairs] or NULL: the estimate after each term.
 * Errors as rd_query (no per-pair status; disconnected pairs are not detected). */
rd_status rd_power_method(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs, int32_t steps,
                          int32_t mode, double* r_out, double* r_hist_out, void* stream);

/* Electric flows (Section 6.3, Definition electric_flow): for every stored entry e = (u -> v),
 * flow_out[p][e] = phi_p(u) - phi_p(v), with phi_p the Lanczos potential of pair p as in
 * rd_potential (Section 6.3, Algorithm 5). The current through the edge is w_e * flow.
 *  flow_out : float[npairs][nnz] (nnz as passed to create, caller's entry order; entries that
 *             were self-loops get 0), host or device.
 *  r_out    : double[npairs] or NULL. Errors as rd_query. */
rd_status rd_flow(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs,
                  const rd_query_opts* opts, float* flow_out, double* r_out, void* stream);

/* Batched query without any device allocation -- no counterpart in the paper; it exists
 * for callers that cannot call cudaMalloc (code running under another framework's
 * allocator or memory pool, processes that reserve all device memory up front, or
 * contexts where allocation is forbidden). It runs the same recurrence as rd_query with
 * the row-group SpMM kernel (or, for graphs whose three vectors fit in one SM's shared
 * memory, the whole-recurrence kernel of RD_Q_NO_ONCHIP), taking the graph straight from
 * the caller's device CSR (no rd_graph is created) and using, as its only scratch, one fixed 32 MiB device
 * array compiled into this library (every GPU that loads the library holds it until the
 * process exits).
 *  n, nnz, row_ptr, col_idx, weights : symmetric CSR as for rd_graph_create, DEVICE pointers;
 *                    self-loops are rejected (RD_ERR_UNSUPPORTED) since the CSR is used as is.
 *  s, t            : int32[npairs] device pointers.
 *  opts            : as rd_query, except: RD_Q_PROFILE is ignored; the SpMM kernel is
 *                    row-group; RD_MODE_DF64 runs as RD_MODE_FP64 (FP64 vectors, the same
 *                    accuracy class, 8-byte elements in the same scratch); disconnected pairs
 *                    are not labelled and end as RD_ERR_NUMERIC.
 *  r_out           : double[npairs] device pointer; iters_out: int32[npairs] device or NULL.
 * Limits: the scratch must hold 24*n bytes of degrees plus the query workspace
 * (2*n*ld vector elements, (k_max+1)*4*ld coefficients, the per-pair state); a request that
 * does not fit returns RD_ERR_INVALID_ARG with the sizes in rd_last_error() and launches
 * nothing. Host pointers are rejected with RD_ERR_INVALID_ARG.
 * Set-up: the first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current); make that first call before any
 * stream capture. The address is kept for the life of the process: it does not survive
 * cudaDeviceReset (or any other destruction of the device's primary context), after which
 * this entry point must not be called again in that process.
 * Polls: the call waits on the stream for per-pair convergence counts every chunk_steps
 * steps and copies them into pageable host memory (it allocates no pinned buffer), so each
 * poll is a synchronous copy; the outputs are ready on return. Sharing: every call uses the same array, which keeps the previous
 * call's contents (the call clears what must start at zero itself); calls that overlap on
 * the GPU (other streams, other host threads) race on it. Returns as rd_query. */
rd_status rd_query_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                           const float* weights, const int32_t* s, const int32_t* t, int64_t npairs,
                           const rd_query_opts* opts, double* r_out, int32_t* iters_out, void* stream);

/* SpMM autotuner. No counterpart in the paper: it picks the right-hand-side tile, the rows
 * per warp and the kernel of the SpMM step of Algorithm 3 for this graph and GPU by
 * timing, not by a fixed rule. For a query of npairs pairs in opts->mode it times every
 * instantiated candidate (tiles from a quarter of the pair count's power-of-two width up to
 * that width; the row-stream kernel and the row-group kernel with 1, 2 or 4 nonzero lanes
 * per row group; for one column the warp-per-task SpMV, the row-stream and the row-group
 * SpMV) on g's own CSR with zeroed vectors, one warm-up and three timed launches each (CUDA
 * events on `stream`), and keeps the fastest per width class in g. Without RD_Q_PLAIN (and
 * npairs > 1) the narrower classes a compacting query passes through are tuned as well,
 * unless RD_Q_NO_COMPACT is set. Calls on g whose opts leave rhs_tile, rows_per_warp and
 * kernel at 0 without RD_Q_NO_TUNE use the table, and tune a missing class on first use.
 *  npairs  : 1 .. 2^24.
 *  opts    : mode and flags as for rd_query (NULL = defaults); rhs_tile, rows_per_warp and
 *            kernel must be 0 and RD_Q_NO_TUNE unset, else RD_ERR_INVALID_ARG.
 *  rhs_tile_out, rows_per_warp_out, kernel_out : nullable; the configuration a query of
 *            npairs pairs now starts with (kernel numbered as in rd_call_stats).
 * Uses (and may grow) g's workspace; the GPU work is on `stream`, which is synchronised
 * before return. Returns RD_OK, RD_ERR_INVALID_ARG, RD_ERR_CUDA or RD_ERR_OOM (a candidate
 * whose workspace does not fit is skipped; RD_ERR_OOM only if none fits). */
rd_status rd_autotune(rd_graph* g, int64_t npairs, const rd_query_opts* opts, int32_t* rhs_tile_out,
                      int32_t* rows_per_warp_out, int32_t* kernel_out, void* stream);

/* Statistics of the last call on g (host struct). */
rd_status rd_last_call_stats(const rd_graph* g, rd_call_stats* out);

/* Static text for a status code. */
const char* rd_status_string(rd_status s);

/* Detail of the last error raised on the calling thread ("" if none). */
const char* rd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RD_H */

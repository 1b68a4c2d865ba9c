// Internal declarations of librd: graph object, workspace, kernel argument
// blocks and the launcher table. Not part of the public ABI (see include/rd.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rd.h"
#include "df64.cuh"

namespace rd {

// ----------------------------------------------------------------- errors
void set_error(const std::string& msg);
rd_status cuda_status(cudaError_t e, const char* what);

#define RD_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return ::rd::cuda_status(_e, #call);     \
    } while (0)

#define RD_TRY(call)                                                    \
    do {                                                                \
        rd_status _s = (call);                                          \
        if (_s < 0) return _s;                                          \
    } while (0)

// ------------------------------------------------------- SpMM configuration
// One warp is split into row groups of GS*NZL lanes. GS lanes span the
// right-hand-side tile (VEC elements each, so the tile is TP = VEC*GS
// columns); NZL lanes share the nonzeros of one row; RPW = 32/(GS*NZL) rows
// are in flight per warp.
// kind 0: row-group kernel (k_spmm, grid-stride over rows); kind 1: row-stream kernel
// (k_spmm_rows, grid-stride over tasks of consecutive rows; nzl must be 1); kind 2:
// warp-per-task SpMV (one column); kind 3: row-stream kernel with cp.async gathers into a
// shared-memory ring (k_spmm_async, FP32 vectors, vec 4, nzl 1).
struct SpmmCfg {
    int vec = 4, gs = 32, nzl = 1, kind = 0;
    int order = 0;  // row-group kernel: 1 = visit rows by decreasing degree (rd_graph::row_order)
    int tp() const { return vec * gs; }
    int rpw() const { return 32 / (gs * nzl); }
    bool operator==(const SpmmCfg& o) const
    {
        return vec == o.vec && gs == o.gs && nzl == o.nzl && kind == o.kind && order == o.order;
    }
};

// Configuration of the heavy-row pre-pass that goes with a step configuration: the same
// column tile, one whole warp per chunk of a heavy row (GS column lanes x 32/GS nonzero
// lanes), so that a chunk's gathers are spread over the warp instead of one row group.
// The async kernel (kind 3) has its own pre-pass with one row group per chunk.
inline SpmmCfg heavy_cfg(const SpmmCfg& c)
{
    SpmmCfg h;
    h.vec = c.vec;
    h.gs = c.gs;
    h.nzl = c.kind == 3 ? 1 : 32 / c.gs;
    h.kind = c.kind == 3 ? 3 : 0;
    return h;
}

constexpr int kBlock = 256;        // threads per block of the SpMM kernels
constexpr int kWarps = kBlock / 32;
constexpr int kRing = 4;           // increments kept for the delayed error estimate

// Argument block of one Lanczos step's SpMM (q-space: q = D^{-1/2} v).
template <typename T>
struct StepArgs {
    int64_t n, ld;                 // rows, padded columns (row stride of vector blocks)
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w;                // nullable (unweighted)
    const T* invdeg;               // 1/d_u
    const T* deg;                  // d_u
    const T* qcur;                 // q_i  (n x ld)
    T* qprev_w;                    // in: q_{i-1}; out: W = D^{-1} W_adj q_i - beta_i q_{i-1}
    const T* cf_beta;              // beta_i per column (ld)
    // heavy rows (degree > heavy_thr): chunk partial sums made by the heavy kernel
    int heavy_thr;
    int64_t n_heavy_rows, n_chunks;
    const int32_t* heavy_rows;     // sorted row ids
    const int32_t* heavy_first;    // n_heavy_rows + 1 chunk offsets
    const int32_t* chunk_beg;      // nnz range of each chunk
    const int32_t* chunk_end;
    T* heavy_part;                 // n_chunks x ld
    int64_t hot_rows;              // gathers of rows below this id keep L2 priority (the rest evict first)
    int64_t ntasks;                // row-stream tasks: rows [task_row[i], task_row[i+1])
    const int32_t* task_row;
    double* block_part;            // [slab][block][3][TP]
    const int32_t* active_prev;    // early exit when *active_prev == 0 (nullable)
    int do_reduce;
    int lazy_walk;                 // Power Method step: W = (1/2) q + (1/2) D^{-1} W_adj q (no recurrence)
    // Step index read from device memory (graph replay; nullable): then the step j's
    // beta_i row is cf_beta + j * cf_stride and the early-exit count is act_count[j].
    const int32_t* step_dev;
    int64_t cf_stride;
    const int32_t* act_count;
    // row-group kernel: visiting order of the rows (nullable = 0 .. n-1); rows of equal
    // degree are adjacent, so the row groups of a warp finish their rows together
    const int32_t* row_order;
};

// Step-dependent operands of a StepArgs launch (fixed pointers, or derived from the step
// index in device memory when the launch is replayed from a CUDA graph).
template <typename T>
__device__ __forceinline__ const T* step_cf_beta(const StepArgs<T>& a)
{
    return a.step_dev ? a.cf_beta + (int64_t)(*a.step_dev) * a.cf_stride : a.cf_beta;
}

template <typename T>
__device__ __forceinline__ bool step_inactive(const StepArgs<T>& a)
{
    const int32_t* p = a.step_dev ? a.act_count + *a.step_dev : a.active_prev;
    return p != nullptr && *p == 0;
}

template <typename T>
struct NormArgs {
    int64_t n, ld;
    T* w_to_qnext;                 // in: W, out: q_{i+1} (in place)
    const T* qcur;
    const T* cf;                   // [4][ld]: beta_i, alpha_i, c_i, 1/beta_{i+1}
    T* phi;                        // nullable: phi += coef * q_i (replay pass)
    const T* coef;                 // ld, with phi
    const int32_t* active_prev;
    const int32_t* step_dev;       // as StepArgs: cf + j * cf_stride, act_count[j]
    int64_t cf_stride;
    const int32_t* act_count;
    // potential accumulated during the forward pass (nullable pvec: off)
    T* pvec;                       // p_{i-1} in, p_i out
    T* xvec;                       // x += mu_i p_i
    const T* xcf;                  // [2][ld]: lambda_i, mu_i (+ j * xcf_stride with step_dev)
    int64_t xcf_stride;
};

// Normalise pass fused with a column compaction (k_normalize_pack).
template <typename T>
struct NormPackArgs {
    int64_t n, ld_old, ld_new;
    const T* w;                    // W, old layout
    const T* qcur;                 // q_i, old layout
    const T* cf;                   // [4][ld_old]: beta_i, alpha_i, c_i, 1/beta_{i+1} of the step
    const int32_t* old_slot;       // [ld_new]: source column of each packed column, -1 none
    T* qnext_new;                  // q_{i+1}, packed (n x ld_new)
    T* qcur_new;                   // q_i, packed (n x ld_new)
};

// Per-pair FP64 state of the running LDL^T factorisation of I - T_k.
struct PairState {
    double* b2;        // ||b||^2 = 1/d_s + 1/d_t
    double* delta;     // last pivot
    double* g;         // last entry of L^{-1} e_1
    double* S;         // e_1^T (I - T_k)^{-1} e_1
    double* beta;      // beta_{k+1}
    double* ring;      // kRing x ld increments
    double* r;         // b2 * S
    double* err;       // estimated relative error
    double* resid;     // relative residual
    int32_t* k;        // steps done
    int32_t* status;   // rd_status per pair
    int32_t* active;   // 1 while iterating
    double* hist_alpha;   // k_max x ld
    double* hist_beta;    // (k_max + 1) x ld: beta_1 .. beta_{k_max+1}
    int32_t* act_count;   // k_max + 1 counters: active pairs entering step j
};

struct FinArgs {
    int64_t ld;
    int npairs, tp, nblocks, step;      // step: 0-based index of the step just reduced
    int k_max, deflate, fixed_k, fp64;
    double rel_tol, resid_tol, sumdeg;
    double inv_sumdeg;                  // 1 / sumdeg
    int est_delayed;                    // 1: delayed-sum error estimate (RD_Q_EST_DELAYED)
    const double* block_part;
    PairState st;
    int64_t pstride;                    // stride of the per-pair [k][pair] arrays (original ld)
    const int32_t* slot_pair;           // column slot -> pair (-1: empty); NULL = identity
    void* cf_step;                      // T [4][ld]: rows 1..3 receive alpha_i, c_i, 1/beta_{i+1}
    void* cf_next;                      // T [4][ld]: row 0 receives beta_{i+1} for the next step
    int elem_size;
    const int32_t* step_dev;            // nullable: step index from device memory (graph replay);
    int64_t cf_stride;                  // then cf_step/cf_next advance by j * cf_stride
    int df;                             // 1: coefficients are stored as double-float pairs
    void* xcf;                          // nullable T [k_max][2][ld]: step j receives lambda_i, mu_i
                                        // of the potential's direct update (identity slot map only)
};

// Whole recurrence of one pair per CTA with q_{i-1}, q_i and W in shared memory (graphs
// small enough); reads the CSR from global memory (L1/L2 resident).
struct OnchipArgs {
    int64_t n;
    int npairs;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w;
    const double* deg64;
    const double* invdeg64;
    const float* deg32;
    const float* invdeg32;
    const int32_t* s;
    const int32_t* t;
    int heavy_thr;
    int64_t n_heavy_rows;
    const int32_t* heavy_rows;
    FinArgs fin;                  // stop rule, tolerances, per-pair state
    int elem_size, weighted;
    int sm_count;                 // SMs of the device (cluster size choice)
    int allow_cluster;            // 0: one CTA per pair (RD_Q_NO_CLUSTER)
};
size_t onchip_smem_bytes(int64_t n, int elem_size);
// Launches the whole-recurrence kernel; returns the CTAs per pair used (1: one CTA per pair,
// 2..16: a thread-block cluster per pair), or 0 if the graph does not fit.
int launch_onchip(cudaStream_t st, const OnchipArgs& a);

// Column compaction: keep the slots whose pair is still active, in slot order.
struct CompactArgs {
    int64_t n, ld_old, ld_new;
    const int32_t* slot_pair_old;       // NULL = identity over npairs
    int npairs;
    int32_t* slot_pair_new;             // ld_new
    int32_t* old_slot;                  // ld_new: source slot or -1
    const int32_t* active;              // per pair
    const void* cf_old;                 // T [4][ld_old]
    void* cf_new;                       // T [4][ld_new]
    const void* q_src0;                 // T n x ld_old
    const void* q_src1;
    void* q_dst0;                       // T n x ld_new
    void* q_dst1;
    int elem_size;
};
void launch_compact(cudaStream_t st, int grid, const CompactArgs& a);
// the slot maps and the packed coefficients only (the q blocks packed by the caller)
void launch_compact_map(cudaStream_t st, const CompactArgs& a);

// Power Method (Algorithm 1) in y = D^{-1} r: start y = D^{-1}(e_s - e_t), accumulate
// rbar += (y_s - y_t)/2 per step (r(s)/(2 d_s) - r(t)/(2 d_t) of Algorithm 1).
struct PmArgs {
    int64_t n, ld;
    int npairs;
    const int32_t* s;
    const int32_t* t;
    const double* deg64;
    void* y;                      // T n x ld
    double* rbar;                 // npairs
    double* hist;                 // nullable: [step][npairs]
    int step, elem_size;
    int32_t* err_flag;
};
void launch_pm_init(cudaStream_t st, const PmArgs& a);
void launch_pm_accum(cudaStream_t st, const PmArgs& a);

// --------------------------------------------------------------- graph
struct Workspace {
    void* base = nullptr;
    size_t bytes = 0;
};

}  // namespace rd

struct rd_graph {
    int device = 0, sm_count = 0;
    int64_t n = 0, nnz = 0, nnz_in = 0;
    bool weighted = false;
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    float* w = nullptr;
    int64_t* keep_idx = nullptr;      // internal entry -> original entry (only if self-loops dropped)
    double* deg64 = nullptr;
    double* invdeg64 = nullptr;
    float* deg32 = nullptr;
    float* invdeg32 = nullptr;
    rd::df64* degdf = nullptr;        // double-float copies (built on first use)
    rd::df64* invdegdf = nullptr;
    double sumdeg = 0.0;
    int32_t* comp = nullptr;
    int32_t ncomp = 0;
    // heavy-row chunks
    int heavy_thr = 256;
    int64_t n_heavy_rows = 0, n_chunks = 0;
    int32_t* heavy_rows = nullptr;
    int32_t* heavy_first = nullptr;
    int32_t* chunk_beg = nullptr;
    int32_t* chunk_end = nullptr;
    // row-stream tasks: consecutive rows with at most task_nnz nonzeros, heavy rows alone
    int task_nnz = 512;
    int64_t ntasks = 0;
    int32_t* task_row = nullptr;
    // rows by decreasing degree (stable: equal degrees in row order)
    int32_t* row_order = nullptr;
    // row of every stored entry (built on first use by the per-entry kernels)
    int32_t* entry_row = nullptr;

    bool rows_sorted_sym = false;     // rows strictly increasing in column, entries symmetric
    double mean_deg = 0.0;
    rd::Workspace ws;
    rd_call_stats stats{};
    int* h_pinned = nullptr;          // small pinned host buffer for polls
    int64_t l2_bytes = 0;             // device L2 size
    // SpMM configurations chosen by the autotuner on this graph, per width class
    struct TunedCfg {
        int prec = 0, single = 0;     // element precision (0 FP32, 1 FP64, 2 double-float); one column or many
        int64_t width = 0;            // width class (power-of-two tile holding the pairs; 1 if single)
        rd::SpmmCfg cfg;
        float us = 0.f;               // measured time of one SpMM launch pair
    };
    std::vector<TunedCfg> tuned;
    // instantiated CUDA graphs of two Lanczos steps, keyed by the bytes of their launch
    // arguments (oldest evicted first), and the stream they are captured on
    std::vector<std::pair<std::string, cudaGraphExec_t>> graphs;
    cudaStream_t capture_stream = nullptr;
};

namespace rd {

// Launchers (defined in the kernel translation units).
// Returns false if the configuration is not instantiated.
bool launch_spmm_f32(const SpmmCfg& c, bool weighted, bool heavy, int grid, cudaStream_t st,
                     const StepArgs<float>& a);
bool launch_spmm_df64(const SpmmCfg& c, bool weighted, bool heavy, int grid, cudaStream_t st,
                      const StepArgs<df64>& a);
bool launch_spmm_f64(const SpmmCfg& c, bool weighted, bool heavy, int grid, cudaStream_t st,
                     const StepArgs<double>& a);
// prec: 0 FP32 vectors, 1 FP64, 2 double-float
int spmm_blocks_per_sm(const SpmmCfg& c, bool weighted, bool heavy, int prec);
std::vector<SpmmCfg> spmm_configs(bool fp64);

void launch_normalize_f32(int grid, cudaStream_t st, const NormArgs<float>& a);
void launch_normalize_f64(int grid, cudaStream_t st, const NormArgs<double>& a);
void launch_normalize_df64(int grid, cudaStream_t st, const NormArgs<df64>& a);
// false when the packed layout has no whole 16-byte units (the caller then packs separately)
bool launch_normalize_pack_f32(int grid, cudaStream_t st, const NormPackArgs<float>& a);
bool launch_normalize_pack_f64(int grid, cudaStream_t st, const NormPackArgs<double>& a);
bool launch_normalize_pack_df64(int grid, cudaStream_t st, const NormPackArgs<df64>& a);
void launch_split_df(cudaStream_t st, int grid, int64_t n, const double* src, df64* dst);
void launch_finalize(cudaStream_t st, const FinArgs& a);
// Advance the device step index by one, saturating at `limit` (end of a replayed step).
void launch_step_advance(cudaStream_t st, int32_t* step, int limit);
// Condition kernels of the device-resident step loop (a conditional while node). Before step
// j (*step = j): continue while pairs are active, k_max is not reached and no column
// compaction is due. After step j's finalize (after_finalize = 1): stop if a compaction is
// due before step j + 1, with step j's normalise pass still to run (the host runs it fused
// with the packing). On stop, record j, the active count the compaction test read, the
// active count entering the next step, and where the loop stopped (0 before the step, 1
// after its finalize) in saved[0..3], and park *step at k_max + 1.
void launch_loop_cond(cudaStream_t st, cudaGraphConditionalHandle h, int32_t* step, const int32_t* act_count,
                      int32_t* saved, const int32_t* compact_from, int k_max, int64_t ld, int compact_check, int lag,
                      int after_finalize);

struct InitArgs {
    int64_t n, ld;
    int npairs, k_max, elem_size;
    int df;                       // 1: vectors are double-float pairs (elem_size 8)
    const int32_t* s;
    const int32_t* t;
    const double* deg64;
    const int32_t* comp;          // nullable
    void* qcur;                   // T n x ld (zeroed before)
    PairState st;
    int32_t* err_flag;
    int replay;                   // 1: only rebuild q_1 (the per-pair state is left untouched)
};
void launch_init(cudaStream_t st, const InitArgs& a);

struct OutArgs {
    int npairs;
    int64_t ld;
    PairState st;
    double* r_out;
    int32_t* iters_out;
    double* err_out;
    int32_t* status_out;
    int32_t* summary;            // [0]: any not converged, [1]: any numeric
};
void launch_output(cudaStream_t st, const OutArgs& a);

struct ZsolveArgs {
    int npairs;
    int64_t ld;
    int k_max;
    PairState st;
    const double* grad_r;         // nullable (ones)
    void* coef_hist;              // T [k_max][ld]: sqrt(b2) * z_j (0 beyond k_p)
    void* gbar;                   // T [ld]: upstream gradient per column (0 if unused)
    double* zscratch;             // [k_max][2][ld]
    int elem_size;
};
void launch_zsolve(cudaStream_t st, const ZsolveArgs& a);

template <typename T>
struct EdgeGradArgs {
    int64_t n, ld, nnz;
    int npairs;
    const int64_t* row_ptr;
    const int32_t* col;
    const int32_t* entry_row;     // row of each stored entry (nnz)
    const T* phi;                 // n x ld
    const T* gbar;                // ld
    float* grad_out;              // internal entries
};
void launch_edge_grad_f32(int grid, cudaStream_t st, const EdgeGradArgs<float>& a);
void launch_edge_grad_f64(int grid, cudaStream_t st, const EdgeGradArgs<double>& a);
void launch_entry_rows(int grid, cudaStream_t st, int64_t n, const int64_t* row_ptr, int32_t* entry_row);


// First Lanczos step from the sparse start vector (two nonzeros per column).
template <typename T>
struct Step0Args {
    int64_t n, ld;
    int npairs;
    int tp;                       // column tile of the plan (layout of block_part)
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w;               // nullable
    const T* invdeg;
    const double* deg64;
    const int32_t* s;
    const int32_t* t;
    const T* q1;                  // q_1 block (n x ld)
    T* wout;                      // W, written over the zeroed q_0 block
    double* block_part;           // [slab][1][3][TP]: each column's sums as one block (nullable)
};
// Step 0's normalise pass after the sparse first step, in two parts: the rows of
// N(s) ∪ N(t) ∪ {s, t} of each column (k_normalize_step0, marking them in `mask`), then every
// other entry (k_normalize_step0_fill), where W_1 and q_1 are zero.
template <typename T>
struct Step0NormArgs {
    int64_t n, ld;
    int npairs;
    const int64_t* row_ptr;
    const int32_t* col;
    const int32_t* s;
    const int32_t* t;
    const T* q1;                  // q_1 block
    T* w;                         // in: W_1 on those rows (k_step0_sparse's output), out: q_2
    const T* cf;                  // [4][ld]: beta_1, alpha_1, c_1, 1/beta_2
    uint32_t* mask;               // n x ld bits, zero on entry: the entries the first part wrote
};
void launch_normalize_step0_f32(int grid, cudaStream_t st, const Step0NormArgs<float>& a);
void launch_normalize_step0_f64(int grid, cudaStream_t st, const Step0NormArgs<double>& a);
void launch_normalize_step0_df64(int grid, cudaStream_t st, const Step0NormArgs<df64>& a);
void launch_step0_f32(cudaStream_t st, const Step0Args<float>& a);
void launch_step0_f64(cudaStream_t st, const Step0Args<double>& a);
void launch_step0_df64(cudaStream_t st, const Step0Args<df64>& a);

// Graph preparation kernels.
rd_status graph_prepare(rd_graph* g, cudaStream_t st, uint32_t flags);
rd_status rows_sorted_symmetric(rd_graph* g, cudaStream_t st, bool* out);
rd_status graph_weights_changed(rd_graph* g, cudaStream_t st);

}  // namespace rd

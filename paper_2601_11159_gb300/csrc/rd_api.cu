// C ABI of librd (declared in include/rd.h): graph ingest, batched Lanczos queries,
// the recomputing adjoint for edge-weight gradients, and potentials.
//
// The driver runs Algorithm 3 (Section 3) for all pairs at once: per step an SpMM
// (plus a pre-pass for heavy rows), an FP64 finalisation of alpha/beta and of the
// running LDL^T factorisation of I - T_k, and a normalisation pass. The host polls
// the number of active pairs every `chunk_steps` steps; kernels of steps after the
// last active pair has stopped return at once.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "rd_internal.cuh"

namespace rd {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

rd_status cuda_status(cudaError_t e, const char* what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    cudaGetLastError();  // clear a sticky-free error so later calls can proceed
    return e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA;
}

rd_status check_csr(rd_graph* g, cudaStream_t st, int64_t* self_loops);
rd_status compute_degrees(rd_graph* g, cudaStream_t st);
int spmm_blocks_per_sm_f32(const SpmmCfg& c, bool weighted, bool heavy);
int spmm_blocks_per_sm_f64(const SpmmCfg& c, bool weighted, bool heavy);
int spmm_blocks_per_sm_df64(const SpmmCfg& c, bool weighted, bool heavy);
std::vector<SpmmCfg> spmm_configs_f32();
std::vector<SpmmCfg> spmm_configs_f64();

int spmm_blocks_per_sm(const SpmmCfg& c, bool weighted, bool heavy, int prec)
{
    if (prec == 2) return spmm_blocks_per_sm_df64(c, weighted, heavy);
    return prec == 1 ? spmm_blocks_per_sm_f64(c, weighted, heavy) : spmm_blocks_per_sm_f32(c, weighted, heavy);
}

// Element precision of a mode: 0 FP32 vectors, 1 FP64, 2 double-float (8-byte elements
// for 1 and 2, which share the tile configurations).
static int mode_prec(int32_t mode) { return mode == RD_MODE_FP64 ? 1 : (mode == RD_MODE_DF64 ? 2 : 0); }

std::vector<SpmmCfg> spmm_configs(bool fp64) { return fp64 ? spmm_configs_f64() : spmm_configs_f32(); }

static bool cfg_listed(const SpmmCfg& c, bool fp64)
{
    if (c.order && c.kind != 0) return false;  // the row order is a row-group kernel option
    for (const auto& x : spmm_configs(fp64))
        if (x.vec == c.vec && x.gs == c.gs && x.nzl == c.nzl && x.kind == c.kind) return true;
    return false;
}

// A step configuration is usable when it and its heavy-row pre-pass are instantiated.
static bool cfg_known(const SpmmCfg& c, bool fp64) { return cfg_listed(c, fp64) && cfg_listed(heavy_cfg(c), fp64); }

// ------------------------------------------------------------- helpers
static bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename X>
    X* take(size_t count)
    {
        off = (off + 255) & ~size_t(255);
        X* p = reinterpret_cast<X*>(base ? base + off : nullptr);
        off += sizeof(X) * (count ? count : 1);
        return p;
    }
};

static rd_status ensure_ws(rd_graph* g, size_t bytes)
{
    if (g->ws.bytes >= bytes) return RD_OK;
    if (g->ws.base) {
        cudaFree(g->ws.base);
        g->ws.base = nullptr;
        g->ws.bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("workspace allocation of " + std::to_string(bytes) + " bytes failed");
        return RD_ERR_OOM;
    }
    g->ws.base = p;
    g->ws.bytes = bytes;
    return RD_OK;
}

// --------------------------------------------------------------- graph
static void free_graph(rd_graph* g)
{
    if (!g) return;
    void* ptrs[] = {g->row_ptr, g->col, g->w, g->keep_idx, g->deg64, g->invdeg64, g->deg32, g->invdeg32,
                    g->comp, g->heavy_rows, g->heavy_first, g->chunk_beg, g->chunk_end, g->task_row,
                    g->row_order, g->entry_row, g->degdf, g->invdegdf, g->ws.base};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (g->h_pinned) cudaFreeHost(g->h_pinned);
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    delete g;
}

// Union-find over the CSR on the host (path halving, union by smaller root id);
// labels are the root id of each vertex's component, made dense afterwards.
static int32_t label_components(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& col,
                                 std::vector<int32_t>& lab)
{
    std::vector<int32_t> par(n);
    std::iota(par.begin(), par.end(), 0);
    auto find = [&](int32_t x) {
        while (par[x] != x) {
            par[x] = par[par[x]];
            x = par[x];
        }
        return x;
    };
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t a = find((int32_t)u), b = find(col[e]);
            if (a != b) {
                if (a < b) par[b] = a; else par[a] = b;
            }
        }
    lab.assign(n, -1);
    std::vector<int32_t> dense(n, -1);
    int32_t nc = 0;
    for (int64_t u = 0; u < n; ++u) {
        int32_t r = find((int32_t)u);
        if (dense[r] < 0) dense[r] = nc++;
        lab[u] = dense[r];
    }
    return nc;
}

static rd_status build_heavy(rd_graph* g, const std::vector<int64_t>& rp)
{
    std::vector<int32_t> rows, first, cb, ce;
    first.push_back(0);
    for (int64_t u = 0; u < g->n; ++u) {
        const int64_t d = rp[u + 1] - rp[u];
        if (d > g->heavy_thr) {
            rows.push_back((int32_t)u);
            for (int64_t e = rp[u]; e < rp[u + 1]; e += g->heavy_thr) {
                cb.push_back((int32_t)e);
                ce.push_back((int32_t)std::min<int64_t>(e + g->heavy_thr, rp[u + 1]));
            }
            first.push_back((int32_t)cb.size());
        }
    }
    g->n_heavy_rows = (int64_t)rows.size();
    g->n_chunks = (int64_t)cb.size();
    // row-stream tasks: greedy runs of consecutive light rows with at most task_nnz nonzeros
    // (a single light row longer than that stays whole); each heavy row is a task of its own
    std::vector<int32_t> tasks;
    tasks.push_back(0);
    int64_t cur = 0;
    for (int64_t u = 0; u < g->n; ++u) {
        const int64_t d = rp[u + 1] - rp[u];
        if (d > g->heavy_thr) {
            if (tasks.back() != (int32_t)u) tasks.push_back((int32_t)u);
            tasks.push_back((int32_t)(u + 1));
            cur = 0;
            continue;
        }
        if (cur > 0 && cur + d > g->task_nnz) {
            tasks.push_back((int32_t)u);
            cur = 0;
        }
        cur += d;
    }
    if (tasks.back() != (int32_t)g->n) tasks.push_back((int32_t)g->n);
    g->ntasks = (int64_t)tasks.size() - 1;
    RD_CUDA(cudaMalloc((void**)&g->task_row, sizeof(int32_t) * tasks.size()));
    RD_CUDA(cudaMemcpy(g->task_row, tasks.data(), sizeof(int32_t) * tasks.size(), cudaMemcpyHostToDevice));
    // rows by decreasing degree, stable (counting sort on the degree)
    {
        int64_t dmax = 0;
        for (int64_t u = 0; u < g->n; ++u) dmax = std::max<int64_t>(dmax, rp[u + 1] - rp[u]);
        std::vector<int64_t> start((size_t)dmax + 2, 0);
        for (int64_t u = 0; u < g->n; ++u) ++start[(size_t)(dmax - (rp[u + 1] - rp[u])) + 1];
        for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
        std::vector<int32_t> order((size_t)std::max<int64_t>(g->n, 1));
        for (int64_t u = 0; u < g->n; ++u) order[(size_t)start[(size_t)(dmax - (rp[u + 1] - rp[u]))]++] = (int32_t)u;
        RD_CUDA(cudaMalloc((void**)&g->row_order, sizeof(int32_t) * order.size()));
        RD_CUDA(cudaMemcpy(g->row_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice));
    }
    if (g->n_heavy_rows == 0) return RD_OK;
    RD_CUDA(cudaMalloc((void**)&g->heavy_rows, sizeof(int32_t) * rows.size()));
    RD_CUDA(cudaMalloc((void**)&g->heavy_first, sizeof(int32_t) * first.size()));
    RD_CUDA(cudaMalloc((void**)&g->chunk_beg, sizeof(int32_t) * cb.size()));
    RD_CUDA(cudaMalloc((void**)&g->chunk_end, sizeof(int32_t) * ce.size()));
    RD_CUDA(cudaMemcpy(g->heavy_rows, rows.data(), sizeof(int32_t) * rows.size(), cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(g->heavy_first, first.data(), sizeof(int32_t) * first.size(), cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(g->chunk_beg, cb.data(), sizeof(int32_t) * cb.size(), cudaMemcpyHostToDevice));
    RD_CUDA(cudaMemcpy(g->chunk_end, ce.data(), sizeof(int32_t) * ce.size(), cudaMemcpyHostToDevice));
    return RD_OK;
}

static rd_status symmetric_check(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& col,
                                 const std::vector<float>& w)
{
    struct E {
        int64_t key;
        float w;
    };
    const int64_t nnz = rp[n];
    std::vector<E> fwd(nnz), bwd(nnz);
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            const float x = w.empty() ? 1.0f : w[e];
            fwd[e] = E{u * n + col[e], x};
            bwd[e] = E{(int64_t)col[e] * n + u, x};
        }
    auto lt = [](const E& a, const E& b) { return a.key < b.key || (a.key == b.key && a.w < b.w); };
    std::sort(fwd.begin(), fwd.end(), lt);
    std::sort(bwd.begin(), bwd.end(), lt);
    for (int64_t e = 0; e < nnz; ++e)
        if (fwd[e].key != bwd[e].key || fwd[e].w != bwd[e].w) {
            set_error("the CSR is not symmetric: entry (" + std::to_string(fwd[e].key / n) + ", " +
                      std::to_string(fwd[e].key % n) + ") has no mirror with equal weight");
            return RD_ERR_INVALID_ARG;
        }
    return RD_OK;
}

static rd_status graph_build(rd_graph* g, const int64_t* row_ptr, const int32_t* col_idx, const float* weights,
                             uint32_t flags, cudaStream_t st)
{
    const int64_t n = g->n, nnz = g->nnz_in;
    RD_CUDA(cudaMalloc((void**)&g->row_ptr, sizeof(int64_t) * (n + 1)));
    RD_CUDA(cudaMalloc((void**)&g->col, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    if (weights) RD_CUDA(cudaMalloc((void**)&g->w, sizeof(float) * std::max<int64_t>(nnz, 1)));
    RD_CUDA(cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, st));
    if (nnz) RD_CUDA(cudaMemcpyAsync(g->col, col_idx, sizeof(int32_t) * nnz, cudaMemcpyDefault, st));
    if (weights && nnz) RD_CUDA(cudaMemcpyAsync(g->w, weights, sizeof(float) * nnz, cudaMemcpyDefault, st));
    g->weighted = weights != nullptr;
    g->nnz = nnz;
    int64_t loops = 0;
    RD_TRY(check_csr(g, st, &loops));

    const bool need_full = loops > 0 || (flags & (RD_CHECK_SYMMETRY | RD_LABEL_COMPONENTS));
    std::vector<int64_t> rp(n + 1);
    std::vector<int32_t> col;
    std::vector<float> w;
    RD_CUDA(cudaMemcpyAsync(rp.data(), g->row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    if (need_full) {
        col.resize(nnz);
        if (nnz) RD_CUDA(cudaMemcpyAsync(col.data(), g->col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st));
        if (g->weighted) {
            w.resize(nnz);
            if (nnz) RD_CUDA(cudaMemcpyAsync(w.data(), g->w, sizeof(float) * nnz, cudaMemcpyDeviceToHost, st));
        }
    }
    RD_CUDA(cudaStreamSynchronize(st));

    if (loops > 0) {  // drop self-loops (they cancel in L = D - W), keep the entry map
        std::vector<int64_t> rp2(n + 1, 0), keep;
        std::vector<int32_t> col2;
        std::vector<float> w2;
        keep.reserve(nnz - loops);
        for (int64_t u = 0; u < n; ++u) {
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                if (col[e] == (int32_t)u) continue;
                keep.push_back(e);
                col2.push_back(col[e]);
                if (g->weighted) w2.push_back(w[e]);
            }
            rp2[u + 1] = (int64_t)col2.size();
        }
        rp.swap(rp2);
        col.swap(col2);
        w.swap(w2);
        g->nnz = (int64_t)col.size();
        RD_CUDA(cudaMalloc((void**)&g->keep_idx, sizeof(int64_t) * std::max<size_t>(keep.size(), 1)));
        RD_CUDA(cudaMemcpy(g->row_ptr, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
        if (g->nnz) {
            RD_CUDA(cudaMemcpy(g->keep_idx, keep.data(), sizeof(int64_t) * keep.size(), cudaMemcpyHostToDevice));
            RD_CUDA(cudaMemcpy(g->col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice));
            if (g->weighted) RD_CUDA(cudaMemcpy(g->w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice));
        }
    }
    if (flags & RD_CHECK_SYMMETRY) RD_TRY(symmetric_check(n, rp, col, w));

    RD_CUDA(cudaMalloc((void**)&g->deg64, sizeof(double) * n));
    RD_CUDA(cudaMalloc((void**)&g->invdeg64, sizeof(double) * n));
    RD_CUDA(cudaMalloc((void**)&g->deg32, sizeof(float) * n));
    RD_CUDA(cudaMalloc((void**)&g->invdeg32, sizeof(float) * n));
    RD_TRY(compute_degrees(g, st));
    RD_TRY(build_heavy(g, rp));
    RD_TRY(rows_sorted_symmetric(g, st, &g->rows_sorted_sym));
    if (flags & RD_LABEL_COMPONENTS) {
        std::vector<int32_t> lab;
        g->ncomp = label_components(n, rp, col, lab);
        RD_CUDA(cudaMalloc((void**)&g->comp, sizeof(int32_t) * n));
        RD_CUDA(cudaMemcpy(g->comp, lab.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    }
    RD_CUDA(cudaMallocHost((void**)&g->h_pinned, 64));
    return RD_OK;
}

// ------------------------------------------------------------- planning
struct Plan {
    bool fp64;              // 8-byte vector elements (FP64 or double-float)
    int prec = 0;           // mode_prec
    bool tuned = false;     // cfg taken from the autotuner's table
    SpmmCfg cfg;
    int64_t ld;
    int grid_main, grid_heavy, grid_norm, nslab;
    int k_max;
    size_t elem;
};

// ------------------------------------------------------------- autotuner keys
// The tuner times the candidate SpMM configurations of a query width on the graph itself
// and keeps the fastest per (precision, single-column or batched, width class); widths are
// classed by the smallest power-of-two tile that holds them.
// rd_query_opts::kernel / rd_call_stats::kernel number of a configuration.
static int kernel_code(const SpmmCfg& c)
{
    if (c.kind == 3) return 5;
    if (c.kind == 2) return 4;
    if (c.kind == 1) return 2;
    return c.order ? 3 : 1;
}

static bool tuning_allowed(const rd_query_opts& o)
{
    return o.kernel == 0 && o.rhs_tile <= 0 && o.rows_per_warp <= 0 && (o.flags & RD_Q_NO_TUNE) == 0;
}

static int64_t tune_width(int64_t P, bool fp64, bool single)
{
    if (single) return 1;
    const int64_t tmin = fp64 ? 8 : 16, tmax = fp64 ? 128 : 256;
    int64_t w = tmin;
    while (w < P && w < tmax) w <<= 1;
    return w;
}

static const rd_graph::TunedCfg* find_tuned(const rd_graph* g, int prec, bool single, int64_t width)
{
    for (const auto& t : g->tuned)
        if (t.prec == prec && t.single == (int)single && t.width == width) return &t;
    return nullptr;
}

static SpmmCfg pick_cfg(const rd_graph* g, int64_t P, const rd_query_opts& o, bool fp64, bool plain,
                        bool* from_table = nullptr)
{
    const double mdeg = g->n ? (double)g->nnz / (double)g->n : 0.0;
    if (from_table) *from_table = false;
    if (tuning_allowed(o)) {
        const bool single = plain || P == 1;
        const rd_graph::TunedCfg* t = find_tuned(g, mode_prec(o.mode), single, tune_width(P, fp64, single));
        if (t) {
            if (from_table) *from_table = true;
            return t->cfg;
        }
    }
    SpmmCfg c;
    if (plain || P == 1) {
        c.vec = 1;
        c.gs = 1;
        // warp-per-task SpMV (also for kernel 5, whose slabs need more than one column)
        if ((o.kernel == 0 || o.kernel == 4 || o.kernel == 5) && g->ntasks > 0) {
            c.nzl = 1;
            c.kind = 2;
            return c;
        }
        if (o.kernel == 2) {  // row-stream with one lane per task
            c.nzl = 1;
            c.kind = 1;
            return c;
        }
        c.nzl = mdeg <= 6 ? 4 : (mdeg <= 12 ? 8 : (mdeg <= 24 ? 16 : 32));
        if (o.rows_per_warp > 0) c.nzl = std::max(1, std::min(32, 32 / o.rows_per_warp));
        c.order = o.kernel == 3 && g->row_order ? 1 : 0;
        return c;
    }
    if (o.kernel == 4) {  // single-column only: no such tile (make_plan reports it)
        c.kind = 2;
        c.vec = 2;
        return c;
    }
    if (o.kernel == 5) {  // async row-stream: tiles of 16 to 128 FP32 columns, 16 to 64 of 8-byte elements
        int tpa = o.rhs_tile > 0 ? o.rhs_tile : (P <= 16 ? 16 : (P <= 32 ? 32 : (P <= 64 || fp64 ? 64 : 128)));
        c.vec = fp64 ? 2 : 4;
        c.gs = std::max(1, tpa / c.vec);
        c.nzl = 1;
        c.kind = 3;
        return c;
    }
    int tp = o.rhs_tile;
    if (tp <= 0) {
        if (fp64) tp = P <= 8 ? 8 : (P <= 16 ? 16 : (P <= 32 ? 32 : 64));
        else tp = P <= 16 ? 16 : (P <= 32 ? 32 : (P <= 64 ? 64 : (P <= 128 ? 128 : 256)));
    }
    c.vec = fp64 ? (tp >= 128 ? 4 : 2) : (tp >= 256 ? 8 : 4);
    c.gs = std::max(1, tp / c.vec);
    c.nzl = 1;
    c.kind = o.kernel == 1 || o.kernel == 3 ? 0 : 1;  // row-stream unless a row-group kernel is asked for
    c.order = o.kernel == 3 && g->row_order ? 1 : 0;
    if (c.kind == 0 && o.rows_per_warp > 0) c.nzl = std::max(1, 32 / (c.gs * o.rows_per_warp));
    return c;
}

static rd_status make_plan_cfg(rd_graph* g, int64_t P, const rd_query_opts& o, const SpmmCfg& cfg, Plan* pl)
{
    pl->prec = mode_prec(o.mode);
    pl->fp64 = pl->prec != 0;
    pl->elem = pl->fp64 ? 8 : 4;
    pl->cfg = cfg;
    if (!cfg_known(pl->cfg, pl->fp64)) {
        set_error("no SpMM kernel for rhs_tile/rows_per_warp = " + std::to_string(pl->cfg.tp()) + "/" +
                  std::to_string(pl->cfg.rpw()));
        return RD_ERR_UNSUPPORTED;
    }
    const int tp = pl->cfg.tp();
    pl->ld = ((P + tp - 1) / tp) * tp;
    pl->nslab = (int)(pl->ld / tp);
    pl->k_max = o.k_max;
    const int rows_per_block = kWarps * pl->cfg.rpw();
    int bps = spmm_blocks_per_sm(pl->cfg, g->weighted, false, pl->prec);
    if (bps < 1) bps = 1;
    int64_t gm = (int64_t)bps * g->sm_count;
    int64_t units = pl->cfg.kind == 1 || pl->cfg.kind == 3 ? g->ntasks : g->n;  // rows or tasks, one per row group
    int64_t per_block = rows_per_block;
    if (pl->cfg.kind == 2) {  // one task per warp
        units = g->ntasks;
        per_block = kWarps;
    }
    gm = std::min<int64_t>(gm, (units + per_block - 1) / per_block);
    pl->grid_main = (int)std::max<int64_t>(gm, 1);
    int bph = spmm_blocks_per_sm(pl->cfg, g->weighted, true, pl->prec);
    if (bph < 1) bph = 1;
    int64_t gh = (int64_t)bph * g->sm_count;
    const int chunks_per_block = kWarps * heavy_cfg(pl->cfg).rpw();
    gh = std::min<int64_t>(gh, (g->n_chunks + chunks_per_block - 1) / chunks_per_block);
    pl->grid_heavy = (int)std::max<int64_t>(gh, 1);
    const int64_t vunits = (g->n * pl->ld) / (16 / (int64_t)pl->elem) + 1;
    pl->grid_norm = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * 8, (vunits + 255) / 256));
    return RD_OK;
}

static rd_status make_plan(rd_graph* g, int64_t P, const rd_query_opts& o, bool plain, Plan* pl)
{
    bool from_table = false;
    const SpmmCfg cfg = pick_cfg(g, P, o, mode_prec(o.mode) != 0, plain, &from_table);
    RD_TRY(make_plan_cfg(g, P, o, cfg, pl));
    pl->tuned = from_table;
    return RD_OK;
}

// ---------------------------------------------------------- workspace map
struct Buffers {
    void* q[2];               // current q_{i-1}/W (slot 0) and q_i (slot 1)
    void* region_a;           // the two n x ld0 blocks q[] start in
    void* region_x;           // n x ld0 elements: target of a column compaction (NULL if off)
    void* heavy_part;
    double* block_part;
    void* cf_hist;            // [k_max+1][4][ld0] (fixed layout: gradient, potential, no-alloc)
    void* cf_cur[2];          // [4][ld0] current coefficients by slot (compacting query)
    int32_t* slot_pair[2];    // [ld0] slot -> pair after a compaction
    int32_t* old_slot;        // [ld0] scratch of the compaction
    PairState st;
    int32_t* s;
    int32_t* t;
    double* r;
    int32_t* iters;
    double* err;
    int32_t* status;
    int32_t* summary;
    int32_t* err_flag;
    int32_t* step_dev;        // step index of graph-replayed steps (zeroed per query)
    int32_t* loop_saved;      // [4]: where the device-resident loop stopped (see launch_loop_cond)
    int32_t* loop_cfrom;      // first step at which the loop tests for a column compaction
    uint32_t* row_mask;       // n x ld bits: entries of q_2 the sparse first normalise pass wrote
    // gradient / potential
    void* phi;
    void* pvec;               // n x ld0: direction vectors of the potential's direct update
    void* xcf;                // [k_max][2][ld0]: their coefficients (zeroed per query)
    void* coef_hist;
    void* gbar;
    double* zscratch;
    float* grad;
    size_t state_bytes_begin, state_bytes_end;  // offsets of the region zeroed per query
};

// Byte size of an n x ld block rounded up to 256 bytes, so that every block that follows
// another inside a region starts 256-byte aligned (the kernels use 16-byte vector accesses).
static int64_t block_bytes(int64_t n, int64_t ld, size_t elem)
{
    return ((n * ld * (int64_t)elem) + 255) & ~int64_t(255);
}

static size_t carve(Carver& c, const rd_graph* g, const Plan& pl, int64_t P, bool grad, Buffers* b,
                    bool compact = false)
{
    const int64_t ld = pl.ld, n = g->n, K = pl.k_max;
    b->region_a = c.take<char>(2 * block_bytes(n, ld, pl.elem));
    b->q[0] = b->region_a;
    b->q[1] = static_cast<char*>(b->region_a) + block_bytes(n, ld, pl.elem);
    // spare region: two packed blocks of at most ld/2 columns, each rounded to 256 bytes
    b->region_x = compact ? c.take<char>(block_bytes(n, ld, pl.elem) + 512) : nullptr;
    b->heavy_part = c.take<char>(std::max<int64_t>(g->n_chunks, 1) * ld * pl.elem);
    // sized for any column tile and any grid of up to 8 blocks of kBlock threads per SM
    b->block_part = c.take<double>((size_t)ld * 3 * (size_t)std::max(pl.grid_main, g->sm_count * 8));
    b->old_slot = c.take<int32_t>(ld);
    b->slot_pair[0] = c.take<int32_t>(ld);
    b->slot_pair[1] = c.take<int32_t>(ld);
    c.off = (c.off + 255) & ~size_t(255);
    b->state_bytes_begin = c.off;
    b->cf_hist = compact ? nullptr : c.take<char>((K + 1) * 4 * ld * pl.elem);
    b->cf_cur[0] = compact ? c.take<char>(4 * ld * pl.elem) : nullptr;
    b->cf_cur[1] = compact ? c.take<char>(4 * ld * pl.elem) : nullptr;
    PairState& s = b->st;
    s.b2 = c.take<double>(ld);
    s.delta = c.take<double>(ld);
    s.g = c.take<double>(ld);
    s.S = c.take<double>(ld);
    s.beta = c.take<double>(ld);
    s.ring = c.take<double>(kRing * ld);
    s.r = c.take<double>(ld);
    s.err = c.take<double>(ld);
    s.resid = c.take<double>(ld);
    s.k = c.take<int32_t>(ld);
    s.status = c.take<int32_t>(ld);
    s.active = c.take<int32_t>(ld);
    s.hist_alpha = c.take<double>(K * ld);
    s.hist_beta = c.take<double>((K + 1) * ld);
    s.act_count = c.take<int32_t>(K + 2);
    b->summary = c.take<int32_t>(2);
    b->err_flag = c.take<int32_t>(1);
    b->step_dev = c.take<int32_t>(1);
    b->loop_saved = c.take<int32_t>(4);
    b->loop_cfrom = c.take<int32_t>(1);
    // queries on graphs that take the sparse first step (rows sorted, symmetric)
    b->row_mask = (!grad && g->rows_sorted_sym) ? c.take<uint32_t>((n * ld + 31) / 32) : nullptr;
    b->xcf = grad ? c.take<char>(K * 2 * ld * pl.elem) : nullptr;
    c.off = (c.off + 255) & ~size_t(255);
    b->state_bytes_end = c.off;
    b->s = c.take<int32_t>(P);
    b->t = c.take<int32_t>(P);
    b->r = c.take<double>(P);
    b->iters = c.take<int32_t>(P);
    b->err = c.take<double>(P);
    b->status = c.take<int32_t>(P);
    if (grad) {
        b->phi = c.take<char>(n * ld * pl.elem);
        b->pvec = c.take<char>(n * ld * pl.elem);
        b->coef_hist = c.take<char>(K * ld * pl.elem);
        b->gbar = c.take<char>(ld * pl.elem);
        b->zscratch = c.take<double>(K * 2 * ld);
        b->grad = c.take<float>(std::max<int64_t>(g->nnz_in, 1));
    } else {
        b->phi = b->coef_hist = b->gbar = nullptr;
        b->zscratch = nullptr;
        b->grad = nullptr;
    }
    return c.off + 256;
}

struct EventPool {
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    cudaEvent_t get()
    {
        if (used == ev.size()) {
            cudaEvent_t e;
            cudaEventCreateWithFlags(&e, cudaEventDefault);
            ev.push_back(e);
        }
        return ev[used++];
    }
    ~EventPool()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

// --------------------------------------------------------------- one run
struct RunCtx {
    rd_graph* g;
    Plan pl;                // plan the workspace was carved for (ld0 = pl.ld)
    Plan cur;               // plan in force (narrower after a column compaction)
    Buffers b;
    rd_query_opts o;
    cudaStream_t st;
    int64_t P;
    int steps = 0;          // steps enqueued
    int64_t launches = 0, spmm_launches = 0;
    double spmm_bytes = 0.0;
    bool profile = false;
    bool compact = false;   // coefficients by slot in cf_cur, columns packed as pairs finish
    bool lagged_polls = false;
    int cf_sel = 0, slot_sel = -1;  // slot_sel < 0: identity slot map
    bool in_region_x = false;
    bool lazy_walk = false;  // Power Method steps instead of Lanczos steps
    bool onchip = false;     // whole recurrence per pair in one kernel (small graphs, queries only)
    int onchip_ctas = 0;     // CTAs per pair it ran with (1, or a cluster of 2..16)
    bool graph = false;      // steps replayed from a captured CUDA graph of one step
    bool device_loop = false;  // steps after the first run by the device-resident loop
    bool sparse_first = false;  // first step run by k_step0_sparse
    bool pot_x = false;      // potential accumulated during the forward steps (k_normalize_pot)
    int compactions = 0;
    EventPool* ev = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spmm_ev;
};

static double spmm_launch_bytes(const rd_graph* g, const Plan& p)
{
    const double nnz = (double)g->nnz;
    return 4.0 * nnz + (g->weighted ? 4.0 * nnz : 0.0) + 8.0 * (double)(g->n + 1) +
           3.0 * (double)p.ld * (double)g->n * (double)p.elem;
}

template <typename T>
static const T* coef_block(RunCtx& c, int j)
{
    if (c.compact) return static_cast<const T*>(c.b.cf_cur[c.cf_sel]);
    return static_cast<const T*>(c.b.cf_hist) + (int64_t)j * 4 * c.cur.ld;
}

template <typename T>
static StepArgs<T> step_args(RunCtx& c, int j, bool reduce)
{
    rd_graph* g = c.g;
    StepArgs<T> a{};
    a.n = g->n;
    a.ld = c.cur.ld;
    a.row_ptr = g->row_ptr;
    a.col = g->col;
    a.w = g->w;
    if constexpr (std::is_same<T, df64>::value) {
        a.invdeg = g->invdegdf;
        a.deg = g->degdf;
    } else if constexpr (sizeof(T) == 8) {
        a.invdeg = g->invdeg64;
        a.deg = g->deg64;
    } else {
        a.invdeg = g->invdeg32;
        a.deg = g->deg32;
    }
    a.qcur = static_cast<const T*>(c.b.q[1]);
    a.qprev_w = static_cast<T*>(c.b.q[0]);
    a.cf_beta = coef_block<T>(c, j);
    a.heavy_thr = g->heavy_thr;
    a.n_heavy_rows = g->n_heavy_rows;
    a.n_chunks = g->n_chunks;
    a.heavy_rows = g->heavy_rows;
    a.heavy_first = g->heavy_first;
    a.chunk_beg = g->chunk_beg;
    a.chunk_end = g->chunk_end;
    a.heavy_part = static_cast<T*>(c.b.heavy_part);
    a.ntasks = g->ntasks;
    a.task_row = g->task_row;
    a.row_order = c.cur.cfg.kind == 0 && c.cur.cfg.order ? g->row_order : nullptr;
    // rows whose current slab fits in half of L2 are gathered with L2 priority
    a.hot_rows = g->l2_bytes > 0 ? (int64_t)(g->l2_bytes / 2) / (c.cur.cfg.tp() * (int64_t)sizeof(T)) : 0;
    a.block_part = c.b.block_part;
    a.active_prev = reduce ? c.b.st.act_count + j : nullptr;
    a.do_reduce = reduce ? 1 : 0;
    a.lazy_walk = c.lazy_walk ? 1 : 0;
    return a;
}

// Launchers by element type.
static bool launch_spmm_t(const SpmmCfg& cfg, bool weighted, bool heavy, int grid, cudaStream_t st,
                          const StepArgs<float>& a)
{
    return launch_spmm_f32(cfg, weighted, heavy, grid, st, a);
}
static bool launch_spmm_t(const SpmmCfg& cfg, bool weighted, bool heavy, int grid, cudaStream_t st,
                          const StepArgs<double>& a)
{
    return launch_spmm_f64(cfg, weighted, heavy, grid, st, a);
}
static bool launch_spmm_t(const SpmmCfg& cfg, bool weighted, bool heavy, int grid, cudaStream_t st,
                          const StepArgs<df64>& a)
{
    return launch_spmm_df64(cfg, weighted, heavy, grid, st, a);
}
static void launch_normalize_t(int grid, cudaStream_t st, const NormArgs<float>& a) { launch_normalize_f32(grid, st, a); }
static void launch_normalize_t(int grid, cudaStream_t st, const NormArgs<double>& a) { launch_normalize_f64(grid, st, a); }
static void launch_normalize_t(int grid, cudaStream_t st, const NormArgs<df64>& a) { launch_normalize_df64(grid, st, a); }
static bool launch_normalize_pack_t(int grid, cudaStream_t st, const NormPackArgs<float>& a)
{
    return launch_normalize_pack_f32(grid, st, a);
}
static bool launch_normalize_pack_t(int grid, cudaStream_t st, const NormPackArgs<double>& a)
{
    return launch_normalize_pack_f64(grid, st, a);
}
static bool launch_normalize_pack_t(int grid, cudaStream_t st, const NormPackArgs<df64>& a)
{
    return launch_normalize_pack_df64(grid, st, a);
}

template <typename T>
static rd_status enqueue_spmm(RunCtx& c, int j, bool reduce)
{
    StepArgs<T> a = step_args<T>(c, j, reduce);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c.profile) {
        e0 = c.ev->get();
        e1 = c.ev->get();
        cudaEventRecord(e0, c.st);
    }
    if (c.g->n_chunks > 0) {
        if (!launch_spmm_t(c.cur.cfg, c.g->weighted, true, c.cur.grid_heavy, c.st, a)) return RD_ERR_UNSUPPORTED;
        ++c.launches;
    }
    if (!launch_spmm_t(c.cur.cfg, c.g->weighted, false, c.cur.grid_main, c.st, a)) return RD_ERR_UNSUPPORTED;
    ++c.launches;
    ++c.spmm_launches;
    c.spmm_bytes += spmm_launch_bytes(c.g, c.cur);
    if (c.profile) {
        cudaEventRecord(e1, c.st);
        c.spmm_ev.emplace_back(e0, e1);
    }
    return RD_OK;
}

template <typename T>
static void enqueue_normalize(RunCtx& c, int j, bool with_phi)
{
    NormArgs<T> a{};
    a.n = c.g->n;
    a.ld = c.cur.ld;
    a.w_to_qnext = static_cast<T*>(c.b.q[0]);
    a.qcur = static_cast<const T*>(c.b.q[1]);
    a.cf = coef_block<T>(c, j);
    a.phi = with_phi ? static_cast<T*>(c.b.phi) : nullptr;
    a.coef = with_phi ? static_cast<const T*>(c.b.coef_hist) + (int64_t)j * c.cur.ld : nullptr;
    a.active_prev = with_phi ? nullptr : c.b.st.act_count + j;
    if (c.pot_x && !with_phi) {
        a.pvec = static_cast<T*>(c.b.pvec);
        a.xvec = static_cast<T*>(c.b.phi);
        a.xcf = static_cast<const T*>(c.b.xcf) + (int64_t)j * 2 * c.cur.ld;
    }
    launch_normalize_t(c.cur.grid_norm, c.st, a);
    ++c.launches;
}

// The first step's product from the sparse start vector (k_step0_sparse) instead of the
// SpMM: for CSR with sorted, symmetric rows (checked once per graph and weight set).
static bool sparse_first_step(const RunCtx& c)
{
    return c.g->rows_sorted_sym && !c.lazy_walk && (c.o.flags & RD_Q_DENSE_FIRST) == 0;
}

// The first step's normalise pass in two sparse-aware parts (k_normalize_step0 + fill): for
// queries (the potential's pass also updates its direction vectors), with the row mask carved
// and whole 16-byte units per row.
static bool sparse_norm_ok(const RunCtx& c)
{
    return !c.pot_x && !c.lazy_walk && c.b.row_mask && c.cur.ld % (16 / (int64_t)c.cur.elem) == 0;
}

static void launch_step0_t(cudaStream_t st, const Step0Args<float>& a) { launch_step0_f32(st, a); }
static void launch_step0_t(cudaStream_t st, const Step0Args<double>& a) { launch_step0_f64(st, a); }
static void launch_step0_t(cudaStream_t st, const Step0Args<df64>& a) { launch_step0_df64(st, a); }
static void launch_norm0_t(int grid, cudaStream_t st, const Step0NormArgs<float>& a)
{
    launch_normalize_step0_f32(grid, st, a);
}
static void launch_norm0_t(int grid, cudaStream_t st, const Step0NormArgs<double>& a)
{
    launch_normalize_step0_f64(grid, st, a);
}
static void launch_norm0_t(int grid, cudaStream_t st, const Step0NormArgs<df64>& a)
{
    launch_normalize_step0_df64(grid, st, a);
}

// Step 0's normalise pass after the sparse first step: the rows next to s and t of each column
// (k_normalize_step0), then every other entry, whose value is the same per column
// (k_normalize_step0_fill); bit for bit the dense pass.
template <typename T>
static void enqueue_normalize_step0(RunCtx& c)
{
    Step0NormArgs<T> a{};
    a.n = c.g->n;
    a.ld = c.cur.ld;
    a.npairs = (int)c.P;
    a.row_ptr = c.g->row_ptr;
    a.col = c.g->col;
    a.s = c.b.s;
    a.t = c.b.t;
    a.q1 = static_cast<const T*>(c.b.q[1]);
    a.w = static_cast<T*>(c.b.q[0]);
    a.cf = coef_block<T>(c, 0);
    a.mask = c.b.row_mask;
    launch_norm0_t(c.cur.grid_norm, c.st, a);
    c.launches += 2;
}

template <typename T>
static void enqueue_step0(RunCtx& c, bool reduce)
{
    const rd_graph* g = c.g;
    Step0Args<T> a{};
    a.n = g->n;
    a.ld = c.cur.ld;
    a.npairs = (int)c.P;
    a.tp = c.cur.cfg.tp();
    a.row_ptr = g->row_ptr;
    a.col = g->col;
    a.w = g->w;
    if constexpr (std::is_same<T, df64>::value) a.invdeg = g->invdegdf;
    else if constexpr (sizeof(T) == 8) a.invdeg = g->invdeg64;
    else a.invdeg = g->invdeg32;
    a.deg64 = g->deg64;
    a.s = c.b.s;
    a.t = c.b.t;
    a.q1 = static_cast<const T*>(c.b.q[1]);
    a.wout = static_cast<T*>(c.b.q[0]);
    a.block_part = reduce ? c.b.block_part : nullptr;
    launch_step0_t(c.st, a);
    ++c.launches;
}

static void enqueue_init(RunCtx& c, bool replay)
{
    const int64_t vbytes = c.g->n * c.cur.ld * (int64_t)c.cur.elem;
    // after the sparse first step the normalise pass writes every entry of the q_0 block
    // (k_normalize_step0 and its fill) and nothing reads it before: no zeros needed there
    if (replay || !sparse_first_step(c) || !sparse_norm_ok(c)) cudaMemsetAsync(c.b.q[0], 0, vbytes, c.st);
    cudaMemsetAsync(c.b.q[1], 0, vbytes, c.st);
    InitArgs a{};
    a.n = c.g->n;
    a.ld = c.cur.ld;
    a.npairs = (int)c.P;
    a.k_max = c.pl.k_max;
    a.elem_size = (int)c.pl.elem;
    a.df = c.pl.prec == 2 ? 1 : 0;
    a.s = c.b.s;
    a.t = c.b.t;
    a.deg64 = c.g->deg64;
    a.comp = c.g->comp;
    a.qcur = c.b.q[1];
    a.err_flag = c.b.err_flag;
    a.replay = replay ? 1 : 0;
    a.st = c.b.st;
    if (!replay) {
        char* base = static_cast<char*>(c.g->ws.base);
        cudaMemsetAsync(base + c.b.state_bytes_begin, 0, c.b.state_bytes_end - c.b.state_bytes_begin, c.st);
    }
    launch_init(c.st, a);
    c.launches += 1;
}

// Pack the columns of the still-active pairs into a block of ld_new columns (ld_new holds
// at least `active_upper` slots, an upper bound on the active count read one step ago).
// With fuse_step >= 0 the packing is fused with that step's normalise pass (its SpMM and
// finalize have run: q[0] holds W and q[1] holds q_j): k_normalize_pack writes q_{j+1} and
// q_j packed, and *fused reports whether it ran. When it did not (no narrower layout, or one
// without whole 16-byte units, such as the single-column layout of the last active pair),
// the caller runs the plain pass and then the packing without fusion.
template <typename T>
static rd_status enqueue_compaction(RunCtx& c, int active_upper, int fuse_step = -1, bool* fused = nullptr)
{
    if (fused) *fused = false;
    Plan np;
    rd_query_opts o2 = c.o;
    o2.rhs_tile = 0;
    RD_TRY(make_plan(c.g, active_upper, o2, false, &np));
    if (np.ld >= c.cur.ld) return RD_OK;
    // the spare region holds n x ld0 elements: two packed blocks must fit in it
    if (!c.in_region_x && 2 * np.ld > c.pl.ld) return RD_OK;
    if (fuse_step >= 0 && np.ld % (16 / (int64_t)np.elem) != 0) return RD_OK;
    const int64_t n = c.g->n;
    void* dst0;
    void* dst1;
    if (c.in_region_x) {
        dst0 = c.b.region_a;
    } else {
        dst0 = c.b.region_x;
    }
    dst1 = static_cast<char*>(dst0) + block_bytes(n, np.ld, np.elem);
    CompactArgs a{};
    a.n = n;
    a.ld_old = c.cur.ld;
    a.ld_new = np.ld;
    a.slot_pair_old = c.slot_sel >= 0 ? c.b.slot_pair[c.slot_sel] : nullptr;
    a.npairs = (int)c.P;
    const int new_sel = c.slot_sel == 0 ? 1 : 0;
    a.slot_pair_new = c.b.slot_pair[new_sel];
    a.old_slot = c.b.old_slot;
    a.active = c.b.st.active;
    a.cf_old = c.b.cf_cur[c.cf_sel];
    a.cf_new = c.b.cf_cur[1 - c.cf_sel];
    a.q_src0 = c.b.q[0];
    a.q_src1 = c.b.q[1];
    a.q_dst0 = dst0;
    a.q_dst1 = dst1;
    a.elem_size = (int)np.elem;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c.g->sm_count * 8,
                                                                 (n * np.ld + 255) / 256));
    if (fuse_step >= 0) {
        launch_compact_map(c.st, a);
        NormPackArgs<T> na{};
        na.n = n;
        na.ld_old = c.cur.ld;
        na.ld_new = np.ld;
        na.w = static_cast<const T*>(c.b.q[0]);
        na.qcur = static_cast<const T*>(c.b.q[1]);
        na.cf = coef_block<T>(c, fuse_step);
        na.old_slot = c.b.old_slot;
        na.qnext_new = static_cast<T*>(dst1);  // q_{j+1}: the current block of the next step
        na.qcur_new = static_cast<T*>(dst0);   // q_j: its previous block
        if (!launch_normalize_pack_t(grid, c.st, na)) {
            set_error("normalise-and-pack launch rejected");
            return RD_ERR_UNSUPPORTED;
        }
        *fused = true;
    } else {
        launch_compact(c.st, grid, a);
    }
    c.launches += 2;
    c.b.q[0] = dst0;
    c.b.q[1] = dst1;
    c.in_region_x = !c.in_region_x;
    c.slot_sel = new_sel;
    c.cf_sel = 1 - c.cf_sel;
    c.cur = np;
    ++c.compactions;
    return RD_OK;
}

// ------------------------------------------------------------- CUDA graphs
// One Lanczos step -- heavy-row pre-pass and SpMM, finalize, normalize, step advance -- is
// captured once per argument set and replayed. Its kernels read the step index from
// device memory (StepArgs::step_dev) and advance it themselves, so one graph per vector
// block orientation serves every step of a query (the host swaps the two blocks' roles
// after each step, as in the launch-per-kernel loop) and later queries with the same
// layout. Polls, compaction and the stop test are the same as in that loop.
constexpr size_t kGraphCache = 16;

template <typename T>
static void graph_step_args(RunCtx& c, const FinArgs& base, StepArgs<T>* sa, FinArgs* fa, NormArgs<T>* na)
{
    const int64_t ld = c.cur.ld;
    const int64_t stride = c.compact ? 0 : 4 * ld;
    T* cf0 = const_cast<T*>(coef_block<T>(c, 0));
    memset(sa, 0, sizeof(*sa));
    *sa = step_args<T>(c, 0, true);
    sa->cf_beta = cf0;
    sa->active_prev = nullptr;
    sa->step_dev = c.b.step_dev;
    sa->cf_stride = stride;
    sa->act_count = c.b.st.act_count;
    memset(fa, 0, sizeof(*fa));
    *fa = base;
    fa->step = 0;
    fa->ld = ld;
    fa->tp = c.cur.cfg.tp();
    fa->nblocks = c.cur.grid_main;
    fa->slot_pair = c.compact && c.slot_sel >= 0 ? c.b.slot_pair[c.slot_sel] : nullptr;
    fa->cf_step = cf0;
    fa->cf_next = c.compact ? cf0 : cf0 + 4 * ld;
    fa->step_dev = c.b.step_dev;
    fa->cf_stride = stride;
    memset(na, 0, sizeof(*na));
    na->n = c.g->n;
    na->ld = ld;
    na->w_to_qnext = static_cast<T*>(c.b.q[0]);
    na->qcur = static_cast<const T*>(c.b.q[1]);
    na->cf = cf0;
    na->step_dev = c.b.step_dev;
    na->cf_stride = stride;
    na->act_count = c.b.st.act_count;
    if (c.pot_x) {
        na->pvec = static_cast<T*>(c.b.pvec);
        na->xvec = static_cast<T*>(c.b.phi);
        na->xcf = static_cast<const T*>(c.b.xcf);
        na->xcf_stride = 2 * ld;
    }
}

// Launch one step from the graph cache (capturing and instantiating it on a miss).
template <typename T>
static rd_status launch_step_graph(RunCtx& c, const FinArgs& base)
{
    rd_graph* g = c.g;
    StepArgs<T> sa;
    FinArgs fa;
    NormArgs<T> na;
    graph_step_args<T>(c, base, &sa, &fa, &na);
    const bool heavy = g->n_chunks > 0;
    int misc[8] = {c.cur.cfg.vec, c.cur.cfg.gs, c.cur.cfg.nzl, c.cur.cfg.kind, c.cur.grid_main, c.cur.grid_heavy,
                   c.cur.grid_norm, c.pl.k_max};
    std::string key(reinterpret_cast<const char*>(misc), sizeof(misc));
    key.append(reinterpret_cast<const char*>(&sa), sizeof(sa));
    key.append(reinterpret_cast<const char*>(&fa), sizeof(fa));
    key.append(reinterpret_cast<const char*>(&na), sizeof(na));
    key.push_back(std::is_same<T, df64>::value ? 'w' : (sizeof(T) == 8 ? 'd' : 'f'));
    cudaGraphExec_t exec = nullptr;
    for (const auto& kv : g->graphs)
        if (kv.first == key) {
            exec = kv.second;
            break;
        }
    if (!exec) {
        if (!g->capture_stream) RD_CUDA(cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking));
        cudaStream_t cs = g->capture_stream;
        RD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        bool ok = true;
        if (heavy) ok = launch_spmm_t(c.cur.cfg, g->weighted, true, c.cur.grid_heavy, cs, sa);
        if (ok) ok = launch_spmm_t(c.cur.cfg, g->weighted, false, c.cur.grid_main, cs, sa);
        if (ok) {
            launch_finalize(cs, fa);
            launch_normalize_t(c.cur.grid_norm, cs, na);
            launch_step_advance(cs, c.b.step_dev, c.pl.k_max);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        if (!ok) {
            if (graph) cudaGraphDestroy(graph);
            set_error("no SpMM kernel for this configuration");
            return RD_ERR_UNSUPPORTED;
        }
        RD_CUDA(ec);
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        RD_CUDA(ei);
        if (g->graphs.size() >= kGraphCache) {
            cudaGraphExecDestroy(g->graphs.front().second);
            g->graphs.erase(g->graphs.begin());
        }
        g->graphs.emplace_back(std::move(key), exec);
    }
    RD_CUDA(cudaGraphLaunch(exec, c.st));
    c.launches += (heavy ? 2 : 1) + 3;
    ++c.spmm_launches;
    c.spmm_bytes += spmm_launch_bytes(g, c.cur);
    return RD_OK;
}

// The device-resident step loop: one CUDA graph whose conditional while node repeats a body of
// one Lanczos step for each orientation of the two vector blocks, each step with a condition
// before it and one after its finalize, so that the steps of a query run without the host
// until every pair has stopped, k_max is reached or a column compaction is due (then after the
// finalize of the step before it, so that the host runs that step's normalise pass fused with
// the packing). Where it stopped is read back by the caller (loop_saved).
template <typename T>
static rd_status launch_step_loop(RunCtx& c, const FinArgs& base, int compact_check, int lag)
{
    rd_graph* g = c.g;
    StepArgs<T> sa[2];
    FinArgs fa[2];
    NormArgs<T> na[2];
    graph_step_args<T>(c, base, &sa[0], &fa[0], &na[0]);
    std::swap(c.b.q[0], c.b.q[1]);
    graph_step_args<T>(c, base, &sa[1], &fa[1], &na[1]);
    std::swap(c.b.q[0], c.b.q[1]);
    const bool heavy = g->n_chunks > 0;
    int misc[10] = {c.cur.cfg.vec, c.cur.cfg.gs, c.cur.cfg.nzl, c.cur.cfg.kind, c.cur.grid_main, c.cur.grid_heavy,
                    c.cur.grid_norm, c.pl.k_max, compact_check, lag};
    std::string key("loop");
    key.append(reinterpret_cast<const char*>(misc), sizeof(misc));
    for (int o = 0; o < 2; ++o) {
        key.append(reinterpret_cast<const char*>(&sa[o]), sizeof(sa[o]));
        key.append(reinterpret_cast<const char*>(&fa[o]), sizeof(fa[o]));
        key.append(reinterpret_cast<const char*>(&na[o]), sizeof(na[o]));
    }
    key.push_back(std::is_same<T, df64>::value ? 'w' : (sizeof(T) == 8 ? 'd' : 'f'));
    cudaGraphExec_t exec = nullptr;
    for (const auto& kv : g->graphs)
        if (kv.first == key) {
            exec = kv.second;
            break;
        }
    if (!exec) {
        if (!g->capture_stream) RD_CUDA(cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking));
        cudaStream_t cs = g->capture_stream;
        cudaGraph_t graph = nullptr;
        RD_CUDA(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault);
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_status(e, "building the device-resident step loop");
        }
        bool ok = true;
        for (int o = 0; o < 2 && ok; ++o) {
            launch_loop_cond(cs, h, c.b.step_dev, c.b.st.act_count, c.b.loop_saved, c.b.loop_cfrom, c.pl.k_max,
                             c.cur.ld, compact_check, lag, 0);
            if (heavy) ok = launch_spmm_t(c.cur.cfg, g->weighted, true, c.cur.grid_heavy, cs, sa[o]);
            if (ok) ok = launch_spmm_t(c.cur.cfg, g->weighted, false, c.cur.grid_main, cs, sa[o]);
            if (ok) {
                launch_finalize(cs, fa[o]);
                launch_loop_cond(cs, h, c.b.step_dev, c.b.st.act_count, c.b.loop_saved, c.b.loop_cfrom,
                                 c.pl.k_max, c.cur.ld, compact_check, lag, 1);
                launch_normalize_t(c.cur.grid_norm, cs, na[o]);
                launch_step_advance(cs, c.b.step_dev, c.pl.k_max);
            }
        }
        cudaGraph_t body = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &body);
        if (!ok || ec != cudaSuccess) {
            cudaGraphDestroy(graph);
            if (!ok) {
                set_error("no SpMM kernel for this configuration");
                return RD_ERR_UNSUPPORTED;
            }
            return cuda_status(ec, "cudaStreamEndCapture (step loop)");
        }
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        RD_CUDA(ei);
        if (g->graphs.size() >= kGraphCache) {
            cudaGraphExecDestroy(g->graphs.front().second);
            g->graphs.erase(g->graphs.begin());
        }
        g->graphs.emplace_back(std::move(key), exec);
    }
    RD_CUDA(cudaGraphLaunch(exec, c.st));
    return RD_OK;
}

// Algorithmic bytes of one SpMM launch above which rd_query polls without lag (about a
// quarter of a millisecond of HBM traffic on this part, against a host reaction of tens of
// microseconds).
constexpr double kNoLagBytes = 1.5e9;

template <typename T>
static rd_status run_forward(RunCtx& c)
{
    c.cur = c.pl;
    enqueue_init(c, false);
    const int chunk = c.o.chunk_steps > 0 ? c.o.chunk_steps : 8;
    FinArgs fa{};
    fa.npairs = (int)c.P;
    fa.pstride = c.pl.ld;
    fa.k_max = c.pl.k_max;
    fa.deflate = (c.o.flags & RD_Q_NO_DEFLATE) ? 0 : 1;
    fa.fixed_k = (c.o.flags & RD_Q_FIXED_K) ? 1 : 0;
    fa.fp64 = sizeof(T) == 8;
    fa.df = std::is_same<T, df64>::value ? 1 : 0;
    fa.rel_tol = c.o.rel_tol;
    fa.resid_tol = c.o.resid_tol;
    fa.est_delayed = (c.o.flags & RD_Q_EST_DELAYED) ? 1 : 0;
    fa.sumdeg = c.g->sumdeg;
    fa.inv_sumdeg = c.g->sumdeg > 0.0 ? 1.0 / c.g->sumdeg : 0.0;
    fa.block_part = c.b.block_part;
    fa.st = c.b.st;
    fa.elem_size = (int)c.pl.elem;
    fa.xcf = c.pot_x ? c.b.xcf : nullptr;
    int* h = c.g->h_pinned;
    // first poll: ids valid and at least one active pair
    RD_CUDA(cudaMemcpyAsync(h, c.b.err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    RD_CUDA(cudaMemcpyAsync(h + 1, c.b.st.act_count, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    RD_CUDA(cudaStreamSynchronize(c.st));
    if (h[0]) {
        set_error("a pair id is outside [0, n)");
        return RD_ERR_INVALID_ARG;
    }
    if (h[1] == 0) return RD_OK;
    if (c.onchip) {
        OnchipArgs oa{};
        oa.n = c.g->n;
        oa.npairs = (int)c.P;
        oa.row_ptr = c.g->row_ptr;
        oa.col = c.g->col;
        oa.w = c.g->w;
        oa.deg64 = c.g->deg64;
        oa.invdeg64 = c.g->invdeg64;
        oa.deg32 = c.g->deg32;
        oa.invdeg32 = c.g->invdeg32;
        oa.s = c.b.s;
        oa.t = c.b.t;
        oa.heavy_thr = c.g->heavy_thr;
        oa.n_heavy_rows = c.g->n_heavy_rows;
        oa.heavy_rows = c.g->heavy_rows;
        oa.fin = fa;
        oa.elem_size = (int)c.pl.elem;
        oa.weighted = c.g->weighted ? 1 : 0;
        oa.sm_count = c.g->sm_count;
        oa.allow_cluster = (c.o.flags & RD_Q_NO_CLUSTER) ? 0 : 1;
        const int ctas = launch_onchip(c.st, oa);
        if (ctas > 0) {
            c.onchip_ctas = ctas;
            ++c.launches;
            RD_CUDA(cudaGetLastError());
            return RD_OK;
        }
    }
    c.graph = !c.profile && (c.o.flags & RD_Q_NO_GRAPH) == 0;
    constexpr int kSlots = 4;   // pinned poll slots h[4 .. 7]
    cudaEvent_t poll_ev[kSlots] = {};
    if (c.lagged_polls)
        for (int i = 0; i < kSlots; ++i) poll_ev[i] = c.ev->get();
    int last_known = h[1];
    const bool sparse0 = sparse_first_step(c);
    c.sparse_first = sparse0;
    // rd_query: after the first step, a device-resident loop over the steps (the host steps in
    // only for column compactions)
    const bool dloop = c.graph && c.lagged_polls && (c.o.flags & RD_Q_NO_DEVICE_LOOP) == 0;
    c.device_loop = dloop;
    for (int j = 0; j < c.pl.k_max; ++j) {
        if (dloop && j > 0) {
            const int compact_check = c.compact ? 1 : 0;
            const int per_step = (c.g->n_chunks > 0 ? 2 : 1) + 5;
            while (true) {
                const int j0 = c.steps;
                const double bytes_per_step = spmm_launch_bytes(c.g, c.cur);
                const int lag = bytes_per_step > kNoLagBytes ? 0 : 1;  // as the host polls below
                RD_TRY(launch_step_loop<T>(c, fa, compact_check, lag));
                // the step index back from the sentinel, for the next launch
                RD_CUDA(cudaMemcpyAsync(c.b.step_dev, c.b.loop_saved, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                        c.st));
                RD_CUDA(cudaMemcpyAsync(h + 8, c.b.loop_saved, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
                RD_CUDA(cudaStreamSynchronize(c.st));
                const int jn = h[8];
                const int ran = jn - j0;  // steps run whole inside the loop
                // body passes: the stop shows in pass ran/2 + 1, and every kernel of a pass launches
                c.launches += (int64_t)(ran / 2 + 1) * 2 * per_step;
                c.spmm_launches += ran;
                c.spmm_bytes += bytes_per_step * ran;
                if (ran & 1) std::swap(c.b.q[0], c.b.q[1]);
                const int act_lag = h[9], act = h[10];  // the count the compaction test read; entering the next step
                if (h[11]) {
                    // stopped after step jn's finalize: its normalise pass, fused with the packing
                    ++c.spmm_launches;
                    c.spmm_bytes += bytes_per_step;
                    bool fused = false;
                    RD_TRY(enqueue_compaction<T>(c, act_lag, jn, &fused));
                    if (!fused) {  // the plain pass, then the packing if there is one to make
                        enqueue_normalize<T>(c, jn, false);
                        std::swap(c.b.q[0], c.b.q[1]);
                        RD_TRY(enqueue_compaction<T>(c, act_lag));
                    }
                    launch_step_advance(c.st, c.b.step_dev, c.pl.k_max);
                    ++c.launches;
                    c.steps = jn + 1;
                } else {
                    c.steps = jn;
                    if (act == 0 || jn >= c.pl.k_max) break;
                    RD_TRY(enqueue_compaction<T>(c, act_lag));
                }
                // the next test after one more step, as the host polls make it
                h[12] = c.steps + 1;
                RD_CUDA(cudaMemcpyAsync(c.b.loop_cfrom, h + 12, sizeof(int32_t), cudaMemcpyHostToDevice, c.st));
            }
            break;
        }
        const bool sparse = j == 0 && sparse0;
        if (c.graph && !sparse) {
            RD_TRY(launch_step_graph<T>(c, fa));
        } else {
            if (sparse) enqueue_step0<T>(c, true);
            else RD_TRY(enqueue_spmm<T>(c, j, true));
            fa.step = j;
            fa.ld = c.cur.ld;
            fa.tp = c.cur.cfg.tp();
            fa.nblocks = sparse ? 1 : c.cur.grid_main;
            const bool sparse_norm = sparse && sparse_norm_ok(c);
            if (c.compact) {
                fa.slot_pair = c.slot_sel >= 0 ? c.b.slot_pair[c.slot_sel] : nullptr;
                fa.cf_step = c.b.cf_cur[c.cf_sel];
                fa.cf_next = c.b.cf_cur[c.cf_sel];
            } else {
                fa.slot_pair = nullptr;
                fa.cf_step = static_cast<T*>(c.b.cf_hist) + (int64_t)j * 4 * c.cur.ld;
                fa.cf_next = static_cast<T*>(c.b.cf_hist) + (int64_t)(j + 1) * 4 * c.cur.ld;
            }
            launch_finalize(c.st, fa);
            ++c.launches;
            if (sparse_norm) enqueue_normalize_step0<T>(c);
            else enqueue_normalize<T>(c, j, false);
            if (c.graph) {  // graph-replayed steps read the step index from device memory
                launch_step_advance(c.st, c.b.step_dev, c.pl.k_max);
                ++c.launches;
            }
        }
        std::swap(c.b.q[0], c.b.q[1]);
        c.steps = j + 1;
        if (j + 1 >= c.pl.k_max) break;
        if (dloop) continue;  // the device-resident loop reads the active counts itself
        if (c.lagged_polls) {
            // count of active pairs after step j lands in h[4 + j % kSlots]; read the count
            // of the previous step, whose copy has usually completed while step j runs --
            // or, when a step is long enough (a step's SpMM moves more than kNoLagBytes),
            // wait for step j's own count: the GPU idles for the host's reaction time, but
            // converged pairs are packed out one step earlier
            const int lag = spmm_launch_bytes(c.g, c.cur) > kNoLagBytes ? 0 : 1;
            const int sl = j % kSlots;
            RD_CUDA(cudaMemcpyAsync(h + 4 + sl, c.b.st.act_count + j + 1, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    c.st));
            RD_CUDA(cudaEventRecord(poll_ev[sl], c.st));
            if (j >= lag) {
                const int ps = (j - lag) % kSlots;
                RD_CUDA(cudaEventSynchronize(poll_ev[ps]));
                last_known = h[4 + ps];
                if (last_known == 0) break;  // steps enqueued since return at once
                if (c.compact && last_known * 2 <= c.cur.ld && c.cur.ld > 16)
                    RD_TRY(enqueue_compaction<T>(c, last_known));
            }
        } else if ((j + 1) % chunk == 0) {
            RD_CUDA(cudaMemcpyAsync(h, c.b.st.act_count + j + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
            RD_CUDA(cudaStreamSynchronize(c.st));
            if (h[0] == 0) break;
        }
    }
    RD_CUDA(cudaGetLastError());
    return RD_OK;
}

static rd_status stage_pairs(RunCtx& c, const int32_t* s, const int32_t* t)
{
    RD_CUDA(cudaMemcpyAsync(c.b.s, s, sizeof(int32_t) * c.P, cudaMemcpyDefault, c.st));
    RD_CUDA(cudaMemcpyAsync(c.b.t, t, sizeof(int32_t) * c.P, cudaMemcpyDefault, c.st));
    return RD_OK;
}

static rd_status finish_outputs(RunCtx& c, double* r_out, int32_t* iters_out, double* err_out, int32_t* status_out,
                                rd_status* call_status)
{
    OutArgs oa{};
    oa.npairs = (int)c.P;
    oa.ld = c.pl.ld;
    oa.st = c.b.st;
    oa.r_out = c.b.r;
    oa.iters_out = c.b.iters;
    oa.err_out = c.b.err;
    oa.status_out = c.b.status;
    oa.summary = c.b.summary;
    launch_output(c.st, oa);
    ++c.launches;
    if (r_out) RD_CUDA(cudaMemcpyAsync(r_out, c.b.r, sizeof(double) * c.P, cudaMemcpyDefault, c.st));
    if (iters_out) RD_CUDA(cudaMemcpyAsync(iters_out, c.b.iters, sizeof(int32_t) * c.P, cudaMemcpyDefault, c.st));
    if (err_out) RD_CUDA(cudaMemcpyAsync(err_out, c.b.err, sizeof(double) * c.P, cudaMemcpyDefault, c.st));
    if (status_out) RD_CUDA(cudaMemcpyAsync(status_out, c.b.status, sizeof(int32_t) * c.P, cudaMemcpyDefault, c.st));
    int* h = c.g->h_pinned;
    RD_CUDA(cudaMemcpyAsync(h, c.b.summary, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    RD_CUDA(cudaStreamSynchronize(c.st));
    RD_CUDA(cudaGetLastError());
    *call_status = h[0] ? RD_WARN_NOT_CONVERGED : RD_OK;
    return RD_OK;
}

static void record_stats(RunCtx& c)
{
    rd_call_stats& s = c.g->stats;
    s.launches += c.launches;
    s.spmm_launches += c.spmm_launches;
    s.steps = std::max(s.steps, c.steps);
    s.rhs_tile = c.pl.cfg.tp();
    s.rows_per_warp = c.pl.cfg.rpw();
    s.nnz_lanes = c.pl.cfg.nzl;
    s.kernel = kernel_code(c.pl.cfg);
    s.ld = c.pl.ld;
    s.spmm_bytes += c.spmm_bytes;
    s.compactions += c.compactions;
    s.tuned = c.pl.tuned ? 1 : 0;
    s.row_order = c.pl.cfg.order;
    s.sparse_first = c.sparse_first ? 1 : 0;
    s.onchip_ctas = c.onchip_ctas;
    s.device_loop = c.device_loop ? 1 : 0;
    if (c.profile) {
        double ms = 0.0;
        for (auto& pr : c.spmm_ev) {
            float x = 0.f;
            if (cudaEventElapsedTime(&x, pr.first, pr.second) == cudaSuccess) ms += x;
        }
        cudaGetLastError();
        s.spmm_ms += ms;
    }
}

static rd_status validate_common(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs,
                                 const rd_query_opts* opts, rd_query_opts* o)
{
    if (!g) {
        set_error("graph is NULL");
        return RD_ERR_INVALID_ARG;
    }
    if (npairs < 0 || npairs > (1ll << 24)) {
        set_error("npairs must be in [0, 2^24]");
        return RD_ERR_INVALID_ARG;
    }
    if (npairs > 0 && (!s || !t)) {
        set_error("s and t must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    if (opts) *o = *opts;
    else rd_query_opts_init(o);
    if (o->k_max < 1 || o->k_max > (1 << 22)) {
        set_error("k_max must be in [1, 2^22]");
        return RD_ERR_INVALID_ARG;
    }
    if (o->kernel < 0 || o->kernel > 5) {
        set_error("kernel must be 0, 1, 2, 3, 4 or 5");
        return RD_ERR_INVALID_ARG;
    }
    if (o->mode != RD_MODE_FP64 && o->mode != RD_MODE_FP32V_FP64S && o->mode != RD_MODE_DF64) {
        set_error("unknown mode");
        return RD_ERR_INVALID_ARG;
    }
    if (!(o->rel_tol >= 0.0) || !(o->resid_tol >= 0.0)) {
        set_error("tolerances must be >= 0");
        return RD_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device) {
        cudaGetLastError();
        set_error("the current CUDA device is not the graph's device");
        return RD_ERR_INVALID_ARG;
    }
    return RD_OK;
}

// ------------------------------------------------------------- autotuner
// Candidates for one width class: for each tile from a quarter of the width up to the
// width, the row-stream kernel and the row-group kernel with 1, 2 or 4 nonzero lanes per
// row group; for one column, the warp-per-task SpMV, the row-stream kernel with one lane
// per task and the row-group kernel with 4 to 32 nonzero lanes per row.
static std::vector<SpmmCfg> tune_candidates(const rd_graph* g, int64_t width, bool fp64, bool single)
{
    std::vector<SpmmCfg> v;
    auto add = [&](int vec, int gs, int nzl, int kind, int order) {
        SpmmCfg c;
        c.vec = vec;
        c.gs = gs;
        c.nzl = nzl;
        c.kind = kind;
        c.order = order;
        if (order && !g->row_order) return;
        if (cfg_known(c, fp64)) v.push_back(c);
    };
    if (single) {
        if (g->ntasks > 0) add(1, 1, 1, 2, 0);
        add(1, 1, 1, 1, 0);
        for (int z : {4, 8, 16, 32})
            for (int o : {0, 1}) add(1, 1, z, 0, o);
        return v;
    }
    const int64_t tmin = fp64 ? 8 : 16;
    for (int64_t tp = std::max(tmin, width / 4); tp <= width; tp <<= 1) {
        const int vec = fp64 ? (tp >= 128 ? 4 : 2) : (tp >= 256 ? 8 : 4);
        const int gs = (int)(tp / vec);
        add(vec, gs, 1, 1, 0);
        for (int z : {1, 2, 4})
            if (gs * z <= 32)
                for (int o : {0, 1}) add(vec, gs, z, 0, o);
    }
    // async row-stream: column slabs of 16 to 128 FP32 columns (16 to 64 of 8-byte elements),
    // down to an eighth of the width
    const int avec = fp64 ? 2 : 4;
    for (int64_t tp = std::max<int64_t>(16, width / 8); tp <= std::min<int64_t>(width, 32 * avec); tp <<= 1)
        add(avec, (int)(tp / avec), 1, 3, 0);
    return v;
}

// Mean time of one SpMM step launch pair (heavy-row pre-pass + main kernel) of cfg on g's
// CSR with `width` columns: zeroed vectors, one warm-up and three timed launches.
template <typename T>
static rd_status time_cfg(rd_graph* g, int64_t width, const rd_query_opts& o, const SpmmCfg& cfg, cudaStream_t st,
                          EventPool& ev, float* us_out)
{
    RunCtx c;
    c.g = g;
    c.o = o;
    c.st = st;
    c.P = width;
    c.ev = &ev;
    RD_TRY(make_plan_cfg(g, width, o, cfg, &c.pl));
    c.cur = c.pl;
    Carver dry(nullptr);
    const size_t bytes = carve(dry, g, c.pl, width, false, &c.b, false);
    RD_TRY(ensure_ws(g, bytes));
    Carver real(g->ws.base);
    carve(real, g, c.pl, width, false, &c.b, false);
    RD_CUDA(cudaMemsetAsync(c.b.region_a, 0, 2 * block_bytes(g->n, c.pl.ld, c.pl.elem), st));
    RD_CUDA(cudaMemsetAsync(static_cast<char*>(g->ws.base) + c.b.state_bytes_begin, 0,
                            c.b.state_bytes_end - c.b.state_bytes_begin, st));
    RD_CUDA(cudaMemsetAsync(c.b.st.act_count, 0x01, sizeof(int32_t), st));  // step 0 "active"
    RD_TRY(enqueue_spmm<T>(c, 0, true));
    cudaEvent_t e0 = ev.get(), e1 = ev.get();
    RD_CUDA(cudaEventRecord(e0, st));
    constexpr int kReps = 3;
    for (int r = 0; r < kReps; ++r) RD_TRY(enqueue_spmm<T>(c, 0, true));
    RD_CUDA(cudaEventRecord(e1, st));
    RD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    *us_out = 1e3f * ms / kReps;
    return RD_OK;
}

// Tune the width classes a query of P pairs can use (all of them down to the narrowest
// tile when the query compacts), skipping classes already in g's table.
static rd_status ensure_tuned(rd_graph* g, int64_t P, const rd_query_opts& o, bool plain, bool compact,
                              cudaStream_t st)
{
    if (!tuning_allowed(o) || P < 1 || g->n == 0) return RD_OK;
    const int prec = mode_prec(o.mode);
    const bool fp64 = prec != 0;
    const bool single = plain || P == 1;
    std::vector<int64_t> widths{tune_width(P, fp64, single)};
    const int64_t tmin = fp64 ? 8 : 16;
    if (compact && !single)
        for (int64_t w = widths[0] / 2; w >= tmin; w /= 2) widths.push_back(w);
    EventPool ev;
    for (int64_t w : widths) {
        if (find_tuned(g, prec, single, w)) continue;
        rd_graph::TunedCfg best;
        best.us = -1.f;
        for (const SpmmCfg& cfg : tune_candidates(g, w, fp64, single)) {
            float us = 0.f;
            rd_status r = prec == 2 ? time_cfg<df64>(g, w, o, cfg, st, ev, &us)
                          : (prec == 1 ? time_cfg<double>(g, w, o, cfg, st, ev, &us)
                                       : time_cfg<float>(g, w, o, cfg, st, ev, &us));
            if (r == RD_ERR_OOM) continue;  // a wider padding that does not fit is not a candidate
            if (r < 0) return r;
            if (best.us < 0.f || us < best.us) {
                best.cfg = cfg;
                best.us = us;
            }
        }
        if (best.us < 0.f) continue;  // nothing fitted: the fixed rule decides
        best.prec = prec;
        best.single = single ? 1 : 0;
        best.width = w;
        g->tuned.push_back(best);
    }
    return RD_OK;
}

static rd_status prepare_run(RunCtx& c, rd_graph* g, int64_t P, const rd_query_opts& o, bool plain, bool grad,
                             cudaStream_t st, bool compact = false, bool lagged_polls = false)
{
    c.g = g;
    c.o = o;
    c.st = st;
    c.P = P;
    c.profile = (o.flags & RD_Q_PROFILE) != 0;
    c.compact = compact;
    c.lagged_polls = lagged_polls && c.ev != nullptr;
    if (mode_prec(o.mode) == 2 && !g->degdf && g->n > 0) {  // double-float degrees, once per graph
        RD_CUDA(cudaMalloc((void**)&g->degdf, sizeof(df64) * g->n));
        RD_CUDA(cudaMalloc((void**)&g->invdegdf, sizeof(df64) * g->n));
        const int grid = std::max(1, std::min(g->sm_count * 8, (int)((g->n + 255) / 256)));
        launch_split_df(st, grid, g->n, g->deg64, g->degdf);
        launch_split_df(st, grid, g->n, g->invdeg64, g->invdegdf);
    }
    RD_TRY(ensure_tuned(g, P, o, plain, compact, st));
    RD_TRY(make_plan(g, P, o, plain, &c.pl));
    c.cur = c.pl;
    Carver dry(nullptr);
    const size_t bytes = carve(dry, g, c.pl, P, grad, &c.b, compact);
    RD_TRY(ensure_ws(g, bytes));
    Carver real(g->ws.base);
    carve(real, g, c.pl, P, grad, &c.b, compact);
    return RD_OK;
}

// Host-side query of a batch of pairs (all device work on st).
static rd_status query_batch(rd_graph* g, const int32_t* s, const int32_t* t, int64_t P, const rd_query_opts& o,
                             bool plain, double* r_out, int32_t* iters_out, double* err_out, int32_t* status_out,
                             cudaStream_t st, rd_status* call_status, EventPool* ev, bool compact = false,
                             bool lagged_polls = false)
{
    RunCtx c;
    c.ev = ev;
    RD_TRY(prepare_run(c, g, P, o, plain, false, st, compact && !plain, lagged_polls));
    c.onchip = (o.flags & RD_Q_NO_ONCHIP) == 0 && onchip_smem_bytes(g->n, (int)c.pl.elem) <= 220 * 1024;
    RD_TRY(stage_pairs(c, s, t));
    rd_status rs = c.pl.prec == 2 ? run_forward<df64>(c)
                   : (c.pl.prec == 1 ? run_forward<double>(c) : run_forward<float>(c));
    if (rs < 0) return rs;
    RD_TRY(finish_outputs(c, r_out, iters_out, err_out, status_out, call_status));
    record_stats(c);
    return RD_OK;
}

template <typename T>
static rd_status run_replay(RunCtx& c, int K)
{
    // Replay of the forward recurrence with the stored coefficients; phi += coef_j q_j.
    c.cur = c.pl;
    const int64_t vbytes = c.g->n * c.pl.ld * (int64_t)c.pl.elem;
    RD_CUDA(cudaMemsetAsync(c.b.phi, 0, vbytes, c.st));
    enqueue_init(c, true);
    const bool sparse0 = sparse_first_step(c);
    for (int j = 0; j < K; ++j) {
        if (j == 0 && sparse0) enqueue_step0<T>(c, false);
        else RD_TRY(enqueue_spmm<T>(c, j, false));
        enqueue_normalize<T>(c, j, true);
        std::swap(c.b.q[0], c.b.q[1]);
    }
    RD_CUDA(cudaGetLastError());
    return RD_OK;
}

static rd_status forward_and_potential(RunCtx& c, const int32_t* s, const int32_t* t, const double* grad_r,
                                       rd_status* call_status)
{
    RD_TRY(stage_pairs(c, s, t));
    // the potential: accumulated during the forward steps (direct update), or, with
    // RD_Q_REPLAY_POTENTIAL, by a second pass that regenerates the vectors
    c.pot_x = (c.o.flags & RD_Q_REPLAY_POTENTIAL) == 0;
    if (c.pot_x) {
        const int64_t vbytes = c.g->n * c.pl.ld * (int64_t)c.pl.elem;
        RD_CUDA(cudaMemsetAsync(c.b.phi, 0, vbytes, c.st));
        RD_CUDA(cudaMemsetAsync(c.b.pvec, 0, vbytes, c.st));
    }
    rd_status rs = c.pl.fp64 ? run_forward<double>(c) : run_forward<float>(c);
    if (rs < 0) return rs;
    // z-solve and gbar; a host grad_r is staged in the output buffer (free until the end)
    const double* d_grad = nullptr;
    if (grad_r) {
        if (is_device_ptr(grad_r)) {
            d_grad = grad_r;
        } else {
            RD_CUDA(cudaMemcpyAsync(c.b.r, grad_r, sizeof(double) * c.P, cudaMemcpyHostToDevice, c.st));
            d_grad = c.b.r;
        }
    }
    ZsolveArgs za{};
    za.npairs = (int)c.P;
    za.ld = c.pl.ld;
    za.k_max = c.pl.k_max;
    za.st = c.b.st;
    za.coef_hist = c.b.coef_hist;
    za.gbar = c.b.gbar;
    za.zscratch = c.b.zscratch;
    za.elem_size = (int)c.pl.elem;
    za.grad_r = d_grad;
    launch_zsolve(c.st, za);
    ++c.launches;
    if (!c.pot_x) {
        // K = max steps over pairs
        std::vector<int32_t> ks(c.P);
        RD_CUDA(cudaMemcpyAsync(ks.data(), c.b.st.k, sizeof(int32_t) * c.P, cudaMemcpyDeviceToHost, c.st));
        RD_CUDA(cudaStreamSynchronize(c.st));
        int K = 0;
        for (int32_t k : ks) K = std::max(K, (int)k);
        rs = c.pl.fp64 ? run_replay<double>(c, K) : run_replay<float>(c, K);
        if (rs < 0) return rs;
    }
    *call_status = RD_OK;
    return RD_OK;
}

}  // namespace rd

using namespace rd;

// =================================================================== C ABI
extern "C" {

void rd_query_opts_init(rd_query_opts* o)
{
    if (!o) return;
    o->k_max = 1000;
    o->rel_tol = 1e-7;
    o->resid_tol = 0.0;
    o->mode = RD_MODE_FP32V_FP64S;
    o->rhs_tile = 0;
    o->rows_per_warp = 0;
    o->chunk_steps = 8;
    o->flags = 0;
    o->kernel = 0;
}

const char* rd_status_string(rd_status s)
{
    switch (s) {
        case RD_OK: return "ok";
        case RD_WARN_NOT_CONVERGED: return "not converged within k_max";
        case RD_ERR_INVALID_ARG: return "invalid argument";
        case RD_ERR_ZERO_DEGREE: return "vertex of degree zero";
        case RD_ERR_DISCONNECTED: return "s and t are disconnected";
        case RD_ERR_CUDA: return "CUDA error";
        case RD_ERR_OOM: return "out of device memory";
        case RD_ERR_TIMEOUT: return "timeout";
        case RD_ERR_NUMERIC: return "numerical breakdown";
        case RD_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* rd_last_error(void) { return g_last_error.c_str(); }

rd_status rd_graph_create(rd_graph** out, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                          const float* weights, uint32_t flags, void* stream)
{
    g_last_error.clear();
    if (!out) {
        set_error("out is NULL");
        return RD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (n < 1 || n >= (1ll << 31) || nnz < 0 || nnz >= (1ll << 31)) {
        set_error("need 1 <= n < 2^31 and 0 <= nnz < 2^31");
        return RD_ERR_INVALID_ARG;
    }
    if (!row_ptr || (nnz > 0 && !col_idx)) {
        set_error("row_ptr/col_idx must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    rd_graph* g = new rd_graph();
    g->n = n;
    g->nnz_in = nnz;
    int l2 = 0;
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device) != cudaSuccess) {
        rd_status s = cuda_status(cudaGetLastError(), "cudaGetDevice");
        delete g;
        return s == RD_OK ? RD_ERR_CUDA : s;
    }
    g->l2_bytes = l2;
    rd_status s = graph_build(g, row_ptr, col_idx, weights, flags, static_cast<cudaStream_t>(stream));
    if (s < 0) {
        free_graph(g);
        return s;
    }
    *out = g;
    return RD_OK;
}

rd_status rd_graph_set_weights(rd_graph* g, const float* weights, void* stream)
{
    g_last_error.clear();
    if (!g || !weights) {
        set_error("graph and weights must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!g->w) RD_CUDA(cudaMalloc((void**)&g->w, sizeof(float) * std::max<int64_t>(g->nnz_in, 1)));
    if (g->keep_idx) {
        std::vector<float> win(g->nnz_in), wk(g->nnz);
        std::vector<int64_t> keep(g->nnz);
        RD_CUDA(cudaMemcpyAsync(win.data(), weights, sizeof(float) * g->nnz_in, cudaMemcpyDefault, st));
        RD_CUDA(cudaMemcpyAsync(keep.data(), g->keep_idx, sizeof(int64_t) * g->nnz, cudaMemcpyDeviceToHost, st));
        RD_CUDA(cudaStreamSynchronize(st));
        for (int64_t e = 0; e < g->nnz; ++e) wk[e] = win[keep[e]];
        RD_CUDA(cudaMemcpy(g->w, wk.data(), sizeof(float) * g->nnz, cudaMemcpyHostToDevice));
    } else if (g->nnz) {
        RD_CUDA(cudaMemcpyAsync(g->w, weights, sizeof(float) * g->nnz, cudaMemcpyDefault, st));
    }
    g->weighted = true;
    int64_t loops = 0;
    RD_TRY(check_csr(g, st, &loops));
    RD_TRY(compute_degrees(g, st));
    return rows_sorted_symmetric(g, st, &g->rows_sorted_sym);
}

rd_status rd_graph_destroy(rd_graph* g)
{
    free_graph(g);
    return RD_OK;
}

rd_status rd_graph_info(const rd_graph* g, int64_t* n, int64_t* nnz, int32_t* weighted, int32_t* ncomponents)
{
    if (!g) {
        set_error("graph is NULL");
        return RD_ERR_INVALID_ARG;
    }
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (weighted) *weighted = g->weighted ? 1 : 0;
    if (ncomponents) *ncomponents = g->ncomp;
    return RD_OK;
}

rd_status rd_last_call_stats(const rd_graph* g, rd_call_stats* out)
{
    if (!g || !out) {
        set_error("graph and out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    *out = g->stats;
    return RD_OK;
}

rd_status rd_query(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs, const rd_query_opts* opts,
                   double* r_out, int32_t* iters_out, double* err_est_out, int32_t* pair_status_out, void* stream)
{
    g_last_error.clear();
    rd_query_opts o;
    RD_TRY(validate_common(g, s, t, npairs, opts, &o));
    if (npairs > 0 && !r_out) {
        set_error("r_out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    g->stats = rd_call_stats{};
    if (npairs == 0) return RD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EventPool ev;
    rd_status call = RD_OK;
    if (o.flags & RD_Q_PLAIN) {
        // one pair per run through the single-vector SpMV path
        for (int64_t p = 0; p < npairs; ++p) {
            rd_status one = RD_OK;
            RD_TRY(query_batch(g, s + p, t + p, 1, o, true, r_out + p, iters_out ? iters_out + p : nullptr,
                               err_est_out ? err_est_out + p : nullptr,
                               pair_status_out ? pair_status_out + p : nullptr, st, &one, &ev, false, true));
            if (one == RD_WARN_NOT_CONVERGED) call = one;
        }
        return call;
    }
    const bool compact = (o.flags & RD_Q_NO_COMPACT) == 0;
    RD_TRY(query_batch(g, s, t, npairs, o, false, r_out, iters_out, err_est_out, pair_status_out, st, &call, &ev,
                       compact, true));
    return call;
}

rd_status rd_autotune(rd_graph* g, int64_t npairs, const rd_query_opts* opts, int32_t* rhs_tile_out,
                      int32_t* rows_per_warp_out, int32_t* kernel_out, void* stream)
{
    g_last_error.clear();
    rd_query_opts o;
    RD_TRY(validate_common(g, nullptr, nullptr, 0, opts, &o));
    if (npairs < 1 || npairs > (1ll << 24)) {
        set_error("npairs must be in [1, 2^24]");
        return RD_ERR_INVALID_ARG;
    }
    if (!tuning_allowed(o)) {
        set_error("rd_autotune needs rhs_tile, rows_per_warp and kernel at 0 and RD_Q_NO_TUNE unset");
        return RD_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool plain = (o.flags & RD_Q_PLAIN) != 0;
    RD_TRY(ensure_tuned(g, npairs, o, plain, !plain && (o.flags & RD_Q_NO_COMPACT) == 0, st));
    RD_CUDA(cudaStreamSynchronize(st));
    Plan pl;
    RD_TRY(make_plan(g, plain ? 1 : npairs, o, plain, &pl));
    if (rhs_tile_out) *rhs_tile_out = pl.cfg.tp();
    if (rows_per_warp_out) *rows_per_warp_out = pl.cfg.rpw();
    if (kernel_out) *kernel_out = kernel_code(pl.cfg);
    return RD_OK;
}

rd_status rd_edge_grad(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs, const double* grad_r,
                       const rd_query_opts* opts, float* grad_w_out, double* r_out, void* stream)
{
    g_last_error.clear();
    rd_query_opts o;
    RD_TRY(validate_common(g, s, t, npairs, opts, &o));
    if (o.mode == RD_MODE_DF64) o.mode = RD_MODE_FP64;  // double-float vectors: rd_query only
    if (!grad_w_out && g->nnz_in > 0) {
        set_error("grad_w_out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    g->stats = rd_call_stats{};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (npairs == 0) {
        if (g->nnz_in) RD_CUDA(cudaMemsetAsync(grad_w_out, 0, sizeof(float) * g->nnz_in, st));
        RD_CUDA(cudaStreamSynchronize(st));
        return RD_OK;
    }
    EventPool ev;
    RunCtx c;
    c.ev = &ev;
    RD_TRY(prepare_run(c, g, npairs, o, false, true, st));
    rd_status call = RD_OK;
    RD_TRY(forward_and_potential(c, s, t, grad_r, &call));
    // edge kernel over internal entries, then map to the caller's entry order
    if (!g->entry_row && g->nnz > 0) {
        RD_CUDA(cudaMalloc((void**)&g->entry_row, sizeof(int32_t) * g->nnz));
        launch_entry_rows(std::max(1, std::min(g->sm_count * 8, (int)((g->n + 7) / 8))), st, g->n, g->row_ptr,
                          g->entry_row);
        ++c.launches;
    }
    const int grid = std::max<int>(1, (int)std::min<int64_t>((int64_t)g->sm_count * 8, (g->nnz + 255) / 256));
    float* gint = c.b.grad;
    if (c.pl.fp64) {
        EdgeGradArgs<double> a{};
        a.n = g->n;
        a.ld = c.pl.ld;
        a.nnz = g->nnz;
        a.npairs = (int)npairs;
        a.row_ptr = g->row_ptr;
        a.col = g->col;
        a.entry_row = g->entry_row;
        a.phi = static_cast<const double*>(c.b.phi);
        a.gbar = static_cast<const double*>(c.b.gbar);
        a.grad_out = gint;
        launch_edge_grad_f64(grid, st, a);
    } else {
        EdgeGradArgs<float> a{};
        a.n = g->n;
        a.ld = c.pl.ld;
        a.nnz = g->nnz;
        a.npairs = (int)npairs;
        a.row_ptr = g->row_ptr;
        a.col = g->col;
        a.entry_row = g->entry_row;
        a.phi = static_cast<const float*>(c.b.phi);
        a.gbar = static_cast<const float*>(c.b.gbar);
        a.grad_out = gint;
        launch_edge_grad_f32(grid, st, a);
    }
    ++c.launches;
    if (g->keep_idx) {
        std::vector<float> gi(g->nnz), go(g->nnz_in, 0.0f);
        std::vector<int64_t> keep(g->nnz);
        RD_CUDA(cudaMemcpyAsync(gi.data(), gint, sizeof(float) * g->nnz, cudaMemcpyDeviceToHost, st));
        RD_CUDA(cudaMemcpyAsync(keep.data(), g->keep_idx, sizeof(int64_t) * g->nnz, cudaMemcpyDeviceToHost, st));
        RD_CUDA(cudaStreamSynchronize(st));
        for (int64_t e = 0; e < g->nnz; ++e) go[keep[e]] = gi[e];
        RD_CUDA(cudaMemcpyAsync(grad_w_out, go.data(), sizeof(float) * g->nnz_in, cudaMemcpyDefault, st));
        RD_CUDA(cudaStreamSynchronize(st));
    } else if (g->nnz) {
        RD_CUDA(cudaMemcpyAsync(grad_w_out, gint, sizeof(float) * g->nnz, cudaMemcpyDefault, st));
    }
    rd_status outs = RD_OK;
    RD_TRY(finish_outputs(c, r_out, nullptr, nullptr, nullptr, &outs));
    record_stats(c);
    return outs;
}

}  // extern "C"

namespace rd {
template <typename T>
__global__ void k_phi_out(int64_t n, int64_t ld, int npairs, const T* phi, float* out)
{
    const int64_t total = n * (int64_t)npairs;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t p = i / n, u = i % n;
        out[i] = (float)phi[u * ld + p];
    }
}
}  // namespace rd

extern "C" rd_status rd_potential(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs,
                                  const rd_query_opts* opts, float* phi_out, double* r_out, void* stream)
{
    g_last_error.clear();
    rd_query_opts o;
    RD_TRY(validate_common(g, s, t, npairs, opts, &o));
    if (o.mode == RD_MODE_DF64) o.mode = RD_MODE_FP64;  // double-float vectors: rd_query only
    if (npairs > 0 && !phi_out) {
        set_error("phi_out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    g->stats = rd_call_stats{};
    if (npairs == 0) return RD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EventPool ev;
    RunCtx c;
    c.ev = &ev;
    RD_TRY(prepare_run(c, g, npairs, o, false, true, st));
    rd_status call = RD_OK;
    RD_TRY(forward_and_potential(c, s, t, nullptr, &call));
    // phi (n x ld, q-space) -> pair-major float output
    float* stage = nullptr;
    const bool dev_out = is_device_ptr(phi_out);
    const size_t bytes = sizeof(float) * (size_t)g->n * (size_t)npairs;
    if (dev_out) {
        stage = phi_out;
    } else {
        RD_CUDA(cudaMallocAsync((void**)&stage, bytes, st));
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g->sm_count * 8, (g->n * npairs + 255) / 256));
    if (c.pl.fp64) k_phi_out<double><<<grid, 256, 0, st>>>(g->n, c.pl.ld, (int)npairs, static_cast<double*>(c.b.phi), stage);
    else k_phi_out<float><<<grid, 256, 0, st>>>(g->n, c.pl.ld, (int)npairs, static_cast<float*>(c.b.phi), stage);
    ++c.launches;
    if (!dev_out) {
        RD_CUDA(cudaMemcpyAsync(phi_out, stage, bytes, cudaMemcpyDeviceToHost, st));
        RD_CUDA(cudaFreeAsync(stage, st));
    }
    rd_status outs = RD_OK;
    RD_TRY(finish_outputs(c, r_out, nullptr, nullptr, nullptr, &outs));
    record_stats(c);
    return outs;
}

namespace rd {
// Potential differences along every stored entry (Section 6.3, Definition electric_flow:
// f(e) = phi(u) - phi(v) for e = (u, v)); one warp per row, lanes over the row's entries,
// output pair-major in the caller's entry order (dropped self-loops get 0).
template <typename T>
__global__ void k_flow(int64_t n, int64_t ld, int npairs, int64_t nnz_in, const int64_t* row_ptr,
                       const int32_t* col, const int64_t* keep_idx, const T* phi, float* out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        for (int64_t e = row_ptr[u] + lane; e < row_ptr[u + 1]; e += 32) {
            const int64_t v = col[e];
            const int64_t oe = keep_idx ? keep_idx[e] : e;
            for (int p = 0; p < npairs; ++p)
                out[(int64_t)p * nnz_in + oe] = (float)(phi[u * ld + p] - phi[v * ld + p]);
        }
    }
}
}  // namespace rd

extern "C" rd_status rd_flow(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs,
                             const rd_query_opts* opts, float* flow_out, double* r_out, void* stream)
{
    g_last_error.clear();
    rd_query_opts o;
    RD_TRY(validate_common(g, s, t, npairs, opts, &o));
    if (o.mode == RD_MODE_DF64) o.mode = RD_MODE_FP64;  // double-float vectors: rd_query only
    if (npairs > 0 && g->nnz_in > 0 && !flow_out) {
        set_error("flow_out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    g->stats = rd_call_stats{};
    if (npairs == 0) return RD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EventPool ev;
    RunCtx c;
    c.ev = &ev;
    RD_TRY(prepare_run(c, g, npairs, o, false, true, st));
    rd_status call = RD_OK;
    RD_TRY(forward_and_potential(c, s, t, nullptr, &call));
    const size_t bytes = sizeof(float) * (size_t)g->nnz_in * (size_t)npairs;
    const bool dev_out = is_device_ptr(flow_out);
    float* stage = dev_out ? flow_out : nullptr;
    if (!dev_out && bytes) RD_CUDA(cudaMallocAsync((void**)&stage, bytes, st));
    if (g->keep_idx && bytes) RD_CUDA(cudaMemsetAsync(stage, 0, bytes, st));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(g->sm_count * 8, (g->n + 7) / 8));
    if (c.pl.fp64)
        k_flow<double><<<grid, 256, 0, st>>>(g->n, c.pl.ld, (int)npairs, g->nnz_in, g->row_ptr, g->col, g->keep_idx,
                                             static_cast<const double*>(c.b.phi), stage);
    else
        k_flow<float><<<grid, 256, 0, st>>>(g->n, c.pl.ld, (int)npairs, g->nnz_in, g->row_ptr, g->col, g->keep_idx,
                                            static_cast<const float*>(c.b.phi), stage);
    ++c.launches;
    if (!dev_out && bytes) {
        RD_CUDA(cudaMemcpyAsync(flow_out, stage, bytes, cudaMemcpyDeviceToHost, st));
        RD_CUDA(cudaFreeAsync(stage, st));
    }
    rd_status outs = RD_OK;
    RD_TRY(finish_outputs(c, r_out, nullptr, nullptr, nullptr, &outs));
    record_stats(c);
    return outs;
}

// ============================================================ Power Method
// Algorithm 1 (Section 2.2) batched over pairs on the same SpMM kernels: in y = D^{-1} r
// the lazy walk r <- (I/2 + P/2) r reads y <- y/2 + D^{-1} W y / 2, and the estimate gains
// r(s)/(2 d_s) - r(t)/(2 d_t) = (y_s - y_t)/2 per step. A comparison baseline for the
// Lanczos iteration, which needs far fewer steps on graphs with large condition number.
namespace rd {
template <typename T>
static rd_status run_power_method(RunCtx& c, int steps, double* d_hist)
{
    const int64_t ld = c.pl.ld, n = c.g->n;
    RD_CUDA(cudaMemsetAsync(c.b.q[0], 0, n * ld * sizeof(T), c.st));
    RD_CUDA(cudaMemsetAsync(c.b.q[1], 0, n * ld * sizeof(T), c.st));
    char* base = static_cast<char*>(c.g->ws.base);
    RD_CUDA(cudaMemsetAsync(base + c.b.state_bytes_begin, 0, c.b.state_bytes_end - c.b.state_bytes_begin, c.st));
    PmArgs pa{};
    pa.n = n;
    pa.ld = ld;
    pa.npairs = (int)c.P;
    pa.s = c.b.s;
    pa.t = c.b.t;
    pa.deg64 = c.g->deg64;
    pa.rbar = c.b.st.r;
    pa.hist = d_hist;
    pa.elem_size = (int)sizeof(T);
    pa.err_flag = c.b.err_flag;
    pa.y = c.b.q[1];
    launch_pm_init(c.st, pa);
    ++c.launches;
    int* h = c.g->h_pinned;
    RD_CUDA(cudaMemcpyAsync(h, c.b.err_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, c.st));
    RD_CUDA(cudaStreamSynchronize(c.st));
    if (h[0]) {
        set_error("a pair id is outside [0, n)");
        return RD_ERR_INVALID_ARG;
    }
    c.lazy_walk = true;
    for (int i = 0; i <= steps; ++i) {
        pa.y = c.b.q[1];
        pa.step = i;
        launch_pm_accum(c.st, pa);
        ++c.launches;
        if (i == steps) break;
        RD_TRY(enqueue_spmm<T>(c, 0, false));  // writes y_{i+1} into q[0]
        std::swap(c.b.q[0], c.b.q[1]);
        c.steps = i + 1;
    }
    RD_CUDA(cudaGetLastError());
    return RD_OK;
}
}  // namespace rd

extern "C" rd_status rd_power_method(rd_graph* g, const int32_t* s, const int32_t* t, int64_t npairs, int32_t steps,
                                     int32_t mode, double* r_out, double* r_hist_out, void* stream)
{
    g_last_error.clear();
    rd_query_opts o;
    rd_query_opts_init(&o);
    o.mode = mode;
    o.k_max = steps + 1;
    o.kernel = 1;  // row-group kernel (the heavy-row pre-pass and chunk sums apply as in rd_query)
    if (steps < 0 || steps >= (1 << 22)) {
        set_error("steps must be in [0, 2^22)");
        return RD_ERR_INVALID_ARG;
    }
    RD_TRY(validate_common(g, s, t, npairs, &o, &o));
    if (o.mode == RD_MODE_DF64) o.mode = RD_MODE_FP64;  // double-float vectors: rd_query only
    if (npairs > 0 && !r_out) {
        set_error("r_out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    g->stats = rd_call_stats{};
    if (npairs == 0) return RD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EventPool ev;
    RunCtx c;
    c.ev = &ev;
    RD_TRY(prepare_run(c, g, npairs, o, false, false, st));
    RD_TRY(stage_pairs(c, s, t));
    // the history reuses the alpha history block: (k_max) x ld doubles >= (steps + 1) x npairs
    double* d_hist = c.b.st.hist_alpha;
    rd_status rs = c.pl.fp64 ? run_power_method<double>(c, steps, d_hist) : run_power_method<float>(c, steps, d_hist);
    if (rs < 0) return rs;
    RD_CUDA(cudaMemcpyAsync(r_out, c.b.st.r, sizeof(double) * npairs, cudaMemcpyDefault, st));
    if (r_hist_out)
        RD_CUDA(cudaMemcpyAsync(r_hist_out, d_hist, sizeof(double) * npairs * (size_t)(steps + 1), cudaMemcpyDefault,
                                st));
    RD_CUDA(cudaStreamSynchronize(st));
    record_stats(c);
    return RD_OK;
}

namespace rd {
rd_status triangle_weights(int64_t n, const int64_t* rp, const int32_t* col, float* w_out, int sm_count,
                           cudaStream_t st, int32_t* flag_dev);
}

extern "C" rd_status rd_triangle_weights(const rd_graph* g, float* w_out, void* stream)
{
    g_last_error.clear();
    if (!g || (!w_out && g->nnz_in > 0)) {
        set_error("graph and w_out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    if (g->keep_idx) {
        set_error("the graph had self-loops; pass a loop-free CSR for triangle weights");
        return RD_ERR_UNSUPPORTED;
    }
    if (g->nnz == 0) return RD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool dev_out = is_device_ptr(w_out);
    float* stage = dev_out ? w_out : nullptr;
    int32_t* flag = nullptr;
    RD_CUDA(cudaMallocAsync((void**)&flag, sizeof(int32_t), st));
    if (!dev_out) RD_CUDA(cudaMallocAsync((void**)&stage, sizeof(float) * g->nnz, st));
    rd_status rs = triangle_weights(g->n, g->row_ptr, g->col, stage, g->sm_count, st, flag);
    if (rs == RD_OK && !dev_out)
        RD_CUDA(cudaMemcpyAsync(w_out, stage, sizeof(float) * g->nnz, cudaMemcpyDeviceToHost, st));
    if (!dev_out) cudaFreeAsync(stage, st);
    cudaFreeAsync(flag, st);
    RD_CUDA(cudaStreamSynchronize(st));
    return rs;
}

// ===================================================== query without allocation
// rd_query_noalloc: the batched query for callers that must not allocate device memory
// (code that runs where cudaMalloc is unavailable or forbidden -- inside another
// framework's memory pool or allocator hooks, or in a process whose device memory is
// fully reserved up front). All of its scratch lives in one fixed, file-scope device
// array; the graph is the caller's device CSR, used in place.
namespace rd {

rd_status check_csr_scratch(rd_graph* g, cudaStream_t st, void* flags_dev, int64_t* self_loops);
rd_status compute_degrees_scratch(rd_graph* g, cudaStream_t st, void* flags_dev, double* block_sums_dev,
                                  double* block_sums_host);
int degree_grid(const rd_graph* g);

// 32 MiB of scratch, held by every GPU that loads this library until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 256;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices];

// Device address of the scratch array on device `dev` (the current device). In host code
// the array's name only stands in for the symbol; the address comes from
// cudaGetSymbolAddress, fetched once per device on that device's first call.
static rd_status noalloc_scratch_address(int dev, void** out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device ordinal out of range for the no-allocation scratch table");
        return RD_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                       "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return RD_OK;
}

}  // namespace rd

extern "C" rd_status rd_query_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                      const float* weights, const int32_t* s, const int32_t* t, int64_t npairs,
                                      const rd_query_opts* opts, double* r_out, int32_t* iters_out, void* stream)
{
    g_last_error.clear();
    if (n < 1 || n >= (1ll << 31) || nnz < 0 || nnz >= (1ll << 31) || npairs < 0) {
        set_error("need 1 <= n < 2^31, 0 <= nnz < 2^31 and npairs >= 0");
        return RD_ERR_INVALID_ARG;
    }
    if (!row_ptr || (nnz > 0 && !col_idx) || (npairs > 0 && (!s || !t || !r_out))) {
        set_error("row_ptr, col_idx, s, t and r_out must not be NULL");
        return RD_ERR_INVALID_ARG;
    }
    const void* need_dev[] = {row_ptr, nnz > 0 ? col_idx : nullptr, weights, npairs > 0 ? s : nullptr,
                              npairs > 0 ? t : nullptr, npairs > 0 ? r_out : nullptr,
                              npairs > 0 ? iters_out : nullptr};
    for (const void* p : need_dev)
        if (p && !is_device_ptr(p)) {
            set_error("rd_query_noalloc takes device pointers only");
            return RD_ERR_INVALID_ARG;
        }
    rd_graph g;
    if (cudaGetDevice(&g.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g.sm_count, cudaDevAttrMultiProcessorCount, g.device) != cudaSuccess) {
        rd_status st = cuda_status(cudaGetLastError(), "cudaGetDevice");
        return st == RD_OK ? RD_ERR_CUDA : st;
    }
    g.n = n;
    g.nnz = g.nnz_in = nnz;
    g.weighted = weights != nullptr;
    g.row_ptr = const_cast<int64_t*>(row_ptr);
    g.col = const_cast<int32_t*>(col_idx);
    g.w = const_cast<float*>(weights);
    g.heavy_thr = INT32_MAX;  // no heavy-row chunk lists: the row-group kernel takes every row whole
    static thread_local int host_poll[16];
    static thread_local double host_block_sums[1 << 14];
    g.h_pinned = host_poll;

    rd_query_opts o;
    RD_TRY(validate_common(&g, s, t, npairs, opts, &o));
    if (o.mode == RD_MODE_DF64) o.mode = RD_MODE_FP64;  // double-float vectors: rd_query only
    o.flags &= ~RD_Q_PROFILE;  // no event objects
    // no timing runs (they could need a larger workspace) and no graph objects
    o.flags |= RD_Q_NO_TUNE | RD_Q_NO_GRAPH;
    o.kernel = 1;              // row-group kernel: needs no task list
    if (npairs == 0) return RD_OK;

    void* base = nullptr;
    RD_TRY(noalloc_scratch_address(g.device, &base));
    // graph-derived arrays first, then the query workspace (same layout as rd_query's)
    Carver cg(base);
    void* flags_dev = cg.take<char>(64);
    double* bsum = cg.take<double>(1 << 14);
    g.deg64 = cg.take<double>(n);
    g.invdeg64 = cg.take<double>(n);
    g.deg32 = cg.take<float>(n);
    g.invdeg32 = cg.take<float>(n);
    const size_t graph_bytes = (cg.off + 255) & ~size_t(255);
    if (degree_grid(&g) > (1 << 14)) {
        set_error("too many SMs for the no-allocation degree buffer");
        return RD_ERR_UNSUPPORTED;
    }
    const bool plain = (o.flags & RD_Q_PLAIN) != 0;
    Plan pl;
    RD_TRY(make_plan(&g, plain ? 1 : npairs, o, plain, &pl));
    Buffers tmp;
    Carver dry(nullptr);
    const size_t query_bytes = carve(dry, &g, pl, plain ? 1 : npairs, false, &tmp);
    if (graph_bytes + query_bytes > kNoAllocScratchBytes) {
        set_error("rd_query_noalloc needs " + std::to_string(graph_bytes + query_bytes) +
                  " bytes of scratch for this graph, pair count and k_max; its fixed scratch holds " +
                  std::to_string(kNoAllocScratchBytes) + " bytes (use rd_graph_create/rd_query instead)");
        return RD_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t loops = 0;
    RD_TRY(check_csr_scratch(&g, st, flags_dev, &loops));
    if (loops > 0) {
        set_error("the CSR holds self-loops; rd_query_noalloc cannot rebuild it (use rd_graph_create)");
        return RD_ERR_UNSUPPORTED;
    }
    RD_TRY(compute_degrees_scratch(&g, st, flags_dev, bsum, host_block_sums));
    g.ws.base = static_cast<char*>(base) + graph_bytes;
    g.ws.bytes = kNoAllocScratchBytes - graph_bytes;  // >= query_bytes, so nothing is allocated
    EventPool ev;
    rd_status call = RD_OK;
    if (plain) {
        for (int64_t p = 0; p < npairs; ++p) {
            rd_status one = RD_OK;
            RD_TRY(query_batch(&g, s + p, t + p, 1, o, true, r_out + p, iters_out ? iters_out + p : nullptr,
                               nullptr, nullptr, st, &one, &ev));
            if (one == RD_WARN_NOT_CONVERGED) call = one;
        }
        return call;
    }
    RD_TRY(query_batch(&g, s, t, npairs, o, false, r_out, iters_out, nullptr, nullptr, st, &call, &ev));
    return call;
}

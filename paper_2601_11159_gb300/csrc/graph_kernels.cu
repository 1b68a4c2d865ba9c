// Graph ingest kernels: CSR validation and degrees (Section 2.1: d_u = sum of the
// weights of u's edges; Section 2.2: the D^{-1/2} scaling of Ahat, applied here as
// 1/d_u per row because vectors are kept as q = D^{-1/2} v).
#include <math.h>

#include "rd_internal.cuh"

namespace rd {

struct CheckFlags {
    int32_t bad_rowptr;
    int32_t bad_col;
    int32_t bad_weight;
    int32_t zero_degree;
    unsigned long long self_loops;
};

__global__ void k_check_csr(int64_t n, int64_t nnz, const int64_t* rp, const int32_t* col, const float* w,
                            CheckFlags* f)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t u = tid; u < n; u += stride) {
        const int64_t a = rp[u], b = rp[u + 1];
        if (a > b || a < 0 || b > nnz) atomicOr(&f->bad_rowptr, 1);
    }
    if (tid == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(&f->bad_rowptr, 1);
    for (int64_t e = tid; e < nnz; e += stride) {
        const int32_t c = col[e];
        if (c < 0 || (int64_t)c >= n) atomicOr(&f->bad_col, 1);
        if (w) {
            const float x = w[e];
            if (!(x > 0.0f) || !isfinite(x)) atomicOr(&f->bad_weight, 1);
        }
    }
}

// Flags a CSR whose rows are not strictly increasing in column, or which is not symmetric
// entry for entry (row v holds u with the same weight bits as row u holds v): the sparse
// first Lanczos step reads row s's weights in place of row u's.
__global__ void k_rows_not_sorted_symmetric(int64_t n, const int64_t* rp, const int32_t* col, const float* w,
                                            int32_t* flag)
{
    // one warp per row, lanes over its entries
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += nwarps) {
        const int64_t beg = rp[u], end = rp[u + 1];
        bool bad = false;
        for (int64_t e = beg + lane; e < end && !bad; e += 32) {
            const int32_t v = col[e];
            if (e > beg && v <= col[e - 1]) {
                bad = true;
                break;
            }
            const int64_t vend = rp[v + 1];
            int64_t lo = rp[v], hi = vend;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (col[mid] < (int32_t)u) lo = mid + 1; else hi = mid;
            }
            bad = lo >= vend || col[lo] != (int32_t)u ||
                  (w != nullptr && __float_as_uint(w[lo]) != __float_as_uint(w[e]));
        }
        if (bad) atomicOr(flag, 1);
    }
}

// Self-loops need the row of each entry: one thread per row.
__global__ void k_count_self_loops(int64_t n, const int64_t* rp, const int32_t* col, CheckFlags* f)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        unsigned long long c = 0;
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) c += (col[e] == (int32_t)u);
        if (c) atomicAdd(&f->self_loops, c);
    }
}

// Degrees in FP64 (fixed order along the row), derived FP32/FP64 copies, and
// per-block partial sums of the degrees (summed on the host in block order).
__global__ void k_degrees(int64_t n, const int64_t* rp, const float* w, double* deg64, double* invdeg64,
                          float* deg32, float* invdeg32, double* block_sum, CheckFlags* f)
{
    __shared__ double red[256];
    double local = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        double d = 0.0;
        if (w) {
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) d += (double)w[e];
        } else {
            d = (double)(rp[u + 1] - rp[u]);
        }
        deg64[u] = d;
        invdeg64[u] = d > 0.0 ? 1.0 / d : 0.0;
        deg32[u] = (float)d;
        invdeg32[u] = d > 0.0 ? (float)(1.0 / d) : 0.0f;
        if (!(d > 0.0)) atomicOr(&f->zero_degree, 1);
        local += d;
    }
    red[threadIdx.x] = local;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sum[blockIdx.x] = red[0];
}

static int grid_for(int64_t work, int sm)
{
    int64_t g = (work + 255) / 256;
    const int64_t cap = (int64_t)sm * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

rd_status rows_sorted_symmetric(rd_graph* g, cudaStream_t st, bool* out)
{
    int32_t* f = nullptr;
    RD_CUDA(cudaMallocAsync((void**)&f, sizeof(int32_t), st));
    RD_CUDA(cudaMemsetAsync(f, 0, sizeof(int32_t), st));
    if (g->n > 0)
        k_rows_not_sorted_symmetric<<<grid_for(g->n, g->sm_count), 256, 0, st>>>(g->n, g->row_ptr, g->col, g->w, f);
    int32_t h = 0;
    RD_CUDA(cudaMemcpyAsync(&h, f, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaFreeAsync(f, st));
    RD_CUDA(cudaStreamSynchronize(st));
    *out = h == 0;
    return RD_OK;
}

rd_status check_csr(rd_graph* g, cudaStream_t st, int64_t* self_loops)
{
    CheckFlags* f = nullptr;
    RD_CUDA(cudaMallocAsync((void**)&f, sizeof(CheckFlags), st));
    RD_CUDA(cudaMemsetAsync(f, 0, sizeof(CheckFlags), st));
    k_check_csr<<<grid_for(g->nnz > g->n ? g->nnz : g->n, g->sm_count), 256, 0, st>>>(g->n, g->nnz, g->row_ptr,
                                                                                       g->col, g->w, f);
    CheckFlags h{};
    RD_CUDA(cudaMemcpyAsync(&h, f, sizeof(CheckFlags), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaStreamSynchronize(st));
    if (h.bad_rowptr) {
        cudaFreeAsync(f, st);
        set_error("row_ptr must start at 0, be non-decreasing and end at nnz");
        return RD_ERR_INVALID_ARG;
    }
    if (h.bad_col) {
        cudaFreeAsync(f, st);
        set_error("a column index is outside [0, n)");
        return RD_ERR_INVALID_ARG;
    }
    if (h.bad_weight) {
        cudaFreeAsync(f, st);
        set_error("edge weights must be finite and > 0");
        return RD_ERR_INVALID_ARG;
    }
    k_count_self_loops<<<grid_for(g->n, g->sm_count), 256, 0, st>>>(g->n, g->row_ptr, g->col, f);
    RD_CUDA(cudaMemcpyAsync(&h, f, sizeof(CheckFlags), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaFreeAsync(f, st));
    RD_CUDA(cudaStreamSynchronize(st));
    *self_loops = (int64_t)h.self_loops;
    return RD_OK;
}

rd_status compute_degrees(rd_graph* g, cudaStream_t st)
{
    const int grid = grid_for(g->n, g->sm_count);
    CheckFlags* f = nullptr;
    double* bs = nullptr;
    RD_CUDA(cudaMallocAsync((void**)&f, sizeof(CheckFlags), st));
    RD_CUDA(cudaMallocAsync((void**)&bs, sizeof(double) * grid, st));
    RD_CUDA(cudaMemsetAsync(f, 0, sizeof(CheckFlags), st));
    k_degrees<<<grid, 256, 0, st>>>(g->n, g->row_ptr, g->w, g->deg64, g->invdeg64, g->deg32, g->invdeg32, bs, f);
    CheckFlags h{};
    std::vector<double> hb(grid);
    RD_CUDA(cudaMemcpyAsync(&h, f, sizeof(CheckFlags), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaMemcpyAsync(hb.data(), bs, sizeof(double) * grid, cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaFreeAsync(f, st));
    RD_CUDA(cudaFreeAsync(bs, st));
    RD_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double x : hb) s += x;
    g->sumdeg = s;
    g->mean_deg = g->n ? s / (double)g->n : 0.0;
    if (h.zero_degree && g->n > 1) {
        set_error("a vertex has degree 0 (isolated vertex)");
        return RD_ERR_ZERO_DEGREE;
    }
    return RD_OK;
}

}  // namespace rd

namespace rd {

// Variants of check_csr / compute_degrees for callers that cannot allocate: the flag
// block and the per-block degree sums live in caller-provided device scratch, and the
// block sums come back through a fixed host buffer.
rd_status check_csr_scratch(rd_graph* g, cudaStream_t st, void* flags_dev, int64_t* self_loops)
{
    CheckFlags* f = static_cast<CheckFlags*>(flags_dev);
    CheckFlags h{};
    RD_CUDA(cudaMemsetAsync(f, 0, sizeof(CheckFlags), st));
    k_check_csr<<<grid_for(g->nnz > g->n ? g->nnz : g->n, g->sm_count), 256, 0, st>>>(g->n, g->nnz, g->row_ptr,
                                                                                       g->col, g->w, f);
    RD_CUDA(cudaMemcpyAsync(&h, f, sizeof(CheckFlags), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaStreamSynchronize(st));
    if (h.bad_rowptr) {
        set_error("row_ptr must start at 0, be non-decreasing and end at nnz");
        return RD_ERR_INVALID_ARG;
    }
    if (h.bad_col) {
        set_error("a column index is outside [0, n)");
        return RD_ERR_INVALID_ARG;
    }
    if (h.bad_weight) {
        set_error("edge weights must be finite and > 0");
        return RD_ERR_INVALID_ARG;
    }
    k_count_self_loops<<<grid_for(g->n, g->sm_count), 256, 0, st>>>(g->n, g->row_ptr, g->col, f);
    RD_CUDA(cudaMemcpyAsync(&h, f, sizeof(CheckFlags), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaStreamSynchronize(st));
    *self_loops = (int64_t)h.self_loops;
    return RD_OK;
}

int degree_grid(const rd_graph* g) { return grid_for(g->n, g->sm_count); }

rd_status compute_degrees_scratch(rd_graph* g, cudaStream_t st, void* flags_dev, double* block_sums_dev,
                                  double* block_sums_host)
{
    const int grid = grid_for(g->n, g->sm_count);
    CheckFlags* f = static_cast<CheckFlags*>(flags_dev);
    CheckFlags h{};
    RD_CUDA(cudaMemsetAsync(f, 0, sizeof(CheckFlags), st));
    k_degrees<<<grid, 256, 0, st>>>(g->n, g->row_ptr, g->w, g->deg64, g->invdeg64, g->deg32, g->invdeg32,
                                    block_sums_dev, f);
    RD_CUDA(cudaMemcpyAsync(&h, f, sizeof(CheckFlags), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaMemcpyAsync(block_sums_host, block_sums_dev, sizeof(double) * grid, cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int i = 0; i < grid; ++i) s += block_sums_host[i];
    g->sumdeg = s;
    g->mean_deg = g->n ? s / (double)g->n : 0.0;
    if (h.zero_degree && g->n > 1) {
        set_error("a vertex has degree 0 (isolated vertex)");
        return RD_ERR_ZERO_DEGREE;
    }
    return RD_OK;
}

}  // namespace rd

namespace rd {

// Triangle-count weights (the weighted setting of the paper's Exp-2): for stored entry
// e = (u, v), w(e) = |N(u) & N(v)| (the triangles through edge uv), or 1 when that is 0.
// One thread per entry: every element of the shorter adjacency list is looked up in the
// longer one by binary search (rows must be sorted by column).
__global__ void k_triangle_weights(int64_t n, const int64_t* rp, const int32_t* col, float* w_out, int32_t* unsorted)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int64_t a0 = rp[u], a1 = rp[u + 1];
        for (int64_t e = a0; e < a1; ++e) {
            if (e > a0 && col[e] <= col[e - 1]) atomicOr(unsorted, 1);
            const int64_t v = col[e];
            const int64_t b0 = rp[v], b1 = rp[v + 1];
            int64_t s0 = a0, s1 = a1, l0 = b0, l1 = b1;  // shorter list [s0,s1), longer [l0,l1)
            if (a1 - a0 > b1 - b0) {
                s0 = b0; s1 = b1; l0 = a0; l1 = a1;
            }
            int64_t cnt = 0;
            for (int64_t i = s0; i < s1; ++i) {
                const int32_t x = col[i];
                int64_t lo = l0, hi = l1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (col[mid] < x) lo = mid + 1; else hi = mid;
                }
                cnt += (lo < l1 && col[lo] == x);
            }
            w_out[e] = cnt > 0 ? (float)cnt : 1.0f;
        }
    }
}

rd_status triangle_weights(int64_t n, const int64_t* rp, const int32_t* col, float* w_out, int sm_count,
                           cudaStream_t st, int32_t* flag_dev)
{
    RD_CUDA(cudaMemsetAsync(flag_dev, 0, sizeof(int32_t), st));
    k_triangle_weights<<<grid_for(n, sm_count), 256, 0, st>>>(n, rp, col, w_out, flag_dev);
    int32_t h = 0;
    RD_CUDA(cudaMemcpyAsync(&h, flag_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RD_CUDA(cudaStreamSynchronize(st));
    if (h) {
        set_error("triangle weights need every row's columns sorted increasingly and without duplicates");
        return RD_ERR_INVALID_ARG;
    }
    return RD_OK;
}

}  // namespace rd

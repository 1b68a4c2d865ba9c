// SpMM / SpMV step of the batched Lanczos recurrence (Algorithm 3: the product
// w = Ahat v_i - beta_i v_{i-1} of the three-term recurrence, Section 3), fused with the
// partial sums of alpha_i = <w, v_i>, ||w||^2 and the component of w along D^{1/2}1.
//
// Vectors are kept in q-space, q = D^{-1/2} v, so that
//   D^{-1/2}(Ahat v - beta v') = D^{-1} W q - beta q'        (row u: (1/d_u) sum_e w_e q[col_e])
//   <x, y> = sum_u d_u q_x[u] q_y[u],   <x, D^{1/2}1> = sum_u d_u q_x[u].
// No per-nonzero degree scaling is needed: the gather is a plain (weighted) sum.
//
// Layout: vector blocks are n x ld row-major (element (u, p) at u*ld + p), one column
// per (s,t) pair. A warp is split into row groups (see SpmmCfg); the grid sweeps the
// columns in slabs of TP = VEC*GS so that one slab of the gathered block stays hot in
// L2 while all rows are processed. Rows whose degree exceeds heavy_thr are split into
// chunks summed beforehand by k_spmm_heavy, so no warp owns a long row.
//
// Determinism: every sum has a fixed order (row loop order, chunk order, xor-shuffle
// trees, warp order, block order in the finalize kernel), so repeated runs and the
// replay pass of the gradient produce bitwise-identical vectors.
#pragma once

#include <cuda_runtime.h>
#include <string.h>

#include "df64.cuh"
#include "rd_internal.cuh"

namespace rd {

// ---------------------------------------------------------- vector memory ops
template <typename T, int VEC>
__device__ __forceinline__ void ld_gather(T (&r)[VEC], const T* p)
{
    constexpr int B = (int)sizeof(T) * VEC;
    if constexpr (B >= 16) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            float4 x = __ldg(q + i);
            memcpy(&r[i * (16 / (int)sizeof(T))], &x, 16);
        }
    } else if constexpr (B == 8) {
        float2 x = __ldg(reinterpret_cast<const float2*>(p));
        memcpy(&r[0], &x, 8);
    } else {
        float x = __ldg(reinterpret_cast<const float*>(p));
        memcpy(&r[0], &x, 4);
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void ld_stream(T (&r)[VEC], const T* p)
{
    constexpr int B = (int)sizeof(T) * VEC;
    if constexpr (B >= 16) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            float4 x = __ldcs(q + i);
            memcpy(&r[i * (16 / (int)sizeof(T))], &x, 16);
        }
    } else if constexpr (B == 8) {
        float2 x = __ldcs(reinterpret_cast<const float2*>(p));
        memcpy(&r[0], &x, 8);
    } else {
        float x = __ldcs(reinterpret_cast<const float*>(p));
        memcpy(&r[0], &x, 4);
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void ld_plain(T (&r)[VEC], const T* p)
{
    constexpr int B = (int)sizeof(T) * VEC;
    if constexpr (B >= 16) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            float4 x = q[i];
            memcpy(&r[i * (16 / (int)sizeof(T))], &x, 16);
        }
    } else if constexpr (B == 8) {
        float2 x = *reinterpret_cast<const float2*>(p);
        memcpy(&r[0], &x, 8);
    } else {
        float x = *reinterpret_cast<const float*>(p);
        memcpy(&r[0], &x, 4);
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void st_stream(T* p, const T (&r)[VEC])
{
    constexpr int B = (int)sizeof(T) * VEC;
    if constexpr (B >= 16) {
        float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            float4 x;
            memcpy(&x, &r[i * (16 / (int)sizeof(T))], 16);
            __stcs(q + i, x);
        }
    } else if constexpr (B == 8) {
        float2 x;
        memcpy(&x, &r[0], 8);
        __stcs(reinterpret_cast<float2*>(p), x);
    } else {
        float x;
        memcpy(&x, &r[0], 4);
        __stcs(reinterpret_cast<float*>(p), x);
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void st_plain(T* p, const T (&r)[VEC])
{
    constexpr int B = (int)sizeof(T) * VEC;
    if constexpr (B >= 16) {
        float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            float4 x;
            memcpy(&x, &r[i * (16 / (int)sizeof(T))], 16);
            q[i] = x;
        }
    } else if constexpr (B == 8) {
        float2 x;
        memcpy(&x, &r[0], 8);
        *reinterpret_cast<float2*>(p) = x;
    } else {
        float x;
        memcpy(&x, &r[0], 4);
        *reinterpret_cast<float*>(p) = x;
    }
}

// Gathers with an L2 eviction-priority hint (createpolicy + ld.global.nc.L2::cache_hint):
// rows that many nonzeros point to are kept (evict_last), the long tail of rarely
// gathered rows is let go first (evict_first), so the tail does not push the hot rows
// out of L2.
#ifndef RD_GATHER_HINT
#define RD_GATHER_HINT 1
#endif

__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float4 ld_f4_policy(const float4* p, uint64_t pol)
{
    float4 r;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}

template <typename T, int VEC>
__device__ __forceinline__ void ld_gather_pol(T (&r)[VEC], const T* p, uint64_t pol)
{
    constexpr int B = (int)sizeof(T) * VEC;
    if constexpr (B >= 16) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < B / 16; ++i) {
            float4 x = ld_f4_policy(q + i, pol);
            memcpy(&r[i * (16 / (int)sizeof(T))], &x, 16);
        }
    } else {
        ld_gather<T, VEC>(r, p);
    }
}

// ------------------------------------------------------------ accumulators
// FP32 partial sums use Kahan compensation (error independent of the number of
// terms to first order); FP64 sums are plain.
template <typename T>
struct Acc;

template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<df64> {
    df64 s = df64(0);
    __device__ __forceinline__ void add(df64 x) { s += x; }
    __device__ __forceinline__ double value() const { return (double)s; }
};

// Independent gathers in flight per lane per round: 8 for 16-byte lanes, 4 for wider ones.
#ifndef RD_ROWS_UNROLL
#define RD_ROWS_UNROLL 8
#endif
template <typename T, int VEC>
inline constexpr int kUnroll = (int)sizeof(T) * VEC > 16 ? (RD_ROWS_UNROLL > 4 ? 4 : RD_ROWS_UNROLL) : RD_ROWS_UNROLL;

// Sum over the nonzeros [beg, end) of w_e * q[col_e, c0 .. c0+VEC), shared by the G = GS*NZL
// lanes of a row group: the group loads up to G column indices (and weights) with one
// coalesced load, broadcasts them by shuffle, and each of the NZL nonzero lanes issues U
// independent gathers per round (nonzero k of the chunk goes to lane zl = k % NZL).
template <typename T, int VEC, int GS, int NZL, int U, bool WEIGHTED>
__device__ __forceinline__ void gather_row(const StepArgs<T>& a, int64_t beg, int64_t end, int64_t c0, int li,
                                           int zl, unsigned mask, T (&acc)[VEC])
{
    constexpr int G = GS * NZL;
    const T* __restrict__ q = a.qcur + c0;
    const int64_t ld = a.ld;
    if constexpr (GS == 1) {
        // one column: lane zl takes nonzeros zl, zl + NZL, zl + 2 NZL, ... (the order of the
        // general loop below), loading U indices and keeping U gathers in flight per round
        for (int64_t base = beg; base < end; base += (int64_t)NZL * U) {
            int j[U];
            float wu[U];
            T x[U][VEC];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = base + (int64_t)u * NZL + zl;
                j[u] = e < end ? __ldg(a.col + e) : -1;
                if constexpr (WEIGHTED) wu[u] = e < end ? __ldg(a.w + e) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j[u] >= 0) {
                    ld_gather<T, VEC>(x[u], q + (int64_t)j[u] * ld);
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; ++i) x[u][i] = T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    if constexpr (WEIGHTED) acc_mul_add_w(acc[i], wu[u], x[u][i]);
                    else acc_add(acc[i], x[u][i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc_finish(acc[i]);
        return;
    }
    for (int64_t base = beg; base < end; base += G) {
        const int cnt = (int)(end - base < G ? end - base : G);
        const int my_col = li < cnt ? __ldg(a.col + base + li) : 0;
        float my_w = 1.0f;
        if constexpr (WEIGHTED) my_w = li < cnt ? __ldg(a.w + base + li) : 0.0f;
        for (int k0 = 0; k0 < cnt; k0 += NZL * U) {
            T x[U][VEC];
            float wu[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int kk = k0 + zl + u * NZL;
                const int j = __shfl_sync(mask, my_col, kk & (G - 1), G);
                if constexpr (WEIGHTED) wu[u] = __shfl_sync(mask, my_w, kk & (G - 1), G);
                if (kk < cnt) {
                    ld_gather<T, VEC>(x[u], q + (int64_t)j * ld);
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; ++i) x[u][i] = T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    if constexpr (WEIGHTED) acc_mul_add_w(acc[i], wu[u], x[u][i]);
                    else acc_add(acc[i], x[u][i]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < VEC; ++i) acc_finish(acc[i]);
}

template <int GS, int NZL, typename T, int VEC>
__device__ __forceinline__ void reduce_nzl(T (&acc)[VEC], unsigned mask)
{
#pragma unroll
    for (int off = GS; off < GS * NZL; off <<= 1) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[i] += shfl_xor_t(mask, acc[i], off);
    }
}

template <int GS, int NZL>
__device__ __forceinline__ unsigned group_mask(int lane)
{
    constexpr int W = GS * NZL;
    if constexpr (W == 32) {
        return 0xffffffffu;
    } else {
        const int rs = lane / W;
        return ((1u << W) - 1u) << (rs * W);
    }
}

// Block partial sums of the three reductions for one slab: lanes holding the same
// columns are combined by an xor-shuffle tree (fixed order), then warps in warp order.
template <typename T, int VEC, int GW, int TP>
__device__ __forceinline__ void block_partials(const StepArgs<T>& a, const Acc<T> (&sA)[VEC], const Acc<T> (&sB)[VEC],
                                               const Acc<T> (&sC)[VEC], double (&red)[kWarps][TP], int slab,
                                               int lane, int warp, int cl)
{
#pragma unroll
    for (int qn = 0; qn < 3; ++qn) {
        double v[VEC];
#pragma unroll
        for (int i = 0; i < VEC; ++i) v[i] = qn == 0 ? sA[i].value() : (qn == 1 ? sB[i].value() : sC[i].value());
#pragma unroll
        for (int off = GW; off < 32; off <<= 1) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
        }
        if (lane < TP / VEC) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) red[warp][cl * VEC + i] = v[i];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < TP; c += kBlock) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) sum += red[w][c];
            a.block_part[(((int64_t)slab * gridDim.x + blockIdx.x) * 3 + qn) * TP + c] = sum;
        }
        __syncthreads();
    }
}

// Epilogue of one row: W = invd * acc - beta * q_prev written over q_prev, and the
// row's terms of sum d W q_cur, sum d W^2, sum d W added to the lane's accumulators.
template <typename T, int VEC>
__device__ __forceinline__ void row_epilogue(const StepArgs<T>& a, int64_t row, int64_t c0, T invd, T du,
                                             const T (&acc)[VEC], const T (&bt)[VEC], const T (&qp)[VEC],
                                             const T (&qc)[VEC], Acc<T> (&sA)[VEC], Acc<T> (&sB)[VEC],
                                             Acc<T> (&sC)[VEC])
{
    T wv[VEC];
    if (a.lazy_walk) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) wv[i] = T(0.5) * (invd * acc[i]) + T(0.5) * qc[i];
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) wv[i] = invd * acc[i] - bt[i] * qp[i];
    }
    st_stream<T, VEC>(a.qprev_w + row * a.ld + c0, wv);
    if (a.do_reduce) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            const T dw = du * wv[i];
            sA[i].add(dw * qc[i]);
            sB[i].add(dw * wv[i]);
            sC[i].add(dw);
        }
    }
}

// Index of a heavy row in the sorted heavy_rows list (binary search).
template <typename T>
__device__ __forceinline__ int heavy_index(const StepArgs<T>& a, int64_t row)
{
    int64_t lo = 0, hi = a.n_heavy_rows - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a.heavy_rows[mid] < row) lo = mid + 1; else hi = mid;
    }
    return (int)lo;
}

// Sum of the chunk partials [f, l) of a heavy row (chunk order, NZL lanes strided; up to four
// partials loaded before they are added, in the same order, as registers allow).
template <typename T, int VEC, int NZL>
__device__ __forceinline__ void heavy_chunks_sum(const StepArgs<T>& a, int f, int l, int64_t c0, int zl,
                                                 T (&acc)[VEC])
{
    constexpr int U = sizeof(T) * VEC <= 8 ? 4 : (sizeof(T) * VEC <= 16 ? 2 : 1);
    for (int c = f + zl; c < l; c += U * NZL) {
        T x[U][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c + u * NZL < l) ld_plain<T, VEC>(x[u], a.heavy_part + (int64_t)(c + u * NZL) * a.ld + c0);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c + u * NZL < l) {
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc[i] += x[u][i];
            }
    }
}

// Sum of the heavy row's chunk partials (chunk order, NZL lanes strided).
template <typename T, int VEC, int NZL>
__device__ __forceinline__ void heavy_row_sum(const StepArgs<T>& a, int64_t row, int64_t c0, int zl, T (&acc)[VEC])
{
    const int hi = heavy_index(a, row);
    heavy_chunks_sum<T, VEC, NZL>(a, a.heavy_first[hi], a.heavy_first[hi + 1], c0, zl, acc);
}

// Partial sums of each heavy-row chunk: heavy_part[chunk, :] = sum over the chunk's nonzeros.
template <typename T, int VEC, int GS, int NZL, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock) k_spmm_heavy(const StepArgs<T> a)
{
    constexpr int TP = VEC * GS;
    constexpr int RPW = 32 / (GS * NZL);
    if (step_inactive(a)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cl = lane % GS, zl = (lane / GS) % NZL;
    const int rs = lane / (GS * NZL);
    const int li = lane % (GS * NZL);
    const unsigned mask = group_mask<GS, NZL>(lane);
    const int64_t nslots = (int64_t)gridDim.x * kWarps * RPW;
    const int64_t slot0 = ((int64_t)blockIdx.x * kWarps + warp) * RPW + rs;
    const int nslab = (int)(a.ld / TP);
    for (int slab = 0; slab < nslab; ++slab) {
        const int64_t c0 = (int64_t)slab * TP + cl * VEC;
        for (int64_t ch = slot0; ch < a.n_chunks; ch += nslots) {
            T acc[VEC];
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[i] = T(0);
            gather_row<T, VEC, GS, NZL, kUnroll<T, VEC>, WEIGHTED>(a, (int64_t)a.chunk_beg[ch], (int64_t)a.chunk_end[ch],
                                                                  c0, li, zl, mask, acc);
            reduce_nzl<GS, NZL>(acc, mask);
            if (zl == 0) st_plain<T, VEC>(a.heavy_part + ch * a.ld + c0, acc);
        }
    }
}



// Per-thread accumulators of the three reductions kept in shared memory (column
// threadIdx.x of a [quantity][VEC][kBlock] array, bank-conflict free); FP32 sums are
// Kahan-compensated, FP64 sums plain. Used by the row-stream kernel to keep registers
// for gathers in flight.
template <typename T, int VEC>
struct SmemAcc;

template <int VEC>
struct SmemAcc<float, VEC> {
    static constexpr int kWords = 3 * VEC * 2;  // floats per thread
    float* p;
    __device__ __forceinline__ void init(float* base)
    {
        p = base + threadIdx.x;
#pragma unroll
        for (int k = 0; k < kWords; ++k) p[k * kBlock] = 0.f;
    }
    __device__ __forceinline__ void add(int q, int i, float x)
    {
        float* sp = p + ((q * VEC + i) * 2) * kBlock;
        float* cp = sp + kBlock;
        const float s = *sp, c = *cp;
        const float y = x - c;
        const float t = s + y;
        *cp = (t - s) - y;
        *sp = t;
    }
    __device__ __forceinline__ double value(int q, int i) const
    {
        const float* sp = p + ((q * VEC + i) * 2) * kBlock;
        return (double)sp[0] - (double)sp[kBlock];
    }
};

template <int VEC>
struct SmemAcc<double, VEC> {
    static constexpr int kWords = 3 * VEC * 2;  // 32-bit words per thread
    double* p;
    __device__ __forceinline__ void init(float* base)
    {
        p = reinterpret_cast<double*>(base) + threadIdx.x;
#pragma unroll
        for (int k = 0; k < 3 * VEC; ++k) p[k * kBlock] = 0.0;
    }
    __device__ __forceinline__ void add(int q, int i, double x) { p[(q * VEC + i) * kBlock] += x; }
    __device__ __forceinline__ double value(int q, int i) const { return p[(q * VEC + i) * kBlock]; }
};

template <int VEC>
struct SmemAcc<df64, VEC> {
    static constexpr int kWords = 3 * VEC * 2;  // 32-bit words per thread
    df64* p;
    __device__ __forceinline__ void init(float* base)
    {
        p = reinterpret_cast<df64*>(base) + threadIdx.x;
#pragma unroll
        for (int k = 0; k < 3 * VEC; ++k) p[k * kBlock] = df64(0);
    }
    __device__ __forceinline__ void add(int q, int i, df64 x) { p[(q * VEC + i) * kBlock] += x; }
    __device__ __forceinline__ double value(int q, int i) const { return (double)p[(q * VEC + i) * kBlock]; }
};

template <typename T, int VEC, int TP>
constexpr size_t rows_smem_bytes()
{
    return (size_t)SmemAcc<T, VEC>::kWords * 4 * kBlock + (size_t)kWarps * TP * 8;
}

// Block partials from shared-memory accumulators (same tree as block_partials).
template <typename T, int VEC, int GW, int TP>
__device__ __forceinline__ void block_partials_s(const StepArgs<T>& a, const SmemAcc<T, VEC>& acc,
                                                 double (*red)[TP], int slab, int lane, int warp, int cl)
{
#pragma unroll
    for (int qn = 0; qn < 3; ++qn) {
        double v[VEC];
#pragma unroll
        for (int i = 0; i < VEC; ++i) v[i] = acc.value(qn, i);
#pragma unroll
        for (int off = GW; off < 32; off <<= 1) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
        }
        if (lane < TP / VEC) {
#pragma unroll
            for (int i = 0; i < VEC; ++i) red[warp][cl * VEC + i] = v[i];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < TP; c += kBlock) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) sum += red[w][c];
            a.block_part[(((int64_t)slab * gridDim.x + blockIdx.x) * 3 + qn) * TP + c] = sum;
        }
        __syncthreads();
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void row_epilogue_s(const StepArgs<T>& a, int64_t row, int64_t c0, T invd, T du,
                                               const T (&acc)[VEC], const T (&bt)[VEC], const T (&qp)[VEC],
                                               const T (&qc)[VEC], SmemAcc<T, VEC>& sacc)
{
    T wv[VEC];
    if (a.lazy_walk) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) wv[i] = T(0.5) * (invd * acc[i]) + T(0.5) * qc[i];
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) wv[i] = invd * acc[i] - bt[i] * qp[i];
    }
    st_stream<T, VEC>(a.qprev_w + row * a.ld + c0, wv);
    if (a.do_reduce) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            const T dw = du * wv[i];
            sacc.add(0, i, dw * qc[i]);
            sacc.add(1, i, dw * wv[i]);
            sacc.add(2, i, dw);
        }
    }
}

#ifndef RD_ROWS_MINB
#define RD_ROWS_MINB 2
#endif
template <typename T, int VEC>
inline constexpr int kMinBlocks = RD_ROWS_MINB;

#ifndef RD_ROWS_PREFETCH
#define RD_ROWS_PREFETCH 1  // prefetch each chunk's gathered rows into L1 at the chunk start
#endif
#ifndef RD_ROWS_BATCH
#define RD_ROWS_BATCH 4     // rows whose terms are summed in registers before one Kahan update
#endif

// Row terms of the three reductions summed over a batch of rows in registers, then added
// to the Kahan accumulators in shared memory (one compensated update per batch).
template <typename T, int VEC>
struct RowBatch {
    T b[3][VEC];
    int cnt;
    __device__ __forceinline__ void reset()
    {
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int i = 0; i < VEC; ++i) b[q][i] = T(0);
        cnt = 0;
    }
    __device__ __forceinline__ void flush(SmemAcc<T, VEC>& acc)
    {
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc.add(q, i, b[q][i]);
        reset();
    }
};

template <typename T, int VEC>
__device__ __forceinline__ void row_epilogue_b(const StepArgs<T>& a, int row, int64_t c0, T invd, T du,
                                               const T (&acc)[VEC], const T (&bt)[VEC], const T (&qp)[VEC],
                                               const T (&qc)[VEC], RowBatch<T, VEC>& rb, SmemAcc<T, VEC>& sacc)
{
    T wv[VEC];
    if (a.lazy_walk) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) wv[i] = T(0.5) * (invd * acc[i]) + T(0.5) * qc[i];
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) wv[i] = invd * acc[i] - bt[i] * qp[i];
    }
    st_stream<T, VEC>(a.qprev_w + (int64_t)row * a.ld + c0, wv);
    if (a.do_reduce) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            const T dw = du * wv[i];
            rb.b[0][i] += dw * qc[i];
            rb.b[1][i] += dw * wv[i];
            rb.b[2][i] += dw;
        }
        if (++rb.cnt == RD_ROWS_BATCH) rb.flush(sacc);
    }
}

// One step: W = D^{-1} W_adj q_i - beta_i q_{i-1} written over q_{i-1}, plus block
// partial sums of sum_u d_u W q_i, sum_u d_u W^2 and sum_u d_u W per column.
// Blocks per SM the row-group kernel is compiled for. With narrow lanes (16 bytes) the
// Kahan accumulators of the three reductions live in shared memory (SmemAcc) instead of
// registers, which lets more warps be resident to keep gathers in flight.
#ifndef RD_GROUP_MINB
#define RD_GROUP_MINB 4
#endif
#ifndef RD_GROUP_SMEM
#define RD_GROUP_SMEM 1
#endif
template <typename T, int VEC>
inline constexpr bool kGroupSmemAcc = RD_GROUP_SMEM && (int)sizeof(T) * VEC <= 16;
template <typename T, int VEC>
inline constexpr int kGroupMinBlocks = kGroupSmemAcc<T, VEC> ? RD_GROUP_MINB : 1;


template <typename T, int VEC, int GS, int NZL, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock, kGroupMinBlocks<T, VEC>) k_spmm(const StepArgs<T> a)
{
    constexpr int TP = VEC * GS;
    constexpr int RPW = 32 / (GS * NZL);
    constexpr bool kSmem = kGroupSmemAcc<T, VEC>;
    __shared__ double red[kWarps][TP];
    __shared__ __align__(16) float sacc_buf[kSmem ? SmemAcc<T, VEC>::kWords * kBlock : 1];
    if (step_inactive(a)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cl = lane % GS, zl = (lane / GS) % NZL;
    const int rs = lane / (GS * NZL);
    const int li = lane % (GS * NZL);
    const unsigned mask = group_mask<GS, NZL>(lane);
    const int64_t nslots = (int64_t)gridDim.x * kWarps * RPW;
    const int64_t slot0 = ((int64_t)blockIdx.x * kWarps + warp) * RPW + rs;
    const int nslab = (int)(a.ld / TP);
    const int64_t ld = a.ld;

    for (int slab = 0; slab < nslab; ++slab) {
        const int64_t c0 = (int64_t)slab * TP + cl * VEC;
        T bt[VEC];
        ld_plain<T, VEC>(bt, step_cf_beta(a) + c0);
        Acc<T> sA[VEC], sB[VEC], sC[VEC];
        SmemAcc<T, VEC> sacc;
        if constexpr (kSmem) sacc.init(sacc_buf);

        for (int64_t i = slot0; i < a.n; i += nslots) {
            const int64_t row = a.row_order ? (int64_t)a.row_order[i] : i;
            const int64_t beg = a.row_ptr[row], end = a.row_ptr[row + 1];
            T acc[VEC], qp[VEC], qc[VEC];
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[i] = T(0);
            if (zl == 0) {  // own-row operands of the epilogue, issued before the gather
                ld_stream<T, VEC>(qp, a.qprev_w + row * ld + c0);
                ld_gather<T, VEC>(qc, a.qcur + row * ld + c0);
            }
            if (end - beg > a.heavy_thr) {
                heavy_row_sum<T, VEC, NZL>(a, row, c0, zl, acc);
            } else {
                gather_row<T, VEC, GS, NZL, kUnroll<T, VEC>, WEIGHTED>(a, beg, end, c0, li, zl, mask, acc);
            }
            reduce_nzl<GS, NZL>(acc, mask);
            if (zl == 0) {
                if constexpr (kSmem) row_epilogue_s<T, VEC>(a, row, c0, a.invdeg[row], a.deg[row], acc, bt, qp, qc, sacc);
                else row_epilogue<T, VEC>(a, row, c0, a.invdeg[row], a.deg[row], acc, bt, qp, qc, sA, sB, sC);
            }
        }

        if constexpr (kSmem) {
            if (a.do_reduce) block_partials_s<T, VEC, GS * NZL, TP>(a, sacc, red, slab, lane, warp, cl);
            __syncthreads();  // the accumulators are re-initialised by the next slab
        } else {
            if (a.do_reduce) block_partials<T, VEC, GS * NZL, TP>(a, sA, sB, sC, red, slab, lane, warp, cl);
        }
    }
}


__device__ __forceinline__ void prefetch_l1(const void* p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Row-stream variant: a row group of GS lanes (VEC columns each) walks a task -- a
// contiguous row range holding at most a fixed number of nonzeros, or one heavy row --
// as a single stream of nonzeros. Column indices come CH at a time in one coalesced
// load, each lane turning its index into a 32-bit offset (in VEC-element units) and
// optionally prefetching that row's slab into L1; U gathers per lane are in flight per
// round and stay in flight across row boundaries; row_ptr, 1/d and d of the task's rows
// are loaded GS rows at a time and broadcast by shuffle; the epilogue of a row runs
// when the stream crosses its end. Requires n * ld / VEC < 2^32.
template <typename T, int VEC, int GS, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock, kMinBlocks<T, VEC>) k_spmm_rows(const StepArgs<T> a)
{
    constexpr int TP = VEC * GS;
    constexpr int NG = 32 / GS;
    constexpr int U = kUnroll<T, VEC>;
    constexpr int CH = GS > U ? GS : U;  // indices per coalesced index load
    constexpr int NH = CH / GS;          // indices held per lane
    extern __shared__ __align__(16) float smem_f[];
    double(*red)[TP] = reinterpret_cast<double(*)[TP]>(smem_f + SmemAcc<T, VEC>::kWords * kBlock);
    if (step_inactive(a)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % GS, grp = lane / GS;
    const unsigned mask = group_mask<GS, 1>(lane);
    const int ngroups = gridDim.x * kWarps * NG;
    const int gid = (blockIdx.x * kWarps + warp) * NG + grp;
    const int nslab = (int)(a.ld / TP);
    const int64_t ld = a.ld;
    const uint32_t ldv = (uint32_t)(ld / VEC);  // row stride in VEC-element units
    const int ntasks = (int)a.ntasks;
#if RD_GATHER_HINT
    const uint64_t pol_hot = l2_policy_evict_last(), pol_cold = l2_policy_evict_first();
    const uint32_t hot_off = (uint32_t)(a.hot_rows < (int64_t)(0xffffffffu / (ldv ? ldv : 1)) ? a.hot_rows * ldv
                                                                                              : 0xffffffffu);
#endif

    for (int slab = 0; slab < nslab; ++slab) {
        const int64_t c0 = (int64_t)slab * TP + gl * VEC;
        T bt[VEC];
        ld_plain<T, VEC>(bt, step_cf_beta(a) + c0);
        SmemAcc<T, VEC> sacc;
        sacc.init(smem_f);
        RowBatch<T, VEC> rb;
        rb.reset();
        const T* __restrict__ q = a.qcur + c0;
        const T* __restrict__ qslab = a.qcur + (int64_t)slab * TP;  // row starts of this slab

        for (int task = gid; task < ntasks; task += ngroups) {
            const int r0 = a.task_row[task], r1 = a.task_row[task + 1];
            const int e_beg = (int)a.row_ptr[r0], e_end = (int)a.row_ptr[r1];
            T acc[VEC], qp[VEC], qc[VEC];
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[i] = T(0);
            if (r1 == r0 + 1 && e_end - e_beg > a.heavy_thr) {
                ld_stream<T, VEC>(qp, a.qprev_w + (int64_t)r0 * ld + c0);
                ld_gather<T, VEC>(qc, q + (int64_t)r0 * ld);
                heavy_row_sum<T, VEC, 1>(a, r0, c0, 0, acc);
                row_epilogue_b<T, VEC>(a, r0, c0, a.invdeg[r0], a.deg[r0], acc, bt, qp, qc, rb, sacc);
                continue;
            }
            // row window: lane gl holds row_ptr[w0 + gl + 1], 1/d and d of row w0 + gl
            int w0 = r0;
            int my_end = (w0 + gl < r1) ? (int)a.row_ptr[w0 + gl + 1] : e_end;
            T my_invd = (w0 + gl < r1) ? a.invdeg[w0 + gl] : T(0);
            T my_deg = (w0 + gl < r1) ? a.deg[w0 + gl] : T(0);
            int row = r0;
            int row_end = __shfl_sync(mask, my_end, 0, GS);
            ld_stream<T, VEC>(qp, a.qprev_w + (int64_t)row * ld + c0);
            ld_gather<T, VEC>(qc, q + (int64_t)row * ld);
            for (int base = e_beg; base < e_end; base += CH) {
                const int cnt = e_end - base < CH ? e_end - base : CH;
                uint32_t my_off[NH];
                float my_w[NH];
#pragma unroll
                for (int h = 0; h < NH; ++h) {
                    const int idx = h * GS + gl;
                    const uint32_t j = idx < cnt ? (uint32_t)__ldg(a.col + base + idx) : 0u;
                    my_off[h] = j * ldv;
                    if constexpr (WEIGHTED) my_w[h] = idx < cnt ? __ldg(a.w + base + idx) : 0.0f;
#if RD_ROWS_PREFETCH
                    if (idx < cnt) {
                        const char* rowp = reinterpret_cast<const char*>(qslab + (int64_t)j * ld);
#pragma unroll
                        for (int L = 0; L < (TP * (int)sizeof(T) + 127) / 128; ++L) prefetch_l1(rowp + 128 * L);
                    }
#endif
                }
                for (int k0 = 0; k0 < cnt; k0 += U) {
                    T x[U][VEC];
                    float wu[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        // k0 == 0 when GS < U; otherwise k0 + u < GS
                        const int kk = k0 + u;
                        const int hh = GS >= U ? 0 : u / (GS >= U ? 1 : GS);
                        const uint32_t off = __shfl_sync(mask, my_off[hh], kk % GS, GS);
                        if constexpr (WEIGHTED) wu[u] = __shfl_sync(mask, my_w[hh], kk % GS, GS);
                        if (kk < cnt) {
#if RD_GATHER_HINT
                            ld_gather_pol<T, VEC>(x[u], q + (size_t)off * VEC, off < hot_off ? pol_hot : pol_cold);
#else
                            ld_gather<T, VEC>(x[u], q + (size_t)off * VEC);
#endif
                        } else {
#pragma unroll
                            for (int i = 0; i < VEC; ++i) x[u][i] = T(0);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e = base + k0 + u;
                        if (e >= e_end) break;
                        while (e >= row_end) {  // the stream leaves `row`
                            const int wi = row - w0;
                            const T invd = shfl_t(mask, my_invd, wi, GS);
                            const T du = shfl_t(mask, my_deg, wi, GS);
#pragma unroll
                            for (int i = 0; i < VEC; ++i) acc_finish(acc[i]);
                            row_epilogue_b<T, VEC>(a, row, c0, invd, du, acc, bt, qp, qc, rb, sacc);
#pragma unroll
                            for (int i = 0; i < VEC; ++i) acc[i] = T(0);
                            ++row;
                            if (row - w0 >= GS) {  // refill the row window
                                w0 = row;
                                my_end = (w0 + gl < r1) ? (int)a.row_ptr[w0 + gl + 1] : e_end;
                                my_invd = (w0 + gl < r1) ? a.invdeg[w0 + gl] : T(0);
                                my_deg = (w0 + gl < r1) ? a.deg[w0 + gl] : T(0);
                            }
                            row_end = __shfl_sync(mask, my_end, row - w0, GS);
                            ld_stream<T, VEC>(qp, a.qprev_w + (int64_t)row * ld + c0);
                            ld_gather<T, VEC>(qc, q + (int64_t)row * ld);
                        }
                        if constexpr (WEIGHTED) {
#pragma unroll
                            for (int i = 0; i < VEC; ++i) acc_mul_add_w(acc[i], wu[u], x[u][i]);
                        } else {
#pragma unroll
                            for (int i = 0; i < VEC; ++i) acc_add(acc[i], x[u][i]);
                        }
                    }
                }
            }
            // last row of the task (and any rows without nonzeros after it)
            while (row < r1) {
                const int wi = row - w0;
                const T invd = shfl_t(mask, my_invd, wi, GS);
                const T du = shfl_t(mask, my_deg, wi, GS);
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc_finish(acc[i]);
                row_epilogue_b<T, VEC>(a, row, c0, invd, du, acc, bt, qp, qc, rb, sacc);
#pragma unroll
                for (int i = 0; i < VEC; ++i) acc[i] = T(0);
                ++row;
                if (row >= r1) break;
                if (row - w0 >= GS) {
                    w0 = row;
                    my_end = (w0 + gl < r1) ? (int)a.row_ptr[w0 + gl + 1] : e_end;
                    my_invd = (w0 + gl < r1) ? a.invdeg[w0 + gl] : T(0);
                    my_deg = (w0 + gl < r1) ? a.deg[w0 + gl] : T(0);
                }
                ld_stream<T, VEC>(qp, a.qprev_w + (int64_t)row * ld + c0);
                ld_gather<T, VEC>(qc, q + (int64_t)row * ld);
            }
        }
        if (a.do_reduce) {
            rb.flush(sacc);
            block_partials_s<T, VEC, GS, TP>(a, sacc, red, slab, lane, warp, gl);
        }
        __syncthreads();  // accumulators are re-initialised by the next slab
    }
}

// ----------------------------------------------------- async-copy row stream
// Row-stream SpMM whose gathers are per-lane 16-byte cp.async copies (the non-bulk form:
// each lane copies its own column segment of a gathered row) into a ring of D slots in
// shared memory. A lane keeps D gathers in flight without holding them in registers, so
// three blocks per SM (24 warps, about 190 KB of gathered rows in flight per SM) stay
// resident; the ring is refilled as each slot is consumed, so the gathers stay in flight
// across row and round boundaries. Row groups of GS lanes x VEC = 4 FP32 columns walk the
// same tasks as k_spmm_rows (runs of consecutive light rows, each heavy row alone with its
// chunk partials from the pre-pass k_spmm_async_heavy), one column slab of TP = 4 GS
// columns at a time. The three reductions use Kahan accumulators in registers.
//
// Ring protocol (per lane; cp.async groups are per thread): every consumption of a slot is
// followed by exactly one commit (of the refill copy, or of an empty group when there is
// nothing to refill), and the prologue of a nonzero range commits D groups, so before
// consuming a slot at most D groups are pending and wait_group(D - 1) completes the oldest,
// the one that filled this slot. A range ends with no copy in flight (refills are issued
// only for nonzeros inside the range), so ranges need no drain.
#ifndef RD_ASYNC_DEPTH
#define RD_ASYNC_DEPTH 24
#endif
#ifndef RD_ASYNC_MINB
#define RD_ASYNC_MINB 2
#endif
// rows ahead whose own-row operands q_{i-1}[row] and q_i[row] are prefetched into L2 (0: none)
#ifndef RD_ASYNC_PF_DIST
#define RD_ASYNC_PF_DIST 1
#endif
constexpr int kAsyncDepth = RD_ASYNC_DEPTH;  // gathers in flight per lane

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ float4 lds_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}

// elements of T in one 16-byte lane slot: 4 FP32, 2 FP64 or double-float
template <typename T>
inline constexpr int kAsyncVec = 16 / (int)sizeof(T);

template <typename T, int GS>
constexpr size_t async_smem_bytes()
{
    return (size_t)kWarps * kAsyncDepth * 32 * 16 + (size_t)kWarps * (kAsyncVec<T> * GS) * 8;
}

// Column indices (as row offsets in 16-byte units) and weights of the D nonzeros of one
// round starting at `base`: lane gl holds positions gl + h GS (h < NH) of the round.
template <int GS, bool WEIGHTED>
struct AsyncRound {
    static constexpr int NH = (kAsyncDepth + GS - 1) / GS;
    uint32_t off[NH];
    float w[NH];
    template <class Args>
    __device__ __forceinline__ void load(const Args& a, int base, int end, int gl, uint32_t ldv)
    {
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            const int pos = h * GS + gl;
            const bool ok = pos < kAsyncDepth && base + pos < end;
            off[h] = ok ? (uint32_t)__ldg(a.col + base + pos) * ldv : 0u;
            if constexpr (WEIGHTED) w[h] = ok ? __ldg(a.w + base + pos) : 0.0f;
        }
    }
    // value held for round position u by its owner lane (u / GS selects the register)
    __device__ __forceinline__ uint32_t off_at(int u) const
    {
        uint32_t v = off[0];
#pragma unroll
        for (int h = 1; h < NH; ++h)
            if (u >= h * GS) v = off[h];
        return v;
    }
    __device__ __forceinline__ float w_at(int u) const
    {
        float v = w[0];
#pragma unroll
        for (int h = 1; h < NH; ++h)
            if (u >= h * GS) v = w[h];
        return v;
    }
};

// acc += w * x (or acc += x unweighted) on the columns of a lane slot (16 bytes as read from
// the ring): four FP32, two FP64 or two double-float (each as hi, lo)
template <bool WEIGHTED>
__device__ __forceinline__ void acc_add_slot(double (&acc)[2], const float4& x, float wv)
{
    const double x0 = __hiloint2double(__float_as_int(x.y), __float_as_int(x.x));
    const double x1 = __hiloint2double(__float_as_int(x.w), __float_as_int(x.z));
    if constexpr (WEIGHTED) {
        acc[0] = fma((double)wv, x0, acc[0]);
        acc[1] = fma((double)wv, x1, acc[1]);
    } else {
        acc[0] += x0;
        acc[1] += x1;
    }
}
template <bool WEIGHTED>
__device__ __forceinline__ void acc_add_slot(df64 (&acc)[2], const float4& x, float wv)
{
    const df64 x0(x.x, x.y, 0), x1(x.z, x.w, 0);
    if constexpr (WEIGHTED) {
        acc_mul_add_w(acc[0], wv, x0);
        acc_mul_add_w(acc[1], wv, x1);
    } else {
        acc_add(acc[0], x0);
        acc_add(acc[1], x1);
    }
}
template <bool WEIGHTED>
__device__ __forceinline__ void acc_add_slot(float (&acc)[4], const float4& x, float wv)
{
    if constexpr (WEIGHTED) {
        acc[0] = fmaf(wv, x.x, acc[0]);
        acc[1] = fmaf(wv, x.y, acc[1]);
        acc[2] = fmaf(wv, x.z, acc[2]);
        acc[3] = fmaf(wv, x.w, acc[3]);
    } else {
        acc[0] += x.x;
        acc[1] += x.y;
        acc[2] += x.z;
        acc[3] += x.w;
    }
}

// Stream the nonzeros [eb, ee) of one row group through the ring: acc += w_e * q[col_e, slab].
// `enter(e)` runs before nonzero e is added when e may open a new row (it closes the rows
// that end there: row epilogues) and returns the end of the segment that e is in (the first
// nonzero of the next row); each segment is then consumed without a boundary test per nonzero.
template <typename T, int GS, bool WEIGHTED, class Enter>
__device__ __forceinline__ void async_stream(const StepArgs<T>& a, const T* q, uint32_t ldv, int eb, int ee,
                                             uint32_t ring, int gl, unsigned mask, T (&acc)[kAsyncVec<T>],
                                             Enter&& enter)
{
    constexpr int D = kAsyncDepth;
    constexpr uint32_t SS = 32 * 16;  // slot stride: one float4 per lane of the warp
    using R = AsyncRound<GS, WEIGHTED>;
    R cur, nxt, nn;
    cur.load(a, eb, ee, gl, ldv);
    nxt.load(a, eb + D, ee, gl, ldv);
    for (int u = 0; u < D; ++u) {
        const uint32_t o = __shfl_sync(mask, cur.off_at(u), u % GS, GS);
        if (eb + u < ee) cp_async16(ring + u * SS, reinterpret_cast<const char*>(q) + (size_t)o * 16);
        cp_async_commit();
    }
    for (int base = eb; base < ee; base += D) {
        nn.load(a, base + 2 * D, ee, gl, ldv);
        const int cnt = ee - base < D ? ee - base : D;
        const int refill = ee - D - base;  // slots u < refill are refilled from the next round
        auto consume = [&](int u) {
            float wv = 1.0f;
            if constexpr (WEIGHTED) wv = __shfl_sync(mask, cur.w_at(u), u % GS, GS);
            const uint32_t o = __shfl_sync(mask, nxt.off_at(u), u % GS, GS);
            cp_async_wait<D - 1>();
            const float4 x = lds_f4(ring + u * SS);
            acc_add_slot<WEIGHTED>(acc, x, wv);
            if (u < refill) cp_async16(ring + u * SS, reinterpret_cast<const char*>(q) + (size_t)o * 16);
            cp_async_commit();
        };
        for (int u = 0; u < cnt;) {
            const int se = enter(base + u) - base;
            const int stop = se < cnt ? se : cnt;
            for (; u < stop; ++u) consume(u);
        }
        cur = nxt;
        nxt = nn;
    }
}

// Heavy-row pre-pass of the async kernel: the chunk partials heavy_part[chunk, slab].
template <typename T, int GS, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock, RD_ASYNC_MINB) k_spmm_async_heavy(const StepArgs<T> a)
{
    constexpr int V = kAsyncVec<T>;
    constexpr int TP = V * GS;
    constexpr int NG = 32 / GS;
    extern __shared__ __align__(16) float smem_f[];
    if (step_inactive(a)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % GS, grp = lane / GS;
    const unsigned mask = group_mask<GS, 1>(lane);
    const uint32_t ring = smem_addr(smem_f) + (uint32_t)(warp * kAsyncDepth * 32 + lane) * 16u;
    const int64_t ngroups = (int64_t)gridDim.x * kWarps * NG;
    const int64_t gid = ((int64_t)blockIdx.x * kWarps + warp) * NG + grp;
    const int nslab = (int)(a.ld / TP);
    const uint32_t ldv = (uint32_t)(a.ld / V);
    for (int slab = 0; slab < nslab; ++slab) {
        const int64_t c0 = (int64_t)slab * TP + gl * V;
        const T* q = a.qcur + c0;
        for (int64_t ch = gid; ch < a.n_chunks; ch += ngroups) {
            T acc[V];
#pragma unroll
            for (int i = 0; i < V; ++i) acc[i] = T(0);
            async_stream<T, GS, WEIGHTED>(a, q, ldv, a.chunk_beg[ch], a.chunk_end[ch], ring, gl, mask, acc,
                                          [](int) { return INT_MAX; });
#pragma unroll
            for (int i = 0; i < V; ++i) acc_finish(acc[i]);
            st_plain<T, V>(a.heavy_part + ch * a.ld + c0, acc);
        }
    }
}

// Main kernel: W = D^{-1} W_adj q_i - beta_i q_{i-1} over q_{i-1}, and the block partials of
// sum d W q_i, sum d W^2, sum d W per column (slab by slab). Row groups take the tasks
// grid-strided; a task of light rows is one stream of nonzeros through the ring.
template <typename T, int GS, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock, RD_ASYNC_MINB) k_spmm_async(const StepArgs<T> a)
{
    constexpr int V = kAsyncVec<T>;
    constexpr int TP = V * GS;
    constexpr int NG = 32 / GS;
    constexpr int PD = RD_ASYNC_PF_DIST;
    extern __shared__ __align__(16) float smem_f[];
    double(&red)[kWarps][TP] = *reinterpret_cast<double(*)[kWarps][TP]>(smem_f + kWarps * kAsyncDepth * 32 * 4);
    if (step_inactive(a)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % GS, grp = lane / GS;
    const unsigned mask = group_mask<GS, 1>(lane);
    const uint32_t ring = smem_addr(smem_f) + (uint32_t)(warp * kAsyncDepth * 32 + lane) * 16u;
    const int ngroups = gridDim.x * kWarps * NG;
    const int gid = (blockIdx.x * kWarps + warp) * NG + grp;
    const int nslab = (int)(a.ld / TP);
    const int64_t ld = a.ld;
    const uint32_t ldv = (uint32_t)(ld / V);
    const int ntasks = (int)a.ntasks;

    for (int slab = 0; slab < nslab; ++slab) {
        const int64_t c0 = (int64_t)slab * TP + gl * V;
        T bt[V];
        ld_plain<T, V>(bt, step_cf_beta(a) + c0);
        Acc<T> sA[V], sB[V], sC[V];
        const T* q = a.qcur + c0;
        // a heavy row: the sum of its chunk partials [f, l)
        auto heavy_row = [&](int r, int f, int l) {
            T acc[V], qp[V], qc[V];
#pragma unroll
            for (int i = 0; i < V; ++i) acc[i] = T(0);
            ld_stream<T, V>(qp, a.qprev_w + (int64_t)r * ld + c0);
            ld_gather<T, V>(qc, q + (int64_t)r * ld);
            heavy_chunks_sum<T, V, 1>(a, f, l, c0, 0, acc);
            row_epilogue<T, V>(a, r, c0, a.invdeg[r], a.deg[r], acc, bt, qp, qc, sA, sB, sC);
        };
        // light rows [r0, r1): one stream of their nonzeros
        auto light_rows = [&](int r0, int r1) {
            const int eb = (int)a.row_ptr[r0], ee = (int)a.row_ptr[r1];
            T acc[V], qp[V], qc[V];
#pragma unroll
            for (int i = 0; i < V; ++i) acc[i] = T(0);
            // row window: lane gl holds row_ptr[w0 + gl + 1], 1/d and d of row w0 + gl
            int w0 = r0;
            int my_end = (w0 + gl < r1) ? (int)a.row_ptr[w0 + gl + 1] : ee;
            T my_invd = (w0 + gl < r1) ? a.invdeg[w0 + gl] : T(0);
            T my_deg = (w0 + gl < r1) ? a.deg[w0 + gl] : T(0);
            int row = r0;
            int row_end = __shfl_sync(mask, my_end, 0, GS);
            ld_stream<T, V>(qp, a.qprev_w + (int64_t)row * ld + c0);
            ld_gather<T, V>(qc, q + (int64_t)row * ld);
            // the own-row operands of the next PD rows into L2 (no registers held): short rows
            // end before a load from DRAM would return
#pragma unroll
            for (int d = 1; d <= PD; ++d)
                if (row + d < r1) {
                    prefetch_l2(a.qprev_w + (int64_t)(row + d) * ld + c0);
                    prefetch_l2(q + (int64_t)(row + d) * ld);
                }
            // close the current row and open the next one
            auto next_row = [&]() {
                const int wi = row - w0;
                const T invd = shfl_t(mask, my_invd, wi, GS);
                const T du = shfl_t(mask, my_deg, wi, GS);
#pragma unroll
                for (int i = 0; i < V; ++i) acc_finish(acc[i]);
                row_epilogue<T, V>(a, row, c0, invd, du, acc, bt, qp, qc, sA, sB, sC);
#pragma unroll
                for (int i = 0; i < V; ++i) acc[i] = T(0);
                ++row;
                if (row >= r1) return;
                if (row - w0 >= GS) {  // refill the row window
                    w0 = row;
                    my_end = (w0 + gl < r1) ? (int)a.row_ptr[w0 + gl + 1] : ee;
                    my_invd = (w0 + gl < r1) ? a.invdeg[w0 + gl] : T(0);
                    my_deg = (w0 + gl < r1) ? a.deg[w0 + gl] : T(0);
                }
                row_end = __shfl_sync(mask, my_end, row - w0, GS);
                ld_stream<T, V>(qp, a.qprev_w + (int64_t)row * ld + c0);
                ld_gather<T, V>(qc, q + (int64_t)row * ld);
                if (PD > 0 && row + PD < r1) {
                    prefetch_l2(a.qprev_w + (int64_t)(row + PD) * ld + c0);
                    prefetch_l2(q + (int64_t)(row + PD) * ld);
                }
            };
            async_stream<T, GS, WEIGHTED>(a, q, ldv, eb, ee, ring, gl, mask, acc, [&](int e) {
                while (e >= row_end) next_row();
                return row_end;
            });
            while (row < r1) next_row();  // the last row (and any rows without nonzeros after it)
        };
        for (int task = gid; task < ntasks; task += ngroups) {
            const int r0 = a.task_row[task], r1 = a.task_row[task + 1];
            if (r1 == r0 + 1 && a.row_ptr[r1] - a.row_ptr[r0] > a.heavy_thr) {
                const int hi = heavy_index(a, r0);
                heavy_row(r0, a.heavy_first[hi], a.heavy_first[hi + 1]);
                continue;
            }
            light_rows(r0, r1);
        }
        if (a.do_reduce) block_partials<T, V, GS, TP>(a, sA, sB, sC, red, slab, lane, warp, gl);
    }
}

template <typename T, int GS>
void async_smem_attr()
{
    constexpr size_t sm = async_smem_bytes<T, GS>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_spmm_async<T, GS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_spmm_async<T, GS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_spmm_async_heavy<T, GS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_spmm_async_heavy<T, GS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
}

template <typename T, int GS>
bool launch_async_cfg(bool weighted, bool heavy, int grid, cudaStream_t st, const StepArgs<T>& a)
{
    constexpr size_t sm = async_smem_bytes<T, GS>();
    async_smem_attr<T, GS>();
    if (heavy) {
        if (weighted) k_spmm_async_heavy<T, GS, true><<<grid, kBlock, sm, st>>>(a);
        else k_spmm_async_heavy<T, GS, false><<<grid, kBlock, sm, st>>>(a);
    } else {
        if (weighted) k_spmm_async<T, GS, true><<<grid, kBlock, sm, st>>>(a);
        else k_spmm_async<T, GS, false><<<grid, kBlock, sm, st>>>(a);
    }
    return true;
}

template <typename T, int GS>
int occupancy_async_cfg(bool weighted, bool heavy)
{
    int nb = 0;
    constexpr size_t sm = async_smem_bytes<T, GS>();
    async_smem_attr<T, GS>();
    if (heavy) {
        if (weighted) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_async_heavy<T, GS, true>, kBlock, sm);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_async_heavy<T, GS, false>, kBlock, sm);
    } else {
        if (weighted) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_async<T, GS, true>, kBlock, sm);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_async<T, GS, false>, kBlock, sm);
    }
    return nb;
}

// Single-column SpMV (one pair per launch, ld = 1). One warp per task (consecutive rows
// with at most kTaskNnz nonzeros, or one heavy row): the lanes stride over the task's
// nonzeros with coalesced index loads and 8 gathers in flight per lane, leaving the
// products w_e q[col_e] in the warp's slice of shared memory; then each lane sums whole
// rows from shared memory and runs the row epilogue. No block-wide barriers.
constexpr int kTaskNnz = 512;

template <typename T, bool WEIGHTED>
__global__ void __launch_bounds__(kBlock) k_spmv_tasks(const StepArgs<T> a)
{
    __shared__ T prod[kWarps][kTaskNnz];
    __shared__ double red[kWarps][1];
    if (step_inactive(a)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = gridDim.x * kWarps;
    const int ntasks = (int)a.ntasks;
    const T bt = step_cf_beta(a)[0];
    Acc<T> sA, sB, sC;
    T* pw = prod[warp];
    for (int task = blockIdx.x * kWarps + warp; task < ntasks; task += nwarps) {
        const int r0 = a.task_row[task], r1 = a.task_row[task + 1];
        const int64_t e0 = a.row_ptr[r0], e1 = a.row_ptr[r1];
        if (r1 == r0 + 1 && e1 - e0 > a.heavy_thr) {
            // heavy row: sum of its chunk partials (chunk order within each lane, then a tree)
            T acc[1] = {T(0)};
            heavy_row_sum<T, 1, 32>(a, r0, 0, lane, acc);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc[0] += shfl_xor_t(0xffffffffu, acc[0], off);
            if (lane == 0) {
                T qp[1], qc[1], bt1[1] = {bt};
                qp[0] = a.qprev_w[r0];
                qc[0] = a.qcur[r0];
                Acc<T> tA[1] = {sA}, tB[1] = {sB}, tC[1] = {sC};
                row_epilogue<T, 1>(a, r0, 0, a.invdeg[r0], a.deg[r0], acc, bt1, qp, qc, tA, tB, tC);
                sA = tA[0];
                sB = tB[0];
                sC = tC[0];
            }
            continue;
        }
        const int cnt = (int)(e1 - e0);
        // operands of each lane's first row in phase 2, loaded now so that their latency
        // overlaps the gathers of phase 1
        const int rf = r0 + lane;
        int fb0 = 0, fb1 = 0;
        T fqp = T(0), fqc = T(0), finvd = T(0), fdu = T(0);
        if (rf < r1) {
            fb0 = (int)(a.row_ptr[rf] - e0);
            fb1 = (int)(a.row_ptr[rf + 1] - e0);
            fqp = a.qprev_w[rf];
            fqc = a.qcur[rf];
            finvd = a.invdeg[rf];
            fdu = a.deg[rf];
        }
        // phase 1: products into shared memory
        for (int k0 = 0; k0 < cnt; k0 += 32 * 8) {
            T x[8];
            int idx[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                idx[u] = k0 + u * 32 + lane;
                x[u] = T(0);
                if (idx[u] < cnt) {
                    const int64_t j = __ldg(a.col + e0 + idx[u]);
                    T xv[1];
                    ld_gather<T, 1>(xv, a.qcur + j);
                    x[u] = xv[0];
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (idx[u] < cnt) {
                    if constexpr (WEIGHTED) pw[idx[u]] = (T)__ldg(a.w + e0 + idx[u]) * x[u];
                    else pw[idx[u]] = x[u];
                }
            }
        }
        __syncwarp();
        // phase 2: one lane per row
        for (int r = rf; r < r1; r += 32) {
            const bool first = r == rf;
            const int b0 = first ? fb0 : (int)(a.row_ptr[r] - e0);
            const int b1 = first ? fb1 : (int)(a.row_ptr[r + 1] - e0);
            T sum = T(0);
            for (int k = b0; k < b1; ++k) sum += pw[k];
            T acc[1] = {sum}, qp[1], qc[1], bt1[1] = {bt};
            qp[0] = first ? fqp : a.qprev_w[r];
            qc[0] = first ? fqc : a.qcur[r];
            const T invd = first ? finvd : a.invdeg[r];
            const T du = first ? fdu : a.deg[r];
            Acc<T> tA[1] = {sA}, tB[1] = {sB}, tC[1] = {sC};
            row_epilogue<T, 1>(a, r, 0, invd, du, acc, bt1, qp, qc, tA, tB, tC);
            sA = tA[0];
            sB = tB[0];
            sC = tC[0];
        }
        __syncwarp();
    }
    if (a.do_reduce) {
        Acc<T> vA[1] = {sA}, vB[1] = {sB}, vC[1] = {sC};
        block_partials<T, 1, 1, 1>(a, vA, vB, vC, red, 0, lane, warp, 0);
    }
}

template <typename T>
bool launch_spmv_tasks(bool weighted, int grid, cudaStream_t st, const StepArgs<T>& a)
{
    if (weighted) k_spmv_tasks<T, true><<<grid, kBlock, 0, st>>>(a);
    else k_spmv_tasks<T, false><<<grid, kBlock, 0, st>>>(a);
    return true;
}

template <typename T>
int occupancy_spmv_tasks(bool weighted)
{
    int nb = 0;
    if (weighted) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_tasks<T, true>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmv_tasks<T, false>, kBlock, 0);
    return nb;
}

// Dynamic shared-memory limit of the row-stream kernels, set once per instantiation (from
// the occupancy query of planning, i.e. before any launch or stream capture uses it).
template <typename T, int VEC, int GS>
void rows_smem_attr()
{
    constexpr size_t sm = rows_smem_bytes<T, VEC, VEC * GS>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_spmm_rows<T, VEC, GS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_spmm_rows<T, VEC, GS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
}

template <typename T, int VEC, int GS>
bool launch_rows_cfg(bool weighted, int grid, cudaStream_t st, const StepArgs<T>& a)
{
    constexpr size_t sm = rows_smem_bytes<T, VEC, VEC * GS>();
    rows_smem_attr<T, VEC, GS>();
    if (weighted) k_spmm_rows<T, VEC, GS, true><<<grid, kBlock, sm, st>>>(a);
    else k_spmm_rows<T, VEC, GS, false><<<grid, kBlock, sm, st>>>(a);
    return true;
}

template <typename T, int VEC, int GS>
int occupancy_rows_cfg(bool weighted)
{
    int nb = 0;
    constexpr size_t sm = rows_smem_bytes<T, VEC, VEC * GS>();
    rows_smem_attr<T, VEC, GS>();
    if (weighted) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_rows<T, VEC, GS, true>, kBlock, sm);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_rows<T, VEC, GS, false>, kBlock, sm);
    return nb;
}

template <typename T, int VEC, int GS, int NZL>
bool launch_cfg(bool weighted, bool heavy, int grid, cudaStream_t st, const StepArgs<T>& a)
{
    if (heavy) {
        if (weighted) k_spmm_heavy<T, VEC, GS, NZL, true><<<grid, kBlock, 0, st>>>(a);
        else k_spmm_heavy<T, VEC, GS, NZL, false><<<grid, kBlock, 0, st>>>(a);
    } else {
        if (weighted) k_spmm<T, VEC, GS, NZL, true><<<grid, kBlock, 0, st>>>(a);
        else k_spmm<T, VEC, GS, NZL, false><<<grid, kBlock, 0, st>>>(a);
    }
    return true;
}

template <typename T, int VEC, int GS, int NZL>
int occupancy_cfg(bool weighted, bool heavy)
{
    int nb = 0;
    if (heavy) {
        if (weighted) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_heavy<T, VEC, GS, NZL, true>, kBlock, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm_heavy<T, VEC, GS, NZL, false>, kBlock, 0);
    } else {
        if (weighted) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm<T, VEC, GS, NZL, true>, kBlock, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spmm<T, VEC, GS, NZL, false>, kBlock, 0);
    }
    return nb;
}

}  // namespace rd

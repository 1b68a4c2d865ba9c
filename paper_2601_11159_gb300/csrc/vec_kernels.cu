// Per-step vector and per-pair scalar kernels of the batched Lanczos iteration:
// start vector (Algorithm 3), FP64 finalisation of alpha/beta with an O(1)-per-step
// LDL^T update of I - T_k (the quadratic form of Section 3), normalisation
// v_{i+1} = w / beta_{i+1} (Algorithm 3), output, the tridiagonal solve for the
// potential of Algorithm 5 and the edge-weight gradient.
#include <math.h>

#include <cooperative_groups.h>

#include "spmm.cuh"

namespace rd {

// ----------------------------------------------------------------- start
// q_1 = D^{-1/2} v_1 with v_1 = (e_s/sqrt(d_s) - e_t/sqrt(d_t)) / ||b||, so
// q_1[s] = 1/(d_s ||b||), q_1[t] = -1/(d_t ||b||); ||b||^2 = 1/d_s + 1/d_t.
template <typename T>
__global__ void k_init(const InitArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npairs) return;
    const PairState& st = a.st;
    const int32_t s = a.s[p], t = a.t[p];
    if (a.replay) {
        if (st.status[p] == RD_OK || st.status[p] == RD_WARN_NOT_CONVERGED) {
            if (s != t && st.b2[p] > 0.0) {
                const double ds = a.deg64[s], dt = a.deg64[t];
                const double bn = sqrt(1.0 / ds + 1.0 / dt);
                T* q = static_cast<T*>(a.qcur);
                q[(int64_t)s * a.ld + p] = (T)(1.0 / (ds * bn));
                q[(int64_t)t * a.ld + p] = (T)(-1.0 / (dt * bn));
            }
        }
        return;
    }
    if (s < 0 || (int64_t)s >= a.n || t < 0 || (int64_t)t >= a.n) {
        atomicOr(a.err_flag, 1);
        st.status[p] = RD_ERR_INVALID_ARG;
        st.r[p] = NAN;
        return;
    }
    if (s == t) {
        st.status[p] = RD_OK;
        st.r[p] = 0.0;
        st.err[p] = 0.0;
        return;
    }
    if (a.comp && a.comp[s] != a.comp[t]) {
        st.status[p] = RD_ERR_DISCONNECTED;
        st.r[p] = INFINITY;
        return;
    }
    const double ds = a.deg64[s], dt = a.deg64[t];
    const double b2 = 1.0 / ds + 1.0 / dt;
    const double bn = sqrt(b2);
    T* q = static_cast<T*>(a.qcur);
    q[(int64_t)s * a.ld + p] = (T)(1.0 / (ds * bn));
    q[(int64_t)t * a.ld + p] = (T)(-1.0 / (dt * bn));
    st.b2[p] = b2;
    st.err[p] = 1.0;
    st.resid[p] = 1.0;
    st.status[p] = RD_OK;
    st.active[p] = 1;
    atomicAdd(&st.act_count[0], 1);
}

void launch_init(cudaStream_t st, const InitArgs& a)
{
    const int nb = (a.npairs + 127) / 128;
    if (a.df) k_init<df64><<<nb, 128, 0, st>>>(a);
    else if (a.elem_size == 8) k_init<double><<<nb, 128, 0, st>>>(a);
    else k_init<float><<<nb, 128, 0, st>>>(a);
}

// -------------------------------------------------------------- finalise
// Column p: reduce the SpMM block partials in block order, then
//   alpha_i = <w, v_i>, beta_{i+1}^2 = ||w||^2 - alpha_i^2 - gamma^2 (gamma: component along
//   D^{1/2}1, removed when deflating), and update the LDL^T factorisation of J_i = I - T_i:
//   delta_1 = 1 - alpha_1,  delta_i = (1 - alpha_i) - beta_i^2 / delta_{i-1}
//   g_1 = 1,                g_i = beta_i g_{i-1} / delta_{i-1}        (g = L^{-1} e_1)
//   S_i = S_{i-1} + g_i^2 / delta_i = e_1^T J_i^{-1} e_1,   r_i = ||b||^2 S_i
//   residual ||b - (I - Ahat) x_i|| / ||b|| = beta_{i+1} |g_i / delta_i|.
// Step i = j + 1 of pair p from the three reduced sums A = <w, v_i>, B = ||w||^2 and
// C = <w, D^{1/2}1> of w = Ahat v_i - beta_i v_{i-1}:
//   alpha_i = A, beta_{i+1}^2 = B - A^2 - C^2/sum(d) (deflated component removed),
//   LDL^T of J_i = I - T_i: delta_1 = 1 - alpha_1, delta_i = (1 - alpha_i) - beta_i^2/delta_{i-1},
//   g_1 = 1, g_i = beta_i g_{i-1}/delta_{i-1}, S_i = S_{i-1} + g_i^2/delta_i, r_i = ||b||^2 S_i,
//   residual ||b - (I - Ahat) x_i||/||b|| = beta_{i+1} |g_i/delta_i|.
// Writes the pair's state and history; returns true when the pair stops (then active = 0),
// else leaves alpha_i, the deflation constant c_i and beta_{i+1} in the outputs.
// The per-pair scalars of the update (a register copy of one pair's PairState entries).
struct PairScalars {
    double b2, delta, g, S, beta;  // beta: beta_i of the step being reduced
    double inv_delta;              // 1 / delta (0 before the first step)
    double r0, r1, r2, r3;         // increments of S: slot j % kRing holds step j's
    // slot access by a run-time index through selects, so that the scalars stay in registers
    // (an indexed array would live in local memory)
    __device__ __forceinline__ double ring(int q) const { return q == 0 ? r0 : (q == 1 ? r1 : (q == 2 ? r2 : r3)); }
    __device__ __forceinline__ void set_ring(int q, double v)
    {
        r0 = q == 0 ? v : r0;
        r1 = q == 1 ? v : r1;
        r2 = q == 2 ? v : r2;
        r3 = q == 3 ? v : r3;
    }
};
static_assert(kRing == 4, "PairScalars holds four ring slots");

// What one step produced (the values pair_update stores).
struct PairStepOut {
    bool ok;                       // false: a value was not finite or I - T_i lost definiteness
    bool warn_not_converged;       // k_max reached before a tolerance was met
    double alpha, cdef, beta_next, incr, r, resid, est;
};

__device__ __forceinline__ PairScalars pair_load(const PairState& st, int p, int64_t np)
{
    PairScalars s;
    s.b2 = st.b2[p];
    s.delta = st.delta[p];
    s.g = st.g[p];
    s.S = st.S[p];
    s.beta = st.beta[p];
    s.inv_delta = s.delta != 0.0 ? 1.0 / s.delta : 0.0;
    s.r0 = st.ring[p];
    s.r1 = st.ring[np + p];
    s.r2 = st.ring[2 * np + p];
    s.r3 = st.ring[3 * np + p];
    return s;
}

// The arithmetic of one step on the scalars (see pair_update); returns true when the pair
// stops. The state in `s` is advanced exactly as pair_update advances the stored state.
// FP64 division and square root are slow on this part (hundreds of cycles each, one thread
// at a time on the whole-recurrence kernels' critical path), so the step takes four divisions
// and one square root: 1/delta_{i-1} is kept from the previous step, 1/sum(d) is passed in,
// 1/delta_i and 1/S_i serve every quotient by them, and the largest increment ratio is found
// by cross-multiplication (increments are positive) before its one division.
__device__ __forceinline__ bool pair_core(const FinArgs& a, PairScalars& s, int j, double A, double B, double C,
                                          PairStepOut& o)
{
    const double alpha = A;
    const double beta_i = s.beta;
    const double cdef = a.deflate ? C * a.inv_sumdeg : 0.0;
    const double gamma2 = a.deflate ? C * cdef : 0.0;
    const double beta2 = B - alpha * alpha - gamma2;
    double delta, g;
    if (j == 0) {
        delta = 1.0 - alpha;
        g = 1.0;
    } else {
        const double idp = s.inv_delta;
        delta = (1.0 - alpha) - beta_i * beta_i * idp;
        g = s.g * beta_i * idp;
    }
    bool stop = false;
    o.ok = isfinite(alpha) && isfinite(beta2) && isfinite(delta) && delta > 0.0;
    o.warn_not_converged = false;
    o.alpha = alpha;
    o.cdef = cdef;
    o.beta_next = 0.0;
    if (!o.ok) return true;  // frozen at its last good estimate
    const double inv_delta = 1.0 / delta;
    const double gd = g * inv_delta;
    const double incr = g * gd;
    const double S = s.S + incr;
    s.S = S;
    o.incr = incr;
    o.r = s.b2 * S;
    s.set_ring(j % kRing, incr);
    const double beta_next = sqrt(fmax(beta2, 0.0));
    o.beta_next = beta_next;
    const double resid = beta_next * fabs(gd);
    o.resid = resid;
    s.delta = delta;
    s.inv_delta = inv_delta;
    s.g = g;
    const double brk = a.fp64 ? 1e-12 : 1e-6;
    const bool breakdown = beta_next <= brk * (fabs(alpha) + beta_i);  // T_i is exact
    stop = breakdown || (!a.fixed_k && a.resid_tol > 0.0 && resid <= a.resid_tol);
    // Relative error estimate of r_k = b2 * S_k: the increments still to come. Default:
    // their sum as a series whose ratio is the largest of the last kRing-1 increment
    // ratios (at least 1/2), with an extra margin 1/(1 - rho) for slowly converging
    // pairs: incr * rho / (1 - rho)^2. Alternative (est_delayed): the sum of the last
    // kRing increments, i.e. the error of the estimate kRing steps back. Without a rel_tol
    // test it only feeds the output, so it is formed on the step that ends the pair.
    const bool use_est = !a.fixed_k && a.rel_tol > 0.0;
    double est = 0.0;
    if (!breakdown && (use_est || stop || j + 1 >= a.k_max)) {
        const double inv_S = 1.0 / S;
        double tail = 0.0;
        const int nr = j + 1 < kRing ? j + 1 : kRing;
        for (int q = 0; q < nr; ++q) tail += s.ring(q);
        est = tail * inv_S;
        if (!a.est_delayed && j + 1 >= kRing) {
            // the largest num/den over the last kRing-1 pairs of consecutive increments
            double bn = s.ring(j % kRing), bd = s.ring((j - 1) % kRing);
            for (int q = 2; q < kRing; ++q) {
                const double num = s.ring((j - q + 1) % kRing);
                const double den = s.ring((j - q) % kRing);
                if (num * bd > bn * den) {
                    bn = num;
                    bd = den;
                }
            }
            const double rho = fmax(0.5, bn / bd);
            const double om = 1.0 - rho;
            est = rho < 1.0 ? incr * rho * inv_S / (om * om) : INFINITY;
        }
        if (!stop && use_est && j + 1 >= kRing && est <= a.rel_tol) stop = true;
    }
    o.est = est;
    if (!stop && j + 1 >= a.k_max) {
        stop = true;
        o.warn_not_converged = !a.fixed_k;
    }
    if (!stop) s.beta = beta_next;
    return stop;
}

// Store one step's results of pair p (the history, the running factorisation, the status).
__device__ __forceinline__ void pair_store(const PairState& st, int p, int j, int64_t np, const PairScalars& s,
                                           const PairStepOut& o, bool stop)
{
    if (!o.ok) {
        st.status[p] = RD_ERR_NUMERIC;
    } else {
        st.S[p] = s.S;
        st.r[p] = o.r;
        st.ring[(int64_t)(j % kRing) * np + p] = o.incr;
        st.resid[p] = o.resid;
        st.err[p] = o.est;
        st.hist_alpha[(int64_t)j * np + p] = o.alpha;
        st.hist_beta[(int64_t)(j + 1) * np + p] = o.beta_next;
        st.k[p] = j + 1;
        st.delta[p] = s.delta;
        st.g[p] = s.g;
        if (o.warn_not_converged) st.status[p] = RD_WARN_NOT_CONVERGED;
    }
    if (stop) st.active[p] = 0;
    else st.beta[p] = s.beta;
}

__device__ __forceinline__ bool pair_update(const FinArgs& a, const PairState& st, int p, int j, double A, double B,
                                            double C, double* alpha_o, double* cdef_o, double* beta_next_o)
{
    PairScalars s = pair_load(st, p, a.pstride);
    PairStepOut o;
    const bool stop = pair_core(a, s, j, A, B, C, o);
    pair_store(st, p, j, a.pstride, s, o, stop);
    if (stop) return true;
    *alpha_o = o.alpha;
    *cdef_o = o.cdef;
    *beta_next_o = o.beta_next;
    return false;
}

// Columns per finalize block: 32, or the next power of two >= ld for narrower tiles, so
// that the remaining threads of the block split the sum over the SpMM blocks.
__host__ __device__ inline int fin_cols_per_block(int64_t ld)
{
    int cb = 1;
    while (cb < ld && cb < 32) cb <<= 1;
    return cb;
}

template <typename T>
__global__ void __launch_bounds__(256) k_finalize(const FinArgs a)
{
    __shared__ double part[3][256];
    const int cb = fin_cols_per_block(a.ld);
    const int nsplit = 256 / cb;
    const int lane = threadIdx.x & (cb - 1), split = threadIdx.x / cb;
    const int64_t col = (int64_t)blockIdx.x * cb + lane;
    const PairState& st = a.st;
    const int j = a.step_dev ? *a.step_dev : a.step;  // 0-based step index; Lanczos step i = j + 1
    if (st.act_count[j] == 0) return;
    // block partials b = split, split + nsplit, ...: four rows of loads in flight, summed
    // in block order (the order depends only on nblocks and ld, so runs are repeatable)
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (col < a.ld) {
        const int64_t slab = col / a.tp, cin = col % a.tp;
        const double* base = a.block_part + slab * a.nblocks * 3 * a.tp + cin;
        const int64_t bstride = 3 * (int64_t)a.tp;
        int b = split;
        for (; b + 3 * nsplit < a.nblocks; b += 4 * nsplit) {
            double x[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double* bp = base + (int64_t)(b + u * nsplit) * bstride;
                x[u][0] = bp[0];
                x[u][1] = bp[a.tp];
                x[u][2] = bp[2 * a.tp];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s0 += x[u][0];
                s1 += x[u][1];
                s2 += x[u][2];
            }
        }
        for (; b < a.nblocks; b += nsplit) {
            const double* bp = base + (int64_t)b * bstride;
            s0 += bp[0];
            s1 += bp[a.tp];
            s2 += bp[2 * a.tp];
        }
    }
    part[0][threadIdx.x] = s0;
    part[1][threadIdx.x] = s1;
    part[2][threadIdx.x] = s2;
    __syncthreads();
    // fixed-order tree over the splits
    for (int h = nsplit >> 1; h >= 1; h >>= 1) {
        if (split < h) {
            part[0][threadIdx.x] += part[0][threadIdx.x + h * cb];
            part[1][threadIdx.x] += part[1][threadIdx.x + h * cb];
            part[2][threadIdx.x] += part[2][threadIdx.x + h * cb];
        }
        __syncthreads();
    }
    if (split != 0 || col >= a.ld) return;
    const int p = a.slot_pair ? a.slot_pair[col] : (col < a.npairs ? (int)col : -1);
    if (p < 0 || !st.active[p]) return;
    const double A = part[0][lane], B = part[1][lane], C = part[2][lane];
    const int64_t ld = a.ld;
    const int64_t cfo = a.step_dev ? (int64_t)j * a.cf_stride : 0;
    T* cfs = static_cast<T*>(a.cf_step) + cfo;
    T* cfn = static_cast<T*>(a.cf_next) + cfo;
    // factors of the previous step, for the potential's direct update below
    const double lam = j > 0 ? st.beta[p] / st.delta[p] : 0.0;
    double alpha, cdef, beta_next;
    const bool stop = pair_update(a, st, p, j, A, B, C, &alpha, &cdef, &beta_next);
    if (a.xcf && st.status[p] != RD_ERR_NUMERIC) {
        // p_i = q_i + lambda_i p_{i-1}, x += mu_i p_i (a stopping step still contributes)
        T* xc = static_cast<T*>(a.xcf) + (int64_t)j * 2 * ld;
        xc[col] = (T)lam;
        xc[ld + col] = (T)(sqrt(st.b2[p]) * st.g[p] / st.delta[p]);
    }
    if (stop) {
        // zero coefficients: the column's vectors become (and stay) zero
        cfs[1 * ld + col] = T(0);
        cfs[2 * ld + col] = T(0);
        cfs[3 * ld + col] = T(0);
        cfn[col] = T(0);
        return;
    }
    cfs[1 * ld + col] = (T)alpha;
    cfs[2 * ld + col] = (T)cdef;
    cfs[3 * ld + col] = (T)(1.0 / beta_next);
    cfn[col] = (T)beta_next;
    atomicAdd(&st.act_count[j + 1], 1);
}

void launch_finalize(cudaStream_t st, const FinArgs& a)
{
    const int cb = fin_cols_per_block(a.ld);
    const int nb = (int)((a.ld + cb - 1) / cb);
    if (a.df) k_finalize<df64><<<nb, 256, 0, st>>>(a);
    else if (a.elem_size == 8) k_finalize<double><<<nb, 256, 0, st>>>(a);
    else k_finalize<float><<<nb, 256, 0, st>>>(a);
}

// ------------------------------------------------------------- normalise
// One element of q_{i+1} = (W - alpha_i q_i - c_i) * (1/beta_{i+1}); every normalise kernel
// forms it this way, so that the packed form (k_normalize_pack) equals the plain one bit for bit.
template <typename T>
__device__ __forceinline__ T lanczos_next(T w, T al, T qc, T c, T ib)
{
    return (w - al * qc - c) * ib;
}
template <>
__device__ __forceinline__ float lanczos_next<float>(float w, float al, float qc, float c, float ib)
{
    return __fmul_rn(__fsub_rn(__fmaf_rn(-al, qc, w), c), ib);
}
template <>
__device__ __forceinline__ double lanczos_next<double>(double w, double al, double qc, double c, double ib)
{
    return __dmul_rn(__dsub_rn(__fma_rn(-al, qc, w), c), ib);
}

// q_{i+1} = (W - alpha_i q_i - c_i) / beta_{i+1}, written over W; optionally
// phi += coef * q_i for the replay pass. 16-byte units; ld == 1 handled separately.
template <typename T, bool LD1>
__global__ void __launch_bounds__(256) k_normalize(const NormArgs<T> a)
{
    const int32_t* act = a.step_dev ? a.act_count + *a.step_dev : a.active_prev;
    if (act && *act == 0) return;
    const T* cfb = a.step_dev ? a.cf + (int64_t)(*a.step_dev) * a.cf_stride : a.cf;
    constexpr int V = 16 / (int)sizeof(T);
    const int64_t total = a.n * a.ld;
    const int64_t units = total / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t ld = a.ld;
    const T* cf_al = cfb + ld;
    const T* cf_c = cfb + 2 * ld;
    const T* cf_ib = cfb + 3 * ld;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const int64_t e0 = u * V;
        T w[V], qc[V], qn[V];
        ld_stream<T, V>(w, a.w_to_qnext + e0);
        ld_stream<T, V>(qc, a.qcur + e0);
        if constexpr (LD1) {
            const T al = cf_al[0], c = cf_c[0], ib = cf_ib[0];
#pragma unroll
            for (int i = 0; i < V; ++i) qn[i] = lanczos_next<T>(w[i], al, qc[i], c, ib);
            if (a.phi) {
                const T cf = a.coef[0];
                T ph[V];
                ld_plain<T, V>(ph, a.phi + e0);
#pragma unroll
                for (int i = 0; i < V; ++i) ph[i] += cf * qc[i];
                st_plain<T, V>(a.phi + e0, ph);
            }
        } else {
            const int64_t c0 = e0 % ld;
            T al[V], c[V], ib[V];
            ld_plain<T, V>(al, cf_al + c0);
            ld_plain<T, V>(c, cf_c + c0);
            ld_plain<T, V>(ib, cf_ib + c0);
#pragma unroll
            for (int i = 0; i < V; ++i) qn[i] = lanczos_next<T>(w[i], al[i], qc[i], c[i], ib[i]);
            if (a.phi) {
                T cf[V], ph[V];
                ld_plain<T, V>(cf, a.coef + c0);
                ld_plain<T, V>(ph, a.phi + e0);
#pragma unroll
                for (int i = 0; i < V; ++i) ph[i] += cf[i] * qc[i];
                st_plain<T, V>(a.phi + e0, ph);
            }
        }
        st_plain<T, V>(a.w_to_qnext + e0, qn);
    }
    if constexpr (LD1) {
        // scalar tail (ld == 1 and n not a multiple of V)
        const int64_t t0 = units * V;
        for (int64_t e = t0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
            const T w = a.w_to_qnext[e], qc = a.qcur[e];
            a.w_to_qnext[e] = lanczos_next<T>(w, cf_al[0], qc, cf_c[0], cf_ib[0]);
            if (a.phi) a.phi[e] += a.coef[0] * qc;
        }
    }
}

// q_{i+1} as k_normalize, with the potential of each pair accumulated on the fly: the direct
// form of the Lanczos solve (D-Lanczos, Saad, Iterative Methods for Sparse Linear Systems,
// Section 6.7.1). With I - T_i = L D L^T (unit lower bidiagonal L, L[i][i-1] = -beta_i/delta_{i-1};
// D = diag(delta)) and g = L^{-1} e_1, the vectors P = Q L^{-T} obey p_i = q_i + lambda_i p_{i-1},
// lambda_i = beta_i/delta_{i-1}, and x_i = ||b|| Q_i (I - T_i)^{-1} e_1 = x_{i-1} + mu_i p_i with
// mu_i = ||b|| g_i/delta_i: after the last step x is the potential of the replay pass
// (sum_j ||b|| z_j q_j, z = (I - T_k)^{-1} e_1), without a second pass over the steps.
template <typename T, bool VECD>
__global__ void __launch_bounds__(256) k_normalize_pot(const NormArgs<T> a)
{
    const int32_t* act = a.step_dev ? a.act_count + *a.step_dev : a.active_prev;
    if (act && *act == 0) return;
    const int64_t j = a.step_dev ? *a.step_dev : 0;
    const int64_t ld = a.ld;
    const T* cfb = a.cf + j * a.cf_stride;
    const T* xcb = a.xcf + j * a.xcf_stride;
    const T* cf_al = cfb + ld;
    const T* cf_c = cfb + 2 * ld;
    const T* cf_ib = cfb + 3 * ld;
    const T* cf_lam = xcb;
    const T* cf_mu = xcb + ld;
    constexpr int V = VECD ? 16 / (int)sizeof(T) : 1;
    const int64_t units = a.n * ld / V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const int64_t e0 = u * V, c0 = e0 % ld;
        T w[V], qc[V], pv[V], xv[V], al[V], c[V], ib[V], lam[V], mu[V];
        ld_stream<T, V>(w, a.w_to_qnext + e0);
        ld_stream<T, V>(qc, a.qcur + e0);
        ld_plain<T, V>(pv, a.pvec + e0);
        ld_plain<T, V>(xv, a.xvec + e0);
        ld_plain<T, V>(al, cf_al + c0);
        ld_plain<T, V>(c, cf_c + c0);
        ld_plain<T, V>(ib, cf_ib + c0);
        ld_plain<T, V>(lam, cf_lam + c0);
        ld_plain<T, V>(mu, cf_mu + c0);
        T qn[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            qn[i] = lanczos_next<T>(w[i], al[i], qc[i], c[i], ib[i]);
            pv[i] = qc[i] + lam[i] * pv[i];
            xv[i] += mu[i] * pv[i];
        }
        st_plain<T, V>(a.pvec + e0, pv);
        st_plain<T, V>(a.xvec + e0, xv);
        st_plain<T, V>(a.w_to_qnext + e0, qn);
    }
}

template <typename T>
static void launch_norm(int grid, cudaStream_t st, const NormArgs<T>& a)
{
    constexpr int V = 16 / (int)sizeof(T);
    if (a.pvec) {
        if (a.ld % V == 0) k_normalize_pot<T, true><<<grid, 256, 0, st>>>(a);
        else k_normalize_pot<T, false><<<grid, 256, 0, st>>>(a);
    } else if (a.ld == 1) {
        k_normalize<T, true><<<grid, 256, 0, st>>>(a);
    } else {
        k_normalize<T, false><<<grid, 256, 0, st>>>(a);
    }
}

__global__ void k_step_advance(int32_t* step, int limit)
{
    if (*step < limit) *step += 1;
}

void launch_step_advance(cudaStream_t st, int32_t* step, int limit) { k_step_advance<<<1, 1, 0, st>>>(step, limit); }

// Conditions of the device-resident step loop (a conditional while node of a CUDA graph).
// Before step j (j steps done): go on while pairs are active, k_max is not reached and no
// column compaction is due. After step j's finalize: stop when a compaction is due before step
// j + 1 (and step j + 1 is to run), leaving step j's normalise pass to the host, which runs it
// fused with the packing. The compaction test reads the count `lag` steps back (active pairs
// fit in half the width), as rd_query's host polls do, so that both pack the columns at the
// same step; it is skipped before step *compact_from (the host moves that past a step where it
// packed, or found no narrower layout). To stop, record j, the count the test read, the count
// entering the next step, and where the loop stopped in saved[0..3] (one read for the host),
// and move the step index to the sentinel k_max + 1, whose active count is always 0, so that
// the remaining kernels of the loop body return at once; an index at the sentinel stays there.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, int32_t* step, const int32_t* act_count, int32_t* saved,
                            const int32_t* compact_from, int k_max, int64_t ld, int compact_check, int lag,
                            int after_finalize)
{
    const int j = *step;
    if (j > k_max) {
        cudaGraphSetConditional(h, 0);
        return;
    }
    const int jn = j + after_finalize;  // the step the test is for
    const int act = act_count[jn];
    const bool compact_due = compact_check && jn >= lag + 1 && jn >= *compact_from && ld > 16 &&
                             (int64_t)act_count[jn - lag] * 2 <= ld;
    bool stop;
    if (after_finalize) {
        stop = compact_due && act > 0 && jn < k_max;  // otherwise the next condition decides
    } else {
        stop = act == 0 || j >= k_max || compact_due;
    }
    if (stop) {
        saved[0] = j;
        saved[1] = act_count[jn >= lag ? jn - lag : 0];
        saved[2] = act;
        saved[3] = after_finalize;
        *step = k_max + 1;
        cudaGraphSetConditional(h, 0);
    } else if (!after_finalize) {
        cudaGraphSetConditional(h, 1);
    }
}

void launch_loop_cond(cudaStream_t st, cudaGraphConditionalHandle h, int32_t* step, const int32_t* act_count,
                      int32_t* saved, const int32_t* compact_from, int k_max, int64_t ld, int compact_check, int lag,
                      int after_finalize)
{
    k_loop_cond<<<1, 1, 0, st>>>(h, step, act_count, saved, compact_from, k_max, ld, compact_check, lag,
                                 after_finalize);
}

// ------------------------------------------------------- sparse first step
// q_1 is nonzero only in rows s and t of its column, so the first product
// W = D^{-1} A q_1 (Algorithm 3 with q_0 = 0) is nonzero only on the rows adjacent to s or
// t. One block per column: with L the endpoint of larger degree and S the other,
//   pass 1, rows u in N(L):  W_u <- w_{uL} q_1[L]                       (partial row sum)
//   pass 2, rows u in N(S):  u in N(L) (binary search in the sorted row L):
//                              W_u <- W_u + w_{uS} q_1[S]                (still unscaled)
//                            otherwise W_u <- (1/d_u) w_{uS} q_1[S]      (final)
//   pass 3, rows u in N(L):  W_u <- (1/d_u) W_u                           (final)
// and the column's sums A = sum d W q_1, B = sum d W^2, C = sum d W are taken in FP64 as one
// block partial. Needs rows strictly increasing in column and symmetric entries (row u
// holds L and S with the weights rows L and S hold u), so that these are the SpMM's rows.
template <typename T>
__device__ __forceinline__ void step0_term(T& acc, const float* w, int64_t e, T q)
{
    if (w) acc_mul_add_w(acc, __ldg(w + e), q);
    else acc_add(acc, q);
}

template <typename T>
__global__ void __launch_bounds__(256) k_step0_sparse(const Step0Args<T> a)
{
    __shared__ double red[8][3];
    const int p = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t s = a.s[p], t = a.t[p];
    bool live = s >= 0 && (int64_t)s < a.n && t >= 0 && (int64_t)t < a.n && s != t;
    T q1s = T(0), q1t = T(0);
    if (live) {
        q1s = a.q1[(int64_t)s * a.ld + p];
        q1t = a.q1[(int64_t)t * a.ld + p];
        live = to_double(q1s) != 0.0 || to_double(q1t) != 0.0;
    }
    double* out = a.block_part ? a.block_part + (int64_t)(p / a.tp) * 3 * a.tp + p % a.tp : nullptr;
    if (!live) {  // uniform over the block: the column stays zero
        if (threadIdx.x == 0 && out) out[0] = out[a.tp] = out[2 * a.tp] = 0.0;
        return;
    }
    const int64_t ds_n = a.row_ptr[s + 1] - a.row_ptr[s], dt_n = a.row_ptr[t + 1] - a.row_ptr[t];
    const bool s_large = ds_n >= dt_n;
    const int32_t L = s_large ? s : t, S = s_large ? t : s;
    const T q1L = s_large ? q1s : q1t, q1S = s_large ? q1t : q1s;
    const int64_t lb = a.row_ptr[L], le = a.row_ptr[L + 1];
    const int64_t sb = a.row_ptr[S], se = a.row_ptr[S + 1];
    const int64_t ld = a.ld;
    double sA = 0.0, sB = 0.0, sC = 0.0;
    auto add_sums = [&](int32_t u, T W) {
        const double d = a.deg64[u], x = to_double(W);
        sB += d * x * x;
        sC += d * x;
        if (u == s) sA += d * x * to_double(q1s);
        else if (u == t) sA += d * x * to_double(q1t);
    };
    for (int64_t e = lb + threadIdx.x; e < le; e += blockDim.x) {
        const int32_t u = __ldg(a.col + e);
        T acc = T(0);
        step0_term(acc, a.w, e, q1L);
        acc_finish(acc);
        a.wout[(int64_t)u * ld + p] = acc;
    }
    __syncthreads();
    for (int64_t e = sb + threadIdx.x; e < se; e += blockDim.x) {
        const int32_t u = __ldg(a.col + e);
        int64_t lo = lb, hi = le;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(a.col + mid) < u) lo = mid + 1; else hi = mid;
        }
        T* wp = a.wout + (int64_t)u * ld + p;
        if (lo < le && __ldg(a.col + lo) == u) {
            T acc = *wp;
            step0_term(acc, a.w, e, q1S);
            acc_finish(acc);
            *wp = acc;
        } else {
            T acc = T(0);
            step0_term(acc, a.w, e, q1S);
            acc_finish(acc);
            const T W = a.invdeg[u] * acc;
            *wp = W;
            add_sums(u, W);
        }
    }
    __syncthreads();
    for (int64_t e = lb + threadIdx.x; e < le; e += blockDim.x) {
        const int32_t u = __ldg(a.col + e);
        T* wp = a.wout + (int64_t)u * ld + p;
        const T W = a.invdeg[u] * *wp;
        *wp = W;
        add_sums(u, W);
    }
    if (!out) return;
    // fixed-order reduction: xor tree within each warp, then warps in order
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        sA += __shfl_xor_sync(0xffffffffu, sA, off);
        sB += __shfl_xor_sync(0xffffffffu, sB, off);
        sC += __shfl_xor_sync(0xffffffffu, sC, off);
    }
    if (lane == 0) {
        red[warp][0] = sA;
        red[warp][1] = sB;
        red[warp][2] = sC;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
        out[threadIdx.x * a.tp] = v;
    }
}

template <typename T>
static void launch_step0(cudaStream_t st, const Step0Args<T>& a)
{
    if (a.npairs > 0) k_step0_sparse<T><<<a.npairs, 256, 0, st>>>(a);
}
// Step 0's normalise pass after the sparse first step, first part. W_1 is nonzero only on
// N(s) ∪ N(t) and q_1 only on {s, t}; elsewhere q_2 = (W_1 - alpha_1 q_1 - c_1) / beta_2 is the
// same value in every row of a column (left to the fill). One CTA per column updates each row
// of that union once, in place, with k_normalize's arithmetic, and marks its entry in the
// mask: N(L) of the endpoint of larger degree, then N(S) minus N(L) (binary search in the
// sorted row L), then s and t unless they are adjacent (then each is in the other's row).
// Columns whose first step wrote nothing (as k_step0_sparse decides) are left to the fill.
template <typename T>
__global__ void __launch_bounds__(256) k_normalize_step0(const Step0NormArgs<T> a)
{
    const int p = blockIdx.x;
    const int32_t s = a.s[p], t = a.t[p];
    const int64_t ld = a.ld;
    bool live = s >= 0 && (int64_t)s < a.n && t >= 0 && (int64_t)t < a.n && s != t;
    if (live)
        live = to_double(a.q1[(int64_t)s * ld + p]) != 0.0 || to_double(a.q1[(int64_t)t * ld + p]) != 0.0;
    if (!live) return;  // uniform over the block
    const T al = a.cf[ld + p], c = a.cf[2 * ld + p], ib = a.cf[3 * ld + p];
    // w_zero: a row the first step did not write (s or t when they are not adjacent: their
    // W_1 entries are zero, and the block holds no zeros there)
    auto upd = [&](int32_t u, bool w_zero) {
        const int64_t e = (int64_t)u * ld + p;
        a.w[e] = lanczos_next<T>(w_zero ? T(0) : a.w[e], al, a.q1[e], c, ib);
        atomicOr(a.mask + (e >> 5), 1u << (e & 31));
    };
    const int64_t ds_n = a.row_ptr[s + 1] - a.row_ptr[s], dt_n = a.row_ptr[t + 1] - a.row_ptr[t];
    const int32_t L = ds_n >= dt_n ? s : t, S = ds_n >= dt_n ? t : s;
    const int64_t lb = a.row_ptr[L], le = a.row_ptr[L + 1];
    const int64_t sb = a.row_ptr[S], se = a.row_ptr[S + 1];
    auto in_row_L = [&](int32_t u) {
        int64_t lo = lb, hi = le;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(a.col + mid) < u) lo = mid + 1; else hi = mid;
        }
        return lo < le && __ldg(a.col + lo) == u;
    };
    for (int64_t e = lb + threadIdx.x; e < le; e += blockDim.x) upd(__ldg(a.col + e), false);
    for (int64_t e = sb + threadIdx.x; e < se; e += blockDim.x) {
        const int32_t u = __ldg(a.col + e);
        if (!in_row_L(u)) upd(u, false);
    }
    if (threadIdx.x == 0 && !in_row_L(S)) {
        upd(s, true);
        upd(t, true);
    }
}

// Second part: every entry the first part did not mark gets (0 - alpha_1 * 0 - c_1) / beta_2
// formed as k_normalize forms it from the zeros of W_1 and q_1 there, without reading the
// block (it holds no zeros there: the sparse first step leaves it unwritten). Thread t keeps
// one 16-byte column unit (its values in registers) and walks the rows t / units,
// + rows_per_pass, ...; a unit with marked entries is written element by element around them.
template <typename T>
__global__ void __launch_bounds__(256) k_normalize_step0_fill(const Step0NormArgs<T> a)
{
    constexpr int V = 16 / (int)sizeof(T);
    const int64_t ld = a.ld;
    const int64_t units = ld / V;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rows_per_pass = (int64_t)gridDim.x * blockDim.x / units;
    const int64_t r0 = t / units;
    if (r0 >= rows_per_pass) return;
    const int64_t c0 = (t % units) * V;
    T v[V];
#pragma unroll
    for (int i = 0; i < V; ++i)
        v[i] = lanczos_next<T>(T(0), a.cf[ld + c0 + i], T(0), a.cf[2 * ld + c0 + i], a.cf[3 * ld + c0 + i]);
    for (int64_t u = r0; u < a.n; u += rows_per_pass) {
        const int64_t e0 = u * ld + c0;
        const uint32_t bits = (a.mask[e0 >> 5] >> (e0 & 31)) & ((1u << V) - 1u);
        if (bits == 0) {
            st_plain<T, V>(a.w + e0, v);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (!((bits >> i) & 1u)) a.w[e0 + i] = v[i];
        }
    }
}

template <typename T>
static void launch_norm0(int grid, cudaStream_t st, const Step0NormArgs<T>& a)
{
    if (a.npairs > 0) k_normalize_step0<T><<<a.npairs, 256, 0, st>>>(a);
    // at least one row per pass (the host takes this path only for whole 16-byte units)
    const int64_t units = a.ld / (16 / (int64_t)sizeof(T));
    const int g = (int)std::max<int64_t>(grid, (units + 255) / 256);
    k_normalize_step0_fill<T><<<g, 256, 0, st>>>(a);
}
void launch_normalize_step0_f32(int grid, cudaStream_t st, const Step0NormArgs<float>& a)
{
    launch_norm0<float>(grid, st, a);
}
void launch_normalize_step0_f64(int grid, cudaStream_t st, const Step0NormArgs<double>& a)
{
    launch_norm0<double>(grid, st, a);
}
void launch_normalize_step0_df64(int grid, cudaStream_t st, const Step0NormArgs<df64>& a)
{
    launch_norm0<df64>(grid, st, a);
}

void launch_step0_f32(cudaStream_t st, const Step0Args<float>& a) { launch_step0<float>(st, a); }
void launch_step0_f64(cudaStream_t st, const Step0Args<double>& a) { launch_step0<double>(st, a); }
void launch_step0_df64(cudaStream_t st, const Step0Args<df64>& a) { launch_step0<df64>(st, a); }

void launch_normalize_f32(int grid, cudaStream_t st, const NormArgs<float>& a) { launch_norm<float>(grid, st, a); }
void launch_normalize_f64(int grid, cudaStream_t st, const NormArgs<double>& a) { launch_norm<double>(grid, st, a); }
void launch_normalize_df64(int grid, cudaStream_t st, const NormArgs<df64>& a) { launch_norm<df64>(grid, st, a); }

// The normalise pass of the step after which the active columns are packed (a column
// compaction), fused with the packing: new column d takes old column o = old_slot[d] (-1:
// zero), and both q_{i+1} (formed from W, q_i and the step's coefficients as k_normalize
// forms it) and q_i are written in the packed layout. One read of W and q_i and one write of
// each packed block, against a normalise pass plus a packing pass that reads both full blocks
// again. Thread t keeps one 16-byte column unit (its slots and coefficients in registers)
// and walks the rows t / units, + rows_per_pass, ...
template <typename T>
__global__ void __launch_bounds__(256) k_normalize_pack(const NormPackArgs<T> a)
{
    constexpr int V = 16 / (int)sizeof(T);
    const int64_t units = a.ld_new / V;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rows_per_pass = (int64_t)gridDim.x * blockDim.x / units;
    const int64_t r0 = t / units;
    if (r0 >= rows_per_pass) return;
    const int64_t cu = t % units;
    int o[V];
    T al[V], c[V], ib[V];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        o[i] = a.old_slot[cu * V + i];
        const int os = o[i] >= 0 ? o[i] : 0;
        al[i] = a.cf[a.ld_old + os];
        c[i] = a.cf[2 * a.ld_old + os];
        ib[i] = a.cf[3 * a.ld_old + os];
    }
    for (int64_t u = r0; u < a.n; u += rows_per_pass) {
        const T* wr = a.w + u * a.ld_old;
        const T* qr = a.qcur + u * a.ld_old;
        T qn[V], qc[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            if (o[i] >= 0) {
                qc[i] = qr[o[i]];
                qn[i] = lanczos_next<T>(wr[o[i]], al[i], qc[i], c[i], ib[i]);
            } else {
                qc[i] = T(0);
                qn[i] = T(0);
            }
        }
        st_plain<T, V>(a.qnext_new + u * a.ld_new + cu * V, qn);
        st_plain<T, V>(a.qcur_new + u * a.ld_new + cu * V, qc);
    }
}

template <typename T>
static bool launch_npack(int grid, cudaStream_t st, const NormPackArgs<T>& a)
{
    constexpr int64_t V = 16 / (int64_t)sizeof(T);
    if (a.ld_new % V != 0 || (int64_t)grid * 256 < a.ld_new / V) return false;
    k_normalize_pack<T><<<grid, 256, 0, st>>>(a);
    return true;
}
bool launch_normalize_pack_f32(int grid, cudaStream_t st, const NormPackArgs<float>& a) { return launch_npack(grid, st, a); }
bool launch_normalize_pack_f64(int grid, cudaStream_t st, const NormPackArgs<double>& a) { return launch_npack(grid, st, a); }
bool launch_normalize_pack_df64(int grid, cudaStream_t st, const NormPackArgs<df64>& a) { return launch_npack(grid, st, a); }

// Double-float copy of an FP64 array (degrees and their inverses for RD_MODE_DF64).
__global__ void k_split_df(int64_t n, const double* __restrict__ src, df64* __restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = df64(src[i]);
}

void launch_split_df(cudaStream_t st, int grid, int64_t n, const double* src, df64* dst)
{
    k_split_df<<<grid, 256, 0, st>>>(n, src, dst);
}

// ---------------------------------------------------------------- output
__global__ void k_output(const OutArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npairs) return;
    const PairState& st = a.st;
    const int status = st.status[p];
    a.r_out[p] = st.r[p];
    if (a.iters_out) a.iters_out[p] = st.k[p];
    if (a.err_out) a.err_out[p] = st.err[p];
    if (a.status_out) a.status_out[p] = status;
    if (status == RD_WARN_NOT_CONVERGED) atomicOr(&a.summary[0], 1);
    if (status == RD_ERR_NUMERIC) atomicOr(&a.summary[1], 1);
}

void launch_output(cudaStream_t st, const OutArgs& a)
{
    k_output<<<(a.npairs + 127) / 128, 128, 0, st>>>(a);
}

// ---------------------------------------------------- tridiagonal solve
// z = (I - T_k)^{-1} e_1 per pair from the stored alpha_1..alpha_k, beta_2..beta_k by
// forward elimination and back substitution (I - T_k is SPD, so no pivoting);
// coef_j = ||b|| z_j is the weight of q_j in the potential
// phi = ||b|| D^{-1/2} V_k z (the potential of Algorithm 5). Also writes gbar[p], the upstream
// gradient of pair p (0 for pairs without a finite result and for padding columns).
template <typename T>
__global__ void k_zsolve(const ZsolveArgs a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.ld) return;
    T* coef = static_cast<T*>(a.coef_hist);
    T* gbar = static_cast<T*>(a.gbar);
    const PairState& st = a.st;
    const int64_t ld = a.ld;
    const int status = p < a.npairs ? st.status[p] : RD_ERR_INVALID_ARG;
    const int k = p < a.npairs ? st.k[p] : 0;
    const bool use = (status == RD_OK || status == RD_WARN_NOT_CONVERGED) && k > 0;
    if (!use) {
        for (int j = 0; j < a.k_max; ++j) coef[(int64_t)j * ld + p] = T(0);
        gbar[p] = T(0);
        return;
    }
    gbar[p] = (T)(a.grad_r ? a.grad_r[p] : 1.0);
    double* zs = a.zscratch;  // [k_max][2][ld]: c'_j, d'_j
    const double* al = st.hist_alpha;
    const double* be = st.hist_beta;  // be[j*ld + p] = beta_{j+1}
    double cprev = 0.0, dprev = 0.0;
    for (int j = 0; j < k; ++j) {
        const double lower = j > 0 ? -be[(int64_t)j * ld + p] : 0.0;
        const double m = (1.0 - al[(int64_t)j * ld + p]) - lower * cprev;
        const double c = (j + 1 < k) ? -be[(int64_t)(j + 1) * ld + p] / m : 0.0;
        const double d = ((j == 0 ? 1.0 : 0.0) - lower * dprev) / m;
        zs[((int64_t)j * 2) * ld + p] = c;
        zs[((int64_t)j * 2 + 1) * ld + p] = d;
        cprev = c;
        dprev = d;
    }
    const double bn = sqrt(st.b2[p]);
    double x = 0.0;
    for (int j = k - 1; j >= 0; --j) {
        x = zs[((int64_t)j * 2 + 1) * ld + p] - zs[((int64_t)j * 2) * ld + p] * x;
        coef[(int64_t)j * ld + p] = (T)(bn * x);
    }
    for (int j = k; j < a.k_max; ++j) coef[(int64_t)j * ld + p] = T(0);
}

void launch_zsolve(cudaStream_t st, const ZsolveArgs& a)
{
    const int nb = (int)((a.ld + 127) / 128);
    if (a.elem_size == 8) k_zsolve<double><<<nb, 128, 0, st>>>(a);
    else k_zsolve<float><<<nb, 128, 0, st>>>(a);
}

// ---------------------------------------------------------- edge gradient
// grad[e] = -1/2 sum_p gbar_p (phi_p(u) - phi_p(v))^2 for stored entry e = (u -> v).
// Entries are processed in CSR order, kU consecutive entries per row group of GS lanes
// (VEC*GS columns per column chunk), so the gathers of kU entries are in flight at once;
// the row of each entry comes from the graph's entry-row array.
template <typename T, int VEC, int GS>
__global__ void __launch_bounds__(256) k_edge_grad(const EdgeGradArgs<T> a)
{
    constexpr int TP = VEC * GS;
    constexpr int NG = 32 / GS;
    constexpr int kU = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cl = lane % GS, grp = lane / GS;
    const unsigned mask = group_mask<GS, 1>(lane);
    const int64_t ngroups = (int64_t)gridDim.x * (blockDim.x / 32) * NG;
    const int64_t gid = ((int64_t)blockIdx.x * (blockDim.x / 32) + warp) * NG + grp;
    const int nch = (int)(a.ld / TP);
    for (int64_t e0 = gid * kU; e0 < a.nnz; e0 += ngroups * kU) {
        int64_t u[kU], v[kU];
        float s[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const bool ok = e0 + k < a.nnz;
            u[k] = ok ? (int64_t)__ldg(a.entry_row + e0 + k) : 0;
            v[k] = ok ? (int64_t)__ldg(a.col + e0 + k) : 0;
            s[k] = 0.f;
        }
        for (int ch = 0; ch < nch; ++ch) {
            const int64_t c0 = (int64_t)ch * TP + cl * VEC;
            T gb[VEC], pu[kU][VEC], pv[kU][VEC];
            ld_gather<T, VEC>(gb, a.gbar + c0);
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                ld_gather<T, VEC>(pu[k], a.phi + u[k] * a.ld + c0);
                ld_gather<T, VEC>(pv[k], a.phi + v[k] * a.ld + c0);
            }
#pragma unroll
            for (int k = 0; k < kU; ++k)
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    const T d = pu[k][i] - pv[k][i];
                    s[k] += (float)(gb[i] * d * d);
                }
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) {
#pragma unroll
            for (int off = 1; off < GS; off <<= 1) s[k] += __shfl_xor_sync(mask, s[k], off);
            if (cl == 0 && e0 + k < a.nnz) a.grad_out[e0 + k] = -0.5f * s[k];
        }
    }
}

template <typename T>
static void launch_eg(int grid, cudaStream_t st, const EdgeGradArgs<T>& a)
{
    constexpr int VEC = 16 / (int)sizeof(T);
    const int64_t units = a.ld / VEC;  // ld is a multiple of VEC here
    if (units % 32 == 0) k_edge_grad<T, VEC, 32><<<grid, 256, 0, st>>>(a);
    else if (units % 16 == 0) k_edge_grad<T, VEC, 16><<<grid, 256, 0, st>>>(a);
    else if (units % 8 == 0) k_edge_grad<T, VEC, 8><<<grid, 256, 0, st>>>(a);
    else if (units % 4 == 0) k_edge_grad<T, VEC, 4><<<grid, 256, 0, st>>>(a);
    else if (units % 2 == 0) k_edge_grad<T, VEC, 2><<<grid, 256, 0, st>>>(a);
    else k_edge_grad<T, VEC, 1><<<grid, 256, 0, st>>>(a);
}

// Row of every stored entry (one warp per row, lanes strided over the row's entries).
__global__ void __launch_bounds__(256) k_entry_rows(int64_t n, const int64_t* row_ptr, int32_t* entry_row)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); r < n; r += nw)
        for (int64_t e = row_ptr[r] + lane; e < row_ptr[r + 1]; e += 32) entry_row[e] = (int32_t)r;
}

void launch_entry_rows(int grid, cudaStream_t st, int64_t n, const int64_t* row_ptr, int32_t* entry_row)
{
    k_entry_rows<<<grid, 256, 0, st>>>(n, row_ptr, entry_row);
}

void launch_edge_grad_f32(int grid, cudaStream_t st, const EdgeGradArgs<float>& a) { launch_eg<float>(grid, st, a); }
void launch_edge_grad_f64(int grid, cudaStream_t st, const EdgeGradArgs<double>& a) { launch_eg<double>(grid, st, a); }

// --------------------------------------------------------------- compaction
// Slot map of the still-active pairs, in slot order (one block, chunked block scan), and
// the coefficients of the next step moved to the new slots.
template <typename T>
__global__ void __launch_bounds__(1024) k_compact_map(const CompactArgs a)
{
    __shared__ int warp_tot[32];
    __shared__ int base_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < a.ld_old; c0 += blockDim.x) {
        const int64_t slot = c0 + tid;
        int p = -1;
        if (slot < a.ld_old) p = a.slot_pair_old ? a.slot_pair_old[slot] : (slot < a.npairs ? (int)slot : -1);
        const int keep = (p >= 0 && a.active[p]) ? 1 : 0;
        // block-wide exclusive scan of keep
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int in_warp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int i = 0; i < w; ++i) before += warp_tot[i];
        int chunk_total = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) chunk_total += warp_tot[i];
        const int dst = base_s + before + in_warp;
        if (keep && dst < a.ld_new) {
            a.slot_pair_new[dst] = p;
            a.old_slot[dst] = (int)slot;
        }
        __syncthreads();
        if (tid == 0) base_s += chunk_total;
        __syncthreads();
    }
    const int kept = base_s;
    const T* cfo = static_cast<const T*>(a.cf_old);
    T* cfn = static_cast<T*>(a.cf_new);
    for (int64_t d = tid; d < a.ld_new; d += blockDim.x) {
        if (d >= kept) {
            a.slot_pair_new[d] = -1;
            a.old_slot[d] = -1;
        }
    }
    __syncthreads();
    for (int64_t d = tid; d < a.ld_new; d += blockDim.x) {
        const int o = a.old_slot[d];
#pragma unroll
        for (int q = 0; q < 4; ++q) cfn[q * a.ld_new + d] = o >= 0 ? cfo[q * a.ld_old + o] : T(0);
    }
}

// q blocks copied column-wise into the compact layout (empty slots zero), any ld_new.
template <typename T>
__global__ void __launch_bounds__(256) k_compact_cols(const CompactArgs a)
{
    const int64_t total = a.n * a.ld_new;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const T* s0 = static_cast<const T*>(a.q_src0);
    const T* s1 = static_cast<const T*>(a.q_src1);
    T* d0 = static_cast<T*>(a.q_dst0);
    T* d1 = static_cast<T*>(a.q_dst1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const int64_t u = i / a.ld_new, c = i % a.ld_new;
        const int o = a.old_slot[c];
        d0[i] = o >= 0 ? s0[u * a.ld_old + o] : T(0);
        d1[i] = o >= 0 ? s1[u * a.ld_old + o] : T(0);
    }
}

// The same when ld_new is a multiple of the 16-byte unit V: thread t keeps one column unit
// (its V source slots in registers) and walks the rows t / units, + rows_per_pass, ...;
// each new row unit is one 16-byte store per block, and no index division runs per element.
template <typename T>
__global__ void __launch_bounds__(256) k_compact_cols_v(const CompactArgs a)
{
    constexpr int V = 16 / (int)sizeof(T);
    const int64_t units = a.ld_new / V;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rows_per_pass = (int64_t)gridDim.x * blockDim.x / units;
    const int64_t r0 = t / units;
    if (r0 >= rows_per_pass) return;  // threads past the last whole group of units
    const int64_t cu = t % units;
    int o[V];
#pragma unroll
    for (int i = 0; i < V; ++i) o[i] = a.old_slot[cu * V + i];
    const T* s0 = static_cast<const T*>(a.q_src0);
    const T* s1 = static_cast<const T*>(a.q_src1);
    T* d0 = static_cast<T*>(a.q_dst0);
    T* d1 = static_cast<T*>(a.q_dst1);
    for (int64_t u = r0; u < a.n; u += rows_per_pass) {
        T x0[V], x1[V];
        const T* r0p = s0 + u * a.ld_old;
        const T* r1p = s1 + u * a.ld_old;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            x0[i] = o[i] >= 0 ? r0p[o[i]] : T(0);
            x1[i] = o[i] >= 0 ? r1p[o[i]] : T(0);
        }
        st_plain<T, V>(d0 + u * a.ld_new + cu * V, x0);
        st_plain<T, V>(d1 + u * a.ld_new + cu * V, x1);
    }
}

void launch_compact_map(cudaStream_t st, const CompactArgs& a)
{
    if (a.elem_size == 8) k_compact_map<double><<<1, 1024, 0, st>>>(a);
    else k_compact_map<float><<<1, 1024, 0, st>>>(a);
}

void launch_compact(cudaStream_t st, int grid, const CompactArgs& a)
{
    // the unit kernel needs whole 16-byte units per row and at least one row per pass
    const int64_t v = 16 / a.elem_size;
    const bool unit = a.ld_new % v == 0 && (int64_t)grid * 256 >= a.ld_new / v;
    if (a.elem_size == 8) {
        k_compact_map<double><<<1, 1024, 0, st>>>(a);
        if (unit) k_compact_cols_v<double><<<grid, 256, 0, st>>>(a);
        else k_compact_cols<double><<<grid, 256, 0, st>>>(a);
    } else {
        k_compact_map<float><<<1, 1024, 0, st>>>(a);
        if (unit) k_compact_cols_v<float><<<grid, 256, 0, st>>>(a);
        else k_compact_cols<float><<<grid, 256, 0, st>>>(a);
    }
}

// ---------------------------------------------------------- Power Method
template <typename T>
__global__ void k_pm_init(const PmArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npairs) return;
    const int32_t s = a.s[p], t = a.t[p];
    if (s < 0 || (int64_t)s >= a.n || t < 0 || (int64_t)t >= a.n) {
        atomicOr(a.err_flag, 1);
        return;
    }
    a.rbar[p] = 0.0;
    if (s == t) return;
    T* y = static_cast<T*>(a.y);
    y[(int64_t)s * a.ld + p] = (T)(1.0 / a.deg64[s]);
    y[(int64_t)t * a.ld + p] = (T)(-1.0 / a.deg64[t]);
}

template <typename T>
__global__ void k_pm_accum(const PmArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npairs) return;
    const int32_t s = a.s[p], t = a.t[p];
    if (s == t) {
        if (a.hist) a.hist[(int64_t)a.step * a.npairs + p] = 0.0;
        return;
    }
    const T* y = static_cast<const T*>(a.y);
    const double r = a.rbar[p] + 0.5 * ((double)y[(int64_t)s * a.ld + p] - (double)y[(int64_t)t * a.ld + p]);
    a.rbar[p] = r;
    if (a.hist) a.hist[(int64_t)a.step * a.npairs + p] = r;
}

void launch_pm_init(cudaStream_t st, const PmArgs& a)
{
    const int nb = (a.npairs + 127) / 128;
    if (a.elem_size == 8) k_pm_init<double><<<nb, 128, 0, st>>>(a);
    else k_pm_init<float><<<nb, 128, 0, st>>>(a);
}

void launch_pm_accum(cudaStream_t st, const PmArgs& a)
{
    const int nb = (a.npairs + 127) / 128;
    if (a.elem_size == 8) k_pm_accum<double><<<nb, 128, 0, st>>>(a);
    else k_pm_accum<float><<<nb, 128, 0, st>>>(a);
}

// ------------------------------------------------------------- on chip
// One pair per CTA, every step in one launch: SpMV from shared memory (one thread per light
// row, one warp per row above heavy_thr), three FP64 block sums in a fixed order, the same
// per-pair update as k_finalize (pair_update) by thread 0, normalisation in shared memory.
constexpr int kOnchipThreads = 1024;

size_t onchip_smem_bytes(int64_t n, int elem_size) { return (size_t)3 * (size_t)n * (size_t)elem_size + 64; }

template <typename T, bool WEIGHTED>
__global__ void __launch_bounds__(kOnchipThreads) k_lanczos_onchip(const OnchipArgs a)
{
    extern __shared__ __align__(16) unsigned char onchip_raw[];
    __shared__ double red[3][kOnchipThreads / 32];
    __shared__ double coef[3];
    __shared__ int stop_s;
    const int p = blockIdx.x;
    const PairState& st = a.fin.st;
    if (p >= a.npairs || !st.active[p]) return;  // uniform over the block
    const int64_t n = a.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarps = nthr >> 5;
    T* buf[3];
    buf[0] = reinterpret_cast<T*>(onchip_raw);
    buf[1] = buf[0] + n;
    buf[2] = buf[1] + n;
    int iprev = 0, icur = 1, iw = 2;
    for (int64_t u = tid; u < 3 * n; u += nthr) buf[0][u] = T(0);
    __syncthreads();
    if (tid == 0) {
        const int32_t s = a.s[p], t = a.t[p];
        const double ds = a.deg64[s], dt = a.deg64[t];
        const double bn = sqrt(st.b2[p]);
        buf[icur][s] = (T)(1.0 / (ds * bn));
        buf[icur][t] = (T)(-1.0 / (dt * bn));
    }
    __syncthreads();
    T bt = T(0);
    for (int j = 0; j < a.fin.k_max; ++j) {
        const T* qp = buf[iprev];
        const T* qc = buf[icur];
        T* W = buf[iw];
        double pa = 0.0, pb = 0.0, pc = 0.0;
        for (int64_t u = tid; u < n; u += nthr) {
            const int64_t e0 = a.row_ptr[u], e1 = a.row_ptr[u + 1];
            if (e1 - e0 > a.heavy_thr) continue;
            T acc = T(0);
            for (int64_t e = e0; e < e1; ++e) {
                if constexpr (WEIGHTED) acc += (T)__ldg(a.w + e) * qc[__ldg(a.col + e)];
                else acc += qc[__ldg(a.col + e)];
            }
            const T invd = sizeof(T) == 8 ? (T)a.invdeg64[u] : (T)a.invdeg32[u];
            const T du = sizeof(T) == 8 ? (T)a.deg64[u] : (T)a.deg32[u];
            const T wv = invd * acc - bt * qp[u];
            W[u] = wv;
            const T dw = du * wv;
            pa += (double)(dw * qc[u]);
            pb += (double)(dw * wv);
            pc += (double)dw;
        }
        for (int64_t h = warp; h < a.n_heavy_rows; h += nwarps) {
            const int64_t u = a.heavy_rows[h];
            T acc = T(0);
            for (int64_t e = a.row_ptr[u] + lane; e < a.row_ptr[u + 1]; e += 32) {
                if constexpr (WEIGHTED) acc += (T)__ldg(a.w + e) * qc[__ldg(a.col + e)];
                else acc += qc[__ldg(a.col + e)];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) {
                const T invd = sizeof(T) == 8 ? (T)a.invdeg64[u] : (T)a.invdeg32[u];
                const T du = sizeof(T) == 8 ? (T)a.deg64[u] : (T)a.deg32[u];
                const T wv = invd * acc - bt * qp[u];
                W[u] = wv;
                const T dw = du * wv;
                pa += (double)(dw * qc[u]);
                pb += (double)(dw * wv);
                pc += (double)dw;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            pa += __shfl_xor_sync(0xffffffffu, pa, off);
            pb += __shfl_xor_sync(0xffffffffu, pb, off);
            pc += __shfl_xor_sync(0xffffffffu, pc, off);
        }
        if (lane == 0) {
            red[0][warp] = pa;
            red[1][warp] = pb;
            red[2][warp] = pc;
        }
        __syncthreads();
        if (tid == 0) {
            double A = 0.0, B = 0.0, C = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                A += red[0][w];
                B += red[1][w];
                C += red[2][w];
            }
            double al = 0.0, cd = 0.0, bn = 0.0;
            const bool stop = pair_update(a.fin, st, p, j, A, B, C, &al, &cd, &bn);
            stop_s = stop ? 1 : 0;
            coef[0] = al;
            coef[1] = cd;
            coef[2] = bn;
        }
        __syncthreads();
        if (stop_s) break;
        const T al = (T)coef[0], cd = (T)coef[1], ib = (T)(1.0 / coef[2]);
        for (int64_t u = tid; u < n; u += nthr) W[u] = (W[u] - al * qc[u] - cd) * ib;
        bt = (T)coef[2];
        const int old_prev = iprev;
        iprev = icur;
        icur = iw;
        iw = old_prev;
        __syncthreads();
    }
}

// ---------------------------------------------------- on chip, one cluster per pair
// The same recurrence for one pair spread over a thread-block cluster of C CTAs (C = 2..16):
// CTA r holds rows [r R, (r+1) R) of q_{i-1}, q_i and W in its shared memory (R a power of
// two), and the product gathers q_i[col] from the owning CTA's shared memory through the
// cluster's distributed shared memory. Per step: every CTA's three FP64 block sums are
// written into every CTA of the cluster, a cluster barrier, every CTA sums the C partials in
// rank order and runs the same scalar update (pair_core) on its own copy of the pair's
// scalars (identical inputs, identical results; rank 0 also stores them), normalises its
// rows in place, and a second cluster barrier publishes the new vector. The FP64 work of a
// step is spread over C SMs (one CTA per SM) instead of one.
constexpr int kClusterThreads = 256;
constexpr int kClusterMax = 16;

struct ClusterLayout {
    int shift;        // log2 R: rows per CTA
    int C;            // CTAs per pair
};

template <typename T, bool WEIGHTED>
__global__ void __launch_bounds__(kClusterThreads) k_lanczos_cluster(const OnchipArgs a, const ClusterLayout L)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char cl_raw[];
    __shared__ double part[kClusterMax][3];
    __shared__ double tpart[3][kClusterThreads];  // per-thread partial sums of the step
    __shared__ double coef[3];
    __shared__ int stop_s;
    __shared__ T* rbase[3][kClusterMax];  // generic addresses of every rank's buffers
    const int C = L.C;
    const int rank = (int)cluster.block_rank();
    const int p = blockIdx.x / C;
    const PairState& st = a.fin.st;
    // uniform over the cluster: no CTA changes active[p] before the first cluster barrier
    if (p >= a.npairs || !st.active[p]) return;
    const int64_t n = a.n;
    const int64_t R = (int64_t)1 << L.shift;
    const int64_t row0 = (int64_t)rank * R;
    const int64_t nrow = row0 >= n ? 0 : (n - row0 < R ? n - row0 : R);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nthr = kClusterThreads, nwarps = kClusterThreads / 32;
    T* buf0 = reinterpret_cast<T*>(cl_raw);
    if (tid < 3 * C) {
        const int b = tid / C, rr = tid % C;
        rbase[b][rr] = cluster.map_shared_rank(buf0 + b * R, rr);
    }
    for (int64_t u = tid; u < 3 * R; u += nthr) buf0[u] = T(0);
    __syncthreads();
    PairScalars ps;
    if (tid == 0) {
        ps = pair_load(st, p, a.fin.pstride);
        const int32_t s = a.s[p], t = a.t[p];
        const double bn = sqrt(ps.b2);
        if (s >= row0 && s < row0 + nrow) buf0[R + (s - row0)] = (T)(1.0 / (a.deg64[s] * bn));
        if (t >= row0 && t < row0 + nrow) buf0[R + (t - row0)] = (T)(-1.0 / (a.deg64[t] * bn));
    }
    cluster.sync();  // every slice of q_1 is in place
    int iprev = 0, icur = 1, iw = 2;
    const int64_t mask = R - 1;
    T bt = T(0);
    for (int j = 0; j < a.fin.k_max; ++j) {
        T* const* cur = rbase[icur];
        const T* qp = buf0 + iprev * R;
        const T* qc = buf0 + icur * R;
        T* W = buf0 + iw * R;
        double pa = 0.0, pb = 0.0, pc = 0.0;
        for (int64_t ul = tid; ul < nrow; ul += nthr) {
            const int64_t u = row0 + ul;
            const int64_t e0 = a.row_ptr[u], e1 = a.row_ptr[u + 1];
            if (e1 - e0 > a.heavy_thr) continue;
            T acc = T(0);
            for (int64_t e = e0; e < e1; ++e) {
                const int32_t v = __ldg(a.col + e);
                const T x = cur[v >> L.shift][v & mask];
                if constexpr (WEIGHTED) acc += (T)__ldg(a.w + e) * x;
                else acc += x;
            }
            const T invd = sizeof(T) == 8 ? (T)a.invdeg64[u] : (T)a.invdeg32[u];
            const T du = sizeof(T) == 8 ? (T)a.deg64[u] : (T)a.deg32[u];
            const T wv = invd * acc - bt * qp[ul];
            W[ul] = wv;
            const T dw = du * wv;
            pa += (double)(dw * qc[ul]);
            pb += (double)(dw * wv);
            pc += (double)dw;
        }
        for (int64_t h = warp; h < a.n_heavy_rows; h += nwarps) {
            const int64_t u = a.heavy_rows[h];
            if (u < row0 || u >= row0 + nrow) continue;
            T acc = T(0);
            for (int64_t e = a.row_ptr[u] + lane; e < a.row_ptr[u + 1]; e += 32) {
                const int32_t v = __ldg(a.col + e);
                const T x = cur[v >> L.shift][v & mask];
                if constexpr (WEIGHTED) acc += (T)__ldg(a.w + e) * x;
                else acc += x;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += shfl_xor_t(0xffffffffu, acc, off);
            if (lane == 0) {
                const int64_t ul = u - row0;
                const T invd = sizeof(T) == 8 ? (T)a.invdeg64[u] : (T)a.invdeg32[u];
                const T du = sizeof(T) == 8 ? (T)a.deg64[u] : (T)a.deg32[u];
                const T wv = invd * acc - bt * qp[ul];
                W[ul] = wv;
                const T dw = du * wv;
                pa += (double)(dw * qc[ul]);
                pb += (double)(dw * wv);
                pc += (double)dw;
            }
        }
        // the CTA's three sums by one warp (FP64 adds are slow here, and the shuffles of the
        // other warps would contend for the same units): lane l adds threads l, l+32, ... in
        // order, then a fixed xor tree; lane r < C writes them into slot `rank` of CTA r
        tpart[0][tid] = pa;
        tpart[1][tid] = pb;
        tpart[2][tid] = pc;
        __syncthreads();
        if (warp == 0) {
            double A = 0.0, B = 0.0, Cs = 0.0;
            for (int w = 0; w < nwarps; ++w) {
                A += tpart[0][w * 32 + lane];
                B += tpart[1][w * 32 + lane];
                Cs += tpart[2][w * 32 + lane];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                A += __shfl_xor_sync(0xffffffffu, A, off);
                B += __shfl_xor_sync(0xffffffffu, B, off);
                Cs += __shfl_xor_sync(0xffffffffu, Cs, off);
            }
            if (lane < C) {
                double* dst = cluster.map_shared_rank(&part[0][0], lane);
                dst[rank * 3 + 0] = A;
                dst[rank * 3 + 1] = B;
                dst[rank * 3 + 2] = Cs;
            }
        }
        cluster.sync();  // all partial sums have arrived
        if (tid == 0) {
            double A = 0.0, B = 0.0, Cs = 0.0;
            for (int rr = 0; rr < C; ++rr) {
                A += part[rr][0];
                B += part[rr][1];
                Cs += part[rr][2];
            }
            PairStepOut o;
            const bool stop = pair_core(a.fin, ps, j, A, B, Cs, o);
            if (rank == 0) pair_store(st, p, j, a.fin.pstride, ps, o, stop);
            stop_s = stop ? 1 : 0;
            coef[0] = o.alpha;
            coef[1] = o.cdef;
            coef[2] = o.beta_next;
        }
        __syncthreads();
        if (stop_s) break;  // the same decision in every CTA of the cluster
        const T al = (T)coef[0], cd = (T)coef[1], ib = (T)(1.0 / coef[2]);
        for (int64_t ul = tid; ul < nrow; ul += nthr) W[ul] = (W[ul] - al * qc[ul] - cd) * ib;
        bt = (T)coef[2];
        const int old_prev = iprev;
        iprev = icur;
        icur = iw;
        iw = old_prev;
        cluster.sync();  // the new q_i is complete in every CTA before the next product reads it
    }
    cluster.sync();  // no CTA leaves while another may still address its shared memory
}

// Cluster size for the whole-recurrence kernel: as many CTAs per pair as keep every pair's
// cluster resident at once (npairs * C <= SMs), at least 32 rows per CTA, at most 16; 1 when
// a cluster would not help (the single-CTA kernel then runs).
static int cluster_size(const OnchipArgs& a)
{
    if (!a.allow_cluster || a.n_heavy_rows > 64) return 1;
    int C = 1;
    while (C < kClusterMax && (int64_t)a.npairs * C * 2 <= a.sm_count && a.n >= (int64_t)64 * C) C <<= 1;
    return C;
}

template <typename T, bool WEIGHTED>
static int launch_cluster_t(cudaStream_t st, const OnchipArgs& a, int C)
{
    auto k = k_lanczos_cluster<T, WEIGHTED>;
    ClusterLayout L;
    L.C = C;
    const int64_t rows = (a.n + C - 1) / C;
    L.shift = 0;
    while (((int64_t)1 << L.shift) < rows) ++L.shift;
    // three row blocks, but at least 120 KB so that one CTA of the cluster occupies an SM (the
    // FP64 rate per SM is what a cluster multiplies)
    const size_t need = (size_t)3 * ((size_t)1 << L.shift) * sizeof(T);
    if (need > 200 * 1024) return 0;
    const size_t sm = need < 120 * 1024 ? 120 * 1024 : need;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 0;
    if (C > 8 && cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.npairs * C), 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        return 0;
    }
    if (cudaLaunchKernelEx(&cfg, k, a, L) != cudaSuccess) {
        cudaGetLastError();  // a refused configuration is not sticky: try a smaller cluster
        return 0;
    }
    return C;
}

int launch_onchip(cudaStream_t st, const OnchipArgs& a)
{
    for (int C = cluster_size(a); C > 1; C >>= 1) {
        int used = 0;
        if (a.elem_size == 8) used = a.weighted ? launch_cluster_t<double, true>(st, a, C)
                                                : launch_cluster_t<double, false>(st, a, C);
        else used = a.weighted ? launch_cluster_t<float, true>(st, a, C) : launch_cluster_t<float, false>(st, a, C);
        if (used) return used;
    }
    const size_t sm = onchip_smem_bytes(a.n, a.elem_size);
    if (sm > 220 * 1024) return 0;
    if (a.elem_size == 8) {
        auto k = a.weighted ? k_lanczos_onchip<double, true> : k_lanczos_onchip<double, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<a.npairs, kOnchipThreads, sm, st>>>(a);
    } else {
        auto k = a.weighted ? k_lanczos_onchip<float, true> : k_lanczos_onchip<float, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<a.npairs, kOnchipThreads, sm, st>>>(a);
    }
    return 1;
}

}  // namespace rd

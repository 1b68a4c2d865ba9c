// Double-float arithmetic for the FP64-class vector mode on the FP32 pipes.
//
// A df64 is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about
// 48 significant bits (relative rounding about 2^-48). Sums use Knuth's error-free TwoSum,
// products Dekker's exact product through a fused multiply-add; both renormalise with
// the fast two-sum. Written from the published definitions (Knuth, TAOCP vol. 2, 4.2.2;
// Dekker 1971), not from any library. GB300 runs FP64 at a small fraction of its FP32
// rate, so an element operation in df64 (about 10-20 FP32 operations) costs less than one
// in FP64 when the kernel is arithmetic-bound; storage is 8 bytes, as for FP64.
#pragma once

#include <cuda_runtime.h>

namespace rd {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ explicit df64(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ explicit df64(float x) : hi(x), lo(0.f) {}
    __host__ __device__ explicit df64(int x) : hi((float)x), lo(0.f) {}
    __host__ __device__ df64(float h, float l, int /*raw*/) : hi(h), lo(l) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly (no condition on the magnitudes).
__device__ __forceinline__ df64 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df64(s, e, 0);
}

// s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)), 0);
}

// Sum with one error-free transformation of the high parts (Dekker's add): the error is
// at most about 2^-48 (|a| + |b|), the backward-stable bound FP64 arithmetic also has,
// for half the operations of the version that also captures the low parts' rounding.
__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
    const df64 s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo, 0); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact low part of a.hi * b.hi
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b)
{
    a = a + b;
    return a;
}

__device__ __forceinline__ df64& operator-=(df64& a, df64 b)
{
    a = a - b;
    return a;
}

// Accumulation of gathered terms into a running sum (the gather loops of the SpMM). For
// float and double a plain multiply-add. For df64 the leading parts go through TwoSum and the
// trailing parts are summed in FP32 without renormalising after every term (about 11 FP32
// operations per weighted term instead of 17); acc_finish renormalises once per row.
template <typename T>
__device__ __forceinline__ void acc_mul_add(T& acc, T w, T x)
{
    acc += w * x;
}
template <typename T>
__device__ __forceinline__ void acc_add(T& acc, T x)
{
    acc += x;
}
template <typename T>
__device__ __forceinline__ void acc_finish(T&)
{
}
template <>
__device__ __forceinline__ void acc_mul_add<df64>(df64& acc, df64 w, df64 x)
{
    const float p = __fmul_rn(w.hi, x.hi);
    float e = __fmaf_rn(w.hi, x.hi, -p);  // exact low part of w.hi * x.hi
    e = __fmaf_rn(w.hi, x.lo, e);
    e = __fmaf_rn(w.lo, x.hi, e);
    const df64 s = df_two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
template <>
__device__ __forceinline__ void acc_add<df64>(df64& acc, df64 x)
{
    const df64 s = df_two_sum(acc.hi, x.hi);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, x.lo));
}
// The same with an FP32 edge weight (a df64 with a zero low part): the product's w.lo x.hi
// term, an exact zero, is not formed.
template <typename T>
__device__ __forceinline__ void acc_mul_add_w(T& acc, float w, T x)
{
    acc_mul_add(acc, T(w), x);
}
template <>
__device__ __forceinline__ void acc_mul_add_w<df64>(df64& acc, float w, df64 x)
{
    const float p = __fmul_rn(w, x.hi);
    float e = __fmaf_rn(w, x.hi, -p);  // exact low part of w * x.hi
    e = __fmaf_rn(w, x.lo, e);
    const df64 s = df_two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(s.lo, e));
}
template <>
__device__ __forceinline__ void acc_finish<df64>(df64& acc)
{
    acc = df_two_sum(acc.hi, acc.lo);
}

// Warp shuffles of element values (both halves move together).
__device__ __forceinline__ float shfl_xor_t(unsigned mask, float v, int off, int width = 32)
{
    return __shfl_xor_sync(mask, v, off, width);
}
__device__ __forceinline__ double shfl_xor_t(unsigned mask, double v, int off, int width = 32)
{
    return __shfl_xor_sync(mask, v, off, width);
}
__device__ __forceinline__ df64 shfl_xor_t(unsigned mask, df64 v, int off, int width = 32)
{
    return df64(__shfl_xor_sync(mask, v.hi, off, width), __shfl_xor_sync(mask, v.lo, off, width), 0);
}
__device__ __forceinline__ float shfl_t(unsigned mask, float v, int src, int width = 32)
{
    return __shfl_sync(mask, v, src, width);
}
__device__ __forceinline__ double shfl_t(unsigned mask, double v, int src, int width = 32)
{
    return __shfl_sync(mask, v, src, width);
}
__device__ __forceinline__ df64 shfl_t(unsigned mask, df64 v, int src, int width = 32)
{
    return df64(__shfl_sync(mask, v.hi, src, width), __shfl_sync(mask, v.lo, src, width), 0);
}

// Conversions of element values to double (identity for float and double).
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(df64 v) { return (double)v; }

}  // namespace rd

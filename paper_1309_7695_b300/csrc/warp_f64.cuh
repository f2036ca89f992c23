// Warp-level building blocks of the FP64 reference kernels: propensities,
// the canonical 32-slot sum and its selection, warp reductions.
#pragma once

#include "device_f64.cuh"
#include "engine.h"

namespace tl {

constexpr unsigned kFull = 0xffffffffu;

// Slot tree over the warp: L[0] = this lane's slot sum, L[k] = L[k-1] +
// L[k-1] of lane ^ (16 >> (k-1)).  Every lane ends with the same L[5].
__device__ __forceinline__ double slot_tree(double v, double L[6])
{
    L[0] = v;
#pragma unroll
    for (int k = 1; k <= 5; ++k) L[k] = L[k - 1] + __shfl_xor_sync(kFull, L[k - 1], 16 >> (k - 1));
    return L[5];
}

// Pick j with probability v_j / total given target = u * total: descend the
// slot tree (second child when target >= first child and second child > 0),
// then walk the chosen slot's reactions in increasing j.  When `crit_only`
// the weights are the critical propensities (0 for noncritical reactions).
// All weights, sums and the target are non-negative, so the comparisons run
// on their bit patterns.
__device__ __forceinline__ int slot_select(const double L[6], double target, const double *a,
                                           const unsigned char *crit, bool crit_only, int M)
{
    int cls = 0;
#pragma unroll
    for (int k = 4; k >= 0; --k) {
        const int step = 1 << (4 - k);
        const double left = __shfl_sync(kFull, L[k], cls);
        const double right = __shfl_sync(kFull, L[k], cls + step);
        if (f64::nn_ge(target, left) && f64::nn_pos(right)) {
            target = target - left;
            cls += step;
        }
    }
    double cum = 0.0;
    int last = -1;
    for (int j = cls; j < M; j += 32) {
        const double v = (crit_only && !crit[j]) ? 0.0 : a[j];
        if (j == cls) cum = f64::first_term(v);
        else cum = cum + v;
        if (f64::nn_pos(v)) last = j;
        if (f64::nn_gt(cum, target)) return j;
    }
    return last;
}

__device__ __forceinline__ double propensity(int info, double c, const int *x)
{
    const int kind = info & 3;
    const int s0 = (info >> 2) & 0x7fff;
    const int s1 = (info >> 17) & 0x7fff;
    if (kind == 0) return c;
    if (kind == 1) return c * (double)x[s0];
    if (kind == 2) return (c * (double)x[s0]) * (double)x[s1];
    const long long xi = x[s0];
    return c * (double)((xi * (xi - 1)) / 2);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, v, d);
        v = o < v ? o : v;
    }
    return v;
}

__device__ __forceinline__ long long warp_sum_i64(long long v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// Propensity with the counts stored as one column of a [N][stride] array.
// Counts are non-negative, so their conversions to double are assembled
// from bits (same values as the rounding conversion).
__device__ __forceinline__ double propensity_col(int info, double c, const int *X, int stride, int col)
{
    const int kind = info & 3;
    const int s0 = (info >> 2) & 0x7fff;
    const int s1 = (info >> 17) & 0x7fff;
    if (kind == 0) return c;
    if (kind == 1) return c * f64::count_to_double(X[s0 * stride + col]);
    if (kind == 2) return (c * f64::count_to_double(X[s0 * stride + col])) * f64::count_to_double(X[s1 * stride + col]);
    const long long xi = X[s0 * stride + col];
    return c * f64::u53_to_double((unsigned long long)((xi * (xi - 1)) / 2));
}

}  // namespace tl

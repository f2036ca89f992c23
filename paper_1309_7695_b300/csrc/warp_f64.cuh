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
    // the minimum of the high words, then the minimum low word among the
    // lanes that hold it (two hardware reductions instead of five shuffle
    // rounds of 64-bit values)
    const unsigned hi = __reduce_min_sync(kFull, (unsigned)(v >> 32));
    const unsigned lo = __reduce_min_sync(kFull, (unsigned)(v >> 32) == hi ? (unsigned)v : 0xFFFFFFFFu);
    return ((unsigned long long)hi << 32) | lo;
}

// Sum over the warp of 0 <= v < 2^50 (a lane's Poisson counts of one leap:
// at most 2^14 reactions per lane, each at most 2^40 + 1): the low 24 and the
// high 26 bits are summed by two 32-bit hardware reductions without overflow.
__device__ __forceinline__ long long warp_sum_counts(long long v)
{
    const unsigned lo = __reduce_add_sync(kFull, (unsigned)(v & 0xFFFFFF));
    const unsigned hi = __reduce_add_sync(kFull, (unsigned)(v >> 24));
    return ((long long)hi << 24) + (long long)lo;
}

__device__ __forceinline__ long long warp_sum_i64(long long v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// Propensity with the counts stored as one column of a [N][stride] array.
// Counts are non-negative, so their conversions to double are assembled
// from bits (same values as the rounding conversion).  Written without
// branches on the reaction kind, so that lanes of a warp holding reactions
// of different kinds issue the same two multiplies: a = (c h0) h1 with
// (h0, h1) = (1, 1), (x, 1), (x, y) or (x(x-1)/2, 1); a product with 1.0 is
// exact, so the values are those of c, c x, (c x) y and c (x(x-1)/2).
__device__ __forceinline__ double propensity_col(int info, double c, const int *X, int stride, int col)
{
    const int kind = info & 3;
    const int s0 = (info >> 2) & 0x7fff;
    const int s1 = (info >> 17) & 0x7fff;
    const long long x0 = X[s0 * stride + col];
    const int x1 = X[s1 * stride + col];
    const unsigned long long h0 = (kind == 3) ? (unsigned long long)((x0 * (x0 - 1)) / 2) : (unsigned long long)x0;
    const double d0 = (kind == 0) ? 1.0 : f64::u53_to_double(h0);
    const double d1 = (kind == 2) ? f64::count_to_double(x1) : 1.0;
    return (c * d0) * d1;
}

}  // namespace tl

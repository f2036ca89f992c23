// Device arithmetic of fast mode: FP32 propensities and Poisson means and an
// FP32 Poisson sampler, on the same Philox stream words as the FP64
// reference mode (a fast run and a reference run of one simulation use
// common random numbers).  Uses CUDA's single-precision math functions.
#pragma once

#include <stdint.h>

#include "device_f64.cuh"
#include "engine.h"

namespace tl {
namespace fast {

// Conversions between FP32 and FP64 assembled from bits on the integer pipe
// (on this GPU a conversion instruction costs as much as an FP64 add).
// Both give the IEEE result: float -> double is exact, double -> float
// rounds to nearest even.  Values outside the normal float range (zero
// aside) take the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if ((u << 1) == 0) return __longlong_as_double((long long)sign);   // +-0
    if (e == 0 || e == 255) return (double)f;
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)(e + (1023 - 127)) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

__device__ __forceinline__ float f64_to_f32(double d)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    if ((b << 1) == 0) return __uint_as_float(sign);   // +-0
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e < -126 || e > 127) return __double2float_rn(d);
    const unsigned long long mant = b & 0x000FFFFFFFFFFFFFull;
    const unsigned m23 = (unsigned)(mant >> 29);
    const unsigned rem = (unsigned)(mant & 0x1FFFFFFFull);
    unsigned r = ((unsigned)(e + 127) << 23) | m23;
    if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) r += 1;   // a carry moves into the exponent
    return __uint_as_float(sign | r);
}

// Uniform in (0,1) from the top 23 bits of one word: ((w >> 9) + 1/2) 2^-23.
// It takes the leading bits of the reference mode's 52-bit uniform.
__device__ __forceinline__ float u23(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

constexpr int kInversionCap = 100;
// PTRS means from here on run the FP64 sampler: FP32 no longer resolves
// the integers around such a mean.
constexpr float kPtrsF32Limit = 0x1p22f;

// Inversion by sequential search for 0 < lam < 10 with the FP32 cdf, on the
// leading 23 bits of the reference mode's inversion uniform.
__device__ __forceinline__ long long inversion(float lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    const uint4 w = f64::draw(seed, sim, attempt, PURPOSE_POISSON, j, 0);
    const float u = u23(w.x);
    float p = __expf(-lam);
    float F = p;
    int k = 0;
    while (u > F && k < kInversionCap) {
        ++k;
        p = __fdividef(p * lam, (float)k);
        const float Fn = F + p;
        if (Fn == F) break;
        F = Fn;
    }
    return k;
}

// ln of the Poisson pmf, k ln lam - lam - ln k!, in FP32 without the
// cancellation of its large terms.  For k >= 10, with Stirling's series for
// ln k!, it equals -D - ln(2 pi k)/2 - (1/(12k) - 1/(360k^3)), where
// D = k ln(k/lam) + lam - k >= 0 is the deviance.  Near k = lam, D is summed
// from v = (k - lam)/(k + lam) as v (k - lam) + 2k (v^3/3 + v^5/5 + ...),
// since k ln(k/lam) = 2k atanh(v) and k - lam = v (k + lam) (the saddle-point
// form of Loader, "Fast and accurate computation of binomial probabilities",
// 2000); every term there is small, so no precision is lost.
__device__ __forceinline__ float log_pmf(float k, float lam)
{
    if (k < 10.0f) {
        float f = 1.0f;
        for (int i = 2; i <= (int)k; ++i) f *= (float)i;   // k! <= 9! is exact in FP32
        return k * __logf(lam) - lam - __logf(f);
    }
    const float d = k - lam;
    const float v = d / (k + lam);
    float D;
    if (fabsf(v) < 0.25f) {
        const float v2 = v * v;
        // sum_{n=1..7} v^(2n+1)/(2n+1); the first omitted term is below 2^-32 of the lead
        float s = 1.0f / 15.0f;
        s = s * v2 + 1.0f / 13.0f;
        s = s * v2 + 1.0f / 11.0f;
        s = s * v2 + 1.0f / 9.0f;
        s = s * v2 + 1.0f / 7.0f;
        s = s * v2 + 1.0f / 5.0f;
        s = s * v2 + 1.0f / 3.0f;
        D = v * d + 2.0f * k * (v * v2 * s);
    } else {
        D = k * logf(k / lam) + lam - k;
    }
    const float rk = 1.0f / k;
    const float corr = rk * (1.0f / 12.0f - (rk * rk) * (1.0f / 360.0f));
    return -D - 0.5f * logf(6.283185307f * k) - corr;
}

// PTRS (Hormann 1993) in FP32 for 10 <= lam < kPtrsF32Limit: the candidate
// integer, the squeeze and the acceptance test (through log_pmf) all in
// FP32, one stream block per iteration, on the leading 23 bits of the
// reference mode's words.
__device__ __forceinline__ long long ptrs(float lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    const float slam = sqrtf(lam);
    const float b = 0.931f + 2.53f * slam;
    const float a = -0.059f + 0.02483f * b;
    const float vr = 0.9277f - __fdividef(3.6224f, b - 2.0f);
    const float inv_alpha = 1.1239f + __fdividef(1.1328f, b - 3.4f);
    for (uint32_t it = 0; it < (uint32_t)f64::kPtrsMaxIters; ++it) {
        const uint4 w = f64::draw(seed, sim, attempt, PURPOSE_POISSON, j, it);
        const float U = u23(w.x) - 0.5f;
        const float V = u23(w.z);
        const float us = 0.5f - fabsf(U);
        const float kf = floorf((__fdividef(2.0f * a, us) + b) * U + lam + 0.43f);
        if (us >= 0.07f && V <= vr) return (long long)__float2int_rz(kf);   // kf >= 0 here for lam >= 10
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        const float lhs = __logf(V * inv_alpha / (a / (us * us) + b));
        if (lhs <= log_pmf(kf, lam)) return (long long)__float2int_rz(kf);
    }
    return -1;
}

}  // namespace fast
}  // namespace tl

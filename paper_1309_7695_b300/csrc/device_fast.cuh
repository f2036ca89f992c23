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

using f64::f32_to_f64;
using f64::f64_to_f32;

// Uniform in (0,1) from the top 23 bits of one word: ((w >> 9) + 1/2) 2^-23.
// It takes the leading bits of the reference mode's 52-bit uniform.
__device__ __forceinline__ float u23(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

constexpr int kInversionCap = 100;
// PTRS means from here on run the FP64 sampler: FP32 no longer resolves
// the integers around such a mean.
constexpr float kPtrsF32Limit = 0x1p22f;

// Inversion by sequential search for 0 < lam < 10 with the FP32 cdf, on the
// leading 23 bits of the reference mode's inversion uniform.
__device__ __forceinline__ long long inversion_u(float lam, float u)
{
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
__device__ __forceinline__ long long inversion(float lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    const uint4 w = f64::draw(seed, sim, attempt, PURPOSE_POISSON, j, 0);
    return inversion_u(lam, u23(w.x));
}

using f64::log_pmf_f32;

// PTRS (Hormann 1993) in FP32 for 10 <= lam < kPtrsF32Limit: the candidate
// integer, the squeeze and the acceptance test (through log_pmf) all in
// FP32, one stream block per iteration, on the leading 23 bits of the
// reference mode's words.
// `work` (optional): [0] += iterations, [1] += acceptance tests after the squeeze.
__device__ __forceinline__ long long ptrs(float lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j,
                                          unsigned *work = nullptr)
{
    const float slam = sqrtf(lam);
    const float b = 0.931f + 2.53f * slam;
    const float a = -0.059f + 0.02483f * b;
    const float vr = 0.9277f - __fdividef(3.6224f, b - 2.0f);
    const float inv_alpha = 1.1239f + __fdividef(1.1328f, b - 3.4f);
    for (uint32_t it = 0; it < (uint32_t)f64::kPtrsMaxIters; ++it) {
        if (work) work[0] += 1;
        const uint4 w = f64::draw(seed, sim, attempt, PURPOSE_POISSON, j, it);
        const float U = u23(w.x) - 0.5f;
        const float V = u23(w.z);
        const float us = 0.5f - fabsf(U);
        const float kf = floorf((__fdividef(2.0f * a, us) + b) * U + lam + 0.43f);
        if (us >= 0.07f && V <= vr) return (long long)__float2int_rz(kf);   // kf >= 0 here for lam >= 10
        if (kf < 0.0f || (us < 0.013f && V > us)) continue;
        if (work) work[1] += 1;
        const float lhs = __logf(V * inv_alpha / (a / (us * us) + b));
        if (lhs <= log_pmf_f32(kf, lam)) return (long long)__float2int_rz(kf);
    }
    return -1;
}

}  // namespace fast
}  // namespace tl

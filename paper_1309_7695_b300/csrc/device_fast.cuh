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

// Uniform in (0,1) from the top 23 bits of one word: ((w >> 9) + 1/2) 2^-23.
// It takes the leading bits of the reference mode's 52-bit uniform.
__device__ __forceinline__ float u23(uint32_t w) { return ((float)(w >> 9) + 0.5f) * 0x1p-23f; }

constexpr int kInversionCap = 100;

// k ~ Poisson(lam), FP32.  lam < 10: inversion by sequential search (FP32
// cdf, compared with the reference mode's 53-bit uniform); lam >= 10: PTRS (Hormann 1993) in FP32, with the final integer
// formed in FP64 (so large means keep integer resolution) and the rare
// acceptance test against the log-pmf in FP64 (its terms cancel heavily).
__device__ __forceinline__ long long poisson(float lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    if (!(lam > 0.0f)) return 0;
    if (!(lam < 0x1p40f)) return f64::kCountLimit + 1;
    if (lam < 10.0f) {
        const uint4 w = f64::draw(seed, sim, attempt, PURPOSE_POISSON, j, 0);
        const double u = f64::u01(w.x, w.y);   // the reference mode's uniform
        float p = __expf(-lam);
        float F = p;
        int k = 0;
        while (u > (double)F && k < kInversionCap) {
            ++k;
            p = __fdividef(p * lam, (float)k);
            const float Fn = F + p;
            if (Fn == F) break;
            F = Fn;
        }
        return k;
    }
    const float slam = sqrtf(lam);
    const float b = 0.931f + 2.53f * slam;
    const float a = -0.059f + 0.02483f * b;
    const float vr = 0.9277f - __fdividef(3.6224f, b - 2.0f);
    for (uint32_t it = 0; it < (uint32_t)f64::kPtrsMaxIters; ++it) {
        const uint4 w = f64::draw(seed, sim, attempt, PURPOSE_POISSON, j, it);
        const float U = u23(w.x) - 0.5f;
        const float V = u23(w.z);
        const float us = 0.5f - fabsf(U);
        const double kd = floor((double)((__fdividef(2.0f * a, us) + b) * U) + (double)lam + 0.43);
        if (us >= 0.07f && V <= vr) return (kd > (double)f64::kCountLimit) ? f64::kCountLimit + 1 : (long long)kd;
        if (kd < 0.0 || (us < 0.013f && V > us)) continue;
        if (kd > (double)f64::kCountLimit) return f64::kCountLimit + 1;
        const double inv_alpha = 1.1239 + 1.1328 / ((double)b - 3.4);
        const double usd = (double)us;
        const double lhs = log((double)V * inv_alpha / ((double)a / (usd * usd) + (double)b));
        const double rhs = -(double)lam + kd * log((double)lam) - lgamma(kd + 1.0);
        if (lhs <= rhs) return (long long)kd;
    }
    return -1;
}

}  // namespace fast
}  // namespace tl

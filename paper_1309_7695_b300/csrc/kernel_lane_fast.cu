// Fast-mode instantiation of the lane-per-simulation kernel.
//
// FP32: propensities a_j, Poisson means a_j tau and the Poisson sampler
// (inversion, and PTRS below means of 2^22 with an FP32 acceptance test),
// -ln u and the event times E/a.  FP64: the simulated clock, the slot tree
// (a0 and a0c as FP64 sums of the FP32 propensities), the critical test and
// tau' (mu_i, sigma_i^2, the bounds and their minimum), as the reference
// mode.  Counts stay exact integers.  Random numbers come from the same
// Philox words as the reference mode, so the two modes are coupled.
#include <algorithm>

#include "device_fast.cuh"
#include "lane_kernel.cuh"

namespace tl {
namespace {

struct FastArith {
    // The SSA step sums each slot's propensities in FP32 and promotes the
    // slot sum to FP64 for the tree (a0 and its partial sums stay FP64).
    static constexpr bool kFloatSlots = true;
    // FP32 propensity from the FP32 rate constant (its RN image)
    __device__ static __forceinline__ float prop_f(int info, float cf, const int *X, int stride, int col)
    {
        const int kind = info & 3;
        const int s0 = (info >> 2) & 0x7fff;
        const int s1 = (info >> 17) & 0x7fff;
        if (kind == 0) return cf;
        if (kind == 1) return cf * (float)X[s0 * stride + col];
        if (kind == 2) return (cf * (float)X[s0 * stride + col]) * (float)X[s1 * stride + col];
        const int xi = X[s0 * stride + col];
        return cf * (0.5f * ((float)xi * (float)(xi - 1)));
    }
    // Conversions go through f64::f32_to_f64 / f64_to_f32 (integer pipe).
    __device__ static __forceinline__ double prop(int info, double c, const int *X, int stride, int col)
    {
        return f64::f32_to_f64(prop_f(info, f64::f64_to_f32(c), X, stride, col));
    }
    __device__ static __forceinline__ void uniforms(uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t purpose,
                                                    double &ua, double &ub)
    {
        // the reference mode's 53-bit uniforms: -ln u is then taken in FP32,
        // while selection targets u * a0 keep the full resolution
        const uint4 w = f64::draw(seed, sim, attempt, purpose, 0, 0);
        ua = f64::u01(w.x, w.y);
        ub = f64::u01(w.z, w.w);
    }
    __device__ static __forceinline__ double neglog(double u)
    {
        // u in (0,1) rounded to FP32 stays in (0,1]; -ln 1 = 0 is a zero-length step
        return f64::f32_to_f64(-logf(f64::f64_to_f32(u)));
    }
    __device__ static __forceinline__ double tau_of(double E, double a)
    {
        return f64::f32_to_f64(f64::f64_to_f32(E) / f64::f64_to_f32(a));
    }
    __device__ static __forceinline__ double mean(double a, double tau)
    {
        return f64::f32_to_f64(f64::f64_to_f32(a) * f64::f64_to_f32(tau));
    }
    __device__ static __forceinline__ int inv_certain(double lam, uint64_t seed, uint32_t sim, uint32_t attempt,
                                                      uint32_t j)
    {
        // the FP32 inversion is the fast-mode definition: always decided here
        return (int)fast::inversion(f64::f64_to_f32(lam), seed, sim, attempt, j);
    }
    __device__ static __forceinline__ void uniforms_of(uint4 w, double &ua, double &ub)
    {
        ua = f64::u01(w.x, w.y);
        ub = f64::u01(w.z, w.w);
    }
    __device__ static __forceinline__ int inv_certain_of(double lam, uint4 w)
    {
        return (int)fast::inversion_u(f64::f64_to_f32(lam), fast::u23(w.x));
    }
    __device__ static __forceinline__ long long inversion(double lam, uint64_t seed, uint32_t sim, uint32_t attempt,
                                                          uint32_t j, const double *)
    {
        return fast::inversion(f64::f64_to_f32(lam), seed, sim, attempt, j);
    }
    __device__ static __forceinline__ long long ptrs(double lam, uint64_t seed, uint32_t sim, uint32_t attempt,
                                                     uint32_t j, unsigned *work)
    {
        if (f64::nn_gt((double)fast::kPtrsF32Limit, lam))
            return fast::ptrs(f64::f64_to_f32(lam), seed, sim, attempt, j, work);
        return f64::ptrs_draw(lam, seed, sim, attempt, j, work);
    }
};

__global__ void params_to_f32(const double *__restrict__ in, float *__restrict__ out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

}  // namespace

cudaError_t launch_params_to_f32(const double *in, float *out, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 148ll * 8);
    params_to_f32<<<(int)blocks, 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_lane_fast(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s)
{
    return launch_lane_impl<FastArith, false>(a, block_warps, grid, smem, carveout, reg_cap, s);
}

int lane_fast_occupancy(int block_warps, size_t smem, int reg_cap) { return lane_occupancy_impl<FastArith, false>(block_warps, smem, reg_cap); }

cudaError_t launch_lane_multi_fast(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s)
{
    return launch_lane_impl<FastArith, true>(a, block_warps, grid, smem, carveout, reg_cap, s);
}

int lane_multi_fast_occupancy(int block_warps, size_t smem, int reg_cap)
{
    return lane_occupancy_impl<FastArith, true>(block_warps, smem, reg_cap);
}

}  // namespace tl

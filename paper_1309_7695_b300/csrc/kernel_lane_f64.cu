// FP64 reference instantiation of the lane-per-simulation kernel.
//
// Compiled with -fmad=false: every double operation is one correctly rounded
// IEEE operation in the order the CPU oracle performs it, so trajectories,
// counters and times match the oracle bit for bit.
#include "lane_kernel.cuh"

namespace tl {
namespace {

struct RefArith {
    // slot sums in FP64, in the canonical order (no FP32 path)
    static constexpr bool kFloatSlots = false;
    __device__ static __forceinline__ double prop(int info, double c, const int *X, int stride, int col)
    {
        return propensity_col(info, c, X, stride, col);
    }
    __device__ static __forceinline__ void uniforms(uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t purpose,
                                                    double &ua, double &ub)
    {
        const uint4 w = f64::draw(seed, sim, attempt, purpose, 0, 0);
        ua = f64::u01(w.x, w.y);
        ub = f64::u01(w.z, w.w);
    }
    __device__ static __forceinline__ double neglog(double u) { return -f64::dlog(u); }
    __device__ static __forceinline__ double tau_of(double E, double a) { return E / a; }
    __device__ static __forceinline__ double mean(double a, double tau) { return a * tau; }
    __device__ static __forceinline__ int inv_certain(double lam, uint64_t seed, uint32_t sim, uint32_t attempt,
                                                      uint32_t j)
    {
        return f64::inversion_certain(lam, f64::inversion_uniform(seed, sim, attempt, j));
    }
    // the same decisions from a Philox block already drawn: the leap's block, and
    // block 0 of reaction j's Poisson stream
    __device__ static __forceinline__ void uniforms_of(uint4 w, double &ua, double &ub)
    {
        ua = f64::u01(w.x, w.y);
        ub = f64::u01(w.z, w.w);
    }
    __device__ static __forceinline__ int inv_certain_of(double lam, uint4 w)
    {
        return f64::inversion_certain(lam, f64::u01(w.x, w.y));
    }
    __device__ static __forceinline__ long long inversion(double lam, uint64_t seed, uint32_t sim, uint32_t attempt,
                                                          uint32_t j, const double *inv)
    {
        return f64::inversion_draw(lam, f64::inversion_uniform(seed, sim, attempt, j), inv);
    }
    __device__ static __forceinline__ long long ptrs(double lam, uint64_t seed, uint32_t sim, uint32_t attempt,
                                                     uint32_t j, unsigned *work)
    {
        return f64::ptrs_draw(lam, seed, sim, attempt, j, work);
    }
};

}  // namespace

size_t lane_f64_smem_bytes(const ModelLayout &L, int block_warps) { return lane_smem_bytes(L, block_warps); }

cudaError_t launch_lane_ref(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s)
{
    return launch_lane_impl<RefArith, false>(a, block_warps, grid, smem, carveout, reg_cap, s);
}

int lane_ref_occupancy(int block_warps, size_t smem, int reg_cap) { return lane_occupancy_impl<RefArith, false>(block_warps, smem, reg_cap); }

size_t lane_multi_smem_bytes(int max_N, int max_M, int block_warps) { return lane_multi_bytes(max_N, max_M, block_warps); }

cudaError_t launch_lane_multi_ref(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s)
{
    return launch_lane_impl<RefArith, true>(a, block_warps, grid, smem, carveout, reg_cap, s);
}

int lane_multi_ref_occupancy(int block_warps, size_t smem, int reg_cap)
{
    return lane_occupancy_impl<RefArith, true>(block_warps, smem, reg_cap);
}

}  // namespace tl

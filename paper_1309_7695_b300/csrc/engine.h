// Internal declarations shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tauleap.h"

namespace tl {

// Packed network, one int32 blob (uploaded once, staged into shared memory
// by every CTA).  Sections, in order:
//   rinfo [M]      kind | sp0 << 2 | sp1 << 17   (kind 0: order 0, 1: X,
//                  2: X+Y with sp0 < sp1, 3: 2X)
//   nu_ptr [M+1]   net-change CSR of reaction j
//   nu_ent [nnz]   species << 8 | (nu & 0xff)    species ascending
//   tr_ptr [N+1]   transpose: reactions that change species i
//   tr_ent [nnz]   j << 8 | (nu & 0xff)          j ascending
//   hor [N]        highest-order class of species i: 0 none, 1 first order,
//                  2 second order as X+Y only, 3 some reaction takes 2X
//   dep_ptr [N+1]  reactions whose propensity reads species i (i is a reactant)
//   dep_ent [ndep] reaction indices
//   cinfo [M]      the species reaction j consumes (nu < 0), for the
//                  critical test: sp_a | n_a << 14 | sp_b << 16 | n_b << 30,
//                  n = |nu| in {1, 2}, 0 for an absent entry (a reaction of
//                  order <= 2 consumes at most two species)
//   dmask [M]      slots (k mod 32) of the reactions k whose propensity
//                  changes when reaction j fires (they read a species j
//                  changes): the dirty slots of an SSA step
struct ModelLayout {
    int32_t N, M, nnz, ndep;
    int32_t off_rinfo, off_nu_ptr, off_nu_ent, off_tr_ptr, off_tr_ent, off_hor, off_dep_ptr, off_dep_ent, off_cinfo,
        off_dmask;
    int32_t words;
    int32_t max_nu_len;
};

enum : uint32_t { PURPOSE_LEAP = 1u, PURPOSE_POISSON = 2u, PURPOSE_SSA = 3u };

// One group of a multi-network launch: its network (packed blob in global
// memory), its inputs and outputs, and the flattened index of its first
// simulation.
struct GroupArgs {
    ModelLayout L;
    const int32_t *blob;
    const double *params;
    const float *params_f;   // fast mode: the FP32 images of params, or null (converted on use)
    const int32_t *x0;
    const double *T;
    int32_t S;
    double t_end;
    int64_t n_sims;
    int64_t sim_offset;
    uint64_t seed;
    int32_t *samples;
    ssa_sim_stats *stats;
    int64_t first;
    // optional completion signal (the serving loop): every finished
    // simulation adds 1 to *done_count; the one that brings it to n_sims
    // sets *done_flag (host-mapped memory) to 1 after a system-scope fence,
    // so the host learns that this group's results are complete while the
    // launch is still running other groups
    unsigned long long *done_count;
    volatile int32_t *done_flag;
};

struct SimArgs {
    // multi-network launch: groups[0..n_groups) in schedule order, flattened
    // over total_sims simulations; n_groups == 0 for a single-network launch
    const GroupArgs *groups;
    int32_t n_groups;
    int32_t max_N, max_M;
    int64_t total_sims;
    ModelLayout L;
    const int32_t *blob;
    const double *params;
    const float *params_f;   // fast mode: the FP32 images of params, or null (converted on use)
    const int32_t *x0;
    const double *T;
    int32_t S;
    double t_end;
    int64_t n_sims;
    int64_t sim_offset;
    uint64_t seed;
    int32_t mode;
    int32_t n_c;
    double eps;
    double ssa_factor;
    int32_t ssa_block;
    int32_t max_halvings;
    int64_t max_attempts;
    int32_t sims_per_warp;
    int32_t *samples;
    ssa_sim_stats *stats;
    unsigned long long *work_counter;
    // optional per-launch work counters (SSA_WORK_* indices), added to
    unsigned long long *work;
    // sweep moments (single-network lane launches): when non-null, every
    // recorded count x of cell (k, i) adds x, (x^2 mod 2^32) and (x^2 >> 32)
    // to moments[(k*N + i)*3 + 0..2]; samples may then be null
    unsigned long long *moments;
    // sweep histograms (single-network lane launches): when non-null, every
    // recorded count x of cell (k, i) adds 1 to hist[(k*N + i)*(hist_bins+2) + b],
    // b = 0 for x < hist_lo, 1 + (x - hist_lo) / hist_width up to hist_bins, and
    // hist_bins + 1 above; samples may then be null
    unsigned long long *hist;
    int32_t hist_lo, hist_width, hist_bins;
};

// Shared-memory bytes of one warp's simulation workspace.
__host__ __device__ inline size_t warp_workspace_bytes(int N, int M)
{
    auto r16 = [](size_t v) { return (v + 15) & ~size_t(15); };
    size_t b = 0;
    b += r16(8 * (size_t)M);        // a_j
    b += r16(8 * (size_t)M);        // c_j
    b += r16(8 * (size_t)M);        // k_j
    b += r16(8 * (size_t)N);        // x' (int64)
    b += r16(4 * (size_t)N);        // x
    b += r16((size_t)M);            // critical flags
    b += r16((size_t)N);            // I_rs flags
    return b;
}

__host__ __device__ inline size_t model_smem_bytes(const ModelLayout &L)
{
    return ((size_t)L.words * 4 + 15) & ~size_t(15);
}

// Lane-per-simulation FP64 reference kernel (kernel_lane_f64.cu): SSA steps
// one simulation per lane, leaps and step-size selection warp-cooperative.
size_t lane_f64_smem_bytes(const ModelLayout &L, int block_warps);
// `carveout`: shared-memory carve-out in percent for this launch, -1 = the driver's default;
// `reg_cap`: 1 selects the kernel build limited to 168 registers (three 4-warp CTAs per SM).
cudaError_t launch_lane_ref(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s);
int lane_ref_occupancy(int block_warps, size_t smem, int reg_cap);
// Fast-mode instantiation (kernel_lane_fast.cu), same shared-memory layout.
cudaError_t launch_lane_fast(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s);
int lane_fast_occupancy(int block_warps, size_t smem, int reg_cap);
// FP32 images (round to nearest) of n rate constants, for fast mode.
cudaError_t launch_params_to_f32(const double *in, float *out, long long n, cudaStream_t s);
// Multi-network persistent instantiations (model read from global memory;
// workspace sized for the largest network, no model staged in shared memory).
size_t lane_multi_smem_bytes(int max_N, int max_M, int block_warps);
cudaError_t launch_lane_multi_ref(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s);
int lane_multi_ref_occupancy(int block_warps, size_t smem, int reg_cap);
cudaError_t launch_lane_multi_fast(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap, cudaStream_t s);
int lane_multi_fast_occupancy(int block_warps, size_t smem, int reg_cap);

// ssa_simulate_multi_dev with optional per-group completion signals
// (abi.cu): group g counts its finished simulations in done_counts[g]
// (device memory, zeroed by the caller on `stream`) and its last simulation
// sets done_flags[g] (host-mapped) to 1.  Both may be null.
int simulate_multi_impl(int32_t n_groups, const ssa_group *groups, const ssa_options *opts, void *stream,
                        unsigned long long *done_counts, volatile int32_t *done_flags);

// Sweep moments (moments.cu): mean[c] and unbiased var[c] of every cell c =
// k*N + i from the exact integer sums accumulated by the lane kernels.
cudaError_t launch_moments_finalize(const unsigned long long *acc, long long n, int cells, double *mean, double *var,
                                    cudaStream_t s);

// Reaction-rate equations, one warp per system (kernel_rre.cu): states
// out[n][S][N] (double) at the sample times; stats as for simulations (leaps
// = accepted steps, rejected = rejected steps).
cudaError_t launch_rre(const ModelLayout &L, const int32_t *blob, int64_t n_sims, const double *params,
                       const int32_t *x0, const double *T, int32_t S, double rtol, double atol, int64_t max_steps,
                       double *out, ssa_sim_stats *stats, unsigned long long *counter, cudaStream_t s);
size_t rre_smem_bytes(const ModelLayout &L);

// Warp-per-simulation FP64 reference kernel (kernel_warp_f64.cu).
size_t warp_f64_smem_bytes(const ModelLayout &L, int block_warps);
cudaError_t launch_warp_ref(const SimArgs &a, int block_warps, int grid, size_t smem, cudaStream_t s);
int warp_ref_occupancy(int block_warps, size_t smem);

}  // namespace tl

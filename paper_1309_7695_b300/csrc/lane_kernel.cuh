// Lane-per-simulation kernel template (see kernel_lane_f64.cu for the FP64
// reference instantiation and kernel_lane_fast.cu for fast mode).
//
// Each lane of a warp owns one simulation (the paper's one thread per
// simulation, Methods, last paragraph) for its exact SSA steps.  An SSA step
// is mostly scalar work (ln u, tau = E/a0, a tree descent), so giving every
// lane its own simulation keeps all 32 FP64 lanes busy instead of repeating
// the same scalar on 32 lanes.  The step-size selection and the leaps,
// which are O(M + N) vector work, run warp-cooperatively for one
// simulation at a time.
//
// Per-simulation state in shared memory, one column per lane (row stride 33,
// so both lane-local rows and one-column-across-lanes accesses are free of
// bank conflicts):
//   X [N][33]  int32   molecule counts
//   V [63][33] double  the 32-slot tree of the propensities: nodes 0..31 are
//                      the slot sums S_l = sum_c a_{32c+l} (increasing c),
//                      level k nodes c < 32>>k are V_k[c] = V_{k-1}[c] +
//                      V_{k-1}[c + (32>>k)], node 62 is a0.
// After an SSA firing only the slots holding a reaction whose reactants
// changed, and their ancestors, are recomputed; every node is always the sum
// of its two children in the same order, so the tree equals a full
// recomputation bit for bit.
//
// Per-lane control state (registers), a small state machine:
//   NEED -> (take the next simulation index)  -> TOP
//   TOP  -> (cooperative: record samples, propensities, critical set, a0c,
//            tau'; then an SSA block, or one leap attempt and its retries)
//        -> SSA | TOP | DONE
//   SSA  -> (lane-local: one SSA step per warp iteration) -> SSA | TOP | DONE
//   DONE -> (record the remaining samples, write the counters) -> NEED
// In exact-SSA mode TOP is lane-local too.
//
// The arithmetic policy `Arith` supplies the mode-dependent operations:
//   prop(info, c, X, stride, col)  propensity of one reaction (as double)
//   uniforms(seed, sim, attempt, purpose, u_a, u_b)   two uniforms of a block
//   neglog(u)                       -ln u
//   tau_of(E, a)                    E / a (time to the next event)
//   mean(a, tau)                    the Poisson mean a tau of a leap
//   inv_certain(lam, stream)        k of the inversion draw when decided
//                                   cheaply, else -1 (then inversion())
//   inversion(lam, stream, inv)     k ~ Poisson(lam) for 0 < lam < 10
//   ptrs(lam, stream, work)         k ~ Poisson(lam) for lam >= 10 (work: optional
//                                   iteration / acceptance-test counts)
// Everything else -- the slot tree and its order, the critical set, tau',
// the control flow and counters -- is shared and runs in FP64, except that
// decisions whose FP64 operands only feed a comparison (the SSA-fallback
// test, whether tau'' can be the step) are first taken in FP32 with a
// margin that certifies the canonical outcome.  Recorded states go to the
// trajectory array and/or the sweep-moment sums (record_count).
#pragma once

#include <climits>
#include <type_traits>

#include "device_f64.cuh"
#include "engine.h"
#include "warp_f64.cuh"

namespace tl {
namespace lane {

constexpr int kStride = 33;
constexpr int kNodes = 63;

// Repeated visits of long simulations.  The cooperative part of a warp
// iteration visits every lane in TOP once, so a simulation that needs many
// leaps advances one leap per iteration while its warp-mates' visits and
// the SSA pass run in between.  A simulation that has already made
// kHeavyLeaps leaps is visited up to kLeapRepeat times in a row instead:
// the warp does the same work in a different order, and the simulations
// that would otherwise be left running alone at the end of a launch are
// further along (one 65,536-simulation batch of the 32 x 64 workload:
// 13-20 s, median about 15 s over 12 launches, instead of 17-21 s).  Each
// simulation's arithmetic and random streams are its own, so results do
// not change.
constexpr int kLeapRepeat = 16;
constexpr long long kHeavyLeaps = 256;

enum : int { P_NEED = 0, P_TOP = 1, P_SSA = 2, P_DONE = 3, P_IDLE = 4 };

__host__ __device__ constexpr int node_base(int k) { return 64 - (64 >> k); }

__host__ __device__ inline size_t r16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline size_t lane_warp_bytes(int N, int M)
{
    return r16(4 * (size_t)kStride * N) + r16(8 * (size_t)kStride * kNodes) + r16(8 * (size_t)M) +
           r16(8 * (size_t)M) + r16(8 * (size_t)N) + r16((size_t)M) + r16((size_t)N) + r16(4 * (size_t)M) +
           r16(8 * (size_t)M) + r16(4 * (size_t)M) + r16(8 * (size_t)N);
}

struct LaneSmem {
    int *X;
    double *V;
    double *a;
    long long *k;
    long long *xn;
    unsigned char *crit;
    unsigned char *irs;
    unsigned short *jl;   // [2M] reactions queued for inversion ([0, M)) and PTRS ([M, 2M))
    double *c;            // [M] rate constants of the simulation the warp last worked on together
    float *af;            // [M] FP32 image of a_j for noncritical a_j > 0, else 0 (NaN: out of FP32 range)
    float2 *lo;           // [N] certified lower bounds of the species' two tau' terms
};

__device__ __forceinline__ LaneSmem carve_lane(unsigned char *p, int N, int M)
{
    LaneSmem w;
    w.X = reinterpret_cast<int *>(p);
    p += r16(4 * (size_t)kStride * N);
    w.V = reinterpret_cast<double *>(p);
    p += r16(8 * (size_t)kStride * kNodes);
    w.a = reinterpret_cast<double *>(p);
    p += r16(8 * (size_t)M);
    w.k = reinterpret_cast<long long *>(p);
    p += r16(8 * (size_t)M);
    w.xn = reinterpret_cast<long long *>(p);
    p += r16(8 * (size_t)N);
    w.crit = p;
    p += r16((size_t)M);
    w.irs = p;
    p += r16((size_t)N);
    w.jl = reinterpret_cast<unsigned short *>(p);
    p += r16(4 * (size_t)M);
    w.c = reinterpret_cast<double *>(p);
    p += r16(8 * (size_t)M);
    w.af = reinterpret_cast<float *>(p);
    p += r16(4 * (size_t)M);
    w.lo = reinterpret_cast<float2 *>(p);
    return w;
}

constexpr double kDblMax = 1.7976931348623157e308;

// Everything one simulation group needs: network arrays and run arguments.
struct GroupView {
    const int *rinfo, *nu_ptr, *nu_ent, *tr_ptr, *tr_ent, *hor, *dep_ptr, *dep_ent, *cinfo, *dmask;
    int N, M, S;
    double t_end;
    const double *params;
    const float *params_f;   // fast mode: FP32 images of params, or null
    const int32_t *x0;
    const double *T;
    int32_t *samples;
    ssa_sim_stats *stats;
    unsigned long long *moments;
    unsigned long long *hist;
    int hist_lo, hist_width, hist_bins;
    long long sim_offset, n_sims, first;
    uint64_t seed;
    unsigned long long *done_count;
    volatile int32_t *done_flag;
};

// One recorded count of simulation `row`, sample k, species i: stored in the
// trajectory array and/or added to the sweep moments of cell (k, i) (exact
// integer sums: x, and x^2 split at bit 32 so neither word can overflow)
// and/or counted in the cell's histogram bin.
__device__ __forceinline__ void record_count(const GroupView &G, long long row, int k, int i, int x)
{
    if (G.samples) G.samples[((size_t)row * G.S + k) * (size_t)G.N + i] = x;
    if (G.hist) {
        const long long d = (long long)x - G.hist_lo;
        const long long b = d < 0 ? 0 : min(d / G.hist_width + 1, (long long)G.hist_bins + 1);
        atomicAdd(G.hist + ((size_t)k * G.N + i) * (size_t)(G.hist_bins + 2) + (size_t)b, 1ull);
    }
    if (G.moments && x != 0) {
        // adding zero changes no sum: a zero count adds nothing, and a count
        // below 2^16 has no high square word
        unsigned long long *c = G.moments + ((size_t)k * G.N + i) * 3;
        const unsigned long long ux = (unsigned)x, sq = ux * ux;
        atomicAdd(c, ux);
        atomicAdd(c + 1, sq & 0xFFFFFFFFull);
        if (sq >> 32) atomicAdd(c + 2, sq >> 32);
    }
}

__device__ __forceinline__ void view_model(GroupView &G, const int *blob, const ModelLayout &L)
{
    G.rinfo = blob + L.off_rinfo;
    G.nu_ptr = blob + L.off_nu_ptr;
    G.nu_ent = blob + L.off_nu_ent;
    G.tr_ptr = blob + L.off_tr_ptr;
    G.tr_ent = blob + L.off_tr_ent;
    G.hor = blob + L.off_hor;
    G.dep_ptr = blob + L.off_dep_ptr;
    G.dep_ent = blob + L.off_dep_ent;
    G.cinfo = blob + L.off_cinfo;
    G.dmask = blob + L.off_dmask;
    G.N = L.N;
    G.M = L.M;
}

// single-network launch: the model staged in shared memory
__device__ __forceinline__ GroupView view_single(const SimArgs &A, const int *smem_blob)
{
    GroupView G;
    view_model(G, smem_blob, A.L);
    G.S = A.S;
    G.t_end = A.t_end;
    G.params = A.params;
    G.params_f = A.params_f;
    G.x0 = A.x0;
    G.T = A.T;
    G.samples = A.samples;
    G.stats = A.stats;
    G.moments = A.moments;
    G.hist = A.hist;
    G.hist_lo = A.hist_lo;
    G.hist_width = A.hist_width;
    G.hist_bins = A.hist_bins;
    G.sim_offset = A.sim_offset;
    G.n_sims = A.n_sims;
    G.first = 0;
    G.seed = A.seed;
    G.done_count = nullptr;
    G.done_flag = nullptr;
    return G;
}

// multi-network launch: group g read from global memory (L1-cached)
__device__ __forceinline__ GroupView view_group(const GroupArgs *groups, int g)
{
    const GroupArgs &R = groups[g];
    GroupView G;
    view_model(G, R.blob, R.L);
    G.S = R.S;
    G.t_end = R.t_end;
    G.params = R.params;
    G.params_f = R.params_f;
    G.x0 = R.x0;
    G.T = R.T;
    G.samples = R.samples;
    G.stats = R.stats;
    G.moments = nullptr;
    G.hist = nullptr;
    G.hist_lo = G.hist_width = G.hist_bins = 0;
    G.sim_offset = R.sim_offset;
    G.n_sims = R.n_sims;
    G.first = R.first;
    G.seed = R.seed;
    G.done_count = R.done_count;
    G.done_flag = R.done_flag;
    return G;
}

// kRegCap = 0: up to 255 registers per thread (8-warp CTAs allowed);
// kRegCap = 1: compiled for three 4-warp CTAs per SM (at most 168 registers),
// the register budget a launch can choose when shared memory allows the
// extra CTA.  Both compute the same values.
template <class Arith, bool kMulti, int kRegCap>
__global__ void __launch_bounds__(kRegCap ? 128 : 256, kRegCap ? 3 : 1) lane_kernel(const SimArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    int *blob = reinterpret_cast<int *>(smem);
    size_t model_bytes = 0;
    if (!kMulti) {
        for (int i = threadIdx.x; i < A.L.words; i += blockDim.x) blob[i] = A.blob[i];
        model_bytes = model_smem_bytes(A.L);
    }
    double *inv = reinterpret_cast<double *>(smem + model_bytes);
    for (int k = threadIdx.x; k < f64::kInvTable; k += blockDim.x) inv[k] = k ? 1.0 / (double)k : 0.0;
    __syncthreads();
    const size_t inv_bytes = r16((size_t)f64::kInvTable * 8);
    const int wN = kMulti ? A.max_N : A.L.N, wM = kMulti ? A.max_M : A.L.M;
    const LaneSmem w = carve_lane(smem + model_bytes + inv_bytes + (size_t)warp * lane_warp_bytes(wN, wM), wN, wM);
    int *const X = w.X;
    double *const V = w.V;
    GroupView G0;
    if (!kMulti) G0 = view_single(A, blob);
    auto gview = [&](int g) -> GroupView { return kMulti ? view_group(A.groups, g) : G0; };
    const long long total = kMulti ? A.total_sims : A.n_sims;
    const bool exact = (A.mode == SSA_MODE_EXACT);
    const double kInf = __longlong_as_double(0x7FF0000000000000ll);

    // this lane's simulation: group grp, row within the group
    int grp = 0;
    long long row = -1;
    uint32_t sim = 0;
    double t = 0.0;
    int ks = 0;
    uint32_t attempt = 0;
    int status = SSA_STATUS_OK;
    int phase = P_NEED;
    int ssa_left = 0;
    int first = 0;
    long long leaps = 0, rejected = 0, ssa_steps = 0, firings = 0;
    double tnext = kInf;   // T[ks], or +inf once every sample is recorded
    // warp-uniform: the (group, row) whose rate constants are in w.c
    long long c_row = -1;
    int c_grp = -1;
    // FP32 images of eps and ssa_factor for the certified bounds (a factor
    // above 1e30 leaves every SSA-fallback test to FP64)
    const float epsf = f64::f64_to_f32(A.eps);
    const float ssaf = f64::f64_to_f32(A.ssa_factor);
    const bool ssaf_ok = f64::nn_ge(1e30, A.ssa_factor);

    // FP32 rate constant of this lane's simulation (fast mode): the staged
    // image, or the RN conversion of the FP64 constant (the same value)
    auto own_cf = [&](const GroupView &G, int j) -> float {
        return G.params_f ? __ldg(G.params_f + (size_t)row * G.M + j)
                          : f64::f64_to_f32(__ldg(G.params + (size_t)row * G.M + j));
    };
    auto own_prop = [&](const GroupView &G, int j) -> double {
        if constexpr (Arith::kFloatSlots)
            return f64::f32_to_f64(Arith::prop_f(G.rinfo[j], own_cf(G, j), X, kStride, lane));
        return Arith::prop(G.rinfo[j], __ldg(G.params + (size_t)row * G.M + j), X, kStride, lane);
    };
    // Slot sum of this lane's simulation, S_l = sum over j = l, l+32, ... of
    // a_j in increasing j (the canonical order).  Up to four reactions per
    // slot (M <= 128) their rate constants are loaded together before the
    // first is used, so the global-memory latency is paid once per slot.
    auto own_slot_sum = [&](const GroupView &G, int l) -> double {
        const int M = G.M;
        if constexpr (Arith::kFloatSlots) {
            // fast mode: the slot's FP32 propensities summed in FP32, promoted once
            float sf = Arith::prop_f(G.rinfo[l], own_cf(G, l), X, kStride, lane);
            for (int j = l + 32; j < M; j += 32) sf = sf + Arith::prop_f(G.rinfo[j], own_cf(G, j), X, kStride, lane);
            return f64::first_term(f64::f32_to_f64(sf));
        }
        const double *c = G.params + (size_t)row * G.M;
        if (M <= 128) {
            const double c0 = __ldg(c + l);
            const double c1 = (l + 32 < M) ? __ldg(c + l + 32) : 0.0;
            const double c2 = (l + 64 < M) ? __ldg(c + l + 64) : 0.0;
            const double c3 = (l + 96 < M) ? __ldg(c + l + 96) : 0.0;
            double s = f64::first_term(Arith::prop(G.rinfo[l], c0, X, kStride, lane));
            if (l + 32 < M) s = s + Arith::prop(G.rinfo[l + 32], c1, X, kStride, lane);
            if (l + 64 < M) s = s + Arith::prop(G.rinfo[l + 64], c2, X, kStride, lane);
            if (l + 96 < M) s = s + Arith::prop(G.rinfo[l + 96], c3, X, kStride, lane);
            return s;
        }
        double s = f64::first_term(own_prop(G, l));
        for (int j = l + 32; j < M; j += 32) s = s + own_prop(G, j);
        return s;
    };
    // The SSA step's propensity arithmetic: FP64 in the reference mode, FP32
    // (with FP32 rate constants, and slot sums promoted to FP64 once) in fast mode
    using acc_t = typename std::conditional<Arith::kFloatSlots, float, double>::type;
    auto load_c = [&](const GroupView &G, int j) -> acc_t {
        if constexpr (Arith::kFloatSlots) return own_cf(G, j);
        else return __ldg(G.params + (size_t)row * G.M + j);
    };
    auto prop_c = [&](int info, acc_t c) -> acc_t {
        if constexpr (Arith::kFloatSlots) return Arith::prop_f(info, c, X, kStride, lane);
        else return Arith::prop(info, c, X, kStride, lane);
    };
    auto to_f64 = [](acc_t v) -> double {
        if constexpr (Arith::kFloatSlots) return f64::f32_to_f64(v);
        else return v;
    };
    auto first_acc = [](acc_t v) -> acc_t {   // +0 + v: the sign of a zero cleared
        if constexpr (Arith::kFloatSlots) return __int_as_float(__float_as_int(v) & 0x7fffffff);
        else return f64::first_term(v);
    };
    auto lane_record = [&](const GroupView &G, int k) {
        for (int i = 0; i < G.N; ++i) record_count(G, row, k, i, X[i * kStride + lane]);
    };
    auto lane_build_tree = [&](const GroupView &G) {
        for (int l = 0; l < 32; ++l) {
            double s = (l < G.M) ? f64::first_term(own_prop(G, l)) : 0.0;
            for (int j = l + 32; j < G.M; j += 32) s = s + own_prop(G, j);
            V[l * kStride + lane] = s;
        }
        for (int k = 1; k <= 5; ++k) {
            const int width = 32 >> k;
            for (int c = 0; c < width; ++c)
                V[(node_base(k) + c) * kStride + lane] =
                    V[(node_base(k - 1) + c) * kStride + lane] + V[(node_base(k - 1) + c + width) * kStride + lane];
        }
    };

    for (;;) {
        // ---- hand out simulation indices to lanes that need one
        if (phase == P_NEED && lane >= A.sims_per_warp) phase = P_IDLE;   // lanes without a simulation slot
        const unsigned need = __ballot_sync(kFull, phase == P_NEED);
        if (need) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(A.work_counter, (unsigned long long)__popc(need));
            base = __shfl_sync(kFull, base, 0);
            if (phase == P_NEED) {
                const unsigned long long r = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                if (r < (unsigned long long)total) {
                    if (kMulti) {
                        int g = 0;
                        while (g + 1 < A.n_groups && (long long)r >= A.groups[g + 1].first) ++g;
                        grp = g;
                    }
                    const GroupView G = gview(grp);
                    const int N = G.N, S = G.S;
                    const double *T = G.T;
                    row = (long long)r - G.first;
                    sim = (uint32_t)(G.sim_offset + row);
                    t = 0.0;
                    ks = 0;
                    attempt = 0;
                    status = SSA_STATUS_OK;
                    leaps = rejected = ssa_steps = firings = 0;
                    tnext = (S > 0) ? T[0] : kInf;
                    for (int i = 0; i < N; ++i) X[i * kStride + lane] = G.x0[(size_t)row * N + i];
                    if (exact) lane_build_tree(G);
                    phase = P_TOP;
                } else {
                    row = -1;
                    phase = P_IDLE;
                }
            }
        }
        if (__all_sync(kFull, phase == P_IDLE)) break;
        __syncwarp();

        // ---- cooperative top of the loop, one simulation at a time
        if (!exact) {
            unsigned todo = __ballot_sync(kFull, phase == P_TOP);
            int again = 0;   // warp-uniform: repeated visits of the current lane so far
            while (todo) {
                const int L = __ffs(todo) - 1;
                todo &= todo - 1;
                const GroupView GL = gview(__shfl_sync(kFull, grp, L));
                const int *rinfo = GL.rinfo, *tr_ptr = GL.tr_ptr, *tr_ent = GL.tr_ent, *hor = GL.hor;
                const int N = GL.N, M = GL.M, S = GL.S;
                const double *T = GL.T;
                const double t_end = GL.t_end;
                const long long rL = __shfl_sync(kFull, row, L);
                const uint32_t sL = __shfl_sync(kFull, sim, L);
                double tL = __shfl_sync(kFull, t, L);
                int ksL = __shfl_sync(kFull, ks, L);
                uint32_t attL = __shfl_sync(kFull, attempt, L);
                long long lpL = __shfl_sync(kFull, leaps, L);
                long long rjL = __shfl_sync(kFull, rejected, L);
                const long long fi0 = __shfl_sync(kFull, firings, L);
                long long fiL = fi0;
                int stL = SSA_STATUS_OK;
                int nphase = P_TOP, nleft = 0, nfirst = 0;
                // rate constants of simulation L, cached per warp in shared memory: a
                // long simulation's consecutive leaps read them from there
                const int gL = kMulti ? __shfl_sync(kFull, grp, L) : 0;
                if (rL != c_row || gL != c_grp) {
                    const double *cL = GL.params + (size_t)rL * M;
                    for (int j = lane; j < M; j += 32) w.c[j] = __ldg(cL + j);
                    c_row = rL;
                    c_grp = gL;
                }

                double tnL = __shfl_sync(kFull, tnext, L);
                while (ksL < S && tnL <= tL) {
                    for (int i = lane; i < N; i += 32) record_count(GL, rL, ksL, i, X[i * kStride + L]);
                    ++ksL;
                    tnL = (ksL < S) ? T[ksL] : kInf;
                }
                if (tL >= t_end) {
                    nphase = P_DONE;
                } else if ((long long)attL >= A.max_attempts) {
                    stL = SSA_STATUS_STEP_LIMIT;
                    nphase = P_DONE;
                } else {
                    // The Philox blocks of this visit's first leap attempt depend only on
                    // (simulation, attempt, reaction): drawn here, the three independent
                    // chains (the leap's block and block 0 of the Poisson streams of this
                    // lane's first two reactions) run together, off the leap's path.
                    const uint32_t att1 = attL + 1;
                    const uint4 w_leap1 = f64::draw(GL.seed, sL, att1, PURPOSE_LEAP, 0, 0);
                    const uint4 w_pois1a = f64::draw(GL.seed, sL, att1, PURPOSE_POISSON, (uint32_t)lane, 0);
                    const uint4 w_pois1b = f64::draw(GL.seed, sL, att1, PURPOSE_POISSON, (uint32_t)(lane + 32), 0);
                    // One pass over this lane's reactions j = lane, lane + 32, ...: the
                    // propensity and its slot sum, the critical test (CGP 2005: L_j = min
                    // over the species j consumes of floor(x_i / |nu_ij|), from the packed
                    // consumed-species word), the FP32 image of a noncritical positive
                    // propensity for the tau' bounds (NaN outside the range they are
                    // proved for), and the reactant species of the noncritical reactions
                    // (I_rs).  The results are used only when a0 turns out positive.
                    const int *cinfo = GL.cinfo;
                    for (int i = lane; i < N; i += 32) w.irs[i] = 0;
                    __syncwarp();
                    bool any_crit = false;
                    int n_crit = 0;   // this lane's critical reactions (work counters only)
                    auto reaction = [&](int j) -> double {
                        const int info = rinfo[j];
                        const double a = Arith::prop(info, w.c[j], X, kStride, L);
                        w.a[j] = a;
                        const unsigned ci = (unsigned)cinfo[j];
                        const unsigned na = (ci >> 14) & 3u, nb = ci >> 30;
                        const int xa = X[(ci & 0x3fffu) * kStride + L];
                        const int xb = X[((ci >> 16) & 0x3fffu) * kStride + L];
                        int Lj = INT_MAX;
                        if (na) Lj = (na == 1) ? xa : (xa >> 1);
                        if (nb) Lj = min(Lj, (nb == 1) ? xb : (xb >> 1));
                        const bool cr = f64::nn_pos(a) && (Lj < A.n_c);
                        w.crit[j] = cr;
                        any_crit |= cr;
                        n_crit += cr;
                        float af = 0.0f;
                        if (!cr) {
                            if (f64::nn_pos(a)) {
                                const int ea = (int)(f64::dbits(a) >> 52);
                                af = (ea >= 1023 - 100 && ea <= 1023 + 100) ? f64::f64_to_f32(a)
                                                                           : __int_as_float(0x7fc00000);
                            }
                            const int kind = info & 3;
                            if (kind >= 1) w.irs[(info >> 2) & 0x7fff] = 1;
                            if (kind == 2) w.irs[(info >> 17) & 0x7fff] = 1;
                        }
                        w.af[j] = af;
                        return a;
                    };
                    double s = 0.0;
                    if (lane < M) s = f64::first_term(reaction(lane));   // first term of the slot sum (no add to +0)
                    for (int j = lane + 32; j < M; j += 32) s = s + reaction(j);
                    double Lv[6];
                    const double a0 = slot_tree(s, Lv);
#pragma unroll
                    for (int k = 0; k <= 5; ++k)
                        if (lane < (32 >> k)) V[(node_base(k) + lane) * kStride + L] = Lv[k];
                    __syncwarp();
                    if (a0 == 0.0) {
                        tL = t_end;
                        nphase = P_DONE;
                    } else if (!(a0 <= kDblMax)) {
                        stL = SSA_STATUS_INVALID;
                        nphase = P_DONE;
                    } else {
                        any_crit = __any_sync(kFull, any_crit);
                        if (A.work) n_crit = __reduce_add_sync(kFull, (unsigned)n_crit);
                        // Certified FP32 bounds on every tau' term (CGP 2006).  mu and sigma^2
                        // summed in FP32 from the FP32 images of the a_j are within
                        // (n + 4) 2^-20 of the sum of |nu a| of the exact sums (n terms), and
                        // bound = max(eps x / g, 1) within 2^-20 relative; each bound below
                        // carries a further 1e-4.  A term whose mu is not certainly nonzero
                        // gets the upper bound +inf.  From these:
                        //  - the SSA-fallback decision "tau' < ssa_factor / a0" is certain when
                        //    the smallest upper bound lies below a lower bound of the threshold;
                        //  - otherwise tau' = the smallest exact term, and only terms whose lower
                        //    bound does not exceed the smallest upper bound can be that term, so
                        //    only those are computed in FP64 (in the canonical operations).
                        const float kNoTerm = __int_as_float(0x7fc00000);   // NaN: never a candidate
                        unsigned hmin = 0x7F800000u;                          // +inf as float bits
                        unsigned n_terms = 0, n_species = 0;                  // work counters
                        for (int i = lane; i < N; i += 32) {
                            float2 lo = make_float2(kNoTerm, kNoTerm);
                            if (w.irs[i]) {
                                float muf = 0.0f, s2f = 0.0f, absf = 0.0f;
                                int n = 0;
                                for (int e = tr_ptr[i]; e < tr_ptr[i + 1]; ++e) {
                                    const int ent = tr_ent[e];
                                    const float af = w.af[ent >> 8];
                                    if (af == 0.0f) continue;
                                    const float nvf = (float)(signed char)(ent & 0xff);
                                    muf = muf + nvf * af;
                                    s2f = s2f + (nvf * nvf) * af;
                                    absf = absf + fabsf(nvf) * af;
                                    ++n;
                                }
                                if (n > 0) {
                                    n_terms += n;
                                    n_species += 1;
                                    const int xi = X[i * kStride + L];
                                    const float xf = (float)xi;
                                    const int h = hor[i];
                                    float bf = epsf * xf;
                                    if (h == 2 || (h != 1 && xi < 2)) bf = bf * 0.5f;
                                    else if (h != 1) bf = bf / (2.0f + 1.0f / (xf - 1.0f));
                                    bf = fmaxf(bf, 1.0f);
                                    const float b_hi = bf * (1.0f + 0x1p-20f), b_lo = bf * (1.0f - 0x1p-20f);
                                    const float rel = (float)(n + 4) * 0x1p-20f;
                                    const float err = rel * absf;
                                    const float amu = fabsf(muf);
                                    // term 1: bound / |mu|
                                    float lo1 = (b_lo / (amu + err)) * (1.0f - 1e-4f);
                                    float hi1 = (amu > err) ? (b_hi / (amu - err)) * (1.0f + 1e-4f) : __int_as_float(0x7F800000);
                                    // term 2: bound^2 / sigma^2 (all terms positive: no cancellation)
                                    float lo2 = ((b_lo * b_lo) / (s2f * (1.0f + rel))) * (1.0f - 2e-4f);
                                    float hi2 = ((b_hi * b_hi) / (s2f * (1.0f - rel))) * (1.0f + 2e-4f);
                                    // outside the proved range (NaN inputs, overflow, underflow):
                                    // always a candidate, never an upper bound
                                    if (!(lo1 >= 0x1p-120f && hi1 <= 0x1p120f)) {
                                        lo1 = 0.0f;
                                        hi1 = __int_as_float(0x7F800000);
                                    }
                                    if (!(lo2 >= 0x1p-120f && hi2 <= 0x1p120f)) {
                                        lo2 = 0.0f;
                                        hi2 = __int_as_float(0x7F800000);
                                    }
                                    lo = make_float2(lo1, lo2);
                                    hmin = min(hmin, min(__float_as_uint(hi1), __float_as_uint(hi2)));
                                }
                            }
                            w.lo[i] = lo;
                        }
                        hmin = __reduce_min_sync(kFull, hmin);
                        const float tau1_hi = __uint_as_float(hmin);
                        if (A.work) {
                            n_terms = __reduce_add_sync(kFull, n_terms);
                            n_species = __reduce_add_sync(kFull, n_species);
                            if (lane == 0) {
                                atomicAdd(A.work + SSA_WORK_SELECTIONS, 1ull);
                                atomicAdd(A.work + SSA_WORK_TAU_TERMS, (unsigned long long)n_terms);
                                atomicAdd(A.work + SSA_WORK_TAU_SPECIES, (unsigned long long)n_species);
                            }
                        }
                        // the threshold ssa_factor / a0 in FP32, and whether its image is trusted
                        const int e0 = (int)(f64::dbits(a0) >> 52);
                        const bool thr_ok = ssaf_ok && (e0 >= 1023 - 100 && e0 <= 1023 + 100);
                        const float thr_f = ssaf / f64::f64_to_f32(a0);
                        const float thr_lo = thr_f * (1.0f - 1e-5f), thr_hi = thr_f * (1.0f + 1e-5f);
                        if (thr_ok && tau1_hi < thr_lo) {
                            nphase = P_SSA;
                            nleft = A.ssa_block;
                            nfirst = 1;
                        } else {
                        // tau' exactly: the canonical FP64 terms of the candidate species
                        unsigned long long tmin = 0x7FF0000000000000ull;
                        for (int i = lane; i < N; i += 32) {
                            const float2 lo = w.lo[i];
                            const bool need1 = lo.x <= tau1_hi, need2 = lo.y <= tau1_hi;
                            if (!(need1 || need2)) continue;
                            double mu = 0.0, sig2 = 0.0;
                            for (int e = tr_ptr[i]; e < tr_ptr[i + 1]; ++e) {
                                const int ent = tr_ent[e];
                                const int j = ent >> 8;
                                // af[j] is 0 exactly when j is critical or a_j is not positive
                                // (an out-of-range a_j has a NaN image): the canonical terms
                                const float af = w.af[j];
                                const double a = w.a[j];
                                if (af == 0.0f) continue;
                                const int nv = (signed char)(ent & 0xff);
                                // nu a and nu^2 a: for |nu| <= 2 exact power-of-two scalings and a
                                // sign flip (exponent arithmetic on a > 0, normal, far from
                                // overflow), else the FP64 products; same values either way
                                const long long ab = f64::dbits(a);
                                const int ea = (int)(ab >> 52);
                                const int an = nv < 0 ? -nv : nv;
                                double tm, ts;
                                if (an <= 2 && ea >= 1 && ea <= 0x7FC) {
                                    const long long two = (an == 2) ? (1ll << 52) : 0ll;
                                    tm = __longlong_as_double((ab + two) | (nv < 0 ? (long long)0x8000000000000000ull : 0ll));
                                    ts = __longlong_as_double(ab + 2 * two);
                                } else {
                                    tm = f64::small_to_double(nv) * a;
                                    ts = f64::count_to_double(nv * nv) * a;
                                }
                                mu = mu + tm;
                                sig2 = sig2 + ts;
                            }
                            const int xi = X[i * kStride + L];
                            const double xd = f64::count_to_double(xi);
                            // bound = (eps x_i) / g_i; dividing by g = 1 or 2 is exact, so
                            // those cases multiply (same value, no division)
                            const int h = hor[i];
                            const double ex = A.eps * xd;
                            double bound;
                            if (h == 1) bound = ex;
                            else if (h == 2 || xi < 2) bound = ex * 0.5;
                            else bound = ex / (2.0 + 1.0 / (xd - 1.0));
                            if (f64::dbits(bound) < f64::dbits(1.0)) bound = 1.0;
                            if (need1 && (f64::dbits(mu) << 1) != 0) {   // mu != 0
                                const unsigned long long b1 =
                                    (unsigned long long)__double_as_longlong(bound / fabs(mu));
                                tmin = b1 < tmin ? b1 : tmin;
                            }
                            if (need2 && f64::nn_pos(sig2)) {   // sig2 >= 0; != 0
                                const unsigned long long b2 =
                                    (unsigned long long)__double_as_longlong((bound * bound) / sig2);
                                tmin = b2 < tmin ? b2 : tmin;
                            }
                        }
                        double tau1 = __longlong_as_double((long long)warp_min_u64(tmin));
                        // a0c (the canonical sum of the critical propensities), needed only
                        // when a critical reaction exists; otherwise it is +0
                        double Lc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                        double a0c = 0.0;
                        if (any_crit) {
                            double sc = 0.0;
                            bool sc_started = false;   // the first critical term is taken, not added to +0
                            for (int j = lane; j < M; j += 32) {
                                if (!w.crit[j]) continue;
                                const double a = w.a[j];   // > 0
                                if (sc_started) sc = sc + a;
                                else sc = a;
                                sc_started = true;
                            }
                            a0c = slot_tree(sc, Lc);
                        }
                        // the SSA-fallback test tau' < ssa_factor / a0: decided on the FP32
                        // images when they are clear of the threshold's margin, else by the
                        // FP64 division (formed once)
                        double ssa_thr = 0.0;
                        bool thr_ready = false;
                        auto below_threshold = [&](double tau) -> bool {
                            const int et = (int)(f64::dbits(tau) >> 52);   // tau > 0
                            if (thr_ok && et >= 1023 - 120 && et <= 1023 + 120) {
                                const float tf = f64::f64_to_f32(tau);
                                if (tf < thr_lo) return true;
                                if (tf > thr_hi) return false;
                            }
                            if (!thr_ready) {
                                ssa_thr = A.ssa_factor / a0;
                                thr_ready = true;
                            }
                            return tau < ssa_thr;
                        };

                        int halvings = 0;
                        for (;;) {
                            if (below_threshold(tau1)) {
                                nphase = P_SSA;
                                nleft = A.ssa_block;
                                nfirst = 1;
                                break;
                            }
                            if ((long long)attL >= A.max_attempts) {
                                stL = SSA_STATUS_STEP_LIMIT;
                                nphase = P_DONE;
                                break;
                            }
                            attL = attL + 1;
                            double u_tau, u_sel;
                            if (attL == att1) Arith::uniforms_of(w_leap1, u_tau, u_sel);
                            else Arith::uniforms(GL.seed, sL, attL, PURPOSE_LEAP, u_tau, u_sel);
                            const double t_stop = (ksL < S) ? tnL : t_end;
                            const double delta = t_stop - tL;
                            // tau'' matters only if it can be the smallest of tau'', tau' and
                            // delta; when a certified FP32 lower bound says it cannot, +inf
                            // stands in for it in the comparisons below
                            double tau2 = kInf;
                            if (f64::nn_pos(a0c)) {
                                const double m = f64::nn_ge(delta, tau1) ? tau1 : delta;
                                if (!f64::tau2_surely_later(u_tau, a0c, m))
                                    tau2 = Arith::tau_of(Arith::neglog(u_tau), a0c);
                            }
                            double tau;
                            int jc = -1;
                            bool clamp = false;
                            // tau2, tau1 and delta are positive (or +inf): compare bit patterns
                            if (f64::nn_ge(tau1, tau2) && f64::nn_ge(delta, tau2)) {
                                tau = tau2;
                                jc = slot_select(Lc, u_sel * a0c, w.a, w.crit, true, M);
                            } else if (f64::nn_ge(tau1, delta)) {
                                tau = delta;
                                clamp = true;
                            } else {
                                tau = tau1;
                            }
                            // Poisson counts of the noncritical reactions.  A first pass
                            // forms the means and settles what it can (critical reactions,
                            // zero means, inversion draws decided in FP32 with a certified
                            // margin); the rest are queued by sampler and drawn in two
                            // compacted passes, so a warp runs each sampler once per 32
                            // queued draws instead of branching over both for every
                            // reaction.  Each draw depends only on its own mean and stream,
                            // so the order is free.
                            int krej = 0, kover = 0;
                            long long ksum = 0;
                            int n_inv = 0, n_ptrs = 0;
                            unsigned w_inv = 0, w_inv_terms = 0;   // work counters
                            const unsigned lt = (1u << lane) - 1u;
                            for (int j0 = 0; j0 < M; j0 += 32) {
                                const int j = j0 + lane;
                                int cls = 0;   // 0 settled, 1 inversion, 2 PTRS
                                if (j < M) {
                                    long long kj = 0;
                                    if (w.crit[j]) {
                                        kj = (j == jc) ? 1 : 0;
                                    } else {
                                        // a_j >= 0 and tau is finite and positive, so lam is a
                                        // finite non-negative double and compares by its bits
                                        const double lam = Arith::mean(w.a[j], tau);
                                        if (f64::nn_pos(lam)) {
                                            if (f64::dbits(lam) >= f64::dbits(0x1p40)) {
                                                kj = f64::kCountLimit + 1;
                                                kover = 1;
                                            } else if (f64::dbits(lam) < f64::dbits(10.0)) {
                                                const int kc =
                                                    (attL == att1 && j0 < 64)
                                                        ? Arith::inv_certain_of(lam, j0 == 0 ? w_pois1a : w_pois1b)
                                                        : Arith::inv_certain(lam, GL.seed, sL, attL, (uint32_t)j);
                                                w_inv += 1;
                                                if (kc >= 0) {
                                                    kj = kc;
                                                    w_inv_terms += (unsigned)kc;
                                                } else {
                                                    cls = 1;
                                                }
                                            } else {
                                                cls = 2;
                                            }
                                            if (cls) kj = __double_as_longlong(lam);   // mean parked until drawn
                                        }
                                    }
                                    w.k[j] = kj;
                                    if (!cls) ksum += kj;
                                }
                                const unsigned bi = __ballot_sync(kFull, cls == 1);
                                const unsigned bp = __ballot_sync(kFull, cls == 2);
                                if (cls == 1) w.jl[n_inv + __popc(bi & lt)] = (unsigned short)j;
                                if (cls == 2) w.jl[M + n_ptrs + __popc(bp & lt)] = (unsigned short)j;
                                n_inv += __popc(bi);
                                n_ptrs += __popc(bp);
                            }
                            __syncwarp();
                            for (int q = lane; q < n_inv; q += 32) {
                                const int j = w.jl[q];
                                const long long kj =
                                    Arith::inversion(__longlong_as_double(w.k[j]), GL.seed, sL, attL, (uint32_t)j, inv);
                                w.k[j] = kj;
                                ksum += kj;
                                w_inv_terms += (unsigned)kj;
                            }
                            unsigned w_ptrs[2] = {0u, 0u};   // PTRS iterations, acceptance tests
                            for (int q = lane; q < n_ptrs; q += 32) {
                                const int j = w.jl[M + q];
                                const double lam = __longlong_as_double(w.k[j]);
                                const long long kj = (A.mode == SSA_MODE_CLE && f64::nn_ge(lam, f64::kCleMinMean))
                                                         ? f64::normal_leap(lam, GL.seed, sL, attL, (uint32_t)j)
                                                         : Arith::ptrs(lam, GL.seed, sL, attL, (uint32_t)j,
                                                                       A.work ? w_ptrs : nullptr);
                                if (kj < 0) krej = 1;
                                else if (kj > f64::kCountLimit) kover = 1;
                                w.k[j] = kj;
                                ksum += kj;
                            }
                            if (A.work) {
                                w_inv = __reduce_add_sync(kFull, w_inv);
                                w_inv_terms = __reduce_add_sync(kFull, w_inv_terms);
                                w_ptrs[0] = __reduce_add_sync(kFull, w_ptrs[0]);
                                w_ptrs[1] = __reduce_add_sync(kFull, w_ptrs[1]);
                                if (lane == 0) {
                                    if (f64::nn_pos(a0c)) atomicAdd(A.work + SSA_WORK_TAU2, 1ull);
                                    atomicAdd(A.work + SSA_WORK_MEANS, (unsigned long long)(M - n_crit));
                                    atomicAdd(A.work + SSA_WORK_INV_DRAWS, (unsigned long long)w_inv);
                                    atomicAdd(A.work + SSA_WORK_INV_TERMS, (unsigned long long)w_inv_terms);
                                    atomicAdd(A.work + SSA_WORK_PTRS_DRAWS, (unsigned long long)n_ptrs);
                                    atomicAdd(A.work + SSA_WORK_PTRS_ITERS, (unsigned long long)w_ptrs[0]);
                                    atomicAdd(A.work + SSA_WORK_PTRS_TESTS, (unsigned long long)w_ptrs[1]);
                                }
                            }
                            if (__any_sync(kFull, krej)) {
                                stL = SSA_STATUS_REJECT_LIMIT;
                                nphase = P_DONE;
                                break;
                            }
                            if (__any_sync(kFull, kover)) {
                                stL = SSA_STATUS_OVERFLOW;
                                nphase = P_DONE;
                                break;
                            }
                            __syncwarp();
                            int neg = 0, big = 0;
                            for (int i = lane; i < N; i += 32) {
                                long long xn = X[i * kStride + L];
                                for (int e = tr_ptr[i]; e < tr_ptr[i + 1]; ++e) {
                                    const int ent = tr_ent[e];
                                    xn += w.k[ent >> 8] * (long long)(signed char)(ent & 0xff);
                                }
                                w.xn[i] = xn;
                                neg |= (xn < 0);
                                big |= (xn > INT_MAX);
                            }
                            if (__any_sync(kFull, neg)) {
                                rjL += 1;
                                halvings += 1;
                                if (halvings > A.max_halvings) {
                                    stL = SSA_STATUS_REJECT_LIMIT;
                                    nphase = P_DONE;
                                    break;
                                }
                                tau1 = tau1 / 2.0;
                                continue;
                            }
                            if (__any_sync(kFull, big)) {
                                stL = SSA_STATUS_OVERFLOW;
                                nphase = P_DONE;
                                break;
                            }
                            for (int i = lane; i < N; i += 32) X[i * kStride + L] = (int)w.xn[i];
                            fiL += warp_sum_counts(ksum);
                            tL = clamp ? t_stop : tL + tau;
                            lpL += 1;
                            break;
                        }
                        }   // not certain_ssa
                    }
                }
                __syncwarp();
                if (lane == L) {
                    t = tL;
                    ks = ksL;
                    tnext = tnL;
                    attempt = attL;
                    status = stL;
                    leaps = lpL;
                    rejected = rjL;
                    firings = fiL;
                    phase = nphase;
                    ssa_left = nleft;
                    first = nfirst;
                }
                if (kLeapRepeat > 1 && nphase == P_TOP && lpL >= kHeavyLeaps && again + 1 < kLeapRepeat) {
                    todo |= 1u << L;   // L was the lowest bit: visited again next
                    ++again;
                } else {
                    again = 0;
                }
            }
            __syncwarp();
        }

        // ---- lane-local part: exact-mode top of the loop
        if (exact && phase == P_TOP) {
            const GroupView G = gview(grp);
            const int S = G.S;
            const double *T = G.T;
            const double t_end = G.t_end;
            while (ks < S && tnext <= t) {
                lane_record(G, ks++);
                tnext = (ks < S) ? T[ks] : kInf;
            }
            if (t >= t_end) {
                phase = P_DONE;
            } else if ((long long)attempt >= A.max_attempts) {
                status = SSA_STATUS_STEP_LIMIT;
                phase = P_DONE;
            } else {
                const double a0 = V[62 * kStride + lane];
                if (a0 == 0.0) {
                    t = t_end;
                    phase = P_DONE;
                } else if (!(a0 <= kDblMax)) {
                    status = SSA_STATUS_INVALID;
                    phase = P_DONE;
                } else {
                    phase = P_SSA;
                    ssa_left = 1;
                    first = 1;
                }
            }
        }

        // ---- lane-local part: one exact SSA step (direct method)
        if (phase == P_SSA) {
            const GroupView G = gview(grp);
            const int *nu_ptr = G.nu_ptr, *nu_ent = G.nu_ent;
            const int M = G.M, S = G.S;
            const double *T = G.T;
            const double t_end = G.t_end;
            if (!first && !f64::nn_gt(t_end, t)) {
                phase = P_TOP;
            } else {
                const double a0 = V[62 * kStride + lane];
                if (f64::dbits(a0) == 0) {
                    t = t_end;
                    phase = P_DONE;
                } else if (f64::dbits(a0) > 0x7FEFFFFFFFFFFFFFll) {
                    status = SSA_STATUS_INVALID;
                    phase = P_DONE;
                } else if ((long long)attempt >= A.max_attempts) {
                    status = SSA_STATUS_STEP_LIMIT;
                    phase = P_DONE;
                } else {
                    attempt = attempt + 1;
                    // -ln u1 and u2 of this attempt.  Every lane in this phase draws in
                    // the same iteration, so the FP64 work of the logarithm is one
                    // converged pass for the whole warp (an FP64 instruction costs the
                    // same however many lanes are active).
                    double u1, u2;
                    Arith::uniforms(G.seed, sim, attempt, PURPOSE_SSA, u1, u2);
                    const double E = Arith::neglog(u1);
                    const double tau = Arith::tau_of(E, a0);
                    const double t_new = t + tau;
                    while (ks < S && !f64::nn_ge(tnext, t_new)) {
                        lane_record(G, ks++);
                        tnext = (ks < S) ? T[ks] : kInf;
                    }
                    if (f64::nn_gt(t_new, t_end)) {
                        t = t_end;
                        phase = P_DONE;
                    } else {
                        // descend the slot tree, then walk the chosen slot
                        double target = u2 * a0;
                        int cls = 0;
#pragma unroll
                        for (int k = 4; k >= 0; --k) {
                            const int step = 1 << (4 - k);
                            const double left = V[(node_base(k) + cls) * kStride + lane];
                            const double right = V[(node_base(k) + cls + step) * kStride + lane];
                            if (f64::nn_ge(target, left) && f64::nn_pos(right)) {
                                target = target - left;
                                cls += step;
                            }
                        }
                        acc_t cum = 0;
                        int jf = -1, last = -1;
                        // walk the slot; the next member's rate constant is loaded one step ahead
                        acc_t cnext = load_c(G, cls);
                        for (int j = cls; j < M; j += 32) {
                            const acc_t cj = cnext;
                            if (j + 32 < M) cnext = load_c(G, j + 32);
                            const acc_t v = prop_c(G.rinfo[j], cj);
                            if (j == cls) cum = first_acc(v);
                            else cum = cum + v;
                            if (f64::nn_pos(to_f64(v))) last = j;
                            if (f64::nn_gt(to_f64(cum), target)) {
                                jf = j;
                                break;
                            }
                        }
                        if (jf < 0) jf = last;
                        if (jf < 0) {
                            status = SSA_STATUS_INVALID;
                            phase = P_DONE;
                        } else {
                            const int e0 = nu_ptr[jf], e1 = nu_ptr[jf + 1];
                            bool over = false;
                            for (int e = e0; e < e1; ++e) {
                                const int ent = nu_ent[e];
                                if ((long long)X[(ent >> 8) * kStride + lane] + (signed char)(ent & 0xff) > INT_MAX)
                                    over = true;
                            }
                            if (over) {
                                status = SSA_STATUS_OVERFLOW;
                                phase = P_DONE;
                            } else {
                                unsigned dirty = (unsigned)G.dmask[jf];
                                for (int e = e0; e < e1; ++e) {
                                    const int ent = nu_ent[e];
                                    X[(ent >> 8) * kStride + lane] += (signed char)(ent & 0xff);
                                }
                                // re-sum the dirty slots (l < M: a dirty slot holds a reaction); up
                                // to four reactions per slot, the next slot's rate constants are
                                // loaded while the current slot is summed
                                unsigned m = dirty;
                                if (m != 0 && M <= 128) {
                                    int l = __ffs(m) - 1;
                                    m &= m - 1;
                                    acc_t c0 = load_c(G, l), c1 = (l + 32 < M) ? load_c(G, l + 32) : acc_t(0);
                                    acc_t c2 = (l + 64 < M) ? load_c(G, l + 64) : acc_t(0);
                                    acc_t c3 = (l + 96 < M) ? load_c(G, l + 96) : acc_t(0);
                                    for (;;) {
                                        const int ln = m ? __ffs(m) - 1 : -1;
                                        m &= m - 1;
                                        acc_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
                                        if (ln >= 0) {
                                            n0 = load_c(G, ln);
                                            if (ln + 32 < M) n1 = load_c(G, ln + 32);
                                            if (ln + 64 < M) n2 = load_c(G, ln + 64);
                                            if (ln + 96 < M) n3 = load_c(G, ln + 96);
                                        }
                                        acc_t sl = first_acc(prop_c(G.rinfo[l], c0));
                                        if (l + 32 < M) sl = sl + prop_c(G.rinfo[l + 32], c1);
                                        if (l + 64 < M) sl = sl + prop_c(G.rinfo[l + 64], c2);
                                        if (l + 96 < M) sl = sl + prop_c(G.rinfo[l + 96], c3);
                                        V[l * kStride + lane] = to_f64(sl);
                                        if (ln < 0) break;
                                        l = ln;
                                        c0 = n0;
                                        c1 = n1;
                                        c2 = n2;
                                        c3 = n3;
                                    }
                                } else {
                                    while (m) {
                                        const int l = __ffs(m) - 1;
                                        m &= m - 1;
                                        V[l * kStride + lane] = own_slot_sum(G, l);
                                    }
                                }
#pragma unroll
                                for (int k = 1; k <= 5; ++k) {
                                    const int width = 32 >> k;
                                    dirty = (dirty | (dirty >> width)) & ((1u << width) - 1u);
                                    unsigned q = dirty;
                                    while (q) {
                                        const int c = __ffs(q) - 1;
                                        q &= q - 1;
                                        V[(node_base(k) + c) * kStride + lane] =
                                            V[(node_base(k - 1) + c) * kStride + lane] +
                                            V[(node_base(k - 1) + c + width) * kStride + lane];
                                    }
                                }
                                t = t_new;
                                ssa_steps += 1;
                                firings += 1;
                                first = 0;
                                if (--ssa_left == 0) phase = P_TOP;
                            }
                        }
                    }
                }
            }
        }

        // ---- finished simulations: remaining samples hold the final state
        if (phase == P_DONE) {
            const GroupView G = gview(grp);
            while (ks < G.S) lane_record(G, ks++);
            if (G.stats != nullptr) {
                ssa_sim_stats st;
                st.status = status;
                st.reserved = 0;
                st.leaps = leaps;
                st.rejected = rejected;
                st.ssa_steps = ssa_steps;
                st.firings = firings;
                st.attempts = attempt;
                st.t_final = t;
                G.stats[row] = st;
            }
            if (kMulti && G.done_count != nullptr) {
                // this simulation's samples and counters are written: count it, and the
                // group's last simulation tells the host that the group is complete
                __threadfence();
                const unsigned long long prev = atomicAdd(G.done_count, 1ull);
                if (prev + 1 == (unsigned long long)G.n_sims) {
                    __threadfence_system();
                    *G.done_flag = 1;
                }
            }
            phase = P_NEED;
        }
        __syncwarp();
    }
}

}  // namespace lane

inline size_t lane_smem_bytes(const ModelLayout &L, int block_warps)
{
    return model_smem_bytes(L) + lane::r16((size_t)f64::kInvTable * 8) + (size_t)block_warps * lane::lane_warp_bytes(L.N, L.M);
}

inline size_t lane_multi_bytes(int max_N, int max_M, int block_warps)
{
    return lane::r16((size_t)f64::kInvTable * 8) + (size_t)block_warps * lane::lane_warp_bytes(max_N, max_M);
}

template <class Arith, bool kMulti, int kRegCap>
cudaError_t launch_lane_variant(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(lane::lane_kernel<Arith, kMulti, kRegCap>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(lane::lane_kernel<Arith, kMulti, kRegCap>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             carveout);
    if (e != cudaSuccess) return e;
    lane::lane_kernel<Arith, kMulti, kRegCap><<<grid, block_warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

// reg_cap: 0 = the default build, 1 = the 168-register build (block_warps <= 4)
template <class Arith, bool kMulti>
cudaError_t launch_lane_impl(const SimArgs &a, int block_warps, int grid, size_t smem, int carveout, int reg_cap,
                             cudaStream_t s)
{
    cudaError_t e = f64::ensure_log_table(s);
    if (e != cudaSuccess) return e;
    if (reg_cap) return launch_lane_variant<Arith, kMulti, 1>(a, block_warps, grid, smem, carveout, s);
    return launch_lane_variant<Arith, kMulti, 0>(a, block_warps, grid, smem, carveout, s);
}

template <class Arith, bool kMulti, int kRegCap>
int lane_occupancy_variant(int block_warps, size_t smem)
{
    int nb = 0;
    // the carve-out a previous launch may have set would cap the answer: query at the default
    if (cudaFuncSetAttribute(lane::lane_kernel<Arith, kMulti, kRegCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(lane::lane_kernel<Arith, kMulti, kRegCap>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             -1) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lane::lane_kernel<Arith, kMulti, kRegCap>, block_warps * 32,
                                                      smem) != cudaSuccess)
        return 0;
    return nb;
}

template <class Arith, bool kMulti>
int lane_occupancy_impl(int block_warps, size_t smem, int reg_cap)
{
    return reg_cap ? lane_occupancy_variant<Arith, kMulti, 1>(block_warps, smem)
                   : lane_occupancy_variant<Arith, kMulti, 0>(block_warps, smem);
}

}  // namespace tl

// Deterministic reaction-rate equations for a batch of parameter sets.
//
// The mean-field model of the network (Methods section: for abundant
// species the intrinsic noise averages out and X(t) follows dX/dt =
// sum_j nu_j a_j(X) with continuous X; the stochastic 2X propensity
// c x(x-1)/2 becomes c x^2/2), one ODE system per parameter set, integrated
// by the Dormand-Prince 5(4) pair (Dormand & Prince 1980) with FSAL and a
// power-of-two step controller:
//   - h starts at T[S-1] / 64;
//   - a step is accepted when err = max_i |e_i| / (atol + rtol max(|x_i|,
//     |x_new_i|)) <= 1, and then, unless it was shortened to land on a
//     sample time, h doubles when err <= 2^-6;
//   - a rejected step halves the step it tried;
//   - a step that would pass the next sample time is shortened to end on it.
// Compiled with -fmad=false: every value is one IEEE operation in the
// written order, so trajectories equal the CPU oracle's bit for bit.
//
// One warp integrates one system at a time, drawing systems from a work
// counter.  Lane l owns species i = l, l+32, ... (their x, stage values and
// derivatives) and reactions j = l, l+32, ... (their propensities); the
// stage state and the propensities pass between lanes through shared
// memory.  The FP64 work of a right-hand side is one warp-instruction per
// 32 species or reactions.
#include <algorithm>
#include <climits>

#include "device_f64.cuh"
#include "engine.h"

namespace tl {
namespace {

constexpr unsigned kAll = 0xffffffffu;

// Dormand-Prince 5(4) coefficients (c_i, a_ij, b_i and b_i - b*_i).
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 44.0 / 45.0, A42 = -56.0 / 15.0, A43 = 32.0 / 9.0;
constexpr double A51 = 19372.0 / 6561.0, A52 = -25360.0 / 2187.0, A53 = 64448.0 / 6561.0, A54 = -212.0 / 729.0;
constexpr double A61 = 9017.0 / 3168.0, A62 = -355.0 / 33.0, A63 = 46732.0 / 5247.0, A64 = 49.0 / 176.0,
                 A65 = -5103.0 / 18656.0;
constexpr double B1 = 35.0 / 384.0, B3 = 500.0 / 1113.0, B4 = 125.0 / 192.0, B5 = -2187.0 / 6784.0, B6 = 11.0 / 84.0;
constexpr double E1 = 35.0 / 384.0 - 5179.0 / 57600.0, E3 = 500.0 / 1113.0 - 7571.0 / 16695.0,
                 E4 = 125.0 / 192.0 - 393.0 / 640.0, E5 = -2187.0 / 6784.0 - (-92097.0 / 339200.0),
                 E6 = 11.0 / 84.0 - 187.0 / 2100.0, E7 = 0.0 - 1.0 / 40.0;

__host__ __device__ inline size_t r16(size_t v) { return (v + 15) & ~size_t(15); }

// per-warp workspace: c[M], a[M], x[N], xs[N], xn[N], k1..k7[N] (doubles)
__host__ __device__ inline size_t rre_warp_bytes(int N, int M) { return r16(8 * (size_t)(2 * M + 10 * N)); }

struct RreSpace {
    double *c, *a, *x, *xs, *xn, *k1, *k2, *k3, *k4, *k5, *k6, *k7;
};

__device__ __forceinline__ RreSpace carve(unsigned char *p, int N, int M)
{
    RreSpace w;
    double *d = reinterpret_cast<double *>(p);
    w.c = d;
    w.a = d + M;
    w.x = d + 2 * M;
    w.xs = w.x + N;
    w.xn = w.xs + N;
    w.k1 = w.xn + (size_t)N;
    w.k2 = w.k1 + N;
    w.k3 = w.k2 + N;
    w.k4 = w.k3 + N;
    w.k5 = w.k4 + N;
    w.k6 = w.k5 + N;
    w.k7 = w.k6 + N;
    return w;
}

struct RreArgs {
    ModelLayout L;
    const int32_t *blob;
    const double *params;
    const int32_t *x0;
    const double *T;
    int32_t S;
    int64_t n_sims;
    double rtol, atol;
    int64_t max_steps;
    double *out;
    ssa_sim_stats *stats;
    unsigned long long *work_counter;
};

// dst = f(src): mass-action (mean-field) propensities, then per species the
// sum over the reactions that change it, in increasing j.
__device__ __forceinline__ void rhs(const RreSpace &w, const int *rinfo, const int *tr_ptr, const int *tr_ent, int N,
                                    int M, const double *src, double *dst, int lane)
{
    __syncwarp();
    for (int j = lane; j < M; j += 32) {
        const int info = rinfo[j];
        const int kind = info & 3;
        const int s0 = (info >> 2) & 0x7fff, s1 = (info >> 17) & 0x7fff;
        const double c = w.c[j];
        double a;
        if (kind == 0) a = c;
        else if (kind == 1) a = c * src[s0];
        else if (kind == 2) a = (c * src[s0]) * src[s1];
        else a = c * ((src[s0] * src[s0]) * 0.5);
        w.a[j] = a;
    }
    __syncwarp();
    for (int i = lane; i < N; i += 32) {
        double f = 0.0;
        bool started = false;
        for (int e = tr_ptr[i]; e < tr_ptr[i + 1]; ++e) {
            const int ent = tr_ent[e];
            const double t = f64::small_to_double((signed char)(ent & 0xff)) * w.a[ent >> 8];
            f = started ? f + t : t;
            started = true;
        }
        dst[i] = f;
    }
    __syncwarp();
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kAll, v, d);
        v = o > v ? o : v;
    }
    return v;
}

__global__ void __launch_bounds__(128, 1) rre_kernel(const RreArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int *blob = reinterpret_cast<int *>(smem);
    for (int q = threadIdx.x; q < A.L.words; q += blockDim.x) blob[q] = A.blob[q];
    __syncthreads();
    const int N = A.L.N, M = A.L.M, S = A.S;
    const int *rinfo = blob + A.L.off_rinfo, *tr_ptr = blob + A.L.off_tr_ptr, *tr_ent = blob + A.L.off_tr_ent;
    const RreSpace w = carve(smem + model_smem_bytes(A.L) + (size_t)warp * rre_warp_bytes(N, M), N, M);
    const double *T = A.T;

    for (;;) {
        unsigned long long r = 0;
        if (lane == 0) r = atomicAdd(A.work_counter, 1ull);
        r = __shfl_sync(kAll, r, 0);
        if (r >= (unsigned long long)A.n_sims) break;
        for (int j = lane; j < M; j += 32) w.c[j] = A.params[(size_t)r * M + j];
        for (int i = lane; i < N; i += 32) w.x[i] = f64::count_to_double(A.x0[(size_t)r * N + i]);
        double *outr = A.out + (size_t)r * S * (size_t)N;
        int status = SSA_STATUS_OK;
        long long acc = 0, rej = 0;
        double t = 0.0;
        double h = (S > 0) ? T[S - 1] / 64.0 : 0.0;
        rhs(w, rinfo, tr_ptr, tr_ent, N, M, w.x, w.k1, lane);
        for (int ks = 0; ks < S; ++ks) {
            const double target = T[ks];
            while (t < target && status == SSA_STATUS_OK) {
                if (acc + rej >= A.max_steps) {
                    status = SSA_STATUS_STEP_LIMIT;
                    break;
                }
                double hh = h;
                bool clamped = false;
                if (t + hh >= target) {
                    hh = target - t;
                    clamped = true;
                }
                for (int i = lane; i < N; i += 32) w.xs[i] = w.x[i] + hh * (A21 * w.k1[i]);
                rhs(w, rinfo, tr_ptr, tr_ent, N, M, w.xs, w.k2, lane);
                for (int i = lane; i < N; i += 32) {
                    double s = A31 * w.k1[i];
                    s = s + A32 * w.k2[i];
                    w.xs[i] = w.x[i] + hh * s;
                }
                rhs(w, rinfo, tr_ptr, tr_ent, N, M, w.xs, w.k3, lane);
                for (int i = lane; i < N; i += 32) {
                    double s = A41 * w.k1[i];
                    s = s + A42 * w.k2[i];
                    s = s + A43 * w.k3[i];
                    w.xs[i] = w.x[i] + hh * s;
                }
                rhs(w, rinfo, tr_ptr, tr_ent, N, M, w.xs, w.k4, lane);
                for (int i = lane; i < N; i += 32) {
                    double s = A51 * w.k1[i];
                    s = s + A52 * w.k2[i];
                    s = s + A53 * w.k3[i];
                    s = s + A54 * w.k4[i];
                    w.xs[i] = w.x[i] + hh * s;
                }
                rhs(w, rinfo, tr_ptr, tr_ent, N, M, w.xs, w.k5, lane);
                for (int i = lane; i < N; i += 32) {
                    double s = A61 * w.k1[i];
                    s = s + A62 * w.k2[i];
                    s = s + A63 * w.k3[i];
                    s = s + A64 * w.k4[i];
                    s = s + A65 * w.k5[i];
                    w.xs[i] = w.x[i] + hh * s;
                }
                rhs(w, rinfo, tr_ptr, tr_ent, N, M, w.xs, w.k6, lane);
                for (int i = lane; i < N; i += 32) {
                    double s = B1 * w.k1[i];
                    s = s + B3 * w.k3[i];
                    s = s + B4 * w.k4[i];
                    s = s + B5 * w.k5[i];
                    s = s + B6 * w.k6[i];
                    w.xn[i] = w.x[i] + hh * s;
                }
                rhs(w, rinfo, tr_ptr, tr_ent, N, M, w.xn, w.k7, lane);
                // scaled error: max over species of non-negative ratios (order-free), by bit pattern
                unsigned long long emax = 0;
                int bad = 0;
                for (int i = lane; i < N; i += 32) {
                    double s = E1 * w.k1[i];
                    s = s + E3 * w.k3[i];
                    s = s + E4 * w.k4[i];
                    s = s + E5 * w.k5[i];
                    s = s + E6 * w.k6[i];
                    s = s + E7 * w.k7[i];
                    const double ei = fabs(hh * s);
                    const double sc = A.atol + A.rtol * fmax(fabs(w.x[i]), fabs(w.xn[i]));
                    const double q = ei / sc;
                    if (!(q == q) || !isfinite(w.xn[i])) bad = 1;
                    else emax = (unsigned long long)__double_as_longlong(q) > emax
                                    ? (unsigned long long)__double_as_longlong(q) : emax;
                }
                if (__any_sync(kAll, bad)) {
                    status = SSA_STATUS_INVALID;
                    break;
                }
                const double err = __longlong_as_double((long long)warp_max_u64(emax));
                if (err <= 1.0) {
                    t = clamped ? target : t + hh;
                    for (int i = lane; i < N; i += 32) {
                        w.x[i] = w.xn[i];
                        w.k1[i] = w.k7[i];
                    }
                    acc += 1;
                    if (!clamped && err <= 0x1p-6) h = 2.0 * h;
                } else {
                    rej += 1;
                    h = hh * 0.5;
                }
                __syncwarp();
            }
            for (int i = lane; i < N; i += 32) outr[(size_t)ks * N + i] = w.x[i];
        }
        if (lane == 0 && A.stats) {
            ssa_sim_stats *st = A.stats + r;
            st->status = status;
            st->reserved = 0;
            st->leaps = acc;
            st->rejected = rej;
            st->ssa_steps = 0;
            st->firings = 0;
            st->attempts = acc + rej;
            st->t_final = t;
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_rre(const ModelLayout &L, const int32_t *blob, int64_t n_sims, const double *params,
                       const int32_t *x0, const double *T, int32_t S, double rtol, double atol, int64_t max_steps,
                       double *out, ssa_sim_stats *stats, unsigned long long *counter, cudaStream_t s)
{
    int dev = 0, sms = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int warps = 4;
    const size_t smem = model_smem_bytes(L) + warps * rre_warp_bytes(L.N, L.M);
    if (smem > (size_t)optin) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(rre_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rre_kernel, warps * 32, smem);
    if (e != cudaSuccess) return e;
    const long long need = (n_sims + warps - 1) / warps;
    const int grid = (int)std::min<long long>((long long)(per_sm > 0 ? per_sm : 1) * sms, need);
    RreArgs a{};
    a.L = L;
    a.blob = blob;
    a.params = params;
    a.x0 = x0;
    a.T = T;
    a.S = S;
    a.n_sims = n_sims;
    a.rtol = rtol;
    a.atol = atol;
    a.max_steps = max_steps;
    a.out = out;
    a.stats = stats;
    a.work_counter = counter;
    rre_kernel<<<grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

size_t rre_smem_bytes(const ModelLayout &L) { return model_smem_bytes(L) + 4 * rre_warp_bytes(L.N, L.M); }

}  // namespace tl

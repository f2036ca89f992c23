// Warp-per-simulation kernel, FP64 reference mode.
//
// One warp advances one simulation at a time and pulls the next simulation
// index from a global work counter when it finishes, so warps stay busy
// however unevenly the step counts of the simulations are spread (one
// thread per simulation: Methods, last paragraph; here a warp, because the
// per-step work over M reactions and N species parallelises across lanes).
//
// Lane l owns reactions j = l, l+32, ... and species i = l, l+32, ...  The
// network (packed CSR, see engine.h) is staged once per CTA into shared
// memory; each warp keeps its simulation's c_j, a_j, Poisson counts k_j,
// counts x_i and candidate counts x'_i in shared memory.
//
// Sums over reactions use the canonical 32-slot order: lane l adds its
// reactions in increasing j, then an xor-butterfly over distances 16..1.
// Sums over the reactions that change a species run in increasing j.  With
// -fmad=false every result matches the plain sequential statement of the
// algorithm bit for bit.
//
// Algorithm per simulation (sources):
//   propensities a_j = c_j h_j(x), mass action (Methods; Gillespie 1977)
//   critical set, a0c, tau' (Cao-Gillespie-Petzold 2005/2006)
//   SSA fallback block when tau' < ssa_factor / a0 (CGP 2006)
//   tau'' ~ Exp(a0c), one critical firing if tau'' wins (CGP 2006)
//   Poisson(a_j tau) for noncritical reactions; negativity -> tau' / 2
//   exact SSA step: direct method (Gillespie 1977)
#include <climits>

#include "device_f64.cuh"
#include "engine.h"
#include "warp_f64.cuh"

namespace tl {
namespace {

struct Workspace {
    double *a, *c;
    long long *k, *xn;
    int *x;
    unsigned char *crit, *irs;
};

__device__ __forceinline__ Workspace carve(unsigned char *p, int N, int M)
{
    auto r16 = [](size_t v) { return (v + 15) & ~size_t(15); };
    Workspace w;
    w.a = reinterpret_cast<double *>(p);
    p += r16(8 * (size_t)M);
    w.c = reinterpret_cast<double *>(p);
    p += r16(8 * (size_t)M);
    w.k = reinterpret_cast<long long *>(p);
    p += r16(8 * (size_t)M);
    w.xn = reinterpret_cast<long long *>(p);
    p += r16(8 * (size_t)N);
    w.x = reinterpret_cast<int *>(p);
    p += r16(4 * (size_t)N);
    w.crit = p;
    p += r16((size_t)M);
    w.irs = p;
    return w;
}

__device__ void run_simulation(const SimArgs &A, long long row, const Workspace &w, const int *blob,
                               const double *inv, int lane)
{
    const int N = A.L.N, M = A.L.M, S = A.S;
    const int *rinfo = blob + A.L.off_rinfo;
    const int *nu_ptr = blob + A.L.off_nu_ptr;
    const int *nu_ent = blob + A.L.off_nu_ent;
    const int *tr_ptr = blob + A.L.off_tr_ptr;
    const int *tr_ent = blob + A.L.off_tr_ent;
    const int *hor = blob + A.L.off_hor;
    const uint32_t sim = (uint32_t)(A.sim_offset + row);
    const double t_end = A.t_end;
    const double *T = A.T;
    int *out = A.samples + (size_t)row * (size_t)S * (size_t)N;

    for (int j = lane; j < M; j += 32) w.c[j] = A.params[(size_t)row * M + j];
    for (int i = lane; i < N; i += 32) w.x[i] = A.x0[(size_t)row * N + i];
    __syncwarp();

    double t = 0.0;
    int ks = 0;
    uint32_t attempt = 0;
    int status = SSA_STATUS_OK;
    long long leaps = 0, rejected = 0, ssa_steps = 0, firings = 0;
    double L[6], Lc[6];

    auto record = [&](int k) {
        int *dst = out + (size_t)k * N;
        for (int i = lane; i < N; i += 32) dst[i] = w.x[i];
    };
    auto compute_props = [&]() -> double {
        double s = 0.0;
        for (int j = lane; j < M; j += 32) {
            const double a = propensity(rinfo[j], w.c[j], w.x);
            w.a[j] = a;
            s = s + a;
        }
        __syncwarp();
        return slot_tree(s, L);
    };

    for (;;) {
        while (ks < S && T[ks] <= t) record(ks++);
        if (t >= t_end) break;
        if ((long long)attempt >= A.max_attempts) {
            status = SSA_STATUS_STEP_LIMIT;
            break;
        }
        double a0 = compute_props();
        if (a0 == 0.0) {
            t = t_end;
            break;
        }
        if (!(a0 <= 1.7976931348623157e308)) {
            status = SSA_STATUS_INVALID;
            break;
        }
        const bool exact = (A.mode == SSA_MODE_EXACT);
        double tau1 = __longlong_as_double(0x7FF0000000000000ll);
        double a0c = 0.0;
        if (!exact) {
            // critical reactions and their canonical sum a0c
            double sc = 0.0;
            for (int j = lane; j < M; j += 32) {
                long long Lj = LLONG_MAX;
                for (int e = nu_ptr[j]; e < nu_ptr[j + 1]; ++e) {
                    const int ent = nu_ent[e];
                    const int nv = (signed char)(ent & 0xff);
                    if (nv < 0) {
                        const long long q = (long long)w.x[ent >> 8] / (long long)(-nv);
                        Lj = q < Lj ? q : Lj;
                    }
                }
                const double a = w.a[j];
                const bool cr = (a > 0.0) && (Lj < (long long)A.n_c);
                w.crit[j] = cr;
                sc = sc + (cr ? a : 0.0);
            }
            for (int i = lane; i < N; i += 32) w.irs[i] = 0;
            __syncwarp();
            a0c = slot_tree(sc, Lc);
            // reactant species of noncritical reactions
            for (int j = lane; j < M; j += 32) {
                if (w.crit[j]) continue;
                const int info = rinfo[j];
                const int kind = info & 3;
                if (kind >= 1) w.irs[(info >> 2) & 0x7fff] = 1;
                if (kind == 2) w.irs[(info >> 17) & 0x7fff] = 1;
            }
            __syncwarp();
            // tau' over I_rs
            unsigned long long tmin = 0x7FF0000000000000ull;
            for (int i = lane; i < N; i += 32) {
                if (!w.irs[i]) continue;
                double mu = 0.0, sig2 = 0.0;
                for (int e = tr_ptr[i]; e < tr_ptr[i + 1]; ++e) {
                    const int ent = tr_ent[e];
                    const int j = ent >> 8;
                    if (w.crit[j]) continue;
                    const double a = w.a[j];
                    if (!(a > 0.0)) continue;
                    const int nv = (signed char)(ent & 0xff);
                    mu = mu + (double)nv * a;
                    sig2 = sig2 + (double)(nv * nv) * a;
                }
                const int xi = w.x[i];
                const double xd = (double)xi;
                double g;
                const int h = hor[i];
                if (h == 1) g = 1.0;
                else if (h == 2) g = 2.0;
                else g = (xi >= 2) ? 2.0 + 1.0 / (xd - 1.0) : 2.0;
                double bound = (A.eps * xd) / g;
                if (bound < 1.0) bound = 1.0;
                if (mu != 0.0) {
                    const unsigned long long b1 = (unsigned long long)__double_as_longlong(bound / fabs(mu));
                    tmin = b1 < tmin ? b1 : tmin;
                }
                if (sig2 != 0.0) {
                    const unsigned long long b2 =
                        (unsigned long long)__double_as_longlong((bound * bound) / sig2);
                    tmin = b2 < tmin ? b2 : tmin;
                }
            }
            tau1 = __longlong_as_double((long long)warp_min_u64(tmin));
        }

        int halvings = 0;
        for (;;) {
            if (exact || tau1 < A.ssa_factor / a0) {
                // block of exact SSA steps (direct method)
                const int n_steps = exact ? 1 : A.ssa_block;
                for (int n = 0; n < n_steps; ++n) {
                    if (n > 0) {
                        if (t >= t_end) break;
                        a0 = compute_props();
                    }
                    if (a0 == 0.0) {
                        t = t_end;
                        goto finished;
                    }
                    if (!(a0 <= 1.7976931348623157e308)) {
                        status = SSA_STATUS_INVALID;
                        goto finished;
                    }
                    if ((long long)attempt >= A.max_attempts) {
                        status = SSA_STATUS_STEP_LIMIT;
                        goto finished;
                    }
                    attempt = attempt + 1;
                    const uint4 wb = f64::draw(A.seed, sim, attempt, PURPOSE_SSA, 0, 0);
                    const double u1 = f64::u01(wb.x, wb.y);
                    const double u2 = f64::u01(wb.z, wb.w);
                    const double tau = -f64::dlog(u1) / a0;
                    const double t_new = t + tau;
                    while (ks < S && T[ks] < t_new) record(ks++);
                    if (t_new > t_end) {
                        t = t_end;
                        goto finished;
                    }
                    const int jf = slot_select(L, u2 * a0, w.a, w.crit, false, M);
                    if (jf < 0) {
                        status = SSA_STATUS_INVALID;
                        goto finished;
                    }
                    const int e0 = nu_ptr[jf], e1 = nu_ptr[jf + 1];
                    int over = 0;
                    for (int e = e0 + lane; e < e1; e += 32) {
                        const int ent = nu_ent[e];
                        const long long nx = (long long)w.x[ent >> 8] + (signed char)(ent & 0xff);
                        if (nx > INT_MAX) over = 1;
                    }
                    if (__any_sync(kFull, over)) {
                        status = SSA_STATUS_OVERFLOW;
                        goto finished;
                    }
                    __syncwarp();
                    for (int e = e0 + lane; e < e1; e += 32) {
                        const int ent = nu_ent[e];
                        w.x[ent >> 8] += (signed char)(ent & 0xff);
                    }
                    __syncwarp();
                    t = t_new;
                    ssa_steps += 1;
                    firings += 1;
                }
                break;
            }

            // one tau-leap attempt
            if ((long long)attempt >= A.max_attempts) {
                status = SSA_STATUS_STEP_LIMIT;
                goto finished;
            }
            attempt = attempt + 1;
            const uint4 wl = f64::draw(A.seed, sim, attempt, PURPOSE_LEAP, 0, 0);
            const double u_tau = f64::u01(wl.x, wl.y);
            const double u_sel = f64::u01(wl.z, wl.w);
            const double tau2 = (a0c > 0.0) ? -f64::dlog(u_tau) / a0c : __longlong_as_double(0x7FF0000000000000ll);
            const double t_stop = (ks < S) ? T[ks] : t_end;
            const double delta = t_stop - t;
            double tau;
            int jc = -1;
            bool clamp = false;
            if (tau2 <= tau1 && tau2 <= delta) {
                tau = tau2;
                jc = slot_select(Lc, u_sel * a0c, w.a, w.crit, true, M);
            } else if (delta <= tau1) {
                tau = delta;
                clamp = true;
            } else {
                tau = tau1;
            }
            int krej = 0, kover = 0;
            long long ksum = 0;
            for (int j = lane; j < M; j += 32) {
                long long kj;
                if (w.crit[j]) {
                    kj = (j == jc) ? 1 : 0;
                } else {
                    kj = f64::poisson(w.a[j] * tau, A.seed, sim, attempt, (uint32_t)j, inv);
                    if (kj < 0) krej = 1;
                    else if (kj > f64::kCountLimit) kover = 1;
                }
                w.k[j] = kj;
                ksum += kj;
            }
            if (__any_sync(kFull, krej)) {
                status = SSA_STATUS_REJECT_LIMIT;
                goto finished;
            }
            if (__any_sync(kFull, kover)) {
                status = SSA_STATUS_OVERFLOW;
                goto finished;
            }
            __syncwarp();
            int neg = 0, big = 0;
            for (int i = lane; i < N; i += 32) {
                long long xn = w.x[i];
                for (int e = tr_ptr[i]; e < tr_ptr[i + 1]; ++e) {
                    const int ent = tr_ent[e];
                    xn += w.k[ent >> 8] * (long long)(signed char)(ent & 0xff);
                }
                w.xn[i] = xn;
                neg |= (xn < 0);
                big |= (xn > INT_MAX);
            }
            if (__any_sync(kFull, neg)) {
                rejected += 1;
                halvings += 1;
                if (halvings > A.max_halvings) {
                    status = SSA_STATUS_REJECT_LIMIT;
                    goto finished;
                }
                tau1 = tau1 / 2.0;
                continue;
            }
            if (__any_sync(kFull, big)) {
                status = SSA_STATUS_OVERFLOW;
                goto finished;
            }
            for (int i = lane; i < N; i += 32) w.x[i] = (int)w.xn[i];
            __syncwarp();
            firings += warp_sum_i64(ksum);
            t = clamp ? t_stop : t + tau;
            leaps += 1;
            break;
        }
    }
finished:
    __syncwarp();
    while (ks < S) record(ks++);
    if (A.stats != nullptr && lane == 0) {
        ssa_sim_stats st;
        st.status = status;
        st.reserved = 0;
        st.leaps = leaps;
        st.rejected = rejected;
        st.ssa_steps = ssa_steps;
        st.firings = firings;
        st.attempts = attempt;
        st.t_final = t;
        A.stats[row] = st;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256, 1) warp_f64_kernel(const SimArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    int *blob = reinterpret_cast<int *>(smem);
    for (int i = threadIdx.x; i < A.L.words; i += blockDim.x) blob[i] = A.blob[i];
    const size_t model_bytes = model_smem_bytes(A.L);
    double *inv = reinterpret_cast<double *>(smem + model_bytes);
    for (int k = threadIdx.x; k < f64::kInvTable; k += blockDim.x) inv[k] = k ? 1.0 / (double)k : 0.0;
    __syncthreads();
    const size_t inv_bytes = ((size_t)f64::kInvTable * 8 + 15) & ~size_t(15);
    unsigned char *mine = smem + model_bytes + inv_bytes + (size_t)warp * warp_workspace_bytes(A.L.N, A.L.M);
    const Workspace w = carve(mine, A.L.N, A.L.M);
    for (;;) {
        unsigned long long r = 0;
        if (lane == 0) r = atomicAdd(A.work_counter, 1ull);
        r = __shfl_sync(kFull, r, 0);
        if (r >= (unsigned long long)A.n_sims) break;
        run_simulation(A, (long long)r, w, blob, inv, lane);
    }
}

}  // namespace

size_t warp_f64_smem_bytes(const ModelLayout &L, int block_warps)
{
    const size_t inv_bytes = ((size_t)f64::kInvTable * 8 + 15) & ~size_t(15);
    return model_smem_bytes(L) + inv_bytes + (size_t)block_warps * warp_workspace_bytes(L.N, L.M);
}

cudaError_t launch_warp_ref(const SimArgs &a, int block_warps, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = f64::ensure_log_table(s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(warp_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    warp_f64_kernel<<<grid, block_warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

int warp_ref_occupancy(int block_warps, size_t smem)
{
    int nb = 0;
    if (cudaFuncSetAttribute(warp_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, warp_f64_kernel, block_warps * 32, smem) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace tl

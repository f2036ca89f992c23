// C ABI of the engine (declared in include/tauleap.h): network validation
// and packing, device-memory ownership for host-buffer jobs, launch-shape
// selection, and job polling / fetching.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"

namespace {

thread_local std::string g_error;

int fail(int code, const std::string &msg)
{
    g_error = msg;
    return code;
}

#define TL_CUDA(expr)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) return fail(SSA_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Makes the model's device current for the scope of one call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Shared-memory carve-out (percent of the SM's maximum) that holds `per_sm`
// CTAs of `smem` bytes each plus the 1 KB the system reserves per CTA; the
// rest of the on-chip memory is L1 cache.
int smem_carveout_pct(int device, size_t smem, int per_sm)
{
    int max_sm = 0;
    if (cudaDeviceGetAttribute(&max_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess || max_sm <= 0)
        return -1;
    const double need = (double)per_sm * (double)(smem + 1024);
    return std::min(100, (int)std::ceil(100.0 * need / (double)max_sm));
}

}  // namespace

struct ssa_model {
    tl::ModelLayout L{};
    int32_t *d_blob = nullptr;
    int device = 0;
};

struct ssa_job {
    ssa_model_t model = nullptr;
    int64_t n_sims = 0;
    int32_t S = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaEvent_t done = nullptr;
    double *d_params = nullptr;
    int32_t *d_x0 = nullptr;
    double *d_T = nullptr;
    int32_t *d_samples = nullptr;
    ssa_sim_stats *d_stats = nullptr;
};

extern "C" {

const char *ssa_last_error(void) { return g_error.c_str(); }

int ssa_abi_version(void) { return SSA_ABI_VERSION; }

void ssa_default_options(ssa_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->mode = SSA_MODE_TAU_LEAP;
    o->precision = SSA_FP64_REF;
    o->eps = 0.03;
    o->n_c = 10;
    o->ssa_block = 100;
    o->ssa_factor = 10.0;
    o->max_halvings = 64;
    o->layout = SSA_LAYOUT_AUTO;
    o->max_attempts = 100000000ll;
    o->block_warps = 0;
}

int ssa_load_model(const ssa_model_desc *d, ssa_model_t *out)
{
    g_error.clear();
    if (!d || !out) return fail(SSA_EINVAL, "null argument");
    *out = nullptr;
    const int N = d->n_species, M = d->n_reactions;
    if (N < 1 || N > 16384 || M < 1 || M > 16384) return fail(SSA_EINVAL, "n_species and n_reactions must be in 1..16384");
    if (!d->react_ptr || !d->prod_ptr) return fail(SSA_EINVAL, "null CSR pointer");
    if (d->react_ptr[0] != 0 || d->prod_ptr[0] != 0) return fail(SSA_EINVAL, "CSR row pointers must start at 0");
    for (int j = 0; j < M; ++j)
        if (d->react_ptr[j + 1] < d->react_ptr[j] || d->prod_ptr[j + 1] < d->prod_ptr[j])
            return fail(SSA_EINVAL, "CSR row pointers must be non-decreasing");
    if ((d->react_ptr[M] > 0 && (!d->react_species || !d->react_coef)) ||
        (d->prod_ptr[M] > 0 && (!d->prod_species || !d->prod_coef)))
        return fail(SSA_EINVAL, "null CSR entry array");

    std::vector<int32_t> rinfo(M);
    std::vector<std::vector<int32_t>> nu_rows(M);
    std::vector<std::vector<int32_t>> tr_rows(N);
    std::vector<std::vector<int32_t>> dep_rows(N);
    std::vector<int32_t> hor(N, 0);
    std::vector<int32_t> dense(N, 0);
    std::vector<int32_t> seen(N, -1);
    int max_nu_len = 0;
    for (int j = 0; j < M; ++j) {
        int order = 0, n = 0, sp[2] = {0, 0}, cf[2] = {0, 0};
        for (int e = d->react_ptr[j]; e < d->react_ptr[j + 1]; ++e) {
            const int s = d->react_species[e], c = d->react_coef[e];
            if (s < 0 || s >= N) return fail(SSA_EINVAL, "reaction " + std::to_string(j) + ": reactant species out of range");
            if (c < 1) return fail(SSA_EINVAL, "reaction " + std::to_string(j) + ": reactant coefficient < 1");
            if (seen[s] == 2 * j) return fail(SSA_EINVAL, "reaction " + std::to_string(j) + ": repeated reactant species");
            seen[s] = 2 * j;
            order += c;
            if (order > 2) return fail(SSA_EINVAL, "reaction " + std::to_string(j) + ": order > 2");
            sp[n] = s;
            cf[n] = c;
            ++n;
        }
        int kind = 0, s0 = 0, s1 = 0;
        if (order == 1) {
            kind = 1;
            s0 = sp[0];
        } else if (order == 2 && n == 1) {
            kind = 3;
            s0 = sp[0];
        } else if (order == 2) {
            kind = 2;
            s0 = std::min(sp[0], sp[1]);
            s1 = std::max(sp[0], sp[1]);
        }
        rinfo[j] = kind | (s0 << 2) | (s1 << 17);
        for (int q = 0; q < n; ++q) dep_rows[sp[q]].push_back(j);
        for (int q = 0; q < n; ++q) {
            const int cls = (order == 1) ? 1 : (cf[q] == 2 ? 3 : 2);
            hor[sp[q]] = std::max(hor[sp[q]], cls);
            dense[sp[q]] -= cf[q];
        }
        for (int e = d->prod_ptr[j]; e < d->prod_ptr[j + 1]; ++e) {
            const int s = d->prod_species[e], c = d->prod_coef[e];
            if (s < 0 || s >= N) return fail(SSA_EINVAL, "reaction " + std::to_string(j) + ": product species out of range");
            if (c < 1 || c > 100) return fail(SSA_EINVAL, "reaction " + std::to_string(j) + ": product coefficient outside 1..100");
            if (seen[s] == 2 * j + 1) return fail(SSA_EINVAL, "reaction " + std::to_string(j) + ": repeated product species");
            seen[s] = 2 * j + 1;
            dense[s] += c;
        }
        // net change, species ascending (touch only the involved species)
        std::vector<int> involved;
        for (int e = d->react_ptr[j]; e < d->react_ptr[j + 1]; ++e) involved.push_back(d->react_species[e]);
        for (int e = d->prod_ptr[j]; e < d->prod_ptr[j + 1]; ++e) involved.push_back(d->prod_species[e]);
        std::sort(involved.begin(), involved.end());
        involved.erase(std::unique(involved.begin(), involved.end()), involved.end());
        for (int s : involved) {
            if (dense[s] != 0) {
                nu_rows[j].push_back((s << 8) | (dense[s] & 0xff));
                tr_rows[s].push_back((j << 8) | (dense[s] & 0xff));
            }
            dense[s] = 0;
        }
        max_nu_len = std::max(max_nu_len, (int)nu_rows[j].size());
    }

    tl::ModelLayout L{};
    L.N = N;
    L.M = M;
    int nnz = 0;
    for (auto &r : nu_rows) nnz += (int)r.size();
    L.nnz = nnz;
    L.off_rinfo = 0;
    L.off_nu_ptr = L.off_rinfo + M;
    L.off_nu_ent = L.off_nu_ptr + M + 1;
    L.off_tr_ptr = L.off_nu_ent + nnz;
    L.off_tr_ent = L.off_tr_ptr + N + 1;
    int ndep = 0;
    for (auto &r : dep_rows) ndep += (int)r.size();
    L.ndep = ndep;
    L.off_hor = L.off_tr_ent + nnz;
    L.off_dep_ptr = L.off_hor + N;
    L.off_dep_ent = L.off_dep_ptr + N + 1;
    L.off_cinfo = L.off_dep_ent + ndep;
    L.off_dmask = L.off_cinfo + M;
    L.words = L.off_dmask + M;
    L.max_nu_len = max_nu_len;
    std::vector<int32_t> blob(L.words);
    std::copy(rinfo.begin(), rinfo.end(), blob.begin() + L.off_rinfo);
    int pos = 0;
    for (int j = 0; j < M; ++j) {
        blob[L.off_nu_ptr + j] = pos;
        for (int v : nu_rows[j]) blob[L.off_nu_ent + pos++] = v;
    }
    blob[L.off_nu_ptr + M] = pos;
    pos = 0;
    for (int i = 0; i < N; ++i) {
        blob[L.off_tr_ptr + i] = pos;
        for (int v : tr_rows[i]) blob[L.off_tr_ent + pos++] = v;
    }
    blob[L.off_tr_ptr + N] = pos;
    std::copy(hor.begin(), hor.end(), blob.begin() + L.off_hor);
    pos = 0;
    for (int i = 0; i < N; ++i) {
        blob[L.off_dep_ptr + i] = pos;
        for (int v : dep_rows[i]) blob[L.off_dep_ent + pos++] = v;
    }
    blob[L.off_dep_ptr + N] = pos;
    for (int j = 0; j < M; ++j) {
        uint32_t ci = 0;
        int slot = 0;
        for (int v : nu_rows[j]) {
            const int nv = (int)(signed char)(v & 0xff);
            if (nv >= 0) continue;
            // |nu| <= 2: only reactants are consumed, with coefficients <= 2
            ci |= ((uint32_t)(v >> 8) | ((uint32_t)(-nv) << 14)) << (16 * slot);
            ++slot;
        }
        blob[L.off_cinfo + j] = (int32_t)ci;
        uint32_t dm = 0;
        for (int v : nu_rows[j])
            for (int k : dep_rows[v >> 8]) dm |= 1u << (k & 31);
        blob[L.off_dmask + j] = (int32_t)dm;
    }

    auto *m = new ssa_model();
    m->L = L;
    if (cudaGetDevice(&m->device) != cudaSuccess) {
        delete m;
        return fail(SSA_ECUDA, "no CUDA device");
    }
    cudaError_t e = cudaMalloc(&m->d_blob, sizeof(int32_t) * (size_t)L.words);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_blob, blob.data(), sizeof(int32_t) * (size_t)L.words, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (m->d_blob) cudaFree(m->d_blob);
        delete m;
        return fail(SSA_ECUDA, std::string("model upload: ") + cudaGetErrorString(e));
    }
    *out = m;
    return SSA_OK;
}

int ssa_free_model(ssa_model_t m)
{
    g_error.clear();
    if (!m) return SSA_OK;
    DeviceGuard g(m->device);
    cudaFree(m->d_blob);
    delete m;
    return SSA_OK;
}

int ssa_model_info(ssa_model_t m, int32_t *n_species, int32_t *n_reactions)
{
    if (!m) return fail(SSA_EINVAL, "null model");
    if (n_species) *n_species = m->L.N;
    if (n_reactions) *n_reactions = m->L.M;
    return SSA_OK;
}

static int check_options(const ssa_options *o)
{
    if (o->mode != SSA_MODE_TAU_LEAP && o->mode != SSA_MODE_EXACT && o->mode != SSA_MODE_CLE)
        return fail(SSA_EINVAL, "unknown mode");
    if (o->mode == SSA_MODE_CLE && o->layout == SSA_LAYOUT_WARP)
        return fail(SSA_EUNSUPPORTED, "Langevin increments run in the lane layout only");
    if (o->precision != SSA_FP64_REF && o->precision != SSA_FAST) return fail(SSA_EINVAL, "unknown precision");
    if (o->precision == SSA_FAST && o->layout == SSA_LAYOUT_WARP)
        return fail(SSA_EUNSUPPORTED, "fast mode runs in the lane layout only");
    if (!(o->eps > 0.0) || !(o->eps < 1.0)) return fail(SSA_EINVAL, "eps must be in (0,1)");
    if (o->n_c < 0) return fail(SSA_EINVAL, "n_c must be >= 0");
    if (o->ssa_block < 1) return fail(SSA_EINVAL, "ssa_block must be >= 1");
    if (!(o->ssa_factor >= 0.0) || !std::isfinite(o->ssa_factor)) return fail(SSA_EINVAL, "ssa_factor must be finite and >= 0");
    if (o->max_halvings < 0) return fail(SSA_EINVAL, "max_halvings must be >= 0");
    if (o->max_attempts < 0 || o->max_attempts > 0xFFFFFFFFll) return fail(SSA_EINVAL, "max_attempts must be in 0..2^32-1");
    if (o->layout != SSA_LAYOUT_AUTO && o->layout != SSA_LAYOUT_WARP && o->layout != SSA_LAYOUT_LANE)
        return fail(SSA_EUNSUPPORTED, "unknown layout");
    if (o->block_warps < 0 || o->block_warps > 8) return fail(SSA_EINVAL, "block_warps must be in 0..8");
    if (o->sims_per_warp < 0 || o->sims_per_warp > 32) return fail(SSA_EINVAL, "sims_per_warp must be in 0..32");
    if (o->ctas_per_sm < 0 || o->ctas_per_sm > 32) return fail(SSA_EINVAL, "ctas_per_sm must be in 0..32");
    if (o->reg_cap != 0 && o->reg_cap != 1) return fail(SSA_EINVAL, "reg_cap must be 0 or 1");
    if (o->reg_cap == 1 && o->block_warps > 4) return fail(SSA_EINVAL, "the 168-register build runs at most 4 warps per CTA");
    return SSA_OK;
}

}  // extern "C"

namespace {

// Validation, launch-shape choice and launch shared by the device-pointer
// entry points.  `counter` is the caller-provided work counter (zeroed on
// `stream` before the launch) or nullptr to allocate a stream-ordered one.
int simulate_dev_impl(ssa_model_t m, int64_t n_sims, int64_t sim_offset, const double *params,
                      const int32_t *x0, double t_end, const double *sample_times, int32_t n_samples,
                      uint64_t seed, const ssa_options *opts, int32_t *samples, ssa_sim_stats *stats,
                      void *stream, unsigned long long *counter_in, unsigned long long *moments = nullptr,
                      unsigned long long *hist = nullptr, int32_t hist_lo = 0, int32_t hist_width = 1,
                      int32_t hist_bins = 0)
{
    if (!m) return fail(SSA_EINVAL, "null model");
    ssa_options o;
    if (opts) o = *opts;
    else ssa_default_options(&o);
    int rc = check_options(&o);
    if (rc) return rc;
    if (n_sims < 0 || sim_offset < 0 || sim_offset + n_sims > (1ll << 32)) return fail(SSA_EINVAL, "n_sims/sim_offset out of range");
    if (n_samples < 0) return fail(SSA_EINVAL, "n_samples < 0");
    if (!(t_end >= 0.0) || !std::isfinite(t_end)) return fail(SSA_EINVAL, "t_end must be finite and >= 0");
    if (n_sims == 0) return SSA_OK;
    if (!params || !x0 || (n_samples > 0 && (!sample_times || (!samples && !moments && !hist))))
        return fail(SSA_EINVAL, "null device array");
    DeviceGuard g(m->device);
    if (!g.ok) return fail(SSA_ECUDA, "cannot select the model's device");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int sms = 0, smem_optin = 0;
    TL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    TL_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    // Launch shape: the lane layout (one simulation per lane for SSA steps)
    // unless asked otherwise or its per-warp workspace does not fit.
    int layout = o.layout;
    if (layout == SSA_LAYOUT_AUTO)
        layout = (tl::lane_f64_smem_bytes(m->L, 1) <= (size_t)smem_optin) ? SSA_LAYOUT_LANE : SSA_LAYOUT_WARP;
    if ((moments || hist) && layout != SSA_LAYOUT_LANE)
        return fail(SSA_EUNSUPPORTED, "sweep moments and histograms are accumulated by the lane layout only");
    if (o.mode == SSA_MODE_CLE && layout != SSA_LAYOUT_LANE)
        return fail(SSA_EUNSUPPORTED, "network too large for the lane layout, which Langevin increments need");
    auto smem_of = [&](int w) {
        return layout == SSA_LAYOUT_LANE ? tl::lane_f64_smem_bytes(m->L, w) : tl::warp_f64_smem_bytes(m->L, w);
    };
    int warps = o.block_warps > 0 ? o.block_warps : 4;
    while (warps > 1 && smem_of(warps) > (size_t)smem_optin) --warps;
    const size_t smem = smem_of(warps);
    if (smem > (size_t)smem_optin) return fail(SSA_EUNSUPPORTED, "network too large for the shared-memory workspace");
    const bool fast = (o.precision == SSA_FAST);
    const int rc_var = layout == SSA_LAYOUT_LANE ? o.reg_cap : 0;
    const int occ = layout == SSA_LAYOUT_LANE
                        ? (fast ? tl::lane_fast_occupancy(warps, smem, rc_var) : tl::lane_ref_occupancy(warps, smem, rc_var))
                        : tl::warp_ref_occupancy(warps, smem);
    int per_sm = std::max(1, occ);
    int carveout = -1;   // the driver's default carve-out
    if (layout == SSA_LAYOUT_LANE && o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) {
        per_sm = o.ctas_per_sm;
        carveout = smem_carveout_pct(m->device, smem, per_sm);
    }
    const int spw = o.sims_per_warp > 0 ? o.sims_per_warp : 32;
    const long long sims_per_block = (long long)warps * (layout == SSA_LAYOUT_LANE ? spw : 1);
    const long long need_blocks = (n_sims + sims_per_block - 1) / sims_per_block;
    const int grid = (int)std::min<long long>((long long)per_sm * sms, need_blocks);

    tl::SimArgs a{};
    a.L = m->L;
    a.blob = m->d_blob;
    a.params = params;
    a.x0 = x0;
    a.T = sample_times;
    a.S = n_samples;
    a.t_end = t_end;
    a.n_sims = n_sims;
    a.sim_offset = sim_offset;
    a.seed = seed;
    a.mode = o.mode;
    a.n_c = o.n_c;
    a.eps = o.eps;
    a.ssa_factor = o.ssa_factor;
    a.ssa_block = o.ssa_block;
    a.max_halvings = o.max_halvings;
    a.max_attempts = o.max_attempts;
    a.sims_per_warp = spw;
    a.work = layout == SSA_LAYOUT_LANE ? reinterpret_cast<unsigned long long *>(o.work_counters) : nullptr;
    a.samples = samples;
    a.stats = stats;
    a.moments = moments;
    a.hist = hist;
    a.hist_lo = hist_lo;
    a.hist_width = hist_width;
    a.hist_bins = hist_bins;
    void *counter = counter_in;
    if (!counter_in) TL_CUDA(cudaMallocAsync(&counter, sizeof(unsigned long long), s));
    a.work_counter = static_cast<unsigned long long *>(counter);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    // fast mode: the rate constants' FP32 images, formed once for the launch (the
    // allocation-free path, which has no place for them, converts them on use instead)
    void *params_f = nullptr;
    const long long n_par = n_sims * (long long)m->L.M;
    if (e == cudaSuccess && fast && layout == SSA_LAYOUT_LANE && !counter_in) {
        e = cudaMallocAsync(&params_f, sizeof(float) * (size_t)n_par, s);
        if (e == cudaSuccess) e = tl::launch_params_to_f32(params, static_cast<float *>(params_f), n_par, s);
        a.params_f = static_cast<const float *>(params_f);
    }
    if (e == cudaSuccess)
        e = layout == SSA_LAYOUT_LANE ? (fast ? tl::launch_lane_fast(a, warps, grid, smem, carveout, rc_var, s)
                                              : tl::launch_lane_ref(a, warps, grid, smem, carveout, rc_var, s))
                                      : tl::launch_warp_ref(a, warps, grid, smem, s);
    if (params_f) cudaFreeAsync(params_f, s);
    cudaError_t e2 = counter_in ? cudaSuccess : cudaFreeAsync(counter, s);
    if (e != cudaSuccess) return fail(SSA_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(SSA_ECUDA, std::string("cudaFreeAsync: ") + cudaGetErrorString(e2));
    return SSA_OK;
}


// ---------------------------------------------------------------------
// Allocation-free launch path (ssa_simulate_dev_noalloc).
//
// The simulation kernels need one piece of scratch memory besides their
// inputs and outputs: the 8-byte work counter from which warps take
// simulation indices.  ssa_simulate_dev allocates it per call with
// cudaMallocAsync.  Callers that may not allocate device memory (code
// running where allocation is forbidden or would deadlock, such as a custom
// allocator's own callbacks, or programs that reserve all device memory up
// front) use the variant below, whose counter lives in this file-scope
// array instead.  Every GPU that loads the library holds these 256 bytes
// until the process exits.  In host code the symbol is only a host-side
// stand-in, so its device address is looked up with cudaGetSymbolAddress
// (with the model's device current) and passed to the kernel.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[32];
constexpr size_t kNoallocScratchBytes = sizeof(g_noalloc_scratch);
constexpr size_t kNoallocCounterBytes = sizeof(unsigned long long);

// Device address of the static scratch on the current device.  It is looked
// up on every call (cheap, and it allocates nothing), so the address is never
// one cached from before a cudaDeviceReset.
int noalloc_scratch(unsigned long long **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(SSA_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    *out = static_cast<unsigned long long *>(p);
    return SSA_OK;
}

}  // namespace

extern "C" {

int ssa_simulate_dev(ssa_model_t m, int64_t n_sims, int64_t sim_offset, const double *params,
                     const int32_t *x0, double t_end, const double *sample_times, int32_t n_samples,
                     uint64_t seed, const ssa_options *opts, int32_t *samples, ssa_sim_stats *stats,
                     void *stream)
{
    g_error.clear();
    return simulate_dev_impl(m, n_sims, sim_offset, params, x0, t_end, sample_times, n_samples, seed, opts,
                             samples, stats, stream, nullptr);
}

int ssa_integrate_rre_dev(ssa_model_t m, int64_t n_sims, const double *params, const int32_t *x0,
                          const double *sample_times, int32_t n_samples, double rtol, double atol, int64_t max_steps,
                          double *out, ssa_sim_stats *stats, void *stream)
{
    g_error.clear();
    if (!m) return fail(SSA_EINVAL, "null model");
    if (n_sims < 0 || n_samples < 0) return fail(SSA_EINVAL, "n_sims and n_samples must be >= 0");
    if (!(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(rtol) || !std::isfinite(atol))
        return fail(SSA_EINVAL, "rtol and atol must be finite and > 0");
    if (max_steps < 1) return fail(SSA_EINVAL, "max_steps must be >= 1");
    if (n_sims == 0 || n_samples == 0) return SSA_OK;
    if (!params || !x0 || !sample_times || !out) return fail(SSA_EINVAL, "null device array");
    DeviceGuard g(m->device);
    if (!g.ok) return fail(SSA_ECUDA, "cannot select the model's device");
    int optin = 0;
    TL_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    if (tl::rre_smem_bytes(m->L) > (size_t)optin) return fail(SSA_EUNSUPPORTED, "network too large for the RRE workspace");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *counter = nullptr;
    TL_CUDA(cudaMallocAsync(&counter, sizeof(unsigned long long), s));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = tl::launch_rre(m->L, m->d_blob, n_sims, params, x0, sample_times, n_samples, rtol, atol, max_steps, out,
                           stats, static_cast<unsigned long long *>(counter), s);
    cudaError_t e2 = cudaFreeAsync(counter, s);
    if (e != cudaSuccess) return fail(SSA_ECUDA, std::string("rre: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(SSA_ECUDA, std::string("cudaFreeAsync: ") + cudaGetErrorString(e2));
    return SSA_OK;
}

int ssa_simulate_moments_dev(ssa_model_t m, int64_t n_sims, int64_t sim_offset, const double *params,
                             const int32_t *x0, double t_end, const double *sample_times, int32_t n_samples,
                             uint64_t seed, const ssa_options *opts, double *mean, double *var,
                             ssa_sim_stats *stats, void *stream)
{
    g_error.clear();
    if (!m) return fail(SSA_EINVAL, "null model");
    if (n_samples <= 0) return fail(SSA_EINVAL, "sweep moments need at least one sample time");
    if (n_sims <= 0) return fail(SSA_EINVAL, "sweep moments need at least one simulation");
    if (!mean || !var) return fail(SSA_EINVAL, "null mean/var array");
    const long long cells = (long long)n_samples * m->L.N;
    if (cells > (1ll << 30)) return fail(SSA_EINVAL, "too many (sample, species) cells");
    DeviceGuard g(m->device);
    if (!g.ok) return fail(SSA_ECUDA, "cannot select the model's device");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void *acc = nullptr;
    const size_t acc_bytes = sizeof(unsigned long long) * 3 * (size_t)cells;
    TL_CUDA(cudaMallocAsync(&acc, acc_bytes, s));
    cudaError_t e = cudaMemsetAsync(acc, 0, acc_bytes, s);
    int rc = SSA_OK;
    if (e == cudaSuccess) {
        rc = simulate_dev_impl(m, n_sims, sim_offset, params, x0, t_end, sample_times, n_samples, seed, opts, nullptr,
                               stats, stream, nullptr, static_cast<unsigned long long *>(acc));
        if (rc == SSA_OK)
            e = tl::launch_moments_finalize(static_cast<const unsigned long long *>(acc), n_sims, (int)cells, mean,
                                            var, s);
    }
    const std::string msg = g_error;
    cudaError_t e2 = cudaFreeAsync(acc, s);
    if (rc != SSA_OK) return fail(rc, msg);
    if (e != cudaSuccess) return fail(SSA_ECUDA, std::string("moments: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(SSA_ECUDA, std::string("cudaFreeAsync: ") + cudaGetErrorString(e2));
    return SSA_OK;
}

int ssa_simulate_histograms_dev(ssa_model_t m, int64_t n_sims, int64_t sim_offset, const double *params,
                                const int32_t *x0, double t_end, const double *sample_times, int32_t n_samples,
                                uint64_t seed, const ssa_options *opts, int32_t bin_lo, int32_t bin_width,
                                int32_t n_bins, uint64_t *counts, ssa_sim_stats *stats, void *stream)
{
    g_error.clear();
    if (!m) return fail(SSA_EINVAL, "null model");
    if (n_bins < 1 || bin_width < 1) return fail(SSA_EINVAL, "n_bins and bin_width must be >= 1");
    if (n_samples <= 0) return fail(SSA_EINVAL, "sweep histograms need at least one sample time");
    if (!counts) return fail(SSA_EINVAL, "null counts array");
    if ((long long)n_samples * m->L.N * (long long)(n_bins + 2) > (1ll << 34))
        return fail(SSA_EINVAL, "too many histogram bins");
    return simulate_dev_impl(m, n_sims, sim_offset, params, x0, t_end, sample_times, n_samples, seed, opts, nullptr,
                             stats, stream, nullptr, nullptr, reinterpret_cast<unsigned long long *>(counts), bin_lo,
                             bin_width, n_bins);
}

static void job_free_buffers(ssa_job *j)
{
    cudaStream_t s = j->stream;
    if (j->d_params) cudaFreeAsync(j->d_params, s);
    if (j->d_x0) cudaFreeAsync(j->d_x0, s);
    if (j->d_T) cudaFreeAsync(j->d_T, s);
    if (j->d_samples) cudaFreeAsync(j->d_samples, s);
    if (j->d_stats) cudaFreeAsync(j->d_stats, s);
    j->d_params = nullptr;
    j->d_x0 = nullptr;
    j->d_T = nullptr;
    j->d_samples = nullptr;
    j->d_stats = nullptr;
}

int ssa_submit_batch(ssa_model_t m, int64_t n_sims, const double *params, const int32_t *x0,
                     double t_end, const double *sample_times, int32_t n_samples, uint64_t seed,
                     const ssa_options *opts, void *stream, ssa_job_t *out)
{
    g_error.clear();
    if (!m || !out) return fail(SSA_EINVAL, "null argument");
    *out = nullptr;
    if (n_sims < 0 || n_sims > (1ll << 32)) return fail(SSA_EINVAL, "n_sims out of range");
    if (n_samples < 0) return fail(SSA_EINVAL, "n_samples < 0");
    if (!(t_end >= 0.0) || !std::isfinite(t_end)) return fail(SSA_EINVAL, "t_end must be finite and >= 0");
    const int N = m->L.N, M = m->L.M;
    if (n_sims > 0 && (!params || !x0)) return fail(SSA_EINVAL, "null host array");
    if (n_samples > 0 && !sample_times) return fail(SSA_EINVAL, "null sample_times");
    for (int32_t k = 0; k < n_samples; ++k) {
        const double v = sample_times[k];
        if (!(v >= 0.0) || !(v <= t_end) || (k > 0 && v < sample_times[k - 1]))
            return fail(SSA_EINVAL, "sample_times must be non-decreasing within [0, t_end]");
    }
    for (int64_t i = 0; i < n_sims * (int64_t)M; ++i)
        if (!(params[i] >= 0.0) || !std::isfinite(params[i])) return fail(SSA_EINVAL, "params must be finite and >= 0");
    for (int64_t i = 0; i < n_sims * (int64_t)N; ++i)
        if (x0[i] < 0) return fail(SSA_EINVAL, "x0 must be >= 0");
    ssa_options o;
    if (opts) o = *opts;
    else ssa_default_options(&o);
    int rc = check_options(&o);
    if (rc) return rc;

    DeviceGuard g(m->device);
    if (!g.ok) return fail(SSA_ECUDA, "cannot select the model's device");
    const size_t b_params = sizeof(double) * (size_t)n_sims * M;
    const size_t b_x0 = sizeof(int32_t) * (size_t)n_sims * N;
    const size_t b_T = sizeof(double) * (size_t)n_samples;
    const size_t b_samples = sizeof(int32_t) * (size_t)n_sims * n_samples * N;
    const size_t b_stats = sizeof(ssa_sim_stats) * (size_t)n_sims;
    size_t free_b = 0, total_b = 0;
    TL_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t need = b_params + b_x0 + b_T + b_samples + b_stats + (64u << 20);
    if (need > free_b) return fail(SSA_ENOMEM, "job needs " + std::to_string(need) + " bytes, " + std::to_string(free_b) + " free");

    auto *j = new ssa_job();
    j->model = m;
    j->n_sims = n_sims;
    j->S = n_samples;
    if (stream) {
        j->stream = reinterpret_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete j;
            return fail(SSA_ECUDA, "cannot create a stream");
        }
        j->own_stream = true;
    }
    auto bail = [&](int code, const std::string &msg) {
        job_free_buffers(j);
        cudaStreamSynchronize(j->stream);
        if (j->done) cudaEventDestroy(j->done);
        if (j->own_stream) cudaStreamDestroy(j->stream);
        delete j;
        return fail(code, msg);
    };
    cudaError_t e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(SSA_ECUDA, "event create");
    auto alloc = [&](void **p, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        return cudaMallocAsync(p, bytes, j->stream);
    };
    e = alloc((void **)&j->d_params, b_params);
    if (e == cudaSuccess) e = alloc((void **)&j->d_x0, b_x0);
    if (e == cudaSuccess) e = alloc((void **)&j->d_T, b_T);
    if (e == cudaSuccess) e = alloc((void **)&j->d_samples, b_samples);
    if (e == cudaSuccess) e = alloc((void **)&j->d_stats, b_stats);
    if (e != cudaSuccess) return bail(SSA_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
    if (b_params) e = cudaMemcpyAsync(j->d_params, params, b_params, cudaMemcpyHostToDevice, j->stream);
    if (e == cudaSuccess && b_x0) e = cudaMemcpyAsync(j->d_x0, x0, b_x0, cudaMemcpyHostToDevice, j->stream);
    if (e == cudaSuccess && b_T) e = cudaMemcpyAsync(j->d_T, sample_times, b_T, cudaMemcpyHostToDevice, j->stream);
    if (e != cudaSuccess) return bail(SSA_ECUDA, std::string("input copy: ") + cudaGetErrorString(e));
    rc = ssa_simulate_dev(m, n_sims, 0, j->d_params, j->d_x0, t_end, j->d_T, n_samples, seed, &o, j->d_samples,
                          j->d_stats, j->stream);
    if (rc != SSA_OK) {
        std::string msg = g_error;
        return bail(rc, msg);
    }
    e = cudaEventRecord(j->done, j->stream);
    if (e != cudaSuccess) return bail(SSA_ECUDA, std::string("event record: ") + cudaGetErrorString(e));
    *out = j;
    return SSA_OK;
}

int ssa_poll(ssa_job_t j, int32_t *state)
{
    g_error.clear();
    if (!j || !state) return fail(SSA_EINVAL, "null argument");
    cudaError_t e = cudaEventQuery(j->done);
    if (e == cudaSuccess) *state = SSA_JOB_DONE;
    else if (e == cudaErrorNotReady) *state = SSA_JOB_RUNNING;
    else {
        *state = SSA_JOB_FAILED;
        return fail(SSA_ECUDA, std::string("job: ") + cudaGetErrorString(e));
    }
    return SSA_OK;
}

int ssa_wait(ssa_job_t j)
{
    g_error.clear();
    if (!j) return fail(SSA_EINVAL, "null job");
    TL_CUDA(cudaEventSynchronize(j->done));
    return SSA_OK;
}

int ssa_fetch(ssa_job_t j, int32_t *samples, ssa_sim_stats *stats)
{
    g_error.clear();
    if (!j) return fail(SSA_EINVAL, "null job");
    DeviceGuard g(j->model->device);
    const size_t b_samples = sizeof(int32_t) * (size_t)j->n_sims * j->S * j->model->L.N;
    const size_t b_stats = sizeof(ssa_sim_stats) * (size_t)j->n_sims;
    if (samples && b_samples)
        TL_CUDA(cudaMemcpyAsync(samples, j->d_samples, b_samples, cudaMemcpyDeviceToHost, j->stream));
    if (stats && b_stats) TL_CUDA(cudaMemcpyAsync(stats, j->d_stats, b_stats, cudaMemcpyDeviceToHost, j->stream));
    TL_CUDA(cudaStreamSynchronize(j->stream));
    return SSA_OK;
}

int ssa_release_job(ssa_job_t j)
{
    g_error.clear();
    if (!j) return SSA_OK;
    DeviceGuard g(j->model->device);
    cudaEventSynchronize(j->done);
    job_free_buffers(j);
    cudaError_t e = cudaStreamSynchronize(j->stream);
    cudaEventDestroy(j->done);
    if (j->own_stream) cudaStreamDestroy(j->stream);
    delete j;
    if (e != cudaSuccess) return fail(SSA_ECUDA, std::string("release: ") + cudaGetErrorString(e));
    return SSA_OK;
}

int ssa_simulate_multi_dev(int32_t n_groups, const ssa_group *groups, const ssa_options *opts, void *stream)
{
    g_error.clear();
    return tl::simulate_multi_impl(n_groups, groups, opts, stream, nullptr, nullptr);
}

}  // extern "C"

namespace tl {

int simulate_multi_impl(int32_t n_groups, const ssa_group *groups, const ssa_options *opts, void *stream,
                        unsigned long long *done_counts, volatile int32_t *done_flags)
{
    if (n_groups < 0 || (n_groups > 0 && !groups)) return fail(SSA_EINVAL, "bad group list");
    if (n_groups == 0) return SSA_OK;
    ssa_options o;
    if (opts) o = *opts;
    else ssa_default_options(&o);
    int rc = check_options(&o);
    if (rc) return rc;
    if (o.layout == SSA_LAYOUT_WARP) return fail(SSA_EUNSUPPORTED, "multi-network launches use the lane layout");
    const int device = groups[0].model ? groups[0].model->device : -1;
    std::vector<tl::GroupArgs> table((size_t)n_groups);
    int64_t first = 0;
    int max_N = 1, max_M = 1;
    for (int g = 0; g < n_groups; ++g) {
        const ssa_group &G = groups[g];
        if (!G.model) return fail(SSA_EINVAL, "group " + std::to_string(g) + ": null model");
        if (G.model->device != device) return fail(SSA_EINVAL, "all groups must use models on one device");
        if (G.n_sims < 0 || G.sim_offset < 0 || G.sim_offset + G.n_sims > (1ll << 32))
            return fail(SSA_EINVAL, "group " + std::to_string(g) + ": n_sims/sim_offset out of range");
        if (G.n_samples < 0 || !(G.t_end >= 0.0) || !std::isfinite(G.t_end))
            return fail(SSA_EINVAL, "group " + std::to_string(g) + ": bad t_end or n_samples");
        if (G.n_sims > 0 && (!G.params || !G.x0 || (G.n_samples > 0 && (!G.sample_times || !G.samples))))
            return fail(SSA_EINVAL, "group " + std::to_string(g) + ": null device array");
        tl::GroupArgs &R = table[(size_t)g];
        R.L = G.model->L;
        R.blob = G.model->d_blob;
        R.params = G.params;
        R.x0 = G.x0;
        R.T = G.sample_times;
        R.S = G.n_samples;
        R.t_end = G.t_end;
        R.n_sims = G.n_sims;
        R.sim_offset = G.sim_offset;
        R.seed = G.seed;
        R.samples = G.samples;
        R.stats = G.stats;
        R.first = first;
        R.done_count = done_counts ? done_counts + g : nullptr;
        R.done_flag = done_flags ? done_flags + g : nullptr;
        first += G.n_sims;
        max_N = std::max(max_N, R.L.N);
        max_M = std::max(max_M, R.L.M);
    }
    if (first == 0) return SSA_OK;
    DeviceGuard guard(device);
    if (!guard.ok) return fail(SSA_ECUDA, "cannot select the models' device");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int sms = 0, smem_optin = 0;
    TL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    TL_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    const bool fast = (o.precision == SSA_FAST);
    int warps = o.block_warps > 0 ? o.block_warps : 4;
    while (warps > 1 && tl::lane_multi_smem_bytes(max_N, max_M, warps) > (size_t)smem_optin) --warps;
    const size_t smem = tl::lane_multi_smem_bytes(max_N, max_M, warps);
    if (smem > (size_t)smem_optin) return fail(SSA_EUNSUPPORTED, "largest network too large for the workspace");
    const int occ = fast ? tl::lane_multi_fast_occupancy(warps, smem, o.reg_cap)
                         : tl::lane_multi_ref_occupancy(warps, smem, o.reg_cap);
    int per_sm = std::max(1, occ);
    int carveout = -1;
    if (o.ctas_per_sm > 0 && o.ctas_per_sm < per_sm) {
        per_sm = o.ctas_per_sm;
        carveout = smem_carveout_pct(device, smem, per_sm);
    }
    const int spw = o.sims_per_warp > 0 ? o.sims_per_warp : 32;
    const long long per_block = (long long)warps * spw;
    const int grid = (int)std::min<long long>((long long)per_sm * sms, (first + per_block - 1) / per_block);

    tl::SimArgs a{};
    a.n_groups = n_groups;
    a.max_N = max_N;
    a.max_M = max_M;
    a.total_sims = first;
    a.mode = o.mode;
    a.n_c = o.n_c;
    a.eps = o.eps;
    a.ssa_factor = o.ssa_factor;
    a.ssa_block = o.ssa_block;
    a.max_halvings = o.max_halvings;
    a.max_attempts = o.max_attempts;
    a.sims_per_warp = spw;
    a.work = reinterpret_cast<unsigned long long *>(o.work_counters);
    void *d_table = nullptr, *counter = nullptr, *params_f = nullptr;
    cudaError_t e = cudaSuccess;
    if (fast) {
        // the rate constants' FP32 images, formed once for the launch
        long long total = 0;
        for (const auto &R : table) total += R.n_sims * (long long)R.L.M;
        if (total > 0) e = cudaMallocAsync(&params_f, sizeof(float) * (size_t)total, s);
        long long off = 0;
        for (auto &R : table) {
            const long long cnt = R.n_sims * (long long)R.L.M;
            if (e == cudaSuccess && cnt > 0) {
                float *dst = static_cast<float *>(params_f) + off;
                e = tl::launch_params_to_f32(R.params, dst, cnt, s);
                R.params_f = dst;
            }
            off += cnt;
        }
        if (e != cudaSuccess) {
            if (params_f) cudaFreeAsync(params_f, s);
            return fail(SSA_ECUDA, std::string("rate constants to FP32: ") + cudaGetErrorString(e));
        }
    }
    const size_t table_bytes = sizeof(tl::GroupArgs) * table.size();
    e = cudaMallocAsync(&d_table, table_bytes, s);
    if (e != cudaSuccess) {
        if (params_f) cudaFreeAsync(params_f, s);
        return fail(SSA_ECUDA, std::string("group table: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(d_table, table.data(), table_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&counter, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        a.groups = static_cast<const tl::GroupArgs *>(d_table);
        a.work_counter = static_cast<unsigned long long *>(counter);
        e = fast ? tl::launch_lane_multi_fast(a, warps, grid, smem, carveout, o.reg_cap, s)
                 : tl::launch_lane_multi_ref(a, warps, grid, smem, carveout, o.reg_cap, s);
    }
    // the table copy is from pageable host memory, so the copy has been staged
    // before cudaMemcpyAsync returned and `table` may go out of scope
    if (counter) cudaFreeAsync(counter, s);
    if (d_table) cudaFreeAsync(d_table, s);
    if (params_f) cudaFreeAsync(params_f, s);
    if (e != cudaSuccess) return fail(SSA_ECUDA, std::string("multi launch: ") + cudaGetErrorString(e));
    return SSA_OK;
}

}  // namespace tl

extern "C" {

int ssa_simulate_dev_noalloc(ssa_model_t m, int64_t n_sims, int64_t sim_offset, const double *params,
                             const int32_t *x0, double t_end, const double *sample_times, int32_t n_samples,
                             uint64_t seed, const ssa_options *opts, int32_t *samples, ssa_sim_stats *stats,
                             void *stream)
{
    g_error.clear();
    if (!m) return fail(SSA_EINVAL, "null model");
    if (kNoallocCounterBytes > kNoallocScratchBytes)
        return fail(SSA_EINVAL, "launch needs more scratch than the static array holds");
    DeviceGuard g(m->device);
    if (!g.ok) return fail(SSA_ECUDA, "cannot select the model's device");
    unsigned long long *counter = nullptr;
    int rc = noalloc_scratch(&counter);
    if (rc) return rc;
    return simulate_dev_impl(m, n_sims, sim_offset, params, x0, t_end, sample_times, n_samples, seed, opts,
                             samples, stats, stream, counter);
}

}  // extern "C"


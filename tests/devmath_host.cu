// Host build of the engine's device arithmetic (csrc/device_f64.cuh is
// __host__ __device__; host code takes the portable paths), exported for
// tests/test_devmath_host.py, which compares it with the oracle bit for bit.
// Only the test builds and loads this file.
#include <stdint.h>

#include "../paper_1309_7695_b300/csrc/device_f64.cuh"

using namespace tl;

static const double *inv_table()
{
    static double t[f64::kInvTable];
    static bool ready = false;
    if (!ready) {
        for (int k = 0; k < f64::kInvTable; ++k) t[k] = k ? 1.0 / (double)k : 0.0;
        ready = true;
    }
    return t;
}

extern "C" {
void dm_log_array(const double *x, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::dlog(x[i]);
}
void dm_exp_array(const double *x, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::dexp(x[i]);
}
void dm_lnfact_array(const int64_t *k, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::dlnfact(k[i]);
}
void dm_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    const uint4 r = f64::philox4x32_10(make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]), key[0], key[1]);
    out[0] = r.x;
    out[1] = r.y;
    out[2] = r.z;
    out[3] = r.w;
}
// the Poisson draw of reaction 0 at attempt 1 of simulations 0..n-1, as the
// oracle's poisson_array draws it
void dm_poisson_array(double lam, uint64_t seed, int64_t n, int64_t *out)
{
    const double *inv = inv_table();
    for (int64_t i = 0; i < n; ++i) out[i] = f64::poisson(lam, seed, (uint32_t)i, 1u, 0u, inv);
}
// the lane kernels' route: the certified FP32 inversion first, the FP64 search
// only when it declines; PTRS from 10 on
void dm_poisson_certified_array(double lam, uint64_t seed, int64_t n, int64_t *out, int64_t *n_fallback)
{
    const double *inv = inv_table();
    int64_t fb = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (lam > 0.0 && lam < 10.0) {
            const int k = f64::inversion_certain(lam, f64::inversion_uniform(seed, (uint32_t)i, 1u, 0u));
            if (k >= 0) {
                out[i] = k;
                continue;
            }
            ++fb;
        }
        out[i] = f64::poisson(lam, seed, (uint32_t)i, 1u, 0u, inv);
    }
    *n_fallback = fb;
}
void dm_normal_leap_array(double lam, uint64_t seed, int64_t n, int64_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = f64::normal_leap(lam, seed, (uint32_t)i, 1u, 0u);
}
}

extern "C" {
void dm_f64_to_f32_array(const double *x, float *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::f64_to_f32(x[i]);
}
void dm_f32_to_f64_array(const float *x, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::f32_to_f64(x[i]);
}
void dm_floor_array(const double *x, int64_t *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::floor_to_ll(x[i]);
}
void dm_u53_array(const uint64_t *v, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::u53_to_double(v[i]);
}
void dm_small_array(const int32_t *v, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = f64::small_to_double(v[i]);
}
}

extern "C" {
void dm_tau2_screen_array(const double *u, const double *a0c, const double *m, uint8_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = f64::tau2_surely_later(u[i], a0c[i], m[i]) ? 1 : 0;
}
}

// Device arithmetic of the FP64 reference mode.
//
// Every function that produces a value of the algorithm is a fixed sequence
// of correctly rounded IEEE-754 double operations (add, sub, mul, div, sqrt,
// explicit fma) plus exact bit manipulation, compiled with -fmad=false so no
// multiply-add is fused.  A CPU program that performs the same operations in
// the same order gets bit-identical values.  No CUDA math-library function
// determines a result: CUDA's FP32 expf / logf appear only inside the
// certified decisions below, which return the canonical decision or defer to
// the FP64 computation.
#pragma once

#include <stdint.h>
#include <string.h>

#include <mutex>

#include "engine.h"

namespace tl {
namespace f64 {

// Every function below is __host__ __device__: on the device it compiles to
// the intrinsics named here, on the host to portable code with the same
// values (a test builds them for the CPU and compares them with the oracle).
#define TL_HD __host__ __device__ __forceinline__

namespace bits {
TL_HD long long d2ll(double x)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(x);
#else
    long long r;
    memcpy(&r, &x, sizeof r);
    return r;
#endif
}
TL_HD double ll2d(long long v)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(v);
#else
    double r;
    memcpy(&r, &v, sizeof r);
    return r;
#endif
}
TL_HD unsigned f2u(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    unsigned r;
    memcpy(&r, &x, sizeof r);
    return r;
#endif
}
TL_HD float u2f(unsigned v)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(v);
#else
    float r;
    memcpy(&r, &v, sizeof r);
    return r;
#endif
}
TL_HD int clzll(long long v)
{
#ifdef __CUDA_ARCH__
    return __clzll(v);
#else
    return v == 0 ? 64 : __builtin_clzll((unsigned long long)v);
#endif
}
TL_HD uint32_t umulhi(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}
TL_HD double ull2d_rn(unsigned long long v)
{
#ifdef __CUDA_ARCH__
    return __ull2double_rn(v);
#else
    return (double)v;
#endif
}
TL_HD float d2f_rn(double v)
{
#ifdef __CUDA_ARCH__
    return __double2float_rn(v);
#else
    return (float)v;
#endif
}
}  // namespace bits


// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by the two round constants, mixes the
// high halves with words 1 and 3 and the key, and the key advances by the
// two Weyl increments between rounds.
TL_HD uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = bits::umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = bits::umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Stream block (sim, attempt, purpose<<24 | j, block) under key = seed.
TL_HD uint4 draw(uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t purpose,
                                      uint32_t j, uint32_t block)
{
    return philox4x32_10(make_uint4(sim, attempt, (purpose << 24) | j, block), (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// Uniform in (0,1): with m the top 52 bits of (w0:w1), the value
// (2m + 1) * 2^-53.  It is exact in double, so it is assembled from integer
// bits here: the odd 53-bit integer 2m+1 is normalised with a leading-zero
// count and given the matching exponent.
TL_HD double u01(uint32_t w0, uint32_t w1)
{
    const uint64_t m = ((((uint64_t)w0) << 32) | (uint64_t)w1) >> 12;
    const uint64_t n = 2 * m + 1;                   // odd, < 2^53
    const int lz = bits::clzll((long long)n);           // >= 11
    const uint64_t mant = (n << (lz - 11)) & 0x000FFFFFFFFFFFFFull;
    const uint64_t expo = (uint64_t)(1033 - lz);    // value = n * 2^-53
    return bits::ll2d((long long)((expo << 52) | mant));
}

// ------------------------------------------- exact bit-level helpers
// For doubles that are never negative and never -0.0 (propensities, their
// sums, times), IEEE order equals the order of the bit patterns read as
// signed 64-bit integers, so these comparisons run on the integer pipe.
TL_HD long long dbits(double v) { return bits::d2ll(v); }
TL_HD bool nn_ge(double a, double b) { return dbits(a) >= dbits(b); }
TL_HD bool nn_gt(double a, double b) { return dbits(a) > dbits(b); }
TL_HD bool nn_pos(double a) { return dbits(a) > 0; }

// Exact conversion of a count 0 <= v < 2^53 to double, assembled from bits
// (normalise with a leading-zero count; no rounding can occur).  Larger
// values use the round-to-nearest conversion.
TL_HD double u53_to_double(unsigned long long v)
{
    if (v == 0) return 0.0;
    if (v >= (1ull << 53)) return bits::ull2d_rn(v);
    const int p = 63 - bits::clzll((long long)v);                       // v in [2^p, 2^(p+1))
    const unsigned long long frac = (v << (52 - p)) & 0x000FFFFFFFFFFFFFull;
    return bits::ll2d((long long)(((unsigned long long)(1023 + p) << 52) | frac));
}
TL_HD double count_to_double(int x) { return u53_to_double((unsigned long long)(unsigned)x); }
// Conversions between FP32 and FP64 assembled from bits on the integer pipe
// (on this GPU a conversion instruction costs as much as an FP64 add).
// Both give the IEEE result: float -> double is exact, double -> float
// rounds to nearest even.  Values outside the normal float range (zero
// aside) take the conversion instruction.
TL_HD double f32_to_f64(float f)
{
    const unsigned u = bits::f2u(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if ((u << 1) == 0) return bits::ll2d((long long)sign);   // +-0
    if (e == 0 || e == 255) return (double)f;
    return bits::ll2d(
        (long long)(sign | ((unsigned long long)(e + (1023 - 127)) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

TL_HD float f64_to_f32(double d)
{
    const unsigned long long b = (unsigned long long)bits::d2ll(d);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    if ((b << 1) == 0) return bits::u2f(sign);   // +-0
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    if (e < -126 || e > 127) return bits::d2f_rn(d);
    const unsigned long long mant = b & 0x000FFFFFFFFFFFFFull;
    const unsigned m23 = (unsigned)(mant >> 29);
    const unsigned rem = (unsigned)(mant & 0x1FFFFFFFull);
    unsigned r = ((unsigned)(e + 127) << 23) | m23;
    if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) r += 1;   // a carry moves into the exponent
    return bits::u2f(sign | r);
}

// +0 + a for a propensity a (>= +0, or -0 from a -0 rate): the canonical
// sums start from +0, and adding the first term to +0 only clears the sign
// of a zero, so the first term is taken with its sign bit cleared (integer
// pipe) instead of being added.
TL_HD double first_term(double a)
{
    return bits::ll2d(bits::d2ll(a) & 0x7FFFFFFFFFFFFFFFll);
}

// Exact conversion of a small signed integer (|v| < 2^31), from bits.
TL_HD double small_to_double(int v)
{
    const double m = u53_to_double((unsigned long long)(v < 0 ? -(long long)v : (long long)v));
    return v < 0 ? bits::ll2d(bits::d2ll(m) | (long long)0x8000000000000000ull) : m;
}

// ------------------------------------------------------ log, exp, log k!
// ln 2 split: the high part keeps 32 significant bits so that e * LN2_HI
// is exact for every exponent e that occurs.
#define TL_LN2_HI 0x1.62e42feep-1
#define TL_LN2_LO 0x1.a39ef35793c76p-33
#define TL_INV_LN2 0x1.71547652b82fep+0
#define TL_HALF_LN_2PI 0x1.d67f1c864beb5p-1

// ---- logarithm table, built on the host in double-double arithmetic ----
// Entry j = 0..256 belongs to the grid point F_j = 1 + j/256:
//   inv[j] = RN(1/F_j),
//   (hi[j], lo[j]) = ln F_j for j <= 106 (F_j <= sqrt 2), ln(F_j / 2) above,
// the latter from ln y = 2 atanh(s), s = (y-1)/(y+1), with the series
// summed in double-double arithmetic (exact products by fma, exact sums by
// Knuth's and Dekker's two-sum) to about 2^-104.  The values are a fixed
// function of this sequence of IEEE operations.
constexpr int kLogTableN = 257;
constexpr int kLogSeriesTerms = 36;   // |s| <= 1/3: first omitted term below 2^-115

namespace logtab {
struct DD {
    double hi, lo;
};
inline DD two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
inline DD fast_two_sum(double a, double b)   // |a| >= |b| or a == 0
{
    const double s = a + b;
    return {s, b - (s - a)};
}
inline DD add(DD x, DD y)
{
    DD s = two_sum(x.hi, y.hi);
    const DD t = two_sum(x.lo, y.lo);
    s.lo = s.lo + t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo = s.lo + t.lo;
    return fast_two_sum(s.hi, s.lo);
}
inline DD mul(DD x, DD y)
{
    const double p = x.hi * y.hi;
    double e = fma(x.hi, y.hi, -p);
    e = e + (x.hi * y.lo + x.lo * y.hi);
    return fast_two_sum(p, e);
}
inline DD div_d(double a, double b)   // RN(a/b) and the exact remainder over b
{
    const double q = a / b;
    return {q, fma(-q, b, a) / b};
}
// tab[0..257) = inv, tab[257..514) = hi, tab[514..771) = lo
inline void build(double *tab)
{
    for (int j = 0; j < kLogTableN; ++j) {
        const double F = 1.0 + (double)j * 0x1p-8;
        tab[j] = 1.0 / F;
        const double y = (j <= 106) ? F : F * 0.5;
        const DD sv = div_d(y - 1.0, y + 1.0);
        const DD z = mul(sv, sv);
        DD acc = div_d(1.0, (double)(2 * kLogSeriesTerms + 1));
        for (int k = kLogSeriesTerms - 1; k >= 0; --k) acc = add(mul(acc, z), div_d(1.0, (double)(2 * k + 1)));
        DD r = mul(sv, acc);
        r.hi = 2.0 * r.hi;
        r.lo = 2.0 * r.lo;
        const DD n = fast_two_sum(r.hi, r.lo);
        tab[kLogTableN + j] = n.hi;
        tab[2 * kLogTableN + j] = n.lo;
    }
}
}  // namespace logtab

// This translation unit's device copy of the table (without relocatable
// device code every unit that evaluates dlog holds its own).
static __device__ double g_log_tab[3 * kLogTableN];

// Entry i of the table: the device copy in device code, a host copy built
// by the same builder in host code.
TL_HD double log_tab(int i)
{
#ifdef __CUDA_ARCH__
    return __ldg(&g_log_tab[i]);
#else
    static const double *tab = [] {
        static double t[3 * kLogTableN];
        logtab::build(t);
        return (const double *)t;
    }();
    return tab[i];
#endif
}

// Upload this unit's table to the current device, once per device: the
// first launch on a device copies it on that launch's stream `s` and waits
// for the copy to finish before marking the device done, so that launches
// on any other stream afterwards read a complete table (a copy from pageable
// memory may return before the data has reached the device, and is not
// ordered with non-blocking streams).  It allocates nothing.  A
// cudaDeviceReset discards the device copy; the library does not notice, so
// a process that resets a device must not use the library on it again.
static inline cudaError_t ensure_log_table(cudaStream_t s)
{
    static std::mutex mu;
    static bool built = false, done[256] = {false};
    static double host[3 * kLogTableN];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    if (!built) {
        logtab::build(host);
        built = true;
    }
    e = cudaMemcpyToSymbolAsync(g_log_tab, host, sizeof host, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

// ln x for finite x > 0 (Tang's table method, written from the
// mathematics).  x = 2^e m, m in [1, 2); F = 1 + j/256 is the grid point
// nearest m and f = m - F is exact, |f| <= 2^-9.  Then
//   ln x = e ln 2 + ln F + ln(1 + r),  r = f RN(1/F),
// with ln(F/2) and e + 1 in place of ln F and e when F > sqrt 2, so that x
// near 1 from either side meets the entry ln 1 = 0.  ln(1 + r) = r + r^2
// (-1/2 + r/3 - r^2/4 + r^3/5 - r^4/6), first omitted term below 2^-56
// relative.  e LN2_HI is exact; its sum with the table's high part keeps its
// rounding error (Fast2Sum), and the low parts and ln(1 + r) are added after.
// F and e as doubles are assembled from bits (exact, off the FP64 unit).
TL_HD double dlog(double x)
{
    long long bits = bits::d2ll(x);
    int biased = (int)((bits >> 52) & 0x7ff);
    int adj = 0;
    if (biased == 0) {
        x = x * 0x1p54;
        bits = bits::d2ll(x);
        biased = (int)((bits >> 52) & 0x7ff);
        adj = -54;
    }
    int e = biased - 1023 + adj;
    const unsigned long long mant = (unsigned long long)bits & 0x000FFFFFFFFFFFFFull;
    const int j = (int)((mant + (1ull << 43)) >> 44);   // nearest 1/256 step, 0..256
    const double m = bits::ll2d((long long)(mant | 0x3FF0000000000000ull));
    const double F = bits::ll2d(j < 256 ? (long long)(0x3FF0000000000000ull | ((unsigned long long)j << 44))
                                                  : (long long)0x4000000000000000ull);
    if (j > 106) e = e + 1;
    const double f = m - F;
    const double r = f * log_tab(j);
    double p = -1.0 / 6.0;
    p = p * r + 1.0 / 5.0;
    p = p * r - 1.0 / 4.0;
    p = p * r + 1.0 / 3.0;
    p = p * r - 1.0 / 2.0;
    const double q = r + (r * r) * p;
    const double de = small_to_double(e);
    const double a = de * TL_LN2_HI;
    const double ghi = log_tab(kLogTableN + j);
    const double hi = a + ghi;
    const double err = ghi - (hi - a);
    const double lo = ((de * TL_LN2_LO + log_tab(2 * kLogTableN + j)) + err) + q;
    return hi + lo;
}

// e^x: n = floor(x/ln2 + 1/2), r = (x - n LN2_HI) - n LN2_LO, e^r by the
// Taylor polynomial through r^13 in Horner form, then scaled by 2^n.
TL_HD double dexp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return bits::ll2d(0x7FF0000000000000ll);
    if (x < -745.0) return 0.0;
    const double n = floor(x * TL_INV_LN2 + 0.5);
    const double r = (x - n * TL_LN2_HI) - n * TL_LN2_LO;
    double p = 1.0 / 6227020800.0;
    p = p * r + 1.0 / 479001600.0;
    p = p * r + 1.0 / 39916800.0;
    p = p * r + 1.0 / 3628800.0;
    p = p * r + 1.0 / 362880.0;
    p = p * r + 1.0 / 40320.0;
    p = p * r + 1.0 / 5040.0;
    p = p * r + 1.0 / 720.0;
    p = p * r + 1.0 / 120.0;
    p = p * r + 1.0 / 24.0;
    p = p * r + 1.0 / 6.0;
    p = p * r + 1.0 / 2.0;
    p = p * r + 1.0;
    p = p * r + 1.0;
    int ni = (int)n;
    if (ni < -1020) {
        p = p * 0x1p-60;
        ni += 60;
    }
    return p * bits::ll2d((long long)((uint64_t)(ni + 1023) << 52));
}

// ln k!: exact product then ln for k < 10; Stirling's series through the
// k^-13 term for k >= 10.
TL_HD double dlnfact(long long k)
{
    if (k < 10) {
        double f = 1.0;
        for (long long i = 2; i <= k; ++i) f = f * (double)i;
        return dlog(f);
    }
    const double kd = (double)k;
    const double r = 1.0 / kd;
    const double r2 = r * r;
    double ser = 1.0 / 156.0;
    ser = ser * r2 - 691.0 / 360360.0;
    ser = ser * r2 + 1.0 / 1188.0;
    ser = ser * r2 - 1.0 / 1680.0;
    ser = ser * r2 + 1.0 / 1260.0;
    ser = ser * r2 - 1.0 / 360.0;
    ser = ser * r2 + 1.0 / 12.0;
    ser = ser * r;
    return ((kd + 0.5) * dlog(kd) - kd) + (TL_HALF_LN_2PI + ser);
}

// --------------------------------------------------------------- Poisson
constexpr long long kCountLimit = 1ll << 40;
constexpr int kInversionCap = 100;
constexpr int kPtrsMaxIters = 1000;
// entries of the 1/k table: k = 0..kInversionCap+1 (the inversion loop reads
// one entry ahead of the term it adds)
constexpr int kInvTable = kInversionCap + 2;

// The inversion draw of reaction j uses the first word pair of block 0 of
// its stream.
TL_HD double inversion_uniform(uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    const uint4 w = draw(seed, sim, attempt, PURPOSE_POISSON, j, 0);
    return u01(w.x, w.y);
}

// Inversion by sequential search for 0 < lam < 10: the smallest k with
// u <= F(k), where p_0 = dexp(-lam), p_k = (p_{k-1} lam) / k and F(k) =
// F(k-1) + p_k, stopping once a term no longer changes F (the rest of the
// tail is below the rounding of F) or at kInversionCap.  `inv` holds
// RN(1/k), so multiplying by it equals dividing by k.  The next term is
// formed before the current one is tested, so the multiply chain of p and
// the add chain of F overlap; u, F and p are positive, so the comparisons
// run on their bit patterns (same order as the IEEE comparison).
TL_HD long long inversion_draw(double lam, double u, const double *__restrict__ inv)
{
    double p = dexp(-lam);
    double F = p;
    double pn = (p * lam) * inv[1];
    long long k = 0;
    while (nn_gt(u, F) && k < kInversionCap) {
        k = k + 1;
        p = pn;
        pn = (p * lam) * inv[k + 1];
        const double Fn = F + p;
        if (dbits(Fn) == dbits(F)) break;
        F = Fn;
    }
    return k;
}

// ln of the Poisson pmf, k ln lam - lam - ln k!, in FP32 without the
// cancellation of its large terms.  For k >= 10, with Stirling's series for
// ln k!, it equals -D - ln(2 pi k)/2 - (1/(12k) - 1/(360k^3)), where
// D = k ln(k/lam) + lam - k >= 0 is the deviance.  Near k = lam, D is summed
// from v = (k - lam)/(k + lam) as v (k - lam) + 2k (v^3/3 + v^5/5 + ...),
// since k ln(k/lam) = 2k atanh(v) and k - lam = v (k + lam) (the saddle-point
// form of Loader, "Fast and accurate computation of binomial probabilities",
// 2000); every term there is small, so no precision is lost.
TL_HD float log_pmf_f32(float k, float lam)
{
    if (k < 10.0f) {
        float f = 1.0f;
        for (int i = 2; i <= (int)k; ++i) f *= (float)i;   // k! <= 9! is exact in FP32
        return k * logf(lam) - lam - logf(f);
    }
    const float d = k - lam;
    const float v = d / (k + lam);
    float D;
    if (fabsf(v) < 0.25f) {
        const float v2 = v * v;
        // sum_{n=1..7} v^(2n+1)/(2n+1); the first omitted term is below 2^-32 of the lead
        float s = 1.0f / 15.0f;
        s = s * v2 + 1.0f / 13.0f;
        s = s * v2 + 1.0f / 11.0f;
        s = s * v2 + 1.0f / 9.0f;
        s = s * v2 + 1.0f / 7.0f;
        s = s * v2 + 1.0f / 5.0f;
        s = s * v2 + 1.0f / 3.0f;
        D = v * d + 2.0f * k * (v * v2 * s);
    } else {
        D = k * logf(k / lam) + lam - k;
    }
    const float rk = 1.0f / k;
    const float corr = rk * (1.0f / 12.0f - (rk * rk) * (1.0f / 360.0f));
    return -D - 0.5f * logf(6.283185307f * k) - corr;
}

// ---------------------------------------------------- certified FP32 decisions
// On this GPU an FP32 operation is ~64x cheaper than an FP64 one.  Where an
// FP64 value of the canonical algorithm only feeds a comparison, the
// comparison is first made on an FP32 evaluation whose distance from the
// canonical FP64 value is bounded; when the FP32 value lies outside that
// bound of the decision boundary the decision is the canonical one, and
// otherwise the caller runs the exact FP64 computation.  Bounds use the
// documented accuracy of CUDA's expf (2 ulp) and logf (1 ulp) and allow a
// factor of at least two over the worst case of the rounding of every
// operation; results are identical to the FP64 path by construction.

// Inversion for 0 < lam < 10: the canonical search stops at the smallest k
// with u <= F(k).  In FP32, each term p_k = e^-lam lam^k / k! carries a
// relative error below 8.4e-7 + 2.4e-7 k (expf, the rounding of lam, three
// roundings per step) and F(k) below 9e-7 + 3e-7 k; u rounds by 2^-25.  The
// margin 4e-6 + 6e-7 k covers their sum twice.  Returns k, or -1 when a
// comparison is within the margin (or after 40 terms): then the FP64 search
// decides.  The FP64 search's early stop (a term below the rounding of F)
// happens only for u within 1e-15 of 1, which is always within the margin.
TL_HD int inversion_certain(double lam, double u)
{
    const float lf = f64_to_f32(lam);
    const float uf = f64_to_f32(u);
    float p = expf(-lf);
    float F = p;
    for (int k = 0; k < 40; ++k) {
        const float m = 4e-6f + 6e-7f * (float)k;
        if (uf <= F - m) return k;
        if (!(uf > F + m)) return -1;
        p = (p * lf) / (float)(k + 1);
        F = F + p;
    }
    return -1;
}

// PTRS acceptance after the squeeze: accept iff
//   ln(V inv_alpha / (a / us^2 + b)) <= -lam + k ln lam - ln k!.
// FP32: the left side from FP32 images of V, us, a, b (relative error of
// the argument below 13 * 2^-24 when a and b are rounded from their FP64
// values, logf within 1 ulp of |ln| <= 40: 5e-6 in all); the right side by
// log_pmf_f32 (deviance form; the rounding of lam to FP32 moves it by at
// most |k - lam| 2^-23).  `extra` widens the margin for a and b that carry
// more error (the FP32 setup of ptrs_draw: 2^-19 relative, 1e-5 more on the
// left side).  Returns +1 (accept), -1 (reject) or 0 (within the margin:
// decide in FP64).
TL_HD int ptrs_accept_certain_f(float lf, long long k, float Vf, float usf, float af, float bf, float extra)
{
    const float kf = (float)k;
    const float inv_alpha = 1.1239f + 1.1328f / (bf - 3.4f);
    const float lhs = logf(Vf * inv_alpha / (af / (usf * usf) + bf));
    const float rhs = log_pmf_f32(kf, lf);
    const float d = fabsf(kf - lf);
    float m = 5e-5f + extra + 4e-6f * (fabsf(rhs) + d);
    if (k < 10) m += 0x1p-20f * lf;
    else if (d >= 0.25f * (kf + lf)) m += 4e-6f * kf * fabsf(logf(kf / lf));
    if (lhs < rhs - m) return 1;
    if (lhs > rhs + m) return -1;
    return 0;
}

TL_HD int ptrs_accept_certain(double lam, long long k, double V, double us, double a, double b)
{
    if (!(lam < 0x1p22)) return 0;
    return ptrs_accept_certain_f(f64_to_f32(lam), k, f64_to_f32(V), f64_to_f32(us), f64_to_f32(a), f64_to_f32(b), 0.0f);
}

// The leap's tau'' = -ln(u)/a0c matters only if it can be the smallest of
// tau'', tau' and the gap to the next sample time.  True when an FP32 lower
// bound of it (logf within 1 ulp, u and a0c rounded to FP32, 1e-4 slack,
// 2^-20 absolute for u near 1) lies above m = min(tau', gap) > 0, so that the
// canonical comparisons certainly find no critical firing.  Requires a0c > 0
// and u >= 2^-126 (FP32-normal); the uniforms here are all >= 2^-53.
TL_HD bool tau2_surely_later(double u, double a0c, double m)
{
    const float a0cf = f64_to_f32(a0c);
    const float Ef = -logf(f64_to_f32(u));
    const float lo = fmaxf(Ef * 0.9999f - 0x1p-20f, 0.0f) / (a0cf * 1.0001f);
    return a0cf >= 0x1p-126f && lo <= 0x1p127f && nn_gt(f32_to_f64(lo), m);
}

// K * 2^-53 for an integer 0 < K < 2^53, exactly, from bits.
TL_HD double scaled53(unsigned long long K)
{
    return bits::ll2d(bits::d2ll(u53_to_double(K)) - (53ll << 52));
}

// floor(x) of a finite double as an integer, from bits (exact; the same
// value as the rounding instruction followed by a conversion).  |x| >= 2^62
// is returned as +-2^62: callers only test such values for sign and for
// exceeding the count limit.
TL_HD long long floor_to_ll(double x)
{
    const long long bits = bits::d2ll(x);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;   // x = 1.f * 2^e
    const bool neg = bits < 0;
    if (e < 0) return (neg && (bits << 1) != 0) ? -1 : 0;   // |x| < 1
    if (e >= 62) return neg ? -(1ll << 62) : (1ll << 62);
    const unsigned long long mant = ((unsigned long long)bits & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    long long t;
    bool frac;
    if (e >= 52) {
        t = (long long)(mant << (e - 52));
        frac = false;
    } else {
        t = (long long)(mant >> (52 - e));
        frac = (mant & ((1ull << (52 - e)) - 1)) != 0;
    }
    return neg ? -(t + (frac ? 1 : 0)) : t;
}

// PTRS, transformed rejection with squeeze (Hormann 1993), for lam >= 10:
// one stream block per iteration (block index = iteration).  Returns -1 if
// it exhausts kPtrsMaxIters and kCountLimit + 1 for a draw above
// kCountLimit.
//
// Every step that is exact in IEEE arithmetic runs on the integer pipe with
// the same result: U = u - 1/2 and us = 1/2 - |U| are integer multiples of
// 2^-53 (u = (2m+1) 2^-53), 2a doubles a positive number, and the floor, its
// conversion and the comparisons of non-negative values use bit patterns.
//
// For lam < 2^16 the iteration's decisions are first taken in FP32 with
// certified margins, and the FP64 constants and candidate are formed only
// when a decision falls inside its margin:
//   - b, a, v_r from FP32 lam: relative errors below 5, 12 and (on v_r,
//     absolute) 5 times 2^-24, bounded by 2^-19 and 1e-6;
//   - the candidate x = (2a/us + b) U + lam + 0.43 as T + (lam + 0.43) with
//     T in FP32 (relative error below 1.3 * 2^-19) and lam + 0.43 split into
//     two floats: |x_FP32 - x_FP64| <= |T| 2^-17 + |x| 2^-22 + 2^-20, so its
//     floor is certain when the fraction of x_FP32 is farther than that from
//     0 and 1;
//   - V <= v_r is certain outside a 1e-6 band; us >= 0.07 and the us < 0.013
//     squeeze are exact;
//   - the acceptance test after the squeeze is ptrs_accept_certain_f with
//     the FP32 a and b.
// The FP64 pieces of a PTRS iteration, kept out of line: they run only when
// a certified FP32 decision falls inside its margin (or for means of 2^16 and
// above), so the common iteration stays a short instruction sequence.
struct PtrsConsts {
    double b, a, two_a, vr;
};
static __host__ __device__ __noinline__ PtrsConsts ptrs_consts64(double lam)
{
    PtrsConsts c;
    const double slam = sqrt(lam);
    c.b = 0.931 + 2.53 * slam;
    c.a = -0.059 + 0.02483 * c.b;                          // > 0 for lam >= 10
    c.two_a = bits::ll2d(bits::d2ll(c.a) + (1ll << 52));   // 2a, exactly
    c.vr = 0.9277 - 3.6224 / (c.b - 2.0);                  // > 0 for lam >= 10
    return c;
}
// The acceptance test after the squeeze, in FP64:
//   ln(V inv_alpha / (a / us^2 + b)) <= -lam + k ln lam - ln k!.
static __host__ __device__ __noinline__ bool ptrs_accept64(double lam, long long k, double V, double us, const PtrsConsts &c)
{
    const double loglam = dlog(lam);
    const double inv_alpha = 1.1239 + 1.1328 / (c.b - 3.4);
    const double kd = u53_to_double((unsigned long long)k);
    const double lhs = dlog(V * inv_alpha / (c.a / (us * us) + c.b));
    const double rhs = -lam + kd * loglam - dlnfact(k);
    return lhs <= rhs;
}
static __host__ __device__ __noinline__ long long ptrs_floor64(double lam, double U, double us, const PtrsConsts &c)
{
    return floor_to_ll((c.two_a / us + c.b) * U + lam + 0.43);
}

// `work` (optional): [0] += iterations, [1] += acceptance tests after the
// squeeze (the log-pmf comparison), for the launch's work counters.
TL_HD long long ptrs_draw(double lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j,
                          unsigned *work = nullptr)
{
    // FP64 constants, formed on first need
    bool set64 = false;
    PtrsConsts c{0.0, 0.0, 0.0, 0.0};
    // FP32 images for the certified decisions
    const bool f32 = nn_gt(0x1p16, lam);
    float lf = 0.0f, bf = 0.0f, af = 0.0f, vrf = 0.0f, Lhi = 0.0f, Llo = 0.0f;
    if (f32) {
        lf = f64_to_f32(lam);
        bf = 0.931f + 2.53f * sqrtf(lf);
        af = -0.059f + 0.02483f * bf;
        vrf = 0.9277f - 3.6224f / (bf - 2.0f);
        const double L = lam + 0.43;
        Lhi = f64_to_f32(L);
        Llo = f64_to_f32(L - f32_to_f64(Lhi));
    }
    for (uint32_t it = 0; it < (uint32_t)kPtrsMaxIters; ++it) {
        if (work) work[0] += 1;
        const uint4 w = draw(seed, sim, attempt, PURPOSE_POISSON, j, it);
        const unsigned long long n = 2 * (((((uint64_t)w.x) << 32) | (uint64_t)w.y) >> 12) + 1;   // u = n 2^-53
        const long long dU = (long long)n - (1ll << 52);                                        // U = dU 2^-53
        const unsigned long long aU = (unsigned long long)(dU < 0 ? -dU : dU);
        const double U = dU < 0 ? -scaled53(aU) : scaled53(aU);
        const double us = scaled53((1ull << 52) - aU);                                          // 1/2 - |U| > 0
        const double V = u01(w.z, w.w);
        const bool us_ok = nn_ge(us, 0.07);
        const bool squeeze_rej = nn_gt(0.013, us) && nn_gt(V, us);
        // decisions of this iteration: accept (squeeze), and the candidate k
        int acc = -1;          // 1 / 0, or -1 undecided
        bool k_known = false;
        long long k = 0;
        if (f32) {
            const float Vf = f64_to_f32(V);
            if (!us_ok) acc = 0;
            else if (Vf <= vrf - 1e-6f) acc = 1;
            else if (Vf > vrf + 1e-6f) acc = 0;
            if (acc == 1 || (acc == 0 && !squeeze_rej)) {
                const float T = ((2.0f * af) / f64_to_f32(us) + bf) * f64_to_f32(U);
                const float x = (T + Llo) + Lhi;
                const float E = fabsf(T) * 0x1p-17f + fabsf(x) * 0x1p-22f + 0x1p-20f;
                if (fabsf(x) < 0x1p22f) {
                    const float fl = floorf(x);
                    const float fr = x - fl;   // exact
                    if (fr > E && fr < 1.0f - E) {
                        k = (long long)(int)fl;   // |fl| < 2^22
                        k_known = true;
                    }
                }
            }
        }
        const bool need_k = (acc != 0) || !squeeze_rej;
        if (acc < 0 || (need_k && !k_known)) {
            if (!set64) {
                c = ptrs_consts64(lam);
                set64 = true;
            }
            if (acc < 0) acc = (us_ok && nn_ge(c.vr, V)) ? 1 : 0;
            if (!k_known && ((acc != 0) || !squeeze_rej)) {
                k = ptrs_floor64(lam, U, us, c);
                k_known = true;
            }
        }
        if (acc == 1) return (k > kCountLimit) ? kCountLimit + 1 : k;
        if (squeeze_rej || k < 0) continue;
        if (k > kCountLimit) return kCountLimit + 1;
        if (work) work[1] += 1;
        const int sure = f32 ? ptrs_accept_certain_f(lf, k, f64_to_f32(V), f64_to_f32(us), af, bf, 2e-5f)
                             : (set64 ? ptrs_accept_certain(lam, k, V, us, c.a, c.b) : 0);
        if (sure > 0) return k;
        if (sure < 0) continue;
        if (!set64) {
            c = ptrs_consts64(lam);
            set64 = true;
        }
        if (ptrs_accept64(lam, k, V, us, c)) return k;
    }
    return -1;
}

// Langevin increment for a leap mean lam >= kCleMinMean (SSA_MODE_CLE; the
// chemical Langevin equation, Gillespie 2000): the Poisson count replaced
// by its normal approximation rounded to the nearest count,
// k = max(0, floor(lam + sqrt(lam) z + 1/2)), z ~ N(0,1) by Marsaglia's
// polar method with one stream block per try (v = 2u - 1, accepted when
// 0 < s = v1^2 + v2^2 < 1, z = v1 sqrt(-2 ln s / s)).  Returns -1 after
// kPtrsMaxIters rejected tries, kCountLimit + 1 above the count limit.
constexpr double kCleMinMean = 1000.0;
TL_HD long long normal_leap(double lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    for (uint32_t it = 0; it < (uint32_t)kPtrsMaxIters; ++it) {
        const uint4 w = draw(seed, sim, attempt, PURPOSE_POISSON, j, it);
        const double v1 = 2.0 * u01(w.x, w.y) - 1.0;
        const double v2 = 2.0 * u01(w.z, w.w) - 1.0;
        const double s = v1 * v1 + v2 * v2;
        if (!(s < 1.0) || !(s > 0.0)) continue;
        const double z = v1 * sqrt((-2.0 * dlog(s)) / s);
        const double k = floor((lam + sqrt(lam) * z) + 0.5);
        if (k < 0.0) return 0;
        if (k > (double)kCountLimit) return kCountLimit + 1;
        return (long long)k;
    }
    return -1;
}

// k ~ Poisson(lam) on the stream (sim, attempt, reaction j): 0 for lam <= 0,
// kCountLimit + 1 for a mean at or above 2^40, inversion below 10, PTRS
// from 10 on.
TL_HD long long poisson(double lam, uint64_t seed, uint32_t sim, uint32_t attempt,
                                             uint32_t j, const double *__restrict__ inv)
{
    if (!(lam > 0.0)) return 0;
    if (!(lam < 0x1p40)) return kCountLimit + 1;
    if (lam < 10.0) return inversion_draw(lam, inversion_uniform(seed, sim, attempt, j), inv);
    return ptrs_draw(lam, seed, sim, attempt, j);
}

}  // namespace f64
}  // namespace tl

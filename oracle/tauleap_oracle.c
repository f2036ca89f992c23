/*
 * CPU oracle for batched stochastic simulation of mass-action networks.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously
 * checkable statement of what the CUDA engine computes.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant generator with the CUDA
 * engine; both follow the same written algorithm.
 *
 * Compile with -O2 -ffp-contract=off (no -ffast-math): every double
 * operation below is a single correctly rounded IEEE-754 operation, in the
 * order written, so the FP64 reference mode of the engine can reproduce it
 * bit for bit.
 *
 * What is computed (sources):
 *  - The state X(t) is the vector of molecule counts; reactions fire
 *    according to mass-action propensities and X(t) is a continuous-time
 *    Markov chain whose sample paths are generated by Gillespie's direct
 *    method (Methods section, stochastic formulation; Gillespie 1977).
 *  - Many independent simulations of one model, each with its own kinetic
 *    constants and initial amounts (Aims and motivation; Methods, last
 *    paragraph: the simulations are mutually independent).
 *  - Tau-leaping with the step-size selection of Cao, Gillespie & Petzold,
 *    J. Chem. Phys. 124, 044109 (2006) ("CGP 2006"), the critical-reaction
 *    treatment of Cao, Gillespie & Petzold, J. Chem. Phys. 123, 054104
 *    (2005) ("CGP 2005"), and the exact-SSA fallback of CGP 2006's
 *    procedure.
 *  - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
 *  - Poisson variates: inversion by sequential search for small means and
 *    the transformed-rejection method PTRS (Hormann 1993, Insurance: Math.
 *    and Economics 12) for means >= 10.
 *  - log / exp / log k!: self-contained functions built from +,-,*,/ and
 *    fma only (Tang's table method for log, its table summed from the atanh
 *    series in double-double arithmetic; Cody-Waite reduction + Taylor
 *    polynomial for exp; Stirling series for log k!), so no platform libm
 *    enters a result.
 *
 * Pinning: see tests/test_oracle_*.py (closed forms, exact CME solutions,
 * libm ulp bounds, Poisson pmf, Philox known-answer values, invariants).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* status codes and options                                            */
/* ------------------------------------------------------------------ */
enum { ST_OK = 0, ST_STEP_LIMIT = 1, ST_OVERFLOW = 2, ST_REJECT_LIMIT = 3, ST_INVALID = 4 };
enum { MODE_TAU_LEAP = 0, MODE_EXACT_SSA = 1, MODE_CLE = 2 };
enum { PURPOSE_LEAP = 1, PURPOSE_POISSON = 2, PURPOSE_SSA = 3 };

typedef struct {
    int32_t mode;          /* MODE_TAU_LEAP, MODE_EXACT_SSA or MODE_CLE */
    int32_t n_c;           /* critical threshold on L_j (CGP 2005), 10 */
    double eps;            /* error-control parameter epsilon (CGP 2006), 0.03 */
    double ssa_factor;     /* leap abandoned when tau' < ssa_factor / a0 (CGP 2006), 10 */
    int32_t ssa_block;     /* SSA steps per fallback block (CGP 2006), 100 */
    int32_t max_halvings;  /* negativity retries per leap, 64 */
    int64_t max_attempts;  /* cap on leap attempts + SSA steps per simulation */
} oracle_opts;

typedef struct {
    int32_t status;
    int32_t reserved;
    int64_t leaps;      /* accepted tau-leaps */
    int64_t rejected;   /* leap attempts undone because a count went negative */
    int64_t ssa_steps;  /* reactions fired by exact SSA steps */
    int64_t firings;    /* total reaction firings represented */
    int64_t attempts;   /* random-stream attempt counter at exit */
    double t_final;
} oracle_stats;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64     */
/* multiplies, key bumped by the Weyl constants between rounds.          */
/* ------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One block of the stream of simulation `sim`: counter words are
 * (sim, attempt, purpose<<24 | j, block); key = (seed lo, seed hi). */
static void draw_block(uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t purpose,
                       uint32_t j, uint32_t block, uint32_t w[4])
{
    uint32_t ctr[4] = { sim, attempt, (purpose << 24) | j, block };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    oracle_philox4x32_10(ctr, key, w);
}

/* Uniform in (0,1) from two words: 52 high bits of (w0:w1), centred. */
double oracle_u01(uint32_t w0, uint32_t w1)
{
    uint64_t m = ((((uint64_t)w0) << 32) | (uint64_t)w1) >> 12;
    return ((double)m + 0.5) * 0x1p-52;
}

/* ------------------------------------------------------------------ */
/* Deterministic elementary functions                                    */
/* ------------------------------------------------------------------ */
/* ln 2 split: LN2_HI is ln 2 truncated to 32 significant bits, so that
 * n*LN2_HI is exact for |n| < 2^21; LN2_LO = ln 2 - LN2_HI rounded. */
static const double LN2_HI = 0x1.62e42feep-1;
static const double LN2_LO = 0x1.a39ef35793c76p-33;
static const double INV_LN2 = 0x1.71547652b82fep+0;   /* 1/ln 2 rounded */
static const double HALF_LN_2PI = 0x1.d67f1c864beb5p-1; /* ln(2 pi)/2 rounded */

/* ---- table of the logarithm (built once, in double-double arithmetic) ----
 * For j = 0..256 the grid point F_j = 1 + j/256 (exact).  LOG_INV[j] =
 * RN(1/F_j).  (LOG_HI[j], LOG_LO[j]) is ln F_j for F_j <= sqrt 2 (j <= 106)
 * and ln(F_j / 2) above, as an unevaluated sum of two doubles.  The pair is
 * computed by the atanh series ln y = 2 atanh(s), s = (y-1)/(y+1), summed in
 * double-double arithmetic (Dekker's exact products via fma, Knuth's exact
 * sums) to about 2^-104; the engine builds its own copy by the same
 * sequence of operations, so the two tables agree bit for bit. */
typedef struct { double hi, lo; } dd_t;

static dd_t dd_two_sum(double a, double b)
{
    dd_t r;
    r.hi = a + b;
    double bb = r.hi - a;
    r.lo = (a - (r.hi - bb)) + (b - bb);
    return r;
}

static dd_t dd_fast_two_sum(double a, double b)   /* |a| >= |b| or a = 0 */
{
    dd_t r;
    r.hi = a + b;
    r.lo = b - (r.hi - a);
    return r;
}

static dd_t dd_add(dd_t x, dd_t y)
{
    dd_t s = dd_two_sum(x.hi, y.hi);
    dd_t t = dd_two_sum(x.lo, y.lo);
    s.lo = s.lo + t.hi;
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo = s.lo + t.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}

static dd_t dd_mul(dd_t x, dd_t y)
{
    double p = x.hi * y.hi;
    double e = fma(x.hi, y.hi, -p);
    e = e + (x.hi * y.lo + x.lo * y.hi);
    return dd_fast_two_sum(p, e);
}

/* a / b for doubles, to double-double: RN quotient plus the exact remainder
 * divided by b. */
static dd_t dd_div_d(double a, double b)
{
    dd_t q;
    q.hi = a / b;
    q.lo = fma(-q.hi, b, a) / b;
    return q;
}

#define LOG_TABLE_N 257
#define LOG_SERIES_TERMS 36 /* |s| <= 1/3: the first omitted term is below 2^-115 */
static double LOG_INV[LOG_TABLE_N], LOG_HI[LOG_TABLE_N], LOG_LO[LOG_TABLE_N];

static void build_log_table(void)
{
    for (int j = 0; j < LOG_TABLE_N; ++j) {
        double F = 1.0 + (double)j * 0x1p-8;
        LOG_INV[j] = 1.0 / F;
        double y = (j <= 106) ? F : F * 0.5;
        dd_t s = dd_div_d(y - 1.0, y + 1.0);
        dd_t z = dd_mul(s, s);
        /* atanh(s)/s = sum_k z^k / (2k+1), Horner from the last term */
        dd_t acc = dd_div_d(1.0, (double)(2 * LOG_SERIES_TERMS + 1));
        for (int k = LOG_SERIES_TERMS - 1; k >= 0; --k)
            acc = dd_add(dd_mul(acc, z), dd_div_d(1.0, (double)(2 * k + 1)));
        dd_t r = dd_mul(s, acc);
        r.hi = 2.0 * r.hi;   /* exact */
        r.lo = 2.0 * r.lo;
        dd_t n = dd_fast_two_sum(r.hi, r.lo);
        LOG_HI[j] = n.hi;
        LOG_LO[j] = n.lo;
    }
}

/* built when the library is loaded, before any caller can use oracle_log */
__attribute__((constructor)) static void oracle_init_tables(void) { build_log_table(); }

/* Natural log of a finite x > 0 (Tang's table method, written from the
 * mathematics).  x = 2^e m with m in [1, 2); F = 1 + j/256 is the grid
 * point nearest m, and f = m - F is exact with |f| <= 2^-9.  Then
 *   ln x = e ln 2 + ln F + ln(1 + r),  r = f * RN(1/F),
 * where, for F > sqrt 2, ln F is replaced by ln(F/2) and e by e + 1 so that
 * x near 1 from either side meets the table entry ln 1 = 0 (no
 * cancellation).  ln(1 + r) = r + r^2 (-1/2 + r/3 - r^2/4 + r^3/5 - r^4/6);
 * the first omitted term is below 2^-56 relative for |r| <= 2^-9.  The
 * exact product e * LN2_HI and the table's high part are added with their
 * rounding error kept (Fast2Sum), the low parts and ln(1 + r) after. */
double oracle_log(double x)
{
    uint64_t bits;
    int adj = 0;
    memcpy(&bits, &x, sizeof bits);
    int biased = (int)((bits >> 52) & 0x7ff);
    if (biased == 0) {            /* subnormal: scale into the normal range */
        x = x * 0x1p54;
        memcpy(&bits, &x, sizeof bits);
        biased = (int)((bits >> 52) & 0x7ff);
        adj = -54;
    }
    int e = biased - 1023 + adj;
    uint64_t mant = bits & 0x000fffffffffffffULL;
    int j = (int)((mant + (1ULL << 43)) >> 44);   /* nearest 1/256 step, 0..256 */
    uint64_t mb = mant | 0x3ff0000000000000ULL;
    double m;
    memcpy(&m, &mb, sizeof m);                    /* m in [1, 2) */
    double F = 1.0 + (double)j * 0x1p-8;          /* exact */
    if (j > 106) e = e + 1;
    double f = m - F;                             /* exact */
    double r = f * LOG_INV[j];
    double p = -1.0 / 6.0;
    p = p * r + 1.0 / 5.0;
    p = p * r - 1.0 / 4.0;
    p = p * r + 1.0 / 3.0;
    p = p * r - 1.0 / 2.0;
    double q = r + (r * r) * p;
    double de = (double)e;
    double a = de * LN2_HI;                       /* exact */
    double hi = a + LOG_HI[j];
    double err = LOG_HI[j] - (hi - a);            /* |a| >= |LOG_HI| or a = 0 */
    double lo = ((de * LN2_LO + LOG_LO[j]) + err) + q;
    return hi + lo;
}

/* e^x.  x = n ln2 + r with n = floor(x/ln2 + 1/2) and |r| <= ln2/2
 * (Cody-Waite, two-part ln 2); e^r by its Taylor polynomial through r^13
 * (first omitted term < 5e-18 relative); scaled by 2^n. */
double oracle_exp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return INFINITY;
    if (x < -745.0) return 0.0;
    double n = floor(x * INV_LN2 + 0.5);
    double r = (x - n * LN2_HI) - n * LN2_LO;
    double p = 1.0 / 6227020800.0;   /* 1/13! */
    p = p * r + 1.0 / 479001600.0;   /* 1/12! */
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
    /* multiply by 2^ni in at most two exact steps */
    if (ni < -1020) {
        p = p * 0x1p-60;
        ni += 60;
    }
    uint64_t sb = (uint64_t)(ni + 1023) << 52;
    double scale;
    memcpy(&scale, &sb, sizeof scale);
    return p * scale;
}

/* ln k! for k >= 0.  k < 10: log of the exact product.  k >= 10: Stirling
 * series (k+1/2) ln k - k + ln(2 pi)/2 + 1/(12k) - 1/(360k^3) + 1/(1260k^5)
 * - 1/(1680k^7) + 1/(1188k^9) - 691/(360360k^11) + 1/(156k^13). */
double oracle_lnfact(int64_t k)
{
    if (k < 10) {
        double f = 1.0;
        for (int64_t i = 2; i <= k; ++i) f = f * (double)i;
        return oracle_log(f);
    }
    double kd = (double)k;
    double r = 1.0 / kd;
    double r2 = r * r;
    double ser = 1.0 / 156.0;
    ser = ser * r2 - 691.0 / 360360.0;
    ser = ser * r2 + 1.0 / 1188.0;
    ser = ser * r2 - 1.0 / 1680.0;
    ser = ser * r2 + 1.0 / 1260.0;
    ser = ser * r2 - 1.0 / 360.0;
    ser = ser * r2 + 1.0 / 12.0;
    ser = ser * r;
    return ((kd + 0.5) * oracle_log(kd) - kd) + (HALF_LN_2PI + ser);
}

/* ------------------------------------------------------------------ */
/* Poisson variates                                                      */
/* ------------------------------------------------------------------ */
#define POISSON_INV_CAP 100      /* inversion stops here (P(k>100 | mean<10) < 1e-60) */
#define PTRS_MAX_ITERS 1000
#define COUNT_LIMIT (((int64_t)1) << 40)

/* k ~ Poisson(lam) for reaction j on the stream (sim, attempt).
 * Returns k >= 0, or -1 when PTRS exhausted its iteration cap. */
int64_t oracle_poisson(double lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    uint32_t w[4];
    if (!(lam > 0.0)) return 0;
    if (!(lam < 0x1p40)) return COUNT_LIMIT + 1;   /* mean beyond the count limit */
    if (lam < 10.0) {
        /* inversion by sequential search: smallest k with u <= F(k) */
        draw_block(seed, sim, attempt, PURPOSE_POISSON, j, 0, w);
        double u = oracle_u01(w[0], w[1]);
        double p = oracle_exp(-lam);
        double F = p;
        int64_t k = 0;
        while (u > F && k < POISSON_INV_CAP) {
            k = k + 1;
            p = (p * lam) * (1.0 / (double)k);
            double Fn = F + p;
            if (Fn == F) break;   /* remaining tail below rounding of F */
            F = Fn;
        }
        return k;
    }
    /* PTRS: transformed rejection with squeeze (Hormann 1993) */
    double slam = sqrt(lam);
    double loglam = oracle_log(lam);
    double b = 0.931 + 2.53 * slam;
    double a = -0.059 + 0.02483 * b;
    double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
    double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (uint32_t it = 0; it < PTRS_MAX_ITERS; ++it) {
        draw_block(seed, sim, attempt, PURPOSE_POISSON, j, it, w);
        double U = oracle_u01(w[0], w[1]) - 0.5;
        double V = oracle_u01(w[2], w[3]);
        double us = 0.5 - fabs(U);
        double kd = floor((2.0 * a / us + b) * U + lam + 0.43);
        if (us >= 0.07 && V <= vr) return (kd > (double)COUNT_LIMIT) ? COUNT_LIMIT + 1 : (int64_t)kd;
        if (kd < 0.0 || (us < 0.013 && V > us)) continue;
        if (kd > (double)COUNT_LIMIT) return COUNT_LIMIT + 1;
        double lhs = oracle_log(V * inv_alpha / (a / (us * us) + b));
        double rhs = -lam + kd * loglam - oracle_lnfact((int64_t)kd);
        if (lhs <= rhs) return (int64_t)kd;
    }
    return -1;
}

/* Langevin increment for a large leap mean (chemical Langevin equation,
 * Gillespie 2000, cited by the paper as the CLE): the Poisson count of a
 * reaction whose mean lam is at least CLE_MIN_MEAN is replaced by its normal
 * approximation rounded to the nearest count, k = max(0, floor(lam +
 * sqrt(lam) z + 1/2)), z ~ N(0,1) by Marsaglia's polar method (one stream
 * block per try: v1 = 2u1 - 1, v2 = 2u2 - 1, accepted when 0 < s = v1^2 +
 * v2^2 < 1, z = v1 sqrt(-2 ln s / s)).  Returns -1 after PTRS_MAX_ITERS
 * rejected tries and COUNT_LIMIT + 1 for a mean at or above 2^40 or a draw
 * above the count limit. */
#define CLE_MIN_MEAN 1000.0
int64_t oracle_normal_leap(double lam, uint64_t seed, uint32_t sim, uint32_t attempt, uint32_t j)
{
    uint32_t w[4];
    if (!(lam < 0x1p40)) return COUNT_LIMIT + 1;   /* mean beyond the count limit, as for Poisson */
    for (uint32_t it = 0; it < PTRS_MAX_ITERS; ++it) {
        draw_block(seed, sim, attempt, PURPOSE_POISSON, j, it, w);
        double v1 = 2.0 * oracle_u01(w[0], w[1]) - 1.0;
        double v2 = 2.0 * oracle_u01(w[2], w[3]) - 1.0;
        double s = v1 * v1 + v2 * v2;
        if (!(s < 1.0) || !(s > 0.0)) continue;
        double z = v1 * sqrt((-2.0 * oracle_log(s)) / s);
        double k = floor((lam + sqrt(lam) * z) + 0.5);
        if (k < 0.0) return 0;
        if (k > (double)COUNT_LIMIT) return COUNT_LIMIT + 1;
        return (int64_t)k;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Model                                                                 */
/* ------------------------------------------------------------------ */
typedef struct {
    int N, M;
    /* reactants of reaction j: up to two (species, coef) entries */
    int *r_n, *r_sp0, *r_sp1, *r_kind; /* kind: 0 order0, 1 X, 2 X+Y, 3 2X */
    /* net change nu_j as a sparse list (species ascending, nu != 0) */
    int *nu_ptr, *nu_sp, *nu_val;
    /* highest-order-of-reaction class per species: 0 none, 1, 2 (X+Y only), 3 (2X present) */
    int *hor;
} model_t;

static void model_free(model_t *m)
{
    free(m->r_n); free(m->r_sp0); free(m->r_sp1); free(m->r_kind);
    free(m->nu_ptr); free(m->nu_sp); free(m->nu_val); free(m->hor);
}

static int model_build(model_t *m, int N, int M,
                       const int32_t *rp, const int32_t *rs, const int32_t *rc,
                       const int32_t *pp, const int32_t *ps, const int32_t *pc)
{
    memset(m, 0, sizeof *m);
    m->N = N; m->M = M;
    m->r_n = calloc(M > 0 ? M : 1, sizeof(int));
    m->r_sp0 = calloc(M > 0 ? M : 1, sizeof(int));
    m->r_sp1 = calloc(M > 0 ? M : 1, sizeof(int));
    m->r_kind = calloc(M > 0 ? M : 1, sizeof(int));
    m->nu_ptr = calloc(M + 1, sizeof(int));
    m->hor = calloc(N > 0 ? N : 1, sizeof(int));
    int *dense = calloc((size_t)(N > 0 ? N : 1), sizeof(int));
    int cap = 0, nnz = 0;
    for (int j = 0; j < M; ++j) cap += (rp[j + 1] - rp[j]) + (pp[j + 1] - pp[j]);
    m->nu_sp = calloc(cap > 0 ? cap : 1, sizeof(int));
    m->nu_val = calloc(cap > 0 ? cap : 1, sizeof(int));
    for (int j = 0; j < M; ++j) {
        int order = 0, n = rp[j + 1] - rp[j];
        for (int e = rp[j]; e < rp[j + 1]; ++e) {
            if (rs[e] < 0 || rs[e] >= N || rc[e] < 1) { free(dense); return -1; }
            order += rc[e];
        }
        for (int e = pp[j]; e < pp[j + 1]; ++e)
            if (ps[e] < 0 || ps[e] >= N || pc[e] < 1) { free(dense); return -1; }
        if (order > 2 || n > 2) { free(dense); return -1; }
        m->r_n[j] = n;
        if (order == 0) m->r_kind[j] = 0;
        else if (order == 1) { m->r_kind[j] = 1; m->r_sp0[j] = rs[rp[j]]; }
        else if (n == 1) { m->r_kind[j] = 3; m->r_sp0[j] = rs[rp[j]]; }
        else {
            m->r_kind[j] = 2;
            int s0 = rs[rp[j]], s1 = rs[rp[j] + 1];
            m->r_sp0[j] = s0 < s1 ? s0 : s1;
            m->r_sp1[j] = s0 < s1 ? s1 : s0;
        }
        /* highest order of reaction per reactant species (CGP 2006, g_i) */
        for (int e = rp[j]; e < rp[j + 1]; ++e) {
            int i = rs[e];
            int cls = (order == 1) ? 1 : (rc[e] == 2 ? 3 : 2);
            if (cls > m->hor[i]) m->hor[i] = cls;
        }
        /* net change nu_ij = product coef - reactant coef */
        for (int e = rp[j]; e < rp[j + 1]; ++e) dense[rs[e]] -= rc[e];
        for (int e = pp[j]; e < pp[j + 1]; ++e) dense[ps[e]] += pc[e];
        m->nu_ptr[j] = nnz;
        for (int i = 0; i < N; ++i) {
            if (dense[i] != 0) {
                m->nu_sp[nnz] = i;
                m->nu_val[nnz] = dense[i];
                ++nnz;
                dense[i] = 0;
            }
        }
    }
    m->nu_ptr[M] = nnz;
    free(dense);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Canonical summation over 32 lane-striped slots                        */
/* ------------------------------------------------------------------ */
/* Sum of v[0..M-1] in a fixed order: slot l accumulates v[l], v[l+32],
 * v[l+64], ... sequentially (slot starts at +0); the 32 slots are then
 * combined pairwise with partner distances 16, 8, 4, 2, 1 (level k keeps
 * L_k[l] = L_{k-1}[l] + L_{k-1}[l ^ (16 >> (k-1))]).  The total is L_5[0].
 * levels[k][l] receives every intermediate value for the search below. */
static double canon_sum(const double *v, int M, double levels[6][32])
{
    for (int l = 0; l < 32; ++l) {
        double s = 0.0;
        for (int j = l; j < M; j += 32) s = s + v[j];
        levels[0][l] = s;
    }
    for (int k = 1; k <= 5; ++k) {
        int d = 16 >> (k - 1);
        for (int l = 0; l < 32; ++l) levels[k][l] = levels[k - 1][l] + levels[k - 1][l ^ d];
    }
    return levels[5][0];
}

/* Pick j with probability v[j]/total, given target = u * total.
 * Descend the slot tree: at level k (4..0) the current slot set splits into
 * children `lane` and `lane + (1 << (4-k))`; go to the second child when
 * target >= first child and the second child is positive (subtracting the
 * first).  Inside the chosen slot walk j = lane, lane+32, ... and return the
 * first j whose running sum exceeds the target; if rounding leaves none,
 * return the highest-index j of the slot with v[j] > 0. */
static int canon_select(const double *v, int M, double levels[6][32], double target)
{
    int lane = 0;
    for (int k = 4; k >= 0; --k) {
        int step = 1 << (4 - k);
        double left = levels[k][lane];
        double right = levels[k][lane + step];
        if (target >= left && right > 0.0) {
            target = target - left;
            lane = lane + step;
        }
    }
    double cum = 0.0;
    int last_pos = -1;
    for (int j = lane; j < M; j += 32) {
        cum = cum + v[j];
        if (v[j] > 0.0) last_pos = j;
        if (cum > target) return j;
    }
    return last_pos;
}

/* ------------------------------------------------------------------ */
/* Per-simulation state and the main loop                               */
/* ------------------------------------------------------------------ */
typedef struct {
    double *a, *a_crit, *mu, *sig2;
    int64_t *k, *xnew;
    int *crit, *irs;
} scratch_t;

/* Mass-action propensity a_j = c_j h_j(x) (Methods: firing of reactions
 * between species; combinatorial h of Gillespie 1977): order 0: c;
 * X: c*x; X+Y: (c*x)*y; 2X: c*(x(x-1)/2). */
static double propensity(const model_t *m, int j, double c, const int32_t *x)
{
    switch (m->r_kind[j]) {
    case 0: return c;
    case 1: return c * (double)x[m->r_sp0[j]];
    case 2: return (c * (double)x[m->r_sp0[j]]) * (double)x[m->r_sp1[j]];
    default: {
        int64_t xi = x[m->r_sp0[j]];
        return c * (double)((xi * (xi - 1)) / 2);
    }
    }
}


/* Critical set, a0c and tau' for the current state (propensities already in
 * w->a).  Returns tau' (INFINITY when no species bounds the step).
 *  - critical reactions (CGP 2005): a_j > 0 and L_j < n_c, where
 *    L_j = min over species with nu_ij < 0 of floor(x_i / |nu_ij|);
 *  - a0c = canonical sum of the critical propensities;
 *  - tau' (CGP 2006): over the reactant species I_rs of the noncritical
 *    reactions J_ncr (every reaction that is not critical, including those
 *    with a_j = 0, so a species whose consumers are momentarily idle still
 *    bounds the step):
 *      mu_i = sum_{j in J_ncr} nu_ij a_j,  sigma2_i = sum_{j in J_ncr} nu_ij^2 a_j,
 *      tau' = min_i min( max(eps x_i / g_i, 1) / |mu_i| , max(eps x_i / g_i, 1)^2 / sigma2_i ),
 *    a term with mu_i = 0 (sigma2_i = 0) being infinite; g_i from the
 *    highest order of reaction of species i: 1, 2, or 2 + 1/(x_i - 1) when
 *    some reaction consumes two molecules of i (2 when x_i < 2). */
static double leap_prepare(const model_t *m, const oracle_opts *o, const int32_t *x,
                           scratch_t *w, double levels_c[6][32], double *a0c_out)
{
    const int N = m->N, M = m->M;
    double tau1 = INFINITY;
    for (int j = 0; j < M; ++j) {
        int64_t L = INT64_MAX;
        for (int e = m->nu_ptr[j]; e < m->nu_ptr[j + 1]; ++e) {
            if (m->nu_val[e] < 0) {
                int64_t q = (int64_t)x[m->nu_sp[e]] / (int64_t)(-m->nu_val[e]);
                if (q < L) L = q;
            }
        }
        w->crit[j] = (w->a[j] > 0.0 && L < (int64_t)o->n_c);
        w->a_crit[j] = w->crit[j] ? w->a[j] : 0.0;
    }
    *a0c_out = canon_sum(w->a_crit, M, levels_c);
    for (int i = 0; i < N; ++i) { w->mu[i] = 0.0; w->sig2[i] = 0.0; w->irs[i] = 0; }
    for (int j = 0; j < M; ++j) {
        if (w->crit[j]) continue;
        int kind = m->r_kind[j];
        if (kind >= 1) w->irs[m->r_sp0[j]] = 1;
        if (kind == 2) w->irs[m->r_sp1[j]] = 1;
        if (!(w->a[j] > 0.0)) continue;   /* zero terms change no sum */
        for (int e = m->nu_ptr[j]; e < m->nu_ptr[j + 1]; ++e) {
            int i = m->nu_sp[e];
            int nv = m->nu_val[e];
            w->mu[i] = w->mu[i] + (double)nv * w->a[j];
            w->sig2[i] = w->sig2[i] + (double)(nv * nv) * w->a[j];
        }
    }
    for (int i = 0; i < N; ++i) {
        if (!w->irs[i]) continue;
        double xd = (double)x[i];
        double g;
        switch (m->hor[i]) {
        case 1: g = 1.0; break;
        case 2: g = 2.0; break;
        default: g = (x[i] >= 2) ? 2.0 + 1.0 / (xd - 1.0) : 2.0; break;
        }
        double bound = (o->eps * xd) / g;
        if (bound < 1.0) bound = 1.0;
        if (w->mu[i] != 0.0) {
            double t1 = bound / fabs(w->mu[i]);
            if (t1 < tau1) tau1 = t1;
        }
        if (w->sig2[i] != 0.0) {
            double t2 = (bound * bound) / w->sig2[i];
            if (t2 < tau1) tau1 = t2;
        }
    }
    return tau1;
}

static void record_until(int32_t *out, int N, const int32_t *x, const double *T, int S,
                         int *ks, double t_inclusive, int strict)
{
    while (*ks < S && (strict ? (T[*ks] < t_inclusive) : (T[*ks] <= t_inclusive))) {
        memcpy(out + (size_t)(*ks) * N, x, sizeof(int32_t) * (size_t)N);
        *ks = *ks + 1;
    }
}

static void record_rest(int32_t *out, int N, const int32_t *x, int S, int *ks)
{
    while (*ks < S) {
        memcpy(out + (size_t)(*ks) * N, x, sizeof(int32_t) * (size_t)N);
        *ks = *ks + 1;
    }
}

static void simulate_one(const model_t *m, const oracle_opts *o, uint64_t seed, uint32_t sim,
                         const double *c, const int32_t *x0, double t_end, const double *T,
                         int S, int32_t *out, oracle_stats *st, scratch_t *w)
{
    const int N = m->N, M = m->M;
    int32_t *x = malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    memcpy(x, x0, sizeof(int32_t) * (size_t)N);
    double levels[6][32], levels_c[6][32];
    double t = 0.0;
    int ks = 0;
    uint32_t attempt = 0;
    memset(st, 0, sizeof *st);
    st->status = ST_OK;

    for (;;) {
        /* samples whose time has been reached hold the current state */
        record_until(out, N, x, T, S, &ks, t, 0);
        if (t >= t_end) break;
        if ((int64_t)attempt >= o->max_attempts) { st->status = ST_STEP_LIMIT; break; }

        /* propensities and their total a0 */
        for (int j = 0; j < M; ++j) w->a[j] = propensity(m, j, c[j], x);
        double a0 = canon_sum(w->a, M, levels);
        if (a0 == 0.0) { t = t_end; break; }   /* no reaction can fire again */
        if (!(a0 <= DBL_MAX)) { st->status = ST_INVALID; break; }   /* non-finite rates */

        int do_ssa = (o->mode == MODE_EXACT_SSA);
        double tau1 = INFINITY, a0c = 0.0;
        if (!do_ssa) tau1 = leap_prepare(m, o, x, w, levels_c, &a0c);

        int halvings = 0;
        int leap_done = 0;
        while (!leap_done) {
            if (do_ssa || tau1 < o->ssa_factor / a0) {
                /* exact SSA steps (direct method, Gillespie 1977); a block of
                 * ssa_block steps in tau-leaping mode (CGP 2006) */
                int n_steps = (o->mode == MODE_EXACT_SSA) ? 1 : o->ssa_block;
                for (int n = 0; n < n_steps; ++n) {
                    if (n > 0) {
                        if (t >= t_end) break;
                        for (int j = 0; j < M; ++j) w->a[j] = propensity(m, j, c[j], x);
                        a0 = canon_sum(w->a, M, levels);
                    }
                    if (a0 == 0.0) { t = t_end; goto finished; }
                    if (!(a0 <= DBL_MAX)) { st->status = ST_INVALID; goto finished; }
                    if ((int64_t)attempt >= o->max_attempts) { st->status = ST_STEP_LIMIT; goto finished; }
                    attempt = attempt + 1;
                    uint32_t wb[4];
                    draw_block(seed, sim, attempt, PURPOSE_SSA, 0, 0, wb);
                    double u1 = oracle_u01(wb[0], wb[1]);
                    double u2 = oracle_u01(wb[2], wb[3]);
                    double tau = -oracle_log(u1) / a0;
                    double t_new = t + tau;
                    /* samples strictly before the event see the pre-event state */
                    record_until(out, N, x, T, S, &ks, t_new, 1);
                    if (t_new > t_end) { t = t_end; goto finished; }
                    int jf = canon_select(w->a, M, levels, u2 * a0);
                    if (jf < 0) { st->status = ST_INVALID; goto finished; }
                    int overflow = 0;
                    for (int e = m->nu_ptr[jf]; e < m->nu_ptr[jf + 1]; ++e) {
                        int64_t nx = (int64_t)x[m->nu_sp[e]] + m->nu_val[e];
                        if (nx > INT32_MAX) overflow = 1;
                    }
                    if (overflow) { st->status = ST_OVERFLOW; goto finished; }
                    for (int e = m->nu_ptr[jf]; e < m->nu_ptr[jf + 1]; ++e)
                        x[m->nu_sp[e]] = (int32_t)((int64_t)x[m->nu_sp[e]] + m->nu_val[e]);
                    t = t_new;
                    st->ssa_steps += 1;
                    st->firings += 1;
                }
                leap_done = 1;
                break;
            }

            /* one tau-leap attempt (CGP 2006 procedure with CGP 2005 critical set) */
            if ((int64_t)attempt >= o->max_attempts) { st->status = ST_STEP_LIMIT; goto finished; }
            attempt = attempt + 1;
            uint32_t wl[4];
            draw_block(seed, sim, attempt, PURPOSE_LEAP, 0, 0, wl);
            double u_tau = oracle_u01(wl[0], wl[1]);
            double u_sel = oracle_u01(wl[2], wl[3]);
            double tau2 = (a0c > 0.0) ? -oracle_log(u_tau) / a0c : INFINITY;
            double t_stop = (ks < S) ? T[ks] : t_end;
            double delta = t_stop - t;
            double tau;
            int jc = -1, clamp = 0;
            if (tau2 <= tau1 && tau2 <= delta) {
                tau = tau2;
                jc = canon_select(w->a_crit, M, levels_c, u_sel * a0c);
            } else if (delta <= tau1) {
                tau = delta;
                clamp = 1;
            } else {
                tau = tau1;
            }
            int kover = 0, krej = 0;
            for (int j = 0; j < M; ++j) {
                if (w->crit[j]) { w->k[j] = (j == jc) ? 1 : 0; continue; }
                double lam = w->a[j] * tau;
                int64_t kj = (o->mode == MODE_CLE && lam >= CLE_MIN_MEAN)
                                 ? oracle_normal_leap(lam, seed, sim, attempt, (uint32_t)j)
                                 : oracle_poisson(lam, seed, sim, attempt, (uint32_t)j);
                if (kj < 0) krej = 1;
                else if (kj > COUNT_LIMIT) kover = 1;
                w->k[j] = kj;
            }
            if (krej) { st->status = ST_REJECT_LIMIT; goto finished; }
            if (kover) { st->status = ST_OVERFLOW; goto finished; }
            for (int i = 0; i < N; ++i) w->xnew[i] = x[i];
            for (int j = 0; j < M; ++j) {
                if (w->k[j] == 0) continue;
                for (int e = m->nu_ptr[j]; e < m->nu_ptr[j + 1]; ++e)
                    w->xnew[m->nu_sp[e]] += w->k[j] * (int64_t)m->nu_val[e];
            }
            int neg = 0, big = 0;
            for (int i = 0; i < N; ++i) {
                if (w->xnew[i] < 0) neg = 1;
                if (w->xnew[i] > INT32_MAX) big = 1;
            }
            if (neg) {
                /* CGP 2006: reduce tau' by half and return to the SSA test */
                st->rejected += 1;
                halvings = halvings + 1;
                if (halvings > o->max_halvings) { st->status = ST_REJECT_LIMIT; goto finished; }
                tau1 = tau1 / 2.0;
                continue;
            }
            if (big) { st->status = ST_OVERFLOW; goto finished; }
            int64_t fired = 0;
            for (int j = 0; j < M; ++j) fired += w->k[j];
            for (int i = 0; i < N; ++i) x[i] = (int32_t)w->xnew[i];
            t = clamp ? t_stop : t + tau;
            st->leaps += 1;
            st->firings += fired;
            leap_done = 1;
        }
    }
finished:
    record_rest(out, N, x, S, &ks);
    st->t_final = t;
    st->attempts = attempt;
    free(x);
}

/* ------------------------------------------------------------------ */
/* Batch entry point                                                     */
/* ------------------------------------------------------------------ */
/* Simulates rows r = 0..n_rows-1.  Row r uses params[r*M..], x0[r*N..] and
 * the random stream of simulation index sim_ids[r] (or sim_offset + r when
 * sim_ids is NULL), so any subset of a large batch can be recomputed alone.
 * samples: [n_rows][S][N] int32; stats: [n_rows].  Returns 0, or -1 on an
 * invalid model. */
int oracle_simulate(int32_t N, int32_t M,
                    const int32_t *react_ptr, const int32_t *react_species, const int32_t *react_coef,
                    const int32_t *prod_ptr, const int32_t *prod_species, const int32_t *prod_coef,
                    int64_t n_rows, const int64_t *sim_ids, int64_t sim_offset,
                    const double *params, const int32_t *x0, double t_end,
                    const double *sample_times, int32_t S, uint64_t seed,
                    const oracle_opts *opts, int32_t *samples, oracle_stats *stats, int n_threads)
{
    model_t m;
    if (model_build(&m, N, M, react_ptr, react_species, react_coef,
                    prod_ptr, prod_species, prod_coef) != 0) {
        model_free(&m);
        return -1;
    }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        scratch_t w;
        size_t MM = (size_t)(M > 0 ? M : 1), NN = (size_t)(N > 0 ? N : 1);
        w.a = malloc(sizeof(double) * MM);
        w.a_crit = malloc(sizeof(double) * MM);
        w.mu = malloc(sizeof(double) * NN);
        w.sig2 = malloc(sizeof(double) * NN);
        w.k = malloc(sizeof(int64_t) * MM);
        w.xnew = malloc(sizeof(int64_t) * NN);
        w.crit = calloc(MM, sizeof(int));
        w.irs = calloc(NN, sizeof(int));
#pragma omp for schedule(dynamic, 1)
        for (int64_t r = 0; r < n_rows; ++r) {
            uint32_t sim = (uint32_t)(sim_ids ? sim_ids[r] : sim_offset + r);
            simulate_one(&m, opts, seed, sim, params + (size_t)r * M, x0 + (size_t)r * N, t_end,
                         sample_times, S, samples + (size_t)r * S * N, stats + r, &w);
        }
        free(w.a); free(w.a_crit); free(w.mu); free(w.sig2);
        free(w.k); free(w.xnew); free(w.crit); free(w.irs);
    }
    model_free(&m);
    return 0;
}


/* ------------------------------------------------------------------ */
/* Reaction-rate equations: deterministic integration of a batch         */
/* ------------------------------------------------------------------ */
/* The mean-field model of the network (Methods: for abundant species the
 * state follows the reaction-rate equations dX/dt = sum_j nu_j a_j(X) with
 * continuous X; the stochastic 2X propensity c x(x-1)/2 becomes c x^2/2),
 * one system per parameter set, integrated by the Dormand-Prince 5(4)
 * pair (Dormand & Prince, J. Comput. Appl. Math. 6, 1980) with its FSAL
 * property and a power-of-two step controller:
 *   - h starts at t_last / 64 (t_last = the last sample time);
 *   - a step whose scaled error err = max_i |e_i| / (atol + rtol max(|x_i|,
 *     |x_new_i|)) is <= 1 is accepted; after an accepted step that was not
 *     shortened to land on a sample time, h doubles when err <= 2^-6;
 *   - a rejected step halves the step it tried;
 *   - a step that would pass the next sample time is shortened to end on it
 *     exactly, and the state there is recorded.
 * Every quantity is one correctly rounded IEEE operation in the order
 * written.  Accepted steps are counted in stats.leaps, rejected ones in
 * stats.rejected; accepted + rejected >= max_steps stops the system with
 * STEP_LIMIT, a non-finite state with INVALID, and the remaining samples
 * repeat the last state. */
static const double DP_A21 = 1.0 / 5.0;
static const double DP_A31 = 3.0 / 40.0, DP_A32 = 9.0 / 40.0;
static const double DP_A41 = 44.0 / 45.0, DP_A42 = -56.0 / 15.0, DP_A43 = 32.0 / 9.0;
static const double DP_A51 = 19372.0 / 6561.0, DP_A52 = -25360.0 / 2187.0, DP_A53 = 64448.0 / 6561.0,
                    DP_A54 = -212.0 / 729.0;
static const double DP_A61 = 9017.0 / 3168.0, DP_A62 = -355.0 / 33.0, DP_A63 = 46732.0 / 5247.0,
                    DP_A64 = 49.0 / 176.0, DP_A65 = -5103.0 / 18656.0;
static const double DP_B1 = 35.0 / 384.0, DP_B3 = 500.0 / 1113.0, DP_B4 = 125.0 / 192.0,
                    DP_B5 = -2187.0 / 6784.0, DP_B6 = 11.0 / 84.0;
/* error weights b - b*, b* the embedded fourth-order weights */
static const double DP_E1 = 35.0 / 384.0 - 5179.0 / 57600.0, DP_E3 = 500.0 / 1113.0 - 7571.0 / 16695.0,
                    DP_E4 = 125.0 / 192.0 - 393.0 / 640.0, DP_E5 = -2187.0 / 6784.0 - (-92097.0 / 339200.0),
                    DP_E6 = 11.0 / 84.0 - 187.0 / 2100.0, DP_E7 = 0.0 - 1.0 / 40.0;

/* f = dX/dt at state x: a_j by mass action (mean-field), then per species
 * the sum over the reactions that change it, in increasing j. */
static void rre_rhs(const model_t *m, const double *c, const double *x, double *a, double *f)
{
    for (int j = 0; j < m->M; ++j) {
        switch (m->r_kind[j]) {
        case 0: a[j] = c[j]; break;
        case 1: a[j] = c[j] * x[m->r_sp0[j]]; break;
        case 2: a[j] = (c[j] * x[m->r_sp0[j]]) * x[m->r_sp1[j]]; break;
        default: a[j] = c[j] * ((x[m->r_sp0[j]] * x[m->r_sp0[j]]) * 0.5); break;
        }
    }
    for (int i = 0; i < m->N; ++i) f[i] = 0.0;
    int *started = calloc((size_t)m->N, sizeof(int));
    for (int j = 0; j < m->M; ++j) {
        for (int e = m->nu_ptr[j]; e < m->nu_ptr[j + 1]; ++e) {
            int i = m->nu_sp[e];
            double t = (double)m->nu_val[e] * a[j];
            f[i] = started[i] ? f[i] + t : t;
            started[i] = 1;
        }
    }
    free(started);
}

static void rre_one(const model_t *m, const double *c, const int32_t *x0i, const double *T, int S,
                    double rtol, double atol, int64_t max_steps, double *out, oracle_stats *st)
{
    const int N = m->N;
    size_t NN = (size_t)(N > 0 ? N : 1), MM = (size_t)(m->M > 0 ? m->M : 1);
    double *x = malloc(sizeof(double) * NN), *xs = malloc(sizeof(double) * NN), *xn = malloc(sizeof(double) * NN);
    double *k[8], *a = malloc(sizeof(double) * MM);
    for (int q = 1; q <= 7; ++q) k[q] = malloc(sizeof(double) * NN);
    for (int i = 0; i < N; ++i) x[i] = (double)x0i[i];
    memset(st, 0, sizeof *st);
    st->status = ST_OK;
    double t = 0.0;
    double h = (S > 0) ? T[S - 1] / 64.0 : 0.0;
    rre_rhs(m, c, x, a, k[1]);
    int ks = 0;
    while (ks < S) {
        const double target = T[ks];
        while (t < target && st->status == ST_OK) {
            if (st->leaps + st->rejected >= max_steps) { st->status = ST_STEP_LIMIT; break; }
            double hh = h;
            int clamped = 0;
            if (t + hh >= target) { hh = target - t; clamped = 1; }
            for (int i = 0; i < N; ++i) xs[i] = x[i] + hh * (DP_A21 * k[1][i]);
            rre_rhs(m, c, xs, a, k[2]);
            for (int i = 0; i < N; ++i) { double s = DP_A31 * k[1][i]; s = s + DP_A32 * k[2][i]; xs[i] = x[i] + hh * s; }
            rre_rhs(m, c, xs, a, k[3]);
            for (int i = 0; i < N; ++i) {
                double s = DP_A41 * k[1][i]; s = s + DP_A42 * k[2][i]; s = s + DP_A43 * k[3][i];
                xs[i] = x[i] + hh * s;
            }
            rre_rhs(m, c, xs, a, k[4]);
            for (int i = 0; i < N; ++i) {
                double s = DP_A51 * k[1][i]; s = s + DP_A52 * k[2][i]; s = s + DP_A53 * k[3][i]; s = s + DP_A54 * k[4][i];
                xs[i] = x[i] + hh * s;
            }
            rre_rhs(m, c, xs, a, k[5]);
            for (int i = 0; i < N; ++i) {
                double s = DP_A61 * k[1][i]; s = s + DP_A62 * k[2][i]; s = s + DP_A63 * k[3][i]; s = s + DP_A64 * k[4][i];
                s = s + DP_A65 * k[5][i];
                xs[i] = x[i] + hh * s;
            }
            rre_rhs(m, c, xs, a, k[6]);
            for (int i = 0; i < N; ++i) {
                double s = DP_B1 * k[1][i]; s = s + DP_B3 * k[3][i]; s = s + DP_B4 * k[4][i]; s = s + DP_B5 * k[5][i];
                s = s + DP_B6 * k[6][i];
                xn[i] = x[i] + hh * s;
            }
            rre_rhs(m, c, xn, a, k[7]);
            double err = 0.0;
            int bad = 0;
            for (int i = 0; i < N; ++i) {
                double s = DP_E1 * k[1][i]; s = s + DP_E3 * k[3][i]; s = s + DP_E4 * k[4][i]; s = s + DP_E5 * k[5][i];
                s = s + DP_E6 * k[6][i]; s = s + DP_E7 * k[7][i];
                double ei = fabs(hh * s);
                double sc = atol + rtol * fmax(fabs(x[i]), fabs(xn[i]));
                double r = ei / sc;
                if (!(r == r) || !isfinite(xn[i])) bad = 1;
                if (r > err) err = r;
            }
            if (bad) { st->status = ST_INVALID; break; }
            if (err <= 1.0) {
                t = clamped ? target : t + hh;
                for (int i = 0; i < N; ++i) { x[i] = xn[i]; k[1][i] = k[7][i]; }
                st->leaps += 1;
                if (!clamped && err <= 0x1p-6) h = 2.0 * h;
            } else {
                st->rejected += 1;
                h = hh * 0.5;
            }
        }
        for (int i = 0; i < N; ++i) out[(size_t)ks * N + i] = x[i];
        ++ks;
    }
    st->attempts = st->leaps + st->rejected;
    st->t_final = t;
    free(x); free(xs); free(xn); free(a);
    for (int q = 1; q <= 7; ++q) free(k[q]);
}

int oracle_rre(int32_t N, int32_t M,
               const int32_t *react_ptr, const int32_t *react_species, const int32_t *react_coef,
               const int32_t *prod_ptr, const int32_t *prod_species, const int32_t *prod_coef,
               int64_t n_rows, const double *params, const int32_t *x0, const double *sample_times, int32_t S,
               double rtol, double atol, int64_t max_steps, double *out, oracle_stats *stats)
{
    model_t m;
    if (model_build(&m, N, M, react_ptr, react_species, react_coef, prod_ptr, prod_species, prod_coef) != 0) {
        model_free(&m);
        return -1;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < n_rows; ++r)
        rre_one(&m, params + (size_t)r * M, x0 + (size_t)r * N, sample_times, S, rtol, atol, max_steps,
                out + (size_t)r * S * N, stats + r);
    model_free(&m);
    return 0;
}


/* ------------------------------------------------------------------ */
/* Bulk entry points used by the pinning tests                           */
/* ------------------------------------------------------------------ */
void oracle_log_array(const double *x, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = oracle_log(x[i]);
}

void oracle_exp_array(const double *x, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = oracle_exp(x[i]);
}

void oracle_lnfact_array(const int64_t *k, double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = oracle_lnfact(k[i]);
}

/* n draws of Poisson(lam): draw i uses simulation index i, attempt 1, j 0. */
void oracle_poisson_array(double lam, uint64_t seed, int64_t n, int64_t *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_poisson(lam, seed, (uint32_t)i, 1u, 0u);
}

void oracle_normal_leap_array(double lam, uint64_t seed, int64_t n, int64_t *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = oracle_normal_leap(lam, seed, (uint32_t)i, 1u, 0u);
}

double oracle_canon_sum(const double *v, int32_t M)
{
    double levels[6][32];
    return canon_sum(v, M, levels);
}

int32_t oracle_canon_select(const double *v, int32_t M, double u)
{
    double levels[6][32];
    double total = canon_sum(v, M, levels);
    return canon_select(v, M, levels, u * total);
}

/* a_j, a0, the critical flags, a0c and tau' for one state (x, c). */
int oracle_leap_quantities(int32_t N, int32_t M,
                           const int32_t *react_ptr, const int32_t *react_species, const int32_t *react_coef,
                           const int32_t *prod_ptr, const int32_t *prod_species, const int32_t *prod_coef,
                           const double *c, const int32_t *x, const oracle_opts *opts,
                           double *a_out, int32_t *crit_out, double *scalars_out /* a0, a0c, tau1 */)
{
    model_t m;
    if (model_build(&m, N, M, react_ptr, react_species, react_coef,
                    prod_ptr, prod_species, prod_coef) != 0) {
        model_free(&m);
        return -1;
    }
    size_t MM = (size_t)(M > 0 ? M : 1), NN = (size_t)(N > 0 ? N : 1);
    scratch_t w;
    w.a = calloc(MM, sizeof(double)); w.a_crit = calloc(MM, sizeof(double));
    w.mu = malloc(sizeof(double) * NN); w.sig2 = malloc(sizeof(double) * NN);
    w.k = malloc(sizeof(int64_t) * MM); w.xnew = malloc(sizeof(int64_t) * NN);
    w.crit = calloc(MM, sizeof(int)); w.irs = calloc(NN, sizeof(int));
    double levels[6][32] = {{0}}, levels_c[6][32] = {{0}}, a0c = 0.0;
    for (int j = 0; j < M; ++j) w.a[j] = propensity(&m, j, c[j], x);
    double a0 = canon_sum(w.a, M, levels);
    double tau1 = leap_prepare(&m, opts, x, &w, levels_c, &a0c);
    for (int j = 0; j < M; ++j) { a_out[j] = w.a[j]; crit_out[j] = w.crit[j]; }
    scalars_out[0] = a0; scalars_out[1] = a0c; scalars_out[2] = tau1;
    free(w.a); free(w.a_crit); free(w.mu); free(w.sig2); free(w.k); free(w.xnew);
    free(w.crit); free(w.irs);
    model_free(&m);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

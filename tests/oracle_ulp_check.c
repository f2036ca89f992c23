/* The oracle's ln and exp against the C library's, over 10^8 inputs each:
 * prints the largest distance in ulps and how many inputs lie more than one
 * ulp away.  Built and run by tests/test_oracle_primitives.py, linked with
 * the oracle library. */
#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

double oracle_log(double x);
double oracle_exp(double x);

/* doubles mapped to integers in the same order, so that a difference of
 * mapped values is a distance in ulps */
static int64_t ordered(double x)
{
    int64_t i;
    memcpy(&i, &x, 8);
    return i < 0 ? INT64_MIN - i : i;
}

static uint64_t state = 88172645463325252ull;
static uint64_t next(void)   /* xorshift64 */
{
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return state;
}

static double u53(uint64_t r) { return (double)(r >> 11) * 0x1p-53; }

int main(int argc, char **argv)
{
    long n = argc > 1 ? atol(argv[1]) : 100000000L;
    int64_t max_log = 0, max_exp = 0, max_sub = 0;
    long over_log = 0, over_exp = 0, over_sub = 0;
    for (long i = 0; i < n; ++i) {
        double x;
        uint64_t r = next();
        switch (i & 3) {
        case 0: {   /* every positive finite binade */
            uint64_t b = r & 0x7fefffffffffffffull;
            memcpy(&x, &b, 8);
            if (x == 0.0) x = 1.0;
            break;
        }
        case 1: x = u53(r) + 0x1p-54; break;                        /* uniforms in (0, 1) */
        case 2: x = 1.0 + (u53(r) - 0.5) * 0x1p-10; break;           /* near 1 */
        default: x = 0.5 + u53(r) * 1.5; break;                      /* [0.5, 2) */
        }
        int64_t d = ordered(oracle_log(x)) - ordered(log(x));
        if (d < 0) d = -d;
        if (d > max_log) max_log = d;
        over_log += d > 1;

        double e = (i & 1) ? (u53(next()) - 0.5) * 2.0 : -708.3 + u53(next()) * 1417.0;
        d = ordered(oracle_exp(e)) - ordered(exp(e));
        if (d < 0) d = -d;
        if (d > max_exp) max_exp = d;
        over_exp += d > 1;

        /* results in the subnormal range */
        double s = -745.1 + u53(next()) * (745.1 - 708.4);
        d = ordered(oracle_exp(s)) - ordered(exp(s));
        if (d < 0) d = -d;
        if (d > max_sub) max_sub = d;
        over_sub += d > 1;
    }
    printf("%ld %lld %ld %lld %ld %lld %ld\n", n, (long long)max_log, over_log, (long long)max_exp, over_exp,
           (long long)max_sub, over_sub);
    return 0;
}

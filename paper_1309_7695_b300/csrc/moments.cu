// Sweep moments across the simulations of a batch: per cell c = (sample k,
// species i), the mean and the unbiased variance of the recorded counts.
//
// The lane kernels accumulate, per cell, the exact integer sums
//   S1 = sum x,   S2 = sum x^2   (S2 as hi * 2^32 + lo, two 64-bit words),
// with 64-bit atomic adds while they record each sample, so the trajectory
// array need not be written at all.  This kernel turns the sums into
//   mean = RN(RN(S1) / RN(n)),
//   var  = RN(RN(n S2 - S1^2) / RN(n (n - 1)))   (0 for n < 2),
// where n S2 - S1^2 = n^2 * (sample variance) (n - 1)/n is formed exactly in
// 128-bit integers.  Both results are fixed functions of the integer sums,
// so they do not depend on the order in which the atomics landed.
#include <stdint.h>

#include "engine.h"

namespace tl {
namespace {

// Round-to-nearest-even conversion of an unsigned 128-bit integer to double.
__device__ __forceinline__ double u128_to_double_rn(unsigned __int128 v)
{
    const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
    if (hi == 0) return __ull2double_rn(lo);
    const int p = 128 - __clzll((long long)hi);          // bit length, 65..128
    const int drop = p - 53;                               // >= 12
    unsigned long long mant = (unsigned long long)(v >> drop);
    const unsigned __int128 rem = v & (((unsigned __int128)1 << drop) - 1);
    const unsigned __int128 half = (unsigned __int128)1 << (drop - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;   // may carry to 2^53: still exact below
    return ldexp((double)mant, drop);
}

__global__ void moments_finalize(const unsigned long long *__restrict__ acc, long long n, int cells,
                                 double *__restrict__ mean, double *__restrict__ var)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    const unsigned long long s1 = acc[3 * (size_t)c], lo = acc[3 * (size_t)c + 1], hi = acc[3 * (size_t)c + 2];
    const unsigned long long un = (unsigned long long)n;
    mean[c] = __ull2double_rn(s1) / __ull2double_rn(un);
    if (n < 2) {
        var[c] = 0.0;
        return;
    }
    const unsigned __int128 s2 = ((unsigned __int128)hi << 32) + lo;
    const unsigned __int128 num = (unsigned __int128)un * s2 - (unsigned __int128)s1 * s1;
    var[c] = u128_to_double_rn(num) / __ull2double_rn(un * (un - 1));
}

}  // namespace

cudaError_t launch_moments_finalize(const unsigned long long *acc, long long n, int cells, double *mean, double *var,
                                    cudaStream_t s)
{
    if (cells <= 0) return cudaSuccess;
    moments_finalize<<<(cells + 255) / 256, 256, 0, s>>>(acc, n, cells, mean, var);
    return cudaGetLastError();
}

}  // namespace tl

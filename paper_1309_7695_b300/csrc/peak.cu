// Issue-rate microbenchmarks: the denominators of the ALU rooflines.
//
// The simulation kernels are bound by FP64 (reference mode) or FP32 (fast
// mode) instruction issue, not by HBM or tensor cores.  Neither figure is
// among the measured peaks, so the library measures them itself:
// every thread of a full-device grid runs kChains independent add chains
// of `iters` dependent adds each (no fused multiply-add: this unit is built
// with -fmad=false), and the rate is the number of adds divided by the
// CUDA-event time of the launch.  A single warp with one dependent chain
// gives the latency of one FP64 add in SM clock cycles.
#include <algorithm>

#include "engine.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) add_chains(T *out, int iters, T step)
{
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] + step;
    }
    T s = a[0];
#pragma unroll
    for (int c = 1; c < kChains; ++c) s = s + a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dep_chain_f64(double *out, long long *cycles, int iters, double step)
{
    double a = (double)threadIdx.x;
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) a = a + step;
    const long long t1 = clock64();
    out[threadIdx.x] = a;
    if (threadIdx.x == 0) *cycles = t1 - t0;
}

template <class T>
cudaError_t time_adds(int sms, cudaStream_t s, double *rate)
{
    const int blocks = sms * (2048 / kThreads);
    const int iters = 4096;
    T *out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, sizeof(T) * (size_t)blocks * kThreads, s);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) {
            add_chains<T><<<blocks, kThreads, 0, s>>>(out, iters, (T)1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;   // rep 0 warms up
    }
    if (e == cudaSuccess) *rate = (double)blocks * kThreads * kChains * iters / (best * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const cudaError_t ef = cudaFreeAsync(out, s);
    return e != cudaSuccess ? e : ef;
}

}  // namespace

extern "C" int ssa_measure_issue_rates(void *stream, double *fp64_adds_per_s, double *fp32_adds_per_s,
                                       double *fp64_add_latency_cycles)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SSA_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double r64 = 0.0, r32 = 0.0;
    if (time_adds<double>(sms, s, &r64) != cudaSuccess) return SSA_ECUDA;
    if (time_adds<float>(sms, s, &r32) != cudaSuccess) return SSA_ECUDA;
    double *out = nullptr;
    long long *cyc = nullptr;
    const int iters = 4096;
    cudaError_t e = cudaMallocAsync(&out, sizeof(double) * 32, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&cyc, sizeof(long long), s);
    long long cycles = 0;
    if (e == cudaSuccess) {
        dep_chain_f64<<<1, 32, 0, s>>>(out, cyc, iters, 1.0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cycles, cyc, sizeof cycles, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (out) cudaFreeAsync(out, s);
    if (cyc) cudaFreeAsync(cyc, s);
    if (e != cudaSuccess) return SSA_ECUDA;
    if (fp64_adds_per_s) *fp64_adds_per_s = r64;
    if (fp32_adds_per_s) *fp32_adds_per_s = r32;
    if (fp64_add_latency_cycles) *fp64_add_latency_cycles = (double)cycles / iters;
    return SSA_OK;
}

// Measurement aid (no counterpart in the paper): the FP64 arithmetic rate of
// the GPU, the denominator against which the FP64 stored-velocity step (bound
// by the FP64 pipe, not by HBM) is reported.  Every thread runs eight
// independent FMA chains in registers; nothing is read from memory.
#include "mr_internal.cuh"

namespace mr {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double* out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (double)threadIdx.x + (double)c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0 && out) out[0] = s;   // never true for a, b > 0: keeps the chains live
}

}  // namespace
}  // namespace mr

using namespace mr;

extern "C" int mr_fp64_fma_rate(double* tflops, mr_stream stream)
{
    if (!tflops) return set_error(MR_ERR_ARG, "mr_fp64_fma_rate: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(e, "mr_fp64_fma_rate: device query");
    const int blocks = sms * 8, threads = 256, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    // one untimed launch, then the best of three
    for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            k_fp64_fma<<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999999, 1e-7);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_check(e, "mr_fp64_fma_rate");
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * (double)threads;
    *tflops = flops / ((double)best * 1e-3) / 1e12;
    return MR_OK;
}

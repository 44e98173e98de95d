// FP64 fused multiply-add rate of the device: a register-only kernel (no memory
// traffic in its loop), timed with CUDA events on the caller's stream.  It measures
// the denominator the FP64-bound stage kernels are compared with; it changes no
// device setting.  Not part of the paper's method.
#include <cuda_runtime.h>

#include "../../include/grmhd.h"

namespace grmhd {
void set_last_error(const char* msg);
}

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kIters = 4096;   // iterations of the chains

// each thread runs kChains independent chains x <- x * a + b, kIters times; the
// result is stored only when it is impossible (a guard the compiler cannot prove),
// so the loop is not removed and nothing is written
__global__ void __launch_bounds__(256) k_fp64_fma(double a, double b, double* __restrict__ sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < kIters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == -1.2345e300) sink[0] = s;
}

}  // namespace

extern "C" grmhd_status grmhd_fp64_fma_rate(double* tflops, grmhd_stream_t stream)
{
    if (!tflops) {
        grmhd::set_last_error("grmhd_fp64_fma_rate: tflops is NULL");
        return GRMHD_ERR_ARG;
    }
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || nsm < 1) {
        grmhd::set_last_error("grmhd_fp64_fma_rate: no CUDA device");
        return GRMHD_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = nsm * 8, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GRMHD_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GRMHD_ERR_CUDA;
    }
    // a (slightly below 1) and b keep every chain bounded
    k_fp64_fma<<<blocks, threads, 0, st>>>(0.999999, 1e-6, nullptr);   // warm-up
    float best = 0.0f;
    for (int rep = 0; rep < 5 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, st);
        k_fp64_fma<<<blocks, threads, 0, st>>>(0.999999, 1e-6, nullptr);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || !(best > 0.0f)) {
        grmhd::set_last_error("grmhd_fp64_fma_rate: kernel or timing failed");
        return GRMHD_ERR_CUDA;
    }
    const double flop = 2.0 * kChains * (double)kIters * blocks * threads;
    *tflops = flop / (best * 1e-3) / 1e12;
    return GRMHD_OK;
}

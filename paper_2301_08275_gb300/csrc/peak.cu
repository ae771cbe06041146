// peak.cu - measured arithmetic peak of this GPU for the roofline of the
// complex128 workloads (a measurement aid; the paper has no counterpart).
//
// gpe_measure_fp64_peak launches a kernel of independent double-precision
// fused multiply-add chains (eight per thread, no memory traffic inside the
// timed loop) on every SM and returns the achieved FLOP/s (2 per FMA), timed
// with CUDA events on the given stream.  The complex128 sweeps of the library
// are bound by this rate, not by HBM.
#include <cuda_runtime.h>

#include "../../include/gpe.h"
#include "gpe_internal.h"

namespace {

__device__ double g_peak_sink;   // keeps the chains live; written by one thread

__global__ void __launch_bounds__(256) k_dfma_chains(int iters, double a, double b)
{
    double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (threadIdx.x == 0 && blockIdx.x == 0) g_peak_sink = s;
}

}  // namespace

extern "C" gpe_status gpe_measure_fp64_peak(void *cuda_stream, double *flops_per_s)
{
    using namespace gpe;
    if (!flops_per_s) {
        set_last_error("gpe_measure_fp64_peak: NULL argument");
        return GPE_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("gpe_measure_fp64_peak: no device");
        return GPE_ECUDA;
    }
    const int blocks = sms * 8, threads = 256, iters = 512;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gpe_status rc = GPE_OK;
    float best = 0.0f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        set_last_error("gpe_measure_fp64_peak: cudaEventCreate failed");
        rc = GPE_ECUDA;
    }
    for (int rep = 0; rc == GPE_OK && rep < 4; ++rep) {
        cudaEventRecord(e0, st);
        k_dfma_chains<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            rc = GPE_ECUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;     // the first launch warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != GPE_OK) return rc;
    const double flop = 2.0 * 64.0 * (double)iters * (double)blocks * threads;
    *flops_per_s = flop / (best * 1e-3);
    return GPE_OK;
}

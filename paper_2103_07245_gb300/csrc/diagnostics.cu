// Diagnostics of the library's device helpers (not part of the paper's method):
// pbpqlp_newton_check evaluates the Newton-refined reciprocal and reciprocal
// square root and the one-step Goldschmidt reciprocal that replace FP64
// division and square root on the pivot chains of the Cholesky and QR
// kernels, so that tests can hold them to an ulp bound against correctly
// rounded results.
#include "../../include/pbpqlp.h"
#include "internal.h"
#include "newton_device.cuh"

namespace {

__global__ void k_newton_check(int64_t n, const double* __restrict__ d, double* __restrict__ rcp,
                               double* __restrict__ rsq, double* __restrict__ rgs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = d[i];
        rcp[i] = pbq::rcp_nr(x);
        rsq[i] = pbq::rsqrt_nr(x);
        if (rgs) rgs[i] = pbq::rcp_gs(x);
    }
}

}  // namespace

extern "C" int pbpqlp_newton_check(const double* d, int64_t n, double* rcp, double* rsqrt, double* rcp_gs,
                                   void* stream) {
    if (n < 0 || (n > 0 && (!d || !rcp || !rsqrt))) return PBPQLP_EINVAL;
    if (n == 0) return PBPQLP_OK;
    const int64_t blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    k_newton_check<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, d, rcp, rsqrt, rcp_gs);
    pbq::count_launches(1);
    return cudaGetLastError() == cudaSuccess ? PBPQLP_OK : PBPQLP_ECUDA;
}

namespace {

// Independent FP64 FMA chains (8 per thread) for the issue-rate probe; the
// result is stored so the chains are not removed.
__global__ void __launch_bounds__(256) k_dfma_probe(int iters, double seed, double* __restrict__ sink) {
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + 1e-3 * (threadIdx.x + j);
    const double x = 1.0 - 1e-9, y = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.678) sink[blockIdx.x] = s;   // practically never true; keeps the work alive
}

}  // namespace

extern "C" int pbpqlp_fp64_rate_probe(double* sink, double* tflops_out, void* stream) {
    if (!sink || !tflops_out) return PBPQLP_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PBPQLP_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PBPQLP_ECUDA;
    const int blocks = sms * 4, threads = 256, iters = 4096;
    k_dfma_probe<<<blocks, threads, 0, s>>>(64, 1.0, sink);   // warm-up
    cudaEventRecord(e0, s);
    k_dfma_probe<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
    cudaEventRecord(e1, s);
    pbq::count_launches(2);
    int rc = PBPQLP_OK;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
        rc = PBPQLP_ECUDA;
    else
        *tflops_out = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

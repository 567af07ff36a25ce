// Diagnostics of the library's device helpers (not part of the paper's method):
// pbpqlp_newton_check evaluates the Newton-refined reciprocal and reciprocal
// square root and the one-step Goldschmidt reciprocal that replace FP64
// division and square root on the pivot chains of the Cholesky and QR
// kernels, so that tests can hold them to an ulp bound against correctly
// rounded results; pbpqlp_oz_convert_check evaluates both forms of the
// exact-integer-to-FP64 conversion that ends every FP64-accurate digit
// product, so that tests can hold them to Python's correctly rounded
// integer-to-float conversion.
#include "../../include/pbpqlp.h"
#include "internal.h"
#include "newton_device.cuh"
#include "oz_convert.cuh"

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

__global__ void k_oz_convert_check(int64_t n, const int64_t* __restrict__ hi, const int64_t* __restrict__ lo,
                                   const int* __restrict__ e, double* __restrict__ fast, double* __restrict__ exact) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        fast[i] = pbq::oz_to_double_fast(hi[i], lo[i], e[i]);
        exact[i] = pbq::oz_to_double(hi[i], lo[i], e[i]);
    }
}

}  // namespace

extern "C" int pbpqlp_oz_convert_check(const int64_t* hi, const int64_t* lo, const int* e, int64_t n, double* fast,
                                       double* exact, void* stream) {
    if (n < 0 || (n > 0 && (!hi || !lo || !e || !fast || !exact))) return PBPQLP_EINVAL;
    if (n == 0) return PBPQLP_OK;
    const int64_t blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    k_oz_convert_check<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, hi, lo, e, fast, exact);
    pbq::count_launches(1);
    return cudaGetLastError() == cudaSuccess ? PBPQLP_OK : PBPQLP_ECUDA;
}

namespace {

// The FP64 issue-rate probe runs the inner loop of a register-blocked FP64
// GEMM: each k step loads 4 values of a 64-row tile and 4 of a 64-column tile
// from shared memory and updates a 4 x 4 block of accumulators (16 FMA
// chains per thread).  The result is stored only on a sentinel value, so the
// work is kept.
__global__ void __launch_bounds__(256) k_dfma_probe(int iters, double seed, double* __restrict__ sink) {
    __shared__ double As[16][65], Bs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int e = tid; e < 16 * 64; e += 256) {
        As[e / 64][e % 64] = 1e-9 * (e % 61 + 1);
        Bs[e / 64][e % 64] = 1e-9 * (e % 59 + 1);
    }
    __syncthreads();
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = seed + 1e-3 * (i * 4 + j);
    for (int it = 0; it < iters; ++it) {
#pragma unroll 2
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
    }
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sum += acc[i][j];
    if (sum == 12345.678) sink[blockIdx.x] = sum;   // practically never true; keeps the work alive
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
    // 1, 2 and 4 CTAs of 256 threads per SM; the best rate is reported
    const int threads = 256, iters = 128;   // 16 k steps of 16 FMAs per iteration
    int rc = PBPQLP_OK;
    double best = 0.0;
    k_dfma_probe<<<sms, threads, 0, s>>>(64, 1.0, sink);   // warm-up
    pbq::count_launches(1);
    for (int per = 1; per <= 4 && rc == PBPQLP_OK; per *= 2) {
        const int blocks = sms * per;
        cudaEventRecord(e0, s);
        k_dfma_probe<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
        cudaEventRecord(e1, s);
        pbq::count_launches(1);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
            rc = PBPQLP_ECUDA;
            break;
        }
        const double tf = 2.0 * 16.0 * 16.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
        best = tf > best ? tf : best;
    }
    if (rc == PBPQLP_OK) *tflops_out = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

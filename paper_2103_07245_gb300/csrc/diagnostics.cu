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

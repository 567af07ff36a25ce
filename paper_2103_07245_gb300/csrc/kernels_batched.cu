// Work-list kernels of the batched path: each launch walks a list of units
// that may belong to different matrices (one CTA per unit), so a whole batch
// of uneven factorizations advances one step of Algorithm 3 per launch.
// The arithmetic is the single-matrix code (fp64_device.cuh).
#include "batched.h"
#include "fp64_device.cuh"

namespace pbq {

template <int TN, bool TA>
__global__ void __launch_bounds__(256) k_dgemm_list(const GemmUnit* __restrict__ units) {
    const GemmUnit u = units[blockIdx.x];
    if (u.cond && *u.cond == 0) return;
    dev_dgemm_tile<TN, TA>(u.M, u.N, u.A, u.lda, u.B, u.ldb, u.C, u.ldc, u.m0, u.kbeg, u.kend);
}

template <bool TA>
static cudaError_t dgemm_list_tn(int TN, const GemmUnit* units, int nunits, cudaStream_t s) {
    switch (TN) {
#define PBQ_L(T) case T: k_dgemm_list<T, TA><<<nunits, 256, 0, s>>>(units); break;
        PBQ_L(1) PBQ_L(2) PBQ_L(3) PBQ_L(4) PBQ_L(5) PBQ_L(6) PBQ_L(7)
        PBQ_L(8) PBQ_L(9) PBQ_L(10) PBQ_L(11) PBQ_L(12) PBQ_L(13) PBQ_L(14)
#undef PBQ_L
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dgemm_list(int TN, bool transA, const GemmUnit* units, int nunits, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    return transA ? dgemm_list_tn<true>(TN, units, nunits, s) : dgemm_list_tn<false>(TN, units, nunits, s);
}

__global__ void __launch_bounds__(256) k_reduce_list(const ReduceUnit* __restrict__ units) {
    const ReduceUnit u = units[blockIdx.x];
    if (u.cond && *u.cond == 0) return;
    const int64_t total = u.M * (int64_t)u.N;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int64_t i = e / u.N;
        const int c = (int)(e - i * u.N);
        const double* p = u.part + i * u.ldp + c;
        double acc = 0.0;
        for (int t = 0; t < u.S; ++t) acc += p[(int64_t)t * u.ps];
        u.C[i * u.ldc + c] = acc;
    }
}

cudaError_t launch_reduce_list(const ReduceUnit* units, int nunits, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    k_reduce_list<<<nunits, 256, 0, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_cholesky_list(const MatUnit* __restrict__ units) {
    extern __shared__ double sm[];
    const MatUnit& u = units[blockIdx.x];
    dev_cholesky(u.l, u.rows, u.G, u.Rp, u.status, u.ctl, u.pass, sm);
}

cudaError_t launch_cholesky_list(const MatUnit* units, int nunits, int lmax, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    const size_t smem = (size_t)(packed_tri(lmax) + 2 * (int64_t)lmax) * sizeof(double);
    cudaError_t e = func_smem_attr((const void*)k_cholesky_list, smem);
    if (e != cudaSuccess) return e;
    // 256 threads: the batched factors are small (l <= 224) and many CTAs share an SM
    k_cholesky_list<<<nunits, 256, smem, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

template <int U, typename T>
__global__ void __launch_bounds__(256) k_trsm_list(const TrsmUnit* __restrict__ units) {
    extern __shared__ __align__(16) unsigned char sraw[];
    T* sR = (T*)sraw;
    const TrsmUnit u = units[blockIdx.x];
    if (u.cond && *u.cond == 0) return;
    const int64_t P = (int64_t)u.l * (u.l + 1) / 2;
    for (int64_t e = threadIdx.x; e < P + u.l; e += blockDim.x) sR[e] = (T)u.Rp[e];
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    dev_trsm_rows<U, T>(u.l, sR, u.X, u.ldx, u.Y, u.ldy, u.r0 + warp, u.r1, 8);
}

template <typename T>
static cudaError_t trsm_list_t(const TrsmUnit* units, int nunits, int lmax, cudaStream_t s) {
    const size_t smem = (size_t)(packed_tri(lmax) + lmax) * sizeof(T);
    const int U = (lmax + 31) / 32;
    cudaError_t e = cudaSuccess;
    switch (U) {
#define PBQ_T(UU) case UU: \
        e = func_smem_attr((const void*)k_trsm_list<UU, T>, smem); \
        if (e != cudaSuccess) return e; \
        k_trsm_list<UU, T><<<nunits, 256, smem, s>>>(units); break;
        PBQ_T(1) PBQ_T(2) PBQ_T(3) PBQ_T(4) PBQ_T(5) PBQ_T(6) PBQ_T(7)
#undef PBQ_T
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trsm_list(const TrsmUnit* units, int nunits, int lmax, cudaStream_t s, bool f32) {
    if (nunits <= 0) return cudaSuccess;
    return f32 ? trsm_list_t<float>(units, nunits, lmax, s) : trsm_list_t<double>(units, nunits, lmax, s);
}

__global__ void __launch_bounds__(1024) k_small_qr_list(const MatUnit* __restrict__ units, int use_smem) {
    extern __shared__ double qsm[];
    const MatUnit& u = units[blockIdx.x];
    dev_small_qr(u.l, u.G, u.L, u.Pt, u.work, use_smem ? qsm : nullptr);
}

cudaError_t launch_small_qr_list(const MatUnit* units, int nunits, int lmax, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)lmax * lmax * sizeof(double);
    const bool fits = smem <= 220 * 1024;
    if (fits) {
        cudaError_t e = func_smem_attr((const void*)k_small_qr_list, smem);
        if (e != cudaSuccess) return e;
    }
    k_small_qr_list<<<nunits, 256, fits ? smem : 0, s>>>(units, fits ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_gaussian_list(const MatUnit* __restrict__ units) {
    const MatUnit& u = units[blockIdx.x];
    // pairs [b0, b1) of the matrix's stream; the last unit's b1 is the stream end
    const int64_t npairs = (u.rows * (int64_t)u.l + 1) / 2;
    const int64_t end = u.b1 < npairs ? u.b1 : npairs;
    for (int64_t b = u.b0 + threadIdx.x; b < end; b += blockDim.x)
        dev_gaussian(u.seed, u.rows, u.l, u.out, u.ld, b, npairs);   // one pair (stride past the end)
}

cudaError_t launch_gaussian_list(const MatUnit* units, int nunits, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    k_gaussian_list<<<nunits, 256, 0, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq

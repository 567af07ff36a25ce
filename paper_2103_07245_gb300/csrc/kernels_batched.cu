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
    // rows by warp, columns by lane (coalesced, no index division)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t i = warp; i < u.M; i += nw)
        for (int c = lane; c < u.N; c += 32) {
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
    // 512 threads: the per-column row updates of a small factor (l <= 224) split
    // over 16 warps, and four such CTAs share an SM (one wave for 600 matrices)
    k_cholesky_list<<<nunits, 512, smem, s>>>(units);
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

// Step t of the row solve and, recursively, the steps after it: every index
// into x is a compile-time constant, so the row stays in registers; row t of
// R (square layout, 16-byte aligned rows) is read as 16-byte broadcasts.
template <int T, int LMAX>
struct RowSolveF32 {
    static __device__ __forceinline__ void run(float (&x)[LMAX], int l, const float* __restrict__ sR,
                                               const float* __restrict__ sD) {
        if (T >= l) return;
        const float y = x[T] * sD[T];
        x[T] = y;
#pragma unroll
        for (int c4 = (T + 1) & ~3; c4 < LMAX; c4 += 4) {
            const float4 r = *reinterpret_cast<const float4*>(sR + T * LMAX + c4);
            if (c4 > T) x[c4] -= y * r.x;
            if (c4 + 1 > T) x[c4 + 1] -= y * r.y;
            if (c4 + 2 > T) x[c4 + 2] -= y * r.z;
            if (c4 + 3 > T) x[c4 + 3] -= y * r.w;
        }
        RowSolveF32<T + 1, LMAX>::run(x, l, sR, sD);
    }
};
template <int LMAX>
struct RowSolveF32<LMAX, LMAX> {
    static __device__ __forceinline__ void run(float (&)[LMAX], int, const float*, const float*) {}
};

// FP32 solves (TF32 modes), one row per thread: the row x[0 .. LMAX) sits in
// registers and the substitution is unrolled over the compile-time bound LMAX
// (columns past l are zero and stay zero).  Blocks of 128 rows pass through
// shared memory (row stride LMAX + 1: coalesced global loads and stores,
// conflict-free row reads); R (LMAX x LMAX, zero on and below the diagonal
// and past l) and 1 / diag are shared-memory broadcasts.  Same arithmetic, in
// the same order, as dev_trsm_rows<U, float>.
template <int LMAX>
__global__ void __launch_bounds__(128) k_trsm_rows_f32(const TrsmUnit* __restrict__ units) {
    constexpr int SX = LMAX + 1;
    extern __shared__ __align__(16) float sRf[];   // R [LMAX][LMAX], then 1 / diag [LMAX], then rows [128][SX]
    const TrsmUnit u = units[blockIdx.x];
    if (u.cond && *u.cond == 0) return;
    const int l = u.l;
    const int64_t P = (int64_t)l * (l + 1) / 2;
    float* sD = sRf + LMAX * LMAX;
    float* sX = sD + LMAX;
    constexpr int CW = (LMAX + 31) / 32;   // 32-column chunks of a row
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // loads are issued in batches (registers first, then shared memory) so
    // that many are in flight: these copies are latency-bound otherwise
    for (int t0 = warp; t0 < LMAX; t0 += 4 * 8) {
        float v[8][CW];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < CW; ++q) {
                const int t = t0 + 4 * j, c = lane + 32 * q;
                v[j][q] = (t < l && c > t && c < l) ? (float)u.Rp[pidx(l, t, 0) + c] : 0.f;
            }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int q = 0; q < CW; ++q) {
                const int t = t0 + 4 * j, c = lane + 32 * q;
                if (t < LMAX && c < LMAX) sRf[t * LMAX + c] = v[j][q];
            }
    }
    for (int t = tid; t < LMAX; t += 128) sD[t] = t < l ? (float)u.Rp[P + t] : 0.f;
    for (int64_t rb = u.r0; rb < u.r1; rb += 128) {
        const int nr = (int)(u.r1 - rb < 128 ? u.r1 - rb : 128);
        __syncthreads();   // R is in place; the previous block's rows are written out
        for (int i0 = warp; i0 < nr; i0 += 4 * 8) {
            float v[8][CW];
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int q = 0; q < CW; ++q) {
                    const int i = i0 + 4 * j, c = lane + 32 * q;
                    v[j][q] = (i < nr && c < l) ? (float)u.X[(rb + i) * u.ldx + c] : 0.f;
                }
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int q = 0; q < CW; ++q) {
                    const int i = i0 + 4 * j, c = lane + 32 * q;
                    if (i < nr && c < l) sX[i * SX + c] = v[j][q];
                }
        }
        __syncthreads();
        if (tid < nr) {
            float x[LMAX];
#pragma unroll
            for (int c = 0; c < LMAX; ++c) x[c] = c < l ? sX[tid * SX + c] : 0.f;
            RowSolveF32<0, LMAX>::run(x, l, sRf, sD);
#pragma unroll
            for (int c = 0; c < LMAX; ++c)
                if (c < l) sX[tid * SX + c] = x[c];
        }
        __syncthreads();
        for (int i = warp; i < nr; i += 4)
#pragma unroll
            for (int q = 0; q < CW; ++q) {
                const int c = lane + 32 * q;
                if (c < l) u.Y[(rb + i) * u.ldy + c] = (double)sX[i * SX + c];
            }
    }
}

static cudaError_t trsm_rows_f32(const TrsmUnit* units, int nunits, int lmax, cudaStream_t s) {
    const int LM = (lmax + 15) / 16 * 16;
    const size_t smem = (size_t)(LM * LM + LM + 128 * (LM + 1)) * sizeof(float);
    cudaError_t e = cudaSuccess;
    switch (LM) {
#define PBQ_R(LL) case LL: \
        e = func_smem_attr((const void*)k_trsm_rows_f32<LL>, smem); \
        if (e != cudaSuccess) return e; \
        k_trsm_rows_f32<LL><<<nunits, 128, smem, s>>>(units); break;
        PBQ_R(16) PBQ_R(32) PBQ_R(48) PBQ_R(64) PBQ_R(80) PBQ_R(96) PBQ_R(112) PBQ_R(128)
#undef PBQ_R
        default: return trsm_list_t<float>(units, nunits, lmax, s);   // l > 128: warp per row
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trsm_list(const TrsmUnit* units, int nunits, int lmax, cudaStream_t s, bool f32) {
    if (nunits <= 0) return cudaSuccess;
    return f32 ? trsm_rows_f32(units, nunits, lmax, s) : trsm_list_t<double>(units, nunits, lmax, s);
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

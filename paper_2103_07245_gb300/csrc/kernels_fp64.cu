// FP64 kernels of the PbP-QLP path (Algorithm 3): Gaussian test matrix,
// skinny DFMA GEMMs for the products with A and A^T, deterministic split-K
// reduction, CholeskyQR passes (Gram -> Cholesky -> row-wise triangular
// solve) with a shifted retry, and the one-CTA Householder QR of R^T.
//
// GB300 has 2 FP64 FMA lanes per SM per clock (~1.2 TFLOP/s for the chip), so
// every FP64 kernel here is DFMA-issue bound and the tiling aims at keeping
// all 152 SMs issuing DFMAs with no wasted (padded) lanes.
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "fp64_device.cuh"

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

namespace pbq {

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t func_smem_attr(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[{dev, func}];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

// With PBPQLP_DEBUG=1 in the environment, failing CUDA calls of the library
// are reported on stderr (call site and CUDA's error text).
cudaError_t debug_report(cudaError_t e, const char* what, const char* file, int line) {
    static const bool on = [] {
        const char* v = std::getenv("PBPQLP_DEBUG");
        return v && v[0] == '1';
    }();
    if (e != cudaSuccess && on) std::fprintf(stderr, "pbpqlp: %s:%d: %s -> %s\n", file, line, what, cudaGetErrorString(e));
    return e;
}
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller.
// ---------------------------------------------------------------------------
__global__ void k_gaussian(uint64_t seed, int64_t rows, int l, double* __restrict__ out, int64_t ld) {
    dev_gaussian(seed, rows, l, out, ld, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

cudaError_t launch_gaussian(uint64_t seed, int64_t rows, int l, double* out, int64_t ld, cudaStream_t s) {
    const int64_t npairs = (rows * (int64_t)l + 1) / 2;
    int64_t blocks = (npairs + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_gaussian<<<(unsigned)blocks, 256, 0, s>>>(seed, rows, l, out, ld);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Skinny FP64 GEMM: C (M x N, N <= 224) = op(A) B.  256 threads = 16 column
// lanes x 16 row groups; a thread owns 4 rows x TN columns (column stride 16),
// so the CTA tile is 64 x 16*TN and TN = ceil(N/16) wastes < 16 columns.
// The split-K index is blockIdx.y.
// ---------------------------------------------------------------------------
template <int TN, bool TA>
__global__ void __launch_bounds__(256)
k_dgemm_skinny(int64_t M, int N, int64_t K, const double* __restrict__ A, int64_t lda,
               const double* __restrict__ B, int64_t ldb, double* __restrict__ C, int64_t ldc,
               int64_t kchunk, int64_t part_stride, const int* __restrict__ cond) {
    if (cond && *cond == 0) return;
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = (kbeg + kchunk < K) ? kbeg + kchunk : K;
    dev_dgemm_tile<TN, TA>(M, N, A, lda, B, ldb, C + (int64_t)blockIdx.y * part_stride, ldc,
                           (int64_t)blockIdx.x * kGemmBM, kbeg, kend);
}

template <bool TA>
static cudaError_t dispatch_dgemm(int TN, dim3 grid, int64_t M, int N, int64_t K, const double* A, int64_t lda,
                                  const double* B, int64_t ldb, double* C, int64_t ldc, int64_t kchunk,
                                  int64_t ps, const int* cond, cudaStream_t s) {
#define PBQ_CASE(T) case T: k_dgemm_skinny<T, TA><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, kchunk, ps, cond); break;
    switch (TN) {
        PBQ_CASE(1) PBQ_CASE(2) PBQ_CASE(3) PBQ_CASE(4) PBQ_CASE(5) PBQ_CASE(6) PBQ_CASE(7)
        PBQ_CASE(8) PBQ_CASE(9) PBQ_CASE(10) PBQ_CASE(11) PBQ_CASE(12) PBQ_CASE(13) PBQ_CASE(14)
        default: return cudaErrorInvalidValue;
    }
#undef PBQ_CASE
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_dgemm_skinny(bool transA, int64_t M, int N, int64_t K, const double* A, int64_t lda,
                                const double* B, int64_t ldb, double* C, int64_t ldc, int S, int64_t kchunk,
                                int64_t part_stride, const int* cond, cudaStream_t s) {
    if (N < 1 || N > kMaxEll || M < 1 || S < 1) return cudaErrorInvalidValue;
    const int TN = (N + 15) / 16;
    dim3 grid((unsigned)((M + kGemmBM - 1) / kGemmBM), (unsigned)S);
    return transA ? dispatch_dgemm<true>(TN, grid, M, N, K, A, lda, B, ldb, C, ldc, kchunk, part_stride, cond, s)
                  : dispatch_dgemm<false>(TN, grid, M, N, K, A, lda, B, ldb, C, ldc, kchunk, part_stride, cond, s);
}

cudaError_t launch_upper_product(int l, int64_t K, const double* A, const double* B, int64_t ld, double* part,
                                 int64_t part_stride, int S, int64_t kchunk, const int* cond, cudaStream_t s) {
    for (int m0 = 0; m0 < l; m0 += kGemmBM) {
        const int M = (l - m0 < kGemmBM) ? l - m0 : kGemmBM;
        const int N = l - m0;
        const int TN = (N + 15) / 16;
        dim3 grid(1u, (unsigned)S);
        cudaError_t e = dispatch_dgemm<true>(TN, grid, M, N, K, A + m0, ld, B + m0, ld, part + (int64_t)m0 * ld + m0,
                                             ld, kchunk, part_stride, cond, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int dgemm_skinny_occupancy(int N) {
    const int TN = (N + 15) / 16;
    int occ = 1;
    cudaError_t e = cudaSuccess;
#define PBQ_OCC(T) case T: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dgemm_skinny<T, false>, 256, 0); break;
    switch (TN) {
        PBQ_OCC(1) PBQ_OCC(2) PBQ_OCC(3) PBQ_OCC(4) PBQ_OCC(5) PBQ_OCC(6) PBQ_OCC(7)
        PBQ_OCC(8) PBQ_OCC(9) PBQ_OCC(10) PBQ_OCC(11) PBQ_OCC(12) PBQ_OCC(13) PBQ_OCC(14)
        default: break;
    }
#undef PBQ_OCC
    if (e != cudaSuccess || occ < 1) occ = 1;
    return occ;
}

// ---------------------------------------------------------------------------
// Deterministic split-K reduction.
// ---------------------------------------------------------------------------
__global__ void k_reduce_partials(int64_t M, int N, int S, const double* __restrict__ part, int64_t ps,
                                  int64_t ldp, double* __restrict__ C, int64_t ldc, const int* __restrict__ cond,
                                  int upper) {
    if (cond && *cond == 0) return;
    const int64_t total = M * (int64_t)N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N;
        const int c = (int)(e - i * N);
        if (upper && c < i) continue;   // only the upper triangle was computed
        const double* p = part + i * ldp + c;
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc += p[(int64_t)s * ps];
        C[i * ldc + c] = acc;
    }
}

cudaError_t launch_reduce_partials(int64_t M, int N, int S, const double* part, int64_t ps, int64_t ldp,
                                   double* C, int64_t ldc, const int* cond, cudaStream_t s, bool upper) {
    const int64_t total = M * (int64_t)N;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_reduce_partials<<<(unsigned)blocks, 256, 0, s>>>(M, N, S, part, ps, ldp, C, ldc, cond, upper ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cholesky of the l x l Gram in shared memory (packed upper triangle).
// ctl (ints): ctl[p] = 1 if pass p (1-based) used the shift; ctl[8 + j] = 1 if
// pass pair j (passes 2j-1, 2j) must run.  Pair 1 always runs; pair j+1 runs
// iff a pass of pair j was shifted.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_cholesky(int l, int64_t rows, const double* __restrict__ G, double* __restrict__ Rp,
           uint32_t* __restrict__ status, int* __restrict__ ctl, int pass) {
    extern __shared__ double sm[];
    dev_cholesky(l, rows, G, Rp, status, ctl, pass, sm);
}

cudaError_t launch_cholesky(int l, int64_t rows, const double* G, double* Rp, uint32_t* status, int* ctl, int pass,
                            cudaStream_t s) {
    const size_t smem = (size_t)(packed_tri(l) + 2 * (int64_t)l) * sizeof(double);
    cudaError_t e = func_smem_attr((const void*)k_cholesky, smem);
    if (e != cudaSuccess) return e;
    k_cholesky<<<1, 1024, smem, s>>>(l, rows, G, Rp, status, ctl, pass);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Y = X R^{-1}: one warp per row, forward substitution y_t = x_t / r_tt then
// x_c -= y_t r_tc (c > t); lane owns columns lane + 32u.  R (packed) and
// 1/diag(R) sit in shared memory.
// ---------------------------------------------------------------------------
template <int U, typename T>
__global__ void __launch_bounds__(256)
k_trsm_rows(int64_t rows, int l, const double* __restrict__ Rp, const double* __restrict__ X, int64_t ldx,
            double* __restrict__ Y, int64_t ldy, const int* __restrict__ cond) {
    if (cond && *cond == 0) return;
    extern __shared__ __align__(16) unsigned char sraw[];
    T* sR = (T*)sraw;
    const int64_t P = (int64_t)l * (l + 1) / 2;
    for (int64_t e = threadIdx.x; e < P + l; e += blockDim.x) sR[e] = (T)Rp[e];
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    dev_trsm_rows<U, T>(l, sR, X, ldx, Y, ldy, (int64_t)blockIdx.x * 8 + warp, rows, (int64_t)gridDim.x * 8);
}

template <typename T>
static cudaError_t trsm_launch_t(int64_t rows, int l, const double* Rp, const double* X, int64_t ldx, double* Y,
                                 int64_t ldy, const int* cond, cudaStream_t s) {
    const size_t smem = (size_t)(packed_tri(l) + l) * sizeof(T);
    const int64_t per_sm = 227 * 1024 / (int64_t)(smem + 1024) > 0 ? 227 * 1024 / (int64_t)(smem + 1024) : 1;
    int64_t blocks = (rows + 7) / 8;
    if (blocks > 152 * per_sm) blocks = 152 * per_sm;
    if (blocks < 1) blocks = 1;
    const int U = (l + 31) / 32;
    cudaError_t e = cudaSuccess;
#define PBQ_TR(UU) case UU: \
        e = func_smem_attr((const void*)k_trsm_rows<UU, T>, smem); \
        if (e != cudaSuccess) return e; \
        k_trsm_rows<UU, T><<<(unsigned)blocks, 256, smem, s>>>(rows, l, Rp, X, ldx, Y, ldy, cond); break;
    switch (U) {
        PBQ_TR(1) PBQ_TR(2) PBQ_TR(3) PBQ_TR(4) PBQ_TR(5) PBQ_TR(6) PBQ_TR(7)
        default: return cudaErrorInvalidValue;
    }
#undef PBQ_TR
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trsm_rows(int64_t rows, int l, const double* Rp, const double* X, int64_t ldx, double* Y,
                             int64_t ldy, const int* cond, cudaStream_t s, bool f32) {
    return f32 ? trsm_launch_t<float>(rows, l, Rp, X, ldx, Y, ldy, cond, s)
               : trsm_launch_t<double>(rows, l, Rp, X, ldx, Y, ldy, cond, s);
}

// ---------------------------------------------------------------------------
// Householder QR of W = R^T (Eq. 7), one CTA.  The kernel stores W transposed
// (Wt = R, so a column of W is a contiguous row of Wt); reflector j (entries
// i >= j) is row j of V.  Rtil = upper(W) with signs fixed to diag >= 0,
// L = Rtil^T, Ptil = H_0 ... H_{l-1} [I] with the matching column signs.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_small_qr(int l, const double* __restrict__ R, double* __restrict__ L, double* __restrict__ Ptil,
           double* __restrict__ work, int use_smem) {
    extern __shared__ double qsm[];
    dev_small_qr(l, R, L, Ptil, work, use_smem ? qsm : nullptr);
}

cudaError_t launch_small_qr(int l, const double* R, double* L, double* Ptil, double* work, cudaStream_t s) {
    const size_t smem = 2 * (size_t)l * l * sizeof(double);
    const bool fits = smem <= 220 * 1024;
    if (fits) {
        cudaError_t e = func_smem_attr((const void*)k_small_qr, smem);
        if (e != cudaSuccess) return e;
    }
    k_small_qr<<<1, 1024, fits ? smem : 0, s>>>(l, R, L, Ptil, work, fits ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_triu(int l, double* R) {
    const int64_t ll = (int64_t)l * l;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ll; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / l), j = (int)(e - (int64_t)i * l);
        if (j < i) R[e] = 0.0;
    }
}

cudaError_t launch_triu(int l, double* R, cudaStream_t s) {
    k_triu<<<64, 256, 0, s>>>(l, R);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// General C = A B^T (reconstruction), 64 x 64 tiles, 4 x 4 per thread, with
// an optional fused residual epilogue sum((Aref - A B^T)^2) per CTA.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_dgemm_nt(int64_t M, int64_t N, int K, const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
           int64_t ldb, double* __restrict__ C, int64_t ldc, const void* __restrict__ Aref, int aref_f32,
           int64_t ldref, double* __restrict__ sqpart) {
    __shared__ double As[16][64];
    __shared__ double Bs[16][64];
    __shared__ double red[8];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * 64, n0 = (int64_t)blockIdx.y * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = tid + 256 * i, r = idx >> 4, kk = idx & 15;
            const int gk = k0 + kk;
            As[kk][r] = (m0 + r < M && gk < K) ? A[(m0 + r) * lda + gk] : 0.0;
            Bs[kk][r] = (n0 + r < N && gk < K) ? B[(n0 + r) * ldb + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    double sq = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gm = m0 + ty * 4 + r;
        if (gm >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gn = n0 + tx + 16 * c;
            if (gn >= N) continue;
            if (Aref) {
                const double ref = aref_f32 ? (double)((const float*)Aref)[gm * ldref + gn]
                                            : ((const double*)Aref)[gm * ldref + gn];
                const double d = ref - acc[r][c];
                sq += d * d;
            } else {
                C[gm * ldc + gn] = acc[r][c];
            }
        }
    }
    if (Aref) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if ((tid & 31) == 0) red[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += red[w];
            sqpart[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
    }
}

cudaError_t launch_dgemm_nt(int64_t M, int64_t N, int K, const double* A, int64_t lda, const double* B, int64_t ldb,
                            double* C, int64_t ldc, const void* Aref, int aref_f32, int64_t ldref, double* sqpart,
                            int* nblocks, cudaStream_t s) {
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64));
    if (nblocks) *nblocks = (int)(grid.x * grid.y);
    k_dgemm_nt<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, Aref, aref_f32, ldref, sqpart);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic sums of squares.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_sumsq(int64_t rows, int64_t cols, const void* __restrict__ X, int x_f32, int64_t ldx,
        const double* __restrict__ Ysub, int64_t ldy, double* __restrict__ part) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
            double v = x_f32 ? (double)((const float*)X)[r * ldx + c] : ((const double*)X)[r * ldx + c];
            if (Ysub) v -= Ysub[r * ldy + c];
            s += v * v;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_sum(int n, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    // fixed assignment: thread t sums t, t+blockDim, ... in order
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[0] = t;
    }
}

cudaError_t launch_sum(int n, const double* part, double* out, cudaStream_t s) {
    k_sum<<<1, 1024, 0, s>>>(n, part, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(int64_t rows, int64_t cols, const void* X, int x_f32, int64_t ldx, const double* Ysub,
                         int64_t ldy, double* part, double* out, cudaStream_t s) {
    int64_t nb = rows < 1024 ? rows : 1024;
    if (nb < 1) nb = 1;
    k_sumsq<<<(unsigned)nb, 256, 0, s>>>(rows, cols, X, x_f32, ldx, Ysub, ldy, part);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_sum((int)nb, part, out, s);
}

// L-values |L_ii|, the 2-norm estimate |L_11| and the count of |L_ii| > tol |L_11|.
__global__ void k_lvalues(int l, const double* __restrict__ L, double tol, double* __restrict__ lv,
                          double* __restrict__ out2) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const double l11 = fabs(L[0]);
    int c = 0;
    for (int i = threadIdx.x; i < l; i += blockDim.x) {
        const double d = fabs(L[(int64_t)i * l + i]);
        lv[i] = d;
        c += (d > tol * l11) ? 1 : 0;
    }
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) { out2[0] = l11; out2[1] = (double)cnt; }
}

cudaError_t launch_lvalues(int l, const double* L, double tol, double* lv, double* out2, cudaStream_t s) {
    k_lvalues<<<1, 256, 0, s>>>(l, L, tol, lv, out2);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_add2d(int64_t rows, int64_t cols, const double* __restrict__ src, int64_t lds,
                        double* __restrict__ dst, int64_t ldd) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e - i * cols;
        dst[i * ldd + j] += src[i * lds + j];
    }
}

cudaError_t launch_add2d(int64_t rows, int64_t cols, const double* src, int64_t lds, double* dst, int64_t ldd,
                         cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    int64_t blocks = (rows * cols + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_add2d<<<(unsigned)blocks, 256, 0, s>>>(rows, cols, src, lds, dst, ldd);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t copy2d(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                   cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst, (size_t)ldd * sizeof(double), src, (size_t)lds * sizeof(double),
                             (size_t)cols * sizeof(double), (size_t)rows, cudaMemcpyDeviceToDevice, s);
}

}  // namespace pbq

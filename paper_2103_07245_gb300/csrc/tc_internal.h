// Internal interface of the tcgen05 products (kernels_tc.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbq {

// Geometry of one product C (rows x N) = Aop (rows x K) Bt^T.
struct TcGeom {
    int BN = 16;            // N rounded up to 16 (UMMA N)
    int64_t tiles = 0;      // 128-row tiles
    int KI = 0;             // 64-element k-blocks per tile
    int G = 1;              // CTAs (one per SM, stream-K)
    int smax = 1;           // partial slots per CTA
    int64_t part_floats = 0;
};
TcGeom tc_geometry(int64_t rows, int64_t K, int N, int num_sms);

// Leading dimension (elements) of the BF16 copies: K rounded up to 64.
int64_t tc_ld(int64_t K);

struct TcOperands {
    const void* Ahi = nullptr;   // rows x K BF16, ld lda (K-major)
    const void* Alo = nullptr;   // split mode only
    int64_t rows = 0, K = 0, lda = 0;
    const void* Bhi = nullptr;   // N x K BF16, ld ldb (K-major)
    const void* Blo = nullptr;
    int N = 0;
    int64_t ldb = 0;
};

// C (FP64, rows x N, ldc) = Aop Bt^T with 1 (BF16) or 3 (split BF16) products.
// after_gemm (optional) is recorded between the tensor-core kernel and the reduction.
cudaError_t launch_tc_product(int nprod, const TcOperands& op, const TcGeom& g, float* part, double* C, int64_t ldc,
                              uint32_t* status, cudaStream_t s, cudaEvent_t after_gemm = nullptr);

// A (m x n, FP32 or FP64, lda) -> hi/lo BF16 (m x n, ld ldh) and, when thi is
// given, the transposed hi/lo (n x m, ld ldt).  lo / tlo may be null.
cudaError_t launch_split_a(int64_t m, int64_t n, const void* A, int a_f32, int64_t lda, void* hi, void* lo, int64_t ldh,
                           void* thi, void* tlo, int64_t ldt, cudaStream_t s);

// Panel P (rows x N FP64, ld ldp) -> transposed BF16 hi/lo (N x rows, ld ldt); tlo may be null.
cudaError_t launch_split_panel_t(int64_t rows, int N, const double* P, int64_t ldp, void* thi, void* tlo, int64_t ldt,
                                 cudaStream_t s);

}  // namespace pbq

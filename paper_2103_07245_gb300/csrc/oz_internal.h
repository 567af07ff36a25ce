// Internal interface of the FP64-accurate tensor-core products (kernels_oz.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbq {

constexpr int kOzDigits = 7;    // balanced base-256 digits per element (56 bits)
constexpr int kOzBM = 128;      // output rows per tile (one TMEM lane per row)
constexpr int kOzBN = 48;       // output columns per tile
constexpr int kOzBK = 32;       // contraction depth of one shared-memory stage

// One operand in digit form: kOzDigits BF16 matrices of `rows` x K (K-major,
// leading dimension ld elements, digit d at S + d*slice_stride), and the
// per-row maximum biased FP64 exponent eraw[rows] (the row scale is
// 2^(eraw - 1021)).
struct OzOperand {
    const void* S = nullptr;
    int64_t rows = 0, ld = 0, slice_stride = 0;
    const int* eraw = nullptr;
};

// Work split of one product C (Mrows x N) = X Y^T over K: 128 x 48 tiles
// (with `upper`, only the tiles that touch the upper triangle), stream-K over
// (tile, 32-deep window) iterations, FP64 partials of kOzBM x kOzBN per slot.
struct OzGeom {
    int64_t tiles = 0;
    int NT = 1, KI = 1, G = 1, smax = 1, upper = 0;
    int64_t part_doubles = 0;
};
OzGeom oz_geometry(int64_t Mrows, int N, int64_t K, bool upper, int num_sms);

// Leading dimension of a digit matrix with contraction length K.
inline int64_t oz_ld(int64_t K) { return (K + 63) / 64 * 64; }

// C[i*ldc + j] = sum_k X[i][k] Y[j][k] (FP64), i < X.rows, j < Y.rows.
// cond (device, optional): nothing runs when *cond == 0.
cudaError_t launch_oz_product(const OzOperand& X, const OzOperand& Y, int64_t K, const OzGeom& g, double* part,
                              double* C, int64_t ldc, uint32_t* status, const int* cond, cudaStream_t s,
                              cudaEvent_t after_gemm = nullptr);

// Panel P (rows x N FP64, ld ldp) as the operand P^T (N rows, contraction
// over the panel rows): column exponents into eraw[N] and digits into S
// (ld ldS, digit stride slice_stride).
cudaError_t launch_oz_panel(int64_t rows, int N, const double* P, int64_t ldp, int* eraw, void* S, int64_t ldS,
                            int64_t slice_stride, const int* cond, cudaStream_t s);

// A (m x n, FP64 or FP32, lda) as both operands: A itself (rows m, row
// exponents er, digits Srow) and A^T (rows n, column exponents ec, digits
// Scol).  Either digit set may be null (its exponents are still formed).
cudaError_t launch_oz_a(int64_t m, int64_t n, const void* A, int a_f32, int64_t lda, int* er, int* ec, void* Srow,
                        int64_t ldr, int64_t srow_stride, void* Scol, int64_t ldcol, int64_t scol_stride,
                        cudaStream_t s);

}  // namespace pbq

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
TcGeom tc_geometry(int64_t rows, int64_t K, int N, int num_sms, bool tf32 = false);

// Leading dimension (elements) of the operand copies: K rounded up to one
// 128-byte row (64 BF16 or 32 FP32 elements).
int64_t tc_ld(int64_t K, bool tf32 = false);

struct TcOperands {
    const void* Ahi = nullptr;   // rows x K BF16, ld lda (K-major)
    const void* Alo = nullptr;   // split mode only
    int64_t rows = 0, K = 0, lda = 0;
    const void* Bhi = nullptr;   // N x K BF16, ld ldb (K-major)
    const void* Blo = nullptr;
    int N = 0;
    int64_t ldb = 0;
    int tf32 = 0;                // operands are TF32 held in FP32 (else BF16)
};

// C (FP64, rows x N, ldc) = Aop Bt^T with 1 (BF16) or 3 (split BF16) products.
// after_gemm (optional) is recorded between the tensor-core kernel and the reduction.
// stall != 0 is the failure-detection test: the producer issues nothing, the
// bounded waits expire after 50 ms and the status word gets the timeout bit.
cudaError_t launch_tc_product(int nprod, const TcOperands& op, const TcGeom& g, float* part, double* C, int64_t ldc,
                              uint32_t* status, cudaStream_t s, cudaEvent_t after_gemm = nullptr, int stall = 0);

// A (m x n, FP32 or FP64, lda) -> hi/lo BF16 (m x n, ld ldh) and, when thi is
// given, the transposed hi/lo (n x m, ld ldt).  lo / tlo may be null.
cudaError_t launch_split_a(int64_t m, int64_t n, const void* A, int a_f32, int64_t lda, void* hi, void* lo, int64_t ldh,
                           void* thi, void* tlo, int64_t ldt, cudaStream_t s, bool tf32 = false);

// Panel P (rows x N FP64, ld ldp) -> transposed BF16 hi/lo (N x rows, ld ldt); tlo may be null.
cudaError_t launch_split_panel_t(int64_t rows, int N, const double* P, int64_t ldp, void* thi, void* tlo, int64_t ldt,
                                 cudaStream_t s, bool tf32 = false);

// ---- grouped TF32 products of the batched path (kernels_tc_list.cu) ----------
// One unit: C[m0 .. m0+127, 0 .. N) = Aop Bt^T over the full contraction
// (KI k-blocks of 32 FP32 elements), operands given by tensor-map indices.
struct TcUnit {
    int amap_hi, amap_lo, bmap_hi, bmap_lo;
    int m0, N, npad, KI;
    double* C;
    int64_t ldc, rows;
};
constexpr int kTcListBNMax = 128;   // largest padded N of the grouped kernel
// nprod 1 (TF32) or 3 (split TF32); units should be sorted by cost (largest first).
cudaError_t launch_tc_list(int nprod, const void* maps, const TcUnit* units, int nunits, int num_sms, uint32_t* status,
                           cudaStream_t s);
// Host: encode a 2-D FP32 tensor map (rows x cols, ld elements, box {32, box_rows}, 128-byte swizzle).
bool make_map_f32(void* map128, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows);

// A strip of one matrix for the TF32 split: rows [r0, r0+32) of A (m x n) into
// hi/lo (ld ldh) and transposed hi/lo (ld ldt).
struct SplitUnit {
    const void* A;
    float *hi, *lo, *thi, *tlo;
    int64_t lda, ldh, ldt, m, n, r0;   // rows r0 .. r0 + 63
    int a_f32;
    int vec_ok;                        // 16-byte aligned pointers and leading dimensions
};
// col_tiles: 64-column tiles of the widest matrix; a_f32: element type of
// every unit's A (one launch handles one type)
cudaError_t launch_split_tf32_list(const SplitUnit* units, int nunits, int col_tiles, int a_f32, cudaStream_t s);
// A row block of one panel: Y (rows x N FP64, ld ldy) into transposed TF32 hi/lo (N x rows, ld ldt).
struct PanelUnit {
    const double* Y;
    float *thi, *tlo;
    int64_t rows, ldy, ldt;   // this unit converts panel rows [r0, r0 + rows)
    int N;
    int64_t r0;
};
cudaError_t launch_split_panel_tf32_list(const PanelUnit* units, int nunits, cudaStream_t s);

}  // namespace pbq

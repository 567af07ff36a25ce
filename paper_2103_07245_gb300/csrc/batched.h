// Work-list descriptors of the batched PbP-QLP path (many matrices per launch).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbq {

// One CTA tile of a skinny FP64 product: C[m0:m0+64, :N] (+)= op(A)[m0:m0+64, kbeg:kend] B[kbeg:kend, :N].
struct GemmUnit {
    const double* A;
    const double* B;
    double* C;
    int64_t lda, ldb, ldc;
    int64_t M, m0, kbeg, kend;
    int N;
    int transA;
    const int* cond;     // skip when *cond == 0 (null: always run)
};

// Sum S partial panels of one matrix (M x N, stride ps, ld ldp) into C (ldc).
struct ReduceUnit {
    const double* part;
    double* C;
    int64_t ps, ldp, ldc, M;
    int N, S;
    const int* cond;
};

// One matrix for the one-CTA kernels (Cholesky, small QR) and the Gaussian draw.
struct MatUnit {
    int l;
    int pass;
    int64_t rows;
    const double* G;     // Cholesky input / small-QR input R
    double* Rp;          // Cholesky output (packed + 1/diag)
    int* ctl;            // retry flags of this matrix's current orth
    uint32_t* status;    // this matrix's status word
    double* L;           // small QR outputs
    double* Pt;
    double* work;
    double* out;         // Gaussian output (rows x l, ld)
    int64_t ld;
    uint64_t seed;
    int64_t b0, b1;      // Gaussian: Box-Muller pairs [b0, b1) of this matrix's stream
};

// A block of rows of one panel for the row-wise triangular solve Y = X R^{-1}.
struct TrsmUnit {
    const double* X;
    double* Y;
    const double* Rp;
    int64_t ldx, ldy, r0, r1;
    int l;
    const int* cond;
};

cudaError_t launch_dgemm_list(int TN, bool transA, const GemmUnit* units, int nunits, cudaStream_t s);
cudaError_t launch_reduce_list(const ReduceUnit* units, int nunits, cudaStream_t s);
cudaError_t launch_cholesky_list(const MatUnit* units, int nunits, int lmax, cudaStream_t s);
cudaError_t launch_trsm_list(const TrsmUnit* units, int nunits, int lmax, cudaStream_t s, bool f32 = false);
cudaError_t launch_small_qr_list(const MatUnit* units, int nunits, int lmax, cudaStream_t s);
cudaError_t launch_gaussian_list(const MatUnit* units, int nunits, cudaStream_t s);

}  // namespace pbq

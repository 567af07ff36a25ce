// Internal launcher interface of the PbP-QLP CUDA library (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pbq {

constexpr int kMaxEll = 224;          // l handled by the one-cluster l x l kernels (factor in shared memory)
constexpr int kMaxEllBlocked = 4096;  // l limit of the blocked l x l steps (kernels_blocked.cu)
constexpr int kCholBlock = 128;       // diagonal block of the blocked Cholesky
constexpr int kGemmBM = 64;           // rows per CTA tile of the skinny FP64 GEMM
constexpr int kGemmBK = 16;           // contraction depth per shared-memory stage

// Device status bits (latched in the workspace status word).
constexpr uint32_t kStShifted = 1u;    // a shifted Cholesky retry was used
constexpr uint32_t kStBreakdown = 2u;  // Cholesky failed even with the shift
constexpr uint32_t kStNonFinite = 4u;  // NaN/Inf met
constexpr uint32_t kStTimeout = 8u;    // bounded wait gave up
constexpr uint32_t kStBadInput = 16u;  // a sparse A's CSR structure failed the device check

// Process-wide launch counter (incremented by every launcher below).
void count_launches(int64_t n);
int64_t launch_count();
// cudaFuncAttributeMaxDynamicSharedMemorySize for func on the current device,
// set through the driver only when a larger size than before is asked for
// (the attribute call costs host time on every launch otherwise).
cudaError_t func_smem_attr(const void* func, size_t bytes);

// Report a failing CUDA call on stderr when PBPQLP_DEBUG=1; returns e.
cudaError_t debug_report(cudaError_t e, const char* what, const char* file, int line);
#define PBQ_DBG(expr) ::pbq::debug_report((expr), #expr, __FILE__, __LINE__)

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline int64_t packed_tri(int l) { return (int64_t)l * (l + 1) / 2; }

// ---- Sparse A (kernels_sparse.cu) ---------------------------------------
// A CSR matrix on the device: ptr[rows + 1], idx[nnz], val[nnz].
struct CsrT {
    const int64_t* ptr = nullptr;
    const int32_t* idx = nullptr;
    const double* val = nullptr;
};
// Scratch bytes of launch_csr_transpose for an A with n columns and nnz entries.
size_t csr_transpose_bytes(int64_t n, int64_t nnz);
// Checks A's CSR structure (kStBadInput in *status on a violation) and builds
// A^T as a CSR in `scratch` (*out points into it), each row of A^T in
// ascending position of A's CSR.  After a violation no kernel reads through
// the structure.
cudaError_t launch_csr_transpose(int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
                                 const double* values, void* scratch, CsrT* out, uint32_t* status, int num_sms,
                                 cudaStream_t s);
// C (rows x l, ldc) = S X for a CSR S with `rows` rows and X row-major (ldx);
// zeros after a structure violation (kStBadInput in *status).
cudaError_t launch_csr_spmm(int64_t rows, const int64_t* ptr, const int32_t* idx, const double* val, const double* X,
                            int64_t ldx, int l, double* C, int64_t ldc, const uint32_t* status, int num_sms,
                            cudaStream_t s);

// ---- FP64 kernels (kernels_fp64.cu) -------------------------------------
// Phi[i*ld + j] = sample (i*l + j) of the Philox4x32-10 / Box-Muller stream.
cudaError_t launch_gaussian(uint64_t seed, int64_t rows, int l, double* out, int64_t ld, cudaStream_t s);

// C (M x N) = op(A) B, op(A) = A (M x K, lda) or A^T (A stored K x M).  B is K x N (ldb).
// With S > 1 the contraction is split in S chunks of kchunk rows; chunk s
// writes C + s*part_stride (a partial sum) and reduce_partials adds them in
// chunk order.  N <= kMaxEll.  cond (device, optional): skip when *cond == 0.
cudaError_t launch_dgemm_skinny(bool transA, int64_t M, int N, int64_t K, const double* A, int64_t lda,
                                const double* B, int64_t ldb, double* C, int64_t ldc, int S, int64_t kchunk,
                                int64_t part_stride, const int* cond, cudaStream_t s);
// Max resident CTAs per SM of the skinny GEMM for this N.
int dgemm_skinny_occupancy(int N);

// C[i*ldc + c] = sum_{s<S} part[s*part_stride + i*ldp + c]  (fixed order; deterministic);
// with upper, only c >= i.
cudaError_t launch_reduce_partials(int64_t M, int N, int S, const double* part, int64_t part_stride,
                                   int64_t ldp, double* C, int64_t ldc, const int* cond, cudaStream_t s,
                                   bool upper = false);

// Upper triangle of A^T B (A, B: K x l, ld ld) into the split-K partial
// buffer: one launch per 64-row tile, columns from the tile's first row
// (the Gram of CholeskyQR and R = Q^T D need only that triangle).
cudaError_t launch_upper_product(int l, int64_t K, const double* A, const double* B, int64_t ld, double* part,
                                 int64_t part_stride, int S, int64_t kchunk, const int* cond, cudaStream_t s);

// One-CTA Cholesky G = R^T R of the l x l Gram (ld l) of a rows x l panel.
// Writes R packed (upper, row-major packed) plus 1/diag (l values after the
// packed triangle).  On a pivot below tau*G0_jj retries once on G + shift*I
// (shifted CholeskyQR, Fukaya et al. 2020).  ctl layout: see kernels_fp64.cu.
cudaError_t launch_cholesky(int l, int64_t rows, const double* G, double* Rpacked, uint32_t* status,
                            int* ctl, int pass, cudaStream_t s);

// The same Cholesky by a cluster of 8 CTAs (rows dealt cyclically, the pivot
// row shared through distributed shared memory), for l > 128.
bool cholesky_cluster_fits(int l);
cudaError_t launch_cholesky_cluster(int l, int64_t rows, const double* G, double* Rpacked, uint32_t* status, int* ctl,
                                    int pass, cudaStream_t s);

// Cholesky G = R^T R with T = R^{-T} (l x l row-major, lower triangular) by
// an 8-CTA cluster (kernels_cholinv.cu).  Rpacked, ctl, status and the
// shifted retry as launch_cholesky.  T may be null.
bool chol_inv_fits(int l);
cudaError_t launch_chol_inv(int l, int64_t rows, const double* G, double* Rpacked, double* T, uint32_t* status,
                            int* ctl, int pass, cudaStream_t s);

// One b x b diagonal block (b <= kMaxEll) of the blocked Cholesky: the cluster
// kernel on S (leading dimension ld), pivot thresholds from gdiag (stride
// ld + 1), R_tt (upper) into R and T_tt = R_tt^{-T} (lower) into T (both ld);
// runs only if *bstate == want, sets *bstate = want + 1 on a failed pivot (4
// on a non-finite one, with the status bit).
cudaError_t launch_chol_inv_block(int b, const double* S, int64_t ld, const double* gdiag, double* R, double* T,
                                  uint32_t* status, int* bstate, int want, cudaStream_t s);

// ---- Blocked l x l steps (kernels_blocked.cu), any l <= kMaxEllBlocked ---
// C (M x N, ldc) = alpha op(A) op(B) + beta C in FP64 (op(A) = A, M x K, or
// A^T with A stored K x M; op(B) = B, K x N, or B^T with B stored N x K);
// with upper, only C[i][j] with j >= i is written.  Each output sums its
// contraction in index order.  Runs only if state is null or *state == want.
cudaError_t launch_dgemm_gen(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                             int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, bool upper,
                             const int* state, int want, cudaStream_t s);
// Cholesky G = R^T R of the l x l Gram (ld l) of a rows x l panel, with
// T = R^{-T} (lower, ld l), right-looking over kCholBlock diagonal blocks,
// one shifted retry of the whole factorization, identity fallback on
// breakdown; ctl / status / pass as launch_chol_inv.  work: the bytes below.
size_t chol_inv_blocked_work_bytes(int l);
cudaError_t launch_chol_inv_blocked(int l, int64_t rows, const double* G, double* T, void* work, uint32_t* status,
                                    int* ctl, int pass, cudaStream_t s);
// Householder QR of R^T (R upper, ld l): L = Rtil^T and Ptil (ld l) with
// diag(Rtil) >= 0, blocked in 32-column panels.  work: the bytes below.
bool qr_blocked_fits(int l);
size_t qr_blocked_work_bytes(int l);
cudaError_t launch_qr_blocked(int l, const double* R, double* L, double* Ptil, void* work, cudaStream_t s);

// Y = X R^{-1} row by row (R from launch_cholesky), rows x l panels; f32
// solves in FP32 (the mixed modes) instead of FP64.
cudaError_t launch_trsm_rows(int64_t rows, int l, const double* Rpacked, const double* X, int64_t ldx,
                             double* Y, int64_t ldy, const int* cond, cudaStream_t s, bool f32 = false);

// One-CTA Householder QR of R^T (R upper, l x l dense ld l, only upper part read):
// R^T = Ptil Rtil with diag(Rtil) >= 0.  Writes L = Rtil^T (l x l, ld l) and
// Ptil (l x l row-major, ld l).  work: 2*l*l doubles (unused when they fit in
// shared memory, l <= 121).
cudaError_t launch_small_qr(int l, const double* R, double* L, double* Ptil, double* work, cudaStream_t s);

// The same QR by an 8-CTA cluster (columns dealt cyclically), for l > 128.
bool small_qr_cluster_fits(int l);
cudaError_t launch_small_qr_cluster(int l, const double* R, double* L, double* Ptil, cudaStream_t s);

// Zero the strictly-lower part of an l x l matrix (ld l) in place.
cudaError_t launch_triu(int l, double* R, cudaStream_t s);

// C (M x N) = A (M x K) B^T with B stored N x K; general N (reconstruction).
// If Aref != nullptr, C is not written; instead per-CTA partial sums of
// (Aref - A B^T)^2 go to sqpart[blockId] (FP64).  Returns the CTA count via *nblocks.
cudaError_t launch_dgemm_nt(int64_t M, int64_t N, int K, const double* A, int64_t lda, const double* B,
                            int64_t ldb, double* C, int64_t ldc, const void* Aref, int aref_f32,
                            int64_t ldref, double* sqpart, int* nblocks, cudaStream_t s);

// Sum of squares of a rows x cols matrix X (FP64 or FP32 elements), minus
// Ysub (FP64) when given: per-CTA partials to part[0..nb) (nb <= 1024) then a
// one-CTA sum to out[0].  Fixed reduction order (deterministic).
cudaError_t launch_sumsq(int64_t rows, int64_t cols, const void* X, int x_f32, int64_t ldx, const double* Ysub,
                         int64_t ldy, double* part, double* out, cudaStream_t s);
// out[0] = sum of part[0..n) in index order (one CTA).
cudaError_t launch_sum(int n, const double* part, double* out, cudaStream_t s);

// L-values |L_ii| into lv (l), out2[0] = |L_11|, out2[1] = #{i : |L_ii| > tol |L_11|} (as a double).
cudaError_t launch_lvalues(int l, const double* L, double tol, double* lv, double* out2, cudaStream_t s);

// dst += src for a rows x cols FP64 block (each element once; deterministic).
cudaError_t launch_add2d(int64_t rows, int64_t cols, const double* src, int64_t lds, double* dst, int64_t ldd,
                         cudaStream_t s);

// Copy a rows x cols FP64 block between leading dimensions.
cudaError_t copy2d(const double* src, int64_t lds, double* dst, int64_t ldd, int64_t rows, int64_t cols,
                   cudaStream_t s);

}  // namespace pbq

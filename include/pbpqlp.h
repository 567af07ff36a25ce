/*
 * pbpqlp.h — C ABI of the GB300 (sm_103a) Projection-based Partial QLP library.
 *
 * The method (Kaloorazi & Chen, "Projection-based QLP Algorithm for
 * Efficiently Computing Low-Rank Approximation of Matrices", Section III,
 * Algorithm 3) factors a dense A (m x n) as A ~= Qa L Qb^T with Qa (m x l) and
 * Qb (n x l) orthonormal and L (l x l) lower triangular, l = k + p (the
 * paper's sampling size d), using q power iterations:
 *     Phi = randn(m, l);  C = A^T Phi;  Pbar = orth(C);
 *     repeat q times: C = A Pbar, Pbar = orth(C); C = A^T Pbar, Pbar = orth(C);
 *     D = A Pbar;  [Qa, R] = qr(D);  [Ptil, Rtil] = qr(R^T);
 *     Qb = Pbar Ptil;  L = Rtil^T.
 * Every orth/qr is an unpivoted thin QR with diag(R) >= 0, so diag(L) >= 0.
 *
 * Conventions shared by every entry point:
 *   - Matrices are row-major.  A has leading dimension lda >= n (elements).
 *     Qa, Qb, L and the Gaussian Phi are contiguous (leading dimension l).
 *   - Pointers named A, Qa, L, Qb, Ahat, omega, workspace are DEVICE pointers
 *     the caller allocates and owns; pointers named *_host are host memory.
 *   - Work is enqueued on the plan's CUDA stream and returns before it runs.
 *     Argument errors are returned at once; numerical failures found on the
 *     device (breakdown, non-finite data) are latched in a status word inside
 *     the workspace and reported by pbpqlp_sync_status() or by the synchronous
 *     calls (pbpqlp_error).
 *   - A plan is used by one host thread / one stream at a time.  Nothing
 *     throws across the ABI.  No entry point allocates device memory except
 *     where stated.
 */
#ifndef PBPQLP_H
#define PBPQLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum {
    PBPQLP_OK = 0,
    PBPQLP_EINVAL = 1,       /* bad argument (sizes, null pointers, modes) */
    PBPQLP_ENOMEM = 2,       /* host allocation failed */
    PBPQLP_ECUDA = 3,        /* a CUDA runtime call failed */
    PBPQLP_ENONFINITE = 4,   /* NaN/Inf met in A or in an intermediate panel */
    PBPQLP_EBREAKDOWN = 5,   /* orthonormalisation failed even after the shifted retries */
    PBPQLP_ETIMEOUT = 6,     /* a bounded device wait gave up */
    PBPQLP_EUNSUPPORTED = 7, /* mode / size combination the library does not support */
    PBPQLP_EWORKSPACE = 8    /* workspace missing or smaller than pbpqlp_workspace_bytes() */
};

/* Arithmetic modes of the three products with A (the sketch, the power
 * iterations and the projection).  Gram accumulation, Cholesky and the final
 * l x l QR are FP64-accurate in every mode: the Grams of CholeskyQR and
 * R = Q^T D run on the tensor cores in the exact-digit form described under
 * PBPQLP_MODE_FP64_EMU (environment PBPQLP_NO_OZ_GRAM=1 at plan creation
 * selects FP64 FMA kernels instead), the Cholesky and QR in FP64 FMA. */
enum {
    PBPQLP_MODE_FP64 = 0,    /* A FP64, FP64 products */
    PBPQLP_MODE_BF16 = 1,    /* A and panels rounded to BF16, FP32 accumulate */
    PBPQLP_MODE_BF16X3 = 2,  /* BF16 hi/lo split, three products hi*hi + lo*hi + hi*lo */
    PBPQLP_MODE_TF32 = 3,    /* TF32 operands, FP32 accumulate */
    PBPQLP_MODE_TF32X3 = 4,  /* TF32 hi/lo split, three products */
    /* FP64-accurate products on the BF16 tensor cores (not in the paper; the
     * error-free splitting of Ozaki, Ogita, Oishi & Rump 2012): every row of
     * an operand is scaled by a power of two and written as 8 balanced
     * base-128 digits (56 bits), the 36 digit products of weight >= 2^-56
     * are summed exactly in FP32 over 32-deep windows and combined in int64.
     * Digit rounding and the dropped digit products add at most
     * 2^-51 max|x_i.| max|y_j.| per term (all digits extreme); on data of
     * even magnitude the error is that of an FP64 dot product.  Rows holding
     * Inf or NaN give NaN products.  A is turned into digits once per call
     * (32 bytes per element of workspace, both orientations). */
    PBPQLP_MODE_FP64_EMU = 5
};

/* Flag OR-ed into the mode of pbpqlp_plan: stream A through the mixed and
 * emulated products instead of holding whole converted copies of it (the
 * pass-efficient setting of Section III-C, where A is stored externally and
 * read once per pass).  Every pass splits (BF16 / TF32 modes) or digitises
 * (MODE_FP64_EMU) one block of rows of A at a time into a staging area of
 * about 512 MB (PBPQLP_STREAM_ROWS in the environment at plan creation sets
 * the rows per block), so A may sit in pinned host memory larger than the
 * device's memory.  C = A Y is written block by block; C = A^T Y adds the
 * blocks' FP64 partial sums in block order, so results are deterministic but
 * not bitwise those of the unstreamed plan.  MODE_FP64 reads A in place in
 * every pass already and ignores the flag. */
#define PBPQLP_STREAM_A 256

/* Element type of A. */
enum { PBPQLP_F64 = 0, PBPQLP_F32 = 1 };

/* Methods of pbpqlp_error. */
enum {
    PBPQLP_ERR_IDENTITY = 0, /* sqrt(||A||_F^2 - ||L_r||_F^2) / ||A||_F (exact in exact arithmetic) */
    PBPQLP_ERR_RESIDUAL = 1, /* ||A - Qa_r L_r Qb_r^T||_F / ||A||_F, formed explicitly */
    PBPQLP_ERR_PROBES = 2    /* randomized estimate from Gaussian probes */
};

typedef struct pbpqlp_plan_s* pbpqlp_plan_t;

/* Library version as major*10000 + minor*100 + patch. */
int pbpqlp_version(void);

/* Human-readable text of a status code (static string; never NULL). */
const char* pbpqlp_strerror(int status);

/*
 * Create a plan for one factorization shape (Algorithm 3 inputs).
 *   m, n   : rows / columns of A (m, n >= 1).
 *   k, p   : target rank and oversampling; l = k + p must satisfy
 *            1 <= k <= l <= min(m, n) and l <= 4096.  Up to l = 224 the
 *            l x l steps run in one thread-block cluster; beyond, they are
 *            blocked (the Cholesky over 128-row diagonal blocks, the QR of
 *            R^T in 32-column Householder panels), the products with A run
 *            in column chunks of at most 224, and the plan needs the
 *            digit-form Grams (PBPQLP_EUNSUPPORTED with PBPQLP_NO_OZ_GRAM=1
 *            or PBPQLP_NO_CLUSTER=1).
 *   q      : power iterations, q >= 0 (q = 0 is the basic form, Eqs. 3-8).
 *   seed   : seed of the Philox4x32-10 Gaussian stream of Phi.
 *   mode   : PBPQLP_MODE_*.
 *   stream : cudaStream_t to enqueue on (NULL = legacy default stream).
 * Host memory only; *out is owned by the caller and freed by
 * pbpqlp_plan_destroy.  Returns PBPQLP_EINVAL on bad sizes.
 */
int pbpqlp_plan(pbpqlp_plan_t* out, int64_t m, int64_t n, int k, int p, int q,
                uint64_t seed, int mode, void* stream);

/* Release a plan (NULL is accepted). */
int pbpqlp_plan_destroy(pbpqlp_plan_t plan);

/* Bytes of device workspace pbpqlp_factor / _reconstruct / _error need
 * (256-byte aligned base required).  Returns 0 for a NULL plan. */
size_t pbpqlp_workspace_bytes(pbpqlp_plan_t plan);

/*
 * Write the Gaussian test matrix Phi (m x l, FP64, row-major) the plan's seed
 * defines into the device buffer omega (Section III-A, randn(n1, d)).
 * Element (i, j) is sample t = i*l + j of the stream: Philox4x32-10 block
 * t/2 with counter {t/2 lo, t/2 hi, 0, 0} and key {seed lo, seed hi}; its
 * words give u1 = (a53 + 1) 2^-53 and u2 = b53 2^-53, and sample t is
 * sqrt(-2 ln u1) * (t even ? cos : sin)(2 pi u2)  (Box-Muller).
 */
int pbpqlp_generate_omega(pbpqlp_plan_t plan, double* omega);

/*
 * Algorithm 3: factor A ~= Qa L Qb^T.
 *   A         : device memory, or pinned host memory the device can address
 *               (out-of-core: every pass then streams A over the host link;
 *               the FP64 passes need ~8 bytes per 2 l flops, far below
 *               NVLink-C2C bandwidth), m x n, row-major, leading dimension lda >= n,
 *               element type a_dtype (PBPQLP_F64 in MODE_FP64; PBPQLP_F32 or
 *               PBPQLP_F64 in the mixed modes, which split A into BF16 hi/lo
 *               copies in the workspace once per call, and in MODE_FP64_EMU,
 *               which writes the digits of A and A^T there).
 *   workspace : device, >= pbpqlp_workspace_bytes(plan) bytes, 256-aligned;
 *               ws_bytes is its size.  Contents are scratch between calls.
 *   omega     : optional device m x l FP64 test matrix; NULL draws Phi from
 *               the plan's seed (as pbpqlp_generate_omega).
 *   Qa        : device, m x l FP64 output (orthonormal columns).
 *   L         : device, l x l FP64 output, lower triangular, diag >= 0.
 *   Qb        : device, n x l FP64 output (orthonormal columns).
 * Asynchronous; device-side failures are read with pbpqlp_sync_status.
 */
int pbpqlp_factor(pbpqlp_plan_t plan, const void* A, int64_t lda, int a_dtype,
                  void* workspace, size_t ws_bytes, const double* omega,
                  double* Qa, double* L, double* Qb);

/*
 * Algorithm 3 continued from a basis (Section III-B: the power iterations
 * only need the current orthonormal basis Pbar).  Because every orth is a
 * thin QR, the first l' columns of orth(C) are orth of the first l' columns
 * of C, and A Pbar[:, :l'] is the first l' columns of A Pbar; so a run started
 * from the first l columns of the basis of a wider run with the same Phi
 * reproduces, up to rounding, the run with Phi's first l columns, and the
 * q-th basis of a run is the basis a q-iteration run projects on.  This lets
 * a caller keep one trajectory and branch off it (the learned (q, p)
 * proposer continues its q = 0 sketch instead of starting over).
 *   pbar0     : optional device n x l basis with orthonormal columns, leading
 *               dimension ld_pbar0 >= l (e.g. the first l columns of a wider
 *               basis).  It replaces Phi, Eq. 3 and the first orth (Eq. 4);
 *               the plan's q power iterations follow.  NULL: start from the
 *               plan's Phi exactly as pbpqlp_factor.
 *   pbar_out  : optional device n x l (contiguous) output: the basis after the
 *               power iterations, the one Eq. 5 projects on.
 *   Qa, L, Qb : as pbpqlp_factor; all three NULL stops after the power
 *               iterations (pbar_out then required): no projection pass.
 * Workspace, asynchrony and status as pbpqlp_factor.
 */
int pbpqlp_factor_from(pbpqlp_plan_t plan, const void* A, int64_t lda, int a_dtype,
                       void* workspace, size_t ws_bytes, const double* pbar0, int64_t ld_pbar0,
                       double* pbar_out, double* Qa, double* L, double* Qb);

/*
 * One product of Algorithm 3 on its own (Eq. 3 / Eq. 5): C = A Y (trans = 0;
 * Y is n x ncols, C is m x ncols) or C = A^T Y (trans = 1; Y is m x ncols,
 * C is n x ncols), in the plan's arithmetic mode (FP64 DFMA, or the
 * tcgen05 BF16 / split-BF16 products with FP32 accumulation).
 *   Y, C : device FP64, row-major, leading dimensions ldy, ldc >= ncols.
 *   1 <= ncols <= l.  A and a_dtype as in pbpqlp_factor.
 * Uses the workspace (same size rule as pbpqlp_factor); asynchronous.
 */
int pbpqlp_sketch(pbpqlp_plan_t plan, const void* A, int64_t lda, int a_dtype, int trans,
                  const double* Y, int64_t ldy, int ncols, double* C, int64_t ldc,
                  void* workspace, size_t ws_bytes);

/*
 * Rank-r reconstruction Ahat = Qa[:, :r] L[:r, :r] Qb[:, :r]^T (Eq. 8 and its
 * truncation), FP64, m x n row-major with leading dimension ldh >= n.
 * 1 <= r <= l.  Uses the workspace (same size rule as pbpqlp_factor).
 */
int pbpqlp_reconstruct(pbpqlp_plan_t plan, const double* Qa, const double* L, const double* Qb,
                       int r, double* Ahat, int64_t ldh, void* workspace, size_t ws_bytes);

/*
 * Relative Frobenius error of the rank-r truncation, returned in *rel_err
 * (host).  Synchronous (waits on the plan's stream).  method is
 * PBPQLP_ERR_IDENTITY, _RESIDUAL or _PROBES (nprobes Gaussian probes drawn
 * from probe_seed).  A and a_dtype as in pbpqlp_factor.  Also returns any
 * latched device status of the preceding factorization.
 */
int pbpqlp_error(pbpqlp_plan_t plan, const void* A, int64_t lda, int a_dtype,
                 const double* Qa, const double* L, const double* Qb, int r,
                 int method, int nprobes, uint64_t probe_seed,
                 void* workspace, size_t ws_bytes, double* rel_err);

/*
 * Rank-revealing outputs of a factorization (Section IV-C: the diagonal of L
 * approximates sigma_1..sigma_l; Section V-D: |L_11| estimates ||A||_2, and
 * Theorem 7 bounds sigma_min(L_11) <= sigma_k).
 *   L        : device, l x l factor from pbpqlp_factor.
 *   lvalues  : device output, l doubles: |L_ii|.
 *   *norm2_est (host): |L_11| (never above ||A||_2: |L_11| <= sigma_1(L) <= sigma_1(A)).
 *   *rank_est  (host): number of i with |L_ii| > tol |L_11| (numerical rank at
 *               relative tolerance tol >= 0).
 * Synchronous; uses the workspace for two scalars.
 */
int pbpqlp_rank_revealing(pbpqlp_plan_t plan, const double* L, double tol, double* lvalues,
                          void* workspace, size_t ws_bytes, double* norm2_est, int* rank_est);

/*
 * Sparse A (Section III-C: with z nonzeros the products with A and A^T cost
 * O(z d) instead of O(m n d)).  Same factorization, outputs and status as
 * pbpqlp_factor, for A (plan's m x n) in CSR form on the device (or in
 * pinned host memory mapped at the same address):
 *   rowptr[m + 1] (int64): rowptr[0] = 0, nondecreasing, rowptr[m] = nnz;
 *   colind[nnz] (int32): 0 <= colind < n, any order within a row, repeated
 *   (row, column) pairs add;  values[nnz] (FP64).
 * A^T is built as a second CSR in the workspace on every call (its rows keep
 * the order of A's entries), so both products are deterministic.  The
 * structure is checked on the device before anything indexes through it: a
 * violation makes pbpqlp_sync_status return PBPQLP_EINVAL (status bit 16)
 * and the outputs hold no meaningful values.  The plan's mode must be
 * PBPQLP_MODE_FP64 (PBPQLP_EUNSUPPORTED otherwise); workspace >=
 * pbpqlp_csr_workspace_bytes(plan, nnz) bytes, 256-aligned (the plan's
 * workspace plus 24 bytes per nonzero and 12 per column).
 */
size_t pbpqlp_csr_workspace_bytes(pbpqlp_plan_t plan, int64_t nnz);
int pbpqlp_factor_csr(pbpqlp_plan_t plan, const int64_t* rowptr, const int32_t* colind, const double* values,
                      int64_t nnz, void* workspace, size_t ws_bytes, const double* omega, double* Qa,
                      double* L, double* Qb);

/*
 * Wait for the plan's stream and return the latched device status of the
 * last pbpqlp_factor (or pbpqlp_factor_csr) on this plan's workspace
 * (PBPQLP_OK, _EINVAL for a bad CSR structure, _ENONFINITE, _EBREAKDOWN or
 * _ETIMEOUT), then clear it.  *flags_host (optional) gets the raw status
 * bits: 1 = a shifted Cholesky retry was used, 2 = breakdown after all
 * retries, 4 = non-finite value, 8 = timeout, 16 = bad CSR structure.
 */
int pbpqlp_sync_status(pbpqlp_plan_t plan, uint32_t* flags_host);

/*
 * Batched factorization: `count` independent matrices of uneven shapes, each
 * factored by Algorithm 3 exactly as pbpqlp_factor would (same kernels, same
 * results), advanced together one step per launch over work lists; the whole
 * launch sequence is captured into one CUDA graph on the first call and
 * replayed while the buffers stay the same.
 *   m, n, k (host arrays of count): shapes and target ranks; p and q are
 *   shared; l_i = k_i + p must satisfy 1 <= k_i <= l_i <= min(m_i, n_i), l_i <= 224.
 *   Matrix i draws Phi_i from the Philox stream keyed by seed + i.
 *   mode: PBPQLP_MODE_FP64, or PBPQLP_MODE_TF32 / PBPQLP_MODE_TF32X3 (the
 *   products with A_i on the tensor cores, kind::tf32 with FP32
 *   accumulation, split hi/lo in the X3 form; Cholesky and the small QR stay
 *   FP64; l_i <= 128 in these modes).  a_dtype PBPQLP_F32 or PBPQLP_F64 in
 *   the TF32 modes, PBPQLP_F64 in FP64 mode.  In every mode the Grams of
 *   the orth (Eq. 4) and R = Q^T D (Eq. 6) are exact-digit products on the
 *   BF16 tensor cores, FP64-accurate as in pbpqlp_factor (environment
 *   PBPQLP_NO_OZ_GRAM=1 at plan creation: FP64 FMA Grams instead).
 *   A, lda, Qa, L, Qb (host arrays of count): device pointers / leading
 *   dimensions per matrix, layouts as in pbpqlp_factor.
 *   workspace: device, >= pbpqlp_batch_workspace_bytes(batch), 256-aligned;
 *   it also holds the work lists, which every call rewrites.
 * pbpqlp_batch_sync_status waits and returns the worst device status of the
 * batch; flags_host (optional, count entries) gets each matrix's status bits.
 */
typedef struct pbpqlp_batch_s* pbpqlp_batch_t;
int pbpqlp_plan_batched(pbpqlp_batch_t* out, int count, const int64_t* m, const int64_t* n,
                        const int* k, int p, int q, uint64_t seed, int mode, void* stream);
int pbpqlp_batch_destroy(pbpqlp_batch_t batch);
size_t pbpqlp_batch_workspace_bytes(pbpqlp_batch_t batch);
int pbpqlp_factor_batched(pbpqlp_batch_t batch, const void* const* A, const int64_t* lda, int a_dtype,
                          void* workspace, size_t ws_bytes, double* const* Qa, double* const* L,
                          double* const* Qb);
int pbpqlp_batch_sync_status(pbpqlp_batch_t batch, uint32_t* flags_host);

/*
 * Autotuner of the batched launch geometry: times the batched factorization
 * on the caller's data for each candidate (Gram row chunk 256/512/1024/2048
 * for the FP64 FMA Grams only, triangular-solve rows per unit 64/128/256, and
 * in the TF32 modes the order of the grouped product units) and keeps the
 * fastest in the plan.  Runs the
 * factorization 2 x (number of candidates) times; outputs hold the last run.
 * table_path (optional): appends one JSON line with the batch signature and
 * the chosen values.  *best_ms (optional) gets the best time per call.
 */
int pbpqlp_batch_autotune(pbpqlp_batch_t batch, const void* const* A, const int64_t* lda, int a_dtype,
                          void* workspace, size_t ws_bytes, double* const* Qa, double* const* L,
                          double* const* Qb, const char* table_path, double* best_ms);

/* Event timing of the batched tensor-core product launches (TF32 modes),
 * as pbpqlp_set_timing / pbpqlp_read_timing. */
int pbpqlp_batch_set_timing(pbpqlp_batch_t batch, int enable);
int pbpqlp_batch_read_timing(pbpqlp_batch_t batch, double* pass_ms_total, int64_t* pass_launches);

/*
 * Learned (q, p) proposer.  Not in the paper: a small network proposes the
 * power-iteration count q in {0..4} and the oversampling p in {5, 10, 20}
 * from cheap features of a first q = 0, l = k + 20 sketch; the caller keeps
 * the plain fixed-q method (q = 2, p = 10) as the fallback, judged by the
 * a-posteriori estimator of pbpqlp_error (PBPQLP_ERR_PROBES).
 *
 * Features (pbpqlp_features): from the L-values d_i = |L_ii| of that sketch
 * (the paper's rank-revealing diagonal, Section IV-C) and m, n, k, 32 floats
 * per matrix: log m / 8, log n / 8, log k / 4, 10 k / min(m, n);
 * log10(d_j / d_1) / 4 at j = round(t k), t = 0.1 .. 1.0 (10 values) and at
 * j = k + 1, 2, 5, 10, 15, 20; log10 of d_k/d_{k+1}, d_k/d_{k+5},
 * d_k/d_{k+20}, d_{k/2}/d_k, d_{k+10}/d_{k+20}; log10 of the sketch tail
 * ratio sqrt(sum_{i>k} d_i^2 / sum_{i<=k} d_i^2) / 4; least-squares slopes
 * of log10 d over [k/2, k] and [k, l] (times k); log10(d_l / d_1) / 4;
 * 10 l / min(m, n); m / n - 1; the constant 1.
 *   L, l, k, m, n: host arrays of count (L[i] a device pointer to the l_i x l_i
 *   factor); features: device, count x 32 FP32; workspace: device,
 *   >= pbpqlp_features_workspace_bytes(count).
 *
 * Network (pbpqlp_mlp_*): 32 -> 128 -> 128 -> 8 with GELU (erf form); the
 * outputs are 5 logits for q and 3 for p.  Parameters are one FP32 vector of
 * pbpqlp_mlp_param_count() floats: W1 (128 x 32), b1, W2 (128 x 128), b2,
 * W3 (8 x 128), b3.  Every linear layer rounds both operands to BF16 and
 * accumulates in FP32 on the tensor cores (forward and backward); the loss is
 * the mean over the batch of the two heads' cross-entropies.  pbpqlp_mlp_adamw
 * is AdamW on the FP32 master parameters (bias-corrected, decoupled decay).
 * pbpqlp_propose writes q and the p index (0, 1, 2 -> p = 5, 10, 20) per row.
 * All pointers are device pointers; workspaces >= pbpqlp_mlp_workspace_bytes(batch).
 */
size_t pbpqlp_features_workspace_bytes(int count);
int pbpqlp_features(int count, const double* const* L, const int* l, const int* k, const int64_t* m,
                    const int64_t* n, float* features, void* workspace, size_t ws_bytes, void* stream);
int pbpqlp_mlp_param_count(void);
size_t pbpqlp_mlp_workspace_bytes(int batch);
int pbpqlp_mlp_init(float* params, uint64_t seed, void* stream);
int pbpqlp_mlp_forward(const float* params, const float* X, int batch, float* logits, void* workspace,
                       size_t ws_bytes, void* stream);
int pbpqlp_mlp_loss_grad(const float* params, const float* X, const int* yq, const int* yp, int batch,
                         float* grad, float* loss, void* workspace, size_t ws_bytes, void* stream);
int pbpqlp_mlp_adamw(float* params, float* m, float* v, const float* grad, int step, float lr, float beta1,
                     float beta2, float eps, float weight_decay, void* stream);
int pbpqlp_propose(const float* features, int count, const float* params, int* q_out, int* p_index_out,
                   void* workspace, size_t ws_bytes, void* stream);

/*
 * pbpqlp_factor_static — the paper has no counterpart; this is a deployment
 * variant of pbpqlp_factor for callers that cannot allocate device memory
 * (code whose host framework owns every device allocation, such as an
 * inference-engine plugin, or a path that must not pay cudaMalloc's implicit
 * synchronisation).  It takes the same inputs and outputs as pbpqlp_factor
 * but no workspace: the scratch is a fixed array of
 * PBPQLP_STATIC_SCRATCH_BYTES inside the library.  Once reserved on a GPU,
 * the array stays reserved there until the process exits.
 *   - Plans with pbpqlp_workspace_bytes(plan) > PBPQLP_STATIC_SCRATCH_BYTES
 *     are rejected with PBPQLP_EWORKSPACE before anything is enqueued.
 *   - The first call on a device does a one-time set-up with that device
 *     current: it looks up the array's device address and caches it.  Under
 *     CUDA's default lazy module loading that lookup is also what loads the
 *     array's module, so the 32 MiB are reserved (an implicit device
 *     allocation that may synchronise) at that first call, not when the
 *     library is loaded; with CUDA_MODULE_LOADING=EAGER they are reserved at
 *     load time.  Make that first call as a warm-up, outside any path that
 *     must not allocate or synchronise, and before any stream capture.
 *     Later calls allocate nothing.  The current device must own the plan's
 *     stream and the buffers.
 *   - Every call shares the one array, so calls whose work overlaps on the
 *     GPU (other streams, other plans, other host threads) race and corrupt
 *     each other; serialise them.  State that must start at zero is cleared
 *     by each call.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.
 *     pbpqlp_sync_status reports its device status like pbpqlp_factor's.
 */
#define PBPQLP_STATIC_SCRATCH_BYTES (32u << 20)
int pbpqlp_factor_static(pbpqlp_plan_t plan, const void* A, int64_t lda, int a_dtype,
                         const double* omega, double* Qa, double* L, double* Qb);

/*
 * Observability (not part of the paper's method).
 * pbpqlp_set_timing: when enable != 0, every later pbpqlp_factor on this plan
 * records a CUDA event pair on the plan's stream around each launch of the
 * kernel that multiplies by A or A^T (the 2q+2 passes of Algorithm 3).
 * pbpqlp_read_timing waits for the stream, returns the summed milliseconds
 * and the number of such launches since the last read, and clears them.
 * Event pairs are created on first use and kept by the plan.
 */
int pbpqlp_set_timing(pbpqlp_plan_t plan, int enable);
int pbpqlp_read_timing(pbpqlp_plan_t plan, double* pass_ms_total, int64_t* pass_launches);

/*
 * Timing by class of launch (observability, not part of the method): bit c
 * of mask enables event pairs around every launch group of class c on later
 * pbpqlp_factor calls (mask 0 disables all; pbpqlp_set_timing toggles bit
 * PBPQLP_TIME_PASS only).  Classes: the products with A or A^T (Eqs. 3 and 5
 * and the power iterations); the Cholesky of the CholeskyQR Gram (with
 * T = R^-T where used); the Grams of CholeskyQR (Eq. 4); the CholeskyQR
 * solve Q = C R^-1; the l x l QR of R^T (Eq. 7); the rest (R = Q^T D and
 * Qb = Pbar Ptil).  pbpqlp_read_timing_class waits for the stream, returns
 * the summed milliseconds and number of groups of class cls since its last
 * read, and clears them.  PBPQLP_EINVAL for an unknown class or mask bit.
 */
enum {
    PBPQLP_TIME_PASS = 0,
    PBPQLP_TIME_CHOL = 1,
    PBPQLP_TIME_GRAM = 2,
    PBPQLP_TIME_SOLVE = 3,
    PBPQLP_TIME_SMALLQR = 4,
    PBPQLP_TIME_OTHER = 5
};
int pbpqlp_set_timing_classes(pbpqlp_plan_t plan, unsigned mask);
int pbpqlp_read_timing_class(pbpqlp_plan_t plan, int cls, double* ms_total, int64_t* groups);

/* Process-wide count of CUDA kernels this library has launched so far. */
int64_t pbpqlp_kernel_launch_count(void);

/*
 * Diagnostic of the library's internal FP64 helpers (not part of the paper's
 * method): for each of the n doubles d[i] (device), writes the Newton-refined
 * reciprocal rcp[i] ~ 1/d[i] and reciprocal square root rsqrt[i] ~
 * 1/sqrt(d[i]) (device outputs) and, when rcp_gs is not NULL, the one-step
 * Goldschmidt reciprocal rcp_gs[i] ~ 1/d[i] of the Cholesky pivot chain; the
 * kernels use them in place of FP64 division and square root.  Positive
 * normal inputs are within 2 ulp of the correctly rounded results; for every
 * other input (zero, subnormal, negative, Inf, NaN, and d >= 2^1023 for the
 * reciprocal) rcp and rsqrt take CUDA's own division / square root, while
 * rcp_gs is meaningless there (its callers reject such pivots first).
 * Asynchronous on `stream`; PBPQLP_EINVAL for n < 0 or null pointers with n > 0.
 */
int pbpqlp_newton_check(const double* d, int64_t n, double* rcp, double* rsqrt, double* rcp_gs, void* stream);

/*
 * Diagnostic of the conversion that ends every FP64-accurate digit product
 * (not part of the paper's method): the digit products accumulate each
 * output as two exact 64-bit integer sums hi and lo, worth (hi 2^28 + lo) 2^e.
 * For each of the n triples (hi[i], lo[i], e[i]) (device arrays), writes
 * fast[i] from the form the kernels use (64-bit operations and one hardware
 * integer-to-double conversion) and exact[i] from the reference form (92-bit
 * integer normalisation); both are the value rounded once to the nearest
 * double, ties to even, for |hi| < 2^62 (device outputs).  Asynchronous on
 * `stream`; PBPQLP_EINVAL for n < 0 or null pointers with n > 0.
 */
int pbpqlp_oz_convert_check(const int64_t* hi, const int64_t* lo, const int* e, int64_t n, double* fast,
                            double* exact, void* stream);

/*
 * Measured FP64 FMA issue rate of the current device (a microbenchmark, not
 * part of the method): CTAs of 256 threads, 1, 2 and 4 per SM, running the
 * inner loop of a register-blocked FP64 GEMM (operands from shared memory,
 * a 4 x 4 block of accumulators per thread);
 * *tflops_out (host) gets the best of 2 x FMAs / the CUDA-event time of a
 * launch, in TFLOP/s.  sink: device scratch of at least 4 x (SM count)
 * doubles (written only if a chain hits a sentinel value).  Synchronous.
 * The benchmark reports FP64 roofline fractions against this measured rate
 * beside the rate derived from unit counts and the maximum clock.
 */
int pbpqlp_fp64_rate_probe(double* sink, double* tflops_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PBPQLP_H */

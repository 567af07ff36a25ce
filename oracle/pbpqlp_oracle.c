/*
 * FP64 CPU oracle for Projection-based Partial QLP (PbP-QLP).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library's product path never
 * does.  It shares no code, header or constant table with the CUDA sources.
 *
 * What it computes (Kaloorazi & Chen, "Projection-based QLP Algorithm for
 * Efficiently Computing Low-Rank Approximation of Matrices"):
 *   - Algorithm 3 (power-iteration-coupled PbP-QLP), executed step by step in
 *     the paper's orientation: Phi is m x l, C = A^T Phi, Pbar = orth(C), q
 *     power iterations with an orth after every product with A or A^T,
 *     D = A Pbar, [Q,R] = qr(D), [Ptil,Rtil] = qr(R^T), P = Pbar Ptil,
 *     L = Rtil^T (Section III, Eqs. 3-8 for q = 0).
 *   - orth() and qr() are the unpivoted thin QR (the paper's "packaged QR",
 *     Section III-A), computed here by Householder reflections with the sign
 *     convention diag(R) >= 0, which makes the thin factors unique for
 *     full-rank inputs.
 *   - The Gaussian test matrix (Section III-A, randn) is drawn from the
 *     counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     SC'11, "Parallel random numbers: as easy as 1, 2, 3") followed by the
 *     Box-Muller transform, written here from those published definitions.
 *
 * Everything is FP64; GEMMs are plain loops that sum over the contraction
 * index in ascending order.  An OpenMP "parallel for" splits independent
 * output rows across host cores and changes no arithmetic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011, Section 3.3 / Table 2).          */
/* Round: two 32x32->64 multiplies by the round multipliers, the high  */
/* halves xor-ed with the other two counter words and the round key;   */
/* the key advances by the Weyl constants between rounds.              */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/*
 * Standard normal samples for linear indices [offset, offset+count).
 * Sample t uses the Philox block b = t / 2 (counter = {b lo, b hi, 0, 0},
 * key = {seed lo, seed hi}).  The four 32-bit outputs give two 53-bit
 * uniforms u1 in (0,1] and u2 in [0,1); Box-Muller then gives
 *   z0 = sqrt(-2 ln u1) cos(2 pi u2),  z1 = sqrt(-2 ln u1) sin(2 pi u2),
 * and sample t takes z0 when t is even, z1 when t is odd.
 */
void orc_gaussian(uint64_t seed, int64_t offset, int64_t count, double* out)
{
    const double two_pi = 6.283185307179586476925286766559;
    const double inv53 = 1.0 / 9007199254740992.0; /* 2^-53 */
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        uint64_t t = (uint64_t)(offset + i);
        uint64_t b = t >> 1;
        uint32_t ctr[4] = {(uint32_t)b, (uint32_t)(b >> 32), 0u, 0u};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        uint64_t a53 = ((uint64_t)(r[0] >> 5) << 26) | (uint64_t)(r[1] >> 6);
        uint64_t b53 = ((uint64_t)(r[2] >> 5) << 26) | (uint64_t)(r[3] >> 6);
        double u1 = ((double)a53 + 1.0) * inv53;   /* (0, 1] */
        double u2 = (double)b53 * inv53;           /* [0, 1) */
        double rad = sqrt(-2.0 * log(u1));
        double ang = two_pi * u2;
        out[i] = (t & 1u) ? rad * sin(ang) : rad * cos(ang);
    }
}

/* ------------------------------------------------------------------ */
/* Plain GEMM.  C (M x N) = op(A) * B with op(A) = A (M x K, lda) or    */
/* A^T (A stored K x M, lda); B is K x N (ldb); all row-major.  Each   */
/* entry sums over the contraction index in ascending order.           */
/* ------------------------------------------------------------------ */
void orc_gemm(int transA, int64_t M, int64_t N, int64_t K,
              const double* A, int64_t lda, const double* B, int64_t ldb,
              double* C, int64_t ldc)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        double* c = C + i * ldc;
        for (int64_t j = 0; j < N; ++j) c[j] = 0.0;
        for (int64_t p = 0; p < K; ++p) {
            double a = transA ? A[p * lda + i] : A[i * lda + p];
            const double* b = B + p * ldb;
            for (int64_t j = 0; j < N; ++j) c[j] += a * b[j];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Unpivoted thin QR by Householder reflections.                        */
/* In: X (rows x cols, ldx), rows >= cols.  Out: Q (rows x cols, ldq)   */
/* with orthonormal columns and R (cols x cols, row-major, upper) with  */
/* diag(R) >= 0 so that X = Q R.  Either output may be NULL.            */
/* For column j the reflector H_j = I - 2 v v^T / (v^T v) maps          */
/* x = W[j:, j] onto alpha e_1 with alpha = -sign(x_0) ||x||; a zero    */
/* column gives H_j = I.  Q = H_0 ... H_{cols-1} [I; 0] is built by     */
/* applying the reflectors in reverse order to [I; 0]; finally the      */
/* signs of the rows of R (and the matching columns of Q) are flipped   */
/* where R[j][j] < 0.                                                   */
/* Returns 0, or -1 on bad sizes / allocation failure.                  */
/* ------------------------------------------------------------------ */
int orc_qr(int64_t rows, int64_t cols, const double* X, int64_t ldx,
           double* Q, int64_t ldq, double* R)
{
    if (rows < cols || cols < 0) return -1;
    if (cols == 0) return 0;
    double* W = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)cols);
    double* V = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)cols); /* reflectors */
    double* vnorm2 = (double*)malloc(sizeof(double) * (size_t)cols);
    double* sgn = (double*)malloc(sizeof(double) * (size_t)cols);
    if (!W || !V || !vnorm2 || !sgn) { free(W); free(V); free(vnorm2); free(sgn); return -1; }
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) W[i * cols + j] = X[i * ldx + j];
    memset(V, 0, sizeof(double) * (size_t)rows * (size_t)cols);

    for (int64_t j = 0; j < cols; ++j) {
        double nrm2 = 0.0;
        for (int64_t i = j; i < rows; ++i) nrm2 += W[i * cols + j] * W[i * cols + j];
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) { vnorm2[j] = 0.0; continue; }
        double x0 = W[j * cols + j];
        double alpha = (x0 >= 0.0) ? -nrm : nrm;
        for (int64_t i = j; i < rows; ++i) V[i * cols + j] = W[i * cols + j];
        V[j * cols + j] = x0 - alpha;
        double vv = 0.0;
        for (int64_t i = j; i < rows; ++i) vv += V[i * cols + j] * V[i * cols + j];
        vnorm2[j] = vv;
        if (vv == 0.0) continue;
        /* apply H_j to the trailing columns W[j:, j:] */
        #pragma omp parallel for schedule(static) if (rows * (cols - j) > 65536)
        for (int64_t c = j; c < cols; ++c) {
            double dot = 0.0;
            for (int64_t i = j; i < rows; ++i) dot += V[i * cols + j] * W[i * cols + c];
            double f = 2.0 * dot / vv;
            for (int64_t i = j; i < rows; ++i) W[i * cols + c] -= f * V[i * cols + j];
        }
    }
    for (int64_t j = 0; j < cols; ++j) sgn[j] = (W[j * cols + j] < 0.0) ? -1.0 : 1.0;
    if (R) {
        for (int64_t i = 0; i < cols; ++i)
            for (int64_t j = 0; j < cols; ++j)
                R[i * cols + j] = (j >= i) ? sgn[i] * W[i * cols + j] : 0.0;
    }
    if (Q) {
        for (int64_t i = 0; i < rows; ++i)
            for (int64_t j = 0; j < cols; ++j) Q[i * ldq + j] = (i == j) ? 1.0 : 0.0;
        for (int64_t j = cols - 1; j >= 0; --j) {
            double vv = vnorm2[j];
            if (vv == 0.0) continue;
            #pragma omp parallel for schedule(static) if (rows * cols > 65536)
            for (int64_t c = 0; c < cols; ++c) {
                double dot = 0.0;
                for (int64_t i = j; i < rows; ++i) dot += V[i * cols + j] * Q[i * ldq + c];
                double f = 2.0 * dot / vv;
                for (int64_t i = j; i < rows; ++i) Q[i * ldq + c] -= f * V[i * cols + j];
            }
        }
        for (int64_t i = 0; i < rows; ++i)
            for (int64_t j = 0; j < cols; ++j) Q[i * ldq + j] *= sgn[j];
    }
    free(W); free(V); free(vnorm2); free(sgn);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Plain sparse product.  A (m x n) in CSR form: the entries of row i    */
/* are (colind[e], values[e]) for rowptr[i] <= e < rowptr[i+1];          */
/* repeated (row, column) pairs add.  C = A B (m x N, B n x N) or        */
/* C = A^T B (n x N, B m x N); B and C row-major (ldb, ldc).  Each       */
/* entry of C sums its terms in ascending e.                            */
/* ------------------------------------------------------------------ */
void orc_csr_mult(int trans, int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colind,
                  const double* values, int64_t N, const double* B, int64_t ldb, double* C, int64_t ldc)
{
    const int64_t rowsC = trans ? n : m;
    for (int64_t i = 0; i < rowsC; ++i)
        for (int64_t j = 0; j < N; ++j) C[i * ldc + j] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const int64_t c = colind[e];
            const double a = values[e];
            /* A: C[i] += a B[c];  A^T: C[c] += a B[i] */
            const double* b = B + (trans ? i : c) * ldb;
            double* o = C + (trans ? c : i) * ldc;
            for (int64_t j = 0; j < N; ++j) o[j] += a * b[j];
        }
}

/* The operand A of Algorithm 3: dense (lda) or CSR. */
typedef struct {
    int64_t m, n;
    const double* A; int64_t lda;                                   /* dense */
    const int64_t* rowptr; const int32_t* colind; const double* values; /* CSR   */
} orc_amat;

/* C (rows x l) = A B (trans = 0) or A^T B (trans = 1). */
static void amat_mult(const orc_amat* a, int trans, int64_t l, const double* B, double* C)
{
    if (a->A) {
        if (trans) orc_gemm(1, a->n, l, a->m, a->A, a->lda, B, l, C, l);
        else orc_gemm(0, a->m, l, a->n, a->A, a->lda, B, l, C, l);
    } else {
        orc_csr_mult(trans, a->m, a->n, a->rowptr, a->colind, a->values, l, B, l, C, l);
    }
}

/* ------------------------------------------------------------------ */
/* Algorithm 3 (PbP-QLP with power iterations, Section III-B).          */
/* In : A (m x n; dense or CSR), l = k + p (the paper's d), q >= 0,     */
/*      Phi (m x l, row-major, contiguous).                             */
/* Out: Q (m x l), L (l x l, lower), P (n x l); optional R (l x l, the  */
/*      first-stage factor of Eq. 6), Pbar (n x l, final basis before   */
/*      the projection), D (m x l, Eq. 5).  All contiguous row-major.   */
/* Returns 0, or -1 on bad sizes / allocation failure.                  */
/* ------------------------------------------------------------------ */
static int pbpqlp_steps(const orc_amat* a, int64_t l, int q,
                        const double* Phi, double* Q, double* L, double* P,
                        double* R_out, double* Pbar_out, double* D_out)
{
    const int64_t m = a->m, n = a->n;
    if (l < 1 || l > m || l > n || q < 0) return -1;
    int rc = 0;
    double* Cn = (double*)malloc(sizeof(double) * (size_t)n * (size_t)l);  /* n x l panel */
    double* Cm = (double*)malloc(sizeof(double) * (size_t)m * (size_t)l);  /* m x l panel */
    double* Pb = (double*)malloc(sizeof(double) * (size_t)n * (size_t)l);  /* Pbar (n x l) */
    double* Pm = (double*)malloc(sizeof(double) * (size_t)m * (size_t)l);  /* orth of the m x l panel */
    double* R = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
    double* RT = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
    double* Pt = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
    double* Rt = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
    if (!Cn || !Cm || !Pb || !Pm || !R || !RT || !Pt || !Rt) { rc = -1; goto done; }

    /* C = A^T Phi (Eq. 3), Pbar = orth(C) (Eq. 4) */
    amat_mult(a, 1, l, Phi, Cn);
    if (orc_qr(n, l, Cn, l, Pb, l, NULL)) { rc = -1; goto done; }
    /* power iterations, an orth after every product (Section III-B) */
    for (int it = 0; it < q; ++it) {
        amat_mult(a, 0, l, Pb, Cm);                                 /* C = A Pbar   */
        if (orc_qr(m, l, Cm, l, Pm, l, NULL)) { rc = -1; goto done; }
        amat_mult(a, 1, l, Pm, Cn);                                 /* C = A^T Pbar */
        if (orc_qr(n, l, Cn, l, Pb, l, NULL)) { rc = -1; goto done; }
    }
    /* D = A Pbar (Eq. 5), [Q, R] = qr(D) (Eq. 6) */
    amat_mult(a, 0, l, Pb, Cm);
    if (D_out) memcpy(D_out, Cm, sizeof(double) * (size_t)m * (size_t)l);
    if (orc_qr(m, l, Cm, l, Q, l, R)) { rc = -1; goto done; }
    /* [Ptil, Rtil] = qr(R^T) (Eq. 7); L = Rtil^T, P = Pbar Ptil (Eq. 8) */
    for (int64_t i = 0; i < l; ++i)
        for (int64_t j = 0; j < l; ++j) RT[i * l + j] = R[j * l + i];
    if (orc_qr(l, l, RT, l, Pt, l, Rt)) { rc = -1; goto done; }
    for (int64_t i = 0; i < l; ++i)
        for (int64_t j = 0; j < l; ++j) L[i * l + j] = Rt[j * l + i];
    orc_gemm(0, n, l, l, Pb, l, Pt, l, P, l);
    if (R_out) memcpy(R_out, R, sizeof(double) * (size_t)l * (size_t)l);
    if (Pbar_out) memcpy(Pbar_out, Pb, sizeof(double) * (size_t)n * (size_t)l);
done:
    free(Cn); free(Cm); free(Pb); free(Pm); free(R); free(RT); free(Pt); free(Rt);
    return rc;
}

/* Dense A (m x n, lda, row-major). */
int orc_pbpqlp(int64_t m, int64_t n, const double* A, int64_t lda, int64_t l, int q,
               const double* Phi, double* Q, double* L, double* P,
               double* R_out, double* Pbar_out, double* D_out)
{
    if (lda < n) return -1;
    orc_amat a = {m, n, A, lda, NULL, NULL, NULL};
    return pbpqlp_steps(&a, l, q, Phi, Q, L, P, R_out, Pbar_out, D_out);
}

/* Sparse A (Section III-C): CSR as in orc_csr_mult. */
int orc_pbpqlp_csr(int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colind, const double* values,
                   int64_t l, int q, const double* Phi, double* Q, double* L, double* P,
                   double* R_out, double* Pbar_out, double* D_out)
{
    orc_amat a = {m, n, NULL, 0, rowptr, colind, values};
    return pbpqlp_steps(&a, l, q, Phi, Q, L, P, R_out, Pbar_out, D_out);
}

/* Number of OpenMP threads a parallel region here uses (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// Blocked l x l steps of Algorithm 3 for sampling sizes beyond one
// thread-block cluster's shared memory (l > 224): the paper's runtime
// workloads (Section V-A, Tables I-III) take d = 0.04n, 0.2n and 0.3n, i.e.
// l up to thousands, where the skinny products become regular GEMMs and the
// orth and the small QR become blocked factorizations.
//
//  - k_dgemm_gen: a general FP64 GEMM, C = alpha op(A) op(B) + beta C, with an
//    upper-triangle-only form, for the trailing updates below.  Each output
//    sums its contraction in index order, so results are deterministic.
//  - The Cholesky of the CholeskyQR Gram G = R^T R together with T = R^{-T}:
//    right-looking over b x b diagonal blocks of the augmented matrix [G | I]
//    (the same elimination as the one-cluster kernel, one level up).  Block t:
//      R_tt, T_tt     = the cluster kernel on S_tt (kernels_cholinv.cu);
//      R[t, r]        = T_tt S[t, r]                (r > t)
//      S[r, r]       -= R[t, r]^T R[t, r]          (upper triangle)
//      T[t, 0:t]      = T_tt Aug[t, 0:t]
//      Aug[r, 0:t+1] -= R[t, r]^T T[t, 0:t+1]      (r > t)
//    with Aug the accumulated left part of the identity half.  A pivot below
//    its threshold makes the whole factorization retry once on G + shift I
//    (shifted CholeskyQR, Fukaya et al. 2020), decided on the device: every
//    launch of an attempt checks a state word and exits at once when its
//    attempt is not the live one.
//  - The Householder QR of R^T (Eq. 7) with diag(Rtil) >= 0: panels of 32
//    columns factored by a thread-block cluster (rows split over the CTAs,
//    column norms and reflector products reduced through distributed shared
//    memory in rank order), the compact-WY factor T of each panel (Schreiber
//    and Van Loan 1989) and GEMM updates of the trailing columns; Ptil is
//    accumulated backwards from the identity; the signs are fixed last.
#include <cooperative_groups.h>
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace cg = cooperative_groups;

namespace pbq {

namespace {

constexpr int kGenBK = 16;
constexpr int kQrNb = 32;          // Householder panel width
constexpr int kQrThreads = 256;
constexpr int kQrCtasMax = 8;

template <int BM, bool TA, bool TB>
__global__ void __launch_bounds__(256)
k_dgemm_gen(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A, int64_t lda,
            const double* __restrict__ B, int64_t ldb, double beta, double* __restrict__ C, int64_t ldc, int upper,
            const int* __restrict__ state, int want) {
    if (state && *state != want) return;
    constexpr int TM = BM / 16;
    const int64_t r0 = (int64_t)blockIdx.y * BM, c0 = (int64_t)blockIdx.x * BM;
    if (upper && c0 + BM <= r0) return;   // tile strictly below the diagonal
    __shared__ double As[kGenBK][BM + 1], Bs[kGenBK][BM + 1];   // As[k][row], Bs[k][col]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = 0; k0 < K; k0 += kGenBK) {
        for (int e = tid; e < BM * kGenBK; e += 256) {
            int rr, kk;
            if (TA) { rr = e % BM; kk = e / BM; }         // A stored K x M: rows contiguous
            else { kk = e % kGenBK; rr = e / kGenBK; }    // A stored M x K: k contiguous
            const int64_t r = r0 + rr, k = k0 + kk;
            As[kk][rr] = (r < M && k < K) ? (TA ? A[k * lda + r] : A[r * lda + k]) : 0.0;
        }
        for (int e = tid; e < BM * kGenBK; e += 256) {
            int cc, kk;
            if (TB) { kk = e % kGenBK; cc = e / kGenBK; }  // B stored N x K
            else { cc = e % BM; kk = e / BM; }             // B stored K x N
            const int64_t c = c0 + cc, k = k0 + kk;
            Bs[kk][cc] = (c < N && k < K) ? (TB ? B[c * ldb + k] : B[k * ldb + c]) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGenBK; ++kk) {
            double a[TM], b[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TM; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = r0 + ty + 16 * i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            const int64_t c = c0 + tx + 16 * j;
            if (c >= N || (upper && c < r)) continue;
            double v = alpha * acc[i][j];
            if (beta != 0.0) v = fma(beta, C[r * ldc + c], v);
            C[r * ldc + c] = v;
        }
    }
}

template <int BM>
cudaError_t dgemm_gen_bm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                         int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, bool upper,
                         const int* state, int want, cudaStream_t s) {
    dim3 grid((unsigned)((N + BM - 1) / BM), (unsigned)((M + BM - 1) / BM));
    const int up = upper ? 1 : 0;
    if (ta && tb) k_dgemm_gen<BM, true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, up, state, want);
    else if (ta) k_dgemm_gen<BM, true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, up, state, want);
    else if (tb) k_dgemm_gen<BM, false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, up, state, want);
    else k_dgemm_gen<BM, false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, up, state, want);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Blocked Cholesky with T = R^{-T}: state words and their kernels
// ---------------------------------------------------------------------------
// bst[0] (the state word): 0 = attempt 0 live, 1 = attempt 0 failed (attempt 1,
// shifted, live), 2 = attempt 1 failed (breakdown), 3 = pass not run,
// 4 = a non-finite pivot.
__global__ void k_bchol_init(int l, int64_t rows, const double* __restrict__ G, double* __restrict__ S,
                             double* __restrict__ Aug, double* __restrict__ T, int* __restrict__ bst,
                             const int* __restrict__ ctl, int pass, int attempt) {
    double shift = 0.0;
    if (attempt == 0) {
        const bool active = !(pass >= 3 && ctl[8 + (pass + 1) / 2] == 0);
        if (blockIdx.x == 0 && threadIdx.x == 0) *bst = active ? 0 : 3;
        if (!active) return;
    } else {
        if (*bst != 1) return;   // nothing writes the state word in this launch
        __shared__ double s_tr;
        if (threadIdx.x == 0) {
            double tr = 0.0;
            for (int j = 0; j < l; ++j) tr += G[(int64_t)j * l + j];
            double sh = 11.0 * ((double)rows * l + (double)l * (l + 1)) * 1.1102230246251565e-16 * tr;
            if (!(sh > 0.0) || !isfinite(sh)) sh = 1.0;
            s_tr = sh;
        }
        __syncthreads();
        shift = s_tr;
    }
    const int64_t total = (int64_t)l * l;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / l, j = e - i * l;
        S[e] = j >= i ? G[e] + (i == j ? shift : 0.0) : 0.0;
        Aug[e] = 0.0;
        T[e] = 0.0;
    }
}

__global__ void k_bchol_final(int l, double* __restrict__ T, const int* __restrict__ bst, int* __restrict__ ctl,
                              int pass, uint32_t* __restrict__ status) {
    const int st = *bst;
    if (st == 3) return;
    if (st == 2 || st == 4) {
        const int64_t total = (int64_t)l * l;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
             e += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = e / l, j = e - i * l;
            T[e] = (i == j) ? 1.0 : 0.0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int shifted = (st == 1 || st == 2) ? 1 : 0;
        ctl[pass] = shifted;
        if ((pass & 1) == 0) ctl[8 + pass / 2 + 1] = (ctl[pass - 1] | ctl[pass]) ? 1 : 0;
        if (shifted) atomicOr(status, kStShifted);
        if (st == 2) atomicOr(status, kStBreakdown);
    }
}

// ---------------------------------------------------------------------------
// Blocked Householder QR of R^T
// ---------------------------------------------------------------------------
// M = R^T (R upper, ld l): M[i][j] = R[j][i] for i >= j, else 0.
__global__ void k_transpose_upper(int l, const double* __restrict__ R, double* __restrict__ M) {
    __shared__ double tile[32][33];
    const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = bj + r, j = bi + tx;        // read R[bj + r][bi + tx]
        tile[r][tx] = (i < l && j < l) ? R[i * l + j] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = bi + r, j = bj + tx;        // M[i][j] = R[j][i]
        if (i < l && j < l) M[i * l + j] = (i >= j) ? tile[tx][r] : 0.0;
    }
}

// Householder factorization of the panel M[c0:l, c0:c0+w] (h = l - c0 rows)
// by a cluster: CTA r holds panel rows [r hc, (r+1) hc) in shared memory.
// Column j: x = M[c0+j:, c0+j], alpha = x_0, beta = -sign(alpha) ||x||,
// v = x / (alpha - beta) with v_0 = 1, tau = (beta - alpha) / beta (tau = 0,
// beta = alpha when x has no entries below the pivot), then the remaining
// panel columns get (I - tau v v^T).  Writes the reduced panel back to M
// (R rows on and above the diagonal), v explicitly into V[c0:, c0:c0+w]
// (zeros above the unit diagonal) and tau into taus[c0 .. c0+w).
__global__ void __launch_bounds__(kQrThreads)
k_hqr_panel(int l, int c0, int w, double* __restrict__ M, double* __restrict__ V, double* __restrict__ taus) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int h = l - c0;
    const int hc = (h + C - 1) / C;
    const int rbeg = rank * hc, rend = min(h, rbeg + hc);
    const int ld = w + 1;
    extern __shared__ double smq[];
    double* pan = smq;                               // hc x (w + 1)
    double* red0 = pan + (int64_t)hc * ld;           // 2: [sum of squares below the pivot, pivot]
    double* red1 = red0 + 2;                         // kQrNb: partial products v^T M[:, k]
    double* wsum = red1 + kQrNb;                     // 8 warps x kQrNb scratch
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = kQrThreads / 32;
    for (int e = tid; e < (rend - rbeg) * w; e += kQrThreads) {
        const int i = e / w, k = e - i * w;
        pan[i * ld + k] = M[(int64_t)(c0 + rbeg + i) * l + c0 + k];
    }
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        // (1) sum of squares of column j below the pivot and the pivot itself
        double sq = 0.0, piv = 0.0;
        for (int i = rbeg + tid; i < rend; i += kQrThreads) {
            const double x = pan[(i - rbeg) * ld + j];
            if (i > j) sq = fma(x, x, sq);
            if (i == j) piv = x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_xor_sync(0xffffffffu, sq, o);
            piv += __shfl_xor_sync(0xffffffffu, piv, o);
        }
        if (lane == 0) { wsum[warp * 2] = sq; wsum[warp * 2 + 1] = piv; }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < nwarp; ++q) { a += wsum[q * 2]; b += wsum[q * 2 + 1]; }
            red0[0] = a;
            red0[1] = b;
        }
        cluster.sync();
        double xsq = 0.0, alpha = 0.0;
        for (int r = 0; r < C; ++r) {
            const double* rr = cluster.map_shared_rank(red0, r);
            xsq += rr[0];
            alpha += rr[1];
        }
        double beta = alpha, tau = 0.0, scale = 0.0;
        if (xsq > 0.0) {
            const double nrm = sqrt(fma(alpha, alpha, xsq));
            beta = alpha >= 0.0 ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            scale = 1.0 / (alpha - beta);
        }
        // (2) v below the pivot, the pivot row gets beta; record v and tau
        for (int i = rbeg + tid; i < rend; i += kQrThreads) {
            double* x = &pan[(i - rbeg) * ld + j];
            if (i > j) *x *= scale;
            if (i == j) *x = beta;
        }
        if (rank == 0 && tid == 0) taus[c0 + j] = tau;
        __syncthreads();
        // (3) partial products p_k = sum_i v_i M[i][k] over own rows (v_j = 1), k > j
        for (int k = j + 1 + warp; k < w; k += nwarp) {
            double acc = 0.0;
            for (int i = max(rbeg, j) + lane; i < rend; i += 32) {
                const double v = (i == j) ? 1.0 : pan[(i - rbeg) * ld + j];
                acc = fma(v, pan[(i - rbeg) * ld + k], acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) red1[k] = acc;
        }
        cluster.sync();
        // (4) M[i][k] -= tau v_i p_k over own rows i >= j
        if (tau != 0.0) {
            for (int e = tid; e < (w - j - 1) * 32; e += kQrThreads) {
                const int k = j + 1 + e / 32, li = e % 32;
                double p = 0.0;
                for (int r = 0; r < C; ++r) p += cluster.map_shared_rank(red1, r)[k];
                const double tp = tau * p;
                for (int i = max(rbeg, j) + li; i < rend; i += 32) {
                    const double v = (i == j) ? 1.0 : pan[(i - rbeg) * ld + j];
                    pan[(i - rbeg) * ld + k] -= tp * v;
                }
            }
        }
        __syncthreads();
    }
    // write back the panel and the explicit reflectors
    for (int e = tid; e < (rend - rbeg) * w; e += kQrThreads) {
        const int i = e / w, k = e - i * w;
        const int gi = rbeg + i;   // panel row
        const double x = pan[i * ld + k];
        M[(int64_t)(c0 + gi) * l + c0 + k] = x;
        V[(int64_t)(c0 + gi) * l + c0 + k] = gi > k ? x : (gi == k ? 1.0 : 0.0);
    }
    cluster.sync();   // no CTA leaves while another may still read its reductions
}

// Compact-WY factor of one panel: T (w x w upper, ld kQrNb) with
// H_1 ... H_w = I - V T V^T, from VtV = V^T V and tau (forward, columnwise):
// T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] VtV[0:j, j].
__global__ void k_build_t(int w, const double* __restrict__ VtV, int ldv, const double* __restrict__ tau,
                          double* __restrict__ T) {
    const int i = threadIdx.x;
    for (int e = i; e < kQrNb * kQrNb; e += blockDim.x) T[e] = 0.0;
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        const double tj = tau[j];
        double y = 0.0;
        if (i < j) {
            for (int k = i; k < j; ++k) y = fma(T[i * kQrNb + k], VtV[k * ldv + j], y);
        }
        __syncthreads();
        if (i < j) T[i * kQrNb + j] = -tj * y;
        if (i == j) T[j * kQrNb + j] = tj;
        __syncthreads();
    }
}

__global__ void k_eye(int l, double* __restrict__ P) {
    const int64_t total = (int64_t)l * l;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / l, j = e - i * l;
        P[e] = (i == j) ? 1.0 : 0.0;
    }
}

// diag(Rtil) >= 0: d_j = sign(M[j][j]) (+1 for 0); L = (D Rtil)^T, Ptil <- Ptil D.
__global__ void k_qr_signs(int l, const double* __restrict__ M, double* __restrict__ L, double* __restrict__ P) {
    const int64_t total = (int64_t)l * l;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / l, j = e - i * l;
        const double d = M[j * l + j] < 0.0 ? -1.0 : 1.0;
        // Rtil = upper triangle of M: L[i][j] = d_j Rtil[j][i] for i >= j
        L[e] = (i >= j) ? d * M[j * l + i] : 0.0;
        P[e] *= d;
    }
}

unsigned grid_for(int64_t elems) {
    int64_t b = (elems + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_dgemm_gen(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                             int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, bool upper,
                             const int* state, int want, cudaStream_t s) {
    if (M < 1 || N < 1) return cudaSuccess;
    if (K < 0) return cudaErrorInvalidValue;
    // 64 x 64 tiles when they fill the SMs, 32 x 32 tiles otherwise
    const int64_t tiles64 = ((M + 63) / 64) * ((N + 63) / 64);
    if (tiles64 >= 152) return dgemm_gen_bm<64>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, upper, state, want, s);
    return dgemm_gen_bm<32>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, upper, state, want, s);
}

size_t chol_inv_blocked_work_bytes(int l) { return sizeof(double) * 3 * (size_t)l * l + 256; }

cudaError_t launch_chol_inv_blocked(int l, int64_t rows, const double* G, double* T, void* work, uint32_t* status,
                                    int* ctl, int pass, cudaStream_t s) {
    const int b = kCholBlock;
    double* S = (double*)work;
    double* Aug = S + (int64_t)l * l;
    double* R = Aug + (int64_t)l * l;
    int* bst = (int*)(R + (int64_t)l * l);
    cudaError_t e;
    for (int attempt = 0; attempt < 2; ++attempt) {
        k_bchol_init<<<grid_for((int64_t)l * l), 256, 0, s>>>(l, rows, G, S, Aug, T, bst, ctl, pass, attempt);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (int a0 = 0; a0 < l; a0 += b) {
            const int a1 = a0 + b < l ? a0 + b : l, nb = a1 - a0;
            const int64_t o = (int64_t)a0 * l;
            if ((e = launch_chol_inv_block(nb, S + o + a0, l, G + o + a0, R + o + a0, T + o + a0, status, bst, attempt,
                                           s)) != cudaSuccess)
                return e;
            if (a1 < l) {
                // R[t, r] = T_tt S[t, r]; S[r, r] -= R[t, r]^T R[t, r] (upper)
                if ((e = launch_dgemm_gen(false, false, nb, l - a1, nb, 1.0, T + o + a0, l, S + o + a1, l, 0.0,
                                          R + o + a1, l, false, bst, attempt, s)) != cudaSuccess)
                    return e;
                if ((e = launch_dgemm_gen(true, false, l - a1, l - a1, nb, -1.0, R + o + a1, l, R + o + a1, l, 1.0,
                                          S + (int64_t)a1 * l + a1, l, true, bst, attempt, s)) != cudaSuccess)
                    return e;
            }
            if (a0 > 0) {
                // T[t, 0:t] = T_tt Aug[t, 0:t]
                if ((e = launch_dgemm_gen(false, false, nb, a0, nb, 1.0, T + o + a0, l, Aug + o, l, 0.0, T + o, l, false,
                                          bst, attempt, s)) != cudaSuccess)
                    return e;
            }
            if (a1 < l) {
                // Aug[r, 0:t+1] -= R[t, r]^T T[t, 0:t+1]
                if ((e = launch_dgemm_gen(true, false, l - a1, a1, nb, -1.0, R + o + a1, l, T + o, l, 1.0,
                                          Aug + (int64_t)a1 * l, l, false, bst, attempt, s)) != cudaSuccess)
                    return e;
            }
        }
    }
    k_bchol_final<<<grid_for((int64_t)l * l), 256, 0, s>>>(l, T, bst, ctl, pass, status);
    count_launches(1);
    return cudaGetLastError();
}

size_t qr_blocked_work_bytes(int l) {
    const size_t nblk = (size_t)(l + kQrNb - 1) / kQrNb;
    return sizeof(double) * (2 * (size_t)l * l + nblk * kQrNb * kQrNb + (size_t)l + 2 * (size_t)kQrNb * l +
                             (size_t)kQrNb * kQrNb) + 256;
}

static size_t hqr_smem(int h, int C) {
    const int hc = (h + C - 1) / C;
    return sizeof(double) * ((size_t)hc * (kQrNb + 1) + 2 + kQrNb + 2 * 8 * kQrNb);
}

bool qr_blocked_fits(int l) { return l >= 1 && l <= kMaxEllBlocked && hqr_smem(l, kQrCtasMax) <= 200 * 1024; }

cudaError_t launch_qr_blocked(int l, const double* R, double* L, double* Pt, void* work, cudaStream_t s) {
    if (!qr_blocked_fits(l)) return cudaErrorInvalidValue;
    double* M = (double*)work;
    double* V = M + (int64_t)l * l;
    const int nblk = (l + kQrNb - 1) / kQrNb;
    double* Tall = V + (int64_t)l * l;
    double* tau = Tall + (int64_t)nblk * kQrNb * kQrNb;
    double* W1 = tau + l;
    double* W2 = W1 + (int64_t)kQrNb * l;
    double* VtV = W2 + (int64_t)kQrNb * l;
    cudaError_t e;
    {
        dim3 grid((unsigned)((l + 31) / 32), (unsigned)((l + 31) / 32)), block(32, 8);
        k_transpose_upper<<<grid, block, 0, s>>>(l, R, M);
        count_launches(1);
    }
    auto ctas = [](int h) {
        const int C = h / 64;
        return C < 1 ? 1 : (C > kQrCtasMax ? kQrCtasMax : C);
    };
    size_t smax = 0;
    for (int c0 = 0; c0 < l; c0 += kQrNb) {
        const size_t b = hqr_smem(l - c0, ctas(l - c0));
        smax = b > smax ? b : smax;
    }
    if ((e = func_smem_attr((const void*)k_hqr_panel, smax)) != cudaSuccess) return e;
    for (int p = 0; p < nblk; ++p) {
        const int c0 = p * kQrNb, w = l - c0 < kQrNb ? l - c0 : kQrNb, h = l - c0;
        const int C = ctas(h);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kQrThreads);
        cfg.dynamicSmemBytes = hqr_smem(h, C);
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if ((e = cudaLaunchKernelEx(&cfg, k_hqr_panel, l, c0, w, M, V, tau)) != cudaSuccess) return e;
        count_launches(1);
        const double* Vp = V + (int64_t)c0 * l + c0;
        double* Tp = Tall + (int64_t)p * kQrNb * kQrNb;
        // VtV = V_p^T V_p (w x w), T_p from it
        if ((e = launch_dgemm_gen(true, false, w, w, h, 1.0, Vp, l, Vp, l, 0.0, VtV, kQrNb, false, nullptr, 0, s)))
            return e;
        k_build_t<<<1, kQrNb, 0, s>>>(w, VtV, kQrNb, tau + c0, Tp);
        count_launches(1);
        const int wc = l - c0 - w;
        if (wc > 0) {
            // M[c0:, c0+w:] -= V_p (T_p^T (V_p^T M[c0:, c0+w:]))
            double* Cm = M + (int64_t)c0 * l + c0 + w;
            if ((e = launch_dgemm_gen(true, false, w, wc, h, 1.0, Vp, l, Cm, l, 0.0, W1, wc, false, nullptr, 0, s)))
                return e;
            if ((e = launch_dgemm_gen(true, false, w, wc, w, 1.0, Tp, kQrNb, W1, wc, 0.0, W2, wc, false, nullptr, 0, s)))
                return e;
            if ((e = launch_dgemm_gen(false, false, h, wc, w, -1.0, Vp, l, W2, wc, 1.0, Cm, l, false, nullptr, 0, s)))
                return e;
        }
    }
    // Ptil = H_1 ... H_l = Q_1 (Q_2 (... Q_P I)), Q_p = I - V_p T_p V_p^T on rows/columns c0:
    k_eye<<<grid_for((int64_t)l * l), 256, 0, s>>>(l, Pt);
    count_launches(1);
    for (int p = nblk - 1; p >= 0; --p) {
        const int c0 = p * kQrNb, w = l - c0 < kQrNb ? l - c0 : kQrNb, h = l - c0;
        const double* Vp = V + (int64_t)c0 * l + c0;
        const double* Tp = Tall + (int64_t)p * kQrNb * kQrNb;
        double* Qs = Pt + (int64_t)c0 * l + c0;
        if ((e = launch_dgemm_gen(true, false, w, h, h, 1.0, Vp, l, Qs, l, 0.0, W1, h, false, nullptr, 0, s))) return e;
        if ((e = launch_dgemm_gen(false, false, w, h, w, 1.0, Tp, kQrNb, W1, h, 0.0, W2, h, false, nullptr, 0, s)))
            return e;
        if ((e = launch_dgemm_gen(false, false, h, h, w, -1.0, Vp, l, W2, h, 1.0, Qs, l, false, nullptr, 0, s))) return e;
    }
    k_qr_signs<<<grid_for((int64_t)l * l), 256, 0, s>>>(l, M, L, Pt);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq

// Cholesky of the l x l CholeskyQR Gram together with the inverse of its
// factor, by a thread-block cluster of 16 CTAs (8 where 16-CTA clusters cannot
// be scheduled): G = R^T R and T = R^{-T}.
// With T the CholeskyQR step Q = C R^{-1} = C T^T is one product, which runs
// on the tensor cores in FP64-accurate digit form (kernels_oz.cu) instead of
// a row-by-row triangular solve.
//
// Method: block right-looking elimination of the augmented matrix [G | I]
// (row operations with R^{-T} turn it into [R | R^{-T}]), 16-row blocks.
// Columns of both halves are dealt cyclically over the C CTAs (column j lives
// in CTA j % C at local column j / C, full length l in shared memory), so the
// trailing updates, which hold nearly all the l^3 / 3 FMAs, are spread over
// all C SMs.  Block t:
//   (a) every CTA gathers the 16 x 16 diagonal block through distributed
//       shared memory and factors it (one warp, redundantly: all CTAs take the
//       same pivot decisions without communicating);
//   (b) each CTA solves its own columns' block rows, R[t, j] = R_tt^{-T} S[t, j]
//       (columns right of the block) and T[t, j] = R_tt^{-T} T[t, j];
//   cluster barrier; each CTA copies block row t of R (columns right of the
//   block) from the owners;
//   (c) trailing updates of own columns: S[i][j] -= sum_k R[t,k][i] R[t,k][j]
//       (a1 <= i <= j) and T[i][j] -= sum_k R[t,k][i] T[t,k][j] (i >= a1);
//   cluster barrier.
// FP64 has few lanes per SM on GB300 and long latencies, so the sequential
// parts are kept short: the diagonal block is factored in LDL^T form (one
// reciprocal per pivot, an FP32 seed refined by Newton-Raphson steps in FP64;
// the square roots of all pivots come afterwards, in parallel), and the
// block-row solve updates all remaining right-hand sides after each unknown
// (two dependent operations per step).  Pivot thresholds and the shifted retry
// (shifted CholeskyQR, Fukaya et al. 2020) follow the one-CTA kernel; ctl /
// status conventions are the same.
#include <cooperative_groups.h>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "newton_device.cuh"

namespace cg = cooperative_groups;

namespace pbq {

namespace {
constexpr int kCiCtasMax = 16;
constexpr int kCiThreads = 512;
constexpr int kCiNb = 16;

// Latencies measured on GB300: a dependent FP64 FMA takes 64 cycles, an FP64
// square root ~670 and a division ~430, an FP32 FMA 4.5.  The sequential
// chains below therefore avoid FP64 square roots and divisions (rcp_nr,
// rsqrt_nr).

}  // namespace

// kBlock: the kernel factors one l x l diagonal block S_tt of a blocked
// factorization (kernels_blocked.cu) instead of a whole Gram: it reads the
// block at G (leading dimension ld), its pivot thresholds from the original
// Gram's diagonal at gdiag (stride ld + 1), writes R_tt (upper, into Rp with
// leading dimension ld) and T_tt (lower, into Tout, ld), makes one attempt,
// and on a failed pivot sets *bstate = want + 1 (4 for a non-finite pivot,
// with the status bit) instead of retrying.  It runs only if *bstate == want.
template <bool kBlock>
__global__ void __launch_bounds__(kCiThreads)
k_chol_inv_cluster(int l, int64_t rows, const double* __restrict__ G, double* __restrict__ Rp,
                   double* __restrict__ Tout, uint32_t* __restrict__ status, int* __restrict__ ctl, int pass,
                   int64_t ld, const double* __restrict__ gdiag, int* __restrict__ bstate, int want) {
    if (kBlock) {
        if (*bstate != want) return;   // uniform: nothing writes it before the first cluster barrier
    } else {
        if (pass >= 3 && ctl[8 + (pass + 1) / 2] == 0) return;   // uniform over the cluster
        ld = l;
    }
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int ncol = (l + C - 1) / C;
    const int nblk = (l + kCiNb - 1) / kCiNb;
    extern __shared__ double smi[];
    double* Sown = smi;                                  // ncol x l: own columns of S (then R)
    double* Town = Sown + (int64_t)ncol * l;             // ncol x l: own columns of T
    double* Rbuf = Town + (int64_t)ncol * l;             // 16 x l: block row t of R
    double* Rtt = Rbuf + (int64_t)kCiNb * l;             // 16 x 16: factored diagonal block (upper), [p][k]
    double* Rinv = Rtt + kCiNb * kCiNb;                  // 16: 1 / R_tt[k][k]
    __shared__ int s_fail;
    __shared__ double s_shift;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const double tau = 1e-12;

    if (tid == 0) { s_fail = 0; s_shift = 0.0; }
    __syncthreads();
    int shifted = 0, fail = 0;
    for (int attempt = 0; attempt < (kBlock ? 1 : 2); ++attempt) {
        const double shift = s_shift;
        for (int e = tid; e < ncol * l; e += nth) {
            const int jl = e / l, i = e - jl * l, j = jl * C + rank;
            double sv = 0.0, tv = 0.0;
            if (j < l) {
                if (i <= j) sv = G[(int64_t)i * ld + j] + (i == j ? shift : 0.0);
                tv = (i == j) ? 1.0 : 0.0;
            }
            Sown[e] = sv;
            Town[e] = tv;
        }
        fail = 0;
        cluster.sync();
        for (int t = 0; t < nblk; ++t) {
            const int a0 = t * kCiNb, a1 = min(l, a0 + kCiNb), nb = a1 - a0;
            // (a) gather and factor the diagonal block (warp 0 of every CTA).  LDL^T
            // form: step p needs only 1/d_p (the chain from one pivot to the
            // next is a reciprocal and two FMAs); the rows of R are scaled by
            // 1/sqrt(d_p) afterwards, all pivots at once.
            if (warp == 0) {
                double s[kCiNb];
                const int j = a0 + lane;
                double thr_mine = 0.0, d_mine = 1.0;
                if (lane < nb) {
                    const double* col = cluster.map_shared_rank(Sown, j % C) + (int64_t)(j / C) * l;
#pragma unroll
                    for (int i = 0; i < kCiNb; ++i) s[i] = (i <= lane) ? col[a0 + i] : 0.0;
                    // the shifted retry (attempt 1, or want 1 in block mode) only asks for d > 0
                    if (attempt == 0 && !(kBlock && want == 1))
                        thr_mine = tau * (kBlock ? gdiag[(int64_t)j * (ld + 1)] : G[(int64_t)j * l + j]);
                } else {
#pragma unroll
                    for (int i = 0; i < kCiNb; ++i) s[i] = 0.0;
                }
                int f = 0;
#pragma unroll
                for (int p = 0; p < kCiNb; ++p) {
                    if (p < nb && f == 0) {
                        const double d = __shfl_sync(0xffffffffu, s[p], p);
                        const double thr = __shfl_sync(0xffffffffu, thr_mine, p);
                        f = !isfinite(d) ? 2 : (!(d > thr) ? 1 : 0);
                        if (f == 0) {
                            const double c = rcp_nr(d);
                            if (lane == p) d_mine = d;
                            const double lk = s[p] * c;   // L[lane][p] = S[p][lane] / d_p
#pragma unroll
                            for (int i = p + 1; i < kCiNb; ++i) {
                                const double spi = __shfl_sync(0xffffffffu, s[p], i);
                                if (lane >= i) s[i] -= spi * lk;
                            }
                        }
                    }
                }
                if (f == 0) {
                    // R[p][k] = S_p[k] / sqrt(d_p) (p < k), R[k][k] = sqrt(d_k)
                    const double rs = rsqrt_nr(d_mine);
#pragma unroll
                    for (int p = 0; p < kCiNb; ++p) {
                        const double rsp = __shfl_sync(0xffffffffu, rs, p);
                        if (lane < nb) Rtt[p * kCiNb + lane] = (p < lane) ? s[p] * rsp : (p == lane ? d_mine * rs : 0.0);
                    }
                    if (lane < nb) Rinv[lane] = rs;
                }
                if (lane == 0) s_fail = f;
            }
            __syncthreads();
            fail = s_fail;
            if (fail) break;   // every CTA factored the same block: same decision everywhere
            // (b) block-row solves R_tt^T y = x on own columns (one thread per column):
            // after each unknown all later right-hand sides are updated at once
            if (tid < 2 * ncol) {
                const bool right = tid >= ncol;
                const int jl = right ? tid - ncol : tid;
                const int j = jl * C + rank;
                if (j < l && (right ? (j < a1) : (j >= a1))) {
                    double* x = (right ? Town : Sown) + (int64_t)jl * l + a0;
                    double acc[kCiNb];
#pragma unroll
                    for (int k = 0; k < kCiNb; ++k) acc[k] = (k < nb) ? x[k] : 0.0;
#pragma unroll
                    for (int p = 0; p < kCiNb; ++p) {
                        if (p < nb) {
                            const double y = acc[p] * Rinv[p];
                            acc[p] = y;
#pragma unroll
                            for (int k = p + 1; k < kCiNb; ++k) acc[k] -= Rtt[p * kCiNb + k] * y;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < kCiNb; ++k)
                        if (k < nb) x[k] = acc[k];
                }
            }
            cluster.sync();   // block row t of R is final in its owners
            // copy block row t of R, columns a1 .. l-1, from the owners
            const int w1 = l - a1;
            for (int e = tid; e < nb * w1; e += nth) {
                const int k = e / w1, j = a1 + (e - k * w1);
                Rbuf[(int64_t)k * l + j] = cluster.map_shared_rank(Sown, j % C)[(int64_t)(j / C) * l + a0 + k];
            }
            __syncthreads();
            // (c) trailing updates, one warp per own column
            for (int jl = warp; jl < ncol; jl += nwarp) {
                const int j = jl * C + rank;
                if (j >= l) continue;
                if (j >= a1) {
                    double* col = Sown + (int64_t)jl * l;
                    double rj[kCiNb];
#pragma unroll
                    for (int k = 0; k < kCiNb; ++k) rj[k] = (k < nb) ? col[a0 + k] : 0.0;
                    for (int i = a1 + lane; i <= j; i += 32) {
                        double acc = col[i];
#pragma unroll
                        for (int k = 0; k < kCiNb; ++k)
                            if (k < nb) acc -= Rbuf[(int64_t)k * l + i] * rj[k];
                        col[i] = acc;
                    }
                } else {
                    double* tcol = Town + (int64_t)jl * l;
                    double tj[kCiNb];
#pragma unroll
                    for (int k = 0; k < kCiNb; ++k) tj[k] = (k < nb) ? tcol[a0 + k] : 0.0;
                    for (int i = a1 + lane; i < l; i += 32) {
                        double acc = tcol[i];
#pragma unroll
                        for (int k = 0; k < kCiNb; ++k)
                            if (k < nb) acc -= Rbuf[(int64_t)k * l + i] * tj[k];
                        tcol[i] = acc;
                    }
                    if (j >= a0) {
                        // own column of the diagonal block: its rows a0 .. a1-1 of R are R_tt's column
                        double* col = Sown + (int64_t)jl * l;
                        for (int k = lane; k < nb; k += 32) col[a0 + k] = Rtt[k * kCiNb + (j - a0)];
                    }
                }
            }
            cluster.sync();   // updates visible before the next gather
        }
        __syncthreads();
        if (!fail) break;
        if (kBlock) {
            // every CTA saw the same failure; the host-side sequence retries or falls back
            if (rank == 0 && tid == 0) {
                if (fail == 2) atomicOr(status, kStNonFinite);
                *bstate = fail == 2 ? 4 : want + 1;
            }
            cluster.sync();
            return;
        }
        if (fail == 2 || attempt == 1) {
            if (rank == 0 && tid == 0) atomicOr(status, fail == 2 ? kStNonFinite : kStBreakdown);
            for (int e = tid; e < ncol * l; e += nth) {
                const int jl = e / l, i = e - jl * l, j = jl * C + rank;
                Sown[e] = (i == j) ? 1.0 : 0.0;
                Town[e] = (i == j) ? 1.0 : 0.0;
            }
            __syncthreads();
            break;
        }
        if (tid == 0) {
            double tr = 0.0;
            for (int j = 0; j < l; ++j) tr += G[(int64_t)j * l + j];
            double sh = 11.0 * ((double)rows * l + (double)l * (l + 1)) * 1.1102230246251565e-16 * tr;
            if (!(sh > 0.0) || !isfinite(sh)) sh = 1.0;
            s_shift = sh;
        }
        shifted = 1;
        cluster.sync();   // every CTA is past its reads of the other CTAs' columns
    }
    if (kBlock) {
        // R_tt (upper) and T_tt (lower) into the blocked factorization's matrices
        for (int e = tid; e < ncol * l; e += nth) {
            const int jl = e / l, i = e - jl * l, j = jl * C + rank;
            if (j >= l) continue;
            if (i <= j) Rp[(int64_t)i * ld + j] = Sown[e];
            if (i >= j) Tout[(int64_t)i * ld + j] = Town[e];
        }
        cluster.sync();   // no CTA leaves while another may still read its shared memory
        return;
    }
    // R packed (row a at a(2l - a + 1)/2, columns a .. l-1), 1/diag after it; T row-major
    const int64_t P = (int64_t)l * (l + 1) / 2;
    for (int e = tid; e < ncol * l; e += nth) {
        const int jl = e / l, i = e - jl * l, j = jl * C + rank;
        if (j >= l) continue;
        if (i <= j) Rp[(int64_t)i * (2 * l - i + 1) / 2 + (j - i)] = Sown[e];
        if (i == j) Rp[P + j] = 1.0 / Sown[e];
        if (Tout) Tout[(int64_t)i * l + j] = (i >= j) ? Town[e] : 0.0;
    }
    if (rank == 0 && tid == 0) {
        ctl[pass] = shifted;
        if ((pass & 1) == 0) ctl[8 + pass / 2 + 1] = (ctl[pass - 1] | ctl[pass]) ? 1 : 0;
        if (shifted) atomicOr(status, kStShifted);
    }
    cluster.sync();   // no CTA leaves while another may still read its shared memory
}

// Shared memory of one CTA, at least 120 KB so that no two CTAs of the cluster
// share an SM (and its FP64 lanes).
static size_t chol_inv_smem(int l, int C) {
    const int ncol = (l + C - 1) / C;
    const size_t need = ((size_t)2 * ncol * l + (size_t)kCiNb * l + kCiNb * kCiNb + kCiNb) * sizeof(double);
    return need > 120 * 1024 ? need : 120 * 1024;
}

// Cluster size: 16 CTAs when the device can schedule such clusters with this
// kernel's shared memory, else the portable 8 (decided once per process).
static int chol_inv_ctas(int l) {
    static int best = 0;
    if (best == 0) {
        best = 8;
        cudaFuncAttributes fa;
        if (cudaFuncSetAttribute(k_chol_inv_cluster<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_chol_inv_cluster<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_chol_inv_cluster<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)chol_inv_smem(kMaxEll, 8)) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, k_chol_inv_cluster<false>) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = kCiCtasMax;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(kCiCtasMax);
            cfg.blockDim = dim3(kCiThreads);
            cfg.dynamicSmemBytes = chol_inv_smem(kMaxEll, kCiCtasMax);
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, k_chol_inv_cluster<false>, &cfg) == cudaSuccess &&
                clusters > 0)
                best = kCiCtasMax;
        }
        cudaGetLastError();
    }
    (void)l;
    return best;
}

bool chol_inv_fits(int l) { return l >= 1 && l <= kMaxEll && chol_inv_smem(l, 8) <= 200 * 1024; }

template <bool kBlock>
static cudaError_t chol_inv_launch(int l, int64_t rows, const double* G, double* Rp, double* T, uint32_t* status,
                                   int* ctl, int pass, int64_t ld, const double* gdiag, int* bstate, int want,
                                   cudaStream_t s) {
    const int C = chol_inv_ctas(l);
    const size_t smem = chol_inv_smem(l, C);
    cudaError_t e = func_smem_attr((const void*)k_chol_inv_cluster<kBlock>, smem);
    if (e != cudaSuccess) return e;
    // (the non-portable cluster size was allowed once, when C = 16 was chosen)
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kCiThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_chol_inv_cluster<kBlock>, l, rows, G, Rp, T, status, ctl, pass, ld, gdiag, bstate,
                           want);
    count_launches(1);
    return e;
}

cudaError_t launch_chol_inv(int l, int64_t rows, const double* G, double* Rp, double* T, uint32_t* status, int* ctl,
                            int pass, cudaStream_t s) {
    return chol_inv_launch<false>(l, rows, G, Rp, T, status, ctl, pass, l, nullptr, nullptr, 0, s);
}

cudaError_t launch_chol_inv_block(int b, const double* S, int64_t ld, const double* gdiag, double* R, double* T,
                                  uint32_t* status, int* bstate, int want, cudaStream_t s) {
    if (b < 1 || b > kMaxEll) return cudaErrorInvalidValue;
    return chol_inv_launch<true>(b, 0, S, R, T, status, nullptr, 0, ld, gdiag, bstate, want, s);
}

}  // namespace pbq

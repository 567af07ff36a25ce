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
//   (a) every CTA factors the 16 x 16 diagonal block (four warps,
//       redundantly: all CTAs take the same pivot decisions without
//       communicating), which gives R_tt and T_tt = R_tt^{-T} at once (the
//       identity beside it is eliminated along with it);
//   (b) each CTA forms its own columns' block rows as small products,
//       R[t, j] = T_tt S[t, j] (columns right of the block) and
//       T[t, j] = T_tt T[t, j], and writes the R values into every CTA's
//       block-row buffer (distributed shared memory); cluster barrier;
//   (c1) the owners of block t+1's columns update them first and write them
//       into every CTA's diagonal-block buffer; cluster barrier;
//   (a) of block t+1 on warps 0-3, while warps 4-7 run (c2), the trailing
//       updates of all other own columns: S[i][j] -= sum_k R[t,k][i] R[t,k][j]
//       (a1 <= i <= j) and T[i][j] -= sum_k R[t,k][i] T[t,k][j] (i >= a1).
// So the sequential pivot chain of the next block overlaps the trailing
// update, every value crosses between CTAs as a store (no remote loads), and
// a block costs two cluster barriers.  FP64 has few lanes per SM on GB300 and
// long latencies: the pivot chain is LDL^T with one reciprocal per pivot (an
// FP32 seed and one Goldschmidt step) and the square roots of all pivots come
// afterwards, in parallel.  Pivot thresholds and the shifted retry (shifted
// CholeskyQR, Fukaya et al. 2020) follow the one-CTA kernel; ctl / status
// conventions are the same.
#include <cooperative_groups.h>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "newton_device.cuh"

namespace cg = cooperative_groups;

namespace pbq {

namespace {
constexpr int kCiCtasMax = 16;
constexpr int kCiThreads = 256;   // 8 warps: the block factor's 32 live doubles per lane fit in registers
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
//
// Shared memory of a CTA: its columns of S (then R) and of T (ncol x l
// each), two buffers of one block row of R for every column (the owners
// write them into every CTA), the next diagonal block's columns (written by
// their owners into every CTA), the factored diagonal block's R_tt and T_tt,
// and the pivot thresholds.
// Factor the 16 x 16 diagonal block in Dnx with 4 warps (threads t = 0..127,
// one warp per SM sub-partition: GB300 issues FP64 at half a lane per clock
// per sub-partition, so one warp alone would serialise the updates).  The
// augmented block [S_tt | I] (16 x 32, in W) is eliminated by LDL^T row
// operations: thread t owns column t % 32 (0..15 of S, 16..31 of I) in rows
// t / 32 + 4r, r = 0..3.  Pivot p: warp 0 forms 1/d_p (an FP32 seed and one
// Goldschmidt step) and the multipliers S[p][i] / d_p; after a 128-thread
// barrier every thread updates its rows below p (row i -= multiplier_i row p;
// S only on and above the diagonal), and a second barrier publishes row p + 1.  The S part ends as D U and the I
// part as L^{-1} = U^{-T}, so R_tt = D^{1/2} U and T_tt = D^{-1/2} L^{-1}.
// No branches on the data: the pivots are checked after the elimination, and
// a failed one (not above its threshold, or not finite) is recorded and the
// block discarded.  Rows and columns past the
// block's width nb are padded with identity.  Not inlined: inlined at both
// call sites, its row array was given a stack frame.
__device__ __noinline__ void chol_block16(double* __restrict__ W, const double* __restrict__ Dnx,
                                          const double* __restrict__ thr, int a0, int nb, double* __restrict__ Rtt,
                                          double* __restrict__ Ttt, int* s_fail, int t) {
    const int c = t & 31, w = t >> 5;
    const bool idl = c >= kCiNb;
    double v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = w + 4 * r;
        double x;
        if (idl) x = (i == c - kCiNb) ? 1.0 : 0.0;
        else if (c < nb) x = (i <= c) ? Dnx[c * kCiNb + i] : 0.0;
        else x = (i == c) ? 1.0 : 0.0;
        v[r] = x;
        W[i * 32 + c] = x;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    double* Mv = W + kCiNb * 32;   // 16: the multipliers S[p][i] / d_p of the current pivot
#pragma unroll
    for (int p = 0; p < kCiNb; ++p) {
        // warp 0: 1/d_p and the multipliers, four FP64 instructions (each FP64 warp
        // instruction occupies a sub-partition's FP64 unit for 64 cycles, so the
        // other warps do not repeat them, and the pivots are checked after the loop)
        if (w == 0) {
            const double cp = rcp_gs(W[p * 32 + p]);
            if (c > p && c < kCiNb) Mv[c] = W[p * 32 + c] * cp;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        const double rowp = W[p * 32 + c];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = w + 4 * r;
            if (i > p) {
                if (idl || c >= i) v[r] = fma(-Mv[i], rowp, v[r]);
                W[i * 32 + c] = v[r];
            }
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
    }
    // The pivots d_i = W[i][i] (row i is final after pivot i - 1), one per lane:
    // every warp forms the 16 values 1 / sqrt(d_i) in one instruction sequence,
    // and warp 0 checks them; the first failed pivot in order decides the flag
    // (2: not finite, 1: not above its threshold), as a check at each pivot would.
    const int il = c & (kCiNb - 1);
    const double dl = W[il * 33];
    const double rsl = rsqrt_nr(dl);
    if (w == 0) {
        const double th = il < nb ? thr[a0 + il] : 0.0;
        const int fp = c >= kCiNb ? 0 : (!isfinite(dl) ? 2 : (!(dl > th) ? 1 : 0));
        const unsigned bad = __ballot_sync(0xffffffffu, fp != 0);
        const int f = bad ? __shfl_sync(0xffffffffu, fp, __ffs((int)bad) - 1) : 0;
        if (c == 0) *s_fail = f;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = w + 4 * r;
        const double rs = __shfl_sync(0xffffffffu, rsl, i);
        const double di = __shfl_sync(0xffffffffu, dl, i);
        if (!idl) Rtt[i * kCiNb + c] = (i < c) ? v[r] * rs : (i == c ? di * rs : 0.0);
        else Ttt[i * kCiNb + (c - kCiNb)] = v[r] * rs;   // row i of L^{-1} scaled by 1/sqrt(d_i)
    }
}

// Own S columns of block rows [a0, a0 + 16) into Dnx of every CTA of the
// cluster (rows <= column; the rest 0).
__device__ __forceinline__ void push_diag16(cg::cluster_group& cluster, const double* __restrict__ Sown, double* Dnx,
                                            int l, int ncol, int C, int rank, int a0, int tid, int nth) {
    const int a1 = min(l, a0 + kCiNb);
    for (int e = tid; e < ncol * kCiNb; e += nth) {
        const int jl = e / kCiNb, i = e - jl * kCiNb, j = jl * C + rank;
        if (j < a0 || j >= a1) continue;
        const double v = (a0 + i <= j) ? Sown[(int64_t)jl * l + a0 + i] : 0.0;
        for (int r = 0; r < C; ++r) cluster.map_shared_rank(Dnx, r)[(j - a0) * kCiNb + i] = v;
    }
}

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
    double* Rbuf = Town + (int64_t)ncol * l;             // 2 x 16 x l: block row of R, by block parity
    double* Dnx = Rbuf + (int64_t)2 * kCiNb * l;         // 16 x 16: next diagonal block, [column][row]
    double* Rtt = Dnx + kCiNb * kCiNb;                   // 16 x 16: R_tt, [row][column]
    double* Ttt = Rtt + kCiNb * kCiNb;                   // 16 x 16: T_tt = R_tt^{-T}, [row][column]
    double* Wfb = Ttt + kCiNb * kCiNb;                   // 16 x 32 + 16: the block factor's rows, multipliers
    double* thr = Wfb + kCiNb * 32 + kCiNb;              // l: pivot thresholds
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
        // the shifted retry (attempt 1, or want 1 in block mode) only asks for d > 0
        for (int i = tid; i < l; i += nth)
            thr[i] = (attempt == 0 && !(kBlock && want == 1))
                         ? tau * (kBlock ? gdiag[(int64_t)i * (ld + 1)] : G[(int64_t)i * l + i]) : 0.0;
        fail = 0;
        __syncthreads();
        push_diag16(cluster, Sown, Dnx, l, ncol, C, rank, 0, tid, nth);
        cluster.sync();                         // Dnx holds diagonal block 0 everywhere
        if (warp < 4) chol_block16(Wfb, Dnx, thr, 0, min(l, kCiNb), Rtt, Ttt, &s_fail, tid);
        __syncthreads();
        fail = s_fail;
        for (int t = 0; t < nblk && !fail; ++t) {
            const int a0 = t * kCiNb, a1 = min(l, a0 + kCiNb), nb = a1 - a0;
            const int a2 = min(l, a1 + kCiNb);
            double* Rb = Rbuf + (int64_t)(t & 1) * kCiNb * l;
            // (b) block row t of R for own columns right of the block, R[t, j] = T_tt S[t, j], and
            // T[t, j] = T_tt T[t, j] for own columns left of its end; R_tt into the block's own columns
            // (at most 4 items per thread: 2 ncol 16 <= 4 x 256 for l <= 256 on 8 CTAs)
            double yv[4];
#pragma unroll
            for (int rep = 0; rep < 4; ++rep) {
                const int e = tid + rep * nth;
                const int side = e / (ncol * kCiNb), r = e - side * ncol * kCiNb;
                const int jl = r / kCiNb, k = r - jl * kCiNb, j = jl * C + rank;
                double y = 0.0;
                if (side < 2 && j < l && k < nb && (side == 0 ? j >= a1 : j < a1)) {
                    const double* x = (side == 0 ? Sown : Town) + (int64_t)jl * l + a0;
#pragma unroll
                    for (int i = 0; i < kCiNb; ++i)
                        if (i <= k) y = fma(Ttt[k * kCiNb + i], x[i], y);
                }
                yv[rep] = y;
            }
            __syncthreads();                    // every x read before any is overwritten
#pragma unroll
            for (int rep = 0; rep < 4; ++rep) {
                const int e = tid + rep * nth;
                const int side = e / (ncol * kCiNb), r = e - side * ncol * kCiNb;
                const int jl = r / kCiNb, k = r - jl * kCiNb, j = jl * C + rank;
                if (side >= 2 || j >= l || k >= nb) continue;
                if (side == 0 && j >= a1) {
                    Sown[(int64_t)jl * l + a0 + k] = yv[rep];
                    for (int rr = 0; rr < C; ++rr) cluster.map_shared_rank(Rb, rr)[(int64_t)k * l + j] = yv[rep];
                } else if (side == 0 && j >= a0) {
                    Sown[(int64_t)jl * l + a0 + k] = Rtt[k * kCiNb + (j - a0)];
                } else if (side == 1 && j < a1) {
                    Town[(int64_t)jl * l + a0 + k] = yv[rep];
                }
            }
            cluster.sync();                     // block row t of R is in every CTA's Rb
            if (a1 >= l) break;
            // (c1) own columns of block t+1: their rows [a1, j] first, then into every CTA's Dnx
            for (int e = tid; e < ncol * kCiNb; e += nth) {
                const int jl = e / kCiNb, i = a1 + (e - jl * kCiNb), j = jl * C + rank;
                if (j < a1 || j >= a2 || i > j) continue;
                double* col = Sown + (int64_t)jl * l;
                double acc = col[i];
#pragma unroll
                for (int k = 0; k < kCiNb; ++k)
                    if (k < nb) acc = fma(-Rb[(int64_t)k * l + i], col[a0 + k], acc);
                col[i] = acc;
            }
            __syncthreads();
            push_diag16(cluster, Sown, Dnx, l, ncol, C, rank, a1, tid, nth);
            cluster.sync();                     // Dnx holds diagonal block t+1 everywhere
            // (a) of block t+1 by warp 0, while the other warps run (c2): the trailing
            // updates of own columns past block t+1 and of own T columns left of a1
            if (warp < 4) chol_block16(Wfb, Dnx, thr, a1, a2 - a1, Rtt, Ttt, &s_fail, tid);
            if (warp >= 4) {
                for (int jl = warp - 4; jl < ncol; jl += nwarp - 4) {
                    const int j = jl * C + rank;
                    if (j >= l || (j >= a1 && j < a2)) continue;
                    const bool scol = j >= a2;
                    double* col = (scol ? Sown : Town) + (int64_t)jl * l;
                    double rj[kCiNb];
#pragma unroll
                    for (int k = 0; k < kCiNb; ++k) rj[k] = (k < nb) ? col[a0 + k] : 0.0;
                    const int iend = scol ? j + 1 : l;
                    for (int i = a1 + lane; i < iend; i += 32) {
                        double acc = col[i];
#pragma unroll
                        for (int k = 0; k < kCiNb; ++k) acc = fma(-Rb[(int64_t)k * l + i], rj[k], acc);
                        col[i] = acc;
                    }
                }
            }
            __syncthreads();
            fail = s_fail;                      // the same in every CTA
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
    const size_t need =
        ((size_t)2 * ncol * l + (size_t)2 * kCiNb * l + 3 * kCiNb * kCiNb + kCiNb * 33 + (size_t)l) * sizeof(double);
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

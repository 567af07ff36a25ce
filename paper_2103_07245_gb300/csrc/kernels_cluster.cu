// Cholesky of the l x l CholeskyQR Gram and Householder QR of R^T (Eq. 7) by
// a thread-block cluster (8 CTAs on 8 SMs) for large l, where one SM's FP64
// rate (2 lanes per clock on GB300) makes the one-CTA kernels the bottleneck.
#include <cooperative_groups.h>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "newton_device.cuh"

namespace cg = cooperative_groups;

namespace pbq {

namespace {
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 512;
constexpr int kCholNb = 16;   // rows per block of the blocked Cholesky
}  // namespace

// Blocked right-looking Cholesky G = R^T R by the cluster.  Blocks of 16 rows
// are dealt cyclically (block t lives in CTA t % C; each owned row is stored at
// full length l in shared memory, row a at local row (t / C) * 16 + a % 16).
// The owner of block t factors its 16 rows completely (pivots, scaling and the
// in-block updates, with block barriers only); after one cluster barrier every
// CTA copies that block row through distributed shared memory and applies the
// rank-16 update S_ab -= sum_i R_ia R_ib to its own later rows.  One cluster
// barrier per block.  Thresholds and the shifted retry follow the one-CTA kernel.
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
k_cholesky_cluster(int l, int64_t rows, const double* __restrict__ G, double* __restrict__ Rp,
                   uint32_t* __restrict__ status, int* __restrict__ ctl, int pass) {
    if (pass >= 3 && ctl[8 + (pass + 1) / 2] == 0) return;   // uniform over the cluster
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int nblk = (l + kCholNb - 1) / kCholNb;
    const int nbmax = (nblk + C - 1) / C;                    // blocks per CTA (same layout everywhere)
    extern __shared__ double smc[];
    double* S = smc;                                         // nbmax*16 rows x l
    double* Rb = S + (int64_t)nbmax * kCholNb * l;           // copy of the current block row (16 x l)
    double* dinv = Rb + (int64_t)kCholNb * l;                // 1/diag of own rows (nbmax*16)
    __shared__ int s_fail;
    __shared__ double s_shift, s_inv;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const double tau = 1e-12;
    auto lrow = [&](int a) { return ((a / kCholNb) / C) * kCholNb + (a % kCholNb); };

    if (tid == 0) { s_fail = 0; s_shift = 0.0; }
    __syncthreads();
    int shifted = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = s_shift;
        for (int t = rank; t < nblk; t += C)
            for (int r = warp; r < kCholNb; r += nwarp) {
                const int a = t * kCholNb + r;
                if (a >= l) continue;
                double* sa = S + (int64_t)lrow(a) * l;
                for (int b = a + lane; b < l; b += 32) sa[b] = G[(int64_t)a * l + b] + (a == b ? shift : 0.0);
            }
        if (tid == 0) s_fail = 0;
        __syncthreads();
        // factor the 16 rows of own block t: pivots, scaling, in-block updates
        auto factor_block = [&](int t) {
            const int a0 = t * kCholNb, a1 = min(l, a0 + kCholNb);
            for (int i = a0; i < a1; ++i) {
                double* si = S + (int64_t)lrow(i) * l;
                if (tid == 0) {
                    const double d = si[i];
                    const double thr = (attempt == 0) ? tau * G[(int64_t)i * l + i] : 0.0;
                    const int f = !isfinite(d) ? 2 : (!(d > thr) ? 1 : 0);
                    if (f) s_fail = f;
                    else {
                        const double rr = sqrt(d);
                        si[i] = rr;
                        s_inv = 1.0 / rr;
                        dinv[lrow(i)] = s_inv;
                    }
                }
                __syncthreads();
                if (s_fail) return;
                const double inv = s_inv;
                for (int c = i + 1 + tid; c < l; c += nth) si[c] *= inv;
                __syncthreads();
                for (int a = i + 1 + warp; a < a1; a += nwarp) {
                    double* sa = S + (int64_t)lrow(a) * l;
                    const double ria = si[a];
                    for (int b = a + lane; b < l; b += 32) sa[b] -= ria * si[b];
                }
                __syncthreads();
            }
        };
        if (rank == 0) factor_block(0);
        cluster.sync();
        int fail = 0;
        for (int t = 0; t < nblk; ++t) {
            const int owner = t % C;
            fail = *cluster.map_shared_rank(&s_fail, owner);
            if (fail) break;
            const int a0 = t * kCholNb, a1 = min(l, a0 + kCholNb), nb = a1 - a0;
            // copy block row t (rows a0..a1-1, columns >= a0) from its owner
            const double* orows = cluster.map_shared_rank(S, owner) + (int64_t)((t / C) * kCholNb) * l;
            for (int e = tid; e < nb * (l - a0); e += nth) {
                const int r = e / (l - a0), b = a0 + e % (l - a0);
                Rb[(int64_t)r * l + b] = orows[(int64_t)r * l + b];
            }
            __syncthreads();
            // rank-nb update of own rows a >= a1
            for (int u = rank; u < nblk; u += C)
                for (int r = warp; r < kCholNb; r += nwarp) {
                    const int a = u * kCholNb + r;
                    if (a < a1 || a >= l) continue;
                    double* sa = S + (int64_t)lrow(a) * l;
                    double ra[kCholNb];
#pragma unroll
                    for (int i = 0; i < kCholNb; ++i) ra[i] = (i < nb) ? Rb[(int64_t)i * l + a] : 0.0;
                    for (int b = a + lane; b < l; b += 32) {
                        double acc = sa[b];
#pragma unroll
                        for (int i = 0; i < kCholNb; ++i)
                            if (i < nb) acc -= ra[i] * Rb[(int64_t)i * l + b];
                        sa[b] = acc;
                    }
                }
            __syncthreads();
            if (t + 1 < nblk && (t + 1) % C == rank) factor_block(t + 1);
            cluster.sync();
        }
        __syncthreads();
        if (!fail) break;
        if (fail == 2 || attempt == 1) {
            if (rank == 0 && tid == 0) atomicOr(status, fail == 2 ? kStNonFinite : kStBreakdown);
            for (int t = rank; t < nblk; t += C)
                for (int r = warp; r < kCholNb; r += nwarp) {
                    const int a = t * kCholNb + r;
                    if (a >= l) continue;
                    double* sa = S + (int64_t)lrow(a) * l;
                    for (int b = a + lane; b < l; b += 32) sa[b] = (a == b) ? 1.0 : 0.0;
                    if (lane == 0) dinv[lrow(a)] = 1.0;
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
        cluster.sync();   // every CTA has read the failing owner's flag before it is reset
    }
    // own rows to the global packed layout (index a(2l - a + 1)/2 + (b - a)) and 1/diag
    const int64_t P = (int64_t)l * (l + 1) / 2;
    for (int t = rank; t < nblk; t += C)
        for (int r = warp; r < kCholNb; r += nwarp) {
            const int a = t * kCholNb + r;
            if (a >= l) continue;
            const double* sa = S + (int64_t)lrow(a) * l;
            const int64_t ga = (int64_t)a * (2 * l - a + 1) / 2 - a;
            for (int b = a + lane; b < l; b += 32) Rp[ga + b] = sa[b];
            if (lane == 0) Rp[P + a] = dinv[lrow(a)];
        }
    if (rank == 0 && tid == 0) {
        ctl[pass] = shifted;
        if ((pass & 1) == 0) ctl[8 + pass / 2 + 1] = (ctl[pass - 1] | ctl[pass]) ? 1 : 0;
        if (shifted) atomicOr(status, kStShifted);
    }
    cluster.sync();   // no CTA leaves while another may still read its shared memory
}

static size_t chol_cluster_smem(int l) {
    const int nblk = (l + kCholNb - 1) / kCholNb;
    const int nbmax = (nblk + kClusterCtas - 1) / kClusterCtas;
    return ((size_t)nbmax * kCholNb * l + (size_t)kCholNb * l + (size_t)nbmax * kCholNb) * sizeof(double);
}

bool cholesky_cluster_fits(int l) { return l > 64 && chol_cluster_smem(l) <= 200 * 1024; }

cudaError_t launch_cholesky_cluster(int l, int64_t rows, const double* G, double* Rp, uint32_t* status, int* ctl,
                                    int pass, cudaStream_t s) {
    const size_t smem = chol_cluster_smem(l);
    cudaError_t e = func_smem_attr((const void*)k_cholesky_cluster, smem);
    if (e != cudaSuccess) return e;
    k_cholesky_cluster<<<kClusterCtas, kClusterThreads, smem, s>>>(l, rows, G, Rp, status, ctl, pass);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Householder QR of W = R^T (Eq. 7) by an 8-CTA cluster, for large l.
// Columns of W (rows of Wt = R) are dealt cyclically: column c lives in CTA
// c % C.  Step j: the owner of column j has already formed reflector v_j (and
// alpha_j); every CTA copies v_j through distributed shared memory and applies
// H_j to its columns c > j; the owner of column j + 1 applies H_j to it first
// and forms v_{j+1} before the step's cluster barrier.  Ptil = H_0 ... H_{l-1}
// [I] needs no barriers: every reflector is final, each CTA forms its own
// columns.  Same arithmetic and sign convention as the one-CTA kernel.
// ---------------------------------------------------------------------------
namespace {
constexpr int kQrThreads = 512;
}

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kQrThreads)
k_small_qr_cluster(int l, const double* __restrict__ R, double* __restrict__ L, double* __restrict__ Ptil) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    extern __shared__ double smq[];
    const int nloc = (l - rank + C - 1) / C;
    const int nmax = (l + C - 1) / C;             // same layout in every CTA: remote pointers map 1:1
    double* Wt = smq;                             // own rows of Wt (= own columns of W), nloc x l
    double* V = Wt + (int64_t)nmax * l;           // reflectors owned here (row lj = v_j, entries >= j)
    double* vb = V + (int64_t)nmax * l;           // local copy of the current reflector (l)
    double* sgall = vb + l;                       // signs of diag(Rtil), all l
    __shared__ double tvv_own[kMaxEll], sg_own[kMaxEll];
    __shared__ double s_t2;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;

    for (int lc = warp; lc < nloc; lc += nwarp) {
        const int c = lc * C + rank;
        for (int i = lane; i < l; i += 32) {
            Wt[(int64_t)lc * l + i] = (i >= c) ? R[(int64_t)c * l + i] : 0.0;
            V[(int64_t)lc * l + i] = 0.0;
        }
    }
    __syncthreads();
    // form reflector j from own column j (warp 0 only)
    auto form = [&](int j) {
        const int lj = j / C;
        double* wj = Wt + (int64_t)lj * l;
        double* vj = V + (int64_t)lj * l;
        double t = 0.0;
        for (int i = j + 1 + lane; i < l; i += 32) t += wj[i] * wj[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        double alpha = 0.0, t2 = 0.0;
        if (lane == 0) {
            const double x0 = wj[j];
            const double s2 = x0 * x0 + t;
            if (s2 != 0.0) {
                const double nrm = s2 * rsqrt_nr(s2);
                alpha = (x0 >= 0.0) ? -nrm : nrm;
                const double v0 = x0 - alpha;
                vj[j] = v0;
                t2 = 2.0 * rcp_nr(v0 * v0 + t);
            }
            tvv_own[lj] = t2;
        }
        t2 = __shfl_sync(0xffffffffu, t2, 0);
        alpha = __shfl_sync(0xffffffffu, alpha, 0);
        for (int i = j + 1 + lane; i < l; i += 32) vj[i] = wj[i];
        __syncwarp();
        if (t2 != 0.0) {
            if (lane == 0) wj[j] = alpha;
            for (int i = j + 1 + lane; i < l; i += 32) wj[i] = 0.0;
        }
        __syncwarp();
    };
    if (rank == 0 && warp == 0) form(0);
    cluster.sync();
    for (int j = 0; j < l; ++j) {
        const int owner = j % C, lj = j / C;
        const double* ov = cluster.map_shared_rank(V, owner) + (int64_t)lj * l;
        for (int i = j + tid; i < l; i += nth) vb[i] = ov[i];
        if (tid == 0) s_t2 = *cluster.map_shared_rank(&tvv_own[lj], owner);
        __syncthreads();
        const double t2 = s_t2;
        if (t2 != 0.0) {
            // apply H_j to every own column c > j; the barrier below separates this
            // from forming v_{j+1} out of (own) column j + 1
            for (int lc = warp; lc < nloc; lc += nwarp) {
                const int c = lc * C + rank;
                if (c <= j) continue;
                double* wc = Wt + (int64_t)lc * l;
                double d = 0.0;
                for (int i = j + lane; i < l; i += 32) d += vb[i] * wc[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                const double f = d * t2;
                for (int i = j + lane; i < l; i += 32) wc[i] -= f * vb[i];
            }
        }
        __syncthreads();
        if (j + 1 < l && (j + 1) % C == rank && warp == 0) form(j + 1);
        cluster.sync();
    }
    // signs of diag(Rtil) (own), gathered by every CTA
    for (int lc = tid; lc < nloc; lc += nth) {
        const int c = lc * C + rank;
        sg_own[lc] = (Wt[(int64_t)lc * l + c] < 0.0) ? -1.0 : 1.0;
    }
    cluster.sync();
    for (int a = tid; a < l; a += nth) sgall[a] = *cluster.map_shared_rank(&sg_own[a / C], a % C);
    __syncthreads();
    // L[b][a] = sg[a] * W[a][b] = sg[a] * Wt[b][a] (b >= a): own rows b of L
    for (int lc = warp; lc < nloc; lc += nwarp) {
        const int b = lc * C + rank;
        for (int a = lane; a < l; a += 32) L[(int64_t)b * l + a] = (a <= b) ? sgall[a] * Wt[(int64_t)lc * l + a] : 0.0;
    }
    __syncthreads();
    // Ptil columns c owned here, formed in the storage of Wt: Pt[lc] = column c of Ptil
    double* Pt = Wt;
    for (int lc = warp; lc < nloc; lc += nwarp) {
        const int c = lc * C + rank;
        for (int i = lane; i < l; i += 32) Pt[(int64_t)lc * l + i] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = l - 1; j >= 0; --j) {
        const int owner = j % C, lj = j / C;
        const double t2 = *cluster.map_shared_rank(&tvv_own[lj], owner);
        if (t2 == 0.0) continue;   // uniform: every thread reads the same value
        const double* ov = cluster.map_shared_rank(V, owner) + (int64_t)lj * l;
        for (int i = j + tid; i < l; i += nth) vb[i] = ov[i];
        __syncthreads();
        for (int lc = warp; lc < nloc; lc += nwarp) {
            const int c = lc * C + rank;
            if (c < j) continue;   // columns c < j are still unit vectors with zeros in rows >= j
            double* pc = Pt + (int64_t)lc * l;
            double d = 0.0;
            for (int i = j + lane; i < l; i += 32) d += vb[i] * pc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const double f = d * t2;
            for (int i = j + lane; i < l; i += 32) pc[i] -= f * vb[i];
        }
        __syncthreads();
    }
    // Ptil[i][c] = sg[c] * Pt[c][i]
    for (int lc = warp; lc < nloc; lc += nwarp) {
        const int c = lc * C + rank;
        for (int i = lane; i < l; i += 32) Ptil[(int64_t)i * l + c] = sgall[c] * Pt[(int64_t)lc * l + i];
    }
    cluster.sync();   // reflectors and signs stay readable until every CTA is done
}

bool small_qr_cluster_fits(int l) {
    const int nloc = (l + kClusterCtas - 1) / kClusterCtas;
    return l > 64 && ((int64_t)2 * nloc * l + 2 * (int64_t)l) * (int64_t)sizeof(double) <= 200 * 1024;
}

cudaError_t launch_small_qr_cluster(int l, const double* R, double* L, double* Ptil, cudaStream_t s) {
    const int nloc = (l + kClusterCtas - 1) / kClusterCtas;
    const size_t smem = ((size_t)2 * nloc * l + 2 * (size_t)l) * sizeof(double);
    cudaError_t e = func_smem_attr((const void*)k_small_qr_cluster, smem);
    if (e != cudaSuccess) return e;
    k_small_qr_cluster<<<kClusterCtas, kQrThreads, smem, s>>>(l, R, L, Ptil);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq

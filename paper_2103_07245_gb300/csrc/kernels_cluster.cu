// Cholesky of the l x l CholeskyQR Gram by a thread-block cluster (8 CTAs on
// 8 SMs) for large l, where one SM's FP64 rate (2 lanes per clock on GB300)
// makes the one-CTA kernel the bottleneck.
//
// Rows of the packed upper triangle are dealt cyclically: row a lives in the
// shared memory of CTA a % C.  Step j copies the finished pivot row j from its
// owner through distributed shared memory, every CTA updates its own rows
// (S_ab -= R_ja R_jb), and the owner of row j + 1 finishes that row (pivot,
// sqrt, one reciprocal, row scaling) before the step's cluster barrier.  The
// arithmetic, thresholds and shifted retry are those of the one-CTA kernel.
#include <cooperative_groups.h>
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace cg = cooperative_groups;

namespace pbq {

namespace {
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 512;

// First packed entry of local row la (global row la*C + rank) in a CTA's store.
__device__ __forceinline__ int64_t lrow_start(int l, int C, int rank, int la) {
    return (int64_t)la * (l - rank) - (int64_t)C * la * (la - 1) / 2;
}
}  // namespace

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
k_cholesky_cluster(int l, int64_t rows, const double* __restrict__ G, double* __restrict__ Rp,
                   uint32_t* __restrict__ status, int* __restrict__ ctl, int pass) {
    if (pass >= 3 && ctl[8 + (pass + 1) / 2] == 0) return;   // uniform over the cluster
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    extern __shared__ double smc[];
    const int nloc = (l - rank + C - 1) / C;                 // rows this CTA owns
    const int64_t nstore = lrow_start(l, C, rank, nloc);
    double* S = smc;                                         // own rows, packed
    double* rowj = S + nstore;                               // copy of the current pivot row (l doubles)
    double* dinv = rowj + l;                                 // 1/diag of own rows (nloc)
    __shared__ int s_fail;
    __shared__ double s_shift;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const double tau = 1e-12;

    if (tid == 0) { s_fail = 0; s_shift = 0.0; }
    __syncthreads();
    int shifted = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = s_shift;
        for (int la = warp; la < nloc; la += nwarp) {
            const int a = la * C + rank;
            const int64_t ra = lrow_start(l, C, rank, la) - a;   // index of (a, b) is ra + b
            for (int b = a + lane; b < l; b += 32) S[ra + b] = G[(int64_t)a * l + b] + (a == b ? shift : 0.0);
        }
        if (tid == 0) s_fail = 0;
        __syncthreads();
        // finish pivot row i (owned here): lane 0 of warp 0 takes the pivot, the warp scales
        auto finish_row = [&](int i) {
            const int li = i / C;
            const int64_t ri = lrow_start(l, C, rank, li) - i;
            double inv = 0.0;
            int f = 0;
            if (lane == 0) {
                const double d = S[ri + i];
                const double thr = (attempt == 0) ? tau * G[(int64_t)i * l + i] : 0.0;
                f = !isfinite(d) ? 2 : (!(d > thr) ? 1 : 0);
                if (f) s_fail = f;
                else {
                    const double r = sqrt(d);
                    S[ri + i] = r;
                    inv = 1.0 / r;
                    dinv[li] = inv;
                }
            }
            f = __shfl_sync(0xffffffffu, f, 0);
            inv = __shfl_sync(0xffffffffu, inv, 0);
            if (!f)
                for (int c = i + 1 + lane; c < l; c += 32) S[ri + c] *= inv;
            __syncwarp();
        };
        if (rank == 0 && warp == 0) finish_row(0);
        cluster.sync();
        int fail = 0;
        for (int j = 0; j < l; ++j) {
            const int owner = j % C;
            // a failed pivot stops every CTA at the same step
            const int* ofail = cluster.map_shared_rank(&s_fail, owner);
            fail = *ofail;
            if (fail) break;
            const double* orow = cluster.map_shared_rank(S, owner) + (lrow_start(l, C, owner, j / C) - j);
            for (int b = j + tid; b < l; b += nth) rowj[b] = orow[b];
            __syncthreads();
            for (int la = warp; la < nloc; la += nwarp) {
                const int a = la * C + rank;
                if (a <= j) continue;
                const double rja = rowj[a];
                const int64_t ra = lrow_start(l, C, rank, la) - a;
                for (int b = a + lane; b < l; b += 32) S[ra + b] -= rja * rowj[b];
            }
            __syncthreads();
            if (j + 1 < l && (j + 1) % C == rank && warp == 0) finish_row(j + 1);
            cluster.sync();
        }
        __syncthreads();
        if (!fail) break;
        if (fail == 2 || attempt == 1) {
            if (rank == 0 && tid == 0) atomicOr(status, fail == 2 ? kStNonFinite : kStBreakdown);
            for (int la = warp; la < nloc; la += nwarp) {
                const int a = la * C + rank;
                const int64_t ra = lrow_start(l, C, rank, la) - a;
                for (int b = a + lane; b < l; b += 32) S[ra + b] = (a == b) ? 1.0 : 0.0;
            }
            for (int la = tid; la < nloc; la += nth) dinv[la] = 1.0;
            __syncthreads();
            break;
        }
        // shifted retry on G + s I (every CTA computes the same shift from G's diagonal)
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
    for (int la = warp; la < nloc; la += nwarp) {
        const int a = la * C + rank;
        const int64_t ra = lrow_start(l, C, rank, la) - a;
        const int64_t ga = (int64_t)a * (2 * l - a + 1) / 2 - a;
        for (int b = a + lane; b < l; b += 32) Rp[ga + b] = S[ra + b];
        if (lane == 0) Rp[P + a] = dinv[la];
    }
    if (rank == 0 && tid == 0) {
        ctl[pass] = shifted;
        if ((pass & 1) == 0) ctl[8 + pass / 2 + 1] = (ctl[pass - 1] | ctl[pass]) ? 1 : 0;
        if (shifted) atomicOr(status, kStShifted);
    }
    cluster.sync();   // no CTA leaves while another may still read its shared memory
}

bool cholesky_cluster_fits(int l) {
    const int nloc = (l + kClusterCtas - 1) / kClusterCtas;
    const int64_t store = (int64_t)nloc * l + 2 * (int64_t)l + 64;
    return l > 128 && store * (int64_t)sizeof(double) <= 200 * 1024;
}

cudaError_t launch_cholesky_cluster(int l, int64_t rows, const double* G, double* Rp, uint32_t* status, int* ctl,
                                    int pass, cudaStream_t s) {
    // rank 0 stores the most: ceil(l/C) rows of at most l entries (bounded loosely), + rowj + dinv
    const int nloc = (l + kClusterCtas - 1) / kClusterCtas;
    const size_t smem = ((size_t)nloc * l + 2 * (size_t)l + 64) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_cholesky_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
            const double nrm = sqrt(x0 * x0 + t);
            if (nrm != 0.0) {
                alpha = (x0 >= 0.0) ? -nrm : nrm;
                const double v0 = x0 - alpha;
                vj[j] = v0;
                t2 = 2.0 / (v0 * v0 + t);
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
    cudaError_t e = cudaFuncSetAttribute(k_small_qr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_small_qr_cluster<<<kClusterCtas, kQrThreads, smem, s>>>(l, R, L, Ptil);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq

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

}  // namespace pbq

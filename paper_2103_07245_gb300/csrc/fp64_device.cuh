// Device bodies of the FP64 kernels, shared by the single-matrix kernels
// (kernels_fp64.cu) and the work-list kernels of the batched path
// (kernels_batched.cu).  See kernels_fp64.cu for what each computes.
#pragma once
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "newton_device.cuh"

namespace pbq {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

// Box-Muller pairs b = b0, b0 + stride, ... of the test-matrix stream.
__device__ __forceinline__ void dev_gaussian(uint64_t seed, int64_t rows, int l, double* __restrict__ out, int64_t ld,
                                             int64_t b0, int64_t stride) {
    const int64_t total = rows * (int64_t)l;
    const int64_t npairs = (total + 1) / 2;
    const double inv53 = 1.0 / 9007199254740992.0;
    for (int64_t b = b0; b < npairs; b += stride) {
        uint32_t c[4] = {(uint32_t)b, (uint32_t)((uint64_t)b >> 32), 0u, 0u};
        philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint64_t a53 = ((uint64_t)(c[0] >> 5) << 26) | (uint64_t)(c[1] >> 6);
        const uint64_t b53 = ((uint64_t)(c[2] >> 5) << 26) | (uint64_t)(c[3] >> 6);
        const double u1 = ((double)a53 + 1.0) * inv53;
        const double u2 = (double)b53 * inv53;
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const int64_t t0 = 2 * b;
        out[(t0 / l) * ld + (t0 % l)] = rad * cs;
        if (t0 + 1 < total) out[((t0 + 1) / l) * ld + ((t0 + 1) % l)] = rad * sn;
    }
}

// One 64 x 16*TN tile of C = op(A) B over the contraction range [kbeg, kend),
// written to Cb (the tile's rows m0.., leading dimension ldc).  256 threads.
template <int TN, bool TA>
__device__ __forceinline__ void dev_dgemm_tile(int64_t M, int N, const double* __restrict__ A, int64_t lda,
                                               const double* __restrict__ B, int64_t ldb, double* __restrict__ Cb,
                                               int64_t ldc, int64_t m0, int64_t kbeg, int64_t kend) {
    constexpr int BM = kGemmBM, BK = kGemmBK, BN = 16 * TN;
    __shared__ double As[BK][BM];
    __shared__ double Bs[BK][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    double acc[4][TN];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = 0.0;

    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = tid + 256 * i;
            int r, kk;
            if (!TA) { r = idx >> 4; kk = idx & 15; }
            else     { kk = idx >> 6; r = idx & 63; }
            const int64_t gm = m0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < kend) v = TA ? A[gk * lda + gm] : A[gm * lda + gk];
            As[kk][r] = v;
        }
        for (int idx = tid; idx < BK * BN; idx += 256) {
            const int kk = idx / BN, c = idx - kk * BN;
            const int64_t gk = k0 + kk;
            Bs[kk][c] = (c < N && gk < kend) ? B[gk * ldb + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[TN];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < TN; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t gm = m0 + ty * 4 + r;
        if (gm >= M) continue;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int col = tx + 16 * c;
            if (col < N) Cb[gm * ldc + col] = acc[r][c];
        }
    }
}

__device__ __forceinline__ int64_t pidx(int l, int a, int b) {
    return (int64_t)a * (2 * l - a + 1) / 2 + (b - a);
}

// Cholesky of one l x l Gram by the whole CTA (sm: packed triangle + 2l doubles).
__device__ __forceinline__ void dev_cholesky(int l, int64_t rows, const double* __restrict__ G, double* __restrict__ Rp,
                                             uint32_t* __restrict__ status, int* __restrict__ ctl, int pass,
                                             double* sm) {
    if (pass >= 3 && ctl[8 + (pass + 1) / 2] == 0) return;
    const int64_t P = (int64_t)l * (l + 1) / 2;
    double* S = sm;
    double* dg0 = sm + P;
    double* dinv = dg0 + l;
    __shared__ int s_fail;
    __shared__ double s_shift;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const double tau = 1e-12;

    for (int j = tid; j < l; j += nth) dg0[j] = G[(int64_t)j * l + j];
    if (tid == 0) { s_shift = 0.0; s_fail = 0; }
    __syncthreads();

    int shifted = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double shift = s_shift;
        for (int a = warp; a < l; a += nwarp)
            for (int b = a + lane; b < l; b += 32)
                S[pidx(l, a, b)] = G[(int64_t)a * l + b] + (a == b ? shift : 0.0);
        if (tid == 0) s_fail = 0;
        __syncthreads();
        // right-looking, one barrier per column.  Warp 0 owns row j + 1 of the
        // update of step j: right after updating it, its lane 0 takes the pivot
        // (checks it, sqrt and one reciprocal) and the warp scales the row, so
        // the next step starts from a finished row and all scalar FP64 work
        // runs on one thread (GB300 issues 2 FP64 lanes per SM per clock).
        auto pivot_row = [&](int i) {   // warp 0 only, row i already updated
            double inv = 0.0;
            int f = 0;
            if (lane == 0) {
                const double d = S[pidx(l, i, i)];
                const double thr = (attempt == 0) ? tau * dg0[i] : 0.0;
                f = !isfinite(d) ? 2 : (!(d > thr) ? 1 : 0);
                if (f) s_fail = f;
                else {
                    inv = rsqrt_nr(d);   // no FP64 square root or division on the pivot chain
                    S[pidx(l, i, i)] = d * inv;
                    dinv[i] = inv;
                }
            }
            f = __shfl_sync(0xffffffffu, f, 0);
            inv = __shfl_sync(0xffffffffu, inv, 0);
            if (!f) {
                const int64_t ri = pidx(l, i, 0);
                for (int c = i + 1 + lane; c < l; c += 32) S[ri + c] *= inv;
            }
            __syncwarp();
        };
        if (warp == 0) pivot_row(0);
        __syncthreads();
        for (int j = 0; j < l; ++j) {
            if (s_fail) break;   // uniform: read after a barrier
            const int64_t rj = pidx(l, j, 0);
            for (int a = j + 1 + warp; a < l; a += nwarp) {
                const double rja = S[rj + a];
                const int64_t ra = pidx(l, a, 0);
                for (int b = a + lane; b < l; b += 32) S[ra + b] -= rja * S[rj + b];
                if (a == j + 1) {   // only warp 0 reaches this row
                    __syncwarp();
                    pivot_row(a);
                }
            }
            __syncthreads();
        }
        const int fail = s_fail;
        __syncthreads();
        if (!fail) break;
        if (fail == 2 || attempt == 1) {
            if (tid == 0) atomicOr(status, fail == 2 ? kStNonFinite : kStBreakdown);
            // leave a finite identity factor so later kernels stay finite
            for (int a = warp; a < l; a += nwarp)
                for (int b = a + lane; b < l; b += 32) S[pidx(l, a, b)] = (a == b) ? 1.0 : 0.0;
            for (int j = tid; j < l; j += nth) dinv[j] = 1.0;
            __syncthreads();
            break;
        }
        // shifted retry: G + s I, s = 11 (rows*l + l(l+1)) u tr(G)  (u = 2^-53)
        if (tid == 0) {
            double tr = 0.0;
            for (int j = 0; j < l; ++j) tr += dg0[j];
            double sh = 11.0 * ((double)rows * l + (double)l * (l + 1)) * 1.1102230246251565e-16 * tr;
            if (!(sh > 0.0) || !isfinite(sh)) sh = 1.0;  // all-zero panel: any factor will do
            s_shift = sh;
        }
        shifted = 1;
        __syncthreads();
    }
    for (int64_t e = tid; e < P; e += nth) Rp[e] = S[e];
    for (int j = tid; j < l; j += nth) Rp[P + j] = dinv[j];
    if (tid == 0) {
        ctl[pass] = shifted;
        if ((pass & 1) == 0) ctl[8 + pass / 2 + 1] = (ctl[pass - 1] | ctl[pass]) ? 1 : 0;
        if (shifted) atomicOr(status, kStShifted);
    }
}

// Y = X R^{-1} for rows r_first, r_first + r_step, ... < r_end, one warp per
// row; sR holds R packed + 1/diag (already in shared memory) in type T, the
// arithmetic type (double, or float for the mixed modes).
template <int U, typename T>
__device__ __forceinline__ void dev_trsm_rows(int l, const T* __restrict__ sR, const double* __restrict__ X,
                                              int64_t ldx, double* __restrict__ Y, int64_t ldy, int64_t r_first,
                                              int64_t r_end, int64_t r_step) {
    const int64_t P = (int64_t)l * (l + 1) / 2;
    const T* dinv = sR + P;
    const int lane = threadIdx.x & 31;
    for (int64_t r = r_first; r < r_end; r += r_step) {
        T x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = lane + 32 * u;
            x[u] = (c < l) ? (T)X[r * ldx + c] : (T)0;
        }
#pragma unroll
        for (int u0 = 0; u0 < U; ++u0) {
            for (int tt = 0; tt < 32; ++tt) {
                const int t = 32 * u0 + tt;
                if (t >= l) break;
                if (lane == tt) x[u0] *= dinv[t];   // only the owner lane forms y_t
                const T y = __shfl_sync(0xffffffffu, x[u0], tt);
                const int64_t rt = pidx(l, t, 0);
#pragma unroll
                for (int u = u0; u < U; ++u) {
                    const int c = lane + 32 * u;
                    if (c > t && c < l) x[u] -= y * sR[rt + c];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = lane + 32 * u;
            if (c < l) Y[r * ldy + c] = (double)x[u];
        }
    }
}

// Householder QR of W = R^T (Eq. 7) by the whole CTA.  The factor is stored
// transposed (Wt = R, so a column of W is a contiguous row of Wt); reflector j
// (entries i >= j) is row j of V.  Rtil = upper(W) with signs fixed to
// diag >= 0, L = Rtil^T, Ptil = H_0 ... H_{l-1} [I] with the matching column
// signs.  Wt and V (2 l^2 doubles) live in sm when given, else in work; Ptil
// is formed in the storage of Wt once L has been written.
__device__ __forceinline__ void dev_small_qr(int l, const double* __restrict__ R, double* __restrict__ L,
                                             double* __restrict__ Ptil, double* __restrict__ work, double* sm) {
    double* Wt = sm ? sm : work;
    double* V = Wt + (int64_t)l * l;
    double* Pt = Wt;
    __shared__ double vv[kMaxEll], sg[kMaxEll], tvv[kMaxEll];   // tvv = 2 / vv (0 for no reflector)
    __shared__ double s_alpha;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const int64_t ll = (int64_t)l * l;
    for (int64_t e = tid; e < ll; e += nth) {
        const int c = (int)(e / l), i = (int)(e - (int64_t)c * l);
        Wt[e] = (i >= c) ? R[e] : 0.0;
        V[e] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < l; ++j) {
        double* wj = Wt + (int64_t)j * l;
        if (warp == 0) {
            double t = 0.0;
            for (int i = j + 1 + lane; i < l; i += 32) t += wj[i] * wj[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) {
                const double x0 = wj[j];
                const double nrm = sqrt(x0 * x0 + t);
                if (nrm == 0.0) { vv[j] = 0.0; tvv[j] = 0.0; s_alpha = 0.0; }
                else {
                    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
                    const double v0 = x0 - alpha;
                    V[(int64_t)j * l + j] = v0;
                    vv[j] = v0 * v0 + t;
                    tvv[j] = 2.0 / vv[j];
                    s_alpha = alpha;
                }
            }
        }
        __syncthreads();
        double* vj = V + (int64_t)j * l;
        for (int i = j + 1 + tid; i < l; i += nth) vj[i] = wj[i];
        __syncthreads();
        const double vvj = vv[j], t2 = tvv[j];
        if (vvj != 0.0) {
            for (int c = j + 1 + warp; c < l; c += nwarp) {
                double* wc = Wt + (int64_t)c * l;
                double d = 0.0;
                for (int i = j + lane; i < l; i += 32) d += vj[i] * wc[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                const double f = d * t2;
                for (int i = j + lane; i < l; i += 32) wc[i] -= f * vj[i];
            }
            if (tid == 0) wj[j] = s_alpha;
            for (int i = j + 1 + tid; i < l; i += nth) wj[i] = 0.0;
        }
        __syncthreads();
    }
    for (int j = tid; j < l; j += nth) sg[j] = (Wt[(int64_t)j * l + j] < 0.0) ? -1.0 : 1.0;
    __syncthreads();
    // L[b][a] = Rtil[a][b] = sg[a] * W[a][b] = sg[a] * Wt[b][a]  (b >= a)
    for (int64_t e = tid; e < ll; e += nth) {
        const int b = (int)(e / l), a = (int)(e - (int64_t)b * l);
        L[e] = (b >= a) ? sg[a] * Wt[e] : 0.0;
    }
    __syncthreads();
    // Ptil = H_0 ... H_{l-1} [I] in the storage of Wt: columns c < j are
    // untouched unit vectors at step j
    for (int64_t e = tid; e < ll; e += nth) {
        const int c = (int)(e / l), i = (int)(e - (int64_t)c * l);
        Pt[e] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = l - 1; j >= 0; --j) {
        const double vvj = vv[j], t2 = tvv[j];
        if (vvj != 0.0) {
            const double* vj = V + (int64_t)j * l;
            for (int c = j + warp; c < l; c += nwarp) {
                double* pc = Pt + (int64_t)c * l;
                double d = 0.0;
                for (int i = j + lane; i < l; i += 32) d += vj[i] * pc[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                const double f = d * t2;
                for (int i = j + lane; i < l; i += 32) pc[i] -= f * vj[i];
            }
        }
        __syncthreads();
    }
    // Ptil[i][c] = sg[c] * Pt[c][i]
    for (int64_t e = tid; e < ll; e += nth) {
        const int i = (int)(e / l), c = (int)(e - (int64_t)i * l);
        Ptil[e] = sg[c] * Pt[(int64_t)c * l + i];
    }
}

}  // namespace pbq

// The learned (q, p) proposer: features from the L-values of a cheap q = 0
// sketch, and a small MLP 32 -> 128 -> 128 -> (5 + 3) with GELU, trained and
// evaluated by these kernels.
//
// Arithmetic: every linear layer rounds its operands to BF16 and multiplies on
// the tensor cores (mma.sync m16n8k16, FP32 accumulation); biases, GELU,
// softmax / cross-entropy and AdamW run in FP32 on FP32 master weights.
#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "mlp_internal.h"

namespace pbq {

// ---------------------------------------------------------------------------
// C (M x N, FP32, ldc) = alpha * sum_k A(m,k) B(k,n) (+ beta * C), operands in
// FP32 memory addressed by (row stride, column stride), rounded to BF16.
// 128 threads = 2 x 2 warps, warp tile 32 x 32 = 2 x 4 mma tiles of 16 x 8.
// ---------------------------------------------------------------------------
constexpr int kMmBM = 64, kMmBN = 64, kMmBK = 16;

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(128)
k_mm_bf16(int M, int N, int K, const float* __restrict__ A, int64_t sam, int64_t sak, const float* __restrict__ B,
          int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t ldc, int accumulate) {
    __shared__ __nv_bfloat16 As[kMmBM][kMmBK + 8];
    __shared__ __nv_bfloat16 Bs[kMmBK][kMmBN + 8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t4 = lane & 3;
    const int m0 = blockIdx.y * kMmBM, n0 = blockIdx.x * kMmBN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    for (int k0 = 0; k0 < K; k0 += kMmBK) {
        for (int e = tid; e < kMmBM * kMmBK; e += 128) {
            const int r = e / kMmBK, kk = e - r * kMmBK;
            const int gm = m0 + r, gk = k0 + kk;
            As[r][kk] = __float2bfloat16_rn((gm < M && gk < K) ? A[(int64_t)gm * sam + (int64_t)gk * sak] : 0.f);
        }
        for (int e = tid; e < kMmBK * kMmBN; e += 128) {
            const int kk = e / kMmBN, cc = e - kk * kMmBN;
            const int gk = k0 + kk, gn = n0 + cc;
            Bs[kk][cc] = __float2bfloat16_rn((gk < K && gn < N) ? B[(int64_t)gk * sbk + (int64_t)gn * sbn] : 0.f);
        }
        __syncthreads();
        uint32_t af[2][4], bf[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm + i * 16 + g;
            af[i][0] = pack_bf16(As[r][t4 * 2], As[r][t4 * 2 + 1]);
            af[i][1] = pack_bf16(As[r + 8][t4 * 2], As[r + 8][t4 * 2 + 1]);
            af[i][2] = pack_bf16(As[r][t4 * 2 + 8], As[r][t4 * 2 + 9]);
            af[i][3] = pack_bf16(As[r + 8][t4 * 2 + 8], As[r + 8][t4 * 2 + 9]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cidx = wn + j * 8 + g;
            bf[j][0] = pack_bf16(Bs[t4 * 2][cidx], Bs[t4 * 2 + 1][cidx]);
            bf[j][1] = pack_bf16(Bs[t4 * 2 + 8][cidx], Bs[t4 * 2 + 9][cidx]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};\n"
                    : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                    : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int gm = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int gn = n0 + wn + j * 8 + t4 * 2 + (r & 1);
                if (gm < M && gn < N) {
                    float* c = C + (int64_t)gm * ldc + gn;
                    *c = accumulate ? *c + acc[i][j][r] : acc[i][j][r];
                }
            }
}

cudaError_t launch_mm_bf16(int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbk,
                           int64_t sbn, float* C, int64_t ldc, int accumulate, cudaStream_t s) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + kMmBN - 1) / kMmBN), (unsigned)((M + kMmBM - 1) / kMmBM));
    k_mm_bf16<<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, accumulate);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Elementwise pieces.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    const float cdf = 0.5f * (1.f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

// Z[b][j] += bias[j]; when act: pre[b][j] = Z, Z = gelu(Z).
__global__ void k_bias_act(int Bn, int N, float* __restrict__ Z, const float* __restrict__ bias, float* __restrict__ pre,
                           int act) {
    const int64_t total = (int64_t)Bn * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e % N);
        const float z = Z[e] + bias[j];
        if (act) { pre[e] = z; Z[e] = gelu(z); }
        else Z[e] = z;
    }
}

// dZ = dH * gelu'(pre)
__global__ void k_gelu_back(int64_t total, const float* __restrict__ dH, const float* __restrict__ pre, float* __restrict__ dZ) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        dZ[e] = dH[e] * gelu_grad(pre[e]);
}

// Cross-entropy of both heads (logits[:, 0:5] for q, [:, 5:8] for p), mean over
// the batch; dlogits and per-sample losses (summed by k_colsum into loss).
__global__ void k_ce_grad(int Bn, const float* __restrict__ logits, const int* __restrict__ yq,
                          const int* __restrict__ yp, float* __restrict__ dlog, float* __restrict__ lossv) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bn) return;
    const float* z = logits + (int64_t)b * kMlpOut;
    float* d = dlog + (int64_t)b * kMlpOut;
    float loss = 0.f;
    const int heads[2][2] = {{0, kMlpQ}, {kMlpQ, kMlpQ + kMlpP}};
    const int ys[2] = {yq[b], yp[b]};
    for (int h = 0; h < 2; ++h) {
        const int a = heads[h][0], e = heads[h][1];
        float mx = z[a];
        for (int j = a + 1; j < e; ++j) mx = fmaxf(mx, z[j]);
        float se = 0.f;
        for (int j = a; j < e; ++j) se += expf(z[j] - mx);
        const float lse = mx + logf(se);
        for (int j = a; j < e; ++j) {
            const float pj = expf(z[j] - lse);
            d[j] = (pj - (j - a == ys[h] ? 1.f : 0.f)) / (float)Bn;
        }
        loss += lse - z[a + ys[h]];
    }
    lossv[b] = loss / (float)Bn;
}

// out[j] (+)= sum_b X[b][j], fixed order per column.
__global__ void k_colsum(int Bn, int N, const float* __restrict__ X, float* __restrict__ out, int accumulate) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int b = 0; b < Bn; ++b) s += X[(int64_t)b * N + j];
    out[j] = accumulate ? out[j] + s : s;
}

__global__ void k_adamw(int n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                        const float* __restrict__ g, float lr, float b1, float b2, float eps, float wd, float bc1,
                        float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] = p[i] - lr * ((mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * p[i]);
}

__global__ void k_argmax_heads(int Bn, const float* __restrict__ logits, int* __restrict__ q, int* __restrict__ p) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bn) return;
    const float* z = logits + (int64_t)b * kMlpOut;
    int bq = 0, bp = 0;
    for (int j = 1; j < kMlpQ; ++j) if (z[j] > z[bq]) bq = j;
    for (int j = 1; j < kMlpP; ++j) if (z[kMlpQ + j] > z[kMlpQ + bp]) bp = j;
    q[b] = bq;
    p[b] = bp;
}

// Uniform(-a_j, a_j) init from the Philox stream (a = 1/sqrt(fan_in) for
// weights, biases zero).
__device__ __forceinline__ uint32_t mix32(uint64_t x) {
    x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ull; x ^= x >> 33;
    return (uint32_t)x;
}
__global__ void k_mlp_init(float* __restrict__ P, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float a = 0.f;
    if (i < kMlpOffB1) a = 1.f / sqrtf((float)kMlpIn);
    else if (i >= kMlpOffW2 && i < kMlpOffB2) a = 1.f / sqrtf((float)kMlpHidden);
    else if (i >= kMlpOffW3 && i < kMlpOffB3) a = 1.f / sqrtf((float)kMlpHidden);
    const float u = (float)(mix32(seed * 0x9E3779B97F4A7C15ull + (uint64_t)i) >> 8) * (1.f / 16777216.f);
    P[i] = a * (2.f * u - 1.f);
}

// ---------------------------------------------------------------------------
// Features of one matrix from the L-values d_i = |L_ii| (i = 1..l) of a q = 0,
// l = k + 20 sketch, and m, n, k (32 floats; see the header for the list).
// ---------------------------------------------------------------------------
__global__ void k_features(int count, const double* const* __restrict__ Ls, const int* __restrict__ ls,
                           const int* __restrict__ ks, const int64_t* __restrict__ ms, const int64_t* __restrict__ ns,
                           float* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double* L = Ls[i];
    const int l = ls[i], k = ks[i];
    const double m = (double)ms[i], n = (double)ns[i];
    auto d = [&](int j) -> double {   // 1-based, clamped into [1, l]
        j = j < 1 ? 1 : (j > l ? l : j);
        const double v = fabs(L[(int64_t)(j - 1) * l + (j - 1)]);
        return v > 1e-300 ? v : 1e-300;
    };
    const double d1 = d(1);
    float* f = F + (int64_t)i * kMlpIn;
    int o = 0;
    f[o++] = (float)(log(m) / 8.0);
    f[o++] = (float)(log(n) / 8.0);
    f[o++] = (float)(log((double)k) / 4.0);
    f[o++] = (float)(k / fmin(m, n) * 10.0);
    const double fr[10] = {0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0};
    for (int t = 0; t < 10; ++t) f[o++] = (float)(log10(d((int)lround(fr[t] * k)) / d1) / 4.0);
    const int off[6] = {1, 2, 5, 10, 15, 20};
    for (int t = 0; t < 6; ++t) f[o++] = (float)(log10(d(k + off[t]) / d1) / 4.0);
    f[o++] = (float)log10(d(k) / d(k + 1));
    f[o++] = (float)log10(d(k) / d(k + 5));
    f[o++] = (float)log10(d(k) / d(k + 20));
    f[o++] = (float)log10(d((k + 1) / 2) / d(k));
    f[o++] = (float)log10(d(k + 10) / d(k + 20));
    double head = 0.0, tail = 0.0;
    for (int j = 1; j <= l; ++j) (j <= k ? head : tail) += d(j) * d(j);
    f[o++] = (float)(0.5 * log10(tail / head + 1e-300) / 4.0);
    // least-squares slopes of log10 d over [k/2, k] and [k, l], times k
    for (int seg = 0; seg < 2; ++seg) {
        const int a = seg == 0 ? (k + 1) / 2 : k, b = seg == 0 ? k : l;
        double sx = 0, sy = 0, sxx = 0, sxy = 0, cnt = 0;
        for (int j = a; j <= b; ++j) {
            const double y = log10(d(j));
            sx += j; sy += y; sxx += (double)j * j; sxy += j * y; cnt += 1;
        }
        const double den = cnt * sxx - sx * sx;
        f[o++] = (float)(den > 0 ? (cnt * sxy - sx * sy) / den * k : 0.0);
    }
    f[o++] = (float)log10(d(l) / d1) / 4.0f;
    f[o++] = (float)((double)l / fmin(m, n) * 10.0);
    f[o++] = (float)(m / n - 1.0);
    f[o++] = 1.0f;   // constant input
    for (; o < kMlpIn; ++o) f[o] = 0.f;
}

// ---------------------------------------------------------------------------
// Host-side layer sequence.
// ---------------------------------------------------------------------------
static int64_t nblk(int64_t total) { int64_t b = (total + 255) / 256; return b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b); }

cudaError_t mlp_forward(const float* P, const float* X, int Bn, MlpWs& w, cudaStream_t s) {
    cudaError_t e;
    // H1 = gelu(X W1^T + b1): A = X (Bn x 32), B(k, n) = W1[n][k]
    if ((e = launch_mm_bf16(Bn, kMlpHidden, kMlpIn, X, kMlpIn, 1, P + kMlpOffW1, 1, kMlpIn, w.H1, kMlpHidden, 0, s))) return e;
    k_bias_act<<<(unsigned)nblk((int64_t)Bn * kMlpHidden), 256, 0, s>>>(Bn, kMlpHidden, w.H1, P + kMlpOffB1, w.Z1, 1);
    if ((e = launch_mm_bf16(Bn, kMlpHidden, kMlpHidden, w.H1, kMlpHidden, 1, P + kMlpOffW2, 1, kMlpHidden, w.H2, kMlpHidden, 0, s))) return e;
    k_bias_act<<<(unsigned)nblk((int64_t)Bn * kMlpHidden), 256, 0, s>>>(Bn, kMlpHidden, w.H2, P + kMlpOffB2, w.Z2, 1);
    if ((e = launch_mm_bf16(Bn, kMlpOut, kMlpHidden, w.H2, kMlpHidden, 1, P + kMlpOffW3, 1, kMlpHidden, w.O, kMlpOut, 0, s))) return e;
    k_bias_act<<<(unsigned)nblk((int64_t)Bn * kMlpOut), 256, 0, s>>>(Bn, kMlpOut, w.O, P + kMlpOffB3, nullptr, 0);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t mlp_backward(const float* P, const float* X, const int* yq, const int* yp, int Bn, MlpWs& w, float* G,
                         float* loss, cudaStream_t s) {
    cudaError_t e;
    k_ce_grad<<<(Bn + 255) / 256, 256, 0, s>>>(Bn, w.O, yq, yp, w.dO, w.lossv);
    k_colsum<<<1, 32, 0, s>>>(Bn, 1, w.lossv, loss, 0);
    // layer 3: dW3 = dO^T H2 (8 x 128), db3 = colsum dO, dH2 = dO W3
    if ((e = launch_mm_bf16(kMlpOut, kMlpHidden, Bn, w.dO, 1, kMlpOut, w.H2, kMlpHidden, 1, G + kMlpOffW3, kMlpHidden, 0, s))) return e;
    k_colsum<<<1, 32, 0, s>>>(Bn, kMlpOut, w.dO, G + kMlpOffB3, 0);
    if ((e = launch_mm_bf16(Bn, kMlpHidden, kMlpOut, w.dO, kMlpOut, 1, P + kMlpOffW3, kMlpHidden, 1, w.dH, kMlpHidden, 0, s))) return e;
    k_gelu_back<<<(unsigned)nblk((int64_t)Bn * kMlpHidden), 256, 0, s>>>((int64_t)Bn * kMlpHidden, w.dH, w.Z2, w.dZ);
    // layer 2
    if ((e = launch_mm_bf16(kMlpHidden, kMlpHidden, Bn, w.dZ, 1, kMlpHidden, w.H1, kMlpHidden, 1, G + kMlpOffW2, kMlpHidden, 0, s))) return e;
    k_colsum<<<(kMlpHidden + 127) / 128, 128, 0, s>>>(Bn, kMlpHidden, w.dZ, G + kMlpOffB2, 0);
    if ((e = launch_mm_bf16(Bn, kMlpHidden, kMlpHidden, w.dZ, kMlpHidden, 1, P + kMlpOffW2, kMlpHidden, 1, w.dH, kMlpHidden, 0, s))) return e;
    k_gelu_back<<<(unsigned)nblk((int64_t)Bn * kMlpHidden), 256, 0, s>>>((int64_t)Bn * kMlpHidden, w.dH, w.Z1, w.dZ);
    // layer 1
    if ((e = launch_mm_bf16(kMlpHidden, kMlpIn, Bn, w.dZ, 1, kMlpHidden, X, kMlpIn, 1, G + kMlpOffW1, kMlpIn, 0, s))) return e;
    k_colsum<<<(kMlpHidden + 127) / 128, 128, 0, s>>>(Bn, kMlpHidden, w.dZ, G + kMlpOffB1, 0);
    count_launches(9);
    return cudaGetLastError();
}

cudaError_t mlp_adamw(float* P, float* m, float* v, const float* G, int t, float lr, float b1, float b2, float eps,
                      float wd, cudaStream_t s) {
    const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
    k_adamw<<<(kMlpParams + 255) / 256, 256, 0, s>>>(kMlpParams, P, m, v, G, lr, b1, b2, eps, wd, bc1, bc2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t mlp_argmax(const float* logits, int Bn, int* q, int* p, cudaStream_t s) {
    k_argmax_heads<<<(Bn + 255) / 256, 256, 0, s>>>(Bn, logits, q, p);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t mlp_init(float* P, uint64_t seed, cudaStream_t s) {
    k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, s>>>(P, seed);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t mlp_features(int count, const double* const* Ls, const int* ls, const int* ks, const int64_t* ms,
                         const int64_t* ns, float* F, cudaStream_t s) {
    k_features<<<(count + 127) / 128, 128, 0, s>>>(count, Ls, ls, ks, ms, ns, F);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq

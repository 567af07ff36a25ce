// Internal interface of the (q, p) proposer MLP (kernels_mlp.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbq {

constexpr int kMlpIn = 32, kMlpHidden = 128, kMlpQ = 5, kMlpP = 3, kMlpOut = kMlpQ + kMlpP;
// Flat FP32 parameter vector: W1 (128 x 32), b1, W2 (128 x 128), b2, W3 (8 x 128), b3.
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpHidden * kMlpIn;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpHidden;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpHidden * kMlpHidden;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpHidden;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpOut * kMlpHidden;
constexpr int kMlpParams = kMlpOffB3 + kMlpOut;   // 21768

// Activations of one batch (all FP32, Bn rows).
struct MlpWs {
    float *H1, *Z1, *H2, *Z2, *O, *dO, *dH, *dZ, *lossv;
};
inline size_t mlp_ws_floats(int Bn) { return (size_t)Bn * (6 * kMlpHidden + 2 * kMlpOut + 1) + 64; }
inline MlpWs mlp_carve(float* base, int Bn) {
    MlpWs w;
    size_t o = 0;
    auto take = [&](size_t n) { float* p = base + o; o += (n + 15) / 16 * 16; return p; };
    w.H1 = take((size_t)Bn * kMlpHidden); w.Z1 = take((size_t)Bn * kMlpHidden);
    w.H2 = take((size_t)Bn * kMlpHidden); w.Z2 = take((size_t)Bn * kMlpHidden);
    w.O = take((size_t)Bn * kMlpOut); w.dO = take((size_t)Bn * kMlpOut);
    w.dH = take((size_t)Bn * kMlpHidden); w.dZ = take((size_t)Bn * kMlpHidden);
    w.lossv = take((size_t)Bn);
    return w;
}
inline size_t mlp_ws_bytes(int Bn) { return sizeof(float) * (mlp_ws_floats(Bn) + 16 * 16); }

cudaError_t launch_mm_bf16(int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbk,
                           int64_t sbn, float* C, int64_t ldc, int accumulate, cudaStream_t s);
cudaError_t mlp_forward(const float* P, const float* X, int Bn, MlpWs& w, cudaStream_t s);
cudaError_t mlp_backward(const float* P, const float* X, const int* yq, const int* yp, int Bn, MlpWs& w, float* G,
                         float* loss, cudaStream_t s);
cudaError_t mlp_adamw(float* P, float* m, float* v, const float* G, int t, float lr, float b1, float b2, float eps,
                      float wd, cudaStream_t s);
cudaError_t mlp_argmax(const float* logits, int Bn, int* q, int* p, cudaStream_t s);
cudaError_t mlp_init(float* P, uint64_t seed, cudaStream_t s);
cudaError_t mlp_features(int count, const double* const* Ls, const int* ls, const int* ks, const int64_t* ms,
                         const int64_t* ns, float* F, cudaStream_t s);

}  // namespace pbq

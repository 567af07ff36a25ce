// C ABI of the learned (q, p) proposer (features, MLP training and inference).
#include <cstring>
#include <vector>

#include "../../include/pbpqlp.h"
#include "internal.h"
#include "mlp_internal.h"

using namespace pbq;

namespace {
int ok(cudaError_t e) { return e == cudaSuccess ? PBPQLP_OK : PBPQLP_ECUDA; }
bool ws_ok(const void* ws, size_t have, size_t need) { return ws && have >= need && ((uintptr_t)ws & 255u) == 0; }
}  // namespace

extern "C" {

int pbpqlp_mlp_param_count(void) { return kMlpParams; }

size_t pbpqlp_mlp_workspace_bytes(int batch) { return batch < 1 ? 0 : mlp_ws_bytes(batch); }

int pbpqlp_mlp_init(float* params, uint64_t seed, void* stream) {
    if (!params) return PBPQLP_EINVAL;
    return ok(mlp_init(params, seed, (cudaStream_t)stream));
}

int pbpqlp_mlp_forward(const float* params, const float* X, int batch, float* logits, void* workspace, size_t ws_bytes,
                       void* stream) {
    if (!params || !X || !logits || batch < 1) return PBPQLP_EINVAL;
    if (!ws_ok(workspace, ws_bytes, mlp_ws_bytes(batch))) return PBPQLP_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpWs w = mlp_carve((float*)workspace, batch);
    cudaError_t e = mlp_forward(params, X, batch, w, s);
    if (e != cudaSuccess) return PBPQLP_ECUDA;
    return ok(cudaMemcpyAsync(logits, w.O, sizeof(float) * (size_t)batch * kMlpOut, cudaMemcpyDeviceToDevice, s));
}

int pbpqlp_mlp_loss_grad(const float* params, const float* X, const int* yq, const int* yp, int batch, float* grad,
                         float* loss, void* workspace, size_t ws_bytes, void* stream) {
    if (!params || !X || !yq || !yp || !grad || !loss || batch < 1) return PBPQLP_EINVAL;
    if (!ws_ok(workspace, ws_bytes, mlp_ws_bytes(batch))) return PBPQLP_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpWs w = mlp_carve((float*)workspace, batch);
    cudaError_t e = mlp_forward(params, X, batch, w, s);
    if (e != cudaSuccess) return PBPQLP_ECUDA;
    return ok(mlp_backward(params, X, yq, yp, batch, w, grad, loss, s));
}

int pbpqlp_mlp_adamw(float* params, float* m, float* v, const float* grad, int step, float lr, float beta1, float beta2,
                     float eps, float weight_decay, void* stream) {
    if (!params || !m || !v || !grad || step < 1) return PBPQLP_EINVAL;
    return ok(mlp_adamw(params, m, v, grad, step, lr, beta1, beta2, eps, weight_decay, (cudaStream_t)stream));
}

size_t pbpqlp_features_workspace_bytes(int count) {
    return count < 1 ? 0 : (size_t)count * (sizeof(void*) + 2 * sizeof(int) + 2 * sizeof(int64_t)) + 5 * 256;
}

int pbpqlp_features(int count, const double* const* L, const int* l, const int* k, const int64_t* m, const int64_t* n,
                    float* features, void* workspace, size_t ws_bytes, void* stream) {
    if (count < 1 || !L || !l || !k || !m || !n || !features) return PBPQLP_EINVAL;
    if (!ws_ok(workspace, ws_bytes, pbpqlp_features_workspace_bytes(count))) return PBPQLP_EWORKSPACE;
    for (int i = 0; i < count; ++i)
        if (!L[i] || k[i] < 2 || l[i] < k[i] + 1) return PBPQLP_EINVAL;
    // stage the small per-matrix arrays in the workspace
    std::vector<unsigned char> host(pbpqlp_features_workspace_bytes(count));
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes) {
        const size_t o = off;
        std::memcpy(host.data() + o, src, bytes);
        off = (o + bytes + 255) / 256 * 256;
        return o;
    };
    const size_t oL = put(L, sizeof(void*) * count), ol = put(l, sizeof(int) * count), ok_ = put(k, sizeof(int) * count);
    const size_t om = put(m, sizeof(int64_t) * count), on = put(n, sizeof(int64_t) * count);
    cudaStream_t s = (cudaStream_t)stream;
    char* d = (char*)workspace;
    if (cudaMemcpyAsync(d, host.data(), off, cudaMemcpyHostToDevice, s) != cudaSuccess) return PBPQLP_ECUDA;
    return ok(mlp_features(count, (const double* const*)(d + oL), (const int*)(d + ol), (const int*)(d + ok_),
                           (const int64_t*)(d + om), (const int64_t*)(d + on), features, s));
}

int pbpqlp_propose(const float* features, int count, const float* params, int* q_out, int* p_index_out,
                   void* workspace, size_t ws_bytes, void* stream) {
    if (!features || !params || !q_out || !p_index_out || count < 1) return PBPQLP_EINVAL;
    if (!ws_ok(workspace, ws_bytes, mlp_ws_bytes(count))) return PBPQLP_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    MlpWs w = mlp_carve((float*)workspace, count);
    if (mlp_forward(params, features, count, w, s) != cudaSuccess) return PBPQLP_ECUDA;
    return ok(mlp_argmax(w.O, count, q_out, p_index_out, s));
}

}  // extern "C"

// pbpqlp_factor_static: the factorization for callers that cannot allocate
// device memory.  Some callers run under a host framework that owns every
// device allocation (an inference engine's plugin, a memory-budgeted service)
// or on a path where cudaMalloc's implicit device synchronisation is not
// acceptable; they cannot provide the workspace pbpqlp_factor needs.  This
// entry point uses a fixed scratch array that is part of the library image
// instead.  Under CUDA's default lazy module loading the array is reserved on
// a GPU when the first call there looks up its address (that lookup loads
// this file's module); with CUDA_MODULE_LOADING=EAGER it is reserved when the
// library is loaded.  Either way it stays reserved until the process exits,
// so its size is kept modest and larger plans are rejected.  Callers make
// the first call per device as a warm-up, outside the path that must not
// allocate; later calls allocate nothing.
#include <mutex>

#include "../../include/pbpqlp.h"
#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[PBPQLP_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol name is only a host-side stand-in, so the real address is looked
// up once per device (with that device current) and cached.
int scratch_on_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PBPQLP_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return PBPQLP_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return PBPQLP_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PBPQLP_OK;
}

}  // namespace

extern "C" int pbpqlp_factor_static(pbpqlp_plan_t plan, const void* A, int64_t lda, int a_dtype,
                                    const double* omega, double* Qa, double* L, double* Qb) {
    if (!plan) return PBPQLP_EINVAL;
    if (pbpqlp_workspace_bytes(plan) > (size_t)PBPQLP_STATIC_SCRATCH_BYTES) return PBPQLP_EWORKSPACE;
    void* ws = nullptr;
    const int rc = scratch_on_current_device(&ws);
    if (rc != PBPQLP_OK) return rc;
    // pbpqlp_factor clears the status word and retry flags it reads; every
    // other scratch region is written before it is read.
    return pbpqlp_factor(plan, A, lda, a_dtype, ws, (size_t)PBPQLP_STATIC_SCRATCH_BYTES, omega, Qa, L, Qb);
}

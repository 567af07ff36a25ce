"""Python binding of the GB300 PbP-QLP library (argument marshalling only).

Every function here forwards to the C ABI of ``libpbpqlp.so`` (declared in
``include/pbpqlp.h``) under the same name.  Device buffers are torch CUDA
tensors (or raw integer device addresses); the CUDA stream is torch's current
stream unless one is given.  There is no CPU fallback: if the shared library
is missing the import of the binding raises.
"""
import ctypes
import os

from . import build as _build

PBPQLP_OK = 0
PBPQLP_EINVAL = 1
PBPQLP_ENOMEM = 2
PBPQLP_ECUDA = 3
PBPQLP_ENONFINITE = 4
PBPQLP_EBREAKDOWN = 5
PBPQLP_ETIMEOUT = 6
PBPQLP_EUNSUPPORTED = 7
PBPQLP_EWORKSPACE = 8

PBPQLP_MODE_FP64 = 0
PBPQLP_MODE_BF16 = 1
PBPQLP_MODE_BF16X3 = 2
PBPQLP_MODE_TF32 = 3
PBPQLP_MODE_TF32X3 = 4
PBPQLP_MODE_FP64_EMU = 5
PBPQLP_STREAM_A = 256

PBPQLP_F64 = 0
PBPQLP_F32 = 1

PBPQLP_ERR_IDENTITY = 0
PBPQLP_ERR_RESIDUAL = 1
PBPQLP_ERR_PROBES = 2

PBPQLP_TIME_PASS = 0
PBPQLP_TIME_CHOL = 1
PBPQLP_TIME_GRAM = 2
PBPQLP_TIME_SOLVE = 3
PBPQLP_TIME_SMALLQR = 4
PBPQLP_TIME_OTHER = 5
TIME_CLASSES = ("pass", "chol", "gram", "solve", "smallqr", "other")

PBPQLP_STATIC_SCRATCH_BYTES = 32 << 20

MAX_ELL = 4096          # l = k + p limit (blocked l x l steps beyond 224)

_lib = None


class PbpqlpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, strerror(status), status))


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libpbpqlp.so (optionally building it first) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libpbpqlp.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(_build.LIB)
    vp, i64, u64, sz, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
    L.pbpqlp_version.argtypes = []
    L.pbpqlp_version.restype = ci
    L.pbpqlp_strerror.argtypes = [ci]
    L.pbpqlp_strerror.restype = ctypes.c_char_p
    L.pbpqlp_plan.argtypes = [ctypes.POINTER(vp), i64, i64, ci, ci, ci, u64, ci, vp]
    L.pbpqlp_plan.restype = ci
    L.pbpqlp_plan_destroy.argtypes = [vp]
    L.pbpqlp_plan_destroy.restype = ci
    L.pbpqlp_workspace_bytes.argtypes = [vp]
    L.pbpqlp_workspace_bytes.restype = sz
    L.pbpqlp_generate_omega.argtypes = [vp, vp]
    L.pbpqlp_generate_omega.restype = ci
    L.pbpqlp_factor.argtypes = [vp, vp, i64, ci, vp, sz, vp, vp, vp, vp]
    L.pbpqlp_factor.restype = ci
    L.pbpqlp_factor_from.argtypes = [vp, vp, i64, ci, vp, sz, vp, i64, vp, vp, vp, vp]
    L.pbpqlp_factor_from.restype = ci
    L.pbpqlp_csr_workspace_bytes.argtypes = [vp, i64]
    L.pbpqlp_csr_workspace_bytes.restype = sz
    L.pbpqlp_factor_csr.argtypes = [vp, vp, vp, vp, i64, vp, sz, vp, vp, vp, vp]
    L.pbpqlp_factor_csr.restype = ci
    L.pbpqlp_sketch.argtypes = [vp, vp, i64, ci, ci, vp, i64, ci, vp, i64, vp, sz]
    L.pbpqlp_sketch.restype = ci
    L.pbpqlp_reconstruct.argtypes = [vp, vp, vp, vp, ci, vp, i64, vp, sz]
    L.pbpqlp_reconstruct.restype = ci
    L.pbpqlp_error.argtypes = [vp, vp, i64, ci, vp, vp, vp, ci, ci, ci, u64, vp, sz, ctypes.POINTER(ctypes.c_double)]
    L.pbpqlp_error.restype = ci
    L.pbpqlp_sync_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    L.pbpqlp_sync_status.restype = ci
    pvp = ctypes.POINTER(vp)
    L.pbpqlp_plan_batched.argtypes = [ctypes.POINTER(vp), ci, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(ci), ci, ci, u64, ci, vp]
    L.pbpqlp_plan_batched.restype = ci
    L.pbpqlp_batch_destroy.argtypes = [vp]
    L.pbpqlp_batch_destroy.restype = ci
    L.pbpqlp_batch_workspace_bytes.argtypes = [vp]
    L.pbpqlp_batch_workspace_bytes.restype = sz
    L.pbpqlp_factor_batched.argtypes = [vp, pvp, ctypes.POINTER(i64), ci, vp, sz, pvp, pvp, pvp]
    L.pbpqlp_factor_batched.restype = ci
    L.pbpqlp_batch_sync_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32)]
    L.pbpqlp_batch_sync_status.restype = ci
    L.pbpqlp_batch_autotune.argtypes = [vp, pvp, ctypes.POINTER(i64), ci, vp, sz, pvp, pvp, pvp, ctypes.c_char_p,
                                        ctypes.POINTER(ctypes.c_double)]
    L.pbpqlp_batch_autotune.restype = ci
    L.pbpqlp_batch_set_timing.argtypes = [vp, ci]
    L.pbpqlp_batch_set_timing.restype = ci
    L.pbpqlp_batch_read_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.pbpqlp_batch_read_timing.restype = ci
    fp = ctypes.POINTER(ctypes.c_float)
    L.pbpqlp_features_workspace_bytes.argtypes = [ci]
    L.pbpqlp_features_workspace_bytes.restype = sz
    L.pbpqlp_features.argtypes = [ci, pvp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(i64),
                                  ctypes.POINTER(i64), vp, vp, sz, vp]
    L.pbpqlp_features.restype = ci
    L.pbpqlp_mlp_param_count.argtypes = []
    L.pbpqlp_mlp_param_count.restype = ci
    L.pbpqlp_mlp_workspace_bytes.argtypes = [ci]
    L.pbpqlp_mlp_workspace_bytes.restype = sz
    L.pbpqlp_mlp_init.argtypes = [vp, u64, vp]
    L.pbpqlp_mlp_init.restype = ci
    L.pbpqlp_mlp_forward.argtypes = [vp, vp, ci, vp, vp, sz, vp]
    L.pbpqlp_mlp_forward.restype = ci
    L.pbpqlp_mlp_loss_grad.argtypes = [vp, vp, vp, vp, ci, vp, vp, vp, sz, vp]
    L.pbpqlp_mlp_loss_grad.restype = ci
    L.pbpqlp_mlp_adamw.argtypes = [vp, vp, vp, vp, ci, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, vp]
    L.pbpqlp_mlp_adamw.restype = ci
    L.pbpqlp_propose.argtypes = [vp, ci, vp, vp, vp, vp, sz, vp]
    L.pbpqlp_propose.restype = ci
    L.pbpqlp_factor_static.argtypes = [vp, vp, i64, ci, vp, vp, vp, vp]
    L.pbpqlp_factor_static.restype = ci
    L.pbpqlp_rank_revealing.argtypes = [vp, vp, ctypes.c_double, vp, vp, sz, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ci)]
    L.pbpqlp_rank_revealing.restype = ci
    L.pbpqlp_set_timing.argtypes = [vp, ci]
    L.pbpqlp_set_timing.restype = ci
    L.pbpqlp_read_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.pbpqlp_read_timing.restype = ci
    L.pbpqlp_kernel_launch_count.argtypes = []
    L.pbpqlp_kernel_launch_count.restype = ctypes.c_int64
    L.pbpqlp_set_timing_classes.argtypes = [vp, ctypes.c_uint]
    L.pbpqlp_set_timing_classes.restype = ci
    L.pbpqlp_read_timing_class.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.pbpqlp_read_timing_class.restype = ci
    L.pbpqlp_newton_check.argtypes = [vp, i64, vp, vp, vp, vp]
    L.pbpqlp_fp64_rate_probe.argtypes = [vp, ctypes.POINTER(ctypes.c_double), vp]
    L.pbpqlp_fp64_rate_probe.restype = ci
    L.pbpqlp_newton_check.restype = ci
    L.pbpqlp_oz_convert_check.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    L.pbpqlp_oz_convert_check.restype = ci
    _lib = L
    return L


def strerror(status: int) -> str:
    return load().pbpqlp_strerror(int(status)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc, where):
    if rc != PBPQLP_OK:
        raise PbpqlpError(rc, where)


# ------------------------------------------------------------------ C ABI names
def pbpqlp_version() -> int:
    return load().pbpqlp_version()


def pbpqlp_plan(m, n, k, p, q, seed, mode=PBPQLP_MODE_FP64, stream=None):
    """Create a plan; returns the opaque handle (ctypes.c_void_p)."""
    h = ctypes.c_void_p()
    _check(load().pbpqlp_plan(ctypes.byref(h), int(m), int(n), int(k), int(p), int(q),
                              int(seed) & 0xFFFFFFFFFFFFFFFF, int(mode), _stream(stream)), "pbpqlp_plan")
    return h


def pbpqlp_plan_destroy(plan):
    _check(load().pbpqlp_plan_destroy(plan), "pbpqlp_plan_destroy")


def pbpqlp_workspace_bytes(plan) -> int:
    return int(load().pbpqlp_workspace_bytes(plan))


def pbpqlp_generate_omega(plan, omega):
    _check(load().pbpqlp_generate_omega(plan, _ptr(omega)), "pbpqlp_generate_omega")


def pbpqlp_factor(plan, A, lda, a_dtype, workspace, ws_bytes, omega, Qa, L, Qb):
    _check(load().pbpqlp_factor(plan, _ptr(A), int(lda), int(a_dtype), _ptr(workspace), int(ws_bytes),
                                _ptr(omega), _ptr(Qa), _ptr(L), _ptr(Qb)), "pbpqlp_factor")


def pbpqlp_factor_from(plan, A, lda, a_dtype, workspace, ws_bytes, pbar0, ld_pbar0, pbar_out, Qa, L, Qb):
    _check(load().pbpqlp_factor_from(plan, _ptr(A), int(lda), int(a_dtype), _ptr(workspace), int(ws_bytes),
                                     _ptr(pbar0), int(ld_pbar0), _ptr(pbar_out), _ptr(Qa), _ptr(L), _ptr(Qb)),
           "pbpqlp_factor_from")


def pbpqlp_csr_workspace_bytes(plan, nnz) -> int:
    return int(load().pbpqlp_csr_workspace_bytes(plan, int(nnz)))


def pbpqlp_factor_csr(plan, rowptr, colind, values, nnz, workspace, ws_bytes, omega, Qa, L, Qb):
    _check(load().pbpqlp_factor_csr(plan, _ptr(rowptr), _ptr(colind), _ptr(values), int(nnz), _ptr(workspace),
                                    int(ws_bytes), _ptr(omega), _ptr(Qa), _ptr(L), _ptr(Qb)), "pbpqlp_factor_csr")


def pbpqlp_sketch(plan, A, lda, a_dtype, trans, Y, ldy, ncols, C, ldc, workspace, ws_bytes):
    _check(load().pbpqlp_sketch(plan, _ptr(A), int(lda), int(a_dtype), int(trans), _ptr(Y), int(ldy), int(ncols),
                                _ptr(C), int(ldc), _ptr(workspace), int(ws_bytes)), "pbpqlp_sketch")


def pbpqlp_reconstruct(plan, Qa, L, Qb, r, Ahat, ldh, workspace, ws_bytes):
    _check(load().pbpqlp_reconstruct(plan, _ptr(Qa), _ptr(L), _ptr(Qb), int(r), _ptr(Ahat), int(ldh),
                                     _ptr(workspace), int(ws_bytes)), "pbpqlp_reconstruct")


def pbpqlp_error(plan, A, lda, a_dtype, Qa, L, Qb, r, method, nprobes, probe_seed, workspace, ws_bytes) -> float:
    out = ctypes.c_double(0.0)
    _check(load().pbpqlp_error(plan, _ptr(A), int(lda), int(a_dtype), _ptr(Qa), _ptr(L), _ptr(Qb), int(r),
                               int(method), int(nprobes), int(probe_seed) & 0xFFFFFFFFFFFFFFFF,
                               _ptr(workspace), int(ws_bytes), ctypes.byref(out)), "pbpqlp_error")
    return out.value


def pbpqlp_sync_status(plan):
    """Returns (status, flags)."""
    f = ctypes.c_uint32(0)
    rc = load().pbpqlp_sync_status(plan, ctypes.byref(f))
    return rc, int(f.value)


def pbpqlp_factor_static(plan, A, lda, a_dtype, omega, Qa, L, Qb):
    """pbpqlp_factor without a workspace argument (the library's fixed device scratch)."""
    _check(load().pbpqlp_factor_static(plan, _ptr(A), int(lda), int(a_dtype), _ptr(omega), _ptr(Qa), _ptr(L),
                                       _ptr(Qb)), "pbpqlp_factor_static")


def pbpqlp_features_workspace_bytes(count) -> int:
    return int(load().pbpqlp_features_workspace_bytes(int(count)))


def pbpqlp_features(L, l, k, m, n, features, workspace, ws_bytes, stream=None):
    cnt = len(L)
    la = (ctypes.c_int * cnt)(*[int(x) for x in l])
    ka = (ctypes.c_int * cnt)(*[int(x) for x in k])
    ma = (ctypes.c_int64 * cnt)(*[int(x) for x in m])
    na = (ctypes.c_int64 * cnt)(*[int(x) for x in n])
    _check(load().pbpqlp_features(cnt, _ptr_array(L), la, ka, ma, na, _ptr(features), _ptr(workspace), int(ws_bytes),
                                  _stream(stream)), "pbpqlp_features")


def pbpqlp_mlp_param_count() -> int:
    return int(load().pbpqlp_mlp_param_count())


def pbpqlp_mlp_workspace_bytes(batch) -> int:
    return int(load().pbpqlp_mlp_workspace_bytes(int(batch)))


def pbpqlp_mlp_init(params, seed, stream=None):
    _check(load().pbpqlp_mlp_init(_ptr(params), int(seed) & 0xFFFFFFFFFFFFFFFF, _stream(stream)), "pbpqlp_mlp_init")


def pbpqlp_mlp_forward(params, X, batch, logits, workspace, ws_bytes, stream=None):
    _check(load().pbpqlp_mlp_forward(_ptr(params), _ptr(X), int(batch), _ptr(logits), _ptr(workspace), int(ws_bytes),
                                     _stream(stream)), "pbpqlp_mlp_forward")


def pbpqlp_mlp_loss_grad(params, X, yq, yp, batch, grad, loss, workspace, ws_bytes, stream=None):
    _check(load().pbpqlp_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(yq), _ptr(yp), int(batch), _ptr(grad), _ptr(loss),
                                       _ptr(workspace), int(ws_bytes), _stream(stream)), "pbpqlp_mlp_loss_grad")


def pbpqlp_mlp_adamw(params, m, v, grad, step, lr, beta1, beta2, eps, weight_decay, stream=None):
    _check(load().pbpqlp_mlp_adamw(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr), float(beta1),
                                   float(beta2), float(eps), float(weight_decay), _stream(stream)), "pbpqlp_mlp_adamw")


def pbpqlp_propose(features, count, params, q_out, p_index_out, workspace, ws_bytes, stream=None):
    _check(load().pbpqlp_propose(_ptr(features), int(count), _ptr(params), _ptr(q_out), _ptr(p_index_out),
                                 _ptr(workspace), int(ws_bytes), _stream(stream)), "pbpqlp_propose")


def pbpqlp_rank_revealing(plan, L, tol, lvalues, workspace, ws_bytes):
    """Returns (norm2 estimate |L_11|, numerical rank at tol); |L_ii| land in lvalues."""
    nrm = ctypes.c_double(0.0)
    rk = ctypes.c_int(0)
    _check(load().pbpqlp_rank_revealing(plan, _ptr(L), float(tol), _ptr(lvalues), _ptr(workspace), int(ws_bytes),
                                        ctypes.byref(nrm), ctypes.byref(rk)), "pbpqlp_rank_revealing")
    return nrm.value, int(rk.value)


def pbpqlp_set_timing(plan, enable):
    _check(load().pbpqlp_set_timing(plan, 1 if enable else 0), "pbpqlp_set_timing")


def pbpqlp_read_timing(plan):
    """Returns (milliseconds summed over timed pass kernels, number of such launches)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().pbpqlp_read_timing(plan, ctypes.byref(ms), ctypes.byref(n)), "pbpqlp_read_timing")
    return ms.value, int(n.value)


def pbpqlp_set_timing_classes(plan, mask):
    _check(load().pbpqlp_set_timing_classes(plan, int(mask)), "pbpqlp_set_timing_classes")


def pbpqlp_read_timing_class(plan, cls):
    """Returns (milliseconds summed over the timed groups of class cls, number of groups)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().pbpqlp_read_timing_class(plan, int(cls), ctypes.byref(ms), ctypes.byref(n)),
           "pbpqlp_read_timing_class")
    return ms.value, int(n.value)


def pbpqlp_kernel_launch_count() -> int:
    return int(load().pbpqlp_kernel_launch_count())


def pbpqlp_newton_check(d, n, rcp, rsqrt, rcp_gs=None, stream=None):
    """The library's Newton-refined 1/d and 1/sqrt(d), and its one-step Goldschmidt 1/d,
    for n device doubles (a diagnostic)."""
    _check(load().pbpqlp_newton_check(_ptr(d), int(n), _ptr(rcp), _ptr(rsqrt), _ptr(rcp_gs), _stream(stream)),
           "pbpqlp_newton_check")


def pbpqlp_oz_convert_check(hi, lo, e, n, fast, exact, stream=None):
    """Both forms of the digit products' exact-integer-to-FP64 conversion of
    (hi 2^28 + lo) 2^e for n device triples (a diagnostic)."""
    _check(load().pbpqlp_oz_convert_check(_ptr(hi), _ptr(lo), _ptr(e), int(n), _ptr(fast), _ptr(exact),
                                          _stream(stream)), "pbpqlp_oz_convert_check")


def pbpqlp_fp64_rate_probe(sink, stream=None) -> float:
    """Measured FP64 FMA issue rate of the current device in TFLOP/s (sink: >= 4 x SMs device doubles)."""
    out = ctypes.c_double(0.0)
    _check(load().pbpqlp_fp64_rate_probe(_ptr(sink), ctypes.byref(out), _stream(stream)), "pbpqlp_fp64_rate_probe")
    return out.value


def _ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def pbpqlp_plan_batched(m, n, k, p, q, seed, mode=PBPQLP_MODE_FP64, stream=None):
    cnt = len(m)
    h = ctypes.c_void_p()
    ma = (ctypes.c_int64 * cnt)(*[int(x) for x in m])
    na = (ctypes.c_int64 * cnt)(*[int(x) for x in n])
    ka = (ctypes.c_int * cnt)(*[int(x) for x in k])
    _check(load().pbpqlp_plan_batched(ctypes.byref(h), cnt, ma, na, ka, int(p), int(q),
                                      int(seed) & 0xFFFFFFFFFFFFFFFF, int(mode), _stream(stream)),
           "pbpqlp_plan_batched")
    return h


def pbpqlp_batch_destroy(batch):
    _check(load().pbpqlp_batch_destroy(batch), "pbpqlp_batch_destroy")


def pbpqlp_batch_workspace_bytes(batch) -> int:
    return int(load().pbpqlp_batch_workspace_bytes(batch))


def pbpqlp_factor_batched(batch, A, lda, a_dtype, workspace, ws_bytes, Qa, L, Qb):
    cnt = len(A)
    la = (ctypes.c_int64 * cnt)(*[int(x) for x in lda])
    _check(load().pbpqlp_factor_batched(batch, _ptr_array(A), la, int(a_dtype), _ptr(workspace), int(ws_bytes),
                                        _ptr_array(Qa), _ptr_array(L), _ptr_array(Qb)), "pbpqlp_factor_batched")


def pbpqlp_batch_autotune(batch, A, lda, a_dtype, workspace, ws_bytes, Qa, L, Qb, table_path=None):
    cnt = len(A)
    la = (ctypes.c_int64 * cnt)(*[int(x) for x in lda])
    best = ctypes.c_double(0.0)
    _check(load().pbpqlp_batch_autotune(batch, _ptr_array(A), la, int(a_dtype), _ptr(workspace), int(ws_bytes),
                                        _ptr_array(Qa), _ptr_array(L), _ptr_array(Qb),
                                        table_path.encode() if table_path else None, ctypes.byref(best)),
           "pbpqlp_batch_autotune")
    return best.value


def pbpqlp_batch_set_timing(batch, enable):
    _check(load().pbpqlp_batch_set_timing(batch, 1 if enable else 0), "pbpqlp_batch_set_timing")


def pbpqlp_batch_read_timing(batch):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().pbpqlp_batch_read_timing(batch, ctypes.byref(ms), ctypes.byref(n)), "pbpqlp_batch_read_timing")
    return ms.value, int(n.value)


def pbpqlp_batch_sync_status(batch, count):
    """Returns (worst status, per-matrix flag list)."""
    f = (ctypes.c_uint32 * count)()
    rc = load().pbpqlp_batch_sync_status(batch, f)
    return rc, [int(x) for x in f]


# ------------------------------------------------------- torch convenience layer
class Plan:
    """Owns a plan handle and a torch-allocated workspace for one shape."""

    def __init__(self, m, n, k, p, q, seed, mode=PBPQLP_MODE_FP64, stream=None, device="cuda"):
        import torch
        self.m, self.n, self.k, self.p, self.q, self.l = int(m), int(n), int(k), int(p), int(q), int(k) + int(p)
        self.seed, self.mode = int(seed), int(mode)
        self.handle = pbpqlp_plan(m, n, k, p, q, seed, mode, stream)
        self.ws_bytes = pbpqlp_workspace_bytes(self.handle)
        # 256-byte aligned: torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)

    def outputs(self, device="cuda"):
        import torch
        f = torch.float64
        return (torch.empty(self.m, self.l, dtype=f, device=device), torch.empty(self.l, self.l, dtype=f, device=device),
                torch.empty(self.n, self.l, dtype=f, device=device))

    def factor(self, A, omega=None, out=None):
        import torch
        a_dtype = PBPQLP_F32 if A.dtype == torch.float32 else PBPQLP_F64
        # outputs live on the plan's device even when A is pinned host memory
        Qa, L, Qb = out if out is not None else self.outputs(self.workspace.device)
        pbpqlp_factor(self.handle, A, A.stride(0), a_dtype, self.workspace, self.ws_bytes, omega, Qa, L, Qb)
        return Qa, L, Qb

    def factor_from(self, A, pbar0=None, pbar_out=False, out=None, iterations_only=False):
        """Algorithm 3 continued from pbar0 (n x >= l, its first l columns are used),
        or from Phi when pbar0 is None.  Returns (Qa, L, Qb, Pbar) with Pbar the basis
        after the power iterations when pbar_out is true (else None); with
        iterations_only the run stops there and Qa, L, Qb are None."""
        import torch
        a_dtype = PBPQLP_F32 if A.dtype == torch.float32 else PBPQLP_F64
        dev = self.workspace.device
        pb = torch.empty(self.n, self.l, dtype=torch.float64, device=dev) if (pbar_out or iterations_only) else None
        if iterations_only:
            Qa = L = Qb = None
        else:
            Qa, L, Qb = out if out is not None else self.outputs(dev)
        ld0 = 0 if pbar0 is None else pbar0.stride(0)
        pbpqlp_factor_from(self.handle, A, A.stride(0), a_dtype, self.workspace, self.ws_bytes, pbar0, ld0, pb,
                           Qa, L, Qb)
        return Qa, L, Qb, pb

    def factor_csr(self, rowptr, colind, values, omega=None, out=None):
        """Sparse A in CSR form (rowptr int64 [m+1], colind int32 [nnz], values FP64 [nnz], on the device)."""
        import torch
        nnz = int(colind.numel())
        need = pbpqlp_csr_workspace_bytes(self.handle, nnz)
        if getattr(self, "_csr_ws", None) is None or self._csr_ws.numel() < need:
            self._csr_ws = torch.empty(need, dtype=torch.uint8, device=self.workspace.device)
        Qa, L, Qb = out if out is not None else self.outputs(self.workspace.device)
        pbpqlp_factor_csr(self.handle, rowptr, colind if nnz else None, values if nnz else None, nnz, self._csr_ws,
                          self._csr_ws.numel(), omega, Qa, L, Qb)
        return Qa, L, Qb

    def omega(self, device="cuda"):
        import torch
        o = torch.empty(self.m, self.l, dtype=torch.float64, device=device)
        pbpqlp_generate_omega(self.handle, o)
        return o

    def sketch(self, A, Y, trans=False):
        """C = A Y (or A^T Y) in the plan's mode; Y is FP64 with <= l columns."""
        import torch
        a_dtype = PBPQLP_F32 if A.dtype == torch.float32 else PBPQLP_F64
        rows = self.n if trans else self.m
        C = torch.empty(rows, Y.shape[1], dtype=torch.float64, device=A.device)
        pbpqlp_sketch(self.handle, A, A.stride(0), a_dtype, 1 if trans else 0, Y, Y.stride(0), Y.shape[1], C,
                      C.stride(0), self.workspace, self.ws_bytes)
        return C

    def reconstruct(self, Qa, L, Qb, r=None):
        import torch
        r = self.k if r is None else r
        Ahat = torch.empty(self.m, self.n, dtype=torch.float64, device=Qa.device)
        pbpqlp_reconstruct(self.handle, Qa, L, Qb, r, Ahat, self.n, self.workspace, self.ws_bytes)
        return Ahat

    def error(self, A, Qa, L, Qb, r=None, method=PBPQLP_ERR_RESIDUAL, nprobes=10, probe_seed=0):
        import torch
        r = self.k if r is None else r
        a_dtype = PBPQLP_F32 if A.dtype == torch.float32 else PBPQLP_F64
        return pbpqlp_error(self.handle, A, A.stride(0), a_dtype, Qa, L, Qb, r, method, nprobes, probe_seed,
                            self.workspace, self.ws_bytes)

    def sync_status(self):
        return pbpqlp_sync_status(self.handle)

    def rank_revealing(self, L, tol=1e-8):
        """(L-values tensor, ||A||_2 estimate, numerical rank at tol)."""
        import torch
        lv = torch.empty(self.l, dtype=torch.float64, device=L.device)
        nrm, rk = pbpqlp_rank_revealing(self.handle, L, tol, lv, self.workspace, self.ws_bytes)
        return lv, nrm, rk

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.pbpqlp_plan_destroy(h)
            self.handle = None


class Batch:
    """Owns a batched plan and its workspace; factors lists of torch matrices."""

    def __init__(self, shapes_m, shapes_n, ks, p, q, seed, mode=PBPQLP_MODE_FP64, stream=None, device="cuda"):
        import torch
        self.m = [int(x) for x in shapes_m]
        self.n = [int(x) for x in shapes_n]
        self.k = [int(x) for x in ks]
        self.p, self.q, self.seed, self.mode = int(p), int(q), int(seed), int(mode)
        self.l = [k + self.p for k in self.k]
        self.handle = pbpqlp_plan_batched(self.m, self.n, self.k, p, q, seed, mode, stream)
        self.ws_bytes = pbpqlp_batch_workspace_bytes(self.handle)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)

    def outputs(self, device="cuda"):
        import torch
        f = torch.float64
        return ([torch.empty(m, l, dtype=f, device=device) for m, l in zip(self.m, self.l)],
                [torch.empty(l, l, dtype=f, device=device) for l in self.l],
                [torch.empty(n, l, dtype=f, device=device) for n, l in zip(self.n, self.l)])

    def factor(self, As, out=None):
        import torch
        a_dtype = PBPQLP_F32 if As[0].dtype == torch.float32 else PBPQLP_F64
        Qa, L, Qb = out if out is not None else self.outputs(As[0].device)
        pbpqlp_factor_batched(self.handle, As, [a.stride(0) for a in As], a_dtype, self.workspace, self.ws_bytes,
                              Qa, L, Qb)
        return Qa, L, Qb

    def sync_status(self):
        return pbpqlp_batch_sync_status(self.handle, len(self.m))

    def autotune(self, As, out, table_path=None):
        import torch
        a_dtype = PBPQLP_F32 if As[0].dtype == torch.float32 else PBPQLP_F64
        Qa, L, Qb = out
        return pbpqlp_batch_autotune(self.handle, As, [a.stride(0) for a in As], a_dtype, self.workspace,
                                     self.ws_bytes, Qa, L, Qb, table_path)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.pbpqlp_batch_destroy(h)
            self.handle = None

#!/usr/bin/env python3
"""PbP-QLP benchmark on GB300: factorizations/s of Algorithm 3.

Default workload (one GPU): plain FP64, A = U diag(exp(-i/40)) V^T with Haar
U, V, m = n = 8000, k = 100, p = 10, q = 2 — one step is one whole
factorization (Phi, 2q+2 products with A / A^T, 2q+2 CholeskyQR orths, the
l x l QR and the basis update).  A (512 MB) is larger than the 129 MB L2, so
no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on the same workload instead.
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PbP-QLP factorizations/s & TFLOP/s, mixed vs plain FP64 at equal rel. error"
UNIT = "factorizations/s"

WORKLOADS = {
    "fp64_8000": dict(m=8000, n=8000, k=100, p=10, q=2, gen="svd", spectrum="exp", scale=40.0, rank_cap=1500,
                      mode="FP64", compare="BF16X3", emulated=True,
                      desc="plain FP64, A = U diag(exp(-i/40)) V^T, Haar U V, 8000x8000, k=100 p=10 q=2"),
    "bf16x3_20000": dict(m=20000, n=20000, k=200, p=20, q=2, gen="xyt", rank=200, eps=1e-3, mode="BF16X3",
                         compare=None,
                         desc="split-BF16 mixed, A = X Y^T + 1e-3 E (FP32), 20000x20000, k=200 p=20 q=2"),
    "batched_512": dict(batched=True, count=512, p=8, q=1, mode="TF32X3", compare="FP64",
                        desc="batched split-TF32: 512 matrices, m~U[256,4096], n~U[128,min(m,2048)], Haar U V, "
                             "sigma_i = i^-alpha, alpha~U[1,3], k~U[8,64], p=8, q=1, A in FP32"),
    "batched_64": dict(batched=True, count=64, p=8, q=1, mode="TF32X3", compare="FP64",
                       desc="batched split-TF32: 64 matrices of the 512-matrix distribution (profiling size)"),
    "fp64emu_8000": dict(m=8000, n=8000, k=100, p=10, q=2, gen="svd", spectrum="exp", scale=40.0, rank_cap=1500,
                         mode="FP64_EMU", compare=None,
                         desc="FP64-accurate products as exact BF16 digit sums on the tensor cores, "
                              "A = U diag(exp(-i/40)) V^T, Haar U V, 8000x8000, k=100 p=10 q=2"),
    "paper_t1_5000": dict(m=5000, n=5000, k=190, p=10, q=2, gen="svd", spectrum="exp", scale=40.0, rank_cap=1500,
                          mode="FP64", compare=None, emulated=True, paper_seconds=0.81,
                          desc="plain FP64, the paper's Table I runtime case n = 5000, d = 0.04n = 200 (k=190 p=10), "
                               "q=2; dense A = U diag(exp(-i/40)) V^T (the paper: spectrum immaterial for runtime)"),
    "paper_t1_10000": dict(m=10000, n=10000, k=390, p=10, q=2, gen="svd", spectrum="exp", scale=50.0, rank_cap=800,
                           mode="FP64", compare=None, emulated=True, paper_seconds=5.9,
                           desc="plain FP64, the paper's Table I runtime case n = 10000, d = 0.04n = 400 (k=390 "
                                "p=10), q=2; dense A = U diag(exp(-i/50)) V^T (blocked l x l steps)"),
    "paper_t2_5000": dict(m=5000, n=5000, k=990, p=10, q=2, gen="svd", spectrum="exp", scale=125.0, rank_cap=2000,
                          mode="FP64", compare=None, emulated=True, paper_seconds=4.3,
                          desc="plain FP64, the paper's Table II runtime case n = 5000, d = 0.2n = 1000 (k=990 "
                               "p=10), q=2; dense A = U diag(exp(-i/125)) V^T (blocked l x l steps)"),
    "csr_100k": dict(sparse=True, m=100000, n=100000, k=100, p=10, q=2, nnz_per_row=100.0, rank=110, support=150,
                     mode="FP64",
                     desc="sparse FP64 (CSR, Section III-C): 100000x100000, ~100 N(0,1) entries per row at uniform "
                          "columns plus 110 sparse rank-one terms e^(-i/20) sqrt(mn) u_i v_i^T on 150x150 "
                          "supports (12.4M nonzeros), k=100 p=10 q=2"),
    "bf16x3_10000": dict(m=10000, n=10000, k=200, p=20, q=2, gen="xyt", rank=200, eps=1e-3, mode="BF16X3",
                         compare=None,
                         desc="split-BF16 mixed, A = X Y^T + 1e-3 E (FP32), 10000x10000, k=200 p=20 q=2 (profiling size)"),
}

# FP64 issue rate of GB300: 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, 1900.0, 1700.0, "fallback"


def algorithmic_flops(m, n, l, q):
    """Every A-pass GEMM, CholeskyQR-equivalent orth work, basis update and small QR."""
    return (2 * q + 2) * 2.0 * m * n * l + 4.0 * (q + 1) * (m + n) * l * l + 2.0 * n * l * l + (8.0 / 3.0) * l ** 3


def make_matrix(w, seed, device):
    import synth
    if w["gen"] == "xyt":
        return synth.torch_xyt_plus_noise(seed, w["m"], w["n"], w["rank"], w["eps"], device=device)
    sig = synth.spectrum(w["spectrum"], w["rank_cap"], w["scale"])
    return synth.torch_svd_matrix(seed, w["m"], w["n"], sig, device=device)


def tc_roofline(rows, K, l, nprod, avg_ms, hbm_peak, tc_peak):
    """Roofline of one tensor-core product launch (rows x K operand, l columns).

    Bytes: the BF16 operand copies of A (hi and lo for the split mode, i.e. the
    same 4 bytes per element as an FP32 A), the BF16 panel, the FP32 partials.
    Flops: the MMAs the tensor pipe executes (three per split product, N padded
    to a multiple of 16)."""
    bn = (l + 15) // 16 * 16
    t = avg_ms / 1e3
    eb = 4.0 if nprod == 3 else 2.0
    hw_flops = nprod * 2.0 * rows * K * bn
    nbytes = eb * rows * K + eb * K * bn + 4.0 * rows * bn
    t_tensor = hw_flops / (tc_peak * 1e12)
    t_hbm = nbytes / (hbm_peak * 1e9)
    tensor = t_tensor >= t_hbm
    ach = hw_flops / t / 1e12 if tensor else nbytes / t / 1e9
    peak = tc_peak if tensor else hbm_peak
    return {"kernel": "k_tc_gemm (tcgen05 product with A, %s)" % ("split BF16 x3" if nprod == 3 else "BF16"),
            "bound": "tensor" if tensor else "hbm", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s" if tensor else "GB/s", "frac": ach / peak,
            "achieved_basis": "tensor-pipe MMA flops (%d MMAs per product, N padded to %d)" % (nprod, bn)
            if tensor else "bytes of the BF16 operand copies + panel + partials",
            "tensor_frac": hw_flops / t / 1e12 / tc_peak, "hbm_frac": nbytes / t / 1e9 / hbm_peak,
            "avg_launch_ms": avg_ms}


def oz_roofline(rows, K, l, avg_ms, hbm_peak, tc_peak):
    """Roofline of one FP64-emulated product launch (k_oz_gemm): rows x K
    operand in 8 BF16 digits, l columns in 48-column tiles.

    Bytes: the digits of A (16 bytes per element), read from DRAM once per
    pass when the 2 .. 8 column tiles of a row tile run in lockstep (else once
    per column tile), the panel digits, the FP64 partials.  Flops: the 36
    digit products per element the tensor pipe executes (N padded to the
    tiles); `tensor_frac_l` counts them on the l columns alone."""
    nt = (l + 47) // 48
    t = avg_ms / 1e3
    hw_flops = 36 * 2.0 * rows * K * nt * 48
    reads = 1 if 2 <= nt <= 8 else nt
    nbytes = 16.0 * rows * K * reads + 16.0 * K * nt * 48 + 8.0 * rows * nt * 48
    t_tensor = hw_flops / (tc_peak * 1e12)
    t_hbm = nbytes / (hbm_peak * 1e9)
    tensor = t_tensor >= t_hbm
    ach = hw_flops / t / 1e12 if tensor else nbytes / t / 1e9
    peak = tc_peak if tensor else hbm_peak
    return {"kernel": "k_oz_gemm (FP64 product as 36 exact BF16 digit products, tcgen05)",
            "bound": "tensor" if tensor else "hbm", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s" if tensor else "GB/s", "frac": ach / peak,
            "achieved_basis": "tensor-pipe MMA flops (36 digit products, N padded to %d)" % (nt * 48)
            if tensor else "bytes of the digits of A (once per pass) + panel digits + partials",
            "tensor_frac": hw_flops / t / 1e12 / tc_peak, "hbm_frac": nbytes / t / 1e9 / hbm_peak,
            "tensor_frac_l": 36 * 2.0 * rows * K * l / t / 1e12 / tc_peak,
            # the same launch on the algorithmic bytes of the FP64 product it replaces
            # (A once in FP64, the panels): what the digit re-reads cost
            "frac_algorithmic_bytes": (8.0 * rows * K + 8.0 * (rows + K) * l) / t / 1e9 / hbm_peak,
            "avg_launch_ms": avg_ms}


# Kernels whose DRAM traffic is recorded in profiles/: source file and the
# markers around the device code the figure belongs to.
KERNEL_SOURCES = {
    "dgemm_skinny_fp64_8000": ("fp64_device.cuh", "__device__ __forceinline__ void dev_dgemm_tile",
                               "__device__ __forceinline__ int64_t pidx"),
    "oz_gemm_fp64emu_8000": ("kernels_oz.cu", "// The MMAs of one stage (two 16-deep k-steps)",
                             "// The grouped product kernel"),
}


def read_traffic(kernel_file_tag):
    """ncu DRAM bytes per launch recorded in profiles/, valid only for the kernel source it was taken on."""
    path = os.path.join(ROOT, "profiles", kernel_file_tag + ".md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    mt = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    ms = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    cur = kernel_source_hash(kernel_file_tag)
    if not mt or not ms or cur is None:
        return None
    return float(mt.group(1)) if cur.startswith(ms.group(1)) else None


def kernel_source_hash(kernel_file_tag="dgemm_skinny_fp64_8000"):
    """sha256 of the device code a recorded traffic figure belongs to."""
    import hashlib
    fname, start, end = KERNEL_SOURCES[kernel_file_tag]
    src = os.path.join(ROOT, "paper_2103_07245_gb300", "csrc", fname)
    if not os.path.exists(src):
        return None
    txt = open(src).read()
    a = txt.find(start)
    b = txt.find(end, a)
    if a < 0 or b < 0:
        return None
    return hashlib.sha256(txt[a:b].encode()).hexdigest()


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_max(value, device=None):
    """Maximum of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dense_config(w, world):
    """The `config` object of a dense workload; both arms print this same dict."""
    abytes = (4 if w["gen"] == "xyt" else 8) * w["m"] * w["n"]
    return {"workload": w["desc"], "m": w["m"], "n": w["n"], "k": w["k"], "p": w["p"], "q": w["q"],
            "mode": w["mode"], "l2": "inputs larger than L2 (A is %d MB), no flush" % (abytes // 2 ** 20),
            "parallelism": "independent factorizations per GPU" if world > 1 else "single GPU"}


def sparse_config(w, world, nnz):
    l = w["k"] + w["p"]
    return {"workload": w["desc"], "m": w["m"], "n": w["n"], "k": w["k"], "p": w["p"], "q": w["q"], "nnz": nnz,
            "mode": "FP64",
            "l2": "the n x l panel the SpMM gathers from (%d MB) fits L2; the CSR arrays (%d MB) do not"
                  % (w["n"] * l * 8 // 2 ** 20, (12 * nnz + 8 * w["m"]) // 2 ** 20),
            "parallelism": "one factorization per GPU" if world > 1 else "single GPU"}


def sparse_matrix(w, seed):
    """The CSR workload (host numpy arrays): rowptr int64, colind int32, values FP64."""
    import synth
    return synth.sparse_csr(seed, w["m"], w["n"], w["nnz_per_row"], rank=w["rank"], support=w["support"])


def run_reference_sparse(args, w, world, rank):
    """The oracle's CSR form timed on the host cores (reference arm of the sparse workload)."""
    if rank != 0:
        return 0
    import oracle
    rp, ci, va = sparse_matrix(w, 1000)
    l = w["k"] + w["p"]
    for _ in range(args.warmup):
        oracle.pbpqlp_csr(rp, ci, va, (w["m"], w["n"]), l, w["q"], seed=7)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.pbpqlp_csr(rp, ci, va, (w["m"], w["n"]), l, w["q"], seed=7)
    dt = (time.perf_counter() - t0) / args.steps
    value = 1.0 / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": sparse_config(w, world, int(rp[-1])),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "one full FP64 oracle factorization (CSR form) per step on the same workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sparse(args, w, world, rank, local):
    """Sparse A: value = factorizations/s; roofline of the SpMM launches (FP64 ALU bound)."""
    import numpy as np
    import torch
    import paper_2103_07245_gb300 as pq

    dev = torch.device("cuda", local)
    pq.load(build_if_missing=True)
    m, n, k, p, q = w["m"], w["n"], w["k"], w["p"], w["q"]
    l = k + p
    rp, ci, va = sparse_matrix(w, 1000 + rank)
    nnz = int(rp[-1])
    d_rp, d_ci, d_va = (torch.from_numpy(x).to(dev) for x in (rp, ci, va))
    stream = torch.cuda.current_stream(dev)
    plan = pq.Plan(m, n, k, p, q, seed=7 + rank, mode=pq.PBPQLP_MODE_FP64, stream=stream, device=dev)
    outs = plan.outputs(dev)
    for _ in range(args.warmup):
        plan.factor_csr(d_rp, d_ci, d_va, out=outs)
    rc, flags = plan.sync_status()
    if rc != pq.PBPQLP_OK:
        raise RuntimeError("device status %d flags %d" % (rc, flags))
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    sampler = ClockSampler(int(vis) if vis.isdigit() else local)
    pq.pbpqlp_set_timing(plan.handle, True)
    pq.pbpqlp_read_timing(plan.handle)
    l0 = pq.pbpqlp_kernel_launch_count()
    dist_barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.factor_csr(d_rp, d_ci, d_va, out=outs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dist_barrier()
    clocks = sampler.stop()
    launches = pq.pbpqlp_kernel_launch_count() - l0
    pass_ms, pass_n = pq.pbpqlp_read_timing(plan.handle)
    pq.pbpqlp_set_timing(plan.handle, False)
    rc, flags = plan.sync_status()
    if rc != pq.PBPQLP_OK:
        raise RuntimeError("device status %d flags %d" % (rc, flags))
    ms = dist_max(e0.elapsed_time(e1) / args.steps, dev)
    value = whole_job_rate(1, world, ms)
    # end to end: the CSR arrays from pinned host memory every step, the factors back
    h = [torch.from_numpy(x).pin_memory() for x in (rp, ci, va)]
    ho = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
    h2d = sum(t.numel() * t.element_size() for t in h)
    d2h = sum(t.numel() * t.element_size() for t in ho)
    dist_barrier()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        for d, s_ in zip((d_rp, d_ci, d_va), h):
            d.copy_(s_, non_blocking=True)
        plan.factor_csr(d_rp, d_ci, d_va, out=outs)
        for d, s_ in zip(ho, outs):
            d.copy_(s_, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dist_barrier()
    e2e_ms = dist_max(e0.elapsed_time(e1) / args.steps, dev)
    # roofline of the SpMM launches: 2 nnz l flop each, FP64 FMA issue rate
    avg = pass_ms / max(pass_n, 1)
    achieved = 2.0 * nnz * l / (avg * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": sparse_config(w, world, nnz),
        "tflops_algorithmic": value * (2 * q + 2) * 2.0 * nnz * l / 1e12,
        "roofline": {"kernel": "k_csr_spmm (CSR A times an l-column panel, FP64 FMA, warp per row)",
                     "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA lanes x 2 flop x 2070 MHz",
                     "launches_timed": pass_n, "avg_launch_ms": avg},
        "e2e": {"value": whole_job_rate(1, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches, "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.pbpqlp_csr(rp, ci, va, (m, n), l, q, seed=7)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "one full FP64 oracle factorization (CSR form) of the same matrix"}
        Q, L, P = (t.cpu().numpy() for t in outs)
        # parity at full size without a dense A: the rank-k difference to the
        # oracle's factors through 16 Gaussian probes, E||D G||_F^2 / 16 = ||D||_F^2
        import scipy.sparse
        import scipy.sparse.linalg
        G = np.random.default_rng(5).standard_normal((n, 16))
        D = Q[:, :k] @ (L[:k, :k] @ (P[:, :k].T @ G)) - ref["Q"][:, :k] @ (ref["L"][:k, :k] @ (ref["P"][:, :k].T @ G))
        S = scipy.sparse.csr_matrix((va, ci, rp), shape=(m, n))
        S.sum_duplicates()
        line["parity"] = {"rel_fro_diff_rank_k_probe_estimate": float(np.linalg.norm(D) / 4.0 /
                                                                      scipy.sparse.linalg.norm(S)),
                          "tol": 1e-11, "probes": 16}
    return line


def run_reference(args, w, world, rank):
    """The FP64 CPU oracle timed on the host cores (reference arm)."""
    if rank != 0:
        return 0
    if w.get("sparse"):
        return run_reference_sparse(args, w, world, rank)
    import numpy as np
    import oracle
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = make_matrix(w, 1000, dev).cpu().numpy().astype(np.float64)
    l = w["k"] + w["p"]
    for _ in range(args.warmup):
        oracle.pbpqlp(A, l, w["q"], seed=7)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.pbpqlp(A, l, w["q"], seed=7)
    dt = (time.perf_counter() - t0) / args.steps
    value = 1.0 / dt
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dense_config(w, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one full FP64 oracle factorization per step on the same workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "tflops_algorithmic": value * algorithmic_flops(w["m"], w["n"], l, w["q"]) / 1e12,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, w, world, rank, local):
    """The uneven batch: value = factorizations/s of the whole batch per GPU."""
    import numpy as np
    import torch
    import paper_2103_07245_gb300 as pq
    import synth

    dev = torch.device("cuda", local)
    pq.load(build_if_missing=True)
    hbm_peak, bf16_peak, bf16_sus, peak_src = measured_peaks()
    shapes = synth.batched_shapes(2024 + rank, w["count"])
    p, q = w["p"], w["q"]
    A64, A32 = [], []
    for i, sh in enumerate(shapes):
        r = min(sh["m"], sh["n"])
        sig = synth.spectrum("poly", r, sh["alpha"])
        a = synth.torch_svd_matrix_device(7000 + 131 * rank + i, sh["m"], sh["n"], sig, device=dev)
        A32.append(a.float().contiguous())
        A64.append(A32[-1].double().contiguous())   # the FP32 data, exactly, for the FP64 comparison
    ms_, ns_, ks_ = [s["m"] for s in shapes], [s["n"] for s in shapes], [s["k"] for s in shapes]
    stream = torch.cuda.current_stream(dev)
    mode = getattr(pq, "PBPQLP_MODE_" + w["mode"])
    B = pq.Batch(ms_, ns_, ks_, p, q, seed=11 + rank, mode=mode, stream=stream, device=dev)
    outs = B.outputs(dev)

    barrier = dist_barrier

    B.factor(A32, out=outs)
    tuned_ms = None
    if not args.no_autotune:
        tuned_ms = B.autotune(A32, outs)
    for _ in range(args.warmup):
        B.factor(A32, out=outs)
    rc, flags = B.sync_status()
    if rc != pq.PBPQLP_OK:
        raise RuntimeError("batch status %d" % rc)
    pq.pbpqlp_batch_set_timing(B.handle, True)
    B.factor(A32, out=outs)          # records the graph with the timing events
    torch.cuda.synchronize(dev)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    sampler = ClockSampler(int(vis) if vis.isdigit() else local)
    l0 = pq.pbpqlp_kernel_launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tc_ms, tc_n = 0.0, 0
    e0.record(stream)
    for _ in range(args.steps):
        B.factor(A32, out=outs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    launches = pq.pbpqlp_kernel_launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    tc_ms, tc_n = pq.pbpqlp_batch_read_timing(B.handle)   # the last step's grouped products
    pq.pbpqlp_batch_set_timing(B.handle, False)
    ms = dist_max(ms, dev)
    count = w["count"]
    value = whole_job_rate(count, world, ms)

    def rel_errors(out_t, As):
        e = []
        for i, sh in enumerate(shapes):
            k = sh["k"]
            Ahat = (out_t[0][i][:, :k] @ out_t[1][i][:k, :k]) @ out_t[2][i][:, :k].T
            e.append(float(torch.linalg.norm(As[i] - Ahat) / torch.linalg.norm(As[i])))
        return np.array(e)

    err_tc = rel_errors(outs, A64)
    # end to end: the A_i in pinned host memory, the factors back in host memory, every step.
    # Main leg: A_i passed in place (the library's split kernel, the only reader of A, streams
    # it over NVLink-C2C), the factors of all matrices in one flat buffer and one copy back.
    # Staged leg: every A_i copied to the device first, every factor copied back separately.
    A_host = [a.cpu().pin_memory() for a in A32]
    sizes = [(sh["m"] * (sh["k"] + p), (sh["k"] + p) ** 2, sh["n"] * (sh["k"] + p)) for sh in shapes]
    flat_dev = torch.empty(sum(sum(z) for z in sizes), dtype=torch.float64, device=dev)
    flat_host = torch.empty(flat_dev.numel(), dtype=torch.float64, pin_memory=True)
    outs_flat, off = ([], [], []), 0
    for sh, z in zip(shapes, sizes):
        l_i = sh["k"] + p
        for t, (cnt, rows) in enumerate(zip(z, (sh["m"], l_i, sh["n"]))):
            outs_flat[t].append(flat_dev[off:off + cnt].view(rows, l_i))
            off += cnt
    h2d = sum(a.numel() * a.element_size() for a in A_host)
    d2h = flat_host.numel() * 8

    def e2e_step():
        B.factor(A_host, out=outs_flat)
        flat_host.copy_(flat_dev, non_blocking=True)

    A_dev = [torch.empty_like(a) for a in A32]
    out_host = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in ts] for ts in outs]

    def e2e_staged_step():
        for h, d in zip(A_host, A_dev):
            d.copy_(h, non_blocking=True)
        B.factor(A_dev, out=outs)
        for hs, ds in zip(out_host, outs):
            for h, d in zip(hs, ds):
                h.copy_(d, non_blocking=True)

    def time_e2e(step_fn):
        step_fn()
        barrier()
        torch.cuda.synchronize(dev)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            step_fn()
        f1.record(stream)
        torch.cuda.synchronize(dev)
        return dist_max(f0.elapsed_time(f1) / args.steps, dev)

    ms_e2e = time_e2e(e2e_step)
    rc, flags = B.sync_status()
    if rc != pq.PBPQLP_OK:
        raise RuntimeError("device status %d flags %d (A in host memory)" % (rc, flags))
    same = all(torch.equal(a, b) for ta, tb in zip(outs_flat, outs) for a, b in zip(ta, tb))
    ms_e2e_staged = time_e2e(e2e_staged_step)

    # the batched FP64 form on the same data (the plain-FP64 GPU reference)
    cmp = None
    if w.get("compare"):
        Bf = pq.Batch(ms_, ns_, ks_, p, q, seed=11 + rank, mode=getattr(pq, "PBPQLP_MODE_" + w["compare"]),
                      stream=stream, device=dev)
        of = Bf.outputs(dev)
        Bf.factor(A64, out=of)
        torch.cuda.synchronize(dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        csteps = max(1, min(3, args.steps))
        c0.record(stream)
        for _ in range(csteps):
            Bf.factor(A64, out=of)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        cms = c0.elapsed_time(c1) / csteps
        err_f = rel_errors(of, A64)
        ratio = err_tc / err_f
        cmp = {"mode": w["compare"], "value": count / (cms / 1e3), "unit": UNIT, "ms_per_step": cms,
               "speedup_of_mixed": cms / ms, "error_ratio_mixed_vs_fp64": {
                   "median": float(np.median(ratio)), "max": float(np.max(ratio))}}
        del Bf, of

    # roofline of the grouped tensor-core products (the last step's 2q+2 launches)
    hw, nbytes = 0.0, 0.0
    for sh in shapes:
        npad = (sh["k"] + p + 15) // 16 * 16
        for trans in ([True, False] * (q + 1)):
            M, K = (sh["n"], sh["m"]) if trans else (sh["m"], sh["n"])
            Mp = (M + 127) // 128 * 128
            hw += 3 * 2.0 * Mp * K * npad
            nbytes += 8.0 * M * K + 8.0 * K * npad + 8.0 * M * (sh["k"] + p)
    tc_t = tc_ms / 1e3 if tc_n else None
    tf32_sus = bf16_sus / 2.0
    roofline = None
    if tc_t:
        t_tensor, t_hbm = hw / (tf32_sus * 1e12), nbytes / (hbm_peak * 1e9)
        tensor = t_tensor >= t_hbm
        ach = hw / tc_t / 1e12 if tensor else nbytes / tc_t / 1e9
        peak = tf32_sus if tensor else hbm_peak
        roofline = {"kernel": "k_tc_list (grouped tcgen05 kind::tf32 products, split x3)",
                    "bound": "tensor" if tensor else "hbm", "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s" if tensor else "GB/s", "frac": ach / peak, "traffic": None,
                    "peak_source": "%s: TF32 = bf16 sustained / 2 (nominal ratio), HBM copy" % peak_src,
                    "tensor_frac": hw / tc_t / 1e12 / tf32_sus, "hbm_frac": nbytes / tc_t / 1e9 / hbm_peak,
                    "launches_timed": tc_n, "avg_launch_ms": tc_ms / tc_n}
    flops = sum(algorithmic_flops(sh["m"], sh["n"], sh["k"] + p, q) for sh in shapes)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "tf32x3", "data": "synthetic",
        "config": {"workload": w["desc"], "count": count, "p": p, "q": q, "mode": w["mode"],
                   "l2": "inputs larger than L2 (%d MB of A), no flush" % (sum(a.numel() * 4 for a in A32) // 2 ** 20),
                   "parallelism": "independent batches per GPU" if world > 1 else "single GPU",
                   "graph": "one CUDA graph replay per step", "autotuned_ms": tuned_ms},
        "tflops_algorithmic": value * flops / count / 1e12,
        "rel_err_rank_k": {"median": float(np.median(err_tc)), "max": float(np.max(err_tc))},
        "roofline": roofline,
        "e2e": {"value": world * count / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "how": "A_i read in place from pinned host memory by the split kernel (NVLink-C2C); factors "
                       "copied back in one copy", "factors_equal_device_resident_run": same},
        "e2e_staged": {"value": world * count / (ms_e2e_staged / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h,
                       "how": "every A_i copied to the device, every factor copied back, one copy each"},
        "gpu_launches": launches, "clocks": clocks, "fp64_batched": cmp,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        sample = list(range(0, count, max(1, count // 6)))[:6]
        t0 = time.perf_counter()
        refs = {i: oracle.pbpqlp(A64[i].cpu().numpy(), shapes[i]["k"] + p, q, seed=11 + i) for i in sample}
        dt = time.perf_counter() - t0
        ratios = []
        for i in sample:
            k = shapes[i]["k"]
            An = A64[i].cpu().numpy()
            g = [t[i].cpu().numpy() for t in outs]
            e_g = oracle.rel_fro_error(An, *g, k)
            e_o = oracle.rel_fro_error(An, refs[i]["Q"], refs[i]["L"], refs[i]["P"], k)
            ratios.append(e_g / e_o)
        line["cpu_baseline"] = {"value": len(sample) / dt, "unit": UNIT, "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": "%d matrices of the batch (every %d-th), full FP64 oracle"
                                % (len(sample), max(1, count // 6))}
        line["parity"] = {"error_ratio_vs_oracle": {"max": float(np.max(ratios)), "median": float(np.median(ratios))},
                          "tol_ratio": 1.1, "matrices": len(sample)}
    return line


def class_breakdown(pq, pl, A, outs, reps=2):
    """Milliseconds per factorization of each timing class (events around every
    launch group), from `reps` extra factorizations outside the timed region."""
    ncls = len(pq.TIME_CLASSES)
    pq.pbpqlp_set_timing_classes(pl.handle, (1 << ncls) - 1)
    for c in range(ncls):
        pq.pbpqlp_read_timing_class(pl.handle, c)
    for _ in range(reps):
        pl.factor(A, out=outs)
    res = {}
    for c, name in enumerate(pq.TIME_CLASSES):
        msc, nc = pq.pbpqlp_read_timing_class(pl.handle, c)
        res[name] = {"ms": msc / reps, "groups": nc // reps}
    pq.pbpqlp_set_timing_classes(pl.handle, 0)
    return res


CLASS_KERNELS = {
    "chol": "k_chol_inv_cluster (Cholesky of the CholeskyQR Gram with T = R^-T, FP64, one thread-block cluster)",
    "gram": "CholeskyQR Grams (upper triangle of X^T X, FP64-accurate digit products on the tensor cores)",
    "solve": "CholeskyQR solve Q = C T^T (FP64-accurate digit product)",
    "smallqr": "k_small_qr_cluster (Householder QR of R^T, Eq. 7, FP64, one thread-block cluster)",
    "other": "R = Q^T D and Qb = Pbar Ptil (digit products)",
}


def class_roofline(name, bd, m, n, l, q, fp64_probe=None):
    """Roofline of a non-pass class: its algorithmic FP64 flops per factorization
    (FP64-equivalent for the digit forms) over its measured time, against the
    FP64 issue rate of the whole GPU."""
    orth_rows = [n] + [m, n] * q + [m]          # the orths of Algorithm 3, two CholeskyQR passes each
    eff = 2 * len(orth_rows)                     # passes that run (the retry pairs exit at once)
    if name == "chol":
        flops = eff * (2.0 / 3.0) * l ** 3       # l^3/6 FMA each for R and for T = R^-T
        per = eff
    elif name == "gram":
        flops = sum(2 * r * l * (l + 1) / 2.0 for r in orth_rows) * 2
        per = eff
    elif name == "solve":
        flops = sum(r * l * l for r in orth_rows) * 2
        per = eff
    elif name == "smallqr":
        flops = (8.0 / 3.0) * l ** 3
        per = 1
    else:
        flops = m * l * (l + 1) + 2.0 * n * l * l
        per = 2
    t = bd[name]["ms"] / 1e3
    ach = flops / t / 1e12 if t > 0 else None
    return {"kernel": CLASS_KERNELS[name], "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS if ach else None, "traffic": None,
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz (FP64-equivalent algorithmic flops)",
            "peak_probe": fp64_probe, "frac_probe": ach / fp64_probe if (ach and fp64_probe) else None,
            "launches_timed": per, "avg_launch_ms": bd[name]["ms"] / per,
            "share_of_step": None}


def dominant_roofline(bd, pass_roofline, m, n, l, q, step_ms, fp64_probe=None):
    """The roofline of the class that takes the most time per factorization."""
    name = max(bd, key=lambda c: bd[c]["ms"])
    r = dict(pass_roofline) if name == "pass" else class_roofline(name, bd, m, n, l, q, fp64_probe)
    r["share_of_step"] = bd[name]["ms"] / step_ms if step_ms else None
    r["class"] = name
    return r


def run_dense(args, w, world, rank, local):
    """One dense workload: value = factorizations/s; every leg's roofline points at
    its dominant kernel class (timed live by class of launch)."""
    import numpy as np
    import torch
    import paper_2103_07245_gb300 as pq

    dev = torch.device("cuda", local)
    pq.load(build_if_missing=True)

    m, n, k, p, q = w["m"], w["n"], w["k"], w["p"], w["q"]
    l = k + p
    hbm_peak, bf16_peak, bf16_sus, peak_src = measured_peaks()
    A = make_matrix(w, 1000 + rank, dev)
    stream = torch.cuda.current_stream(dev)
    mode = getattr(pq, "PBPQLP_MODE_" + w["mode"])
    plan = pq.Plan(m, n, k, p, q, seed=7 + rank, mode=mode, stream=stream, device=dev)
    Qa, L, Qb = plan.outputs(dev)

    barrier = dist_barrier

    def timed_run(pl, outs, steps, sampler=None):
        """K factorizations bracketed by barrier + synchronize (the library replays the
        recorded launch sequence), then 2 more with event pairs around each pass kernel,
        outside the timed region, for the pass kernels' launch times.
        Returns (ms/step, pass ms, passes, launches, clocks)."""
        l0 = pq.pbpqlp_kernel_launch_count()
        barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            pl.factor(A, out=outs)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        clk = sampler.stop() if sampler else None
        launches = pq.pbpqlp_kernel_launch_count() - l0
        rc, flags = pl.sync_status()
        if rc != pq.PBPQLP_OK:
            raise RuntimeError("device status %d flags %d" % (rc, flags))
        pq.pbpqlp_set_timing(pl.handle, True)
        pq.pbpqlp_read_timing(pl.handle)
        for _ in range(2):
            pl.factor(A, out=outs)
        pms, pn = pq.pbpqlp_read_timing(pl.handle)
        pq.pbpqlp_set_timing(pl.handle, False)
        return e0.elapsed_time(e1) / steps, pms, pn, launches, clk

    for _ in range(args.warmup):
        plan.factor(A, out=(Qa, L, Qb))
    rc, flags = plan.sync_status()
    if rc != pq.PBPQLP_OK:
        raise RuntimeError("device status %d flags %d" % (rc, flags))

    # ---- device-resident timing (inputs already in HBM)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    sampler = ClockSampler(int(vis) if vis.isdigit() else local)
    ms, pass_ms, pass_launches, launches, clocks = timed_run(plan, (Qa, L, Qb), args.steps, sampler)
    ms = dist_max(ms, dev)
    value = whole_job_rate(1, world, ms)
    err_main = plan.error(A, Qa, L, Qb, k, method=pq.PBPQLP_ERR_RESIDUAL)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    A_host = A.cpu().pin_memory()
    A_dev = torch.empty_like(A)
    out_host = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (Qa, L, Qb)]
    h2d = A_host.numel() * A_host.element_size()
    d2h = sum(t.numel() * t.element_size() for t in out_host)

    def e2e_step():
        A_dev.copy_(A_host, non_blocking=True)
        plan.factor(A_dev, out=(Qa, L, Qb))
        for h, d in zip(out_host, (Qa, L, Qb)):
            h.copy_(d, non_blocking=True)
    e2e_step()
    barrier()
    torch.cuda.synchronize(dev)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    f1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms_e2e = dist_max(f0.elapsed_time(f1) / args.steps, dev)

    flops = algorithmic_flops(m, n, l, q)
    avg_pass_ms = (pass_ms / pass_launches) if pass_launches else None
    sink = torch.zeros(4096, dtype=torch.float64, device=dev)
    fp64_probe = pq.pbpqlp_fp64_rate_probe(sink)   # measured FP64 FMA issue rate, beside the derived peak
    if w["mode"] == "FP64":
        achieved = 2.0 * m * n * l / (avg_pass_ms / 1e3) / 1e12 if avg_pass_ms else None
        roofline = {"kernel": "k_dgemm_skinny (A / A^T pass, 2mnl flop per launch)", "bound": "alu",
                    "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                    "traffic": read_traffic("dgemm_skinny_fp64_8000"),
                    "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz (not in MEASURED_PEAKS.json)",
                    "peak_probe": fp64_probe, "frac_probe": (achieved / fp64_probe) if achieved else None,
                    "peak_probe_source": "pbpqlp_fp64_rate_probe: the shared-memory inner loop of a register-blocked "
                                         "FP64 GEMM (4 x 4 accumulators per thread), best of 1, 2 and 4 CTAs "
                                         "per SM, CUDA events, measured in this run",
                    "launches_timed": pass_launches, "avg_launch_ms": avg_pass_ms}
        dtype = "f64"
    elif w["mode"] == "FP64_EMU":
        roofline = oz_roofline(max(m, n), min(m, n), l, avg_pass_ms, hbm_peak, bf16_sus) if avg_pass_ms else None
        if roofline:
            roofline["traffic"] = read_traffic("oz_gemm_fp64emu_8000") if (m, n, l) == (8000, 8000, 110) else None
            roofline["peak_source"] = "%s (MEASURED_PEAKS.json: HBM copy GB/s, bf16 sustained TFLOP/s)" % peak_src
            roofline["launches_timed"] = pass_launches
        dtype = "f64-emulated (bf16 digit products, exact sums)"
    else:
        nprod = 3 if w["mode"] == "BF16X3" else 1
        roofline = tc_roofline(max(m, n), min(m, n), l, nprod, avg_pass_ms, hbm_peak, bf16_sus)
        roofline["traffic"] = None
        roofline["peak_source"] = "%s (MEASURED_PEAKS.json: HBM copy GB/s, bf16 sustained TFLOP/s)" % peak_src
        roofline["launches_timed"] = pass_launches
        dtype = "bf16x3" if nprod == 3 else "bf16"
    bd = class_breakdown(pq, plan, A, (Qa, L, Qb))
    pass_roofline = roofline
    roofline = dominant_roofline(bd, roofline, m, n, l, q, ms, fp64_probe) if roofline else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        # the paper's own time for this exact configuration (Table I, FP64 MATLAB on a 4-core
        # Core i7 at 1.8 GHz), as factorizations/s: context, another machine
        "vs_baseline": value * w["paper_seconds"] if w.get("paper_seconds") else None,
        "dtype": dtype, "data": "synthetic",
        "config": dense_config(w, world),
        "tflops_algorithmic": value * flops / 1e12,
        "rel_err_rank_k": err_main,
        "roofline": roofline,
        "pass_roofline": pass_roofline,
        "breakdown_ms_per_step": {c: round(v["ms"], 4) for c, v in bd.items()},
        "e2e": {"value": world / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
    }

    # ---- out of core: A left in pinned host memory, streamed over the host link every pass
    if w["mode"] == "FP64" and not args.no_out_of_core:
        ooc_out = plan.outputs(dev)
        for _ in range(1):
            plan.factor(A_host, out=ooc_out)
        torch.cuda.synchronize(dev)
        o0 = torch.cuda.Event(enable_timing=True)
        o1 = torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for _ in range(args.steps):
            plan.factor(A_host, out=ooc_out)
        o1.record(stream)
        torch.cuda.synchronize(dev)
        oms = dist_max(o0.elapsed_time(o1) / args.steps, dev)
        line["out_of_core"] = {"value": whole_job_rate(1, world, oms), "unit": UNIT, "ms_per_step": oms,
                               "bitwise_equal": bool(all(torch.equal(a, b) for a, b in zip(ooc_out, (Qa, L, Qb)))),
                               "note": "A in pinned host memory, read by the kernels over the host link each pass"}

    # ---- the same matrix in the mixed mode: speed at (near) equal relative error
    if w.get("compare"):
        cmode = getattr(pq, "PBPQLP_MODE_" + w["compare"])
        cplan = pq.Plan(m, n, k, p, q, seed=7 + rank, mode=cmode, stream=stream, device=dev)
        couts = cplan.outputs(dev)
        for _ in range(args.warmup):
            cplan.factor(A, out=couts)
        cms, cpms, cpn, _, _ = timed_run(cplan, couts, args.steps)
        err_c = cplan.error(A, *couts, k, method=pq.PBPQLP_ERR_RESIDUAL)
        nprod = 3 if w["compare"] == "BF16X3" else 1
        cpass = tc_roofline(max(m, n), min(m, n), l, nprod, cpms / cpn, hbm_peak, bf16_sus) if cpn else None
        cbd = class_breakdown(pq, cplan, A, couts)
        line["mixed"] = {"mode": w["compare"], "value": world / (cms / 1e3), "unit": UNIT, "ms_per_step": cms,
                         "tflops_algorithmic": world / (cms / 1e3) * flops / 1e12,
                         "rel_err_rank_k": err_c, "rel_err_rank_k_fp64": err_main,
                         "error_ratio_vs_fp64": err_c / err_main, "speedup_vs_fp64": ms / cms,
                         "roofline": dominant_roofline(cbd, cpass, m, n, l, q, cms, fp64_probe) if cpass else None,
                         "pass_roofline": cpass,
                         "breakdown_ms_per_step": {c: round(v["ms"], 4) for c, v in cbd.items()}}
        del cplan

    # ---- the same matrix with the products emulated in FP64 accuracy on the tensor cores
    if w.get("emulated"):
        eplan = pq.Plan(m, n, k, p, q, seed=7 + rank, mode=pq.PBPQLP_MODE_FP64_EMU, stream=stream, device=dev)
        eouts = eplan.outputs(dev)
        for _ in range(args.warmup):
            eplan.factor(A, out=eouts)
        ems, epms, epn, elaunch, _ = timed_run(eplan, eouts, args.steps)
        ems = dist_max(ems, dev)
        err_e = eplan.error(A, *eouts, k, method=pq.PBPQLP_ERR_RESIDUAL)
        ah_e = eplan.reconstruct(*eouts, k)
        ah_f = plan.reconstruct(Qa, L, Qb, k)
        diff = float(torch.linalg.norm(ah_e - ah_f) / torch.linalg.norm(A))
        del ah_e, ah_f
        line["fp64_emulated"] = {
            "mode": "FP64_EMU", "value": whole_job_rate(1, world, ems), "unit": UNIT, "ms_per_step": ems,
            "dtype": "bf16 digit products summed exactly (FP64-accurate)",
            "tflops_algorithmic": whole_job_rate(1, world, ems) * flops / 1e12,
            "rel_err_rank_k": err_e, "rel_err_rank_k_fp64": err_main,
            "rel_fro_diff_vs_fp64_rank_k": diff, "speedup_vs_fp64": ms / ems, "gpu_launches": elaunch}
        epass = dict(oz_roofline(max(m, n), min(m, n), l, epms / epn, hbm_peak, bf16_sus),
                     traffic=read_traffic("oz_gemm_fp64emu_8000") if (m, n, l) == (8000, 8000, 110) else None) \
            if epn else None
        ebd = class_breakdown(pq, eplan, A, eouts)
        line["fp64_emulated"]["roofline"] = dominant_roofline(ebd, epass, m, n, l, q, ems, fp64_probe) if epass else None
        line["fp64_emulated"]["pass_roofline"] = epass
        line["fp64_emulated"]["breakdown_ms_per_step"] = {c: round(v["ms"], 4) for c, v in ebd.items()}
        del eplan, eouts

    # ---- CPU baseline: the oracle, rank 0 at N = 1, and parity of the timed result
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        A_np = A_host.numpy().astype(np.float64)
        t0 = time.perf_counter()
        ref = oracle.pbpqlp(A_np, l, q, seed=7)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "one full FP64 oracle factorization of the same %dx%d matrix (q=%d, l=%d)"
                                          % (m, n, q, l)}
        Qa_n, L_n, Qb_n = (t.numpy() for t in out_host)
        Ag = oracle.reconstruct(Qa_n, L_n, Qb_n, k)
        Ac = oracle.reconstruct(ref["Q"], ref["L"], ref["P"], k)
        if w["mode"] in ("FP64", "FP64_EMU"):
            line["parity"] = {"rel_fro_diff_rank_k": float(np.linalg.norm(Ag - Ac) / np.linalg.norm(A_np)),
                              "tol": 1e-11}
        else:
            e_gpu = float(np.linalg.norm(A_np - Ag) / np.linalg.norm(A_np))
            e_orc = float(np.linalg.norm(A_np - Ac) / np.linalg.norm(A_np))
            line["parity"] = {"rel_err_rank_k": e_gpu, "rel_err_rank_k_oracle": e_orc,
                              "error_ratio": e_gpu / e_orc, "tol_ratio": 1.1}
    return line


DEFAULT_WORKLOAD = "fp64_8000"
# Sub-legs of the default run: the split-BF16 20000^2 workload and the 512-matrix batch.
DEFAULT_SUBLEGS = (("mixed_c3", "bf16x3_20000"), ("batched", "batched_512"))
SUBLEG_KEYS = ("value", "unit", "ms_per_step", "dtype", "config", "tflops_algorithmic", "rel_err_rank_k", "roofline",
               "breakdown_ms_per_step", "e2e", "e2e_staged", "gpu_launches", "clocks", "cpu_baseline", "parity",
               "fp64_batched")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-out-of-core", action="store_true")
    ap.add_argument("--no-sublegs", action="store_true", help="default workload only: skip the c3 and batched legs")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    w = WORKLOADS[args.workload]
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, w, world, rank)
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if w.get("batched"):
        line = run_batched(args, w, world, rank, local)
    elif w.get("sparse"):
        line = run_sparse(args, w, world, rank, local)
    else:
        line = run_dense(args, w, world, rank, local)
    if args.workload == DEFAULT_WORKLOAD and not args.no_sublegs:
        for key, name in DEFAULT_SUBLEGS:
            torch.cuda.empty_cache()
            wl = WORKLOADS[name]
            sub = run_batched(args, wl, world, rank, local) if wl.get("batched") else \
                run_dense(args, wl, world, rank, local)
            line[key] = {kk: sub[kk] for kk in SUBLEG_KEYS if kk in sub}
            # the sub-legs' kernels count toward this run's launches too
            line["gpu_launches"] = line.get("gpu_launches", 0) + sub.get("gpu_launches", 0)
            line.setdefault("gpu_launches_by_leg", {})[key] = sub.get("gpu_launches", 0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

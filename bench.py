#!/usr/bin/env python
"""Benchmark of the two-site H_eff matvec (Section II-C / Fig. 1d) on GB300.

Workload (default): the 6x6 J1-J2 cylinder stand-in at m = 4096: spin-1/2, U(1) Sz,
40 sectors per bond with multinomial(4096, Binom(39, 1/2)) dimensions (seeds 0 and 1),
range-4 chain MPO (k = 14, couplings 1, 0.5, 0.2, 0.1), symmetrised Gaussian
environments, Gaussian two-site tensor (seed 2).  One step = one heff_apply (operator
preparation + pack + the two grouped GEMMs) on inputs resident in HBM.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (bounded sample per step).  With torchrun (N > 1) the default is one
apply spread over the ranks by row shards (the left sectors a' of y, assigned by
longest-processing-time over their GEMM flops): each rank runs its shard's plan into a
zeroed y and an all-reduce of y (NCCL) completes the apply on every rank (strong
scaling).  ``--mode replicas`` instead runs an independent problem per rank (its own
two-site tensor, no collective on the data path; weak scaling).  The time is the maximum
over ranks.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "H_eff applies/s at m=4096 (6x6 J1-J2 stand-in, U(1) Sz, k=14)"

# ncu figures per launch of the four kernels of one apply (DRAM bytes read + written, and
# the tensor pipe's active cycles in % of peak for the GEMMs), keyed by (workload,
# precision, kernel, tile variant), from the committed ncu profile summary of the apply;
# valid only while the device code they were measured on is unchanged (hash below).
NCU_FIGURES = {
    ("spin_m4096", "bf16x3", "mix", 0): {"dram_bytes": 193512192 + 334207744},
    ("spin_m4096", "bf16x3", "pack", 0): {"dram_bytes": 24090112 + 768},
    ("spin_m4096", "bf16x3", "gemm1", 256): {"dram_bytes": 432674048 + 283594496, "tensor_pct": 56.21},
    ("spin_m4096", "bf16x3", "gemm2", 256): {"dram_bytes": 718457088 + 38714880, "tensor_pct": 65.00},
}
NCU_SRC_SHA = "b88c17ecde77e8e5"


def _src_sha():
    """Hash of the device code of tc_gemm.cu and apply.cu (each file up to its host-side
    section), of the PTX wrappers they include and of the planner that orders and assigns
    their tiles: the code the ncu figures were measured on."""
    import hashlib
    h = hashlib.sha256()
    for name, mark in (("tc_gemm.cu", b"// ---------------------------------------------------------------- host side"),
                       ("apply.cu", b"// ------------------------------------------------------------------ host side"),
                       ("tc_ptx.cuh", b""), ("convert.cuh", b""), ("plan.cpp", b"")):
        with open(os.path.join(ROOT, "paper_2007_05540_gb300", "csrc", name), "rb") as f:
            txt = f.read()
        cut = txt.find(mark) if mark else -1
        h.update(txt[:cut] if cut >= 0 else txt)
    return h.hexdigest()[:16]


def algorithmic_bytes(lays, io_bytes):
    """Bytes one apply must move at least: read L, W1, W2, R and x, write y (io dtype)."""
    Ll, W1l, W2l, Rl, xl = lays
    return io_bytes * (Ll.nelem + W1l.nelem + W2l.nelem + Rl.nelem + 2 * xl.nelem)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--mode", default="shard", choices=["shard", "replicas"],
                    help="N > 1: row shards of one apply + all-reduce of y (default), or independent problems")
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3", "fp64"])
    ap.add_argument("--workload", default="spin_m4096")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--tiles", default="",
                    help="tile variants of GEMM 1 and GEMM 2 (256, 128 or 512 = CTA pairs), e.g. 512,256; "
                         "skips the autotuner")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the planner's default tile widths (for profiling: serialised launches under a "
                         "profiler would time the candidates differently)")
    ap.add_argument("--part", default="",
                    choices=["", "lanczos", "svd", "env_update", "backward", "energy", "batched", "dmrg"],
                    help="time one step of the DMRG bond update alone and print its own JSON line "
                         "(the profiling cases): the FP64 Lanczos eigensolver (30 iterations, BF16x3 "
                         "matvecs), the block SVD truncation, the environment update, the gradients")
    ap.add_argument("--block-precisions", default="fp64,bf16x3",
                    help="--part env_update / backward: the block-product precisions to time")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary measurements (other precisions, eigensolver, SVD, batched graph)")
    return ap.parse_args()


# ------------------------------------------------------------------ peaks and clocks
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks
def sum_over_ranks(v, device):
    """The sum of a per-rank float over the process group; the identity without one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())


def max_over_ranks(v, device):
    """The maximum of a per-rank float over the process group (the job's time is the
    slowest rank's); the identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_batch(rank):
    """Each rank's problem in replicas mode: the shared L, W, R of the workload and its own
    two-site tensor (batch entry = rank), so ranks are independent (weak scaling, no
    data-path collective)."""
    return int(rank)


def sharded_step(apply_shard, y):
    """One row-sharded apply: the other shards' y blocks are zero here, this rank writes its
    own (apply_shard(y)), and the sum over the ranks (an all-reduce) is the whole y on every
    rank.  Without a process group of more than one rank it is the plain apply."""
    import torch.distributed as dist
    multi = dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    if multi:
        y.zero_()
    apply_shard(y)
    if multi:
        dist.all_reduce(y)


# ------------------------------------------------------------------ problem
def make_problem(name, batch):
    import workloads as wl
    from paper_2007_05540_gb300 import heff
    w = wl.workload_by_name(name)
    lays = heff.heff_layouts((w.alpha_q, w.alpha_d), (w.beta_q, w.beta_d), w.phys, w.ql, w.qm, w.qr)
    Ll, W1l, W2l, Rl, xl = lays
    bufs = {"L": Ll.assemble(lambda k: w.L_block(k)), "R": Rl.assemble(lambda k: w.R_block(k)),
            "W1": W1l.assemble(lambda k: w.W1[k]), "W2": W2l.assemble(lambda k: w.W2[k]),
            "x": xl.assemble(lambda k: w.x_block(k, batch))}
    return w, lays, bufs


def cpu_baseline(name, seconds, batch=0, threads=None):
    """The FP64 oracle (as it stands) on the host cores, on sampled output sectors.

    threads=None: all cores (NumPy's BLAS threads); threads=1: a child process with every
    BLAS thread pool limited to one thread (the pools read their size at start-up)."""
    if threads is not None:
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
        code = ("import json, sys; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.cpu_baseline(%r, %r, %r)))" % (ROOT, name, float(seconds), int(batch)))
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            return {"error": r.stderr[-300:]}
        out = json.loads(r.stdout.strip().splitlines()[-1])
        out["cores"] = int(threads)
        return out
    import workloads as wl
    from oracle import heff as oh
    w = wl.workload_by_name(name)
    L, W1, W2, R, x = oh.problem_from_workload(w, batch)
    total = oh.canonical_flops(L, W1, W2, R, x)["total"]
    nsec = len(w.alpha_d)
    order = list(range(nsec))
    t0 = time.perf_counter()
    done_flops, ns = 0.0, 0
    while time.perf_counter() - t0 < seconds and ns < nsec:
        s = order[(ns * 7) % nsec] if nsec % 7 else order[ns]
        cnt = {}
        oh.heff_apply(L, W1, W2, R, x, count=cnt, left_sectors={s})
        done_flops += cnt["gemm1"] + cnt["gemm2"]
        ns += 1
    dt = time.perf_counter() - t0
    rate = done_flops / dt
    return {"value": rate / total, "unit": "applies/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{ns} of {nsec} output left sectors of one apply ({done_flops:.3e} of "
                      f"{total:.3e} canonical flops) in {dt:.1f} s; applies/s = flop rate / flops per apply",
            "tflops": rate / 1e12}


# ------------------------------------------------------------------ secondary measurements
def _events_ms(fn, n, stream, flush=None):
    """Mean CUDA-event time of fn() on `stream` over n runs (L2 flushed before each)."""
    import torch
    ts = []
    for _ in range(n):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.mean(ts))


def dense_gemm_rates(dev, stream):
    """cuBLAS dense-GEMM rates of this GPU (through torch.matmul) in TF32 and FP64, and BF16
    as a check against the measured peak: the denominators of the other precisions'
    rooflines (square products, inputs resident, median of timed repetitions)."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, n, reps in (("bf16", torch.bfloat16, 8192, 10), ("tf32", torch.float32, 8192, 10),
                                  ("fp64", torch.float64, 4096, 3)):
            torch.backends.cuda.matmul.allow_tf32 = name == "tf32"
            g = torch.Generator(device=dev).manual_seed(7)
            a = torch.randn(n, n, device=dev, dtype=torch.float32, generator=g).to(dt)
            b = torch.randn(n, n, device=dev, dtype=torch.float32, generator=g).to(dt)
            c = torch.empty(n, n, device=dev, dtype=dt)
            with torch.cuda.stream(stream):
                torch.matmul(a, b, out=c)
                ts = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    torch.matmul(a, b, out=c)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (float(np.median(ts)) * 1e-3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def extras(args, w, lays, bufs, dev, stream, flush, value):
    """Same workload in the other precisions, the eigensolver step around the apply, the
    SVD truncation, and the batched electron workload replayed from a captured graph."""
    import torch
    from paper_2007_05540_gb300 import heff
    Ll, W1l, W2l, Rl, xl = lays
    out = {}
    # other matvec precisions on the same inputs
    rates = {args.precision: value}
    for prec in ("bf16x3", "tf32x3", "fp64"):
        if prec in rates:
            continue
        io = "f64" if prec == "fp64" else "f32"
        dt = torch.float64 if io == "f64" else torch.float32
        P = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], prec, io)
        d = {k: torch.from_numpy(np.asarray(v)).to(dev, dt) for k, v in bufs.items()}
        ws = P.workspace(dev)
        y = torch.empty_like(d["x"])
        if prec != "fp64":
            heff.heff_plan_autotune(P.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], y, ws, stream)

        def f(P=P, d=d, y=y, ws=ws):
            heff.heff_apply(P.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], y, ws, stream)
        n = 3 if prec == "fp64" else 10
        for _ in range(2):
            f()
        rates[prec] = 1000.0 / _events_ms(f, n, stream, flush)
        del P, d, ws, y
    out["applies_per_s"] = rates
    out["speedup_vs_fp64_gpu"] = {p: rates[p] / rates["fp64"] for p in rates if p != "fp64"}
    # whole-apply rooflines of every precision against this GPU's cuBLAS rate for the dtype
    canon = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], "fp64", "f64").flops_canonical
    dense = dense_gemm_rates(dev, stream)
    dt_of = {"bf16x3": "bf16", "tf32x3": "tf32", "fp64": "fp64"}
    out["roofline_by_precision"] = {
        "peaks_tflops": dense,
        "peak_source": "cuBLAS GEMM through torch.matmul on this GPU (bf16, tf32: 8192^3; fp64: 4096^3)",
        "note": "whole apply (prepare + pack + GEMM 1 + GEMM 2): canonical flops x applies/s over the dtype's "
                "dense-GEMM rate; the split precisions issue three tensor-core products per useful "
                "multiply-add (tensor_pipe_frac)"}
    for p, r in rates.items():
        u = canon * r / 1e12
        e = {"useful_tflops": u, "frac": u / dense[dt_of[p]]}
        if p != "fp64":
            e["tensor_pipe_frac"] = 3.0 * e["frac"]
        out["roofline_by_precision"][p] = e

    # eigensolver step: FP64 Lanczos (30 iterations) with BF16x3 and with FP64 matvecs,
    # the FP64 Rayleigh quotient of the mixed Ritz vector, then the block SVD truncation
    n_iter = 30
    d64 = {k: torch.from_numpy(np.asarray(bufs[k])).to(dev, torch.float64) for k in ("L", "W1", "W2", "R")}
    x0 = torch.from_numpy(np.asarray(bufs["x"])).to(dev, torch.float64)
    res = {}
    for prec in ("bf16x3", "fp64"):
        P = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], prec, "f64")
        ws = P.workspace(dev)
        lz = torch.empty(heff.heff_lanczos_workspace_size(P.handle, n_iter), dtype=torch.uint8, device=dev)
        xv = torch.empty_like(x0)
        r = torch.zeros(3 + 2 * (n_iter + 1), dtype=torch.float64, device=dev)

        def f(P=P, ws=ws, lz=lz, xv=xv, r=r):
            heff.heff_lanczos(P.handle, d64["L"], d64["W1"], d64["W2"], d64["R"], x0, n_iter, xv, r, ws, lz, stream)
        f()
        ms = _events_ms(f, 1 if prec == "fp64" else 3, stream)
        res[prec] = (ms, float(r[0].item()), xv, P, ws, float(r[1].item()))
    ms_b, th_b, xb, Pb, wsb, resid_b = res["bf16x3"]
    ms_f, th_f, xf, P64, ws64, resid_f = res["fp64"]
    y = torch.empty_like(xb)

    def rq(P, ws, v):
        heff.heff_apply(P.handle, d64["L"], d64["W1"], d64["W2"], d64["R"], v, y, ws, stream)
        torch.cuda.synchronize()
        return float(torch.dot(v, y) / torch.dot(v, v))
    th_rq = rq(P64, ws64, xb)
    # energy of one vector (the FP64 Ritz vector) under each matvec precision
    Pt = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], "tf32x3", "f64")
    wst = Pt.workspace(dev)
    e64, eb, et = rq(P64, ws64, xf), rq(Pb, wsb, xf), rq(Pt, wst, xf)
    out["lanczos30"] = {
        "ms_bf16x3": ms_b, "ms_fp64": ms_f, "speedup": ms_f / ms_b,
        "ritz_bf16x3": th_b, "ritz_fp64": th_f, "rq_fp64_of_bf16x3_vector": th_rq,
        "residual_estimate": {"bf16x3": resid_b, "fp64": resid_f},
        "rel_diff_ritz": abs(th_b - th_f) / abs(th_f), "rel_diff_refined": abs(th_rq - th_f) / abs(th_f),
        "energy_same_vector_rel_err": {"bf16x3": abs(eb - e64) / abs(e64), "tf32x3": abs(et - e64) / abs(e64)},
        "note": "same start vector, FP64 orthogonalisation and tridiagonal eigensolver in both; 30 steps do "
                "not converge this synthetic spectrum, so the Ritz values differ by Krylov drift; "
                "energy_same_vector compares <v|K|v>/<v|v> of the FP64 Ritz vector under each matvec"}
    del Pt, wst
    del res, y
    # ground energy of config 3, both paths converged (restarted Lanczos to a residual
    # estimate of 1e-8 |E| from the same start vector)
    out["energy_config3"] = ground_state_compare(args.workload, dev, stream)
    s = heff.heff_svd_create(xl.handle)
    sws = torch.empty(heff.heff_svd_workspace_size(s), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sweeps = heff.heff_svd_compute(s, xb, sws, stream)
    q, dims, disc, nrm = heff.heff_svd_truncate(s, int(w.alpha_d.sum()), 1e-12, w.nq, 4096)
    torch.cuda.synchronize()
    sw32, sw64 = heff.heff_svd_info(s)
    out["svd_truncation"] = {"ms": (time.perf_counter() - t0) * 1e3, "jacobi_sweeps": {"fp32": sw32, "fp64": sw64},
                             "kept": int(np.sum(dims)), "sectors": int(len(dims)), "discarded_weight": float(disc),
                             "note": "one-sided Jacobi per charge block: FP32 preconditioning sweeps, FP64 orthonormalisation and FP64 sweeps; host wall time incl. the sync"}
    heff.heff_svd_destroy(s)
    del sws, xb, d64, x0

    # environment update (left side) onto a new bond of the same size with even charges,
    # FP64 block products
    out["env_update"] = env_update_timing(w, dev, stream)
    # Rayleigh-quotient gradients: whole intermediates at m = 1024, streamed at m = 4096
    out["backward"] = backward_timing(dev, stream)

    # lattice MPO windows at m = 4096: the 6 x 6 J1-J2 cylinder (k = 26) and the paper's
    # 20 x 10 J1-J2 cylinder (k = 38, uncompressed)
    for key, name, note in (
            ("paper_block_model_m4096", "spin_paper_m4096",
             "the block-size model of the paper's Table II, b_l = floor((m/4) 0.6^|l|): 27 sectors, centre "
             "block 1024; range-4 chain MPO (k = 14)"),
            ("j1j2_6x6_lattice_m4096", "spin_j1j2_6x6_m4096",
             "two-site window of the snake-ordered 6x6 J1-J2 (J2 = 0.5) cylinder MPO, binomial sectors"),
            ("j1j2_20x10_lattice_m4096", "spin_j1j2_20x10_m4096",
             "two-site window of the snake-ordered 20x10 J1-J2 (J2 = 0.5) cylinder MPO (the paper's spin "
             "lattice), binomial sectors"),
            ("j1j2_20x10_compressed_m4096", "spin_j1j2_20x10c_m4096",
             "the same window of the 20x10 J1-J2 cylinder MPO compressed at the SVD cutoff 1e-13 "
             "(k = 32, SVD basis), binomial sectors"),
            ("j1j2_20x10_compressed_interpolative_m4096", "spin_j1j2_20x10ci_m4096",
             "the same compression keeping a subset of the automaton's channels (k = 32, sparse W), "
             "binomial sectors")):
        out[key] = {**single_apply(name, dev, stream, flush), "note": note}

    # 32 electron-model applies sharing L, W, R in one captured graph (autotuned tiles): the
    # range-5 chain window and the 4 x 8 Hubbard cylinder window
    for name in ("electron_m2048", "electron_hubbard_4x8_m2048", "electron_tri_xc6_m2048", "electron_tri_xc6c_m2048",
                 "electron_tri_xc6ci_m2048"):
        out[name + "_batch32_graph"] = batched_graph(name, 32, dev, stream, flush)
    # the GPU two-site DMRG driver: full sweeps of the 6x6 J1-J2 cylinder, bond caps 16 .. 1024
    out["dmrg_6x6_sweeps"] = dmrg_sweep_timing()
    return out


def ground_state_compare(name, dev, stream, n_iter=120, cycles=6, tol=1e-8):
    """heff_ground_state with BF16x3 matvecs (energy: the FP64 Rayleigh quotient of its Ritz
    vector) and with FP64 matvecs, from the same start vector; host wall time of each (the
    routine synchronises once per restart cycle)."""
    import torch
    from paper_2007_05540_gb300 import heff
    w, lays, bufs = make_problem(name, 0)
    d = {k: torch.from_numpy(np.asarray(bufs[k])).to(dev, torch.float64) for k in ("L", "W1", "W2", "R", "x")}
    P64 = heff.Plan(*lays, bufs["W1"], bufs["W2"], "fp64", "f64")
    Pb = heff.Plan(*lays, bufs["W1"], bufs["W2"], "bf16x3", "f64")
    ws64, wsb = P64.workspace(dev), Pb.workspace(dev)
    gs = torch.empty(heff.heff_ground_state_workspace_size(Pb.handle, n_iter), dtype=torch.uint8, device=dev)
    x = torch.empty_like(d["x"])
    out = {}
    for key, P, P2, ws, ws2 in (("mixed", Pb, P64, wsb, ws64), ("fp64", P64, None, ws64, None)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = heff.heff_ground_state(P.handle, P2.handle if P2 is not None else None, d["L"], d["W1"], d["W2"],
                                   d["R"], d["x"], n_iter, cycles, tol, x, ws, ws2, gs, stream)
        torch.cuda.synchronize()
        r["s"] = time.perf_counter() - t0
        out[key] = r
    E64, Em = out["fp64"]["energy"], out["mixed"]["energy"]
    return {"workload": name, "E_fp64": E64, "E_mixed": Em, "rel_err": abs(Em - E64) / abs(E64),
            "ritz_bf16x3": out["mixed"]["ritz"], "rel_err_ritz_bf16x3": abs(out["mixed"]["ritz"] - E64) / abs(E64),
            "residual_fp64": {"mixed": out["mixed"]["residual_fp64"], "fp64": out["fp64"]["residual_fp64"]},
            "residual_estimate": {"mixed": out["mixed"]["residual_estimate"],
                                  "fp64": out["fp64"]["residual_estimate"]},
            "cycles": {"mixed": out["mixed"]["cycles"], "fp64": out["fp64"]["cycles"]},
            "matvecs": {"mixed": out["mixed"]["matvecs"], "fp64": out["fp64"]["matvecs"]},
            "s": {"mixed": out["mixed"]["s"], "fp64": out["fp64"]["s"]},
            "speedup": out["fp64"]["s"] / out["mixed"]["s"],
            "note": f"restarted Lanczos ({n_iter} steps per cycle) until the residual estimate is <= {tol:g} |E|; "
                    "mixed: BF16x3 matvecs, energy = FP64 Rayleigh quotient of its Ritz vector (one FP64 apply); "
                    "residual_fp64 = ||K x - E x|| / |E| with FP64 matvecs"}


def single_apply(name, dev, stream, flush):
    """One BF16x3 apply of a workload with autotuned tiles: CUDA-event mean of 10 (L2 flushed)."""
    import torch
    from paper_2007_05540_gb300 import heff
    wj, lj, bj = make_problem(name, 0)
    Pj = heff.Plan(*lj, bj["W1"], bj["W2"], "bf16x3", "f32")
    dj = {k: torch.from_numpy(np.asarray(v)).to(dev, torch.float32) for k, v in bj.items()}
    wsj = Pj.workspace(dev)
    yj = torch.empty_like(dj["x"])
    tnj = heff.heff_plan_autotune(Pj.handle, dj["L"], dj["W1"], dj["W2"], dj["R"], dj["x"], yj, wsj, stream)

    def fj():
        heff.heff_apply(Pj.handle, dj["L"], dj["W1"], dj["W2"], dj["R"], dj["x"], yj, wsj, stream)
    for _ in range(3):
        fj()
    msj = _events_ms(fj, 10, stream, flush)
    res = {"applies_per_s": 1000.0 / msj, "ms": msj, "tile_variant": list(tnj), "mpo_k": int(wj.W1.shape[0]),
           "flops_per_apply": Pj.flops_canonical, "tflops_canonical": Pj.flops_canonical / (msj * 1e-3) / 1e12}
    del Pj, dj, wsj, yj
    torch.cuda.synchronize()
    return res


def batched_graph(name, nb, dev, stream, flush):
    """nb applies of one workload sharing L, W, R, captured once in a CUDA graph and replayed."""
    import torch
    from paper_2007_05540_gb300 import heff
    we, le, be = make_problem(name, 0)
    xs_host = [le[4].assemble(lambda k: we.x_block(k, b)) for b in range(nb)]
    Pe = heff.Plan(*le, be["W1"], be["W2"], "bf16x3", "f32", max_batch=nb)
    de = {k: torch.from_numpy(np.asarray(be[k])).to(dev, torch.float32) for k in ("L", "W1", "W2", "R")}
    xs = [torch.from_numpy(v).to(dev, torch.float32) for v in xs_host]
    ys = [torch.empty_like(v) for v in xs]
    wse = Pe.workspace(dev)
    tn = heff.heff_plan_autotune(Pe.handle, de["L"], de["W1"], de["W2"], de["R"], xs[0], ys[0], wse, stream)
    cs = torch.cuda.Stream(device=dev)
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        heff.heff_apply_batched(Pe.handle, de["L"], de["W1"], de["W2"], de["R"], xs, ys, wse, cs)
    torch.cuda.current_stream().wait_stream(cs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        heff.heff_apply_batched(Pe.handle, de["L"], de["W1"], de["W2"], de["R"], xs, ys, wse, cs)
    for _ in range(3):
        g.replay()
    ms = _events_ms(g.replay, 10, torch.cuda.current_stream(), flush)
    fl = Pe.flops_canonical
    res = {"applies_per_s": nb * 1000.0 / ms, "ms_per_batch": ms, "tile_variant": list(tn),
           "tflops_canonical": nb * fl / (ms * 1e-3) / 1e12, "flops_per_apply": fl,
           "sectors": int(len(we.alpha_d)), "max_block": int(we.alpha_d.max()), "mpo_k": int(we.W1.shape[0])}
    del g, Pe, wse, xs, ys, de
    torch.cuda.synchronize()
    return res


def env_update_timing(w, dev, stream, precs=("fp64", "bf16x3")):
    import torch
    import workloads as wl
    from workloads.fill import site_block
    from paper_2007_05540_gb300 import heff
    ones = lambda n: np.ones(n, dtype=np.int32)
    m_new, nsec_new = int(w.alpha_d.sum()), int(len(w.alpha_d)) + 1
    gq, gd = wl.binomial_sectors(m_new, nsec_new, 31, parity=0)
    ph = w.phys
    site_l = heff.Layout([(w.alpha_q, w.alpha_d, 1), (ph, ones(len(ph)), 1), (gq, gd, -1)])
    W_l = heff.Layout([(w.ql, ones(w.W1.shape[0]), 1), (ph, ones(len(ph)), 1), (ph, ones(len(ph)), -1),
                       (w.qm, ones(w.W1.shape[3]), -1)])
    old_l = heff.Layout([(w.alpha_q, w.alpha_d, -1), (w.ql, ones(len(w.ql)), 1), (w.alpha_q, w.alpha_d, 1)])
    new_l = heff.Layout([(gq, gd, -1), (w.qm, ones(len(w.qm)), 1), (gq, gd, 1)])
    site = site_l.assemble(lambda k: site_block(36, k, (int(w.alpha_d[k[0]]), int(gd[k[2]]))))
    Wv = W_l.assemble(lambda k: w.W1[k])
    old = old_l.assemble(lambda k: w.L_block(k))
    plan = heff.heff_env_plan_create(old_l.handle, site_l.handle, W_l.handle, new_l.handle, Wv, "left")
    out = {"m_old": m_new, "m_new": m_new,
           "note": "left environment L[a',w,a] extended by one site; fp64: FP64 block products on CUDA cores, "
                   "bf16x3: the same products on the tensor cores (BF16 hi/lo split, FP32 accumulation); "
                   "rel_err_bf16x3: norm-wise against the FP64 result"}
    try:
        ws = torch.empty(heff.heff_env_workspace_size(plan), dtype=torch.uint8, device=dev)
        d = [torch.from_numpy(v).to(dev) for v in (old, site, Wv)]
        env = {p: torch.empty(new_l.nelem, dtype=torch.float64, device=dev) for p in precs}
        fl = heff.heff_env_flops(plan)
        out["flops"] = fl
        for prec in precs:
            heff.heff_env_plan_set_precision(plan, prec)

            def f(prec=prec):
                heff.heff_env_update(plan, d[0], d[1], d[2], env[prec], ws, stream)
            f()
            ms = _events_ms(f, 3, stream)
            out[prec] = {"ms": ms, "tflops": fl / (ms * 1e-3) / 1e12}
        if len(env) == 2:
            out["rel_err_bf16x3"] = float(torch.linalg.norm(env["bf16x3"] - env["fp64"]) /
                                          torch.linalg.norm(env["fp64"]))
        out["status"] = heff.heff_env_status(plan, ws, stream)
    finally:
        heff.heff_env_plan_destroy(plan)
    return out


def backward_timing(dev, stream, precs=("fp64", "bf16x3")):
    import torch
    import workloads as wl
    from paper_2007_05540_gb300 import heff
    res = {}
    # m = 4096 twice: in one pass (no workspace limit) and streamed through a 256 MB limit
    for key, name, limit in (("spin_m1024", "spin_m1024", 0), ("spin_m4096", "spin_m4096", 0),
                             ("spin_m4096_streamed_256MB", "spin_m4096", 256 << 20)):
        w, lays, bufs = make_problem(name, 0)
        Ll, W1l, W2l, Rl, xl = lays
        g = heff.heff_grad_plan_create(Ll.handle, W1l.handle, W2l.handle, Rl.handle, xl.handle, bufs["W1"],
                                       bufs["W2"], limit)
        try:
            d = {k: torch.from_numpy(np.asarray(v)).to(dev) for k, v in bufs.items()}
            rho = torch.empty((), dtype=torch.float64, device=dev)
            res[key] = {"chunks": heff.heff_grad_chunks(g)}
            grads = {}
            for prec in precs:
                # the apply inside (for rho and dx) and the block products in the same precision
                plan = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], prec, "f64")
                aws = plan.workspace(dev)
                heff.heff_grad_plan_set_precision(g, prec)
                gws = torch.empty(heff.heff_grad_workspace_size(g), dtype=torch.uint8, device=dev)
                outs = [torch.empty_like(d[k]) for k in ("x", "L", "R", "W1", "W2")]

                def f(plan=plan, aws=aws, outs=outs, gws=gws):
                    heff.heff_backward(g, plan.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], rho, *outs, aws,
                                       gws, stream)
                f()
                ms = _events_ms(f, 2, stream)
                grads[prec] = outs
                res[key][prec] = {"ms": ms, "rho": float(rho), "grad_workspace_MB": gws.numel() / 1e6}
                del plan, aws, gws
            if len(grads) == 2:
                res[key]["rel_err_bf16x3"] = {k: float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for k, a, b
                                              in zip(("dx", "dL", "dR", "dW1", "dW2"), grads["bf16x3"],
                                                     grads["fp64"])}
        finally:
            heff.heff_grad_plan_destroy(g)
    return res


# ------------------------------------------------------------------ one step alone
def run_part(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    if args.part == "lanczos":
        return run_lanczos_only(args)
    precs = tuple(args.block_precisions.split(","))
    if args.part == "env_update":
        w, _, _ = make_problem(args.workload, 0)
        out = env_update_timing(w, dev, stream, precs)
    elif args.part == "backward":
        out = backward_timing(dev, stream, precs)
    elif args.part == "energy":
        out = ground_state_compare(args.workload, dev, stream)
    elif args.part == "batched":
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        out = batched_graph(args.workload, 32, dev, stream, flush)
    elif args.part == "dmrg":
        out = dmrg_sweep_timing()
    else:
        out = svd_timing(args, dev, stream)
    print(json.dumps({"part": args.part, "workload": args.workload, **out}), flush=True)


def dmrg_sweep_timing(m_schedule=(16, 32, 64, 128, 256, 512, 1024), precision="bf16x3"):
    """Two-site DMRG on the GPU (dmrg.py: per bond the Lanczos eigensolver, the block SVD
    split and the environment update) for the snake-ordered 6x6 J1-J2 (J2 = 0.5) cylinder
    from the Neel product state, one sweep per bond cap: the host wall time and the energy of
    each sweep (no oracle at these sizes: the test suite checks the driver against the
    oracle's DMRG to m = 64)."""
    import torch
    import workloads as wl
    from paper_2007_05540_gb300 import dmrg
    mpo = wl.heisenberg_mpo(36, wl.cylinder_pairs(6, 6, 1.0, 0.5))
    states = [0] * 36                             # Neel: the state (x + y) mod 2 on site (x, y)
    for x in range(6):
        for y in range(6):
            states[wl.snake_index(x, y, 6)] = (x + y) % 2
    run = dmrg.GpuDMRG(mpo, (0,), precision, 20, 1e-12, states=states)
    sweeps = []
    for m in m_schedule:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = run.sweep(int(m))
        torch.cuda.synchronize()
        sweeps.append({"m_max": int(m), "s": time.perf_counter() - t0, "energy": e,
                       "max_bond": int(max(run.bond_dims()))})
    return {"lattice": "6x6 J1-J2 cylinder (J2 = 0.5), 36 sites, MPO k = 26", "matvec": precision,
            "lanczos_steps_per_bond": 20, "sweeps": sweeps, "refined_energy": run.refined_energy(),
            "note": "one sweep = 70 two-site bond updates (left to right and back), each building its plans, "
                    "Lanczos, block SVD split and environment update on the GPU; host wall time per sweep"}


def svd_timing(args, dev, stream):
    """Block SVD truncation (to m, cutoff 1e-12) of the workload's two-site tensor x: the
    host wall time of heff_svd_compute + heff_svd_truncate (they synchronise)."""
    import torch
    from paper_2007_05540_gb300 import heff
    w, lays, bufs = make_problem(args.workload, 0)
    xl = lays[4]
    x = torch.from_numpy(np.asarray(bufs["x"])).to(dev, torch.float64)
    x /= torch.linalg.norm(x)
    s = heff.heff_svd_create(xl.handle)
    try:
        sws = torch.empty(heff.heff_svd_workspace_size(s), dtype=torch.uint8, device=dev)
        heff.heff_svd_compute(s, x, sws, stream)                 # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        heff.heff_svd_compute(s, x, sws, stream)
        q, dims, disc, nrm = heff.heff_svd_truncate(s, int(w.alpha_d.sum()), 1e-12, w.nq, 4096)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        sw32, sw64 = heff.heff_svd_info(s)
    finally:
        heff.heff_svd_destroy(s)
    return {"ms": ms, "jacobi_sweeps": {"fp32": sw32, "fp64": sw64}, "kept": int(np.sum(dims)),
            "sectors": int(len(dims)), "discarded_weight": float(disc)}


def run_lanczos_only(args):
    """FP64 Lanczos (30 iterations) with BF16x3 matvecs on one GPU: one warm-up run, then the
    CUDA-event time of 3 runs (the L2 is not flushed: the basis vectors exceed it)."""
    import torch
    from paper_2007_05540_gb300 import heff
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    w, lays, bufs = make_problem(args.workload, 0)
    Ll, W1l, W2l, Rl, xl = lays
    n_iter = 30
    d64 = {k: torch.from_numpy(np.asarray(bufs[k])).to(dev, torch.float64) for k in ("L", "W1", "W2", "R")}
    x0 = torch.from_numpy(np.asarray(bufs["x"])).to(dev, torch.float64)
    P = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], "bf16x3", "f64")
    ws = P.workspace(dev)
    lz = torch.empty(heff.heff_lanczos_workspace_size(P.handle, n_iter), dtype=torch.uint8, device=dev)
    xv = torch.empty_like(x0)
    r = torch.zeros(3 + 2 * (n_iter + 1), dtype=torch.float64, device=dev)

    def f():
        heff.heff_lanczos(P.handle, d64["L"], d64["W1"], d64["W2"], d64["R"], x0, n_iter, xv, r, ws, lz, stream)
    f()
    ms = _events_ms(f, 3, stream)
    print(json.dumps({"workload": args.workload, "lanczos_iterations": n_iter, "matvec": "bf16x3",
                      "ms": ms, "ritz": float(r[0].item()), "residual_estimate": float(r[1].item())}),
          flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2007_05540_gb300 import heff

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = args.precision
    io = "f64" if prec == "fp64" else "f32"
    dt = torch.float64 if io == "f64" else torch.float32
    shard = world > 1 and args.mode == "shard"
    w, lays, bufs = make_problem(args.workload, 0 if shard else rank_batch(rank))
    Ll, W1l, W2l, Rl, xl = lays
    plan = heff.Plan(Ll, W1l, W2l, Rl, xl, bufs["W1"], bufs["W2"], prec, io,
                     shard=(rank, world) if shard else None)
    st = plan.stats
    d = {k: torch.from_numpy(np.asarray(v)).to(dev, dt) for k, v in bufs.items()}
    ws = plan.workspace(dev)
    y = torch.empty_like(d["x"])
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2

    def apply_shard(out):
        heff.heff_apply(plan.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], out, ws, stream)

    def step():
        sharded_step(apply_shard, y)

    # one-time plan setup (outside the timed region): tile width per GEMM by measurement
    tune_ms = None
    if args.tiles:
        tile_n = tuple(int(v) for v in args.tiles.split(","))
        heff.heff_plan_select_tiles(plan.handle, *tile_n)
    elif args.no_autotune:
        tile_n = (int(st[15]), int(st[22]) or int(st[15]))
    else:
        tune_ms = []
        tile_n = heff.heff_plan_autotune(plan.handle, d["L"], d["W1"], d["W2"], d["R"], d["x"], y, ws, stream,
                                         times=tune_ms)
    st = plan.stats = heff.heff_plan_stats(plan.handle)
    heff.heff_plan_set_timing(plan.handle, False)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    if not args.no_clocks:
        clocks.start()
        time.sleep(0.3)
    n0 = heff.heff_launch_count()
    step_ms, phases = [], np.zeros(4)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    evs = []
    for _ in range(args.steps):
        flush.zero_()                                   # L2 flush between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    launches = heff.heff_launch_count() - n0
    ck = clocks.stop() if not args.no_clocks else {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    ms = max_over_ranks(float(np.mean(step_ms)), dev)
    # phase breakdown from further steps with events between the kernels: those events keep
    # consecutive kernels from overlapping (dependent launch), so they stay out of the timed steps
    heff.heff_plan_set_timing(plan.handle, True)
    n_ph = min(args.steps, 20)
    for _ in range(n_ph):
        flush.zero_()
        step()
        phases += np.array(heff.heff_plan_timings(plan.handle))   # waits for this step
    heff.heff_plan_set_timing(plan.handle, False)
    phases /= n_ph

    # end to end through the C ABI from pinned host buffers: heff_apply_host copies the
    # step's inputs in, applies and copies y out; two streams alternate (own staging buffer,
    # workspace and host y each), so one step's copies overlap the other's compute
    host = {k: torch.from_numpy(np.asarray(v)).to(dt).pin_memory() for k, v in bufs.items()}
    y_host = [torch.empty(y.numel(), dtype=dt).pin_memory() for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = y_host[0].numel() * y_host[0].element_size()
    e2e_steps = max(4, min(args.steps, 20))
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    staging = [torch.empty(heff.heff_apply_host_staging_size(plan.handle), dtype=torch.uint8, device=dev)
               for _ in range(2)]
    wss = [ws, plan.workspace(dev)]

    def e2e_step(k):
        j = k % 2
        if shard:
            # each rank: its inputs in, its shard, the all-reduce of y, y out
            with torch.cuda.stream(streams[j]):
                dj = {kk: t.to(dev, non_blocking=True) for kk, t in host.items()}
                yj = torch.empty_like(dj["x"])

                def ap(out, dj=dj):
                    heff.heff_apply(plan.handle, dj["L"], dj["W1"], dj["W2"], dj["R"], dj["x"], out, wss[j], streams[j])
                sharded_step(ap, yj)
                y_host[j].copy_(yj, non_blocking=True)
            return
        heff.heff_apply_host(plan.handle, host["L"], host["W1"], host["W2"], host["R"], host["x"], y_host[j],
                             staging[j], wss[j], streams[j])
    heff.heff_plan_set_timing(plan.handle, False)
    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st_ in streams:
        st_.wait_stream(stream)
    for k in range(e2e_steps):
        e2e_step(k)
    for st_ in streams:
        stream.wait_stream(st_)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, dev)
    del staging, wss

    peaks, peak_src = measured_peaks()
    canonical = plan.flops_canonical
    per_step = 1 if shard else world          # applies completed by the job per step
    if shard:                                 # a shard plan counts its own share
        canonical = sum_over_ranks(canonical, dev)
    value = per_step * 1000.0 / ms
    g_ms = {"gemm1": phases[2], "gemm2": phases[3]}
    dom = max(g_ms, key=g_ms.get)
    useful = float(st[18] if dom == "gemm1" else st[19])
    if prec == "fp64":
        # FP64 on CUDA cores: the GB300 FP64 rate (nominal 1.25 TFLOP/s) bounds it
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": 1.25,
                "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)",
                "achieved": useful / (g_ms[dom] * 1e-3) / 1e12}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        # frac counts the method's useful flops (valid rows, columns and contraction of the
        # kernel's tiles); the split issues three tensor-core products per useful
        # multiply-add, so the tensor pipe is busy about three times that (tensor_pipe_frac)
        passes = 3
        base = peaks["bf16_tflops"] * (1.0 if prec == "bf16x3" else 0.5)
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": base,
                "peak_source": ("bf16 burst, " if prec == "bf16x3" else "bf16 burst x 0.5 (nominal tf32/bf16), ")
                + peak_src,
                "achieved": useful / (g_ms[dom] * 1e-3) / 1e12}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["tensor_pipe_frac"] = passes * roof["frac"]
        roof["note"] = (f"achieved/frac: useful flops of the kernel's tiles; tensor_pipe_frac: the {passes} "
                        "tensor-core products per useful multiply-add of the hi/lo split")
    # the whole apply: canonical flops of the method per step against the same peak
    roof["apply_frac"] = canonical / (ms * 1e-3) / 1e12 / roof["peak"]
    roof["kernel"] = dom
    roof["launch_ms"] = g_ms[dom]
    sha = _src_sha()
    tiles = {"gemm1": int(tile_n[0]), "gemm2": int(tile_n[1]), "mix": 0, "pack": 0}
    fig = {k: NCU_FIGURES.get((args.workload, prec, k, tiles[k])) for k in tiles}
    fresh = sha == NCU_SRC_SHA
    roof["traffic"] = fig[dom]["dram_bytes"] if fresh and fig[dom] else None
    roof["traffic_unit"] = "bytes per launch (ncu dram read + write)"
    alg = algorithmic_bytes(lays, 8 if io == "f64" else 4)
    roof["algorithmic_bytes_per_apply"] = alg
    if fresh and all(fig.values()):
        roof["traffic_ratio"] = sum(f["dram_bytes"] for f in fig.values()) / alg
        roof["ncu_tensor_pipe_pct"] = {k: fig[k].get("tensor_pct") for k in ("gemm1", "gemm2")}
    else:
        roof["traffic_ratio"] = None
        roof["ncu_tensor_pipe_pct"] = None

    # the apply an eigensolver pays per Krylov step: heff_apply_prepared (pack + GEMMs) with
    # the operators prepared once
    heff.heff_prepare(plan.handle, d["L"], d["W1"], d["W2"], d["R"], ws, stream)

    def prep_step():
        sharded_step(lambda out: heff.heff_apply_prepared(plan.handle, d["x"], out, ws, stream), y)
    for _ in range(3):
        prep_step()
    prep_ms = max_over_ranks(_events_ms(prep_step, max(args.steps, 10), stream, flush), dev)

    out = {
        "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms,
        "ms_per_step_median": float(np.median(step_ms)), "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": {"bf16x3": "bf16x3->f32", "tf32x3": "tf32x3->f32", "fp64": "f64"}[prec],
        "data": "synthetic (seeded; no dataset)",
        "config": {"workload": args.workload, "m": int(w.alpha_d.sum()), "sectors": int(len(w.alpha_d)),
                   "mpo_k": int(w.W1.shape[0]), "d": int(w.W1.shape[1]), "precision": prec, "io_dtype": io,
                   "tile_variant": list(tile_n),
                   "autotune_ms": [round(v, 4) for v in tune_ms] if tune_ms is not None else None,
                   "l2": "flushed (512 MB write) between timed steps; working set > L2",
                   "parallelism": (f"row shards of one apply x{world} (LPT over left sectors) + NCCL all-reduce of y"
                                   if shard else f"independent problems per rank x{world}")},
        "tflops_canonical": canonical * value / 1e12,
        "flops_per_apply": canonical,
        "phase_ms": {"prepare": phases[0], "pack": phases[1], "gemm1": phases[2], "gemm2": phases[3]},
        "apply_prepared": {"value": per_step * 1000.0 / prep_ms, "unit": "applies/s", "ms": prep_ms,
                           "tflops_canonical": canonical / (prep_ms * 1e-3) / 1e12,
                           "note": "heff_apply_prepared (pack + GEMM 1 + GEMM 2; operators prepared once), "
                                   "the matvec an eigensolver repeats"},
        "wall_s": wall,
        "e2e": {"value": per_step * 1000.0 / e2e_ms, "unit": "applies/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": ck,
    }
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "spin_m4096":
        out["extras"] = extras(args, w, lays, bufs, dev, stream, flush, value)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
        out["cpu_baseline"]["one_thread"] = cpu_baseline(args.workload, args.cpu_seconds / 2, threads=1)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = []
    base = None
    for _ in range(args.warmup + args.steps):
        base = cpu_baseline(args.workload, max(1.0, min(args.cpu_seconds, 120.0 / max(1, args.steps + args.warmup))))
        steps.append(base["value"])
    v = float(np.median(steps[args.warmup:]))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "applies/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded; no dataset)",
           "config": {"workload": args.workload, "precision": "fp64 oracle (CPU)"},
           "cpu_baseline": {"value": v, "unit": "applies/s", "cores": base["cores"], "kind": "oracle",
                            "sample": base["sample"]},
           "e2e": {"value": v, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.part:
        run_part(a)
    else:
        run_ours(a)

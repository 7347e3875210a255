"""Benchmark of the COPA AO-ADMM outer iteration on GB300.

Workload: synthetic EHR-shaped tensor with K = 500,000 subjects, J = 1,500 features,
I_k ~ Pareto(1.5) clipped to [1, 2000] (mean ~40 visits), 1 + Poisson(4) Zipf(1.1) codes
per visit (~1e8 nonzeros), integer counts U{1..50} stored as bf16; rank R = 40,
non-negative W, l1 on V (lambda = 1), 20 ADMM iterations per factor. One step = one
outer iteration (Procrustes for every subject, then H, W, V by ADMM, then the FIT).

Prints ONE JSON line (rank 0). Under torchrun (N > 1) the subjects are split into one
contiguous, nnz-balanced shard per GPU and the partial sums are all-reduced over NCCL
(strong scaling of the same K = 500,000 fit). `--impl reference` times the FP64 CPU oracle
instead, on the host cores, over a bounded random sample of subjects, scaled to the full K.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "ehr_K500k_J1500_R40"
METRIC = "AO-ADMM outer iters/sec (K=500k, J=1500, R=40)"
R_RANK, N_INNER, LAM_V = 40, 20, 1.0

# The other configurations: parity cases of the tests, measured here on request.
#   smoothing (K=20k, J=500, R=10): the B-spline projection once, then the fit on it;
#   backward (K=50k, J=1000, R=20): loss and gradients with Q from one Procrustes step;
#   rank sweep (K=100k, J=1000, R from --rank).
OTHER_WORKLOADS = {
    "ehr_K20k_J500_R10_smooth": dict(gen="ehr_K20k", R=10, n_inner=10, smooth=True),
    "ehr_K50k_J1000_R20_backward": dict(gen="ehr_K50k", R=20, backward=True),
    "ehr_K100k_J1000": dict(gen="ehr_K100k", R=None, n_inner=10),
    # hyperparameter sweep: 8 fits (l1 weight on V over a grid) of the smoothed K=20k tensor
    "ehr_K20k_J500_R10_sweep8": dict(gen="ehr_K20k", R=10, n_inner=10, smooth=True, sweep=8),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--K", type=int, default=500_000, help="subjects (smaller for quick runs)")
    ap.add_argument("--cpu-sample", type=int, default=50_000, help="subjects in the oracle sample")
    ap.add_argument("--gap-outer", type=int, default=10, help="outer iterations of the fit-gap runs")
    ap.add_argument("--gap-oracle-sample", type=int, default=2000,
                    help="subjects of the oracle refit in the fit-gap leg (0: skip)")
    ap.add_argument("--no-fit-gap", action="store_true")
    ap.add_argument("--plain-outer", type=int, default=3,
                    help="outer iterations of the plain per-subject FP64 form in the fit-gap leg (0: skip)")
    ap.add_argument("--no-tune", action="store_true", help="default launch schedule (no copa_tune)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD] + sorted(OTHER_WORKLOADS),
                    help="the headline workload (default) or one of the other configurations, "
                         "which print their own line (no e2e, no CPU baseline)")
    ap.add_argument("--rank", type=int, default=40, help="R for ehr_K100k_J1000 (the rank sweep)")
    return ap.parse_args()


def make_data(K):
    import synth
    t = time.time()
    X = synth.ehr_K500k(K=K)
    H0, V0, W0 = synth.init_factors(X.K, X.J, R_RANK)
    return X, (H0, V0, W0), time.time() - t


# ---------------------------------------------------------------------------------
# CPU oracle leg: the FP64 oracle on the host cores, subjects sharded over a process pool
# ---------------------------------------------------------------------------------

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        for key in ("model name", "CPU part", "Hardware"):
            for ln in txt.splitlines():
                if ln.startswith(key):
                    return f"{key}: {ln.split(':', 1)[1].strip()} ({platform.machine()})"
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _oracle_worker(conn, root, path, n_inner, lam, steps):
    """One shard of the oracle's outer iteration (oracle/sharded.py); the all-reduce goes
    through the parent, which sums the shards' partials in a fixed order."""
    sys.path.insert(0, root)
    import synth
    from oracle import copa_oracle as O
    from oracle import sharded as OS
    d = np.load(path)
    Xs = synth.SparseTensor(int(d["K"]), int(d["J"]), d["subj_ptr"], d["row_ptr"], d["col"], d["val"])
    st = OS.ShardState(d["H"], d["V"], d["W"], np.zeros_like(d["H"]), np.zeros_like(d["V"]), np.zeros_like(d["W"]))
    opt = O.Options(n_inner=n_inner, c_H=O.NONE, c_W=O.NONNEG, c_V=O.L1, lam_V=lam)

    def allreduce(x):
        conn.send(np.ascontiguousarray(x, dtype=np.float64))
        return conn.recv()

    conn.send("ready")
    assert conn.recv() == "go"
    fits = []
    for _ in range(steps):
        st, fit = OS.outer_iteration(Xs, st, opt, allreduce)
        fits.append(fit)
        conn.send(("iter", fit))
    conn.send(("done", fits))
    conn.close()


def sample_subjects(X, init, n_sample, seed=0):
    rng = np.random.default_rng(seed)
    ks = np.sort(rng.choice(X.K, size=min(n_sample, X.K), replace=False))
    H0, V0, W0 = init
    return X.subset(ks), (H0, V0, W0[ks])


def oracle_pool_run(Xs, init, steps):
    """The oracle's outer iteration on the host cores: the subjects of Xs are split into one
    contiguous nnz-balanced shard per core (cores = the affinity mask's size), every shard
    process runs oracle/sharded.py on its subjects (one BLAS thread), and this process sums
    the shards' partial sums (F_H, F_V, the Grams, the FIT terms) and sends them back.
    Returns (seconds per outer iteration for each step, FIT history, cores)."""
    import multiprocessing as mp
    H0, V0, W0 = init
    cores = max(1, min(host_cores(), Xs.K))
    nnz_pre = Xs.row_ptr[Xs.subj_ptr]
    bounds = np.searchsorted(nnz_pre, np.linspace(0, nnz_pre[-1], cores + 1), side="left")
    bounds[0], bounds[-1] = 0, Xs.K
    bounds = np.maximum.accumulate(bounds)
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs, conns = [], []
    with tempfile.TemporaryDirectory() as td:
        try:
            for p in range(cores):
                sub = Xs.subset(np.arange(bounds[p], bounds[p + 1]))
                path = os.path.join(td, f"shard{p}.npz")
                np.savez(path, K=sub.K, J=sub.J, subj_ptr=sub.subj_ptr, row_ptr=sub.row_ptr, col=sub.col,
                         val=sub.val, H=H0, V=V0, W=W0[bounds[p]:bounds[p + 1]])
                a, b = ctx.Pipe()
                pr = ctx.Process(target=_oracle_worker, args=(b, ROOT, path, N_INNER, LAM_V, steps), daemon=True)
                pr.start()
                procs.append(pr)
                conns.append(a)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        for c in conns:
            assert c.recv() == "ready"
        stamps = [time.perf_counter()]
        for c in conns:
            c.send("go")
        fits = None
        while True:
            msgs = [c.recv() for c in conns]
            if isinstance(msgs[0], tuple):
                if msgs[0][0] == "done":
                    fits = msgs[0][1]
                    break
                stamps.append(time.perf_counter())     # every shard finished an iteration
                continue
            total = msgs[0].copy()
            for m in msgs[1:]:
                total += m
            for c in conns:
                c.send(total)
        for pr in procs:
            pr.join(timeout=60)
    return list(np.diff(stamps)), fits, cores


def oracle_pool_leg(X, init, n_sample, steps=1, warmup=0, seed=0):
    """cpu_baseline: iterations of the full-K workload per second from the oracle timed on a
    random sample of n_sample subjects (time per sampled iteration scaled by K/n)."""
    Xs, init_s = sample_subjects(X, init, n_sample, seed)
    secs, fits, cores = oracle_pool_run(Xs, init_s, warmup + steps)
    per_step = float(np.mean(secs[warmup:]))
    return {"value": (Xs.K / X.K) / per_step, "unit": "iter/s", "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{Xs.K} of {X.K} random subjects ({Xs.S} visits, {Xs.nnz} nnz), {steps} timed outer "
                      f"iteration(s) x {N_INNER} inner after {warmup} untimed; numpy FP64 oracle, subjects in "
                      f"{cores} contiguous nnz-balanced shards, one process per core (1 BLAS thread each), "
                      f"partial sums added by the parent; {per_step:.2f} s per sampled iteration scaled by "
                      f"K/{Xs.K}",
            "seconds_per_sampled_iteration": per_step}


# ---------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")
        self.index = index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([float(r[1]) for r in rows])
        mx = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        load = sm[sm > 0.5 * mx] if (sm > 0.5 * mx).any() else sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------------

def kernel_breakdown(h, P, Xd, R, H, V, W, reps=2):
    """Time each step of one outer iteration with CUDA events on the handle's stream."""
    torch = h.torch
    stream = h.stream
    K, J = Xd.K, Xd.J
    H, V, W = H.clone(), V.clone(), W.clone()
    DH, DV, DW = torch.zeros_like(H), torch.zeros_like(V), torch.zeros_like(W)
    names = ["procrustes+F_H", "grams+chol+admm H", "admm W (fused F_W)", "mttkrp V (+U^T U)",
             "admm V", "fit"]
    acc = {n: 0.0 for n in names}
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record(stream)
        st = h.procrustes(Xd, R, H, V, W, want_fh=True)
        ev[1].record(stream)
        gW, gV = h.gram(W), h.gram(V)
        h.admm_step(st["F_H"], gW, gV, N_INNER, "none", 0.0, H, DH)
        ev[2].record(stream)
        gH = h.gram(H)
        h.admm_w_fused(st, H, gH, gV, N_INNER, "nonneg", 0.0, W, DW)
        ev[3].record(stream)
        FV, UtU = h.mttkrp("V", Xd, R, st, H=H, W=W, want_utu=True)
        ev[4].record(stream)
        gW = h.gram(W)
        h.admm_step(FV, gH, gW, N_INNER, "l1", LAM_V, V, DV)
        ev[5].record(stream)
        h.fit_value(Xd, R, V, FV, UtU)
        ev[6].record(stream)
        h.sync()
        for i, n in enumerate(names):
            acc[n] += ev[i].elapsed_time(ev[i + 1])
    return {n: acc[n] / reps for n in names}


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_procrustes_step_dram_ehr_K100k_J1500_R40.txt")


def procrustes_traffic(K):
    """DRAM bytes (read + write) of one Procrustes step over K subjects, from the committed
    ncu summary of the same kernels on the K = 100,000 workload, scaled by the number of
    subjects (the workload draws subjects independently, so traffic grows in proportion);
    None when k_procrustes.cu changed since the counters were taken."""
    try:
        with open(TRAFFIC_PROFILE) as f:
            lines = f.read().splitlines()
        with open(os.path.join(ROOT, "paper_1803_04572_gb300", "csrc", "k_procrustes.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if "=" in ln and not ln.lstrip().startswith("#"):
            k, v = ln.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256") != sha or "dram_bytes_per_step" not in kv:
        return None
    return float(kv["dram_bytes_per_step"]) * K / float(kv["subjects"])


PROCRUSTES_KERNELS = ["k_tall_qr", "k_tall_jacobi", "k_tall_pass2", "k_procrustes_warp", "k_fh_stream4",
                      "k_reduce_partials"]


def procrustes_work(X, R):
    """Algorithmic FLOPs of the Procrustes step (a1-a3) by the accounting of the method:
    one pass over X forming P_k = X_k V (2 N R) and the R x R (or dual m_k x m_k) eigen
    problem of every subject at about 50 m_k^3 flops (m_k = min(I_k, R))."""
    m = np.minimum(np.diff(X.subj_ptr), R).astype(np.float64)
    return 2.0 * X.nnz * R + 50.0 * float(np.sum(m ** 3))


def iteration_bytes(X, R, count_bytes=2):
    """Algorithmic bytes of one outer iteration (implicit-Y schedule): two passes over X
    (column index + count per nonzero, row and subject pointers), the S_k and T_k round
    trips (K R(R+1)/2 and K R^2 reals, written and read) and W's state (Zbar_W, D_W read
    and written); V, H, F_H, F_V stay in L2."""
    B_X = X.nnz * (4 + count_bytes) + 4 * (X.S + 1) + 8 * (X.K + 1)
    B_S = 2 * 4 * X.K * R * (R + 1) / 2
    B_T = 2 * 4 * X.K * R * R
    B_W = 4 * 4 * X.K * R
    return float(2 * B_X + B_S + B_T + B_W)


def procrustes_roofline(h, P, Xd, X, R, H, V, W, peaks, reps=3):
    """The dominant step, the Procrustes step (six kernels: the tall QR, Jacobi and second
    pass, the small-subject warp kernel, the F_H stream and its reduction), timed as
    standalone copa_procrustes calls with CUDA events on the handle's stream; achieved =
    algorithmic FLOPs / time against the FP32 unit-count peak (plain ALU work)."""
    torch = h.torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.procrustes(Xd, R, H, V, W, want_fh=True)
    h.sync()
    e0.record(h.stream)
    for _ in range(reps):
        h.procrustes(Xd, R, H, V, W, want_fh=True)
    e1.record(h.stream)
    h.sync()
    ms = e0.elapsed_time(e1) / reps
    work = procrustes_work(X, R)
    achieved = work / (ms * 1e-3) / 1e12
    tally = 2.0 * h.procrustes_work()
    key = "fp32_tflops" if h.precision == "mixed" else "fp64_tflops"
    peak = peaks[key]
    return ms, {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": procrustes_traffic(X.K),
                "kernel": "Procrustes step: " + ", ".join(PROCRUSTES_KERNELS),
                "work_flop_per_launch": work,
                "work_rule": "2 N R (X pass) + 50 sum_k min(I_k,R)^3 (eigen), per launch",
                "ms_per_launch": ms,
                "peak_source": peaks[key.replace("tflops", "source")],
                "kernel_tally": {"flop_per_launch": tally, "achieved": tally / (ms * 1e-3) / 1e12,
                                 "note": "multiply-adds the kernels count for the rows, QR, Jacobi "
                                         "(textbook Hestenes count) and products, x2"}}


def fit_history(h, P, X, init, n_outer, val_dtype):
    """n_outer outer iterations from init on a fresh device copy; (FIT history, ms)."""
    torch = h.torch
    Xd = P.DeviceTensor.from_host(X, h.device, val_dtype)
    H, V, W = (torch.as_tensor(a, dtype=h.dtype, device=h.device) for a in init)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.sync()
    e0.record(h.stream)
    hist = h.fit(Xd, P.Options(R_RANK, n_outer=n_outer, n_inner=N_INNER, c_H="none", c_W="nonneg", c_V="l1",
                               lam_V=LAM_V, use_graph=True), H, V, W)
    e1.record(h.stream)
    h.sync()
    ms = e0.elapsed_time(e1)
    del Xd, H, V, W
    return [float(x) for x in hist], ms


def nccl_sum(t, stream):
    """All-reduce (sum) of a sharded fit's partial sums, ordered on the handle's stream."""
    import torch
    import torch.distributed as dist
    with torch.cuda.stream(stream):
        dist.all_reduce(t)


def gpu_leg(args, X, init, rank, world):
    import torch
    import paper_1803_04572_gb300 as P
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    h = P.Copa(dev, args.precision)
    R = R_RANK
    vd = "bf16" if args.precision == "mixed" else "f64"
    H0, V0, W0 = init
    Xl = X
    if world > 1:
        # one shard of contiguous, nnz-balanced subjects per GPU; H and V replicated, the
        # sums completed by an NCCL all-reduce per mode update
        bounds = P.partition(X.subj_ptr, X.row_ptr, world)
        Xl = X.subset(np.arange(bounds[rank], bounds[rank + 1]))
        W0 = W0[bounds[rank]:bounds[rank + 1]]
        h.set_allreduce(nccl_sum, X.J, R)
    Xd = P.DeviceTensor.from_host(Xl, h.device, vd)
    h.validate(Xd)
    H, V, W = (torch.as_tensor(a, dtype=h.dtype, device=h.device) for a in (H0, V0, W0))
    DH, DV, DW = torch.zeros_like(H), torch.zeros_like(V), torch.zeros_like(W)
    mk = lambda n: P.Options(R, n_outer=n, n_inner=N_INNER, c_H="none", c_W="nonneg", c_V="l1",
                             lam_V=LAM_V, use_graph=True)
    # the launch schedule for this tensor's size distribution (timed once, untimed here)
    tuned = None
    if not args.no_tune:
        t0 = time.perf_counter()
        tuned = h.tune(Xd, R, H, V, W)
        tuned["tuning_s"] = time.perf_counter() - t0
    # warm-up (W outer iterations, untimed)
    h.fit(Xd, mk(args.warmup), H, V, W, DH, DV, DW)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = Clocks(dev)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(h.stream)
    hist = h.fit(Xd, mk(args.steps), H, V, W, DH, DV, DW)
    e1.record(h.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = h.fit_launches()
    clocks = clk.stop()
    if world > 1:
        t = torch.tensor([ms], device=h.device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    out = {"ms_total": ms, "fit_last": float(hist[-1]), "fit_hist": [float(x) for x in hist], "clocks": clocks,
           "launches": launches, "autotune": tuned}
    if rank == 0 and world == 1:
        out["breakdown_ms"] = kernel_breakdown(h, P, Xd, R, H, V, W)
        out["proc_ms"], out["roofline"] = procrustes_roofline(h, P, Xd, X, R, H, V, W, PEAKS)
        out["sparsity_V"] = float((V == 0).double().mean().item())
    # e2e: the public host-buffer entry point, H2D of the step's inputs and D2H of the result
    if not args.no_e2e:
        pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()
        Xh = type("Xh", (), {})()
        Xh.K, Xh.J = Xl.K, Xl.J
        # the counts as bf16 (exact for integers <= 256), as the device tensor holds them
        arr = [pin(Xl.subj_ptr, np.int64), pin(Xl.row_ptr, np.int64), pin(Xl.col, np.int32),
               pin(P.bf16_bits(Xl.val), np.uint16)]
        Xh.subj_ptr, Xh.row_ptr, Xh.col, Xh.val = (a.numpy() for a in arr)
        nd = np.float32 if args.precision == "mixed" else np.float64
        fac = [pin(a, nd) for a in (H0, V0, W0)]
        duals = [pin(np.zeros_like(a), nd) for a in (H0, V0, W0)]
        Hn, Vn, Wn = (f.numpy() for f in fac)
        DHn, DVn, DWn = (d.numpy() for d in duals)
        # warm-up: both sets of staging buffers allocated, the copy path exercised
        for _ in range(2):
            h.stage_host(Xh, val_dtype="bf16")
        for _ in range(2):
            h.fit_host(Xh, mk(1), Hn, Vn, Wn, DHn, DVn, DWn, val_dtype="bf16")
        if world > 1:
            torch.distributed.barrier()
        # each step's X is copied from pinned host memory inside the timed region: the
        # first by its own call, every later one beside the step before it (queued by
        # copa_stage_host, issued by that step's call after its own copies); the factors
        # and duals are copied in and out by each call
        t0 = time.perf_counter()
        h.stage_host(Xh, val_dtype="bf16")
        for s in range(args.e2e_steps):
            if s + 1 < args.e2e_steps:
                h.stage_host(Xh, val_dtype="bf16")
            h.fit_host(Xh, mk(1), Hn, Vn, Wn, DHn, DVn, DWn, val_dtype="bf16")
        dt = (time.perf_counter() - t0) / args.e2e_steps
        if world > 1:
            t = torch.tensor([dt], device=h.device)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        h2d = sum(a.numel() * a.element_size() for a in arr) + sum(a.nbytes for a in (Hn, Vn, Wn, DHn, DVn, DWn))
        d2h = sum(a.nbytes for a in (Hn, Vn, Wn, DHn, DVn, DWn)) + 8
        out["e2e"] = {"value": 1.0 / dt, "unit": "iter/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h),
                      "note": "copa_fit_host, one outer iteration per call, X (bf16 counts) and state from "
                              "pinned host memory; the X of step s+1 is copied (queued by copa_stage_host) "
                              "beside step s" + (" (per rank: its shard; max over ranks)" if world > 1 else "")}
    if world > 1:
        h.set_allreduce(None)
    return out, h, P


def fit_gap_leg(args, X, init, h):
    """The mixed form against the FP64 form of the same kernels at C3, and against the
    oracle on a subject subsample: the FIT after each of 10 outer iterations x 20 inner
    from the same initialisation (equal iterations, so equal work)."""
    import paper_1803_04572_gb300 as P
    n = args.gap_outer
    hist32, ms32 = fit_history(h, P, X, init, n, "bf16")
    h64 = P.Copa(h.device.index, "fp64")
    hist64, ms64 = fit_history(h64, P, X, init, n, "f64")
    plain = None
    if args.plain_outer > 0:
        # the plain per-subject FP64 form (block per subject, FP64 Gram eigendecomposition,
        # explicit Y, unfused launches, no graph) from the same initialisation
        import torch
        npl = min(args.plain_outer, n)
        Xd = P.DeviceTensor.from_host(X, h64.device, "f64")
        Hp, Vp, Wp = (torch.as_tensor(a, dtype=torch.float64, device=h64.device) for a in init)
        h64.sync()
        t0 = time.perf_counter()
        hp = h64.fit_plain(Xd, P.Options(R_RANK, n_outer=npl, n_inner=N_INNER, c_H="none", c_W="nonneg", c_V="l1",
                                         lam_V=LAM_V), Hp, Vp, Wp)
        h64.sync()
        sp = time.perf_counter() - t0
        del Xd, Hp, Vp, Wp
        plain = {"outer_iterations": npl, "fit": [float(x) for x in hp], "iters_per_s": npl / sp,
                 "fit_gap_vs_mixed_max": float(np.max(np.abs(np.array(hp) - np.array(hist32[:npl])))),
                 "mixed_speedup": (1000.0 * n / ms32) / (npl / sp),
                 "note": "copa_fit_plain: one block per subject, FP64 Gram eigendecomposition, explicit Y, "
                         "unfused launches, no graph; host-timed including its set-up"}
    h64.close()
    res = {"outer_iterations": n, "n_inner": N_INNER,
           "fit_mixed": hist32, "fit_fp64": hist64,
           "fit_gap_vs_fp64_max": float(np.max(np.abs(np.array(hist32) - np.array(hist64)))),
           "mixed_iters_per_s": 1000.0 * n / ms32, "fp64_iters_per_s": 1000.0 * n / ms64,
           "note": "same kernels, FP64 handle: every step in double (the Procrustes step by the "
                   "block or lane kernels in FP64)",
           "plain_fp64": plain}
    if args.gap_oracle_sample > 0:
        Xs, init_s = sample_subjects(X, init, args.gap_oracle_sample, seed=5)
        hs, _ = fit_history(h, P, Xs, init_s, n, "bf16")
        _, fo, cores = oracle_pool_run(Xs, init_s, n)
        res["oracle_subsample"] = {"subjects": Xs.K, "fit_mixed": hs, "fit_oracle": [float(x) for x in fo],
                                   "fit_gap_vs_oracle_max": float(np.max(np.abs(np.array(hs) - np.array(fo)))),
                                   "oracle_cores": cores}
    return res


def config_leg(args):
    """One line for a configuration other than the headline one (1 GPU)."""
    import torch
    import synth
    import paper_1803_04572_gb300 as P
    cfg = OTHER_WORKLOADS[args.workload]
    R = cfg["R"] or args.rank
    t = time.time()
    X = getattr(synth, cfg["gen"])()
    gen_s = time.time() - t
    H0, V0, W0 = synth.init_factors(X.K, X.J, R)
    h = P.Copa(0, args.precision)
    vd = "bf16" if args.precision == "mixed" else "f64"
    Xd = P.DeviceTensor.from_host(X, h.device, vd)
    h.validate(Xd)
    H, V, W = (torch.as_tensor(a, dtype=h.dtype, device=h.device) for a in (H0, V0, W0))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    extra = {}
    if cfg.get("backward"):
        metric = f"backward passes/sec (K={X.K // 1000}k, J={X.J}, R={R})"
        st = h.procrustes(Xd, R, H, V, W, want_pi=True)
        for _ in range(args.warmup):
            h.loss_grad(Xd, R, st, H, V, W)
        h.sync()
        clk = Clocks(0)
        clk.start()
        e0.record(h.stream)
        for _ in range(args.steps):
            loss, gH, gV, gW = h.loss_grad(Xd, R, st, H, V, W)
        e1.record(h.stream)
        h.sync()
        extra["loss"] = float(loss.cpu()[0])
        launches = None
    elif cfg.get("sweep"):
        G = cfg["sweep"]
        lams = list(np.geomspace(0.1, 10.0, G))
        days = torch.as_tensor(X.days, dtype=torch.float64, device=h.device)
        Xfit, _ = h.smooth(Xd, days, 7, 3, out_dtype="f64" if args.precision == "fp64" else "f32")
        xn2 = float(np.sum(np.asarray(X.val, dtype=np.float64) ** 2))
        opts = [P.Options(R, n_outer=args.steps, n_inner=cfg["n_inner"], c_V="l1", lam_V=float(l), x_norm2=xn2)
                for l in lams]
        fresh = lambda: [tuple(torch.as_tensor(a, dtype=h.dtype, device=h.device) for a in (H0, V0, W0))
                         for _ in lams]
        h.fit_batch(Xfit, [P.Options(**dict(o.__dict__, n_outer=args.warmup)) for o in opts], fresh())   # warm-up
        for o in opts:
            st0 = fresh()[0]
            h.fit(Xfit, P.Options(**dict(o.__dict__, n_outer=args.warmup)), *st0)
        h.sync()
        clk = Clocks(0)
        clk.start()
        states = fresh()
        h.sync()
        e0.record(h.stream)
        hists = h.fit_batch(Xfit, opts, states)
        e1.record(h.stream)
        h.sync()
        ms_batch = e0.elapsed_time(e1)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        seq_states = fresh()
        h.sync()
        t0.record(h.stream)
        for o, st0 in zip(opts, seq_states):
            h.fit(Xfit, o, *st0)
        t1.record(h.stream)
        h.sync()
        ms_seq = t0.elapsed_time(t1)
        work = G * args.steps
        line = {"metric": f"sweep fit-iterations/sec ({G} fits, l1 weight grid, K={X.K // 1000}k, J={X.J}, R={R}, "
                          "smoothed)", "unit": "1/s", "higher_is_better": True, "data": "synthetic",
                "config": {"workload": args.workload, "K": X.K, "J": X.J, "R": R, "fits": G,
                           "lam_V": [float(l) for l in lams], "precision": args.precision, "parallelism": "1 GPU"},
                "value": 1000.0 * work / ms_batch, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_batch / args.steps, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE[args.precision], "clocks": clk.stop(), "gpu_launches": None,
                "sequential": {"value": 1000.0 * work / ms_seq, "ms_total": ms_seq,
                               "note": "the same fits as separate copa_fit calls, one after the other"},
                "batched_ms_total": ms_batch, "fit_last": [float(x[-1]) for x in hists],
                "sparsity_V": [float((st[1] == 0).double().mean().item()) for st in states],
                "generation_s": gen_s}
        print(json.dumps(line))
        return
    else:
        Xfit, xn2 = Xd, 0.0
        if cfg.get("smooth"):
            days = torch.as_tensor(X.days, dtype=torch.float64, device=h.device)
            h.sync()
            t0 = time.perf_counter()
            Xfit, _ = h.smooth(Xd, days, 7, 3, out_dtype="f64" if args.precision == "fp64" else "f32")
            h.sync()
            extra["smoothing_setup_ms"] = (time.perf_counter() - t0) * 1e3
            xn2 = float(np.sum(np.asarray(X.val, dtype=np.float64) ** 2))
        metric = (f"AO-ADMM outer iters/sec (K={X.K // 1000}k, J={X.J}, R={R}"
                  + (", smoothed)" if cfg.get("smooth") else ")"))
        DH, DV, DW = torch.zeros_like(H), torch.zeros_like(V), torch.zeros_like(W)
        mk = lambda n: P.Options(R, n_outer=n, n_inner=cfg["n_inner"], c_H="none", c_W="nonneg", c_V="l1",
                                 lam_V=LAM_V, x_norm2=xn2, use_graph=True)
        h.fit(Xfit, mk(args.warmup), H, V, W, DH, DV, DW)
        h.sync()
        clk = Clocks(0)
        clk.start()
        e0.record(h.stream)
        hist = h.fit(Xfit, mk(args.steps), H, V, W, DH, DV, DW)
        e1.record(h.stream)
        h.sync()
        launches = h.fit_launches()
        extra["fit_last"] = float(hist[-1])
    ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": metric, "unit": "1/s", "higher_is_better": True, "data": "synthetic",
            "config": {"workload": args.workload, "K": X.K, "J": X.J, "R": R, "nnz": X.nnz, "visits": X.S,
                       "precision": args.precision, "parallelism": "1 GPU"},
            "value": 1000.0 / ms, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision],
            "clocks": clk.stop(), "gpu_launches": launches, "generation_s": gen_s}
    line.update(extra)
    print(json.dumps(line))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = json.load(open(p)) if os.path.exists(p) else {}
    # Plain-ALU peaks from the unit counts at the maximum SM clock (2070 MHz): 152 SMs x
    # 128 FP32 FMA/clk x 2 = 80.5 TFLOP/s; FP64 2 FMA/clk/SM -> 1.26 TFLOP/s (an FMA-loop
    # probe on this machine's GB300 measured 69.4 and 1.19 TFLOP/s).
    return {"hbm_gbs": d.get("hbm_gbs", 6800.0),
            "fp32_tflops": 152 * 128 * 2 * 2.070e9 / 1e12,
            "fp32_source": "unit count 152 SM x 128 FMA/clk at 2070 MHz (FMA-loop probe: 69.4)",
            "fp64_tflops": 152 * 2 * 2 * 2.070e9 / 1e12,
            "fp64_source": "unit count 152 SM x 2 DFMA/clk at 2070 MHz (DFMA-loop probe: 1.19)",
            "hbm_source": "of measured" if "hbm_gbs" in d else "of fallback"}


PEAKS = load_peaks()


DTYPE = {"mixed": "f32 bulk + f32 one-sided-Jacobi Procrustes (bf16 counts), "
                  "f64 Gram/Cholesky/U^T U/FIT sums",
         "fp64": "f64"}


def main():
    args = parse()
    if args.workload != WORKLOAD:
        config_leg(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if args.impl == "reference":
            if rank != 0:
                return
        else:
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
    X, init, gen_s = make_data(args.K)
    base = {"metric": METRIC, "unit": "iter/s", "higher_is_better": True, "data": "synthetic",
            "config": {"workload": WORKLOAD, "K": X.K, "J": X.J, "R": R_RANK, "nnz": X.nnz, "visits": X.S,
                       "n_inner": N_INNER, "constraints": "H none, W nonneg, V l1 (lambda 1)",
                       "l2": "inputs larger than L2 (X is %.2f GB)" % (X.nnz * 6 / 1e9)}}
    if args.impl == "reference":
        ref = oracle_pool_leg(X, init, args.cpu_sample, steps=args.steps, warmup=args.warmup)
        line = dict(base, impl="reference", value=ref["value"], n_gpus=args.gpus, steps=args.steps,
                    warmup=args.warmup, ms_per_step=1000.0 / ref["value"], dtype="f64",
                    scaling="weak", vs_baseline=None, cpu_baseline=ref,
                    e2e={"value": ref["value"], "unit": "iter/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0})
        line["config"]["parallelism"] = f"host cores x{ref['cores']} (oracle)"
        print(json.dumps(line))
        return
    res, h, P = gpu_leg(args, X, init, rank, world)
    if rank != 0:
        return
    ms_step = res["ms_total"] / args.steps
    value = 1000.0 / ms_step          # outer iterations of the whole K-subject fit per second
    line = dict(base, value=value, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_step, scaling="strong" if world > 1 else "weak", vs_baseline=None,
                dtype=DTYPE[args.precision], clocks=res["clocks"], gpu_launches=res["launches"],
                fit_last=res["fit_last"], generation_s=gen_s, autotune=res["autotune"])
    if world == 1:
        B = iteration_bytes(X, R_RANK)
        ach = B / (ms_step * 1e-3) / 1e9
        line.update(roofline=res["roofline"], sparsity_V=res["sparsity_V"], breakdown_ms=res["breakdown_ms"],
                    hbm={"bytes_per_iteration": B, "achieved": ach, "peak": PEAKS["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / PEAKS["hbm_gbs"], "peak_source": PEAKS["hbm_source"],
                         "rule": "2 passes over X (int32 column + bf16 count per nonzero, pointers) + "
                                 "S_k and T_k round trips + W state, per outer iteration"})
    line["config"]["parallelism"] = (f"{world} GPUs, contiguous nnz-balanced subject shards, NCCL all-reduce "
                                     f"of F_H, F_V and the Grams per mode update" if world > 1 else "1 GPU")
    line["config"]["precision"] = args.precision
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    if world == 1 and not args.no_fit_gap and args.precision == "mixed":
        line["fit_gap"] = fit_gap_leg(args, X, init, h)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_pool_leg(X, init, args.cpu_sample)
    print(json.dumps(line))


if __name__ == "__main__":
    main()

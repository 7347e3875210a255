"""Benchmark of the COPA AO-ADMM outer iteration on GB300.

Workload: synthetic EHR-shaped tensor with K = 500,000 subjects, J = 1,500 features,
I_k ~ Pareto(1.5) clipped to [1, 2000] (mean ~40 visits), 1 + Poisson(4) Zipf(1.1) codes
per visit (~1e8 nonzeros), integer counts U{1..50} stored as bf16; rank R = 40,
non-negative W, l1 on V (lambda = 1), 20 ADMM iterations per factor. One step = one
outer iteration (Procrustes for every subject, then H, W, V by ADMM, then the FIT).

Prints ONE JSON line (rank 0). `--impl reference` times the FP64 CPU oracle instead, on
a bounded random sample of subjects, scaled to the full K.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
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
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--K", type=int, default=500_000, help="subjects (smaller for quick runs)")
    ap.add_argument("--cpu-sample", type=int, default=6000, help="subjects in the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
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
# CPU oracle leg (a bounded sample, single thread, in a child process)
# ---------------------------------------------------------------------------------

_ORACLE_CHILD = r"""
import sys, time, json, numpy as np
sys.path.insert(0, sys.argv[1])
import synth
from oracle import copa_oracle as O
d = np.load(sys.argv[2])
X = synth.SparseTensor(int(d["K"]), int(d["J"]), d["subj_ptr"], d["row_ptr"], d["col"], d["val"])
st = O.State.from_init(d["H"], d["V"], d["W"])
opt = O.Options(n_inner=int(d["n_inner"]), c_H=O.NONE, c_W=O.NONNEG, c_V=O.L1, lam_V=float(d["lam"]))
steps = int(d["steps"])
t = time.perf_counter()
for _ in range(steps):
    rec = O.outer_iteration(X, st, opt)
    st = rec.state
dt = time.perf_counter() - t
print(json.dumps({"seconds": dt, "steps": steps}))
"""


def oracle_leg(X, init, n_sample, steps=1, seed=0):
    rng = np.random.default_rng(seed)
    ks = np.sort(rng.choice(X.K, size=min(n_sample, X.K), replace=False))
    Xs = X.subset(ks)
    H0, V0, W0 = init
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sample.npz")
        np.savez(path, K=Xs.K, J=Xs.J, subj_ptr=Xs.subj_ptr, row_ptr=Xs.row_ptr, col=Xs.col, val=Xs.val,
                 H=H0, V=V0, W=W0[ks], n_inner=N_INNER, lam=LAM_V, steps=steps)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        out = subprocess.run([sys.executable, "-c", _ORACLE_CHILD, ROOT, path], env=env,
                             capture_output=True, text=True, check=True)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    per_step = res["seconds"] / res["steps"]
    iters_per_s = (Xs.K / X.K) / per_step      # full-K outer iterations per second
    return {"value": iters_per_s, "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": f"{Xs.K} of {X.K} random subjects ({Xs.S} visits, {Xs.nnz} nnz), "
                      f"{res['steps']} outer iteration(s) x {N_INNER} inner, numpy FP64, 1 thread; "
                      f"{per_step:.2f} s per sampled iteration scaled by K/{Xs.K}"}


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


def procrustes_roofline(h, P, Xd, X, R, H, V, W, peaks, reps=3):
    """Average duration of the Procrustes launch (the dominant kernel), timed with CUDA
    events on the handle's stream, and its algorithmic work: the multiply-adds the kernel
    tallies for the rows, QR, Jacobi rotations and products it performs (2 FLOP each)."""
    torch = h.torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = h.procrustes(Xd, R, H, V, W, want_fh=True)
    h.sync()
    e0.record(h.stream)
    for _ in range(reps):
        st = h.procrustes(Xd, R, H, V, W, want_fh=True)
    e1.record(h.stream)
    h.sync()
    ms = e0.elapsed_time(e1) / reps
    fma = h.procrustes_work()
    achieved = 2.0 * fma / (ms * 1e-3) / 1e12
    key = "fp32_tflops" if h.precision == "mixed" else "fp64_tflops"
    peak = peaks[key]
    return ms, {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": procrustes_traffic(X.K), "kernel": "k_procrustes",
                "work_fma_per_launch": fma, "peak_source": peaks[key.replace("tflops", "source")]}


def gpu_leg(args, X, init, rank, world):
    import torch
    import paper_1803_04572_gb300 as P
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    h = P.Copa(dev, args.precision)
    R = R_RANK
    vd = "bf16" if args.precision == "mixed" else "f64"
    Xd = P.DeviceTensor.from_host(X, h.device, vd)
    h.validate(Xd)
    H0, V0, W0 = init
    H, V, W = (torch.as_tensor(a, dtype=h.dtype, device=h.device) for a in (H0, V0, W0))
    DH, DV, DW = torch.zeros_like(H), torch.zeros_like(V), torch.zeros_like(W)
    mk = lambda n: P.Options(R, n_outer=n, n_inner=N_INNER, c_H="none", c_W="nonneg", c_V="l1",
                             lam_V=LAM_V, use_graph=True)
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
           "launches": launches}
    if rank == 0:
        out["breakdown_ms"] = kernel_breakdown(h, P, Xd, R, H, V, W)
        out["proc_ms"], out["roofline"] = procrustes_roofline(h, P, Xd, X, R, H, V, W, PEAKS)
        out["sparsity_V"] = float((V == 0).double().mean().item())
    # e2e: the public host-buffer entry point, H2D of the step's inputs and D2H of the result
    if not args.no_e2e and rank == 0:
        pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()
        Xh = type("Xh", (), {})()
        Xh.K, Xh.J = X.K, X.J
        arr = [pin(X.subj_ptr, np.int64), pin(X.row_ptr, np.int64), pin(X.col, np.int32),
               pin(X.val, np.float32)]
        Xh.subj_ptr, Xh.row_ptr, Xh.col, Xh.val = (a.numpy() for a in arr)
        nd = np.float32 if args.precision == "mixed" else np.float64
        fac = [pin(a, nd) for a in (H0, V0, W0)]
        duals = [pin(np.zeros_like(a), nd) for a in (H0, V0, W0)]
        Hn, Vn, Wn = (f.numpy() for f in fac)
        DHn, DVn, DWn = (d.numpy() for d in duals)
        h.fit_host(Xh, mk(1), Hn, Vn, Wn, DHn, DVn, DWn)     # warm-up
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            h.fit_host(Xh, mk(1), Hn, Vn, Wn, DHn, DVn, DWn)
        dt = (time.perf_counter() - t0) / args.e2e_steps
        h2d = sum(a.numel() * a.element_size() for a in arr) + sum(a.nbytes for a in (Hn, Vn, Wn, DHn, DVn, DWn))
        d2h = sum(a.nbytes for a in (Hn, Vn, Wn, DHn, DVn, DWn)) + 8
        out["e2e"] = {"value": 1.0 / dt, "unit": "iter/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h),
                      "note": "copa_fit_host, one outer iteration per call, X and state from pinned host memory"}
    return out


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
            "dtype": "f32 bulk (bf16 counts), f64 Gram/eigen/Cholesky/FIT" if args.precision == "mixed" else "f64",
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
        ref = oracle_leg(X, init, args.cpu_sample, steps=max(1, args.steps // max(1, args.steps)))
        line = dict(base, impl="reference", value=ref["value"], n_gpus=args.gpus, steps=args.steps,
                    warmup=args.warmup, ms_per_step=1000.0 / ref["value"], dtype="f64",
                    scaling="weak", vs_baseline=None, cpu_baseline=ref,
                    e2e={"value": ref["value"], "unit": "iter/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 0})
        print(json.dumps(line))
        return
    res = gpu_leg(args, X, init, rank, world)
    if rank != 0:
        return
    ms_step = res["ms_total"] / args.steps
    value = world * 1000.0 / ms_step
    line = dict(base, value=value, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms_step, scaling="weak", vs_baseline=None,
                dtype="f32 bulk (bf16 counts), f64 Gram/eigen/Cholesky/FIT" if args.precision == "mixed" else "f64",
                roofline=res["roofline"], clocks=res["clocks"],
                gpu_launches=res["launches"],
                fit_last=res["fit_last"], sparsity_V=res["sparsity_V"], breakdown_ms=res["breakdown_ms"],
                generation_s=gen_s)
    line["config"]["parallelism"] = "replicas x%d (subjects per replica fixed)" % world if world > 1 else "1 GPU"
    line["config"]["precision"] = args.precision
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_leg(X, init, args.cpu_sample)
    print(json.dumps(line))


if __name__ == "__main__":
    main()

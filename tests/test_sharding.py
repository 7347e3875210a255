"""Subject sharding of the outer iteration (Sec. 3.2: the Procrustes loop is independent
per subject, every other step sees the subjects only through sums).

CPU: libcopa's partitioner (host code) against brute force; the oracle's sharded
iteration with one shard against the plain oracle; two gloo ranks against the
single-process oracle. GPU: two shards of one fit on one GPU, run by two host threads
whose all-reduce is a host-side sum behind a barrier (no kernel waits on another), against
the unsharded fit."""
import os
import socket
import subprocess
import sys
import tempfile
import threading

import numpy as np
import pytest

import synth
from oracle import copa_oracle as O
from oracle import sharded as OS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_OUTER = 3
OPT = O.Options(n_inner=6, c_H=O.NONE, c_W=O.NONNEG, c_V=O.L1, lam_V=0.5)


def CASE():
    X = synth.ehr_custom(60, 25, median=8, lo=1, hi=30, lam=2.0, cmax=10, seed=31)
    return X, synth.init_factors(X.K, X.J, 4)


def _P():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "copa_build", os.path.join(ROOT, "paper_1803_04572_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1803_04572_gb300 as P
    return P


def test_partition_is_nnz_balanced():
    """bounds[p] is the subject boundary whose nonzero prefix is closest to p N / n among
    the boundaries at or after bounds[p-1] (brute force), bounds are non-decreasing and
    cover [0, K]."""
    P = _P()
    rng = np.random.default_rng(0)
    tensors = [synth.ehr_custom(K, 10, median=5, lo=lo, hi=40, seed=s)
               for K, lo, s in [(1, 1, 0), (7, 0, 1), (50, 1, 2), (333, 0, 3)]]
    tensors.append(synth.ehr_tensor(4, 10, np.zeros(4, dtype=np.int64), 2.0, 5, 4))   # all empty
    for X in tensors:
        pre = X.row_ptr[X.subj_ptr]
        N = int(pre[-1])
        for n in (1, 2, 3, 7, X.K + 2):
            b = P.partition(X.subj_ptr, X.row_ptr, n)
            assert b[0] == 0 and b[-1] == X.K and np.all(np.diff(b) >= 0), b
            lo = 0
            for p in range(1, n):
                t = N * p / n
                best = min(abs(pre[k] - t) for k in range(lo, X.K + 1))
                assert abs(pre[b[p]] - t) == best, (X.K, n, p, b)
                lo = b[p]
    with pytest.raises(P.CopaError):
        P.partition(np.zeros(1, np.int64), np.zeros(1, np.int64), 0)
    del rng


def test_one_shard_is_the_oracle_iteration():
    X, init = CASE()
    st = O.State.from_init(*init)
    ss = OS.shard_state(st, 0, X.K)
    for _ in range(N_OUTER):
        rec = O.outer_iteration(X, st, OPT)
        ss, f = OS.outer_iteration(X, ss, OPT, lambda a: a)
        st = rec.state
        for a, b in ((st.H, ss.H), (st.V, ss.V), (st.W, ss.W), (st.DW, ss.DW)):
            np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-13)
        assert abs(f - O.fit_value(X, rec.Q, st.H, st.V, st.W)) < 1e-13


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_match_the_single_process_oracle():
    """world_size 2 over gloo on CPU: each rank holds its shard (libcopa's partition), the
    sums go through torch.distributed.all_reduce; H, V agree across ranks and with the
    single-process oracle, the W rows concatenate to its W, the FIT history matches."""
    _P()
    X, init = CASE()
    port = _free_port()
    with tempfile.TemporaryDirectory() as td:
        outs = [os.path.join(td, f"r{r}.npz") for r in range(2)]
        procs = []
        for r in range(2):
            env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                       PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]),
                       OMP_NUM_THREADS="1")
            procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "tests", "_shard_worker.py"), outs[r]],
                                          env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT))
        logs = []
        for p in procs:
            try:
                out, _ = p.communicate(timeout=240)
            except subprocess.TimeoutExpired:
                p.kill()
                out, _ = p.communicate()
            logs.append(out.decode(errors="replace"))
        assert all(p.returncode == 0 for p in procs), logs
        res = [dict(np.load(o)) for o in outs]
    st, hist, _ = O.fit(X, *init, OPT, N_OUTER)
    b = res[0]["bounds"]
    assert 0 < b[1] < X.K
    for r in range(2):
        np.testing.assert_array_equal(res[r]["bounds"], b)
        np.testing.assert_allclose(res[r]["H"], st.H, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(res[r]["V"], st.V, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(res[r]["fits"], hist, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(res[0]["H"], res[1]["H"])      # replicated: bitwise equal
    np.testing.assert_allclose(np.concatenate([res[0]["W"], res[1]["W"]]), st.W, rtol=1e-10, atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_shards_on_one_gpu_match_the_whole_fit(precision):
    """copa_fit as two shards of one fit on cuda:0 (two handles, two host threads, a host
    all-reduce behind a barrier) against copa_fit over all subjects."""
    import torch
    import paper_1803_04572_gb300 as P
    X = synth.ehr_custom(400, 70, median=12, lo=1, hi=80, lam=3.0, cmax=20, seed=33)
    R = 8
    H0, V0, W0 = synth.init_factors(X.K, X.J, R)
    vd = "f64" if precision == "fp64" else "bf16"
    opt = P.Options(R, n_outer=4, n_inner=8, c_V="l1", lam_V=0.5)
    h = P.Copa(0, precision)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=h.dtype, device=h.device)
    H, V, W = T(H0), T(V0), T(W0)
    hist = h.fit(P.DeviceTensor.from_host(X, h.device, vd), opt, H, V, W)
    bounds = P.partition(X.subj_ptr, X.row_ptr, 2)
    slots, barrier = [None, None], threading.Barrier(2, timeout=120)
    results, errors = [None, None], []

    def shard(r):
        try:
            hr = P.Copa(0, precision)

            def reduce_fn(t, stream):
                stream.synchronize()
                slots[r] = t.cpu()
                barrier.wait()
                total = slots[0] + slots[1]          # same order on both shards
                barrier.wait()
                with torch.cuda.stream(stream):
                    t.copy_(total.to(t.device))
                stream.synchronize()

            hr.set_allreduce(reduce_fn, X.J, R)
            Xr = X.subset(np.arange(bounds[r], bounds[r + 1]))
            Hr, Vr, Wr = T(H0), T(V0), T(W0[bounds[r]:bounds[r + 1]])
            hr_hist = hr.fit(P.DeviceTensor.from_host(Xr, hr.device, vd), opt, Hr, Vr, Wr)
            torch.cuda.synchronize()
            results[r] = (hr_hist, Hr.cpu().double().numpy(), Vr.cpu().double().numpy(), Wr.cpu().double().numpy())
        except Exception as e:   # noqa: BLE001
            errors.append(e)
            barrier.abort()

    th = [threading.Thread(target=shard, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errors, errors
    tol = 1e-10 if precision == "fp64" else 1e-5
    Hn, Vn, Wn = (a.cpu().double().numpy() for a in (H, V, W))
    for r in range(2):
        np.testing.assert_allclose(results[r][0], hist, rtol=0, atol=tol)
        np.testing.assert_allclose(results[r][1], Hn, rtol=tol, atol=tol * np.abs(Hn).max())
        np.testing.assert_allclose(results[r][2], Vn, rtol=tol, atol=100 * tol * np.abs(Vn).max())
    np.testing.assert_array_equal(results[0][1], results[1][1])   # H replicated bitwise
    np.testing.assert_allclose(np.concatenate([results[0][3], results[1][3]]), Wn, rtol=tol,
                               atol=100 * tol * np.abs(Wn).max())

"""The launch-schedule autotuner: its table logic on the host (no GPU) and, on the GPU,
that a tuned schedule changes only the speed of a fit, not its results."""
import os

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _P():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "copa_build", os.path.join(ROOT, "paper_1803_04572_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_1803_04572_gb300 as P
    return P


def test_tune_key_depends_on_rank_precision_and_size_distribution_only():
    P = _P()
    X = synth.ehr_K500k(K=20_000)
    sizes = np.diff(X.subj_ptr)
    k = P.tune_key(X.subj_ptr, 40, "mixed")
    perm = np.random.default_rng(0).permutation(sizes)          # same sizes, other order
    assert P.tune_key(np.concatenate([[0], np.cumsum(perm)]), 40, "mixed") == k
    other = synth.ehr_K500k(seed=3, K=20_000)                     # same distribution, other draw
    assert P.tune_key(other.subj_ptr, 40, "mixed") == k
    assert P.tune_key(X.subj_ptr, 20, "mixed") != k
    assert P.tune_key(X.subj_ptr, 40, "fp64") != k
    small = synth.ehr_custom(20_000, 50, median=5, lo=1, hi=20)   # another size distribution
    assert P.tune_key(small.subj_ptr, 40, "mixed") != k
    assert P.tune_key(np.zeros(1, np.int64), 40, "mixed") == P.tune_key(np.zeros(1, np.int64), 40, "mixed")


def test_tune_table_store_and_lookup():
    P = _P()
    key = P.tune_key(np.array([0, 3, 10, 10, 41], np.int64), 7, "mixed")
    assert P.tune_lookup(key) is None
    P.tune_store(key, split=5, blocks_per_sm=2, fv_path=1, ms=1.5)
    assert P.tune_lookup(key) == {"split": 5, "blocks_per_sm": 2, "fv_path": 1, "ms": 1.5}
    P.tune_store(key, split=7)
    assert P.tune_lookup(key)["split"] == 7 and P.tune_lookup(key)["fv_path"] == 0
    with pytest.raises(P.CopaError):
        P.tune_store(key, split=0)
    P.tune_store(key, split=3, fv_path=2)
    assert P.tune_lookup(key)["fv_path"] == 2
    with pytest.raises(P.CopaError):
        P.tune_store(key, split=3, fv_path=3)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tuned_schedule_changes_speed_not_results(precision):
    """copa_tune picks a schedule from its candidates and stores it; a fit under the tuned
    schedule gives the FIT history of the default schedule (1e-10 FP64, 1e-5 mixed); a
    second copa_tune on another handle finds the stored choice without timing."""
    import torch
    import paper_1803_04572_gb300 as P
    X = synth.ehr_custom(3000, 200, median=20, lo=1, hi=150, lam=3.0, cmax=20, seed=61)
    R = 24
    init = synth.init_factors(X.K, X.J, R)
    vd = "f64" if precision == "fp64" else "bf16"
    opt = P.Options(R, n_outer=4, n_inner=8)
    h0 = P.Copa(0, precision)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=h0.dtype, device=h0.device)
    Xd = P.DeviceTensor.from_host(X, h0.device, vd)
    H, V, W = (T(a) for a in init)
    hist0 = h0.fit(Xd, opt, H, V, W)
    h1 = P.Copa(0, precision)
    H, V, W = (T(a) for a in init)
    choice = h1.tune(Xd, R, H, V, W, force=True)
    assert 1 <= choice["split"] <= min(R, 32) and choice["blocks_per_sm"] in (0, 2) and choice["ms"] > 0
    key = P.tune_key(X.subj_ptr, R, precision)
    assert P.tune_lookup(key) == choice
    hist1 = h1.fit(Xd, opt, H, V, W)
    np.testing.assert_allclose(hist1, hist0, rtol=0, atol=1e-10 if precision == "fp64" else 1e-5)
    # a forced split of 8 as well (the tall kernels take 9 <= I_k <= 24)
    h2 = P.Copa(0, precision)
    P.tune_store(key, split=8, blocks_per_sm=2, fv_path=1)
    assert h2.tune(Xd, R, H, V, W)["split"] == 8
    H, V, W = (T(a) for a in init)
    hist2 = h2.fit(Xd, opt, H, V, W)
    np.testing.assert_allclose(hist2, hist0, rtol=0, atol=1e-10 if precision == "fp64" else 1e-5)

"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/copa.h declares (no compute: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "copa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(copa_[A-Za-z_0-9]+)\s*\(", src)))


def _build():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "copa_build", os.path.join(ROOT, "paper_1803_04572_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def test_library_exports_every_declared_symbol():
    lib_path = _build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 15, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    _build()
    import paper_1803_04572_gb300 as P
    assert sorted(set(P.EXPORTED)) == _declared()


def test_device_tensor_sizes_from_arrays():
    """S is the number of visit rows (row_ptr has S + 1 entries), not K."""
    _build()
    import numpy as np
    import torch
    import paper_1803_04572_gb300 as P
    import synth
    X = synth.ehr_custom(7, 5, median=4, lo=2, hi=6, seed=1)
    t = lambda a, dt: torch.as_tensor(np.asarray(a, dtype=dt))
    d = P.DeviceTensor(X.K, X.J, t(X.subj_ptr, np.int64), t(X.row_ptr, np.int64), t(X.col, np.int32),
                       t(X.val, np.float32), "f32")
    assert (d.K, d.S, d.nnz) == (X.K, X.S, X.nnz)
    c = d.c()
    assert (c.K, c.J, c.S, c.nnz) == (X.K, X.J, X.S, X.nnz)


def test_host_tensor_sizes_from_arrays():
    _build()
    import paper_1803_04572_gb300 as P
    import synth
    X = synth.ehr_custom(9, 6, median=5, lo=2, hi=9, seed=2)
    tc, keep = P.host_tensor_c(X, "f32")
    assert (tc.K, tc.J, tc.S, tc.nnz) == (X.K, X.J, X.S, X.nnz)


def test_bf16_host_values():
    """bf16_bits gives the bf16 patterns of integer counts and refuses anything else; the
    host tensor for copa_fit_host takes them as val_dtype "bf16" and nothing wider."""
    import numpy as np
    import pytest
    _build()
    import paper_1803_04572_gb300 as P
    b = P.bf16_bits(np.array([1.0, 2.0, 50.0, 256.0, -3.0]))
    assert b.dtype == np.uint16
    assert list(b) == [0x3F80, 0x4000, 0x4248, 0x4380, 0xC040]
    with pytest.raises(ValueError):
        P.bf16_bits(np.array([1.5]))
    with pytest.raises(ValueError):
        P.bf16_bits(np.array([257.0]))
    X = type("Xh", (), {})()
    X.K, X.J = 1, 4
    X.subj_ptr, X.row_ptr = np.array([0, 1]), np.array([0, 2])
    X.col, X.val = np.array([0, 3]), b[:2]
    tc, _ = P.host_tensor_c(X, "bf16")
    assert tc.nnz == 2 and tc.val_dtype == P.VAL_DTYPE["bf16"]
    X.val = np.array([1.0, 2.0], dtype=np.float32)
    with pytest.raises(ValueError):
        P.host_tensor_c(X, "bf16")

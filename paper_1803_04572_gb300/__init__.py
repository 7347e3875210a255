"""Python binding of libcopa, the GB300 implementation of COPA's per-iteration hot path
(constrained PARAFAC2 by AO-ADMM, Afshar et al., arXiv 1803.04572).

Argument marshalling only: every step runs in the CUDA kernels of libcopa.so behind the
C ABI declared in include/copa.h. PyTorch supplies device memory and the stream. There
is no CPU fallback: importing this package fails if the library has not been built
(`python -m paper_1803_04572_gb300.build` or `__graft_entry__.build()`).
"""
from __future__ import annotations

import ctypes
import itertools
import os
from ctypes import POINTER, Structure, byref, c_double, c_int32, c_int64, c_void_p
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcopa.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcopa.so is not built ({LIB_PATH}); run paper_1803_04572_gb300/build.py")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NUMERIC, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_COMM = range(8)
PREC = {"mixed": 0, "fp64": 1}
CONSTRAINT = {"none": 0, "nonneg": 1, "l1": 2, "l0": 3}
VAL_DTYPE = {"f32": 0, "f64": 1, "bf16": 2}
MODE = {"H": 0, "V": 1, "W": 2}

EXPORTED = ["copa_create", "copa_destroy", "copa_last_error", "copa_sync", "copa_validate",
            "copa_procrustes", "copa_mttkrp", "copa_gram", "copa_admm_step", "copa_admm_w_fused",
            "copa_fit_value", "copa_fit", "copa_fit_host", "copa_smooth_plan",
            "copa_smooth_project", "copa_loss_grad", "copa_procrustes_work", "copa_gram_noalloc",
            "copa_fit_launches", "copa_debug_set", "copa_partition", "copa_set_allreduce", "copa_factor_U",
            "copa_fit_stats", "copa_fit_batch", "copa_tune", "copa_tune_key", "copa_tune_lookup",
            "copa_tune_store", "copa_fit_plain", "copa_forget_tensor", "copa_stage_host"]
KNOTS = {"uniform": 0, "quantile": 1}


class CopaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"copa error {code}: {msg}")
        self.code = code


class TensorC(Structure):
    _fields_ = [("K", c_int64), ("J", c_int32), ("S", c_int64), ("nnz", c_int64),
                ("subj_ptr", c_void_p), ("row_ptr", c_void_p), ("col_idx", c_void_p),
                ("vals", c_void_p), ("val_dtype", c_int32)]


class ProcOutC(Structure):
    _fields_ = [("Q", c_void_p), ("T", c_void_p), ("Pi", c_void_p), ("rank", c_void_p)]


class TuneC(Structure):
    _fields_ = [("split", c_int32), ("blocks_per_sm", c_int32), ("fv_path", c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"split": self.split, "blocks_per_sm": self.blocks_per_sm, "fv_path": self.fv_path,
                "ms": float(self.ms)}


class OptionsC(Structure):
    _fields_ = [("R", c_int32), ("n_outer", c_int32), ("n_inner", c_int32), ("c_H", c_int32),
                ("c_W", c_int32), ("c_V", c_int32), ("lam_H", c_double), ("lam_W", c_double),
                ("lam_V", c_double), ("tau", c_double), ("x_norm2", c_double),
                ("use_graph", c_int32), ("eps_inner", c_double), ("eps_fit", c_double)]


_V = c_void_p
# int32 (*)(double* buf, int64 count, void* stream, void* user)
ALLREDUCE_FN = ctypes.CFUNCTYPE(c_int32, c_void_p, c_int64, c_void_p, c_void_p)
_sig = {
    "copa_create": [POINTER(c_void_p), c_int32, _V, c_int32],
    "copa_destroy": [_V],
    "copa_sync": [_V],
    "copa_validate": [_V, POINTER(TensorC)],
    "copa_forget_tensor": [_V],
    "copa_procrustes": [_V, POINTER(TensorC), c_int32, _V, _V, _V, c_double, POINTER(ProcOutC), _V],
    "copa_mttkrp": [_V, c_int32, POINTER(TensorC), c_int32, POINTER(ProcOutC), _V, _V, _V, _V],
    "copa_gram": [_V, _V, c_int64, c_int32, _V],
    "copa_admm_step": [_V, _V, _V, _V, c_int32, c_int32, c_double, _V, _V, c_int64, c_int32, _V],
    "copa_admm_w_fused": [_V, POINTER(ProcOutC), _V, _V, _V, c_int32, c_int32, c_double, _V, _V,
                          c_int64, c_int32, _V],
    "copa_fit_value": [_V, POINTER(TensorC), c_int32, _V, _V, _V, c_double, _V],
    "copa_fit": [_V, POINTER(TensorC), POINTER(OptionsC), _V, _V, _V, _V, _V, _V, _V,
                 POINTER(ProcOutC)],
    "copa_fit_host": [_V, POINTER(TensorC), POINTER(OptionsC), _V, _V, _V, _V, _V, _V, _V],
    "copa_stage_host": [_V, POINTER(TensorC)],
    "copa_smooth_plan": [_V, POINTER(TensorC), _V, c_int32, c_int32, c_int32, POINTER(c_int64),
                         POINTER(c_int64)],
    "copa_smooth_project": [_V, POINTER(TensorC), _V, c_int32, c_int32, c_int32, POINTER(TensorC), _V],
    "copa_factor_U": [_V, c_int64, c_int32, _V, c_int64, _V, _V, _V, _V, c_int32, c_int64, _V],
    "copa_fit_stats": [_V, POINTER(c_int32), _V],
    "copa_fit_batch": [_V, POINTER(TensorC), c_int32, _V, _V, _V, _V, _V, _V, _V, _V],
    "copa_tune": [_V, POINTER(TensorC), c_int32, _V, _V, _V, c_int32, POINTER(TuneC)],
    "copa_fit_plain": [_V, POINTER(TensorC), POINTER(OptionsC), _V, _V, _V, _V, _V, _V, _V],
    "copa_tune_key": [_V, c_int64, c_int32, c_int32, POINTER(ctypes.c_uint64)],
    "copa_tune_lookup": [ctypes.c_uint64, POINTER(c_int32), POINTER(TuneC)],
    "copa_tune_store": [ctypes.c_uint64, POINTER(TuneC)],
    "copa_loss_grad": [_V, POINTER(TensorC), c_int32, POINTER(ProcOutC), _V, _V, _V, _V, _V, _V,
                       _V],
    "copa_procrustes_work": [_V, POINTER(c_double)],
    "copa_gram_noalloc": [_V, c_int32, _V, c_int64, c_int32, _V],
    "copa_fit_launches": [_V, POINTER(c_int64)],
    "copa_debug_set": [_V, c_int32, c_int64],
    "copa_partition": [_V, _V, c_int64, c_int32, _V],
    "copa_set_allreduce": [_V, ALLREDUCE_FN, _V, _V, c_int64],
}
for _n, _a in _sig.items():
    getattr(_lib, _n).argtypes = _a
    getattr(_lib, _n).restype = c_int32
_lib.copa_last_error.argtypes = [_V]
_lib.copa_last_error.restype = ctypes.c_char_p


def lib():
    return _lib


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class DeviceTensor:
    """Segmented per-subject CSR storage of {X_k} on the device (torch-owned arrays).

    Each instance has a serial number: a handle called with another instance than the last
    one first drops what it derived from the last one (copa_forget_tensor), since a new
    tensor can sit at a freed one's addresses. After rewriting the arrays of an instance in
    place, call Copa.forget_tensor() before using it again."""

    _serials = itertools.count(1)

    def __init__(self, K, J, subj_ptr, row_ptr, col, vals, val_dtype: str):
        self.serial = next(DeviceTensor._serials)
        self.K, self.J = int(K), int(J)
        self.subj_ptr, self.row_ptr, self.col, self.vals = subj_ptr, row_ptr, col, vals
        self.val_dtype = val_dtype
        self.S = int(row_ptr.numel() - 1)      # visit rows (subj_ptr has K + 1 entries)
        self.nnz = int(col.numel())
        if int(subj_ptr.numel()) != self.K + 1:
            raise ValueError("subj_ptr must have K + 1 entries")

    @staticmethod
    def from_host(X, device="cuda", val_dtype: str = "f32") -> "DeviceTensor":
        """X: any object with K, J, subj_ptr, row_ptr, col, val (numpy arrays)."""
        import torch
        tdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[val_dtype]
        return DeviceTensor(
            X.K, X.J,
            torch.as_tensor(np.ascontiguousarray(X.subj_ptr, dtype=np.int64)).to(device),
            torch.as_tensor(np.ascontiguousarray(X.row_ptr, dtype=np.int64)).to(device),
            torch.as_tensor(np.ascontiguousarray(X.col, dtype=np.int32)).to(device),
            torch.as_tensor(np.ascontiguousarray(X.val, dtype=np.float64)).to(device=device, dtype=tdt),
            val_dtype)

    def c(self) -> TensorC:
        return TensorC(self.K, self.J, self.S, self.nnz, _ptr(self.subj_ptr), _ptr(self.row_ptr),
                       _ptr(self.col), _ptr(self.vals), VAL_DTYPE[self.val_dtype])


def bf16_bits(values) -> np.ndarray:
    """The bf16 bit patterns (uint16) of integer counts |x| <= 256, for host tensors whose
    values are passed as val_dtype "bf16" (exact for such counts; half the bytes of f32)."""
    import torch
    v = torch.as_tensor(np.ascontiguousarray(values, dtype=np.float32))
    if not bool(torch.all((v == torch.round(v)) & (v.abs() <= 256))):
        raise ValueError("bf16 values must be integers of magnitude <= 256")
    return v.to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


def host_tensor_c(X, val_dtype="f32"):
    """TensorC over HOST numpy arrays (for copa_fit_host); returns (struct, keep-alive).
    val_dtype "bf16": X.val holds bf16 bit patterns (a 2-byte integer array, see bf16_bits)."""
    if val_dtype == "bf16":
        val = np.asarray(X.val)
        if val.dtype.itemsize != 2 or val.dtype.kind not in "ui":
            raise ValueError("val_dtype bf16 takes the values as bf16 bit patterns (uint16), see bf16_bits")
        val = np.ascontiguousarray(val)
    else:
        val = np.ascontiguousarray(X.val, dtype={"f32": np.float32, "f64": np.float64}[val_dtype])
    arrs = [np.ascontiguousarray(X.subj_ptr, dtype=np.int64), np.ascontiguousarray(X.row_ptr, dtype=np.int64),
            np.ascontiguousarray(X.col, dtype=np.int32), val]
    if len(arrs[0]) != X.K + 1:
        raise ValueError("subj_ptr must have K + 1 entries")
    tc = TensorC(X.K, X.J, len(arrs[1]) - 1, len(arrs[2]), *(a.ctypes.data for a in arrs),
                 VAL_DTYPE[val_dtype])
    return tc, arrs


def _tensor_key(tc) -> tuple:
    """What copa_fit_host matches a staged copy by: sizes, value type, host addresses."""
    return (tc.K, tc.J, tc.S, tc.nnz, tc.val_dtype, tc.subj_ptr, tc.row_ptr, tc.col_idx, tc.vals)


def partition(subj_ptr, row_ptr, nshards: int) -> np.ndarray:
    """copa_partition on host arrays: the first subject of each of nshards contiguous
    shards balanced by nonzeros (nshards + 1 bounds). Needs no GPU."""
    sp = np.ascontiguousarray(subj_ptr, dtype=np.int64)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    out = np.zeros(nshards + 1, dtype=np.int64)
    code = _lib.copa_partition(sp.ctypes.data, rp.ctypes.data, len(sp) - 1, nshards, out.ctypes.data)
    if code != OK:
        raise CopaError(code, "copa_partition: bad arguments")
    return out


def tune_key(subj_ptr, R: int, precision: str) -> int:
    """copa_tune_key on a host subj_ptr array (no GPU needed)."""
    sp = np.ascontiguousarray(subj_ptr, dtype=np.int64)
    key = ctypes.c_uint64()
    code = _lib.copa_tune_key(sp.ctypes.data, len(sp) - 1, R, PREC[precision], byref(key))
    if code != OK:
        raise CopaError(code, "copa_tune_key: bad arguments")
    return key.value


def tune_lookup(key: int):
    """The table entry of a key as a dict, or None (copa_tune_lookup; no GPU needed)."""
    found, out = c_int32(), TuneC()
    _lib.copa_tune_lookup(key, byref(found), byref(out))
    return out.as_dict() if found.value else None


def tune_store(key: int, split: int, blocks_per_sm: int = 0, fv_path: int = 0, ms: float = 0.0):
    code = _lib.copa_tune_store(key, byref(TuneC(split, blocks_per_sm, fv_path, ms)))
    if code != OK:
        raise CopaError(code, "copa_tune_store: bad choice")


class Options:
    def __init__(self, R, n_outer=10, n_inner=10, c_H="none", c_W="nonneg", c_V="l1", lam_H=0.0,
                 lam_W=0.0, lam_V=1.0, tau=1e-8, x_norm2=0.0, use_graph=True, eps_inner=0.0, eps_fit=0.0):
        self.__dict__.update(locals())
        del self.__dict__["self"]

    def c(self) -> OptionsC:
        return OptionsC(self.R, self.n_outer, self.n_inner, CONSTRAINT[self.c_H], CONSTRAINT[self.c_W],
                        CONSTRAINT[self.c_V], self.lam_H, self.lam_W, self.lam_V, self.tau, self.x_norm2,
                        1 if self.use_graph else 0, self.eps_inner, self.eps_fit)


class Copa:
    """A libcopa handle bound to one device and a dedicated CUDA stream.

    The library enqueues its kernels on its own stream (a real stream object, so that
    libcopa's CUDA runtime and PyTorch's refer to the same queue). Every call first makes
    that stream wait for PyTorch's current stream (so inputs written by PyTorch are
    complete) and afterwards makes PyTorch's current stream wait for it (so outputs are
    complete and freed inputs are not reused too early)."""

    def __init__(self, device: int = 0, precision: str = "mixed", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.precision = precision
        self.dtype = torch.float32 if precision == "mixed" else torch.float64
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = c_void_p()
        self._check(_lib.copa_create(byref(h), device, c_void_p(self.stream.cuda_stream), PREC[precision]), None)
        self.h = h
        self._last_serial = None
        self._staged = []   # (key, arrays) of the pending copa_stage_host copies, oldest first

    def _xc(self, X: DeviceTensor) -> TensorC:
        """X's TensorC, after dropping the handle's caches if X is not the tensor of the last call."""
        if X.serial != self._last_serial:
            if self._last_serial is not None:
                self.forget_tensor()
            self._last_serial = X.serial
        return X.c()

    def forget_tensor(self):
        """copa_forget_tensor: drop the data the handle derived from the tensors it has seen."""
        self._call(_lib.copa_forget_tensor, self.h)

    def close(self):
        if getattr(self, "h", None):
            _lib.copa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, fn, *args):
        cur = self.torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        code = fn(*args)
        cur.wait_stream(self.stream)
        self._check(code)

    def _check(self, code, h="self"):
        if code != OK:
            msg = _lib.copa_last_error(self.h if h == "self" else None)
            raise CopaError(code, msg.decode() if msg else "")

    def empty(self, *shape, dtype=None):
        return self.torch.empty(*shape, dtype=dtype or self.dtype, device=self.device)

    def zeros(self, *shape, dtype=None):
        return self.torch.zeros(*shape, dtype=dtype or self.dtype, device=self.device)

    # ---- steps ----
    def sync(self):
        self._call(_lib.copa_sync, self.h)

    def validate(self, X: DeviceTensor):
        self._call(_lib.copa_validate, self.h, byref(self._xc(X)))

    def procrustes(self, X: DeviceTensor, R, H, V, W, tau=1e-8, want_pi=False, want_rank=False,
                   want_fh=True):
        st = {"Q": self.empty(max(X.S, 1), R), "T": self.empty(X.K, R, R),
              "Pi": self.empty(X.K, R, R) if want_pi else None,
              "rank": self.empty(X.K, dtype=self.torch.int32) if want_rank else None}
        fh = self.empty(R, R) if want_fh else None
        po = self.proc_c(st)
        self._call(_lib.copa_procrustes, self.h, byref(self._xc(X)), R, _ptr(H), _ptr(V), _ptr(W), tau,
                                         byref(po), _ptr(fh))
        st["F_H"] = fh
        return st

    @staticmethod
    def proc_c(st) -> ProcOutC:
        return ProcOutC(_ptr(st.get("Q")), _ptr(st.get("T")), _ptr(st.get("Pi")), _ptr(st.get("rank")))

    def mttkrp(self, mode: str, X: DeviceTensor, R, st, H=None, W=None, want_utu=False):
        rows = {"H": R, "V": X.J, "W": X.K}[mode]
        F = self.empty(rows, R)
        utu = self.empty(R, R, dtype=self.torch.float64) if want_utu else None
        self._call(_lib.copa_mttkrp, self.h, MODE[mode], byref(self._xc(X)), R, byref(self.proc_c(st)), _ptr(H),
                                     _ptr(W), _ptr(F), _ptr(utu))
        return (F, utu) if want_utu else F

    def gram(self, A):
        R = A.shape[1]
        G = self.empty(R, R, dtype=self.torch.float64)
        self._call(_lib.copa_gram, self.h, _ptr(A), A.shape[0], R, _ptr(G))
        return G

    def admm_step(self, F, Ga, Gb, n_inner, constraint, lam, Zbar, D):
        rho = self.empty(1, dtype=self.torch.float64)
        self._call(_lib.copa_admm_step, self.h, _ptr(F), _ptr(Ga), _ptr(Gb), n_inner, CONSTRAINT[constraint],
                                        lam, _ptr(Zbar), _ptr(D), Zbar.shape[0], Zbar.shape[1], _ptr(rho))
        return rho

    def admm_w_fused(self, st, H, Ga, Gb, n_inner, constraint, lam, Wbar, DW):
        rho = self.empty(1, dtype=self.torch.float64)
        self._call(_lib.copa_admm_w_fused, self.h, byref(self.proc_c(st)), _ptr(H), _ptr(Ga), _ptr(Gb), n_inner,
                                           CONSTRAINT[constraint], lam, _ptr(Wbar), _ptr(DW), Wbar.shape[0],
                                           Wbar.shape[1], _ptr(rho))
        return rho

    def fit_value(self, X: DeviceTensor, R, V, F_V, UtU, x_norm2=0.0):
        out = self.empty(1, dtype=self.torch.float64)
        self._call(_lib.copa_fit_value, self.h, byref(self._xc(X)), R, _ptr(V), _ptr(F_V), _ptr(UtU), x_norm2,
                                        _ptr(out))
        return out

    def fit(self, X: DeviceTensor, opt: Options, H, V, W, DH=None, DV=None, DW=None, state=None):
        """Algorithm 1 for opt.n_outer iterations; H, V, W (and the duals) updated in place.
        Returns the FIT history (numpy, float64)."""
        DH = self.torch.zeros_like(H) if DH is None else DH
        DV = self.torch.zeros_like(V) if DV is None else DV
        DW = self.torch.zeros_like(W) if DW is None else DW
        hist = np.zeros(max(1, opt.n_outer), dtype=np.float64)
        po = byref(self.proc_c(state)) if state is not None else None
        self._call(_lib.copa_fit, self.h, byref(self._xc(X)), byref(opt.c()), _ptr(H), _ptr(V), _ptr(W), _ptr(DH),
                                  _ptr(DV), _ptr(DW), hist.ctypes.data, po)
        return hist[:self.fit_stats(opt.n_outer)[0]]

    def fit_batch(self, X: DeviceTensor, opts, states):
        """copa_fit_batch: len(opts) fits of X run concurrently; states is a list of
        (H, V, W) or (H, V, W, DH, DV, DW) tensors per fit, updated in place. Returns the FIT
        histories (G x n_outer numpy array, NaN past a fit's last iteration)."""
        G = len(opts)
        if len(states) != G:
            raise ValueError("one state per option set")
        full = []
        for stt in states:
            H, V, W = stt[:3]
            D = stt[3:] if len(stt) == 6 else tuple(self.torch.zeros_like(a) for a in (H, V, W))
            full.append((H, V, W) + tuple(D))
        arr = (OptionsC * G)(*[o.c() for o in opts])
        ptrs = [(c_void_p * G)(*[_ptr(st[i]) for st in full]) for i in range(6)]
        n_outer = opts[0].n_outer
        hist = np.zeros((G, max(1, n_outer)), dtype=np.float64)
        self._call(_lib.copa_fit_batch, self.h, byref(self._xc(X)), G, arr, *ptrs, hist.ctypes.data)
        return hist[:, :n_outer]

    def tune(self, X: DeviceTensor, R, H, V, W, force=False):
        """copa_tune: times the schedule candidates on X (or reuses the table's choice) and
        applies the fastest to this handle's later calls on X at rank R; returns it."""
        out = TuneC()
        self._call(_lib.copa_tune, self.h, byref(self._xc(X)), R, _ptr(H), _ptr(V), _ptr(W), 1 if force else 0,
                   byref(out))
        return out.as_dict()

    def fit_stats(self, n_outer: int):
        """(outer iterations run, inner ADMM iterations as an n_outer x 3 array (H, W, V))
        of the last fit (copa_fit_stats)."""
        n = c_int32()
        inner = np.zeros(3 * max(n_outer, 1), dtype=np.int32)
        self._check(_lib.copa_fit_stats(self.h, byref(n), inner.ctypes.data))
        return n.value, inner[:3 * n_outer].reshape(n_outer, 3)

    def fit_plain(self, X: DeviceTensor, opt: Options, H, V, W, DH=None, DV=None, DW=None):
        """copa_fit_plain: the plain per-subject FP64 form (FP64 handle); returns the FIT
        history (numpy) and updates H, V, W (and the duals) in place."""
        DH = self.torch.zeros_like(H) if DH is None else DH
        DV = self.torch.zeros_like(V) if DV is None else DV
        DW = self.torch.zeros_like(W) if DW is None else DW
        hist = np.zeros(max(1, opt.n_outer), dtype=np.float64)
        self._call(_lib.copa_fit_plain, self.h, byref(self._xc(X)), byref(opt.c()), _ptr(H), _ptr(V), _ptr(W), _ptr(DH),
                   _ptr(DV), _ptr(DW), hist.ctypes.data)
        return hist[:opt.n_outer]

    def fit_host(self, Xh, opt: Options, H, V, W, DH=None, DV=None, DW=None, val_dtype="f32"):
        """copa_fit_host on numpy arrays (H, V, W, duals updated in place)."""
        nd = np.float32 if self.precision == "mixed" else np.float64
        for a in (H, V, W):
            assert a.dtype == nd and a.flags.c_contiguous
        DH = np.zeros_like(H) if DH is None else DH
        DV = np.zeros_like(V) if DV is None else DV
        DW = np.zeros_like(W) if DW is None else DW
        tc, keep = host_tensor_c(Xh, val_dtype)
        hist = np.zeros(max(1, opt.n_outer), dtype=np.float64)
        # the library takes the oldest staged copy if it is of these arrays, else drops all
        if self._staged and self._staged[0][0] == _tensor_key(tc):
            taken = [self._staged.pop(0)]
        else:
            taken, self._staged = self._staged, []
        self._call(_lib.copa_fit_host, self.h, byref(tc), byref(opt.c()), H.ctypes.data, V.ctypes.data,
                                       W.ctypes.data, DH.ctypes.data, DV.ctypes.data, DW.ctypes.data,
                                       hist.ctypes.data)
        del keep, taken
        return hist[:self.fit_stats(opt.n_outer)[0]]

    def stage_host(self, Xh, val_dtype="f32"):
        """copa_stage_host: queue the copy of a host tensor for a later fit_host call with the
        same arrays; the next fit_host call issues it beside its own work (pinned memory
        makes it asynchronous). The arrays are kept referenced until the call that takes or
        discards the copy, and must not be written meanwhile."""
        tc, keep = host_tensor_c(Xh, val_dtype)
        self._check(_lib.copa_stage_host(self.h, byref(tc)))
        self._staged.append((_tensor_key(tc), keep))

    def smooth(self, X: DeviceTensor, days, n_basis=7, degree=3, out_dtype="f32", want_C=False,
               knots="quantile"):
        """Smoothing set-up of Sec. 3.3.1: returns (X' as DeviceTensor, C or None). knots:
        "quantile" (interior knots at the quantiles of each subject's visit days) or
        "uniform" (equally spaced in days)."""
        S_out, nnz_out = c_int64(), c_int64()
        kr = KNOTS[knots]
        self._call(_lib.copa_smooth_plan, self.h, byref(self._xc(X)), _ptr(days), n_basis, degree, kr, byref(S_out),
                                          byref(nnz_out))
        torch = self.torch
        tdt = torch.float32 if out_dtype == "f32" else torch.float64
        Xp = DeviceTensor(X.K, X.J, self.empty(X.K + 1, dtype=torch.int64),
                          self.empty(S_out.value + 1, dtype=torch.int64),
                          self.empty(max(nnz_out.value, 1), dtype=torch.int32)[:nnz_out.value],
                          self.empty(max(nnz_out.value, 1), dtype=tdt)[:nnz_out.value], out_dtype)
        C = self.empty(X.S, n_basis, dtype=torch.float64) if want_C else None
        xc = Xp.c()
        self._call(_lib.copa_smooth_project, self.h, byref(self._xc(X)), _ptr(days), n_basis, degree, kr, byref(xc),
                                             _ptr(C))
        return Xp, C

    def factor_U(self, X_fit: DeviceTensor, R, Q, H, X: Optional[DeviceTensor] = None, C=None):
        """U_k = Q_k H stacked by rows (S_fit x R), or, with the smoothing basis C of the
        original tensor X, U_k = C_k Q_k H (S x R) (copa_factor_U)."""
        rows = X.S if C is not None else X_fit.S
        U = self.empty(max(rows, 1), R)[:rows]
        self._call(_lib.copa_factor_U, self.h, X_fit.K, R, _ptr(X_fit.subj_ptr), X_fit.S, _ptr(Q), _ptr(H),
                   _ptr(X.subj_ptr) if X is not None else None, _ptr(C),
                   int(C.shape[1]) if C is not None else 0, X.S if X is not None else 0, _ptr(U))
        return U

    def debug_set(self, key: int, value: int):
        """Test hook of copa_debug_set (key 1: force the tensor-core V-mode kernel's first
        wait to run out after `value` ns; 0 switches it off)."""
        self._check(_lib.copa_debug_set(self.h, key, value))

    def set_allreduce(self, reduce_fn, J: int = 0, R: int = 0):
        """Makes this handle one shard of a sharded fit (copa_set_allreduce), or a whole fit
        again with reduce_fn=None. reduce_fn(t, stream) must replace the float64 CUDA tensor
        t by its sum over all shards, on `stream` (this handle's torch stream) or before it
        returns. The buffer is sized for J x R factors."""
        if reduce_fn is None:
            self._check(_lib.copa_set_allreduce(self.h, ALLREDUCE_FN(), None, None, 0))
            self._red = None
            return
        cap = max(1, J * R + 2 * R * R)
        buf = self.torch.zeros(cap, dtype=self.torch.float64, device=self.device)
        stream = self.stream

        def cb(ptr, n, _stream, _user):
            try:
                reduce_fn(buf[:n], stream)
                return 0
            except Exception as e:   # reported as COPA_ERR_COMM by the fit
                self._red_exc = e
                return 1

        fn = ALLREDUCE_FN(cb)
        self._red = (fn, buf)          # keeps the callback and the buffer alive
        self._check(_lib.copa_set_allreduce(self.h, fn, None, buf.data_ptr(), cap))

    def fit_launches(self) -> int:
        """Kernels launched by the last fit() (graph nodes x iterations + set-up), -1 if unknown."""
        v = c_int64()
        self._call(_lib.copa_fit_launches, self.h, byref(v))
        return v.value

    def procrustes_work(self) -> float:
        """Multiply-adds performed by the last procrustes() launch (counted on the device)."""
        v = c_double()
        self._call(_lib.copa_procrustes_work, self.h, byref(v))
        return v.value

    def loss_grad(self, X: DeviceTensor, R, st, H, V, W):
        loss = self.empty(1, dtype=self.torch.float64)
        gH, gV, gW = self.empty(*H.shape), self.empty(*V.shape), self.empty(*W.shape)
        self._call(_lib.copa_loss_grad, self.h, byref(self._xc(X)), R, byref(self.proc_c(st)), _ptr(H), _ptr(V),
                                        _ptr(W), _ptr(loss), _ptr(gH), _ptr(gV), _ptr(gW))
        return loss, gH, gV, gW


def gram_noalloc(A, G, stream):
    """G = A^T A through copa_gram_noalloc, which allocates nothing (see include/copa.h).
    A: rows x R float32/float64 CUDA tensor; G: R x R float64 CUDA tensor (written);
    stream: a torch.cuda.Stream to enqueue on. The call receives raw pointers, so every
    property the kernel relies on (dtype, shape, contiguity, device) is checked here
    first; a mismatch raises CopaError(ERR_INVALID_ARG) before anything is launched."""
    import torch

    def bad(why):
        raise CopaError(ERR_INVALID_ARG, "gram_noalloc: " + why)

    if not (isinstance(A, torch.Tensor) and isinstance(G, torch.Tensor)):
        bad("A and G must be torch tensors")
    if A.dtype not in (torch.float32, torch.float64):
        bad(f"A must be float32 or float64, not {A.dtype}")
    if A.dim() != 2 or not A.is_contiguous():
        bad("A must be a contiguous rows x R matrix")
    R = A.shape[1]
    if G.dtype != torch.float64 or tuple(G.shape) != (R, R) or not G.is_contiguous():
        bad(f"G must be a contiguous {R} x {R} float64 matrix")
    cur = torch.cuda.current_device()
    for name, t in (("A", A), ("G", G)):
        if t.device.type != "cuda" or t.device.index != cur:
            bad(f"{name} must be on the current CUDA device (cuda:{cur}), not {t.device}")
    code = _lib.copa_gram_noalloc(c_void_p(stream.cuda_stream), 1 if A.dtype == torch.float64 else 0,
                                  _ptr(A), A.shape[0], R, _ptr(G))
    if code != OK:
        raise CopaError(code, "copa_gram_noalloc failed")


def reconstruction_loss(handle: Copa, X: DeviceTensor, H, V, W, tau=1e-8):
    """L = sum_k ||X_k - Q_k H S_k V^T||_F^2 with Q_k from the Procrustes step at (H, V, W),
    held fixed; differentiable in H, V, W through the hand-written backward kernels."""
    import torch

    class _Loss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, H_, V_, W_):
            R = H_.shape[0]
            st = handle.procrustes(X, R, H_.detach(), V_.detach(), W_.detach(), tau, want_pi=True, want_fh=False)
            loss, gH, gV, gW = handle.loss_grad(X, R, st, H_.detach(), V_.detach(), W_.detach())
            ctx.save_for_backward(gH, gV, gW)
            return loss[0].to(H_.dtype)

        @staticmethod
        def backward(ctx, g):
            gH, gV, gW = ctx.saved_tensors
            return g * gH, g * gV, g * gW

    return _Loss.apply(H, V, W)

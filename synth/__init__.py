"""Seeded synthetic inputs for the COPA hot path.

This module is the one piece shared by the FP64 oracle and the GPU path: it draws
irregular sparse tensors {X_k} shaped like the EHR data of the paper (Sec. 4.1, data set
description and the summary-statistics table: a few to ~2000 visits per patient, a
heavy-tailed code distribution, integer counts) and the initial factors. It holds none
of the method's arithmetic: no Procrustes, projection, MTTKRP, ADMM or FIT.

Layout (row-major, 0-based, shared by every consumer):
  subj_ptr int64[K+1]  visit-row offsets of each subject
  row_ptr  int64[S+1]  nonzero offsets of each visit row
  col      int32[N]    feature index, strictly increasing within a row
  val      float64[N]  value (an integer count in every recipe here)
  days     float64[S]  visit day of each row (only for the smoothing recipe)

All randomness comes from numpy PCG64 with the seeds given below (data 0, init 1,
days 2), so the CPU and GPU sides read identical arrays.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class SparseTensor:
    """Segmented per-subject CSR storage of {X_k}, X_k of size I_k x J."""

    K: int
    J: int
    subj_ptr: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    days: Optional[np.ndarray] = None

    @property
    def S(self) -> int:
        return int(self.subj_ptr[-1])

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def rows_of(self, k: int) -> range:
        return range(int(self.subj_ptr[k]), int(self.subj_ptr[k + 1]))

    def dense(self, k: int) -> np.ndarray:
        """X_k as a dense float64 I_k x J matrix (small inputs only)."""
        r0, r1 = int(self.subj_ptr[k]), int(self.subj_ptr[k + 1])
        out = np.zeros((r1 - r0, self.J), dtype=np.float64)
        for i in range(r0, r1):
            a, b = int(self.row_ptr[i]), int(self.row_ptr[i + 1])
            out[i - r0, self.col[a:b]] = self.val[a:b]
        return out

    def subset(self, ks) -> "SparseTensor":
        """A tensor holding only the listed subjects, in the order given."""
        ks = np.asarray(ks, dtype=np.int64)
        sizes = self.subj_ptr[ks + 1] - self.subj_ptr[ks]
        subj_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        rows = _ranges(self.subj_ptr[ks], sizes)
        rlen = self.row_ptr[rows + 1] - self.row_ptr[rows]
        row_ptr = np.concatenate([[0], np.cumsum(rlen)]).astype(np.int64)
        idx = _ranges(self.row_ptr[rows], rlen)
        days = None if self.days is None else self.days[rows].copy()
        return SparseTensor(len(ks), self.J, subj_ptr, row_ptr,
                            self.col[idx].copy(), self.val[idx].copy(), days)


def _ranges(starts: np.ndarray, lens: np.ndarray) -> np.ndarray:
    """Concatenation of arange(starts[i], starts[i] + lens[i]) over i (vectorised)."""
    lens = np.asarray(lens, dtype=np.int64)
    n = int(lens.sum())
    if n == 0:
        return np.zeros(0, np.int64)
    off = np.repeat(np.asarray(starts, dtype=np.int64) - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    return off + np.arange(n, dtype=np.int64)


# ----------------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------------

def zipf_columns(rng: np.random.Generator, J: int, n: int, a: float = 1.1,
                 perm: Optional[np.ndarray] = None) -> np.ndarray:
    """n draws of a truncated Zipf(a) rank over 1..J, mapped to columns by perm."""
    w = np.arange(1, J + 1, dtype=np.float64) ** (-a)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    rank = np.minimum(np.searchsorted(cdf, u, side="right"), J - 1)
    if perm is None:
        return rank.astype(np.int32)
    return perm[rank].astype(np.int32)


def _sorted_distinct(keys: np.ndarray) -> np.ndarray:
    s = np.sort(keys)
    if len(s) == 0:
        return s
    keep = np.empty(len(s), dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def distinct_rows(rng: np.random.Generator, J: int, n_per_row: np.ndarray,
                  perm: np.ndarray, a: float = 1.1):
    """For every row r, n_per_row[r] distinct Zipf columns, sorted ascending.

    Draws, removes duplicates and redraws the deficit of the rows still short of
    their target until every row holds its target count (targets are capped at J).
    Returns (row_ptr, col)."""
    S = len(n_per_row)
    target = np.minimum(n_per_row.astype(np.int64), J)
    done = []
    active = np.arange(S, dtype=np.int64)       # rows still short of their target
    have_keys = np.zeros(0, dtype=np.int64)     # distinct keys drawn so far for them
    need = target.copy()
    while len(active):
        rows = np.repeat(active, need)
        cols = zipf_columns(rng, J, len(rows), a, perm).astype(np.int64)
        keys = _sorted_distinct(np.concatenate([have_keys, rows * J + cols]))
        krow = keys // J
        cnt = np.bincount(krow, minlength=S)
        short = cnt < target
        fin = ~short[krow]
        done.append(keys[fin])
        have_keys = keys[~fin]
        active = np.nonzero(short & (np.isin(np.arange(S), active)))[0] if len(have_keys) else \
            np.zeros(0, np.int64)
        need = target[active] - cnt[active]
    keys = np.sort(np.concatenate(done)) if done else np.zeros(0, np.int64)
    row = keys // J
    col = (keys - row * J).astype(np.int32)
    row_ptr = np.zeros(S + 1, dtype=np.int64)
    np.cumsum(np.bincount(row, minlength=S), out=row_ptr[1:])
    return row_ptr, col


def visit_days(rng: np.random.Generator, sizes: np.ndarray) -> np.ndarray:
    """Visit days per row: first visit day 0, then gaps of 1 + Geometric(0.2) with
    probability 0.9 (clustered visits) or U{60..900} (long gaps) otherwise."""
    S = int(sizes.sum())
    # numpy's geometric counts trials (support 1, 2, ...) = 1 + a failure count
    short = rng.geometric(0.2, size=S)
    long_gap = rng.integers(60, 901, size=S)
    gaps = np.where(rng.random(S) < 0.9, short, long_gap).astype(np.float64)
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    gaps[starts[sizes > 0]] = 0.0
    days = np.cumsum(gaps)
    # restart the running sum at every subject so that t_1 = 0
    base = np.repeat(days[starts[sizes > 0]], sizes[sizes > 0])
    return days - base


def _lognormal_sizes(rng, K, median, lo, hi, sigma=1.0):
    x = np.rint(median * np.exp(sigma * rng.standard_normal(K)))
    return np.clip(x, lo, hi).astype(np.int64)


PARETO_XM = 14.3  # scale giving a clipped mean of ~40 visits for alpha = 1.5, [1, 2000]


def _pareto_sizes(rng, K, alpha=1.5, xm=PARETO_XM, lo=1, hi=2000):
    x = np.floor(xm * (1.0 + rng.pareto(alpha, size=K)))
    return np.clip(x, lo, hi).astype(np.int64)


def ehr_tensor(K: int, J: int, sizes: np.ndarray, lam: float, cmax: int, seed: int = 0,
               with_days: bool = False) -> SparseTensor:
    """EHR-shaped counts: every visit holds 1 + Poisson(lam) distinct Zipf(1.1)
    columns (ranks mapped to columns by a seeded permutation), counts U{1..cmax}."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(J)
    S = int(sizes.sum())
    n_per_row = 1 + rng.poisson(lam, size=S)
    row_ptr, col = distinct_rows(rng, J, n_per_row, perm)
    val = rng.integers(1, cmax + 1, size=len(col)).astype(np.float64)
    subj_ptr = np.zeros(K + 1, dtype=np.int64)
    np.cumsum(sizes, out=subj_ptr[1:])
    days = visit_days(np.random.default_rng(2), sizes) if with_days else None
    return SparseTensor(K, J, subj_ptr, row_ptr, col, val, days)


# ----------------------------------------------------------------------------------
# the five workloads (subject count K, features J, rank R)
# ----------------------------------------------------------------------------------

@dataclasses.dataclass
class Planted:
    H: np.ndarray
    V: np.ndarray
    W: np.ndarray
    Q: list


def planted_small(K=200, J=100, R=5, seed=0, keep=0.05, noise_free=False,
                  imin=5, imax=30):
    """Planted rank-R PARAFAC2 counts (K=200, J=100, R=5 workload).

    H ~ U(0,1) R x R; V J x R with 70% zeros and the rest U(0,1); w_k ~ U(0.5,1.5);
    Q_k non-negative with orthonormal columns: each visit gets a component drawn
    uniformly (redrawn until all R components occur), Q_k(i, r_i) = 1/sqrt(n_r).
    The mean is Q_k H diag(w_k) V^T; X_k(i,j) ~ Poisson(mean), then each entry is
    kept with probability `keep`. With noise_free=True X_k is the mean itself."""
    rng = np.random.default_rng(seed)
    H = rng.random((R, R))
    V = rng.random((J, R)) * (rng.random((J, R)) >= 0.7)
    W = rng.uniform(0.5, 1.5, size=(K, R))
    sizes = rng.integers(imin, imax + 1, size=K)
    Qs, rows_c, rows_v, row_len = [], [], [], []
    for k in range(K):
        Ik = int(sizes[k])
        while True:
            comp = rng.integers(0, R, size=Ik)
            if len(np.unique(comp)) == R:
                break
        n_r = np.bincount(comp, minlength=R)
        Q = np.zeros((Ik, R))
        Q[np.arange(Ik), comp] = 1.0 / np.sqrt(n_r[comp])
        Qs.append(Q)
        mean = (Q @ H) * W[k][None, :] @ V.T
        if noise_free:
            Xk = mean
        else:
            Xk = rng.poisson(mean).astype(np.float64)
            Xk *= rng.random(Xk.shape) < keep
        for i in range(Ik):
            nz = np.nonzero(Xk[i])[0]
            rows_c.append(nz.astype(np.int32))
            rows_v.append(Xk[i, nz])
            row_len.append(len(nz))
    subj_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    row_ptr = np.concatenate([[0], np.cumsum(row_len)]).astype(np.int64)
    col = np.concatenate(rows_c).astype(np.int32) if rows_c else np.zeros(0, np.int32)
    val = np.concatenate(rows_v).astype(np.float64) if rows_v else np.zeros(0)
    return SparseTensor(K, J, subj_ptr, row_ptr, col, val), Planted(H, V, W, Qs)


WORKLOADS = {
    # name: (K, J, R, n_outer, n_inner)
    "planted_K200_J100_R5": (200, 100, 5, 20, 10),
    "ehr_K20k_J500_R10_smooth": (20_000, 500, 10, 20, 10),
    "ehr_K500k_J1500_R40": (500_000, 1500, 40, 10, 20),
    "ehr_K50k_J1000_R20": (50_000, 1000, 20, 1, 0),
    "ehr_K100k_J1000": (100_000, 1000, None, 5, 10),
}


def ehr_K20k(seed=0, K=20_000, J=500):
    """Lognormal visits (median 20, clipped to [2, 300]), 1 + Poisson(3) codes per
    visit, counts U{1..20}, visit days for the spline basis."""
    rng = np.random.default_rng(seed + 1000)
    sizes = _lognormal_sizes(rng, K, 20, 2, 300)
    return ehr_tensor(K, J, sizes, 3.0, 20, seed, with_days=True)


def ehr_K500k(seed=0, K=500_000, J=1500):
    """Pareto(1.5) visits (clipped mean ~40, range [1, 2000]), 1 + Poisson(4) codes
    per visit (~1e8 nonzeros at K=500k), counts U{1..50}."""
    rng = np.random.default_rng(seed + 1000)
    sizes = _pareto_sizes(rng, K)
    return ehr_tensor(K, J, sizes, 4.0, 50, seed)


def ehr_K50k(seed=0, K=50_000, J=1000):
    """Lognormal visits (median 30, clipped to [2, 500]), 1 + Poisson(4) codes,
    counts U{1..20}."""
    rng = np.random.default_rng(seed + 1000)
    sizes = _lognormal_sizes(rng, K, 30, 2, 500)
    return ehr_tensor(K, J, sizes, 4.0, 20, seed)


def ehr_K100k(seed=0, K=100_000, J=1000):
    """Lognormal visits (median 25, clipped to [2, 400]), 1 + Poisson(4) codes,
    counts U{1..20}."""
    rng = np.random.default_rng(seed + 1000)
    sizes = _lognormal_sizes(rng, K, 25, 2, 400)
    return ehr_tensor(K, J, sizes, 4.0, 20, seed)


def ehr_custom(K, J, median=20, lo=1, hi=200, lam=4.0, cmax=50, seed=0, with_days=False):
    """Scaled-down EHR-shaped tensor for tests (lognormal visit counts)."""
    rng = np.random.default_rng(seed + 1000)
    sizes = _lognormal_sizes(rng, K, median, lo, hi)
    return ehr_tensor(K, J, sizes, lam, cmax, seed, with_days=with_days)


def init_factors(K: int, J: int, R: int, seed: int = 1):
    """Initial factors: H = I_R, W = 1 (K x R), V ~ U(0,1) (J x R) from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    H = np.eye(R)
    V = rng.random((J, R))
    W = np.ones((K, R))
    return H, V, W


def random_state(K: int, J: int, R: int, seed: int = 3):
    """A generic mid-fit state (for step-isolated checks): H ~ U(0,1) + I, V ~ U(0,1)
    with 30% exact zeros, W ~ U(0,1) with 20% exact zeros."""
    rng = np.random.default_rng(seed)
    H = rng.random((R, R)) + np.eye(R)
    V = rng.random((J, R)) * (rng.random((J, R)) >= 0.3)
    W = rng.random((K, R)) * (rng.random((K, R)) >= 0.2)
    return H, V, W


def from_dense(slices, J: int, days=None) -> SparseTensor:
    """Pack dense per-subject slices (list of I_k x J arrays) into the CSR container;
    exact zeros are not stored, so all-zero rows become empty rows."""
    sizes = np.array([s.shape[0] for s in slices], dtype=np.int64)
    cols, vals, lens = [], [], []
    for s in slices:
        for row in s:
            nz = np.nonzero(row)[0]
            cols.append(nz.astype(np.int32))
            vals.append(row[nz].astype(np.float64))
            lens.append(len(nz))
    subj_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    row_ptr = np.concatenate([[0], np.cumsum(np.array(lens, dtype=np.int64))]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = np.concatenate(vals) if vals else np.zeros(0)
    return SparseTensor(len(slices), J, subj_ptr, row_ptr, col, val, days)


def with_edge_cases(X: SparseTensor, seed: int = 7) -> SparseTensor:
    """Copy of X with an empty subject inserted at the front, in the middle and at the
    end, and the first visit of every 5th subject emptied (a visit with no codes)."""
    rng = np.random.default_rng(seed)
    slices = [X.dense(k) for k in range(X.K)]
    for k in range(0, len(slices), 5):
        if slices[k].shape[0]:
            slices[k][0, :] = 0.0
    e = np.zeros((0, X.J))
    mid = len(slices) // 2
    slices = [e] + slices[:mid] + [e] + slices[mid:] + [e]
    days = None
    if X.days is not None:
        days = np.concatenate([np.sort(rng.integers(0, 500, size=s.shape[0])).astype(np.float64)
                               for s in slices]) if slices else None
    return from_dense(slices, X.J, days)

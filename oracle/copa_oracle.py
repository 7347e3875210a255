"""FP64 CPU oracle of COPA's AO-ADMM outer iteration (Afshar et al., arXiv 1803.04572).

TEST INFRASTRUCTURE ONLY. This module is what the CUDA path is checked against. Only the
test suite, the smoke check and the benchmark's CPU-baseline leg may import it; the
product path never calls it and shares no code with it.

Everything is plain numpy in float64 (a library SVD, Cholesky and triangular solves
serve as single steps), written for readability, not speed: per-subject Python loops,
dense slices X_k, dense projected slices Y_k over the columns X_k uses.

Notation follows the paper: X_k (I_k x J) ~ Q_k H S_k V^T with S_k = diag(W(k,:)),
Q_k^T Q_k = I; Y_k = Q_k^T X_k (R x J) are the frontal slices of the R x J x K tensor Y
that is CP-decomposed as [H; V; W] (Sec. 3.1, Eq. 7).

Readings of the paper used here (the paper is silent or ambiguous at these points):
  * Procrustes (Eq. 5, Algorithm 1): A_k = X_k V S_k H^T = B D C^T (thin SVD,
    B left, C right singular vectors) and Q_k = B C^T, keeping only singular values
    with d_i^2 > TAU * d_max^2 (TAU = 1e-8); A_k = 0 gives Q_k = 0. This is the
    pseudo-polar factor: the Procrustes optimum whenever that optimum is unique.
  * The factor handed to the other modes and returned is the auxiliary Zbar (the
    proximal output), updated in the order H, W, V (Algorithm 1).
  * rho = trace(G) / R (Algorithm 1), recomputed once per mode per outer iteration.
  * Inner ADMM, row form: (G + rho I) z = f + rho (zbar + d); zbar = prox(z - d);
    d = d + zbar - z (Eq. 8 update rules, Algorithm 1).
  * l1 prox: sign(v) max(|v| - lambda/rho, 0); l0 prox: v if v^2 > 2 lambda/rho else 0
    (a tie goes to 0); non-negativity: max(0, v) (Sec. 3.3.2, 3.3.3).
  * Fixed inner and outer iteration counts by default; optionally the inner ADMM stops on
    its primal and dual residuals and the outer loop on the change of the FIT (Algorithm 1
    names both convergence tests without defining them). Zbar and D carried across outer
    iterations.
  * Smoothing basis (Sec. 3.3.1): cubic B-splines by the Cox-de Boor recursion, l = 7
    functions on [t_1, t_n] (the first and last visit day), boundary knots repeated, 3
    interior knots either equally spaced in days or at the quantiles of the visit days
    (the paper leaves their estimation open); C_k = left singular vectors of M_k with
    sigma^2 > 1e-10 sigma_max^2. If t_1 = t_n the basis is the constant function.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
from scipy.linalg import solve_triangular

TAU = 1e-8          # rank cut of the Procrustes step (eigenvalues of A^T A)
TAU_BASIS = 1e-10   # rank cut of the smoothing basis (eigenvalues of M_k^T M_k)

NONE, NONNEG, L1, L0 = "none", "nonneg", "l1", "l0"


# ------------------------------------------------------------------------------------
# Procrustes step and projection (Sec. 3.1, Eq. 5; Algorithm 1, per-subject loop)
# ------------------------------------------------------------------------------------

def procrustes(Xk: np.ndarray, V: np.ndarray, w: np.ndarray, H: np.ndarray,
               tau: float = TAU) -> np.ndarray:
    """Q_k = B C^T from the truncated SVD of A_k = X_k V S_k H^T (Eq. 5)."""
    R = H.shape[0]
    A = Xk @ V @ np.diag(w) @ H.T
    if A.shape[0] == 0:
        return np.zeros((0, R))
    B, d, Ct = np.linalg.svd(A, full_matrices=False)
    if d.size == 0 or d[0] == 0.0:
        return np.zeros_like(A)
    keep = d * d > tau * d[0] * d[0]
    return B[:, keep] @ Ct[keep, :]


def project(Q: np.ndarray, Xk: np.ndarray) -> np.ndarray:
    """Y_k = Q_k^T X_k (Algorithm 1, Sec. 3.1)."""
    return Q.T @ Xk


# ------------------------------------------------------------------------------------
# MTTKRP (Sec. 2 definition) on the R x J x K tensor Y with slices Y_k
# ------------------------------------------------------------------------------------

def khatri_rao(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Column-wise Kronecker product: column r is kron(A[:, r], B[:, r])."""
    return np.einsum("ir,jr->ijr", A, B).reshape(A.shape[0] * B.shape[0], A.shape[1])


def unfold(Y: np.ndarray, mode: int) -> np.ndarray:
    """Mode-n matricization of a 3-way array (n = 1, 2, 3), with the remaining
    indices ordered so that the earlier mode varies fastest (Kolda-Bader)."""
    if mode == 1:
        return np.reshape(np.transpose(Y, (0, 2, 1)), (Y.shape[0], -1))  # col j + J k
    if mode == 2:
        return np.reshape(np.transpose(Y, (1, 2, 0)), (Y.shape[1], -1))  # col r + R k
    return np.reshape(np.transpose(Y, (2, 1, 0)), (Y.shape[2], -1))      # col r + R j


def mttkrp_literal(Y: np.ndarray, H, V, W, mode: int) -> np.ndarray:
    """F = Y_(n) (Khatri-Rao of the other factors), formed literally (tiny inputs).
    Mode 1 (H): Y_(1)(W (.) V); mode 2 (V): Y_(2)(W (.) H); mode 3 (W): Y_(3)(V (.) H)."""
    if mode == 1:
        return unfold(Y, 1) @ khatri_rao(W, V)
    if mode == 2:
        return unfold(Y, 2) @ khatri_rao(W, H)
    return unfold(Y, 3) @ khatri_rao(V, H)


@dataclasses.dataclass
class Slices:
    """Y_k = Q_k^T X_k stored densely over the columns X_k uses (all others are 0)."""
    cols: List[np.ndarray]
    Y: List[np.ndarray]       # R x c_k


def project_all(X, Q: List[np.ndarray]) -> Slices:
    cols, Ys = [], []
    for k in range(X.K):
        Xk = X.dense(k)
        used = np.nonzero(np.any(Xk != 0.0, axis=0))[0]
        cols.append(used)
        Ys.append(project(Q[k], Xk[:, used]))
    return Slices(cols, Ys)


def mttkrp_H(Ys: Slices, V, W) -> np.ndarray:
    """F_H = Y_(1)(W (.) V) = sum_k Y_k V S_k."""
    R = V.shape[1]
    F = np.zeros((R, R))
    for k, (c, Y) in enumerate(zip(Ys.cols, Ys.Y)):
        F += Y @ V[c] @ np.diag(W[k])
    return F


def mttkrp_V(Ys: Slices, H, W, J: int) -> np.ndarray:
    """F_V = Y_(2)(W (.) H) = sum_k Y_k^T H S_k."""
    R = H.shape[1]
    F = np.zeros((J, R))
    for k, (c, Y) in enumerate(zip(Ys.cols, Ys.Y)):
        F[c] += Y.T @ H @ np.diag(W[k])
    return F


def mttkrp_W(Ys: Slices, H, V) -> np.ndarray:
    """F_W = Y_(3)(V (.) H), row k = diag(H^T Y_k V)."""
    K, R = len(Ys.Y), H.shape[1]
    F = np.zeros((K, R))
    for k, (c, Y) in enumerate(zip(Ys.cols, Ys.Y)):
        F[k] = np.diag(H.T @ Y @ V[c])
    return F


# ------------------------------------------------------------------------------------
# ADMM inner loop (Eq. 8 update rules, Algorithm 1) and proximal operators
# ------------------------------------------------------------------------------------

def prox(v: np.ndarray, kind: str, lam: float, rho: float) -> np.ndarray:
    """argmin_zbar c(zbar) + rho/2 ||zbar - v||^2, element-wise (Sec. 3.3)."""
    if kind == NONE:
        return v.copy()
    if kind == NONNEG:
        return np.maximum(0.0, v)
    if kind == L1:
        return np.sign(v) * np.maximum(np.abs(v) - lam / rho, 0.0)
    if kind == L0:
        return np.where(v * v > 2.0 * lam / rho, v, 0.0)
    raise ValueError(kind)


def rho_of(G: np.ndarray) -> float:
    """rho = trace(G) / R (Algorithm 1)."""
    return float(np.trace(G)) / G.shape[0]


def admm_counted(F, G, Zbar, D, n_inner: int, kind: str, lam: float = 0.0, eps: float = 0.0,
                 trace: Optional[list] = None):
    """Inner ADMM for one factor with G, F, rho and L = chol(G + rho I) fixed; at most
    n_inner iterations. With eps > 0 the loop stops after the first iteration whose primal
    and dual residuals are both small relative to the factor (the convergence test that
    Algorithm 1 leaves unspecified; reading used here, norms over the whole factor matrix):
        ||Zbar - Z||_F <= eps ||Zbar||_F   and   ||Zbar - Zbar_prev||_F <= eps ||Zbar||_F
    (Zbar after the iteration's update). Both are measured against the factor: the scaled
    dual D of an unconstrained factor is zero after the first iteration, so a test against
    ||D|| would never pass there. Returns (Z, Zbar, D, rho, L, iterations). `trace`, if a
    list, receives max(primal, dual) / ||Zbar|| of every iteration (the quantity compared
    with eps)."""
    R = G.shape[0]
    rho = rho_of(G)
    L = np.linalg.cholesky(G + rho * np.eye(R))
    Z = np.zeros_like(Zbar)
    it = 0
    for it in range(1, n_inner + 1):
        Zbar_prev = Zbar
        rhs = (F + rho * (Zbar + D)).T
        Z = solve_triangular(L.T, solve_triangular(L, rhs, lower=True), lower=False).T
        Zbar = prox(Z - D, kind, lam, rho)
        D = D + Zbar - Z
        if eps > 0.0:
            nz2 = np.sum(Zbar ** 2)
            p2, d2 = np.sum((Zbar - Z) ** 2), np.sum((Zbar - Zbar_prev) ** 2)
            if trace is not None:
                trace.append(np.sqrt(max(p2, d2) / nz2) if nz2 > 0 else np.inf)
            if p2 <= eps * eps * nz2 and d2 <= eps * eps * nz2:
                break
    return Z, Zbar, D, rho, L, it


def admm(F, G, Zbar, D, n_inner: int, kind: str, lam: float = 0.0):
    """Inner ADMM for one factor with G, F, rho and L = chol(G + rho I) fixed, exactly
    n_inner iterations. Returns (Z, Zbar, D, rho, L); rows of Z, Zbar, D are the factor's
    rows."""
    return admm_counted(F, G, Zbar, D, n_inner, kind, lam)[:5]


def grams(H, V, W):
    """The three Hadamard-product Grams (Algorithm 1): G_H, G_W, G_V."""
    return ((W.T @ W) * (V.T @ V), (H.T @ H) * (V.T @ V), (H.T @ H) * (W.T @ W))


# ------------------------------------------------------------------------------------
# Metrics (Sec. 4.1, evaluation metrics)
# ------------------------------------------------------------------------------------

def residual_norm2(X, Q, H, V, W) -> float:
    """sum_k ||X_k - Q_k H S_k V^T||_F^2 by dense reconstruction."""
    tot = 0.0
    for k in range(X.K):
        Xk = X.dense(k)
        tot += float(np.sum((Xk - Q[k] @ H @ np.diag(W[k]) @ V.T) ** 2))
    return tot


def data_norm2(X) -> float:
    return float(np.sum(np.asarray(X.val, dtype=np.float64) ** 2))


def fit_value(X, Q, H, V, W, x_norm2: Optional[float] = None, proj_norm2=None) -> float:
    """FIT = 1 - sum_k ||X_k - U_k S_k V^T||^2 / sum_k ||X_k||^2 (U_k = Q_k H).

    With smoothing, X holds the projected slices X'_k = C_k^T X_k, x_norm2 is the
    original sum ||X_k||^2 and the part of X_k outside span(C_k) is added back:
    ||X_k - C_k Q_k H S_k V^T||^2 = ||X_k||^2 - ||X'_k||^2 + ||X'_k - Q_k H S_k V^T||^2."""
    res = residual_norm2(X, Q, H, V, W)
    if x_norm2 is None:
        return 1.0 - res / data_norm2(X)
    return 1.0 - (x_norm2 - data_norm2(X) + res) / x_norm2


def sparsity(V: np.ndarray) -> float:
    """SPARSITY = (number of exact zeros of V) / size(V)."""
    return float(np.count_nonzero(V == 0.0)) / V.size


# ------------------------------------------------------------------------------------
# One outer iteration and the whole fit (Algorithm 1)
# ------------------------------------------------------------------------------------

@dataclasses.dataclass
class Options:
    n_inner: int = 10
    c_H: str = NONE
    c_W: str = NONNEG
    c_V: str = L1
    lam_H: float = 0.0
    lam_W: float = 0.0
    lam_V: float = 1.0
    tau: float = TAU
    eps_inner: float = 0.0    # > 0: stop each inner ADMM early (admm_counted); n_inner is the cap


@dataclasses.dataclass
class State:
    """Auxiliary factors (the model) and scaled duals, carried across iterations."""
    H: np.ndarray
    V: np.ndarray
    W: np.ndarray
    DH: np.ndarray
    DV: np.ndarray
    DW: np.ndarray

    @staticmethod
    def from_init(H, V, W):
        H, V, W = (np.array(a, dtype=np.float64) for a in (H, V, W))
        return State(H, V, W, np.zeros_like(H), np.zeros_like(V), np.zeros_like(W))

    def copy(self):
        return State(*(a.copy() for a in (self.H, self.V, self.W, self.DH, self.DV, self.DW)))


@dataclasses.dataclass
class StepRecord:
    """Everything one outer iteration produced (for step-isolated comparisons)."""
    Q: list
    F_H: np.ndarray
    G_H: np.ndarray
    rho_H: float
    F_W: np.ndarray
    G_W: np.ndarray
    rho_W: float
    F_V: np.ndarray
    G_V: np.ndarray
    rho_V: float
    state: State
    inner: tuple = (0, 0, 0)    # ADMM iterations run for H, W, V
    traces: tuple = ((), (), ())  # with eps_inner > 0: the residual ratio of every iteration


def outer_iteration(X, st: State, opt: Options) -> StepRecord:
    """One pass of Algorithm 1: Procrustes for every subject, then H, W, V by ADMM."""
    st = st.copy()
    Q = [procrustes(X.dense(k), st.V, st.W[k], st.H, opt.tau) for k in range(X.K)]
    Ys = project_all(X, Q)
    # H: G = W^T W * V^T V, F = Y_(1)(W (.) V)
    G_H = (st.W.T @ st.W) * (st.V.T @ st.V)
    F_H = mttkrp_H(Ys, st.V, st.W)
    tr = ([], [], [])
    _, st.H, st.DH, rho_H, _, nH = admm_counted(F_H, G_H, st.H, st.DH, opt.n_inner, opt.c_H, opt.lam_H,
                                                opt.eps_inner, tr[0])
    # W: G = H^T H * V^T V, F = Y_(3)(V (.) H)
    G_W = (st.H.T @ st.H) * (st.V.T @ st.V)
    F_W = mttkrp_W(Ys, st.H, st.V)
    _, st.W, st.DW, rho_W, _, nW = admm_counted(F_W, G_W, st.W, st.DW, opt.n_inner, opt.c_W, opt.lam_W,
                                                opt.eps_inner, tr[1])
    # V: G = H^T H * W^T W, F = Y_(2)(W (.) H)
    G_V = (st.H.T @ st.H) * (st.W.T @ st.W)
    F_V = mttkrp_V(Ys, st.H, st.W, X.J)
    _, st.V, st.DV, rho_V, _, nV = admm_counted(F_V, G_V, st.V, st.DV, opt.n_inner, opt.c_V, opt.lam_V,
                                                opt.eps_inner, tr[2])
    return StepRecord(Q, F_H, G_H, rho_H, F_W, G_W, rho_W, F_V, G_V, rho_V, st, (nH, nW, nV),
                      tuple(tuple(t) for t in tr))


def fit(X, H0, V0, W0, opt: Options, n_outer: int, x_norm2: Optional[float] = None, eps_fit: float = 0.0,
        records: Optional[list] = None):
    """Run up to n_outer outer iterations from the given init; returns (state, FIT history,
    last step record). FIT uses the Q_k of each iteration and its final factors. With
    eps_fit > 0 the loop stops after the first iteration t >= 2 (1-based) whose FIT differs
    from the previous one by at most eps_fit (Algorithm 1's outer convergence test, which
    the paper leaves unspecified; reading used here). `records`, if a list, receives every
    iteration's StepRecord."""
    st = State.from_init(H0, V0, W0)
    hist = []
    rec = None
    for _ in range(n_outer):
        rec = outer_iteration(X, st, opt)
        st = rec.state
        hist.append(fit_value(X, rec.Q, st.H, st.V, st.W, x_norm2))
        if records is not None:
            records.append(rec)
        if eps_fit > 0.0 and len(hist) >= 2 and abs(hist[-1] - hist[-2]) <= eps_fit:
            break
    return st, np.array(hist), rec


# ------------------------------------------------------------------------------------
# Smoothness on U_k through a per-subject spline basis (Sec. 3.3.1)
# ------------------------------------------------------------------------------------

KNOTS_UNIFORM, KNOTS_QUANTILE = "uniform", "quantile"


def spline_knots(t1: float, tn: float, l: int = 7, d: int = 3, days=None,
                 rule: str = KNOTS_UNIFORM) -> np.ndarray:
    """Boundary knots t_1 and t_n repeated d+1 times and l-d-1 interior knots, placed
    (Sec. 3.3.1: the knots' number and positions are estimated; reading used here)
      uniform:  equally spaced in days on [t_1, t_n];
      quantile: at the quantiles j/(l-d) of the subject's visit days (linear interpolation
                between order statistics), so that the knots follow the visits: many where
                visits cluster, few across long gaps."""
    n_int = l - d - 1
    p = np.arange(1, n_int + 1) / (n_int + 1)
    if rule == KNOTS_QUANTILE:
        t = np.sort(np.asarray(days, dtype=np.float64))
        h = (len(t) - 1) * p
        j = np.floor(h).astype(int)
        j1 = np.minimum(j + 1, len(t) - 1)
        interior = t[j] + (h - j) * (t[j1] - t[j])
    else:
        interior = t1 + (tn - t1) * p
    return np.concatenate([np.full(d + 1, t1), interior, np.full(d + 1, tn)])


def bspline(i: int, d: int, t: float, knots: np.ndarray) -> float:
    """m_{i,d}(t) by the recursion of Sec. 3.3.1 (0/0 taken as 0). Degree 0 is the
    indicator of [beta_i, beta_{i+1}), closed on the right on the last non-empty span."""
    if d == 0:
        lo, hi = knots[i], knots[i + 1]
        if lo < hi and (lo <= t < hi or (t == knots[-1] and hi == knots[-1])):
            return 1.0
        return 0.0
    a = 0.0
    den = knots[i + d] - knots[i]
    if den > 0:
        a = (t - knots[i]) / den * bspline(i, d - 1, t, knots)
    b = 0.0
    den = knots[i + d + 1] - knots[i + 1]
    if den > 0:
        b = (knots[i + d + 1] - t) / den * bspline(i + 1, d - 1, t, knots)
    return a + b


def subject_basis(days: np.ndarray, l: int = 7, d: int = 3, rule: str = KNOTS_UNIFORM) -> np.ndarray:
    """M_k (I_k x l): the l basis functions evaluated at the visit days."""
    if len(days) == 0:
        return np.zeros((0, l))
    t1, tn = float(days[0]), float(days[-1])
    if tn == t1:
        return np.ones((len(days), 1))
    knots = spline_knots(t1, tn, l, d, days, rule)
    return np.array([[bspline(i, d, float(t), knots) for i in range(l)] for t in days])


def basis_C(M: np.ndarray, tau: float = TAU_BASIS) -> np.ndarray:
    """C_k = left singular vectors of M_k with sigma^2 > tau sigma_max^2."""
    if M.shape[0] == 0:
        return np.zeros((0, 0))
    B, s, _ = np.linalg.svd(M, full_matrices=False)
    keep = s * s > tau * s[0] * s[0]
    return B[:, keep]


def smooth_project(X, l: int = 7, d: int = 3, rule: str = KNOTS_UNIFORM):
    """X'_k = C_k^T X_k for every subject (Sec. 3.3.1); returns the list of C_k and the
    projected slices as a list of dense r_k x J matrices."""
    Cs, Xp = [], []
    for k in range(X.K):
        rows = X.rows_of(k)
        C = basis_C(subject_basis(X.days[rows.start:rows.stop], l, d, rule))
        Cs.append(C)
        Xp.append(C.T @ X.dense(k))
    return Cs, Xp


def factor_U(Q: list, H: np.ndarray, Cs: Optional[list] = None) -> list:
    """The paper's output U_k = Q_k H, or U_k = C_k Q_k H when the fit ran on the smoothed
    projection X'_k = C_k^T X_k (Sec. 3.3.1, Algorithm 1 output)."""
    if Cs is None:
        return [q @ H for q in Q]
    return [C @ q @ H for C, q in zip(Cs, Q)]


# ------------------------------------------------------------------------------------
# Reconstruction loss and its gradient with Q_k fixed (no 1/2 factor)
# ------------------------------------------------------------------------------------

def loss_and_grad(X, Q, H, V, W):
    """L = sum_k ||X_k - Q_k H S_k V^T||_F^2 and dL/dH, dL/dV, dL/dW (Q_k fixed)."""
    L = 0.0
    gH, gV, gW = np.zeros_like(H), np.zeros_like(V), np.zeros_like(W)
    for k in range(X.K):
        Xk = X.dense(k)
        Sk = np.diag(W[k])
        Rk = Xk - Q[k] @ H @ Sk @ V.T
        L += float(np.sum(Rk * Rk))
        gH += -2.0 * Q[k].T @ Rk @ V @ Sk
        gV += -2.0 * Rk.T @ Q[k] @ H @ Sk
        gW[k] = -2.0 * np.diag(H.T @ Q[k].T @ Rk @ V)
    return L, gH, gV, gW


def slices_to_tensor(Xp, J: int):
    """Pack dense slices (a list of r_k x J arrays) into the shared CSR container."""
    from synth import SparseTensor
    sizes = np.array([x.shape[0] for x in Xp], dtype=np.int64)
    rows = [x[i] for x in Xp for i in range(x.shape[0])]
    cols = [np.nonzero(r)[0].astype(np.int32) for r in rows]
    vals = [r[c] for r, c in zip(rows, cols)]
    subj_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    row_ptr = np.concatenate([[0], np.cumsum([len(c) for c in cols])]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = np.concatenate(vals) if vals else np.zeros(0)
    return SparseTensor(len(Xp), J, subj_ptr, row_ptr, col, val)

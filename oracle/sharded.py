"""The FP64 oracle's outer iteration over subject shards (test infrastructure only).

TEST INFRASTRUCTURE ONLY, like copa_oracle.py: only the test suite and the benchmark's
CPU-baseline leg use it; the product path never does.

Algorithm 1 processes the subjects independently in its Procrustes loop (Sec. 3.2, the
per-subject parallel loop) and touches them otherwise only through sums: the MTTKRPs for
H and V (F_H = sum_k Y_k V S_k, F_V = sum_k Y_k^T H S_k), the Gram W^T W = sum_k w_k^T w_k
and the residual of the FIT. So the subjects can be split into shards, each holding its
slices X_k and its rows of W (and of the dual D_W), with H, V and their duals replicated:
every shard runs the same iteration on its own subjects, and the sums are completed by an
all-reduce (sum over shards) before the step that needs them. The ADMM updates of H and V
then see identical inputs on every shard and stay replicated; the W update is row-wise
and stays local.

This module restates copa_oracle.outer_iteration in that form, with the same steps in the
same order, calling copa_oracle for every piece of arithmetic. `allreduce(a)` must return
the elementwise sum of `a` over all shards (identity for a single shard).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

from . import copa_oracle as O


@dataclasses.dataclass
class ShardState:
    """H, V and their duals (replicated) and this shard's rows of W and D_W."""
    H: np.ndarray
    V: np.ndarray
    W: np.ndarray
    DH: np.ndarray
    DV: np.ndarray
    DW: np.ndarray

    def copy(self):
        return ShardState(*(a.copy() for a in (self.H, self.V, self.W, self.DH, self.DV, self.DW)))


def shard_state(st: O.State, k0: int, k1: int) -> ShardState:
    """The part of a full state that the shard of subjects [k0, k1) holds."""
    return ShardState(st.H.copy(), st.V.copy(), st.W[k0:k1].copy(), st.DH.copy(), st.DV.copy(),
                      st.DW[k0:k1].copy())


def outer_iteration(Xs, st: ShardState, opt: O.Options, allreduce: Callable[[np.ndarray], np.ndarray],
                    x_norm2: Optional[float] = None):
    """One outer iteration of Algorithm 1 on the shard Xs (its subjects only). Returns the
    new shard state and the FIT of the whole tensor after the iteration."""
    assert opt.eps_inner <= 0.0, "sharded iteration: fixed inner counts only"
    st = st.copy()
    Q = [O.procrustes(Xs.dense(k), st.V, st.W[k], st.H, opt.tau) for k in range(Xs.K)]
    Ys = O.project_all(Xs, Q)
    # H: G = W^T W .* V^T V, F_H = sum over all subjects
    WtW = allreduce(st.W.T @ st.W)
    G_H = WtW * (st.V.T @ st.V)
    F_H = allreduce(O.mttkrp_H(Ys, st.V, st.W))
    _, st.H, st.DH, _, _ = O.admm(F_H, G_H, st.H, st.DH, opt.n_inner, opt.c_H, opt.lam_H)
    # W: row-wise, local to the shard (G needs only the replicated H and V)
    G_W = (st.H.T @ st.H) * (st.V.T @ st.V)
    F_W = O.mttkrp_W(Ys, st.H, st.V)
    _, st.W, st.DW, _, _ = O.admm(F_W, G_W, st.W, st.DW, opt.n_inner, opt.c_W, opt.lam_W)
    # V: G = H^T H .* W^T W (the updated W of every shard), F_V = sum over all subjects
    G_V = (st.H.T @ st.H) * allreduce(st.W.T @ st.W)
    F_V = allreduce(O.mttkrp_V(Ys, st.H, st.W, Xs.J))
    _, st.V, st.DV, _, _ = O.admm(F_V, G_V, st.V, st.DV, opt.n_inner, opt.c_V, opt.lam_V)
    # FIT: residual and data norm summed over shards
    sums = allreduce(np.array([O.residual_norm2(Xs, Q, st.H, st.V, st.W), O.data_norm2(Xs)]))
    xn = sums[1] if x_norm2 is None else x_norm2
    fit = 1.0 - (xn - sums[1] + sums[0]) / xn
    return st, fit

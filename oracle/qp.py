"""Oracle of the assembly front end: the reduced SPD system of a branch-MPC
QP, written out densely from its definition (App. A, "Linear System Sparsity
in IPM and ADMM"): with the equality constraints A x = b and the
inequalities h_l <= G x <= h_u of the QP, eliminating the second and third
block rows of the regularized KKT matrix (Eq. appendix_ipm_kkt; the ADMM
matrix of Eq. appendix_admm_kkt has the same form) leaves

    K = P + tau I + delta^{-1} A^T A + G^T (W + delta I)^{-1} G.

Variables are ordered as the solver's right-hand side (natural order): the
stages z_1..z_N of scenario 1, ..., of scenario S, then the root u_0; a
stage is z_k = (x_k, u_k). The constraints are the dynamics
x_{k+1} = A_k x_k + B_k u_k (k = 1..N-1) and the first step
x_1 - B_0 u_0 = A_0 x_init of every scenario; G = I (bounds on every
variable). Test infrastructure only: nothing on the product path imports
this module.
"""
from __future__ import annotations

import numpy as np


def _np(a):
    return np.asarray(a.cpu().numpy() if hasattr(a, "cpu") else a, dtype=np.float64)


def layout(qp: dict) -> dict:
    S, N, nx, nu = qp["S"], qp["N"], qp["nx"], qp["nu"]
    nb = nx + nu
    n0 = S * N * nb
    return {"S": S, "N": N, "nx": nx, "nu": nu, "nb": nb, "n0": n0, "n": n0 + nu}


def _x(L, s, k):
    """Column range of x_k (1-based k) of scenario s."""
    o = s * L["N"] * L["nb"] + (k - 1) * L["nb"]
    return slice(o, o + L["nx"])


def _u(L, s, k):
    o = s * L["N"] * L["nb"] + (k - 1) * L["nb"] + L["nx"]
    return slice(o, o + L["nu"])


def equality_matrix(qp: dict) -> np.ndarray:
    """The rows of A: per scenario, the first step (x_1 - B_0 u_0) and the
    dynamics x_{k+1} - A_k x_k - B_k u_k, k = 1..N-1."""
    L = layout(qp)
    A, B = _np(qp["A"]), _np(qp["B"])
    S, N, nx = L["S"], L["N"], L["nx"]
    root = slice(L["n0"], L["n"])
    rows = []
    for s in range(S):
        M = np.zeros((nx, L["n"]))
        M[:, _x(L, s, 1)] = np.eye(nx)
        M[:, root] = -B[s, 0]
        rows.append(M)
        for k in range(1, N):
            M = np.zeros((nx, L["n"]))
            M[:, _x(L, s, k + 1)] = np.eye(nx)
            M[:, _x(L, s, k)] = -A[s, k]
            M[:, _u(L, s, k)] = -B[s, k]
            rows.append(M)
    return np.vstack(rows)


def cost_diagonal(qp: dict) -> np.ndarray:
    """Diagonal of P: q on the states, rw on the stage inputs, r0w on u_0."""
    L = layout(qp)
    q, rw, r0w = _np(qp["q"]), _np(qp["rw"]), _np(qp["r0w"])
    stages = np.concatenate([q, rw], axis=-1)          # [S][N][nb] = (x_k, u_k)
    return np.concatenate([stages.reshape(-1), r0w])


def weight_diagonal(qp: dict) -> np.ndarray:
    """Diagonal of W (the inequality weights), same order as the variables."""
    return np.concatenate([_np(qp["w"]).reshape(-1), _np(qp["w0"])])


def reduced_kkt(qp: dict) -> np.ndarray:
    """Dense K = P + tau I + A^T A / delta + G^T (W + delta I)^{-1} G with G = I."""
    tau, delta = qp["tau"], qp["delta"]
    A = equality_matrix(qp)
    n = A.shape[1]
    return (np.diag(cost_diagonal(qp)) + tau * np.eye(n) + A.T @ A / delta
            + np.diag(1.0 / (weight_diagonal(qp) + delta)))


def quadratic_form(qp: dict, v) -> float:
    """v^T K v from the definition term by term, without forming A^T A: the
    cost and regularization terms, ||A v||^2 / delta with A v evaluated
    constraint by constraint from the dynamics, and the inequality term."""
    L = layout(qp)
    v = _np(v)
    A, B = _np(qp["A"]), _np(qp["B"])
    tau, delta = qp["tau"], qp["delta"]
    val = float(np.sum(cost_diagonal(qp) * v * v) + tau * np.sum(v * v)
                + np.sum(v * v / (weight_diagonal(qp) + delta)))
    u0 = v[L["n0"]:]
    acc = 0.0
    for s in range(L["S"]):
        res = v[_x(L, s, 1)] - B[s, 0] @ u0
        acc += float(res @ res)
        for k in range(1, L["N"]):
            res = v[_x(L, s, k + 1)] - A[s, k] @ v[_x(L, s, k)] - B[s, k] @ v[_u(L, s, k)]
            acc += float(res @ res)
    return val + acc / delta

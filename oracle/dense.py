"""Dense NumPy/SciPy oracle of the two-level factor.

ORACLE -- test infrastructure only (see oracle/__init__.py).

Everything here is the plain definition, evaluated on assembled dense
matrices with library routines:

* ``gamma(n)`` is the recursive block permutation Gamma_n of Sec. II: take
  every other block starting with the first, keep their order, and recurse
  on the blocks left over.
* ``tail_order(N)`` is Pi_i of Sec. IV-A as a sequence of 1-based stage
  indices: reverse the tail (Omega_i), apply Gamma_{N-1} to
  (x_N, ..., x_2) and keep x_1 last.
* ``permuted_factor`` is the Cholesky factor L of Pi K Pi^T
  (Eq. permuted_root_coupled_matrix) from ``numpy.linalg.cholesky``; the
  blocks L_i, F_i and L_R of Alg. 1 are read off it.

These cost O((S N nb)^3) and are meant for small systems, or one tail at a
time (``permuted_tail_factor``).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _np(a):
    return np.asarray(a.cpu().numpy() if hasattr(a, "cpu") else a, dtype=np.float64)


def gamma(n: int) -> list:
    """Gamma_n as the list of 1-based positions in permuted order (Sec. II)."""
    def rec(seq):
        if not seq:
            return []
        return seq[0::2] + rec(seq[1::2])
    return rec(list(range(1, n + 1)))


def gamma_groups(n: int) -> list:
    """The groups produced by the recursive calls of Gamma_n (Sec. II)."""
    out = []
    seq = list(range(1, n + 1))
    while seq:
        out.append(seq[0::2])
        seq = seq[1::2]
    return out


def tail_order(N: int) -> list:
    """Pi_i = blkdiag(Gamma_{N-1}, I) Omega_i (Sec. IV-A), as the natural
    1-based stage indices in permuted order."""
    rev = list(range(N, 0, -1))           # Omega_i: (x_N, ..., x_1)
    head = rev[:-1]                       # (x_N, ..., x_2)
    return [head[j - 1] for j in gamma(len(head))] + [1]


def assemble_tail(D_s, E_s) -> np.ndarray:
    """Dense K_i (Eq. tail_block_tridiagonal) from the lower triangles of D
    and the sub-diagonal blocks E."""
    D_s, E_s = _np(D_s), _np(E_s)
    N, nb, _ = D_s.shape
    K = np.zeros((N * nb, N * nb))
    for k in range(N):
        Dl = np.tril(D_s[k])
        K[k * nb:(k + 1) * nb, k * nb:(k + 1) * nb] = Dl + np.tril(Dl, -1).T
    for k in range(N - 1):
        K[(k + 1) * nb:(k + 2) * nb, k * nb:(k + 1) * nb] = E_s[k]
        K[k * nb:(k + 1) * nb, (k + 1) * nb:(k + 2) * nb] = E_s[k].T
    return K


def assemble_system(D, E, C, R) -> np.ndarray:
    """Dense K of Eq. root_coupled_matrix in natural order (dx^1..dx^M, dx_0)."""
    D, E, C, R = _np(D), _np(E), _np(C), _np(R)
    S, N, nb, _ = D.shape
    nr = R.shape[0]
    n0 = S * N * nb
    K = np.zeros((n0 + nr, n0 + nr))
    for s in range(S):
        o = s * N * nb
        K[o:o + N * nb, o:o + N * nb] = assemble_tail(D[s], E[s])
        K[n0:, o:o + nb] = C[s]               # C_i = [C_{i,1} 0 ... 0]
        K[o:o + nb, n0:] = C[s].T
    Rl = np.tril(R)
    K[n0:, n0:] = Rl + np.tril(Rl, -1).T
    return K


def permutation_vector(S: int, N: int, nb: int, nr: int, order=None) -> np.ndarray:
    """Scalar index vector P with (Pi K Pi^T) = K[P][:, P] for
    Pi = blkdiag(Pi_1, ..., Pi_M, I)."""
    order = tail_order(N) if order is None else order
    idx = []
    for s in range(S):
        for k in order:
            base = s * N * nb + (k - 1) * nb
            idx.extend(range(base, base + nb))
    idx.extend(range(S * N * nb, S * N * nb + nr))
    return np.asarray(idx)


def permuted_factor(D, E, C, R, order=None) -> dict:
    """Cholesky factor of Pi K Pi^T for the whole (small) system."""
    D = _np(D)
    S, N, nb, _ = D.shape
    nr = _np(R).shape[0]
    K = assemble_system(D, E, C, R)
    P = permutation_vector(S, N, nb, nr, order)
    Kh = K[np.ix_(P, P)]
    L = np.linalg.cholesky(Kh)
    return {"K": K, "P": P, "Khat": Kh, "L": L}


def permuted_tail_factor(D_s, E_s, C_s=None, order=None) -> dict:
    """For one tail: L_i = chol(Pi_i K_i Pi_i^T) and, if C_s is given,
    F_i = C_hat_i L_i^{-T} with C_hat_i = C_i Pi_i^T (Eq. permuted_tail_coupling)
    and U_i = F_i F_i^T."""
    D_s = _np(D_s)
    N, nb, _ = D_s.shape
    order = tail_order(N) if order is None else order
    Kt = assemble_tail(D_s, E_s)
    P = np.concatenate([np.arange((k - 1) * nb, k * nb) for k in order])
    L = np.linalg.cholesky(Kt[np.ix_(P, P)])
    out = {"order": order, "L": L, "P": P}
    if C_s is not None:
        C_s = _np(C_s)
        nr = C_s.shape[0]
        Ci = np.zeros((nr, N * nb))
        Ci[:, :nb] = C_s                              # C_i = [C_{i,1} 0 ... 0]
        Chat = Ci[:, P]                               # C_i Pi_i^T
        F = sla.solve_triangular(L, Chat.T, lower=True).T   # F L^T = C_hat
        out.update({"Chat": Chat, "F": F, "U": F @ F.T})
    return out


def block(L: np.ndarray, nb: int, i: int, j: int) -> np.ndarray:
    """Block (i, j) (0-based block indices) of a dense matrix with nb-blocks."""
    return L[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]


def root_factor(D, E, C, R) -> dict:
    """R_tilde = R - sum_i U_i and L_R = chol(R_tilde) (Alg. 1, steps 4-5),
    with each U_i taken from the dense permuted tail factor."""
    D, E, C, R = _np(D), _np(E), _np(C), _np(R)
    S = D.shape[0]
    Rl = np.tril(R)
    Rt = Rl + np.tril(Rl, -1).T
    for s in range(S):
        Rt = Rt - permuted_tail_factor(D[s], E[s], C[s])["U"]
    return {"Rt": Rt, "LR": np.linalg.cholesky(Rt)}


def dense_solve(D, E, C, R, r) -> np.ndarray:
    """x = K^{-1} r through a dense LU with partial pivoting (scipy)."""
    K = assemble_system(D, E, C, R)
    return sla.lu_solve(sla.lu_factor(K), _np(r))

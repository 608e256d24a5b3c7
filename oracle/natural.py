"""ctypes front end of the natural-order C oracle (oracle/bm_oracle.c).

ORACLE -- test infrastructure only (see oracle/__init__.py).

Natural order = (dx^1, ..., dx^M, dx_0) with each tail dx^i = (dx_1, ..., dx_N)
(Sec. III-B); this is Fig. 2(a)'s ordering, whose factor carries a dense root
row. Every function takes and returns float64 NumPy arrays in the layouts of
``bmgen``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.bmo_factor.restype = ctypes.c_long
        lib.bmo_factor.argtypes = [ctypes.c_int] * 4 + [_dp] * 9 + [ctypes.c_int]
        lib.bmo_solve.restype = None
        lib.bmo_solve.argtypes = [ctypes.c_int] * 4 + [_dp] * 6 + [ctypes.c_int]
        lib.bmo_residual.restype = None
        lib.bmo_residual.argtypes = [ctypes.c_int] * 4 + [_dp] * 8 + [ctypes.c_int]
        lib.bmo_tail_schur_first.restype = ctypes.c_long
        lib.bmo_tail_schur_first.argtypes = [ctypes.c_int] * 3 + [_dp] * 3 + [ctypes.c_int]
        lib.bmo_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    a = np.asarray(a.cpu().numpy() if hasattr(a, "cpu") else a, dtype=np.float64)
    return np.ascontiguousarray(a)


class NotSPD(RuntimeError):
    pass


def max_threads() -> int:
    return int(_load().bmo_max_threads())


def factor(D, E, C, R, nthreads: int = 0) -> dict:
    """Natural-order block Cholesky. Returns Ld[S,N,nb,nb], Lsub[S,N-1,nb,nb],
    Z[S,N,nr,nb] (dense root row of the factor), LR[nr,nr] = chol(R - sum U),
    Rt = R - sum U and logdet(K) = 2 sum log diag(L)."""
    D, E, C, R = _f64(D), _f64(E), _f64(C), _f64(R)
    S, N, nb, _ = D.shape
    nr = R.shape[0]
    if nb > 256:
        raise ValueError("oracle supports nb <= 256")
    Ld = np.zeros((S, N, nb, nb))
    Lsub = np.zeros((S, max(N - 1, 0), nb, nb))
    Z = np.zeros((S, N, nr, nb))
    LR = np.zeros((nr, nr))
    Rt = np.zeros((nr, nr))
    Ep = E if E.size else np.zeros(1)
    Lsp = Lsub if Lsub.size else np.zeros(1)
    rc = _load().bmo_factor(S, N, nb, nr, _p(D), _p(Ep), _p(C), _p(R), _p(Ld), _p(Lsp), _p(Z),
                            _p(LR), _p(Rt), int(nthreads))
    if rc != 0:
        raise NotSPD("oracle: non-positive pivot (code %d)" % rc)
    logdet = 2.0 * (np.log(np.diagonal(Ld, axis1=-2, axis2=-1)).sum() + np.log(np.diag(LR)).sum())
    return {"Ld": Ld, "Lsub": Lsub, "Z": Z, "LR": LR, "Rt": Rt, "logdet": float(logdet),
            "shape": (S, N, nb, nr)}


def solve(fac: dict, r, nthreads: int = 0) -> np.ndarray:
    S, N, nb, nr = fac["shape"]
    r = _f64(r)
    x = np.zeros_like(r)
    Lsub = fac["Lsub"] if fac["Lsub"].size else np.zeros(1)
    _load().bmo_solve(S, N, nb, nr, _p(fac["Ld"]), _p(Lsub), _p(fac["Z"]), _p(fac["LR"]),
                      _p(r), _p(x), int(nthreads))
    return x


def abs_kx(D, E, C, R, x) -> np.ndarray:
    """|K| |x| for the root-coupled matrix of Sec. III-B (Eq.
    root_coupled_matrix): stage blocks D (lower triangles, mirrored),
    sub-diagonal blocks E and their transposes, C_{s,1} coupling stage 1 of
    tail s to the root, root block R; written out block by block."""
    D, E, C, R, x = (_f64(a) for a in (D, E, C, R, x))
    S, N, nb, _ = D.shape
    nr = R.shape[0]
    n0 = S * N * nb
    X = np.abs(x[:n0]).reshape(S, N, nb)
    x0 = np.abs(x[n0:])
    Dl = np.tril(D)
    Dfull = np.abs(Dl + np.swapaxes(np.tril(Dl, -1), -1, -2))
    out = np.einsum("snij,snj->sni", Dfull, X)
    if N > 1:
        Ea = np.abs(E)
        out[:, 1:] += np.einsum("snij,snj->sni", Ea, X[:, :-1])     # block (k+1, k) = E_k
        out[:, :-1] += np.einsum("snji,snj->sni", Ea, X[:, 1:])     # block (k, k+1) = E_k^T
    Ca = np.abs(C)
    out[:, 0] += np.einsum("sji,j->si", Ca, x0)                     # block (1, root) = C^T
    Rl = np.tril(R)
    Rfull = np.abs(Rl + np.tril(Rl, -1).T)
    root = Rfull @ x0 + np.einsum("sij,sj->i", Ca, X[:, 0])
    return np.concatenate([out.reshape(-1), root])


def residual_rows(D, E, C, R, x, r, rows) -> dict:
    """rho_i = r_i - (K x)_i and omega_i = |rho_i| / (|K||x| + |r|)_i for a
    set of row indices of K only (natural order), each row formed from the
    blocks it touches (Eq. root_coupled_matrix): for systems too large to
    check whole on the host."""
    D, E, C, R, x, r = (_f64(a) for a in (D, E, C, R, x, r))
    S, N, nb, _ = D.shape
    nr = R.shape[0]
    n0 = S * N * nb
    rows = np.asarray(rows, dtype=np.int64)
    rho = np.zeros(rows.size)
    den = np.zeros(rows.size)
    for t, g in enumerate(rows):
        if g < n0:
            s, rem = divmod(int(g), N * nb)
            k, i = divmod(rem, nb)
            xs = x[s * N * nb:(s + 1) * N * nb].reshape(N, nb)
            Dk = D[s, k]
            row = np.array([Dk[i, j] if j <= i else Dk[j, i] for j in range(nb)])
            terms = [row * xs[k]]
            if k > 0:
                terms.append(E[s, k - 1][i] * xs[k - 1])          # block (k, k-1)
            if k + 1 < N:
                terms.append(E[s, k][:, i] * xs[k + 1])           # block (k, k+1) = E^T
            if k == 0:
                terms.append(C[s][:, i] * x[n0:])                 # block (1, root) = C^T
        else:
            c = int(g) - n0
            row = np.array([R[c, j] if j <= c else R[j, c] for j in range(nr)])
            terms = [row * x[n0:]] + [C[s][c] * x[s * N * nb:s * N * nb + nb] for s in range(S)]
        prod = np.concatenate(terms)
        rho[t] = r[g] - prod.sum()
        den[t] = np.abs(prod).sum() + abs(r[g])
    with np.errstate(divide="ignore", invalid="ignore"):
        om = np.where(den > 0, np.abs(rho) / np.where(den > 0, den, 1.0), np.where(rho != 0, np.inf, 0.0))
    return {"rho": rho, "omega": float(om.max()) if om.size else 0.0}


def residual_rows_exact(D, E, C, R, x, r, rows) -> dict:
    """rho_i = r_i - (K x)_i computed exactly in rational arithmetic (every
    FP64 entry is a dyadic rational, so each product and the sum are exact)
    and rounded once to FP64, with (|K| |x|)_i, for a set of row indices of
    K (natural order, the blocks of Eq. root_coupled_matrix as in
    ``residual_rows``). The reference for residuals that claim more than
    FP64 summation accuracy."""
    from fractions import Fraction
    D, E, C, R, x, r = (_f64(a) for a in (D, E, C, R, x, r))
    S, N, nb, _ = D.shape
    nr = R.shape[0]
    n0 = S * N * nb
    rows = np.asarray(rows, dtype=np.int64)
    rho = np.zeros(rows.size)
    kx = np.zeros(rows.size)
    for t, g in enumerate(rows):
        pairs = []
        if g < n0:
            s, rem = divmod(int(g), N * nb)
            k, i = divmod(rem, nb)
            base = s * N * nb
            pairs += [(D[s, k, i, j] if j <= i else D[s, k, j, i], x[base + k * nb + j]) for j in range(nb)]
            if k > 0:
                pairs += [(E[s, k - 1, i, j], x[base + (k - 1) * nb + j]) for j in range(nb)]
            if k + 1 < N:
                pairs += [(E[s, k, j, i], x[base + (k + 1) * nb + j]) for j in range(nb)]
            if k == 0:
                pairs += [(C[s, j, i], x[n0 + j]) for j in range(nr)]
        else:
            c = int(g) - n0
            pairs += [(R[c, j] if j <= c else R[j, c], x[n0 + j]) for j in range(nr)]
            pairs += [(C[s, c, j], x[s * N * nb + j]) for s in range(S) for j in range(nb)]
        acc = Fraction(float(r[g]))
        for a, b in pairs:
            acc -= Fraction(float(a)) * Fraction(float(b))
        rho[t] = float(acc)
        kx[t] = float(sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in pairs))
    return {"rho": rho, "abs_kx": kx}


def residual(D, E, C, R, x, r, nthreads: int = 0) -> dict:
    """rho = r - K x in FP64, the normwise backward error
    eta = ||rho||_inf / (||K||_inf ||x||_inf + ||r||_inf), the componentwise
    (Oettli-Prager) backward error omega = max_i |rho_i| / (|K| |x| + |r|)_i
    and the relative residuals ||rho||_inf / ||r||_inf (rel_inf) and
    ||rho||_2 / ||r||_2."""
    D, E, C, R, x, r = (_f64(a) for a in (D, E, C, R, x, r))
    S, N, nb, _ = D.shape
    nr = R.shape[0]
    rho = np.zeros_like(r)
    out = np.zeros(6)
    Ep = E if E.size else np.zeros(1)
    _load().bmo_residual(S, N, nb, nr, _p(D), _p(Ep), _p(C), _p(R), _p(x), _p(r), _p(rho), _p(out),
                         int(nthreads))
    eta = out[0] / (out[1] * out[2] + out[3])
    rel_inf = out[0] / out[3] if out[3] > 0 else (0.0 if out[0] == 0 else float("inf"))
    den = abs_kx(D, E, C, R, x) + np.abs(r)
    num = np.abs(rho)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(den > 0, num / np.where(den > 0, den, 1.0), np.where(num > 0, np.inf, 0.0))
    return {"rho": rho, "eta": float(eta), "rel2": float(out[4] / out[5]), "rel_inf": float(rel_inf),
            "omega": float(ratio.max()), "K_inf": float(out[1])}


def tail_schur_first(D, E, nthreads: int = 0) -> np.ndarray:
    """Per tail, the Schur complement onto stage 1 of the tail matrix K_i
    (eliminating stages N, ..., 2): S_1 = ((K_i^{-1})_{11})^{-1}."""
    D, E = _f64(D), _f64(E)
    S, N, nb, _ = D.shape
    out = np.zeros((S, nb, nb))
    Ep = E if E.size else np.zeros(1)
    rc = _load().bmo_tail_schur_first(S, N, nb, _p(D), _p(Ep), _p(out), int(nthreads))
    if rc != 0:
        raise NotSPD("oracle: non-positive pivot (code %d)" % rc)
    return out


def solve_system(sysd: dict, nthreads: int = 0) -> dict:
    """Factor + solve + residual of one generated system (dict from bmgen)."""
    fac = factor(sysd["D"], sysd["E"], sysd["C"], sysd["R"], nthreads)
    x = solve(fac, sysd["r"], nthreads)
    res = residual(sysd["D"], sysd["E"], sysd["C"], sysd["R"], x, sysd["r"], nthreads)
    return {"x": x, "fac": fac, "res": res}

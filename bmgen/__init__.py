"""Seeded synthetic branch-MPC inputs.

This module only draws inputs: the stage blocks ``D``, the sub-diagonal
blocks ``E``, the root-tail coupling blocks ``C``, the root block ``R`` and a
right-hand side ``r`` of the root-coupled SPD system ``K dx = r`` (Sec. III-B,
Eq. root_coupled_matrix and Eq. tail_block_tridiagonal). It holds none of the
solver's arithmetic (no factorization, no triangular solve of ``K``); the
oracle under ``oracle/`` and the CUDA library both consume what it returns.

Recipe (the paper's quadrotor data are not available; these MPC-shaped
systems stand in for them):

* Every tail is the dual Schur complement ``G H^{-1} G^T`` of the linear
  dynamics ``x_k = A x_{k-1} + B u_{k-1}`` with ``H = blkdiag(Q_k, R_k)``,
  which makes it SPD by construction:
  ``D_k = A Q_{k-1}^{-1} A^T + B R_{k-1}^{-1} B^T + Q_k^{-1}`` and the block
  below the diagonal ``E_k = -A Q_k^{-1}`` (the block above it is its
  transpose).
* ``C_{s,1} = B_s^T`` couples the shared root (size ``nr``) to stage 1.
* The root block is ``R = R0 + sum_s C_{s,1} (K_s^{-1})_{11} C_{s,1}^T`` so
  that the exact root Schur complement ``R - sum_s U_s`` equals ``R0``
  (``nr * I`` by default, or a random Wishart matrix) and ``K`` is SPD by the
  Schur-complement lemma. ``(K_s^{-1})_{11}`` is obtained from the backward
  recursion ``S_N = D_N, S_k = D_k - E_k^T S_{k+1}^{-1} E_k`` with dense
  ``torch.linalg.solve`` calls; it only shapes the input.
* ``A_s = I + 0.1 G_s`` with ``G_s ~ N(0, 1/nb)`` (independent per scenario)
  or, for the larger workloads, ``A_s = A_0 + 0.05 Xi_s`` with a shared
  ``A_0 = I + 0.1 G`` and ``Xi_s ~ N(0, 1)``; ``B_s ~ N(0, 1)``; diagonal
  ``Q_s, R_s ~ U[0.1, 10]``; optional interior-point barrier diagonals
  ``10^U[lo, hi]`` per stage and entry added to ``Q_k`` and ``R_k``.
* ``r ~ N(0, 1)``; the seed of instance ``j`` of workload id ``c`` is
  ``1000 c + j``.

Layouts (row-major, contiguous, float64): ``D[S][N][nb][nb]`` (full symmetric
storage), ``E[S][N-1][nb][nb]`` where ``E[s][k]`` is the paper's ``E_{s,k+1}``,
the block at (stage k+2, stage k+1) in 1-based stages; ``C[S][nr][nb]``;
``R[nr][nr]``; ``r[S*N*nb + nr]`` in the natural order
``(dx^1, ..., dx^S, dx_0)`` with ``dx^s = (dx^s_1, ..., dx^s_N)``.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import Optional, Tuple

import torch

__all__ = ["Workload", "WORKLOADS", "generate", "generate_qp", "n_unknowns", "seed_for",
           "method_flops", "natural_flops", "draw_batched_shapes"]


@dataclass(frozen=True)
class Workload:
    """Shape and draw recipe of one synthetic branch-MPC system."""
    name: str
    S: int                 # scenarios (the paper's M)
    N: int                 # horizon length (stages per tail)
    nb: int                # stage block size (nx)
    nr: int                # root block size (nu)
    workload_id: int = 0   # c in seed = 1000 c + instance
    barrier: Optional[Tuple[float, float]] = None  # log10 range of barrier diagonals
    shared_A: bool = False  # A_s = A_0 + 0.05 Xi_s instead of independent A_s
    root: str = "scaled_identity"  # R0 = nr * I, or "wishart"

    def with_shape(self, **kw) -> "Workload":
        return replace(self, **kw)


WORKLOADS = {
    # plain FP64 single instance
    "plain-s4-n16-nb4": Workload("plain-s4-n16-nb4", 4, 16, 4, 2, workload_id=1),
    # plain FP64, medium
    "medium-s64-n64-nb12": Workload("medium-s64-n64-nb12", 64, 64, 12, 4, workload_id=2,
                                    barrier=(-4.0, 4.0), shared_A=True),
    # FP32 tails + FP64 refinement
    "mixed-s512-n128-nb24": Workload("mixed-s512-n128-nb24", 512, 128, 24, 8, workload_id=3,
                                     barrier=(-6.0, 6.0), shared_A=True),
    # the large serving request shape
    "large-s2048-n256-nb48": Workload("large-s2048-n256-nb48", 2048, 256, 48, 16, workload_id=5,
                                      barrier=(-4.0, 4.0), shared_A=True),
    # one point of the paper's sweep grid (nb = nr = 16), context only
    "grid-s100-n160-nb16": Workload("grid-s100-n160-nb16", 100, 160, 16, 16, workload_id=6,
                                    shared_A=True),
}


def seed_for(w: Workload, instance: int = 0) -> int:
    return 1000 * w.workload_id + instance


def n_unknowns(S: int, N: int, nb: int, nr: int) -> int:
    return S * N * nb + nr


def _levels(N: int) -> int:
    """Number of odd-even levels of the N-1 chain blocks (0 when N <= 1)."""
    return (N - 1).bit_length() if N >= 2 else 0


def method_flops(S: int, N: int, nb: int, nr: int) -> dict:
    """Flop counts of the two-level method (factor and solve), used only to
    convert measured times into GFLOP/s. A chain block with two neighbours
    at elimination costs chol (nb^3/3) + two triangular solves (2 nb^3) + two
    symmetric updates (2 nb^3 counted full) + one fill product (2 nb^3) =
    19/3 nb^3; a block with one neighbour costs 7/3 nb^3."""
    n3 = float(nb) ** 3
    two = one = 0
    for p in range(1, N):
        lvl = (p & -p).bit_length() - 1
        has_left = p > (1 << lvl)
        if has_left:
            two += 1
        else:
            one += 1
    tail = two * 19.0 / 3.0 * n3 + one * 7.0 / 3.0 * n3 + n3 / 3.0  # + x_1 chol
    tail += 2.0 * nr * nb * nb / 2.0 * 2.0 + 2.0 * nr * nr * nb       # coupling trsm + syrk
    factor = S * tail + nr ** 3 / 3.0 + 2.0 * S * nr * nr / 2.0
    # solve: per chain block fwd (trsv nb^2 + up to 2 gemv 2 nb^2 each) and bwd (same)
    solve_tail = 0.0
    for p in range(1, N):
        lvl = (p & -p).bit_length() - 1
        k = 2 if p > (1 << lvl) else 1
        solve_tail += 2.0 * (nb * nb + k * 2.0 * nb * nb)
    solve_tail += 2.0 * nb * nb + 2.0 * 2.0 * nr * nb
    solve = S * solve_tail + 2.0 * nr * nr
    return {"factor": factor, "solve": solve, "total": factor + solve}


def natural_flops(S: int, N: int, nb: int, nr: int) -> float:
    """Riccati-equivalent (natural-order) factor flop count, 7/3 nb^3 per stage."""
    return S * N * 7.0 / 3.0 * float(nb) ** 3


def _uniform(g, shape, lo, hi, dev):
    return lo + (hi - lo) * torch.rand(shape, generator=g, device=dev, dtype=torch.float64)


@torch.no_grad()
def generate(w: Workload, instance: int = 0, device="cpu", seed: Optional[int] = None,
             with_rhs: bool = True) -> dict:
    """Draw one system. Returns float64 tensors D, E, C, R, r on ``device``.

    The draw order is fixed (A, B, Q, R, barriers, R0, r) so a seed always
    yields the same system on a given device type."""
    S, N, nb, nr = w.S, w.N, w.nb, w.nr
    if min(S, N, nb, nr) < 1:
        raise ValueError("S, N, nb, nr must be >= 1")
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(seed_for(w, instance) if seed is None else seed)
    f64 = torch.float64
    eye = torch.eye(nb, dtype=f64, device=dev)

    if w.shared_A:
        G = torch.randn((nb, nb), generator=g, device=dev, dtype=f64) / (nb ** 0.5)
        A0 = eye + 0.1 * G
        Xi = torch.randn((S, nb, nb), generator=g, device=dev, dtype=f64)
        A = A0.unsqueeze(0) + 0.05 * Xi
    else:
        G = torch.randn((S, nb, nb), generator=g, device=dev, dtype=f64) / (nb ** 0.5)
        A = eye.unsqueeze(0) + 0.1 * G
    B = torch.randn((S, nb, nr), generator=g, device=dev, dtype=f64)
    q = _uniform(g, (S, 1, nb), 0.1, 10.0, dev).expand(S, N + 1, nb)
    rr = _uniform(g, (S, 1, nr), 0.1, 10.0, dev).expand(S, N + 1, nr)
    if w.barrier is not None:
        lo, hi = w.barrier
        q = q + torch.pow(10.0, _uniform(g, (S, N + 1, nb), lo, hi, dev))
        rr = rr + torch.pow(10.0, _uniform(g, (S, N + 1, nr), lo, hi, dev))
    qinv = 1.0 / q     # [S, N+1, nb]  stage 0..N
    rinv = 1.0 / rr    # [S, N+1, nr]

    # D_k (k = 1..N) = A Q_{k-1}^{-1} A^T + B R_{k-1}^{-1} B^T + Q_k^{-1}
    AQ = A.unsqueeze(1) * qinv[:, :N, None, :]              # [S,N,nb,nb] = A diag(qinv_{k-1})
    D = AQ @ A.transpose(-1, -2).unsqueeze(1)
    BR = B.unsqueeze(1) * rinv[:, :N, None, :]
    D = D + BR @ B.transpose(-1, -2).unsqueeze(1)
    D = D + torch.diag_embed(qinv[:, 1:N + 1, :])
    D = 0.5 * (D + D.transpose(-1, -2))
    # E_k (k = 1..N-1), block (k+1, k) = -A Q_k^{-1}
    if N >= 2:
        E = -(A.unsqueeze(1) * qinv[:, 1:N, None, :])
    else:
        E = torch.zeros((S, 0, nb, nb), dtype=f64, device=dev)
    C = B.transpose(-1, -2).contiguous()                     # [S, nr, nb]

    # root: R = R0 + sum_s C_s (K_s^{-1})_{11} C_s^T
    Sk = D[:, N - 1]
    for k in range(N - 2, -1, -1):
        Ek = E[:, k]                                         # block (k+2, k+1)
        Sk = D[:, k] - Ek.transpose(-1, -2) @ torch.linalg.solve(Sk, Ek)
        Sk = 0.5 * (Sk + Sk.transpose(-1, -2))
    X = torch.linalg.solve(Sk, C.transpose(-1, -2))          # S_1^{-1} C^T  [S, nb, nr]
    Usum = (C @ X).sum(dim=0)
    if w.root == "wishart":
        Z = torch.randn((nr, 2 * nr), generator=g, device=dev, dtype=f64)
        R0 = Z @ Z.T / (2 * nr) + 0.5 * torch.eye(nr, dtype=f64, device=dev)
    else:
        R0 = nr * torch.eye(nr, dtype=f64, device=dev)
    R = R0 + 0.5 * (Usum + Usum.T)
    out = {"D": D.contiguous(), "E": E.contiguous(), "C": C, "R": R.contiguous(),
           "R0": R0, "S": S, "N": N, "nb": nb, "nr": nr}
    if with_rhs:
        out["r"] = torch.randn((n_unknowns(S, N, nb, nr),), generator=g, device=dev, dtype=f64)
    return out


def draw_batched_shapes(count: int = 256, seed: int = 4000, nb_set=(6, 12, 24, 48),
                        S_range=(8, 256), N_range=(16, 256)):
    """Shapes of a batch of independent systems: S ~ U{8..256}, N ~ U{16..256},
    nb from ``nb_set``, nr = ceil(nb/3)."""
    g = torch.Generator()
    g.manual_seed(seed)
    shapes = []
    for _ in range(count):
        S = int(torch.randint(S_range[0], S_range[1] + 1, (1,), generator=g))
        N = int(torch.randint(N_range[0], N_range[1] + 1, (1,), generator=g))
        nb = int(nb_set[int(torch.randint(0, len(nb_set), (1,), generator=g))])
        shapes.append((S, N, nb, -(-nb // 3)))
    return shapes


def generate_qp(S: int, N: int, nx: int, nu: int, seed: int = 0, device="cpu",
                barrier: Tuple[float, float] = (-3.0, 3.0), tau: float = 1e-6, delta: float = 1e-4) -> dict:
    """Draw the data of a branch-MPC QP (inputs of the assembly front end).

    Stage k = 1..N of scenario s holds z_k = (x_k, u_k) (nb = nx + nu; u_N
    is the padding input of the last stage); the shared root is the first
    input u_0 (nr = nu); the initial state is fixed. Dynamics
    x_{k+1} = A_k x_k + B_k u_k (k = 1..N-1) and x_1 = A_0 x_init + B_0 u_0.
    Returns float64 tensors A[S][N][nx][nx] (A_k at index k; A_0 only acts on
    the fixed initial state), B[S][N][nx][nu] (B_k at index k), diagonal
    costs q[S][N][nx] (x_1..x_N), rw[S][N][nu] (u_1..u_N), r0w[nu] (u_0),
    inequality weights w[S][N][nb] and w0[nu] (the positive diagonal W of
    the interior point method, 10^U[lo, hi]) and the regularizations tau,
    delta. Draws only: no assembly here."""
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    f64 = torch.float64
    eye = torch.eye(nx, dtype=f64, device=dev)
    A0 = eye + 0.1 * torch.randn((nx, nx), generator=g, device=dev, dtype=f64) / (nx ** 0.5)
    A = A0.expand(S, N, nx, nx) + 0.02 * torch.randn((S, N, nx, nx), generator=g, device=dev, dtype=f64)
    B = torch.randn((S, N, nx, nu), generator=g, device=dev, dtype=f64) / (nx ** 0.5)
    q = _uniform(g, (S, N, nx), 0.1, 10.0, dev)
    rw = _uniform(g, (S, N, nu), 0.1, 10.0, dev)
    r0w = _uniform(g, (nu,), 0.1, 10.0, dev)
    lo, hi = barrier
    w = torch.pow(10.0, _uniform(g, (S, N, nx + nu), lo, hi, dev))
    w0 = torch.pow(10.0, _uniform(g, (nu,), lo, hi, dev))
    return {"A": A.contiguous(), "B": B.contiguous(), "q": q, "rw": rw, "r0w": r0w, "w": w, "w0": w0,
            "tau": float(tau), "delta": float(delta), "S": S, "N": N, "nx": nx, "nu": nu,
            "nb": nx + nu, "nr": nu}

"""Pins of the oracle against what the paper and the mathematics fix.

Each test pins one oracle function to something other than itself: the
paper's printed worked examples (tests/golden/), Theorem 1, dense LU with
partial pivoting, closed forms (nb = 1 Thomas recursion, N = 1 arrow
matrix), and invariants of the Cholesky factor (L L^T = K, logdet, the
ordering-invariant blocks L_R and L_{i,1}). The last tests plant plausible
mistakes into the oracle's inputs and check that these pins see them.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import bmgen
from oracle import dense, natural

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def small(S, N, nb, nr, seed=0, barrier=None, root="scaled_identity", shared_A=False):
    w = bmgen.Workload("t", S, N, nb, nr, workload_id=90, barrier=barrier, root=root,
                       shared_A=shared_A)
    d = bmgen.generate(w, seed=seed)
    return {k: (v.numpy() if hasattr(v, "numpy") else v) for k, v in d.items()}


# --- Sec. II: the recursive permutation ---------------------------------------

def test_gamma7_matches_paper_example():
    gold = _read_golden("gamma7.txt")[0]
    groups = [[int(t) for t in g.split()] for g in gold.split("|")]
    assert dense.gamma(7) == [p for g in groups for p in g]
    assert dense.gamma_groups(7) == groups


def test_seven_block_pattern_matches_eq_seven_block_permutation():
    rows = [r.split() for r in _read_golden("seven_block_pattern.txt")]
    order = dense.gamma(7)

    def psi(i, j):  # block (i, j) of the block-tridiagonal Psi, 1-based
        if i == j:
            return "D%d" % i
        if i == j + 1:
            return "E%d" % j
        if j == i + 1:
            return "E%dT" % i
        return "."

    got = [[psi(order[a], order[b]) for b in range(7)] for a in range(7)]
    assert got == rows


@pytest.mark.parametrize("n", list(range(1, 65)))
def test_gamma_is_permutation_with_log_levels(n):
    g = dense.gamma(n)
    assert sorted(g) == list(range(1, n + 1))
    groups = dense.gamma_groups(n)
    assert len(groups) == n.bit_length()            # floor(log2 n) + 1 levels
    # blocks of one group are never neighbours in the chain (mutually uncoupled)
    for grp in groups:
        assert all(b - a >= 2 for a, b in zip(grp, grp[1:]))


def test_tail_order_definition():
    # Pi_i: reverse, Gamma_{N-1} on (x_N..x_2), x_1 last (Sec. IV-A)
    assert dense.tail_order(1) == [1]
    assert dense.tail_order(2) == [2, 1]
    # N = 8: (x8..x2) = xi_1..xi_7 -> Gamma_7 = (1,3,5,7,2,6,4) -> stages (8,6,4,2,7,3,5), then 1
    assert dense.tail_order(8) == [8, 6, 4, 2, 7, 3, 5, 1]


# --- natural-order C oracle vs dense LU ---------------------------------------

CASES = [(1, 1, 1, 1), (1, 2, 3, 2), (2, 3, 2, 1), (3, 9, 4, 2), (2, 8, 3, 3), (1, 5, 1, 1),
         (4, 16, 4, 2), (2, 7, 5, 4)]


@pytest.mark.parametrize("S,N,nb,nr", CASES)
def test_natural_oracle_matches_dense_lu(S, N, nb, nr):
    d = small(S, N, nb, nr, seed=S * 100 + N, barrier=(-2, 2))
    out = natural.solve_system(d)
    xref = dense.dense_solve(d["D"], d["E"], d["C"], d["R"], d["r"])
    K = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    kappa = np.linalg.cond(K)
    err = np.abs(out["x"] - xref).max() / np.abs(xref).max()
    assert err < 1e-15 * kappa * 50
    assert out["res"]["eta"] < 1e-15


@pytest.mark.parametrize("S,N,nb,nr", CASES)
def test_natural_factor_reconstructs_K(S, N, nb, nr):
    d = small(S, N, nb, nr, seed=7 + N, barrier=(-1, 1))
    f = natural.factor(d["D"], d["E"], d["C"], d["R"])
    n0 = S * N * nb
    L = np.zeros((n0 + nr, n0 + nr))
    for s in range(S):
        for k in range(N):
            o = s * N * nb + k * nb
            L[o:o + nb, o:o + nb] = f["Ld"][s, k]
            L[n0:, o:o + nb] = f["Z"][s, k]
            if k + 1 < N:
                L[o + nb:o + 2 * nb, o:o + nb] = f["Lsub"][s, k]
    L[n0:, n0:] = f["LR"]
    K = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    assert np.abs(L @ L.T - K).max() <= 1e-14 * np.abs(K).max()
    assert np.allclose(np.triu(L, 1), 0.0)
    sign, ld = np.linalg.slogdet(K)
    assert sign > 0 and abs(f["logdet"] - ld) <= 1e-10 * max(1.0, abs(ld))


# --- Theorem 1 and the ordering study of Fig. 2 --------------------------------

@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 9, 16, 17])
def test_theorem1_coupling_solve_is_single_block(N):
    nb, nr = 3, 2
    d = small(1, N, nb, nr, seed=N)
    t = dense.permuted_tail_factor(d["D"][0], d["E"][0], d["C"][0])
    F = t["F"]
    assert np.all(F[:, :(N - 1) * nb] == 0.0)      # exact zeros before the last block
    assert np.abs(F[:, (N - 1) * nb:]).max() > 0.0
    # and the reduced formula F_{i,1} = C_{i,1} L_{i,1}^{-T} of Sec. IV-B
    L11 = dense.block(t["L"], nb, N - 1, N - 1)
    F1 = sla.solve_triangular(L11, d["C"][0].T, lower=True).T
    assert np.allclose(F[:, (N - 1) * nb:], F1, rtol=1e-13, atol=0)


def _root_row_blocks(order, N, nb, nr, d):
    pf = dense.permuted_factor(d["D"], d["E"], d["C"], d["R"], order=order)
    L = pf["L"]
    S = d["D"].shape[0]
    n0 = S * N * nb
    cnt = []
    for s in range(S):
        c = 0
        for j in range(N):
            o = s * N * nb + j * nb
            if np.any(L[n0:, o:o + nb] != 0.0):
                c += 1
        cnt.append(c)
    return cnt


def test_fill_in_orderings_of_fig2():
    # M = 2, N = 9 as in Fig. 2; root-row blocks of the factor per tail
    N, nb, nr = 9, 3, 3
    d = small(2, N, nb, nr, seed=3)
    fwd = list(range(1, N + 1))                          # (a)
    rev = list(range(N, 0, -1))                          # (b)
    full = [rev[j - 1] for j in dense.gamma(N)]          # (c) Gamma_N on the whole reversed tail
    prop = dense.tail_order(N)                           # (d)
    assert _root_row_blocks(fwd, N, nb, nr, d) == [N, N]
    assert _root_row_blocks(rev, N, nb, nr, d) == [1, 1]
    assert min(_root_row_blocks(full, N, nb, nr, d)) > 1
    assert _root_row_blocks(prop, N, nb, nr, d) == [1, 1]


def test_proposed_ordering_has_at_most_two_subdiagonal_blocks_per_column():
    N, nb = 23, 2
    d = small(1, N, nb, 1, seed=5)
    t = dense.permuted_tail_factor(d["D"][0], d["E"][0])
    L = t["L"]
    for c in range(N):
        nz = [r for r in range(c + 1, N) if np.any(dense.block(L, nb, r, c) != 0.0)]
        assert len(nz) <= 2


# --- ordering-invariant blocks --------------------------------------------------

@pytest.mark.parametrize("S,N,nb,nr", [(3, 9, 4, 2), (2, 16, 3, 3), (1, 1, 2, 2), (2, 2, 3, 1)])
def test_root_factor_and_logdet_are_ordering_invariant(S, N, nb, nr):
    d = small(S, N, nb, nr, seed=11, root="wishart", barrier=(-2, 2))
    nat = natural.factor(d["D"], d["E"], d["C"], d["R"])
    pf = dense.permuted_factor(d["D"], d["E"], d["C"], d["R"])
    n0 = S * N * nb
    LR_dense = pf["L"][n0:, n0:]
    assert np.allclose(nat["LR"], LR_dense, rtol=1e-9, atol=1e-12)
    ld = 2 * np.log(np.diag(pf["L"])).sum()
    assert abs(ld - nat["logdet"]) <= 1e-10 * max(1.0, abs(ld))
    # the generator fixes the exact root Schur complement to R0
    scale = np.abs(d["R"]).max()
    assert np.abs(nat["Rt"] - d["R0"]).max() <= 1e-12 * scale


@pytest.mark.parametrize("N", [1, 2, 5, 12])
def test_last_tail_block_equals_schur_onto_first_stage(N):
    S, nb = 2, 4
    d = small(S, N, nb, 2, seed=N + 40, barrier=(-2, 2))
    S1 = natural.tail_schur_first(d["D"], d["E"])
    for s in range(S):
        t = dense.permuted_tail_factor(d["D"][s], d["E"][s])
        L11 = dense.block(t["L"], nb, N - 1, N - 1)
        assert np.allclose(L11 @ L11.T, S1[s], rtol=1e-10, atol=1e-12 * np.abs(S1[s]).max())
        # S_1 is the inverse of the (1,1) block of K_i^{-1}
        Kt = dense.assemble_tail(d["D"][s], d["E"][s])
        inv11 = np.linalg.inv(Kt)[:nb, :nb]
        assert np.allclose(np.linalg.inv(S1[s]), inv11, rtol=1e-8, atol=1e-12)


# --- closed forms ---------------------------------------------------------------

def _thomas(a, b, c, d):
    """Scalar tridiagonal solve (sub a, diag b, super c), textbook recursion."""
    n = len(b)
    cp, dp = np.zeros(n), np.zeros(n)
    cp[0] = c[0] / b[0] if n > 1 else 0.0
    dp[0] = d[0] / b[0]
    for i in range(1, n):
        m = b[i] - a[i - 1] * cp[i - 1]
        cp[i] = c[i] / m if i < n - 1 else 0.0
        dp[i] = (d[i] - a[i - 1] * dp[i - 1]) / m
    x = np.zeros(n)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def test_nb1_is_bordered_scalar_tridiagonal():
    S, N = 4, 11
    d = small(S, N, 1, 1, seed=2, barrier=(-1, 1))
    out = natural.solve_system(d)
    # block elimination of the border with Thomas solves: x_i = w_i - z_i x0
    r = d["r"]
    zs, ws = [], []
    rhs0, schur = r[-1], np.tril(d["R"])[0, 0]
    for s in range(S):
        diag = d["D"][s, :, 0, 0]
        sub = d["E"][s, :, 0, 0]
        e1 = np.zeros(N)
        e1[0] = d["C"][s, 0, 0]
        z = _thomas(sub, diag, sub, e1)
        w = _thomas(sub, diag, sub, r[s * N:(s + 1) * N])
        zs.append(z)
        ws.append(w)
        schur -= e1 @ z
        rhs0 -= e1 @ w
    x0 = rhs0 / schur
    xref = np.concatenate([w - z * x0 for z, w in zip(zs, ws)] + [[x0]])
    assert np.allclose(out["x"], xref, rtol=1e-10, atol=1e-12 * np.abs(xref).max())


def _block_thomas(D, E, rhs):
    """Block tridiagonal solve, textbook block LU recursion: diagonal blocks
    D[k] (full symmetric), sub-diagonal E[k] = block (k+1, k), super-diagonal
    E[k]^T; rhs is (N*nb, m)."""
    N, nb = D.shape[0], D.shape[1]
    rhs = rhs.reshape(N, nb, -1)
    Cp, dp = [None] * N, [None] * N
    M = D[0]
    for k in range(N):
        if k > 0:
            M = D[k] - E[k - 1] @ Cp[k - 1]
        r = rhs[k] - (E[k - 1] @ dp[k - 1] if k > 0 else 0.0)
        dp[k] = np.linalg.solve(M, r)
        if k + 1 < N:
            Cp[k] = np.linalg.solve(M, E[k].T)
    x = [None] * N
    x[-1] = dp[-1]
    for k in range(N - 2, -1, -1):
        x[k] = dp[k] - Cp[k] @ x[k + 1]
    return np.concatenate(x).reshape(N * nb, -1)


def test_s1_is_bordered_block_tridiagonal():
    """One tail: a block tridiagonal matrix bordered by the root on its first
    stage, solved by block Thomas recursions and the border's Schur complement."""
    N, nb, nr = 9, 3, 2
    d = small(1, N, nb, nr, seed=6, barrier=(-2, 2))
    out = natural.solve_system(d)
    D = np.array([np.tril(b) + np.tril(b, -1).T for b in d["D"][0]])
    E = d["E"][0]
    C, r = d["C"][0], d["r"]
    Rl = np.tril(d["R"])
    B = np.zeros((N * nb, nr))
    B[:nb] = C.T                       # border: root coupled to stage 1 only
    Z = _block_thomas(D, E, B)
    w = _block_thomas(D, E, r[:N * nb].reshape(-1, 1))[:, 0]
    schur = Rl + np.tril(Rl, -1).T - B.T @ Z
    x0 = np.linalg.solve(schur, r[N * nb:] - B.T @ w)
    xref = np.concatenate([w - Z @ x0, x0])
    assert np.allclose(out["x"], xref, rtol=1e-10, atol=1e-12 * np.abs(xref).max())


def test_n1_is_arrow_matrix():
    S, nb, nr = 5, 3, 2
    d = small(S, 1, nb, nr, seed=4)
    out = natural.solve_system(d)
    r = d["r"]
    Rl = np.tril(d["R"])
    schur = Rl + np.tril(Rl, -1).T
    rhs0 = r[S * nb:].copy()
    Dfull = []
    for s in range(S):
        Dl = np.tril(d["D"][s, 0])
        Ds = Dl + np.tril(Dl, -1).T
        Dfull.append(Ds)
        Cs = d["C"][s]
        schur = schur - Cs @ np.linalg.solve(Ds, Cs.T)
        rhs0 = rhs0 - Cs @ np.linalg.solve(Ds, r[s * nb:(s + 1) * nb])
    x0 = np.linalg.solve(schur, rhs0)
    xs = [np.linalg.solve(Dfull[s], r[s * nb:(s + 1) * nb] - d["C"][s].T @ x0) for s in range(S)]
    xref = np.concatenate(xs + [x0])
    assert np.allclose(out["x"], xref, rtol=1e-11, atol=1e-13 * np.abs(xref).max())


def test_dense_permuted_factor_solves_the_system():
    d = small(3, 9, 3, 2, seed=8, barrier=(-2, 2))
    pf = dense.permuted_factor(d["D"], d["E"], d["C"], d["R"])
    L, P = pf["L"], pf["P"]
    rh = d["r"][P]
    y = sla.solve_triangular(L, rh, lower=True)
    xh = sla.solve_triangular(L.T, y, lower=False)
    x = np.empty_like(xh)
    x[P] = xh
    xref = dense.dense_solve(d["D"], d["E"], d["C"], d["R"], d["r"])
    assert np.allclose(x, xref, rtol=1e-10, atol=1e-12 * np.abs(xref).max())


# --- the generator's recipe --------------------------------------------------------

def test_generator_is_spd_and_deterministic():
    w = bmgen.WORKLOADS["plain-s4-n16-nb4"]
    a = bmgen.generate(w)
    b = bmgen.generate(w)
    for k in ("D", "E", "C", "R", "r"):
        assert np.array_equal(a[k].numpy(), b[k].numpy())
    K = dense.assemble_system(a["D"], a["E"], a["C"], a["R"])
    assert np.linalg.eigvalsh(K).min() > 0
    # stage block formula D_k = A Q^-1 A^T + B R^-1 B^T + Q^-1 is symmetric
    D = a["D"].numpy()
    assert np.array_equal(D, np.swapaxes(D, -1, -2))


# --- residual measures: |K| |x| and the componentwise backward error ---------------

@pytest.mark.parametrize("S,N,nb,nr", CASES)
def test_abs_kx_matches_dense_assembly(S, N, nb, nr):
    d = small(S, N, nb, nr, seed=7 * S + N, barrier=(-2, 2))
    g = np.random.default_rng(S + N + nb)
    x = g.standard_normal(S * N * nb + nr)
    K = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    want = np.abs(K) @ np.abs(x)
    got = natural.abs_kx(d["D"], d["E"], d["C"], d["R"], x)
    assert np.allclose(got, want, rtol=1e-14, atol=0.0)
    # a transposed sub-diagonal block is seen (E_k is not symmetric)
    if N > 1 and nb > 1:
        bad = natural.abs_kx(d["D"], np.swapaxes(d["E"], -1, -2), d["C"], d["R"], x)
        assert not np.allclose(bad, want, rtol=1e-8, atol=0.0)


def test_omega_closed_form_two_by_two():
    # K = [[2, 1], [1, 3]] (S = N = nb = nr = 1), x = (1, 1), r = (4, 3):
    # K x = (3, 4), rho = (1, -1), |K||x| + |r| = (7, 7) -> omega = 1/7
    D = np.array([[[[2.0]]]])
    E = np.zeros((1, 0, 1, 1))
    C = np.array([[[1.0]]])
    R = np.array([[3.0]])
    res = natural.residual(D, E, C, R, np.array([1.0, 1.0]), np.array([4.0, 3.0]))
    assert res["omega"] == pytest.approx(1.0 / 7.0, rel=1e-15)
    assert res["rel_inf"] == pytest.approx(0.25, rel=1e-15)
    assert res["eta"] == pytest.approx(1.0 / (4.0 * 1.0 + 4.0), rel=1e-15)


@pytest.mark.parametrize("S,N,nb,nr", CASES[:5])
def test_omega_against_dense_definition(S, N, nb, nr):
    d = small(S, N, nb, nr, seed=11 * S + N, barrier=(-2, 2))
    xref = dense.dense_solve(d["D"], d["E"], d["C"], d["R"], d["r"])
    # the exact solution has a tiny componentwise backward error
    assert natural.residual(d["D"], d["E"], d["C"], d["R"], xref, d["r"])["omega"] < 1e-14
    # a perturbed one: omega equals the definition on the dense matrix
    g = np.random.default_rng(N)
    x = xref * (1.0 + 1e-6 * g.standard_normal(xref.shape))
    K = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    want = (np.abs(d["r"] - K @ x) / (np.abs(K) @ np.abs(x) + np.abs(d["r"]))).max()
    got = natural.residual(d["D"], d["E"], d["C"], d["R"], x, d["r"])["omega"]
    assert got == pytest.approx(want, rel=1e-6)


# --- the pins catch plausible mistakes (planted into the oracle's inputs) ---------

def test_pins_detect_transposed_subdiagonal():
    d = small(2, 6, 3, 2, seed=21)
    xref = dense.dense_solve(d["D"], d["E"], d["C"], d["R"], d["r"])
    bad = dict(d)
    bad["E"] = np.swapaxes(d["E"], -1, -2).copy()
    x_bad = natural.solve_system(bad)["x"]
    assert np.abs(x_bad - xref).max() > 1e-6 * np.abs(xref).max()


def test_pins_detect_shifted_stage_alignment():
    d = small(2, 6, 3, 2, seed=22, barrier=(-2, 2))   # stage-varying E_k
    xref = dense.dense_solve(d["D"], d["E"], d["C"], d["R"], d["r"])
    bad = dict(d)
    bad["E"] = np.roll(d["E"], 1, axis=1)
    try:
        x_bad = natural.solve_system(bad)["x"]
    except natural.NotSPD:
        return                                       # the misaligned matrix is not even SPD
    assert np.abs(x_bad - xref).max() > 1e-6 * np.abs(xref).max()


def test_pins_detect_wrong_gamma_start():
    # a Gamma that starts with the second block instead of the first breaks the example
    def gamma_wrong(n):
        def rec(seq):
            if not seq:
                return []
            if len(seq) == 1:
                return seq
            return seq[1::2] + rec(seq[0::2])
        return rec(list(range(1, n + 1)))
    gold = _read_golden("gamma7.txt")[0]
    want = [int(t) for t in gold.replace("|", " ").split()]
    assert gamma_wrong(7) != want


@pytest.mark.parametrize("S,N,nb,nr", CASES[:6])
def test_residual_rows_matches_dense_rows(S, N, nb, nr):
    d = small(S, N, nb, nr, seed=13 * S + N, barrier=(-2, 2))
    g = np.random.default_rng(S * N)
    x = g.standard_normal(S * N * nb + nr)
    K = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    rows = np.arange(K.shape[0])
    got = natural.residual_rows(d["D"], d["E"], d["C"], d["R"], x, d["r"], rows)
    assert np.allclose(got["rho"], d["r"] - K @ x, rtol=1e-12, atol=1e-12 * np.abs(K @ x).max())
    want = (np.abs(d["r"] - K @ x) / (np.abs(K) @ np.abs(x) + np.abs(d["r"]))).max()
    assert got["omega"] == pytest.approx(want, rel=1e-9)


def test_exact_residual_rows():
    """residual_rows_exact: zero residual where r = K x holds exactly (small
    integer entries, where the FP64 product K x is itself exact), agreement
    with the FP64 rows to FP64 rounding elsewhere, and the exact value where
    FP64 summation cancels to zero."""
    d = small(2, 5, 3, 2, seed=4, barrier=(-1, 1))
    g = np.random.default_rng(7)
    D, E, C, R = (np.round(4 * np.asarray(d[k])) for k in ("D", "E", "C", "R"))
    x = g.integers(-5, 6, size=2 * 5 * 3 + 2).astype(np.float64)
    K = dense.assemble_system(D, E, C, R)
    r = K @ x                                   # exact: small integers
    rows = np.arange(K.shape[0])
    ex = natural.residual_rows_exact(D, E, C, R, x, r, rows)
    assert np.array_equal(ex["rho"], np.zeros(rows.size))
    assert np.allclose(ex["abs_kx"], np.abs(K) @ np.abs(x))
    y = g.standard_normal(x.size)
    ex = natural.residual_rows_exact(d["D"], d["E"], d["C"], d["R"], y, d["r"], rows)
    Kd = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    assert np.allclose(ex["rho"], np.asarray(d["r"]) - Kd @ y, rtol=0,
                       atol=1e-13 * (np.abs(Kd) @ np.abs(y)).max())
    # a row whose FP64 sum, left to right, loses the 1: 1e16 * 1 + 1 * 1 + 1e16 * (-1)
    D1 = np.zeros((1, 1, 3, 3))
    D1[0, 0, 2] = [1e16, 1.0, 1e16]
    C1, R1, E1 = np.zeros((1, 1, 3)), np.eye(1), np.zeros((1, 0, 3, 3))
    x1, r1 = np.array([1.0, 1.0, -1.0, 0.0]), np.zeros(4)
    assert (1e16 * 1.0 + 1.0 * 1.0) + 1e16 * -1.0 == 0.0
    ex = natural.residual_rows_exact(D1, E1, C1, R1, x1, r1, [2])
    assert ex["rho"][0] == -1.0 and ex["abs_kx"][0] == 2e16 + 1

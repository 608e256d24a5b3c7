"""Pins of the assembly front end's oracle (oracle/qp.py) against what the
paper and the mathematics fix: App. A's reduced matrix
K = P + tau I + delta^{-1} A^T A + G^T (W + delta I)^{-1} G is symmetric
positive definite, its quadratic form equals the cost, regularization,
constraint-residual and inequality terms evaluated one constraint at a time,
it has the block pattern of Sec. III-B (block-tridiagonal tails, the root
coupled to stage 1 of each tail only), and a 3 x 3 case matches a hand
computation.
"""
import numpy as np
import pytest

import bmgen
from oracle import qp as oq

SHAPES = [(1, 1, 1, 1), (2, 3, 2, 1), (3, 4, 3, 2), (2, 6, 4, 2), (1, 5, 2, 3)]


@pytest.mark.parametrize("S,N,nx,nu", SHAPES)
def test_quadratic_form_matches_definition(S, N, nx, nu):
    d = bmgen.generate_qp(S, N, nx, nu, seed=S + 10 * N)
    K = oq.reduced_kkt(d)
    g = np.random.default_rng(N)
    for _ in range(3):
        v = g.standard_normal(K.shape[0])
        assert v @ K @ v == pytest.approx(oq.quadratic_form(d, v), rel=1e-12)


@pytest.mark.parametrize("S,N,nx,nu", SHAPES)
def test_reduced_matrix_is_spd_with_the_branch_pattern(S, N, nx, nu):
    d = bmgen.generate_qp(S, N, nx, nu, seed=7 * S + N)
    K = oq.reduced_kkt(d)
    assert np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() > 0
    nb = nx + nu
    n0 = S * N * nb

    def blk(s, k):                        # stage k (1-based) of scenario s
        o = s * N * nb + (k - 1) * nb
        return slice(o, o + nb)
    for s in range(S):
        for t in range(S):
            for k in range(1, N + 1):
                for l in range(1, N + 1):
                    if s != t or abs(k - l) > 1:
                        assert not K[blk(s, k), blk(t, l)].any()
        for k in range(2, N + 1):
            assert not K[blk(s, k), n0:].any()      # the root sees stage 1 only
    # the stage-(k+1, k) block is delta^{-1} [[-A_k, -B_k], [0, 0]]
    if N > 1:
        A, B = d["A"].numpy(), d["B"].numpy()
        E = K[blk(0, 2), blk(0, 1)]
        want = np.zeros((nb, nb))
        want[:nx, :nx] = -A[0, 1] / d["delta"]
        want[:nx, nx:] = -B[0, 1] / d["delta"]
        assert np.allclose(E, want, rtol=1e-14, atol=0.0)


def test_three_by_three_by_hand():
    # S = N = nx = nu = 1: variables (x_1, u_1, u_0); one constraint x_1 - b u_0 = 0
    d = bmgen.generate_qp(1, 1, 1, 1, seed=3)
    q, rw, r0 = float(d["q"][0, 0, 0]), float(d["rw"][0, 0, 0]), float(d["r0w"][0])
    wx, wu, w0 = float(d["w"][0, 0, 0]), float(d["w"][0, 0, 1]), float(d["w0"][0])
    b, tau, dl = float(d["B"][0, 0, 0, 0]), d["tau"], d["delta"]
    want = np.array([[q + tau + 1 / (wx + dl) + 1 / dl, 0.0, -b / dl],
                     [0.0, rw + tau + 1 / (wu + dl), 0.0],
                     [-b / dl, 0.0, r0 + tau + 1 / (w0 + dl) + b * b / dl]])
    assert np.allclose(oq.reduced_kkt(d), want, rtol=1e-14, atol=0.0)


def test_pins_detect_transposed_dynamics():
    d = bmgen.generate_qp(2, 4, 3, 1, seed=9)
    bad = dict(d)
    bad["A"] = d["A"].transpose(-1, -2).contiguous()
    v = np.random.default_rng(1).standard_normal(oq.layout(d)["n"])
    assert abs(v @ oq.reduced_kkt(bad) @ v - oq.quadratic_form(d, v)) > 1e-6 * abs(oq.quadratic_form(d, v))

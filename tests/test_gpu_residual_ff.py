"""Float-float refinement residual of the mixed path, through the C ABI.

With tol >= 1e-11 (and no BM_FLAG_RESIDUAL_FP64) the refinement computes
rho = r - K x on the FP32 pipe: K and x split into hi + lo floats, exact
products (TwoProduct), TwoSum for the running sum and FP64 accumulation of
every 8 terms, with |rho_ff - rho|_i <= 4e-12 (|K||x|)_i (the bound in
bm_mixed.cuh), and stops at omega <= tol - 4e-12. These tests check:
  * bm_residual row by row against the exact residual (rational
    arithmetic, oracle.natural.residual_rows_exact) within that bound, on
    barrier-scaled systems at a refined iterate (where r - K x cancels most);
  * that accepted iterates meet tol by the oracle's FP64 omega, that the
    reported omega is the oracle's to within the bound, and that the
    iteration counts are those of FP64 residuals;
  * the mode selection (tolerance, flag) and the fallback to FP64 residuals
    when an entry of K or x leaves 2^-50..2^50;
  * repeatability.
"""
import numpy as np
import pytest
import torch

import bmgen
from oracle import natural

pytestmark = pytest.mark.gpu

BETA = 4e-12


def _bm():
    import paper_2609_29977_gb300 as bm
    return bm


def gen(S, N, nb, nr, seed=0, barrier=(-6.0, 6.0), root_scale=1.0, root="wishart"):
    w = bmgen.Workload("f", S, N, nb, nr, workload_id=94, barrier=barrier, root=root, shared_A=True)
    d = bmgen.generate(w, seed=seed)
    if root_scale != 1.0:
        d["R"] = d["R"] - (1.0 - root_scale) * d["R0"]
        d["R0"] = root_scale * d["R0"]
    return d


def solve(d, tol=1e-10, flags=0, max_refine=10, residual_of=None):
    bm = _bm()
    g = {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
    solver = bm.BranchKKTSolver(d["S"], d["N"], d["nb"], d["nr"], precision=bm.BM_PREC_FP32_IR,
                                max_refine=max_refine, tol=tol, flags=flags)
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    x = solver.solve(g["r"])
    x2 = solver.solve(g["r"])
    info = solver.query()
    rho = None
    if residual_of is not None:
        rho = solver.residual(g["r"], torch.as_tensor(residual_of, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    out = {"x": x.cpu().numpy(), "x2": x2.cpu().numpy(), "info": info, "rho": rho}
    solver.close()
    return out


def sample_rows(d, count=360, seed=0):
    S, N, nb, nr = d["S"], d["N"], d["nb"], d["nr"]
    n = S * N * nb + nr
    if n <= count:
        return np.arange(n)
    g = np.random.default_rng(seed)
    # first and last block rows of every tail, the root rows, then random rows
    fixed = [s * N * nb + k * nb + i for s in range(S) for k in (0, N - 1) for i in range(nb)]
    fixed += list(range(S * N * nb, n))
    rest = g.choice(n, size=max(count - len(fixed), 0), replace=False)
    return np.unique(np.concatenate([np.asarray(fixed, dtype=np.int64), rest]))


SHAPES = [(4, 16, 4, 2), (3, 2, 3, 3), (2, 33, 12, 4), (3, 20, 16, 5), (2, 12, 24, 8), (1, 7, 48, 16),
          (5, 31, 8, 9), (2, 1, 6, 2)]


@pytest.mark.parametrize("S,N,nb,nr", SHAPES)
def test_float_float_residual_rows_match_exact(S, N, nb, nr):
    d = gen(S, N, nb, nr, seed=5 * S + N + nb)
    bm = _bm()
    first = solve(d, tol=1e-10)
    x = first["x"]
    ff = solve(d, tol=1e-10, residual_of=x)
    f64 = solve(d, tol=1e-10, flags=bm.BM_FLAG_RESIDUAL_FP64, residual_of=x)
    assert ff["info"]["residual_float_float"] == 1 and f64["info"]["residual_float_float"] == 0
    rows = sample_rows(d, seed=S + N)
    ex = natural.residual_rows_exact(d["D"], d["E"], d["C"], d["R"], x, d["r"], rows)
    kx = ex["abs_kx"]
    err_ff = np.abs(ff["rho"][rows] - ex["rho"])
    err_64 = np.abs(f64["rho"][rows] - ex["rho"])
    assert np.all(err_ff <= BETA * kx + 1e-300), (err_ff / np.maximum(kx, 1e-300)).max()
    # the FP64 residual: about (terms in the row) 2^-53 |K||x| at most
    assert np.all(err_64 <= (3 * nb + S * nb + nr) * 2.0 ** -53 * kx + 1e-300)
    # at a refined iterate the residual is far below |K||x| (the check is not
    # vacuous: rho is what is left after cancelling |K||x| by 6+ digits)
    assert np.median(np.abs(ex["rho"]) / np.maximum(kx, 1e-300)) < 1e-6, first["info"]


@pytest.mark.parametrize("S,N,nb,nr,scale,b", [(8, 24, 12, 4, 1.0, 6), (6, 40, 24, 8, 3.1e-4, 4),
                                               (4, 64, 24, 8, 1.0, 6), (3, 17, 16, 5, 1.0, 6)])
def test_float_float_refinement_meets_tolerance(S, N, nb, nr, scale, b):
    """Barrier 10^(+-b); scale < 1: a root that cancels by about 1e3 / scale,
    with the coupling columns refined."""
    bm = _bm()
    d = gen(S, N, nb, nr, seed=S * N, barrier=(-b, b), root_scale=scale, root="scaled_identity")
    cf = bm.BM_FLAG_COUPLING_REFINE if scale < 1.0 else 0
    ff = solve(d, tol=1e-10, flags=cf)
    f64 = solve(d, tol=1e-10, flags=cf | bm.BM_FLAG_RESIDUAL_FP64)
    info = ff["info"]
    assert info["status"] == 0 and info["residual_float_float"] == 1, info
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], ff["x"], d["r"])
    assert res["omega"] <= 1e-10, res["omega"]
    assert abs(info["backward_error"] - res["omega"]) <= BETA + 1e-3 * res["omega"], (info, res["omega"])
    assert abs(info["iters"] - f64["info"]["iters"]) <= 1, (info, f64["info"])
    assert np.array_equal(ff["x"], ff["x2"])


def test_float_float_mode_selection():
    bm = _bm()
    d = gen(2, 9, 6, 3, seed=1)
    assert solve(d, tol=1e-11)["info"]["residual_float_float"] == 1
    assert solve(d, tol=0)["info"]["residual_float_float"] == 1            # default 1e-10
    assert solve(d, tol=1e-12)["info"]["residual_float_float"] == 0
    assert solve(d, tol=1e-8, flags=bm.BM_FLAG_RESIDUAL_FP64)["info"]["residual_float_float"] == 0
    assert bm.ff_residual(1e-11) and not bm.ff_residual(1e-12)
    # FP64 handles have no refinement residual
    solver = bm.BranchKKTSolver(2, 9, 6, 3)
    g = {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    with pytest.raises(RuntimeError):
        solver.residual(g["r"], g["r"].clone())
    solver.close()


def test_float_float_falls_back_outside_its_range():
    """A diagonal entry of 2^55 (outside 2^-50..2^50; K stays SPD): the
    refinement computes FP64 residuals instead and still meets tol."""
    d = gen(3, 12, 8, 3, seed=2, barrier=(-2.0, 2.0))
    d["D"][1, 5, 2, 2] *= 2.0 ** 55
    out = solve(d, tol=1e-10)
    info = out["info"]
    assert info["status"] == 0 and info["residual_float_float"] == 0, info
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], out["x"], d["r"])
    assert res["omega"] <= 1e-10

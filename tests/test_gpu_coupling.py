"""Mixed precision with refined coupling columns, through the C ABI.

The FP32 tail factor gives each local Schur update U_i = C_{i,1}
(K_i^{-1})_{11} C_{i,1}^T (Alg. 1 step 3) only to FP32-level accuracy, and
R - sum_i U_i (step 4) cancels strongly on barrier-scaled systems. The
library then refines X_i = K_i^{-1} C_i^T with the FP32 factor and a
float-float residual, forms U_i from X_i in FP64 and uses X_i for the root
coupling of every solve. These tests check, against the FP64 oracle:
  * the root factor L_R built from the refined columns (element by element,
    at a bound set by the cancellation of the root block),
  * the solution (componentwise backward error omega <= tol of the oracle's
    own FP64 residual, forward error bounded by omega times cond(K)),
  * the automatic choice (engaged when the root's cancellation times the
    FP32 factor's pivot spread times 2^-24 exceeds 16, or when the
    FP32-based root is not positive definite, or later by the solve when the
    refinement fails without it),
  * graph and direct launches bit for bit, and repeatability.
"""
import numpy as np
import pytest
import torch

import bmgen
from oracle import dense, natural

pytestmark = pytest.mark.gpu


def _bm():
    import paper_2609_29977_gb300 as bm
    return bm


def gen(S, N, nb, nr, seed=0, barrier=(-2.0, 2.0), root="scaled_identity", shared_A=False, root_scale=1.0):
    """A generated system; root_scale < 1 shrinks the exact root Schur
    complement R0 to root_scale * R0 (R -> R - (1 - root_scale) R0), which
    keeps K SPD and raises the cancellation of R - sum_i U_i by 1/root_scale."""
    w = bmgen.Workload("c", S, N, nb, nr, workload_id=93, barrier=barrier, root=root, shared_A=shared_A)
    d = bmgen.generate(w, seed=seed)
    if root_scale != 1.0:
        d["R"] = d["R"] - (1.0 - root_scale) * d["R0"]
        d["R0"] = root_scale * d["R0"]
    return d


def run(d, flags=0, tol=1e-10, max_refine=10, export=False, direct=False):
    bm = _bm()
    g = {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
    f = flags | (bm.BM_FLAG_NO_GRAPH if direct else 0)
    solver = bm.BranchKKTSolver(d["S"], d["N"], d["nb"], d["nr"], precision=bm.BM_PREC_FP32_IR,
                                max_refine=max_refine, tol=tol, flags=f)
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    x = solver.solve(g["r"])
    info = solver.query()
    fac = solver.export_factor() if export else None
    torch.cuda.synchronize()
    out = {"x": x.cpu().numpy(), "info": info,
           "fac": {k: v.cpu().numpy() for k, v in fac.items()} if fac else None}
    solver.close()
    return out


def cancellation(d):
    """max_j R_jj / R~_jj of the exact root Schur complement R~ = R0."""
    return float((d["R"].diagonal() / d["R0"].diagonal()).max())


SHAPES = [(4, 16, 4, 2), (1, 1, 3, 2), (3, 2, 3, 3), (2, 9, 6, 3), (2, 33, 12, 4), (3, 20, 16, 5),
          (2, 12, 24, 8), (1, 7, 48, 16), (2, 10, 2, 1), (5, 31, 8, 9), (3, 40, 24, 12)]


@pytest.mark.parametrize("S,N,nb,nr", SHAPES)
def test_refined_coupling_reaches_tolerance(S, N, nb, nr):
    bm = _bm()
    d = gen(S, N, nb, nr, seed=3 * S + N + nb, barrier=(-5, 5), root="wishart")
    out = run(d, flags=bm.BM_FLAG_COUPLING_REFINE, tol=1e-12)
    info = out["info"]
    assert info["status"] == 0 and info["coupling_refined"] == 1, info
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], out["x"], d["r"])
    assert res["omega"] <= 2e-12, res
    assert abs(info["backward_error"] - res["omega"]) <= 0.1 * res["omega"] + 1e-16, (info, res["omega"])
    ref = natural.solve_system(d)
    K = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    kappa = np.linalg.cond(K)
    fwd = np.abs(out["x"] - ref["x"]).max() / np.abs(ref["x"]).max()
    assert fwd <= max(1e-12, 1e-12 * kappa * 10), (fwd, kappa)


@pytest.mark.parametrize("S,N,nb,nr,scale", [(8, 24, 12, 4, 6.7e-3), (6, 40, 24, 8, 3.1e-4), (4, 17, 6, 3, 2.4e-3)])
def test_refined_root_factor_matches_oracle(S, N, nb, nr, scale):
    """L_R from the refined columns against the oracle's FP64 L_R, on roots
    that cancel by about 3e4, 3e5 and 1e4 (the mixed workload's is 2.7e4).
    The root block R~ = R - sum_i U_i is a scaled identity, so L_R's
    relative error is about half that of R~, which is at most the
    cancellation gamma times the relative error of the U_i. One refinement
    step with an exact residual leaves the U_i with at least 8 correct
    digits on these tails (about 5 from the FP32 factor alone), and the
    refined root must beat the FP32-based one by at least 2 digits."""
    bm = _bm()
    d = gen(S, N, nb, nr, seed=S + N, barrier=(-4, 4), shared_A=True, root_scale=scale)
    gamma = cancellation(d)
    ref = natural.factor(d["D"], d["E"], d["C"], d["R"])
    LRo = ref["LR"]
    fine = run(d, flags=bm.BM_FLAG_COUPLING_REFINE, export=True)
    coarse = run(d, flags=bm.BM_FLAG_COUPLING_FP32, export=True)
    assert fine["info"]["coupling_refined"] == 1 and coarse["info"]["coupling_refined"] == 0
    assert fine["info"]["status"] == 0, fine["info"]
    e_fine = np.abs(np.tril(fine["fac"]["LR"]) - LRo).max() / np.abs(LRo).max()
    assert e_fine <= 1e-8 * gamma, (e_fine, gamma)
    if coarse["info"]["status"] != 2:
        e_coarse = np.abs(np.tril(coarse["fac"]["LR"]) - LRo).max() / np.abs(LRo).max()
        assert e_fine <= 1e-2 * e_coarse, (e_fine, e_coarse)


def test_automatic_mode_engages_on_cancellation():
    """Default flags: a root that cancels by 1.6e6 after these FP32 tails
    (pivot spread about 3e3) engages the refinement and converges; the same
    tails with a root that cancels by 1.6e2 do not engage it."""
    d_hi = gen(8, 24, 12, 4, seed=21, barrier=(-4, 4), shared_A=True, root_scale=1e-4)
    d_lo = gen(8, 24, 12, 4, seed=21, barrier=(-4, 4), shared_A=True)
    assert cancellation(d_hi) > 1e6 and cancellation(d_lo) < 1e3
    hi = run(d_hi)
    lo = run(d_lo)
    assert hi["info"]["coupling_refined"] == 1 and hi["info"]["status"] == 0, hi["info"]
    assert lo["info"]["coupling_refined"] == 0 and lo["info"]["status"] == 0, lo["info"]
    for d, out in ((d_hi, hi), (d_lo, lo)):
        res = natural.residual(d["D"], d["E"], d["C"], d["R"], out["x"], d["r"])
        assert res["omega"] <= 2e-10, res


def test_automatic_mode_resolves_cancellation_of_1e6():
    """A root that cancels by about 1e6 (the FP32-based root is then not
    positive definite): the automatic mode refines and converges."""
    bm = _bm()
    d = gen(6, 40, 24, 8, seed=5, barrier=(-5, 5), shared_A=True, root_scale=1.4e-4)
    assert 5e5 < cancellation(d) < 2e6
    coarse = run(d, flags=bm.BM_FLAG_COUPLING_FP32)
    auto = run(d)
    assert coarse["info"]["status"] != 0, coarse["info"]
    assert auto["info"]["coupling_refined"] == 1 and auto["info"]["status"] == 0, auto["info"]
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], auto["x"], d["r"])
    assert res["omega"] <= 2e-10, res


RESUME_CASES = [(2, 12, 24, 8, 46, "wishart"), (4, 64, 24, 8, 256, "wishart"), (6, 40, 24, 8, 240, "scaled_identity")]


@pytest.mark.parametrize("S,N,nb,nr,seed,root", RESUME_CASES)
def test_automatic_mode_resumes_a_failed_refinement(S, N, nb, nr, seed, root):
    """Barrier 10^+-6 systems whose FP32-based root passes the factor's probe
    (indicator 0.9 to 5) but on which the refinement stalls near 1e-8 with
    it: the default mode resumes the same solve with refined coupling
    columns and converges; the next solve on that factor uses them from the
    start; the graph and direct forms give the same bits; forcing the
    FP32-based root still reports the stall."""
    bm = _bm()
    w = bmgen.Workload("c", S, N, nb, nr, workload_id=94, barrier=(-6.0, 6.0), root=root, shared_A=True)
    d = bmgen.generate(w, seed=seed)
    coarse = run(d, flags=bm.BM_FLAG_COUPLING_FP32)
    assert coarse["info"]["status"] == 5 and coarse["info"]["coupling_refined"] == 0, coarse["info"]
    outs = []
    for direct in (False, True):
        g = {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
        solver = bm.BranchKKTSolver(S, N, nb, nr, precision=bm.BM_PREC_FP32_IR, tol=1e-10,
                                    flags=bm.BM_FLAG_NO_GRAPH if direct else 0)
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        x1 = solver.solve(g["r"]).cpu().numpy()
        i1 = solver.query()
        x2 = solver.solve(g["r"]).cpu().numpy()
        i2 = solver.query()
        solver.close()
        outs.append((x1, i1, x2, i2))
        assert i1["status"] == 0 and i1["coupling_refined"] == 1, i1
        assert i2["status"] == 0 and i2["coupling_refined"] == 1, i2
        for x in (x1, x2):
            res = natural.residual(d["D"], d["E"], d["C"], d["R"], x, d["r"])
            assert res["omega"] <= 1e-10, res["omega"]
        assert i2["iters"] <= i1["iters"], (i1, i2)
    (a1, ai1, a2, ai2), (b1, bi1, b2, bi2) = outs
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    for k in ("status", "iters", "backward_error"):
        assert ai1[k] == bi1[k] and ai2[k] == bi2[k], (k, ai1, bi1)


def test_unresolvable_cancellation_is_reported():
    """A root that cancels by about 1e9 is beyond one refinement step of the
    coupling columns (their U_i carry 8 to 11 digits): the path must report
    the failure (BM_ERR_NOT_CONVERGED, or BM_ERR_NOT_SPD at the root), and
    its reported backward error must be the oracle's, not a false success."""
    d = gen(6, 40, 24, 8, seed=5, barrier=(-5, 5), shared_A=True, root_scale=1e-7)
    assert cancellation(d) > 5e8
    auto = run(d)
    info = auto["info"]
    assert info["coupling_refined"] == 1, info
    if info["status"] == 5:
        res = natural.residual(d["D"], d["E"], d["C"], d["R"], auto["x"], d["r"])
        assert res["omega"] > 1e-10 and abs(info["backward_error"] - res["omega"]) <= 0.1 * res["omega"], (info, res)
    else:
        assert info["status"] == 2 and info["fail_scenario"] == -1, info


@pytest.mark.parametrize("tol,max_refine", [(1e-10, 10), (1e-30, 2)])
def test_refined_graph_and_direct_agree_bitwise(tol, max_refine):
    bm = _bm()
    d = gen(5, 31, 8, 9, seed=8, barrier=(-4, 4), shared_A=True, root_scale=1e-4)
    outs = [run(d, flags=bm.BM_FLAG_COUPLING_REFINE, tol=tol, max_refine=max_refine, direct=direct)
            for direct in (False, True)]
    (a, b) = outs
    assert np.array_equal(a["x"], b["x"])
    for k in ("status", "iters", "backward_error", "coupling_refined"):
        assert a["info"][k] == b["info"][k], (k, a["info"], b["info"])
    assert a["info"]["coupling_refined"] == 1


def test_refined_is_deterministic_and_refactors():
    """Repeated factor + solve on one handle gives the same bits, and a new
    factor with other values (same pointers) is used by the next solve."""
    bm = _bm()
    d = gen(3, 21, 8, 3, seed=5, barrier=(-4, 4), root_scale=1e-4)
    g = {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
    solver = bm.BranchKKTSolver(3, 21, 8, 3, precision=bm.BM_PREC_FP32_IR, tol=1e-12,
                                flags=bm.BM_FLAG_COUPLING_REFINE)
    xs = []
    for _ in range(3):
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        xs.append(solver.solve(g["r"]).cpu().numpy())
    assert all(np.array_equal(xs[0], x) for x in xs[1:])
    # scaling K by 4 scales x by 1/4 exactly (powers of two are exact)
    for k in ("D", "E", "C", "R"):
        g[k].mul_(4.0)
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    x4 = solver.solve(g["r"]).cpu().numpy()
    info = solver.query()
    solver.close()
    assert info["status"] == 0
    assert np.array_equal(x4, xs[0] / 4.0)


def test_conflicting_coupling_flags_are_rejected():
    bm = _bm()
    with pytest.raises(RuntimeError):
        bm.BranchKKTSolver(2, 4, 4, 2, precision=bm.BM_PREC_FP32_IR,
                           flags=bm.BM_FLAG_COUPLING_REFINE | bm.BM_FLAG_COUPLING_FP32)

"""The FP32-tail + FP64-refinement path (BM_PREC_FP32_IR) through the C ABI.

Parity bar (mixed path): refinement stops on the componentwise backward
error omega = max_i |r - K x|_i / (|K||x| + |r|)_i <= tol (1e-10 unless a
test asks for less); the oracle's omega of the returned x must meet it
(within a factor 2: two differently rounded FP64 residuals, and FP32 weights
on the device), and the solution is compared with the FP64 oracle, the
difference bounded by omega times a condition estimate. The FP32 tail
factor is checked against the dense FP64 factor within FP32 rounding
(well-conditioned systems), and the library's FP64->FP32 rounding is
checked bit for bit against the hardware conversion.
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


def gen(S, N, nb, nr, seed=0, barrier=(-2.0, 2.0), root="scaled_identity", shared_A=False):
    w = bmgen.Workload("m", S, N, nb, nr, workload_id=92, barrier=barrier, root=root, shared_A=shared_A)
    return bmgen.generate(w, seed=seed)


def to_dev(d):
    return {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}


def run_mixed(d, tol=1e-10, max_refine=10, export=False):
    bm = _bm()
    g = to_dev(d)
    solver = bm.BranchKKTSolver(d["S"], d["N"], d["nb"], d["nr"], precision=bm.BM_PREC_FP32_IR,
                                max_refine=max_refine, tol=tol)
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    x = solver.solve(g["r"])
    info = solver.query()
    fac = solver.export_factor() if export else None
    torch.cuda.synchronize()
    out = {"x": x.cpu().numpy(), "info": info,
           "fac": {k: v.cpu().numpy() for k, v in fac.items()} if fac else None}
    solver.close()
    return out


def test_round_to_fp32_matches_hardware_conversion():
    bm = _bm()
    g = torch.Generator().manual_seed(0)
    parts = [
        torch.randn(200000, dtype=torch.float64, generator=g) * torch.pow(10.0, torch.randint(-40, 40, (200000,),
                                                                                             generator=g).double()),
        torch.tensor([0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, 1e39, -1e39,
                      float("inf"), float("-inf"), 1.1754943508222875e-38, 1.401298464324817e-45,
                      7.006492321624085e-46, 7.006492321624087e-46, 2.1019476964872256e-45, 1e-50, -1e-310,
                      1.0000000596046448, 1.0000001788139343, 1.0000000596046446], dtype=torch.float64),
        # values exactly halfway between two floats, both parities
        (torch.arange(1, 2001, dtype=torch.float64) * 2.0 + 1.0) * 2.0 ** -24,
    ]
    src = torch.cat(parts).cuda()
    dst = torch.empty(src.numel(), dtype=torch.float32, device="cuda")
    bm.bm_round_to_fp32(src, dst)
    ref = src.float()
    assert torch.equal(dst.view(torch.int32), ref.view(torch.int32))
    nan = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    bm.bm_round_to_fp32(nan, out)
    assert torch.isnan(out).all()


@pytest.mark.parametrize("S,N,nb,nr", [(4, 16, 4, 2), (1, 1, 3, 2), (3, 2, 3, 3), (2, 9, 6, 3), (2, 33, 12, 4),
                                       (3, 20, 16, 5), (2, 12, 24, 8), (1, 7, 48, 16), (2, 10, 2, 1)])
def test_mixed_reaches_tolerance(S, N, nb, nr):
    d = gen(S, N, nb, nr, seed=S + 7 * N + nb, root="wishart")
    out = run_mixed(d, tol=1e-12)
    assert out["info"]["status"] == 0, out["info"]
    x = out["x"]
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], x, d["r"])
    assert res["omega"] <= 2e-12 and res["eta"] <= 1e-12, res
    # the device's own figure agrees with the oracle's
    dev = out["info"]["backward_error"]
    assert dev <= 1e-12 and abs(dev - res["omega"]) <= 0.1 * res["omega"] + 1e-16, (dev, res["omega"])
    ref = natural.solve_system(d)
    K = dense.assemble_system(d["D"], d["E"], d["C"], d["R"])
    kappa = np.linalg.cond(K)
    fwd = np.abs(x - ref["x"]).max() / np.abs(ref["x"]).max()
    assert fwd <= max(1e-12, 1e-12 * kappa * 10), (fwd, kappa)


def test_mixed_fp32_factor_is_the_rounded_factor():
    S, N, nb, nr = 2, 17, 6, 3
    d = gen(S, N, nb, nr, seed=3, barrier=None)
    out = run_mixed(d, export=True)
    fac = out["fac"]
    order = dense.tail_order(N)
    pos = {st: i for i, st in enumerate(order)}
    worst = 0.0
    for s in range(S):
        L = dense.permuted_tail_factor(d["D"][s], d["E"][s])["L"]
        scale = np.abs(L).max()
        for k in range(1, N + 1):
            ref = dense.block(L, nb, pos[k], pos[k])
            worst = max(worst, np.abs(fac["Ld"][s, k - 1] - ref).max() / scale)
    assert 0.0 < worst <= 2e-5, worst       # FP32 rounding, not FP64 agreement


def test_mixed_refines_and_reports_iterations():
    w = bmgen.WORKLOADS["medium-s64-n64-nb12"]
    d = bmgen.generate(w)
    loose = run_mixed(d, tol=1e-8)
    tight = run_mixed(d, tol=1e-14)
    assert loose["info"]["status"] == 0 and tight["info"]["status"] == 0
    assert tight["info"]["iters"] > loose["info"]["iters"]
    for out, tol in ((loose, 1e-8), (tight, 1e-14)):
        res = natural.residual(d["D"], d["E"], d["C"], d["R"], out["x"], d["r"])
        assert res["omega"] <= 2 * tol, (res["omega"], tol)
    # at 1e-14 the mixed solution agrees with the FP64 oracle's to the
    # oracle's own accuracy on this workload
    ref = natural.solve_system(d)
    fwd = np.abs(tight["x"] - ref["x"]).max() / np.abs(ref["x"]).max()
    assert fwd <= 1e-9, fwd


def test_mixed_not_converged_is_reported():
    d = gen(2, 9, 4, 2, seed=11, barrier=(-3, 3))
    out = run_mixed(d, tol=1e-30, max_refine=1)
    assert out["info"]["status"] == 5, out["info"]          # BM_ERR_NOT_CONVERGED
    assert np.all(np.isfinite(out["x"]))
    assert out["info"]["iters"] == 1


def test_mixed_is_deterministic():
    bm = _bm()
    d = gen(3, 21, 8, 3, seed=5)
    g = to_dev(d)
    solver = bm.BranchKKTSolver(3, 21, 8, 3, precision=bm.BM_PREC_FP32_IR, tol=1e-13)
    xs = []
    for _ in range(3):
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        xs.append(solver.solve(g["r"]).cpu().numpy())
    assert all(np.array_equal(xs[0], x) for x in xs[1:])
    solver.close()


@pytest.mark.parametrize("tol,max_refine", [(1e-10, 10), (1e-14, 10), (1e-30, 3), (1e-30, 1), (1e-30, 0)])
def test_mixed_graph_loop_and_direct_launch_agree_bitwise(tol, max_refine):
    """The captured solve (refinement as a conditional loop node) and the
    directly launched, unrolled solve give the same bits, iteration count,
    status and backward error: on convergence, on reaching max_refine and
    on a stall."""
    bm = _bm()
    S, N, nb, nr = 3, 21, 8, 3
    d = gen(S, N, nb, nr, seed=12, barrier=(-3, 3))
    g = to_dev(d)
    outs = []
    for flags in (0, bm.BM_FLAG_NO_GRAPH):
        solver = bm.BranchKKTSolver(S, N, nb, nr, precision=bm.BM_PREC_FP32_IR, max_refine=max_refine, tol=tol,
                                    flags=flags)
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        x = solver.solve(g["r"])
        outs.append((x.cpu().numpy(), solver.query()))
        solver.close()
    (xa, ia), (xb, ib) = outs
    assert np.array_equal(xa, xb)
    for k in ("status", "iters", "backward_error"):
        assert ia[k] == ib[k], (k, ia, ib)
    assert ia["iters"] <= (max_refine if max_refine > 0 else 10)   # <= 0 selects the default, 10
    if tol == 1e-30:
        assert ia["status"] == 5, ia


def test_mixed_graph_loop_restarts_on_replay():
    """A replay of the captured solve runs the whole loop again: with the
    right-hand side scaled by -2 in place (same pointers, so the same graph),
    every step of the method scales exactly, so the solution must be exactly
    -2 times the first one after the same number of corrections."""
    bm = _bm()
    S, N, nb, nr = 2, 17, 6, 3
    d = gen(S, N, nb, nr, seed=4, barrier=(-3, 3))
    g = to_dev(d)
    solver = bm.BranchKKTSolver(S, N, nb, nr, precision=bm.BM_PREC_FP32_IR, tol=1e-13)
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    r = g["r"].clone()
    x = torch.empty_like(r)
    solver.solve(r, x)
    i1 = solver.query()
    x1 = x.clone()
    r.mul_(-2.0)
    solver.solve(r, x)
    i2 = solver.query()
    solver.close()
    assert i1["status"] == 0 and i2["status"] == 0 and i1["iters"] >= 1
    assert i2["iters"] == i1["iters"]
    assert torch.equal(x, -2.0 * x1)


def test_mixed_not_spd_is_reported():
    bm = _bm()
    d = gen(2, 8, 4, 2, seed=6)
    g = to_dev(d)
    D = g["D"].clone()
    D[1, 4] = -torch.eye(4, dtype=torch.float64, device="cuda")
    solver = bm.BranchKKTSolver(2, 8, 4, 2, precision=bm.BM_PREC_FP32_IR)
    solver.factor(D, g["E"], g["C"], g["R"])
    solver.solve(g["r"])
    info = solver.query()
    assert info["status"] == 2 and info["fail_scenario"] == 1 and info["fail_stage"] == 5, info
    solver.close()


def test_mixed_workload_full_size():
    """The mixed-precision workload at full size (S=512, N=128, nb=24, nr=8,
    barrier 10^U[-6,6]) at the 1e-10 target. Its root Schur complement
    R - sum_i U_i cancels by 2.7e4 on the diagonal (the generator makes it
    exactly R0 = nr I) while FP32 tail factors give each U_i only to about
    1e-5, so the FP32-based root is wrong by O(1). The automatic mode must
    see that, refine the coupling columns, and reach omega <= 1e-10 against
    the oracle's own FP64 residual."""
    w = bmgen.WORKLOADS["mixed-s512-n128-nb24"]
    d = bmgen.generate(w)
    out = run_mixed(d, tol=1e-10, max_refine=8)
    info = out["info"]
    assert info["status"] == 0, info
    assert info["coupling_refined"] == 1, info
    assert info["backward_error"] <= 1e-10, info
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], out["x"], d["r"])
    assert res["omega"] <= 2e-10, res
    assert abs(info["backward_error"] - res["omega"]) <= 0.1 * res["omega"] + 1e-16, (info, res["omega"])
    # sanity bound on the forward error against the oracle's FP64 solution
    # (omega <= 1e-10 bounds it by 1e-10 times the componentwise condition
    # number, which is far below 1e6 on these systems)
    ref = natural.solve_system(d)
    fwd = np.abs(out["x"] - ref["x"]).max() / np.abs(ref["x"]).max()
    assert fwd <= 1e-4, fwd

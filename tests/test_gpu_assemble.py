"""The assembly front end (bm_assemble_reduced) through the C ABI: the
library's D, E, C, R of App. A's reduced matrix against the dense oracle
(oracle/qp.py) entry by entry, then the assembled system factored and solved
on the GPU and checked against the oracle's residual."""
import numpy as np
import pytest
import torch

import bmgen
from oracle import dense, natural
from oracle import qp as oq

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1, 1), (2, 3, 2, 1), (3, 9, 4, 2), (5, 17, 8, 4), (2, 33, 12, 4), (4, 20, 20, 4),
          (2, 7, 36, 12)]


def _bm():
    import paper_2609_29977_gb300 as bm
    return bm


def _to(d, dev):
    return {k: (v.to(dev) if isinstance(v, torch.Tensor) else v) for k, v in d.items()}


@pytest.mark.parametrize("S,N,nx,nu", SHAPES)
def test_assembly_matches_dense_oracle(S, N, nx, nu):
    bm = _bm()
    qp = bmgen.generate_qp(S, N, nx, nu, seed=S + 3 * N + nx)
    out = bm.bm_assemble_reduced(_to(qp, "cuda"))
    torch.cuda.synchronize()
    K = dense.assemble_system(*(out[k].cpu().numpy() for k in ("D", "E", "C", "R")))
    want = oq.reduced_kkt(qp)
    scale = np.abs(want).max()
    assert np.abs(K - want).max() <= 1e-14 * scale, np.abs(K - want).max() / scale
    D = out["D"].cpu().numpy()
    assert np.array_equal(D, np.swapaxes(D, -1, -2))       # full symmetric stage blocks


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_assembled_system_is_solved(precision):
    bm = _bm()
    S, N, nx, nu = 6, 40, 12, 4
    qp = bmgen.generate_qp(S, N, nx, nu, seed=77, barrier=(-2.0, 2.0), delta=1e-2)
    sysd = bm.bm_assemble_reduced(_to(qp, "cuda"))
    n = bmgen.n_unknowns(S, N, nx + nu, nu)
    r = torch.randn(n, dtype=torch.float64, generator=torch.Generator().manual_seed(5)).cuda()
    solver = bm.BranchKKTSolver(S, N, nx + nu, nu, precision=precision, tol=1e-12)
    solver.factor(sysd["D"], sysd["E"], sysd["C"], sysd["R"])
    x = solver.solve(r)
    info = solver.query()
    solver.close()
    assert info["status"] == 0, info
    host = {k: sysd[k].cpu().numpy() for k in ("D", "E", "C", "R")}
    res = natural.residual(host["D"], host["E"], host["C"], host["R"], x.cpu().numpy(), r.cpu().numpy())
    assert res["eta"] <= 1e-12 and res["omega"] <= (1e-12 if precision else 1e-13), res


def test_assembly_rejects_bad_arguments():
    bm = _bm()
    qp = _to(bmgen.generate_qp(2, 3, 2, 1, seed=1), "cuda")
    bad = dict(qp)
    bad["delta"] = 0.0
    with pytest.raises(bm.BMError):
        bm.bm_assemble_reduced(bad)
    big = _to(bmgen.generate_qp(1, 2, 60, 8, seed=1), "cuda")     # nb = 68 > 64
    with pytest.raises(bm.BMError):
        bm.bm_assemble_reduced(big)

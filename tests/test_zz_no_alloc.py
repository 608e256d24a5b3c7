"""bm_factor_solve_noalloc: the entry point for callers that cannot
allocate device memory (allocator callbacks, real-time loops, fixed
memory budgets). It keeps the whole FP64 factor in the library's fixed
scratch array; here it must give the same x as the handle-based entry
points (bm_analyze + bm_factor + bm_solve) on two calls in a row, the
second on a different system, so nothing left in the shared array from the
first call leaks into the second, and meet the FP64 path's bar against the
oracle's residual. It synchronizes before returning, so a stream that is
being captured into a CUDA graph is refused. Kept in its own file,
collected last."""
import numpy as np
import pytest
import torch

import bmgen
from oracle import natural

pytestmark = pytest.mark.gpu


def _system(S, N, nb, nr, seed):
    w = bmgen.Workload("noalloc", S, N, nb, nr, workload_id=93, barrier=(-3.0, 3.0), root="wishart")
    d = bmgen.generate(w, seed=seed)
    return {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}


def _handle_solution(bm, g):
    solver = bm.BranchKKTSolver(g["S"], g["N"], g["nb"], g["nr"])
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    x = solver.solve(g["r"])
    assert solver.query()["status"] == 0
    solver.close()
    return x


def test_noalloc_matches_handle_entry_points_on_two_calls():
    import paper_2609_29977_gb300 as bm
    for seed, shape in ((1, (64, 64, 12, 4)), (2, (5, 23, 7, 3))):
        g = _system(*shape, seed=seed)
        ref = _handle_solution(bm, g)
        x = torch.full_like(g["r"], float("nan"))
        code = bm.bm_factor_solve_noalloc(*shape, g["D"], g["E"], g["C"], g["R"], g["r"], x)
        assert code == 0
        xr, xn = ref.cpu().numpy(), x.cpu().numpy()
        assert np.all(np.isfinite(xn))
        assert np.abs(xn - xr).max() <= 1e-12 * np.abs(xr).max()
        # the FP64 path's parity bar against the oracle's own residual
        res = natural.residual(g["D"], g["E"], g["C"], g["R"], xn, g["r"])
        assert res["eta"] <= 1e-12, res


def test_noalloc_rejects_systems_larger_than_the_scratch_array():
    import paper_2609_29977_gb300 as bm
    S, N, nb, nr = 512, 128, 24, 8          # needs far more than 32 MiB
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    code = bm.bm_factor_solve_noalloc(S, N, nb, nr, t, t, t, t, t, torch.zeros_like(t))
    assert code == 1                         # BM_ERR_INVALID_ARG, before any work


def test_noalloc_refuses_a_capturing_stream():
    import paper_2609_29977_gb300 as bm
    S, N, nb, nr = 2, 9, 4, 2
    g = _system(S, N, nb, nr, seed=3)
    x = torch.zeros_like(g["r"])
    marker = torch.zeros(1, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        code = bm.bm_factor_solve_noalloc(S, N, nb, nr, g["D"], g["E"], g["C"], g["R"], g["r"], x)
        marker.add_(1.0)
    assert code == 1                         # BM_ERR_INVALID_ARG, nothing launched
    torch.cuda.synchronize()
    assert float(x.abs().max()) == 0.0
    # still usable outside the capture
    assert bm.bm_factor_solve_noalloc(S, N, nb, nr, g["D"], g["E"], g["C"], g["R"], g["r"], x) == 0

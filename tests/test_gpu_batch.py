"""The batched form (bm_batch_*): many systems of uneven S, N, nb, nr
factored in one persistent launch and solved with FP32 tails + FP64
refinement. Each system must reach the tolerance on the componentwise
backward error against the oracle's FP64 residual, and must give bitwise the
same x as the single-system path
(bm_factor/bm_solve in BM_PREC_FP32_IR) -- the same result alone and in the
mix. A failing system reports its own status without disturbing the others.
"""
import os

import numpy as np
import pytest
import torch

import bmgen
from oracle import natural

pytestmark = pytest.mark.gpu


def _bm():
    import paper_2609_29977_gb300 as bm
    return bm


def _shapes(seed, count, nbs=(4, 6, 12, 24, 48), Smax=10, Nmax=40):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nb = int(g.choice(nbs))
        out.append((int(g.integers(1, Smax + 1)), int(g.integers(1, Nmax + 1)), nb, -(-nb // 3)))
    return out


def _gen(shapes, seed0=100):
    systems = []
    for j, (S, N, nb, nr) in enumerate(shapes):
        w = bmgen.Workload("b", S, N, nb, nr, workload_id=94, barrier=(-3.0, 3.0), shared_A=True)
        systems.append(bmgen.generate(w, seed=seed0 + j))
    return systems


def _solve_batch(shapes, systems, tol=1e-12, max_refine=10):
    bm = _bm()
    dev = [{k: v.cuda() for k, v in d.items() if isinstance(v, torch.Tensor)} for d in systems]
    batch = bm.BranchKKTBatch(shapes, max_refine=max_refine, tol=tol)
    batch.factor([d["D"] for d in dev], [d["E"] for d in dev], [d["C"] for d in dev], [d["R"] for d in dev])
    xs = batch.solve([d["r"] for d in dev])
    infos = batch.query()
    out = [x.cpu().numpy() for x in xs]
    sched = batch.schedule()
    batch.close()
    return out, infos, sched


def test_batch_matches_oracle_and_single_path(tmp_path, monkeypatch):
    monkeypatch.setenv("BM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    bm = _bm()
    shapes = _shapes(1, 12) + [(1, 1, 4, 2), (3, 2, 6, 2), (2, 17, 24, 8), (1, 9, 48, 16)]
    systems = _gen(shapes)
    xs, infos, sched = _solve_batch(shapes, systems)
    assert sched["status"] == 0 and sched["threads_per_cta"] in (64, 128, 256)
    for (S, N, nb, nr), d, x, info in zip(shapes, systems, xs, infos):
        assert info["status"] == 0, (S, N, nb, nr, info)
        res = natural.residual(d["D"], d["E"], d["C"], d["R"], x, d["r"])
        assert res["omega"] <= 2e-12 and res["eta"] <= 1e-12, ((S, N, nb, nr), res)
        # the same system alone through the single-system path
        g = {k: v.cuda() for k, v in d.items() if isinstance(v, torch.Tensor)}
        single = bm.BranchKKTSolver(S, N, nb, nr, precision=bm.BM_PREC_FP32_IR, tol=1e-12)
        single.factor(g["D"], g["E"], g["C"], g["R"])
        xs1 = single.solve(g["r"]).cpu().numpy()
        assert single.query()["iters"] == info["iters"]
        single.close()
        assert np.array_equal(xs1, x), (S, N, nb, nr)


def test_batch_autotune_cache_is_reused(tmp_path, monkeypatch):
    monkeypatch.setenv("BM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    shapes = _shapes(2, 6)
    systems = _gen(shapes, 300)
    _, _, s1 = _solve_batch(shapes, systems)
    assert not s1["from_cache"]
    assert os.path.exists(tmp_path / "tune.json")
    _, _, s2 = _solve_batch(shapes, systems)
    assert s2["from_cache"]
    assert (s2["threads_per_cta"], s2["ctas_per_sm"]) == (s1["threads_per_cta"], s1["ctas_per_sm"])


def test_batch_isolates_a_failing_system(tmp_path, monkeypatch):
    monkeypatch.setenv("BM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    shapes = [(3, 9, 6, 2), (2, 12, 12, 4), (4, 7, 4, 2)]
    systems = _gen(shapes, 500)
    bad = dict(systems[1])
    bad["D"] = bad["D"].clone()
    bad["D"][1, 3] = -torch.eye(12, dtype=torch.float64)
    systems[1] = bad
    xs, infos, _ = _solve_batch(shapes, systems)
    assert infos[1]["status"] == 2 and infos[1]["fail_scenario"] == 1 and infos[1]["fail_stage"] == 4, infos[1]
    for k in (0, 2):
        assert infos[k]["status"] == 0
        d = systems[k]
        res = natural.residual(d["D"], d["E"], d["C"], d["R"], xs[k], d["r"])
        assert res["omega"] <= 2e-12


def test_batch_rejects_unsupported_shapes():
    bm = _bm()
    with pytest.raises(bm.BMError):
        bm.BranchKKTBatch([(2, 4, 5, 2)])        # nb = 5 is not a batched block size
    assert bm.bm_batch_workspace_bytes([(2, 4, 6, 2), (3, 5, 12, 4)]) > 0

"""Parity at full benchmark sizes, in the launch configurations the bench
times, on outputs the oracle can check one by one.

- The batched workload (256 systems, S ~ U{8..256}, N ~ U{16..256},
  nb in {6, 12, 24, 48}) in one persistent launch: every system's device
  componentwise backward error <= tol, and sampled systems checked by the
  oracle (whole systems for the smaller ones, sampled rows for the rest).
- The large serving request (S=2048, N=256, nb=48, nr=16) with FP32 tails
  and refinement: the oracle's residual on every row of four sampled
  scenarios and on all root rows.
"""
import numpy as np
import pytest
import torch

import bmgen
from oracle import natural

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _bm():
    import paper_2609_29977_gb300 as bm
    return bm


def _host(t):
    return t.cpu().numpy()


def test_batched_workload_full_size(tmp_path, monkeypatch):
    monkeypatch.setenv("BM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    bm = _bm()
    shapes = bmgen.draw_batched_shapes(256)
    base = bmgen.Workload("batched", 1, 1, 1, 1, workload_id=4, barrier=(-4.0, 4.0), shared_A=True)
    systems = [bmgen.generate(base.with_shape(S=S, N=N, nb=nb, nr=nr), instance=j, device="cuda")
               for j, (S, N, nb, nr) in enumerate(shapes)]
    batch = bm.BranchKKTBatch(shapes, tol=TOL)
    batch.factor([d["D"] for d in systems], [d["E"] for d in systems], [d["C"] for d in systems],
                 [d["R"] for d in systems])
    xs = batch.solve([d["r"] for d in systems])
    infos = batch.query()
    batch.close()
    assert all(i["status"] == 0 for i in infos), [i for i in infos if i["status"]]
    assert max(i["backward_error"] for i in infos) <= TOL
    # sampled systems against the oracle: the smallest whole, the others by rows
    sizes = [S * N * nb * nb for (S, N, nb, _) in shapes]
    small = int(np.argmin(sizes))
    picks = [small] + [j for j in (1, 77, 200) if j != small]
    g = np.random.default_rng(4)
    for j in picks:
        d = {k: _host(systems[j][k]) for k in ("D", "E", "C", "R", "r")}
        x = _host(xs[j])
        S, N, nb, nr = shapes[j]
        if j == small:
            res = natural.residual(d["D"], d["E"], d["C"], d["R"], x, d["r"])
            om = res["omega"]
        else:
            n = S * N * nb + nr
            rows = np.concatenate([g.choice(S * N * nb, 1500, replace=False), np.arange(S * N * nb, n)])
            om = natural.residual_rows(d["D"], d["E"], d["C"], d["R"], x, d["r"], rows)["omega"]
        assert om <= 2 * TOL, (j, shapes[j], om, infos[j])


def test_large_request_full_size():
    bm = _bm()
    w = bmgen.WORKLOADS["large-s2048-n256-nb48"]
    d = bmgen.generate(w, device="cuda")
    S, N, nb, nr = w.S, w.N, w.nb, w.nr
    solver = bm.BranchKKTSolver(S, N, nb, nr, precision=bm.BM_PREC_FP32_IR, tol=TOL)
    solver.factor(d["D"], d["E"], d["C"], d["R"])
    x = solver.solve(d["r"])
    info = solver.query()
    solver.close()
    assert info["status"] == 0 and info["backward_error"] <= TOL, info
    n0 = S * N * nb
    # every row of four sampled scenarios (their tail rows need only their own blocks)
    for s in (0, 511, 1500, 2047):
        sub = {"D": _host(d["D"][s:s + 1]), "E": _host(d["E"][s:s + 1]), "C": _host(d["C"][s:s + 1]),
               "R": _host(d["R"])}
        xs = np.concatenate([_host(x[s * N * nb:(s + 1) * N * nb]), _host(x[n0:])])
        rs = np.concatenate([_host(d["r"][s * N * nb:(s + 1) * N * nb]), np.zeros(nr)])
        om = natural.residual_rows(sub["D"], sub["E"], sub["C"], sub["R"], xs, rs, np.arange(N * nb))["omega"]
        assert om <= 2 * TOL, (s, om)
    # all root rows: R x_0 + sum_s C_s x_1^s (a one-stage view of every tail's first block)
    x1 = _host(x[:n0].view(S, N, nb)[:, 0].reshape(-1))
    xr = np.concatenate([x1, _host(x[n0:])])
    rr = np.concatenate([np.zeros(S * nb), _host(d["r"][n0:])])
    D1 = np.zeros((S, 1, nb, nb))
    E1 = np.zeros((S, 0, nb, nb))
    om = natural.residual_rows(D1, E1, _host(d["C"]), _host(d["R"]), xr, rr, np.arange(S * nb, S * nb + nr))["omega"]
    assert om <= 2 * TOL, om

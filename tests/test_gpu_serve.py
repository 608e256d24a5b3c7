"""The serving runtime (bm_server_*) through the C ABI.

Each request is one system of Sec. III-B factored once (Alg. 1) and solved
for several right-hand sides (Alg. 2) against its resident factor. The
kernels and launch shapes of a request depend only on its shape, so a
request's solutions are bit-for-bit the same whether it runs alone or
overlapped with other requests; these tests check exactly that, check the
solutions against the oracle's FP64 residual, and check admission by device
memory (first in, first out; nothing admitted beyond the budget).
"""
import numpy as np
import pytest
import torch

import bmgen
from oracle import natural

pytestmark = pytest.mark.gpu

NRHS = 4
SHAPES = [(3, 17, 6, 2), (5, 40, 12, 4), (2, 9, 24, 8), (8, 33, 6, 2), (4, 64, 12, 4), (1, 1, 6, 2),
          (6, 20, 24, 8), (2, 130, 12, 4), (3, 5, 48, 16), (7, 16, 12, 4), (4, 28, 6, 2), (2, 3, 24, 8)]


def _bm():
    import paper_2609_29977_gb300 as bm
    return bm


def make_requests(shapes, seed0=0, barrier=(-3.0, 3.0)):
    out = []
    for i, (S, N, nb, nr) in enumerate(shapes):
        w = bmgen.Workload("serve", S, N, nb, nr, workload_id=93, barrier=barrier, shared_A=True)
        d = bmgen.generate(w, seed=seed0 + 17 * i, with_rhs=False)
        n = bmgen.n_unknowns(S, N, nb, nr)
        g = torch.Generator().manual_seed(seed0 + 17 * i + 1)
        d["rs"] = torch.randn((NRHS, n), generator=g, dtype=torch.float64)
        out.append(d)
    return out


def to_dev(d):
    return {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}


def submit(server, rid, g, x):
    server.submit(rid, g["S"], g["N"], g["nb"], g["nr"], g["D"], g["E"], g["C"], g["R"], g["rs"], x)


def run_alone(reqs, precision, tol=1e-12):
    """Each request alone: a one-slot server, one request at a time."""
    bm = _bm()
    server = bm.BranchKKTServer(2 << 30, slots=1, precision=precision, tol=tol)
    xs, comps = [], []
    for i, d in enumerate(reqs):
        g = to_dev(d)
        x = torch.empty_like(g["rs"])
        submit(server, i, g, x)
        comps += server.drain()
        xs.append(x.cpu().numpy())
    server.close()
    return xs, comps


def run_mix(reqs, precision, slots=8, budget=2 << 30, tol=1e-12, stagger=True):
    """All requests through one server: half submitted up front, the rest
    while the first ones are on the GPU."""
    bm = _bm()
    server = bm.BranchKKTServer(budget, slots=slots, precision=precision, tol=tol)
    gs = [to_dev(d) for d in reqs]
    xs = [torch.empty_like(g["rs"]) for g in gs]
    comps = []
    half = len(gs) // 2 if stagger else len(gs)
    for i in range(half):
        submit(server, i, gs[i], xs[i])
    for i in range(half, len(gs)):
        comps += server.poll()
        submit(server, i, gs[i], xs[i])
    comps += server.drain()
    stats = server.stats()
    server.close()
    return [x.cpu().numpy() for x in xs], comps, stats


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32ir"])
def test_same_result_alone_and_in_the_mix(precision):
    tol = 1e-12 if precision == 0 else 1e-11
    reqs = make_requests(SHAPES)
    alone, comps_alone = run_alone(reqs, precision, tol=tol)
    mixed, comps_mix, stats = run_mix(reqs, precision, tol=tol)
    assert stats["completed"] == len(reqs) and stats["queued"] == 0 and stats["in_flight"] == 0
    assert sorted(c["id"] for c in comps_mix) == list(range(len(reqs)))
    for c in comps_alone + comps_mix:
        assert c["status"] == 0, c
    for i, d in enumerate(reqs):
        assert np.array_equal(alone[i], mixed[i]), ("request", i, SHAPES[i])
        for j in range(NRHS):
            res = natural.residual(d["D"], d["E"], d["C"], d["R"], mixed[i][j], d["rs"][j])
            assert res["eta"] <= tol, (i, j, res["eta"])
            if precision == 1:
                assert res["omega"] <= 2 * tol, (i, j, res["omega"])
    # the same kernels as the single-system entry points (FP64: first rhs)
    if precision == 0:
        bm = _bm()
        for i in (0, 2, 8):
            g = to_dev(reqs[i])
            solver = bm.BranchKKTSolver(g["S"], g["N"], g["nb"], g["nr"])
            solver.factor(g["D"], g["E"], g["C"], g["R"])
            x = solver.solve(g["rs"][0].contiguous())
            assert np.array_equal(x.cpu().numpy(), mixed[i][0])
            solver.close()


def test_mixed_requests_report_refinement_per_rhs():
    bm = _bm()
    reqs = make_requests(SHAPES[:4])
    _, comps, _ = run_mix(reqs, bm.BM_PREC_FP32_IR, tol=1e-11)
    for c in comps:
        assert len(c["iters"]) == NRHS and all(it >= 1 for it in c["iters"])
        assert all(0.0 <= e <= 1e-11 for e in c["backward_error"]), c


def test_admission_respects_the_budget_fifo():
    """A budget that holds one request at a time: the requests run one after
    another in submission order, and the arena never holds more than that."""
    bm = _bm()
    one = to_dev(make_requests([(4, 40, 12, 4)], seed0=50)[0])
    gs = [one] * 5                                   # the same system five times
    xs = [torch.empty_like(g["rs"]) for g in gs]
    server = bm.BranchKKTServer(1 << 30, slots=4, precision=bm.BM_PREC_FP64)
    need = server.request_bytes(4, 40, 12, 4, gs[0]["D"], gs[0]["E"], gs[0]["C"], gs[0]["R"], gs[0]["rs"], xs[0])
    server.close()
    budget = need + need // 2                        # one fits, two do not
    server = bm.BranchKKTServer(budget, slots=4, precision=bm.BM_PREC_FP64)
    for i, g in enumerate(gs):
        submit(server, i, g, xs[i])
        st = server.stats()
        assert st["in_flight"] <= 1 and st["bytes_in_use"] <= budget
    comps = sorted(server.drain(), key=lambda c: c["id"])
    st = server.stats()
    server.close()
    assert st["peak_bytes_in_use"] == need and st["completed"] == 5
    for a, b in zip(comps, comps[1:]):
        assert b["t_start_us"] >= a["t_done_us"] - 1.0, (a, b)    # strictly one after another
    for c in comps:
        assert c["status"] == 0 and c["t_submit_us"] <= c["t_start_us"] + 5e3
        assert c["t_start_us"] <= c["t_factor_us"] <= c["t_done_us"]
    ref = xs[0].cpu().numpy()
    for x in xs[1:]:
        assert np.array_equal(x.cpu().numpy(), ref)   # the same system five times


def test_larger_budget_overlaps_requests():
    bm = _bm()
    reqs = make_requests([(16, 64, 12, 4)] * 6, seed0=70)
    _, comps, stats = run_mix(reqs, bm.BM_PREC_FP64, slots=6, stagger=False)
    comps.sort(key=lambda c: c["t_start_us"])
    # with six slots the later requests start before the first has finished
    assert comps[1]["t_start_us"] < comps[0]["t_done_us"]
    assert stats["peak_bytes_in_use"] > 0


def test_invalid_and_oversize_requests_are_rejected():
    bm = _bm()
    d = to_dev(make_requests([(2, 8, 6, 2)])[0])
    x = torch.empty_like(d["rs"])
    server = bm.BranchKKTServer(1 << 20, slots=2, precision=bm.BM_PREC_FP32_IR)
    big = to_dev(make_requests([(64, 64, 12, 4)])[0])
    xb = torch.empty_like(big["rs"])
    with pytest.raises(bm.BMError) as e:
        submit(server, 1, big, xb)                   # larger than the whole budget
    assert e.value.code == 1
    with pytest.raises(bm.BMError):
        server.submit(2, 2, 8, 6, 2, d["D"], d["E"], d["C"], d["R"], d["rs"], d["rs"])   # x aliases r
    bad = make_requests([(2, 8, 5, 2)])[0]           # nb = 5 has no FP32 tail kernel
    bad = to_dev(bad)
    with pytest.raises(bm.BMError):
        submit(server, 3, bad, torch.empty_like(bad["rs"]))
    nine = torch.zeros((9, d["rs"].shape[1]), dtype=torch.float64, device="cuda")
    with pytest.raises(bm.BMError):
        server.submit(4, 2, 8, 6, 2, d["D"], d["E"], d["C"], d["R"], nine, torch.empty_like(nine))
    submit(server, 5, d, x)
    comps = server.drain()
    assert [c["id"] for c in comps] == [5] and comps[0]["status"] == 0
    server.close()
    with pytest.raises(bm.BMError):
        bm.BranchKKTServer(0, slots=2)
    with pytest.raises(bm.BMError):
        bm.BranchKKTServer(1 << 20, slots=65)


def test_host_io_requests_match_device_requests():
    bm = _bm()
    reqs = make_requests(SHAPES[:5], seed0=90)
    dev_x, _, _ = run_mix(reqs, bm.BM_PREC_FP32_IR, tol=1e-11)
    server = bm.BranchKKTServer(1 << 30, slots=4, precision=bm.BM_PREC_FP32_IR, tol=1e-11)
    hx = []
    for i, d in enumerate(reqs):
        h = {k: (v.pin_memory() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}
        x = torch.empty_like(h["rs"]).pin_memory()
        hx.append((h, x))
        server.submit(i, h["S"], h["N"], h["nb"], h["nr"], h["D"], h["E"], h["C"], h["R"], h["rs"], x,
                      host_io=True)
    comps = server.drain()
    server.close()
    assert all(c["status"] == 0 for c in comps)
    for i in range(len(reqs)):
        assert np.array_equal(hx[i][1].numpy(), dev_x[i])


def test_failing_request_is_isolated():
    bm = _bm()
    reqs = make_requests(SHAPES[:6], seed0=110)
    alone, _ = run_alone(reqs, bm.BM_PREC_FP64)
    bad = 3
    S, N = reqs[bad]["S"], reqs[bad]["N"]
    reqs[bad]["D"] = reqs[bad]["D"].clone()
    reqs[bad]["D"][S - 1, N - 1] = -torch.eye(reqs[bad]["nb"], dtype=torch.float64)
    mixed, comps, _ = run_mix(reqs, bm.BM_PREC_FP64)
    by_id = {c["id"]: c for c in comps}
    assert by_id[bad]["status"] == 2, by_id[bad]
    assert by_id[bad]["fail_scenario"] == S - 1 and by_id[bad]["fail_stage"] == N
    for i in range(len(reqs)):
        if i != bad:
            assert by_id[i]["status"] == 0
            assert np.array_equal(mixed[i], alone[i])


def test_mixed_failure_falls_back_to_fp64():
    """A root Schur complement R - sum_i U_i that cancels to 1e-9 of R0: FP64
    resolves it, FP32 tails cannot. Without the fallback flag the mixed
    request reports its failure; with it, the server re-runs the request in
    FP64 and returns exactly the FP64 result."""
    bm = _bm()
    reqs = make_requests([(6, 24, 12, 4), (3, 17, 6, 2)], seed0=130)
    d = reqs[0]
    d["R"] = (d["R"] - (1.0 - 1e-9) * d["R0"]).contiguous()
    fp64_x, fp64_c = run_alone(reqs, bm.BM_PREC_FP64)
    assert all(c["status"] == 0 for c in fp64_c)
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], fp64_x[0][0], d["rs"][0])
    assert res["eta"] <= 1e-12
    _, plain, _ = run_mix(reqs, bm.BM_PREC_FP32_IR, tol=1e-12)
    by_id = {c["id"]: c for c in plain}
    assert by_id[0]["status"] in (2, 5) and by_id[0]["fallback"] == 0, by_id[0]
    assert by_id[1]["status"] == 0
    server = bm.BranchKKTServer(2 << 30, slots=4, precision=bm.BM_PREC_FP32_IR, tol=1e-12, fp64_fallback=True)
    gs = [to_dev(q) for q in reqs]
    xs = [torch.empty_like(g["rs"]) for g in gs]
    for i, g in enumerate(gs):
        submit(server, i, g, xs[i])
    comps = {c["id"]: c for c in server.drain()}
    st = server.stats()
    server.close()
    assert comps[0]["status"] == 0 and comps[0]["fallback"] == 1, comps[0]
    assert comps[1]["status"] == 0 and comps[1]["fallback"] == 0
    assert st["fallbacks"] == 1 and st["completed"] == 2
    assert np.array_equal(xs[0].cpu().numpy(), fp64_x[0])
    assert comps[0]["t_start_us"] <= comps[0]["t_factor_us"] <= comps[0]["t_done_us"]

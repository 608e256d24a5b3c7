"""Parity of the FP64 CUDA path (through the C ABI) with the oracle.

The factor of a fixed SPD ordering is unique, so every exported block of
L (Ld, Ll, Lr, F_{i,1}, L_R) is compared element by element with the dense
Cholesky factor of Pi K Pi^T from oracle.dense; the solution x is compared
with the natural-order oracle through the FP64 residual.

Tolerances (FP64 path): normwise backward error eta <= 1e-12 and relative
residual ||r - K x||_2 / ||r||_2 <= max(1e-12, 10 x the oracle's own); factor
blocks within 1e-12 of the largest entry of the tail factor (both sides are
backward-stable Cholesky factorizations of the same matrix in the same
order, so they differ by rounding only).
"""
import numpy as np
import pytest
import torch

import bmgen
from oracle import dense, natural

pytestmark = pytest.mark.gpu

ETA_TOL = 1e-12


def _bm():
    import paper_2609_29977_gb300 as bm
    return bm


def gen(S, N, nb, nr, seed=0, barrier=(-2.0, 2.0), root="scaled_identity", shared_A=False):
    w = bmgen.Workload("t", S, N, nb, nr, workload_id=91, barrier=barrier, root=root, shared_A=shared_A)
    return bmgen.generate(w, seed=seed)


def to_dev(d):
    return {k: (v.cuda() if isinstance(v, torch.Tensor) else v) for k, v in d.items()}


def run_gpu(d, flags=0, precision=0):
    bm = _bm()
    S, N, nb, nr = d["S"], d["N"], d["nb"], d["nr"]
    g = to_dev(d)
    solver = bm.BranchKKTSolver(S, N, nb, nr, precision=precision, flags=flags)
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    x = solver.solve(g["r"])
    info = solver.query()
    fac = solver.export_factor()
    torch.cuda.synchronize()
    out = {"x": x.cpu().numpy(), "info": info, "fac": {k: v.cpu().numpy() for k, v in fac.items()}}
    solver.close()
    return out


def neighbour_stages(N, k):
    """Natural stages of the left/right neighbours of stage k >= 2 at its
    elimination level (chain position p = N+1-k, level ctz(p))."""
    p = N + 1 - k
    lvl = (p & -p).bit_length() - 1
    h = 1 << lvl
    b = p + h if p + h <= N - 1 else N
    a = p - h if p > h else None
    return (None if a is None else N + 1 - a), N + 1 - b


def check_factor_blocks(d, fac, tails=None, tol=1e-12):
    S, N, nb = d["S"], d["N"], d["nb"]
    D, E, C = d["D"].numpy(), d["E"].numpy(), d["C"].numpy()
    order = dense.tail_order(N)
    pos = {st: i for i, st in enumerate(order)}
    worst = 0.0
    for s in (range(S) if tails is None else tails):
        t = dense.permuted_tail_factor(D[s], E[s], C[s])
        L = t["L"]
        scale = np.abs(L).max()
        for k in range(1, N + 1):
            pk = pos[k]
            ref = dense.block(L, nb, pk, pk)
            worst = max(worst, np.abs(fac["Ld"][s, k - 1] - ref).max() / scale)
            if k >= 2:
                a, b = neighbour_stages(N, k)
                ref_r = dense.block(L, nb, pos[b], pk)
                worst = max(worst, np.abs(fac["Lr"][s, k - 1] - ref_r).max() / scale)
                ref_l = dense.block(L, nb, pos[a], pk) if a is not None else np.zeros((nb, nb))
                worst = max(worst, np.abs(fac["Ll"][s, k - 1] - ref_l).max() / scale)
                # the factor column has no other non-zero block (fill confined)
                others = [r for r in range(N) if r not in (pk, pos[b]) and (a is None or r != pos[a])]
                for r in others:
                    if r > pk:
                        assert np.all(dense.block(L, nb, r, pk) == 0.0)
            else:
                assert np.all(fac["Ll"][s, 0] == 0.0) and np.all(fac["Lr"][s, 0] == 0.0)
        Fref = t["F"][:, (N - 1) * nb:]
        worst = max(worst, np.abs(fac["F"][s] - Fref).max() / max(1.0, np.abs(Fref).max()))
    assert worst <= tol, worst
    return worst


def check_solution(d, x, eta_tol=ETA_TOL):
    ref = natural.solve_system(d)
    res = natural.residual(d["D"], d["E"], d["C"], d["R"], x, d["r"])
    assert np.all(np.isfinite(x))
    assert res["eta"] <= eta_tol, res["eta"]
    assert res["rel2"] <= max(1e-12, 10 * ref["res"]["rel2"]), (res["rel2"], ref["res"]["rel2"])
    return res, ref


SHAPES = [
    (4, 16, 4, 2),     # the plain FP64 single-instance shape
    (1, 1, 3, 2),      # N = 1: pure arrow matrix
    (3, 2, 3, 3),      # N = 2: one chain position + x_1
    (2, 3, 2, 1),
    (2, 9, 5, 3),      # N - 1 = 2^3
    (2, 17, 4, 4),     # N - 1 = 2^4
    (3, 33, 6, 2),
    (2, 12, 1, 1),     # nb = 1: scalar tridiagonal + border
    (1, 20, 7, 9),     # nr > nb
    (5, 7, 12, 4),
    (2, 6, 24, 8),
    (1, 5, 48, 16),    # multi-warp blocks
    (2, 4, 64, 64),    # largest supported blocks
]


@pytest.mark.parametrize("S,N,nb,nr", SHAPES)
def test_fp64_factor_blocks_and_solution(S, N, nb, nr):
    d = gen(S, N, nb, nr, seed=S * 31 + N * 7 + nb, root="wishart")
    out = run_gpu(d)
    assert out["info"]["status"] == 0, out["info"]
    check_factor_blocks(d, out["fac"])
    nat = natural.factor(d["D"], d["E"], d["C"], d["R"])
    assert np.allclose(out["fac"]["LR"], nat["LR"], rtol=0, atol=1e-12 * np.abs(nat["LR"]).max())
    check_solution(d, out["x"])


def test_fp64_plain_workload_parity():
    w = bmgen.WORKLOADS["plain-s4-n16-nb4"]
    d = bmgen.generate(w)
    out = run_gpu(d)
    assert out["info"]["status"] == 0
    check_factor_blocks(d, out["fac"])
    res, ref = check_solution(d, out["x"])
    fwd = np.abs(out["x"] - ref["x"]).max() / np.abs(ref["x"]).max()
    assert fwd <= 1e-10, fwd


def test_fp64_medium_workload_full_size():
    """The medium FP64 workload at full size, in the launch configuration the
    benchmark times (graphs on): x against the oracle (backward error, and
    element by element within the condition-number bound), L_R exactly, and
    the tail factors of sampled scenarios element by element."""
    w = bmgen.WORKLOADS["medium-s64-n64-nb12"]
    d = bmgen.generate(w)
    out = run_gpu(d)
    assert out["info"]["status"] == 0
    check_factor_blocks(d, out["fac"], tails=[0, 17, 63])
    res, ref = check_solution(d, out["x"])
    nat = ref["fac"]
    assert np.allclose(out["fac"]["LR"], nat["LR"], rtol=0, atol=1e-9 * np.abs(nat["LR"]).max())
    # x element by element against the oracle's x: two backward-stable FP64
    # solves differ by at most about kappa_1(K) times the sum of their
    # normwise backward errors (||K||_1 = ||K||_inf, K symmetric; ||K^-1||_1
    # estimated by Higham's method through the oracle's own factor)
    import scipy.sparse.linalg as spla
    n = ref["x"].size
    kinv = spla.LinearOperator((n, n), matvec=lambda v: natural.solve(nat, np.ascontiguousarray(v, dtype=np.float64)),
                               rmatvec=lambda v: natural.solve(nat, np.ascontiguousarray(v, dtype=np.float64)),
                               dtype=np.float64)
    kappa = res["K_inf"] * spla.onenormest(kinv)
    bound = 10.0 * kappa * (res["eta"] + ref["res"]["eta"]) + 1e-15
    diff = np.abs(out["x"] - ref["x"]) / np.abs(ref["x"]).max()
    assert diff.max() <= bound, (diff.max(), bound, kappa)
    # L_{i,1} of every tail against the Schur complement onto stage 1
    S1 = natural.tail_schur_first(d["D"], d["E"])
    L11 = out["fac"]["Ld"][:, 0]
    for s in range(w.S):
        rec = L11[s] @ L11[s].T
        assert np.abs(rec - S1[s]).max() <= 1e-11 * np.abs(S1[s]).max()


def test_fp64_graph_and_direct_launch_agree_bitwise():
    bm = _bm()
    d = gen(3, 21, 6, 3, seed=5)
    a = run_gpu(d)
    b = run_gpu(d, flags=bm.BM_FLAG_NO_GRAPH)
    assert np.array_equal(a["x"], b["x"])
    for k in a["fac"]:
        assert np.array_equal(a["fac"][k], b["fac"][k])


def test_fp64_repeat_is_deterministic_and_reuses_factor():
    bm = _bm()
    d = gen(4, 30, 8, 3, seed=9)
    g = to_dev(d)
    solver = bm.BranchKKTSolver(4, 30, 8, 3)
    xs = []
    for _ in range(3):
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        xs.append(solver.solve(g["r"]).cpu().numpy())
    assert all(np.array_equal(xs[0], x) for x in xs[1:])
    # several right-hand sides on one factor
    for j in range(3):
        r = torch.randn(solver.n, dtype=torch.float64, generator=torch.Generator().manual_seed(j)).cuda()
        x = solver.solve(r).cpu().numpy()
        dd = dict(d)
        dd["r"] = r.cpu()
        check_solution(dd, x)
    solver.close()


# (S, N, nb, nr, pipelined): nb = 5 has no compiled tail kernels (serial
# copies); the others overlap the copies of later chunks of tails with the
# first level of earlier ones from the second call on (S = 3: one tail per
# chunk; S = 12 and 19: uneven chunks; N = 2: no level before the top kernel)
HOST_CASES = [(3, 11, 5, 2, False), (3, 16, 4, 2, True), (12, 64, 4, 2, True), (19, 33, 12, 3, True),
              (9, 2, 6, 3, True)]


@pytest.mark.parametrize("S,N,nb,nr,piped", HOST_CASES)
def test_fp64_host_entry_matches_device_entry(S, N, nb, nr, piped):
    bm = _bm()
    d = gen(S, N, nb, nr, seed=13)
    dev = run_gpu(d)
    solver = bm.BranchKKTSolver(S, N, nb, nr)
    pin = {k: d[k].contiguous().pin_memory() for k in ("D", "E", "C", "R", "r")}
    x = torch.empty_like(pin["r"]).pin_memory()
    for call in range(3):
        x.fill_(float("nan"))
        x, code = solver.factor_solve_host(pin["D"], pin["E"], pin["C"], pin["R"], pin["r"], x)
        assert code == 0
        assert solver.query()["host_pipelined"] == (1 if piped and call > 0 else 0)
        assert np.array_equal(x.numpy(), dev["x"])
    # pageable inputs take the serial copies, with the same result
    page = {k: d[k].contiguous().clone() for k in ("D", "E", "C", "R", "r")}
    xp = torch.empty_like(page["r"])
    xp, code = solver.factor_solve_host(page["D"], page["E"], page["C"], page["R"], page["r"], xp)
    assert code == 0 and solver.query()["host_pipelined"] == 0
    assert np.array_equal(xp.numpy(), dev["x"])
    solver.close()


@pytest.mark.parametrize("direct", [False, True])   # captured graph, or BM_FLAG_NO_GRAPH
def test_fp64_host_entry_pipelined_new_buffers(direct):
    """The pipelined host entry follows new host buffers (the captured form
    is captured again) and gives the device entry's bits for each system,
    also when its copies and kernels are launched directly."""
    bm = _bm()
    flags = bm.BM_FLAG_NO_GRAPH if direct else 0
    S, N, nb, nr = 10, 40, 6, 3
    d1, d2 = gen(S, N, nb, nr, seed=21), gen(S, N, nb, nr, seed=22)
    ref1, ref2 = run_gpu(d1)["x"], run_gpu(d2)["x"]
    p1 = {k: d1[k].contiguous().pin_memory() for k in ("D", "E", "C", "R", "r")}
    p2 = {k: d2[k].contiguous().pin_memory() for k in ("D", "E", "C", "R", "r")}
    solver = bm.BranchKKTSolver(S, N, nb, nr, flags=flags)
    x = torch.empty_like(p1["r"]).pin_memory()
    for call, (p, ref) in enumerate(((p1, ref1), (p2, ref2), (p1, ref1), (p1, ref1))):
        x, code = solver.factor_solve_host(p["D"], p["E"], p["C"], p["R"], p["r"], x)
        assert code == 0
        assert solver.query()["host_pipelined"] == (1 if call > 0 else 0)
        assert np.array_equal(x.numpy(), ref)
    solver.close()


@pytest.mark.parametrize("scenario,stage", [(8, 2), (8, 3), (11, 57), (0, 1), (7, 64)])
def test_fp64_host_entry_pipelined_reports_location(scenario, stage):
    """A non-SPD block in a later chunk of tails is reported with the
    system-wide scenario index by the pipelined host entry (chunks of S = 12
    tails: [0,1) [1,3) [3,4) [4,6) [6,7) [7,9) [9,10) [10,12)); stages 2 and
    64 are eliminated at level 0 (run per chunk), 3 at level 1 (over all
    tails), 57 at level 3 (the top kernel) and 1 is x_1."""
    bm = _bm()
    d = gen(12, 64, 4, 2, seed=5)
    pin = {k: d[k].contiguous().pin_memory() for k in ("D", "E", "C", "R", "r")}
    bad = d["D"].clone()
    bad[scenario, stage - 1] = -torch.eye(4, dtype=torch.float64)
    bad = bad.contiguous().pin_memory()
    solver = bm.BranchKKTSolver(12, 64, 4, 2, flags=bm.BM_FLAG_NO_TUNE)   # default schedule: top level 3
    x = torch.empty_like(pin["r"]).pin_memory()
    _, code = solver.factor_solve_host(pin["D"], pin["E"], pin["C"], pin["R"], pin["r"], x)
    assert code == 0
    _, code = solver.factor_solve_host(bad, pin["E"], pin["C"], pin["R"], pin["r"], x)
    info = solver.query()
    assert info["host_pipelined"] == 1
    assert code == 2 and info["fail_scenario"] == scenario and info["fail_stage"] == stage, info
    # the same location as the device entry
    g = to_dev(d)
    ref = bm.BranchKKTSolver(12, 64, 4, 2)
    ref.factor(bad.cuda(), g["E"], g["C"], g["R"])
    rinfo = ref.query()
    assert (rinfo["fail_scenario"], rinfo["fail_stage"]) == (scenario, stage)
    ref.close()
    # the status is cleared by the next call
    _, code = solver.factor_solve_host(pin["D"], pin["E"], pin["C"], pin["R"], pin["r"], x)
    assert code == 0 and solver.query()["host_pipelined"] == 1
    solver.close()


@pytest.mark.parametrize("stage", [1, 2, 7, 16])
def test_fp64_not_spd_reports_location(stage):
    bm = _bm()
    d = gen(3, 16, 4, 2, seed=3)
    D = d["D"].clone()
    D[1, stage - 1] = -torch.eye(4, dtype=torch.float64)
    g = to_dev(d)
    g["D"] = D.cuda()
    solver = bm.BranchKKTSolver(3, 16, 4, 2)
    solver.factor(g["D"], g["E"], g["C"], g["R"])
    x = solver.solve(g["r"])
    info = solver.query()
    assert info["status"] == 2 and info["fail_scenario"] == 1 and info["fail_stage"] == stage, info
    assert torch.isfinite(x).all()
    # the status is sticky until the next factor, which clears it
    solver.factor(to_dev(d)["D"], g["E"], g["C"], g["R"])
    assert solver.query()["status"] == 0
    solver.close()


def test_fp64_nan_input_is_reported_and_root_failure_located():
    bm = _bm()
    d = gen(2, 8, 3, 2, seed=4)
    g = to_dev(d)
    D = g["D"].clone()
    D[0, 3, 1, 1] = float("nan")
    solver = bm.BranchKKTSolver(2, 8, 3, 2)
    solver.factor(D, g["E"], g["C"], g["R"])
    assert solver.query()["status"] == 2
    # a root block that makes R - sum U indefinite is reported at the root
    R = g["R"].clone() - 100.0 * torch.eye(2, dtype=torch.float64, device="cuda")
    solver.factor(g["D"], g["E"], g["C"], R)
    info = solver.query()
    assert info["status"] == 2 and info["fail_scenario"] == -1 and info["fail_stage"] == 0, info
    solver.close()


def test_fp64_invalid_arguments_are_rejected():
    bm = _bm()
    with pytest.raises(bm.BMError):
        bm.BranchKKTSolver(0, 4, 4, 2)
    with pytest.raises(bm.BMError):
        bm.BranchKKTSolver(2, 4, 65, 2)
    solver = bm.BranchKKTSolver(2, 4, 3, 2)
    r = torch.zeros(solver.n, dtype=torch.float64, device="cuda")
    with pytest.raises(bm.BMError):
        solver.solve(r)                      # before any factor
    solver.close()


def test_fp64_analyze_reports_allocation_failure():
    """A workspace far beyond the device's memory: bm_analyze returns
    BM_ERR_OOM and the context stays usable."""
    bm = _bm()
    with pytest.raises(bm.BMError) as e:
        bm.BranchKKTSolver(40000, 1 << 16, 48, 16)
    assert e.value.code == 3
    solver = bm.BranchKKTSolver(2, 4, 3, 2)      # still works afterwards
    solver.close()


def test_bounded_device_wait_times_out():
    """The bounded wait of the batched factor, on a counter that nothing
    increments, gives up after its limit (~1 ms here) with BM_ERR_TIMEOUT."""
    bm = _bm()
    import time
    t0 = time.perf_counter()
    assert bm.bm_test_bounded_wait(2_000_000) == 6
    assert time.perf_counter() - t0 < 5.0
    assert bm.bm_test_bounded_wait(0) == 1      # invalid limit


def test_fp64_handles_with_different_block_sizes_coexist():
    """Analyzing a small-block handle after a large-block one must not break
    the large one (kernel attributes are process-wide)."""
    bm = _bm()
    big = gen(2, 5, 48, 16, seed=31)
    gb = to_dev(big)
    h_big = bm.BranchKKTSolver(2, 5, 48, 16)
    h_small = bm.BranchKKTSolver(2, 5, 3, 2)
    h_big.factor(gb["D"], gb["E"], gb["C"], gb["R"])
    x = h_big.solve(gb["r"]).cpu().numpy()
    assert h_big.query()["status"] == 0
    check_solution(big, x)
    h_small.close()
    h_big.close()


def test_fp64_schedule_is_tuned_cached_and_does_not_change_the_bits(tmp_path, monkeypatch):
    """The first factor of a handle tunes the launch schedule (team size per
    grid-wide level, top level of the per-tail kernel) and stores it; a second
    handle of the same shape takes it from the cache. Every element of every
    block is computed by one thread in a fixed order whatever the schedule,
    so the tuned, cached and default schedules give the same bits."""
    monkeypatch.setenv("BM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    bm = _bm()
    S, N, nb, nr = 16, 40, 12, 4
    d = gen(S, N, nb, nr, seed=3, barrier=(-3, 3))
    g = to_dev(d)
    outs = []
    for flags in (0, 0, bm.BM_FLAG_NO_TUNE):
        solver = bm.BranchKKTSolver(S, N, nb, nr, flags=flags)
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        x = solver.solve(g["r"]).cpu().numpy()
        outs.append((x, solver.schedule(), solver.query()))
        solver.close()
    (x1, s1, i1), (x2, s2, i2), (x3, s3, i3) = outs
    assert s1["source"] == "tuned" and s2["source"] == "cache" and s3["source"] == "rule", (s1, s2, s3)
    assert s1["top_level"] == s2["top_level"] and s1["teams"] == s2["teams"]
    assert 0 <= s1["top_level"] <= 6 and all(t in (8, 16, 32, 64) for t in s1["teams"]), s1
    assert i1["status"] == i2["status"] == i3["status"] == 0
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)
    assert "fp64-schedule" in (tmp_path / "tune.json").read_text()
    # mixed-precision handles have no tunable schedule
    mixed = bm.BranchKKTSolver(S, N, nb, nr, precision=bm.BM_PREC_FP32_IR)
    with pytest.raises(bm.BMError):
        mixed.schedule()
    mixed.close()

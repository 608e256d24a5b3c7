"""Benchmark: factor + solve of one branch-MPC KKT system per step.

Default workload: the mixed-precision system of the headline metric (S=512
scenarios, N=128 stages, nb=24, nr=8, barrier diagonals 10^U[-6,6]),
factored (Alg. 1) and solved (Alg. 2) through the C ABI with the inputs
resident in HBM (605 MB of FP64 blocks, larger than L2; L2 is also flushed
by a 256 MiB write between timed steps, outside the timed events). One step
= bm_factor + bm_solve.

Prints ONE JSON line (rank 0). value = whole-job GFLOP/s of the plain FP64
path, counting the method's flops of one factor + solve per step (the same
per-step count for every arm, so value is proportional to KKT systems per
second). Beside it, on the same system: "fp32ir_same_workload" (FP32 tails +
FP64 refinement to omega <= 1e-10, with its status, backward errors and
forward error against the FP64 solution) and, for the default workload on
one GPU, "batched" (256 uneven systems in one persistent launch against the
FP64 path one system at a time) and "serving" (the Poisson request stream,
FP32+IR against FP64, p50/p99 latency); --no-forms skips those two.
  --impl reference : the CPU oracle (natural-order FP64 block Cholesky) on
                     the host cores, timed on the same workload.
  --workload NAME  : another synthetic workload (see bmgen.WORKLOADS).
  --precision fp32ir : the FP32-tail + FP64-refinement path.
Multi-GPU (torchrun): every rank factors and solves its own replica (the
scenarios of one system are not split across GPUs); weak scaling.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "mixed-s512-n128-nb24"
METRIC = "factor+solve µs and GFLOP/s per branch KKT; FP32+IR vs FP64 at rel. residual 1e-10"
L2_FLUSH_BYTES = 256 << 20


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp64_peak_gflops(sm_mhz=None):
    """FP64 ALU peak of the GPU: 152 SMs x 2 FMA lanes per clock (one 32-lane
    warp instruction per 64 cycles on each of the 4 SM sub-partitions,
    measured) x 2 flop per FMA x the maximum SM clock."""
    peaks, _ = _peaks()
    mhz = sm_mhz or peaks.get("sm_max_mhz", 2070.0)
    return 152 * 2 * 2 * mhz * 1e6 / 1e9


def fp32_peak_gflops(sm_mhz=None):
    """FP32 ALU peak: 152 SMs x 128 FMA lanes per clock x 2 flop x the
    maximum SM clock (121 lane-ops per SM per clock measured with FFMA)."""
    peaks, _ = _peaks()
    mhz = sm_mhz or peaks.get("sm_max_mhz", 2070.0)
    return 152 * 128 * 2 * mhz * 1e6 / 1e9


def _factor_kernels(N, nb, precision):
    """Names of the kernels one factor launches (one CUDA graph)."""
    from paper_2609_29977_gb300 import bm as core   # plain Python: does not load the library
    Lc, top = core.chain_levels(N), core.top_level(N)
    if precision == "fp64":
        if nb in core.TAIL_NB:
            return "k_factor_level_team x%d + k_factor_top (its last CTA does the root step)" % top
        return "k_factor_level x%d + k_factor_x1 + k_factor_root" % Lc
    suffix = "" if nb <= 32 else "_w"
    return ("k_level_rows%s x%d + k_top_rows%s + k_pivot_spread + k_factor_root (probe), then when refined "
            "k_cx_bwd + k_cx_residual + k_cx_fwd + k_cx_bwd + k_factor_root" % (suffix, top, suffix))


def _kernel_source_hash():
    """Hash of every CUDA source of the library (any change makes the
    committed DRAM counters stale)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2609_29977_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def _profile_traffic(workload, precision):
    """Per-launch DRAM traffic of the factor pipeline from the committed ncu
    summary (profiles/factor_<precision>_<workload>.txt), if the kernels have
    not changed since it was taken; else None."""
    p = os.path.join(ROOT, "profiles", "factor_%s_%s.txt" % (precision, workload))
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line and line.split(":", 1)[0].strip() in ("source_hash", "traffic_bytes_per_factor"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_hash") != _kernel_source_hash():
        return None
    try:
        return float(vals["traffic_bytes_per_factor"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest per-rank value over all ranks (the slowest replica sets
    the whole-job time); the value itself without a process group."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(world, flops_per_step, steps, slowest_ms):
    """Whole-job throughput: every rank solves its own replica (weak
    scaling), so the job does world x steps systems in the slowest rank's
    time."""
    return world * flops_per_step * steps / (slowest_ms * 1e-3) / 1e9


def time_oracle(sysd, budget_s, min_reps=3, nthreads=0):
    """The oracle's factor + solve (no residual check), repeated on the full
    system until the budget is spent; returns (seconds per factor+solve,
    threads, reps)."""
    from oracle import natural
    threads = nthreads or natural.max_threads()
    reps, t0 = 0, time.perf_counter()
    while True:
        fac = natural.factor(sysd["D"], sysd["E"], sysd["C"], sysd["R"], nthreads=threads)
        natural.solve(fac, sysd["r"], nthreads=threads)
        reps += 1
        el = time.perf_counter() - t0
        if reps >= min_reps and el >= budget_s:
            break
    return el / reps, threads, reps


def gpu_residual_measures(g, x):
    """Residual measures of x in plain PyTorch FP64: normwise backward error
    eta = ||r - K x||_inf / (||K||_inf ||x||_inf + ||r||_inf), componentwise
    backward error omega = max_i |r - K x|_i / (|K||x| + |r|)_i, and the
    relative residuals in the infinity and 2-norms."""
    import torch
    D, E, C, R, r = g["D"], g["E"], g["C"], g["R"], g["r"]
    S, N, nb, _ = D.shape
    nr = R.shape[0]
    n0 = S * N * nb
    X = x[:n0].view(S, N, nb, 1)
    x0 = x[n0:]
    Dl = torch.tril(D)
    Df = Dl + torch.tril(Dl, -1).transpose(-1, -2)
    Kx = (Df @ X).squeeze(-1)
    AKx = (Df.abs() @ X.abs()).squeeze(-1)
    rows = Df.abs().sum(-1)
    if N > 1:
        Kx[:, 1:] += (E @ X[:, :-1]).squeeze(-1)
        Kx[:, :-1] += (E.transpose(-1, -2) @ X[:, 1:]).squeeze(-1)
        AKx[:, 1:] += (E.abs() @ X[:, :-1].abs()).squeeze(-1)
        AKx[:, :-1] += (E.abs().transpose(-1, -2) @ X[:, 1:].abs()).squeeze(-1)
        rows[:, 1:] += E.abs().sum(-1)
        rows[:, :-1] += E.abs().sum(-2)
    Kx[:, 0] += (C.transpose(-1, -2) @ x0.view(1, nr, 1)).squeeze(-1)
    AKx[:, 0] += (C.abs().transpose(-1, -2) @ x0.abs().view(1, nr, 1)).squeeze(-1)
    rows[:, 0] += C.abs().sum(-2)
    Rl = torch.tril(R)
    Rf = Rl + torch.tril(Rl, -1).T
    k0 = Rf @ x0 + (C @ X[:, 0]).squeeze(-1).sum(0)
    a0 = Rf.abs() @ x0.abs() + (C.abs() @ X[:, 0].abs()).squeeze(-1).sum(0)
    rows0 = Rf.abs().sum(-1) + C.abs().sum(-1).sum(0)
    rho = torch.cat([(r[:n0] - Kx.reshape(-1)), r[n0:] - k0])
    den = torch.cat([AKx.reshape(-1), a0]) + r.abs()
    kinf = torch.maximum(rows.max(), rows0.max())
    eta = rho.abs().max() / (kinf * x.abs().max() + r.abs().max())
    omega = torch.where(den > 0, rho.abs() / den.clamp_min(1e-300), (rho != 0).double() * float("inf")).max()
    return {"backward_error": float(eta), "omega": float(omega), "rel_residual_inf": float(rho.abs().max() / r.abs().max()),
            "rel_residual_2": float(rho.norm() / r.norm())}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import bmgen
    w = bmgen.WORKLOADS[args.workload]
    sysd = bmgen.generate(w)
    fl = bmgen.method_flops(w.S, w.N, w.nb, w.nr)
    budget = args.ref_budget
    for _ in range(args.warmup):
        time_oracle(sysd, 0.0, min_reps=1)
    per = []
    threads = 0
    for _ in range(args.steps):
        sec, threads, reps = time_oracle(sysd, budget / max(1, args.steps), min_reps=1)
        per.append(sec)
    sec = statistics.mean(per)
    value = fl["total"] / sec / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "S": w.S, "N": w.N, "nb": w.nb, "nr": w.nr, "precision": "fp64",
                   "solver": "oracle: natural-order FP64 block Cholesky (C, OpenMP over tails)"},
        "us_per_kkt": sec * 1e6,
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": "full workload, factor+solve repeated per step for ~%.1f s" %
                                   (budget / max(1, args.steps))},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    print(json.dumps(batched_line(args, args.steps, args.warmup)), flush=True)
    return 0


def batched_line(args, steps, warmup):
    """The batched workload: 256 systems with S~U{8..256}, N~U{16..256},
    nb in {6,12,24,48}, nr = ceil(nb/3), barrier 10^U[-4,4], factored in one
    persistent launch and solved with FP32 tails + FP64 refinement. One step
    = bm_batch_factor + bm_batch_solve of the whole batch. Beside it, the
    same systems through the plain FP64 path, one handle per system."""
    import torch

    import bmgen
    import paper_2609_29977_gb300 as bm

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    count = args.batch_count
    shapes = bmgen.draw_batched_shapes(count)
    base = bmgen.Workload("batched", 1, 1, 1, 1, workload_id=4, barrier=(-4.0, 4.0), shared_A=True)
    t0 = time.perf_counter()
    systems = []
    for j, (S, N, nb, nr) in enumerate(shapes):
        d = bmgen.generate(base.with_shape(S=S, N=N, nb=nb, nr=nr), instance=j, device=args.gen_device)
        systems.append({k: (v.to(dev) if isinstance(v, torch.Tensor) else v) for k, v in d.items()})
    gen_s = time.perf_counter() - t0
    flops = sum(bmgen.method_flops(S, N, nb, nr)["total"] for (S, N, nb, nr) in shapes)
    batch = bm.BranchKKTBatch(shapes, max_refine=args.max_refine, tol=args.tol)
    Ds, Es, Cs, Rs, rs = ([d[k] for d in systems] for k in ("D", "E", "C", "R", "r"))
    xs = [torch.empty_like(r) for r in rs]
    t0 = time.perf_counter()
    batch.factor(Ds, Es, Cs, Rs)     # first call autotunes the persistent launch
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    for _ in range(max(3, warmup)):
        batch.factor(Ds, Es, Cs, Rs)
        batch.solve(rs, xs)
    infos = batch.query()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler("0")
    sampler.start()
    time.sleep(0.5)
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        a, b, c = ev[i]
        a.record(stream)
        batch.factor(Ds, Es, Cs, Rs)
        b.record(stream)
        batch.solve(rs, xs)
        c.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    fac = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
    sol = statistics.mean(b.elapsed_time(c) for _, b, c in ev)
    infos = batch.query()
    omegas = [i["backward_error"] for i in infos]
    bad = [i for i in infos if i["status"] != 0]
    sched = batch.schedule()
    batch.close()
    # the plain FP64 path on the same systems, one handle per system, back to back
    fp64_ms = None
    fwd_max = None
    if not args.no_fp64_compare:
        # one system at a time (a handle per system would not fit beside the
        # batch): factor + solve timed with events after a warm-up, summed
        fp64_ms = 0.0
        fwd_max = 0.0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for (S, N, nb, nr), d, xb in zip(shapes, systems, xs):
            hnd = bm.BranchKKTSolver(S, N, nb, nr)
            x64 = torch.empty_like(d["r"])
            hnd.factor(d["D"], d["E"], d["C"], d["R"])
            hnd.solve(d["r"], x64)
            flush.zero_()
            a.record(stream)
            hnd.factor(d["D"], d["E"], d["C"], d["R"])
            hnd.solve(d["r"], x64)
            b.record(stream)
            torch.cuda.synchronize()
            fp64_ms += a.elapsed_time(b)
            fwd_max = max(fwd_max, float((xb - x64).abs().max() / x64.abs().max()))
            hnd.close()
            del x64
    ms = fac + sol
    line = {
        "metric": METRIC, "value": flops / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1, "steps": steps,
        "warmup": max(3, warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded MPC-shaped generator)",
        "config": {"workload": "batched-%d" % count, "systems": count, "stages": sum(S * N for S, N, _, _ in shapes),
                   "precision": "fp32ir", "tol": args.tol, "l2": "flushed between timed steps"},
        "factor_ms": fac, "solve_ms": sol, "fp64_sequential_ms": fp64_ms,
        "speedup_vs_fp64_sequential": (fp64_ms / ms) if fp64_ms else None,
        "omega_max": max(omegas), "failed_systems": len(bad), "schedule": sched,
        "forward_error_vs_fp64_max": fwd_max if fp64_ms is not None else None,
        "autotune_s": tune_s, "generate_s": gen_s, "clocks": clocks,
    }
    del systems, Ds, Es, Cs, Rs, rs, xs
    torch.cuda.empty_cache()
    return line


def _percentile(vals, q):
    v = sorted(vals)
    if not v:
        return None
    k = (len(v) - 1) * q
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def run_serving(args):
    print(json.dumps(serving_line(args)), flush=True)
    return 0


def serving_line(args):
    """Serving: a Poisson stream of requests (mean --rate per second), each a
    branch-MPC system drawn as in the batched workload (S~U{8..256},
    N~U{16..256}, nb in {6,12,24,48}, nr = ceil(nb/3)) or, with probability
    5%, the large system (S=2048, N=256, nb=48, nr=16); every request is
    factored once and solved for 4 right-hand sides against its resident
    factor. The requests go through the library's serving runtime (admission
    by an HBM budget, one stream per slot), first with the FP32-tail +
    refinement path (a request it cannot resolve is re-run in FP64 by the
    server), then with the plain FP64 path, on the same arrival
    trace; then both again at half the throughput the first run sustained.
    The inputs of a request are drawn from a pool of distinct systems and are
    resident in HBM before the stream starts; latency = completion of the
    last solve - arrival."""
    import random

    import torch

    import bmgen
    import paper_2609_29977_gb300 as bm

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    rng = random.Random(args.seed)
    nrhs = 4
    t0 = time.perf_counter()
    small_shapes = bmgen.draw_batched_shapes(args.pool, seed=5000)
    base = bmgen.Workload("serve", 1, 1, 1, 1, workload_id=7, barrier=(-4.0, 4.0), shared_A=True)
    pool = []
    for j, (S, N, nb, nr) in enumerate(small_shapes):
        pool.append(bmgen.generate(base.with_shape(S=S, N=N, nb=nb, nr=nr), instance=j, device=dev, with_rhs=False))
    large_w = bmgen.WORKLOADS["large-s2048-n256-nb48"]
    if args.large_frac > 0:
        pool.append(bmgen.generate(large_w, device=dev, with_rhs=False))
    for j, d in enumerate(pool):
        n = bmgen.n_unknowns(d["S"], d["N"], d["nb"], d["nr"])
        g = torch.Generator(device=dev).manual_seed(9000 + j)
        d["rs"] = torch.randn((nrhs, n), generator=g, device=dev, dtype=torch.float64)
    gen_s = time.perf_counter() - t0
    n_small = len(small_shapes)
    kinds = []
    for _ in range(args.requests):
        if args.large_frac > 0 and rng.random() < args.large_frac:
            kinds.append(n_small)
        else:
            kinds.append(rng.randrange(n_small))
    gaps = [rng.expovariate(1.0) for _ in range(args.requests)]   # unit-rate gaps, scaled per run
    flops = []
    for k in kinds:
        d = pool[k]
        f = bmgen.method_flops(d["S"], d["N"], d["nb"], d["nr"])
        flops.append(f["factor"] + nrhs * f["solve"])
    xs = [torch.empty_like(pool[k]["rs"]) for k in kinds]
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    budget = int(args.serve_budget_gb * (1 << 30))

    def one_run(precision, rate):
        server = bm.BranchKKTServer(budget, slots=args.slots, precision=precision, max_refine=args.max_refine,
                                    tol=args.tol, fp64_fallback=(precision == bm.BM_PREC_FP32_IR))

        def submit(rid, k, x):
            d = pool[k]
            server.submit(rid, d["S"], d["N"], d["nb"], d["nr"], d["D"], d["E"], d["C"], d["R"], d["rs"], x)

        # warm-up: every distinct system once (kernel attributes, allocator)
        for j in range(len(pool)):
            submit(10 ** 9 + j, j, torch.empty_like(pool[j]["rs"]))
        server.drain()
        arrivals, t = [], 0.0
        for gp in gaps:
            t += gp / rate
            arrivals.append(t)
        sampler = ClockSampler("0")
        sampler.start()
        time.sleep(0.3)
        comps, delay = {}, {}
        i = 0
        start = time.perf_counter()
        while len(comps) < args.requests:
            now = time.perf_counter() - start
            while i < args.requests and arrivals[i] <= now:
                submit(i, kinds[i], xs[i])
                delay[i] = (time.perf_counter() - start) - arrivals[i]
                i += 1
            for c in server.poll(wait=(i >= args.requests)):
                comps[c["id"]] = c
        wall = time.perf_counter() - start
        clocks = sampler.stop()
        stats = server.stats()
        server.close()
        lat, bad, etas = [], 0, []
        first_submit = min(c["t_submit_us"] - delay[c["id"]] * 1e6 for c in comps.values())
        last_done = max(c["t_done_us"] for c in comps.values())
        for rid, c in comps.items():
            # arrival on the server's clock = submission - how late the submission was
            arrival_us = c["t_submit_us"] - delay[rid] * 1e6
            lat.append((c["t_done_us"] - arrival_us) * 1e-3)
            bad += c["status"] != 0
            etas += [e for e in c["backward_error"] if e >= 0]
        span_s = (last_done - first_submit) * 1e-6
        # the solutions of a sample of requests against plain PyTorch FP64 residuals
        sample_eta = 0.0
        for rid in range(min(8, args.requests)):
            d = pool[kinds[rid]]
            gd = {"D": d["D"], "E": d["E"], "C": d["C"], "R": d["R"], "r": d["rs"][0]}
            sample_eta = max(sample_eta, gpu_residual_measures(gd, xs[rid][0])["omega"])
        return {"offered_rate": rate, "throughput_req_s": args.requests / span_s,
                "gflops": sum(flops) / span_s / 1e9, "p50_ms": _percentile(lat, 0.5), "p99_ms": _percentile(lat, 0.99),
                "max_ms": max(lat), "makespan_s": span_s, "wall_s": wall, "failed": bad,
                "device_omega_max": max(etas) if etas else None, "sample_omega_max": sample_eta,
                "peak_arena_gb": stats["peak_bytes_in_use"] / 2 ** 30, "fp64_fallbacks": stats["fallbacks"],
                "clocks": clocks}

    runs = {}
    runs["fp32ir"] = one_run(bm.BM_PREC_FP32_IR, args.rate)
    runs["fp64"] = one_run(bm.BM_PREC_FP64, args.rate)
    half = 0.5 * runs["fp32ir"]["throughput_req_s"]
    runs["fp32ir_half_load"] = one_run(bm.BM_PREC_FP32_IR, half)
    runs["fp64_half_load"] = one_run(bm.BM_PREC_FP64, half)
    main = runs["fp32ir"]
    line = {
        "metric": "serving: requests/s (factor + 4 RHS per request) with p50/p99 latency; FP32+IR vs FP64",
        "value": main["throughput_req_s"], "unit": "req/s", "n_gpus": 1, "steps": args.requests, "warmup": len(pool),
        "ms_per_step": 1e3 * main["makespan_s"] / args.requests, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded MPC-shaped generator)",
        "config": {"workload": "serving-poisson-%g-per-s" % args.rate, "requests": args.requests,
                   "large_fraction": args.large_frac, "pool_small_systems": n_small, "rhs_per_request": nrhs,
                   "slots": args.slots, "hbm_budget_gb": args.serve_budget_gb, "tol": args.tol,
                   "l2": "inputs of the stream (pool of %d systems, %.1f GB) exceed L2" %
                         (len(pool), sum(sum(d[k].numel() for k in ("D", "E")) * 8 for d in pool) / 1e9)},
        "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"], "runs": runs,
        "throughput_vs_fp64": main["throughput_req_s"] / runs["fp64"]["throughput_req_s"],
        "generate_s": gen_s,
    }
    del pool, xs
    torch.cuda.empty_cache()
    return line


def run_assembly(args):
    """Assembly front end: App. A's reduced matrix of a branch-MPC QP formed
    on the GPU (bm_assemble_reduced) in the solver's block layout, timed
    alone (value: GB/s of inputs read and D, E, C, R written once; roofline:
    the FP64 FMAs of the [A_k B_k]^T [A_k B_k] lower triangles, which bound
    it on GB300), then QP -> K -> factor -> solve with the FP64 path and with
    FP32+IR."""
    import torch

    import bmgen
    import paper_2609_29977_gb300 as bm

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    S, N, nx, nu = (int(t) for t in (args.shape or "512,128,24,8").split(","))
    qp = bmgen.generate_qp(S, N, nx, nu, seed=6000, device=dev, barrier=(-3.0, 3.0), delta=1e-2)
    nb = nx + nu
    for _ in range(max(3, args.warmup)):
        out = bm.bm_assemble_reduced(qp)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    k = min(args.steps, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    sampler = ClockSampler("0")
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        out = bm.bm_assemble_reduced(qp)
        b.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    n_in = sum(qp[key].numel() for key in ("A", "B", "q", "rw", "r0w", "w", "w0"))
    n_out = sum(out[key].numel() for key in ("D", "E", "C", "R"))
    byts = 8.0 * (n_in + n_out)
    peaks, src = _peaks()
    gbs = byts / (ms * 1e-3) / 1e9
    flops = 2.0 * nx * (nb * (nb + 1) / 2) * S * (N - 1) + 2.0 * nx * nu * nu * S
    gflops = flops / (ms * 1e-3) / 1e9
    n = bmgen.n_unknowns(S, N, nb, nu)
    r = torch.randn(n, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(6001))
    paths = {}
    for name, prec in (("fp64", bm.BM_PREC_FP64), ("fp32ir", bm.BM_PREC_FP32_IR)):
        solver = bm.BranchKKTSolver(S, N, nb, nu, precision=prec, max_refine=args.max_refine, tol=args.tol)
        x = torch.empty_like(r)
        for _ in range(3):
            o2 = bm.bm_assemble_reduced(qp)
            solver.factor(o2["D"], o2["E"], o2["C"], o2["R"])
            solver.solve(r, x)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tt = []
        for _ in range(5):
            flush.zero_()
            a.record(stream)
            o2 = bm.bm_assemble_reduced(qp)
            solver.factor(o2["D"], o2["E"], o2["C"], o2["R"])
            solver.solve(r, x)
            b.record(stream)
            torch.cuda.synchronize()
            tt.append(a.elapsed_time(b))
        info = solver.query()
        meas = gpu_residual_measures({"D": o2["D"], "E": o2["E"], "C": o2["C"], "R": o2["R"], "r": r}, x)
        paths[name] = {"ms_qp_to_solution": statistics.median(tt), "device_status": info["name"],
                       "refinement_steps": info["iters"], **meas}
        solver.close()
    line = {
        "metric": "assembly front end: GB/s of K formed from QP data; QP -> solution ms", "value": gbs,
        "unit": "GB/s", "n_gpus": 1, "steps": k, "warmup": max(3, args.warmup), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic branch-MPC QP (seeded)",
        "config": {"workload": "qp-assembly-s%d-n%d-nx%d-nu%d" % (S, N, nx, nu), "S": S, "N": N, "nx": nx,
                   "nu": nu, "l2": "flushed between timed steps"},
        "roofline": {"kernel": "k_assemble_stage + k_assemble_coupling + k_assemble_root", "bound": "alu", "achieved": gflops,
                     "peak": fp64_peak_gflops(), "unit": "GFLOP/s", "frac": gflops / fp64_peak_gflops(),
                     "traffic": None, "peak_source": "FP64 ALU derived (as the factor)",
                     "algorithmic_flops": flops, "algorithmic_bytes": byts,
                     "hbm_frac": gbs / peaks["hbm_gbs"], "hbm_peak_source": src},
        "paths": paths, "clocks": clocks, "gpu_launches": 3 * k,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_grid(args):
    """Context sweep over the paper's experiment grid (Sec. V): nb = nr = 16,
    scenario counts M and horizons N, factor and solve (FP64, or FP32+IR
    with --precision fp32ir) timed with the
    paper's protocol (device-resident data, analysis and graph capture
    excluded, median of 50 after 10 warm-ups; L2 not flushed). Synthetic
    systems stand in for the paper's quadrotor model (barrier off)."""
    import torch

    import bmgen
    import paper_2609_29977_gb300 as bm

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    base = bmgen.WORKLOADS["grid-s100-n160-nb16"]
    pts = [(m, 30) for m in (20, 60, 100, 140, 200)] + [(100, n) for n in (40, 80, 120, 160)] + [(200, 160)]
    out = []
    for m, n in pts:
        w = base.with_shape(S=m, N=n)
        d = bmgen.generate(w, device=dev)
        prec = bm.BM_PREC_FP64 if args.precision == "fp64" else bm.BM_PREC_FP32_IR
        solver = bm.BranchKKTSolver(m, n, w.nb, w.nr, precision=prec, max_refine=args.max_refine, tol=args.tol)
        x = torch.empty_like(d["r"])
        for _ in range(10):
            solver.factor(d["D"], d["E"], d["C"], d["R"])
            solver.solve(d["r"], x)
        fac, sol = [], []
        for _ in range(50):
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            solver.factor(d["D"], d["E"], d["C"], d["R"])
            b.record(stream)
            solver.solve(d["r"], x)
            c.record(stream)
            torch.cuda.synchronize()
            fac.append(a.elapsed_time(b))
            sol.append(b.elapsed_time(c))
        info = solver.query()
        solver.close()
        meas = gpu_residual_measures(d, x)
        out.append({"M": m, "N": n, "factor_ms": statistics.median(fac), "solve_ms": statistics.median(sol),
                    "status": info["name"], "omega": meas["omega"], "refinement_steps": info["iters"]})
        del d, x
    at = {(p["M"], p["N"]): p for p in out}
    line = {
        "metric": "paper grid (nb = nr = 16): %s factor and solve ms per point, median of 50" % args.precision,
        "value": at[(100, 160)]["factor_ms"], "unit": "ms (factor, M=100, N=160)", "n_gpus": 1, "steps": 50,
        "warmup": 10, "ms_per_step": at[(100, 160)]["factor_ms"] + at[(100, 160)]["solve_ms"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded MPC-shaped generator, barrier off)",
        "config": {"workload": "paper-grid-nb16", "points": len(out), "l2": "not flushed (the paper's protocol)"},
        "points": out,
        "factor_growth_N40_to_160_at_M100": at[(100, 160)]["factor_ms"] / at[(100, 40)]["factor_ms"],
        "solve_growth_N40_to_160_at_M100": at[(100, 160)]["solve_ms"] / at[(100, 40)]["solve_ms"],
        "paper_context_rtx5090": {"factor_ms_N30_M20_to_200": [0.15, 0.35], "solve_ms_N30_M20_to_200": [0.10, 0.16],
                                  "factor_ms_M100_N160": "< 1", "solve_ms_M100_N160": "< 0.35",
                                  "growth_N40_to_160_at_M100": {"factor": 3.1, "solve": 2.3}},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    import bmgen
    import paper_2609_29977_gb300 as bm

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = bm.BM_PREC_FP64 if args.precision == "fp64" else bm.BM_PREC_FP32_IR
    w = bmgen.WORKLOADS[args.workload]
    if args.shape:
        S_, N_, nb_, nr_ = (int(t) for t in args.shape.split(","))
        w = w.with_shape(name="%s-shape-%d-%d-%d-%d" % (w.name, S_, N_, nb_, nr_), S=S_, N=N_, nb=nb_, nr=nr_)
    sysd = bmgen.generate(w, instance=rank)
    g = {k: v.to(dev) for k, v in sysd.items() if isinstance(v, torch.Tensor)}
    fl = bmgen.method_flops(w.S, w.N, w.nb, w.nr)
    solver = bm.BranchKKTSolver(w.S, w.N, w.nb, w.nr, precision=prec, max_refine=args.max_refine,
                                tol=args.tol, flags=(bm.BM_FLAG_NO_GRAPH if args.direct else 0) | _coupling_flags(args))
    x = torch.empty_like(g["r"])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        solver.solve(g["r"], x)

    for _ in range(max(3, args.warmup)):
        step()
    info = solver.query()
    # FP32 tails that cannot resolve the system are a reported outcome of the
    # mixed path (NOT_CONVERGED, or NOT_SPD of the FP32-based root), not a crash
    if info["status"] != 0 and not (prec == bm.BM_PREC_FP32_IR and info["status"] in (2, 5)):
        raise RuntimeError("device status after warm-up: %s" % info)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [t for t in vis.split(",") if t.strip()]
    smi_index = ids[local] if local < len(ids) and ids[local].strip().isdigit() else str(local)
    sampler = ClockSampler(smi_index)
    sampler.start()
    time.sleep(0.5)   # let nvidia-smi start sampling before the timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        a, b, c = ev[i]
        a.record(stream)
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        b.record(stream)
        solver.solve(g["r"], x)
        c.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    fac_ms = [a.elapsed_time(b) for a, b, _ in ev]
    sol_ms = [b.elapsed_time(c) for _, b, c in ev]
    tot_ms = sum(f + s for f, s in zip(fac_ms, sol_ms))
    info = solver.query()
    tot_ms = max_over_ranks(tot_ms, dist, dev)
    ms_per_step = tot_ms / args.steps
    value = whole_job_gflops(world, fl["total"], args.steps, tot_ms)

    # end to end through the public host-buffer entry point (pinned memory)
    pin = {k: sysd[k].contiguous().pin_memory() for k in ("D", "E", "C", "R", "r")}
    xh = torch.empty_like(pin["r"]).pin_memory()
    for _ in range(2):
        solver.factor_solve_host(pin["D"], pin["E"], pin["C"], pin["R"], pin["r"], xh)
    e2e_ms = []
    for _ in range(min(args.steps, 200)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, code = solver.factor_solve_host(pin["D"], pin["E"], pin["C"], pin["R"], pin["r"], xh)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        if code != 0 and not (prec == bm.BM_PREC_FP32_IR and code in (2, 5)):
            raise RuntimeError("host entry status %d" % code)
    e2e_piped = solver.query().get("host_pipelined", 0)
    e2e_step = max_over_ranks(statistics.mean(e2e_ms), dist, dev)
    h2d = sum(pin[k].numel() * 8 for k in ("D", "E", "C", "R", "r"))
    d2h = xh.numel() * 8

    meas = gpu_residual_measures(g, x)
    fwd_vs_fp64 = None
    if args.precision != "fp64" and not args.no_fp64_compare:
        # the error of the mixed result against the FP64 path's solution
        ref = bm.BranchKKTSolver(w.S, w.N, w.nb, w.nr)
        ref.factor(g["D"], g["E"], g["C"], g["R"])
        x64 = ref.solve(g["r"])
        fwd_vs_fp64 = float((x - x64).abs().max() / x64.abs().max())
        ref.close()
        del x64
    # a captured solve stops its refinement loop after the last iteration that
    # runs; directly launched, every unrolled iteration is a launch
    graph_loop = prec == bm.BM_PREC_FP32_IR and not args.direct
    launches_per_step = solver.launches_per_step(info.get("iters") if graph_loop else None)
    fmean = statistics.mean(fac_ms)
    # minimum bytes of one factor: A (D, E, C, R in FP64) read once, L (three
    # blocks per stage, FP64 or FP32) written once
    wbytes = 8 if args.precision == "fp64" else 4
    a_bytes = 8 * (w.S * (2 * w.N - 1) * w.nb * w.nb + w.S * w.nr * w.nb + w.nr * w.nr)
    l_bytes = wbytes * 3 * w.S * w.N * w.nb * w.nb
    factor_gbs = (a_bytes + l_bytes) / (fmean * 1e-3) / 1e9
    # the same steps with L2 left warm (no flush between steps)
    warm = []
    for _ in range(min(args.steps, 1000)):
        a_, b_, c_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True), \
            torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        solver.factor(g["D"], g["E"], g["C"], g["R"])
        b_.record(stream)
        solver.solve(g["r"], x)
        c_.record(stream)
        warm.append((a_, b_, c_))
    torch.cuda.synchronize()
    warm_fac = statistics.median(a_.elapsed_time(b_) for a_, b_, _ in warm)
    warm_sol = statistics.median(b_.elapsed_time(c_) for _, b_, c_ in warm)
    mhz = _peaks()[0].get("sm_max_mhz", 2070.0)
    if args.precision == "fp64":
        peak_alu = fp64_peak_gflops()
        peak_src = "FP64 ALU derived: 152 SMs x 2 FMA/clk x 2 flop x %.0f MHz" % mhz
    else:
        peak_alu = fp32_peak_gflops()
        peak_src = "FP32 ALU derived: 152 SMs x 128 FMA/clk x 2 flop x %.0f MHz (tails are FP32)" % mhz
    achieved = fl["factor"] / (fmean * 1e-3) / 1e9
    traffic = _profile_traffic(w.name, args.precision)
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded MPC-shaped generator; the paper's quadrotor data are not available)",
        "config": {"workload": w.name, "S": w.S, "N": w.N, "nb": w.nb, "nr": w.nr,
                   "precision": args.precision, "l2": "flushed between timed steps (256 MiB write)",
                   "launch": "direct" if args.direct else "graph",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "factor_us": fmean * 1e3, "solve_us": statistics.mean(sol_ms) * 1e3,
        "factor_us_median": statistics.median(fac_ms) * 1e3, "solve_us_median": statistics.median(sol_ms) * 1e3,
        "l2_warm": {"factor_us_median": warm_fac * 1e3, "solve_us_median": warm_sol * 1e3,
                    "us_per_kkt": (warm_fac + warm_sol) * 1e3, "steps": len(warm)},
        "factor_hbm": {"algorithmic_bytes": a_bytes + l_bytes, "achieved_gbs": factor_gbs,
                       "frac_of_measured_hbm": factor_gbs / _peaks()[0]["hbm_gbs"]},
        "us_per_kkt": ms_per_step * 1e3, **meas,
        "forward_error_vs_fp64": fwd_vs_fp64, "refinement_steps": info.get("iters"),
        "device_status": info["name"],
        "residual_float_float": info.get("residual_float_float") if args.precision == "fp32ir" else None,
        "flops_per_kkt": {"method": fl["total"], "natural_order_factor": bmgen.natural_flops(w.S, w.N, w.nb, w.nr)},
        "roofline": {"kernel": "factor pipeline (%s, one graph)" % _factor_kernels(w.N, w.nb, args.precision),
                     "bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "GFLOP/s",
                     "frac": achieved / peak_alu, "traffic": traffic, "peak_source": peak_src,
                     "achieved_basis": "method flops of one factor (%.4g) / mean factor time over the timed "
                                       "steps (CUDA events on the launching stream)" % fl["factor"]},
        "e2e": {"value": whole_job_gflops(world, fl["total"], 1, e2e_step), "unit": "GFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step,
                "copies_overlap_factor": bool(e2e_piped)},
        "gpu_launches": launches_per_step * args.steps,
        "schedule": _schedule_of(solver, bm),
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sec, threads, reps = time_oracle(sysd, args.ref_budget)
        line["cpu_baseline"] = {"value": fl["total"] / sec / 1e9, "unit": "GFLOP/s", "cores": threads,
                                "kind": "oracle",
                                "sample": "full workload factor+solve x%d (%.1f s)" % (reps, sec * reps)}
        sec1, _, reps1 = time_oracle(sysd, min(3.0, args.ref_budget), min_reps=1, nthreads=1)
        line["cpu_baseline_single_thread"] = {"value": fl["total"] / sec1 / 1e9, "unit": "GFLOP/s", "cores": 1,
                                              "kind": "oracle", "us_per_kkt": sec1 * 1e6,
                                              "sample": "full workload factor+solve x%d" % reps1}
    solver.close()
    if args.precision == "fp64" and not args.no_fp32ir_compare:
        # the FP32-tail + FP64-refinement path on the same system, same timing
        mixed = bm.BranchKKTSolver(w.S, w.N, w.nb, w.nr, precision=bm.BM_PREC_FP32_IR,
                                   max_refine=args.max_refine, tol=args.tol, flags=_coupling_flags(args))
        xm = torch.empty_like(g["r"])
        for _ in range(max(3, args.warmup)):
            mixed.factor(g["D"], g["E"], g["C"], g["R"])
            mixed.solve(g["r"], xm)
        k = min(args.steps, 1000)
        evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize()
        for a, b, c in evm:
            flush.zero_()
            a.record(stream)
            mixed.factor(g["D"], g["E"], g["C"], g["R"])
            b.record(stream)
            mixed.solve(g["r"], xm)
            c.record(stream)
        torch.cuda.synchronize()
        mfac = statistics.mean(a.elapsed_time(b) for a, b, _ in evm)
        msol = statistics.mean(b.elapsed_time(c) for _, b, c in evm)
        mms = mfac + msol
        minfo = mixed.query()
        mmeas = gpu_residual_measures(g, xm)
        line["fp32ir_same_workload"] = {
            "us_per_kkt": mms * 1e3, "factor_us": mfac * 1e3, "solve_us": msol * 1e3,
            "value": world * fl["total"] / (mms * 1e-3) / 1e9, "unit": "GFLOP/s",
            "steps": k, **mmeas, "refinement_steps": minfo["iters"],
            "coupling_refined": minfo["coupling_refined"],
            "residual_float_float": minfo["residual_float_float"],
            "forward_error_vs_fp64": float((xm - x).abs().max() / x.abs().max()),
            "device_status": minfo["name"], "speedup_vs_fp64": ms_per_step / mms,
            "gpu_launches_per_step": mixed.launches_per_step(minfo.get("iters"))}
        mixed.close()
        del xm
    if world == 1 and rank == 0 and not args.no_forms and w.name == DEFAULT_WORKLOAD and not args.shape:
        # the batched and serving forms of the method on their own workloads,
        # reported beside the single-system line (each its own timed region)
        del g, x
        torch.cuda.empty_cache()
        line["batched"] = _sub_line(lambda: _batched_summary(batched_line(args, min(args.steps, 3), 2)))
        line["serving"] = _sub_line(lambda: _serving_summary(serving_line(args)))
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _schedule_of(solver, bm):
    """The FP64 factor's launch schedule (autotuned on the first factor), or
    None for the mixed path."""
    try:
        return solver.schedule()
    except bm.BMError:
        return None


def _coupling_flags(args):
    import paper_2609_29977_gb300 as bm
    f = {"auto": 0, "refine": bm.BM_FLAG_COUPLING_REFINE, "fp32": bm.BM_FLAG_COUPLING_FP32}[args.coupling]
    return f | (bm.BM_FLAG_RESIDUAL_FP64 if args.residual == "fp64" else 0)


def _sub_line(fn):
    try:
        return fn()
    except Exception as e:   # a failing form is reported, not fatal to the main line
        return {"error": "%s: %s" % (type(e).__name__, e)}


def _batched_summary(b):
    keep = ("value", "unit", "ms_per_step", "factor_ms", "solve_ms", "fp64_sequential_ms",
            "speedup_vs_fp64_sequential", "omega_max", "failed_systems", "forward_error_vs_fp64_max",
            "schedule", "steps", "warmup", "clocks")
    out = {k: b.get(k) for k in keep}
    out["config"] = b.get("config")
    return out


def _serving_summary(sv):
    out = {k: sv.get(k) for k in ("value", "unit", "p50_ms", "p99_ms", "throughput_vs_fp64", "config")}
    out["runs"] = {name: {k: r.get(k) for k in ("offered_rate", "throughput_req_s", "gflops", "p50_ms", "p99_ms",
                                                 "failed", "fp64_fallbacks", "device_omega_max",
                                                 "sample_omega_max")}
                   for name, r in sv.get("runs", {}).items()}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32ir"])
    ap.add_argument("--max-refine", type=int, default=10)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--ref-budget", type=float, default=10.0, help="seconds of oracle work")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape", default="", help="S,N,nb,nr override of the workload's shape (profiling)")
    ap.add_argument("--batch-count", type=int, default=256, help="systems in the batched workload")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the FP64 reference run of the batched and mixed-precision lines")
    ap.add_argument("--no-fp32ir-compare", action="store_true")
    ap.add_argument("--direct", action="store_true",
                    help="launch the kernels directly instead of replaying CUDA graphs (for ncu launch lists: ncu "
                         "does not list the kernels inside a graph's conditional refinement loop)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean Poisson arrivals per second")
    ap.add_argument("--requests", type=int, default=200, help="serving: requests per run")
    ap.add_argument("--pool", type=int, default=24, help="serving: distinct small systems")
    ap.add_argument("--large-frac", type=float, default=0.05, help="serving: fraction of large requests")
    ap.add_argument("--slots", type=int, default=8, help="serving: requests in flight at most")
    ap.add_argument("--serve-budget-gb", type=float, default=160.0, help="serving: HBM arena")
    ap.add_argument("--seed", type=int, default=2000)
    ap.add_argument("--gen-device", default="cuda", help="batched: where the systems are drawn (cuda or cpu)")
    ap.add_argument("--coupling", default="auto", choices=["auto", "refine", "fp32"],
                    help="mixed precision: refine the coupling columns automatically, always, or never")
    ap.add_argument("--residual", default="auto", choices=["auto", "fp64"],
                    help="fp32ir refinement residual: float-float when tol >= 1e-11 (auto) or always FP64")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the batched and serving sub-runs reported beside the main line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batched"):
        return run_batched(args)
    if args.workload.startswith("serving"):
        return run_serving(args)
    if args.workload.startswith("assembly"):
        return run_assembly(args)
    if args.workload.startswith("paper-grid"):
        return run_grid(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

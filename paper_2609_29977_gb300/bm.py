"""ctypes binding of libbm.so (include/bm.h): argument marshalling only.

Every function named ``bm_*`` here calls the C entry point of the same name.
Tensors are torch tensors (device tensors for bm_factor / bm_solve, host
tensors for bm_factor_solve_host); streams default to torch's current CUDA
stream. There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(HERE, "libbm.so")

BM_PREC_FP64 = 0
BM_PREC_FP32_IR = 1
BM_FLAG_NO_GRAPH = 1
BM_FLAG_COUPLING_REFINE = 2   # mixed precision: always refine the coupling columns
BM_FLAG_COUPLING_FP32 = 4     # mixed precision: never (root from the FP32 tail factor alone)
BM_FLAG_NO_TUNE = 8           # FP64: keep the default launch schedule (no autotuning)
BM_FLAG_RESIDUAL_FP64 = 16    # FP32_IR: FP64 refinement residuals, never float-float

BM_OK = 0
STATUS_NAMES = {0: "BM_OK", 1: "BM_ERR_INVALID_ARG", 2: "BM_ERR_NOT_SPD", 3: "BM_ERR_OOM",
                4: "BM_ERR_CUDA", 5: "BM_ERR_NOT_CONVERGED", 6: "BM_ERR_TIMEOUT",
                7: "BM_ERR_NOT_FACTORED"}

EXPORTED_SYMBOLS = ("bm_version", "bm_status_string", "bm_workspace_bytes", "bm_analyze", "bm_factor",
                    "bm_solve", "bm_residual", "bm_query", "bm_schedule", "bm_export_factor", "bm_factor_solve_host", "bm_destroy",
                    "bm_factor_solve_noalloc", "bm_round_to_fp32", "bm_batch_workspace_bytes",
                    "bm_batch_analyze", "bm_batch_factor", "bm_batch_solve", "bm_batch_query",
                    "bm_batch_schedule", "bm_batch_destroy", "bm_server_request_bytes", "bm_server_create",
                    "bm_server_submit", "bm_server_poll", "bm_server_get_stats", "bm_server_destroy",
                    "bm_assemble_reduced", "bm_test_bounded_wait")
BATCH_NB = (4, 6, 12, 24, 48)
BM_NOALLOC_SCRATCH_BYTES = 32 << 20
BM_SERVE_MAX_RHS = 8
BM_SERVE_MAX_SLOTS = 64
BM_REQ_HOST_IO = 1
BM_SERVE_FP64_FALLBACK = 1


class bm_desc(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("N", ctypes.c_int), ("nb", ctypes.c_int), ("nr", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_refine", ctypes.c_int), ("tol", ctypes.c_double),
                ("flags", ctypes.c_uint)]


class bm_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("fail_scenario", ctypes.c_int), ("fail_stage", ctypes.c_int),
                ("iters", ctypes.c_int), ("backward_error", ctypes.c_double), ("coupling_refined", ctypes.c_int),
                ("residual_float_float", ctypes.c_int), ("host_pipelined", ctypes.c_int)]


class bm_qp_desc(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("N", ctypes.c_int), ("nx", ctypes.c_int), ("nu", ctypes.c_int),
                ("tau", ctypes.c_double), ("delta", ctypes.c_double)]


class bm_server_desc(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("slots", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("flags", ctypes.c_int), ("tol", ctypes.c_double)]


class bm_request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_ulonglong), ("S", ctypes.c_int), ("N", ctypes.c_int), ("nb", ctypes.c_int),
                ("nr", ctypes.c_int), ("nrhs", ctypes.c_int), ("flags", ctypes.c_int),
                ("D", ctypes.c_void_p), ("E", ctypes.c_void_p), ("C", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("r", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class bm_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_ulonglong), ("status", ctypes.c_int), ("fail_scenario", ctypes.c_int),
                ("fail_stage", ctypes.c_int), ("fallback", ctypes.c_int), ("iters", ctypes.c_int * BM_SERVE_MAX_RHS),
                ("backward_error", ctypes.c_double * BM_SERVE_MAX_RHS), ("t_submit_us", ctypes.c_double),
                ("t_start_us", ctypes.c_double), ("t_factor_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


class bm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("admitted", ctypes.c_ulonglong),
                ("completed", ctypes.c_ulonglong), ("fallbacks", ctypes.c_ulonglong), ("queued", ctypes.c_int),
                ("in_flight", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("peak_bytes_in_use", ctypes.c_size_t),
                ("budget", ctypes.c_size_t)]


class BMError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = int(code)
        super().__init__("%s: %s (%s)" % (what, STATUS_NAMES.get(self.code, self.code),
                                          bm_status_string(self.code)))


_lib = None


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("libbm.so is not built (expected at %s); run __graft_entry__.build()" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    vp, dp, sz = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t
    lib.bm_version.restype = ctypes.c_int
    lib.bm_version.argtypes = []
    lib.bm_status_string.restype = ctypes.c_char_p
    lib.bm_status_string.argtypes = [ctypes.c_int]
    lib.bm_workspace_bytes.restype = sz
    lib.bm_workspace_bytes.argtypes = [ctypes.POINTER(bm_desc)]
    lib.bm_analyze.restype = ctypes.c_int
    lib.bm_analyze.argtypes = [ctypes.POINTER(bm_desc), vp, ctypes.POINTER(vp)]
    lib.bm_factor.restype = ctypes.c_int
    lib.bm_factor.argtypes = [vp, dp, dp, dp, dp, vp]
    lib.bm_solve.restype = ctypes.c_int
    lib.bm_solve.argtypes = [vp, dp, dp, vp]
    lib.bm_residual.restype = ctypes.c_int
    lib.bm_residual.argtypes = [vp, dp, dp, dp, vp]
    lib.bm_query.restype = ctypes.c_int
    lib.bm_query.argtypes = [vp, vp, ctypes.POINTER(bm_info)]
    lib.bm_export_factor.restype = ctypes.c_int
    lib.bm_export_factor.argtypes = [vp, dp, dp, dp, dp, dp, vp]
    lib.bm_factor_solve_host.restype = ctypes.c_int
    lib.bm_factor_solve_host.argtypes = [vp, dp, dp, dp, dp, dp, dp, vp]
    lib.bm_destroy.restype = None
    lib.bm_destroy.argtypes = [vp]
    lib.bm_batch_workspace_bytes.restype = sz
    lib.bm_batch_workspace_bytes.argtypes = [ctypes.POINTER(bm_desc), ctypes.c_int]
    lib.bm_batch_analyze.restype = ctypes.c_int
    lib.bm_batch_analyze.argtypes = [ctypes.POINTER(bm_desc), ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.bm_batch_factor.restype = ctypes.c_int
    lib.bm_batch_factor.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.bm_batch_solve.restype = ctypes.c_int
    lib.bm_batch_solve.argtypes = [vp, vp, vp, vp]
    lib.bm_batch_query.restype = ctypes.c_int
    lib.bm_batch_query.argtypes = [vp, vp, ctypes.POINTER(bm_info)]
    lib.bm_schedule.restype = ctypes.c_int
    lib.bm_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)]
    lib.bm_batch_schedule.restype = ctypes.c_int
    lib.bm_batch_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
    lib.bm_batch_destroy.restype = None
    lib.bm_batch_destroy.argtypes = [vp]
    lib.bm_round_to_fp32.restype = ctypes.c_int
    lib.bm_round_to_fp32.argtypes = [dp, dp, ctypes.c_size_t, vp]
    lib.bm_factor_solve_noalloc.restype = ctypes.c_int
    lib.bm_factor_solve_noalloc.argtypes = [ctypes.c_int] * 4 + [dp] * 6 + [vp]
    lib.bm_test_bounded_wait.restype = ctypes.c_int
    lib.bm_test_bounded_wait.argtypes = [ctypes.c_ulonglong, vp]
    lib.bm_assemble_reduced.restype = ctypes.c_int
    lib.bm_assemble_reduced.argtypes = [ctypes.POINTER(bm_qp_desc)] + [dp] * 11 + [vp]
    lib.bm_server_request_bytes.restype = sz
    lib.bm_server_request_bytes.argtypes = [ctypes.POINTER(bm_server_desc), ctypes.POINTER(bm_request)]
    lib.bm_server_create.restype = ctypes.c_int
    lib.bm_server_create.argtypes = [ctypes.POINTER(bm_server_desc), ctypes.POINTER(vp)]
    lib.bm_server_submit.restype = ctypes.c_int
    lib.bm_server_submit.argtypes = [vp, ctypes.POINTER(bm_request)]
    lib.bm_server_poll.restype = ctypes.c_int
    lib.bm_server_poll.argtypes = [vp, ctypes.c_int, ctypes.POINTER(bm_completion), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]
    lib.bm_server_get_stats.restype = ctypes.c_int
    lib.bm_server_get_stats.argtypes = [vp, ctypes.POINTER(bm_server_stats)]
    lib.bm_server_destroy.restype = None
    lib.bm_server_destroy.argtypes = [vp]
    _lib = lib
    return lib


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t, name, device=True):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if t.dtype != torch.float64:
        raise TypeError("%s must be float64" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if device != t.is_cuda:
        raise ValueError("%s must be a %s tensor" % (name, "CUDA" if device else "host"))
    return ctypes.c_void_p(t.data_ptr())


def _check(code, what):
    if code != BM_OK:
        raise BMError(code, what)


def bm_version() -> int:
    return int(_load().bm_version())


def bm_status_string(code: int) -> str:
    return _load().bm_status_string(int(code)).decode()


# block sizes with compiled tail kernels (factor and cluster solve)
TAIL_NB = (2, 3, 4, 6, 8, 12, 16, 24, 32, 48)


def chain_levels(N: int) -> int:
    """Odd-even levels of the N - 1 chain positions of a tail (Sec. II)."""
    return (N - 1).bit_length() if N > 1 else 0


def top_level(N: int) -> int:
    """First level with at most four positions per tail: it and the levels
    above it run in one launch per tail."""
    for lvl in range(chain_levels(N)):
        if (N // 2 if lvl == 0 else ((N - 1) >> lvl) + 1) <= 4:
            return lvl
    return chain_levels(N)


FF_RESIDUAL_MIN_TOL = 1e-11   # FP32_IR: float-float refinement residuals from this tolerance up


def ff_residual(tol=1e-10, flags=0) -> bool:
    """Whether a BM_PREC_FP32_IR handle computes float-float residuals."""
    tol = tol if tol > 0 else 1e-10
    return not (flags & BM_FLAG_RESIDUAL_FP64) and tol >= FF_RESIDUAL_MIN_TOL


def launches_per_step(S, N, nb, nr, precision=BM_PREC_FP64, max_refine=10, iters=None, flags=0,
                      tol=1e-10) -> int:
    """Kernels that one bm_factor + one bm_solve launch.

    Factor: one launch per level below ``top_level(N)``, one for the top
    levels, x_1 and (FP64) the root, whose last CTA does the root step; the
    mixed path launches the root separately (with the per-level generic kernels,
    used for block sizes without compiled tail kernels: one per level, one
    for x_1, one for the root). FP64 solve: tail forward, root, tail
    backward (generic kernels: one per level each way, plus x_1 forward,
    root and x_1 backward). Mixed factor: the tail launches, then with
    BM_FLAG_COUPLING_FP32 the root; with BM_FLAG_COUPLING_REFINE the four
    coupling-column launches and the root; by default the pivot-spread
    reduction, the probing root, the four coupling-column launches and a
    second root (the last five return at once when the probe does not engage
    the refinement). Mixed solve: with
    coupling columns (both modes but BM_FLAG_COUPLING_FP32) one launch for
    the first correction's root terms, then three kernels per refinement
    iteration; in the automatic mode one more, which resumes a failed
    refinement with refined coupling columns; pass the corrections of the solve
    (``query()["iters"]``) for a captured graph, whose loop stops after the
    last iteration that runs; without it the count is the unrolled
    direct-launch bound (``max_refine <= 0`` selects 10). With float-float
    refinement residuals (``ff_residual(tol, flags)``) the mixed factor
    first splits K into hi + lo floats: one more launch."""
    Lc = chain_levels(N)
    if precision == BM_PREC_FP32_IR:
        mr = max_refine if max_refine > 0 else 10
        runs = mr + 1 if iters is None else min(int(iters), mr) + 1
        split = 1 if ff_residual(tol, flags) else 0
        if flags & BM_FLAG_COUPLING_FP32:
            return split + (top_level(N) + 2) + 3 * runs
        # refined coupling columns: the first correction's root terms are
        # one more launch per solve (it returns at once when not refined)
        if flags & BM_FLAG_COUPLING_REFINE:
            return split + top_level(N) + 6 + 1 + 3 * runs
        # automatic: the retry decision after the refinement; launched
        # directly, also the resumed refinement's launches, which return at
        # once unless it runs (in a graph they are a conditional node: when
        # it runs, add 6 + 3 per resumed iteration)
        retry = 1 if iters is not None else 1 + 6 + 3 * mr
        return split + top_level(N) + 8 + 1 + 3 * runs + retry
    if nb not in TAIL_NB:
        return (Lc + 2) + (2 * Lc + 3)
    return (top_level(N) + 1) + 3


def make_desc(S, N, nb, nr, precision=BM_PREC_FP64, max_refine=10, tol=1e-10, flags=0) -> bm_desc:
    return bm_desc(int(S), int(N), int(nb), int(nr), int(precision), int(max_refine), float(tol), int(flags))


def bm_workspace_bytes(desc: bm_desc) -> int:
    return int(_load().bm_workspace_bytes(ctypes.byref(desc)))


def bm_analyze(desc: bm_desc, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_load().bm_analyze(ctypes.byref(desc), _stream(stream), ctypes.byref(h)), "bm_analyze")
    return h


def bm_factor(h, D, E, C, R, stream=None) -> None:
    _check(_load().bm_factor(h, _ptr(D, "D"), _ptr(E, "E") if E is not None and E.numel() else None,
                             _ptr(C, "C"), _ptr(R, "R"), _stream(stream)), "bm_factor")


def bm_solve(h, r, x, stream=None) -> None:
    _check(_load().bm_solve(h, _ptr(r, "r"), _ptr(x, "x"), _stream(stream)), "bm_solve")


def bm_residual(h, r, x, rho, stream=None) -> None:
    """rho = r - K x with the handle's refinement arithmetic (FP32_IR handles)."""
    _check(_load().bm_residual(h, _ptr(r, "r"), _ptr(x, "x"), _ptr(rho, "rho"), _stream(stream)), "bm_residual")


def bm_query(h, stream=None) -> dict:
    info = bm_info()
    code = _load().bm_query(h, _stream(stream), ctypes.byref(info))
    return {"status": int(code), "name": STATUS_NAMES.get(int(code), str(code)),
            "fail_scenario": info.fail_scenario, "fail_stage": info.fail_stage, "iters": info.iters,
            "backward_error": info.backward_error, "coupling_refined": int(info.coupling_refined),
            "residual_float_float": int(info.residual_float_float), "host_pipelined": int(info.host_pipelined)}


def bm_schedule(h) -> dict:
    """The FP64 factor's launch schedule (see include/bm.h): top level of the
    per-tail kernel, team size of each grid-wide level, and where it came
    from ("cache", "tuned" or "rule")."""
    top = ctypes.c_int()
    teams = (ctypes.c_int * 32)()
    src = ctypes.c_int()
    _check(_load().bm_schedule(h, ctypes.byref(top), teams, ctypes.byref(src)), "bm_schedule")
    return {"top_level": int(top.value), "teams": [int(teams[l]) for l in range(int(top.value))],
            "source": {1: "cache", 0: "tuned", -1: "rule"}.get(int(src.value), str(src.value))}


def bm_export_factor(h, Ld=None, Ll=None, Lr=None, F=None, LR=None, stream=None) -> None:
    _check(_load().bm_export_factor(h, _ptr(Ld, "Ld"), _ptr(Ll, "Ll"), _ptr(Lr, "Lr"), _ptr(F, "F"),
                                    _ptr(LR, "LR"), _stream(stream)), "bm_export_factor")


def bm_factor_solve_host(h, D, E, C, R, r, x, stream=None) -> int:
    """Host tensors in, host x out; returns the device status code."""
    return int(_load().bm_factor_solve_host(
        h, _ptr(D, "D", False), _ptr(E, "E", False) if E is not None and E.numel() else None,
        _ptr(C, "C", False), _ptr(R, "R", False), _ptr(r, "r", False), _ptr(x, "x", False), _stream(stream)))


def bm_destroy(h) -> None:
    if h:
        _load().bm_destroy(h)


def bm_factor_solve_noalloc(S, N, nb, nr, D, E, C, R, r, x, stream=None) -> int:
    """FP64 factor + solve in the library's fixed device scratch array, for
    callers that cannot allocate device memory; synchronizes the stream and
    returns the device status code (see include/bm.h)."""
    return int(_load().bm_factor_solve_noalloc(
        int(S), int(N), int(nb), int(nr), _ptr(D, "D"), _ptr(E, "E") if E is not None and E.numel() else None,
        _ptr(C, "C"), _ptr(R, "R"), _ptr(r, "r"), _ptr(x, "x"), _stream(stream)))


def bm_round_to_fp32(src, dst, stream=None) -> None:
    """Round a float64 device tensor into a float32 device tensor (same size)."""
    import torch
    if dst.dtype != torch.float32 or not dst.is_cuda or not dst.is_contiguous() or dst.numel() != src.numel():
        raise ValueError("dst must be a contiguous float32 CUDA tensor of src's size")
    _check(_load().bm_round_to_fp32(_ptr(src, "src"), ctypes.c_void_p(dst.data_ptr()), src.numel(),
                                    _stream(stream)), "bm_round_to_fp32")


class BranchKKTSolver:
    """Owns one bm_handle: analyze once, then factor / solve many times."""

    def __init__(self, S, N, nb, nr, precision=BM_PREC_FP64, max_refine=10, tol=1e-10, flags=0, stream=None):
        self.desc = make_desc(S, N, nb, nr, precision, max_refine, tol, flags)
        self.shape = (S, N, nb, nr)
        self.n = S * N * nb + nr
        self.h = bm_analyze(self.desc, stream)

    def factor(self, D, E, C, R, stream=None):
        bm_factor(self.h, D, E, C, R, stream)
        return self

    def solve(self, r, x=None, stream=None):
        import torch
        if x is None:
            x = torch.empty_like(r)
        bm_solve(self.h, r, x, stream)
        return x

    def residual(self, r, x, rho=None, stream=None):
        import torch
        if rho is None:
            rho = torch.empty_like(r)
        bm_residual(self.h, r, x, rho, stream)
        return rho

    def launches_per_step(self, iters=None) -> int:
        """Kernels one bm_factor + one bm_solve of this handle launch (see
        the module-level ``launches_per_step``)."""
        S, N, nb, nr = self.shape
        return launches_per_step(S, N, nb, nr, self.desc.precision, self.desc.max_refine, iters, self.desc.flags,
                                 self.desc.tol)

    def query(self, stream=None) -> dict:
        return bm_query(self.h, stream)

    def schedule(self) -> dict:
        return bm_schedule(self.h)

    def export_factor(self, stream=None) -> dict:
        import torch
        S, N, nb, nr = self.shape
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {k: torch.empty((S, N, nb, nb), dtype=torch.float64, device=dev) for k in ("Ld", "Ll", "Lr")}
        out["F"] = torch.empty((S, nr, nb), dtype=torch.float64, device=dev)
        out["LR"] = torch.empty((nr, nr), dtype=torch.float64, device=dev)
        bm_export_factor(self.h, out["Ld"], out["Ll"], out["Lr"], out["F"], out["LR"], stream)
        return out

    def factor_solve_host(self, D, E, C, R, r, x=None, stream=None):
        import torch
        if x is None:
            x = torch.empty_like(r)
        code = bm_factor_solve_host(self.h, D, E, C, R, r, x, stream)
        return x, code

    def close(self):
        if self.h:
            bm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched form ---------------------------------------------------------------

def _desc_array(shapes, max_refine, tol):
    arr = (bm_desc * len(shapes))()
    for i, (S, N, nb, nr) in enumerate(shapes):
        arr[i] = make_desc(S, N, nb, nr, BM_PREC_FP32_IR, max_refine, tol)
    return arr


def bm_batch_workspace_bytes(shapes, max_refine=10, tol=1e-10) -> int:
    arr = _desc_array(shapes, max_refine, tol)
    return int(_load().bm_batch_workspace_bytes(arr, len(shapes)))


def bm_batch_analyze(shapes, max_refine=10, tol=1e-10, stream=None):
    arr = _desc_array(shapes, max_refine, tol)
    h = ctypes.c_void_p()
    _check(_load().bm_batch_analyze(arr, len(shapes), _stream(stream), ctypes.byref(h)), "bm_batch_analyze")
    return h


def _ptr_array(tensors, name, allow_empty=False):
    import torch
    ptrs = []
    for t in tensors:
        if t is None or (allow_empty and t.numel() == 0):
            ptrs.append(0)
        else:
            ptrs.append(_ptr(t, name).value)
    return torch.tensor(ptrs, dtype=torch.int64, device="cuda")


def bm_batch_factor(h, Dp, Ep, Cp, Rp, stream=None) -> None:
    """Dp, Ep, Cp, Rp: int64 CUDA tensors holding the device pointers."""
    _check(_load().bm_batch_factor(h, ctypes.c_void_p(Dp.data_ptr()), ctypes.c_void_p(Ep.data_ptr()),
                                   ctypes.c_void_p(Cp.data_ptr()), ctypes.c_void_p(Rp.data_ptr()),
                                   _stream(stream)), "bm_batch_factor")


def bm_batch_solve(h, rp, xp, stream=None) -> None:
    _check(_load().bm_batch_solve(h, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(xp.data_ptr()),
                                  _stream(stream)), "bm_batch_solve")


def bm_batch_query(h, count, stream=None) -> list:
    infos = (bm_info * count)()
    _load().bm_batch_query(h, _stream(stream), infos)
    return [{"status": i.status, "name": STATUS_NAMES.get(i.status, str(i.status)), "fail_scenario": i.fail_scenario,
             "fail_stage": i.fail_stage, "iters": i.iters, "backward_error": i.backward_error} for i in infos]


def bm_batch_schedule(h) -> dict:
    t, c, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    code = _load().bm_batch_schedule(h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(f))
    return {"status": code, "threads_per_cta": t.value, "ctas_per_sm": c.value, "from_cache": bool(f.value)}


def bm_batch_destroy(h) -> None:
    if h:
        _load().bm_batch_destroy(h)


class BranchKKTBatch:
    """Many independent systems (list of (S, N, nb, nr)) factored in one
    persistent launch and solved with FP32 tails + FP64 refinement."""

    def __init__(self, shapes, max_refine=10, tol=1e-10, stream=None):
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.count = len(self.shapes)
        self.h = bm_batch_analyze(self.shapes, max_refine, tol, stream)
        self._keep = []

    def factor(self, Ds, Es, Cs, Rs, stream=None):
        arrs = (_ptr_array(Ds, "D"), _ptr_array(Es, "E", True), _ptr_array(Cs, "C"), _ptr_array(Rs, "R"))
        self._keep = [arrs, list(Ds), list(Es), list(Cs), list(Rs)]
        bm_batch_factor(self.h, *arrs, stream=stream)
        return self

    def solve(self, rs, xs=None, stream=None):
        import torch
        if xs is None:
            xs = [torch.empty_like(r) for r in rs]
        rp, xp = _ptr_array(rs, "r"), _ptr_array(xs, "x")
        self._keep_solve = [rp, xp, list(rs), list(xs)]
        bm_batch_solve(self.h, rp, xp, stream)
        return xs

    def query(self, stream=None) -> list:
        return bm_batch_query(self.h, self.count, stream)

    def schedule(self) -> dict:
        return bm_batch_schedule(self.h)

    def close(self):
        if self.h:
            bm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# Serving runtime (include/bm.h, "Serving runtime")

def make_server_desc(hbm_budget, slots=8, precision=BM_PREC_FP32_IR, max_refine=10, tol=1e-10,
                     fp64_fallback=False) -> bm_server_desc:
    return bm_server_desc(int(hbm_budget), int(slots), int(precision), int(max_refine),
                          BM_SERVE_FP64_FALLBACK if fp64_fallback else 0, float(tol))


def _request(rid, S, N, nb, nr, D, E, C, R, r, x, host_io):
    dev = not host_io
    nrhs = r.shape[0] if r.dim() == 2 else 1
    return bm_request(int(rid), int(S), int(N), int(nb), int(nr), int(nrhs), BM_REQ_HOST_IO if host_io else 0,
                      _ptr(D, "D", dev), _ptr(E, "E", dev) if N > 1 else None, _ptr(C, "C", dev),
                      _ptr(R, "R", dev), _ptr(r, "r", dev), _ptr(x, "x", dev))


def bm_server_request_bytes(desc: bm_server_desc, req: bm_request) -> int:
    return int(_load().bm_server_request_bytes(ctypes.byref(desc), ctypes.byref(req)))


def bm_server_create(desc: bm_server_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_load().bm_server_create(ctypes.byref(desc), ctypes.byref(h)), "bm_server_create")
    return h


def bm_server_submit(s, req: bm_request) -> None:
    _check(_load().bm_server_submit(s, ctypes.byref(req)), "bm_server_submit")


def _completion_dict(c: bm_completion, nrhs: int) -> dict:
    return {"id": int(c.id), "status": int(c.status), "fail_scenario": int(c.fail_scenario),
            "fail_stage": int(c.fail_stage), "fallback": int(c.fallback),
            "iters": [int(c.iters[j]) for j in range(nrhs)],
            "backward_error": [float(c.backward_error[j]) for j in range(nrhs)],
            "t_submit_us": float(c.t_submit_us), "t_start_us": float(c.t_start_us),
            "t_factor_us": float(c.t_factor_us), "t_done_us": float(c.t_done_us)}


def bm_server_poll(s, wait=False, max_out=256) -> list:
    buf = (bm_completion * max_out)()
    n = ctypes.c_int(0)
    _check(_load().bm_server_poll(s, 1 if wait else 0, buf, max_out, ctypes.byref(n)), "bm_server_poll")
    return [buf[i] for i in range(n.value)]


def bm_server_get_stats(s) -> dict:
    st = bm_server_stats()
    _check(_load().bm_server_get_stats(s, ctypes.byref(st)), "bm_server_get_stats")
    return {k: int(getattr(st, k)) for k, _ in bm_server_stats._fields_}


def bm_server_destroy(s) -> None:
    _load().bm_server_destroy(s)


class BranchKKTServer:
    """A request loop over one GPU: admits requests by device memory (first in,
    first out), keeps each request's factor resident while its right-hand
    sides are solved, and overlaps admitted requests on separate streams.
    Tensors of a request are held here until its completion is returned.
    """

    def __init__(self, hbm_budget, slots=8, precision=BM_PREC_FP32_IR, max_refine=10, tol=1e-10,
                 fp64_fallback=False):
        self.desc = make_server_desc(hbm_budget, slots, precision, max_refine, tol, fp64_fallback)
        self.h = bm_server_create(self.desc)
        self._held = {}

    def request_bytes(self, S, N, nb, nr, D, E, C, R, r, x, host_io=False) -> int:
        return bm_server_request_bytes(self.desc, _request(0, S, N, nb, nr, D, E, C, R, r, x, host_io))

    def submit(self, rid, S, N, nb, nr, D, E, C, R, r, x, host_io=False) -> None:
        """r, x: [nrhs, S*N*nb + nr] (or one vector); device tensors, or host
        tensors (page-locked for speed) with host_io=True."""
        if rid in self._held:
            raise ValueError("request id %r is already in flight" % (rid,))
        req = _request(rid, S, N, nb, nr, D, E, C, R, r, x, host_io)
        bm_server_submit(self.h, req)
        self._held[rid] = (D, E, C, R, r, x, req.nrhs)

    def poll(self, wait=False) -> list:
        out = []
        for c in bm_server_poll(self.h, wait):
            nrhs = self._held.pop(int(c.id))[6]
            out.append(_completion_dict(c, nrhs))
        return out

    def drain(self) -> list:
        out = []
        while self._held:
            out.extend(self.poll(wait=True))
        return out

    def stats(self) -> dict:
        return bm_server_get_stats(self.h)

    def close(self):
        if self.h is not None and self.h.value:
            bm_server_destroy(self.h)
        self.h = None
        self._held = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# Assembly front end (include/bm.h, "Assembly front end")

def bm_assemble_reduced(qp: dict, stream=None) -> dict:
    """K = P + tau I + delta^{-1} A^T A + G^T (W + delta I)^{-1} G of a
    branch-MPC QP (device tensors A, B, q, rw, r0w, w, w0 and the scalars of
    bmgen.generate_qp's layout) in the D, E, C, R layout of bm_factor."""
    import torch
    S, N, nx, nu = int(qp["S"]), int(qp["N"]), int(qp["nx"]), int(qp["nu"])
    nb = nx + nu
    dev = qp["A"].device
    D = torch.empty((S, N, nb, nb), dtype=torch.float64, device=dev)
    E = torch.empty((S, max(N - 1, 0), nb, nb), dtype=torch.float64, device=dev)
    C = torch.empty((S, nu, nb), dtype=torch.float64, device=dev)
    R = torch.empty((nu, nu), dtype=torch.float64, device=dev)
    desc = bm_qp_desc(S, N, nx, nu, float(qp["tau"]), float(qp["delta"]))
    _check(_load().bm_assemble_reduced(ctypes.byref(desc), _ptr(qp["A"], "A"), _ptr(qp["B"], "B"),
                                       _ptr(qp["q"], "q"), _ptr(qp["rw"], "rw"), _ptr(qp["r0w"], "r0w"),
                                       _ptr(qp["w"], "w"), _ptr(qp["w0"], "w0"), _ptr(D, "D"),
                                       _ptr(E, "E") if N > 1 else None, _ptr(C, "C"), _ptr(R, "R"),
                                       _stream(stream)), "bm_assemble_reduced")
    return {"D": D, "E": E, "C": C, "R": R, "S": S, "N": N, "nb": nb, "nr": nu}


def bm_test_bounded_wait(limit_cycles: int, stream=None) -> int:
    """Status left by the batched factor's bounded wait on a counter that
    nothing increments (BM_ERR_TIMEOUT = 6 when the wait behaves)."""
    return int(_load().bm_test_bounded_wait(int(limit_cycles), _stream(stream)))

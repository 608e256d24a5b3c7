"""Host-side logic of the serving runtime, on CPU: bm_server_request_bytes
sizes an admitted request's arena range (the factor workspace, plus the
staging of inputs and outputs for host-buffer requests) and rejects
malformed requests, without touching a GPU (the pointers are only checked,
never dereferenced)."""
import ctypes

import pytest

import paper_2609_29977_gb300 as bm
from paper_2609_29977_gb300 import bm as core


def _req(S, N, nb, nr, nrhs=4, flags=0, base=1 << 20, r_off=0, x_off=None):
    n = S * N * nb + nr
    if x_off is None:
        x_off = r_off + 8 * n * nrhs + 256
    p = lambda k: ctypes.c_void_p(base + 4096 * k)       # aligned, distinct, never dereferenced
    return core.bm_request(7, S, N, nb, nr, nrhs, flags, p(1), p(2), p(3), p(4),
                           ctypes.c_void_p(base + (1 << 30) + r_off), ctypes.c_void_p(base + (1 << 30) + x_off))


def _bytes(desc, req):
    return core.bm_server_request_bytes(desc, req)


def test_request_bytes_cover_the_workspace_and_host_staging():
    for prec in (core.BM_PREC_FP64, core.BM_PREC_FP32_IR):
        desc = core.make_server_desc(1 << 30, 4, prec)
        S, N, nb, nr, nrhs = 3, 17, 12, 4, 4
        dev = _bytes(desc, _req(S, N, nb, nr, nrhs))
        work = core.bm_workspace_bytes(core.make_desc(S, N, nb, nr, precision=prec))
        assert dev >= work and dev - work < 256
        host = _bytes(desc, _req(S, N, nb, nr, nrhs, flags=core.BM_REQ_HOST_IO))
        n = S * N * nb + nr
        staged = 8 * (S * N * nb * nb + S * (N - 1) * nb * nb + S * nr * nb + nr * nr + 2 * nrhs * n)
        assert staged <= host - dev < staged + 6 * 256
    # FP32 tails make the mixed workspace smaller than the FP64 one
    f64 = _bytes(core.make_server_desc(1 << 30, 4, core.BM_PREC_FP64), _req(8, 64, 24, 8))
    mix = _bytes(core.make_server_desc(1 << 30, 4, core.BM_PREC_FP32_IR), _req(8, 64, 24, 8))
    assert mix < f64


def test_malformed_requests_size_to_zero():
    desc = core.make_server_desc(1 << 30, 4, core.BM_PREC_FP32_IR)
    assert _bytes(desc, _req(2, 8, 6, 2)) > 0
    assert _bytes(desc, _req(2, 8, 6, 2, nrhs=0)) == 0
    assert _bytes(desc, _req(2, 8, 6, 2, nrhs=core.BM_SERVE_MAX_RHS + 1)) == 0
    assert _bytes(desc, _req(2, 8, 5, 2)) == 0                       # no FP32 tail kernel for nb = 5
    assert _bytes(desc, _req(2, 8, 6, 2, flags=4)) == 0              # unknown flag
    assert _bytes(desc, _req(2, 8, 6, 2, r_off=0, x_off=8)) == 0     # x overlaps r
    bad = _req(2, 8, 6, 2)
    bad.D = ctypes.c_void_p((1 << 20) + 4)                           # device pointer not 16-byte aligned
    assert _bytes(desc, bad) == 0
    f64 = core.make_server_desc(1 << 30, 4, core.BM_PREC_FP64)
    assert _bytes(f64, _req(2, 8, 5, 2)) > 0                         # the FP64 path takes any nb <= 64
    assert _bytes(f64, _req(2, 8, 65, 2)) == 0


def test_server_descriptor_is_validated_before_any_device_call():
    with pytest.raises(bm.BMError):
        bm.BranchKKTServer(0, slots=2)                                # no budget
    with pytest.raises(bm.BMError):
        bm.BranchKKTServer(1 << 20, slots=core.BM_SERVE_MAX_SLOTS + 1)
    with pytest.raises(bm.BMError):
        bm.BranchKKTServer(1 << 20, slots=2, precision=7)

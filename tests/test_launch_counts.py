"""The kernel counts the bench reports (``gpu_launches``), checked on CPU
against counts taken by hand from the launch sequence of the library:
factor = one launch per level below the top level, one top launch (FP64:
its last CTA does the root step; mixed: a root launch follows); FP64 solve = forward, root, backward; mixed factor = the tail
launches plus the root (FP32-based root), plus four coupling-column
launches (always refined), plus a pivot-spread reduction and a probing root
(automatic); mixed solve =
one root-term launch when coupling columns may be used, then three kernels
per refinement iteration."""
from paper_2609_29977_gb300 import bm as core


def test_levels_of_the_medium_workload():
    # N = 64: 63 chain positions, levels 0..5 (+ x_1); per-tail positions by
    # level 32, 32, 16, 8, 4 -> level 4 is the first with at most four
    assert core.chain_levels(64) == 6
    assert core.top_level(64) == 4
    assert core.chain_levels(1) == 0 and core.top_level(1) == 0
    assert core.chain_levels(2) == 1 and core.top_level(2) == 0     # one chain position
    assert core.top_level(9) == 0      # level 0 already has N/2 = 4 positions
    assert core.top_level(10) == 2     # levels 0, 1, 2: 5, 5, 3 positions (level 1 holds 4 eliminations + x_1's update)


def test_fp64_counts():
    # medium: 4 level launches + top (whose last CTA does the root), then
    # forward + root + backward
    assert core.launches_per_step(64, 64, 12, 4) == 8
    # a block size without compiled tail kernels (generic per-level path)
    Lc = core.chain_levels(9)
    assert Lc == 4
    assert core.launches_per_step(2, 9, 5, 3) == (Lc + 2) + (2 * Lc + 3) == 17


def test_mixed_counts():
    # FP64 refinement residuals (the float-float split kernel is counted below)
    fp32 = core.BM_FLAG_COUPLING_FP32 | core.BM_FLAG_RESIDUAL_FP64
    # medium, FP32-based root, 2 corrections in a captured graph: 6 factor + 3 x 3 solve
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2, flags=fp32) == 15
    # directly launched: all 11 iterations
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, flags=fp32) == 6 + 33
    # max_refine <= 0 selects 10; the count never exceeds max_refine + 1 iterations
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 0, flags=fp32) == 6 + 33
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 3, iters=7, flags=fp32) == 6 + 12
    # refined coupling columns: 5 tail launches (top level 4 of N = 64),
    # bwd X0, residual, fwd, bwd correction, root; the solve adds the first
    # correction's root terms
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2,
                                  flags=core.BM_FLAG_COUPLING_REFINE | core.BM_FLAG_RESIDUAL_FP64) == 10 + 1 + 9
    # automatic (default): pivot-spread reduction and probing root in addition
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2,
                                  flags=core.BM_FLAG_RESIDUAL_FP64) == 12 + 1 + 9 + 1
    # float-float residuals (tol >= 1e-11, the default 1e-10): one split launch in the factor
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2,
                                  flags=core.BM_FLAG_COUPLING_REFINE) == 1 + 10 + 1 + 9
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2) == 1 + 12 + 1 + 9 + 1
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2, tol=1e-11) == 1 + 12 + 1 + 9 + 1
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2, tol=1e-12) == 12 + 1 + 9 + 1
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10, iters=2, tol=0) == 1 + 12 + 1 + 9 + 1
    # automatic mode launched directly: all 11 iterations, the retry decision,
    # the resumed refinement's 4 + 1 + 1 launches and its 10 iterations
    assert core.launches_per_step(64, 64, 12, 4, core.BM_PREC_FP32_IR, 10) == 1 + 12 + 1 + 33 + 1 + 6 + 30
    # the mixed workload (N = 128: levels 0..6, top level 5): 6 tail launches
    assert core.top_level(128) == 5
    assert core.launches_per_step(512, 128, 24, 8, core.BM_PREC_FP32_IR, 8, iters=3) == 1 + 13 + 1 + 12 + 1

"""ORACLE -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything from this package. The CUDA library never
imports it and it never imports the CUDA library.

Two independent FP64 references of the root-coupled SPD solve of Sec. III-B:

* ``oracle.natural`` -- a C block Cholesky in the natural variable order
  (tails forward, root last; the ordering of Fig. 2(a)), with solve,
  residual and the per-tail Schur complement onto the first stage.
* ``oracle.dense`` -- NumPy/SciPy on assembled dense matrices: the
  permutation Gamma_N of Sec. II and Pi_i of Sec. IV-A written from their
  definitions, and the Cholesky factor of the permuted matrix Pi K Pi^T
  (Eq. permuted_root_coupled_matrix) by a library dense Cholesky, from which
  every block of the two-level factor (Alg. 1) is read off.

Both are pinned by ``tests/test_oracle_pins.py`` against what the paper and
the mathematics fix (the Gamma_7 example, the printed seven-block pattern,
Theorem 1, dense LU on small systems, closed forms for nb = 1 and N = 1,
invariants of the factor).
"""

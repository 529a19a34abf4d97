"""CPU oracle for the LR-SPIKE hot path (FP64, plain loops, written from the paper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything in
this package.  The product library (``paper_2504_11167_gb300``) never imports it
and shares no code with it: the only thing both sides use is the seeded input
generator module ``paper_2504_11167_gb300.inputs``, which holds none of the
method's arithmetic.

Parity status per function (see the module docstrings for the pins):
  band LU / solves / matvec ..... pinned (dense LU, LAPACK gbtrf/gbsv, L*U = A)
  partitioning, B_i, C_i ........ pinned (dense slices of A)
  spikes ........................ pinned (A_i T_i = [0; B_i] by dense product)
  compression (SPIKE, COUPLING) . pinned (Eckart-Young, r = k exactness, rank <= r exactness)
  reduced system FULL ........... pinned (r = k gives A^{-1}; dense (D S~)^{-1})
  reduced system TRUNCATED ...... pinned (paper's x-tip 2x2 kernel + Woodbury form; p = 2)
  transpose ..................... pinned (dense M^{-1} transposed; adjoint identity)
  IR / BiCGStab ................. pinned (final residual, dense solve)
"""

"""Oracle for resistance distance by Lanczos iteration: plain, slow, FP64, CPU.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import, call, link or run
anything in this package. The product library (``paper_2601_11159_gb300``)
never does, and the two share no code.

* ``oracle.dense``   -- L^+ = (L + J/n)^{-1} - J/n, r, potentials, edge gradients (small n).
* ``oracle.lanczos`` -- Algorithm 3 in plain C (``lanczos_ref.c``), any n, one pair per thread.

Every function cites the passage of the paper it follows. All parts are pinned by
tests in ``tests/test_oracle_pins.py`` against closed forms, invariants and the
paper's one exact printed value (the running example's r(1,4) = 1).
"""

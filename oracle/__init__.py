"""FP64 CPU oracle for batched Orthogonal Matching Pursuit (test infrastructure).

This package is the independent checker of the CUDA path. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may import it; the
library ``paper_2407_06434_gb300`` never does, and the two share no code (the only common
dependency is the input generator package ``workloads``, which holds none of OMP's arithmetic).

Modules:
  omp    -- Alg. 1 in FP64: reference mode (least squares re-solved each step), timed mode
            (progressive Cholesky append, Sec. 2.1), inverse-Cholesky recurrence (Sec. 2.3),
            forced-support replay.
  quant  -- BF16 and FP8 E4M3 round-to-nearest-even conversions written from the formats'
            definitions, and the per-column / per-signal FP8 scaling the correlation uses.
  mlp    -- FP64 forward/backward of the learned proposal network (two dense layers + GELU +
            BCE-with-logits), for gradient checks.

Parity status: every function here is pinned by tests in ``tests/test_oracle_*.py`` against
brute force, closed forms, hand-worked examples or library routines; none is "parity unpinned".
"""

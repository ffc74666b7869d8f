"""CPU oracle for the single-pass online randomized interpolative decomposition.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the method of Li, Becker & Doostan, "Online randomized interpolative
decomposition with a posteriori error estimator for temporal PDE data
reduction" (arXiv 2405.16076), written from the paper's text:

* Algorithm 3 (single-pass randomized ID: sketching, streaming ridge-leverage
  column subset selection, batch step every t columns),
* Algorithms 4-7 (the four coefficient updates),
* Algorithm 8 with Eqs. 35-37 (NA-Hutch++ error estimate per candidate),
* Sec. 2.1, Eqs. 5-11 (offline CPQR-based ID), Eq. 16 (exact ridge leverage
  score), Sec. 3.4, Eqs. 38-43 (simplex-gradient operator),
* and, for the reduced-precision sketch forms (not in the paper), the E4M3
  block-scaled operands of an FP8 sketch (``oracle.fp8``).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library: the two
sides each implement the Philox4x32-10 counter generator from its published
definition and meet only on seeded inputs.

Parity status per function is listed in each module header; every function
here is pinned by a ``-m "not gpu"`` test against closed forms, brute force,
invariants or published known-answer values.
"""

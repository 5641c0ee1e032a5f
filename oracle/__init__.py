"""Plain FP64 CPU oracle for the phase-field fracture solver (test infrastructure only).

This package is the checker against which the CUDA library is compared.  It is written from
the paper (Farrell & Maurini, "Linear and nonlinear solvers for variational phase-field models
of brittle fracture"): assembled sparse matrices, sparse direct solves, and the nonlinear
algorithms (Algorithms 1-4) taken step by step in the paper's order.  It is slow on purpose.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The product path (``paper_1511_08463_gb300``) never imports it, and it never imports
the product path; both read problem descriptions from ``workloads``.

Parity status per function is listed in each module header.
"""

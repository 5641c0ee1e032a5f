"""Writes notched32_step31.npz: the oracle's state after load step 31 of the 32 x 32 notched
square on its 50-step schedule to t = 2 (AT1, ell = 4h, ORAM omega = 1.5, stopping tolerance
1e-10).  The GPU parity test of the crack-propagation steps starts both implementations from it
instead of re-running the 31 pre-initiation steps in the oracle each time.

Only the oracle computes it: python tests/golden/make_notched32_state.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import am  # noqa: E402
from oracle.problem import Problem  # noqa: E402

N, LAST = 32, 31


def main():
    w = W.notched_square(n=N)
    p = Problem(w)
    for (t, dT) in w.loads[:LAST]:
        r = am.load_step(p, t, dT, omega=w.omega, tol=1e-10, maxit=5000)
        assert r["status"] == "converged"
    np.savez_compressed(os.path.join(HERE, f"notched{N}_step{LAST}.npz"), u=p.u, alpha=p.alpha,
                        alpha_prev=p.alpha_prev, n=N, step=LAST, t=w.loads[LAST - 1][0])


if __name__ == "__main__":
    main()

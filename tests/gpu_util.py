"""Helpers shared by the GPU parity tests (no solver arithmetic: they only compare)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_08463_gb300 import _build

    _build.build()
    return torch


def rel_max(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def tight_opts(S, **kw):
    base = dict(am_tol=1e-10, u_rtol=1e-12, rs_rtol=1e-12, alpha_cg_rtol=1e-12, cg_maxit=5000,
                am_maxit=5000, precision="fp64")
    base.update(kw)
    return S.make_opts(**base)

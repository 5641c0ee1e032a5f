"""The seeded synthetic inputs (workloads.py) are reproducible and follow the distributions the
batch and serving configurations state; no GPU."""
import numpy as np

import workloads as W


def test_batch_of_notched_distribution_and_seed():
    a = W.batch_of_notched(n_instances=256, seed=0)
    b = W.batch_of_notched(n_instances=256, seed=0)
    c = W.batch_of_notched(n_instances=256, seed=1)
    key = lambda ws: [(w.nx, w.ell, w.nu, w.loads[0]) for w in ws]
    assert key(a) == key(b) and key(a) != key(c)
    ns = np.array([w.nx for w in a])
    assert np.all(ns % 16 == 0) and ns.min() >= 64 and ns.max() <= 256
    assert len(set(ns)) > 5  # spread over the log-uniform range
    ratio = np.array([w.ell * w.nx / w.lx for w in a])  # ell / h
    assert ratio.min() >= 2.0 - 1e-12 and ratio.max() <= 8.0 + 1e-12
    nu = np.array([w.nu for w in a])
    assert nu.min() >= 0.2 and nu.max() <= 0.35
    t = np.array([w.loads[0][0] for w in a])
    assert np.all(t >= 0.5 * 2.0 - 1e-12) and np.all(t <= 2.0 + 1e-12)
    assert all(len(w.loads) == 1 and w.nx == w.ny and w.kind == "crossed" for w in a)


def test_serving_stream_arrivals_sizes_and_steps():
    jobs = W.serving_stream(n_jobs=400, rate=4.0, seed=0)
    again = W.serving_stream(n_jobs=400, rate=4.0, seed=0)
    assert [(j.arrival, j.workload.nx, len(j.workload.loads)) for j in jobs] == \
        [(j.arrival, j.workload.nx, len(j.workload.loads)) for j in again]
    t = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 4.0) < 0.05  # Poisson arrivals at the stated rate
    steps = np.array([len(j.workload.loads) for j in jobs])
    assert steps.min() >= 10 and steps.max() <= 60
    kinds = {j.workload.kind for j in jobs}
    assert kinds == {"crossed", "right"}  # notched squares and bars
    for j in jobs:
        w = j.workload
        assert w.nx % 16 == 0 and 32 <= w.nx <= 1024
        if w.kind == "right":  # bar N x N/8
            assert w.ny * 8 == w.nx

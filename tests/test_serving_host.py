"""The serving workload's host side (no GPU): the seeded request trace is a
Poisson process with the stated rate, uniform kernel and storage-type mix and
log-uniform sizes, identical for a seed; and each request's compulsory bytes
follow the kernels' definitions (Table I: GEMVER reads A, writes and reads B;
the others read their matrices once)."""
import numpy as np

from paper_1205_1098_gb300.serve import OPS, compulsory_bytes, make_trace


def test_trace_is_seeded_and_well_formed():
    a = make_trace(seed=4, rate=20000.0, duration=1.0)
    b = make_trace(seed=4, rate=20000.0, duration=1.0)
    assert a == b and a != make_trace(seed=5, rate=20000.0, duration=1.0)
    t = np.array([r["t"] for r in a])
    assert np.all(np.diff(t) > 0) and t[-1] < 1.0 and t[0] > 0
    assert [r["id"] for r in a] == list(range(len(a)))


def test_trace_statistics():
    rate, dur, nmin, nmax = 20000.0, 2.0, 64, 8192
    tr = make_trace(seed=7, rate=rate, duration=dur, nmin=nmin, nmax=nmax)
    n_req = len(tr)
    assert abs(n_req - rate * dur) < 4 * np.sqrt(rate * dur)            # Poisson count
    gaps = np.diff([r["t"] for r in tr])
    assert abs(gaps.mean() * rate - 1) < 0.02 and abs(gaps.std() * rate - 1) < 0.03   # exponential gaps
    for op in OPS:
        frac = sum(r["op"] == op for r in tr) / n_req
        assert abs(frac - 1 / len(OPS)) < 0.02, op
    assert abs(sum(r["dtype"] == "bf16" for r in tr) / n_req - 0.5) < 0.02
    n = np.array([r["n"] for r in tr])
    assert n.min() >= nmin and n.max() <= nmax
    # Log-uniform sizes: log n is uniform, its median at the geometric mean.
    assert abs(np.median(np.log(n)) - 0.5 * (np.log(nmin) + np.log(nmax))) < 0.05


def test_fixed_count_trace():
    tr = make_trace(seed=9, rate=20000.0, duration=0.0, nmin=512, nmax=4096, count=48)
    assert len(tr) == 48 and all(512 <= r["n"] <= 4096 for r in tr)


def test_compulsory_bytes():
    n = 1000
    assert compulsory_bytes("bicgk", n, "f32") == 4 * n * n + 16 * n
    assert compulsory_bytes("bicgk", n, "bf16") == 2 * n * n + 16 * n
    assert compulsory_bytes("gemver", n, "f32") == 12 * n * n + 32 * n      # A read, B written and read
    assert compulsory_bytes("gesummv", n, "bf16") == 4 * n * n + 8 * n     # two matrices
    assert compulsory_bytes("atax", n, "f32") == 4 * n * n + 8 * n

"""The synthetic inputs are what the design notes say they are (CPU).

Graphs: exactly m distinct undirected edges, no self-loops, ids in [0, n), deterministic for a
seed; Chung-Lu weights sum to 2m and are capped at sqrt(2m); the bucketed generator for the
largest graph (run here on the CPU) keeps the same properties. Serving trace: Poisson arrivals in
[0, duration), the request mix and parameter ranges of its recipe, deterministic for a seed.
"""
import importlib.util
import os

import numpy as np
import pytest

from synth import graphs as SG

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check_edges(n, m, u, v):
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    assert u.shape == v.shape == (m,)
    assert u.min() >= 0 and v.min() >= 0 and u.max() < n and v.max() < n
    assert not np.any(u == v)
    key = np.minimum(u, v) * n + np.maximum(u, v)
    assert np.unique(key).size == m


def test_rmat_exact_distinct_edges_and_determinism():
    n, m = 4096, 30000
    u, v = SG.rmat_edges(n, m, seed=5)
    _check_edges(n, m, u, v)
    u2, v2 = SG.rmat_edges(n, m, seed=5)
    assert np.array_equal(u, u2) and np.array_equal(v, v2)
    u3, _ = SG.rmat_edges(n, m, seed=6)
    assert not np.array_equal(u, u3)
    # R-MAT skew: the heaviest node has far more than the average degree
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    assert deg.max() > 10 * deg.mean()


def test_chung_lu_weights_sum_and_cap():
    n, m = 100000, 1_000_000
    for gamma in (2.0, 2.1, 2.5):
        w = SG.chung_lu_weights(n, m, gamma)
        assert abs(w.sum() - 2 * m) < 1e-6 * 2 * m
        assert w.max() <= np.sqrt(2 * m) * (1 + 1e-12)
        assert np.all(np.diff(w) <= 1e-9)  # non-increasing with the node index


def test_chung_lu_edges_follow_the_weights():
    n, m = 20000, 200000
    u, v = SG.chung_lu_edges(n, m, 2.1, seed=3)
    _check_edges(n, m, u, v)
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    # ids are relabelled, so compare the degree distributions, not node by node
    w = np.sort(SG.chung_lu_weights(n, m, 2.1))[::-1]
    d = np.sort(deg)[::-1]
    top = slice(0, 200)
    assert abs(d[top].sum() / w[top].sum() - 1.0) < 0.15


@pytest.mark.parametrize("bucket_keys", [1 << 30, 1 << 18])
def test_bucketed_generator_on_cpu(bucket_keys):
    n, m = 50000, 400000
    u, v = SG.chung_lu_edges_cuda(n, m, 2.0, seed=11, device="cpu", chunk=1 << 18, bucket_keys=bucket_keys)
    _check_edges(n, m, u.numpy(), v.numpy())
    u2, v2 = SG.chung_lu_edges_cuda(n, m, 2.0, seed=11, device="cpu", chunk=1 << 18, bucket_keys=bucket_keys)
    assert torch.equal(u, u2) and torch.equal(v, v2)


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_serving_trace_recipe():
    bench = _bench()
    n = 20000
    rng = np.random.default_rng(0)
    u = rng.integers(0, n, 100000).astype(np.int32)
    v = rng.integers(0, n, 100000).astype(np.int32)
    rate, duration = 2000.0, 10.0
    tr = bench.serve_trace(n, u, v, rate, duration, 7, 1e-3)
    assert tr == bench.serve_trace(n, u, v, rate, duration, 7, 1e-3)
    t = np.array([r[0] for r in tr])
    assert np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < duration
    assert abs(len(tr) - rate * duration) < 5 * np.sqrt(rate * duration)
    kinds = np.array([r[1] for r in tr])
    frac = {k: np.mean(kinds == k) for k in ("ppr", "katz", "hkpr", "transition", "features")}
    assert abs(frac["features"] - 0.10) < 0.02
    for k in ("ppr", "katz", "hkpr", "transition"):
        assert abs(frac[k] - 0.225) < 0.02
    assert {r[2] for r in tr} == {1e-6, 1e-7, 1e-8, 1e-9}
    L = np.array([r[3] for r in tr])
    assert L.min() >= 5 and L.max() <= 40
    cols = np.array([r[5] for r in tr])
    assert cols.min() >= 1 and cols.max() <= 64
    src = np.array([r[4] for r in tr])
    assert src.min() >= 0 and src.max() < n

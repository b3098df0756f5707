"""The dependence-robust unbiasedness check (tests/_stats.py) on synthetic runs: it accepts unbiased
estimates whose nodes share a strong common fluctuation within each run, and rejects a 1% bias
confined to one degree class."""
import numpy as np
import pytest

from tests._stats import unbiased


def _runs(rng, N, exact, common_sd, node_sd):
    # every run scales all nodes by one shared factor (a sampled hub lifts them together) and adds
    # independent noise per node; both have mean zero, so the runs are unbiased
    common = rng.normal(0.0, common_sd, size=(N, 1))
    noise = rng.normal(0.0, node_sd, size=(N, exact.size))
    return exact[None, :] * (1.0 + common + noise)


def test_accepts_unbiased_dependent_runs():
    rng = np.random.default_rng(7)
    n, N = 5000, 200
    deg = rng.integers(1, 1000, n)
    exact = rng.random(n) + 0.1
    ok = 0
    for _ in range(20):
        runs = _runs(rng, N, exact, common_sd=0.05, node_sd=0.05)
        try:
            st = unbiased(runs, exact, deg)
            ok += 1
        except AssertionError:
            pass
    # the criteria are at 4 and 6 standard deviations: a failure on unbiased data is very rare
    assert ok >= 19
    # the naive fraction of nodes beyond the 99% bound swings with the common mode
    assert 0.0 <= st["frac_beyond_99"] <= 1.0


def test_rejects_class_bias():
    rng = np.random.default_rng(8)
    n, N = 5000, 200
    deg = rng.integers(1, 1000, n)
    exact = rng.random(n) + 0.1
    runs = _runs(rng, N, exact, common_sd=0.0, node_sd=0.05)
    cls = (deg >= 16) & (deg < 64)
    runs[:, cls] *= 1.01  # a planted 1% bias in one degree class
    with pytest.raises(AssertionError):
        unbiased(runs, exact, deg)


def test_rejects_node_bias():
    rng = np.random.default_rng(9)
    n, N = 5000, 200
    deg = rng.integers(1, 1000, n)
    exact = rng.random(n) + 0.1
    runs = _runs(rng, N, exact, common_sd=0.0, node_sd=0.05)
    runs[:, 123] += 0.1 * exact[123]  # 28 standard errors at one node
    with pytest.raises(AssertionError):
        unbiased(runs, exact, deg)

"""Pins for the oracle's Algorithm 2 (Randomized Propagation), both subset samplers.

The randomized oracle is pinned to what the paper proves about Algorithm 2 and to exact
distributions: eps = 0 reduces it to Algorithm 1; Lemma 4.1 (unbiased residues and reserves);
Lemma 4.2 (Var[pi_hat(v)] <= L(L+1) eps pi(v) / 2); the expected-cost bound of the proof of
Theorem 4.3 (E[cost] <= (1/eps) sum_{i=1..L} ||r^(i)||_1); the sampled count on a star, which is
exactly Binomial(N, p); and per-neighbour inclusion frequencies p_v across several degree groups.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from tests import _graphs as G


def _graph(seed=3, n=120, m=420):
    n, src, dst = G.random_multigraph(n, m, seed, loops=False)
    return oracle.build_csr(n, src, dst), G.dense_adjacency(n, src, dst)


def _runs(g, a, b, L, w, Y, eps, x, seeds, groups):
    return np.stack([oracle.randomized(g, a, b, L, w, Y, eps, x, s, groups=groups) for s in seeds])


@pytest.mark.parametrize("groups", [False, True])
def test_eps_zero_is_exact(groups):
    g, _ = _graph()
    rng = np.random.default_rng(0)
    x = rng.standard_normal(g.n)
    for a, b in ((0, 1), (0.5, 0.5), (1, 0), (0.3, 0.8)):
        w, Y = oracle.tail_sums(oracle.PPR, 10, 0.2)
        exact = oracle.basic(g, a, b, 10, w, Y, x)
        got = oracle.randomized(g, a, b, 10, w, Y, 0.0, x, 7, groups=groups)
        np.testing.assert_allclose(got, exact, rtol=1e-13, atol=1e-16)


CASES = [
    # (a, b, kind, L, param, eps)
    (0.0, 1.0, oracle.PPR, 8, 0.2, 2e-3),
    (0.5, 0.5, oracle.PPR, 6, 0.1, 1e-3),
    (1.0, 0.0, oracle.HKPR, 6, 3.0, 2e-3),
]


@pytest.mark.parametrize("groups", [False, True])
@pytest.mark.parametrize("case", CASES)
def test_unbiased_variance_and_cost(case, groups):
    a, b, kind, L, param, eps = case
    g, A = _graph()
    nz = np.flatnonzero(g.deg > 0)
    x = np.zeros(g.n)
    x[nz[:3]] = [0.5, 0.3, 0.2]
    w, Y = oracle.tail_sums(kind, L, param)
    exact = oracle.basic(g, a, b, L, w, Y, x)
    N = 600
    runs = []
    costs = []
    for s in range(N):
        pi, st = oracle.randomized(g, a, b, L, w, Y, eps, x, 1000 + s, groups=groups, stats=True)
        runs.append(pi)
        costs.append(sum(int(t[0] + t[2]) for t in st))
    runs = np.stack(runs)
    mean, var = runs.mean(0), runs.var(0, ddof=1)
    # Lemma 4.1: unbiased. z-scores of the mean over N independent runs.
    sd = np.sqrt(var / N)
    live = sd > 0
    z = (mean[live] - exact[live]) / sd[live]
    assert np.mean(np.abs(z) > 2.576) <= 0.01 + 3 * np.sqrt(0.01 * 0.99 / live.sum()) + 1e-9
    assert np.abs(z).max() < 5.5
    # Lemma 4.2: Var <= L(L+1) eps pi / 2 (pi = exact, x >= 0 with ||x||_1 = 1, Y_0 = 1 here)
    bound = L * (L + 1) * eps * exact / 2 * Y[0]
    assert np.all(var <= 1.35 * bound + 1e-18)
    # Theorem 4.3 proof: E[cost] <= (1/eps) sum_{i=1..L} ||r^(i)||_1, r^(i) = (Y_i/Y_0) P^i x
    d = A.sum(1)
    with np.errstate(divide="ignore"):
        da = np.where(d > 0, d ** (-a), 0.0)
        db = np.where(d > 0, d ** (-b), 0.0)
    P = da[:, None] * A * db[None, :]
    v, rsum = x.copy(), 0.0
    for i in range(1, L + 1):
        v = P @ v
        rsum += Y[i] / Y[0] * v.sum()
    cbound = rsum / eps
    assert np.mean(costs) <= cbound * (1 + 3 / np.sqrt(N))


@pytest.mark.parametrize("groups", [False, True])
def test_star_sample_count_is_binomial(groups):
    """Star K_{1,N}, a=0, one level: the number of sampled leaves is Binomial(N, p) exactly."""
    leaves = 200
    n, src, dst = G.star(leaves)
    g = oracle.build_csr(n, src, dst)
    x = np.zeros(n); x[0] = 1.0
    w, Y = oracle.tail_sums(oracle.TRANSITION, 1)        # w_1 = 1: pi = r^(1)
    eps = 1.0 / (leaves * 0.07)                          # p = (1/leaves)/eps = 0.07
    p = (1.0 / leaves) / eps
    counts = []
    for s in range(3000):
        pi = oracle.randomized(g, 0, 1, 1, w, Y, eps, x, s, groups=groups)
        k = pi[1:] / eps
        assert np.allclose(k, np.round(k)) and set(np.unique(np.round(k))) <= {0.0, 1.0}
        counts.append(int(round(k.sum())))
    counts = np.array(counts)
    # chi-square goodness of fit against Binomial(leaves, p), bins pooled to expected >= 5
    ks = np.arange(leaves + 1)
    pmf = stats.binom.pmf(ks, leaves, p)
    obs = np.bincount(counts, minlength=leaves + 1).astype(float)
    exp = pmf * counts.size
    lo, hi = np.searchsorted(np.cumsum(exp), 5), leaves - np.searchsorted(np.cumsum(exp[::-1]), 5)
    o = np.concatenate([[obs[:lo].sum()], obs[lo:hi], [obs[hi:].sum()]])
    e = np.concatenate([[exp[:lo].sum()], exp[lo:hi], [exp[hi:].sum()]])
    chi2 = ((o - e) ** 2 / e).sum()
    assert stats.chi2.sf(chi2, o.size - 1) > 1e-3


@pytest.mark.parametrize("groups", [False, True])
@pytest.mark.parametrize("a", [0.5, 1.0])
def test_inclusion_frequency_per_neighbour(groups, a):
    """Centre whose neighbours span degree groups: neighbour v is reached w.p. min(1, inc/eps)."""
    degrees = [1, 2, 3, 5, 8, 9, 15, 17, 30, 33, 60, 64, 100]
    n, src, dst = G.graded_fan(degrees)
    g = oracle.build_csr(n, src, dst)
    x = np.zeros(n); x[0] = 1.0
    w, Y = oracle.tail_sums(oracle.TRANSITION, 1)
    dc = len(degrees)
    eps = 1.0 / 3.0 ** a                                 # neighbours of degree <= 3 are pushed
    hubs = np.arange(1, dc + 1)
    inc = 1.0 / g.deg[hubs].astype(float) ** a           # b = 0, r(centre) = 1: inc = 1 / d_v^a
    p = np.minimum(1.0, inc / eps)
    N = 4000
    hits = np.zeros(dc)
    for s in range(N):
        pi = oracle.randomized(g, a, 0, 1, w, Y, eps, x, s, groups=groups)
        det = inc >= eps
        np.testing.assert_allclose(pi[hubs][det], inc[det], rtol=1e-14)
        hits += (pi[hubs] > 0)
    freq = hits / N
    samp = p < 1
    z = (freq[samp] - p[samp]) / np.sqrt(p[samp] * (1 - p[samp]) / N)
    assert np.abs(z).max() < 4.0
    assert np.all(freq[~samp] == 1.0)


@pytest.mark.parametrize("groups", [False, True])
def test_directed_unbiased(groups):
    """Lemma 4.1 carries over to the directed propagation (Section 4, "Propagation on directed
    graph"): on a directed graph with sinks, PPR with a = 0, b = 1 is unbiased over 600 runs."""
    n, src, dst = G.random_multigraph(120, 300, 5, loops=False)
    g = oracle.build_csr(n, src, dst, directed=True)
    assert np.any(g.deg == 0)
    nz = np.flatnonzero(g.deg > 0)
    x = np.zeros(n)
    x[nz[:3]] = [0.5, 0.3, 0.2]
    w, Y = oracle.tail_sums(oracle.PPR, 8, 0.2)
    exact = oracle.basic(g, 0.0, 1.0, 8, w, Y, x)
    np.testing.assert_allclose(exact, G.dense_directed_propagation(G.dense_directed_adjacency(n, src, dst), 0, 1, w, x),
                               rtol=1e-12, atol=1e-16)
    N = 600
    runs = _runs(g, 0.0, 1.0, 8, w, Y, 2e-3, x, range(2000, 2000 + N), groups)
    mean, sd = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(N)
    # a source whose mass rarely comes back has an almost deterministic estimate: its standard
    # error can fall below FP64 rounding of the mean, so the z-test uses a rounding floor
    sd = np.maximum(sd, 1e-13 * np.abs(exact))
    live = sd > 0
    z = (mean[live] - exact[live]) / sd[live]
    assert np.mean(np.abs(z) > 2.576) <= 0.01 + 3 * np.sqrt(0.01 * 0.99 / live.sum()) + 1e-9
    assert np.abs(z).max() < 5.5

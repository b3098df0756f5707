"""Pins for the oracle's CSR builder, tail sums and Algorithm 1 (exact propagation).

Everything here runs on the CPU. Each check compares the oracle with something that is not the
oracle: known-answer vectors, brute-force set logic, dense matrix powers, closed forms on regular
graphs, linear solves, the paper's Figure 1 example and the mass invariant of a column-stochastic
propagation matrix.
"""
import math
import os

import numpy as np
import pytest

import oracle
from tests import _graphs as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox known answers
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(t, 16) for t in r]
        out = oracle.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


# ---------------------------------------------------------------- CSR builder
def _csr_by_sets(n, src, dst, loops):
    nb = [set() for _ in range(n)]
    for s, d in zip(src.tolist(), dst.tolist()):
        if s != d:
            nb[s].add(d)
            nb[d].add(s)
    if loops:
        for u in range(n):
            nb[u].add(u)
    deg = np.array([len(s) for s in nb], np.int32)
    rows = [sorted(s, key=lambda v: (deg[v], v)) for s in nb]
    return deg, rows


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("loops", [False, True])
def test_csr_matches_set_construction(seed, loops):
    n, src, dst = G.random_multigraph(60, 150, seed)
    g = oracle.build_csr(n, src, dst, add_self_loops=loops)
    deg, rows = _csr_by_sets(n, src, dst, loops)
    np.testing.assert_array_equal(g.deg, deg)
    assert g.rowptr[0] == 0 and np.all(np.diff(g.rowptr) == deg)
    for u in range(n):
        assert g.colidx[g.rowptr[u]:g.rowptr[u + 1]].tolist() == rows[u]


def test_csr_rows_sorted_and_symmetric():
    n, src, dst = G.random_multigraph(300, 2000, 7)
    g = oracle.build_csr(n, src, dst)
    for u in range(n):
        row = g.colidx[g.rowptr[u]:g.rowptr[u + 1]]
        keys = [(g.deg[v], v) for v in row]
        assert keys == sorted(keys) and len(set(row.tolist())) == row.size and u not in row
        for v in row:
            rv = g.colidx[g.rowptr[v]:g.rowptr[v + 1]]
            assert u in rv


def test_csr_empty_and_isolated():
    g = oracle.build_csr(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.nnz == 0 and g.deg.tolist() == [0] * 5
    g = oracle.build_csr(3, np.array([1], np.int32), np.array([1], np.int32))  # only a self-loop
    assert g.nnz == 0
    g = oracle.build_csr(3, np.array([0], np.int32), np.array([2], np.int32), add_self_loops=True)
    assert g.deg.tolist() == [2, 1, 2]


def test_csr_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.build_csr(3, np.array([0], np.int32), np.array([3], np.int32))


# ---------------------------------------------------------------- tail sums (Def. 3.1)
def test_tail_sums_closed_forms():
    L = 12
    w, Y = oracle.tail_sums(oracle.PPR, L, 0.2)
    np.testing.assert_allclose(w, 0.2 * 0.8 ** np.arange(L + 1), rtol=1e-15)
    np.testing.assert_allclose(Y, 0.8 ** np.arange(L + 2), rtol=1e-15)
    # HKPR: Y_0 = 1 (Poisson pmf sums to 1) and Y_i = 1 - P(N < i) for N ~ Poisson(t)
    t = 5.0
    w, Y = oracle.tail_sums(oracle.HKPR, 30, t)
    pmf = np.array([math.exp(-t) * t ** k / math.factorial(k) for k in range(31)])
    np.testing.assert_allclose(w, pmf, rtol=1e-12)
    assert abs(Y[0] - 1.0) < 1e-14
    cdf_lt = np.concatenate([[0.0], np.cumsum(pmf)])
    for i in range(0, 8):  # where 1 - cdf has no cancellation problem
        assert abs(Y[i] - (1.0 - cdf_lt[i])) < 1e-14
    # deep tail is positive, decreasing and matches the next-term dominated estimate
    assert np.all(np.diff(Y) < 0) and Y[31] > 0
    assert abs(Y[30] / pmf[30] - 1.0) < 0.25
    # Katz: Y_i = beta^i / (1 - beta)
    w, Y = oracle.tail_sums(oracle.KATZ, 10, 0.3)
    np.testing.assert_allclose(Y, 0.3 ** np.arange(12) / 0.7, rtol=1e-15)
    # transition: w_L = 1
    w, Y = oracle.tail_sums(oracle.TRANSITION, 4)
    assert w.tolist() == [0, 0, 0, 0, 1] and Y.tolist() == [1, 1, 1, 1, 1, 0]
    # finite list
    w, Y = oracle.tail_sums(oracle.FINITE, 3, w=[0.5, 0.25, 0.0, 0.25])
    assert Y.tolist() == [1.0, 0.5, 0.25, 0.25, 0.0]


# ---------------------------------------------------------------- Algorithm 1 vs brute force
@pytest.mark.parametrize("seed", range(6))
def test_basic_matches_dense_matrix_powers(seed):
    rng = np.random.default_rng(100 + seed)
    n, src, dst = G.random_multigraph(40, 90, seed)
    loops = bool(seed % 2)
    g = oracle.build_csr(n, src, dst, add_self_loops=loops)
    A = G.dense_adjacency(n, src, dst, loops)
    a, b = rng.random(), rng.random()
    L = int(rng.integers(1, 9))
    w = rng.random(L + 1)
    x = rng.standard_normal(n)
    x[rng.random(n) < 0.5] = 0.0
    wl, Y = oracle.tail_sums(oracle.FINITE, L, w=w)
    got = oracle.basic(g, a, b, L, wl, Y, x)
    want = G.dense_propagation(A, a, b, w, x)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


def test_basic_weight_rescaling_is_invisible():
    """Section 3: propagating w/sum(w) and rescaling gives the same vector as w itself."""
    n, src, dst = G.random_multigraph(30, 70, 11)
    g = oracle.build_csr(n, src, dst)
    x = np.zeros(n); x[3] = 1.0
    w = np.array([0.3, 0.9, 0.0, 2.0])
    wl, Y = oracle.tail_sums(oracle.FINITE, 3, w=w)
    got = oracle.basic(g, 0.5, 0.5, 3, wl, Y, x)
    want = G.dense_propagation(G.dense_adjacency(n, src, dst), 0.5, 0.5, w, x)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- closed forms
def test_complete_graph_closed_forms():
    n, s = 9, 4
    g = oracle.build_csr(*G.complete(n))
    e = np.zeros(n); e[s] = 1.0
    # L-hop transition: P^L e_s = 1/n + (-1/(n-1))^L (e_s - 1/n)
    for L in (1, 2, 5):
        w, Y = oracle.tail_sums(oracle.TRANSITION, L)
        want = 1.0 / n + (-1.0 / (n - 1)) ** L * (e - 1.0 / n)
        np.testing.assert_allclose(oracle.basic(g, 0, 1, L, w, Y, e), want, rtol=1e-13)
    # PPR truncated at L: 1/n * (1-(1-alpha)^{L+1}) + alpha (1-q^{L+1})/(1-q) (e_s - 1/n), q = -(1-alpha)/(n-1)
    alpha, L = 0.2, 20
    w, Y = oracle.tail_sums(oracle.PPR, L, alpha)
    q = -(1 - alpha) / (n - 1)
    want = (1 - (1 - alpha) ** (L + 1)) / n + alpha * (1 - q ** (L + 1)) / (1 - q) * (e - 1.0 / n)
    np.testing.assert_allclose(oracle.basic(g, 0, 1, L, w, Y, e), want, rtol=1e-13)
    # HKPR, infinite sum (L large): 1/n + exp(-t n/(n-1)) (e_s - 1/n)
    t = 3.0
    w, Y = oracle.tail_sums(oracle.HKPR, 60, t)
    want = 1.0 / n + math.exp(-t * n / (n - 1)) * (e - 1.0 / n)
    np.testing.assert_allclose(oracle.basic(g, 0, 1, 60, w, Y, e), want, rtol=1e-12)
    # on a regular graph D^-1/2 A D^-1/2 = D^-1 A = A D^-1 (SGC / single-target PPR forms)
    for a, b in ((0.5, 0.5), (1.0, 0.0)):
        np.testing.assert_allclose(oracle.basic(g, a, b, 60, w, Y, e), want, rtol=1e-12)


def test_cycle_ppr_closed_form():
    n, alpha = 11, 0.2
    g = oracle.build_csr(*G.cycle(n))
    e = np.zeros(n); e[0] = 1.0
    L = 200  # (1-alpha)^{L+1} < 1e-19
    w, Y = oracle.tail_sums(oracle.PPR, L, alpha)
    got = oracle.basic(g, 0, 1, L, w, Y, e)
    rho = (1 - math.sqrt(1 - (1 - alpha) ** 2)) / (1 - alpha)
    Cc = math.sqrt(alpha / (2 - alpha))
    j = np.arange(n)
    closed = Cc * (rho ** j + rho ** (n - j)) / (1 - rho ** n)
    np.testing.assert_allclose(got, closed, rtol=1e-12)
    # and the DFT form of the same circulant inverse
    k = np.arange(n)
    dft = np.array([(alpha / n) * np.sum(np.cos(2 * np.pi * k * jj / n) / (1 - (1 - alpha) * np.cos(2 * np.pi * k / n))) for jj in j])
    np.testing.assert_allclose(got, dft, rtol=1e-12)


def test_cycle_transition_binomial_fold():
    n, L = 7, 9
    g = oracle.build_csr(*G.cycle(n))
    e = np.zeros(n); e[0] = 1.0
    w, Y = oracle.tail_sums(oracle.TRANSITION, L)
    want = np.zeros(n)
    for k in range(L + 1):
        want[(2 * k - L) % n] += math.comb(L, k) / 2 ** L
    np.testing.assert_allclose(oracle.basic(g, 0, 1, L, w, Y, e), want, rtol=1e-14)


def test_ppr_linear_solve():
    """PPR fixed point pi = alpha (I - (1-alpha) A D^-1)^-1 x (Section 2, PageRank definition)."""
    n, src, dst = G.random_multigraph(50, 160, 5, loops=False)
    g = oracle.build_csr(n, src, dst)
    A = G.dense_adjacency(n, src, dst)
    keep = A.sum(1) > 0
    alpha = 0.25
    x = np.where(keep, np.random.default_rng(1).random(n), 0.0)
    x /= x.sum()
    d = A.sum(1)
    P = A / np.where(d > 0, d, 1.0)[None, :]
    want = alpha * np.linalg.solve(np.eye(n) - (1 - alpha) * P, x)
    L = 150
    w, Y = oracle.tail_sums(oracle.PPR, L, alpha)
    np.testing.assert_allclose(oracle.basic(g, 0, 1, L, w, Y, x), want, rtol=1e-12, atol=1e-16)


def test_katz_linear_solve_and_lambda():
    """Katz: sum beta^i A^i e_s = (I - beta A)^-1 e_s for beta < 1/lambda_1 (Table 1)."""
    n, src, dst = G.random_multigraph(40, 100, 9, loops=False)
    g = oracle.build_csr(n, src, dst)
    A = G.dense_adjacency(n, src, dst)
    lam_np = np.linalg.eigvalsh(A).max()
    lam = oracle.power_lambda(g, iters=5000, tol=1e-15)
    assert abs(lam - lam_np) < 1e-9 * lam_np
    beta = 0.5 / lam_np
    L = 80  # (beta lambda)^{L+1} / (1 - beta lambda) < 1e-24
    w, Y = oracle.tail_sums(oracle.KATZ, L, beta)
    s = int(np.argmax(A.sum(1)))
    e = np.zeros(n); e[s] = 1.0
    want = np.linalg.solve(np.eye(n) - beta * A, e)
    np.testing.assert_allclose(oracle.basic(g, 0, 0, L, w, Y, e), want, rtol=1e-12)


def test_figure1_two_step_transition():
    golden = {l.split()[0]: float(l.split()[1]) for l in open(os.path.join(GOLDEN, "fig1_toy_graph.txt"))
              if l.strip() and not l.startswith("#")}
    k = 25
    n, src, dst = G.fig1(k)
    g = oracle.build_csr(n, src, dst)
    e = np.zeros(n); e[0] = 1.0
    w, Y = oracle.tail_sums(oracle.TRANSITION, 2)
    pi = oracle.basic(g, 0, 1, 2, w, Y, e)
    assert abs(pi[0] - golden["s"]) < 1e-15 and abs(pi[1] - golden["v"]) < 1e-15
    assert np.all(pi[2:] == golden["u"])


def test_mass_invariant_column_stochastic():
    """a=0, b=1, no isolated node: ||r^(i)||_1 = Y_i ||x||_1 and sum pi = sum_{i<=L} w_i ||x||_1."""
    n, src, dst = G.random_multigraph(80, 300, 21, loops=False)
    g = oracle.build_csr(n, src, dst)
    keep = g.deg > 0
    x = np.where(keep, np.random.default_rng(2).random(n), 0.0)
    w, Y = oracle.tail_sums(oracle.HKPR, 15, 4.0)
    pi = oracle.basic(g, 0, 1, 15, w, Y, x)
    assert abs(pi.sum() - w.sum() * x.sum()) < 1e-12 * x.sum()


def test_signed_signal_is_linear():
    n, src, dst = G.random_multigraph(30, 80, 4)
    g = oracle.build_csr(n, src, dst)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n)
    w, Y = oracle.tail_sums(oracle.PPR, 8, 0.1)
    whole = oracle.basic(g, 0.5, 0.5, 8, w, Y, x)
    plus = oracle.basic(g, 0.5, 0.5, 8, w, Y, np.maximum(x, 0))
    minus = oracle.basic(g, 0.5, 0.5, 8, w, Y, np.maximum(-x, 0))
    np.testing.assert_allclose(whole, plus - minus, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- directed graphs
# Section 4, "Propagation on directed graph": pi = sum_i w_i (D^-a A^T D^-b)^i x with D the
# out-degree matrix, for PageRank, PPR, HKPR and Katz. A push goes from u to its out-neighbours.
def _directed_by_sets(n, src, dst, loops):
    out = [set() for _ in range(n)]
    for s, d in zip(src.tolist(), dst.tolist()):
        if s != d:
            out[s].add(d)
    if loops:
        for u in range(n):
            out[u].add(u)
    deg = np.array([len(s) for s in out], np.int32)
    rows = [sorted(s, key=lambda v: (deg[v], v)) for s in out]
    return deg, rows


@pytest.mark.parametrize("seed", [1, 2])
@pytest.mark.parametrize("loops", [False, True])
def test_directed_csr_matches_set_construction(seed, loops):
    n, src, dst = G.random_multigraph(60, 150, seed)
    g = oracle.build_csr(n, src, dst, add_self_loops=loops, directed=True)
    deg, rows = _directed_by_sets(n, src, dst, loops)
    np.testing.assert_array_equal(g.deg, deg)
    assert g.rowptr[0] == 0 and np.all(np.diff(g.rowptr) == deg)
    for u in range(n):
        assert g.colidx[g.rowptr[u]:g.rowptr[u + 1]].tolist() == rows[u]


@pytest.mark.parametrize("seed", range(6))
def test_directed_basic_matches_dense_matrix_powers(seed):
    """Random directed multigraphs with sinks (out-degree 0): a = 0 (the presets) or a random a,
    random b, weights and signed signal, against dense powers of D^-a A^T D^-b."""
    rng = np.random.default_rng(300 + seed)
    n, src, dst = G.random_multigraph(40, 70, seed)
    loops = bool(seed % 2)
    g = oracle.build_csr(n, src, dst, add_self_loops=loops, directed=True)
    if not loops:
        assert np.any(g.deg == 0)  # sinks present
    A = G.dense_directed_adjacency(n, src, dst, loops)
    a = 0.0 if seed < 3 else rng.random()
    b = rng.random()
    L = int(rng.integers(1, 9))
    w = rng.random(L + 1)
    x = rng.standard_normal(n)
    x[rng.random(n) < 0.5] = 0.0
    wl, Y = oracle.tail_sums(oracle.FINITE, L, w=w)
    got = oracle.basic(g, a, b, L, wl, Y, x)
    want = G.dense_directed_propagation(A, a, b, w, x)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


def _directed_cycle(n):
    src = np.arange(n, dtype=np.int32)
    return src, ((src + 1) % n).astype(np.int32)


def test_directed_cycle_transition_is_a_shift():
    """On the directed cycle 0 -> 1 -> ... -> n-1 -> 0 every node has out-degree 1, so
    A^T D^-1 moves all mass one step forward: the L-step transition vector is e_{s+L mod n}."""
    n, s = 7, 2
    src, dst = _directed_cycle(n)
    g = oracle.build_csr(n, src, dst, directed=True)
    for L in (1, 5, 9):
        w, Y = oracle.tail_sums(oracle.TRANSITION, L)
        x = np.zeros(n); x[s] = 1.0
        pi = oracle.basic(g, 0, 1, L, w, Y, x)
        want = np.zeros(n); want[(s + L) % n] = 1.0
        np.testing.assert_allclose(pi, want, atol=1e-15)


def test_directed_cycle_ppr_closed_form():
    """PPR on the directed cycle: the walk sits at s+i mod n after i steps, so the truncated PPR
    is pi(v) = sum over i <= L with s+i = v (mod n) of alpha (1-alpha)^i."""
    n, s, alpha, L = 5, 1, 0.15, 23
    src, dst = _directed_cycle(n)
    g = oracle.build_csr(n, src, dst, directed=True)
    w, Y = oracle.tail_sums(oracle.PPR, L, alpha)
    x = np.zeros(n); x[s] = 1.0
    pi = oracle.basic(g, 0, 1, L, w, Y, x)
    want = np.zeros(n)
    for i in range(L + 1):
        want[(s + i) % n] += alpha * (1 - alpha) ** i
    np.testing.assert_allclose(pi, want, rtol=1e-13)


def test_directed_mass_invariant_and_sink_loss():
    """a = 0, b = 1: A^T D^-1 is column stochastic on nodes with out-edges. On a strongly connected
    graph (a cycle plus chords) sum pi = sum_{i<=L} w_i. A sink keeps what reaches it as reserve
    and passes nothing on (D^-1 := 0), so the total falls short by exactly the dense prediction."""
    n = 50
    rng = np.random.default_rng(9)
    cs, cd = _directed_cycle(n)
    ch_s = rng.integers(0, n, 120).astype(np.int32)
    ch_d = rng.integers(0, n, 120).astype(np.int32)
    src, dst = np.concatenate([cs, ch_s]), np.concatenate([cd, ch_d])
    g = oracle.build_csr(n, src, dst, directed=True)
    w, Y = oracle.tail_sums(oracle.HKPR, 12, 3.0)
    x = np.zeros(n); x[4] = 1.0
    pi = oracle.basic(g, 0, 1, 12, w, Y, x)
    assert abs(pi.sum() - w.sum()) < 1e-12
    keep = src != 7  # node 7 loses its out-edges and becomes a sink
    g2 = oracle.build_csr(n, src[keep], dst[keep], directed=True)
    assert g2.deg[7] == 0
    pi2 = oracle.basic(g2, 0, 1, 12, w, Y, x)
    want = G.dense_directed_propagation(G.dense_directed_adjacency(n, src[keep], dst[keep]), 0, 1, w, x)
    np.testing.assert_allclose(pi2, want, rtol=1e-12, atol=1e-16)
    assert pi2.sum() < w.sum() - 1e-6


# ---------------------------------------------------------------- local-clustering sweep
def _conductance_by_sets(n, src, dst, S):
    """Phi(S) from the definition on the undirected simple graph of the edge list."""
    E = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist()) if a != b}
    deg = np.zeros(n)
    for a, b in E:
        deg[a] += 1
        deg[b] += 1
    S = set(S)
    vol = sum(deg[v] for v in S)
    cut = sum(1 for a, b in E if (a in S) != (b in S))
    den = min(vol, deg.sum() - vol)
    return cut / den if den > 0 else np.inf


def test_sweep_finds_the_clique_of_a_barbell():
    """Two K_6 joined by one edge, HKPR from a node of the first clique: the sweep stops at that
    clique, whose conductance is 1 / (6*5 + 1) (one cut edge, volume 31 on either side)."""
    k = 6
    src, dst = [], []
    for off in (0, k):
        for i in range(k):
            for j in range(i + 1, k):
                src.append(off + i); dst.append(off + j)
    src.append(0); dst.append(k)
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    g = oracle.build_csr(2 * k, src, dst)
    w, Y = oracle.tail_sums(oracle.HKPR, 30, 3.0)
    x = np.zeros(2 * k); x[2] = 1.0
    pi = oracle.basic(g, 0, 1, 30, w, Y, x)
    size, phi, order = oracle.sweep_conductance(g, pi)
    assert size == k and sorted(order[:k].tolist()) == list(range(k))
    assert abs(phi - 1.0 / (k * (k - 1) + 1)) < 1e-15


@pytest.mark.parametrize("seed", range(4))
def test_sweep_matches_set_conductance(seed):
    """The sweep's order is by pi(v)/d_v (largest first, ties by id) over nodes with pi > 0, and its
    answer is the first prefix of least conductance computed from the definition."""
    n, src, dst = G.random_multigraph(50, 120, seed, loops=False)
    g = oracle.build_csr(n, src, dst)
    w, Y = oracle.tail_sums(oracle.PPR, 6, 0.15)
    x = np.zeros(n); x[int(np.argmax(g.deg))] = 1.0
    pi = oracle.basic(g, 0, 1, 6, w, Y, x)
    size, phi, order = oracle.sweep_conductance(g, pi)
    live = [v for v in range(n) if g.deg[v] > 0 and pi[v] > 0]
    want_order = sorted(live, key=lambda v: (-pi[v] / g.deg[v], v))
    assert order.tolist() == want_order
    phis = [_conductance_by_sets(n, src, dst, want_order[:i]) for i in range(1, min(len(live), n - 1) + 1)]
    best = int(np.argmin(phis))
    assert size == best + 1 and abs(phi - phis[best]) < 1e-12
    # scaling pi does not change the answer
    assert oracle.sweep_conductance(g, 7.5 * pi)[:2] == (size, phi)


# Untransposed adjacency (single-target PPR on a directed graph): r^(i+1)(v) sums over the
# out-neighbours u of v, so u pushes to its in-neighbours; degrees stay out-degrees.
@pytest.mark.parametrize("seed", [1, 2])
def test_untransposed_csr_matches_set_construction(seed):
    n, src, dst = G.random_multigraph(60, 150, seed)
    g = oracle.build_csr(n, src, dst, directed="untransposed")
    inn = [set() for _ in range(n)]
    outdeg = np.zeros(n, np.int32)
    pairs = {(s, d) for s, d in zip(src.tolist(), dst.tolist()) if s != d}
    for s_, d_ in pairs:
        inn[d_].add(s_)
        outdeg[s_] += 1
    np.testing.assert_array_equal(g.deg, outdeg)
    assert np.array_equal(np.diff(g.rowptr), [len(r) for r in inn])
    for u in range(n):
        assert g.colidx[g.rowptr[u]:g.rowptr[u + 1]].tolist() == sorted(inn[u], key=lambda v: (outdeg[v], v))


@pytest.mark.parametrize("seed", range(4))
def test_untransposed_basic_matches_dense_matrix_powers(seed):
    rng = np.random.default_rng(500 + seed)
    n, src, dst = G.random_multigraph(40, 70, seed)
    g = oracle.build_csr(n, src, dst, directed="untransposed")
    A = G.dense_directed_adjacency(n, src, dst)
    a, b = (1.0, 0.0) if seed == 0 else (rng.random(), rng.random())  # seed 0: the preset
    L = int(rng.integers(1, 9))
    w = rng.random(L + 1)
    x = rng.standard_normal(n)
    wl, Y = oracle.tail_sums(oracle.FINITE, L, w=w)
    got = oracle.basic(g, a, b, L, wl, Y, x)
    want = G.dense_directed_propagation(A, a, b, w, x, transposed=False)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


def test_untransposed_cycle_goes_backwards():
    """With the untransposed adjacency the directed cycle carries mass backwards: e_s -> e_{s-L}."""
    n, s = 7, 2
    src, dst = _directed_cycle(n)
    g = oracle.build_csr(n, src, dst, directed="untransposed")
    for L in (1, 4, 10):
        w, Y = oracle.tail_sums(oracle.TRANSITION, L)
        x = np.zeros(n); x[s] = 1.0
        pi = oracle.basic(g, 0, 1, L, w, Y, x)
        want = np.zeros(n); want[(s - L) % n] = 1.0
        np.testing.assert_allclose(pi, want, atol=1e-15)

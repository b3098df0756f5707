"""Dense signals through agp_query_dense against the FP64 oracle.

Table 1's PageRank row propagates the uniform signal x = 1/n (a = 0, b = 1, PPR weights); other
dense signals are split into sign parts (Section 3) exactly as sparse ones. eps = 0 results match
the oracle to relative 1e-5 per entry; eps > 0 keeps the expected total mass (Lemma 4.1).
"""
import numpy as np
import pytest

import oracle
from synth import graphs as SG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def agp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_03058_gb300 as agp
    agp.lib()
    return agp


@pytest.fixture(scope="module")
def graph(agp):
    n = 16384
    u, v = SG.rmat_edges(n, 131072, seed=20210604)
    return n, agp.build_graph(n, u, v), oracle.build_csr(n, u, v)


def _rel(got, want, scale=None):
    ref = np.abs(want) if scale is None else scale
    err = np.abs(np.asarray(got, np.float64) - want)
    assert np.all(err <= REL * ref + 1e-30), f"worst rel {np.max(err / np.maximum(ref, 1e-300)):.3e}"


def test_global_pagerank(agp, graph):
    n, g, og = graph
    L, alpha = 30, 0.15
    X = torch.full((1, n), 1.0 / n, dtype=torch.float32, device="cuda")
    out, _ = agp.query_dense(g, agp.ppr(alpha, L, 0.0), X)
    w, Y = oracle.tail_sums(oracle.PPR, L, alpha)
    want = oracle.basic(og, 0.0, 1.0, L, w, Y, np.full(n, 1.0 / n))
    _rel(out[0].cpu().numpy(), want)
    # the host path (input and output on the host) gives the same numbers
    out_h, _ = agp.query_dense(g, agp.ppr(alpha, L, 0.0), np.full((1, n), 1.0 / n, np.float32))
    _rel(out_h[0], want)


def test_signed_dense_rows_fp32_and_bf16(agp, graph):
    n, g, og = graph
    rng = np.random.default_rng(4)
    Q = 3
    Xf = rng.standard_normal((Q, n + 5)).astype(np.float32)   # ldx > n
    Xf[1, ::3] = 0.0
    Xf[2] = np.abs(Xf[2])                                      # one sign only: a single lane
    wts = np.array([0.05, 0.3, 0.4, 0.25])
    p = agp.finite(wts, 0.5, 0.5, 0.0)
    wl, Y = oracle.tail_sums(oracle.FINITE, 3, w=wts)
    for dtype in (torch.float32, torch.bfloat16):
        Xd = torch.as_tensor(Xf, device="cuda").to(dtype)
        out, _ = agp.query_dense(g, p, Xd[:, :n] if dtype == torch.float32 else Xd)
        xs = Xd.float().cpu().numpy().astype(np.float64)[:, :n]
        for q in range(Q):
            xp, xm = np.maximum(xs[q], 0), np.maximum(-xs[q], 0)
            pp = oracle.basic(og, 0.5, 0.5, 3, wl, Y, xp) if xp.any() else np.zeros(n)
            pm = oracle.basic(og, 0.5, 0.5, 3, wl, Y, xm) if xm.any() else np.zeros(n)
            _rel(out[q].cpu().numpy(), pp - pm, scale=np.abs(pp) + np.abs(pm))


def test_dense_eps_unbiased_mass(agp, graph):
    """eps > 0, 200 seeds of PageRank from x = 1/n: every run's expected total mass is that of the
    exact propagation (Lemma 4.1). It is below sum_{i<=L} w_i on this graph: R-MAT leaves isolated
    nodes, whose share of x is reserved once and never pushed (D^-1 := 0 there)."""
    n, g, og = graph
    N = 200
    L, alpha = 20, 0.15
    X = torch.full((N, n), 1.0 / n, dtype=torch.float32, device="cuda")
    out, _ = agp.query_dense(g, [agp.ppr(alpha, L, 1e-6, seed=k) for k in range(N)], X)
    mass = out.sum(1, dtype=torch.float64).cpu().numpy()
    w, Y = oracle.tail_sums(oracle.PPR, L, alpha)
    want = oracle.basic(og, 0.0, 1.0, L, w, Y, np.full(n, 1.0 / n)).sum()
    assert want < 1.0 - (1 - alpha) ** (L + 1) - 0.01  # the isolated nodes' loss is visible
    assert abs(mass.mean() - want) <= 4.0 * mass.std(ddof=1) / np.sqrt(N) + 1e-6
    assert np.all(np.abs(mass - want) < 0.05)


def test_dense_errors(agp, graph):
    n, g, og = graph
    bad = torch.zeros((1, n), dtype=torch.float32, device="cuda")
    bad[0, 7] = float("nan")
    with pytest.raises(agp.AgpError) as e:
        agp.query_dense(g, agp.ppr(0.2, 5, 0.0), bad)
    assert e.value.code == 1
    with pytest.raises(agp.AgpError):
        agp.query_dense(g, agp.ppr(0.2, 5, 0.0), torch.zeros((1, n - 1), dtype=torch.float32, device="cuda"))
    # zero rows have no lanes and give zero output
    out, _ = agp.query_dense(g, agp.ppr(0.2, 5, 0.0), torch.zeros((2, n), dtype=torch.float32, device="cuda"))
    assert not out.any()

"""The local-clustering sweep (Section 6) on the GPU against the oracle's sweep of the same pi.

Both order the nodes by the FP64 score pi(v)/d_v of the same FP32 pi (ties by id) and evaluate the
conductance of every prefix as a quotient of exact integers, so the order, the per-prefix
conductances and the best prefix are compared exactly. The oracle's sweep is pinned on the CPU
(barbell graph, conductance from the definition).
"""
import numpy as np
import pytest

import oracle
from synth import graphs as SG
from tests import _graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def agp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_03058_gb300 as agp
    agp.lib()
    return agp


def _compare(agp, g, og, pi_row):
    best, phi, order, phis = agp.sweep(g, pi_row)
    pi64 = pi_row.cpu().numpy().astype(np.float64)
    k_o, phi_o, order_o = oracle.sweep_conductance(og, pi64)
    np.testing.assert_array_equal(order.cpu().numpy(), order_o)
    assert best == k_o
    if k_o > 0:
        assert phi == phi_o
    # every prefix's conductance from the definition (exact integers)
    o = order_o
    in_s = np.zeros(og.n, bool)
    vol, cut, two_m = 0, 0, int(og.deg.sum())
    want = []
    for v in o[: min(len(o), og.n - 1)]:
        row = og.colidx[og.rowptr[v]:og.rowptr[v + 1]]
        loops = int((row == v).sum())
        inside = int(in_s[row[row != v]].sum())
        in_s[v] = True
        vol += int(og.deg[v])
        cut += int(og.deg[v]) - loops - 2 * inside
        den = min(vol, two_m - vol)
        want.append(cut / den if den > 0 else np.inf)
    np.testing.assert_array_equal(phis.cpu().numpy(), np.array(want))


def test_sweep_hkpr_rows(agp):
    n = 16384
    u, v = SG.rmat_edges(n, 131072, seed=20210604)
    g = agp.build_graph(n, u, v)
    og = oracle.build_csr(n, u, v)
    srcs = np.flatnonzero(og.deg > 0)[::1500][:6]
    out, _ = agp.query_sources(g, agp.hkpr(5.0, 20, 1e-7, seed=11), srcs)
    for q in range(len(srcs)):
        _compare(agp, g, og, out[q])
    g.destroy()


def test_sweep_barbell_and_loops(agp):
    """Two cliques joined by one edge: the sweep from inside one clique cuts at the bridge. With one
    self-loop per node (the self-looped graph of SGC) the loops count in d_v but never in the cut."""
    n, src, dst = G.barbell(12)
    for loops in (False, True):
        g = agp.build_graph(n, src, dst, add_self_loops=loops)
        og = oracle.build_csr(n, src, dst, add_self_loops=loops)
        out, _ = agp.query_sources(g, agp.hkpr(3.0, 20, 0.0), [1])
        _compare(agp, g, og, out[0])
        best, phi, order, _ = agp.sweep(g, out[0])
        assert best == 12 and set(order.cpu().numpy()[:12].tolist()) == set(range(12))
        g.destroy()


def test_sweep_degenerate(agp):
    n = 50
    u, v = SG.rmat_edges(64, 200, seed=3)
    keep = (u < n) & (v < n)
    g = agp.build_graph(n, u[keep], v[keep])
    og = oracle.build_csr(n, u[keep], v[keep])
    zero = torch.zeros(n, dtype=torch.float32, device="cuda")
    best, phi, order, phis = agp.sweep(g, zero)        # nothing to sweep
    assert best == 0 and np.isnan(phi) and order.numel() == 0
    one = zero.clone()
    one[int(np.flatnonzero(og.deg > 0)[0])] = 1.0      # a single swept node
    _compare(agp, g, og, one)
    ties = torch.as_tensor(og.deg.astype(np.float32), device="cuda")  # equal scores: order by id
    _compare(agp, g, og, ties)
    gd = agp.build_graph(n, u[keep], v[keep], directed=True)
    with pytest.raises(agp.AgpError):
        agp.sweep(gd, zero)
    g.destroy()
    gd.destroy()

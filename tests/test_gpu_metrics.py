"""Approximation-quality measures of the paper's experiments (agp_compare): MaxError and
Precision@k (Section 6, local clustering with HKPR; the appendix's Katz experiments).

Both are compared exactly with the definitions computed on the host: MaxError in FP64 from the same
FP32 inputs, normalised by the degree (0 for d_v = 0) or plain, and Precision@k from the top-k sets
in the order value descending, id ascending, on the FP32 normalised values. The inputs include an
HKPR estimate and its exact propagation on an R-MAT graph (isolated nodes included), ties at zero,
k = 1 and k = 2048.
"""
import numpy as np
import pytest

import oracle
from synth import graphs as SG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def agp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_03058_gb300 as agp
    agp.lib()
    return agp


def _normalised(x, deg):
    if deg is None:
        return x.astype(np.float32)
    d = deg.astype(np.float32)
    return np.where(deg > 0, x.astype(np.float32) / np.where(deg > 0, d, np.float32(1)), np.float32(0)).astype(np.float32)


def _host(est, ref, deg, k):
    if deg is None:
        me = np.abs(est.astype(np.float64) - ref.astype(np.float64)).max()
    else:
        dd = deg.astype(np.float64)
        ne = np.where(deg > 0, est.astype(np.float64) / np.where(deg > 0, dd, 1.0), 0.0)
        nr = np.where(deg > 0, ref.astype(np.float64) / np.where(deg > 0, dd, 1.0), 0.0)
        me = np.abs(ne - nr).max()
    top = lambda v: set(np.lexsort((np.arange(v.size), -np.where(v == 0, 0, v).astype(np.float64)))[:k].tolist())
    prec = len(top(_normalised(est, deg)) & top(_normalised(ref, deg))) / k
    return me, prec


@pytest.mark.parametrize("normalise", [True, False], ids=["normalised", "plain"])
def test_hkpr_estimate_against_exact(agp, normalise):
    n = 16384
    u, v = SG.rmat_edges(n, 131072, seed=20210604)
    g = agp.build_graph(n, u, v)
    og = oracle.build_csr(n, u, v)
    s = int(np.argsort(og.deg)[-50])
    est, _ = agp.query_sources(g, agp.hkpr(5.0, 20, 1e-6, seed=3), [s])
    ref, _ = agp.query_sources(g, agp.hkpr(5.0, 20, 0.0), [s])
    _, _, deg = g.csr()
    e, r = est[0].contiguous(), ref[0].contiguous()
    for k in (1, 50, 2048):
        me, prec = agp.compare(e, r, deg if normalise else None, k=k)
        want_me, want_prec = _host(e.cpu().numpy(), r.cpu().numpy(), og.deg if normalise else None, k)
        assert me == want_me
        assert prec == want_prec
    # an estimate equal to the reference: no error, full precision
    me, prec = agp.compare(r, r, deg if normalise else None, k=50)
    assert me == 0.0 and prec == 1.0
    g.destroy()


def test_ties_and_max_error_only(agp):
    rng = np.random.default_rng(4)
    n = 5000
    ref = np.zeros(n, np.float32)
    ref[rng.choice(n, 300, replace=False)] = rng.random(300).astype(np.float32)
    est = ref.copy()
    est[rng.choice(n, 40, replace=False)] += np.float32(1e-3)
    deg = rng.integers(0, 20, n).astype(np.int32)  # some isolated nodes
    e, r, d = (torch.as_tensor(x, device="cuda") for x in (est, ref, deg))
    for k in (1, 100, 300, 1000):  # k = 1000 reaches into the zeros (ties by id)
        me, prec = agp.compare(e, r, d, k=k)
        want_me, want_prec = _host(est, ref, deg, k)
        assert me == want_me and prec == want_prec
    me, prec = agp.compare(e, r, None)
    assert prec is None and me == np.abs(est.astype(np.float64) - ref.astype(np.float64)).max()

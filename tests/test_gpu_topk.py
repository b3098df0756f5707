"""Sparse output (agp_topk): the k largest entries of each row, ties by ascending node id.

The order is fully defined (value descending, id ascending), so the result is compared bit-exactly
with a sort of the same FP32 rows on the host (numpy lexsort), including rows with many equal entries
(zeros, repeated values), negative values, -0, k = 1, k = n and the largest k.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def agp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_03058_gb300 as agp
    agp.lib()
    return agp


def _host_topk(rows, k):
    vals, ids = [], []
    for r in rows:
        v = np.where(r == 0, np.float32(0), r)  # -0 counts as +0
        order = np.lexsort((np.arange(r.size), -v.astype(np.float64)))[:k]
        vals.append(v[order])
        ids.append(order.astype(np.int32))
    return np.array(vals), np.array(ids)


def _check(agp, rows, k):
    pi = torch.as_tensor(rows, device="cuda")
    val, idx = agp.topk(pi, k)
    wv, wi = _host_topk(rows, k)
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    np.testing.assert_array_equal(val.cpu().numpy(), wv)


def test_topk_random_and_ties(agp):
    rng = np.random.default_rng(0)
    n = 100_000
    rows = rng.random((6, n), dtype=np.float32) * 1e-3
    rows[1, rng.random(n) < 0.97] = 0.0                        # mostly zeros (a sparse pi)
    rows[2] = np.round(rows[2] * 1e5) / 1e5                    # many repeated values
    rows[3] = rng.standard_normal(n).astype(np.float32)        # signed (pi+ - pi-)
    rows[4, :] = 0.0                                           # all equal: ids decide
    rows[4, ::7] = -0.0
    rows[5, 123] = np.float32(np.inf)
    for k in (1, 17, 1000, 2048):
        _check(agp, rows, k)


def test_topk_small_rows_and_limits(agp):
    rng = np.random.default_rng(1)
    rows = rng.random((3, 37), dtype=np.float32)
    rows[1, :20] = rows[1, 20:] [:17].max()  # a tie across the boundary
    for k in (1, 36, 37):
        _check(agp, rows, k)
    pi = torch.as_tensor(rows, device="cuda")
    with pytest.raises(agp.AgpError):
        agp.topk(pi, 38)
    with pytest.raises(agp.AgpError):
        agp.topk(torch.zeros((1, 5000), device="cuda"), 2049)


def test_topk_of_a_propagation(agp):
    """On query output: the top entries of exact PPR rows against the host sort of the same rows."""
    from synth import graphs as SG
    n = 16384
    u, v = SG.rmat_edges(n, 131072, seed=20210604)
    g = agp.build_graph(n, u, v)
    deg = np.bincount(u, minlength=n) + np.bincount(v, minlength=n)
    srcs = np.flatnonzero(deg > 0)[:8]
    out, _ = agp.query_sources(g, agp.ppr(0.2, 10, 1e-6, seed=3), srcs)
    val, idx = agp.topk(out, 100)
    wv, wi = _host_topk(out.cpu().numpy(), 100)
    np.testing.assert_array_equal(idx.cpu().numpy(), wi)
    np.testing.assert_array_equal(val.cpu().numpy(), wv)
    assert np.all(idx.cpu().numpy()[:, 0] == srcs)  # the source holds the largest PPR entry here
    g.destroy()

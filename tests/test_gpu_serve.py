"""Continuous-batching server (agp_serve_*): every result is the same alone and in the mix.

A request's lanes draw their random numbers from (seed, node, level, segment) counters, never from
the batch they share sweeps with, so a result computed in the mix equals the same request run
alone up to FP32 atomic summation order. At eps = 0 that is 1e-5 of the result's largest entry,
and the served results are also checked against the FP64 oracle (relative 1e-5 per entry). At
eps > 0 a different summation order can, rarely, flip one sampling decision (see _same_draws).
"""
import numpy as np
import pytest

import oracle
from synth import graphs as SG
from tests._compare import close, equally_accurate, same_draws

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    g = agp.build_graph(n, u, v)
    og = oracle.build_csr(n, u, v)
    yield n, g, og, u, v
    g.destroy()


def _mixed_requests(agp, og, count, seed):
    rng = np.random.default_rng(seed)
    beta = 0.85 / oracle.power_lambda(og)
    live = np.flatnonzero(og.deg > 0)
    reqs = []
    for k in range(count):
        kind = k % 4
        L = int(rng.integers(5, 21))
        eps = float(rng.choice([1e-5, 1e-6, 1e-7]))
        s = int(rng.choice(live))
        if kind == 0:
            p = agp.ppr(0.2, L, eps, seed=1000 + k)
        elif kind == 1:
            p = agp.katz(beta, L, eps, seed=1000 + k)
        elif kind == 2:
            p = agp.hkpr(5.0, L, eps, seed=1000 + k)
        else:
            p = agp.transition(min(L, 6), eps, seed=1000 + k)
        reqs.append((p, s))
    return reqs


def _exact(agp, p):
    """The same request at eps = 0 (named weight kinds only, as in the mix)."""
    return agp._params(p.a, p.b, p.L, p.kind, p.param, eps=0.0, seed=p.seed)


def test_mix_equals_alone(agp, graph):
    n, g, og, _, _ = graph
    reqs = _mixed_requests(agp, og, 48, 1)
    with agp.Server(g, max_lanes=16) as srv:
        tickets = [srv.submit(p, source=s) for p, s in reqs]
        results = []
        for t in tickets:
            r = srv.wait(t, timeout_us=120_000_000)
            assert r is not None and r.status == 0
            results.append(srv.result_array(r).cpu().numpy())
            srv.release(t)
        st = srv.stats()
        assert st["completed"] >= len(reqs) and st["sweeps"] > 0
    drifted = 0
    for (p, s), got in zip(reqs, results):
        alone, _ = agp.query_sources(g, p, [s])
        want = alone[0].cpu().numpy()
        if close(got, want):
            continue
        # a summation-order flip of one sampling decision: same accuracy against the exact result
        drifted += 1
        exact, _ = agp.query_sources(g, _exact(agp, p), [s])
        assert equally_accurate(got, want, exact[0].cpu().numpy())
    print(f"[drift] served mix vs alone: {drifted} of {len(reqs)} requests differ beyond 1e-5")
    assert drifted <= max(1, len(reqs) // 20)  # at most 5% (measured on GB300: none)


def test_mix_exact_matches_oracle(agp, graph):
    n, g, og, _, _ = graph
    live = np.flatnonzero(og.deg > 0)
    cases = [(agp.ppr(0.2, 12, 0.0), oracle.PPR, 12, 0.2, 0, 1), (agp.hkpr(3.0, 15, 0.0), oracle.HKPR, 15, 3.0, 0, 1),
             (agp.transition(3, 0.0, a=0.5, b=0.5), oracle.TRANSITION, 3, 0.0, 0.5, 0.5)]
    with agp.Server(g, max_lanes=8) as srv:
        tickets = [(srv.submit(p, source=int(live[7 * i])), kind, L, prm, a, b, int(live[7 * i]))
                   for i, (p, kind, L, prm, a, b) in enumerate(cases)]
        for t, kind, L, prm, a, b, s in tickets:
            r = srv.wait(t, timeout_us=60_000_000)
            got = srv.result_array(r).cpu().numpy().astype(np.float64)
            srv.release(t)
            w, Y = oracle.tail_sums(kind, L, prm)
            x = np.zeros(n); x[s] = 1.0
            want = oracle.basic(og, a, b, L, w, Y, x)
            assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-30)


@pytest.mark.parametrize("eps", [0.0, 1e-6])
def test_feature_request_in_mix(agp, graph, eps):
    """A BF16 feature block served among queries equals the same block propagated alone.

    eps = 0: identical up to FP32 summation order (1e-5 of the column's largest entry). eps > 0:
    the random streams are the same, but a different FP32 atomic order can move a residue across
    a sampling threshold by one ulp and flip that decision; the change then propagates through the
    decisions downstream (with geometric skips, a changed probability moves every later trial of that
    node), so the two blocks can drift apart within the estimator's own error. Every column must
    either agree with the block run alone (same_draws) or be as accurate as it against the exact
    propagation."""
    n, g, og, u, v = graph
    X = torch.randn(n, 6, generator=torch.Generator().manual_seed(4)).to(torch.bfloat16).cuda()
    pf = agp._params(0.5, 0.5, 6, agp.W_PPR, 0.1, eps=eps, seed=77)
    reqs = _mixed_requests(agp, og, 12, 2)
    with agp.Server(g, max_lanes=24) as srv:
        ts = [srv.submit(p, source=s) for p, s in reqs[:6]]
        tf = srv.submit(pf, X=X)
        ts += [srv.submit(p, source=s) for p, s in reqs[6:]]
        r = srv.wait(tf, timeout_us=120_000_000)
        assert r.status == 0 and r.cols == 6
        Zs = srv.result_array(r).cpu().numpy().astype(np.float64)
        srv.release(tf)
        for t in ts:
            assert srv.wait(t, timeout_us=120_000_000).status == 0
            srv.release(t)
    Za = agp.feature_propagate(g, pf, X).cpu().numpy().astype(np.float64)
    if eps == 0.0:
        for c in range(6):
            assert close(Zs[:, c], Za[:, c])
        return
    Z0 = agp.feature_propagate(g, agp._params(0.5, 0.5, 6, agp.W_PPR, 0.1, eps=0.0, seed=77), X)
    Z0 = Z0.cpu().numpy().astype(np.float64)
    for c in range(6):
        if not same_draws(Zs[:, c], Za[:, c]):
            assert equally_accurate(Zs[:, c], Za[:, c], Z0[:, c])


def test_cancel_deadline_and_release(agp, graph):
    n, g, og, _, _ = graph
    reqs = _mixed_requests(agp, og, 40, 3)
    with agp.Server(g, max_lanes=2) as srv:
        tickets = [srv.submit(p, source=s) for p, s in reqs]
        late = srv.submit(reqs[0][0], source=reqs[0][1], deadline_us=1)
        srv.cancel(tickets[-1])
        assert srv.wait(tickets[-1], timeout_us=60_000_000).status == 7      # AGP_ECANCELED
        assert srv.wait(late, timeout_us=60_000_000).status == 6             # AGP_ETIMEDOUT
        for t in tickets[:-1]:
            r = srv.wait(t, timeout_us=120_000_000)
            assert r is not None and r.status == 0
            srv.release(t)
        with pytest.raises(agp.AgpError):
            srv.release(10 ** 9)
        with pytest.raises(agp.AgpError):
            srv.submit(reqs[0][0], source=n)  # source outside the graph


def test_fifo_plain_mode_matches(agp, graph):
    """The FIFO-plain baseline draws the same random numbers as a batched call. As in the mix, an
    FP32 summation-order flip of one sampling decision can move a result within the estimator's
    error: at most 5% of the results (at least one) may do so, and those stay as accurate."""
    n, g, og, _, _ = graph
    reqs = _mixed_requests(agp, og, 8, 5)
    drifted = 0
    with agp.Server(g, mode=agp.SERVE_FIFO_PLAIN, results_on_host=True) as srv:
        ts = [srv.submit(p, source=s) for p, s in reqs]
        for (p, s), t in zip(reqs, ts):
            r = srv.wait(t, timeout_us=120_000_000)
            assert r.status == 0 and r.on_host == 1
            got = srv.result_array(r).numpy().copy()
            srv.release(t)
            alone, _ = agp.query_sources(g, p, [s])
            want = alone[0].cpu().numpy()
            if same_draws(got, want):
                continue
            drifted += 1
            exact, _ = agp.query_sources(g, _exact(agp, p), [s])
            assert equally_accurate(got, want, exact[0].cpu().numpy())
    print(f"[drift] FIFO-plain vs alone: {drifted} of {len(reqs)} requests beyond the same-draws bound")
    assert drifted <= max(1, len(reqs) // 20)


@pytest.mark.parametrize("mode", ["batched", "fifo_plain"])
def test_completion_order_next(agp, graph, mode):
    """agp_serve_next reports every finished request once, in completion order, and skips one that
    was released before it was reported; its results equal those of agp_serve_wait."""
    n, g, og, _, _ = graph
    reqs = _mixed_requests(agp, og, 24, 3)
    m = agp.SERVE_BATCHED if mode == "batched" else agp.SERVE_FIFO_PLAIN
    with agp.Server(g, mode=m, max_lanes=8) as srv:
        tickets = [srv.submit(p, source=s) for p, s in reqs]
        # take the first one by its ticket and release it before next() can report it
        first = srv.wait(tickets[0], timeout_us=120_000_000)
        assert first is not None and first.status == 0
        want0 = srv.result_array(first).cpu().numpy().copy()
        srv.release(tickets[0])
        seen, lat = [], []
        while len(seen) < len(tickets) - 1:
            r = srv.next(timeout_us=120_000_000)
            assert r is not None
            tk, res = r
            assert res.status == 0 and tk != tickets[0] and tk not in seen
            seen.append(tk)
            lat.append(res.latency_us)
            got = srv.result_array(res).cpu().numpy()
            again = srv.poll(tk)
            assert again is not None and np.array_equal(srv.result_array(again).cpu().numpy(), got)
            srv.release(tk)
        assert sorted(seen) == sorted(tickets[1:])
        assert srv.next(timeout_us=1000) is None  # nothing left to report
    assert np.isfinite(want0).all() and want0.sum() > 0

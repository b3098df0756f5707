"""The device's level coefficients (Def. 3.1) against the FP64 oracle's tail sums, element by element.

At eps = 0 the output is sum_i w_i P^i x whatever the tail sums Y_i are (they cancel between the
reserve factor w_i/Y_i and the push factor Y_{i+1}/Y_i), so exact-propagation parity cannot see a
wrong Y_i; at eps > 0 the estimator stays unbiased for any positive Y_i. A mistake there would only
change variance and cost. This test therefore reads the table the level kernels use, through
agp_coefficients (the same device routine), and compares it with the oracle:
    keep_i = Y_0 w_i / Y_i,  push_i = Y_{i+1} / Y_i (0 at i = L),  Y_0,
to relative 1e-12 in FP64. The device derives these as ratios (closed forms per Table 1 row, a
downward ratio recurrence for the heat kernel, compensated suffix sums for explicit weights); the
oracle sums the tails as written, so the two share no arithmetic.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def agp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_03058_gb300 as agp
    agp.lib()
    return agp


def _oracle_table(kind, L, param=0.0, w=None):
    wl, Y = oracle.tail_sums(kind, L, param, w)
    keep = np.zeros(L + 1)
    push = np.zeros(L + 1)
    for i in range(L + 1):
        if Y[i] > 0:
            keep[i] = Y[0] * wl[i] / Y[i]
            push[i] = Y[i + 1] / Y[i] if i < L else 0.0
    return keep, push, Y[0]


def _check(agp, params, kind, L, param=0.0, w=None):
    keep, push, y0 = agp.coefficients(params)
    k_o, p_o, y0_o = _oracle_table(kind, L, param, w)
    for name, got, want in (("keep", keep, k_o), ("push", push, p_o)):
        zero = want == 0
        assert np.all(got[zero] == 0), (name, np.flatnonzero(got[zero] != 0))
        rel = np.abs(got[~zero] - want[~zero]) / np.abs(want[~zero])
        assert rel.size == 0 or rel.max() <= REL, (name, int(np.argmax(rel)), rel.max())
    assert abs(y0 - y0_o) <= REL * abs(y0_o)


@pytest.mark.parametrize("t", [0.5, 5.0, 40.0, 200.0])
@pytest.mark.parametrize("L", [1, 10, 30, 63])
def test_hkpr(agp, t, L):
    _check(agp, agp.hkpr(t, L, 1e-7), oracle.HKPR, L, t)


@pytest.mark.parametrize("alpha", [0.01, 0.1, 0.2, 0.5, 1.0])
def test_ppr(agp, alpha):
    for L in (0, 20, 63):
        _check(agp, agp.ppr(alpha, L, 1e-7), oracle.PPR, L, alpha)


@pytest.mark.parametrize("beta", [1e-6, 0.85 / 2151.35, 0.3, 0.99])
def test_katz(agp, beta):
    # beta^i must stay representable in the oracle's FP64 tail (beta = 1e-6 underflows past i ~ 50)
    for L in ((0, 8, 20) if beta < 1e-3 else (0, 8, 20, 63)):
        _check(agp, agp.katz(beta, L, 1e-8), oracle.KATZ, L, beta)


def test_transition(agp):
    for L in (0, 1, 4, 63):
        _check(agp, agp.transition(L, 1e-6), oracle.TRANSITION, L)


def test_finite_weights(agp):
    rng = np.random.default_rng(3)
    cases = [np.array([0.1, 0.0, 0.5, 0.3, 0.25]),        # a zero weight inside
             np.array([0.0, 0.0, 1.0]),                    # zeros first
             np.array([0.4, 0.6, 0.0, 0.0]),               # zero tail: levels 2, 3 get nothing
             np.array([2.0]),                              # L = 0, unnormalised
             rng.exponential(size=64) * 10.0 ** rng.uniform(-12, 3, 64)]  # L = 63, 15 decades
    for w in cases:
        _check(agp, agp.finite(w, 0.5, 0.5, 1e-6), oracle.FINITE, w.size - 1, w=w)


def test_invalid_parameters(agp):
    with pytest.raises(agp.AgpError) as e:
        agp.coefficients(agp.ppr(0.0, 5, 1e-6))
    assert e.value.code == 1
    with pytest.raises(agp.AgpError):
        agp.coefficients(agp.katz(1.0, 5, 1e-6))
    with pytest.raises(agp.AgpError):
        agp.coefficients(agp.finite(np.zeros(4), 0.0, 1.0, 1e-6))

"""The FP32 forms of the push decision c / d^a >= eps agree with its FP64 evaluation.

The kernels decide in FP32 and fall back to FP64 only inside a bracket around eps (lane parameters
eps_up, eps_lo, eps_hi). This checks the two facts that make that exact, with numpy's IEEE FP32
arithmetic (correctly rounded division and square root, as __fdiv_rn and __fsqrt_rn):
  * a = 0: c >= eps_up, with eps_up the smallest float not below eps, equals (double)c >= eps;
  * a in {1, 1/2}: an FP32 quotient at or above eps_hi = eps (1 + 2^-20), or below
    eps_lo = eps (1 - 2^-20), gives the same answer as the FP64 test, because the FP32 quotient
    is within 2 ulp (2^-22 relative) of the exact value.
No device code runs here.
"""
import numpy as np

M = 2.0 ** -20


def eps_up(e):
    f = np.float32(e)
    if float(f) < e:
        f = np.nextafter(f, np.float32(np.inf))
    return f


def fp64_decision(c, d, mode, e):
    cd = c.astype(np.float64)
    dd = d.astype(np.float64)
    q = cd / dd if mode == 1 else cd / np.sqrt(dd)
    return q >= e


def fp32_screen(c, d, mode, e):
    d32 = d.astype(np.float32)
    q = c / d32 if mode == 1 else c / np.sqrt(d32)
    lo, hi = np.float32(e * (1 - M)), np.float32(e * (1 + M))
    return q >= hi, q < lo


def test_a0_threshold_is_exact():
    rng = np.random.default_rng(1)
    for e in np.concatenate([10.0 ** rng.uniform(-12, -1, 200), [1e-8, 1e-7, 0.1, 2.0 ** -30]]):
        f = eps_up(e)
        # floats at and around the boundary, and a random spread
        near = np.array([np.nextafter(f, np.float32(0)), f, np.nextafter(f, np.float32(np.inf))], np.float32)
        c = np.concatenate([near, (e * 10.0 ** rng.uniform(-1, 1, 1000)).astype(np.float32)])
        assert np.array_equal(c >= f, c.astype(np.float64) >= e)


def test_screen_agrees_with_fp64_outside_bracket():
    rng = np.random.default_rng(2)
    for mode in (1, 2):
        for _ in range(40):
            e = 10.0 ** rng.uniform(-12, -2)
            d = rng.integers(1, 1 << 26, 20000).astype(np.int64)
            scale = d.astype(np.float64) if mode == 1 else np.sqrt(d.astype(np.float64))
            # c spread around the boundary c = eps d^a, including within a few ulp of it
            rel = np.concatenate([rng.uniform(-1e-3, 1e-3, 10000), rng.integers(-64, 65, 10000) * 2.0 ** -24])
            c = (e * scale * (1.0 + rel)).astype(np.float32)
            yes, no = fp32_screen(c, d, mode, e)
            truth = fp64_decision(c, d, mode, e)
            assert not np.any(yes & no)
            assert np.all(truth[yes]) and not np.any(truth[no])
            # the bracket is narrow: almost every case of the +-1e-3 spread is decided in FP32
            assert np.mean((yes | no)[:10000]) > 0.99

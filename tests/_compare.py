"""Comparisons of two GPU results computed with the same random draws (no method arithmetic)."""
import numpy as np


def close(a, b, tol=1e-5):
    """Identical up to FP32 summation order: every entry within `tol` of b's largest entry."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    return np.abs(a - b).max() <= tol * scale


def same_draws(a, b, tol=1e-5):
    """eps > 0: both runs draw the same random numbers, but FP32 atomic sums in another order can
    move a residue by one ulp across a sampling threshold and flip that one decision, which moves
    about eps of mass (and what it pushes later). Such flips are rare: at least 99% of the entries
    agree to `tol` of the largest entry and the relative L1 difference stays below 1e-2."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    agree = np.mean(np.abs(a - b) <= tol * scale)
    l1 = np.abs(a - b).sum() / max(np.abs(b).sum(), 1e-30)
    return agree >= 0.99 and l1 <= 1e-2


def equally_accurate(a, b, exact, slack=1.5):
    """eps > 0, when the coupling has drifted: a is as accurate as b against the exact (eps = 0)
    result, in L1. A flipped sampling decision changes one residue by eps, and that residue then
    changes the decisions drawn downstream, so two runs can drift apart within the estimator's own
    error; they remain equally good estimates."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    x = np.asarray(exact, np.float64)
    err_a = np.abs(a - x).sum()
    err_b = np.abs(b - x).sum()
    return err_a <= slack * err_b + 1e-6 * np.abs(x).sum()

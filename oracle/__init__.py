"""FP64 CPU oracle for Approximate Graph Propagation (arXiv:2106.03058).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this package; the CUDA library never does. The arithmetic lives in plain C
(``agp_oracle.c``, FP64); this module compiles it with gcc, loads it with ctypes and adds the
signal handling the paper states around Algorithm 2:

* Section 3, "Assumption on graph signal x": x is split into its non-negative and negative parts,
  each part is propagated separately after normalising it to unit L1 norm, and the parts are
  recombined, pi = ||x+||_1 pi(x+ / ||x+||_1) - ||x-||_1 pi(x- / ||x-||_1).
* Section 3, "Assumptions on w_i": if sum w != 1, propagate with w / sum w and rescale by sum w.
  The C routines only use the scale-free ratios w_i/Y_i and Y_{i+1}/Y_i, so the rescaling is a
  multiplication of their output by Y_0.

Every function of ``agp_oracle.c`` is pinned by tests against closed forms, brute-force matrix
powers, invariants and the paper's statistical lemmas; see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "agp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# weight-sequence kinds of ora_tail_sums (Table 1)
FINITE, PPR, HKPR, KATZ, TRANSITION = 0, 1, 2, 3, 4

_P = np.ctypeslib.ndpointer
_i64p = _P(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = _P(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = _P(dtype=np.uint32, flags="C_CONTIGUOUS")
_f64p = _P(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``agp_oracle.c`` into ``liboracle.so`` next to it (plain gcc, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.ora_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.ora_philox4x32_10.restype = None
        L.ora_build_csr.argtypes = [C.c_int64, C.c_int64, _i32p, _i32p, C.c_int, _i64p, _i32p, _i32p]
        L.ora_build_csr.restype = C.c_int64
        L.ora_build_csr_directed.argtypes = [C.c_int64, C.c_int64, _i32p, _i32p, C.c_int, _i64p, _i32p, _i32p]
        L.ora_build_csr_directed.restype = C.c_int64
        L.ora_build_csr_directed_in.argtypes = [C.c_int64, C.c_int64, _i32p, _i32p, C.c_int, _i64p, _i32p, _i32p]
        L.ora_build_csr_directed_in.restype = C.c_int64
        L.ora_sweep_conductance.argtypes = [C.c_int64, _i64p, _i32p, _i32p, _f64p, _i32p, C.POINTER(C.c_double)]
        L.ora_sweep_conductance.restype = C.c_int64
        L.ora_tail_sums.argtypes = [C.c_int, C.c_int, C.c_double, _f64p, _f64p, _f64p]
        L.ora_tail_sums.restype = C.c_int
        L.ora_basic.argtypes = [C.c_int64, _i64p, _i32p, _i32p, C.c_double, C.c_double, C.c_int,
                                _f64p, _f64p, _f64p, _f64p, _i64p]
        L.ora_basic.restype = C.c_int
        for f in (L.ora_randomized, L.ora_randomized_groups):
            f.argtypes = [C.c_int64, _i64p, _i32p, _i32p, C.c_double, C.c_double, C.c_int,
                          _f64p, _f64p, C.c_double, _f64p, C.c_uint64, _f64p, _i64p]
            f.restype = C.c_int
        L.ora_power_lambda.argtypes = [C.c_int64, _i64p, _i32p, C.c_int, C.c_double]
        L.ora_power_lambda.restype = C.c_double
        _lib = L
    return _lib


def philox4x32_10(counter, key):
    """Philox4x32-10 block for a 4-word counter and a 2-word key (Salmon et al., SC'11)."""
    out = np.zeros(4, np.uint32)
    lib().ora_philox4x32_10(np.asarray(counter, np.uint32), np.asarray(key, np.uint32), out)
    return out


class CSR:
    """Undirected CSR with rows sorted by (neighbour degree, neighbour id)."""

    def __init__(self, n, rowptr, colidx, deg):
        self.n = int(n)
        self.rowptr = rowptr
        self.colidx = colidx
        self.deg = deg

    @property
    def nnz(self):
        return int(self.rowptr[-1])


def build_csr(n, src, dst, add_self_loops=False, directed=False) -> CSR:
    """Section 4 pre-sorting: see ``ora_build_csr``. directed=True (or "transposed"): rows are
    out-neighbours and degrees out-degrees (``ora_build_csr_directed``); directed="untransposed":
    rows are in-neighbours, degrees still out-degrees (``ora_build_csr_directed_in``), so a row's
    length is not its degree there."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    m = src.size
    rowptr = np.zeros(n + 1, np.int64)
    colidx = np.zeros(max(2 * m + (n if add_self_loops else 0), 1), np.int32)
    deg = np.zeros(max(n, 1), np.int32)
    if directed == "untransposed":
        fn = lib().ora_build_csr_directed_in
    elif directed in (True, "transposed"):
        fn = lib().ora_build_csr_directed
    elif not directed:
        fn = lib().ora_build_csr
    else:
        raise ValueError("directed must be False, True, 'transposed' or 'untransposed'")
    nnz = fn(n, m, src, dst, int(bool(add_self_loops)), rowptr, colidx, deg)
    if nnz < 0:
        raise ValueError("ora_build_csr: bad argument")
    return CSR(n, rowptr, colidx[:nnz].copy(), deg[:n].copy())


def tail_sums(kind: int, L: int, param: float = 0.0, w=None):
    """(w[0..L], Y[0..L+1]) for a Table-1 weight sequence, Def. 3.1 tail sums."""
    w_in = np.zeros(L + 1, np.float64) if w is None else np.ascontiguousarray(w, np.float64)
    if w_in.size != L + 1:
        raise ValueError("w must have L+1 entries")
    w_out = np.zeros(L + 1, np.float64)
    Y = np.zeros(L + 2, np.float64)
    if lib().ora_tail_sums(kind, L, float(param), w_in, w_out, Y) != 0:
        raise ValueError("ora_tail_sums: bad argument")
    return w_out, Y


def _split(x):
    x = np.asarray(x, np.float64)
    parts = []
    for sign, part in ((1.0, np.where(x > 0, x, 0.0)), (-1.0, np.where(x < 0, -x, 0.0))):
        s = part.sum()
        if s > 0:
            parts.append((sign, s, np.ascontiguousarray(part / s)))
    return parts


def basic(g: CSR, a, b, L, w, Y, x, frontier_sizes=False):
    """Algorithm 1 on a signed signal x (split, normalised and rescaled as Section 3 states)."""
    out = np.zeros(g.n, np.float64)
    fronts = []
    for sign, scale, xp in _split(x):
        pi = np.zeros(g.n, np.float64)
        fs = np.zeros(L + 1, np.int64)
        lib().ora_basic(g.n, g.rowptr, g.colidx, g.deg, float(a), float(b), int(L),
                        np.ascontiguousarray(w, np.float64), np.ascontiguousarray(Y, np.float64),
                        xp, pi, fs)
        out += sign * scale * Y[0] * pi
        fronts.append(fs)
    return (out, fronts) if frontier_sizes else out


def randomized(g: CSR, a, b, L, w, Y, eps, x, seed, groups=False, stats=False):
    """Algorithm 2 on a signed signal x; the two sign parts use seeds 2*seed and 2*seed+1."""
    out = np.zeros(g.n, np.float64)
    all_stats = []
    fn = lib().ora_randomized_groups if groups else lib().ora_randomized
    for k, (sign, scale, xp) in enumerate(_split(x)):
        pi = np.zeros(g.n, np.float64)
        st = np.zeros(3 + L + 1, np.int64)
        part_seed = (2 * int(seed) + (0 if sign > 0 else 1)) & 0xFFFFFFFFFFFFFFFF
        fn(g.n, g.rowptr, g.colidx, g.deg, float(a), float(b), int(L),
           np.ascontiguousarray(w, np.float64), np.ascontiguousarray(Y, np.float64),
           float(eps), xp, part_seed, pi, st)
        out += sign * scale * Y[0] * pi
        all_stats.append(st)
    return (out, all_stats) if stats else out


def power_lambda(g: CSR, iters=1000, tol=1e-13):
    """lambda_1(A) by FP64 power iteration (for Katz beta = fraction / lambda_1)."""
    return lib().ora_power_lambda(g.n, g.rowptr, g.colidx, int(iters), float(tol))


def sweep_conductance(g: CSR, pi):
    """Local-clustering sweep over pi(v)/d_v (see ``ora_sweep_conductance``):
    returns (best prefix size, its conductance, the swept nodes in order)."""
    pi = np.ascontiguousarray(pi, np.float64)
    order = np.full(max(g.n, 1), -1, np.int32)
    phi = C.c_double(0.0)
    k = lib().ora_sweep_conductance(g.n, g.rowptr, g.colidx, g.deg, pi, order, C.byref(phi))
    swept = order[: g.n]
    return int(k), float(phi.value), swept[swept >= 0].copy()

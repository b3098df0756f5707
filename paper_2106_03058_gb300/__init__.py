"""GB300 library for Approximate Graph Propagation (Wang et al., KDD'21, arXiv:2106.03058).

Thin Python binding of the C ABI declared in ``include/agp.h``: every function below only
marshals arguments (pointers, sizes, flags) and calls the entry point of the same name in
``libagp.so``; every step of the propagation runs in the library's CUDA kernels. PyTorch is used
for device memory and streams only.

If ``libagp.so`` is missing it is built from ``csrc/`` with nvcc; if that is impossible, loading
fails with an error (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

__all__ = [
    "AgpError", "Params", "Stats", "lib", "build_graph", "Graph", "query_batch", "query_sources",
    "feature_propagate", "katz_beta", "coefficients", "query_dense", "DENSE_BF16", "QUERY_TIMES", "SAMPLER_GROUPS", "topk", "sweep", "katz_lambda_noalloc", "threshold", "ppr", "hkpr", "katz", "transition", "finite",
    "W_FINITE", "W_PPR", "W_HKPR", "W_KATZ", "W_TRANSITION", "INPUT_ON_DEVICE", "OUTPUT_ON_DEVICE",
    "PLAIN", "COLLECT_STATS", "PROFILE", "EPS_ABSOLUTE", "KERNELS", "profile_read", "autotune", "Server", "ServeConfig",
    "Request", "Result", "SERVE_BATCHED", "SERVE_FIFO_PLAIN", "REQ_X_ON_DEVICE", "REQ_EPS_ABSOLUTE", "ADMIT_COST", "ADMIT_FIFO", "ADD_SELF_LOOPS", "EDGES_ON_DEVICE", "DIRECTED", "DIRECTED_IN", "MAX_LEVELS",
]

W_FINITE, W_PPR, W_HKPR, W_KATZ, W_TRANSITION = 0, 1, 2, 3, 4
INPUT_ON_DEVICE, OUTPUT_ON_DEVICE, PLAIN, COLLECT_STATS, PROFILE, EPS_ABSOLUTE = 0x1, 0x2, 0x4, 0x8, 0x10, 0x20
DENSE_BF16, QUERY_TIMES, SAMPLER_GROUPS = 0x40, 0x80, 0x100
KERNELS = ("compact", "expand", "push", "sample", "level_end")
ADD_SELF_LOOPS, EDGES_ON_DEVICE, DIRECTED, DIRECTED_IN = 0x1, 0x2, 0x4, 0x8
MAX_LEVELS = 64


class AgpError(RuntimeError):
    def __init__(self, func, code, detail):
        self.code = code
        self.detail = detail
        super().__init__(f"{func}: {_strerror(code)}: {detail}")


class Params(C.Structure):
    """``agp_params_t``: a, b, L, weight kind and parameter, eps, seed (Eq. 1, Algorithm 2)."""
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("L", C.c_int32), ("kind", C.c_int32),
                ("param", C.c_double), ("w", C.POINTER(C.c_double)), ("eps", C.c_double),
                ("seed", C.c_uint64)]


class Stats(C.Structure):
    """``agp_stats_t``: per-query frontier sizes and cost counters."""
    _fields_ = [("frontier", C.c_int64 * MAX_LEVELS), ("det_edge_ops", C.c_int64),
                ("samples_drawn", C.c_int64), ("samples_accepted", C.c_int64),
                ("by_kernel", (C.c_int64 * 4) * 3), ("levels", C.c_int32), ("done_ms", C.c_float)]

    def as_dict(self):
        return {"frontier": list(self.frontier)[: self.levels], "det_edge_ops": self.det_edge_ops,
                "samples_drawn": self.samples_drawn, "samples_accepted": self.samples_accepted,
                "by_kernel": [list(r) for r in self.by_kernel]}


class ServeConfig(C.Structure):
    """``agp_serve_config_t``."""
    _fields_ = [("mode", C.c_int32), ("max_lanes", C.c_int32), ("result_budget", C.c_int64),
                ("results_on_host", C.c_int32), ("admission", C.c_int32)]


class Request(C.Structure):
    """``agp_request_t``: a single-source query (source >= 0) or a BF16 feature block (source = -1)."""
    _fields_ = [("params", Params), ("source", C.c_int32), ("cols", C.c_int32), ("X", C.c_void_p),
                ("ldx", C.c_int64), ("deadline_us", C.c_int64), ("flags", C.c_uint32), ("reserved", C.c_int32)]


class Result(C.Structure):
    """``agp_result_t``."""
    _fields_ = [("status", C.c_int32), ("on_host", C.c_int32), ("pi", C.c_void_p), ("n", C.c_int64),
                ("cols", C.c_int64), ("queue_us", C.c_double), ("latency_us", C.c_double)]


SERVE_BATCHED, SERVE_FIFO_PLAIN, REQ_X_ON_DEVICE, REQ_EPS_ABSOLUTE = 0, 1, 0x1, 0x2
ADMIT_COST, ADMIT_FIFO = 0, 1

_lib = None
_lock = threading.Lock()
_vp, _i32, _i64, _u32, _dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double


def lib():
    """Load ``libagp.so`` (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            L = C.CDLL(path)
            L.agp_strerror.restype = C.c_char_p
            L.agp_strerror.argtypes = [C.c_int]
            L.agp_last_error_detail.restype = C.c_char_p
            L.agp_last_error_detail.argtypes = []
            L.agp_version.restype = C.c_int
            L.agp_build_graph.argtypes = [_i64, _i64, _vp, _vp, _u32, C.c_int, _vp, C.POINTER(_vp)]
            L.agp_graph_info.argtypes = [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp)]
            L.agp_graph_destroy.argtypes = [_vp]
            L.agp_graph_set_memory_budget.argtypes = [_vp, _i64]
            L.agp_query_batch.argtypes = [_vp, C.POINTER(Params), _i32, _i32, _vp, _vp, _vp, _vp, _i64, _u32,
                                          C.POINTER(Stats), _vp]
            L.agp_query.argtypes = [_vp, C.POINTER(Params), _i64, _vp, _vp, _vp, _u32, C.POINTER(Stats), _vp]
            L.agp_feature_propagate.argtypes = [_vp, C.POINTER(Params), _vp, _i64, _i64, _vp, _i64, _u32, _vp]
            L.agp_katz_beta.argtypes = [_vp, _dbl, _i32, _dbl, C.POINTER(_dbl), C.POINTER(_dbl), _vp]
            L.agp_threshold.argtypes = [_vp, _dbl, _dbl, _i64, _vp, _vp, _vp, _vp]
            L.agp_query_dense.argtypes = [_vp, C.POINTER(Params), _i32, _i32, _vp, _i64, _vp, _i64, _u32,
                                          C.POINTER(Stats), _vp]
            L.agp_sweep.argtypes = [_vp, _vp, _vp, _vp, C.POINTER(_i64), C.POINTER(_dbl), C.POINTER(_i64), _vp]
            L.agp_topk.argtypes = [_vp, _i64, _i64, _i32, _i32, _vp, _vp, _i64, _vp]
            L.agp_compare.argtypes = [_vp, _vp, _i64, _vp, _i32, C.POINTER(_dbl), C.POINTER(_dbl), _vp]
            L.agp_coefficients.argtypes = [C.POINTER(Params), _vp, _vp, C.POINTER(_dbl), C.c_int, _vp]
            L.agp_profile_read.argtypes = [_vp, C.POINTER(_dbl), C.POINTER(_i64), C.POINTER(_i64), C.c_int]
            L.agp_graph_set_wave_lanes.argtypes = [_vp, _i32]
            L.agp_katz_lambda_noalloc.argtypes = [_i64, _vp, _vp, _i32, _dbl, C.POINTER(_dbl), _vp]
            L.agp_katz_lambda_noalloc.restype = C.c_int
            L.agp_autotune.argtypes = [_vp, C.POINTER(Params), _i32, _i32, _vp, _vp, _vp, _vp, _i64, _u32, _vp, _i32,
                                       C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_dbl), _vp]
            L.agp_graph_set_group_width.argtypes = [_vp, _i32]
            L.agp_graph_set_column_tile.argtypes = [_vp, _i32]
            L.agp_graph_set_pull_threshold.argtypes = [_vp, _i32]
            L.agp_serve_create.argtypes = [_vp, C.POINTER(ServeConfig), C.POINTER(_vp)]
            L.agp_serve_submit.argtypes = [_vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
            L.agp_serve_poll.argtypes = [_vp, C.c_uint64, C.POINTER(Result)]
            L.agp_serve_wait.argtypes = [_vp, C.c_uint64, _i64, C.POINTER(Result)]
            L.agp_serve_next.argtypes = [_vp, _i64, C.POINTER(C.c_uint64), C.POINTER(Result)]
            L.agp_serve_release.argtypes = [_vp, C.c_uint64]
            L.agp_serve_cancel.argtypes = [_vp, C.c_uint64]
            L.agp_serve_stats.argtypes = [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i32), C.POINTER(_i32)]
            L.agp_serve_destroy.argtypes = [_vp]
            for f in ("agp_serve_create", "agp_serve_submit", "agp_serve_poll", "agp_serve_wait", "agp_serve_next",
                      "agp_serve_release",
                      "agp_serve_cancel", "agp_serve_stats", "agp_serve_destroy"):
                getattr(L, f).restype = C.c_int
            for f in ("agp_build_graph", "agp_graph_info", "agp_graph_destroy", "agp_graph_set_memory_budget",
                      "agp_query_batch", "agp_query", "agp_feature_propagate", "agp_katz_beta", "agp_threshold",
                      "agp_profile_read", "agp_graph_set_wave_lanes", "agp_autotune", "agp_coefficients", "agp_query_dense",
                      "agp_graph_set_group_width", "agp_topk", "agp_compare", "agp_sweep", "agp_graph_set_column_tile",
                      "agp_graph_set_pull_threshold"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


def _strerror(code):
    return lib().agp_strerror(code).decode()


def _check(func, rc):
    if rc != 0:
        raise AgpError(func, rc, lib().agp_last_error_detail().decode())


def _ptr(x):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ---------------------------------------------------------------- parameter presets (Table 1)
def _params(a, b, L, kind, param=0.0, w=None, eps=0.0, seed=0):
    p = Params(float(a), float(b), int(L), int(kind), float(param), None, float(eps), int(seed) & (2**64 - 1))
    if w is not None:
        arr = np.ascontiguousarray(w, np.float64)
        p._w_keep = arr  # keep the host array alive with the struct
        p.w = arr.ctypes.data_as(C.POINTER(C.c_double))
    return p


def ppr(alpha, L, eps, seed=0, a=0.0, b=1.0):
    """Personalized PageRank w_i = alpha (1-alpha)^i (APPNP with a = b = 1/2)."""
    return _params(a, b, L, W_PPR, alpha, eps=eps, seed=seed)


def hkpr(t, L, eps, seed=0, a=0.0, b=1.0):
    """Heat kernel PageRank w_i = e^-t t^i / i! (GDC with a = b = 1/2)."""
    return _params(a, b, L, W_HKPR, t, eps=eps, seed=seed)


def katz(beta, L, eps, seed=0):
    """Katz w_i = beta^i, a = b = 0."""
    return _params(0.0, 0.0, L, W_KATZ, beta, eps=eps, seed=seed)


def transition(L, eps, seed=0, a=0.0, b=1.0):
    """L-hop transition probability (SGC with a = b = 1/2): w_L = 1."""
    return _params(a, b, L, W_TRANSITION, eps=eps, seed=seed)


def finite(w, a, b, eps, seed=0):
    """Explicit weights w_0..w_L."""
    w = np.asarray(w, np.float64)
    return _params(a, b, w.size - 1, W_FINITE, w=w, eps=eps, seed=seed)


# ---------------------------------------------------------------- graph
class Graph:
    """Handle of a device CSR built by ``agp_build_graph``."""

    def __init__(self, handle, n, nnz, device):
        self.handle = handle
        self.n = n
        self.nnz = nnz
        self.device = device

    def destroy(self):
        if self.handle:
            lib().agp_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def set_wave_lanes(self, lanes):
        """``agp_graph_set_wave_lanes`` (0 = automatic)."""
        _check("agp_graph_set_wave_lanes", lib().agp_graph_set_wave_lanes(self.handle, int(lanes)))

    def set_group_width(self, width):
        """``agp_graph_set_group_width`` (0 = automatic; 1, 2 or 4)."""
        _check("agp_graph_set_group_width", lib().agp_graph_set_group_width(self.handle, int(width)))

    def set_pull_threshold(self, shift):
        """``agp_graph_set_pull_threshold``: pull a level when the frontier holds >= n >> shift nodes
        (-1 = never; 62 = always)."""
        _check("agp_graph_set_pull_threshold", lib().agp_graph_set_pull_threshold(self.handle, int(shift)))

    def set_column_tile(self, columns):
        """``agp_graph_set_column_tile`` (0 = automatic; 8, 16 or 32)."""
        _check("agp_graph_set_column_tile", lib().agp_graph_set_column_tile(self.handle, int(columns)))

    def set_memory_budget(self, nbytes):
        _check("agp_graph_set_memory_budget", lib().agp_graph_set_memory_budget(self.handle, int(nbytes)))

    def csr(self):
        """Copies of (rowptr int64[n+1], colidx int32[nnz], deg int32[n]) as CUDA torch tensors."""
        import torch
        n, nnz = _i64(), _i64()
        rp, ci, dg = _vp(), _vp(), _vp()
        _check("agp_graph_info", lib().agp_graph_info(self.handle, C.byref(n), C.byref(nnz), C.byref(rp), C.byref(ci), C.byref(dg)))

        def view(ptr, count, typestr, dtype):
            out = torch.empty(max(count, 0), dtype=dtype, device=f"cuda:{self.device}")
            if count > 0:
                src = _CudaArray(ptr.value, count, typestr)
                out.copy_(torch.as_tensor(src, device=f"cuda:{self.device}"))
            return out

        return (view(rp, n.value + 1, "<i8", torch.int64), view(ci, nnz.value, "<i4", torch.int32),
                view(dg, n.value, "<i4", torch.int32))


class _CudaArray:
    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False), "version": 3}


def build_graph(n, src, dst, add_self_loops=False, device=0, stream=None, directed=False):
    """``agp_build_graph``: src/dst are int32 numpy arrays (host) or CUDA tensors (device).
    directed=True (or "transposed"): edges are src -> dst, rows are out-neighbour lists (AGP_DIRECTED;
    queries need a = 0); directed="untransposed": rows are in-neighbour lists, deg out-degrees
    (AGP_DIRECTED_IN, single-target PPR)."""
    dflag = DIRECTED_IN if directed == "untransposed" else (DIRECTED if directed else 0)
    flags = (ADD_SELF_LOOPS if add_self_loops else 0) | dflag
    on_dev = not isinstance(src, np.ndarray)
    if on_dev:
        flags |= EDGES_ON_DEVICE
    else:
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
    h = _vp()
    m = int(src.shape[0])
    _check("agp_build_graph", lib().agp_build_graph(int(n), m, _ptr(src), _ptr(dst), flags, int(device),
                                                     _stream(stream), C.byref(h)))
    nn, nnz = _i64(), _i64()
    _check("agp_graph_info", lib().agp_graph_info(h, C.byref(nn), C.byref(nnz), None, None, None))
    return Graph(h, nn.value, nnz.value, device)


# ---------------------------------------------------------------- queries
def _params_array(params, Q):
    if isinstance(params, Params):
        arr = (Params * 1)(params)
        return arr, 1, [params]
    params = list(params)
    if len(params) != Q:
        raise ValueError("need one Params or Q of them")
    arr = (Params * Q)(*params)
    return arr, Q, params


def query_batch(g, params, x_off, x_idx, x_val, out, ld_out=None, flags=0, stats=None, stream=None):
    """``agp_query_batch`` with raw arrays (numpy = host, torch CUDA = device)."""
    Q = int(x_off.shape[0]) - 1
    parr, np_, keep = _params_array(params, Q)
    st = (Stats * Q)() if (flags & (COLLECT_STATS | QUERY_TIMES)) and stats is None else stats
    ld = int(ld_out if ld_out is not None else g.n)
    _check("agp_query_batch", lib().agp_query_batch(g.handle, parr, np_, Q, _ptr(x_off), _ptr(x_idx), _ptr(x_val),
                                                     _ptr(out), ld, int(flags), st, _stream(stream)))
    return st


def query_dense(g, params, X, out=None, flags=0, stats=None, stream=None):
    """``agp_query_dense``: X is [Q, >= n] float32 or bfloat16 (numpy on the host, torch CUDA on the
    device); returns (out [Q, n] float32 on X's side, stats)."""
    import torch
    on_dev = torch.is_tensor(X) and X.is_cuda
    Q = int(X.shape[0])
    bf16 = (X.dtype == torch.bfloat16) if torch.is_tensor(X) else False
    if torch.is_tensor(X) and not on_dev:
        X = X.contiguous().numpy() if not bf16 else X.contiguous().view(torch.int16).numpy()
    ldx = int(X.stride(0) if torch.is_tensor(X) else X.strides[0] // X.itemsize)
    if out is None:
        out = (torch.empty((Q, g.n), dtype=torch.float32, device=f"cuda:{g.device}") if on_dev
               else np.zeros((Q, g.n), np.float32))
    ld = int(out.stride(0) if torch.is_tensor(out) else out.strides[0] // 4)
    fl = int(flags) | (INPUT_ON_DEVICE if on_dev else 0) | (DENSE_BF16 if bf16 else 0)
    if torch.is_tensor(out) and out.is_cuda:
        fl |= OUTPUT_ON_DEVICE
    parr, np_, keep = _params_array(params, Q)
    st = (Stats * Q)() if (fl & (COLLECT_STATS | QUERY_TIMES)) and stats is None else stats
    _check("agp_query_dense", lib().agp_query_dense(g.handle, parr, np_, Q, _ptr(X), ldx, _ptr(out), ld, fl, st,
                                                     _stream(stream)))
    return out, st


def autotune(g, params, x_off, x_idx, x_val, out, ld_out=None, flags=INPUT_ON_DEVICE | OUTPUT_ON_DEVICE,
             candidates=None, stream=None):
    """``agp_autotune``: returns (best lanes, best group width, best ms or -1 when taken from the cache)."""
    Q = int(x_off.shape[0]) - 1
    parr, np_, keep = _params_array(params, Q)
    cand = None if candidates is None else (C.c_int32 * len(candidates))(*candidates)
    best, width, ms = _i32(), _i32(), _dbl()
    _check("agp_autotune", lib().agp_autotune(g.handle, parr, np_, Q, _ptr(x_off), _ptr(x_idx), _ptr(x_val), _ptr(out),
                                               int(ld_out if ld_out is not None else g.n), int(flags), cand,
                                               0 if candidates is None else len(candidates), C.byref(best),
                                               C.byref(width), C.byref(ms), _stream(stream)))
    return best.value, width.value, ms.value


class Server:
    """``agp_serve_*``: continuous-batching server over a graph (see include/agp.h)."""

    def __init__(self, g, mode=SERVE_BATCHED, max_lanes=0, result_budget=0, results_on_host=False, admission=ADMIT_COST):
        self.g = g
        cfg = ServeConfig(int(mode), int(max_lanes), int(result_budget), int(bool(results_on_host)), int(admission))
        h = _vp()
        _check("agp_serve_create", lib().agp_serve_create(g.handle, C.byref(cfg), C.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, params, source=None, X=None, deadline_us=0, eps_absolute=False):
        """Queue a query from `source` or a feature block X (CUDA bf16 [n, cols], read in place)."""
        fl = REQ_EPS_ABSOLUTE if eps_absolute else 0
        if source is not None:
            req = Request(params, int(source), 0, None, 0, int(deadline_us), fl, 0)
        else:
            req = Request(params, -1, int(X.shape[1]), X.data_ptr(), int(X.stride(0)), int(deadline_us),
                          REQ_X_ON_DEVICE | fl, 0)
        t = C.c_uint64()
        _check("agp_serve_submit", lib().agp_serve_submit(self.handle, C.byref(req), C.byref(t)))
        if X is not None:
            self._keep[t.value] = X  # the device block must outlive the request
        return t.value

    def poll(self, ticket):
        r = Result()
        rc = lib().agp_serve_poll(self.handle, int(ticket), C.byref(r))
        if rc == 5:  # AGP_EAGAIN
            return None
        _check("agp_serve_poll", rc)
        return r

    def wait(self, ticket, timeout_us=-1):
        r = Result()
        rc = lib().agp_serve_wait(self.handle, int(ticket), int(timeout_us), C.byref(r))
        if rc == 6:  # AGP_ETIMEDOUT
            return None
        _check("agp_serve_wait", rc)
        return r

    def next(self, timeout_us=-1):
        """The next finished request in completion order: (ticket, Result), or None on timeout."""
        r, t = Result(), C.c_uint64()
        rc = lib().agp_serve_next(self.handle, int(timeout_us), C.byref(t), C.byref(r))
        if rc == 6:  # AGP_ETIMEDOUT
            return None
        _check("agp_serve_next", rc)
        return int(t.value), r

    def result_array(self, r):
        """Copy a finished result into a torch tensor ([n] or [n, cols], on its device or the host)."""
        import torch
        count = int(r.n * r.cols)
        if r.on_host:
            buf = (C.c_float * count).from_address(r.pi)
            t = torch.from_numpy(np.ctypeslib.as_array(buf).copy())
        else:
            t = torch.empty(count, dtype=torch.float32, device=f"cuda:{self.g.device}")
            if count:
                t.copy_(torch.as_tensor(_CudaArray(r.pi, count, "<f4"), device=f"cuda:{self.g.device}"))
        return t if r.cols == 1 else t.view(int(r.n), int(r.cols))

    def release(self, ticket):
        _check("agp_serve_release", lib().agp_serve_release(self.handle, int(ticket)))
        self._keep.pop(ticket, None)

    def cancel(self, ticket):
        _check("agp_serve_cancel", lib().agp_serve_cancel(self.handle, int(ticket)))

    def stats(self):
        c, sw = _i64(), _i64()
        a, q = _i32(), _i32()
        _check("agp_serve_stats", lib().agp_serve_stats(self.handle, C.byref(c), C.byref(sw), C.byref(a), C.byref(q)))
        return {"completed": c.value, "sweeps": sw.value, "lanes_active": a.value, "queued": q.value}

    def destroy(self):
        if self.handle:
            lib().agp_serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def profile_read(g, reset=False):
    """``agp_profile_read``: ({kernel: ms}, {kernel: launches}, all kernel launches)."""
    ms = (_dbl * 5)()
    ln = (_i64 * 5)()
    tot = _i64()
    _check("agp_profile_read", lib().agp_profile_read(g.handle, ms, ln, C.byref(tot), int(bool(reset))))
    return dict(zip(KERNELS, list(ms))), dict(zip(KERNELS, list(ln))), tot.value


def query_sources(g, params, sources, out=None, plain=False, collect_stats=False, stream=None, profile=False,
                  sampler_groups=False):
    """One query per source node (x = e_s). Inputs/outputs on the device; returns (out, stats)."""
    import torch
    dev = f"cuda:{g.device}"
    src = torch.as_tensor(np.asarray(sources, np.int32), device=dev) if not torch.is_tensor(sources) else sources.to(dev, torch.int32)
    Q = int(src.numel())
    off = torch.arange(Q + 1, dtype=torch.int64, device=dev)
    if out is None:
        out = torch.empty((Q, g.n), dtype=torch.float32, device=dev)
    flags = (INPUT_ON_DEVICE | OUTPUT_ON_DEVICE | (PLAIN if plain else 0) | (COLLECT_STATS if collect_stats else 0)
             | (PROFILE if profile else 0) | (SAMPLER_GROUPS if sampler_groups else 0))
    st = query_batch(g, params, off, src, None, out, out.stride(0), flags, None, stream)
    return out, st


def feature_propagate(g, params, X, Z=None, plain=False, stream=None, eps_absolute=False):
    """``agp_feature_propagate``: X CUDA bfloat16 [n, d] (row stride X.stride(0)), Z CUDA float32 [n, d]."""
    import torch
    if X.dtype != torch.bfloat16 or not X.is_cuda:
        raise TypeError("X must be a CUDA bfloat16 tensor")
    n, d = X.shape
    if Z is None:
        Z = torch.empty((n, d), dtype=torch.float32, device=X.device)
    _check("agp_feature_propagate", lib().agp_feature_propagate(g.handle, C.byref(params), X.data_ptr(), d, X.stride(0),
                                                                 Z.data_ptr(), Z.stride(0),
                                                                 (PLAIN if plain else 0) | (EPS_ABSOLUTE if eps_absolute else 0),
                                                                 _stream(stream)))
    return Z


def katz_beta(g, fraction=0.85, iters=1000, tol=1e-12, stream=None):
    """``agp_katz_beta``: returns (beta, lambda_1)."""
    beta, lam = _dbl(), _dbl()
    _check("agp_katz_beta", lib().agp_katz_beta(g.handle, float(fraction), int(iters), float(tol), C.byref(beta),
                                                 C.byref(lam), _stream(stream)))
    return beta.value, lam.value


def katz_lambda_noalloc(n, rowptr, colidx, iters=1000, tol=1e-12, stream=None):
    """``agp_katz_lambda_noalloc``: lambda_1 of a caller-owned device CSR (CUDA tensors), no allocation."""
    lam = _dbl()
    _check("agp_katz_lambda_noalloc", lib().agp_katz_lambda_noalloc(int(n), rowptr.data_ptr(), colidx.data_ptr(), int(iters),
                                                                     float(tol), C.byref(lam), _stream(stream)))
    return lam.value


def threshold(g, a, eps, nodes, c, k_out, stream=None):
    """``agp_threshold`` on CUDA tensors nodes (int32), c (float32), k_out (int32)."""
    _check("agp_threshold", lib().agp_threshold(g.handle, float(a), float(eps), int(nodes.numel()), nodes.data_ptr(),
                                                 c.data_ptr(), k_out.data_ptr(), _stream(stream)))
    return k_out


def coefficients(params, device=0, stream=None):
    """``agp_coefficients``: (keep[0..L], push[0..L], Y_0) in FP64 as the device computes them."""
    L = int(params.L)
    keep = np.zeros(L + 1, np.float64)
    push = np.zeros(L + 1, np.float64)
    y0 = _dbl()
    _check("agp_coefficients", lib().agp_coefficients(C.byref(params), keep.ctypes.data, push.ctypes.data, C.byref(y0),
                                                       int(device), _stream(stream)))
    return keep, push, y0.value


def topk(pi, k, stream=None):
    """``agp_topk``: pi CUDA float32 [Q, >= n] (row stride pi.stride(0), n = pi.shape[1]); returns
    (values [Q, k] float32, ids [Q, k] int32) on the device, largest first, ties by ascending id."""
    import torch
    Q, n = int(pi.shape[0]), int(pi.shape[1])
    val = torch.empty((Q, k), dtype=torch.float32, device=pi.device)
    idx = torch.empty((Q, k), dtype=torch.int32, device=pi.device)
    _check("agp_topk", lib().agp_topk(pi.data_ptr(), n, int(pi.stride(0)), Q, int(k), val.data_ptr(), idx.data_ptr(),
                                       k, _stream(stream)))
    return val, idx


def compare(pi_est, pi_ref, deg=None, k=None, stream=None):
    """``agp_compare`` on CUDA float32 n-vectors: returns (MaxError, Precision@k or None). deg: the
    graph's int32 degrees (CUDA) to normalise by d_v, or None for the plain values."""
    n = int(pi_est.numel())
    me, pk = _dbl(), _dbl()
    _check("agp_compare", lib().agp_compare(pi_est.data_ptr(), pi_ref.data_ptr(), n,
                                             deg.data_ptr() if deg is not None else None, int(k or 0), C.byref(me),
                                             C.byref(pk) if k else None, _stream(stream)))
    return me.value, (pk.value if k else None)


def sweep(g, pi, stream=None):
    """``agp_sweep`` on a CUDA float32 row pi [n]: returns (best prefix size, its conductance, the
    swept nodes in order (CUDA int32), Phi of every prefix (CUDA float64))."""
    import torch
    n = g.n
    order = torch.empty(n, dtype=torch.int32, device=pi.device)
    phi = torch.empty(max(n - 1, 1), dtype=torch.float64, device=pi.device)
    best, bphi, swept = _i64(), _dbl(), _i64()
    _check("agp_sweep", lib().agp_sweep(g.handle, pi.data_ptr(), order.data_ptr(), phi.data_ptr(), C.byref(best),
                                         C.byref(bphi), C.byref(swept), _stream(stream)))
    k = swept.value
    return best.value, bphi.value, order[:k], phi[:max(min(k, n - 1), 0)]

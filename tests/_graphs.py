"""Small deterministic test graphs (edge lists) and dense brute-force helpers for the tests."""
import numpy as np


def complete(n):
    u, v = np.triu_indices(n, 1)
    return n, u.astype(np.int32), v.astype(np.int32)


def cycle(n):
    u = np.arange(n, dtype=np.int32)
    return n, u, ((u + 1) % n).astype(np.int32)


def star(leaves):
    """Centre 0 joined to leaves 1..leaves."""
    v = np.arange(1, leaves + 1, dtype=np.int32)
    return leaves + 1, np.zeros(leaves, np.int32), v


def fig1(k):
    """Figure 1: s=0 joined to u_1..u_k (nodes 2..k+1), each u_i joined to v=1."""
    us = np.arange(2, k + 2, dtype=np.int32)
    src = np.concatenate([np.zeros(k, np.int32), us])
    dst = np.concatenate([us, np.ones(k, np.int32)])
    return k + 2, src, dst


def random_multigraph(n, m, seed, loops=True):
    """Random edge list with duplicates, reversed duplicates, self-loops and isolated nodes."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if not loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    # repeat a few edges, both orientations
    k = max(1, m // 10)
    src = np.concatenate([src, dst[:k], src[:k]])
    dst = np.concatenate([dst, src[:k], dst[:k]])
    return n, src, dst


def graded_fan(degrees, seed=0):
    """Centre 0 joined to hubs 1..K; hub j gets (degrees[j]-1) private leaves so deg = degrees[j].

    The centre's neighbours then span several degree groups [2^k, 2^{k+1}).
    """
    K = len(degrees)
    src, dst = [], []
    nxt = K + 1
    for j, d in enumerate(degrees):
        src.append(0); dst.append(j + 1)
        for _ in range(d - 1):
            src.append(j + 1); dst.append(nxt); nxt += 1
    return nxt, np.array(src, np.int32), np.array(dst, np.int32)


def dense_adjacency(n, src, dst, add_self_loops=False):
    A = np.zeros((n, n))
    for s, d in zip(src, dst):
        if s != d:
            A[s, d] = 1.0
            A[d, s] = 1.0
    if add_self_loops:
        A += np.eye(n)
    return A


def dense_propagation(A, a, b, w, x):
    """sum_i w_i (D^-a A D^-b)^i x with dense FP64 matrix powers (D^-p := 0 for d = 0)."""
    d = A.sum(1)
    with np.errstate(divide="ignore"):
        da = np.where(d > 0, d ** (-a), 0.0)
        db = np.where(d > 0, d ** (-b), 0.0)
    M = da[:, None] * A * db[None, :]
    out = np.zeros(A.shape[0])
    v = np.asarray(x, np.float64).copy()
    for i, wi in enumerate(w):
        if i > 0:
            v = M @ v
        out += wi * v
    return out


def dense_directed_adjacency(n, src, dst, add_self_loops=False):
    """A[u, v] = 1 for every directed edge u -> v (repeats merged, input loops dropped)."""
    A = np.zeros((n, n))
    for s, d in zip(src, dst):
        if s != d:
            A[s, d] = 1.0
    if add_self_loops:
        A += np.eye(n)
    return A


def dense_directed_propagation(A, a, b, w, x, transposed=True):
    """sum_i w_i (D^-a Ã D^-b)^i x with D the out-degree matrix, Ã = A^T (transposed, PageRank,
    PPR, HKPR, Katz) or A (single-target PPR); dense FP64 powers; D^0 = I, and D^-p := 0 at
    out-degree 0 for p > 0."""
    d = A.sum(1)
    with np.errstate(divide="ignore"):
        da = np.ones_like(d) if a == 0 else np.where(d > 0, d ** (-a), 0.0)
        db = np.ones_like(d) if b == 0 else np.where(d > 0, d ** (-b), 0.0)
    M = da[:, None] * (A.T if transposed else A) * db[None, :]
    out = np.zeros(A.shape[0])
    v = np.asarray(x, np.float64).copy()
    for i, wi in enumerate(w):
        if i > 0:
            v = M @ v
        out += wi * v
    return out


def barbell(k):
    """Two complete graphs K_k joined by the edge (0, k): nodes 0..k-1 and k..2k-1."""
    src, dst = [], []
    for off in (0, k):
        for i in range(k):
            for j in range(i + 1, k):
                src.append(off + i)
                dst.append(off + j)
    src.append(0)
    dst.append(k)
    return 2 * k, np.array(src, np.int32), np.array(dst, np.int32)

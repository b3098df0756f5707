"""Seeded synthetic graphs shaped like the paper's workloads.

This module only draws inputs: edge lists, sources and feature matrices. It holds none of the
propagation arithmetic, so both the FP64 oracle and the CUDA library can take their inputs from it.

The paper evaluates on social and citation graphs (YouTube, Orkut, Twitter, Friendster, Reddit,
Yelp, Amazon, Papers100M; Section 5, Tables 3 and 4). Those datasets are not available here, so
the generators below stand in for them with the same node counts, edge counts and power-law degree
skew:

* R-MAT (Chakrabarti et al., SDM'04): recursive quadrant choice with probabilities (a, b, c, d).
* Chung-Lu (Chung and Lu, 2002): edge (u, v) drawn with probability proportional to w_u * w_v,
  expected degrees w following a power law with the given exponent, capped at sqrt(sum w).

Every generator returns exactly ``m`` distinct undirected edges without self-loops, as two int32
arrays ``(u, v)`` with ``u < v`` before the random relabelling of node ids. Draws are repeated
until at least ``m`` distinct edges exist; a uniformly random subset of any surplus is dropped.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

__all__ = [
    "rmat_edges",
    "chung_lu_edges",
    "chung_lu_weights",
    "cached",
]


def _distinct_sorted(keys):
    """Sorted distinct values of an int64 array (sort + adjacent compare)."""
    keys = np.sort(keys)
    if keys.size == 0:
        return keys
    keep = np.empty(keys.size, bool)
    keep[0] = True
    np.not_equal(keys[1:], keys[:-1], out=keep[1:])
    return keys[keep]


def _canonical(u, v, n):
    lo = np.minimum(u, v).astype(np.int64)
    hi = np.maximum(u, v).astype(np.int64)
    keep = lo != hi
    return lo[keep] * n + hi[keep]


def _draw_until(m, n, draw, rng):
    """Call ``draw(k)`` -> (u, v) until ``m`` distinct non-loop undirected edges exist.

    If the draws hold more than ``m`` distinct edges, a uniformly random subset of the surplus is
    removed, so the result is exactly ``m`` edges, sorted by (lo, hi).
    """
    keys = np.empty(0, np.int64)
    want = int(m * 1.05) + 1024
    while True:
        u, v = draw(want)
        keys = _distinct_sorted(np.concatenate([keys, _canonical(u, v, n)]))
        if keys.size >= m:
            break
        want = int((m - keys.size) * 1.5) + 1024
    surplus = keys.size - m
    if surplus:
        drop = rng.choice(keys.size, size=surplus, replace=False)
        keep = np.ones(keys.size, bool)
        keep[drop] = False
        keys = keys[keep]
    return keys // n, keys % n


def _relabel(lo, hi, n, rng):
    perm = rng.permutation(n).astype(np.int32)
    return perm[lo], perm[hi]


def rmat_edges(n: int, m: int, seed: int, a=0.57, b=0.19, c=0.19, scale: int | None = None):
    """R-MAT graph with ``n`` nodes and exactly ``m`` distinct undirected edges.

    Node ids are drawn on a ``2**scale`` grid (``scale`` defaults to ceil(log2 n)); draws with an
    endpoint >= n are discarded and redrawn. Ids are randomly relabelled afterwards.
    """
    if scale is None:
        scale = max(1, int(np.ceil(np.log2(max(n, 2)))))
    rng = np.random.default_rng(seed)
    ab, abc = a + b, a + b + c

    def draw(k):
        u = np.zeros(k, np.int64)
        v = np.zeros(k, np.int64)
        for _ in range(scale):
            r = rng.random(k)
            bu = (r >= ab).astype(np.int64)                       # quadrants c, d: lower half
            bv = ((r >= a) & (r < ab)) | (r >= abc)               # quadrants b, d: right half
            u = (u << 1) | bu
            v = (v << 1) | bv.astype(np.int64)
        keep = (u < n) & (v < n)
        return u[keep], v[keep]

    lo, hi = _draw_until(m, n, draw, rng)
    return _relabel(lo, hi, n, rng)


def chung_lu_weights(n: int, m: int, gamma: float):
    """Expected degrees w_i proportional to (i+1)^(-1/(gamma-1)), sum 2m, capped at sqrt(2m).

    The cap is applied iteratively with renormalisation so that the uncapped nodes carry the rest
    of the total 2m.
    """
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
    total = 2.0 * m
    cap = np.sqrt(total)
    capped = np.zeros(n, bool)
    for _ in range(64):
        free = ~capped
        scale = (total - cap * capped.sum()) / w[free].sum()
        ww = np.where(capped, cap, w * scale)
        newly = (ww > cap) & free
        if not newly.any():
            return ww
        capped |= newly
    return np.minimum(ww, cap)


def chung_lu_edges(n: int, m: int, gamma: float, seed: int):
    """Chung-Lu graph with ``n`` nodes and exactly ``m`` distinct undirected edges.

    Each draw picks both endpoints independently with probability proportional to the expected
    degree, so the pair (u, v) has probability proportional to w_u * w_v. Ids are randomly
    relabelled afterwards.
    """
    rng = np.random.default_rng(seed)
    w = chung_lu_weights(n, m, gamma)
    p = w / w.sum()

    def draw(k):
        # k iid endpoint pairs: the multiset of first endpoints comes from multinomial counts;
        # the second endpoints are drawn the same way and put in random order, which pairs
        # them independently with the first ones.
        ids = np.arange(n, dtype=np.int64)
        u = np.repeat(ids, rng.multinomial(k, p))
        v = np.repeat(ids, rng.multinomial(k, p))
        rng.shuffle(v)
        return u, v

    lo, hi = _draw_until(m, n, draw, rng)
    return _relabel(lo, hi, n, rng)


def cached(tag: str, fn, *args, **kwargs):
    """Run ``fn(*args, **kwargs)`` -> tuple of arrays, caching to ``$AGP_SYNTH_CACHE`` if set."""
    root = os.environ.get("AGP_SYNTH_CACHE")
    if not root:
        return fn(*args, **kwargs)
    key = hashlib.sha1(repr((tag, args, sorted(kwargs.items()))).encode()).hexdigest()[:16]
    path = os.path.join(root, f"{tag}_{key}.npz")
    if os.path.exists(path):
        with np.load(path) as z:
            return tuple(z[f"a{i}"] for i in range(len(z.files)))
    out = fn(*args, **kwargs)
    os.makedirs(root, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, **{f"a{i}": x for i, x in enumerate(out)})
    os.replace(tmp, path)
    return out


def chung_lu_edges_cuda(n: int, m: int, gamma: float, seed: int, device: str = "cuda", chunk: int = 1 << 27,
                        log=None, bucket_keys: int = 1 << 30):
    """Chung-Lu graph drawn on a CUDA device (for graphs too large to draw quickly on the host).

    Same model and weights as ``chung_lu_edges``: endpoints are drawn independently by inverse
    CDF of the capped power-law weights (torch RNG seeded with ``seed``), non-loop pairs are
    canonicalised and deduplicated on the device, draws repeat until at least ``m`` distinct edges
    exist and a random surplus is dropped (uniformly within hash buckets, in proportion to their
    sizes); node ids are then randomly relabelled. Pairs are spread over hash buckets of about ``bucket_keys`` (2^30) keys, so that no tensor
    operation sees 2^31 elements or more. Returns CUDA int32 tensors ``(u, v)`` of length m. Deterministic for a
    given seed on a given GPU model.
    """
    import torch

    say = log or (lambda *_: None)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    w = chung_lu_weights(n, m, gamma)
    cdf = torch.from_numpy(np.cumsum(w) / w.sum()).to(device)
    del w
    P = max(1, -(-int(m * 1.1) // bucket_keys))
    parts = [torch.empty(0, dtype=torch.int64, device=device) for _ in range(P)]
    want = int(m * 1.05) + 1024
    while True:
        new = [[] for _ in range(P)]
        left = want
        while left > 0:
            k = min(chunk, left)
            left -= k
            u = torch.searchsorted(cdf, torch.rand(k, dtype=torch.float64, generator=gen, device=device), right=True)
            v = torch.searchsorted(cdf, torch.rand(k, dtype=torch.float64, generator=gen, device=device), right=True)
            u.clamp_(max=n - 1)
            v.clamp_(max=n - 1)
            lo, hi = torch.minimum(u, v), torch.maximum(u, v)
            del u, v
            keep = lo != hi
            lo, hi = lo[keep], hi[keep]
            key = lo * n + hi
            if P == 1:
                new[0].append(key)
            else:
                b = torch.remainder(lo + hi, P)
                for p in range(P):
                    new[p].append(key[b == p])
                del b
            del lo, hi, keep, key
        count = 0
        for p in range(P):
            parts[p] = torch.unique(torch.cat([parts[p]] + new[p]))
            new[p] = None
            count += parts[p].numel()
        say(f"[synth] {count} distinct edges after drawing {want} pairs ({P} buckets)")
        if count >= m:
            break
        want = int((m - count) * 1.5) + 1024
    surplus = count - m
    if surplus:
        # the surplus is split over the buckets in proportion to their sizes (the buckets are a
        # hash partition, so this is a uniform drop up to rounding of the split)
        sizes = np.array([t.numel() for t in parts], dtype=np.int64)
        drops = (sizes * surplus) // count
        drops[: surplus - int(drops.sum())] += 1
        for p in range(P):
            if drops[p]:
                idx = torch.randperm(int(sizes[p]), generator=gen, device=device)[: int(drops[p])]
                mask = torch.ones(int(sizes[p]), dtype=torch.bool, device=device)
                mask[idx] = False
                parts[p] = parts[p][mask]
                del idx, mask
    perm = torch.randperm(n, generator=gen, device=device).to(torch.int32)
    lo = torch.empty(m, dtype=torch.int32, device=device)
    hi = torch.empty(m, dtype=torch.int32, device=device)
    off = 0
    for p in range(P):
        keys = parts[p]
        parts[p] = None
        c = keys.numel()
        lo[off:off + c] = perm[keys // n]
        hi[off:off + c] = perm[keys % n]
        off += c
        del keys
    del perm
    return lo, hi

"""Seeded synthetic graph generators.

These produce the *inputs* of the solver (edge lists and weights) and nothing
else: no part of the method's arithmetic lives here.  Both the CUDA path and the
FP64 oracle consume the same arrays, so this module is the only code the two
sides share.

The paper's own workloads (Bhoslib frb59-26-*, SNAP Amazon/DBLP/Google+, Sec. 4.2)
are not available; these generators stand in for them with seeded graphs of
the shapes used in the benchmarks:

* ``er_graph``      -- Erdos-Renyi G(n, M): M distinct undirected edges, uniform.
* ``chung_lu``      -- power-law expected-degree graph (exponent gamma), M edges.
* ``grid_graph``    -- 4-neighbour W x H grid, the multiway-cut image workload.

Every edge list is canonical: ``eu < ev`` elementwise, no duplicates, sorted by
``(eu, ev)``.  Vertex ids of the random graphs are a seeded random relabelling,
so id order carries no structure.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph",
    "er_graph",
    "chung_lu",
    "grid_graph",
    "int_weights",
    "unit_interval_weights",
    "lognormal_weights",
    "batch_instances",
]


@dataclass
class Graph:
    """An undirected simple graph with optional vertex / edge weights."""

    n: int
    eu: np.ndarray  # int32[m], eu < ev
    ev: np.ndarray  # int32[m]
    w: np.ndarray | None = None  # float32[n] vertex weights (VC / IS)
    ce: np.ndarray | None = None  # float32[m] edge weights (multiway cut)
    terminals: np.ndarray | None = None  # int32[k] (multiway cut)
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])


def _canonical_unique(u: np.ndarray, v: np.ndarray, n: int, m: int):
    """Canonicalise pairs, drop loops, keep the first ``m`` distinct pairs in
    draw order.  Returns the kept keys (u*n+v) or fewer if not enough."""
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v).astype(np.int64)
    hi = np.maximum(u, v).astype(np.int64)
    key = lo * n + hi
    _, first = np.unique(key, return_index=True)
    first.sort()
    return key[first[:m]]


def _finish(keys: np.ndarray, n: int, relabel: np.ndarray | None):
    eu = (keys // n).astype(np.int64)
    ev = (keys % n).astype(np.int64)
    if relabel is not None:
        eu, ev = relabel[eu], relabel[ev]
        lo = np.minimum(eu, ev)
        hi = np.maximum(eu, ev)
        eu, ev = lo, hi
    order = np.lexsort((ev, eu))
    return eu[order].astype(np.int32), ev[order].astype(np.int32)


def er_graph(n: int, m: int, seed: int) -> Graph:
    """G(n, M): ``m`` distinct edges drawn uniformly without loops."""
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges for a simple graph")
    rng = np.random.default_rng(seed)
    # draw pairs until at least m distinct ones exist, then keep a uniformly
    # random m-subset of the distinct pairs (uniform over m-edge graphs)
    keys = np.empty(0, np.int64)
    draw = int(m * 1.1) + 64
    while True:
        u = rng.integers(0, n, size=draw)
        v = rng.integers(0, n, size=draw)
        keep = u != v
        lo = np.minimum(u[keep], v[keep]).astype(np.int64)
        hi = np.maximum(u[keep], v[keep]).astype(np.int64)
        keys = np.sort(np.concatenate([keys, lo * n + hi]))
        if keys.shape[0] > 1:
            keys = keys[np.concatenate([[True], keys[1:] != keys[:-1]])]
        if keys.shape[0] >= m:
            break
        draw = int((m - keys.shape[0]) * 1.5) + 64
    if keys.shape[0] > m:
        keys = keys[np.sort(rng.choice(keys.shape[0], size=m, replace=False))]
    eu = (keys // n).astype(np.int32)
    ev = (keys % n).astype(np.int32)
    return Graph(n=n, eu=eu, ev=ev, meta={"kind": "er", "n": n, "m": m, "seed": seed})


def chung_lu(n: int, m: int, gamma: float, seed: int) -> Graph:
    """Chung-Lu power-law graph.

    Expected degrees w_i proportional to (i+1)^(-1/(gamma-1)), scaled to mean 2m/n
    and capped at sqrt(sum w) (the usual Chung-Lu admissibility cap).  Endpoint
    pairs are drawn independently from w; loops and repeated pairs are dropped
    until ``m`` distinct edges remain.  Vertex ids are randomly relabelled.
    """
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (gamma - 1.0))
    target = 2.0 * m / n
    for _ in range(8):
        w *= target / w.mean()
        cap = np.sqrt(w.sum())
        w = np.minimum(w, cap)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    keys = np.empty(0, np.int64)
    need = m
    while keys.shape[0] < m:
        draw = int(need * 1.3) + 1024
        u = np.searchsorted(cdf, rng.random(draw), side="right")
        v = np.searchsorted(cdf, rng.random(draw), side="right")
        u = np.minimum(u, n - 1)
        v = np.minimum(v, n - 1)
        new = _canonical_unique(u, v, n, draw)
        allk = np.concatenate([keys, new])
        _, first = np.unique(allk, return_index=True)
        first.sort()
        keys = allk[first][:m]
        need = m - keys.shape[0]
    relabel = rng.permutation(n).astype(np.int64)
    eu, ev = _finish(keys, n, relabel)
    return Graph(n=n, eu=eu, ev=ev,
                 meta={"kind": "chung_lu", "n": n, "m": m, "gamma": gamma, "seed": seed})


def grid_graph(width: int, height: int, k: int, seed: int) -> Graph:
    """4-neighbour grid with ``k`` distinct terminal pixels and lognormal(0,1)
    edge weights (FP32).  Vertex id = row*width + col."""
    n = width * height
    idx = np.arange(n, dtype=np.int64).reshape(height, width)
    hu = idx[:, :-1].ravel()
    hv = idx[:, 1:].ravel()
    vu = idx[:-1, :].ravel()
    vv = idx[1:, :].ravel()
    eu = np.concatenate([hu, vu])
    ev = np.concatenate([hv, vv])
    order = np.lexsort((ev, eu))
    eu = eu[order].astype(np.int32)
    ev = ev[order].astype(np.int32)
    rng = np.random.default_rng(seed)
    terminals = rng.choice(n, size=k, replace=False).astype(np.int32)
    ce = lognormal_weights(eu.shape[0], rng)
    return Graph(n=n, eu=eu, ev=ev, ce=ce, terminals=terminals,
                 meta={"kind": "grid", "width": width, "height": height, "k": k, "seed": seed})


def int_weights(n: int, lo: int, hi: int, rng) -> np.ndarray:
    """Integer weights uniform in [lo, hi], stored as FP32 (exact)."""
    return rng.integers(lo, hi + 1, size=n).astype(np.float32)


def unit_interval_weights(n: int, rng) -> np.ndarray:
    """Weights uniform in (0, 1] on the 2^-24 lattice, exact in FP32."""
    return (rng.integers(1, (1 << 24) + 1, size=n).astype(np.float64) / float(1 << 24)).astype(np.float32)


def lognormal_weights(m: int, rng) -> np.ndarray:
    return rng.lognormal(0.0, 1.0, size=m).astype(np.float32)


def batch_instances(count: int, n_lo: int, n_hi: int, d_lo: float, d_hi: float,
                    w_lo: int, w_hi: int, seed: int):
    """Batched workload: ``count`` ER instances, the first half vertex cover, the
    second half independent set.  n ~ U[n_lo, n_hi], average degree
    d ~ U[d_lo, d_hi], M = round(n*d/2), integer weights U[w_lo, w_hi].

    Returns a list of (kind, Graph) with kind in {"vc", "is"}.
    """
    rng = np.random.default_rng(seed)
    out = []
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    ds = rng.uniform(d_lo, d_hi, size=count)
    seeds = rng.integers(0, 2**62, size=count)
    for t in range(count):
        n = int(ns[t])
        m = int(round(n * ds[t] / 2.0))
        g = er_graph(n, m, int(seeds[t]))
        g.w = int_weights(n, w_lo, w_hi, np.random.default_rng(int(seeds[t]) ^ 0x5DEECE66D))
        out.append(("vc" if t < count // 2 else "is", g))
    return out


def serving_pool(count: int, seed: int, n_lo: float = 1e3, n_hi: float = 1e6, d_lo: float = 4.0,
                 d_hi: float = 16.0, side_lo: int = 64, side_hi: int = 512, k: int = 4,
                 mix=(0.4, 0.4, 0.2)):
    """Request pool of the serving workload: ``count`` graphs whose kinds follow
    ``mix`` (vertex cover, independent set, multiway cut) in proportion.  VC/IS:
    ER with n log-uniform in [n_lo, n_hi], average degree U[d_lo, d_hi],
    integer weights U[1, 10].  MC: a side x side 4-neighbour grid, side
    U[side_lo, side_hi], ``k`` terminals, lognormal(0, 1) edge weights.

    Returns a list of (kind, Graph)."""
    rng = np.random.default_rng(seed)
    n_vc = int(round(count * mix[0]))
    n_is = int(round(count * mix[1]))
    kinds = ["vc"] * n_vc + ["is"] * n_is + ["mc"] * (count - n_vc - n_is)
    out = []
    for kind in kinds:
        s = int(rng.integers(0, 2**62))
        if kind == "mc":
            side = int(rng.integers(side_lo, side_hi + 1))
            out.append((kind, grid_graph(side, side, k, s)))
            continue
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        m = int(round(n * rng.uniform(d_lo, d_hi) / 2.0))
        g = er_graph(n, m, s)
        g.w = int_weights(n, 1, 10, np.random.default_rng(s ^ 0x5DEECE66D))
        out.append((kind, g))
    return out


def poisson_trace(rate: float, count: int, kinds, seed: int, mix=(0.4, 0.4, 0.2)):
    """Open-loop arrival trace: ``count`` arrival times (seconds from the start)
    of a Poisson process with ``rate`` per second, and for each arrival the
    index of a pool entry: the kind is drawn from ``mix``, then an entry of that
    kind uniformly.  ``kinds`` lists the pool's kinds."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    by_kind = {c: np.flatnonzero(np.asarray(kinds) == c) for c in ("vc", "is", "mc")}
    names = np.array(["vc", "is", "mc"])
    pick = names[rng.choice(3, size=count, p=np.asarray(mix, np.float64) / np.sum(mix))]
    idx = np.array([by_kind[c][rng.integers(len(by_kind[c]))] for c in pick], np.int64)
    return t, idx


class SetSystem:
    """A set system for set cover: set j holds elems[ptr[j]:ptr[j+1]]
    (increasing element ids); cost[j] integer-valued FP32."""

    def __init__(self, n_elements, ptr, elems, cost):
        self.n_elements = int(n_elements)
        self.ptr = ptr
        self.elems = elems
        self.cost = cost

    @property
    def n_sets(self):
        return int(self.ptr.shape[0]) - 1


def set_cover_instance(n_elements: int, n_sets: int, f_lo: int, f_hi: int, seed: int) -> SetSystem:
    """Every element is put in f ~ U[f_lo, f_hi] distinct random sets (draws
    that repeat a set for the same element are dropped, so a few elements get
    fewer); set costs integer U[1, 10]."""
    rng = np.random.default_rng(seed)
    f = rng.integers(f_lo, f_hi + 1, size=n_elements)
    cand = rng.integers(0, n_sets, size=(n_elements, f_hi))
    cand = np.sort(np.where(np.arange(f_hi)[None, :] < f[:, None], cand, n_sets), axis=1)
    keep = cand < n_sets
    keep[:, 1:] &= cand[:, 1:] != cand[:, :-1]
    elem = np.repeat(np.arange(n_elements, dtype=np.int64), f_hi)[keep.ravel()]
    sets = cand.ravel()[keep.ravel()].astype(np.int64)
    order = np.lexsort((elem, sets))
    sets, elem = sets[order], elem[order]
    ptr = np.zeros(n_sets + 1, np.int64)
    np.cumsum(np.bincount(sets, minlength=n_sets), out=ptr[1:])
    cost = rng.integers(1, 11, size=n_sets).astype(np.float32)
    return SetSystem(n_elements, ptr, elem.astype(np.int32), cost)


class PairwiseMRF:
    """Pairwise factor graph: n variables with k labels, edges eu[e] -- ev[e],
    scores theta_node (n, k) and theta_edge (m, k, k), FP32."""

    def __init__(self, n, k, eu, ev, theta_node, theta_edge):
        self.n, self.k = int(n), int(k)
        self.eu, self.ev = eu, ev
        self.theta_node, self.theta_edge = theta_node, theta_edge

    @property
    def m(self):
        return int(self.eu.shape[0])


def skip_chain_crf(n: int, k: int, sent_len: int, skip_frac: float, seed: int) -> PairwiseMRF:
    """Skip-chain-CRF-shaped MRF (the shape of the paper's text-chunking factor
    graph): the variables form sentences of `sent_len` consecutive tokens with a
    chain factor between neighbours; a `skip_frac` share of tokens also gets a
    skip factor to a random earlier token within 500 positions.  Unary scores
    N(0, 1); chain factors share one transition matrix N(0, 0.5) (tied CRF
    weights); skip factors reward equal labels by a weight U(0, 1)."""
    rng = np.random.default_rng(seed)
    i = np.arange(n - 1)
    chain = i[(i + 1) % sent_len != 0]
    cu, cv = chain, chain + 1
    src = np.flatnonzero(rng.random(n) < skip_frac)
    src = src[src > 0]
    dst = np.maximum(0, src - rng.integers(2, 501, size=src.shape[0]))
    ok = dst < src - 1  # not a chain neighbour
    su, sv = dst[ok], src[ok]
    eu = np.concatenate([cu, su]).astype(np.int32)
    ev = np.concatenate([cv, sv]).astype(np.int32)
    tn = rng.normal(size=(n, k)).astype(np.float32)
    trans = rng.normal(scale=0.5, size=(k, k)).astype(np.float32)
    te = np.empty((eu.shape[0], k, k), np.float32)
    te[: cu.shape[0]] = trans
    lam = rng.random(su.shape[0]).astype(np.float32)
    te[cu.shape[0]:] = lam[:, None, None] * np.eye(k, dtype=np.float32)[None]
    return PairwiseMRF(n, k, eu, ev, tn, te)

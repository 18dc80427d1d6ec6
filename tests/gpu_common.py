"""Shared helpers of the GPU tests: build the same seeded workload on both
sides (CUDA library through the C ABI, FP64 oracle) and compare."""
import numpy as np

import oracle
from paper_1311_2661_gb300 import synth

X_TOL = 1e-4      # max |x_gpu - x_oracle|
OBJ_RTOL = 1e-5   # relative objective difference


def gpu():
    from paper_1311_2661_gb300 import thetis

    return thetis


def vc_graph(n, m, seed, wmax=10):
    g = synth.er_graph(n, m, seed)
    g.w = synth.int_weights(n, 1, wmax, np.random.default_rng(seed + 1000))
    return g


def is_graph(n, m, seed):
    g = synth.chung_lu(n, m, 2.1, seed)
    g.w = synth.unit_interval_weights(n, np.random.default_rng(seed + 2000))
    return g


def hub_graph(n, m, hub_deg, seed):
    """ER graph plus one hub of degree hub_deg (exercises the CTA-per-column class)."""
    g = synth.er_graph(n, m, seed)
    rng = np.random.default_rng(seed + 7)
    hub = 0
    nb = rng.choice(np.arange(1, n), size=hub_deg, replace=False)
    key = set(zip(g.eu.tolist(), g.ev.tolist()))
    extra = [(hub, int(v)) for v in nb if (hub, int(v)) not in key]
    eu = np.concatenate([g.eu, np.array([e[0] for e in extra], np.int32)])
    ev = np.concatenate([g.ev, np.array([e[1] for e in extra], np.int32)])
    o = np.lexsort((ev, eu))
    g.eu, g.ev = eu[o].astype(np.int32), ev[o].astype(np.int32)
    g.w = synth.int_weights(n, 1, 10, rng)
    return g


def multi_hub_graph(n, m, hubs, seed):
    """ER graph plus hubs {vertex: degree} at scattered vertex ids: columns and
    vertex lists long enough for every per-group sort tier of the build (more
    than 8, 32, 128 and 4096 entries) in warps other than the first."""
    g = synth.er_graph(n, m, seed)
    rng = np.random.default_rng(seed + 11)
    key = set(zip(g.eu.tolist(), g.ev.tolist()))
    extra = []
    for hub, deg in hubs.items():
        nb = rng.choice(np.delete(np.arange(n), hub), size=deg, replace=False)
        for v in nb.tolist():
            e = (min(hub, v), max(hub, v))
            if e not in key:
                key.add(e)
                extra.append(e)
    eu = np.concatenate([g.eu, np.array([e[0] for e in extra], np.int32)])
    ev = np.concatenate([g.ev, np.array([e[1] for e in extra], np.int32)])
    o = np.lexsort((ev, eu))
    g.eu, g.ev = eu[o].astype(np.int32), ev[o].astype(np.int32)
    g.w = synth.int_weights(n, 1, 10, rng)
    return g


def build_gpu(kind, g, seed=0, device=False, stream=None):
    T = gpu()
    if device:
        import torch

        dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    else:
        dv = lambda a: a
    if kind == "vc":
        return T.thetis_build_vc(g.n, dv(g.eu), dv(g.ev), dv(g.w), seed=seed, stream=stream)
    if kind == "is":
        return T.thetis_build_is(g.n, dv(g.eu), dv(g.ev), dv(g.w), seed=seed, stream=stream)
    return T.thetis_build_mc(g.n, dv(g.eu), dv(g.ev), dv(g.ce), len(g.terminals), dv(g.terminals),
                             seed=seed, stream=stream)


def gpu_full_x(h):
    return np.concatenate([h.get_x().astype(np.float64), h.get_slack().astype(np.float64)])


def rel(a, b):
    return abs(a - b) / max(1.0, abs(b))

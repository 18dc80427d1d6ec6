"""Oracle pins for set cover (App. B.1): the covering LP, the covering repair
(App. C.2 lemma with q(P) = 1), the f-threshold rounding (Hochbaum) and the
randomized rounding (Srinivasan) with the uncovered-element fix-up."""
import itertools

import numpy as np
import pytest
from scipy.optimize import linprog

from paper_1311_2661_gb300 import synth


def _set_system(n_elem, k_sets, seed, fmax=4):
    """Every element in 1..fmax random sets; costs integer U[1, 10]."""
    rng = np.random.default_rng(seed)
    members = [[] for _ in range(k_sets)]
    for a in range(n_elem):
        for s in rng.choice(k_sets, size=int(rng.integers(1, fmax + 1)), replace=False):
            members[s].append(a)
    ptr = np.concatenate([[0], np.cumsum([len(m) for m in members])]).astype(np.int64)
    elems = np.array([a for m in members for a in sorted(m)], np.int32)
    cost = rng.integers(1, 11, size=k_sets).astype(np.float64)
    return ptr, elems, cost


def _lp_opt(lp):
    e = lp.export()
    res = linprog(e["c"], A_eq=lp.dense_A(), b_eq=e["b"],
                  bounds=list(zip(e["lo"], np.where(np.isinf(e["hi"]), None, e["hi"]))), method="highs")
    assert res.status == 0
    return res.x, res.fun


def _covers(ptr, elems, n_elem, take):
    cov = np.zeros(n_elem, bool)
    for s in np.flatnonzero(take):
        cov[elems[ptr[s]:ptr[s + 1]]] = True
    return cov.all()


def test_vertex_cover_is_set_cover_with_f2(oracle_mod):
    """Sets = vertices, elements = edges: the set-cover LP is the vertex-cover LP
    and the f-threshold (f = 2) is the VC threshold, label for label."""
    g = synth.er_graph(200, 600, 3)
    w = synth.int_weights(200, 1, 10, np.random.default_rng(4)).astype(np.float64)
    members = [[] for _ in range(g.n)]
    for e, (u, v) in enumerate(zip(g.eu, g.ev)):
        members[u].append(e)
        members[v].append(e)
    ptr = np.concatenate([[0], np.cumsum([len(m) for m in members])]).astype(np.int64)
    elems = np.array([e for m in members for e in m], np.int32)
    sc = oracle_mod.OracleLP.set_cover(g.m, ptr, elems, w)
    vc = oracle_mod.OracleLP.vc(g.n, g.eu, g.ev, w)
    vc.n_vertices = g.n
    assert sc.sc_frequency() == 2
    assert abs(_lp_opt(sc)[1] - _lp_opt(vc)[1]) < 1e-7
    x, _ = sc.solve(beta=100.0, epochs=200, refresh_every=10)
    for xx in (x[: g.n], np.clip(x[: g.n] * 0.9, 0, 1)):  # feasible-ish and infeasible (repair) points
        a, b = sc.round_sc(xx), vc.round_vc(xx)
        assert a["status"] == b["status"] == 0
        assert np.array_equal(a["labels"], b["labels"])
        assert abs(a["eps"] - b["eps"]) < 1e-15 and a["obj"] == b["obj"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_threshold_is_an_f_approximation(oracle_mod, seed):
    ptr, elems, cost = _set_system(40, 16, seed)
    lp = oracle_mod.OracleLP.set_cover(40, ptr, elems, cost)
    f = lp.sc_frequency()
    xs, lp_star = _lp_opt(lp)
    r = lp.round_sc(xs[:16])
    assert r["status"] == 0 and lp.valid_sc(r["labels"]) and _covers(ptr, elems, 40, r["labels"])
    ip_star = min(cost @ np.array(t) for t in itertools.product([0, 1], repeat=16)
                  if _covers(ptr, elems, 40, np.array(t, np.uint8)))
    assert lp_star - 1e-9 <= ip_star <= r["obj"] <= f * lp_star + 1e-9
    rr = lp.round_sc_rand(xs[:16], seed=5, reps=10)
    assert rr["status"] == 0 and lp.valid_sc(rr["labels"]) and rr["obj"] >= ip_star


def test_randomized_pick_and_fixup_probabilities(oracle_mod):
    """One element in sets {0, 1} with x~ = (0.6, 0.5): set 1 is taken with
    probability 0.5; set 0 with 0.6 + P(neither picked) = 0.6 + 0.4 * 0.5 = 0.8
    (the fix-up adds the larger-x~ set)."""
    lp = oracle_mod.OracleLP.set_cover(1, np.array([0, 1, 2]), np.array([0, 0], np.int32), np.ones(2))
    xt = np.array([0.6, 0.5])
    reps = 20000
    takes = np.array([lp.round_sc_rand_rep(xt, 7, r) for r in range(reps)], np.float64)
    p = takes.mean(axis=0)
    for got, want in ((p[0], 0.8), (p[1], 0.5)):
        assert abs(got - want) <= 4 * np.sqrt(want * (1 - want) / reps)
    assert np.all(takes.sum(axis=1) >= 1)  # always a cover


def test_repair_makes_every_element_covered(oracle_mod):
    ptr, elems, cost = _set_system(60, 25, 9)
    lp = oracle_mod.OracleLP.set_cover(60, ptr, elems, cost)
    xs, _ = _lp_opt(lp)
    x = np.clip(xs[:25] * 0.7, 0, 1)  # infeasible: every coverage scaled by 0.7
    r = lp.round_sc(x)
    assert 0 < r["eps"] < 1
    xt = np.minimum(1.0, x / (1 - r["eps"]))
    for a in range(60):
        sets = [s for s in range(25) if a in elems[ptr[s]:ptr[s + 1]]]
        assert xt[sets].sum() >= 1 - 1e-12
    assert r["status"] == 0 and lp.valid_sc(r["labels"])
    # a point that cannot be repaired
    assert lp.round_sc(np.zeros(25))["status"] == 6

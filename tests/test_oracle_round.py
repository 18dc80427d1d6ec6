"""Oracle pins for repair and rounding: the feasibility lemmas of App. C,
the factor-2 bound of Sec. 2, exact selection probabilities of the packing
rounding (App. B.2), the CKR expectation (App. B.3) and validity."""
import itertools

import numpy as np
import pytest

from paper_1311_2661_gb300 import synth


def _graph_lp(oracle_mod, kind, n, m, seed, wmax=10):
    g = synth.er_graph(n, m, seed)
    g.w = synth.int_weights(n, 1, wmax, np.random.default_rng(seed))
    return g, oracle_mod.build_problem(kind, g)


@pytest.mark.parametrize("seed", range(5))
def test_vc_repair_feasible_and_factor_two(oracle_mod, seed):
    g, lp = _graph_lp(oracle_mod, "vc", 40, 120, seed)
    rng = np.random.default_rng(seed)
    # an infeasible point with eps < 1
    x = np.clip(rng.uniform(0.2, 0.7, g.n), 0, 1)
    r = lp.round_vc(x)
    eps = max(0.0, float(np.max(1 - x[g.eu] - x[g.ev])))
    assert r["status"] == 0 and r["eps"] == eps
    xt = np.minimum(1.0, x / (1 - eps))
    assert np.all(xt[g.eu] + xt[g.ev] >= 1 - 1e-12)  # Lemma: x~ feasible
    lab = r["labels"].astype(bool)
    assert np.array_equal(lab, xt >= 0.5)
    assert lp.valid(r["labels"])
    assert r["obj"] == float(g.w[lab].sum())
    assert r["obj"] <= 2 * float(g.w @ xt) + 1e-9  # Sec. 2: at most twice the LP cost at x~


def test_vc_repair_eps_ge_one(oracle_mod):
    g, lp = _graph_lp(oracle_mod, "vc", 10, 20, 3)
    r = lp.round_vc(np.zeros(10))
    assert r["status"] == 6


@pytest.mark.parametrize("seed", range(3))
def test_vc_rounded_vs_ip_enumeration(oracle_mod, seed):
    """Round the converged QP point; with x~ feasible and delta' from the LP,
    cost <= 2 (1 + delta') LP* <= 2(1+delta') IP* (2^n enumeration)."""
    g, lp = _graph_lp(oracle_mod, "vc", 12, 24, seed)
    x, info = lp.solve(beta=100.0, epochs=20000, tol=1e-9, refresh_every=50)
    r = lp.round_vc(x[: g.n])
    best = None
    w = g.w.astype(np.float64)
    for bits in itertools.product((0, 1), repeat=g.n):
        b = np.array(bits, bool)
        if np.all(b[g.eu] | b[g.ev]):
            c = float(w[b].sum())
            best = c if best is None else min(best, c)
    xt = np.minimum(1.0, x[: g.n] / (1 - r["eps"]))
    assert lp.valid(r["labels"])
    assert r["obj"] <= 2 * float(w @ xt) + 1e-9
    assert float(w @ xt) >= best / 2 - 1e-9  # LP value at a feasible point >= LP* >= IP*/2


@pytest.mark.parametrize("seed", range(4))
def test_is_repair_and_validity(oracle_mod, seed):
    g, lp = _graph_lp(oracle_mod, "is", 60, 200, seed)
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 0.9, g.n)
    r = lp.round_is(x, seed=seed, reps=10)
    alpha = max(0.0, float(np.max(x[g.eu] + x[g.ev] - 1)))
    assert r["alpha"] == alpha
    xt = x / (1 + alpha)
    assert np.all(xt[g.eu] + xt[g.ev] <= 1 + 1e-12)  # App. C.3: x~ feasible
    assert lp.valid(r["labels"])
    assert r["obj"] == float(g.w[r["labels"].astype(bool)].sum())
    # best of reps: no single repetition beats it, ties go to the lowest rep
    objs = [float(g.w[lp.round_is_rep(xt, seed, q).astype(bool)].sum()) for q in range(10)]
    assert r["obj"] == max(objs) and r["best_rep"] == int(np.argmax(objs))


def test_is_selection_probabilities_single_edge(oracle_mod):
    """Algorithm 2 with theta = 1/k: u (lower id) is kept with probability
    x~_u, v with probability x~_v (1 - x~_u)."""
    lp = oracle_mod.OracleLP.is_(2, np.array([0], np.int32), np.array([1], np.int32), np.ones(2))
    lp.n_vertices = 2
    xt = np.array([0.3, 0.6])
    reps = 20000
    keep = np.array([lp.round_is_rep(xt, 99, q) for q in range(reps)], np.float64)
    p = keep.mean(0)
    for got, want in zip(p, [0.3, 0.6 * 0.7]):
        assert abs(got - want) < 5 * np.sqrt(want * (1 - want) / reps)
    assert not np.any(keep.sum(1) == 2)


def _mc_lp(oracle_mod, w, h, k, seed):
    g = synth.grid_graph(w, h, k, seed)
    lp = oracle_mod.build_problem("mc", g)
    return g, lp


def _random_simplex_x(g, k, rng):
    x = rng.dirichlet(np.ones(k) * 0.7, size=g.n)
    for i, t in enumerate(g.terminals):
        x[t] = 0
        x[t, i] = 1
    return x.ravel()


def test_ckr_k2_expectation_equals_lp_cost(oracle_mod):
    """For k = 2 an edge is cut with probability exactly |x_u1 - x_v1| =
    d(u,v), so the expected CKR cost equals the LP cost at x."""
    g, lp = _mc_lp(oracle_mod, 5, 4, 2, 3)
    rng = np.random.default_rng(3)
    x = _random_simplex_x(g, 2, rng)
    X = x.reshape(g.n, 2)
    ce = g.ce.astype(np.float64)
    lpcost = float(np.sum(ce * 0.5 * np.abs(X[g.eu] - X[g.ev]).sum(1)))
    reps = 6000
    costs = np.array([lp.mc_cut_cost(lp.round_mc_rep(x, 5, q)) for q in range(reps)])
    assert abs(costs.mean() - lpcost) < 5 * costs.std() / np.sqrt(reps)


@pytest.mark.parametrize("k", [3, 4])
def test_ckr_bound_and_terminals(oracle_mod, k):
    """CKR: every terminal keeps its own label and E[cost] <= (3/2 - 1/k) LP(x)."""
    g, lp = _mc_lp(oracle_mod, 5, 5, k, 7 + k)
    rng = np.random.default_rng(k)
    x = _random_simplex_x(g, k, rng)
    X = x.reshape(g.n, k)
    ce = g.ce.astype(np.float64)
    lpcost = float(np.sum(ce * 0.5 * np.abs(X[g.eu] - X[g.ev]).sum(1)))
    reps = 4000
    costs = []
    for q in range(reps):
        lab = lp.round_mc_rep(x, 11, q)
        assert lp.valid(lab)
        assert all(lab[t] == i for i, t in enumerate(g.terminals))
        costs.append(lp.mc_cut_cost(lab))
    costs = np.array(costs)
    assert costs.mean() <= (1.5 - 1.0 / k) * lpcost + 5 * costs.std() / np.sqrt(reps)
    r = lp.round_mc(x, 11, reps=10)
    assert r["obj"] == costs[:10].min() and r["best_rep"] == int(np.argmin(costs[:10]))


def test_ckr_radius_and_permutation_streams(oracle_mod):
    """The radius is U(seed, rep, 2, 0) and the order a Fisher-Yates shuffle on
    stream 3: a vertex exactly at a terminal's unit vector gets that label, and
    a vertex at the barycentre falls in the first ball iff 1/k >= 1 - rho."""
    g, lp = _mc_lp(oracle_mod, 3, 3, 3, 1)
    k = 3
    x = np.tile(np.full(k, 1.0 / k), g.n)
    for i, t in enumerate(g.terminals):
        x[t * k:(t + 1) * k] = 0
        x[t * k + i] = 1
    for rep in range(50):
        rho = oracle_mod.rng_uniform(11, rep, 2, 0)
        sig = list(range(k))
        for i in range(k - 1, 0, -1):
            j = int(np.floor(oracle_mod.rng_uniform(11, rep, 3, i) * (i + 1)))
            sig[i], sig[j] = sig[j], sig[i]
        lab = lp.round_mc_rep(x, 11, rep)
        free = [v for v in range(g.n) if v not in set(g.terminals.tolist())]
        want = sig[0] if 1.0 / k >= 1 - rho else sig[k - 1]
        assert all(lab[v] == want for v in free)

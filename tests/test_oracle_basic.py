"""Oracle pins: random numbers, standard-form builders, colouring, simplex
projection.  Each pin compares the oracle with something other than itself:
published test vectors, LP optima from scipy's HiGHS and closed forms,
networkx's greedy colouring, an independent bisection projection."""
import json
import os

import numpy as np
import pytest

from paper_1311_2661_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# splitmix64
# --------------------------------------------------------------------------
def test_splitmix64_published_vectors(oracle_mod):
    g = _gold("splitmix64.json")
    for i, h in enumerate(g["seed_0_hex"]):
        assert oracle_mod.splitmix64_at(0, i) == int(h, 16)
    for i, v in enumerate(g["seed_1234567"]):
        assert oracle_mod.splitmix64_at(1234567, i) == v


def test_rng_uniform_range_and_mean(oracle_mod):
    u = np.array([oracle_mod.rng_uniform(7, 3, 1, i) for i in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    # distinct (rep, stream) keys give distinct streams
    a = [oracle_mod.rng_u64(7, 0, 1, i) for i in range(64)]
    b = [oracle_mod.rng_u64(7, 1, 1, i) for i in range(64)]
    c = [oracle_mod.rng_u64(7, 0, 2, i) for i in range(64)]
    assert len(set(a) | set(b) | set(c)) == 192


# --------------------------------------------------------------------------
# standard form builders, pinned through LP optima
# --------------------------------------------------------------------------
def _lp_opt(lp, upper=True):
    """LP optimum of the oracle's standard form by scipy HiGHS."""
    from scipy.optimize import linprog

    e = lp.export()
    A = lp.dense_A()
    bounds = [(lo, None if (not upper or not np.isfinite(hi)) else hi) for lo, hi in zip(e["lo"], e["hi"])]
    res = linprog(e["c"], A_eq=A, b_eq=e["b"], bounds=bounds, method="highs")
    assert res.status == 0
    return res


def _complete(n):
    eu, ev = np.triu_indices(n, 1)
    return eu.astype(np.int32), ev.astype(np.int32)


def _cycle(n):
    eu = np.arange(n)
    ev = (eu + 1) % n
    lo, hi = np.minimum(eu, ev), np.maximum(eu, ev)
    return lo.astype(np.int32), hi.astype(np.int32)


@pytest.mark.parametrize("n", [3, 4, 5, 7])
def test_vc_lp_complete_graph_is_n_over_2(oracle_mod, n):
    eu, ev = _complete(n)
    lp = oracle_mod.OracleLP.vc(n, eu, ev, np.ones(n))
    assert abs(_lp_opt(lp).fun - n / 2) < 1e-9


@pytest.mark.parametrize("n", [3, 5, 9])
def test_vc_lp_odd_cycle(oracle_mod, n):
    eu, ev = _cycle(n)
    lp = oracle_mod.OracleLP.vc(n, eu, ev, np.ones(n))
    assert abs(_lp_opt(lp).fun - n / 2) < 1e-9


def test_vc_lp_bipartite_is_matching(oracle_mod):
    # K_{2,3}: maximum matching 2 (Konig: LP* = IP* = 2)
    eu = np.array([0, 0, 0, 1, 1, 1], np.int32)
    ev = np.array([2, 3, 4, 2, 3, 4], np.int32)
    lp = oracle_mod.OracleLP.vc(5, eu, ev, np.ones(5))
    assert abs(_lp_opt(lp).fun - 2.0) < 1e-9


def _half_integral_opt(n, eu, ev, w, sense):
    """Brute force over {0,1/2,1}^n (edge LPs are half-integral)."""
    best = None
    vals = np.array([0.0, 0.5, 1.0])
    import itertools

    for t in itertools.product(range(3), repeat=n):
        x = vals[list(t)]
        s = x[eu] + x[ev]
        if sense == "vc" and np.any(s < 1 - 1e-12):
            continue
        if sense == "is" and np.any(s > 1 + 1e-12):
            continue
        o = float(w @ x)
        if best is None or (sense == "vc" and o < best) or (sense == "is" and o > best):
            best = o
    return best


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_vc_is_lp_vs_half_integral_enumeration(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = 7
    g = synth.er_graph(n, 10, seed)
    w = rng.integers(1, 11, n).astype(np.float64)
    vc = oracle_mod.OracleLP.vc(n, g.eu, g.ev, w)
    assert abs(_lp_opt(vc).fun - _half_integral_opt(n, g.eu, g.ev, w, "vc")) < 1e-9
    isp = oracle_mod.OracleLP.is_(n, g.eu, g.ev, w)
    # the IS form is a minimisation of -w^T x
    assert abs(-_lp_opt(isp).fun - _half_integral_opt(n, g.eu, g.ev, w, "is")) < 1e-9


def test_standard_form_shapes(oracle_mod):
    g = synth.er_graph(30, 60, 5)
    lp = oracle_mod.OracleLP.vc(30, g.eu, g.ev, np.ones(30))
    assert (lp.M, lp.Ns, lp.N, lp.nnz) == (60, 30, 90, 3 * 60)
    e = lp.export()
    A = lp.dense_A()
    # each row: x_u + x_v - s_e = 1
    for r in range(60):
        assert A[r, g.eu[r]] == 1 and A[r, g.ev[r]] == 1 and A[r, 30 + r] == -1
        assert abs(A[r]).sum() == 3
    assert np.all(e["b"] == 1)
    isp = oracle_mod.OracleLP.is_(30, g.eu, g.ev, np.ones(30))
    assert np.all(isp.dense_A()[:, 30:] == np.eye(60))
    assert np.all(isp.export()["c"][:30] == -1)


def test_mc_lp_path_two_terminals(oracle_mod):
    """Path 0-1-2-3 with terminals 0 and 3: the multiway-cut LP optimum is the
    cheapest edge (a path LP is integral)."""
    eu = np.array([0, 1, 2], np.int32)
    ev = np.array([1, 2, 3], np.int32)
    ce = np.array([3.0, 1.5, 2.0])
    lp = oracle_mod.OracleLP.mc(4, eu, ev, ce, 2, np.array([0, 3], np.int32))
    res = _lp_opt_mc(lp, 2, 4)
    assert abs(res - 1.5) < 1e-9


def _lp_opt_mc(lp, k, n):
    from scipy.optimize import linprog

    e = lp.export()
    A = lp.dense_A()
    N = lp.N
    Aeq = [A]
    beq = [e["b"]]
    # simplex rows sum_i x_{v,i} = 1 (the oracle enforces them by projection)
    S = np.zeros((n, N))
    for v in range(n):
        S[v, v * k:(v + 1) * k] = 1
    Aeq.append(S)
    beq.append(np.ones(n))
    bounds = [(lo, None if not np.isfinite(hi) else hi) for lo, hi in zip(e["lo"], e["hi"])]
    res = linprog(e["c"], A_eq=np.vstack(Aeq), b_eq=np.concatenate(beq), bounds=bounds, method="highs")
    assert res.status == 0
    return res.fun


def test_mc_lp_triangle_three_terminals(oracle_mod):
    """Triangle of terminals: every edge is cut, LP* = sum of weights."""
    eu = np.array([0, 0, 1], np.int32)
    ev = np.array([1, 2, 2], np.int32)
    ce = np.array([1.0, 2.0, 4.0])
    lp = oracle_mod.OracleLP.mc(3, eu, ev, ce, 3, np.array([0, 1, 2], np.int32))
    assert abs(_lp_opt_mc(lp, 3, 3) - 7.0) < 1e-9
    assert lp.U == 3 * 3 + 2 * 3 * 3  # z columns + slacks; terminal blocks are fixed


def test_mc_lp_star_fractional(oracle_mod):
    """Star with centre 3 and leaves = 3 terminals, unit weights: the LP and IP
    both cut two of the three edges (cost 2)."""
    eu = np.array([0, 1, 2], np.int32)
    ev = np.array([3, 3, 3], np.int32)
    lp = oracle_mod.OracleLP.mc(4, eu, ev, np.ones(3), 3, np.array([0, 1, 2], np.int32))
    assert abs(_lp_opt_mc(lp, 3, 4) - 2.0) < 1e-9


# --------------------------------------------------------------------------
# colouring
# --------------------------------------------------------------------------
def _conflict_graph(lp):
    import networkx as nx

    A = lp.dense_A() != 0
    us, ul, _ = lp.units()
    col_unit = -np.ones(lp.N, np.int64)
    for u, (s, l) in enumerate(zip(us, ul)):
        col_unit[s:s + l] = u
    G = nx.Graph()
    G.add_nodes_from(range(lp.U))
    for r in range(lp.M):
        units = sorted({int(col_unit[j]) for j in np.nonzero(A[r])[0] if col_unit[j] >= 0})
        for a in range(len(units)):
            for b in range(a + 1, len(units)):
                G.add_edge(units[a], units[b])
    return G, A, us, ul


@pytest.mark.parametrize("kind", ["vc", "is", "mc"])
def test_coloring_matches_networkx_greedy(oracle_mod, kind):
    nx = pytest.importorskip("networkx")
    if kind == "mc":
        g = synth.grid_graph(4, 3, 3, 11)
        lp = oracle_mod.OracleLP.mc(g.n, g.eu, g.ev, g.ce.astype(np.float64), 3, g.terminals)
    else:
        g = synth.er_graph(25, 60, 4)
        mk = oracle_mod.OracleLP.vc if kind == "vc" else oracle_mod.OracleLP.is_
        lp = mk(25, g.eu, g.ev, np.ones(25))
    seed = 12345
    G, A, us, ul = _conflict_graph(lp)
    # priority key restated here: (structural before slack, nnz desc, splitmix64_at(seed, u) desc, u asc)
    nnz = np.array([int(A[:, s:s + l].sum()) for s, l in zip(us, ul)])
    slack = [int(s >= lp.Ns) for s in us]
    keys = [(slack[u], -nnz[u], -oracle_mod.splitmix64_at(seed, u), u) for u in range(lp.U)]
    order = [k[3] for k in sorted(keys)]
    assert list(lp.priority_order(seed)) == order
    ref = nx.greedy_color(G, strategy=lambda G_, colors: iter(order))
    col, nc = lp.color(seed)
    assert nc == max(ref.values()) + 1
    assert all(col[u] == ref[u] for u in range(lp.U))
    for a, b in G.edges():
        assert col[a] != col[b]


# --------------------------------------------------------------------------
# simplex projection
# --------------------------------------------------------------------------
def _bisect_simplex(y):
    lo, hi = y.min() - 1.0, y.max()
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.maximum(y - mid, 0).sum() > 1.0:
            lo = mid
        else:
            hi = mid
    return np.maximum(y - 0.5 * (lo + hi), 0)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 17])
def test_simplex_projection(oracle_mod, k):
    rng = np.random.default_rng(k)
    for _ in range(200):
        y = rng.normal(0, 1.5, k)
        if rng.random() < 0.2:
            y[rng.integers(k)] = y[0]  # ties
        x = oracle_mod.project_simplex(y)
        assert abs(x.sum() - 1.0) < 1e-12 and x.min() >= 0
        assert np.max(np.abs(x - _bisect_simplex(y))) < 1e-10
        # KKT: x = max(y - theta, 0) with one theta for the support
        sup = x > 0
        th = (y - x)[sup]
        assert np.ptp(th) < 1e-12
        assert np.all(y[~sup] <= th[0] + 1e-12)

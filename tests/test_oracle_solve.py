"""Oracle pins for the coordinate-descent solve of eq. QP (Sec. 3.2-3.3):
single-edge closed forms, brute-force active-set enumeration of x(beta),
the exact fixed point x(beta) = x* when (xbar, ubar) is an LP primal-dual
optimal pair (Thm. 1 with C* = 0), the Thm. 1 residual bound, monotone
descent of f_beta, and the LCP of App. A at convergence."""
import itertools
import json
import os

import numpy as np
import pytest

from paper_1311_2661_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _closed():
    with open(os.path.join(GOLD, "closed_forms.json")) as f:
        return json.load(f)


def _single(oracle_mod, kind):
    mk = oracle_mod.OracleLP.vc if kind == "vc" else oracle_mod.OracleLP.is_
    lp = mk(2, np.array([0], np.int32), np.array([1], np.int32), np.ones(2))
    lp.n_vertices = 2
    return lp


@pytest.mark.parametrize("kind", ["vc", "is"])
def test_single_edge_closed_form(oracle_mod, kind):
    cf = _closed()[f"{kind}_single_edge"]
    beta, t = cf["beta"], cf["t"]
    lp = _single(oracle_mod, kind)
    x, info = lp.solve(beta=beta, epochs=400000, tol=1e-13, refresh_every=100)
    assert info["converged"]
    assert abs(x[0] - t) < 1e-9 and abs(x[1] - t) < 1e-9 and abs(x[2]) < 1e-12
    # checks at the closed-form point: obj, infeasibility, f_beta
    sgn = 1.0 if kind == "vc" else -1.0
    xs = np.array([t, t, 0.0])
    chk = lp.checks(xs, beta)
    f = sgn * 2 * t + beta / 2 * (2 * t - 1) ** 2 + t * t / beta
    assert abs(chk["obj"] - sgn * 2 * t) < 1e-14
    assert abs(chk["infeas"] - abs(2 * t - 1)) < 1e-14
    assert abs(chk["fbeta"] - f) < 1e-12
    assert chk["rho"] < 1e-12
    if kind == "vc":
        r = lp.round_vc(xs[:2])
        assert abs(r["eps"] - (1 - 2 * t)) < 1e-15
        assert r["near"] == 2  # x~ = 1/2: threshold tie
    else:
        r = lp.round_is(xs[:2], seed=1, reps=1)
        assert abs(r["alpha"] - (2 * t - 1)) < 1e-15


def _enumerate_qp(H, q, lo, hi):
    """Brute force over active sets {lo, hi, free}^N of min 1/2 x'Hx + q'x on a box."""
    N = len(q)
    states = [[0, 2] if not np.isfinite(hi[i]) else [0, 1, 2] for i in range(N)]
    for st in itertools.product(*states):
        st = np.array(st)
        x = np.where(st == 0, lo, np.where(st == 1, np.where(np.isfinite(hi), hi, 0), 0.0))
        F = np.nonzero(st == 2)[0]
        if F.size:
            Bx = np.nonzero(st != 2)[0]
            rhs = -(q[F] + H[np.ix_(F, Bx)] @ x[Bx])
            x[F] = np.linalg.solve(H[np.ix_(F, F)], rhs)
            if np.any(x[F] < lo[F] - 1e-12) or np.any(x[F] > hi[F] + 1e-12):
                continue
        g = H @ x + q
        if np.any(g[st == 0] < -1e-10) or np.any(g[st == 1] > 1e-10):
            continue
        return x
    raise AssertionError("no KKT point found")


def _qp_data(lp, beta, ubar=None, xbar=None):
    e = lp.export()
    A = lp.dense_A()
    ub = np.zeros(lp.M) if ubar is None else ubar
    xb = np.zeros(lp.N) if xbar is None else xbar
    H = beta * A.T @ A + np.eye(lp.N) / beta
    q = e["c"] - A.T @ ub - beta * A.T @ e["b"] - xb / beta
    return H, q, e


@pytest.mark.parametrize("kind,seed,beta", [("vc", 1, 3.0), ("vc", 2, 10.0), ("is", 3, 3.0), ("is", 4, 7.0)])
def test_solve_matches_active_set_enumeration(oracle_mod, kind, seed, beta):
    rng = np.random.default_rng(seed)
    g = synth.er_graph(4, 4, seed)
    w = rng.integers(1, 5, 4).astype(np.float64)
    mk = oracle_mod.OracleLP.vc if kind == "vc" else oracle_mod.OracleLP.is_
    lp = mk(4, g.eu, g.ev, w)
    H, q, e = _qp_data(lp, beta)
    xref = _enumerate_qp(H, q, e["lo"], e["hi"])
    for rule in (0, 1):
        x, info = lp.solve(beta=beta, epochs=200000, tol=1e-13, refresh_every=50, step_rule=rule)
        assert info["converged"], info
        assert np.max(np.abs(x - xref)) < 1e-9
        assert abs(info["fbeta"] - (0.5 * xref @ H @ xref + q @ xref + 0.5 * beta * e["b"] @ e["b"])) < 1e-8


def test_solve_with_ubar_xbar_matches_enumeration(oracle_mod):
    rng = np.random.default_rng(9)
    g = synth.er_graph(4, 5, 9)
    lp = oracle_mod.OracleLP.vc(4, g.eu, g.ev, rng.integers(1, 5, 4).astype(np.float64))
    beta = 4.0
    ub = rng.normal(0, 1, lp.M)
    xb = rng.uniform(0, 1, lp.N)
    H, q, e = _qp_data(lp, beta, ub, xb)
    xref = _enumerate_qp(H, q, e["lo"], e["hi"])
    x, info = lp.solve(beta=beta, epochs=200000, tol=1e-13, refresh_every=50, ubar=ub, xbar=xb)
    assert info["converged"]
    assert np.max(np.abs(x - xref)) < 1e-9


def _lp_pair(lp):
    """A primal-dual optimal pair of the standard form without upper bounds."""
    from scipy.optimize import linprog

    e = lp.export()
    A = lp.dense_A()
    res = linprog(e["c"], A_eq=A, b_eq=e["b"], bounds=[(0, None)] * lp.N, method="highs")
    assert res.status == 0
    return res.x, res.eqlin.marginals, A, e


@pytest.mark.parametrize("seed", [1, 5, 8])
def test_fixed_point_at_lp_pair(oracle_mod, seed):
    """With xbar = x*, ubar = u*, x* solves the LCP of App. A for every beta
    (c - A'u* >= 0 complementary to x* >= 0, Ax* = b), so SCD must return x*."""
    rng = np.random.default_rng(seed)
    g = synth.er_graph(6, 9, seed)
    lp = oracle_mod.OracleLP.vc(6, g.eu, g.ev, rng.integers(1, 5, 6).astype(np.float64))
    xs, us, A, e = _lp_pair(lp)
    assert np.all(xs[:6] <= 1 + 1e-12)  # the [0,1] box is inactive at x*
    x, info = lp.solve(beta=50.0, epochs=300000, tol=1e-13, refresh_every=100, ubar=us, xbar=xs)
    assert info["converged"]
    assert np.max(np.abs(x - xs)) < 1e-8


@pytest.mark.parametrize("seed,beta", [(2, 10.0), (3, 30.0), (4, 100.0)])
def test_theorem1_residual_bound(oracle_mod, seed, beta):
    """Thm. 1: ||A x(beta) - b|| <= (1+sqrt 2) C*/beta and ||x(beta)-x*|| <= sqrt 6 C*."""
    rng = np.random.default_rng(seed)
    g = synth.er_graph(6, 9, seed)
    lp = oracle_mod.OracleLP.vc(6, g.eu, g.ev, rng.integers(1, 5, 6).astype(np.float64))
    xs, us, A, e = _lp_pair(lp)
    Cs = max(np.linalg.norm(xs), np.linalg.norm(us))
    x, info = lp.solve(beta=beta, epochs=2000000, tol=1e-12, refresh_every=200)
    assert info["converged"]
    assert np.all(x[:6] < 1)  # upper bound inactive: the QP is the one of Thm. 1
    assert np.linalg.norm(A @ x - e["b"]) <= (1 + np.sqrt(2)) * Cs / beta + 1e-9
    assert np.linalg.norm(x - xs) <= np.sqrt(6) * Cs + 1e-9


@pytest.mark.parametrize("kind,rule", [("vc", 0), ("is", 0), ("vc", 1), ("mc", 0)])
def test_fbeta_monotone_per_step(oracle_mod, kind, rule):
    if kind == "mc":
        g = synth.grid_graph(4, 4, 3, 2)
        lp = oracle_mod.OracleLP.mc(g.n, g.eu, g.ev, g.ce.astype(np.float64), 3, g.terminals)
    else:
        g = synth.er_graph(30, 70, 3)
        mk = oracle_mod.OracleLP.vc if kind == "vc" else oracle_mod.OracleLP.is_
        lp = mk(30, g.eu, g.ev, np.arange(1, 31, dtype=np.float64) % 7 + 1)
    col, nc = lp.color(0)
    x = lp.initial_x()
    f0 = lp.checks(x, 20.0)["fbeta"]
    for _ in range(3):
        f, x = lp.fbeta_steps(x, 20.0, col, step_rule=rule)
        seq = np.concatenate([[f0], f])
        assert np.all(np.diff(seq) <= 1e-9 * (1 + np.abs(seq[:-1])))
        f0 = f[-1]


def test_mc_solve_matches_slsqp(oracle_mod):
    """Block SCD with simplex projection (App. E) on a tiny multiway-cut QP
    versus scipy SLSQP with explicit simplex equalities."""
    from scipy.optimize import minimize

    eu = np.array([0, 1, 1, 2], np.int32)
    ev = np.array([1, 2, 3, 3], np.int32)
    ce = np.array([1.0, 2.0, 0.5, 1.5])
    k = 2
    lp = oracle_mod.OracleLP.mc(4, eu, ev, ce, k, np.array([0, 3], np.int32))
    beta = 3.0
    H, q, e = _qp_data(lp, beta)
    # simplex equalities for the free vertices; terminals are fixed by their bounds
    cons = [{"type": "eq", "fun": (lambda x, v=v: x[v * k:(v + 1) * k].sum() - 1.0)} for v in (1, 2)]
    bounds = [(lo, hi if np.isfinite(hi) else None) for lo, hi in zip(e["lo"], e["hi"])]
    x0 = lp.initial_x()
    res = minimize(lambda x: 0.5 * x @ H @ x + q @ x, x0, jac=lambda x: H @ x + q, bounds=bounds,
                   constraints=cons, method="SLSQP", options={"ftol": 1e-16, "maxiter": 5000})
    x, info = lp.solve(beta=beta, epochs=200000, tol=1e-13, refresh_every=50)
    assert info["converged"]
    for v in range(4):
        assert abs(x[v * k:(v + 1) * k].sum() - 1) < 1e-12
    assert np.max(np.abs(x - res.x)) < 1e-6
    fo = 0.5 * x @ H @ x + q @ x
    assert fo <= res.fun + 1e-10


def test_lcp_at_convergence(oracle_mod):
    """App. A: the QP solution satisfies 0 <= x - lo  perp  F_beta(x) >= 0 on the box."""
    g = synth.er_graph(12, 25, 7)
    lp = oracle_mod.OracleLP.is_(12, g.eu, g.ev, np.linspace(1, 3, 12))
    beta = 5.0
    x, info = lp.solve(beta=beta, epochs=500000, tol=1e-13, refresh_every=100)
    assert info["converged"]
    H, q, e = _qp_data(lp, beta)
    F = H @ x + q
    at_lo = np.abs(x - e["lo"]) < 1e-12
    at_hi = np.abs(x - e["hi"]) < 1e-12
    free = ~at_lo & ~at_hi
    assert np.all(np.abs(F[free]) < 1e-9)
    assert np.all(F[at_lo] > -1e-9)
    assert np.all(F[at_hi] < 1e-9)


def test_cfg1_shape_runs(oracle_mod):
    """Vertex cover on G(2000, 8000): 50 epochs reduce f_beta and rho monotonically
    at the refresh points, and the count of free coordinates is N."""
    g = synth.er_graph(2000, 8000, 1)
    g.w = synth.int_weights(2000, 1, 10, np.random.default_rng(1))
    lp = oracle_mod.build_problem("vc", g)
    assert lp.free_coords == 10000 and lp.nnz == 24000
    x, info = lp.solve(beta=100.0, epochs=50, refresh_every=10)
    tr = info["trace"]
    assert tr.shape[0] == 5
    assert np.all(np.diff(tr[:, 3]) < 0)
    assert info["rho"] < tr[0, 1]

"""Oracle pins for the augmented-Lagrangian outer loop of Sec. 3.4 (proximal
method of multipliers around eq. QP): the iterates reach the LP optimum with
Ax = b, the multiplier estimate closes the duality gap (bound terms included),
the infeasibility falls far below the Theta(1/beta) floor of the fixed-beta
penalty (Thm. 1), and an optimal primal-dual pair is a fixed point."""
import numpy as np
import pytest
from scipy.optimize import linprog

from paper_1311_2661_gb300 import synth


def _instances(oracle_mod):
    out = []
    # K_5 and C_7, unit weights: LP* = n/2 (all one half)
    k5 = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    c7 = [(i, (i + 1) % 7) for i in range(7)]
    for n, edges in ((5, k5), (7, c7)):
        eu = np.array([e[0] for e in edges], np.int32)
        ev = np.array([e[1] for e in edges], np.int32)
        out.append(("vc", oracle_mod.OracleLP.vc(n, eu, ev, np.ones(n)), n / 2))
    # a random graph with integer weights, VC and IS; LP* from HiGHS
    g = synth.er_graph(12, 24, 5)
    w = synth.int_weights(12, 1, 10, np.random.default_rng(3)).astype(np.float64)
    out.append(("vc", oracle_mod.OracleLP.vc(12, g.eu, g.ev, w), None))
    out.append(("is", oracle_mod.OracleLP.is_(12, g.eu, g.ev, w), None))
    return out


def _lp_opt(lp):
    e = lp.export()
    A = lp.dense_A()
    res = linprog(e["c"], A_eq=A, b_eq=e["b"], bounds=list(zip(e["lo"], np.where(np.isinf(e["hi"]), None, e["hi"]))),
                  method="highs")
    assert res.status == 0
    return res.fun


def _dual_objective(lp, u):
    """LP dual value of the multiplier estimate u: b'u plus the bound terms of
    the reduced costs d = c - A'u (lo_j = 0 for every column here)."""
    e = lp.export()
    d = e["c"] - lp.dense_A().T @ u
    fin = np.isfinite(e["hi"])
    return e["b"] @ u + np.sum(e["hi"][fin] * np.minimum(d[fin], 0.0)) + np.sum(e["lo"] * np.maximum(d, 0.0))


@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_al_reaches_lp_optimum_and_closes_duality_gap(oracle_mod, idx):
    kind, lp, lp_star = _instances(oracle_mod)[idx]
    if lp_star is None:
        lp_star = _lp_opt(lp)
    x, u, hist = lp.solve_al(beta=10.0, epochs=200000, tol=1e-12, refresh_every=10, outer=80)
    obj = lp.export()["c"] @ x
    assert np.max(np.abs(lp.residual(x))) <= 1e-6
    assert abs(obj - lp_star) <= 1e-5 * max(1.0, abs(lp_star))
    # the multiplier estimate is dual optimal: its dual value equals LP*
    assert abs(_dual_objective(lp, u) - lp_star) <= 1e-5 * max(1.0, abs(lp_star))
    # outer iterations shrink the infeasibility
    infeas = [h["infeas"] for h in hist]
    assert infeas[-1] < 1e-3 * infeas[0]


def test_al_far_below_fixed_penalty(oracle_mod):
    """Thm. 1: at fixed beta the penalty solution keeps ||Ax - b|| = Theta(1/beta);
    the multiplier updates remove that floor."""
    kind, lp, _ = _instances(oracle_mod)[2]
    x_pen, info_pen = lp.solve(beta=10.0, epochs=200000, tol=1e-12, refresh_every=10)
    x_al, _, _ = lp.solve_al(beta=10.0, epochs=200000, tol=1e-12, refresh_every=10, outer=30)
    pen = np.max(np.abs(lp.residual(x_pen)))
    al = np.max(np.abs(lp.residual(x_al)))
    assert pen > 1e-3  # the floor is there
    assert al < 1e-3 * pen


def test_al_optimal_pair_is_a_fixed_point(oracle_mod):
    kind, lp, _ = _instances(oracle_mod)[0]
    x, u, _ = lp.solve_al(beta=10.0, epochs=200000, tol=1e-12, refresh_every=10, outer=80)
    x2, u2, hist = lp.solve_al(beta=10.0, epochs=200000, tol=1e-12, refresh_every=10, outer=1, ubar=u, xbar=x, x0=x)
    assert np.max(np.abs(x2 - x)) <= 1e-8
    assert np.max(np.abs(u2 - u)) <= 1e-6


def test_al_growth_multiplies_beta(oracle_mod):
    kind, lp, _ = _instances(oracle_mod)[1]
    _, _, hist = lp.solve_al(beta=2.0, epochs=50, refresh_every=10, outer=4, beta_growth=3.0)
    assert [h["beta"] for h in hist] == [2.0, 6.0, 18.0, 54.0]

"""Augmented-Lagrangian outer loop on the GPU (thetis_solve_al, Sec. 3.4)
against the FP64 oracle's loop: iterates, per-outer infeasibility and the
multiplier estimate, then convergence to the LP optimum."""
import numpy as np
import pytest
from scipy.optimize import linprog

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import X_TOL, build_gpu, gpu, is_graph, vc_graph

pytestmark = pytest.mark.gpu


def _full_x(h):
    return np.concatenate([h.get_x(), h.get_slack()]).astype(np.float64)


@pytest.mark.parametrize("kind,n,m,growth", [("vc", 300, 900, 1.0), ("is", 400, 1500, 1.0), ("vc", 250, 700, 2.0)])
def test_al_matches_oracle(kind, n, m, growth):
    T = gpu()
    g = vc_graph(n, m, 4) if kind == "vc" else is_graph(n, m, 4)
    beta, outer, epochs = 20.0, 4, 30
    h = build_gpu(kind, g, seed=5)
    info, hist = h.solve_al(beta=beta, epochs=epochs, refresh_every=10, outer=outer, beta_growth=growth)
    lp = oracle.build_problem(kind, g)
    x_o, u_o, hist_o = lp.solve_al(beta=beta, epochs=epochs, refresh_every=10, outer=outer, beta_growth=growth,
                                   color=lp.color(5)[0])
    assert info["epochs_run"] == outer * epochs
    assert np.max(np.abs(_full_x(h) - x_o)) <= X_TOL
    for k in range(outer):
        assert abs(hist["infeas"][k] - hist_o[k]["infeas"]) <= 4 * X_TOL
    # |d ubar| <= sum_k beta_k * max_i |d r_i| <= sum_k beta_k * (row nnz = 3) * X_TOL
    u_tol = 3 * X_TOL * sum(beta * growth ** k for k in range(outer))
    assert np.max(np.abs(h.duals().astype(np.float64) - u_o)) <= u_tol


def test_al_reaches_lp_optimum():
    T = gpu()
    g = synth.er_graph(60, 150, 8)
    g.w = synth.int_weights(60, 1, 10, np.random.default_rng(8))
    lp = oracle.build_problem("vc", g)
    e = lp.export()
    res = linprog(e["c"], A_eq=lp.dense_A(), b_eq=e["b"],
                  bounds=list(zip(e["lo"], np.where(np.isinf(e["hi"]), None, e["hi"]))), method="highs")
    h = build_gpu("vc", g, seed=1)
    info, hist = h.solve_al(beta=10.0, epochs=5000, tol=1e-5, refresh_every=10, outer=40)
    x = _full_x(h)
    # FP32 iterate: the LP optimum to ~1e-4, and the penalty floor gone
    assert hist["infeas"][-1] <= 1e-4
    assert abs(e["c"] @ x - res.fun) <= 1e-3 * abs(res.fun)
    assert hist["infeas"][-1] < 1e-2 * hist["infeas"][0]


def test_al_rejects_bad_arguments():
    T = gpu()
    g = vc_graph(50, 100, 1)
    h = build_gpu("vc", g)
    with pytest.raises(T.ThetisError):
        h.solve_al(outer=0)
    with pytest.raises(T.ThetisError):
        h.solve_al(outer=2, beta_growth=0.5)
    hb = T.thetis_build_batch_graphs([("vc", g), ("is", g)])
    with pytest.raises(T.ThetisError):
        hb.solve_al(outer=2)
    h2 = build_gpu("vc", g)
    with pytest.raises(T.ThetisError):  # no multiplier yet
        h2.duals()

"""Pairwise MAP on the GPU (thetis_build_map, Sec. 4.1) against the FP64
oracle: colouring, iterates and node rounding on the same point; MAP
recovered on a chain; input checks."""
import numpy as np
import pytest

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import X_TOL, gpu, rel

pytestmark = pytest.mark.gpu


def _pair(g, seed=0):
    T = gpu()
    h = T.thetis_build_map(g.n, g.k, g.eu, g.ev, g.theta_node, g.theta_edge, seed=seed)
    lp = oracle.OracleLP.map_lp(g.n, g.k, g.eu, g.ev, g.theta_node.astype(np.float64),
                                g.theta_edge.astype(np.float64))
    return h, lp


@pytest.mark.parametrize("n,k,seed", [(300, 5, 1), (500, 3, 2), (120, 8, 3)])
def test_map_colouring_iterates_and_rounding(n, k, seed):
    T = gpu()
    g = synth.skip_chain_crf(n, k, 20, 0.1, seed)
    h, lp = _pair(g, seed=3)
    col, _ = lp.color(3)
    assert np.array_equal(h.colors(), col)
    h.solve(beta=100.0, epochs=40, refresh_every=10)
    x_o, _ = lp.solve(beta=100.0, epochs=40, refresh_every=10, color=col)
    x = h.get_x().astype(np.float64)
    assert np.max(np.abs(x - x_o)) <= X_TOL
    lab, ri = h.round()
    r = lp.round_map(x)
    assert np.array_equal(lab, r["labels"]) and ri["valid"]
    assert rel(ri["obj"], r["obj"]) <= 1e-12


def _viterbi(n, k, th_n, th_e):
    score = th_n[0].copy()
    back = np.zeros((n, k), np.int64)
    for i in range(1, n):
        cand = score[:, None] + th_e[i - 1]
        back[i] = np.argmax(cand, axis=0)
        score = cand[back[i], np.arange(k)] + th_n[i]
    lab = np.zeros(n, np.int64)
    lab[-1] = int(np.argmax(score))
    for i in range(n - 1, 0, -1):
        lab[i - 1] = back[i][lab[i]]
    return float(score.max()), lab


def test_map_chain_solved_exactly():
    """On a chain the local polytope is tight: the augmented-Lagrangian solve
    and node rounding give the Viterbi labelling."""
    T = gpu()
    rng = np.random.default_rng(4)
    n, k = 200, 4
    eu = np.arange(n - 1, dtype=np.int32)
    ev = eu + 1
    tn = rng.normal(size=(n, k)).astype(np.float32)
    te = rng.normal(scale=0.7, size=(n - 1, k, k)).astype(np.float32)
    h = T.thetis_build_map(n, k, eu, ev, tn, te)
    h.solve_al(beta=10.0, epochs=4000, tol=1e-5, refresh_every=10, outer=30)
    lab, ri = h.round()
    best, vlab = _viterbi(n, k, tn.astype(np.float64), te.astype(np.float64))
    assert np.array_equal(lab, vlab)
    assert abs(-ri["obj"] - best) <= 1e-9 * abs(best) + 1e-9


def test_map_bad_inputs():
    T = gpu()
    eu, ev = np.array([0], np.int32), np.array([1], np.int32)
    tn, te = np.zeros((2, 3), np.float32), np.zeros((1, 3, 3), np.float32)
    with pytest.raises(T.ThetisError):
        T.thetis_build_map(2, 1, eu, ev, tn[:, :1], te[:, :1, :1])
    with pytest.raises(T.ThetisError):
        T.thetis_build_map(2, 33, eu, ev, np.zeros((2, 33), np.float32), np.zeros((1, 33, 33), np.float32))
    with pytest.raises(T.ThetisError):  # loop
        T.thetis_build_map(2, 3, eu, eu, tn, te)
    bad = tn.copy()
    bad[1, 2] = np.inf
    with pytest.raises(T.ThetisError):
        T.thetis_build_map(2, 3, eu, ev, bad, te)

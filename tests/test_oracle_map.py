"""Oracle pins for pairwise MAP as an LP (Sec. 4.1: the local-polytope
relaxation with node rounding): exact on trees (Viterbi on chains), brute
force on tiny graphs, a relaxation on cycles, and the augmented-Lagrangian
solve followed by node rounding recovering the MAP labels of a chain."""
import itertools

import numpy as np
import pytest
from scipy.optimize import linprog


def _chain(n, k, seed):
    rng = np.random.default_rng(seed)
    eu = np.arange(n - 1, dtype=np.int32)
    ev = np.arange(1, n, dtype=np.int32)
    return eu, ev, rng.normal(size=(n, k)), rng.normal(scale=0.7, size=(n - 1, k, k))


def _viterbi(n, k, th_n, th_e):
    """Max-sum dynamic programming on a chain: (best score, labels)."""
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


def _brute(n, k, eu, ev, th_n, th_e):
    best = -np.inf
    for lab in itertools.product(range(k), repeat=n):
        lab = np.array(lab)
        sc = th_n[np.arange(n), lab].sum() + th_e[np.arange(len(eu)), lab[eu], lab[ev]].sum()
        best = max(best, sc)
    return best


def _lp(lp):
    """The LP with its simplex blocks written as rows (the method projects onto
    them instead), solved by HiGHS."""
    e = lp.export()
    n, k = lp.map_meta[0], lp.map_meta[1]
    S = np.zeros((n, e["c"].shape[0]))
    for i in range(n):
        S[i, i * k:(i + 1) * k] = 1.0
    A = np.vstack([lp.dense_A(), S])
    b = np.concatenate([e["b"], np.ones(n)])
    res = linprog(e["c"], A_eq=A, b_eq=b, bounds=list(zip(e["lo"], e["hi"])), method="highs")
    assert res.status == 0
    return res.x, res.fun


@pytest.mark.parametrize("n,k,seed", [(6, 3, 1), (8, 2, 2), (5, 4, 3)])
def test_chain_lp_is_tight_and_rounds_to_viterbi(oracle_mod, n, k, seed):
    eu, ev, th_n, th_e = _chain(n, k, seed)
    lp = oracle_mod.OracleLP.map_lp(n, k, eu, ev, th_n, th_e)
    x, val = _lp(lp)
    best, lab = _viterbi(n, k, th_n, th_e)
    assert abs(-val - best) < 1e-8                 # local polytope exact on a tree
    r = lp.round_map(x)
    assert np.array_equal(r["labels"], lab) and abs(-r["obj"] - best) < 1e-9
    assert abs(best - _brute(n, k, eu, ev, th_n, th_e)) < 1e-9


def test_single_edge_brute_force(oracle_mod):
    rng = np.random.default_rng(5)
    th_n, th_e = rng.normal(size=(2, 3)), rng.normal(size=(1, 3, 3))
    lp = oracle_mod.OracleLP.map_lp(2, 3, [0], [1], th_n, th_e)
    _, val = _lp(lp)
    assert abs(-val - _brute(2, 3, np.array([0]), np.array([1]), th_n, th_e)) < 1e-9


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_cycle_lp_is_a_relaxation(oracle_mod, seed):
    """A cycle with a skip edge: LP optimum >= MAP score (upper bound on the
    score, i.e. a lower bound on the minimised objective), and the rounded
    labels score no more than the MAP."""
    rng = np.random.default_rng(seed)
    n, k = 6, 2
    eu = np.array([0, 1, 2, 3, 4, 5, 0], np.int32)
    ev = np.array([1, 2, 3, 4, 5, 0, 3], np.int32)
    th_n = rng.normal(size=(n, k))
    th_e = rng.normal(scale=1.5, size=(len(eu), k, k))
    lp = oracle_mod.OracleLP.map_lp(n, k, eu, ev, th_n, th_e)
    x, val = _lp(lp)
    best = _brute(n, k, eu, ev, th_n, th_e)
    assert -val >= best - 1e-9
    assert -lp.round_map(x)["obj"] <= best + 1e-9


def test_al_solve_and_node_rounding_recover_the_chain_map(oracle_mod):
    n, k = 12, 3
    eu, ev, th_n, th_e = _chain(n, k, 9)
    lp = oracle_mod.OracleLP.map_lp(n, k, eu, ev, th_n, th_e)
    x, u, hist = lp.solve_al(beta=10.0, epochs=100000, tol=1e-11, refresh_every=10, outer=60)
    best, lab = _viterbi(n, k, th_n, th_e)
    assert abs(lp.export()["c"] @ x + best) < 1e-5 and np.max(np.abs(lp.residual(x))) < 1e-6
    assert np.array_equal(lp.round_map(x)["labels"], lab)

"""Set cover on the GPU (thetis_build_sc, App. B.1) against the FP64 oracle:
colouring, iterates, the covering repair and both roundings bit-exact on the
same x, validity, and input checks."""
import numpy as np
import pytest

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import X_TOL, gpu

pytestmark = pytest.mark.gpu


def _pair(ss, seed=0):
    T = gpu()
    h = T.thetis_build_sc(ss.n_elements, ss.ptr, ss.elems, ss.cost, seed=seed)
    lp = oracle.OracleLP.set_cover(ss.n_elements, ss.ptr, ss.elems, ss.cost.astype(np.float64))
    return h, lp


@pytest.mark.parametrize("n_elem,n_sets,f_lo,f_hi", [(3000, 800, 1, 6), (5000, 300, 2, 8), (800, 2000, 1, 3)])
def test_sc_colouring_iterates_and_rounding(n_elem, n_sets, f_lo, f_hi):
    T = gpu()
    ss = synth.set_cover_instance(n_elem, n_sets, f_lo, f_hi, n_elem + n_sets)
    h, lp = _pair(ss, seed=4)
    col, _ = lp.color(4)
    assert np.array_equal(h.colors(), col)
    info = h.solve(beta=100.0, epochs=40, refresh_every=10)
    x_o, info_o = lp.solve(beta=100.0, epochs=40, refresh_every=10, color=col)
    x = np.concatenate([h.get_x(), h.get_slack()]).astype(np.float64)
    assert np.max(np.abs(x - x_o)) <= X_TOL
    assert abs(info["rho"] - info_o["rho"]) <= 1e-4
    # rounding on the GPU's own iterate: bit-exact with the oracle
    xs = h.get_x().astype(np.float64)
    lab, ri = h.round(kind=T.ROUND_SC)
    r = lp.round_sc(xs)
    assert r["status"] == 0 and ri["valid"] and lp.valid_sc(lab)
    assert np.array_equal(lab, r["labels"]) and ri["obj"] == r["obj"] and ri["repair"] == r["eps"]
    assert ri["near"] == r["near"]
    lab2, ri2 = h.round(kind=T.ROUND_SC_RAND, seed=9, reps=10)
    r2 = lp.round_sc_rand(xs, 9, 10)
    assert ri2["valid"] and lp.valid_sc(lab2)
    assert np.array_equal(lab2, r2["labels"]) and ri2["obj"] == r2["obj"] and ri2["best_rep"] == r2["best_rep"]


def test_sc_converged_rounding_within_f_of_lp():
    """Solved to rho <= 1e-4: the f-threshold cover costs at most f times the
    (repaired) LP cost at the rounded point."""
    T = gpu()
    ss = synth.set_cover_instance(4000, 600, 1, 4, 7)
    h, lp = _pair(ss)
    info = h.solve(beta=100.0, epochs=20000, tol=1e-4, refresh_every=10)
    assert info["converged"]
    lab, ri = h.round(kind=T.ROUND_SC)
    f = lp.sc_frequency()
    xt = np.minimum(1.0, h.get_x().astype(np.float64) / (1 - ri["repair"]))
    assert ri["valid"] and ri["obj"] <= f * float(ss.cost.astype(np.float64) @ xt) + 1e-6


def test_sc_repair_impossible_and_bad_inputs():
    T = gpu()
    ss = synth.set_cover_instance(100, 40, 1, 3, 1)
    h = T.thetis_build_sc(ss.n_elements, ss.ptr, ss.elems, ss.cost)
    lab, ri = h.round(kind=T.ROUND_SC)  # x = 0 before any solve: eps = 1
    assert lab is None and ri["status"] == T.THETIS_E_REPAIR
    with pytest.raises(T.ThetisError):  # wrong rounding kind for the problem
        h.round(kind=T.ROUND_VC)
    # element 0 in no set
    with pytest.raises(T.ThetisError):
        T.thetis_build_sc(3, np.array([0, 1, 2]), np.array([1, 2], np.int32), np.ones(2, np.float32))
    # repeated element inside a set
    with pytest.raises(T.ThetisError):
        T.thetis_build_sc(2, np.array([0, 2, 3]), np.array([1, 1, 0], np.int32), np.ones(2, np.float32))
    # element id out of range
    with pytest.raises(T.ThetisError):
        T.thetis_build_sc(2, np.array([0, 1, 2]), np.array([0, 5], np.int32), np.ones(2, np.float32))
    # non-positive cost
    with pytest.raises(T.ThetisError):
        T.thetis_build_sc(2, np.array([0, 1, 2]), np.array([0, 1], np.int32), np.array([1, 0], np.float32))

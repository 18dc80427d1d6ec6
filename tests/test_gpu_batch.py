"""Batched solves (thetis_build_batch): every instance of a block-diagonal batch
is coloured, swept and rounded as it would be alone -- checked against the
single-instance GPU path and against the FP64 oracle instance by instance."""
import numpy as np
import pytest

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import OBJ_RTOL, X_TOL, gpu, rel

pytestmark = pytest.mark.gpu


def _batch(count=24, seed=3, nmax=600):
    rng = np.random.default_rng(seed)
    items = []
    for t in range(count):
        n = int(rng.integers(1, nmax)) if t != 5 else 1
        dmax = min(n - 1, 12)
        m = 0 if (n < 2 or t == 7) else int(rng.integers(0, n * dmax // 2 + 1))
        m = min(m, n * (n - 1) // 2)
        g = synth.er_graph(n, m, int(rng.integers(1 << 30)))
        g.w = synth.int_weights(n, 1, 10, np.random.default_rng(t))
        items.append(("vc" if t % 2 == 0 else "is", g))
    return items


def _slices(items):
    noff = np.concatenate([[0], np.cumsum([g.n for _, g in items])])
    eoff = np.concatenate([[0], np.cumsum([g.m for _, g in items])])
    return noff, eoff


def test_batch_colouring_equals_alone_and_oracle():
    T = gpu()
    items = _batch()
    hb = T.thetis_build_batch_graphs(items, seed=11)
    cb = hb.colors()
    noff, eoff = _slices(items)
    Nv = noff[-1]
    for t, (kind, g) in enumerate(items):
        mine = np.concatenate([cb[noff[t]:noff[t + 1]], cb[Nv + eoff[t]:Nv + eoff[t + 1]]])
        lp = oracle.build_problem(kind, g)
        col, _ = lp.color(11)
        assert np.array_equal(mine, col), t
        b = T.thetis_build_vc if kind == "vc" else T.thetis_build_is
        h = b(g.n, g.eu, g.ev, g.w, seed=11)
        assert np.array_equal(mine, h.colors()), t


@pytest.mark.parametrize("engine", [0, 1])
def test_batch_iterates_and_rounding_match_oracle(engine):
    T = gpu()
    items = _batch(seed=4)
    hb = T.thetis_build_batch_graphs(items, seed=2, device=True)
    info = hb.solve(beta=100.0, epochs=40, refresh_every=10, engine=engine)
    x = hb.get_x().astype(np.float64)
    s = hb.get_slack().astype(np.float64)
    lab, obj, status, best = T.thetis_round_batch(hb, seed=9, reps=10)
    noff, eoff = _slices(items)
    rho_max = 0.0
    for t, (kind, g) in enumerate(items):
        lp = oracle.build_problem(kind, g)
        col, _ = lp.color(2)
        x_o, info_o = lp.solve(beta=100.0, epochs=40, refresh_every=10, color=col)
        mine = np.concatenate([x[noff[t]:noff[t + 1]], s[eoff[t]:eoff[t + 1]]])
        assert np.max(np.abs(mine - x_o)) <= X_TOL, t
        assert rel(lp.checks(mine, 100.0)["fbeta"], info_o["fbeta"]) <= OBJ_RTOL, t
        rho_max = max(rho_max, lp.checks(mine, 100.0)["rho"])
        xv = x[noff[t]:noff[t + 1]]
        r = lp.round_vc(xv) if kind == "vc" else lp.round_is(xv, 9, 10)
        if kind == "vc" and r["status"] == 6:
            assert status[t] == -1
            continue
        assert status[t] == 1 and lp.valid(lab[noff[t]:noff[t + 1]])
        assert np.array_equal(lab[noff[t]:noff[t + 1]], r["labels"]), t
        assert obj[t] == r["obj"], t
        if kind == "is":
            assert best[t] == r["best_rep"], t
    assert abs(info["rho"] - rho_max) <= 1e-6


def test_batch_to_tolerance_every_instance_converged():
    T = gpu()
    items = _batch(count=16, seed=8, nmax=400)
    hb = T.thetis_build_batch_graphs(items, seed=0)
    info = hb.solve(beta=100.0, epochs=5000, tol=1e-3, refresh_every=10)
    assert info["converged"] and info["rho"] <= 1e-3
    x, s = hb.get_x().astype(np.float64), hb.get_slack().astype(np.float64)
    noff, eoff = _slices(items)
    for t, (kind, g) in enumerate(items):
        lp = oracle.build_problem(kind, g)
        mine = np.concatenate([x[noff[t]:noff[t + 1]], s[eoff[t]:eoff[t + 1]]])
        assert lp.checks(mine, 100.0)["rho"] <= 1e-3 + 1e-6


def test_batch_rejects_bad_input():
    T = gpu()
    with pytest.raises(T.ThetisError):  # local endpoint beyond its instance
        T.thetis_build_batch(np.array([0, 1], np.uint8), np.array([0, 2, 4]), np.array([0, 1, 2]),
                             np.array([0, 2], np.int32), np.array([1, 3], np.int32), np.ones(4, np.float32))
    with pytest.raises(T.ThetisError):  # bad kind
        T.thetis_build_batch(np.array([7], np.uint8), np.array([0, 2]), np.array([0, 1]),
                             np.array([0], np.int32), np.array([1], np.int32), np.ones(2, np.float32))


def test_batch_instances_stop_where_alone_stops():
    """tol applies per instance: each instance stops at the first check where its
    own rho <= tol -- the same check, iterate and rho as its solve alone -- and
    is no longer swept while the rest of the batch continues."""
    T = gpu()
    items = _batch(count=20, seed=12, nmax=500)
    hb = T.thetis_build_batch_graphs(items, seed=3)
    info = hb.solve(beta=100.0, epochs=3000, tol=1e-3, refresh_every=10)
    ep, rho = T.thetis_batch_info(hb)
    assert info["converged"] and info["rho"] == rho.max() and info["epochs_run"] == ep.max()
    x, s = hb.get_x().astype(np.float64), hb.get_slack().astype(np.float64)
    noff, eoff = _slices(items)
    assert len(set(ep.tolist())) > 1, "every instance stopped at the same check"
    for t, (kind, g) in enumerate(items):
        b = T.thetis_build_vc if kind == "vc" else T.thetis_build_is
        h = b(g.n, g.eu, g.ev, g.w, seed=3)
        ia = h.solve(beta=100.0, epochs=3000, tol=1e-3, refresh_every=10)
        assert ia["epochs_run"] == ep[t], t
        assert abs(ia["rho"] - rho[t]) <= 1e-9 + 1e-6 * rho[t], t
        xa = np.concatenate([h.get_x(), h.get_slack()]).astype(np.float64)
        mine = np.concatenate([x[noff[t]:noff[t + 1]], s[eoff[t]:eoff[t + 1]]])
        assert np.max(np.abs(mine - xa)) <= X_TOL, t
        # and the FP64 oracle, run to the same epoch count in the same colour order
        lp = oracle.build_problem(kind, g)
        col, _ = lp.color(3)
        x_o, _ = lp.solve(beta=100.0, epochs=int(ep[t]), refresh_every=10, color=col)
        assert np.max(np.abs(mine - x_o)) <= X_TOL, t
        assert lp.checks(mine, 100.0)["rho"] <= 1e-3 + 1e-6

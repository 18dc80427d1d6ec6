"""Batched solves (thetis_build_batch): every instance of a block-diagonal batch
is coloured, swept and rounded as it would be alone -- checked against the
single-instance GPU path and against the FP64 oracle instance by instance.
Engine 0 (the default) is the instance-resident engine (one CTA or cluster per
instance); engines 1 and 2 sweep the whole block-diagonal LP."""
import numpy as np
import pytest

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import OBJ_RTOL, X_TOL, gpu, rel

pytestmark = pytest.mark.gpu

# rho of one instance in a batch against its solve alone: the two sum every
# column's dot product in a different FP32 order, so their iterates differ at
# FP32 rounding level and rho (an FP64 function of the iterate) by ~1e-8
RHO_ATOL = 1e-7


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


@pytest.mark.parametrize("engine", [0, 1, 2])
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
        # the batch sums each column's dot in another FP32 order than the solve
        # alone: the iterates agree to FP32 rounding, rho to ~1e-7
        assert abs(ia["rho"] - rho[t]) <= RHO_ATOL, t
        xa = np.concatenate([h.get_x(), h.get_slack()]).astype(np.float64)
        mine = np.concatenate([x[noff[t]:noff[t + 1]], s[eoff[t]:eoff[t + 1]]])
        assert np.max(np.abs(mine - xa)) <= X_TOL, t
        # and the FP64 oracle, run to the same epoch count in the same colour order
        lp = oracle.build_problem(kind, g)
        col, _ = lp.color(3)
        x_o, _ = lp.solve(beta=100.0, epochs=int(ep[t]), refresh_every=10, color=col)
        assert np.max(np.abs(mine - x_o)) <= X_TOL, t
        assert lp.checks(mine, 100.0)["rho"] <= 1e-3 + 1e-6


def _sized_items(sizes, seed):
    """One ER instance per (kind, n, m), weights U[1, 10]."""
    rng = np.random.default_rng(seed)
    items = []
    for kind, n, m in sizes:
        g = synth.er_graph(n, m, int(rng.integers(1 << 30)))
        g.w = synth.int_weights(n, 1, 10, rng)
        items.append((kind, g))
    return items


# instances for every launch class of the instance-resident engine: r and x
# of 4 (n + m) bytes fit one CTA of 256, 512 or 1024 threads, or span a
# cluster of 2, 3 or 4 CTAs (distributed shared memory and halo buffers; x in
# shared memory, or in global memory where that saves a CTA: the (20000,
# 100000) and (19000, 140000) instances), or (without clusters) one CTA keeps
# x and part of r in global memory
CLASS_SIZES = [("vc", 300, 1000), ("is", 3000, 20000), ("vc", 8000, 40000), ("is", 15000, 70000),
               ("vc", 20000, 150000), ("is", 19000, 140000), ("vc", 18000, 130000),
               ("is", 21000, 160000), ("vc", 20000, 100000)]


@pytest.mark.parametrize("step_rule,lanes,clusters", [(0, 1, 0), (1, 1, 0), (0, 1, 1), (1, 8, 1), (0, 4, 0)])
def test_instance_engine_every_launch_class_matches_oracle(step_rule, lanes, clusters):
    T = gpu()
    items = _sized_items(CLASS_SIZES, 31)
    hb = T.thetis_build_batch_graphs(items, seed=6, device=True)
    T.thetis_set_batch_shape(hb, lanes, clusters)
    info = hb.solve(beta=100.0, epochs=30, refresh_every=10, step_rule=step_rule)
    assert info["epochs_run"] == 30
    x = hb.get_x().astype(np.float64)
    s = hb.get_slack().astype(np.float64)
    noff, eoff = _slices(items)
    for t, (kind, g) in enumerate(items):
        lp = oracle.build_problem(kind, g)
        x_o, info_o = lp.solve(beta=100.0, epochs=30, refresh_every=10, step_rule=step_rule, color=lp.color(6)[0])
        mine = np.concatenate([x[noff[t]:noff[t + 1]], s[eoff[t]:eoff[t + 1]]])
        assert np.max(np.abs(mine - x_o)) <= X_TOL, t
        assert rel(lp.checks(mine, 100.0)["fbeta"], info_o["fbeta"]) <= OBJ_RTOL, t
    # the union sweep on the same batch agrees with it to tolerance
    hu = T.thetis_build_batch_graphs(items, seed=6, device=True)
    hu.solve(beta=100.0, epochs=30, refresh_every=10, step_rule=step_rule, engine=2)
    start, ctas = T.thetis_batch_placement(hu)
    assert not start.any() and not ctas.any()
    assert np.max(np.abs(hu.get_x() - hb.get_x())) <= X_TOL


@pytest.mark.parametrize("clusters", [0, 1])
def test_instance_engine_classes_stop_where_alone_stops(clusters):
    T = gpu()
    items = _sized_items(CLASS_SIZES, 32)
    hb = T.thetis_build_batch_graphs(items, seed=1)
    T.thetis_set_batch_shape(hb, 1, clusters)
    info = hb.solve(beta=100.0, epochs=3000, tol=1e-3, refresh_every=20)
    ep, rho = T.thetis_batch_info(hb)
    done = T.thetis_batch_latency(hb)
    assert info["converged"] and np.all(rho <= 1e-3)
    assert np.all(done > 0) and np.all(done <= info["solve_ms"] + 1e-6)
    start, ctas = T.thetis_batch_placement(hb)
    assert np.all(start >= 0) and np.all(start < done)
    # one CTA unless r does not fit one CTA's shared memory (clusters on)
    assert np.all(ctas[:3 if clusters else len(items)] == 1)
    if clusters:
        assert np.all((ctas[3:] >= 2) & (ctas[3:] <= 4))
    x, s = hb.get_x().astype(np.float64), hb.get_slack().astype(np.float64)
    noff, eoff = _slices(items)
    for t, (kind, g) in enumerate(items):
        b = T.thetis_build_vc if kind == "vc" else T.thetis_build_is
        h = b(g.n, g.eu, g.ev, g.w, seed=1)
        ia = h.solve(beta=100.0, epochs=3000, tol=1e-3, refresh_every=20)
        assert ia["epochs_run"] == ep[t], t
        assert abs(ia["rho"] - rho[t]) <= RHO_ATOL, t
        xa = np.concatenate([h.get_x(), h.get_slack()]).astype(np.float64)
        mine = np.concatenate([x[noff[t]:noff[t + 1]], s[eoff[t]:eoff[t + 1]]])
        assert np.max(np.abs(mine - xa)) <= X_TOL, t


def test_batched_workload_shape_parity_sample():
    """The batched benchmark's distribution (ER, n ~ U[200, 20000], average
    degree ~ U[4, 16], half VC half IS), 256 instances solved to rho <= 1e-3:
    every instance's rho checked by the oracle at the GPU iterate, and a seeded
    sample of 8 compared with the oracle's own solve element by element."""
    T = gpu()
    items = synth.batch_instances(256, 200, 20000, 4.0, 16.0, 1, 10, 77)
    hb = T.thetis_build_batch_graphs(items, seed=0, device=True)
    info = hb.solve(beta=100.0, epochs=4000, tol=1e-3, refresh_every=20)
    ep, rho = T.thetis_batch_info(hb)
    assert info["converged"] and np.all(rho <= 1e-3)
    x, s = hb.get_x().astype(np.float64), hb.get_slack().astype(np.float64)
    lab, obj, status, best = T.thetis_round_batch(hb, seed=4, reps=10)
    assert np.all(status == 1)
    noff, eoff = _slices(items)
    sample = set(np.random.default_rng(5).choice(len(items), 8, replace=False).tolist())
    for t, (kind, g) in enumerate(items):
        lp = oracle.build_problem(kind, g)
        mine = np.concatenate([x[noff[t]:noff[t + 1]], s[eoff[t]:eoff[t + 1]]])
        chk = lp.checks(mine, 100.0)
        assert chk["rho"] <= 1e-3 + 1e-9, t
        assert abs(chk["rho"] - rho[t]) <= 1e-9 + 1e-6 * rho[t], t
        assert lp.valid(lab[noff[t]:noff[t + 1]]), t
        if t in sample:
            x_o, info_o = lp.solve(beta=100.0, epochs=int(ep[t]), refresh_every=20, color=lp.color(0)[0])
            assert np.max(np.abs(mine - x_o)) <= X_TOL, t
            assert info_o["rho"] <= 1e-3 + 1e-6, t


@pytest.mark.parametrize("lanes,clusters,epochs", [(1, 0, 40), (1, 1, 40), (4, 0, 25), (1, 0, 0)])
def test_rounding_inside_the_instance_kernel_equals_round_batch(lanes, clusters, epochs):
    """thetis_solve_round_batch rounds every instance in its own CTA / cluster
    the moment it stops (repair, VC threshold / IS best of reps with
    alterations, exact validity): labels, objectives, best repetitions and
    statuses equal thetis_round_batch on the same iterate, bit for bit --
    including the VC repair failure of an unsolved iterate (epochs = 0)."""
    T = gpu()
    items = _sized_items(CLASS_SIZES, 41) + _batch(count=12, seed=9, nmax=500)
    outs = []
    for fused in (True, False):
        hb = T.thetis_build_batch_graphs(items, seed=5, device=True)
        T.thetis_set_batch_shape(hb, lanes, clusters)
        kw = dict(beta=100.0, epochs=epochs, tol=1e-3, refresh_every=10)
        if fused:
            info, lab, obj, status, best = T.thetis_solve_round_batch(hb, seed=21, reps=7, **kw)
        else:
            info = hb.solve(**kw)
            lab, obj, status, best = T.thetis_round_batch(hb, seed=21, reps=7)
        outs.append((hb.get_x(), lab.copy(), obj, status, best, info["epochs_run"]))
    (x1, l1, o1, s1, b1, e1), (x2, l2, o2, s2, b2, e2) = outs
    assert np.array_equal(x1, x2) and e1 == e2
    assert np.array_equal(l1, l2)
    assert np.array_equal(o1, o2)
    assert np.array_equal(s1, s2)
    assert np.array_equal(b1, b2)
    noff, _ = _slices(items)
    for t, (kind, g) in enumerate(items):
        if kind == "vc" and epochs == 0 and g.m > 0:
            assert s1[t] == -1, t
        else:
            assert s1[t] == 1, t
            assert oracle.build_problem(kind, g).valid(l1[noff[t]:noff[t + 1]]), t

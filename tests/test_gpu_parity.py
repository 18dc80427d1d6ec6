"""CUDA path vs FP64 oracle through the C ABI (sizes the oracle finishes in
seconds, several tiles and ragged tails).  Tolerances: iterates max|dx| <= 1e-4,
relative objective <= 1e-5; colouring and rounding decisions bit-exact (rounding
compared outside the 1e-4 threshold band)."""
import numpy as np
import pytest

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import (OBJ_RTOL, X_TOL, build_gpu, gpu, gpu_full_x, hub_graph, is_graph, multi_hub_graph,
                              rel, vc_graph)

pytestmark = pytest.mark.gpu


def _pair(kind, g, seed=0):
    h = build_gpu(kind, g, seed=seed)
    lp = oracle.build_problem(kind, g)
    return h, lp


CASES = [
    ("vc", lambda: vc_graph(2000, 8000, 1)),
    ("is", lambda: is_graph(3000, 20000, 2)),
    ("vc", lambda: hub_graph(5000, 12000, 2600, 3)),
    ("is", lambda: hub_graph(6000, 9000, 4500, 6)),
    ("vc", lambda: multi_hub_graph(9000, 30000, {37: 60, 1413: 300, 2900: 1500, 5071: 4700, 8999: 20}, 8)),
    ("mc", lambda: synth.grid_graph(37, 23, 4, 4)),
    ("mc", lambda: synth.grid_graph(16, 16, 8, 5)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_coloring_bit_exact(case):
    kind, mk = CASES[case]
    g = mk()
    h, lp = _pair(kind, g, seed=77)
    col_o, nc_o = lp.color(77)
    col_g = h.colors()
    assert h.sizes["ncolors"] == nc_o
    assert np.array_equal(col_g, col_o)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("step_rule", [0, 1])
@pytest.mark.parametrize("engine", [0, 1])
def test_scd_iterates_match_oracle(case, step_rule, engine):
    """engine 0: persistent cooperative sweep; engine 1: one launch per colour."""
    kind, mk = CASES[case]
    g = mk()
    h, lp = _pair(kind, g, seed=5)
    beta, epochs = 100.0, 50
    info = h.solve(beta=beta, epochs=epochs, refresh_every=10, step_rule=step_rule, engine=engine)
    col, _ = lp.color(5)
    x_o, info_o = lp.solve(beta=beta, epochs=epochs, refresh_every=10, step_rule=step_rule, color=col)
    x_g = gpu_full_x(h)
    assert info["epochs_run"] == info_o["epochs_run"] == epochs
    assert np.max(np.abs(x_g - x_o)) <= X_TOL
    assert rel(info["obj"], info_o["obj"]) <= OBJ_RTOL
    assert rel(info["fbeta"], info_o["fbeta"]) <= OBJ_RTOL
    # the GPU's own FP64 checks equal the oracle's checks at the GPU iterate
    chk = lp.checks(x_g, beta)
    assert abs(info["rho"] - chk["rho"]) <= 1e-6
    assert rel(info["obj"], chk["obj"]) <= 1e-9
    assert abs(info["infeas"] - chk["infeas"]) <= 1e-6
    assert rel(info["fbeta"], chk["fbeta"]) <= 1e-9


def test_engines_give_identical_iterates():
    """The persistent sweep and the per-colour launches run the same tiles in the
    same colour order, so their iterates agree to the last bit."""
    g = is_graph(3000, 20000, 2)
    h0, h1 = build_gpu("is", g, seed=5), build_gpu("is", g, seed=5)
    i0 = h0.solve(beta=100.0, epochs=23, refresh_every=7, engine=0)
    i1 = h1.solve(beta=100.0, epochs=23, refresh_every=7, engine=1)
    assert np.array_equal(gpu_full_x(h0), gpu_full_x(h1))
    assert i0["fbeta"] == i1["fbeta"]


def test_stop_at_tolerance_matches_oracle():
    g = vc_graph(600, 2400, 9)
    h, lp = _pair("vc", g, seed=1)
    info = h.solve(beta=100.0, epochs=3000, tol=1e-3, refresh_every=10)
    x_o, info_o = lp.solve(beta=100.0, epochs=3000, tol=1e-3, refresh_every=10, color=lp.color(1)[0])
    assert info["converged"] and info_o["converged"]
    assert info["epochs_run"] == info_o["epochs_run"]
    assert info["rho"] <= 1e-3
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL


def test_ubar_xbar_and_warm_start():
    g = vc_graph(500, 1500, 4)
    h, lp = _pair("vc", g, seed=2)
    rng = np.random.default_rng(3)
    ub = rng.normal(0, 0.5, lp.M).astype(np.float32)
    xb = rng.uniform(0, 1, lp.N).astype(np.float32)
    x0 = rng.uniform(0, 1, g.n).astype(np.float32)
    info = h.solve(beta=30.0, epochs=40, refresh_every=7, ubar=ub, xbar=xb, x0=x0)
    xs0 = lp.initial_x()
    xs0[: g.n] = x0
    x_o, info_o = lp.solve(beta=30.0, epochs=40, refresh_every=7, color=lp.color(2)[0],
                           ubar=ub.astype(np.float64), xbar=xb.astype(np.float64), x0=xs0)
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL
    assert rel(info["fbeta"], info_o["fbeta"]) <= OBJ_RTOL


def test_solve_continues_from_current_iterate():
    g = vc_graph(400, 1600, 6)
    h, lp = _pair("vc", g, seed=3)
    h.solve(beta=100.0, epochs=20)
    h.solve(beta=100.0, epochs=30)
    x_o, _ = lp.solve(beta=100.0, epochs=50, color=lp.color(3)[0])
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL


def test_general_lp_with_eq_rows_and_values():
    """thetis_create on a general LP: EQ/GE/LE rows, non-unit coefficients,
    per-column bounds, a fixed column and a simplex block."""
    rng = np.random.default_rng(11)
    M, n = 60, 80
    A = (rng.random((M, n)) < 0.08) * rng.choice([-2.0, -1.0, 0.5, 1.0, 3.0], size=(M, n))
    A[:, 0] = 0
    A[rng.integers(0, M, 4), 0] = 1.0
    cols = [np.nonzero(A[:, j])[0] for j in range(n)]
    colptr = np.concatenate([[0], np.cumsum([len(c) for c in cols])]).astype(np.int64)
    rowidx = np.concatenate(cols).astype(np.int32)
    val = np.concatenate([A[c, j] for j, c in enumerate(cols)]).astype(np.float32)
    b = rng.normal(0, 1, M).astype(np.float32)
    c = rng.normal(0, 1, n).astype(np.float32)
    lo = np.zeros(n, np.float32)
    hi = rng.uniform(0.5, 2.0, n).astype(np.float32)
    lo[5] = hi[5] = 0.25  # fixed column
    rk = rng.integers(0, 3, M).astype(np.uint8)
    bf = np.array([10, 20], np.int64)  # two simplex blocks of 3
    for f in bf:
        lo[f:f + 3] = 0
        hi[f:f + 3] = 1
    T = gpu()
    h = T.thetis_create(M, n, colptr, rowidx, b, c, lo, hi, rk, csc_val=val, block_k=3, block_first=bf, seed=9)
    lp = oracle.OracleLP.general(M, colptr, rowidx, val.astype(np.float64), b.astype(np.float64),
                                 c.astype(np.float64), lo.astype(np.float64), hi.astype(np.float64), rk, 3, bf)
    assert np.array_equal(h.colors(), lp.color(9)[0])
    info = h.solve(beta=5.0, epochs=60, refresh_every=10)
    x_o, info_o = lp.solve(beta=5.0, epochs=60, refresh_every=10, color=lp.color(9)[0])
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL
    assert rel(info["fbeta"], info_o["fbeta"]) <= OBJ_RTOL


# -------------------------------------------------------------------------
# rounding
# -------------------------------------------------------------------------
@pytest.mark.parametrize("kind,mk", [("vc", lambda: vc_graph(2000, 8000, 1)), ("is", lambda: is_graph(3000, 20000, 2)),
                                     ("mc", lambda: synth.grid_graph(37, 23, 4, 4))])
def test_rounding_bit_exact_on_same_x(kind, mk):
    """Same iterate on both sides (the GPU's FP32 x given to the oracle in FP64):
    labels, objective, repair value and best repetition are identical."""
    g = mk()
    h, lp = _pair(kind, g)
    h.solve(beta=100.0, epochs=50)
    x = h.get_x().astype(np.float64)
    lab, info = h.round(seed=123, reps=10)
    if kind == "vc":
        r = lp.round_vc(x[: g.n])
        assert info["repair"] == r["eps"]
    elif kind == "is":
        r = lp.round_is(x[: g.n], 123, 10)
        assert info["repair"] == r["alpha"] and info["best_rep"] == r["best_rep"]
    else:
        r = lp.round_mc(x[: g.n * len(g.terminals)], 123, 10)
        assert info["best_rep"] == r["best_rep"]
    assert np.array_equal(lab, r["labels"])
    assert info["obj"] == r["obj"]
    assert info["valid"] and lp.valid(lab)


@pytest.mark.parametrize("kind,mk", [("vc", lambda: vc_graph(2000, 8000, 1)), ("is", lambda: is_graph(3000, 20000, 2)),
                                     ("mc", lambda: synth.grid_graph(37, 23, 4, 4)),
                                     ("mc", lambda: synth.grid_graph(64, 48, 8, 9))])
def test_rounding_end_to_end_outside_band(kind, mk):
    """GPU solve + round vs oracle solve + round, compared element by element on
    every vertex whose decision no draw within the band of its threshold can
    change.  The band is 1e-4, widened to twice the largest difference of the
    repaired points x~ of the two sides.  IS (App. B.2): a vertex's final label
    depends on its own pick and its neighbours' (alteration), so the vertices
    near the band and their neighbours are masked, in the repetition the GPU
    chose; MC (App. B.3): a vertex's label depends on its own row only.  The
    GPU's choice of repetition must be the oracle's best up to the weight / cut
    cost the masked decisions can move."""
    g = mk()
    h, lp = _pair(kind, g)
    h.solve(beta=100.0, epochs=50)
    reps, seed = 10, 5
    lab, info = h.round(seed=seed, reps=reps)
    x_o, _ = lp.solve(beta=100.0, epochs=50, color=lp.color(0)[0])
    x_g = h.get_x().astype(np.float64)
    n = g.n
    assert info["valid"] and lp.valid(lab)
    if kind == "vc":
        r = lp.round_vc(x_o[:n])
        xt = np.minimum(1, x_o[:n] / (1 - r["eps"]))
        xt_g = np.minimum(1, x_g[:n] / (1 - info["repair"]))
        band = max(1e-4, 2 * float(np.max(np.abs(xt - xt_g))))
        near = np.abs(xt - 0.5) < band
        assert np.array_equal(lab[~near], r["labels"][~near])
        assert near.mean() < 0.05
        return
    if kind == "is":
        r = lp.round_is(x_o[:n], seed, reps)
        xt = x_o[:n] / (1 + r["alpha"])
        xt_g = x_g[:n] / (1 + info["repair"])
        band = max(1e-4, 2 * float(np.max(np.abs(xt - xt_g))))
        nbr = [[] for _ in range(n)]
        for a, b in zip(g.eu.tolist(), g.ev.tolist()):
            nbr[a].append(b)
            nbr[b].append(a)
        w = g.w.astype(np.float64)
        wq, mq, lq = [], [], []
        for q in range(reps):
            u = np.array([oracle.rng_uniform(seed, q, 1, v) for v in range(n)])
            near = np.abs(u - xt) < band
            mask = near.copy()
            for v in np.nonzero(near)[0]:
                mask[nbr[v]] = True
            l_q = lp.round_is_rep(xt, seed, q)
            lq.append(l_q)
            wq.append(float(w @ l_q))
            mq.append(float(w[mask].sum()))
            if q == info["best_rep"]:
                b_mask = mask
        b = info["best_rep"]
        assert b_mask.mean() < 0.2
        assert np.array_equal(lab[~b_mask], lq[b][~b_mask])
        assert wq[b] + mq[b] >= max(wq[q] - mq[q] for q in range(reps))
        if b == r["best_rep"]:
            assert np.array_equal(lq[b], r["labels"])
        return
    k = len(g.terminals)
    r = lp.round_mc(x_o[: n * k], seed, reps)
    X = x_o[: n * k].reshape(n, k)
    Xg = x_g[: n * k].reshape(n, k)
    band = max(1e-4, 2 * float(np.max(np.abs(X - Xg))))
    ce = g.ce.astype(np.float64)
    cq, sq = [], []
    for q in range(reps):
        rad = oracle.rng_uniform(seed, q, 2, 0)
        near = np.any(np.abs(X - (1 - rad)) < band, axis=1)
        l_q = lp.round_mc_rep(x_o[: n * k], seed, q)
        cq.append(lp.mc_cut_cost(l_q))
        sq.append(float(ce[near[g.eu] | near[g.ev]].sum()))
        if q == info["best_rep"]:
            b_near, b_lab = near, l_q
    b = info["best_rep"]
    assert b_near.mean() < 0.2
    assert np.array_equal(lab[~b_near], b_lab[~b_near])
    assert cq[b] - sq[b] <= min(cq[q] + sq[q] for q in range(reps))


def test_vc_repair_error():
    g = vc_graph(50, 100, 2)
    h = build_gpu("vc", g)
    lab, info = h.round(seed=0)  # x = 0: eps = 1
    assert lab is None and info["status"] == gpu().THETIS_E_REPAIR


# -------------------------------------------------------------------------
# edge cases and memory spaces
# -------------------------------------------------------------------------
def test_device_inputs_equal_host_inputs():
    import torch

    g = vc_graph(1500, 5000, 8)
    h1 = build_gpu("vc", g)
    h2 = build_gpu("vc", g, device=True, stream=torch.cuda.current_stream())
    for h in (h1, h2):
        h.solve(beta=100.0, epochs=30)
    assert np.array_equal(h1.get_x(), h2.get_x())
    out = torch.zeros(g.n, dtype=torch.uint8, device="cuda")
    lab1, _ = h1.round(seed=1)
    h2.round(seed=1, out=out)
    assert np.array_equal(lab1, out.cpu().numpy())


def test_empty_and_isolated():
    T = gpu()
    # no edges: every vertex isolated, VC optimum is 0, IS picks every vertex
    e = np.zeros(0, np.int32)
    h = T.thetis_build_vc(5, e, e, np.ones(5, np.float32))
    info = h.solve(beta=10.0, epochs=3)
    assert np.all(h.get_x() == 0)
    lab, r = h.round()
    assert r["valid"] and lab.sum() == 0
    h = T.thetis_build_is(5, e, e, np.ones(5, np.float32))
    h.solve(beta=10.0, epochs=200, tol=1e-9)
    lab, r = h.round(seed=3, reps=4)
    assert r["valid"]
    # single edge: the closed form of eq. QP (Sec. 3.2)
    h = T.thetis_build_vc(2, np.array([0], np.int32), np.array([1], np.int32), np.ones(2, np.float32))
    h.solve(beta=4.0, epochs=20000, tol=1e-7)
    t = (4.0 - 1) / (8.0 + 0.25)
    assert np.max(np.abs(h.get_x() - t)) < 1e-5


def test_invalid_inputs_rejected():
    T = gpu()
    with pytest.raises(T.ThetisError) as ei:
        T.thetis_build_vc(3, np.array([0, 1]), np.array([1, 5]), np.ones(3))
    assert ei.value.status == T.THETIS_E_INVALID
    with pytest.raises(T.ThetisError):
        T.thetis_build_vc(3, np.array([0]), np.array([0]), np.ones(3))  # loop
    with pytest.raises(T.ThetisError):
        T.thetis_build_vc(3, np.array([0]), np.array([1]), np.array([1.0, -1.0, 1.0]))  # weight <= 0
    with pytest.raises(T.ThetisError):
        T.thetis_build_mc(4, np.array([0, 1]), np.array([1, 2]), np.ones(2), 2, np.array([0, 0]))
    with pytest.raises(T.ThetisError):  # repeated row inside a column
        T.thetis_create(2, 1, np.array([0, 2]), np.array([1, 1]), np.ones(2), np.ones(1), np.zeros(1),
                        np.ones(1), np.zeros(2, np.uint8))
    g = vc_graph(30, 50, 1)
    h = build_gpu("vc", g)
    with pytest.raises(T.ThetisError):
        h.solve(beta=-1.0)
    with pytest.raises(T.ThetisError):
        h.round(kind=T.ROUND_IS)


def test_async_mode_converges_to_oracle_solution():
    """Sec. 3.4 asynchronous mode: no iterate parity, but the converged
    objective and residual match the oracle's solution."""
    g = vc_graph(1000, 3000, 12)
    h, lp = _pair("vc", g)
    info = h.solve(beta=20.0, epochs=4000, tol=1e-5, refresh_every=20, mode=gpu().MODE_ASYNC)
    x_o, info_o = lp.solve(beta=20.0, epochs=100000, tol=1e-9, refresh_every=50, color=lp.color(0)[0])
    assert info["rho"] <= 1e-5
    assert rel(info["fbeta"], info_o["fbeta"]) <= 1e-5
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= 1e-2


@pytest.mark.parametrize("step_rule", [0, 1])
def test_tail_colours_match_oracle_and_engines(step_rule):
    """A power-law graph whose last 22 colours hold only a few columns each:
    they run as the three tail phases (partial dots, one-CTA colour chain,
    deferred scatter) in both engines; the iterate matches the oracle's serial
    sweep and the engines agree bit for bit."""
    g = is_graph(8000, 120000, 2)
    T = gpu()
    kw = dict(beta=100.0, epochs=30, refresh_every=10, step_rule=step_rule)
    h0, lp = _pair("is", g, seed=0)
    h0.solve(engine=0, **kw)
    h1 = build_gpu("is", g, seed=0)
    h1.solve(engine=1, **kw)
    x0, x1 = gpu_full_x(h0), gpu_full_x(h1)
    assert np.array_equal(x0, x1)
    x_o, _ = lp.solve(color=lp.color(0)[0], **kw)
    assert np.max(np.abs(x0 - x_o)) <= X_TOL
    # with centres: xbar, ubar given
    rng = np.random.default_rng(1)
    ub = rng.normal(size=g.m).astype(np.float32)
    xb = rng.random(g.n + g.m).astype(np.float32)
    h2, _ = _pair("is", g, seed=0)
    h2.solve(ubar=ub, xbar=xb, **kw)
    x_o2, _ = lp.solve(color=lp.color(0)[0], ubar=ub.astype(np.float64), xbar=xb.astype(np.float64), **kw)
    assert np.max(np.abs(gpu_full_x(h2) - x_o2)) <= X_TOL


@pytest.mark.parametrize("ctas", [1, 4, 64])
def test_async_mode_capped_concurrency_converges(ctas):
    """The asynchronous scheme with at most `ctas` CTAs stepping at once reaches
    the same solution (objective within 1e-5, rho <= tol)."""
    g = vc_graph(1000, 3000, 12)
    h, lp = _pair("vc", g)
    info = h.solve(beta=20.0, epochs=4000, tol=1e-5, refresh_every=20, mode=gpu().MODE_ASYNC, async_ctas=ctas)
    x_o, info_o = lp.solve(beta=20.0, epochs=100000, tol=1e-9, refresh_every=50, color=lp.color(0)[0])
    assert info["rho"] <= 1e-5
    assert rel(info["fbeta"], info_o["fbeta"]) <= 1e-5
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= 1e-2


def test_autotune_keeps_the_iterate_and_parity():
    """Tuning times trial sweeps on the real problem but restores the iterate;
    a solve after tuning still matches the oracle (the lane group only changes
    the FP32 summation order inside small columns)."""
    T = gpu()
    g = is_graph(3000, 20000, 2)
    h, lp = _pair("is", g, seed=5)
    h.solve(beta=100.0, epochs=7)
    x_before = gpu_full_x(h)
    sg, per = T.thetis_autotune(h, beta=100.0, trial_epochs=2)
    assert sg in (1, 2, 4, 8) and per in (0, 1, 2)
    assert np.array_equal(gpu_full_x(h), x_before)
    h.solve(beta=100.0, epochs=33)
    x_o, _ = lp.solve(beta=100.0, epochs=40, refresh_every=10, color=lp.color(5)[0])
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL
    # a second handle of the same shape takes the cached choice
    h2 = build_gpu("is", g, seed=5)
    assert T.thetis_autotune(h2, beta=100.0, trial_epochs=2) == (sg, per)


@pytest.mark.parametrize("group", [1, 2, 4, 8])
def test_every_small_group_matches_oracle(group):
    """Each lane-group variant of the small-column step is exact to tolerance."""
    g = vc_graph(2000, 8000, 1)
    h, lp = _pair("vc", g, seed=5)
    _force_group(h, group)
    h.solve(beta=100.0, epochs=30, refresh_every=10)
    x_o, _ = lp.solve(beta=100.0, epochs=30, refresh_every=10, color=lp.color(5)[0])
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL


def _force_group(h, group):
    gpu().thetis_set_launch_shape(h, group, 0)


def _general_lp_from_rows(rows, n, rng, block_first, block_k):
    """CSC of a general LP whose rows hold the given column sets (coefficients
    +-1 and 2), random row kinds, bounds [0, hi] with simplex blocks."""
    M = len(rows)
    entries = sorted((int(j), i) for i, r in enumerate(rows) for j in r)
    colptr = np.zeros(n + 1, np.int64)
    for j, _ in entries:
        colptr[j + 1] += 1
    colptr = np.cumsum(colptr)
    rowidx = np.array([i for _, i in entries], np.int32)
    val = rng.choice([-1.0, 1.0, 2.0], size=len(entries)).astype(np.float32)
    b = rng.normal(0, 1, M).astype(np.float32)
    c = rng.normal(0, 1, n).astype(np.float32)
    lo = np.zeros(n, np.float32)
    hi = rng.uniform(0.5, 2.0, n).astype(np.float32)
    for f in block_first:
        hi[f:f + block_k] = 1
    rk = rng.integers(0, 3, M).astype(np.uint8)
    return M, colptr, rowidx, val, b, c, lo, hi, rk


def test_colouring_beyond_the_row_masks():
    """Dense rows (320 columns) force more than 300 colours, past the 127 the
    per-row colour masks hold, so the colouring takes its slow path; rows with
    two columns of one block, and rows of exactly two units (one of them a
    block appearing twice), take the repeat and two-unit paths.  Colouring
    equal to the oracle's; a short solve matches."""
    rng = np.random.default_rng(21)
    n, k = 700, 3
    bf = np.array([30, 300, 600], np.int64)
    rows = [rng.choice(n, 320, replace=False) for _ in range(3)]
    rows += [rng.choice(n, 2, replace=False) for _ in range(200)]
    rows += [np.array([30, 31, 300, 301, 302]), np.array([600, 601, 5]), np.array([302, 30, 32, 450])]
    while len(rows) < 420:
        rows.append(rng.choice(n, int(rng.integers(3, 7)), replace=False))
    M, colptr, rowidx, val, b, c, lo, hi, rk = _general_lp_from_rows(rows, n, rng, bf, k)
    T = gpu()
    h = T.thetis_create(M, n, colptr, rowidx, b, c, lo, hi, rk, csc_val=val, block_k=k, block_first=bf, seed=4)
    lp = oracle.OracleLP.general(M, colptr, rowidx, val.astype(np.float64), b.astype(np.float64),
                                 c.astype(np.float64), lo.astype(np.float64), hi.astype(np.float64), rk, k, bf)
    col_o, nc_o = lp.color(4)
    assert nc_o > 300
    assert h.sizes["ncolors"] == nc_o
    assert np.array_equal(h.colors(), col_o)
    h.solve(beta=5.0, epochs=20, refresh_every=10)
    x_o, _ = lp.solve(beta=5.0, epochs=20, refresh_every=10, color=col_o)
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL

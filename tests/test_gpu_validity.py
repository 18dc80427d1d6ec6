"""Exact validity check of integral solutions (thetis_check_labels): it must
accept the roundings' own outputs and reject every labelling that breaks the
problem's constraints -- an uncovered edge (VC, Sec. 2), an edge inside the set
(IS, App. B.2), a terminal with another terminal's label or a label out of range
(MC, App. B.3), an uncovered element (SC, App. B.1), a label out of range (MAP,
Sec. 4.1).  The oracle's own validity check and objective are the reference."""
import numpy as np
import pytest

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import build_gpu, gpu, is_graph, vc_graph

pytestmark = pytest.mark.gpu


def _weight(g, lab):
    return float(g.w.astype(np.float64) @ (lab != 0))


def test_vertex_cover_rejects_an_uncovered_edge():
    g = vc_graph(1500, 6000, 4)
    h = build_gpu("vc", g)
    lp = oracle.build_problem("vc", g)
    h.solve(beta=100.0, epochs=60)
    lab, info = h.round()
    valid, obj = h.check_labels(lab)
    assert valid and lp.valid(lab) and obj == info["obj"] == _weight(g, lab)
    bad = lab.copy()
    e = int(np.nonzero(lab[g.eu] | lab[g.ev])[0][0])
    bad[g.eu[e]] = bad[g.ev[e]] = 0
    assert not lp.valid(bad)
    valid, obj = h.check_labels(bad)
    assert not valid and obj == _weight(g, bad)
    # every vertex chosen is a cover; none is not (when there is an edge)
    assert h.check_labels(np.ones(g.n, np.uint8))[0]
    assert not h.check_labels(np.zeros(g.n, np.uint8))[0]


def test_independent_set_rejects_an_edge_inside():
    g = is_graph(2000, 9000, 5)
    h = build_gpu("is", g)
    lp = oracle.build_problem("is", g)
    h.solve(beta=100.0, epochs=60)
    lab, info = h.round(seed=3, reps=6)
    valid, obj = h.check_labels(lab)
    assert valid and lp.valid(lab) and obj == info["obj"]
    bad = lab.copy()
    bad[g.eu[17]] = bad[g.ev[17]] = 1
    assert not lp.valid(bad)
    assert not h.check_labels(bad)[0]
    assert h.check_labels(np.zeros(g.n, np.uint8))[0]
    # a label value other than 0 / 1 is out of range
    two = lab.copy()
    two[np.nonzero(lab == 0)[0][0]] = 2
    valid, obj = h.check_labels(two)
    assert not valid and np.isnan(obj)


def test_multiway_cut_rejects_wrong_terminal_and_out_of_range_labels():
    T = gpu()
    g = synth.grid_graph(40, 30, 4, 6)
    h = build_gpu("mc", g)
    lp = oracle.build_problem("mc", g)
    h.solve(beta=100.0, epochs=60)
    lab, info = h.round(seed=2, reps=5)
    valid, obj = h.check_labels(lab)
    assert valid and lp.valid(lab) and obj == info["obj"] == lp.mc_cut_cost(lab)
    t0, t1 = int(g.terminals[0]), int(g.terminals[1])
    bad = lab.copy()
    bad[t0] = 1  # terminal 0 must keep label 0
    assert not lp.valid(bad)
    valid, obj = h.check_labels(bad)
    assert not valid and obj == lp.mc_cut_cost(bad)
    swap = lab.copy()
    swap[t0], swap[t1] = 1, 0
    assert not h.check_labels(swap)[0]
    oor = lab.copy()
    oor[int(np.setdiff1d(np.arange(g.n), g.terminals)[0])] = 4  # k = 4
    valid, obj = h.check_labels(oor)
    assert not valid and np.isnan(obj)
    # a labelling with every non-terminal on label 0 is feasible
    ok = np.zeros(g.n, np.uint8)
    ok[g.terminals] = np.arange(4)
    assert h.check_labels(ok, kind=T.ROUND_MC)[0] and lp.valid(ok)


def test_set_cover_rejects_an_uncovered_element():
    T = gpu()
    ss = synth.set_cover_instance(3000, 700, 1, 5, 11)
    h = T.thetis_build_sc(ss.n_elements, ss.ptr, ss.elems, ss.cost, seed=1)
    lp = oracle.OracleLP.set_cover(ss.n_elements, ss.ptr, ss.elems, ss.cost.astype(np.float64))
    h.solve(beta=100.0, epochs=60)
    lab, info = h.round(kind=T.ROUND_SC)
    valid, obj = h.check_labels(lab, kind=T.ROUND_SC)
    assert valid and lp.valid_sc(lab) and obj == info["obj"]
    # drop every set that holds element a
    a = int(ss.elems[ss.ptr[5]])
    holds = [s for s in range(len(ss.ptr) - 1) if a in ss.elems[ss.ptr[s]:ss.ptr[s + 1]]]
    bad = lab.copy()
    bad[holds] = 0
    assert not lp.valid_sc(bad)
    valid, obj = h.check_labels(bad, kind=T.ROUND_SC)
    assert not valid and obj == float(ss.cost.astype(np.float64) @ (bad != 0))


def test_map_rejects_out_of_range_labels_and_scores_valid_ones():
    T = gpu()
    g = synth.skip_chain_crf(300, 5, 20, 0.1, 2)
    h = T.thetis_build_map(g.n, g.k, g.eu, g.ev, g.theta_node, g.theta_edge, seed=0)
    lp = oracle.OracleLP.map_lp(g.n, g.k, g.eu, g.ev, g.theta_node.astype(np.float64),
                                g.theta_edge.astype(np.float64))
    rng = np.random.default_rng(4)
    lab = rng.integers(0, g.k, g.n).astype(np.uint8)
    valid, obj = h.check_labels(lab)
    assert valid
    assert abs(obj - lp.map_energy(lab)) <= 1e-9 * max(1.0, abs(obj))
    lab[7] = g.k
    valid, obj = h.check_labels(lab)
    assert not valid and np.isnan(obj)


def test_check_labels_argument_errors():
    T = gpu()
    g = vc_graph(100, 300, 1)
    h = build_gpu("vc", g)
    with pytest.raises(T.ThetisError):  # kind does not match the problem
        h.check_labels(np.zeros(g.n, np.uint8), kind=T.ROUND_MC)
    items = [("vc", vc_graph(50, 100, 2)), ("is", vc_graph(60, 120, 3))]
    hb = T.thetis_build_batch_graphs(items)
    with pytest.raises(T.ThetisError):  # batch handles report validity per instance through thetis_round_batch
        T.thetis_check_labels(hb, np.zeros(110, np.uint8), kind=T.ROUND_VC)

"""The seeded input generators: shapes and invariants the workloads rely on
(they hold no method arithmetic)."""
import numpy as np

from paper_1311_2661_gb300 import synth


def test_set_cover_instance_shape():
    ss = synth.set_cover_instance(2000, 300, 1, 6, 4)
    assert ss.ptr[0] == 0 and np.all(np.diff(ss.ptr) >= 0) and ss.ptr[-1] == ss.elems.shape[0]
    for j in range(ss.n_sets):
        e = ss.elems[ss.ptr[j]:ss.ptr[j + 1]]
        assert np.all(np.diff(e) > 0) and (e.size == 0 or (e[0] >= 0 and e[-1] < ss.n_elements))
    freq = np.bincount(ss.elems, minlength=ss.n_elements)
    assert freq.min() >= 1 and freq.max() <= 6
    assert np.all(ss.cost == np.round(ss.cost)) and ss.cost.min() >= 1 and ss.cost.max() <= 10
    again = synth.set_cover_instance(2000, 300, 1, 6, 4)
    assert np.array_equal(again.elems, ss.elems) and np.array_equal(again.cost, ss.cost)


def test_skip_chain_crf_shape():
    f = synth.skip_chain_crf(1000, 5, 20, 0.2, 3)
    nchain = 1000 - 1000 // 20  # neighbours inside a sentence
    u, v = f.eu.astype(np.int64), f.ev.astype(np.int64)
    assert np.all(u < v)
    chain, skip = slice(0, nchain), slice(nchain, None)
    assert np.all(v[chain] - u[chain] == 1) and np.all(u[chain] % 20 != 19)
    assert np.all(v[skip] - u[skip] >= 2) and np.all(v[skip] - u[skip] <= 500)
    assert f.theta_node.shape == (1000, 5) and f.theta_edge.shape == (f.m, 5, 5)
    # chain factors share one transition matrix; skip factors reward agreement only
    assert np.all(f.theta_edge[chain] == f.theta_edge[0])
    te = f.theta_edge[skip]
    assert np.all(te[:, ~np.eye(5, dtype=bool)] == 0) and np.all(te[:, 0, 0] == te[:, 1, 1])


def test_serving_pool_and_trace():
    pool = synth.serving_pool(20, 5, n_lo=100, n_hi=2000, side_lo=8, side_hi=12)
    kinds = [k for k, _ in pool]
    assert kinds.count("vc") == 8 and kinds.count("is") == 8 and kinds.count("mc") == 4
    for k, g in pool:
        if k == "mc":
            assert len(g.terminals) == 4
        else:
            assert 100 <= g.n <= 2000 and g.w.shape == (g.n,)
    t, idx = synth.poisson_trace(2000.0, 5000, kinds, 1)
    assert np.all(np.diff(t) > 0) and abs(t[-1] - 2.5) < 0.25  # 5000 arrivals at 2000/s
    got = np.array([kinds[j] for j in idx])
    for k, p in (("vc", 0.4), ("is", 0.4), ("mc", 0.2)):
        assert abs(np.mean(got == k) - p) < 0.03


def test_batch_instances_shape():
    items = synth.batch_instances(12, 50, 400, 4.0, 8.0, 1, 10, 2)
    assert [k for k, _ in items] == ["vc"] * 6 + ["is"] * 6
    for _, g in items:
        assert 50 <= g.n <= 400 and np.all(g.eu < g.ev) and g.w.min() >= 1 and g.w.max() <= 10
        keys = g.eu.astype(np.int64) * g.n + g.ev
        assert np.unique(keys).size == keys.size  # simple graph


def _simple(g):
    keys = g.eu.astype(np.int64) * g.n + g.ev
    return np.all(g.eu < g.ev) and np.unique(keys).size == keys.size and g.eu.min() >= 0 and g.ev.max() < g.n


def test_er_graph_shape():
    g = synth.er_graph(3000, 12000, 5)
    assert g.m == 12000 and _simple(g)
    deg = np.bincount(np.concatenate([g.eu, g.ev]), minlength=g.n)
    assert deg.mean() == 8.0 and deg.max() < 30  # binomial, mean 8
    again = synth.er_graph(3000, 12000, 5)
    assert np.array_equal(again.eu, g.eu) and np.array_equal(again.ev, g.ev)


def test_chung_lu_shape():
    """m distinct edges, a heavy tail whose log-log CCDF slope is near
    -(gamma - 1), and degrees far above the mean on a few hubs."""
    n, m, gamma = 50_000, 400_000, 2.1
    g = synth.chung_lu(n, m, gamma, 3)
    assert g.m == m and _simple(g)
    deg = np.bincount(np.concatenate([g.eu, g.ev]), minlength=n)
    assert deg.mean() == 2 * m / n
    assert np.median(deg) < deg.mean() < deg.max() / 20
    # tail slope of P(D >= d) between d = 2*mean and d = 20*mean
    d = np.array([2, 4, 8, 16]) * deg.mean()
    ccdf = np.array([np.mean(deg >= x) for x in d])
    slope = np.polyfit(np.log(d), np.log(ccdf), 1)[0]
    assert -1.6 < slope < -0.7
    again = synth.chung_lu(n, m, gamma, 3)
    assert np.array_equal(again.eu, g.eu) and np.array_equal(again.ev, g.ev)


def test_grid_graph_shape():
    g = synth.grid_graph(37, 23, 4, 2)
    assert g.n == 37 * 23 and g.m == 2 * 37 * 23 - 37 - 23 and _simple(g)
    d = g.ev.astype(np.int64) - g.eu
    assert np.all((d == 1) | (d == 37))  # right or down neighbour
    assert np.all(g.eu[d == 1] % 37 != 36)  # no wrap-around
    assert np.unique(g.terminals).size == 4 and g.ce.shape == (g.m,) and g.ce.min() > 0

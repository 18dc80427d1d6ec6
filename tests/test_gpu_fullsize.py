"""The CUDA path at the benchmark's full sizes, in the launch shape the
benchmark times (the autotuned sweep), against the FP64 oracle: the IS LP of a
Chung-Lu graph (n = 2^20, M = 1.6e7 edges, gamma = 2.1) and the multiway-cut
LP of a 1024 x 1024 grid with 8 terminals.  The oracle still gets through a
few epochs of these on one core, so the comparison is element by element:

* colouring -- IS: equal to the oracle's sequential greedy colouring; MC (whose
  sequential colouring takes minutes): a proper colouring (no row holds two
  units of one colour) that is first-fit in the priority order on a sample of
  units;
* the full iterate after two epochs with the FP64 refresh (the oracle sweeps
  in the GPU's colour order): max |dx| <= 1e-4;
* rounding on the GPU's own iterate: labels, objective and winning repetition
  identical, and the labels valid.

Full-size frontiers take the colouring's grouped paths (16 or 4 units a warp)
that the small cases never reach."""
import numpy as np
import pytest

import oracle
from paper_1311_2661_gb300 import synth
from tests.gpu_common import X_TOL, build_gpu, gpu, gpu_full_x

pytestmark = pytest.mark.gpu

BETA = 100.0


def _check_proper_and_first_fit(lp, col, seed, sample=3000):
    """On a random sample of units: no unit sharing a row with it has its
    colour, and every colour below its own is held by a higher-priority unit
    sharing a row with it (one pass over the non-zeros finds the sampled
    units' rows)."""
    e = lp.export()
    us, ul, _ = lp.units()
    cp, ri = e["colptr"], e["rowidx"]
    rank = np.empty(lp.U, np.int64)
    rank[lp.priority_order(seed)] = np.arange(lp.U)
    rng = np.random.default_rng(1)
    S = rng.choice(lp.U, size=min(sample, lp.U), replace=False)
    own = [ri[cp[us[u]]:cp[us[u] + ul[u]]] for u in S]
    rows = np.unique(np.concatenate(own))
    q = np.flatnonzero(np.isin(ri, rows))  # the non-zeros of those rows
    c = np.searchsorted(cp, q, side="right") - 1  # their columns
    w = np.searchsorted(us, c, side="right") - 1  # their units (fixed columns: none)
    ok = (w >= 0) & (c < us[np.maximum(w, 0)] + ul[np.maximum(w, 0)])
    rq, wq = ri[q][ok], w[ok]
    o = np.argsort(rq, kind="stable")
    rq, wq = rq[o], wq[o]
    for u, r_u in zip(S, own):
        lo, hi = np.searchsorted(rq, r_u), np.searchsorted(rq, r_u, side="right")
        parts = [wq[a:b] for a, b in zip(lo, hi)]
        nb = np.unique(np.concatenate(parts)) if parts else np.empty(0, np.int64)
        nb = nb[nb != u]
        assert not np.any(col[nb] == col[u]), "two units of one colour share a row"
        held = set(col[nb[rank[nb] < rank[u]]].tolist())
        assert all(cc in held for cc in range(int(col[u])))


def test_is_fullsize():
    T = gpu()
    g = synth.chung_lu(1 << 20, 16_000_000, 2.1, 2)
    g.w = synth.unit_interval_weights(g.n, np.random.default_rng(19))
    h = build_gpu("is", g, seed=0, device=True)
    T.thetis_autotune(h, beta=BETA)  # the benchmark's launch shape; the iterate is restored
    lp = oracle.build_problem("is", g)
    col_o, nc_o = lp.color(0)
    assert h.sizes["ncolors"] == nc_o
    assert np.array_equal(h.colors(), col_o)
    h.solve(beta=BETA, epochs=2, refresh_every=10)
    x_o, _ = lp.solve(beta=BETA, epochs=2, refresh_every=10, color=col_o)
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL
    x = h.get_x().astype(np.float64)
    lab, info = h.round(seed=11, reps=10)
    r = lp.round_is(x[: g.n], 11, 10)
    assert info["repair"] == r["alpha"] and info["best_rep"] == r["best_rep"]
    assert np.array_equal(lab, r["labels"]) and info["obj"] == r["obj"]
    assert info["valid"] and lp.valid(lab)


def test_mc_fullsize():
    T = gpu()
    g = synth.grid_graph(1024, 1024, 8, 3)
    h = build_gpu("mc", g, seed=0, device=True)
    T.thetis_autotune(h, beta=BETA)
    lp = oracle.build_problem("mc", g)
    col = h.colors()
    _check_proper_and_first_fit(lp, col, 0)
    h.solve(beta=BETA, epochs=2, refresh_every=10)
    x_o, _ = lp.solve(beta=BETA, epochs=2, refresh_every=10, color=col)
    assert np.max(np.abs(gpu_full_x(h) - x_o)) <= X_TOL
    k = len(g.terminals)
    x = h.get_x().astype(np.float64)
    lab, info = h.round(seed=11, reps=10)
    r = lp.round_mc(x[: g.n * k], 11, 10)
    assert info["best_rep"] == r["best_rep"]
    assert np.array_equal(lab, r["labels"]) and info["obj"] == r["obj"]
    assert info["valid"] and lp.valid(lab)

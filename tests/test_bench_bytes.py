"""The roofline numerator of bench.py -- algorithmic bytes per epoch, 20 +
12 nnz_j per free structural column and 16 per slack -- against a direct count
over the oracle's standard form on small instances of every workload kind (VC,
IS, multiway cut, set cover, MAP), and against the per-epoch figure of the IS
benchmark configuration (661 MB)."""
from types import SimpleNamespace

import numpy as np

import bench
import oracle
from paper_1311_2661_gb300 import synth


def _direct(lp, n_struct):
    e = lp.export()
    nnz = np.diff(e["colptr"])
    free = e["lo"] < e["hi"]
    struct = np.arange(lp.N) < n_struct
    return int(np.sum((20 + 12 * nnz)[struct & free]) + 16 * np.sum(~struct & free))


def test_is_and_vc_bytes_match_the_standard_form():
    g = synth.er_graph(500, 2000, 3)
    g.w = np.ones(g.n, np.float32)
    for kind in ("vc", "is"):
        lp = oracle.build_problem(kind, g)
        assert bench.algorithmic_bytes_per_epoch({"kind": kind}, g) == _direct(lp, g.n)


def test_mc_bytes_match_the_standard_form():
    g = synth.grid_graph(24, 17, 4, 5)
    lp = oracle.build_problem("mc", g)
    n_struct = g.n * 4 + g.m * 4  # vertex-label columns, then edge-label columns
    assert bench.algorithmic_bytes_per_epoch({"kind": "mc", "k": 4}, g) == _direct(lp, n_struct)


def test_is_benchmark_epoch_is_661_mb():
    g = SimpleNamespace(n=1 << 20, m=16_000_000)
    b = bench.algorithmic_bytes_per_epoch({"kind": "is"}, g)
    assert b == 20 * (1 << 20) + 40 * 16_000_000 and round(b / 1e6) == 661


def test_sc_bytes_match_the_standard_form():
    ss = synth.set_cover_instance(800, 150, 1, 5, 2)
    lp = oracle.OracleLP.set_cover(ss.n_elements, ss.ptr, ss.elems, ss.cost.astype(np.float64))
    g = SimpleNamespace(n=ss.n_sets, m=int(ss.ptr[-1]), n_elements=ss.n_elements)
    assert bench.algorithmic_bytes_per_epoch({"kind": "sc"}, g) == _direct(lp, ss.n_sets)


def test_map_bytes_match_the_standard_form():
    f = synth.skip_chain_crf(120, 4, 12, 0.2, 3)
    lp = oracle.OracleLP.map_lp(f.n, 4, f.eu, f.ev, f.theta_node.astype(np.float64), f.theta_edge.astype(np.float64))
    g = SimpleNamespace(n=f.n, m=f.m)
    assert bench.algorithmic_bytes_per_epoch({"kind": "map", "k": 4}, g) == _direct(lp, lp.N)

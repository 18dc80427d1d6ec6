"""The allocation-free rounding entry point (thetis_round_is_static).

Callers that cannot allocate device memory when they round -- a serving loop
that must not stall on cudaMalloc / cudaFree, a process whose free memory
belongs to another allocator, code recording a stream capture -- use this
entry point instead of thetis_round.  Its scratch is one fixed static device
array, so these tests check that it returns exactly what thetis_round returns,
on two calls in a row (the array keeps the previous call's contents), and that
sizes beyond the array are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests.gpu_common import build_gpu, is_graph

pytestmark = pytest.mark.gpu


def _device_inputs(g, h):
    import torch

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    h.get_x(out=x)
    return dev(g.eu), dev(g.ev), dev(g.w), x


def test_static_rounding_equals_thetis_round_twice():
    import torch

    from paper_1311_2661_gb300 import thetis as T

    g = is_graph(3000, 20000, 2)
    h = build_gpu("is", g)
    h.solve(beta=100.0, epochs=50)
    eu, ev, w, x = _device_inputs(g, h)
    for seed in (123, 123, 7):
        ref_lab, ref = h.round(seed=seed, reps=10)
        out = torch.full((g.n,), 255, dtype=torch.uint8, device="cuda")
        got = T.thetis_round_is_static(g.n, eu, ev, w, x, out, seed=seed, reps=10)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref_lab)
        for key in ("obj", "repair", "best_rep", "near", "valid"):
            assert got[key] == ref[key], key


def test_static_rounding_second_graph_after_first():
    """A smaller problem after a larger one: stale scratch must not leak in."""
    import torch

    from paper_1311_2661_gb300 import thetis as T

    for n, m, seed in ((4000, 30000, 3), (700, 2500, 4)):
        g = is_graph(n, m, seed)
        h = build_gpu("is", g)
        h.solve(beta=100.0, epochs=30)
        eu, ev, w, x = _device_inputs(g, h)
        ref_lab, ref = h.round(seed=9, reps=5)
        out = torch.zeros(g.n, dtype=torch.uint8, device="cuda")
        got = T.thetis_round_is_static(g.n, eu, ev, w, x, out, seed=9, reps=5)
        assert np.array_equal(out.cpu().numpy(), ref_lab)
        assert got["obj"] == ref["obj"] and got["valid"]


def test_static_rounding_rejects_sizes_beyond_scratch():
    import torch

    from paper_1311_2661_gb300 import thetis as T

    n = 33_488_624 // 10 + 1  # n * reps just above the limit at reps = 10
    eu = torch.zeros(0, dtype=torch.int32, device="cuda")
    w = torch.ones(1, dtype=torch.float32, device="cuda")
    with pytest.raises(T.ThetisError) as ei:
        T.thetis_round_is_static(n, eu, eu, w, w, torch.zeros(1, dtype=torch.uint8, device="cuda"), reps=10)
    assert ei.value.status == T.THETIS_E_INVALID
    assert "static scratch limit" in str(ei.value)

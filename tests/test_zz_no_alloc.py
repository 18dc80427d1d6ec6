"""The allocation-free rounding entry point (thetis_round_is_static).

Callers that cannot allocate device memory when they round -- a serving loop
that must not stall on cudaMalloc / cudaFree, or a process whose free memory
already belongs to another allocator -- use this entry point instead of
thetis_round.  Its scratch is one fixed static device array, so these tests
check that it returns exactly what thetis_round returns, on calls in a row (the
array keeps the previous call's contents), that neither the library's memory
pool nor torch's allocator grows during the calls, and that sizes beyond the
array, bad endpoints and host pointers are refused before any kernel reads
them.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_common import build_gpu, is_graph

pytestmark = pytest.mark.gpu


def _device_inputs(g, h):
    import torch

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    h.get_x(out=x)
    return dev(g.eu.astype(np.int32)), dev(g.ev.astype(np.int32)), dev(g.w.astype(np.float32)), x


def _memory():
    import torch

    from paper_1311_2661_gb300 import thetis as T

    torch.cuda.synchronize()
    return T.thetis_cache_info(), torch.cuda.memory_allocated()


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
        before = _memory()
        got = T.thetis_round_is_static(g.n, eu, ev, w, x, out, seed=seed, reps=10)
        assert _memory() == before, "the allocation-free rounding changed device memory use"
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
        before = _memory()
        got = T.thetis_round_is_static(g.n, eu, ev, w, x, out, seed=9, reps=5)
        assert _memory() == before
        assert np.array_equal(out.cpu().numpy(), ref_lab)
        assert got["obj"] == ref["obj"] and got["valid"]


def test_static_rounding_rejects_sizes_beyond_scratch():
    import torch

    from paper_1311_2661_gb300 import thetis as T

    n = 33_488_624 // 10 + 1  # n * reps just above the limit at reps = 10
    eu = torch.zeros(0, dtype=torch.int32, device="cuda")
    w = torch.ones(n, dtype=torch.float32, device="cuda")
    lab = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.ThetisError) as ei:
        T.thetis_round_is_static(n, eu, eu, w, w, lab, reps=10)
    assert ei.value.status == T.THETIS_E_INVALID
    assert "static scratch limit" in str(ei.value)


def test_static_rounding_rejects_bad_endpoints_and_host_pointers():
    """An endpoint outside [0, n) is caught by the on-device check before any
    kernel indexes with it; a host array is refused before any kernel runs."""
    import torch

    from paper_1311_2661_gb300 import thetis as T

    n = 10
    w = torch.ones(n, dtype=torch.float32, device="cuda")
    x = torch.full((n,), 0.5, dtype=torch.float32, device="cuda")
    lab = torch.zeros(n, dtype=torch.uint8, device="cuda")
    eu = torch.tensor([0, 3], dtype=torch.int32, device="cuda")
    ev = torch.tensor([1, n], dtype=torch.int32, device="cuda")  # n is out of range
    with pytest.raises(T.ThetisError) as ei:
        T.thetis_round_is_static(n, eu, ev, w, x, lab, reps=2)
    assert ei.value.status == T.THETIS_E_INVALID and "endpoint" in str(ei.value)
    # the wrapper refuses host tensors; the C entry point refuses host pointers too
    with pytest.raises(ValueError):
        T.thetis_round_is_static(n, eu.cpu(), ev.cpu(), w, x, lab, reps=2)
    w_host = np.ones(n, np.float32)
    ev_ok = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    info = T.RoundInfo()
    st = T._lib.thetis_round_is_static(n, 2, eu.data_ptr(), ev_ok.data_ptr(), w_host.ctypes.data, x.data_ptr(), 0,
                                       2, lab.data_ptr(), C.byref(info), None)
    assert st == T.THETIS_E_INVALID
    # the context is still usable: a valid call succeeds afterwards
    got = T.thetis_round_is_static(n, eu, ev_ok, w, x, lab, reps=2)
    assert got["valid"]

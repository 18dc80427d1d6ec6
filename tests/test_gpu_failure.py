"""Failure path of the bounded device waits.  No fault, trap or endless loop:
the persistent sweep's grid barriers are told to wait for one CTA more than the
launch has (set on the host), so the first wait runs out after its short time
limit, the kernel records the timeout and returns, and the solve reports
THETIS_E_TIMEOUT.  The handle, the context and the GPU stay usable: the same
handle solves again and a fresh solve still matches the oracle."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import X_TOL, build_gpu, gpu, gpu_full_x, vc_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit_ms", [1.0, 20.0])
def test_barrier_wait_runs_out_and_the_gpu_stays_usable(limit_ms):
    import time

    T = gpu()
    g = vc_graph(3000, 12000, 7)
    h = build_gpu("vc", g, seed=2)
    T.thetis_set_wait_limit(h, limit_ms, missing_ctas=1)
    t0 = time.perf_counter()
    with pytest.raises(T.ThetisError) as ei:
        h.solve(beta=100.0, epochs=10, refresh_every=10, engine=0)
    took = time.perf_counter() - t0
    assert ei.value.status == T.THETIS_E_TIMEOUT
    assert took < 5.0  # the wait ended at its limit, not at the 2 s default or later
    # the same handle runs again once the barriers are whole
    T.thetis_set_wait_limit(h, 2000.0, missing_ctas=0)
    info = h.solve(beta=100.0, epochs=10, refresh_every=10, engine=0)
    assert info["epochs_run"] == 10
    # a fresh solve on the same GPU matches the oracle
    h2 = build_gpu("vc", g, seed=2)
    h2.solve(beta=100.0, epochs=30, refresh_every=10, engine=0)
    lp = oracle.build_problem("vc", g)
    x_o, _ = lp.solve(beta=100.0, epochs=30, refresh_every=10, color=lp.color(2)[0])
    assert np.max(np.abs(gpu_full_x(h2) - x_o)) <= X_TOL


def test_wait_limit_argument_checks():
    T = gpu()
    h = build_gpu("vc", vc_graph(50, 100, 1))
    for bad in ((0.0, 0), (-1.0, 0), (10.0, -1), (10.0, 5000)):
        with pytest.raises(T.ThetisError):
            T.thetis_set_wait_limit(h, *bad)

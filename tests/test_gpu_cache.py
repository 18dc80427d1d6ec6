"""The library's device memory pool: memory freed by a destroyed handle stays
reserved and serves the next build, a trim gives back only unused reserve,
and builds before and after a trim agree."""
import numpy as np
import pytest

from tests.gpu_common import gpu, vc_graph

pytestmark = pytest.mark.gpu


def _build(T, g):
    h = T.thetis_build_vc(g.n, g.eu, g.ev, g.w, seed=3)
    h.solve(beta=100.0, epochs=20, refresh_every=10)
    return h


def test_pool_reuse_and_trim():
    T = gpu()
    g = vc_graph(20000, 80000, 5)
    h = _build(T, g)
    x0, c0 = h.get_x(), h.colors()
    r_live, u_live = T.thetis_cache_info()
    assert u_live > 0 and r_live >= u_live
    h.close()
    r_free, u_free = T.thetis_cache_info()
    assert u_free < u_live and r_free >= r_live - (u_live - u_free) and r_free >= u_free
    # the next build of the same size is served from the reserve (a little
    # slack for the pool's chunking)
    h = _build(T, g)
    r_again, _ = T.thetis_cache_info()
    assert r_again <= r_free + (32 << 20)
    np.testing.assert_array_equal(h.get_x(), x0)
    # trimming never touches memory in use, and the handle stays valid
    _, u_held = T.thetis_cache_info()
    T.thetis_trim_cache(0)
    r_trim, u_trim = T.thetis_cache_info()
    assert u_trim == u_held and r_trim >= u_trim and r_trim <= r_again
    np.testing.assert_array_equal(h.get_x(), x0)
    np.testing.assert_array_equal(h.colors(), c0)
    h.close()
    # a build after the trim maps memory again and gives the same result
    h = _build(T, g)
    np.testing.assert_array_equal(h.get_x(), x0)
    h.close()

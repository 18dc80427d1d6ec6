"""The C ABI: libthetis.so builds for sm_103a, loads, and exports every
function include/thetis.h declares (no compute call: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "thetis.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(thetis_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1311_2661_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("thetis_create", "thetis_build_vc", "thetis_build_is", "thetis_build_mc", "thetis_solve",
                 "thetis_round", "thetis_get_x", "thetis_destroy", "thetis_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_exposes_the_same_names(lib):
    from paper_1311_2661_gb300 import thetis

    for n in _declared():
        if n in ("thetis_sync",):
            continue
        assert hasattr(thetis, n), n


def test_calls_fail_cleanly_without_a_device(lib):
    """Without a GPU every call returns an error status, never aborts."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1311_2661_gb300 import thetis

    import numpy as np

    with pytest.raises(thetis.ThetisError) as ei:
        thetis.thetis_build_vc(3, np.array([0, 1]), np.array([1, 2]), np.ones(3))
    assert ei.value.status in (thetis.THETIS_E_CUDA, thetis.THETIS_E_INVALID)

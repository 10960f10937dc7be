"""lbm_fields_static: the field read-back for callers that cannot allocate.

A program whose device memory belongs to another allocator (PyTorch keeps
freed blocks in its own cache, so a raw cudaMalloc may fail while the process
still has memory) or that must not stall other streams with cudaFree can
call lbm_fields_static instead of lbm_fields: it stages the result in a fixed
array built into the library.  These tests call it through the C ABI and
compare it with lbm_fields, which stages through a buffer it allocates.

This file is collected last on purpose, and its tests pass both alone in a
fresh process and after the rest of the suite (the fixed array is set up on
the first call on a device and keeps the last call's contents).
"""
import numpy as np
import pytest

import paper_1303_0625_gb300 as G
from paper_1303_0625_gb300 import lbm as L

pytestmark = pytest.mark.gpu


def _lattice(nx, ny, precision):
    lat = G.Lattice(nx, ny, 0.8, bc_y=G.LBM_WALL, wall_ux=(0.0, 0.02), precision=precision)
    lat.add_disk(0.3 * nx, 0.5 * ny, 7.2, 0.06, 0.01)
    lat.add_disk(0.7 * nx, 0.4 * ny, 5.1, -0.05, 0.02, 0.01)
    return lat


def _both(lat):
    ref = [np.empty((lat.ny, lat.nx)) for _ in range(3)]
    got = [np.full((lat.ny, lat.nx), 7.0) for _ in range(3)]
    L.lbm_fields(lat.handle, *ref)
    L.lbm_fields_static(lat.handle, *got)
    return ref, got


@pytest.mark.parametrize("precision", [G.LBM_FP64, G.LBM_FP32_DEV])
def test_static_fields_match_allocating_fields_twice(precision):
    """Two calls in a row, with steps in between, give what lbm_fields gives
    (identical up to the FP64 tolerance of the parity tests, 1e-12)."""
    lat = _lattice(96, 64, precision)
    for steps in (15, 40):
        lat.step(steps)
        ref, got = _both(lat)
        for a, b in zip(ref, got):
            solid = np.isnan(a)
            assert np.array_equal(solid, np.isnan(b))
            assert np.abs(a[~solid] - b[~solid]).max() <= 1e-12
        assert solid.any() and (~solid).any()


def test_static_fields_after_a_smaller_domain():
    """The fixed array keeps the previous call's contents; a smaller domain
    read afterwards still gets exactly its own values."""
    big = _lattice(128, 96, G.LBM_FP64)
    big.step(5)
    _both(big)
    small = _lattice(40, 32, G.LBM_FP64)
    small.step(7)
    ref, got = _both(small)
    for a, b in zip(ref, got):
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.abs(np.nan_to_num(a) - np.nan_to_num(b)).max() <= 1e-12


def test_static_fields_reject_domains_above_the_maximum():
    nx, ny = 1024, 1024  # 2^20 nodes > LBM_FIELDS_STATIC_MAX_NODES
    assert nx * ny > L.LBM_FIELDS_STATIC_MAX_NODES
    lat = G.Lattice(nx, ny, 0.8, precision=G.LBM_FP32_DEV)
    out = [np.zeros((ny, nx)) for _ in range(3)]
    with pytest.raises(L.LBMError) as e:
        L.lbm_fields_static(lat.handle, *out)
    assert e.value.status == L.LBM_EINVAL
    assert "maximum" in str(e.value)
    assert not out[0].any()

"""Batches of independent channels (one fixed cylinder each) stepped by the
batch kernels: every case against its own single-domain run and against the
FP64 oracle, convergence and retirement, launch policies, isolation of an
unstable case, and the autotuner's cache.

Tolerances are those of the single-domain parity tests: FP64 forces <= 1e-12
relative (scale as in _pairs.force_rel) and populations <= 1e-12 absolute;
FP32 forces <= 1e-5.  A batch case and the same case run alone evaluate the
same expressions, so they are compared at rounding level.
"""
import json

import numpy as np
import pytest

import paper_1303_0625_gb300 as G
import workloads as W
from _pairs import PREC, force_rel, make_gpu, make_oracle
from paper_1303_0625_gb300 import lbm as L

pytestmark = pytest.mark.gpu


def _sweep(n, seed=31, nx=(40, 150), ny=(24, 64), **kw):
    return W.cylinder_sweep(n, seed_offset=seed, nx_range=nx, ny_range=ny, **kw)


def _batch(ws, precision="fp64", ring=256, **kw):
    return G.Batch.from_workloads(ws, precision=PREC[precision], force_ring=ring, **kw)


def _assert_same_case(b, k, w, steps, precision):
    """Case k of the batch agrees with the same workload run alone to
    rounding: the batch computes the open columns in its per-node path (the
    neighbour's update recomputed there) where the single domain reads the
    neighbour's stored update, and it splits a disk's link sums over the
    warps of a block.  Populations within 1e-12 (FP64) / 1e-6 (FP32,
    |f| < 0.5), forces within 1e-13 / 1e-6 of the force scale."""
    alone = make_gpu(w, precision, ring=steps)
    alone.step(steps)
    v = b.case(k)
    assert v.t == steps
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.abs(v.get_f() - alone.get_f()).max() <= (1e-12 if precision == "fp64" else 1e-6)
    radii = [s["r"] for s in w["solids"]]
    assert force_rel(v.forces(0, steps), alone.forces(0, steps), radii) <= tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_cases_equal_single_domain_runs(precision):
    """Six uneven channels; 130 steps with a test every 50 (a partial block
    at the end), graph replay on."""
    ws = _sweep(6)
    b = _batch(ws, precision)
    b.set_convergence(every=50, tol=0.0, max_steps=10**6)
    assert b.run(130) == 6
    st, steps, drag = b.state()
    assert (st == L.LBM_CASE_ACTIVE).all() and (steps == 130).all()
    for k, w in enumerate(ws):
        _assert_same_case(b, k, w, 130, precision)


def test_batch_against_fp64_oracle():
    ws = _sweep(3, seed=37)
    b = _batch(ws, "fp64")
    b.run(60)
    for k, w in enumerate(ws):
        o = make_oracle(w)
        ref = o.step(60)
        v = b.case(k)
        got = v.forces(0, 60)
        assert force_rel(got, ref, [s["r"] for s in w["solids"]]) <= 1e-12
        own = o.owner()
        assert np.array_equal(v.owner(), own)
        fl = own < 0
        assert np.abs(v.get_f()[:, fl] - o.get_f()[:, fl]).max() <= 1e-12


def test_batch_fp32_forces_against_fp64_oracle():
    ws = _sweep(3, seed=41)
    b = _batch(ws, "fp32")
    b.run(100)
    for k, w in enumerate(ws):
        ref = make_oracle(w).step(100)
        got = b.case(k).forces(0, 100)
        assert force_rel(got, ref, [s["r"] for s in w["solids"]]) <= 1e-5


@pytest.mark.parametrize("variant,rows,persistent",
                         [(0, 1, False), (1, 1, False), (2, 1, False), (1, 2, False),
                          (2, 4, False), (1, 3, False), (0, 1, True), (1, 2, True), (2, 1, True)])
def test_batch_launch_policies_agree(variant, rows, persistent):
    """Tile width and height, persistent or per-tile blocks, graph or direct launches:
    the same arithmetic, compiled separately per width, so populations agree
    to FP32 rounding (a few ulp after 40 steps; |f| < 0.5)."""
    ws = _sweep(4, seed=43)
    ref = _batch(ws, "fp32")
    ref.set_launch(0, 1, False, graph=False)
    ref.run(40)
    b = _batch(ws, "fp32")
    b.set_launch(variant, rows, persistent, graph=True)
    b.set_convergence(every=20, tol=0.0, max_steps=10**6)
    b.run(40)
    assert b.launch() == (variant, rows, int(persistent))
    for k in range(len(ws)):
        assert np.abs(b.case(k).get_f() - ref.case(k).get_f()).max() <= 1e-6


def test_convergence_retires_cases_and_freezes_them():
    """With a loose tolerance the low-Re cases converge first; a retired case
    stops stepping (its clock and populations stay as they were) while the
    others go on, and the reported drag is that of its latest record."""
    ws = _sweep(5, seed=47, nx=(48, 96), ny=(24, 40))
    b = _batch(ws, "fp32", ring=8)
    every = 25
    b.set_convergence(every=every, tol=2e-3, max_steps=10**6)
    active = b.run(3000)
    st, steps, drag = b.state()
    done = np.flatnonzero(st == L.LBM_CASE_CONVERGED)
    assert done.size >= 1 and active == int((st == L.LBM_CASE_ACTIVE).sum())
    assert (steps % every == 0).all()
    for k in done:
        v = b.case(int(k))
        rec = v.forces(int(steps[k]) - 1, 1)  # [1][nsolid][2][3]
        assert drag[k] == rec[0, :, 1, 0].sum()
    frozen = {int(k): b.case(int(k)).get_f() for k in done}
    b.run(2 * every)
    st2, steps2, _ = b.state()
    for k, f in frozen.items():
        assert st2[k] == L.LBM_CASE_CONVERGED and steps2[k] == steps[k]
        assert np.array_equal(b.case(k).get_f(), f)
    for k in np.flatnonzero(st == L.LBM_CASE_ACTIVE):
        assert steps2[k] == steps[k] + 2 * every or st2[k] != L.LBM_CASE_ACTIVE


def test_convergence_window_needs_consecutive_calm_tests():
    """With a tolerance every test passes (tol 10), a case retires at the
    first test that finds the drag within tol of the previous one (the second
    test: the first has no history), or, with a window of w tests, after w
    such tests in a row; a window needs w >= 1."""
    ws = _sweep(3, seed=59)
    every = 10
    for window, expect in ((1, 2 * every), (4, 5 * every)):
        b = _batch(ws, "fp32", ring=4)
        b.set_convergence(every=every, tol=10.0, max_steps=10**6, window=window)
        assert b.run(1000) == 0
        st, steps, _ = b.state()
        assert (st == L.LBM_CASE_CONVERGED).all() and (steps == expect).all(), (window, steps)
        b.close()
    b = _batch(ws, "fp32", ring=4)
    with pytest.raises(G.LBMError) as e:
        L.lbm_batch_set_convergence_window(b.handle, 0)
    assert e.value.status == G.LBM_EINVAL
    b.close()


def test_step_cap_and_all_retired():
    ws = _sweep(3, seed=53)
    b = _batch(ws, "fp32", ring=4)
    b.set_convergence(every=10, tol=0.0, max_steps=30)
    assert b.run(1000) == 0
    st, steps, _ = b.state()
    assert (st == L.LBM_CASE_CAPPED).all() and (steps == 30).all()
    n0 = b.launch_count()
    assert b.run(100) == 0  # nothing left to step
    assert b.launch_count() - n0 <= 1  # only the final read-back


def test_unstable_case_is_isolated():
    """A case driven far past the stability limit is retired as unstable;
    the other cases are unaffected (they agree with their runs alone)."""
    ws = _sweep(3, seed=59)
    bad = dict(ws[1], tau=0.5001, inflow_umax=0.9)
    ws2 = [ws[0], bad, ws[2]]
    b = _batch(ws2, "fp32", ring=300)
    b.set_convergence(every=25, tol=0.0, max_steps=10**6)
    b.run(300)
    st, steps, _ = b.state()
    assert st[1] == L.LBM_CASE_UNSTABLE and steps[1] < 300
    assert st[0] == st[2] == L.LBM_CASE_ACTIVE
    for k in (0, 2):
        _assert_same_case(b, k, ws2[k], 300, "fp32")


def test_batch_case_calls_that_step_are_refused():
    ws = _sweep(2, seed=61)
    b = _batch(ws, "fp32")
    v = b.case(0)
    for call in (lambda: L.lbm_step(v.handle, 1), lambda: v.add_disk(10.0, 10.0, 3.0),
                 lambda: L.lbm_destroy(v.handle)):
        with pytest.raises(L.LBMError) as e:
            call()
        assert e.value.status == L.LBM_EINVAL
    with pytest.raises(L.LBMError) as e:
        L.lbm_batch_add_solid(b.handle, 0, L.lbm_disk(cx=20.0, cy=12.0, r=3.0, vx=0.01))
    assert e.value.status == L.LBM_EINVAL
    cfgs = [G.lbm.make_config(64, 32, 0.8, precision=G.LBM_FP32_DEV),
            G.lbm.make_config(64, 32, 0.8, precision=G.LBM_FP64)]
    with pytest.raises(L.LBMError) as e:
        G.Batch(cfgs)
    assert e.value.status == L.LBM_EINVAL and "precision" in str(e.value)


def test_autotune_and_json_cache(tmp_path):
    ws = _sweep(8, seed=67)
    b = _batch(ws, "fp32", ring=4)
    cache = tmp_path / "tune.json"
    best = b.autotune(steps=3, cache=str(cache))
    assert b.launch() == best
    table = json.loads(cache.read_text())
    assert list(table.values()) == [list(best)]
    _, steps, _ = b.state()
    assert (steps == L.LBM_BATCH_TUNE_SHAPES * 4).all()  # every shape x (1 + 3) real steps
    b2 = _batch(ws, "fp32", ring=4)
    assert b2.autotune(steps=3, cache=str(cache)) == best
    _, steps2, _ = b2.state()
    assert (steps2 == 0).all()  # taken from the cache, nothing timed


def test_batch_timing_counts_fused_launches():
    ws = _sweep(4, seed=71)
    b = _batch(ws, "fp32", ring=4)
    b.set_timing(True)
    b.run(12)
    ms, n = b.timing()
    assert n == 12 and ms > 0.0

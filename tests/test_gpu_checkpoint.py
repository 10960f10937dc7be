"""Checkpoints (lbm_save, lbm_load) and the time-out path of the bounded
device waits, through the C ABI.

Resuming from a saved state must give the steps that followed the save bit
for bit, in every precision, with prescribed and free disks crossing nodes.
The time-out test stalls nothing: a wait limit of 0 makes every grid-wide
barrier of the re-rasterisation give up at once, the launch returns, and the
host reports LBM_ETIMEOUT; the context then resumes from a saved state."""
import numpy as np
import pytest

import workloads as W
import paper_1303_0625_gb300 as G
from _pairs import make_gpu, seeded_f

pytestmark = pytest.mark.gpu


def _case(**kw):
    w = dict(nx=72, ny=64, tau=0.7, rho0=1.0, bc_x=W.PERIODIC, bc_y=W.WALL, u0=(0.0, 0.0),
             wall_ux=(0.0, 0.02), body_force=(0.0, 0.0), rho_w_mode=W.RHOW_LOCAL, refill=1,
             gravity=(0.0, -2e-4), lub_range=2.0,
             solids=[dict(cx=18.3, cy=40.1, r=6.2, vx=0.08, vy=-0.05, omega=0.01, rho_s=1.0,
                          motion=0),
                     dict(cx=45.7, cy=30.4, r=5.1, vx=0.0, vy=0.0, omega=0.0, rho_s=1.5,
                          motion=1),
                     dict(cx=58.0, cy=14.0, r=4.0, vx=0.0, vy=0.0, omega=0.0, rho_s=1.0,
                          motion=0)])
    w.update(kw)
    return w


def _lattice(w, precision):
    g = make_gpu(w, precision, ring=64)
    g.set_f(seeded_f(w, 5))
    return g


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_save_load_resumes_bit_for_bit(precision):
    w = _case()
    ref = _lattice(w, precision)
    whole = ref.step_record(60)

    g = _lattice(w, precision)
    first = g.step_record(30)
    state = g.save()
    g.step(17)  # the saving context moves on

    h = _lattice(w, precision)  # a fresh context with the same solids
    h.load(state)
    assert h.t == 30
    second = h.step_record(30)
    assert np.array_equal(np.concatenate([first, second]), whole)
    assert np.array_equal(h.get_f(), ref.get_f())
    assert np.array_equal(h.owner(), ref.owner())
    assert np.array_equal(h.solids(), ref.solids())
    # records from before the save are restored with the state
    assert np.array_equal(h.forces(0, 30), first)

    g.load(state)  # and back into the context that moved on
    assert np.array_equal(g.step_record(30), whole[30:])


def test_load_rejects_other_configurations():
    w = _case()
    g = _lattice(w, "fp32")
    g.step(5)
    state = g.save()
    other = make_gpu(_case(tau=0.71), "fp32")
    with pytest.raises(G.LBMError) as e:
        other.load(state)
    assert e.value.status == G.LBM_EINVAL
    fewer = make_gpu(dict(_case(), solids=_case()["solids"][:2]), "fp32")
    with pytest.raises(G.LBMError) as e:
        fewer.load(state)
    assert e.value.status == G.LBM_EINVAL
    with pytest.raises(G.LBMError) as e:
        g.load(state[: len(state) // 2])
    assert e.value.status == G.LBM_EINVAL
    junk = np.zeros_like(state)
    with pytest.raises(G.LBMError) as e:
        g.load(junk)
    assert e.value.status == G.LBM_EINVAL
    # nothing changed: the context steps on as before
    ref = _lattice(w, "fp32")
    ref.step(5)
    assert np.array_equal(g.step_record(8), ref.step_record(8))


def test_barrier_time_out_is_reported_and_the_saved_state_resumes():
    w = _case()
    ref = _lattice(w, "fp32")
    whole = ref.step_record(20)

    g = _lattice(w, "fp32")
    g.step(10)
    state = g.save()
    g.set_wait_limit(0)  # every grid barrier gives up at once
    g.step(3)
    with pytest.raises(G.LBMError) as e:
        g.sync()
    assert e.value.status == G.LBM_ETIMEOUT
    with pytest.raises(G.LBMError) as e:  # the condition persists
        g.sync()
    assert e.value.status == G.LBM_ETIMEOUT
    with pytest.raises(G.LBMError):  # and such a state is not saved
        g.save()

    g.set_wait_limit(1 << 24)
    g.load(state)
    assert np.array_equal(g.step_record(10), whole[10:])
    g.sync()

"""CUDA path vs the FP64 oracle, element by element, on seeded inputs.

Tolerances (stated by the method's precision targets; a force's scale is the
larger of its largest magnitude over the run and the one-sided pressure force
2 rho0 r / 3 on the disk, see _pairs.force_rel):
  FP64 storage and arithmetic:  forces <= 1e-12 relative; populations at
      fluid nodes <= 1e-12 absolute; owner map,
      link list and solid positions exact (integer and geometric decisions are
      rounded identically on both sides);
  FP32 with f - w_i storage:    forces <= 1e-5 relative;
  FP16 with f - w_i storage:    forces <= 1e-3 relative.
"""
import numpy as np
import pytest

import workloads as W
from _pairs import describe, force_rel, make_gpu, make_oracle, rel, run_pair

pytestmark = pytest.mark.gpu


def _disks(*specs):
    out = []
    for s in specs:
        cx, cy, r = s[:3]
        vx, vy, om = (list(s[3:6]) + [0.0, 0.0, 0.0])[:3]
        out.append(dict(cx=cx, cy=cy, r=r, vx=vx, vy=vy, omega=om, rho_s=s[6] if len(s) > 6 else 1.0,
                        motion=s[7] if len(s) > 7 else 0))
    return out


def _case(nx, ny, tau, solids, **kw):
    w = dict(nx=nx, ny=ny, tau=tau, rho0=1.0, bc_x=W.PERIODIC, bc_y=W.PERIODIC, u0=(0.0, 0.0),
             wall_ux=(0.0, 0.0), body_force=(0.0, 0.0), rho_w_mode=W.RHOW_CONST, refill=1,
             solids=solids)
    w.update(kw)
    return w


def _check_fp64(o, g, ref, got, ftol=1e-12):
    assert got.shape == ref.shape
    radii = [o.solid_radius(s) for s in range(o.nsolid)]
    err = force_rel(got, ref, radii)
    assert err <= ftol, describe(got, ref, radii)
    own = o.owner()
    assert np.array_equal(g.owner(), own)
    fl = own < 0
    fo, fg = o.get_f(), g.get_f()
    assert np.abs(fg[:, fl] - fo[:, fl]).max() <= 1e-12
    for s in range(o.nsolid):
        assert np.allclose(g.solids()[s], o.solid_state(s), rtol=1e-13, atol=1e-15)


MOVING = _disks((15.3, 12.1, 5.2, 0.09, 0.04, 0.01), (31.7, 27.4, 6.1, -0.07, -0.08, -0.02))


@pytest.mark.parametrize("rho_w_mode", [W.RHOW_CONST, W.RHOW_LOCAL])
@pytest.mark.parametrize("bc", [(W.PERIODIC, W.PERIODIC), (W.PERIODIC, W.WALL)])
def test_moving_rotating_disks_fp64(rho_w_mode, bc):
    w = _case(48, 40, 0.7, MOVING, rho_w_mode=rho_w_mode, bc_x=bc[0], bc_y=bc[1],
              wall_ux=(0.0, 0.03) if bc[1] == W.WALL else (0.0, 0.0))
    o, g, ref, got = run_pair(w, 80, perturb=1)
    _check_fp64(o, g, ref, got)


@pytest.mark.parametrize("refill", [1, 2, 3])
def test_refill_variants_fp64(refill):
    w = _case(56, 44, 0.8, _disks((20.2, 20.7, 7.3, 0.1, -0.06), (40.1, 12.9, 4.4, -0.1, 0.1)),
              refill=refill)
    o, g, ref, got = run_pair(w, 60, perturb=2)
    _check_fp64(o, g, ref, got)


@pytest.mark.parametrize("nx,ny", [(77, 45), (130, 33), (64, 64)])
def test_ragged_sizes_fp64(nx, ny):
    """Rows that are not a multiple of the block width or the row pitch."""
    w = _case(nx, ny, 0.9, _disks((nx * 0.3, ny * 0.5, 6.6, 0.05, 0.02), (nx * 0.75, ny * 0.3, 4.1)),
              bc_y=W.WALL, wall_ux=(-0.01, 0.02))
    o, g, ref, got = run_pair(w, 40, perturb=3)
    _check_fp64(o, g, ref, got)


def test_overlapping_disks_lowest_id_fp64():
    """Prescribed disks that run into each other: lowest id owns the overlap."""
    w = _case(64, 40, 0.75, _disks((20.0, 20.0, 6.0, 0.1, 0.0), (36.0, 20.4, 6.0, -0.1, 0.0)))
    o, g, ref, got = run_pair(w, 70, perturb=4)
    assert (o.owner() >= 0).sum() < 2 * 113  # they do overlap by the end
    _check_fp64(o, g, ref, got)


def test_free_disks_walls_gravity_lubrication_fp64():
    w = _case(72, 96, 0.7, _disks((20.0, 70.0, 6.0, 0.0, 0.0, 0.0, 1.5, 1),
                                  (34.5, 71.0, 6.0, 0.0, 0.0, 0.0, 1.5, 1),
                                  (50.0, 60.0, 5.0, 0.0, 0.0, 0.0, 2.0, 1)),
              bc_x=W.WALL, bc_y=W.WALL, gravity=(0.0, -2e-4), lub_range=2.0)
    o, g, ref, got = run_pair(w, 150)
    _check_fp64(o, g, ref, got)


@pytest.mark.parametrize("motion_cme,relative", [(0, 0), (1, 0), (0, 1)])
def test_free_disk_in_moving_frame_fp64(motion_cme, relative):
    """A free disk settling in a channel whose walls, fluid and disk all carry
    the frame velocity V = 0.02 (the Galilean test of Sec. III.A), driven by
    Eq. 5 or, for comparison, Eq. 4, with the node-type momenta of the Eq. 5
    record booked in absolute or relative momentum: the same trajectory and
    records as the oracle."""
    w = _case(80, 40, 0.6, _disks((48.0, 7.1, 5.0, 0.02, 0.0, 0.0, 1.5, 1)), bc_y=W.WALL,
              u0=(0.02, 0.0), wall_ux=(0.02, 0.02), gravity=(-6e-4, 0.0), motion_cme=motion_cme,
              relative_changes=relative)
    o, g, ref, got = run_pair(w, 200)
    _check_fp64(o, g, ref, got)


def test_open_channel_fixed_disk_fp64():
    w = _case(160, 64, 0.6, _disks((40.0, 33.0, 6.4)), bc_x=W.OPEN, bc_y=W.WALL,
              inflow_umax=0.06)
    o, g, ref, got = run_pair(w, 300)
    _check_fp64(o, g, ref, got)


def test_body_force_channel_fp64():
    w = _case(24, 16, 0.9, _disks((12.0, 8.0, 3.0)), bc_y=W.WALL, body_force=(2e-6, 0.0))
    o, g, ref, got = run_pair(w, 200)
    _check_fp64(o, g, ref, got)
    ro, uxo, uyo = o.fields()
    rg, uxg, uyg = g.fields()
    fl = o.owner() < 0
    assert np.abs(uxg[fl] - uxo[fl]).max() < 1e-14
    assert np.isnan(rg[~fl]).all()


def test_link_list_exact():
    w = _case(50, 38, 0.8, _disks((10.2, 11.0, 4.3, 0.05), (30.0, 20.0, 7.7, -0.04, 0.06),
                                  (46.0, 30.0, 5.0)), bc_y=W.WALL)
    o, g, ref, got = run_pair(w, 37)
    assert np.array_equal(g.links(), o.links())


def test_graph_replay_matches_direct_launches():
    w = _case(48, 40, 0.7, MOVING, rho_w_mode=W.RHOW_LOCAL)
    g1 = make_gpu(w, ring=64)
    g2 = make_gpu(w, ring=64)
    g2.set_graph(8)
    a = g1.step_record(40)
    b = g2.step_record(40)
    # every sum runs in a fixed order (no atomics in floating point): the
    # replayed graph gives the same records, bit for bit
    assert np.array_equal(a, b)
    assert np.array_equal(g1.get_f(), g2.get_f())
    assert np.array_equal(g1.solids(), g2.solids())


# -------------------------------------------- the Galilean pair, 256 x 128

@pytest.mark.parametrize("run", ["a", "b"])
def test_galilean_pair_full_run_fp64(run):
    """Disk r = 12 in the 256 x 128 channel, tau 0.8, 5000 steps, both force
    forms every step, local rho_w."""
    w = W.galilean_pair(run)
    o, g, ref, got = run_pair(w, 5000)
    _check_fp64(o, g, ref, got)


# ------------------------------------------------------ precision modes

@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 1e-3)])
def test_precision_modes_against_fp64_oracle(prec, tol):
    """Deviation storage: forces at horizons 1, 10 and 100 steps against FP64."""
    w = W.precision_study(nx=256, ny=192, ndisk=40, seed_offset=2)
    o = make_oracle(w)
    g = make_gpu(w, prec, ring=128)
    for h in (1, 9, 90):
        ref = o.step(h)
        got = g.step_record(h)
        radii = [s["r"] for s in w["solids"]]
        err = force_rel(got, ref, radii)
        assert err <= tol, f"{prec} horizon {o.t}: " + describe(got, ref, radii)
    assert np.array_equal(g.owner(), o.owner())


def test_unstable_run_reports_status():
    """A velocity far beyond the lattice's stability limit is reported as
    LBM_EUNSTABLE by the next synchronising call (host-side check of a device
    flag; nothing faults)."""
    from paper_1303_0625_gb300 import lbm as L
    w = _case(32, 32, 0.5001, _disks((16.0, 16.0, 4.0)), u0=(0.9, 0.0))
    g = make_gpu(w, "fp32")
    g.step(400)
    with pytest.raises(L.LBMError) as e:
        g.sync()
    assert e.value.status == L.LBM_EUNSTABLE

"""Interpolated boundary on the disks (LBM_INTERPOLATED; the boundary
condition of the paper's simulations, Sec. IV, ref. [40]) on the CUDA path
against the FP64 oracle, with the parity tests' tolerances: FP64 populations
and forces to 1e-12, FP32 forces to 1e-5, FP16 to 1e-3."""
import numpy as np
import pytest

import workloads as W
from _pairs import describe, force_rel, run_pair

import paper_1303_0625_gb300 as G

DISKS = [dict(cx=15.3, cy=12.1, r=5.2, vx=0.09, vy=0.04, omega=0.01, rho_s=1.0, motion=0),
         dict(cx=31.7, cy=27.4, r=6.1, vx=-0.07, vy=-0.08, omega=-0.02, rho_s=1.0, motion=0)]


def _case(**kw):
    w = dict(nx=48, ny=40, tau=0.7, rho0=1.0, bc_x=W.PERIODIC, bc_y=W.WALL, u0=(0.0, 0.0),
             wall_ux=(0.0, 0.03), body_force=(0.0, 0.0), rho_w_mode=W.RHOW_CONST, refill=1,
             solids=DISKS, boundary=G.LBM_INTERPOLATED)
    w.update(kw)
    return w


def _radii(w):
    return [s["r"] for s in w["solids"]]


def _check_fp64(o, g, ref, got, w, ftol=1e-12):
    assert force_rel(got, ref, _radii(w)) <= ftol, describe(got, ref, _radii(w))
    assert np.array_equal(g.owner(), o.owner())
    fl = o.owner() < 0
    assert np.abs(g.get_f()[:, fl] - o.get_f()[:, fl]).max() <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("kw", [{}, {"rho_w_mode": W.RHOW_LOCAL},
                                {"bc_y": W.PERIODIC, "wall_ux": (0.0, 0.0)},
                                {"collision": G.LBM_MRT}])
def test_interpolated_moving_disks_fp64(kw):
    w = _case(**kw)
    o, g, ref, got = run_pair(w, 80, perturb=1)
    _check_fp64(o, g, ref, got, w)


@pytest.mark.gpu
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
def test_interpolated_every_launch_variant_fp64(variant):
    """With the interpolated boundary the per-node path runs deferred whatever
    the requested variant; every width gives the oracle's result."""
    w = _case()
    o, g, ref, got = run_pair(w, 40, perturb=2, variant=variant)
    _check_fp64(o, g, ref, got, w)
    launches = g.launch_count()
    g.step(1)
    g.sync()
    assert g.launch_count() - launches == 5  # forces, ring, fused, update, re-rasterisation


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16", 1e-3)])
def test_interpolated_deviation_modes(precision, tol):
    w = _case()
    o, g, ref, got = run_pair(w, 80, precision=precision, perturb=1)
    assert force_rel(got, ref, _radii(w)) <= tol


@pytest.mark.gpu
@pytest.mark.parametrize("motion_cme,relative", [(0, 0), (0, 1)])
def test_interpolated_free_disk_in_moving_frame_fp64(motion_cme, relative):
    """The Galilean test's setting (Sec. III.A) with the paper's boundary: a
    free disk settling in a channel moving at V = 0.02."""
    w = _case(nx=80, ny=40, tau=0.6,
              solids=[dict(cx=48.0, cy=7.1, r=5.0, vx=0.02, vy=0.0, omega=0.0, rho_s=1.5,
                           motion=1)],
              u0=(0.02, 0.0), wall_ux=(0.02, 0.02), gravity=(-6e-4, 0.0), motion_cme=motion_cme,
              relative_changes=relative)
    o, g, ref, got = run_pair(w, 200)
    _check_fp64(o, g, ref, got, w)


def test_batches_reject_the_interpolated_boundary():
    c = G.lbm.make_config(32, 32, 0.8, boundary=G.LBM_INTERPOLATED)
    with pytest.raises(G.LBMError) as e:
        G.lbm.lbm_batch_create([c])
    assert e.value.status == G.LBM_EINVAL

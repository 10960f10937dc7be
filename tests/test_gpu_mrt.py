"""MRT collision (Sec. IV: S = diag(0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1/tau, 1/tau))
on the CUDA path against the FP64 oracle, with the parity tests' tolerances:
FP64 populations and forces to 1e-12, FP32 forces to 1e-5, FP16 to 1e-3."""
import numpy as np
import pytest

import workloads as W
from _pairs import force_rel, run_pair

import paper_1303_0625_gb300 as G

DISKS = [dict(cx=15.3, cy=12.1, r=5.2, vx=0.09, vy=0.04, omega=0.01, rho_s=1.0, motion=0),
         dict(cx=31.7, cy=27.4, r=6.1, vx=-0.07, vy=-0.08, omega=-0.02, rho_s=1.0, motion=0)]


def _case(**kw):
    w = dict(nx=48, ny=40, tau=0.7, rho0=1.0, bc_x=W.PERIODIC, bc_y=W.WALL, u0=(0.0, 0.0),
             wall_ux=(0.0, 0.03), body_force=(0.0, 0.0), rho_w_mode=W.RHOW_CONST, refill=1,
             solids=DISKS, collision=G.LBM_MRT)
    w.update(kw)
    return w


def _radii(w):
    return [s["r"] for s in w["solids"]]


@pytest.mark.gpu
@pytest.mark.parametrize("kw", [{}, {"rho_w_mode": W.RHOW_LOCAL}, {"bc_y": W.PERIODIC,
                                                                  "wall_ux": (0.0, 0.0)}])
def test_mrt_moving_disks_fp64(kw):
    w = _case(**kw)
    o, g, ref, got = run_pair(w, 80, perturb=1)
    assert force_rel(got, ref, _radii(w)) <= 1e-12
    fl = o.owner() < 0
    assert np.array_equal(g.owner(), o.owner())
    assert np.abs(g.get_f()[:, fl] - o.get_f()[:, fl]).max() <= 1e-12


@pytest.mark.gpu
def test_mrt_open_channel_fp64():
    w = _case(nx=160, ny=64, tau=0.6, bc_x=W.OPEN, wall_ux=(0.0, 0.0), inflow_umax=0.06,
              solids=[dict(cx=40.0, cy=33.0, r=6.4, vx=0.0, vy=0.0, omega=0.0, rho_s=1.0,
                           motion=0)])
    o, g, ref, got = run_pair(w, 300)
    assert force_rel(got, ref, _radii(w)) <= 1e-12
    fl = o.owner() < 0
    assert np.abs(g.get_f()[:, fl] - o.get_f()[:, fl]).max() <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("fp16", 1e-3)])
def test_mrt_deviation_modes(precision, tol):
    w = _case()
    o, g, ref, got = run_pair(w, 80, precision=precision, perturb=1)
    assert force_rel(got, ref, _radii(w)) <= tol


def test_mrt_rejects_body_force_and_batches():
    c = G.lbm.make_config(32, 32, 0.8, collision=G.LBM_MRT, body_force=(1e-6, 0.0))
    with pytest.raises(G.LBMError) as e:
        G.lbm.lbm_create(c)
    assert e.value.status == G.LBM_EINVAL
    c = G.lbm.make_config(32, 32, 0.8, collision=G.LBM_MRT)
    with pytest.raises(G.LBMError) as e:
        G.lbm.lbm_batch_create([c])
    assert e.value.status == G.LBM_EINVAL

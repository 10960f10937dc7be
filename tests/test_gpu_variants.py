"""Launch variants of the single-domain advection-collision kernel.

Variants 0-2 (nodes per thread, inline per-node path) and 3-5 (the same
widths, nodes next to solids and edges computed by a second kernel) evaluate
the same expressions, so they agree to the storage precision's rounding; the
deferred variants also match the FP64 oracle with the tolerances of the
parity tests (forces 1e-12 relative in FP64, 1e-5 in FP32).
"""
import numpy as np
import pytest

import workloads as W
from _pairs import force_rel, make_gpu, run_pair, seeded_f

pytestmark = pytest.mark.gpu

DISKS = [dict(cx=15.3, cy=12.1, r=5.2, vx=0.09, vy=0.04, omega=0.01, rho_s=1.0, motion=0),
         dict(cx=31.7, cy=27.4, r=6.1, vx=-0.07, vy=-0.08, omega=-0.02, rho_s=1.0, motion=0),
         dict(cx=52.0, cy=20.5, r=7.4, vx=0.0, vy=0.0, omega=0.0, rho_s=1.0, motion=0)]


def _case(bc_x, bc_y, **kw):
    w = dict(nx=72, ny=40, tau=0.7, rho0=1.0, bc_x=bc_x, bc_y=bc_y, u0=(0.0, 0.0),
             wall_ux=(0.0, 0.03) if bc_y == W.WALL else (0.0, 0.0), body_force=(0.0, 0.0),
             rho_w_mode=W.RHOW_CONST, refill=1, solids=DISKS)
    w.update(kw)
    return w


CASES = {
    "periodic": _case(W.PERIODIC, W.PERIODIC),
    "walls": _case(W.PERIODIC, W.WALL),
    "box": _case(W.WALL, W.WALL),
    "open": _case(W.OPEN, W.WALL, inflow_umax=0.04, wall_ux=(0.0, 0.0)),
    "local": _case(W.PERIODIC, W.WALL, rho_w_mode=W.RHOW_LOCAL),
}
TOL = {"fp64": 1e-13, "fp32": 1e-6, "fp16": 2e-3}


def _run(w, precision, variant, steps=30):
    g = make_gpu(w, precision, ring=steps)
    g.set_f(seeded_f(w, 1))
    g.set_kernel_variant(variant)
    rec = g.step_record(steps)
    g.sync()
    f = g.get_f()
    fl = g.owner() < 0
    g.close()
    return rec, f[:, fl]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_variants_agree(case, precision):
    w = CASES[case]
    ref_rec, ref_f = _run(w, precision, 0)
    radii = [s["r"] for s in w["solids"]]
    for v in range(1, 6):
        rec, f = _run(w, precision, v)
        assert f.shape == ref_f.shape
        assert np.abs(f - ref_f).max() <= TOL[precision], f"variant {v}"
        assert force_rel(rec, ref_rec, radii) <= 10 * TOL[precision], f"variant {v}"


@pytest.mark.parametrize("variant", [3, 4, 5])
@pytest.mark.parametrize("case", ["walls", "box", "open"])
def test_deferred_variants_match_oracle(case, variant):
    w = CASES[case]
    radii = [s["r"] for s in w["solids"]]
    for precision, ftol in (("fp64", 1e-12), ("fp32", 1e-5)):
        o, g, ref, got = run_pair(w, 40, precision=precision, perturb=1, variant=variant)
        assert force_rel(got, ref, radii) <= ftol, precision
        if precision == "fp64":
            fl = o.owner() < 0
            assert np.abs(g.get_f()[:, fl] - o.get_f()[:, fl]).max() <= 1e-12


def test_variant_range_and_autotune():
    g = make_gpu(CASES["walls"], "fp32", ring=8)
    for v in range(6):
        g.set_kernel_variant(v)
        assert g.kernel_variant() == v
    with pytest.raises(Exception):
        g.set_kernel_variant(6)
    best = g.autotune(2)
    assert 0 <= best < 6 and g.kernel_variant() == best
    assert g.force_overlap() in (0, 1)
    g.sync()
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_force_kernel_beside_or_before_gives_the_same_results(precision):
    """The force kernel reads only what the advection-collision kernel of the
    step reads, so running it beside that kernel (second stream) or before it
    changes nothing, bit for bit."""
    w = CASES["walls"]
    runs = []
    for on in (True, False):
        g = make_gpu(w, precision, ring=64)
        g.set_force_overlap(on)
        g.set_f(seeded_f(w, 3))
        runs.append((g.step_record(40), g.get_f(), g.owner(), g.solids()))
        g.close()
    for x, y in zip(*runs):
        assert np.array_equal(x, y)

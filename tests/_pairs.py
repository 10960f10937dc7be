"""Test helper: build the FP64 oracle and the CUDA lattice from one workload
description and compare them."""
import numpy as np

import oracle as O
import paper_1303_0625_gb300 as G

PREC = {"fp64": G.LBM_FP64, "fp32": G.LBM_FP32_DEV, "fp16": G.LBM_FP16_DEV}


def make_oracle(w):
    o = O.Oracle(w["nx"], w["ny"], w["tau"], rho0=w.get("rho0", 1.0), u0=w.get("u0", (0, 0)),
                 bc_x=w["bc_x"], bc_y=w["bc_y"], wall_ux=w.get("wall_ux", (0, 0)),
                 body_force=w.get("body_force", (0, 0)), inflow_umax=w.get("inflow_umax", 0.0),
                 gravity=w.get("gravity", (0, 0)), lub_range=w.get("lub_range", 0.0),
                 rho_w_mode=w.get("rho_w_mode", 0), refill=w.get("refill", 1),
                 motion_cme=w.get("motion_cme", 0),
                 relative_changes=w.get("relative_changes", 0),
                 collision=w.get("collision", 0), boundary=w.get("boundary", 0))
    for s in w["solids"]:
        o.add_disk(s["cx"], s["cy"], s["r"], s["vx"], s["vy"], s["omega"], s["rho_s"], s["motion"])
    return o


def make_gpu(w, precision="fp64", ring=None, **kw):
    return G.Lattice.from_workload(w, precision=PREC.get(precision, precision),
                                   force_ring=ring or 256, **kw)


def rel(got, ref):
    """max |got - ref| / max |ref| (ref's scale taken over the whole series)."""
    scale = np.abs(ref).max()
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / (scale if scale > 0 else 1.0))


def force_rel(got, ref, radii, rho0=1.0):
    """Relative error of force records [steps][nsolid][2][3] per solid and
    component class.  The scale of a force is the larger of the series'
    largest magnitude and the one-sided pressure force on the disk's diameter,
    rho0 c_s^2 d = 2 rho0 r / 3 (the size of the link sums of Eq. 6 before
    they cancel); for the torque it is that force times r."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    worst = 0.0
    for s, r in enumerate(radii):
        f0 = 2.0 * rho0 * r / 3.0
        for comp, s0 in ((slice(0, 2), f0), (slice(2, 3), f0 * r)):
            a = ref[:, s, :, comp]
            scale = max(np.abs(a).max(), s0)
            worst = max(worst, float(np.abs(got[:, s, :, comp] - a).max() / scale))
    return worst


def force_rel_own(got, ref):
    """Worst error of each solid's force and torque relative to that solid's
    own series maximum (no floor): the error of the net force itself, which
    force_rel may scale by the larger link-sum size.  Returns a list over
    solids of (Fx/Fy error, torque error)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    out = []
    for s in range(ref.shape[1]):
        row = []
        for comp in (slice(0, 2), slice(2, 3)):
            a = ref[:, s, :, comp]
            scale = np.abs(a).max()
            row.append(float(np.abs(got[:, s, :, comp] - a).max() / scale) if scale > 0 else 0.0)
        out.append(tuple(row))
    return out


def describe(got, ref, radii):
    """Failure text: the force-scale error and each solid's own-scale error."""
    own = force_rel_own(got, ref)
    worst = max(max(r) for r in own) if own else 0.0
    return (f"force rel err {force_rel(got, ref, radii):.3e} (force scale); "
            f"worst solid relative to its own series {worst:.3e}")


def seeded_f(w, seed, amp=0.01):
    """Equilibrium at u0 times a seeded multiplicative perturbation."""
    import workloads as WL
    base = O.feq(w.get("rho0", 1.0), *w.get("u0", (0.0, 0.0)))
    f = np.broadcast_to(base[:, None, None], (9, w["ny"], w["nx"])).copy()
    f *= 1.0 + WL.perturbation(f.shape, seed, amp)
    return f


def run_pair(w, steps, precision="fp64", perturb=None, graph=0, variant=None):
    o = make_oracle(w)
    g = make_gpu(w, precision, ring=max(steps, 1))
    if graph:
        g.set_graph(graph)
    if variant is not None:
        g.set_kernel_variant(variant)
    if perturb is not None:
        f0 = seeded_f(w, perturb)
        o.set_f(f0)
        g.set_f(f0)
    ref = o.step(steps)
    got = g.step_record(steps)
    g.sync()
    return o, g, ref, got

"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests
and the benchmark.

This module only draws numbers and lays out problem descriptions (domain
sizes, boundary kinds, disk positions, radii and velocities, initial
perturbations).  It holds none of the lattice-Boltzmann arithmetic, so both
implementations can consume it without sharing any of the method.

Every description is a plain dict; ``solids`` is a list of dicts with keys
cx, cy, r, vx, vy, omega, rho_s, motion (0 prescribed, 1 free).

Base seed 13030625; each workload adds its own offset.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 13030625

PERIODIC, WALL, OPEN = 0, 1, 2
PRESCRIBED, FREE = 0, 1
RHOW_CONST, RHOW_LOCAL = 0, 1
FP64, FP32_DEV, FP16_DEV = 0, 1, 2


def _disk(cx, cy, r, vx=0.0, vy=0.0, omega=0.0, rho_s=1.0, motion=PRESCRIBED):
    return dict(cx=float(cx), cy=float(cy), r=float(r), vx=float(vx), vy=float(vy),
                omega=float(omega), rho_s=float(rho_s), motion=int(motion))


def galilean_pair(run: str, *, rho_w_mode=RHOW_LOCAL, moving_walls=True, U=0.05):
    """Channel 256 x 128, periodic in x, bounce-back walls in y, tau 0.8,
    rho0 1, one disk of radius 12 at (128, 64).

    run 'a': the disk moves at (U, 0) through fluid at rest, walls at rest.
    run 'b': the disk is fixed, the fluid starts at (-U, 0); the walls move at
    -U (the exact Galilean transform of 'a') unless moving_walls is False.
    """
    base = dict(nx=256, ny=128, tau=0.8, rho0=1.0, bc_x=PERIODIC, bc_y=WALL,
                rho_w_mode=rho_w_mode, refill=1, body_force=(0.0, 0.0))
    if run == "a":
        base.update(u0=(0.0, 0.0), wall_ux=(0.0, 0.0), solids=[_disk(128, 64, 12, U, 0.0)])
    elif run == "b":
        w = -U if moving_walls else 0.0
        base.update(u0=(-U, 0.0), wall_ux=(w, w), solids=[_disk(128, 64, 12)])
    else:
        raise ValueError(run)
    return base


def rejection_disks(nx, ny, n, rmin, rmax, vmax, seed, *, periodic=(True, True), gap=2.0,
                    margin=0.0, region=None, max_attempts=1_000_000):
    """n non-overlapping disks by seeded rejection sampling.

    Radii uniform in [rmin, rmax], centres uniform in the domain (or in
    region = (x0, x1, y0, y1)), velocity components uniform in [-vmax, vmax].
    Two disks are accepted when their centre distance (nearest periodic image
    along periodic axes) exceeds r_a + r_b + gap.  Along a non-periodic axis a
    centre keeps r + margin from the domain edge.
    """
    rng = np.random.default_rng(seed)
    xs = np.empty(n)
    ys = np.empty(n)
    rs = np.empty(n)
    k = 0
    attempts = 0
    x0, x1, y0, y1 = region if region is not None else (0.0, float(nx), 0.0, float(ny))
    while k < n:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError(f"placed only {k} of {n} disks")
        r = rng.uniform(rmin, rmax)
        lo_x = x0 if periodic[0] else max(x0, r + margin)
        hi_x = x1 if periodic[0] else min(x1, nx - 1 - r - margin)
        lo_y = y0 if periodic[1] else max(y0, r + margin)
        hi_y = y1 if periodic[1] else min(y1, ny - 1 - r - margin)
        cx = rng.uniform(lo_x, hi_x)
        cy = rng.uniform(lo_y, hi_y)
        if k:
            dx = xs[:k] - cx
            dy = ys[:k] - cy
            if periodic[0]:
                dx -= nx * np.round(dx / nx)
            if periodic[1]:
                dy -= ny * np.round(dy / ny)
            if np.any(dx * dx + dy * dy <= (rs[:k] + r + gap) ** 2):
                continue
        xs[k], ys[k], rs[k] = cx, cy, r
        k += 1
    v = rng.uniform(-vmax, vmax, size=(n, 2))
    return [_disk(xs[j], ys[j], rs[j], v[j, 0], v[j, 1]) for j in range(n)]


def precision_study(nx=8192, ny=4096, ndisk=2000, *, tau=None, seed_offset=2, rmin=8.0,
                    rmax=20.0, vmax=0.05):
    """Fully periodic nx x ny domain with ndisk non-overlapping disks, radii
    uniform in [rmin, rmax], constant prescribed velocities with components
    uniform in [-vmax, vmax], and one seeded draw of tau in [0.55, 1.0]
    (shared by every precision mode).  Defaults: the 8192 x 4096 domain with
    2000 disks."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    tau_draw = float(rng.uniform(0.55, 1.0))
    solids = rejection_disks(nx, ny, ndisk, rmin, rmax, vmax, BASE_SEED + seed_offset + 100)
    return dict(nx=nx, ny=ny, tau=tau_draw if tau is None else float(tau), rho0=1.0,
                bc_x=PERIODIC, bc_y=PERIODIC, u0=(0.0, 0.0), wall_ux=(0.0, 0.0),
                body_force=(0.0, 0.0), rho_w_mode=RHOW_CONST, refill=1, solids=solids)


def precision_study_common_velocity(nx=2048, ny=1024, ndisk=125, *, seed_offset=2, rmin=8.0,
                                    rmax=20.0, vmax=0.05):
    """The precision-study recipe with every disk given one velocity, drawn
    with components uniform in [-vmax, vmax]: the disks keep their distances,
    so none overlaps at any horizon (the independent velocities of
    precision_study make disks overlap and trap fluid between them within a
    few hundred steps).  Default: the disk density of the 8192 x 4096 /
    2000-disk domain on a 2048 x 1024 domain."""
    w = precision_study(nx, ny, ndisk, seed_offset=seed_offset, rmin=rmin, rmax=rmax, vmax=vmax)
    rng = np.random.default_rng(BASE_SEED + seed_offset + 200)
    vx, vy = (float(v) for v in rng.uniform(-vmax, vmax, size=2))
    for d in w["solids"]:
        d.update(vx=vx, vy=vy)
    return w


def perturbation(shape, seed, amplitude):
    """Seeded uniform noise in [-amplitude, amplitude] of the given shape."""
    rng = np.random.default_rng(BASE_SEED + 7919 * int(seed))
    return rng.uniform(-amplitude, amplitude, size=shape)


def sedimentation(nx=2048, ny=8192, ndisk=200, *, r=10.0, density_ratio=1.5, g=1e-5, tau=0.7,
                  seed_offset=4):
    """Box with walls on all sides; ndisk free disks of radius r and density
    density_ratio settle under gravity (0, -g); seeded non-overlapping
    positions in the top quarter of the box."""
    region = (0.0, float(nx), 0.75 * ny, float(ny))
    solids = rejection_disks(nx, ny, ndisk, r, r, 0.0, BASE_SEED + seed_offset,
                             periodic=(False, False), gap=4.0, margin=4.0, region=region)
    for s in solids:
        s.update(vx=0.0, vy=0.0, rho_s=float(density_ratio), motion=FREE)
    return dict(nx=nx, ny=ny, tau=tau, rho0=1.0, bc_x=WALL, bc_y=WALL, u0=(0.0, 0.0),
                wall_ux=(0.0, 0.0), body_force=(0.0, 0.0), gravity=(0.0, -g), lub_range=2.0,
                rho_w_mode=RHOW_CONST, refill=1, solids=solids)


def cylinder_sweep(ncase=512, *, seed_offset=3, nx_range=(128, 1024), ny_range=(64, 512),
                   re_range=(1.0, 100.0), tau=0.6, umax_cap=0.1):
    """Sweep of independent channels with one fixed cylinder each.

    Per case: nx uniform in nx_range, ny uniform among the even values of
    ny_range (the pair drawn again while the disk would come closer than 4
    nodes to the inlet, nx/4 - ny/10 < 4; ``shape_redraws`` counts those
    draws), a disk of radius ny/10 at (nx/4, ny/2 + U[-2, 2]), bounce-back
    walls in y, an equilibrium Poiseuille inlet at x = 0 and a copy outlet.
    Re = U_mean d / nu with d = 2 r and nu = (tau - 1/2) / 3 is drawn
    uniformly from re_range and drawn again while the inlet peak
    1.5 U_mean would exceed umax_cap (low Mach number); ``redraws`` counts the
    extra draws.  Returns a list of case descriptions.
    """
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    nu = (tau - 0.5) / 3.0
    out = []
    for _ in range(ncase):
        shape_redraws = -1
        while True:
            shape_redraws += 1
            nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
            ny = 2 * int(rng.integers(ny_range[0] // 2, ny_range[1] // 2 + 1))
            if nx / 4.0 - ny / 10.0 >= 4.0:
                break
        r = ny / 10.0
        cy = ny / 2.0 + float(rng.uniform(-2.0, 2.0))
        redraws = -1
        while True:
            redraws += 1
            re = float(rng.uniform(*re_range))
            umax = 1.5 * re * nu / (2.0 * r)
            if umax <= umax_cap:
                break
        out.append(dict(nx=nx, ny=ny, tau=float(tau), rho0=1.0, bc_x=OPEN, bc_y=WALL,
                        u0=(0.0, 0.0), wall_ux=(0.0, 0.0), body_force=(0.0, 0.0),
                        inflow_umax=umax, re=re, redraws=redraws,
                        shape_redraws=shape_redraws, rho_w_mode=RHOW_CONST,
                        refill=1, solids=[_disk(nx / 4.0, cy, r)]))
    return out


def warm_start_channels(ncase, *, seed_offset=5, nx=256, ny=128, umax=0.05, tau_min=0.53,
                        umax_cap=0.12, re_range=(1.0, 100.0), rmin=6.0, rmax=16.0):
    """Channels of the learned warm start: nx x ny, bounce-back walls in y,
    Poiseuille velocity inlet and pressure outlet, 1-4 fixed disks of radius
    uniform in [rmin, rmax] at seeded non-overlapping positions (gap >= 4),
    each at least its diameter from the walls and twice its diameter from
    the inlet and outlet.  Re uniform in re_range on the largest diameter d
    and the mean inlet speed U_mean = umax / 1.5; tau = 1/2 + 3 U_mean d / Re;
    below tau_min, tau = tau_min and U_mean = Re (tau - 1/2) / (3 d), the case
    drawn again when its peak 1.5 U_mean would exceed umax_cap.  Returns a
    list of case descriptions (with ``re`` and ``u_scale`` = peak speed)."""
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    out = []
    while len(out) < ncase:
        k = int(rng.integers(1, 5))
        disks = []
        for _ in range(200):
            if len(disks) == k:
                break
            r = float(rng.uniform(rmin, rmax))
            cx = float(rng.uniform(4 * r, nx - 4 * r))
            cy = float(rng.uniform(3 * r, ny - 3 * r))
            if all((cx - d["cx"]) ** 2 + (cy - d["cy"]) ** 2 > (r + d["r"] + 4) ** 2 for d in disks):
                disks.append(_disk(cx, cy, r))
        if not disks:
            continue
        re = float(rng.uniform(*re_range))
        d = 2.0 * max(x["r"] for x in disks)
        umean = umax / 1.5
        tau = 0.5 + 3.0 * umean * d / re
        if tau < tau_min:
            tau = tau_min
            umean = re * (tau - 0.5) / (3.0 * d)
            if 1.5 * umean > umax_cap:
                continue
        out.append(dict(nx=nx, ny=ny, tau=tau, rho0=1.0, bc_x=OPEN, bc_y=WALL, u0=(0.0, 0.0),
                        wall_ux=(0.0, 0.0), body_force=(0.0, 0.0), inflow_umax=1.5 * umean,
                        u_scale=1.5 * umean, re=re, rho_w_mode=RHOW_CONST, refill=1,
                        solids=disks))
    return out


def crop_disks(cfg, nx, ny):
    """Copy of a periodic workload restricted to the disks whose whole extent
    (plus a 2-node gap) lies inside [0, nx) x [0, ny)."""
    out = dict(cfg)
    out["nx"], out["ny"] = nx, ny
    out["solids"] = [dict(s) for s in cfg["solids"]
                     if s["cx"] - s["r"] > 2 and s["cx"] + s["r"] < nx - 3
                     and s["cy"] - s["r"] > 2 and s["cy"] + s["r"] < ny - 3]
    return out


def cells(cfg) -> int:
    return int(cfg["nx"]) * int(cfg["ny"])


def describe(cfg) -> str:
    return (f"{cfg['nx']}x{cfg['ny']} tau={cfg['tau']:.4f} solids={len(cfg['solids'])} "
            f"bc=({cfg['bc_x']},{cfg['bc_y']})")


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("math", "np", "annotations")]

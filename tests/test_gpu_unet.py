"""The warm-start network on the GPU (BF16 tensor-core convolutions, FP32
accumulation) against the FP64 oracle network with the same parameters:
forward outputs and every parameter's gradient, on a small network and on
the full 4-level, 32-256-channel network at 128 x 256.

The oracle evaluates the same function (the BF16 weights the GPU multiplies
with, the BF16-rounded input); what remains is the BF16 rounding of
activations and activation gradients between layers (FP32 accumulation).
Tolerance: relative L2 error <= 2e-2."""
import numpy as np
import pytest

import oracle.unet as U
import paper_1303_0625_gb300 as G
from paper_1303_0625_gb300 import lbm as L

pytestmark = pytest.mark.gpu


def _flat(p, levels, base):
    out = []
    for name, co, ci, k in U.layer_shapes(levels, base):
        out += [p[name + ".w"].ravel(), p[name + ".b"].ravel()]
    return np.concatenate(out)


def _unflat(v, levels, base):
    p, o = {}, 0
    for name, co, ci, k in U.layer_shapes(levels, base):
        n = co * ci * k * k
        p[name + ".w"] = v[o:o + n].reshape(co, ci, k, k).astype(np.float64)
        o += n
        p[name + ".b"] = v[o:o + co].astype(np.float64)
        o += co
    return p


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), as the GPU stores
    weights and the network input."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _case(levels, base, H, W, B, seed):
    rng = np.random.default_rng(seed)
    p = U.init_params(levels, base, seed=seed)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0.0, 0.1, p[k].shape)
    x = np.zeros((B, U.IN_CH, H, W))
    yy, xx = np.mgrid[0:H, 0:W]
    for n in range(B):
        for _ in range(2):
            cy, cx, r = rng.uniform(0.3 * H, 0.7 * H), rng.uniform(0.2 * W, 0.8 * W), rng.uniform(1.5, max(H / 5, 2.5))
            x[n, 0] = np.maximum(x[n, 0], ((yy - cy) ** 2 + (xx - cx) ** 2 <= r * r))
        x[n, 1] = rng.uniform(0.01, 1.0)
    t = rng.normal(0.0, 0.5, (B, 3, H, W))
    fl = 1.0 - x[:, 0]
    net = G.UNet(H, W, levels=levels, base=base, max_batch=B)
    net.set_params(_flat(p, levels, base).astype(np.float32))
    # the oracle evaluates the function the GPU evaluates: BF16 weights (the
    # GPU keeps FP32 masters but multiplies with their BF16 copies), FP32
    # biases, the input rounded to BF16
    p = _unflat(net.params(), levels, base)
    for k in p:
        if k.endswith(".w") and not k.startswith("head"):
            p[k] = _bf16(p[k])
    x = _bf16(x)
    return net, p, x, t, fl


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-30))


def test_params_round_trip_in_oracle_layout():
    net = G.UNet(8, 16, levels=2, base=8, max_batch=1)
    v = _flat(U.init_params(2, 8, seed=5), 2, 8).astype(np.float32)
    net.set_params(v)
    assert net.nparam == v.size and np.array_equal(net.params(), v)


@pytest.mark.parametrize("levels,base,H,W,B,gtol", [(2, 8, 16, 32, 2, 2e-2), (3, 16, 32, 64, 2, 2e-2),
                                                     (4, 32, 32, 64, 2, 3e-2)])
def test_forward_and_gradients_small(levels, base, H, W, B, gtol):
    """Gradients of the deepest layers pass through the most BF16 roundings
    (each <= 2^-9 relative): the 4-level chain has 14 of them between the
    loss and enc3a, a worst-case accumulation of 2.8%, hence 3e-2 there."""
    net, p, x, t, fl = _case(levels, base, H, W, B, levels)
    y_ref, cache = U.forward(p, x, levels, keep=True)
    y = net.forward(x)
    assert _rel(y, y_ref) <= 2e-2
    # element by element: no output off by more than 5% of the largest one
    assert np.abs(y - y_ref).max() <= 5e-2 * np.abs(y_ref).max()
    loss_ref, dy = U.loss(y_ref, t, fl)
    g_ref = U.backward(p, cache, dy, levels)
    loss, g = net.gradients(x, t, fl)
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    gv = _unflat(g, levels, base)
    for k in g_ref:
        assert _rel(gv[k], g_ref[k]) <= gtol, (k, _rel(gv[k], g_ref[k]))


def test_full_network_forward_128x256():
    net, p, x, t, fl = _case(4, 32, 128, 256, 1, 7)
    y = net.forward(x)
    y_ref = U.forward(p, x, 4)
    assert _rel(y, y_ref) <= 2e-2
    assert np.abs(y - y_ref).max() <= 5e-2 * np.abs(y_ref).max()


def test_training_lowers_the_loss():
    net, p, x, t, fl = _case(3, 16, 32, 64, 4, 11)
    t = np.tanh(x[:, :3]) + 0.1  # a learnable target
    first = net.train_step(x, t, fl, 1e-3)
    for _ in range(60):
        last = net.train_step(x, t, fl, 1e-3)
    assert last < 0.5 * first


def test_warm_start_sets_the_predicted_equilibrium():
    import torch
    H, W = 32, 64
    lat = G.Lattice(W, H, 0.7, bc_x=G.LBM_OPEN, bc_y=G.LBM_WALL, inflow_umax=0.05,
                    precision=G.LBM_FP32_DEV)
    lat.add_disk(20.3, 15.8, 5.2)
    rng = np.random.default_rng(3)
    pred = rng.normal(0.0, 0.3, (3, H, W)).astype(np.float32)
    U_ = 0.05
    dev = torch.from_numpy(pred).cuda()
    R = 3e-3
    L.lbm_warm_start(lat.handle, dev, U_, R)
    rho, ux, uy = lat.fields()
    fl = lat.owner() < 0
    assert np.allclose(rho[fl], 1.0 + R * pred[0][fl], atol=2e-6)
    assert np.allclose(ux[fl], U_ * pred[1][fl], atol=2e-6)
    assert np.allclose(uy[fl], U_ * pred[2][fl], atol=2e-6)
    # relative to the channel's Poiseuille flow
    from paper_1303_0625_gb300 import warmstart as WS
    case = dict(nx=W, ny=H, tau=0.7, inflow_umax=0.05, rho0=1.0)
    rp, up = WS.poiseuille(case)
    L.lbm_warm_start(lat.handle, dev, U_, R, base=True)
    rho, ux, uy = lat.fields()
    assert np.allclose(rho[fl], (rp + R * pred[0])[fl], atol=2e-6)
    assert np.allclose(ux[fl], (up[:, None] + U_ * pred[1])[fl], atol=2e-6)
    with pytest.raises(G.LBMError):  # the flux correction works on the base
        L.lbm_warm_start(lat.handle, dev, U_, R, flux=True)


def test_warm_start_column_flux_equals_the_inlet_flux():
    """With the column flux correction every column of the initial state
    carries the inlet's mass flux sum_y rho u_P over column 0, u_x of each
    column scaled by one factor (FP64 storage: to rounding); rho and u_y as
    without it."""
    import torch
    H, W = 32, 64
    lat = G.Lattice(W, H, 0.7, bc_x=G.LBM_OPEN, bc_y=G.LBM_WALL, inflow_umax=0.05,
                    precision=G.LBM_FP64)
    lat.add_disk(30.3, 15.8, 6.2)
    lat.add_disk(48.0, 9.5, 3.5)
    rng = np.random.default_rng(5)
    pred = rng.normal(0.0, 0.3, (3, H, W)).astype(np.float32)
    U_, R = 0.05, 3e-3
    L.lbm_warm_start(lat.handle, torch.from_numpy(pred).cuda(), U_, R, base=True, flux=True)
    rho, ux, uy = lat.fields()
    fl = lat.owner() < 0
    from paper_1303_0625_gb300 import warmstart as WS
    rp, up = WS.poiseuille(dict(nx=W, ny=H, tau=0.7, inflow_umax=0.05, rho0=1.0))
    rho_p = rp + R * pred[0].astype(np.float64)
    ux_p = up[:, None] + U_ * pred[1].astype(np.float64)
    q_in = (np.where(fl[:, 0], rho_p[:, 0] * up, 0.0)).sum()
    q = np.where(fl, rho * ux, 0.0).sum(axis=0)
    assert np.abs(q / q_in - 1.0).max() <= 1e-12
    scale = q_in / np.where(fl, rho_p * ux_p, 0.0).sum(axis=0)
    assert np.allclose(ux[fl], (ux_p * scale[None, :])[fl], rtol=0, atol=1e-13)
    assert np.allclose(rho[fl], rho_p[fl], rtol=0, atol=1e-13)
    assert np.allclose(uy[fl], (U_ * pred[2].astype(np.float64))[fl], rtol=0, atol=1e-13)


def test_wait_time_out_is_reported_and_the_network_recovers():
    """A wait limit of 0 makes the mbarrier waits of every tensor-core
    convolution give up at once: each CTA stops issuing MMAs, waits for the
    ones it issued, frees its tensor memory and stores nothing; the host gets
    LBM_ETIMEOUT, and with the limit restored the network computes as
    before (the forward pass bit for bit; the weight gradients, summed with
    FP32 atomics across pixel splits, to rounding)."""
    net, p, x, t, fl = _case(3, 16, 32, 64, 2, seed=11)
    ref = net.forward(x)
    loss_ref, g_ref = net.gradients(x, t, fl)
    net.set_wait_limit(0)
    with pytest.raises(G.LBMError) as e:
        net.forward(x)
    assert e.value.status == G.LBM_ETIMEOUT
    with pytest.raises(G.LBMError) as e:
        net.gradients(x, t, fl)
    assert e.value.status == G.LBM_ETIMEOUT
    with pytest.raises(G.LBMError) as e:
        net.set_wait_limit(-1)
    assert e.value.status == G.LBM_EINVAL
    net.set_wait_limit(1 << 24)
    assert np.array_equal(net.forward(x), ref)
    loss, g = net.gradients(x, t, fl)
    assert abs(loss - loss_ref) <= 1e-6 * abs(loss_ref)
    assert _rel(g, g_ref) <= 1e-5
    net.close()

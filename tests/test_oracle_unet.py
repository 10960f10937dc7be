"""Pins of the FP64 warm-start network oracle (oracle/unet.py): every layer
against an independent statement (a library correlation, closed forms,
adjointness), and the whole backward pass against central finite
differences, so that a dropped term, a flipped kernel or a lost skip
gradient fails."""
import numpy as np
import pytest

import oracle.unet as U


def test_conv_matches_library_correlation():
    # only this pin needs scipy; the others run without it
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy_signal.correlate2d(x[n, c], w[o, c], mode="same")
                             for c in range(3))
            assert np.allclose(y[n, o], ref, rtol=0, atol=1e-12)


def test_conv_identity_and_shift_kernels():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 2, 5, 6))
    w = np.zeros((2, 2, 3, 3))
    w[0, 0, 1, 1] = 1.0   # identity on channel 0
    w[1, 1, 1, 2] = 1.0   # y[i, j] = x[i, j + 1], zero beyond the edge
    y = U.conv(x, w, np.zeros(2))
    assert np.array_equal(y[0, 0], x[0, 0])
    assert np.array_equal(y[0, 1, :, :-1], x[0, 1, :, 1:]) and not y[0, 1, :, -1].any()


def test_pool_and_upsample_are_adjoint():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 3, 4, 5))
    y = rng.normal(size=(2, 3, 8, 10))
    assert np.isclose((U.up(x) * y).sum(), 4.0 * (x * U.pool(y)).sum(), rtol=1e-13)
    assert np.allclose(U.pool(U.up(x)), x)
    assert np.allclose(U.pool_backward(U.pool(y) * 0 + 1).sum(), y.size / 4)
    assert np.allclose(U.up_backward(U.up(x)), 4 * x)


def test_adam_first_step_is_a_signed_step():
    """With zero moments, bias correction makes the first step lr * g / (|g| + eps)."""
    p = {"a": np.array([1.0, -2.0, 0.5])}
    g = {"a": np.array([0.3, -1e-3, 2.0])}
    st = {}
    U.adam(p, g, st, lr=0.01)
    assert np.allclose(p["a"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=0, atol=1e-7)


def test_loss_ignores_solid_nodes():
    rng = np.random.default_rng(3)
    y = rng.normal(size=(1, 3, 4, 4))
    t = rng.normal(size=(1, 3, 4, 4))
    fl = np.ones((1, 4, 4))
    fl[0, 1, 2] = 0
    l0, g0 = U.loss(y, t, fl)
    y2 = y.copy()
    y2[0, :, 1, 2] += 100.0
    l1, _ = U.loss(y2, t, fl)
    assert l0 == l1 and not g0[0, :, 1, 2].any()
    assert np.isclose(l0, ((y - t) ** 2 * fl[:, None]).sum() / (15 * 3))


@pytest.mark.parametrize("levels,base,shape", [(2, 4, (8, 16)), (3, 2, (16, 8))])
def test_backward_matches_finite_differences(levels, base, shape):
    rng = np.random.default_rng(4 + levels)
    p = U.init_params(levels, base, seed=levels)
    for k in p:
        p[k] = p[k] + rng.normal(0.0, 0.05, p[k].shape)
    x = rng.normal(size=(2, U.IN_CH) + shape)
    t = rng.normal(size=(2, 3) + shape)
    fl = (rng.random((2,) + shape) > 0.2).astype(float)
    y, cache = U.forward(p, x, levels, keep=True)
    _, dy = U.loss(y, t, fl)
    g = U.backward(p, cache, dy, levels)
    assert set(g) == set(p)
    h = 1e-6
    for k in p:
        for _ in range(3):
            idx = tuple(int(rng.integers(0, n)) for n in p[k].shape)
            p[k][idx] += h
            lp, _ = U.loss(U.forward(p, x, levels), t, fl)
            p[k][idx] -= 2 * h
            lm, _ = U.loss(U.forward(p, x, levels), t, fl)
            p[k][idx] += h
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(abs(fd), 1e-3), (k, idx, fd, g[k][idx])

"""Host logic of the warm start that needs no GPU: the steady band test
(the same rule as the batch engine's convergence window) and the
Poiseuille base of the network's residual targets."""
import numpy as np

from paper_1303_0625_gb300 import warmstart as WS


def _run(series, tol, window):
    """Index of the test at which the band test first holds `window` calm
    tests in a row, or -1."""
    anchor = np.full(1, np.nan)
    calm = np.zeros(1, dtype=np.int64)
    for k, d in enumerate(series):
        anchor, calm = WS.band_step(anchor, calm, np.array([d]), tol)
        if calm[0] >= window:
            return k
    return -1


def test_band_rejects_an_oscillation_that_a_single_test_passes():
    t = np.arange(400)
    osc = 1.0 + 1e-3 * np.cos(2 * np.pi * t / 40.0)  # turning points every 20 tests
    # one test: the change between two tests near a turning point is below 1e-4
    assert _run(osc, 1e-4, 1) >= 0
    # a band held for 50 tests never holds
    assert _run(osc, 1e-5, 50) == -1


def test_band_accepts_noise_below_it_and_a_settled_decay():
    rng = np.random.default_rng(1)
    noisy = 0.2 * (1.0 + 2e-6 * rng.standard_normal(300))  # round-off noise of a few 1e-6
    assert _run(noisy, 1e-5, 50) == 50  # the 50 tests after the anchor (test 0)
    assert _run(noisy, 1e-8, 10) == -1  # a band below the noise never holds
    decay = 1.0 + 0.5 * np.exp(-np.arange(2000) / 30.0)
    k = _run(decay, 1e-5, 50)
    assert k > 0 and abs(decay[k] - 1.0) < 1e-5 * 30 / 1  # within tol x (decay time / test)


def test_band_restarts_its_run_when_the_drag_leaves_it():
    series = [1.0] * 10 + [1.1] + [1.1] * 10
    assert _run(series, 1e-5, 9) == 9
    assert _run(series, 1e-5, 10) == 20  # the jump at test 10 starts a new run at 1.1


def test_poiseuille_base():
    case = dict(nx=64, ny=32, tau=0.8, inflow_umax=0.05, rho0=1.0)
    rho, u = WS.poiseuille(case)
    y = np.arange(32) + 0.5
    assert np.allclose(u, 4 * 0.05 * y * (32 - y) / 32 ** 2)
    assert rho.shape == (32, 64) and np.all(rho[:, -1] == 1.0)
    nu = (0.8 - 0.5) / 3.0
    # the pressure drop of the parabola: d(rho)/dx = -3 * 8 nu umax / ny^2
    assert np.allclose(np.diff(rho[0]), -24.0 * nu * 0.05 / 32 ** 2)

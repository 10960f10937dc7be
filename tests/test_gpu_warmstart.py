"""Learned warm start on small, fast-converging channels: a warm-started
run reaches the plain (cold) run's converged drag within 1e-4 (steady
states do not depend on the initial state), and a network whose prediction
is unusable is caught by the drift check and the case restarts cold."""
import numpy as np
import pytest

import paper_1303_0625_gb300 as G
from paper_1303_0625_gb300 import warmstart as WS
import workloads as W

pytestmark = pytest.mark.gpu


def _cases(n=6):
    return W.warm_start_channels(n, seed_offset=91, nx=64, ny=32, rmin=3.0, rmax=5.0,
                                 re_range=(1.0, 4.0))


def test_warm_start_reaches_the_cold_drag():
    cases = _cases()
    ref = WS.steady(cases, tol=1e-9, cap=200_000)
    assert (ref["state"] == G.LBM_CASE_CONVERGED).all()
    data = WS.dataset(cases, ref)
    net = G.UNet(32, 64, levels=2, base=8, max_batch=8, seed=1)
    WS.train(net, data, epochs=150, batch=2, lr=2e-3, lr_end=1e-4)
    # a network trained on six samples predicts the pressure level to a few
    # percent: the drift bound here only has to reject unusable states
    warm = WS.time_to_drag(cases, ref["drag"], net=net, cap=100_000, drift_mass=5e-2)
    cold = WS.time_to_drag(cases, ref["drag"], cap=100_000)
    assert (warm["steps"] >= 0).all() and (cold["steps"] >= 0).all()
    assert not warm["fallback"].any(), warm["drift"]


def test_unusable_prediction_falls_back_to_cold():
    cases = _cases(3)
    ref = WS.steady(cases, tol=1e-9, cap=200_000, fields=False)
    net = G.UNet(32, 64, levels=2, base=8, max_batch=4, seed=2)
    p = net.params()
    p[-3:] = 1e3  # head biases: density 1 + 1e3 * scale, far beyond the drift bound
    net.set_params(p)
    warm = WS.time_to_drag(cases, ref["drag"], net=net, cap=100_000)
    assert warm["fallback"].all() and (warm["steps"] >= 0).all()

"""Pins of the pooled on-line delta adaptation (Robbins-Monro on log delta).

- With one chain it is the offline calibration rule of calibrate_delta.calibrate.
- On a small linear-Gaussian model the second-half acceptance settles at the target
  from step sizes far too small and far too large (a sign error diverges instead).
"""
import numpy as np

from oracle import calibrate_delta, mcmc
from paper_2303_00301_gb300 import workloads


def _model(wl):
    em = mcmc.LinearGaussianEmission(wl.y, wl.Ry, wl.mask) if wl.emission == workloads.EMIS_LINEAR_GAUSSIAN \
        else mcmc.SVEmission(wl.y, wl.mask)
    return dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)


def test_one_chain_reduces_to_the_offline_rule():
    wl = workloads.stochastic_volatility(d=3, T=20, n_chains=1, delta=0.05)
    model = _model(wl)
    n = 25
    _, deltas, _ = calibrate_delta.run_chains_adaptive(wl.x_init[:1], model, 0.05, n, target=0.5)
    # calibrate() returns the mean of the second half of its delta history
    mean_half, _ = calibrate_delta.calibrate(model, wl.x_init[0], 0.05, n, target=0.5)
    assert abs(np.mean(deltas[1:][n // 2:]) - mean_half) < 1e-12


def test_acceptance_settles_at_the_target():
    wl = workloads.linear_gaussian(d=2, T=16, n_chains=4)
    model = _model(wl)
    for delta0 in (1e-3, 20.0):
        _, deltas, las = calibrate_delta.run_chains_adaptive(wl.x_init, model, delta0, 400, target=0.4, c=2.0)
        acc = np.exp(np.minimum(0.0, las[200:])).mean()
        assert abs(acc - 0.4) < 0.08, (delta0, acc, deltas[-1])

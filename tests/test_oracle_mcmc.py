"""Pins of the oracle's auxiliary Kalman MH step (no GPU)."""
import numpy as np
import pytest

from oracle import dense, kalman, mcmc, philox
from paper_2303_00301_gb300 import workloads


class LinearPotential:
    """gamma(x) = sum_t c_t . x_t: first-order linearisation is exact."""

    def __init__(self, c):
        self.c = c

    def log_h(self, x):
        return np.sum(self.c * x, axis=1)

    def grad(self, x):
        return self.c.copy()


def _model_from(wl):
    if wl.emission == workloads.EMIS_SV:
        em = mcmc.SVEmission(wl.y, wl.mask)
    else:
        em = mcmc.LinearGaussianEmission(wl.y, wl.Ry, wl.mask)
    return dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)


def test_linear_potential_gives_log_alpha_zero():
    d, T = 3, 10
    m = workloads.random_lgssm(d, T, seed=21)
    c = np.random.default_rng(2).standard_normal((T, d))
    model = dict(m0=m["m0"], P0=m["P0"], F=m["F"], b=m["b"], Q=m["Q"], emission=LinearPotential(c))
    x = np.random.default_rng(3).standard_normal((T, d))
    for it in range(3):
        st = mcmc.aux_step_philox(x, model, 0.4, seed=9, chain=0, iteration=it)
        assert abs(st["log_alpha"]) < 1e-9
        x = st["x_new"]


def _simplified_log_alpha(st, x, model, delta):
    """Section 2.2 algebra: prior terms cancel, N(u;z,R)/N(u+Rv;z,R) = exp(v.(u-z) + v.Rv/2)."""
    em = model["emission"]
    u, v, vs, xs = st["u"], st["v"], st["v_star"], st["x_star"]
    r = 0.5 * delta
    fwd = np.sum(v * (u - xs)) + 0.5 * r * np.sum(v * v)
    rev = np.sum(vs * (u - x)) + 0.5 * r * np.sum(vs * vs)
    return (em.log_h(xs).sum() - em.log_h(x).sum() + fwd - rev
            + st["logZ"] - st["logZ_star"])


@pytest.mark.parametrize("kind", ["lg", "sv"])
def test_simplified_ratio_equals_direct_formula(kind):
    if kind == "lg":
        wl = workloads.linear_gaussian(d=2, T=12)
    else:
        wl = workloads.stochastic_volatility(d=4, T=12, n_chains=1, delta=0.05)
    model = _model_from(wl)
    x = wl.x_init[0]
    for it in range(4):
        st = mcmc.aux_step_philox(x, model, wl.delta, wl.mcmc_seed, 0, it)
        assert st["log_alpha"] == pytest.approx(_simplified_log_alpha(st, x, model, wl.delta),
                                                abs=1e-9)
        x = st["x_new"]


def test_reject_keeps_state_accept_moves():
    wl = workloads.linear_gaussian(d=2, T=8)
    model = _model_from(wl)
    x = wl.x_init[0]
    eps = np.zeros_like(x)
    st_acc = mcmc.aux_step(x, model, wl.delta, eps, eps, log_u=-np.inf)
    st_rej = mcmc.aux_step(x, model, wl.delta, eps, eps, log_u=np.inf)
    assert st_acc["accepted"] and np.array_equal(st_acc["x_new"], st_acc["x_star"])
    assert not st_rej["accepted"] and np.array_equal(st_rej["x_new"], x)


def test_two_step_toy_posterior_closed_form():
    """Section 4.4 model: E[x0|y] = rho y / (1 + r^2), Var = 1 - rho^2 / (1 + r^2)."""
    rho, r2, y = 0.6, 0.3, 5.0
    wl = workloads.two_step_toy(rho=rho, r2=r2, y_obs=y)
    mbar, C = dense.prior_moments(wl.m0, wl.P0, wl.F, wl.b, wl.Q, 2)
    # condition the stacked prior on y = x_1 + N(0, r2)
    h = np.array([0.0, 1.0])
    s = h @ C @ h + r2
    k = C @ h / s
    mean = mbar + k * (y - h @ mbar)
    cov = C - np.outer(k, h @ C)
    assert mean[0] == pytest.approx(rho * y / (1 + r2), rel=1e-13)
    assert cov[0, 0] == pytest.approx(1 - rho ** 2 / (1 + r2), rel=1e-13)
    assert mean[0] == pytest.approx(wl.meta["post_mean_x0"], rel=1e-13)


def _batch_se(samples, n_batches=20):
    n = len(samples) // n_batches * n_batches
    bm = samples[:n].reshape(n_batches, -1, *samples.shape[1:]).mean(axis=1)
    return bm.std(axis=0, ddof=1) / np.sqrt(n_batches)


@pytest.mark.slow
def test_two_step_toy_chain_mean():
    wl = workloads.two_step_toy(rho=0.8, r2=0.5, y_obs=2.0, delta=1.0)
    model = _model_from(wl)
    keep = []
    x, n_acc, kept = mcmc.run_chain(wl.x_init[0], model, wl.delta, seed=5, chain=0,
                                    n_iters=6000, keep=lambda z: z[0, 0])
    s = np.array(kept[500:])
    se = _batch_se(s)
    assert 0.2 < n_acc / 6000 < 0.99
    assert abs(s.mean() - wl.meta["post_mean_x0"]) < 4 * se
    assert abs(s.var() / wl.meta["post_var_x0"] - 1) < 0.25


@pytest.mark.slow
@pytest.mark.parametrize("sampler", ["rts", "bridging"])
def test_linear_gaussian_stationarity(sampler):
    """Chain moments match the exact smoother of the linear-Gaussian model within MC error
    (with either pathwise sampler: RTS, or the divide-and-conquer sampler of Appendix A.2.3)."""
    wl = workloads.linear_gaussian(d=2, T=16)
    model = _model_from(wl)
    kf = kalman.kalman_filter(wl.y, wl.m0, wl.P0, wl.F, wl.b, wl.Q, wl.Ry)
    ms, Ps = kalman.rts_smoother(kf, wl.F)
    x, n_acc, kept = mcmc.run_chain(wl.x_init[0], model, wl.delta, seed=wl.mcmc_seed, chain=0,
                                    n_iters=3000, keep=lambda z: z.copy(), sampler=sampler)
    s = np.stack(kept[300:])
    se = _batch_se(s)
    z = (s.mean(axis=0) - ms) / se
    # Bonferroni over T*d = 32 coordinates at ~4.3 sigma
    assert np.max(np.abs(z)) < 4.3, np.max(np.abs(z))
    assert n_acc / 3000 > 0.3

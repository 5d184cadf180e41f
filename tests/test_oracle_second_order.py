"""Pins of the oracle's second-order auxiliary proposal (Section 2.2, Eqs. (2.8)-(2.9)).

- Gaussian target: the second-order expansion of gamma is exact, so the proposal
  is the exact conditional pi(x | u) and log alpha = 0 from any state.
- Completing the square: the expansion of Eq. (2.8) times N(u_t; z_t, (delta/2) I)
  equals N(omega_t; z_t, Omega_t) up to a constant in z_t.
- With a zero Hessian the step reduces to the first-order step.
- On a 1-D, two-step stochastic-volatility model the chain's stationary mean
  and second moment match the posterior computed by grid quadrature.
"""
import numpy as np
import pytest

from oracle import kalman, mcmc, philox
from paper_2303_00301_gb300 import workloads


def _lg_model(d, T, seed):
    m = workloads.random_lgssm(d, T, seed=seed)
    rng = np.random.default_rng(seed + 1)
    A = rng.standard_normal((d, d))
    Ry = A @ A.T / d + 0.3 * np.eye(d)
    em = mcmc.LinearGaussianEmission(m["y"], Ry)
    return dict(m0=m["m0"], P0=m["P0"], F=m["F"], b=m["b"], Q=m["Q"], emission=em)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gaussian_target_gives_log_alpha_zero(seed):
    d, T, delta = 3, 12, 0.7
    model = _lg_model(d, T, 10 + seed)
    rng = np.random.default_rng(seed)
    x = 2.0 * rng.standard_normal((T, d))          # far from the posterior on purpose
    for it in range(3):
        eps_a = rng.standard_normal((T, d))
        eps_b = rng.standard_normal((T, d))
        st = mcmc.aux_step_second_order(x, model, delta, eps_a, eps_b, np.log(0.5))
        assert abs(st["log_alpha"]) < 1e-8, st["log_alpha"]
        x = st["x_star"]


def test_first_order_proposal_does_not_have_this_property():
    """Control for the pin above: the first-order step on the same target rejects sometimes."""
    d, T, delta = 3, 12, 0.7
    model = _lg_model(d, T, 10)
    rng = np.random.default_rng(0)
    x = 2.0 * rng.standard_normal((T, d))
    st = mcmc.aux_step(x, model, delta, rng.standard_normal((T, d)), rng.standard_normal((T, d)),
                       np.log(0.5))
    assert abs(st["log_alpha"]) > 1e-3


def test_pseudo_observations_complete_the_square():
    d, T, delta = 3, 4, 0.3
    rng = np.random.default_rng(5)
    y = rng.standard_normal((T, d))
    em = mcmc.SVEmission(y)
    model = dict(emission=em)
    x = 0.5 * rng.standard_normal((T, d))
    u = x + np.sqrt(0.5 * delta) * rng.standard_normal((T, d))
    om, Om = mcmc.second_order_obs(x, u, model, delta)
    v, Lam = em.grad(x), em.hess(x)
    R = 0.5 * delta * np.eye(d)
    for t in range(T):
        vals = []
        for _ in range(6):
            z = x[t] + rng.standard_normal(d)
            expansion = v[t] @ (z - x[t]) + 0.5 * (z - x[t]) @ Lam[t] @ (z - x[t])
            vals.append(expansion + kalman.mvn_logpdf(u[t], z, R) - kalman.mvn_logpdf(om[t], z, Om[t]))
        assert np.ptp(vals) < 1e-9, vals


def test_hessians_match_finite_differences():
    d, T = 3, 5
    rng = np.random.default_rng(8)
    y = rng.standard_normal((T, d))
    x = 0.3 * rng.standard_normal((T, d))
    A = rng.standard_normal((d, d))
    for em in (mcmc.SVEmission(y), mcmc.LinearGaussianEmission(y, A @ A.T + np.eye(d))):
        H = em.hess(x)
        h = 1e-5
        for i in range(d):
            e = np.zeros((T, d)); e[:, i] = h
            fd = (em.grad(x + e) - em.grad(x - e)) / (2 * h)      # column i of each Hessian
            assert np.max(np.abs(fd - H[:, :, i])) < 1e-7


class _ZeroHessian:
    def __init__(self, em):
        self.em = em

    def log_h(self, x):
        return self.em.log_h(x)

    def grad(self, x):
        return self.em.grad(x)

    def hess(self, x):
        return np.zeros((x.shape[0], x.shape[1], x.shape[1]))


def test_zero_hessian_reduces_to_first_order():
    wl = workloads.stochastic_volatility(d=4, T=20, n_chains=1, delta=0.05)
    model = dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=_ZeroHessian(mcmc.SVEmission(wl.y)))
    x = wl.x_init[0]
    rng = np.random.default_rng(2)
    ea, eb = rng.standard_normal(x.shape), rng.standard_normal(x.shape)
    a = mcmc.aux_step(x, model, wl.delta, ea, eb, np.log(0.3))
    b = mcmc.aux_step_second_order(x, model, wl.delta, ea, eb, np.log(0.3))
    assert np.allclose(a["x_star"], b["x_star"], rtol=1e-12, atol=1e-12)
    assert abs(a["log_alpha"] - b["log_alpha"]) < 1e-9


def test_two_step_sv_chain_matches_grid_posterior():
    """d = 1, T = 2: x0 ~ N(0, 1), x1 = 0.8 x0 + N(0, 0.5), y_t ~ N(0, exp(x_t))."""
    m0, P0 = np.zeros(1), np.eye(1)
    F, b, Q = 0.8 * np.eye(1), np.zeros(1), 0.5 * np.eye(1)
    y = np.array([[1.7], [0.2]])
    em = mcmc.SVEmission(y)
    model = dict(m0=m0, P0=P0, F=F, b=b, Q=Q, emission=em)
    # posterior moments by quadrature on a grid
    g = np.linspace(-7.0, 7.0, 1401)
    X0, X1 = np.meshgrid(g, g, indexing="ij")
    logp = (-0.5 * X0 ** 2 - 0.5 * (X1 - 0.8 * X0) ** 2 / 0.5
            - 0.5 * X0 - 0.5 * y[0, 0] ** 2 * np.exp(-X0)
            - 0.5 * X1 - 0.5 * y[1, 0] ** 2 * np.exp(-X1))
    w = np.exp(logp - logp.max())
    w /= w.sum()
    mean = np.array([(w * X0).sum(), (w * X1).sum()])
    second = np.array([(w * X0 ** 2).sum(), (w * X1 ** 2).sum()])
    # the chain
    delta, n, burn = 0.8, 6000, 200
    x = np.zeros((2, 1))
    acc, s1, s2 = 0, np.zeros(2), np.zeros(2)
    for k in range(n + burn):
        st = mcmc.aux_step_philox(x, model, delta, seed=11, chain=0, iteration=k, order=2)
        x = st["x_new"]
        if k >= burn:
            acc += st["accepted"]
            s1 += x[:, 0]
            s2 += x[:, 0] ** 2
    assert acc / n > 0.5
    assert np.all(np.abs(s1 / n - mean) < 0.08), (s1 / n, mean)
    assert np.all(np.abs(s2 / n - second) < 0.15), (s2 / n, second)

"""Pins of the oracle's log-likelihood gradient (Fisher identity) by finite differences."""
import numpy as np
import pytest

from oracle import gradient


def _theta(d, seed):
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal(d) * 0.3
    phi = rng.uniform(0.8, 0.99, d)
    Sigma = 0.5 * np.ones((d, d)) + 0.5 * np.eye(d)
    L = np.linalg.cholesky(Sigma) * rng.uniform(0.8, 1.2)
    return mu, phi, L, 0.3


@pytest.mark.parametrize("d,T", [(1, 5), (2, 12), (3, 20)])
def test_fisher_gradient_matches_finite_differences(d, T):
    theta = _theta(d, seed=d * 10 + T)
    yt = np.random.default_rng(T).standard_normal((T, d))
    g_mu, g_phi, g_L, g_delta, logZ = gradient.loglik_grad(theta, yt)
    f_mu, f_phi, f_L, f_delta = gradient.loglik_fd_grad(theta, yt, h=1e-5)
    assert logZ == pytest.approx(gradient.loglik(theta, yt), rel=1e-12)
    for g, f in [(g_mu, f_mu), (g_phi, f_phi), (g_L, f_L), (np.array(g_delta), np.array(f_delta))]:
        scale = max(1.0, np.abs(f).max())
        assert np.abs(g - f).max() < 2e-6 * scale, (g, f)


def test_gradient_is_zero_in_the_upper_triangle_of_L():
    theta = _theta(3, 1)
    yt = np.random.default_rng(0).standard_normal((8, 3))
    g_L = gradient.loglik_grad(theta, yt)[2]
    assert np.all(np.triu(g_L, 1) == 0)


def test_delta_gradient_closed_form_static_case():
    """phi -> 0, d = 1: log Z = sum_t log N(y_t; mu, q + delta/2); d/d delta in closed form."""
    mu, q, delta = 0.2, 0.7, 0.4
    theta = (np.array([mu]), np.array([0.0]), np.array([[np.sqrt(q)]]), delta)
    yt = np.random.default_rng(3).standard_normal((6, 1))
    s2 = q + delta / 2
    expect = np.sum(-0.25 / s2 + 0.25 * (yt[:, 0] - mu) ** 2 / s2 ** 2)
    assert gradient.loglik_grad(theta, yt)[3] == pytest.approx(expect, rel=1e-10)

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


def test_sv_model_is_the_stationary_ar1():
    """The theta -> model map: P0 solves the discrete Lyapunov equation P0 = F P0 F^T + Q
    (scipy's solver) and m0 = b / (1 - phi) is the stationary mean."""
    sl = pytest.importorskip("scipy.linalg")
    mu, phi, L, delta = _theta(4, 7)
    m = gradient.sv_model(mu, phi, L, delta)
    P0 = sl.solve_discrete_lyapunov(m["F"], m["Q"])
    assert np.max(np.abs(m["P0"] - P0)) < 1e-10 * np.max(np.abs(P0))
    assert np.max(np.abs(m["m0"] - m["b"] / (1.0 - phi))) < 1e-12
    assert np.allclose(m["Q"], L @ L.T) and np.allclose(m["R"], 0.5 * delta * np.eye(4))


def test_theta_update_is_a_projected_mean_gradient_step():
    mu, phi, L, _ = _theta(3, 2)
    rng = np.random.default_rng(5)
    C = 4
    g_mu, g_phi, g_L = rng.standard_normal((C, 3)), rng.standard_normal((C, 3)), rng.standard_normal((C, 3, 3))
    lr = 1e-3
    mu2, phi2, L2 = gradient.sv_theta_update(mu, phi, L, g_mu, g_phi, g_L, lr)
    assert np.allclose(mu2, mu + lr * g_mu.sum(0) / C, rtol=0, atol=1e-15)
    assert np.allclose(phi2, phi + lr * g_phi.sum(0) / C, rtol=0, atol=1e-15)
    assert np.allclose(L2, np.tril(L + lr * g_L.sum(0) / C), rtol=0, atol=1e-15)
    # projections: phi kept inside the unit interval, diag(L) positive, upper part zero
    mu3, phi3, L3 = gradient.sv_theta_update(mu, phi, L, g_mu, 1e4 * np.ones((C, 3)), -1e4 * np.ones((C, 3, 3)), 1.0)
    assert np.all(phi3 == gradient.PHI_MAX)
    assert np.all(np.diag(L3) == gradient.L_MIN) and np.all(np.triu(L3, 1) == 0)


def test_a_small_step_along_the_gradient_increases_the_mean_loglik():
    """The ascent property the update relies on: a small step along the mean gradient
    raises the mean log Z over the chains' pseudo-observations."""
    theta = _theta(2, 3)
    rng = np.random.default_rng(9)
    yts = [rng.standard_normal((15, 2)) for _ in range(3)]
    gs = [gradient.loglik_grad(theta, yt) for yt in yts]
    g_mu = np.array([g[0] for g in gs]); g_phi = np.array([g[1] for g in gs]); g_L = np.array([g[2] for g in gs])
    mu2, phi2, L2 = gradient.sv_theta_update(theta[0], theta[1], theta[2], g_mu, g_phi, g_L, 1e-4)
    before = np.mean([gradient.loglik(theta, yt) for yt in yts])
    after = np.mean([gradient.loglik((mu2, phi2, L2, theta[3]), yt) for yt in yts])
    assert after > before

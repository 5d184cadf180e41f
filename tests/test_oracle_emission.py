"""Pins of the oracle's emission models against definitions outside the oracle.

The stochastic-volatility emission of Section 4.1 is y_t(i) ~ N(0, exp(x_t(i))):
its log density is checked against scipy's normal log-pdf with scale
exp(x/2), its gradient against central differences of that scipy density
(not of the oracle's own log_h), and its Hessian against central differences
of the gradient. The linear-Gaussian emission (Appendix A, y_t ~ N(x_t, R_y))
is checked the same way against scipy's multivariate normal. Planted mistakes
(a flipped sign, a dropped -x/2 term, a factor 2) in a copy of the formulas
must fail the same checks, so the checks are sensitive to them.
"""
import numpy as np
import pytest

from oracle import mcmc

stats = pytest.importorskip("scipy.stats")


def _sv_case(seed=0, T=9, d=5):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.5, (T, d))
    y = np.exp(x / 2) * rng.standard_normal((T, d)) + rng.normal(0, 0.3, (T, d))
    return x, y


def _scipy_sv_logh(x, y):
    """sum_i log N(y_t(i); 0, exp(x_t(i))), by scipy (scale = standard deviation)."""
    return stats.norm.logpdf(y, loc=0.0, scale=np.exp(x / 2)).sum(axis=1)


def _central_diff(f, x, h):
    """[T][d] central differences of a per-t scalar function f(x) -> [T] in each x_t(i)."""
    T, d = x.shape
    g = np.zeros((T, d))
    for i in range(d):
        e = np.zeros((T, d))
        e[:, i] = h
        g[:, i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def test_sv_log_density_matches_scipy():
    for seed in range(3):
        x, y = _sv_case(seed)
        em = mcmc.SVEmission(y)
        assert np.max(np.abs(em.log_h(x) - _scipy_sv_logh(x, y))) < 1e-11


def test_sv_mask_switches_terms_off():
    x, y = _sv_case(4)
    mask = np.array([1, 0, 1, 1, 0, 1, 0, 1, 1], bool)
    em = mcmc.SVEmission(y, mask)
    ref = np.where(mask, _scipy_sv_logh(x, y), 0.0)
    assert np.max(np.abs(em.log_h(x) - ref)) < 1e-11
    assert np.all(em.grad(x)[~mask] == 0.0)


def test_sv_gradient_matches_finite_differences_of_scipy():
    for seed in range(3):
        x, y = _sv_case(10 + seed)
        em = mcmc.SVEmission(y)
        fd = _central_diff(lambda z: _scipy_sv_logh(z, y), x, 1e-5)
        scale = np.maximum(1.0, np.abs(fd))
        assert np.max(np.abs(em.grad(x) - fd) / scale) < 1e-7


def test_sv_hessian_matches_finite_differences_of_the_gradient():
    x, y = _sv_case(20)
    em = mcmc.SVEmission(y)
    H = em.hess(x)
    T, d = x.shape
    h = 1e-5
    for i in range(d):
        e = np.zeros((T, d))
        e[:, i] = h
        col = (em.grad(x + e) - em.grad(x - e)) / (2 * h)       # d v / d x_i, [T][d]
        assert np.max(np.abs(H[:, :, i] - col) / np.maximum(1.0, np.abs(col))) < 1e-6


@pytest.mark.parametrize("mistake", ["sign", "drop_half_x", "factor_two"])
def test_sv_pins_catch_planted_mistakes(mistake):
    """A copy of the SV formulas with one plausible slip fails the pins above."""
    x, y = _sv_case(30)

    def log_h(z):
        if mistake == "drop_half_x":
            lh = -0.5 * np.log(2 * np.pi) - 0.5 * y ** 2 * np.exp(-z)
        elif mistake == "factor_two":
            lh = -0.5 * np.log(2 * np.pi) - 0.5 * z - y ** 2 * np.exp(-z)
        else:
            lh = -0.5 * np.log(2 * np.pi) - 0.5 * z - 0.5 * y ** 2 * np.exp(-z)
        return lh.sum(axis=1)

    def grad(z):
        if mistake == "sign":
            return 0.5 - 0.5 * y ** 2 * np.exp(-z)
        return -0.5 + 0.5 * y ** 2 * np.exp(-z)

    ld_err = np.max(np.abs(log_h(x) - _scipy_sv_logh(x, y)))
    fd = _central_diff(lambda z: _scipy_sv_logh(z, y), x, 1e-5)
    g_err = np.max(np.abs(grad(x) - fd) / np.maximum(1.0, np.abs(fd)))
    assert ld_err > 1e-3 or g_err > 1e-3


def _lg_case(seed=0, T=6, d=4):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    Ry = A @ A.T + 0.5 * np.eye(d)
    return rng.standard_normal((T, d)), rng.standard_normal((T, d)), Ry


def _scipy_lg_logh(x, y, Ry):
    return np.array([stats.multivariate_normal(mean=x[t], cov=Ry).logpdf(y[t]) for t in range(len(x))])


def test_linear_gaussian_log_density_matches_scipy():
    for seed in range(3):
        x, y, Ry = _lg_case(seed)
        em = mcmc.LinearGaussianEmission(y, Ry)
        assert np.max(np.abs(em.log_h(x) - _scipy_lg_logh(x, y, Ry))) < 1e-10


def test_linear_gaussian_gradient_and_hessian_match_finite_differences():
    x, y, Ry = _lg_case(5)
    em = mcmc.LinearGaussianEmission(y, Ry)
    fd = _central_diff(lambda z: _scipy_lg_logh(z, y, Ry), x, 1e-5)
    assert np.max(np.abs(em.grad(x) - fd)) < 1e-6
    H = em.hess(x)
    T, d = x.shape
    for i in range(d):
        e = np.zeros((T, d))
        e[:, i] = 1e-5
        col = (em.grad(x + e) - em.grad(x - e)) / 2e-5
        assert np.max(np.abs(H[:, :, i] - col)) < 1e-6


@pytest.mark.parametrize("mistake", ["sign", "drop_logdet", "covariance_for_precision"])
def test_linear_gaussian_pins_catch_planted_mistakes(mistake):
    """A copy of the linear-Gaussian formulas with one plausible slip fails the pins."""
    x, y, Ry = _lg_case(6)
    d = Ry.shape[0]
    P = np.linalg.inv(Ry)
    r = y - x
    q = np.einsum("ti,ij,tj->t", r, P, r)
    const = -0.5 * (d * np.log(2 * np.pi) + np.linalg.slogdet(Ry)[1])
    log_h = (-0.5 * d * np.log(2 * np.pi) - 0.5 * q) if mistake == "drop_logdet" else const - 0.5 * q
    if mistake == "sign":
        grad = -(r @ P)
    elif mistake == "covariance_for_precision":
        grad = r @ Ry
    else:
        grad = r @ P
    ld_err = np.max(np.abs(log_h - _scipy_lg_logh(x, y, Ry)))
    fd = _central_diff(lambda z: _scipy_lg_logh(z, y, Ry), x, 1e-5)
    assert ld_err > 1e-3 or np.max(np.abs(grad - fd)) > 1e-3

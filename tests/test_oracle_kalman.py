"""Pins of the oracle's Kalman filter, RTS sampler and parallel-scan operators.

Each pin compares the oracle with something other than itself: scalar closed
forms, a dense stacked-path Gaussian, a different scan schedule, or an
AR(1) closed form.
"""
import numpy as np
import pytest

from oracle import dense, kalman
from paper_2303_00301_gb300 import workloads


def _scalar_logpdf(y, mean, var):
    return -0.5 * (np.log(2 * np.pi * var) + (y - mean) ** 2 / var)


def test_scalar_T1_closed_form():
    # Bayes for one scalar Gaussian observation (Appendix A.1, t = 0 step)
    m0, p0, r, y = 0.3, 2.0, 0.5, 1.7
    kf = kalman.kalman_filter(np.array([[y]]), np.array([m0]), np.array([[p0]]),
                              np.eye(1), np.zeros(1), np.eye(1), np.array([[r]]))
    assert kf["mf"][0, 0] == pytest.approx(m0 + p0 / (p0 + r) * (y - m0), rel=1e-14)
    assert kf["Pf"][0, 0, 0] == pytest.approx(p0 * r / (p0 + r), rel=1e-14)
    assert kf["logZ"] == pytest.approx(_scalar_logpdf(y, m0, p0 + r), rel=1e-14)


def test_scalar_T2_closed_form():
    # (y0, y1) jointly Gaussian; log Z and E[x1 | y0, y1] written out with 2x2 algebra.
    m0, p0, f, bb, q, r = -0.2, 1.5, 0.7, 0.1, 0.4, 0.3
    y0, y1 = 0.9, -0.4
    mu = np.array([m0, f * m0 + bb])
    s00, s01, s11 = p0 + r, f * p0, f * f * p0 + q + r
    det = s00 * s11 - s01 * s01
    e0, e1 = y0 - mu[0], y1 - mu[1]
    quad = (s11 * e0 * e0 - 2 * s01 * e0 * e1 + s00 * e1 * e1) / det
    logZ = -0.5 * (2 * np.log(2 * np.pi) + np.log(det) + quad)
    # cov(x1, (y0, y1)) = (f p0, f^2 p0 + q)
    c0, c1 = f * p0, f * f * p0 + q
    w0 = (s11 * c0 - s01 * c1) / det
    w1 = (-s01 * c0 + s00 * c1) / det
    mf1 = mu[1] + w0 * e0 + w1 * e1
    Pf1 = (f * f * p0 + q) - (w0 * c0 + w1 * c1)
    kf = kalman.kalman_filter(np.array([[y0], [y1]]), np.array([m0]), np.array([[p0]]),
                              np.array([[f]]), np.array([bb]), np.array([[q]]), np.array([[r]]))
    assert kf["logZ"] == pytest.approx(logZ, rel=1e-13)
    assert kf["mf"][1, 0] == pytest.approx(mf1, rel=1e-13)
    assert kf["Pf"][1, 0, 0] == pytest.approx(Pf1, rel=1e-13)


def test_dense_prior_is_ar1_closed_form():
    # stationary AR(1): cov(x_t, x_s) = q / (1 - phi^2) phi^|t-s|
    phi, q, T = 0.8, 0.5, 6
    p_stat = q / (1 - phi ** 2)
    mean, C = dense.prior_moments(np.zeros(1), np.array([[p_stat]]), np.array([[phi]]),
                                  np.zeros(1), np.array([[q]]), T)
    idx = np.arange(T)
    expect = p_stat * phi ** np.abs(idx[:, None] - idx[None, :])
    assert np.allclose(C, expect, rtol=1e-13, atol=0)
    assert np.all(mean == 0)


@pytest.mark.parametrize("d,T,tv", [(1, 3, False), (2, 5, False), (3, 8, True), (2, 7, True)])
def test_filter_and_smoother_match_dense_gaussian(d, T, tv):
    m = workloads.random_lgssm(d, T, seed=10 * d + T, time_varying=tv)
    R = 0.37 * np.eye(d)
    kf = kalman.kalman_filter(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], R)
    mbar, C = dense.prior_moments(m["m0"], m["P0"], m["F"], m["b"], m["Q"], T)
    post_mean, post_cov, logZ = dense.lgssm_posterior(m["y"], 2 * 0.37, mbar, C)
    assert kf["logZ"] == pytest.approx(logZ, rel=1e-11)
    ms, Ps = kalman.rts_smoother(kf, m["F"])
    assert np.allclose(ms.reshape(-1), post_mean, rtol=0, atol=1e-10)
    for t in range(T):
        blk = post_cov[t * d:(t + 1) * d, t * d:(t + 1) * d]
        assert np.allclose(Ps[t], blk, rtol=0, atol=1e-10)
    # the last filtered marginal equals the last smoothed marginal
    assert np.allclose(kf["mf"][-1], post_mean[-d:], atol=1e-10)


@pytest.mark.parametrize("d,T,tv", [(1, 4, False), (2, 6, True), (3, 5, False)])
def test_rts_sampler_law_is_dense_posterior(d, T, tv):
    """x* is affine in the noise: its mean and covariance must be the dense posterior's."""
    m = workloads.random_lgssm(d, T, seed=d + 100 * T, time_varying=tv)
    R = 0.2 * np.eye(d)
    kf = kalman.kalman_filter(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], R)
    x0 = kalman.rts_sample(kf, m["F"], m["b"], m["Q"], np.zeros((T, d)))
    cols = []
    for k in range(T * d):
        e = np.zeros(T * d); e[k] = 1.0
        cols.append((kalman.rts_sample(kf, m["F"], m["b"], m["Q"], e.reshape(T, d)) - x0).reshape(-1))
    Mmap = np.stack(cols, axis=1)
    mbar, C = dense.prior_moments(m["m0"], m["P0"], m["F"], m["b"], m["Q"], T)
    post_mean, post_cov, _ = dense.lgssm_posterior(m["y"], 0.4, mbar, C)
    assert np.allclose(x0.reshape(-1), post_mean, atol=1e-10)
    assert np.allclose(Mmap @ Mmap.T, post_cov, atol=1e-10)


def test_titsias_form_equals_lgssm_posterior():
    """Section 2.2: with Sigma_t = I the LGSSM proposal is Eq. (2.2)'s proposal."""
    d, T, delta = 2, 5, 0.3
    m = workloads.random_lgssm(d, T, seed=3)
    rng = np.random.default_rng(0)
    u = rng.standard_normal((T, d)); g = rng.standard_normal((T, d))
    mbar, C = dense.prior_moments(m["m0"], m["P0"], m["F"], m["b"], m["Q"], T)
    mean_t, A = dense.titsias_proposal(u, g, delta, mbar, C)
    kf = kalman.kalman_filter(u + 0.5 * delta * g, m["m0"], m["P0"], m["F"], m["b"], m["Q"],
                              0.5 * delta * np.eye(d))
    ms, Ps = kalman.rts_smoother(kf, m["F"])
    assert np.allclose(ms.reshape(-1), mean_t, atol=1e-10)
    for t in range(T):
        assert np.allclose(Ps[t], A[t * d:(t + 1) * d, t * d:(t + 1) * d], atol=1e-10)


@pytest.mark.parametrize("d,T,tv", [(1, 9, False), (2, 16, True), (3, 13, False), (4, 33, True)])
def test_parallel_filter_scan_equals_sequential_filter(d, T, tv):
    m = workloads.random_lgssm(d, T, seed=7 * d + T, time_varying=tv)
    R = 0.25 * np.eye(d)
    kf = kalman.kalman_filter(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], R)
    el = kalman.filter_elements(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], R)
    for scan in (kalman.sequential_scan, kalman.hillis_steele_scan):
        pref = scan(el, kalman.filter_combine)
        mf = np.stack([p[1] for p in pref]); Pf = np.stack([p[2] for p in pref])
        assert np.allclose(mf, kf["mf"], rtol=0, atol=1e-12 * max(1, np.abs(kf["mf"]).max()))
        assert np.allclose(Pf, kf["Pf"], rtol=0, atol=1e-12 * max(1, np.abs(kf["Pf"]).max()))
        # prefixes starting at t = 0 are marginals: A = 0, J = 0, eta = 0
        assert max(np.abs(p[0]).max() for p in pref) == 0.0
        assert max(np.abs(p[4]).max() for p in pref) < 1e-14


def test_filter_combine_is_associative():
    d, T = 3, 5
    m = workloads.random_lgssm(d, T, seed=11, time_varying=True)
    el = kalman.filter_elements(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], 0.3 * np.eye(d))
    a, b, c = el[1], el[2], el[3]
    lhs = kalman.filter_combine(kalman.filter_combine(a, b), c)
    rhs = kalman.filter_combine(a, kalman.filter_combine(b, c))
    for x, y in zip(lhs, rhs):
        assert np.allclose(x, y, atol=1e-12)


@pytest.mark.parametrize("d,T,tv", [(1, 7, False), (3, 12, True), (2, 32, False)])
def test_backward_suffix_scan_is_rts_sampler(d, T, tv):
    """Proposition A.1 pathwise: identical noise gives identical paths."""
    m = workloads.random_lgssm(d, T, seed=5 * d + T, time_varying=tv)
    kf = kalman.kalman_filter(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], 0.3 * np.eye(d))
    eps = np.random.default_rng(1).standard_normal((T, d))
    x_seq = kalman.rts_sample(kf, m["F"], m["b"], m["Q"], eps)
    gu = kalman.backward_elements(kf, m["F"], m["b"], m["Q"], eps)
    x_par = np.stack([e[1] for e in kalman.suffix_scan(gu, kalman.backward_combine)])
    assert np.allclose(x_par, x_seq, rtol=0, atol=1e-12 * max(1, np.abs(x_seq).max()))


def test_two_backward_covariance_forms_agree():
    """Sigma_t = P^f - G (F P^f F^T + Q) G^T equals L = P^f - G F P^f (App. A.2.3 init)."""
    d, T = 3, 6
    m = workloads.random_lgssm(d, T, seed=2)
    kf = kalman.kalman_filter(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], 0.5 * np.eye(d))
    F, Q = m["F"], m["Q"]
    for t in range(T - 1):
        Pf = kf["Pf"][t]
        Ppn = F @ Pf @ F.T + Q
        G = np.linalg.solve(Ppn, F @ Pf).T
        assert np.allclose(Pf - G @ Ppn @ G.T, Pf - G @ F @ Pf, atol=1e-12)


def test_planted_sign_error_is_caught():
    """A plausible mistake in the element operator (sign of the eta correction) fails the scan pin."""
    d, T = 2, 8
    m = workloads.random_lgssm(d, T, seed=4)
    R = 0.25 * np.eye(d)
    kf = kalman.kalman_filter(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], R)
    el = kalman.filter_elements(m["y"], m["m0"], m["P0"], m["F"], m["b"], m["Q"], R)

    def bad_combine(ei, ej):
        Ai, bi, Ci, ei_, Ji = ei
        A, bb, C, eta, J = kalman.filter_combine(ei, ej)
        # flip the sign of the J_j b_i term inside eta
        Aj, bj, Cj, ej_, Jj = ej
        M = np.eye(d) + Ci @ Jj
        eta_bad = Ai.T @ np.linalg.solve(M.T, ej_ + Jj @ bi) + ei_
        return (A, bb, C, eta_bad, J)

    pref = kalman.hillis_steele_scan(el, bad_combine)
    mf = np.stack([p[1] for p in pref])
    assert not np.allclose(mf, kf["mf"], atol=1e-6)

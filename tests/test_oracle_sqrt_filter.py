"""Pins of the oracle's square-root parallel filter (oracle/sqrt_filter.py).

The square-root formulas are derived, not printed by the paper (Section 4.1
names the method only), so every one is pinned against the covariance form
(oracle/kalman.py, itself pinned to closed forms and the dense Gaussian):
- tria: lower triangular, positive diagonal, L L^T = X X^T, also for X of
  deficient rank and for a QR-friendly ill-conditioned X;
- each square-root element against filter_elements (A, b, U U^T = C, eta, Z Z^T = J);
- each square-root combine against filter_combine on the same elements;
- the filter (sequential and Hillis-Steele) against kalman_filter: m^f, P^f, ell_t, log Z.
"""
import numpy as np
import pytest

from oracle import kalman, sqrt_filter as sf
from paper_2303_00301_gb300 import workloads


@pytest.mark.parametrize("d,k,seed", [(1, 2, 0), (3, 6, 1), (5, 10, 2), (4, 12, 3), (6, 7, 4)])
def test_tria_identity(d, k, seed):
    X = np.random.default_rng(seed).standard_normal((d, k))
    L = sf.tria(X)
    assert np.allclose(np.triu(L, 1), 0)
    assert np.all(np.diag(L) > 0)
    assert np.allclose(L @ L.T, X @ X.T, atol=1e-12)
    assert np.allclose(L, np.linalg.cholesky(X @ X.T), atol=1e-10)


def test_tria_rank_deficient_and_ill_conditioned():
    rng = np.random.default_rng(9)
    B = rng.standard_normal((4, 2))
    X = np.hstack([B @ rng.standard_normal((2, 3)), np.zeros((4, 3))])     # rank 2
    L = sf.tria(X)
    assert np.allclose(L @ L.T, X @ X.T, atol=1e-12)
    assert np.all(np.diag(L) >= 0)
    # X X^T with condition number ~1e16: its Cholesky in FP64 is unreliable, tria is not
    X = np.diag([1.0, 1e-8, 1e-8]) @ rng.standard_normal((3, 6))
    L = sf.tria(X)
    assert np.allclose(L @ L.T, X @ X.T, rtol=0, atol=1e-14)


def _model(d, T, seed, tv=False):
    m = workloads.random_lgssm(d, T, seed=seed)
    rng = np.random.default_rng(seed + 50)
    F, b, Q = m["F"], m["b"], m["Q"]
    R = 0.35 * np.eye(d)
    if tv:
        F = np.stack([F * (0.6 + 0.4 * rng.random()) for _ in range(T - 1)])
        b = rng.standard_normal((T - 1, d))
        Q = np.stack([Q * (0.5 + rng.random()) for _ in range(T - 1)])
        A = rng.standard_normal((T, d, d))
        R = np.stack([a @ a.T / d + 0.2 * np.eye(d) for a in A])
    y = rng.standard_normal((T, d)) * 1.3
    return y, m["m0"], m["P0"], F, b, Q, R


@pytest.mark.parametrize("tv", [False, True])
@pytest.mark.parametrize("d,T,seed", [(1, 6, 0), (2, 9, 1), (3, 12, 2), (5, 7, 3)])
def test_elements_and_operator_match_the_covariance_form(d, T, seed, tv):
    y, m0, P0, F, b, Q, R = _model(d, T, seed, tv)
    ref = kalman.filter_elements(y, m0, P0, F, b, Q, R)
    sr = sf.sr_elements(y, m0, P0, F, b, Q, R)
    for (A, bb, C, eta, J), (As, bs, U, es, Z) in zip(ref, sr):
        assert np.allclose(A, As, atol=1e-12)
        assert np.allclose(bb, bs, atol=1e-12)
        assert np.allclose(C, U @ U.T, atol=1e-12)
        assert np.allclose(eta, es, atol=1e-12)
        assert np.allclose(J, Z @ Z.T, atol=1e-12)
    for i in range(T - 1):
        A, bb, C, eta, J = kalman.filter_combine(ref[i], ref[i + 1])
        As, bs, U, es, Z = sf.sr_combine(sr[i], sr[i + 1])
        assert np.allclose(A, As, atol=1e-11)
        assert np.allclose(bb, bs, atol=1e-11)
        assert np.allclose(C, U @ U.T, atol=1e-11)
        assert np.allclose(eta, es, atol=1e-11)
        assert np.allclose(J, Z @ Z.T, atol=1e-11)
        assert np.allclose(np.triu(U, 1), 0) and np.allclose(np.triu(Z, 1), 0)
    # combines of combines (the scan's later rounds)
    e01 = sf.sr_combine(sr[0], sr[1])
    e23 = sf.sr_combine(sr[2], sr[3]) if T > 3 else sr[2]
    r01 = kalman.filter_combine(ref[0], ref[1])
    r23 = kalman.filter_combine(ref[2], ref[3]) if T > 3 else ref[2]
    got, want = sf.sr_combine(e01, e23), kalman.filter_combine(r01, r23)
    assert np.allclose(got[1], want[1], atol=1e-11)
    assert np.allclose(got[2] @ got[2].T, want[2], atol=1e-11)


@pytest.mark.parametrize("schedule", ["sequential", "hillis_steele"])
@pytest.mark.parametrize("tv", [False, True])
@pytest.mark.parametrize("d,T,seed", [(1, 5, 0), (2, 16, 1), (3, 13, 2), (4, 1, 3)])
def test_filter_matches_kalman_filter(d, T, seed, tv, schedule):
    if T == 1 and tv:
        pytest.skip("no transitions")
    y, m0, P0, F, b, Q, R = _model(d, T, seed, tv)
    kf = kalman.kalman_filter(y, m0, P0, F, b, Q, R)
    out = sf.sr_filter(y, m0, P0, F, b, Q, R, schedule=schedule)
    assert np.allclose(out["mf"], kf["mf"], atol=1e-10)
    assert np.allclose(np.einsum("tij,tkj->tik", out["Uf"], out["Uf"]), kf["Pf"], atol=1e-10)
    assert np.allclose(out["ell"], kf["ell"], atol=1e-10)
    assert abs(out["logZ"] - kf["logZ"]) < 1e-9

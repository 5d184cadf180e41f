"""Pins of the oracle's divide-and-conquer sampler (Section 2.4.2, Appendix A.2.3).

Everything is checked against the dense Gaussian of the stacked path
(oracle/dense.py: the prior moments of the dynamics and the exact posterior
given ytilde ~ N(x, (delta/2) I)), never against the tree itself:
- each node's (E, g, L) is the dense conditional law of x_k given x_m;
- each bridge (G, Gamma, w, V) is the dense conditional law of x_l given (x_k, x_m);
- the sampler is affine in eps; its offset is the dense posterior mean and the
  product of its matrix with its transpose the dense posterior covariance;
- with T = 2 the tree is one leaf and the draw is the RTS sampler's;
- every state is drawn exactly once, whatever T.
"""
import numpy as np
import pytest

from oracle import bridging, dense, kalman
from paper_2303_00301_gb300 import workloads


def _setup(d, T, seed, delta=0.6, homogeneous=True):
    m = workloads.random_lgssm(d, T, seed=seed)
    rng = np.random.default_rng(seed + 7)
    F, b, Q = m["F"], m["b"], m["Q"]
    if not homogeneous:     # a time-varying stack exercises the per-step indices
        F = np.stack([F * (0.7 + 0.3 * rng.random()) for _ in range(T - 1)])
        b = rng.standard_normal((T - 1, d))
        Q = np.stack([Q * (0.5 + rng.random()) for _ in range(T - 1)])
    yt = rng.standard_normal((T, d)) * 1.5
    R = 0.5 * delta * np.eye(d)
    kf = kalman.kalman_filter(yt, m["m0"], m["P0"], F, b, Q, R)
    mbar, C = dense.prior_moments(m["m0"], m["P0"], F, b, Q, T)
    mean, cov, _ = dense.lgssm_posterior(yt, delta, mbar, C)
    return kf, F, b, Q, mean, cov


def _blk(i, d):
    return slice(i * d, (i + 1) * d)


def _cond(mean, cov, d, target, given):
    """Dense Gaussian conditioning: x_target | x_given = A x_given + c, covariance S."""
    ti = np.concatenate([np.arange(t * d, (t + 1) * d) for t in target])
    gi = np.concatenate([np.arange(t * d, (t + 1) * d) for t in given])
    A = np.linalg.solve(cov[np.ix_(gi, gi)], cov[np.ix_(gi, ti)]).T
    c = mean[ti] - A @ mean[gi]
    S = cov[np.ix_(ti, ti)] - A @ cov[np.ix_(gi, ti)]
    return A, c, S


CASES = [(1, 3, 0), (2, 5, 1), (3, 8, 2), (2, 9, 3), (1, 13, 4), (3, 6, 5), (2, 17, 6)]


@pytest.mark.parametrize("homogeneous", [True, False])
@pytest.mark.parametrize("d,T,seed", CASES)
def test_node_elements_and_bridges_are_dense_conditionals(d, T, seed, homogeneous):
    kf, F, b, Q, mean, cov = _setup(d, T, seed, homogeneous=homogeneous)
    levels = bridging.build_tree(kf, F, b, Q)
    n_bridges = 0
    for level in levels:
        for node in level:
            k, m = node["k"], node["m"]
            E, g, L = _cond(mean, cov, d, [k], [m])
            assert np.allclose(node["E"], E, atol=1e-9), (k, m)
            assert np.allclose(node["g"], g, atol=1e-9), (k, m)
            assert np.allclose(node["L"], L, atol=1e-9), (k, m)
            if node["l"] is not None:
                n_bridges += 1
                A, c, S = _cond(mean, cov, d, [node["l"]], [k, m])
                assert np.allclose(node["G"], A[:, :d], atol=1e-9)
                assert np.allclose(node["Gam"], A[:, d:], atol=1e-9)
                assert np.allclose(node["w"], c, atol=1e-9)
                assert np.allclose(node["V"], S, atol=1e-9)
    assert n_bridges == max(T - 2, 0)
    assert len(levels[-1]) == 1 and levels[-1][0]["k"] == 0 and levels[-1][0]["m"] == T - 1


@pytest.mark.parametrize("d,T,seed", CASES + [(2, 2, 9), (2, 1, 10)])
def test_sampler_has_the_dense_posterior_law(d, T, seed):
    kf, F, b, Q, mean, cov = _setup(d, T, seed)
    n = T * d
    mu = bridging.dnc_sample(kf, F, b, Q, np.zeros((T, d))).reshape(-1)
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = bridging.dnc_sample(kf, F, b, Q, e.reshape(T, d)).reshape(-1) - mu
    assert np.allclose(mu, mean, atol=1e-9)
    assert np.allclose(A @ A.T, cov, atol=1e-9)


def test_two_states_reduce_to_the_rts_sampler():
    kf, F, b, Q, _, _ = _setup(3, 2, 11)
    eps = np.random.default_rng(0).standard_normal((2, 3))
    assert np.allclose(bridging.dnc_sample(kf, F, b, Q, eps), kalman.rts_sample(kf, F, b, Q, eps),
                       atol=1e-12)


def test_every_state_is_drawn_once():
    for T in range(1, 40):
        kf, F, b, Q, _, _ = _setup(1, T, 100 + T)
        x = bridging.dnc_sample(kf, F, b, Q, np.zeros((T, 1)))
        assert np.all(np.isfinite(x)), T
        if T > 2:
            levels = bridging.build_tree(kf, F, b, Q)
            ls = sorted(nd["l"] for lv in levels for nd in lv if nd["l"] is not None)
            assert ls == list(range(1, T - 1)), T


def test_differs_from_rts_draw_but_not_in_law():
    """Same eps, different factorisation of the same law: paths differ for T > 2."""
    kf, F, b, Q, _, _ = _setup(2, 9, 3)
    eps = np.random.default_rng(1).standard_normal((9, 2))
    assert not np.allclose(bridging.dnc_sample(kf, F, b, Q, eps), kalman.rts_sample(kf, F, b, Q, eps))

"""The matrix identities the wide table-mode kernels evaluate, checked in FP64
against the oracle's definitions (oracle/kalman.py): the covariance-only
element constants, the C-only operator on prefixes (A = J = 0), the prefixes
by doubling over the steps, and the per-step tables (K' = r S^{-1}, G, Sigma)
in the factored forms the kernels use, and the blocked recurrences of the CTA
routines (the triangular inverse by 32 x 32 blocks, the Cholesky factorisation
without square roots in blocks of 8 columns). The GPU parity tests check the
kernels themselves; these check the algebra they rest on, on the CPU.
"""
import numpy as np
import pytest

from oracle import kalman
from paper_2303_00301_gb300 import workloads


def _model(d, T, seed):
    m = workloads.random_lgssm(d, T, seed=seed)
    return m["m0"], m["P0"], m["F"], m["b"], m["Q"]


def _chol(A):
    return np.linalg.cholesky(A)


def _elements_factored(P0, F, Q, r):
    """k_w_elem: C_0 = P0 - Y^T Y (Y = chol(P0 + R)^{-1} P0); for t >= 1 with
    S = Q + R = L L^T: C = Q - Y^T Y (Y = L^{-1} Q), J = W^T W (W = L^{-1} F), A = r L^{-T} W."""
    d = P0.shape[0]
    I = np.eye(d)
    Li0 = np.linalg.inv(_chol(P0 + r * I))
    Y0 = Li0 @ P0
    C0 = P0 - Y0.T @ Y0
    Li = np.linalg.inv(_chol(Q + r * I))
    Y = Li @ Q
    W = Li @ F
    return C0, (r * Li.T @ W, Q - Y.T @ Y, W.T @ W)


def _combine_c_only(Ci, E):
    """k_w_double on a prefix (A_i = 0, J_i = 0): C = C_e + P P^T, P = A_e U chol(N)^{-T},
    U = chol(C_i), N = I + U^T J_e U."""
    Ae, Ce, Je = E
    U = _chol(Ci)
    N = np.eye(len(Ci)) + U.T @ Je @ U
    B = U @ np.linalg.inv(_chol(N)).T
    P = Ae @ B
    return Ce + P @ P.T


def _combine_full(Ei, E):
    """The squaring E^(2^k) (x) E^(2^k) of k_w_double: the full operator in the same form."""
    Ai, Ci, Ji = Ei
    Ae, Ce, Je = E
    U = _chol(Ci)
    N = np.eye(len(Ci)) + U.T @ Je @ U
    B = U @ np.linalg.inv(_chol(N)).T
    P = Ae @ B
    X1 = Je @ Ai
    Z = B.T @ X1
    return (Ae @ Ai - P @ Z, Ce + P @ P.T, Ji + Ai.T @ X1 - Z.T @ Z)


@pytest.mark.parametrize("d,seed", [(1, 0), (3, 1), (6, 2)])
def test_element_constants_match_the_oracle_elements(d, seed):
    m0, P0, F, b, Q = _model(d, 4, seed)
    r = 0.35
    y = np.random.default_rng(seed).standard_normal((4, d))
    el = kalman.filter_elements(y, m0, P0, F, b, Q, r * np.eye(d))
    C0, (A, C, J) = _elements_factored(P0, F, Q, r)
    assert np.allclose(C0, el[0][2], atol=1e-12)
    for t in (1, 2, 3):
        assert np.allclose(A, el[t][0], atol=1e-12)
        assert np.allclose(C, el[t][2], atol=1e-12)
        assert np.allclose(J, el[t][4], atol=1e-12)


@pytest.mark.parametrize("d,seed", [(2, 3), (5, 4)])
def test_operators_match_the_oracle_operator(d, seed):
    m0, P0, F, b, Q = _model(d, 4, seed)
    r = 0.2
    y = np.random.default_rng(seed).standard_normal((4, d))
    el = kalman.filter_elements(y, m0, P0, F, b, Q, r * np.eye(d))
    C0, E = _elements_factored(P0, F, Q, r)
    # C-only operator on a prefix (A = J = 0) against the full operator
    ref = kalman.filter_combine(el[0], el[1])
    assert np.allclose(_combine_c_only(C0, E), ref[2], atol=1e-11)
    # the full operator (squaring) against the oracle's
    e1 = (el[1][0], el[1][2], el[1][4])
    ref = kalman.filter_combine(el[1], el[2])
    got = _combine_full(e1, E)
    assert np.allclose(got[0], ref[0], atol=1e-11)
    assert np.allclose(got[1], ref[2], atol=1e-11)
    assert np.allclose(got[2], ref[4], atol=1e-11)


@pytest.mark.parametrize("d,T,seed", [(1, 9, 5), (4, 37, 6), (7, 64, 7)])
def test_doubling_prefixes_are_the_filtering_covariances(d, T, seed):
    """P_t = P_{t - 2^k} (x) E^(2^k) for 2^k <= t < 2^(k+1), E^(2^(k+1)) = E^(2^k) (x) E^(2^k)."""
    m0, P0, F, b, Q = _model(d, T, seed)
    r = 0.3
    C0, E = _elements_factored(P0, F, Q, r)
    P = [None] * T
    P[0] = C0
    Ek = E
    pow2 = 1
    while pow2 < T:
        for i in range(min(pow2, T - pow2)):
            P[pow2 + i] = _combine_c_only(P[i], Ek)
        Ek = _combine_full(Ek, Ek)
        pow2 *= 2
    y = np.zeros((T, d))
    kf = kalman.kalman_filter(y, m0, P0, F, b, Q, r * np.eye(d))
    assert np.allclose(np.stack(P), kf["Pf"], atol=1e-10)


@pytest.mark.parametrize("d,seed", [(2, 8), (6, 9)])
def test_per_step_tables_in_factored_form(d, seed):
    """k_w_epi: K'_t = r L_S^{-T} L_S^{-1}; with L_P = chol(P^p_{t+1}) and Y = L_P^{-1} F P^f_t:
    G_t^T = L_P^{-T} Y, Sigma_t = P^f_t - Y^T Y (the RTS gain and covariance of Appendix A.1)."""
    T = 6
    m0, P0, F, b, Q = _model(d, T, seed)
    r = 0.25
    kf = kalman.kalman_filter(np.zeros((T, d)), m0, P0, F, b, Q, r * np.eye(d))
    for t in range(T - 1):
        Pp_next = F @ kf["Pf"][t] @ F.T + Q
        assert np.allclose(Pp_next, kf["Pp"][t + 1], atol=1e-12)
        LiS = np.linalg.inv(_chol(kf["Pp"][t] + r * np.eye(d)))
        Kp = r * LiS.T @ LiS
        K = np.linalg.solve(kf["Pp"][t] + r * np.eye(d), kf["Pp"][t]).T
        assert np.allclose(Kp, np.eye(d) - K, atol=1e-12)
        LiP = np.linalg.inv(_chol(Pp_next))
        Y = LiP @ F @ kf["Pf"][t]
        G = (LiP.T @ Y).T
        G_ref = np.linalg.solve(Pp_next, F @ kf["Pf"][t]).T
        assert np.allclose(G, G_ref, atol=1e-11)
        Sig = kf["Pf"][t] - Y.T @ Y
        assert np.allclose(Sig, kf["Pf"][t] - G_ref @ Pp_next @ G_ref.T, atol=1e-11)


def _blocked_trinv(L, nb=32):
    """w_trinv's recurrence: the diagonal blocks inverted on their own, then the
    block columns from the second last to the first, X_(i,j) = -(sum_{k=j+1..i}
    X_(i,k) L_(k,j)) X_(j,j) for the blocks below the diagonal (from X L = I)."""
    n = L.shape[0]
    X = np.zeros_like(L)
    B = n // nb
    sl = [slice(b * nb, (b + 1) * nb) for b in range(B)]
    for b in range(B):
        X[sl[b], sl[b]] = np.linalg.inv(L[sl[b], sl[b]])
    for j in range(B - 2, -1, -1):
        below = slice((j + 1) * nb, n)
        X[below, sl[j]] = -(X[below, below] @ L[below, sl[j]]) @ X[sl[j], sl[j]]
    return X


def _blocked_ldl_chol(A, nk=8):
    """w_chol's recurrence: elimination without square roots in blocks of nk
    columns (S_ik -> L_ik sqrt(p_k)), the diagonal block, the panel below it
    and one rank-nk update of the trailing part per block; then L_ik = S_ik /
    sqrt(p_k)."""
    n = A.shape[0]
    S = np.tril(A.copy())
    p = np.zeros(n)
    for k in range(0, n, nk):
        e = min(n, k + nk)
        for c in range(k, e):   # diagonal block, column by column
            p[c] = S[c, c]
            for c2 in range(c + 1, e):
                S[c2, c + 1:c2 + 1] -= (S[c2, c] / p[c]) * S[c + 1:c2 + 1, c]
        for c in range(k, e):   # panel rows, row-locally
            l = S[e:, c] / p[c]
            S[e:, c + 1:e] -= np.outer(l, S[c + 1:e, c])
        Lm = S[e:, k:e] / p[k:e]   # rank-nk trailing update (lower part)
        S[e:, e:] -= np.tril(Lm @ S[e:, k:e].T)
    L = np.tril(S, -1) / np.sqrt(p)[None, :] + np.diag(np.sqrt(p))
    return L, 0.5 * np.sum(np.log(p))


@pytest.mark.parametrize("n", [64, 128])
def test_blocked_triangular_inverse_is_the_inverse(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    L = _chol(A @ A.T / n + np.eye(n))
    X = _blocked_trinv(L)
    assert np.allclose(X, np.linalg.inv(L), rtol=0, atol=1e-12 * np.abs(np.linalg.inv(L)).max())
    assert np.all(np.triu(X, 1) == 0.0)


@pytest.mark.parametrize("n", [5, 8, 37, 64, 101, 128])
def test_blocked_cholesky_without_square_roots_is_the_cholesky_factor(n):
    rng = np.random.default_rng(100 + n)
    A = rng.standard_normal((n, n))
    A = A @ A.T / n + 0.5 * np.eye(n)
    L, half_logdet = _blocked_ldl_chol(A)
    Lr = _chol(A)
    assert np.max(np.abs(L - Lr)) < 1e-12 * np.abs(Lr).max()
    assert abs(half_logdet - np.sum(np.log(np.diag(Lr)))) < 1e-10

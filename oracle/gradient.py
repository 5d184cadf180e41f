"""FP64 reference gradient of the auxiliary LGSSM log marginal likelihood.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this package.

The paper obtains gradients by automatic differentiation (Section 4) and does
not print a gradient of the Kalman likelihood; this module fixes the
conventions used by the library's ``aux_loglik_grad``:

* theta = (mu, phi, L, delta) of the multivariate SV model (Section 4.1):
  F = diag(phi), b = (I - F) mu, Q = L L^T (L lower triangular), p_0 the
  stationary law (m0 = mu, P0_ij = Q_ij / (1 - phi_i phi_j)), R = (delta/2) I.
* log Z(theta) = log p(ytilde | theta), the Kalman filter likelihood
  (Appendix A.1) of fixed pseudo-observations ytilde; delta enters through R.

Two independent routes:
  loglik_fd_grad   central finite differences of the Kalman filter log Z.
  loglik_grad      Fisher's identity, grad log p(y | theta) =
                   E[grad log p(x, y | theta) | y], with the smoothed means,
                   covariances and lag-one cross-covariances of the RTS
                   smoother (Appendix A.1). Pinned by loglik_fd_grad.
"""
import numpy as np

from . import kalman


def sv_model(mu, phi, L, delta):
    """LGSSM matrices of theta = (mu, phi, L, delta)."""
    mu = np.asarray(mu, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    L = np.tril(np.asarray(L, dtype=np.float64))
    d = len(mu)
    Q = L @ L.T
    P0 = Q / (1.0 - np.outer(phi, phi))
    return dict(m0=mu.copy(), P0=P0, F=np.diag(phi), b=(1.0 - phi) * mu, Q=Q,
                R=0.5 * delta * np.eye(d))


def loglik(theta, ytilde):
    m = sv_model(*theta)
    return kalman.kalman_filter(ytilde, m["m0"], m["P0"], m["F"], m["b"], m["Q"], m["R"])["logZ"]


def loglik_fd_grad(theta, ytilde, h=1e-6):
    """Central differences, step h * max(1, |theta_i|), for every free parameter."""
    mu, phi, L, delta = (np.array(v, dtype=np.float64) for v in theta)
    d = len(mu)

    def f(mu_, phi_, L_, delta_):
        return loglik((mu_, phi_, L_, delta_), ytilde)

    g_mu = np.zeros(d)
    g_phi = np.zeros(d)
    g_L = np.zeros((d, d))
    for i in range(d):
        s = h * max(1.0, abs(mu[i]))
        e = np.zeros(d); e[i] = s
        g_mu[i] = (f(mu + e, phi, L, delta) - f(mu - e, phi, L, delta)) / (2 * s)
        s = h * max(1.0, abs(phi[i]))
        e = np.zeros(d); e[i] = s
        g_phi[i] = (f(mu, phi + e, L, delta) - f(mu, phi - e, L, delta)) / (2 * s)
        for j in range(i + 1):
            s = h * max(1.0, abs(L[i, j]))
            E = np.zeros((d, d)); E[i, j] = s
            g_L[i, j] = (f(mu, phi, L + E, delta) - f(mu, phi, L - E, delta)) / (2 * s)
    s = h * max(1.0, abs(float(delta)))
    g_delta = (f(mu, phi, L, delta + s) - f(mu, phi, L, delta - s)) / (2 * s)
    return g_mu, g_phi, g_L, float(g_delta)


def smoother_moments(theta, ytilde):
    """Filter, then RTS smoother means m_t, covariances P_t and cross-covariances
    C_t = Cov(x_t, x_{t-1} | y) = P_t G_{t-1}^T (t >= 1)."""
    m = sv_model(*theta)
    kf = kalman.kalman_filter(ytilde, m["m0"], m["P0"], m["F"], m["b"], m["Q"], m["R"])
    mf, Pf, Pp = kf["mf"], kf["Pf"], kf["Pp"]
    T, d = mf.shape
    F = m["F"]
    ms, Ps = kalman.rts_smoother(kf, F)
    Cs = np.zeros((T, d, d))
    for t in range(1, T):
        G = np.linalg.solve(Pp[t], F @ Pf[t - 1]).T
        Cs[t] = Ps[t] @ G.T
    return kf, ms, Ps, Cs, m


def loglik_grad(theta, ytilde):
    """Fisher's identity gradient of log Z (conventions in the module docstring)."""
    mu, phi, L, delta = (np.array(v, dtype=np.float64) for v in theta)
    L = np.tril(L)
    kf, ms, Ps, Cs, m = smoother_moments((mu, phi, L, delta), ytilde)
    T, d = ms.shape
    Phi = np.diag(phi)
    Q, P0 = m["Q"], m["P0"]
    Qi, P0i = np.linalg.inv(Q), np.linalg.inv(P0)
    a = ms - mu
    ebar = a[1:] - a[:-1] * phi
    M = np.zeros((d, d))
    D = np.zeros((d, d))
    for t in range(1, T):
        e = ebar[t - 1]
        M += np.outer(e, e) + Ps[t] - Cs[t] @ Phi - Phi @ Cs[t].T + Phi @ Ps[t - 1] @ Phi
        D += np.outer(e, a[t - 1]) + Cs[t] - Phi @ Ps[t - 1]
    S0 = Ps[0] + np.outer(a[0], a[0])
    Gam = 0.5 * (P0i @ S0 @ P0i - P0i)
    W = 1.0 - np.outer(phi, phi)
    g_mu = (1.0 - phi) * (Qi @ ebar.sum(axis=0)) + P0i @ a[0]
    g_phi = np.diag(Qi @ D) + 2.0 * np.sum(Gam * Q * phi[None, :] / W ** 2, axis=1)
    GQ = -0.5 * (T - 1) * Qi + 0.5 * Qi @ M @ Qi + Gam / W
    g_L = np.tril(2.0 * GQ @ L)
    O = np.sum((ytilde - ms) ** 2) + np.einsum("tii->", Ps)
    g_delta = -T * d / (2.0 * delta) + O / delta ** 2
    return g_mu, g_phi, g_L, float(g_delta), kf["logZ"]


# ---------------------------------------------------------------------------
# The gradient-based theta-update inside the Gibbs sweep. The paper updates its
# static parameters inside the sampler (Section 4.3) without stating a rule;
# this one is a projected gradient-ascent step on the mean over chains of the
# auxiliary marginal log-likelihood log p(ytilde_c | theta) (Fisher's identity
# above), applied to (mu, phi, L) with delta left to the sampler:
#   mu  <- mu  + lr * mean_c g_mu[c]
#   phi <- clip(phi + lr * mean_c g_phi[c], -PHI_MAX, PHI_MAX)
#   L   <- tril(L + lr * mean_c g_L[c]),  diag(L) <- max(diag(L), L_MIN)
# then the model is rebuilt from theta by sv_model (stationary p_0).
# ---------------------------------------------------------------------------
PHI_MAX = 0.999
L_MIN = 1e-6


def sv_theta_update(mu, phi, L, g_mu, g_phi, g_L, lr):
    """One theta-update from per-chain gradients g_mu [C][d], g_phi [C][d], g_L [C][d][d]."""
    mu = np.asarray(mu, dtype=np.float64) + lr * np.mean(np.asarray(g_mu, dtype=np.float64), axis=0)
    phi = np.asarray(phi, dtype=np.float64) + lr * np.mean(np.asarray(g_phi, dtype=np.float64), axis=0)
    phi = np.clip(phi, -PHI_MAX, PHI_MAX)
    L = np.tril(np.asarray(L, dtype=np.float64) + lr * np.mean(np.asarray(g_L, dtype=np.float64), axis=0))
    idx = np.arange(len(mu))
    L[idx, idx] = np.maximum(L[idx, idx], L_MIN)
    return mu, phi, L

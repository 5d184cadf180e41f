"""Brute-force dense Gaussian computations over the whole path (tiny T·d only).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.

Section 2.1, Eq. (2.2): with a Gaussian prior N(x; mbar, C) over the stacked
path and a linearised potential, the auxiliary proposal is Gaussian with
covariance A = (C^{-1} + (2/delta) I)^{-1} and mean mbar + (2/delta) A (ytilde - mbar),
ytilde = u + (delta/2) grad f(x) (the zero-mean form of Eq. (2.2) after the
change of variables of its footnote). Section 2.2 states that this proposal
is the pathwise smoothing distribution of the auxiliary LGSSM; these
functions compute it with dense (T·d)-dimensional algebra so that the
sequential and parallel samplers can be checked against it.
"""
import numpy as np


def _at(arr, t, ndim):
    arr = np.asarray(arr, dtype=np.float64)
    return arr if arr.ndim == ndim else arr[t]


def prior_moments(m0, P0, F, b, Q, T):
    """Mean [T*d] and covariance [T*d, T*d] of x_{0:T-1} under the Gaussian dynamics.

    Written as x = Phi e + c with e = (x_0 - m0, w_1, ..., w_{T-1}) independent.
    """
    m0 = np.asarray(m0, dtype=np.float64)
    d = len(m0)
    mean = np.zeros((T, d))
    mean[0] = m0
    # Phi[t, s] = F_{t-1} ... F_s (d x d) maps innovation s to state t
    Phi = np.zeros((T, T, d, d))
    for t in range(T):
        Phi[t, t] = np.eye(d)
        if t > 0:
            Ft = _at(F, t - 1, 2)
            mean[t] = Ft @ mean[t - 1] + _at(b, t - 1, 1)
            for s in range(t):
                Phi[t, s] = Ft @ Phi[t - 1, s]
    covs = [np.asarray(P0, dtype=np.float64)] + [_at(Q, t - 1, 2) for t in range(1, T)]
    C = np.zeros((T * d, T * d))
    for t in range(T):
        for r in range(T):
            acc = np.zeros((d, d))
            for s in range(min(t, r) + 1):
                acc += Phi[t, s] @ covs[s] @ Phi[r, s].T
            C[t * d:(t + 1) * d, r * d:(r + 1) * d] = acc
    return mean.reshape(-1), C


def lgssm_posterior(ytilde, delta, mbar, C):
    """Posterior of the stacked path given ytilde ~ N(x, (delta/2) I).

    Returns (mean, cov, logZ) with logZ = log N(ytilde; mbar, C + (delta/2) I).
    """
    y = np.asarray(ytilde, dtype=np.float64).reshape(-1)
    n = len(y)
    r = 0.5 * delta
    A = np.linalg.inv(np.linalg.inv(C) + np.eye(n) / r)
    mean = mbar + A @ (y - mbar) / r
    S = C + r * np.eye(n)
    sign, logdet = np.linalg.slogdet(S)
    z = np.linalg.solve(S, y - mbar)
    logZ = -0.5 * (n * np.log(2 * np.pi) + logdet + (y - mbar) @ z)
    return mean, A, logZ


def titsias_proposal(u, grad, delta, mbar, C):
    """Eq. (2.2) with the prior mean shifted to mbar: mean and covariance A."""
    u = np.asarray(u, dtype=np.float64).reshape(-1)
    g = np.asarray(grad, dtype=np.float64).reshape(-1)
    n = len(u)
    A = np.linalg.inv(np.linalg.inv(C) + (2.0 / delta) * np.eye(n))
    mean = mbar + (2.0 / delta) * A @ (u + 0.5 * delta * g - mbar)
    return mean, A

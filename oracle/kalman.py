"""FP64 reference of the linear-Gaussian state-space machinery the sampler uses.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product path never does. Plain, slow, sequential numpy code:
one Python loop over time, library solves/Cholesky as single steps.

Model (Appendix A, Eq. (A.1) with H_t = I and c_t = 0, as in the auxiliary
LGSSM of Section 2.2, Eq. (2.7)):

    x_0 ~ N(m0, P0),  x_t = F_{t-1} x_{t-1} + b_{t-1} + N(0, Q_{t-1}),
    y_t = x_t + N(0, R),           t = 0 .. T-1  (T = number of states).

F, b, Q may be a single (homogeneous) value or a stack over t = 0 .. T-2
(index t-1 is the transition into x_t). R may be a single [d,d] matrix or a
stack over t.

Functions and the passages they follow:
  kalman_filter      the Kalman filter algorithm (Appendix A.1, Eqs. (A.3)-(A.6)), with the
                     predictive likelihood terms N(y_t; m^p_t, P^p_t + R).
  rts_sample         the Rauch-Tung-Striebel sampler algorithm (Appendix A.1, Eq. (A.10)).
  rts_smoother       marginal smoother means/covariances (same recursion,
                     Appendix A.1), used for stationarity checks.
  filter_elements,   the per-step conditional-Gaussian elements and their
  filter_combine     associative operator of the parallel Kalman filter
                     (Appendix A.2.1, Eqs. (A.12)-(A.13); element formulas of
                     the cited Sarkka & Garcia-Fernandez construction).
                     parity unpinned by a printed value: pinned by equality
                     with kalman_filter under sequential and Hillis-Steele
                     scans.
  sequential_scan,   prefix scans over any associative operator; the second
  hillis_steele_scan is the Hillis-Steele algorithm of Appendix A.2.1.
  backward_elements, (G_t, U_t) elements and operator of the parallel RTS
  backward_combine,  sampler, Eqs. (A.14)-(A.15), Proposition A.1 and the
  suffix_scan        parallel RTS sampler algorithm (Appendix A.2.2).
"""
import numpy as np

LOG2PI = np.log(2.0 * np.pi)


def _at(arr, t, ndim):
    """Select time t from a homogeneous (ndim) or stacked (ndim+1) array."""
    arr = np.asarray(arr, dtype=np.float64)
    return arr if arr.ndim == ndim else arr[t]


def mvn_logpdf(x, mean, cov):
    """log N(x; mean, cov) via a Cholesky factor."""
    d = len(mean)
    L = np.linalg.cholesky(cov)
    z = np.linalg.solve(L, x - mean)
    return -0.5 * (d * LOG2PI + 2.0 * np.sum(np.log(np.diag(L))) + z @ z)


def kalman_filter(y, m0, P0, F, b, Q, R):
    """The Kalman filter algorithm of Appendix A.1 with H = I.

    Returns a dict with mf, Pf (filtered), mp, Pp (predicted; mp[0]=m0,
    Pp[0]=P0), ell (per-step predictive log-likelihood terms) and logZ.
    """
    y = np.asarray(y, dtype=np.float64)
    T, d = y.shape
    mf = np.zeros((T, d)); Pf = np.zeros((T, d, d))
    mp = np.zeros((T, d)); Pp = np.zeros((T, d, d))
    ell = np.zeros(T)
    m_pred = np.asarray(m0, dtype=np.float64).copy()
    P_pred = np.asarray(P0, dtype=np.float64).copy()
    for t in range(T):
        if t > 0:
            Ft = _at(F, t - 1, 2); bt = _at(b, t - 1, 1); Qt = _at(Q, t - 1, 2)
            m_pred = Ft @ mf[t - 1] + bt
            P_pred = Ft @ Pf[t - 1] @ Ft.T + Qt
        Rt = _at(R, t, 2)
        S = P_pred + Rt
        K = np.linalg.solve(S, P_pred).T          # P_pred S^{-1} (both symmetric)
        mp[t] = m_pred; Pp[t] = P_pred
        ell[t] = mvn_logpdf(y[t], m_pred, S)
        mf[t] = m_pred + K @ (y[t] - m_pred)
        P_f = P_pred - K @ P_pred
        Pf[t] = 0.5 * (P_f + P_f.T)
    return dict(mf=mf, Pf=Pf, mp=mp, Pp=Pp, ell=ell, logZ=float(np.sum(ell)))


def rts_sample(kf, F, b, Q, eps):
    """The RTS sampler algorithm of Appendix A.1 driven by given standard normals eps [T, d].

    x_{T-1} = m^f + chol(P^f) eps_{T-1}; for t < T-1
    x_t = m^f_t + G_t (x_{t+1} - m^p_{t+1}) + chol(P^f_t - G_t P^p_{t+1} G_t^T) eps_t,
    G_t = P^f_t F_t^T (P^p_{t+1})^{-1}. chol is the lower Cholesky factor.
    """
    mf, Pf, mp, Pp = kf["mf"], kf["Pf"], kf["mp"], kf["Pp"]
    T, d = mf.shape
    x = np.zeros((T, d))
    x[T - 1] = mf[T - 1] + np.linalg.cholesky(Pf[T - 1]) @ eps[T - 1]
    for t in range(T - 2, -1, -1):
        Ft = _at(F, t, 2)
        G = np.linalg.solve(Pp[t + 1], Ft @ Pf[t]).T
        mean = mf[t] + G @ (x[t + 1] - mp[t + 1])
        cov = Pf[t] - G @ Pp[t + 1] @ G.T
        cov = 0.5 * (cov + cov.T)
        x[t] = mean + np.linalg.cholesky(cov) @ eps[t]
    return x


def rts_smoother(kf, F):
    """Marginal smoothing means/covariances (RTS smoother)."""
    mf, Pf, mp, Pp = kf["mf"], kf["Pf"], kf["mp"], kf["Pp"]
    T, d = mf.shape
    ms = mf.copy(); Ps = Pf.copy()
    for t in range(T - 2, -1, -1):
        Ft = _at(F, t, 2)
        G = np.linalg.solve(Pp[t + 1], Ft @ Pf[t]).T
        ms[t] = mf[t] + G @ (ms[t + 1] - mp[t + 1])
        Ps[t] = Pf[t] + G @ (Ps[t + 1] - Pp[t + 1]) @ G.T
    return ms, Ps


# ---------------------------------------------------------------------------
# Parallel filter: elements a_t = (A, b, C, eta, J) and their operator.
# Element t represents p(x_t | y_t, x_{t-1}) = N(A x_{t-1} + b, C) together with
# the likelihood p(y_t | x_{t-1}) up to a constant, N_I(x_{t-1}; eta, J).
# ---------------------------------------------------------------------------

def filter_elements(y, m0, P0, F, b, Q, R):
    """Per-step elements of the parallel Kalman filter (H = I)."""
    y = np.asarray(y, dtype=np.float64)
    T, d = y.shape
    I = np.eye(d)
    elems = []
    # t = 0: conditions the prior on y_0; a marginal (A = 0, eta = 0, J = 0).
    R0 = _at(R, 0, 2)
    S0 = P0 + R0
    K0 = np.linalg.solve(S0, P0).T
    A = np.zeros((d, d))
    bb = m0 + K0 @ (y[0] - m0)
    C = P0 - K0 @ S0 @ K0.T
    elems.append((A, bb, 0.5 * (C + C.T), np.zeros(d), np.zeros((d, d))))
    for t in range(1, T):
        Ft = _at(F, t - 1, 2); bt = _at(b, t - 1, 1); Qt = _at(Q, t - 1, 2)
        Rt = _at(R, t, 2)
        S = Qt + Rt
        K = np.linalg.solve(S, Qt).T               # Q S^{-1}
        A = (I - K) @ Ft
        bb = bt + K @ (y[t] - bt)
        C = (I - K) @ Qt
        Sinv_F = np.linalg.solve(S, Ft)
        eta = Sinv_F.T @ (y[t] - bt)
        J = Ft.T @ Sinv_F
        elems.append((A, bb, 0.5 * (C + C.T), eta, 0.5 * (J + J.T)))
    return elems


def filter_combine(ei, ej):
    """a_i (x) a_j for i earlier than j, through an LU solve with M = I + C_i J_j."""
    Ai, bi, Ci, ei_, Ji = ei
    Aj, bj, Cj, ej_, Jj = ej
    d = len(bi)
    I = np.eye(d)
    M = I + Ci @ Jj
    Minv_Ai = np.linalg.solve(M, Ai)
    Minv_rhs = np.linalg.solve(M, bi + Ci @ ej_)
    Minv_Ci = np.linalg.solve(M, Ci)
    Mt = M.T                                       # = I + J_j C_i
    A = Aj @ Minv_Ai
    bb = Aj @ Minv_rhs + bj
    C = Aj @ Minv_Ci @ Aj.T + Cj
    eta = Ai.T @ np.linalg.solve(Mt, ej_ - Jj @ bi) + ei_
    J = Ai.T @ np.linalg.solve(Mt, Jj) @ Ai + Ji
    return (A, bb, 0.5 * (C + C.T), eta, 0.5 * (J + J.T))


def sequential_scan(elems, op):
    """Inclusive prefix scan, left to right: out_t = e_0 op ... op e_t."""
    out = [elems[0]]
    for e in elems[1:]:
        out.append(op(out[-1], e))
    return out


def hillis_steele_scan(elems, op):
    """Hillis-Steele algorithm (Appendix A.2.1): log2 T rounds of out_t <- out_{t-2^k} op out_t."""
    out = list(elems)
    T = len(out)
    k = 1
    while k < T:
        out = [out[t] if t < k else op(out[t - k], out[t]) for t in range(T)]
        k *= 2
    return out


# ---------------------------------------------------------------------------
# Parallel RTS sampler (Appendix A.2.2).
# ---------------------------------------------------------------------------

def backward_elements(kf, F, b, Q, eps):
    """(G_t, U_t) of Eq. (A.14): U_t = m^f_t - G_t (F_t m^f_t + b_t) + chol(Sigma_t) eps_t,
    Sigma_t = P^f_t - G_t (F_t P^f_t F_t^T + Q_t) G_t^T; G_{T-1} = 0 and
    U_{T-1} = m^f_{T-1} + chol(P^f_{T-1}) eps_{T-1}."""
    mf, Pf = kf["mf"], kf["Pf"]
    T, d = mf.shape
    out = []
    for t in range(T - 1):
        Ft = _at(F, t, 2); bt = _at(b, t, 1); Qt = _at(Q, t, 2)
        Ppn = Ft @ Pf[t] @ Ft.T + Qt
        G = np.linalg.solve(Ppn, Ft @ Pf[t]).T
        Sig = Pf[t] - G @ Ppn @ G.T
        Sig = 0.5 * (Sig + Sig.T)
        U = mf[t] - G @ (Ft @ mf[t] + bt) + np.linalg.cholesky(Sig) @ eps[t]
        out.append((G, U))
    out.append((np.zeros((d, d)),
                mf[T - 1] + np.linalg.cholesky(Pf[T - 1]) @ eps[T - 1]))
    return out


def backward_combine(ei, ej):
    """(G_i, U_i) o (G_j, U_j) = (G_i G_j, G_i U_j + U_i), Eq. (A.12)."""
    Gi, Ui = ei
    Gj, Uj = ej
    return (Gi @ Gj, Gi @ Uj + Ui)


def suffix_scan(elems, op):
    """Backward (suffix) scan: out_t = e_t o e_{t+1} o ... o e_{T-1}."""
    out = [None] * len(elems)
    out[-1] = elems[-1]
    for t in range(len(elems) - 2, -1, -1):
        out[t] = op(elems[t], out[t + 1])
    return out

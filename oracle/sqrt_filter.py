"""FP64 reference of the square-root form of the parallel Kalman filter.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product path never does.

Section 4.1 reports that the parallel filter diverged in single precision
on the stochastic-volatility model and points to the square-root version of
the parallel filter (cited there, not printed): every covariance-like block
of an element is carried as a factor, C = U U^T and J = Z Z^T, and new factors
come from an orthogonal triangularisation instead of from sums and
differences of covariances. The formulas below are this module's derivation
(readings, not printed by the paper): the standard elements and operator of
Appendix A.2.1 (oracle/kalman.py: filter_elements, filter_combine) with

  tria(X)   the lower-triangular L with positive diagonal and L L^T = X X^T
            (X is d x k), from a QR factorisation of X^T;

  elements  t = 0:  tria([[chol R, chol P0], [0, chol P0]]) = [[Ls, 0], [Kb, U]],
                    K = Kb Ls^{-1}, A = 0, b = m0 + K (y_0 - m0), eta = 0, Z = 0;
            t >= 1: the same with Q in place of P0: K = Q S^{-1}, A = (I - K) F,
                    b = b_t + K (y_t - b_t), Z = F^T Ls^{-T}, eta = Z Ls^{-1} (y_t - b_t);

  operator  (i earlier, j later) W = U_i^T Z_j, Xi = tria([W, I]), Xi' = tria([W^T, I]),
            M^{-1} = I - U_i Xi^{-T} Xi^{-1} W Z_j^T,
            M^{-T} = I - Z_j Xi'^{-T} Xi'^{-1} W^T U_i^T,
            A = A_j M^{-1} A_i,   b = A_j M^{-1} (b_i + U_i U_i^T eta_j) + b_j,
            U = tria([A_j U_i Xi^{-T}, U_j]),
            eta = A_i^T M^{-T} (eta_j - Z_j Z_j^T b_i) + eta_i,
            Z = tria([A_i^T Z_j Xi'^{-T}, Z_i]),
            which are the standard operator's A, b, eta and factors of its C and J
            (push-through identities with M = I + C_i J_j);

  filter    the inclusive prefix at t has A = 0, b = m^f_t and U = chol(P^f_t);
            the predictive factor Ls_t = tria([F U_{t-1}, chol Q, chol R])
            (tria([chol P0, chol R]) at t = 0) gives
            l_t = log N(y_t; m^p_t, Ls_t Ls_t^T).

parity pins (tests/test_oracle_sqrt_filter.py): tria against its defining
identity; each square-root element and combine against the covariance-form
element and operator of oracle/kalman.py; the filter's m^f, P^f and log Z
against kalman_filter (sequential and Hillis-Steele schedules).
"""
import numpy as np

from . import kalman

LOG2PI = float(np.log(2.0 * np.pi))


def _at(arr, t, ndim):
    arr = np.asarray(arr, dtype=np.float64)
    return arr if arr.ndim == ndim else arr[t]


def tria(X):
    """Lower-triangular L, positive diagonal, with L L^T = X X^T (X: d x k, k >= d)."""
    X = np.asarray(X, dtype=np.float64)
    d = X.shape[0]
    R = np.linalg.qr(X.T, mode="r")[:d, :d]     # X^T = Q R  =>  X X^T = R^T R
    L = R.T.copy()
    s = np.sign(np.diag(L))
    s[s == 0] = 1.0
    return L * s[None, :]


def _solve_lower(L, B):
    return np.linalg.solve(L, B)


def _split(pre, d):
    T = tria(pre)
    return T[:d, :d], T[d:, :d], T[d:, d:]       # Ls, Kb, U


def sr_elements(y, m0, P0, F, b, Q, R):
    """Square-root elements (A, b, U, eta, Z) per step (H = I)."""
    y = np.asarray(y, dtype=np.float64)
    T, d = y.shape
    I = np.eye(d)
    Z0 = np.zeros((d, d))
    elems = []
    cR = np.linalg.cholesky(_at(R, 0, 2))
    cP = np.linalg.cholesky(np.asarray(P0, dtype=np.float64))
    Ls, Kb, U = _split(np.block([[cR, cP], [Z0, cP]]), d)
    K = np.linalg.solve(Ls.T, Kb.T).T             # Kb Ls^{-1}
    elems.append((np.zeros((d, d)), m0 + K @ (y[0] - m0), U, np.zeros(d), np.zeros((d, d))))
    for t in range(1, T):
        Ft = _at(F, t - 1, 2); bt = _at(b, t - 1, 1)
        cQ = np.linalg.cholesky(_at(Q, t - 1, 2))
        cR = np.linalg.cholesky(_at(R, t, 2))
        Ls, Kb, U = _split(np.block([[cR, cQ], [Z0, cQ]]), d)
        K = np.linalg.solve(Ls.T, Kb.T).T
        A = (I - K) @ Ft
        bb = bt + K @ (y[t] - bt)
        Z = _solve_lower(Ls, Ft).T                # F^T Ls^{-T}
        eta = Z @ _solve_lower(Ls, y[t] - bt)
        elems.append((A, bb, U, eta, Z))
    return elems


def sr_combine(ei, ej):
    """Square-root form of a_i (x) a_j, i earlier than j."""
    Ai, bi, Ui, ei_, Zi = ei
    Aj, bj, Uj, ej_, Zj = ej
    d = len(bi)
    I = np.eye(d)
    W = Ui.T @ Zj
    Xi = tria(np.hstack([W, I]))
    Xp = tria(np.hstack([W.T, I]))
    Ninv_WZt = np.linalg.solve(Xi.T, _solve_lower(Xi, W @ Zj.T))          # N^{-1} W Z_j^T
    Minv = I - Ui @ Ninv_WZt
    Npinv_WtUt = np.linalg.solve(Xp.T, _solve_lower(Xp, W.T @ Ui.T))      # N'^{-1} W^T U_i^T
    MinvT = I - Zj @ Npinv_WtUt
    A = Aj @ Minv @ Ai
    bb = Aj @ Minv @ (bi + Ui @ (Ui.T @ ej_)) + bj
    U = tria(np.hstack([Aj @ _solve_lower(Xi, Ui.T).T, Uj]))               # A_j U_i Xi^{-T}
    eta = Ai.T @ MinvT @ (ej_ - Zj @ (Zj.T @ bi)) + ei_
    Z = tria(np.hstack([Ai.T @ _solve_lower(Xp, Zj.T).T, Zi]))             # A_i^T Z_j Xi'^{-T}
    return (A, bb, U, eta, Z)


def sr_filter(y, m0, P0, F, b, Q, R, schedule="sequential"):
    """Filtering means, factors of the filtering covariances and log Z.

    Returns dict(mf [T, d], Uf [T, d, d] (lower, U U^T = P^f), ell [T], logZ)."""
    y = np.asarray(y, dtype=np.float64)
    T, d = y.shape
    elems = sr_elements(y, m0, P0, F, b, Q, R)
    scan = kalman.sequential_scan if schedule == "sequential" else kalman.hillis_steele_scan
    pref = scan(elems, sr_combine)
    mf = np.stack([e[1] for e in pref])
    Uf = np.stack([e[2] for e in pref])
    ell = np.zeros(T)
    for t in range(T):
        cR = np.linalg.cholesky(_at(R, t, 2))
        if t == 0:
            mp = np.asarray(m0, dtype=np.float64)
            Ls = tria(np.hstack([np.linalg.cholesky(np.asarray(P0, dtype=np.float64)), cR]))
        else:
            Ft = _at(F, t - 1, 2)
            mp = Ft @ mf[t - 1] + _at(b, t - 1, 1)
            Ls = tria(np.hstack([Ft @ Uf[t - 1], np.linalg.cholesky(_at(Q, t - 1, 2)), cR]))
        z = _solve_lower(Ls, y[t] - mp)
        ell[t] = -0.5 * (d * LOG2PI + 2.0 * np.sum(np.log(np.diag(Ls))) + z @ z)
    return dict(mf=mf, Uf=Uf, ell=ell, logZ=float(np.sum(ell)))

"""FP64 reference of one step of the first-order auxiliary Kalman sampler.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package; the product path never does.

Target (Section 2.2, Eq. (2.5) and the augmented target Eq. (2.6)):

    pi(x, u) ∝ N(x_0; m0, P0) prod_t N(x_t; F x_{t-1} + b, Q) exp(gamma(x))
               prod_t N(u_t; x_t, (delta/2) I),     gamma(x) = sum_t log h(y_t | x_t).

One step (Algorithm 2 with Gaussian dynamics, so F, b, Q are the model's):
  1. u_t = x_t + sqrt(delta/2) eps_t                 (first line of Alg. 2)
  2. v_t = grad_{x_t} gamma(x);  ytilde_t = u_t + (delta/2) v_t   (Eq. (2.7))
  3. x* ~ q(. | u, x): Kalman filter (Appendix A.1) on ytilde with R = (delta/2) I,
     then the RTS sampler (Appendix A.1) with the backward noise.
  4. v*, ytilde* from x*; the Kalman filter on ytilde* gives log p(ytilde*).
  5. log alpha = log pi(x*, u) + log q(x | u, x*) - log pi(x, u) - log q(x* | u, x)
     (the MRTH line of Alg. 2), with the smoothing density of each proposal
     written as joint over marginal (Eq. (A.7)):
         log q(z | u, x) = log p(z) + sum_t log N(ytilde_t; z_t, R) - log p(ytilde).
     This is the direct formula on full joint densities; the CUDA library
     uses an algebraically simplified form, so agreement between the two is
     a check of that simplification.
  6. accept iff log U < log alpha.

Emission models (gamma and its gradient):
  linear-Gaussian  log h(y|x) = log N(y; x, R_y)           (Appendix A, Eq. (A.1))
  stochastic vol.  log h(y|x) = sum_i log N(y_i; 0, exp(x_i))  (Section 4.1)
  Student-t        log h(y|x) = log t_nu(y; x, Sigma)      (Section 4.2)
An optional observation mask switches gamma_t off (gamma_t = 0, v_t = 0) at
unobserved steps, as in the two-step model of Section 4.4.

aux_step_second_order is the same step with the second-order proposal of
Section 2.2, Eqs. (2.8)-(2.9) (the Hessian of gamma_t enters the
pseudo-observation covariance).
"""
import numpy as np

from . import bridging
from . import kalman
from . import philox

LOG2PI = np.log(2.0 * np.pi)


class LinearGaussianEmission:
    """log h(y_t | x_t) = log N(y_t; x_t, R_y)."""

    def __init__(self, y, Ry, mask=None):
        self.y = np.asarray(y, dtype=np.float64)
        self.Ry = np.asarray(Ry, dtype=np.float64)
        self.mask = np.ones(len(self.y), bool) if mask is None else np.asarray(mask, bool)
        self.Ry_inv = np.linalg.inv(self.Ry)
        d = self.Ry.shape[0]
        self._const = -0.5 * (d * LOG2PI + np.linalg.slogdet(self.Ry)[1])

    def log_h(self, x):
        r = self.y - x
        q = np.einsum("ti,ij,tj->t", r, self.Ry_inv, r)
        return np.where(self.mask, self._const - 0.5 * q, 0.0)

    def grad(self, x):
        g = (self.y - x) @ self.Ry_inv.T
        return g * self.mask[:, None]

    def hess(self, x):
        """Hessian of log h(y_t | x_t) in x_t, [T, d, d]: -R_y^{-1} (0 where masked)."""
        T = len(x)
        return -self.Ry_inv[None, :, :] * self.mask[:, None, None] * np.ones((T, 1, 1))


class SVEmission:
    """log h(y_t | x_t) = sum_i log N(y_t(i); 0, exp(x_t(i)))."""

    def __init__(self, y, mask=None):
        self.y = np.asarray(y, dtype=np.float64)
        self.mask = np.ones(len(self.y), bool) if mask is None else np.asarray(mask, bool)

    def log_h(self, x):
        lh = -0.5 * LOG2PI - 0.5 * x - 0.5 * self.y ** 2 * np.exp(-x)
        return np.where(self.mask, lh.sum(axis=1), 0.0)

    def grad(self, x):
        g = -0.5 + 0.5 * self.y ** 2 * np.exp(-x)
        return g * self.mask[:, None]

    def hess(self, x):
        """Hessian of log h(y_t | x_t) in x_t, [T, d, d]: diag(-y^2 exp(-x) / 2)."""
        h = -0.5 * self.y ** 2 * np.exp(-x) * self.mask[:, None]
        return np.einsum("ti,ij->tij", h, np.eye(x.shape[1]))


class StudentTEmission:
    """log h(y_t | x_t) = log t_nu(y_t; x_t, Sigma): the multivariate t with nu
    degrees of freedom, location x_t and scale matrix Sigma (the observation
    model of Section 4.2; it does not factorise over the coordinates)."""

    def __init__(self, y, Sigma, nu, mask=None):
        from math import lgamma
        self.y = np.asarray(y, dtype=np.float64)
        self.nu = float(nu)
        self.mask = np.ones(len(self.y), bool) if mask is None else np.asarray(mask, bool)
        self.Lam = np.linalg.inv(np.asarray(Sigma, dtype=np.float64))
        d = self.y.shape[1]
        self.d = d
        self._const = (lgamma(0.5 * (self.nu + d)) - lgamma(0.5 * self.nu) - 0.5 * d * np.log(self.nu * np.pi)
                       - 0.5 * np.linalg.slogdet(np.asarray(Sigma, dtype=np.float64))[1])

    def _q(self, x):
        r = self.y - x
        return r, np.einsum("ti,ij,tj->t", r, self.Lam, r)

    def log_h(self, x):
        _, q = self._q(x)
        return np.where(self.mask, self._const - 0.5 * (self.nu + self.d) * np.log1p(q / self.nu), 0.0)

    def grad(self, x):
        r, q = self._q(x)
        g = ((self.nu + self.d) / (self.nu + q))[:, None] * (r @ self.Lam.T)
        return g * self.mask[:, None]


def log_prior(x, m0, P0, F, b, Q):
    """log N(x_0; m0, P0) + sum_{t>=1} log N(x_t; F x_{t-1} + b, Q)."""
    lp = kalman.mvn_logpdf(x[0], m0, P0)
    for t in range(1, len(x)):
        Ft = kalman._at(F, t - 1, 2); bt = kalman._at(b, t - 1, 1); Qt = kalman._at(Q, t - 1, 2)
        lp += kalman.mvn_logpdf(x[t], Ft @ x[t - 1] + bt, Qt)
    return lp


def _log_obs(z, obs, R):
    return sum(kalman.mvn_logpdf(obs[t], z[t], R) for t in range(len(z)))


def _draw(kf, F, b, Q, eps, sampler):
    """A path from the smoothing law: the RTS sampler (Appendix A.1) or the
    divide-and-conquer sampler (Appendix A.2.3); both exact, so the MH ratio
    below is the same for either."""
    if sampler == "rts":
        return kalman.rts_sample(kf, F, b, Q, eps)
    if sampler == "bridging":
        return bridging.dnc_sample(kf, F, b, Q, eps)
    raise ValueError(sampler)


def aux_step(x, model, delta, eps_aux, eps_back, log_u, sampler="rts"):
    """One auxiliary Kalman MH step from state x [T, d].

    model: dict with m0, P0, F, b, Q and 'emission' (an emission object).
    eps_aux, eps_back: standard normals [T, d]; log_u: log of the MH uniform.
    Returns dict(x_new, x_star, log_alpha, accepted, logZ, logZ_star, u, v, v_star).
    """
    m0, P0, F, b, Q = model["m0"], model["P0"], model["F"], model["b"], model["Q"]
    em = model["emission"]
    T, d = x.shape
    R = 0.5 * delta * np.eye(d)
    u = x + np.sqrt(0.5 * delta) * eps_aux
    v = em.grad(x)
    yt = u + 0.5 * delta * v
    kf = kalman.kalman_filter(yt, m0, P0, F, b, Q, R)
    x_star = _draw(kf, F, b, Q, eps_back, sampler)
    v_star = em.grad(x_star)
    yt_star = u + 0.5 * delta * v_star
    kf_star = kalman.kalman_filter(yt_star, m0, P0, F, b, Q, R)

    def log_pi(z):
        return log_prior(z, m0, P0, F, b, Q) + em.log_h(z).sum() + _log_obs(z, u, R)

    def log_q(z, obs, logZ):
        return log_prior(z, m0, P0, F, b, Q) + _log_obs(z, obs, R) - logZ

    log_alpha = (log_pi(x_star) + log_q(x, yt_star, kf_star["logZ"])
                 - log_pi(x) - log_q(x_star, yt, kf["logZ"]))
    accepted = bool(log_u < log_alpha)
    return dict(x_new=x_star if accepted else x.copy(), x_star=x_star,
                log_alpha=float(log_alpha), accepted=accepted,
                logZ=kf["logZ"], logZ_star=kf_star["logZ"], u=u, v=v, v_star=v_star,
                ytilde=yt, ytilde_star=yt_star, kf=kf)


def second_order_obs(x, u, model, delta):
    """Pseudo-observations of the second-order proposal (Section 2.2, the
    expansion Eq. (2.8) and the proposal Eq. (2.9)), Sigma_t = I:
        Lambda_t = Hessian of gamma_t at x_t,
        Omega_t  = ((2/delta) I - Lambda_t)^{-1},
        omega_t  = Omega_t ((2/delta) u_t + v_t - Lambda_t x_t).
    Returns (omega [T, d], Omega [T, d, d])."""
    em = model["emission"]
    T, d = x.shape
    v = em.grad(x)
    Lam = em.hess(x)
    Om = np.zeros((T, d, d))
    om = np.zeros((T, d))
    for t in range(T):
        Om[t] = np.linalg.inv((2.0 / delta) * np.eye(d) - Lam[t])
        om[t] = Om[t] @ ((2.0 / delta) * u[t] + v[t] - Lam[t] @ x[t])
    return om, Om


def aux_step_second_order(x, model, delta, eps_aux, eps_back, log_u, sampler="rts"):
    """One auxiliary Kalman MH step with the second-order proposal.

    Same augmented target as aux_step; the proposal is the smoothing law of the
    LGSSM with the model's dynamics and observations omega_t ~ N(z_t, Omega_t)
    (second_order_obs), sampled by the Kalman filter and RTS sampler of
    Appendix A.1 with a time-varying observation covariance. log alpha is the
    direct formula on full joint densities, as in aux_step.
    """
    m0, P0, F, b, Q = model["m0"], model["P0"], model["F"], model["b"], model["Q"]
    em = model["emission"]
    T, d = x.shape
    R = 0.5 * delta * np.eye(d)
    u = x + np.sqrt(0.5 * delta) * eps_aux
    om, Om = second_order_obs(x, u, model, delta)
    kf = kalman.kalman_filter(om, m0, P0, F, b, Q, Om)
    x_star = _draw(kf, F, b, Q, eps_back, sampler)
    om_s, Om_s = second_order_obs(x_star, u, model, delta)
    kf_star = kalman.kalman_filter(om_s, m0, P0, F, b, Q, Om_s)

    def log_pi(z):
        return log_prior(z, m0, P0, F, b, Q) + em.log_h(z).sum() + _log_obs(z, u, R)

    def log_q(z, obs, covs, logZ):
        return (log_prior(z, m0, P0, F, b, Q)
                + sum(kalman.mvn_logpdf(obs[t], z[t], covs[t]) for t in range(len(z))) - logZ)

    log_alpha = (log_pi(x_star) + log_q(x, om_s, Om_s, kf_star["logZ"])
                 - log_pi(x) - log_q(x_star, om, Om, kf["logZ"]))
    accepted = bool(log_u < log_alpha)
    return dict(x_new=x_star if accepted else x.copy(), x_star=x_star,
                log_alpha=float(log_alpha), accepted=accepted,
                logZ=kf["logZ"], logZ_star=kf_star["logZ"], u=u,
                omega=om, Omega=Om, omega_star=om_s, Omega_star=Om_s, kf=kf)


def aux_step_philox(x, model, delta, seed, chain, iteration, order=1, sampler="rts"):
    """aux_step with the library's Philox streams for (seed, chain, iteration)."""
    T, d = x.shape
    eps_aux = philox.path_normals(seed, chain, iteration, philox.PURPOSE_AUX, T, d)
    eps_back = philox.path_normals(seed, chain, iteration, philox.PURPOSE_BACKWARD, T, d)
    log_u = float(np.log(philox.mh_uniform(seed, chain, iteration)))
    step = aux_step if order == 1 else aux_step_second_order
    return step(x, model, delta, eps_aux, eps_back, log_u, sampler=sampler)


def run_chain(x0, model, delta, seed, chain, n_iters, iter0=0, keep=None, order=1, sampler="rts"):
    """Run n_iters steps; returns (x_final, n_accepted, kept states or None)."""
    x = np.array(x0, dtype=np.float64)
    n_acc = 0
    kept = [] if keep is not None else None
    for k in range(n_iters):
        st = aux_step_philox(x, model, delta, seed, chain, iter0 + k, order=order, sampler=sampler)
        x = st["x_new"]
        n_acc += st["accepted"]
        if keep is not None:
            kept.append(keep(x))
    return x, n_acc, kept

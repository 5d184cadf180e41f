"""Seeded synthetic workloads: the models and simulated data the sampler runs on.

This module holds model definitions and data simulation only — none of the
sampler's arithmetic — so that the CUDA library's tests, the benchmark and
the CPU oracle can all draw the same inputs from it.

Models (all with Gaussian dynamics x_t = F x_{t-1} + b + N(0, Q), x_0 ~ N(m0, P0)):

* ``linear_gaussian``: F = 0.9 I, Q = 0.1 I, P0 = I, y_t = x_t + N(0, 0.5 I),
  delta = 0.1; d = 2, T = 64, one chain by default. The emission is the
  linear-Gaussian observation model of Appendix A (Eq. (A.1)).
* ``stochastic_volatility``: the multivariate SV model of Section 4.1 with the
  parameter laws used here: mu = 0, Phi = diag(phi), phi_i ~ U[0.8, 0.99] iid,
  Sigma_ij = 0.5 + 0.5 [i = j] (equicorrelation 0.5, unit variances), p_0 the
  stationary law (P0_ij = Sigma_ij / (1 - phi_i phi_j), closed form since Phi
  is diagonal), y_t(i) = exp(x_t(i) / 2) eta_t(i), eta ~ N(0, 1). The paper's
  SV datasets are simulated from the model itself; this simulation stands in
  for them.
* ``spatio_temporal``: the lattice model of Section 4.2: independent random
  walks X_t(i, j) = X_{t-1}(i, j) + N(0, sigma_X^2) on a side x side lattice
  (d = side^2), observed through a multivariate t with nu degrees of freedom
  whose precision matrix has entries tau^D for lattice distance D <= r_y and 0
  beyond (D = |i - i'| + |j - j'|); sigma_X = 1, nu = 1, tau = -1/4, r_y = 1,
  T = 1024, d = 64 as in that section. The law of X_0 is not stated; here
  X_0 ~ N(0, sigma_X^2 I). The chains start at the simulated latent path.
* ``two_step_toy``: the two-step failure-mode model of Section 4.4:
  x_0 ~ N(0, 1), x_1 ~ N(rho x_0, 1 - rho^2), one observation y = 5 of x_1
  with variance r^2 (the emission at t = 0 is masked out).

All randomness comes from numpy's PCG64 generator seeded explicitly; the
sampler's own draws come from the Philox streams keyed by ``mcmc_seed``.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

EMIS_LINEAR_GAUSSIAN = 0
EMIS_SV = 1
EMIS_STUDENT_T = 2


@dataclass
class Workload:
    name: str
    d: int
    T: int
    n_chains: int
    m0: np.ndarray
    P0: np.ndarray
    F: np.ndarray
    b: np.ndarray
    Q: np.ndarray
    y: np.ndarray                 # [T, d]
    emission: int                 # EMIS_LINEAR_GAUSSIAN | EMIS_SV | EMIS_STUDENT_T
    delta: float
    x_init: np.ndarray            # [C, T, d]
    mcmc_seed: int = 1
    Ry: Optional[np.ndarray] = None     # linear-Gaussian covariance, or Student-t scale matrix
    mask: Optional[np.ndarray] = None   # [T] uint8, 1 = observed
    nu: float = 0.0                     # Student-t degrees of freedom
    meta: dict = field(default_factory=dict)

    def oracle_model(self):
        """The model as plain arrays (for the CPU oracle's emission classes)."""
        return dict(m0=self.m0, P0=self.P0, F=self.F, b=self.b, Q=self.Q,
                    y=self.y, Ry=self.Ry, mask=self.mask, emission=self.emission)


def _simulate_dynamics(rng, m0, P0, F, b, Q, T):
    d = len(m0)
    x = np.zeros((T, d))
    x[0] = m0 + np.linalg.cholesky(P0) @ rng.standard_normal(d)
    LQ = np.linalg.cholesky(Q)
    for t in range(1, T):
        x[t] = F @ x[t - 1] + b + LQ @ rng.standard_normal(d)
    return x


def linear_gaussian(d=2, T=64, n_chains=1, sim_seed=0, mcmc_seed=1, delta=0.1,
                    phi=0.9, q=0.1, r=0.5):
    """Linear-Gaussian SSM: F = phi I, Q = q I, P0 = I, y = x + N(0, r I)."""
    rng = np.random.default_rng(sim_seed)
    m0 = np.zeros(d); P0 = np.eye(d)
    F = phi * np.eye(d); b = np.zeros(d); Q = q * np.eye(d); Ry = r * np.eye(d)
    x_true = _simulate_dynamics(rng, m0, P0, F, b, Q, T)
    y = x_true + np.sqrt(r) * rng.standard_normal((T, d))
    # initial chain states: independent draws from the prior dynamics
    rng0 = np.random.default_rng(sim_seed + 7919)
    x_init = np.stack([_simulate_dynamics(rng0, m0, P0, F, b, Q, T) for _ in range(n_chains)])
    return Workload(name=f"linear_gaussian_d{d}_T{T}", d=d, T=T, n_chains=n_chains,
                    m0=m0, P0=P0, F=F, b=b, Q=Q, y=y, emission=EMIS_LINEAR_GAUSSIAN,
                    delta=delta, x_init=x_init, mcmc_seed=mcmc_seed, Ry=Ry,
                    meta=dict(x_true=x_true))


def sv_parameters(d, rng):
    phi = rng.uniform(0.8, 0.99, size=d)
    Sigma = 0.5 * np.ones((d, d)) + 0.5 * np.eye(d)
    P0 = Sigma / (1.0 - np.outer(phi, phi))
    return phi, Sigma, P0


# delta per (d, T) for the SV model, frozen once from an oracle calibration run
# (Robbins-Monro on log delta towards ~50% acceptance).
SV_DELTA = {
    (30, 1024): 0.0183,   # 400 oracle steps, acceptance 0.47 over the second half
}


def stochastic_volatility(d=30, T=1024, n_chains=32, sim_seed=0, mcmc_seed=1, delta=None):
    rng = np.random.default_rng(sim_seed)
    phi, Sigma, P0 = sv_parameters(d, rng)
    m0 = np.zeros(d); F = np.diag(phi); b = np.zeros(d); Q = Sigma
    x_true = _simulate_dynamics(rng, m0, P0, F, b, Q, T)
    y = np.exp(0.5 * x_true) * rng.standard_normal((T, d))
    if delta is None:
        delta = SV_DELTA.get((d, T), 0.05)
    # (x_true, y) is a joint draw, so x_true is an exact draw from p(x | y):
    # every chain starts at stationarity.
    x_init = np.repeat(x_true[None], n_chains, axis=0)
    return Workload(name=f"sv_d{d}_T{T}", d=d, T=T, n_chains=n_chains, m0=m0, P0=P0,
                    F=F, b=b, Q=Q, y=y, emission=EMIS_SV, delta=float(delta),
                    x_init=x_init, mcmc_seed=mcmc_seed,
                    meta=dict(phi=phi, Sigma=Sigma, x_true=x_true))


def lattice_precision(side, tau=-0.25, r_y=1):
    """Precision of the spatio-temporal observation noise: tau^D for D <= r_y."""
    idx = [(i, j) for i in range(side) for j in range(side)]
    d = len(idx)
    Lam = np.zeros((d, d))
    for a, (i, j) in enumerate(idx):
        for b_, (k, l) in enumerate(idx):
            D = abs(i - k) + abs(j - l)
            if D <= r_y:
                Lam[a, b_] = tau ** D
    return Lam


def spatio_temporal(side=8, T=1024, n_chains=1, nu=1.0, tau=-0.25, r_y=1, sigma_x=1.0, sim_seed=0,
                    mcmc_seed=1, delta=0.05):
    d = side * side
    rng = np.random.default_rng(sim_seed)
    m0 = np.zeros(d)
    P0 = sigma_x ** 2 * np.eye(d)
    F = np.eye(d)
    b = np.zeros(d)
    Q = sigma_x ** 2 * np.eye(d)
    x_true = _simulate_dynamics(rng, m0, P0, F, b, Q, T)
    Sigma = np.linalg.inv(lattice_precision(side, tau, r_y))
    Ls = np.linalg.cholesky(Sigma)
    z = rng.standard_normal((T, d)) @ Ls.T
    w = rng.chisquare(nu, size=T)
    y = x_true + z / np.sqrt(w / nu)[:, None]
    x_init = np.repeat(x_true[None], n_chains, axis=0)
    return Workload(name=f"spatio_temporal_{side}x{side}_T{T}", d=d, T=T, n_chains=n_chains, m0=m0,
                    P0=P0, F=F, b=b, Q=Q, y=y, emission=EMIS_STUDENT_T, delta=delta, x_init=x_init,
                    mcmc_seed=mcmc_seed, Ry=Sigma, nu=nu, meta=dict(x_true=x_true))


def two_step_toy(rho=0.5, r2=0.1, y_obs=5.0, n_chains=1, delta=0.5, mcmc_seed=1):
    """Section 4.4 model; exact posterior of x_0: mean rho y/(1+r2), var 1 - rho^2/(1+r2)."""
    m0 = np.zeros(1); P0 = np.eye(1)
    F = np.array([[rho]]); b = np.zeros(1); Q = np.array([[1.0 - rho ** 2]])
    y = np.array([[0.0], [y_obs]])
    mask = np.array([0, 1], dtype=np.uint8)
    x_init = np.zeros((n_chains, 2, 1))
    return Workload(name=f"two_step_rho{rho}_r2{r2}", d=1, T=2, n_chains=n_chains,
                    m0=m0, P0=P0, F=F, b=b, Q=Q, y=y, emission=EMIS_LINEAR_GAUSSIAN,
                    delta=delta, x_init=x_init, mcmc_seed=mcmc_seed,
                    Ry=np.array([[r2]]), mask=mask,
                    meta=dict(post_mean_x0=rho * y_obs / (1.0 + r2),
                              post_var_x0=1.0 - rho ** 2 / (1.0 + r2)))


def random_lgssm(d, T, seed, time_varying=False):
    """A random stable LGSSM (for scan/filter equality tests)."""
    rng = np.random.default_rng(seed)

    def spd(scale):
        M = rng.standard_normal((d, d))
        return scale * (M @ M.T / d + 0.5 * np.eye(d))

    def stable():
        M = rng.standard_normal((d, d))
        return 0.9 * M / max(1.0, np.max(np.abs(np.linalg.eigvals(M))))

    m0 = rng.standard_normal(d)
    P0 = spd(1.0)
    if time_varying:
        F = np.stack([stable() for _ in range(T - 1)])
        b = rng.standard_normal((T - 1, d)) * 0.1
        Q = np.stack([spd(0.3) for _ in range(T - 1)])
    else:
        F = stable(); b = rng.standard_normal(d) * 0.1; Q = spd(0.3)
    y = rng.standard_normal((T, d))
    return dict(m0=m0, P0=P0, F=F, b=b, Q=Q, y=y)

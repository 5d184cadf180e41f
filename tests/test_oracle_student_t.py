"""Pins of the Student-t emission (Section 4.2) and the spatio-temporal workload."""
import numpy as np
import pytest

from oracle import mcmc
from paper_2303_00301_gb300 import workloads


def test_log_density_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(0)
    d, T = 5, 7
    A = rng.standard_normal((d, d))
    Sigma = A @ A.T + d * np.eye(d)
    y = rng.standard_normal((T, d))
    x = rng.standard_normal((T, d))
    for nu in (1.0, 3.5, 10.0):
        em = mcmc.StudentTEmission(y, Sigma, nu)
        ref = np.array([stats.multivariate_t(loc=x[t], shape=Sigma, df=nu).logpdf(y[t]) for t in range(T)])
        assert np.max(np.abs(em.log_h(x) - ref)) < 1e-10


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    d, T = 4, 3
    A = rng.standard_normal((d, d))
    em = mcmc.StudentTEmission(rng.standard_normal((T, d)), A @ A.T + np.eye(d), 1.0)
    x = rng.standard_normal((T, d))
    g = em.grad(x)
    h = 1e-6
    for i in range(d):
        e = np.zeros((T, d)); e[:, i] = h
        fd = (em.log_h(x + e) - em.log_h(x - e)) / (2 * h)
        assert np.max(np.abs(fd - g[:, i])) < 1e-6


def test_lattice_precision_structure():
    Lam = workloads.lattice_precision(3, tau=-0.25, r_y=1)
    assert Lam.shape == (9, 9)
    assert np.allclose(np.diag(Lam), 1.0)
    # (0,0) neighbours (0,1) and (1,0): tau; (1,1) at distance 2: 0
    assert Lam[0, 1] == -0.25 and Lam[0, 3] == -0.25 and Lam[0, 4] == 0.0
    assert np.all(np.linalg.eigvalsh(workloads.lattice_precision(8)) > 0)


def test_spatio_temporal_workload_shapes():
    wl = workloads.spatio_temporal(side=3, T=20, n_chains=2)
    assert wl.d == 9 and wl.y.shape == (20, 9) and wl.x_init.shape == (2, 20, 9)
    assert wl.emission == workloads.EMIS_STUDENT_T and wl.nu == 1.0

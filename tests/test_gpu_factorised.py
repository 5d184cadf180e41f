"""Factorised-prior path (Student-t emission, Section 4.2) against the dense FP64 oracle.

The library runs d independent scalar LGSSMs; the oracle runs the same auxiliary
LGSSM as one dense d-dimensional model, so agreement also checks the factorisation.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from oracle import kalman, mcmc, philox  # noqa: E402
from paper_2303_00301_gb300 import AuxKalman, workloads  # noqa: E402

TOL_LA32 = 2e-3


def _tt(a, dt):
    return torch.tensor(np.asarray(a), dtype=dt, device="cuda")


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def _model(wl):
    return dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q,
                emission=mcmc.StudentTEmission(wl.y, wl.Ry, wl.nu, wl.mask))


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("side,T,L", [(3, 40, 8), (2, 17, 5), (4, 33, 1)])
def test_loglik_and_sample_path(dt, side, T, L):
    wl = workloads.spatio_temporal(side=side, T=T, n_chains=2, delta=0.3)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 1e-4
    rng = np.random.default_rng(side * T)
    C, d = 2, wl.d
    yt = rng.standard_normal((C, T, d)) * 2.0
    eps = rng.standard_normal((C, T, d))
    s = AuxKalman(wl, dtype=dt, block_len=L)
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    mf = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    s.loglik(_tt(yt, tdt), logZ, mf)
    xs = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    s.sample_path(_tt(yt, tdt), xs, eps=_tt(eps, tdt))
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert abs(logZ[c].item() - kf["logZ"]) <= (1e-9 if dt == "f64" else 1e-5) * abs(kf["logZ"])
        assert _rel(mf[c].double().cpu().numpy(), kf["mf"]) < tol
        x_ref = kalman.rts_sample(kf, wl.F, wl.b, wl.Q, eps[c])
        assert _rel(xs[c].double().cpu().numpy(), x_ref) < tol
    s.close()


def _steps(wl, dt, L, n_iters, chains, tol_x, tol_la):
    tdt = torch.float64 if dt == "f64" else torch.float32
    s = AuxKalman(wl, dtype=dt, block_len=L)
    x = _tt(wl.x_init, tdt)
    la = torch.zeros(wl.n_chains, dtype=torch.float64, device="cuda")
    model = _model(wl)
    for it in range(n_iters):
        x_before = x.double().cpu().numpy()
        s.step(x, n_iters=1, iter0=it, log_alpha=la)
        torch.cuda.synchronize()
        xg, lag = x.double().cpu().numpy(), la.cpu().numpy()
        for c in chains:
            ref = mcmc.aux_step_philox(x_before[c], model, wl.delta, wl.mcmc_seed, c, it)
            lu = np.log(philox.mh_uniform(wl.mcmc_seed, c, it))
            near_tie = abs(ref["log_alpha"] - lu) < tol_la
            assert abs(lag[c] - ref["log_alpha"]) < tol_la or near_tie, (it, c, lag[c], ref["log_alpha"])
            if bool(lu < lag[c]) != ref["accepted"]:
                assert near_tie
                continue
            if ref["accepted"]:
                assert _rel(xg[c], ref["x_star"]) < tol_x, (it, c)
            else:
                assert np.array_equal(xg[c], x_before[c])
    assert s.status()[0] == 0
    s.close()


def test_kalman_step_f64():
    wl = workloads.spatio_temporal(side=3, T=30, n_chains=3, delta=0.2)
    _steps(wl, "f64", L=6, n_iters=3, chains=[0, 1, 2], tol_x=1e-9, tol_la=1e-8)


def test_kalman_step_f32():
    wl = workloads.spatio_temporal(side=3, T=30, n_chains=3, delta=0.2)
    _steps(wl, "f32", L=6, n_iters=3, chains=[0, 1, 2], tol_x=1e-4, tol_la=TOL_LA32)


def test_kalman_step_full_size_8x8_T1024_f32():
    """The lattice model of Section 4.2 at its size (d = 64, T = 1024), one chain."""
    wl = workloads.spatio_temporal(side=8, T=1024, n_chains=1, delta=0.05)
    _steps(wl, "f32", L=0, n_iters=1, chains=[0], tol_x=1e-4, tol_la=TOL_LA32)


def test_unsupported_calls_raise():
    wl = workloads.spatio_temporal(side=2, T=8, n_chains=1)
    s = AuxKalman(wl, dtype="f32")
    with pytest.raises(RuntimeError, match="unsupported"):
        s.b.aux_set_proposal(s.handle, 2)
    with pytest.raises(RuntimeError, match="unsupported"):
        s.loglik(_tt(np.zeros((1, 8, 4)), torch.float32), torch.zeros(1, dtype=torch.float64, device="cuda"),
                 Pf=torch.zeros((1, 8, 4, 4), device="cuda"))
    s.close()

"""Divide-and-conquer (bridging) sampler of the CUDA path against the FP64 oracle
(Section 2.4.2, Appendix A.2.3; oracle/bridging.py, pinned to dense Gaussian
conditionals in test_oracle_bridging.py).

Tolerances as in test_gpu_parity.py: normwise relative error per chain of
1e-9 (FP64) and 1e-4 (FP32) on paths; log alpha within 1e-8 (FP64) and
TOL_LA32 (FP32) absolute; MH decisions agree except where |log alpha - log U|
is inside the log-alpha tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import bridging, kalman, mcmc, philox  # noqa: E402
from paper_2303_00301_gb300 import MODES, AuxKalman, workloads  # noqa: E402

TOL_LA32 = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00301_gb300 import build
    build.build()


def _tt(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


def _lgssm_workload(d, T, C, seed, delta=0.5):
    m = workloads.random_lgssm(d, T, seed=seed)
    return workloads.Workload(name="rand", d=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"],
                              F=m["F"], b=m["b"], Q=m["Q"], y=m["y"],
                              emission=workloads.EMIS_LINEAR_GAUSSIAN, delta=delta,
                              x_init=np.zeros((C, T, d)), Ry=np.eye(d))


def _oracle_model(wl):
    if wl.emission == workloads.EMIS_SV:
        em = mcmc.SVEmission(wl.y, wl.mask)
    else:
        em = mcmc.LinearGaussianEmission(wl.y, wl.Ry, wl.mask)
    return dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)


# d, T, C, block_len, dtype: several tree levels, ragged T - 1, T = 1 and 2
CASES = [
    (2, 64, 2, 8, "f64"),
    (3, 37, 3, 5, "f64"),
    (1, 2, 2, 1, "f64"),
    (2, 1, 2, 1, "f64"),
    (4, 100, 2, 10, "f64"),
    (16, 50, 2, 9, "f64"),
    (5, 41, 2, 7, "f32"),
    (8, 33, 2, 6, "f32"),
    (30, 128, 2, 16, "f32"),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("d,T,C,L,dt", CASES)
def test_sample_path_matches_the_oracle(d, T, C, L, dt, mode):
    wl = _lgssm_workload(d, T, C, seed=300 + d * T)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 1e-4
    rng = np.random.default_rng(d * T + 1)
    yt = rng.standard_normal((C, T, d))
    eps = rng.standard_normal((C, T, d))
    s = AuxKalman(wl, dtype=dt, block_len=L, mode=mode, sampler="bridging")
    xs = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    s.sample_path(_tt(yt, tdt), xs, eps=_tt(eps, tdt), logZ=logZ)
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        ref = bridging.dnc_sample(kf, wl.F, wl.b, wl.Q, eps[c])
        assert _rel(xs[c].double().cpu().numpy(), ref) < tol, (c, _rel(xs[c].double().cpu().numpy(), ref))
        assert abs(logZ[c].item() - kf["logZ"]) <= (1e-9 if dt == "f64" else 1e-5) * abs(kf["logZ"])
    rc, per_chain = s.status()
    assert rc == 0 and not np.any(per_chain)
    s.close()


@pytest.mark.parametrize("mode", ["per_chain", "cached"])
def test_noise_is_the_backward_stream(mode):
    d, T, C = 3, 45, 2
    wl = _lgssm_workload(d, T, C, seed=5)
    s = AuxKalman(wl, dtype="f64", block_len=7, mode=mode, sampler="bridging")
    rng = np.random.default_rng(3)
    yt = rng.standard_normal((C, T, d))
    xs = torch.zeros((C, T, d), dtype=torch.float64, device="cuda")
    s.sample_path(_tt(yt, torch.float64), xs, iteration=17)
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        eps = philox.path_normals(wl.mcmc_seed, c, 17, philox.PURPOSE_BACKWARD, T, d)
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert _rel(xs[c].cpu().numpy(), bridging.dnc_sample(kf, wl.F, wl.b, wl.Q, eps)) < 1e-9
    s.close()


def _step_parity(wl, dt, L, mode, n_iters, chains=None, order=1):
    """Each iteration from the GPU's state: log alpha, the MH decision (up to near
    ties inside the tolerance) and the new state against the oracle's step with
    the bridging sampler and the same Philox streams."""
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol_x = 1e-9 if dt == "f64" else 1e-4
    tol_la = 1e-8 if dt == "f64" else TOL_LA32
    C = wl.n_chains
    s = AuxKalman(wl, dtype=dt, block_len=L, mode=mode, proposal=order, sampler="bridging")
    x = _tt(wl.x_init, tdt)
    la = torch.zeros(C, dtype=torch.float64, device="cuda")
    model = _oracle_model(wl)
    chains = list(range(C)) if chains is None else chains
    n_acc = 0
    for it in range(n_iters):
        x_before = x.double().cpu().numpy()
        s.step(x, 1, iter0=it, log_alpha=la)
        torch.cuda.synchronize()
        xg = x.double().cpu().numpy()
        lag = la.cpu().numpy()
        for c in chains:
            ref = mcmc.aux_step_philox(x_before[c], model, wl.delta, wl.mcmc_seed, c, it, order=order,
                                       sampler="bridging")
            lu = np.log(philox.mh_uniform(wl.mcmc_seed, c, it))
            near_tie = abs(ref["log_alpha"] - lu) < tol_la
            assert abs(lag[c] - ref["log_alpha"]) < tol_la or near_tie, (it, c, lag[c], ref["log_alpha"])
            if bool(lu < lag[c]) != ref["accepted"]:
                assert near_tie, (it, c, lag[c], ref["log_alpha"], lu)
                continue
            if ref["accepted"]:
                n_acc += 1
                assert _rel(xg[c], ref["x_star"]) < tol_x, (it, c, _rel(xg[c], ref["x_star"]))
            else:
                assert np.array_equal(xg[c], x_before[c]), (it, c)
    assert s.status()[0] == 0
    s.close()
    return n_acc


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_linear_gaussian_f64(mode):
    _step_parity(_lgssm_workload(3, 40, 3, seed=8, delta=0.4), "f64", 6, mode, 4)


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_sv_f64(mode):
    wl = workloads.stochastic_volatility(d=4, T=50, n_chains=3, delta=0.05)
    assert _step_parity(wl, "f64", 7, mode, 4) > 0


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_sv_f32(mode):
    wl = workloads.stochastic_volatility(d=8, T=65, n_chains=3, delta=0.05)
    _step_parity(wl, "f32", 8, mode, 3)


def test_kalman_step_parity_second_order_f64():
    wl = workloads.stochastic_volatility(d=3, T=30, n_chains=2, delta=0.3)
    _step_parity(wl, "f64", 5, "per_chain", 3, order=2)


@pytest.mark.parametrize("mode", ["shared", "cached"])
def test_kalman_step_full_size_sampled_chains(mode):
    """SV d = 30, T = 1024, 32 chains (the timed workload): two chains against the oracle."""
    wl = workloads.stochastic_volatility(d=30, T=1024, n_chains=32)
    _step_parity(wl, "f32", 0, mode, 2, chains=[0, 31])


def test_samplers_agree_in_law_at_full_size():
    """Same chains, either sampler: equal acceptance and path moments within MC error
    (the scan and the tree map the noise differently, so only the law is shared)."""
    wl = workloads.stochastic_volatility(d=30, T=1024, n_chains=32)
    out = {}
    for sampler in ("scan", "bridging"):
        s = AuxKalman(wl, dtype="f32", mode="cached", sampler=sampler)
        x = _tt(wl.x_init, torch.float32)
        acc = torch.zeros(32, dtype=torch.int32, device="cuda")
        s.step(x, 150, iter0=0)
        m1 = torch.zeros_like(x, dtype=torch.float64)
        for k in range(100):
            s.step(x, 1, iter0=150 + k, accept_count=acc)
            m1 += x.double()
        torch.cuda.synchronize()
        out[sampler] = ((m1 / 100).mean(0).cpu().numpy(), acc.sum().item() / (32 * 100))
        s.close()
    (ma, aa), (mb, ab) = out["scan"], out["bridging"]
    assert abs(aa - ab) < 0.08, (aa, ab)
    # posterior means of x_t(i) averaged over 32 chains x 100 iterations
    assert np.mean(np.abs(ma - mb)) < 0.15, np.mean(np.abs(ma - mb))


@pytest.mark.parametrize("mode", ["per_chain", "cached"])
def test_bridging_with_delta_adaptation_follows_the_oracle(mode):
    """On-device delta adaptation with the bridging sampler: delta trajectory and states
    against the oracle's pooled Robbins-Monro rule with the same sampler (FP64)."""
    from oracle import calibrate_delta
    wl = workloads.stochastic_volatility(d=3, T=21, n_chains=3, delta=0.3)
    s = AuxKalman(wl, dtype="f64", block_len=4, mode=mode, sampler="bridging")
    s.adapt_delta(True, target=0.5, gain=1.0)
    x = _tt(wl.x_init, torch.float64)
    n = 5
    s.step(x, n, iter0=0)
    torch.cuda.synchronize()
    xo, deltas, _ = calibrate_delta.run_chains_adaptive(wl.x_init, _oracle_model(wl), wl.delta, n,
                                                        seed=wl.mcmc_seed, sampler="bridging")
    log_d = np.log(deltas[-1])
    assert abs(s.delta() - float(np.exp(log_d))) < 1e-9 * float(np.exp(log_d))
    assert _rel(x.cpu().numpy(), xo) < 1e-9
    s.close()


def test_bridging_is_unsupported_on_the_factorised_path():
    wl = workloads.spatio_temporal(side=2, T=8, n_chains=1, delta=0.3)
    from paper_2303_00301_gb300 import _binding as B
    with pytest.raises(B.AuxError):
        AuxKalman(wl, dtype="f32", sampler="bridging")

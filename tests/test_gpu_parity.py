"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative errors are normwise over each chain's whole array, and
element-wise scaled by the oracle's posterior standard deviation: at every entry
|gpu - oracle| <= tol * (|oracle| + sd), see tests/parity_metrics.py):
  FP64 path: 1e-9 on means, covariances, paths and log Z; 1e-8 absolute on log alpha.
  FP32 path: 1e-4 on filtering means/covariances and sampled paths, 1e-5 on log Z
  (the stated accuracy targets); log alpha within TOL_LA32 absolute, a bound on
  the FP32 rounding of the T*d per-element terms summed into it; MH decisions must
  agree except where |log alpha_oracle - log U| < TOL_LA32. The |d log alpha|
  values and decision mismatches are collected in the session's parity report.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kalman, mcmc, philox  # noqa: E402
from paper_2303_00301_gb300 import MODES, AuxKalman, workloads  # noqa: E402
import parity_metrics as pm  # noqa: E402

TOL_LA32 = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00301_gb300 import build
    build.build()


def _tt(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


_rel = pm.rel


def _check_filter(key, tol, mfg, Pfg, kf):
    """Normwise and element-wise (posterior-sd scaled) parity of m^f and P^f."""
    assert _rel(mfg, kf["mf"]) < tol
    assert _rel(Pfg, kf["Pf"]) < tol
    em, eP = pm.vec_err(mfg, kf["mf"], kf["Pf"]), pm.mat_err(Pfg, kf["Pf"], kf["Pf"])
    pm.note("mf", key, em)
    pm.note("Pf", key, eP)
    assert em < tol, (key, em)
    assert eP < tol, (key, eP)


def _check_path(key, tol, xg, x_ref, Ps):
    """Normwise and element-wise parity of a sampled path (scale: smoothing sd)."""
    assert _rel(xg, x_ref) < tol, (key, _rel(xg, x_ref))
    e = pm.vec_err(xg, x_ref, Ps)
    pm.note("x_star", key, e)
    assert e < tol, (key, e)


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


FILTER_CASES = [
    # d, T, C, block_len, dtype
    (2, 64, 2, 8, "f64"),
    (1, 37, 3, 8, "f64"),
    (3, 37, 3, 5, "f64"),
    (16, 50, 2, 9, "f64"),
    (2, 1, 2, 1, "f64"),
    (3, 20, 2, 1, "f64"),
    (4, 20, 2, 20, "f64"),
    (5, 41, 2, 7, "f32"),
    (8, 33, 2, 6, "f32"),
    (30, 128, 2, 16, "f32"),
]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("d,T,C,L,dt", FILTER_CASES)
def test_loglik_filter_parity(d, T, C, L, dt, mode):
    wl = _lgssm_workload(d, T, C, seed=100 + d * T)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 1e-4
    tol_z = 1e-9 if dt == "f64" else 1e-5
    rng = np.random.default_rng(d + T)
    yt = rng.standard_normal((C, T, d))
    s = AuxKalman(wl, dtype=dt, block_len=L, mode=mode)
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    mf = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    Pf = torch.zeros((C, T, d, d), dtype=tdt, device="cuda")
    s.loglik(_tt(yt, tdt), logZ, mf, Pf)
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert abs(logZ[c].item() - kf["logZ"]) <= tol_z * abs(kf["logZ"]), (c, logZ[c].item(), kf["logZ"])
        pm.note("logZ", f"{dt}_{mode}", abs(logZ[c].item() - kf["logZ"]) / abs(kf["logZ"]))
        _check_filter(f"{dt}_{mode}", tol, mf[c].double().cpu().numpy(), Pf[c].double().cpu().numpy(), kf)
    assert s.status()[0] == 0
    s.close()


@pytest.mark.parametrize("mode", ["shared", "cached"])
@pytest.mark.parametrize("T,L", [(8, 8), (5, 4), (9, 4), (10, 4), (12, 4), (21, 4), (64, 4)])
def test_covariance_doubling_scan_shapes(T, L, mode):
    """p = 16 covariance pass (distinct block aggregates, prefixes by doubling) over
    2, 3 and more covariance blocks with and without a short last block."""
    d, C = 16, 2
    wl = _lgssm_workload(d, T, C, seed=40 + T)
    yt = np.random.default_rng(T).standard_normal((C, T, d))
    s = AuxKalman(wl, dtype="f64", block_len=L, mode=mode)
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    mf = torch.zeros((C, T, d), dtype=torch.float64, device="cuda")
    Pf = torch.zeros((C, T, d, d), dtype=torch.float64, device="cuda")
    s.loglik(_tt(yt, torch.float64), logZ, mf, Pf)
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert abs(logZ[c].item() - kf["logZ"]) <= 1e-9 * abs(kf["logZ"])
        _check_filter(f"f64_{mode}_doubling", 1e-9, mf[c].cpu().numpy(), Pf[c].cpu().numpy(), kf)
    s.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("d,T,C,L,dt", FILTER_CASES)
def test_sample_path_parity(d, T, C, L, dt, mode):
    wl = _lgssm_workload(d, T, C, seed=200 + d * T)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 1e-4
    rng = np.random.default_rng(7 * d + T)
    yt = rng.standard_normal((C, T, d))
    eps = rng.standard_normal((C, T, d))
    s = AuxKalman(wl, dtype=dt, block_len=L, mode=mode)
    xs = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    s.sample_path(_tt(yt, tdt), xs, eps=_tt(eps, tdt), logZ=logZ)
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        x_ref = kalman.rts_sample(kf, wl.F, wl.b, wl.Q, eps[c])
        _, Ps = kalman.rts_smoother(kf, wl.F)
        _check_path(f"{dt}_{mode}", tol, xs[c].double().cpu().numpy(), x_ref, Ps)
    s.close()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_backward_noise_is_the_philox_stream(dt):
    d, T, C = 6, 30, 3
    wl = _lgssm_workload(d, T, C, seed=5)
    tdt = torch.float64 if dt == "f64" else torch.float32
    s = AuxKalman(wl, dtype=dt, block_len=7, seed=77)
    yt = _tt(np.random.default_rng(1).standard_normal((C, T, d)), tdt)
    it = 123456789
    eps = philox.path_normals(77, np.arange(C), it, philox.PURPOSE_BACKWARD, T, d)
    xa = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    xb = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    s.sample_path(yt, xa, eps=None, iteration=it)
    s.sample_path(yt, xb, eps=_tt(eps, tdt), iteration=it)
    torch.cuda.synchronize()
    tol = 1e-12 if dt == "f64" else 2e-6
    assert _rel(xa.double().cpu().numpy(), xb.double().cpu().numpy()) < tol
    s.close()


def _step_and_compare(wl, dt, L, n_iters, chains=None, tol_x=None, tol_la=None, mode="per_chain",
                      proposal=1):
    """Step all chains on the GPU; replay the chosen chains on the oracle from the same state.

    Each oracle step starts from the GPU's state before that step, so a rare
    near-tie decision difference in FP32 does not make the paths diverge."""
    C = wl.n_chains
    tdt = torch.float64 if dt == "f64" else torch.float32
    s = AuxKalman(wl, dtype=dt, block_len=L, mode=mode, proposal=proposal)
    x = _tt(wl.x_init, tdt)
    la = torch.zeros(C, dtype=torch.float64, device="cuda")
    model = _oracle_model(wl)
    chains = list(range(C)) if chains is None else chains
    mismatches, max_dla, dlas = 0, 0.0, []
    key = f"{wl.name}_d{wl.d}_T{wl.T}_{dt}_{mode}_order{proposal}"
    for it in range(n_iters):
        x_before = x.double().cpu().numpy()
        s.step(x, n_iters=1, iter0=it, log_alpha=la)
        torch.cuda.synchronize()
        xg = x.double().cpu().numpy()
        lag = la.cpu().numpy()
        for c in chains:
            ref = mcmc.aux_step_philox(x_before[c], model, wl.delta, wl.mcmc_seed, c, it, order=proposal)
            lu = np.log(philox.mh_uniform(wl.mcmc_seed, c, it))
            dla = abs(lag[c] - ref["log_alpha"])
            max_dla = max(max_dla, dla)
            dlas.append(dla)
            near_tie = abs(ref["log_alpha"] - lu) < tol_la
            assert dla < tol_la or near_tie, (it, c, lag[c], ref["log_alpha"])
            gpu_accepted = bool(lu < lag[c])
            if gpu_accepted != ref["accepted"]:
                assert near_tie, (it, c, lag[c], ref["log_alpha"], lu)
                mismatches += 1
                continue
            if gpu_accepted:
                _, Ps = kalman.rts_smoother(ref["kf"], wl.F)
                _check_path(key, tol_x, xg[c], ref["x_star"], Ps)
            else:
                assert np.array_equal(xg[c], x_before[c]), (it, c)
    assert s.status()[0] == 0
    s.close()
    pm.note_log_alpha(key, dlas, mismatches, tol_la)
    return mismatches, max_dla, lag


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_linear_gaussian_f64(mode):
    wl = workloads.linear_gaussian(d=2, T=64, n_chains=4)
    _step_and_compare(wl, "f64", L=8, n_iters=4, tol_x=1e-9, tol_la=1e-8, mode=mode)


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_masked_toy_f64(mode):
    wl = workloads.two_step_toy(rho=0.7, r2=0.3, n_chains=3)
    _step_and_compare(wl, "f64", L=1, n_iters=4, tol_x=1e-9, tol_la=1e-8, mode=mode)


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_sv_f64(mode):
    wl = workloads.stochastic_volatility(d=6, T=45, n_chains=3, delta=0.05)
    _step_and_compare(wl, "f64", L=8, n_iters=3, tol_x=1e-9, tol_la=1e-8, mode=mode)


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_sv_f32_small(mode):
    wl = workloads.stochastic_volatility(d=6, T=45, n_chains=4, delta=0.05)
    _step_and_compare(wl, "f32", L=8, n_iters=3, tol_x=1e-4, tol_la=TOL_LA32, mode=mode)


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_sv_f32_full_size_sampled_chains(mode):
    """d=30, T=1024, 32 chains in the benchmark's launch configuration; oracle on 4 chains."""
    wl = workloads.stochastic_volatility(d=30, T=1024, n_chains=32)
    _step_and_compare(wl, "f32", L=0, n_iters=1, chains=[0, 9, 22, 31], tol_x=1e-4,
                      tol_la=TOL_LA32, mode=mode)


@pytest.mark.parametrize("mode", MODES)
def test_kalman_step_parity_sv_f64_padded_32(mode):
    """FP64 at the padded width 32 (d = 30, the SV shape of the paper's Section 4.1
    runs, which it ran in FP64): the same FP64 bands as the small FP64 cases."""
    wl = workloads.stochastic_volatility(d=30, T=96, n_chains=3, delta=0.0183)
    _step_and_compare(wl, "f64", L=8, n_iters=2, tol_x=1e-9, tol_la=1e-8, mode=mode)


def test_kalman_step_parity_sv_f64_full_size_sampled_chains():
    """d=30, T=1024, 32 chains in FP64 in the benchmark's shared-mode launch
    configuration; oracle on 3 chains."""
    wl = workloads.stochastic_volatility(d=30, T=1024, n_chains=32)
    _step_and_compare(wl, "f64", L=0, n_iters=1, chains=[0, 17, 31], tol_x=1e-9, tol_la=1e-8, mode="shared")


# ---- second-order proposal (Section 2.2, Eqs. (2.8)-(2.9)), per-chain path

def test_second_order_sv_f64():
    wl = workloads.stochastic_volatility(d=6, T=45, n_chains=3, delta=0.05)
    _step_and_compare(wl, "f64", L=8, n_iters=3, tol_x=1e-9, tol_la=1e-8, proposal=2)


def test_second_order_sv_f32_small():
    wl = workloads.stochastic_volatility(d=6, T=45, n_chains=4, delta=0.05)
    _step_and_compare(wl, "f32", L=8, n_iters=3, tol_x=1e-4, tol_la=TOL_LA32, proposal=2)


def test_second_order_masked_toy_f64():
    wl = workloads.two_step_toy(rho=0.7, r2=0.3, n_chains=3)
    _step_and_compare(wl, "f64", L=1, n_iters=4, tol_x=1e-9, tol_la=1e-8, proposal=2)


def test_second_order_is_exact_on_the_linear_gaussian_model():
    """With a Gaussian emission the second-order proposal is the exact conditional:
    log alpha = 0 on the GPU as in the oracle, and every step is accepted."""
    wl = workloads.linear_gaussian(d=2, T=64, n_chains=4)
    _, max_dla, lag = _step_and_compare(wl, "f64", L=8, n_iters=3, tol_x=1e-9, tol_la=1e-8, proposal=2)
    assert np.max(np.abs(lag)) < 1e-8


def test_second_order_sv_f32_full_size_sampled_chains():
    """d=30, T=1024, 32 chains; oracle on 3 chains."""
    wl = workloads.stochastic_volatility(d=30, T=1024, n_chains=32)
    _step_and_compare(wl, "f32", L=0, n_iters=1, chains=[0, 17, 31], tol_x=1e-4, tol_la=TOL_LA32,
                      proposal=2)


@pytest.mark.parametrize("mode", ["shared", "cached"])
def test_second_order_is_rejected_in_table_modes(mode):
    wl = workloads.stochastic_volatility(d=4, T=16, n_chains=2, delta=0.05)
    s = AuxKalman(wl, dtype="f32", block_len=4, mode=mode, proposal=2)
    x = _tt(wl.x_init, torch.float32)
    with pytest.raises(RuntimeError, match="unsupported"):
        s.step(x, n_iters=1, iter0=0)
    s.close()


# ---- on-device delta adaptation (pooled Robbins-Monro on log delta)

@pytest.mark.parametrize("mode", MODES)
def test_delta_adaptation_follows_the_oracle_f64(mode):
    from oracle import calibrate_delta
    wl = workloads.stochastic_volatility(d=3, T=20, n_chains=3, delta=0.2)
    n, target, gain = 12, 0.5, 1.5
    s = AuxKalman(wl, dtype="f64", block_len=4, mode=mode)
    s.adapt_delta(True, target=target, gain=gain)
    x = _tt(wl.x_init, torch.float64)
    deltas = [s.delta()]
    for k in range(n):
        s.step(x, n_iters=1, iter0=k)
        deltas.append(s.delta())
    x_ref, d_ref, _ = calibrate_delta.run_chains_adaptive(wl.x_init, _oracle_model(wl), 0.2, n,
                                                         target=target, c=gain, seed=wl.mcmc_seed)
    assert np.max(np.abs(np.array(deltas) / d_ref - 1.0)) < 1e-9, (deltas, d_ref)
    assert _rel(x.cpu().numpy(), x_ref) < 1e-9
    s.adapt_delta(False)
    assert abs(s.delta() - d_ref[-1]) < 1e-9 * d_ref[-1]
    s.close()


def test_delta_adaptation_reaches_the_target_f32():
    wl = workloads.stochastic_volatility(d=8, T=64, n_chains=16, delta=2.0)
    s = AuxKalman(wl, dtype="f32", block_len=8, mode="cached")
    s.adapt_delta(True, target=0.4, gain=2.0)
    x = _tt(wl.x_init, torch.float32)
    acc = torch.zeros(16, dtype=torch.int32, device="cuda")
    s.step(x, n_iters=150, iter0=0)
    s.step(x, n_iters=150, iter0=150, accept_count=acc)
    torch.cuda.synchronize()
    rate = acc.float().mean().item() / 150
    assert abs(rate - 0.4) < 0.1, (rate, s.delta())
    s.close()


def test_execution_modes_agree_at_full_size():
    """d=30, T=1024, 32 chains: the three execution modes give the same steps (FP32 rounding)."""
    wl = workloads.stochastic_volatility(d=30, T=1024, n_chains=32)
    out = []
    for mode in MODES:
        s = AuxKalman(wl, dtype="f32", mode=mode)
        x = _tt(wl.x_init, torch.float32)
        la = torch.zeros(32, dtype=torch.float64, device="cuda")
        s.step(x, n_iters=2, iter0=0, log_alpha=la)
        torch.cuda.synchronize()
        out.append((x.double().cpu().numpy(), la.cpu().numpy()))
        assert s.status()[0] == 0
        s.close()
    xa, la_a = out[0]
    for xb, la_b in out[1:]:
        assert np.max(np.abs(la_a - la_b)) < TOL_LA32
        for c in range(32):
            assert _rel(xa[c], xb[c]) < 1e-5, c


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_cached_tables_follow_model_updates(dt):
    """The cached covariance tables are rebuilt after aux_set_model_params and aux_set_mode."""
    d, T, C = 4, 29, 2
    wl = _lgssm_workload(d, T, C, seed=31)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol_z = 1e-9 if dt == "f64" else 1e-5
    yt = np.random.default_rng(3).standard_normal((C, T, d))
    s = AuxKalman(wl, dtype=dt, block_len=6, mode="cached")
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")

    def check(model_wl):
        s.loglik(_tt(yt, tdt), logZ)
        torch.cuda.synchronize()
        R = 0.5 * model_wl.delta * np.eye(d)
        for c in range(C):
            ref = kalman.kalman_filter(yt[c], model_wl.m0, model_wl.P0, model_wl.F, model_wl.b,
                                       model_wl.Q, R)["logZ"]
            assert abs(logZ[c].item() - ref) <= tol_z * abs(ref), (c, logZ[c].item(), ref)

    check(wl)
    check(wl)                       # second call reuses the tables
    wl2 = _lgssm_workload(d, T, C, seed=32, delta=0.37)
    s.b.aux_set_model_params(s.handle, d_x=d, T=T, n_chains=C, m0=wl2.m0, P0=wl2.P0, F=wl2.F,
                             b=wl2.b, Q=wl2.Q, y=wl2.y, delta=wl2.delta, emis_kind=wl2.emission,
                             dtype=s.dtype_code, R_y=wl2.Ry, obs_mask=wl2.mask)
    check(wl2)
    s.b.aux_set_mode(s.handle, s.b.AUX_MODE_PER_CHAIN)
    check(wl2)
    s.b.aux_set_mode(s.handle, s.b.AUX_MODE_CACHED_COV)
    check(wl2)
    s.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_resume_is_bitwise(dt, mode):
    wl = workloads.stochastic_volatility(d=5, T=33, n_chains=3, delta=0.05)
    tdt = torch.float64 if dt == "f64" else torch.float32
    s = AuxKalman(wl, dtype=dt, block_len=6, mode=mode)
    xa = _tt(wl.x_init, tdt)
    xb = _tt(wl.x_init, tdt)
    s.step(xa, n_iters=6, iter0=10)
    s.step(xb, n_iters=2, iter0=10)
    s.step(xb, n_iters=4, iter0=12)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb)
    s.close()


def test_nonfinite_state_is_rejected_and_reported():
    wl = workloads.stochastic_volatility(d=4, T=20, n_chains=3, delta=0.05)
    s = AuxKalman(wl, dtype="f32", block_len=5)
    x0 = wl.x_init.copy()
    x0[1, 7, 2] = np.nan
    x = _tt(x0, torch.float32)
    s.step(x, n_iters=1, iter0=0)
    torch.cuda.synchronize()
    rc, per_chain = s.status()
    assert per_chain[1] != 0 and per_chain[0] == 0 and per_chain[2] == 0
    xg = x.cpu().numpy()
    assert np.isnan(xg[1, 7, 2]) and np.array_equal(np.nan_to_num(xg[1]), np.nan_to_num(x0[1].astype(np.float32)))
    assert s.status()[0] == 0      # cleared by the previous read
    s.close()


def test_two_step_toy_posterior_on_gpu():
    """Section 4.4 model: the ensemble of many chains matches the closed-form posterior of x_0."""
    rho, r2, y = 0.8, 0.5, 2.0
    C = 512
    wl = workloads.two_step_toy(rho=rho, r2=r2, y_obs=y, n_chains=C, delta=1.0, mcmc_seed=3)
    s = AuxKalman(wl, dtype="f64", block_len=1)
    x = _tt(wl.x_init, torch.float64)
    acc = torch.zeros(C, dtype=torch.int32, device="cuda")
    s.step(x, n_iters=300, iter0=0, accept_count=acc)
    torch.cuda.synchronize()
    x0 = x[:, 0, 0].cpu().numpy()
    m, v = wl.meta["post_mean_x0"], wl.meta["post_var_x0"]
    assert abs(x0.mean() - m) < 4.5 * np.sqrt(v / C)
    assert abs(x0.var() / v - 1) < 0.25
    assert 0.2 < acc.float().mean().item() / 300 < 0.99
    s.close()


def test_linear_gaussian_stationarity_on_gpu():
    """Config-1 model: chain ensemble matches the exact smoother (KF + RTS) within MC error."""
    C = 256
    wl = workloads.linear_gaussian(d=2, T=64, n_chains=C)
    s = AuxKalman(wl, dtype="f64", block_len=8)
    x = _tt(wl.x_init, torch.float64)
    s.step(x, n_iters=400, iter0=0)
    torch.cuda.synchronize()
    xe = x.cpu().numpy()
    kf = kalman.kalman_filter(wl.y, wl.m0, wl.P0, wl.F, wl.b, wl.Q, wl.Ry)
    ms, Ps = kalman.rts_smoother(kf, wl.F)
    sd = np.sqrt(np.einsum("tii->ti", Ps))
    z = (xe.mean(axis=0) - ms) / (sd / np.sqrt(C))
    assert np.max(np.abs(z)) < 4.5, np.max(np.abs(z))
    ratio = xe.var(axis=0) / sd ** 2
    assert 0.75 < ratio.mean() < 1.25
    s.close()


# ---- time-varying dynamics (AUX_DYN_TIME_VARYING): per-chain path

def _tv_workload(d, T, C, seed, delta=0.5):
    m = workloads.random_lgssm(d, T, seed=seed, time_varying=True)
    return workloads.Workload(name="tv", d=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"],
                              F=m["F"], b=m["b"], Q=m["Q"], y=m["y"],
                              emission=workloads.EMIS_LINEAR_GAUSSIAN, delta=delta,
                              x_init=np.zeros((C, T, d)), Ry=np.eye(d))


@pytest.mark.parametrize("d,T,C,L,dt", [(3, 37, 2, 5, "f64"), (2, 2, 2, 1, "f64"), (16, 40, 2, 7, "f64"),
                                         (5, 41, 2, 7, "f32"), (30, 128, 2, 16, "f32")])
def test_time_varying_filter_and_path_parity(d, T, C, L, dt):
    """F_t, b_t, Q_t per transition: log Z, m^f, P^f and a sampled path against the
    oracle's filter and RTS sampler on the stacked model (Algorithm 2, local dynamics)."""
    wl = _tv_workload(d, T, C, seed=300 + d * T)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 1e-4
    tol_z = 1e-9 if dt == "f64" else 1e-5
    rng = np.random.default_rng(d * T + 1)
    yt = rng.standard_normal((C, T, d))
    eps = rng.standard_normal((C, T, d))
    s = AuxKalman(wl, dtype=dt, block_len=L)
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    mf = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    Pf = torch.zeros((C, T, d, d), dtype=tdt, device="cuda")
    s.loglik(_tt(yt, tdt), logZ, mf, Pf)
    xs = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    s.sample_path(_tt(yt, tdt), xs, eps=_tt(eps, tdt))
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert abs(logZ[c].item() - kf["logZ"]) <= tol_z * abs(kf["logZ"]), (c, logZ[c].item(), kf["logZ"])
        _check_filter(f"tv_{dt}", tol, mf[c].double().cpu().numpy(), Pf[c].double().cpu().numpy(), kf)
        x_ref = kalman.rts_sample(kf, wl.F, wl.b, wl.Q, eps[c])
        _, Ps = kalman.rts_smoother(kf, wl.F)
        _check_path(f"tv_{dt}", tol, xs[c].double().cpu().numpy(), x_ref, Ps)
    assert s.status()[0] == 0
    s.close()


@pytest.mark.parametrize("proposal", [1, 2])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_time_varying_step_parity(dt, proposal):
    wl = _tv_workload(4, 33, 3, seed=77, delta=0.3)
    tol_x, tol_la = (1e-9, 1e-8) if dt == "f64" else (1e-4, TOL_LA32)
    _step_and_compare(wl, dt, L=6, n_iters=3, tol_x=tol_x, tol_la=tol_la, proposal=proposal)


def test_time_varying_scope_is_reported():
    from paper_2303_00301_gb300 import _binding as B
    wl = _tv_workload(3, 12, 2, seed=1)
    for kw in (dict(mode="shared"), dict(mode="cached"), dict(sampler="bridging"),
               dict(filter_form="square_root")):
        with pytest.raises(B.AuxError):
            AuxKalman(wl, dtype="f64", block_len=4, **kw)
    s = AuxKalman(wl, dtype="f64", block_len=4)
    g = torch.zeros(2, 3, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AuxError):
        s.grad(torch.zeros((2, 12, 3), dtype=torch.float64, device="cuda"), g[:, 0], g[:, 1], g,
               torch.zeros(2, dtype=torch.float64, device="cuda"))
    s.close()

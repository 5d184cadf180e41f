"""Square-root form (aux_set_filter_form) of the per-chain parallel filter and of
the table modes' covariance pass against the FP64 oracle (oracle/sqrt_filter.py,
pinned to the covariance form and the Kalman filter in test_oracle_sqrt_filter.py).

Tolerances: FP64 1e-9 relative on m^f, P^f and log Z; FP32 1e-4 on m^f and P^f,
1e-5 on log Z (normwise per chain), as for the covariance form.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kalman, sqrt_filter  # noqa: E402
from paper_2303_00301_gb300 import AuxKalman, workloads  # noqa: E402
from paper_2303_00301_gb300 import _binding as B  # noqa: E402


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


def _workload(d, T, C, seed, delta=0.5, Q=None):
    m = workloads.random_lgssm(d, T, seed=seed)
    return workloads.Workload(name="rand", d=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"],
                              F=m["F"], b=m["b"], Q=m["Q"] if Q is None else Q, y=m["y"],
                              emission=workloads.EMIS_LINEAR_GAUSSIAN, delta=delta,
                              x_init=np.zeros((C, T, d)), Ry=np.eye(d))


def _run(wl, dt, L, yt, form, mode="per_chain"):
    C, T, d = wl.n_chains, wl.T, wl.d
    tdt = torch.float64 if dt == "f64" else torch.float32
    s = AuxKalman(wl, dtype=dt, block_len=L, filter_form=form, mode=mode)
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    mf = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    Pf = torch.zeros((C, T, d, d), dtype=tdt, device="cuda")
    s.loglik(_tt(yt, tdt), logZ, mf, Pf)
    torch.cuda.synchronize()
    out = logZ.cpu().numpy(), mf.double().cpu().numpy(), Pf.double().cpu().numpy(), s.status()
    s.close()
    return out


CASES = [
    # d, T, C, block_len, dtype: several blocks, ragged tail, one block, T = 1
    (2, 64, 2, 8, "f64"),
    (1, 37, 3, 8, "f64"),
    (3, 37, 3, 5, "f64"),
    (4, 20, 2, 20, "f64"),
    (3, 1, 2, 1, "f64"),
    (16, 50, 2, 9, "f64"),
    (5, 41, 2, 7, "f32"),
    (8, 33, 2, 6, "f32"),
    (30, 128, 2, 16, "f32"),
]


@pytest.mark.parametrize("d,T,C,L,dt", CASES)
def test_square_root_filter_matches_the_oracle(d, T, C, L, dt):
    wl = _workload(d, T, C, seed=700 + d * T)
    rng = np.random.default_rng(d + 3 * T)
    yt = rng.standard_normal((C, T, d))
    logZ, mf, Pf, (rc, st) = _run(wl, dt, L, yt, "square_root")
    tol = 1e-9 if dt == "f64" else 1e-4
    tol_z = 1e-9 if dt == "f64" else 1e-5
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        ref = sqrt_filter.sr_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert abs(logZ[c] - ref["logZ"]) <= tol_z * abs(ref["logZ"]), (c, logZ[c], ref["logZ"])
        assert _rel(mf[c], ref["mf"]) < tol
        assert _rel(Pf[c], np.einsum("tij,tkj->tik", ref["Uf"], ref["Uf"])) < tol
    assert rc == 0 and not np.any(st)


def test_square_root_and_covariance_forms_agree():
    wl = _workload(6, 96, 3, seed=11)
    yt = np.random.default_rng(2).standard_normal((3, 96, 6))
    a = _run(wl, "f64", 12, yt, "square_root")
    b = _run(wl, "f64", 12, yt, "covariance")
    assert np.allclose(a[0], b[0], rtol=1e-12, atol=1e-9)
    assert _rel(a[1], b[1]) < 1e-11 and _rel(a[2], b[2]) < 1e-11


def test_single_precision_stays_accurate_where_the_covariance_form_loses_it():
    """Observations far more precise than the dynamics (r = 1e-6 against Q ~ 1): P^f ~ r I
    is a small difference of O(1) covariances in the covariance form; the square-root
    form never forms it. Both in FP32 against the FP64 oracle."""
    d, T, C = 8, 128, 2
    rng = np.random.default_rng(4)
    A = rng.standard_normal((d, d))
    Q = A @ A.T / d + np.eye(d)
    wl = _workload(d, T, C, seed=21, delta=2e-6, Q=Q)
    yt = rng.standard_normal((C, T, d)) * 2.0
    R = 0.5 * wl.delta * np.eye(d)
    err = {}
    for form in ("square_root", "covariance"):
        logZ, mf, Pf, (rc, st) = _run(wl, "f32", 16, yt, form)
        e_pf, e_z = [], []
        for c in range(C):
            kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
            e_pf.append(_rel(Pf[c], kf["Pf"]))
            e_z.append(abs(logZ[c] - kf["logZ"]) / abs(kf["logZ"]))
        err[form] = (max(e_pf), max(e_z), int(np.any(st)))
    print("P^f rel err, log Z rel err, status:", err)
    assert err["square_root"][0] < 1e-4 and err["square_root"][1] < 1e-5 and err["square_root"][2] == 0
    # measured on GB300: 2.3e-7 against 1.5e-1
    assert 100 * err["square_root"][0] < err["covariance"][0]


def test_scope_is_reported():
    wl = _workload(3, 20, 2, seed=1)
    x = _tt(wl.x_init, torch.float64)
    s = AuxKalman(wl, dtype="f64", block_len=5, filter_form="square_root", sampler="bridging")
    with pytest.raises(B.AuxError):
        s.step(x, 1)
    s.close()


# ---- the table modes: the covariance pass on factors (k_srcov_reduce / _scan_double / _apply)
TAB_CASES = [
    # d, T, C, block_len, dtype, mode: one covariance block, several, ragged tail, T = 1
    (2, 64, 2, 8, "f64", "shared"),
    (1, 37, 3, 8, "f64", "cached"),
    (3, 37, 3, 5, "f64", "shared"),
    (4, 300, 2, 20, "f64", "cached"),
    (3, 1, 2, 1, "f64", "shared"),
    (16, 133, 2, 16, "f64", "cached"),
    (13, 257, 2, 32, "f64", "shared"),
    (30, 257, 2, 32, "f32", "cached"),
    (8, 65, 2, 8, "f32", "cached"),
    (30, 1024, 2, 32, "f32", "shared"),
]


@pytest.mark.parametrize("d,T,C,L,dt,mode", TAB_CASES)
def test_table_modes_square_root_match_the_oracle(d, T, C, L, dt, mode):
    wl = _workload(d, T, C, seed=300 + d * T)
    rng = np.random.default_rng(2 * d + T)
    yt = rng.standard_normal((C, T, d))
    logZ, mf, Pf, (rc, st) = _run(wl, dt, L, yt, "square_root", mode=mode)
    tol = 1e-9 if dt == "f64" else 1e-4
    tol_z = 1e-9 if dt == "f64" else 1e-5
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        ref = sqrt_filter.sr_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert abs(logZ[c] - ref["logZ"]) <= tol_z * abs(ref["logZ"]), (c, logZ[c], ref["logZ"])
        assert _rel(mf[c], ref["mf"]) < tol
        assert _rel(Pf[c], np.einsum("tij,tkj->tik", ref["Uf"], ref["Uf"])) < tol
    assert rc == 0 and not np.any(st)


def test_table_modes_square_root_and_covariance_forms_agree():
    wl = _workload(12, 200, 3, seed=17)
    yt = np.random.default_rng(3).standard_normal((3, 200, 12))
    for mode in ("shared", "cached"):
        a = _run(wl, "f64", 24, yt, "square_root", mode=mode)
        b = _run(wl, "f64", 24, yt, "covariance", mode=mode)
        assert np.allclose(a[0], b[0], rtol=1e-12, atol=1e-9)
        assert _rel(a[1], b[1]) < 1e-11 and _rel(a[2], b[2]) < 1e-11


def test_table_modes_single_precision_at_small_r():
    """The ill-conditioned case of the per-chain test above (r = 1e-6 against Q ~ 1)
    through the covariance pass of the cached mode. There both forms keep single
    precision: the square-root form by its factors, the covariance form because its
    pass builds every covariance without subtracting nearly equal matrices (the
    elements as r S^{-1} P, the prefixes by additions C_e + P P^T), unlike the
    per-chain covariance filter above, whose step P^p - Y^T Y loses the digits."""
    d, T, C = 8, 128, 2
    rng = np.random.default_rng(4)
    A = rng.standard_normal((d, d))
    Q = A @ A.T / d + np.eye(d)
    wl = _workload(d, T, C, seed=21, delta=2e-6, Q=Q)
    yt = rng.standard_normal((C, T, d)) * 2.0
    R = 0.5 * wl.delta * np.eye(d)
    err = {}
    for form in ("square_root", "covariance"):
        logZ, mf, Pf, (rc, st) = _run(wl, "f32", 16, yt, form, mode="cached")
        e_pf, e_z = [], []
        for c in range(C):
            kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
            e_pf.append(_rel(Pf[c], kf["Pf"]))
            e_z.append(abs(logZ[c] - kf["logZ"]) / abs(kf["logZ"]))
        err[form] = (max(e_pf), max(e_z), int(np.any(st)))
    print("cached mode: P^f rel err, log Z rel err, status:", err)
    for form in ("square_root", "covariance"):
        assert err[form][0] < 1e-4 and err[form][1] < 1e-5 and err[form][2] == 0, (form, err[form])


@pytest.mark.parametrize("sampler", ["scan", "bridging"])
@pytest.mark.parametrize("d,T,C,L,dt,mode", [(3, 37, 3, 5, "f64", "cached"), (16, 133, 2, 16, "f64", "shared"),
                                             (8, 65, 2, 8, "f32", "shared")])
def test_table_modes_sample_path(d, T, C, L, dt, mode, sampler):
    """Both samplers on the tables of the square-root covariance pass, against the
    same sampler on the covariance form's tables (the bridging sampler maps eps
    differently, so each form is compared with its own sampler) and, for the
    (G, U) scan, against the RTS sampler of the oracle."""
    wl = _workload(d, T, C, seed=40 + d * T)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 1e-4
    rng = np.random.default_rng(d + T)
    yt = rng.standard_normal((C, T, d))
    eps = rng.standard_normal((C, T, d))
    out = {}
    for form in ("square_root", "covariance"):
        s = AuxKalman(wl, dtype=dt, block_len=L, filter_form=form, mode=mode, sampler=sampler)
        xs = torch.zeros((C, T, d), dtype=tdt, device="cuda")
        logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
        s.sample_path(_tt(yt, tdt), xs, eps=_tt(eps, tdt), logZ=logZ)
        torch.cuda.synchronize()
        out[form] = (xs.double().cpu().numpy(), logZ.cpu().numpy())
        assert s.status()[0] == 0
        s.close()
    assert _rel(out["square_root"][0], out["covariance"][0]) < (1e-10 if dt == "f64" else 1e-3)
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        assert abs(out["square_root"][1][c] - kf["logZ"]) <= (1e-9 if dt == "f64" else 1e-5) * abs(kf["logZ"])
        if sampler == "scan":
            ref = kalman.rts_sample(kf, wl.F, wl.b, wl.Q, eps[c])
            assert _rel(out["square_root"][0][c], ref) < tol


@pytest.mark.parametrize("d,T,C,L,dt", CASES)
def test_sample_path_matches_the_rts_sampler(d, T, C, L, dt):
    """Same filter, the backward elements in Joseph form: the (G, U) scan's path is the
    RTS sampler's (Appendix A.1) for the same eps."""
    wl = _workload(d, T, C, seed=900 + d * T)
    tdt = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 1e-4
    rng = np.random.default_rng(5 * d + T)
    yt = rng.standard_normal((C, T, d))
    eps = rng.standard_normal((C, T, d))
    s = AuxKalman(wl, dtype=dt, block_len=L, filter_form="square_root")
    xs = torch.zeros((C, T, d), dtype=tdt, device="cuda")
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    s.sample_path(_tt(yt, tdt), xs, eps=_tt(eps, tdt), logZ=logZ)
    torch.cuda.synchronize()
    R = 0.5 * wl.delta * np.eye(d)
    for c in range(C):
        kf = kalman.kalman_filter(yt[c], wl.m0, wl.P0, wl.F, wl.b, wl.Q, R)
        ref = kalman.rts_sample(kf, wl.F, wl.b, wl.Q, eps[c])
        assert _rel(xs[c].double().cpu().numpy(), ref) < tol
        assert abs(logZ[c].item() - kf["logZ"]) <= (1e-9 if dt == "f64" else 1e-5) * abs(kf["logZ"])
    s.close()


def _step_parity(wl, dt, L, n_iters, tol_x, tol_la, mode="per_chain"):
    from oracle import mcmc, philox
    C = wl.n_chains
    tdt = torch.float64 if dt == "f64" else torch.float32
    s = AuxKalman(wl, dtype=dt, block_len=L, filter_form="square_root", mode=mode)
    x = _tt(wl.x_init, tdt)
    la = torch.zeros(C, dtype=torch.float64, device="cuda")
    em = mcmc.SVEmission(wl.y, wl.mask)
    model = dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)
    moved = 0
    for it in range(n_iters):
        x_before = x.double().cpu().numpy()
        s.step(x, 1, iter0=it, log_alpha=la)
        torch.cuda.synchronize()
        xg = x.double().cpu().numpy()
        for c in range(C):
            ref = mcmc.aux_step_philox(x_before[c], model, wl.delta, wl.mcmc_seed, c, it)
            lu = np.log(philox.mh_uniform(wl.mcmc_seed, c, it))
            near = abs(ref["log_alpha"] - lu) < tol_la
            assert abs(la[c].item() - ref["log_alpha"]) < tol_la or near
            if bool(lu < la[c].item()) != ref["accepted"]:
                assert near
                continue
            if ref["accepted"]:
                moved += 1
                assert _rel(xg[c], ref["x_star"]) < tol_x
            else:
                assert np.array_equal(xg[c], x_before[c])
    assert s.status()[0] == 0
    s.close()
    return moved


def test_kalman_step_parity_sv_f64():
    wl = workloads.stochastic_volatility(d=5, T=40, n_chains=3, delta=0.05)
    assert _step_parity(wl, "f64", 7, 3, 1e-9, 1e-8) > 0


def test_kalman_step_parity_sv_f32():
    wl = workloads.stochastic_volatility(d=8, T=64, n_chains=3, delta=0.05)
    _step_parity(wl, "f32", 8, 3, 1e-4, 2e-3)


@pytest.mark.parametrize("mode", ["shared", "cached"])
def test_kalman_step_parity_table_modes_sv(mode):
    wl = workloads.stochastic_volatility(d=5, T=40, n_chains=3, delta=0.05)
    assert _step_parity(wl, "f64", 7, 3, 1e-9, 1e-8, mode=mode) > 0
    wl = workloads.stochastic_volatility(d=8, T=64, n_chains=3, delta=0.05)
    _step_parity(wl, "f32", 8, 3, 1e-4, 2e-3, mode=mode)


def test_kalman_step_full_size_sampled_step():
    """d = 30, T = 1024, 32 chains, FP32: one step of every chain against the oracle,
    per chain and on the shared tables."""
    for mode in ("per_chain", "shared"):
        _full_size_step(mode)


def _full_size_step(mode):
    wl = workloads.stochastic_volatility(d=30, T=1024, n_chains=32)
    s = AuxKalman(wl, dtype="f32", filter_form="square_root", mode=mode)
    from oracle import mcmc, philox
    x = _tt(wl.x_init, torch.float32)
    la = torch.zeros(32, dtype=torch.float64, device="cuda")
    s.step(x, 1, iter0=0, log_alpha=la)
    torch.cuda.synchronize()
    em = mcmc.SVEmission(wl.y, wl.mask)
    model = dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)
    for c in (0, 31):
        ref = mcmc.aux_step_philox(wl.x_init[c], model, wl.delta, wl.mcmc_seed, c, 0)
        assert abs(la[c].item() - ref["log_alpha"]) < 2e-3
    assert s.status()[0] == 0
    s.close()

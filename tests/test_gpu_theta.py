"""The SV parameterisation behind the C ABI and the on-device theta-update of the
Gibbs sweep (aux_set_sv_theta, aux_sv_theta_step, aux_loglik_grad with the last
step's pseudo-observations), against the FP64 oracle.

Tolerances: FP64 1e-9 relative (log Z, theta); FP32 1e-5 on log Z and 1e-4 on
theta after an update (the gradient itself is held to 1e-3 in FP32, times a
small learning rate).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import gradient, kalman, mcmc  # noqa: E402
from paper_2303_00301_gb300 import AuxKalman, workloads  # noqa: E402
from paper_2303_00301_gb300 import _binding as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00301_gb300 import build
    build.build()


def _theta(d, seed, delta=0.05):
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal(d) * 0.3
    phi = rng.uniform(0.8, 0.99, d)
    Sigma = 0.5 * np.ones((d, d)) + 0.5 * np.eye(d)
    L = np.linalg.cholesky(Sigma) * rng.uniform(0.8, 1.2)
    return mu, phi, L, delta


def _sv_workload(theta, T, C, y):
    m = gradient.sv_model(*theta)
    d = len(theta[0])
    return workloads.Workload(name="svtheta", d=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"], F=m["F"],
                              b=m["b"], Q=m["Q"], y=y, emission=workloads.EMIS_SV, delta=theta[3],
                              x_init=np.zeros((C, T, d)))


def _logz(s, yt, tdt):
    C = yt.shape[0]
    z = torch.zeros(C, dtype=torch.float64, device="cuda")
    s.loglik(torch.tensor(yt, dtype=tdt, device="cuda"), z)
    torch.cuda.synchronize()
    return z.cpu().numpy()


@pytest.mark.parametrize("dt,d,mode", [("f64", 3, "per_chain"), ("f64", 5, "shared"), ("f32", 30, "shared"),
                                       ("f32", 12, "per_chain")])
def test_set_theta_is_the_stationary_sv_model(dt, d, mode):
    """aux_set_sv_theta forms F, b, Q, P0, m0 on the device: log Z equals the oracle's
    Kalman filter on sv_model(theta), for a theta other than the handle's first."""
    T, C = 40, 2
    th0, th1 = _theta(d, 1), _theta(d, 2, delta=0.07)
    rng = np.random.default_rng(d)
    s = AuxKalman(_sv_workload(th0, T, C, rng.standard_normal((T, d))), dtype=dt, block_len=8, mode=mode)
    s.set_theta(*th1)
    yt = rng.standard_normal((C, T, d))
    tdt = torch.float64 if dt == "f64" else torch.float32
    z = _logz(s, yt, tdt)
    m = gradient.sv_model(*th1)
    tol = 1e-9 if dt == "f64" else 1e-5
    for c in range(C):
        ref = kalman.kalman_filter(yt[c], m["m0"], m["P0"], m["F"], m["b"], m["Q"], m["R"])["logZ"]
        assert abs(z[c] - ref) <= tol * abs(ref), (c, z[c], ref)
    mu, phi, L = s.theta()
    assert np.allclose(mu, th1[0], rtol=0, atol=1e-15) and np.allclose(phi, th1[1], rtol=0, atol=1e-15)
    assert np.allclose(L, np.tril(th1[2]), rtol=0, atol=1e-15)
    s.close()


@pytest.mark.parametrize("dt,d", [("f64", 4), ("f32", 16)])
def test_theta_step_follows_the_oracle_update(dt, d):
    T, C, lr = 30, 3, 2e-3
    th = _theta(d, 5)
    rng = np.random.default_rng(3)
    s = AuxKalman(_sv_workload(th, T, C, rng.standard_normal((T, d))), dtype=dt, block_len=6)
    tdt = torch.float64 if dt == "f64" else torch.float32
    yt = rng.standard_normal((C, T, d))
    g = [torch.zeros(C, d, dtype=torch.float64, device="cuda"), torch.zeros(C, d, dtype=torch.float64, device="cuda"),
         torch.zeros(C, d, d, dtype=torch.float64, device="cuda"), torch.zeros(C, dtype=torch.float64, device="cuda")]
    s.grad(torch.tensor(yt, dtype=tdt, device="cuda"), *g)
    s.theta_step(g[0], g[1], g[2], lr)
    mu, phi, L = s.theta()
    gs = [gradient.loglik_grad(th, yt[c]) for c in range(C)]
    ref = gradient.sv_theta_update(th[0], th[1], th[2], [x[0] for x in gs], [x[1] for x in gs],
                                   [x[2] for x in gs], lr)
    tol = 1e-9 if dt == "f64" else 1e-4
    for a, b in zip((mu, phi, L), ref):
        assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b))), (a, b)
    # the model was rebuilt from the new theta
    z = _logz(s, yt, tdt)
    m = gradient.sv_model(ref[0], ref[1], ref[2], th[3])
    tz = 1e-9 if dt == "f64" else 1e-5
    for c in range(C):
        r = kalman.kalman_filter(yt[c], m["m0"], m["P0"], m["F"], m["b"], m["Q"], m["R"])["logZ"]
        assert abs(z[c] - r) <= tz * abs(r)
    s.close()


@pytest.mark.parametrize("mode", ["per_chain", "shared"])
def test_theta_within_gibbs_sweep_captured_matches_the_oracle(mode):
    """A sweep x-update (aux_kalman_step) -> gradient on that step's pseudo-observations
    (aux_loglik_grad, ytilde = NULL) -> theta-update (aux_sv_theta_step), captured once
    in a CUDA graph and replayed, equals the oracle's sweep (FP64, Philox draws)."""
    d, T, C, lr, sweeps = 3, 20, 2, 5e-3, 3
    th = _theta(d, 8, delta=0.1)
    rng = np.random.default_rng(11)
    x_true = rng.standard_normal((T, d)) * 0.5
    y = np.exp(0.5 * x_true) * rng.standard_normal((T, d))
    wl = _sv_workload(th, T, C, y)
    s = AuxKalman(wl, dtype="f64", block_len=5, mode=mode)
    x = torch.zeros((C, T, d), dtype=torch.float64, device="cuda")
    g = [torch.zeros(C, d, dtype=torch.float64, device="cuda"), torch.zeros(C, d, dtype=torch.float64, device="cuda"),
         torch.zeros(C, d, d, dtype=torch.float64, device="cuda"), torch.zeros(C, dtype=torch.float64, device="cuda")]
    # first call outside the capture: allocates the gradient buffers
    s.step(x, 1, iter0=0)
    s.grad(None, *g)
    s.theta_step(g[0], g[1], g[2], lr)
    s.device_iteration(True, 1)
    st = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        graph.capture_begin()
        s.step(x, 1, stream=st.cuda_stream)
        s.grad(None, *g, stream=st.cuda_stream)
        s.theta_step(g[0], g[1], g[2], lr, stream=st.cuda_stream)
        graph.capture_end()
    for _ in range(sweeps - 1):
        graph.replay()
    torch.cuda.synchronize()
    mu, phi, L = s.theta()
    xg = x.cpu().numpy()
    s.close()
    # the oracle's sweep
    theta = (th[0], th[1], th[2])
    xs = [np.zeros((T, d)) for _ in range(C)]
    for it in range(sweeps):
        m = gradient.sv_model(theta[0], theta[1], theta[2], th[3])
        model = dict(m0=m["m0"], P0=m["P0"], F=m["F"], b=m["b"], Q=m["Q"], emission=mcmc.SVEmission(y))
        gs = []
        for c in range(C):
            st_ = mcmc.aux_step_philox(xs[c], model, th[3], wl.mcmc_seed, c, it)
            gs.append(gradient.loglik_grad((theta[0], theta[1], theta[2], th[3]), st_["ytilde"]))
            xs[c] = st_["x_new"]
        theta = gradient.sv_theta_update(theta[0], theta[1], theta[2], [q[0] for q in gs], [q[1] for q in gs],
                                         [q[2] for q in gs], lr)
    for a, b in zip((mu, phi, L), theta):
        assert np.max(np.abs(a - b)) <= 1e-8 * max(1.0, np.max(np.abs(b))), (a, b)
    for c in range(C):
        assert np.max(np.abs(xg[c] - xs[c])) <= 1e-8 * max(1.0, np.max(np.abs(xs[c])))


def test_theta_scope_is_reported():
    d, T, C = 3, 10, 2
    th = _theta(d, 1)
    s = AuxKalman(_sv_workload(th, T, C, np.zeros((T, d))), dtype="f64", block_len=5, mode="cached")
    g = torch.zeros(C, d, d, dtype=torch.float64, device="cuda")
    with pytest.raises(B.AuxError):          # cached tables would go stale
        s.theta_step(g[:, 0], g[:, 1], g, 1e-3)
    bad_phi = th[1].copy()
    bad_phi[0] = 1.2
    with pytest.raises(B.AuxError):
        s.set_theta(th[0], bad_phi, th[2], th[3])
    bad_L = th[2].copy()
    bad_L[1, 1] = -1.0
    with pytest.raises(B.AuxError):
        s.set_theta(th[0], th[1], bad_L, th[3])
    s.close()

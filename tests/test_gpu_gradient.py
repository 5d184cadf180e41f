"""aux_loglik_grad (Fisher-identity gradient on the GPU) against the FP64 oracle.

Tolerances: FP64 path 1e-8 relative to the oracle's analytic gradient and 1e-5
to central finite differences; FP32 path 1e-3 relative (normwise per parameter
block), the stated target for the gradient.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import gradient  # noqa: E402
from paper_2303_00301_gb300 import AuxKalman, workloads  # noqa: E402


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


def _workload(theta, T, C):
    from paper_2303_00301_gb300.svgrad import sv_model_arrays
    m = sv_model_arrays(*theta)
    d = len(theta[0])
    return workloads.Workload(name="svgrad", d=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"],
                              F=m["F"], b=m["b"], Q=m["Q"], y=np.zeros((T, d)),
                              emission=workloads.EMIS_SV, delta=m["delta"],
                              x_init=np.zeros((C, T, d)))


def _gpu_grad(theta, yt, L_blk, dt, grad_mem=0):
    C, T, d = yt.shape
    s = AuxKalman(_workload(theta, T, C), dtype=dt, block_len=L_blk)
    if grad_mem:
        s.b.aux_set_grad_memory(s.handle, grad_mem)
    tdt = torch.float64 if dt == "f64" else torch.float32
    y = torch.tensor(yt, dtype=tdt, device="cuda")
    out = [torch.zeros(C, d, dtype=torch.float64, device="cuda"),
           torch.zeros(C, d, dtype=torch.float64, device="cuda"),
           torch.zeros(C, d, d, dtype=torch.float64, device="cuda"),
           torch.zeros(C, dtype=torch.float64, device="cuda")]
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    s.b.aux_loglik_grad(s.handle, y, *out, logZ=logZ)
    torch.cuda.synchronize()
    assert s.status()[0] == 0
    s.close()
    return [o.cpu().numpy() for o in out], logZ.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("d,T,L", [(3, 40, 7), (1, 9, 4), (5, 33, 33), (4, 25, 1)])
def test_grad_f64_matches_oracle_and_finite_differences(d, T, L):
    theta = _theta(d, seed=d + T)
    C = 2
    yt = np.random.default_rng(T).standard_normal((C, T, d)) * 0.5
    (g_mu, g_phi, g_L, g_delta), logZ = _gpu_grad(theta, yt, L, "f64")
    for c in range(C):
        r_mu, r_phi, r_L, r_delta, r_logZ = gradient.loglik_grad(theta, yt[c])
        assert abs(logZ[c] - r_logZ) <= 1e-10 * abs(r_logZ)
        assert _rel(g_mu[c], r_mu) < 1e-8
        assert _rel(g_phi[c], r_phi) < 1e-8
        assert _rel(g_L[c], r_L) < 1e-8
        assert abs(g_delta[c] - r_delta) <= 1e-8 * abs(r_delta)
    f_mu, f_phi, f_L, f_delta = gradient.loglik_fd_grad(theta, yt[0], h=1e-5)
    assert _rel(g_mu[0], f_mu) < 1e-5 and _rel(g_phi[0], f_phi) < 1e-5
    assert _rel(g_L[0], f_L) < 1e-5 and abs(g_delta[0] - f_delta) < 1e-5 * abs(f_delta)


@pytest.mark.parametrize("d,T,C,L", [(8, 64, 3, 8), (32, 2048, 64, 0)])
def test_grad_f32_matches_oracle(d, T, C, L):
    """(32, 2048, 64) is the differentiation workload (oracle on two sampled chains)."""
    theta = _theta(d, seed=7 * d)
    rng = np.random.default_rng(d)
    yt = rng.standard_normal((C, T, d)) * 0.5
    (g_mu, g_phi, g_L, g_delta), logZ = _gpu_grad(theta, yt, L, "f32")
    for c in ([0, C - 1] if C > 3 else range(C)):
        r_mu, r_phi, r_L, r_delta, r_logZ = gradient.loglik_grad(theta, yt[c])
        assert abs(logZ[c] - r_logZ) <= 1e-5 * abs(r_logZ)
        assert _rel(g_mu[c], r_mu) < 1e-3, _rel(g_mu[c], r_mu)
        assert _rel(g_phi[c], r_phi) < 1e-3, _rel(g_phi[c], r_phi)
        assert _rel(g_L[c], r_L) < 1e-3, _rel(g_L[c], r_L)
        assert abs(g_delta[c] - r_delta) <= 1e-3 * abs(r_delta)


def test_autograd_function_and_theta_ascent():
    """SVLogZ.backward returns the library gradient; a few ascent steps raise log Z."""
    from paper_2303_00301_gb300.svgrad import SVLogZ
    d, T, C = 4, 64, 3
    theta = _theta(d, seed=3)
    s = AuxKalman(_workload(theta, T, C), dtype="f64", block_len=8)
    yt = torch.tensor(np.random.default_rng(0).standard_normal((C, T, d)), device="cuda")
    mu = torch.tensor(theta[0], requires_grad=True)
    phi = torch.tensor(theta[1], requires_grad=True)
    L = torch.tensor(theta[2], requires_grad=True)
    delta = torch.tensor(theta[3], dtype=torch.float64, requires_grad=True)
    lz = SVLogZ.apply(mu, phi, L, delta, yt, s).sum()
    lz.backward()
    ref = [gradient.loglik_grad(theta, yt[c].cpu().numpy()) for c in range(C)]
    assert _rel(mu.grad.numpy(), sum(r[0] for r in ref)) < 1e-8
    assert _rel(L.grad.numpy(), sum(r[2] for r in ref)) < 1e-8
    assert abs(delta.grad.item() - sum(r[3] for r in ref)) < 1e-8 * abs(delta.grad.item())
    # gradient ascent on mu alone increases the total log-likelihood
    vals = []
    m = mu.detach().clone()
    for _ in range(4):
        m.requires_grad_(True)
        v = SVLogZ.apply(m, phi.detach(), L.detach(), delta.detach(), yt, s).sum()
        v.backward()
        vals.append(v.item())
        m = (m + 1e-3 * m.grad).detach()
    assert all(b > a for a, b in zip(vals, vals[1:]))
    s.close()


def test_grad_refuses_f64_at_padded_width_32():
    """FP64 at d_x > 16: sampling runs, the gradient's smoother does not fit a CTA's
    shared memory and aux_loglik_grad reports AUX_E_UNSUPPORTED instead."""
    from paper_2303_00301_gb300._binding import AuxError
    theta = _theta(20, 3)
    yt = np.zeros((2, 16, 20))
    with pytest.raises(AuxError) as ei:
        _gpu_grad(theta, yt, 4, "f64")
    assert ei.value.code == 7   # AUX_E_UNSUPPORTED


def _store_bytes(C, T, d, es):
    p = next(w for w in (4, 8, 16, 32) if w >= d)
    return C * T * (2 * p * p + p) * es


@pytest.mark.parametrize("d,T,C,L,dt,blocks", [(5, 200, 3, 16, "f64", 1), (5, 200, 3, 16, "f64", 3),
                                               (30, 512, 6, 23, "f32", 2), (32, 2048, 64, 46, "f32", 5)])
def test_grad_recompute_not_store_equals_the_stored_path(d, T, C, L, dt, blocks):
    """With a memory cap the in-block filter is recomputed per chunk of blocks
    (twice) instead of storing G_t, Sigma_t, U_t for all steps: the same
    arithmetic per block, so the same gradient bit for bit; chunks of one, three
    and two blocks, and five at the differentiation workload (d = 32, T = 2048,
    64 chains), where the full store is 1.1 GB and the cap 130 MB. The FP64 case
    is also held to the oracle."""
    theta = _theta(d, seed=11 * d)
    rng = np.random.default_rng(d + T)
    yt = rng.standard_normal((C, T, d)) * 0.5
    es = 8 if dt == "f64" else 4
    p = next(w for w in (4, 8, 16, 32) if w >= d)
    cap = blocks * C * L * (2 * p * p + p) * es          # room for `blocks` blocks per chunk
    assert cap < _store_bytes(C, T, d, es)
    g0, z0 = _gpu_grad(theta, yt, L, dt)
    g1, z1 = _gpu_grad(theta, yt, L, dt, grad_mem=cap)
    for a, b in zip(g0, g1):
        assert np.array_equal(a, b)
    assert np.array_equal(z0, z1)
    if dt == "f64":
        for c in range(C):
            r_mu, r_phi, r_L, r_delta, r_logZ = gradient.loglik_grad(theta, yt[c])
            assert _rel(g1[0][c], r_mu) < 1e-8 and _rel(g1[1][c], r_phi) < 1e-8
            assert _rel(g1[2][c], r_L) < 1e-8 and abs(g1[3][c] - r_delta) <= 1e-8 * abs(r_delta)

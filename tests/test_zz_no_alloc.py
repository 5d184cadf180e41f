"""aux_loglik_noalloc: the log-likelihood entry point that allocates no device memory.

Some callers cannot call cudaMalloc (code inside a host callback, under an
allocator it must not bypass, or with a device-memory budget fixed up front),
so they cannot create a model handle. This entry point serves them from a
fixed scratch array inside the library. These tests call it through the C ABI
and check it against aux_loglik (the handle-based entry point) on two calls in
a row, with the tolerances of the other parity tests; they pass when run alone
in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00301_gb300 import build
    build.build()
    from paper_2303_00301_gb300 import _binding
    return _binding


def _model(d, T, seed):
    from paper_2303_00301_gb300 import workloads
    return workloads.random_lgssm(d, T, seed=seed)


@pytest.mark.parametrize("d,T,C,L,dt", [(30, 256, 4, 16, "f32"), (3, 37, 3, 5, "f64"),
                                         (8, 64, 2, 0, "f32")])
def test_noalloc_matches_aux_loglik_on_two_calls(lib, d, T, C, L, dt):
    m = _model(d, T, seed=11 * d + T)
    delta = 0.5
    code = lib.AUX_F32 if dt == "f32" else lib.AUX_F64
    tdt = torch.float32 if dt == "f32" else torch.float64
    tol = 1e-5 if dt == "f32" else 1e-9
    handle = lib.aux_init_model(d_x=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"], F=m["F"],
                                b=m["b"], Q=m["Q"], y=m["y"], delta=delta, emis_kind=0,
                                dtype=code, R_y=np.eye(d), block_len=L, seed=1)
    rng = np.random.default_rng(d + T)
    try:
        for call in range(2):
            yt = torch.tensor(rng.standard_normal((C, T, d)), dtype=tdt, device="cuda")
            ref = torch.zeros(C, dtype=torch.float64, device="cuda")
            out = torch.full((C,), float("nan"), dtype=torch.float64, device="cuda")
            lib.aux_loglik(handle, yt, ref)
            lib.aux_loglik_noalloc(yt, out, d_x=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"],
                                   F=m["F"], b=m["b"], Q=m["Q"], delta=delta, dtype=code,
                                   block_len=L)
            torch.cuda.synchronize()
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            assert np.all(np.isfinite(o)), (call, o)
            assert np.all(np.abs(o - r) <= tol * np.abs(r)), (call, o, r)
    finally:
        lib.aux_free_model(handle)


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    d, T, C = 32, 4096, 64
    m = _model(d, 4, seed=1)
    yt = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.AuxError) as e:
        lib.aux_loglik_noalloc(yt, out, d_x=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"],
                               F=m["F"], b=m["b"], Q=m["Q"], delta=0.5, dtype=lib.AUX_F32)
    assert e.value.code == lib.AUX_E_TOO_LARGE


def test_noalloc_reports_a_nonfinite_result(lib):
    """A NaN in one chain's pseudo-observations gives a non-finite logZ for that
    chain; the call reports it (AUX_E_NONFINITE) and the other chains still equal
    aux_loglik. A later clean call on the same scratch returns AUX_OK."""
    d, T, C = 6, 40, 3
    m = _model(d, T, seed=3)
    kw = dict(d_x=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"], F=m["F"], b=m["b"], Q=m["Q"],
              delta=0.5, dtype=lib.AUX_F32, block_len=8)
    yt = torch.tensor(np.random.default_rng(0).standard_normal((C, T, d)), dtype=torch.float32,
                      device="cuda")
    ref = torch.zeros(C, dtype=torch.float64, device="cuda")
    lib.aux_loglik_noalloc(yt, ref, **kw)
    bad = yt.clone()
    bad[1, 17, 2] = float("nan")
    out = torch.zeros(C, dtype=torch.float64, device="cuda")
    with pytest.raises(lib.AuxError) as e:
        lib.aux_loglik_noalloc(bad, out, **kw)
    assert e.value.code == lib.AUX_E_NONFINITE
    o, r = out.cpu().numpy(), ref.cpu().numpy()
    assert not np.isfinite(o[1])
    assert np.all(np.abs(o[[0, 2]] - r[[0, 2]]) <= 1e-5 * np.abs(r[[0, 2]]))
    out2 = torch.zeros(C, dtype=torch.float64, device="cuda")
    lib.aux_loglik_noalloc(yt, out2, **kw)
    assert np.all(np.abs(out2.cpu().numpy() - r) <= 1e-12 * np.abs(r))


def test_noalloc_refuses_stream_capture(lib):
    """The call synchronises its stream, so it refuses a capturing stream up front
    (AUX_E_UNSUPPORTED, nothing enqueued) and the capture itself stays valid."""
    d, T, C = 4, 16, 2
    m = _model(d, T, seed=4)
    yt = torch.zeros((C, T, d), dtype=torch.float32, device="cuda")
    out = torch.zeros(C, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    code = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            lib.aux_loglik_noalloc(yt, out, d_x=d, T=T, n_chains=C, m0=m["m0"], P0=m["P0"],
                                   F=m["F"], b=m["b"], Q=m["Q"], delta=0.5, dtype=lib.AUX_F32,
                                   stream=s.cuda_stream)
        except lib.AuxError as e:
            code = e.code
        out.add_(1.0)
        g.capture_end()
    assert code == lib.AUX_E_UNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(out == 1.0)

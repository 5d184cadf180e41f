"""Parity of the batched persistent launch (aux_batch_*) with the FP64 oracle.

A batch of models of uneven T and padded widths 4 .. 64 (SV and linear-Gaussian
emissions, one or two chains each) takes MCMC steps in one persistent launch per
iteration; every chain is replayed on the oracle from the same state with the
same Philox streams (Algorithm 2). Tolerances as in test_gpu_parity: FP32 log
alpha within TOL_LA32 absolute, identical MH decisions except within TOL_LA32 of
log U, accepted paths within 1e-4 (normwise and element-wise, scaled by the
smoothing standard deviation), rejected chains unchanged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kalman, mcmc, philox  # noqa: E402
from paper_2303_00301_gb300 import AuxBatch, AuxKalman, workloads  # noqa: E402
import parity_metrics as pm  # noqa: E402

TOL_LA32 = 2e-3
TOL_X32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00301_gb300 import build
    build.build()


def _oracle_model(wl):
    if wl.emission == workloads.EMIS_SV:
        em = mcmc.SVEmission(wl.y, wl.mask)
    else:
        em = mcmc.LinearGaussianEmission(wl.y, wl.Ry, wl.mask)
    return dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)


# (d, T, chains): padded widths 4, 8, 16, 32 and 64, block lengths that leave ragged
# last blocks, one model of a single block and one of a single step
MIXED = [(3, 37, 2), (8, 50, 1), (13, 61, 2), (30, 45, 1), (40, 23, 2), (64, 31, 1), (5, 6, 1), (9, 2, 1)]


def _mixed_workloads():
    wls = []
    for i, (d, T, C) in enumerate(MIXED):
        delta = 0.05 * np.sqrt(30.0 / d)
        wls.append(workloads.stochastic_volatility(d=d, T=T, n_chains=C, sim_seed=200 + i,
                                                   mcmc_seed=300 + i, delta=delta))
    wls.append(workloads.linear_gaussian(d=2, T=64, n_chains=2, sim_seed=7, mcmc_seed=11))
    # linear-Gaussian emissions whose R_y^{-1} products run at widths 32 and 64, and the
    # two-step toy of Section 4.4 (first observation masked)
    wls.append(workloads.linear_gaussian(d=20, T=40, n_chains=1, sim_seed=9, mcmc_seed=17, delta=0.05))
    wls.append(workloads.linear_gaussian(d=40, T=20, n_chains=1, sim_seed=10, mcmc_seed=19, delta=0.05))
    wls.append(workloads.two_step_toy(n_chains=2, mcmc_seed=13))
    return wls


def _make(wls, mode):
    models = [AuxKalman(wl, dtype="f32", mode=mode) for wl in wls]
    xs = [torch.tensor(np.ascontiguousarray(wl.x_init), dtype=torch.float32, device="cuda") for wl in wls]
    return models, xs


def _compare_step(wls, x_before, xg, lag, it, key):
    """Replay every chain on the oracle from its state before the step."""
    dlas, mism = [], 0
    off = 0
    for wl, xb, xn in zip(wls, x_before, xg):
        model = _oracle_model(wl)
        for c in range(wl.n_chains):
            ref = mcmc.aux_step_philox(xb[c], model, wl.delta, wl.mcmc_seed, c, it)
            lu = np.log(philox.mh_uniform(wl.mcmc_seed, c, it))
            la = lag[off + c]
            dla = abs(la - ref["log_alpha"])
            dlas.append(dla)
            near_tie = abs(ref["log_alpha"] - lu) < TOL_LA32
            assert dla < TOL_LA32 or near_tie, (wl.name, c, it, la, ref["log_alpha"])
            acc = bool(lu < la)
            if acc != ref["accepted"]:
                assert near_tie, (wl.name, c, it)
                mism += 1
                continue
            if acc:
                _, Ps = kalman.rts_smoother(ref["kf"], wl.F)
                assert pm.rel(xn[c], ref["x_star"]) < TOL_X32, (wl.name, c, pm.rel(xn[c], ref["x_star"]))
                e = pm.vec_err(xn[c], ref["x_star"], Ps)
                pm.note("x_star", key, e)
                assert e < TOL_X32, (wl.name, c, e)
            else:
                assert np.array_equal(xn[c], xb[c].astype(np.float32)), (wl.name, c)
        off += wl.n_chains
    pm.note_log_alpha(key, dlas, mism, TOL_LA32)


def _run_and_compare(wls, batch, xs, n_iters, it0, key):
    n = sum(wl.n_chains for wl in wls)
    la = torch.zeros(n, dtype=torch.float64, device="cuda")
    for it in range(it0, it0 + n_iters):
        x_before = [x.double().cpu().numpy() for x in xs]
        batch.step(1, log_alpha=la)
        torch.cuda.synchronize()
        _compare_step(wls, x_before, [x.cpu().numpy() for x in xs], la.cpu().numpy(), it, key)
    assert batch.status() == (0, 0)


CONFIGS = [
    dict(warps_per_cta=8, ctas_per_sm=0, order=0, block_factor=None),
    dict(warps_per_cta=4, ctas_per_sm=1, order=1, block_factor=[0.5, 2.0, 0.5, 2.0]),
    dict(warps_per_cta=16, ctas_per_sm=2, order=0, block_factor=[2.0, 0.5, 2.0, 0.5]),
]


@pytest.mark.parametrize("mode", ["cached", "shared"])
@pytest.mark.parametrize("cfg", range(len(CONFIGS)))
def test_batch_step_matches_the_oracle(mode, cfg):
    wls = _mixed_workloads()
    models, xs = _make(wls, mode)
    b = AuxBatch(models, xs, iteration=5, mode=mode)
    b.set_config(**CONFIGS[cfg])
    _run_and_compare(wls, b, xs, 2, 5, f"batch_mixed_{mode}_cfg{cfg}")
    assert b.iteration() == 7
    b.close()
    for m in models:
        assert m.status()[0] == 0
        m.close()


def test_batch_equals_the_per_model_steps_at_full_size():
    """SV d = 30, T = 1024 and d = 64, T = 512 (4 chains each) in one batch against
    the same handles stepped one by one (aux_kalman_step, same iterations), each
    step from the same state."""
    wls = [workloads.stochastic_volatility(d=30, T=1024, n_chains=4),
           workloads.stochastic_volatility(d=64, T=512, n_chains=4, sim_seed=3, mcmc_seed=4, delta=0.01)]
    models, xs = _make(wls, "cached")
    b = AuxBatch(models, xs, iteration=0)
    la_b = torch.zeros(8, dtype=torch.float64, device="cuda")
    la_r = [torch.zeros(4, dtype=torch.float64, device="cuda") for _ in wls]
    for it in range(3):
        xr = [x.clone() for x in xs]
        b.step(1, log_alpha=la_b)
        for m, x, la in zip(models, xr, la_r):
            m.step(x, 1, iter0=it, log_alpha=la)
        torch.cuda.synchronize()
        lb = la_b.cpu().numpy()
        lr = np.concatenate([la.cpu().numpy() for la in la_r])
        assert np.max(np.abs(lb - lr)) < TOL_LA32, (it, lb, lr)
        for w, (wl, x, y) in enumerate(zip(wls, xs, xr)):
            xa, xb = x.double().cpu().numpy(), y.double().cpu().numpy()
            for c in range(4):
                lu = np.log(philox.mh_uniform(wl.mcmc_seed, c, it))
                if abs(lr[4 * w + c] - lu) < TOL_LA32:
                    continue   # a near tie may be decided either way
                assert pm.rel(xa[c], xb[c]) < 1e-5, (it, w, c, pm.rel(xa[c], xb[c]))
    assert b.status() == (0, 0)
    b.close()
    for m in models:
        m.close()


def test_batch_graph_replays_equal_eager_steps():
    """The step captured once in a CUDA graph (the iteration lives on the device):
    replays are bit-identical to eager steps from the same state and iteration."""
    wls = _mixed_workloads()
    models, xs = _make(wls, "cached")
    x0 = [x.clone() for x in xs]
    b = AuxBatch(models, xs, iteration=3)
    for _ in range(3):
        b.step(1)
    torch.cuda.synchronize()
    x_eager = [x.clone() for x in xs]
    for x, y in zip(xs, x0):
        x.copy_(y)
    b.set_iteration(3)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        b.step(1, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    b.set_iteration(3)
    for x, y in zip(xs, x0):
        x.copy_(y)
    torch.cuda.synchronize()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert b.iteration() == 6
    for x, y in zip(xs, x_eager):
        assert torch.equal(x, y)
    del g
    b.close()
    for m in models:
        m.close()


def test_batch_tuner_restores_the_chains_and_keeps_parity():
    wls = _mixed_workloads()
    models, xs = _make(wls, "cached")
    x0 = [x.clone() for x in xs]
    b = AuxBatch(models, xs, iteration=9)
    best = b.tune(reps=2)
    torch.cuda.synchronize()
    assert best > 0.0
    cfg = b.config()
    assert cfg["warps_per_cta"] in (4, 8, 16) and cfg["order"] in (0, 1)
    assert all(f in (0.5, 1.0, 2.0) for f in cfg["block_factor"])
    assert len(cfg["block_len"]) == len(wls)
    assert b.iteration() == 9
    for x, y in zip(xs, x0):
        assert torch.equal(x, y)
    _run_and_compare(wls, b, xs, 1, 9, "batch_mixed_tuned")
    b.close()
    for m in models:
        m.close()


def test_batch_rejects_unsupported_models():
    from paper_2303_00301_gb300 import _binding as B
    wl = workloads.stochastic_volatility(d=6, T=20, n_chains=1)
    x = torch.zeros((1, 20, 6), dtype=torch.float32, device="cuda")
    for kw in (dict(dtype="f32", mode="per_chain"), dict(dtype="f64", mode="cached")):
        m = AuxKalman(wl, **kw)
        with pytest.raises(B.AuxError) as e:
            AuxBatch([m], [x])
        assert e.value.code == B.AUX_E_UNSUPPORTED
        m.close()
    m = AuxKalman(wl, dtype="f32", mode="cached")
    with pytest.raises(B.AuxError) as e:
        B.aux_batch_create([m.handle, m.handle], [x, x])
    assert e.value.code == B.AUX_E_INVALID_ARG
    m.close()


def test_batch_rejects_a_nonfinite_chain_and_steps_the_others():
    wls = _mixed_workloads()[:3]
    models, xs = _make(wls, "cached")
    xs[2][1, 5, 4] = float("nan")
    x0 = [x.cpu().numpy() for x in xs]
    b = AuxBatch(models, xs)
    acc = torch.zeros(sum(wl.n_chains for wl in wls), dtype=torch.int32, device="cuda")
    b.step(4, accept_count=acc)
    torch.cuda.synchronize()
    rc, aborted = b.status()
    assert aborted == 0 and rc != 0
    rc2, per = models[2].status()
    assert per[1] != 0 and per[0] == 0
    xn = xs[2].cpu().numpy()
    assert np.array_equal(np.nan_to_num(xn[1]), np.nan_to_num(x0[2][1]))   # never accepted
    assert acc.cpu().numpy()[-1] == 0 and acc.cpu().numpy()[:-1].sum() > 0
    b.close()
    for m in models:
        m.close()

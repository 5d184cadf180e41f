"""CUDA-graph replay of MCMC iterations (aux_set_device_iteration).

With the iteration index kept on the device, n MCMC iterations captured once
and replayed k times must be, bit for bit, the k*n iterations that eager
aux_kalman_step calls with successive iter0 produce: the Philox streams are
keyed by the same (seed, chain, iteration) and the launches are the same.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_00301_gb300 import MODES, AuxKalman, workloads  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_00301_gb300 import build
    build.build()


def _tt(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _eager_and_replayed(wl, dt, L, mode="per_chain", proposal=1, adapt=False, n=3, reps=3, **kw):
    tdt = torch.float64 if dt == "f64" else torch.float32
    C = wl.n_chains
    out = []
    for graph in (False, True):
        s = AuxKalman(wl, dtype=dt, block_len=L, mode=mode, proposal=proposal, **kw)
        if adapt:
            s.adapt_delta(True, target=0.5, gain=1.0)
        x = _tt(wl.x_init, tdt)
        acc = torch.zeros(C, dtype=torch.int32, device="cuda")
        la = torch.zeros(C, dtype=torch.float64, device="cuda")
        if not graph:
            s.step(x, 1, 0, acc)                       # the warm-up iteration of the graph run
            for k in range(reps):
                s.step(x, n, 1 + k * n, acc, la)
        else:
            s.device_iteration(True, 0)
            s.step(x, 1, 12345, acc)                   # iter0 is ignored: the counter says 0
            g = s.capture(x, n, acc, la)
            for _ in range(reps):
                g.replay()
        torch.cuda.synchronize()
        it = s.iteration() if graph else None
        out.append((x.clone(), acc.clone(), la.clone(), s.delta(), it))
        s.close()
    return out


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_replayed_iterations_equal_eager_iterations(dt, mode):
    wl = workloads.stochastic_volatility(d=6, T=45, n_chains=3, delta=0.05)
    (xa, aa, la, _, _), (xb, ab, lb, _, itb) = _eager_and_replayed(wl, dt, 9, mode)
    assert torch.equal(xa, xb)
    assert torch.equal(aa, ab)
    assert torch.equal(la, lb)
    assert itb == 1 + 3 * 3


def test_replay_second_order_per_chain():
    wl = workloads.stochastic_volatility(d=4, T=30, n_chains=2, delta=0.2)
    (xa, aa, la, _, _), (xb, ab, lb, _, _) = _eager_and_replayed(wl, "f32", 6, proposal=2)
    assert torch.equal(xa, xb) and torch.equal(aa, ab) and torch.equal(la, lb)


@pytest.mark.parametrize("mode", ["per_chain", "cached"])
def test_replay_with_delta_adaptation(mode):
    wl = workloads.stochastic_volatility(d=5, T=40, n_chains=4, delta=0.5)
    (xa, aa, la, da, _), (xb, ab, lb, db, _) = _eager_and_replayed(wl, "f64", 8, mode, adapt=True)
    assert torch.equal(xa, xb) and torch.equal(aa, ab) and torch.equal(la, lb)
    assert da == db and da != 0.5


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_replay_factorised_path(dt):
    wl = workloads.spatio_temporal(side=3, T=24, n_chains=2, delta=0.3)
    (xa, aa, la, _, _), (xb, ab, lb, _, itb) = _eager_and_replayed(wl, dt, 6)
    assert torch.equal(xa, xb) and torch.equal(aa, ab) and torch.equal(la, lb)
    assert itb == 10


@pytest.mark.parametrize("mode", MODES)
def test_replay_with_the_bridging_sampler(mode):
    wl = workloads.stochastic_volatility(d=5, T=37, n_chains=3, delta=0.05)
    (xa, aa, la, _, _), (xb, ab, lb, _, _) = _eager_and_replayed(wl, "f32", 6, mode, sampler="bridging")
    assert torch.equal(xa, xb) and torch.equal(aa, ab) and torch.equal(la, lb)


def test_replay_with_the_square_root_filter():
    wl = workloads.stochastic_volatility(d=4, T=30, n_chains=2, delta=0.05)
    (xa, aa, la, _, _), (xb, ab, lb, _, _) = _eager_and_replayed(wl, "f32", 5, filter_form="square_root")
    assert torch.equal(xa, xb) and torch.equal(aa, ab) and torch.equal(la, lb)


@pytest.mark.parametrize("mode", ["shared", "cached"])
def test_replay_with_square_root_tables(mode):
    wl = workloads.stochastic_volatility(d=6, T=45, n_chains=3, delta=0.05)
    (xe, ae, le, _, _), (xg, ag, lg, _, it) = _eager_and_replayed(wl, "f32", 8, mode=mode,
                                                                   filter_form="square_root")
    assert torch.equal(xe, xg) and torch.equal(ae, ag) and torch.equal(le, lg) and it == 10


@pytest.mark.parametrize("mode", ["shared", "cached"])
def test_replay_on_the_wide_kernels(mode):
    """d = 40 (padded to 64) and d = 72 (to 128), with and without delta adaptation."""
    for d, adapt in ((40, False), (72, True)):
        wl = workloads.stochastic_volatility(d=d, T=30, n_chains=3, delta=0.02)
        (xe, ae, le, de, _), (xg, ag, lg, dg, it) = _eager_and_replayed(wl, "f32", 6, mode=mode, adapt=adapt)
        assert torch.equal(xe, xg) and torch.equal(ae, ag) and torch.equal(le, lg) and it == 10
        assert de == dg


def test_counter_can_be_reset_and_disabled():
    wl = workloads.stochastic_volatility(d=3, T=16, n_chains=2, delta=0.05)
    s = AuxKalman(wl, dtype="f64", block_len=4)
    x = _tt(wl.x_init, torch.float64)
    s.device_iteration(True, 40)
    s.step(x, 5, 0)
    assert s.iteration() == 45
    s.device_iteration(False)
    s.step(x, 2, 0)                                    # eager indices again: counter untouched
    assert s.iteration() == 45
    s.close()

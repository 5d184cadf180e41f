"""Pick the step size delta of an SV workload with the oracle (run once, offline).

TEST INFRASTRUCTURE: writes no library code; the value it prints is frozen
into the workload table by hand and recorded with the run that produced it.

The paper tunes delta to a target acceptance rate without stating the rule
(Section 4, experiments preamble). This script uses a Robbins-Monro
recursion on log delta, log delta <- log delta + c k^{-0.6} (a_k - target),
with a_k = min(1, exp(log alpha_k)) from the oracle's own MH steps, and
reports the mean of delta over the second half of the run.
run_chains_adaptive is the same rule on line for chains that share delta
(a_k pooled over the chains): the reference of the library's on-device
adaptation (aux_set_delta_adaptation).

usage: python -m oracle.calibrate_delta D T [n_iters] [target]
"""
import sys
import time

import numpy as np

from . import mcmc


def calibrate(wl_model, x0, delta0, n_iters, target=0.5, seed=1, c=1.0):
    log_d = np.log(delta0)
    x = np.array(x0)
    hist = []
    acc = []
    for k in range(n_iters):
        delta = float(np.exp(log_d))
        st = mcmc.aux_step_philox(x, wl_model, delta, seed, 0, k)
        a = float(np.exp(min(0.0, st["log_alpha"])))
        acc.append(a)
        x = st["x_new"]
        log_d += c * (k + 1) ** -0.6 * (a - target)
        hist.append(np.exp(log_d))
    half = n_iters // 2
    return float(np.mean(hist[half:])), float(np.mean(acc[half:]))


def run_chains_adaptive(x0, model, delta0, n_iters, target=0.5, c=1.0, seed=1, order=1, iter0=0,
                        sampler="rts"):
    """Chains that share one delta adapted on line by the rule of `calibrate`,
    with a_k the mean over the chains of min(1, exp(log alpha_k)) (a
    non-finite log alpha counts as 0). Step k of every chain uses the delta
    of step k; chain c draws the library's Philox streams (seed, c, iter0 + k).

    Returns (x [C, T, d], deltas [n_iters + 1], log_alphas [n_iters, C])."""
    x = np.array(x0, dtype=np.float64)
    C = x.shape[0]
    log_d = np.log(delta0)
    deltas = [float(np.exp(log_d))]
    las = np.zeros((n_iters, C))
    for k in range(n_iters):
        delta = float(np.exp(log_d))
        acc = 0.0
        for ch in range(C):
            st = mcmc.aux_step_philox(x[ch], model, delta, seed, ch, iter0 + k, order=order, sampler=sampler)
            x[ch] = st["x_new"]
            las[k, ch] = st["log_alpha"]
            acc += float(np.exp(min(0.0, st["log_alpha"]))) if np.isfinite(st["log_alpha"]) else 0.0
        log_d += c * (k + 1) ** -0.6 * (acc / C - target)
        deltas.append(float(np.exp(log_d)))
    return x, np.array(deltas), las


def main(argv):
    from paper_2303_00301_gb300 import workloads
    d, T = int(argv[0]), int(argv[1])
    n_iters = int(argv[2]) if len(argv) > 2 else 300
    target = float(argv[3]) if len(argv) > 3 else 0.5
    wl = workloads.stochastic_volatility(d=d, T=T, n_chains=1, delta=0.05)
    model = dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q,
                 emission=mcmc.SVEmission(wl.y))
    t0 = time.time()
    delta, acc = calibrate(model, wl.x_init[0], 0.05 * (30.0 * 1024 / (d * T)) ** 0.5,
                           n_iters, target)
    print(f"d={d} T={T} delta={delta:.6g} mean_accept_second_half={acc:.3f} "
          f"iters={n_iters} wall_s={time.time() - t0:.1f}")


if __name__ == "__main__":
    main(sys.argv[1:])

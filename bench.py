#!/usr/bin/env python
"""Throughput of the auxiliary Kalman sampler on GB300: chain·timesteps/s.

Workload (default): multivariate stochastic-volatility model, d_x = 30,
T = 1024, 32 chains, FP32, delta = 0.0183 (oracle-calibrated, ~50%
acceptance), seeded synthetic data. One step = one auxiliary Kalman MH
iteration (linearise, parallel filter, backward sampling scan, reverse filter,
MH test) on all chains. The sampler state and data are resident in HBM when
the timed region starts; L2 is flushed (256 MiB write) before every timed step.

The headline mode (--mode, default "shared") recomputes the covariance half of
the scan once per step for all chains, then runs the per-chain means; the JSON
line also reports the "per_chain" mode (every chain runs the full element
scan: the general path) and the "cached" mode (covariance tables kept across
steps), each with its own roofline line, and ESS / ESJD from a long run.

--impl reference times the FP64 CPU oracle (the only other implementation of
the method here) on the host cores on bounded samples of the same workload.
Under torchrun every rank runs an independent replica (weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "aux-Kalman chain·timesteps/s at d_x=30,T=1024"
UNIT = "chain·timesteps/s"
WORKLOADS = {
    "sv_d30_T1024": dict(kind="sv", d=30, T=1024, C=32, dtype="f32"),
    "lg_d2_T64": dict(kind="lg", d=2, T=64, C=1, dtype="f64"),
}
FP32_LANES_PER_SM = 128
_DEVICE_CAPS = {}


def device_caps(peaks):
    """(multiprocessor count, maximum SM clock in MHz, where the clock came from) of
    the current device: the SM count from the device properties, the clock from
    nvidia-smi's clocks.max.sm, else the measured peaks file."""
    if not _DEVICE_CAPS:
        import torch
        dev = torch.cuda.current_device()
        _DEVICE_CAPS["n_sm"] = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz, src = None, None
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(dev), "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                 timeout=20).stdout.strip()
            mhz, src = float(out.splitlines()[0]), "nvidia-smi clocks.max.sm"
        except Exception:
            pass
        if mhz is None:
            mhz, src = float(peaks.get("sm_max_mhz", 2070.0)), "MEASURED_PEAKS.json sm_max_mhz"
        _DEVICE_CAPS["sm_max_mhz"], _DEVICE_CAPS["clock_source"] = mhz, src
    return _DEVICE_CAPS["n_sm"], _DEVICE_CAPS["sm_max_mhz"], _DEVICE_CAPS["clock_source"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sv_d30_T1024", choices=sorted(WORKLOADS))
    ap.add_argument("--block-len", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="shared", choices=["per_chain", "shared", "cached"],
                    help="execution mode of the headline number (aux_set_mode)")
    ap.add_argument("--sampler", default="scan", choices=["scan", "bridging"],
                    help="pathwise sampler of the headline mode (aux_set_sampler)")
    ap.add_argument("--filter-form", default="covariance", choices=["covariance", "square_root"],
                    help="filter form of the headline mode (aux_set_filter_form)")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the measurements of the other execution modes")
    ap.add_argument("--ess-iters", type=int, default=5000,
                    help="post-burn-in iterations of the ESS / ESJD run (0 = skip)")
    ap.add_argument("--ess-burn", type=int, default=500)
    ap.add_argument("--spatial-only", action="store_true",
                    help="run only the lattice-model line (Section 4.2) and print it")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched multi-instance line and print it")
    ap.add_argument("--wide-only", action="store_true",
                    help="run only the d = 128 line (wide kernels) and print it")
    ap.add_argument("--batched-quick", action="store_true",
                    help="batched line: the full batch in cached mode only (no subset, shared mode or "
                         "per-instance comparison; for profiling)")
    ap.add_argument("--batched-instances", type=int, default=256,
                    help="instances of the batched line (256: the full mix; fewer for profiling)")
    ap.add_argument("--wide-T", type=int, default=4096, help="T of the d = 128 line")
    ap.add_argument("--wide-L", type=int, default=0, help="block length of the d = 128 line (0: default)")
    ap.add_argument("--wide-adapt", type=int, default=150,
                    help="delta adaptation steps before the d = 128 line is timed (0: the workload's delta)")
    ap.add_argument("--cpu-sample-chains", type=int, default=0,
                    help="chain-steps in the CPU baseline sample (0 = 2 per core)")
    return ap.parse_args()


def max_over_ranks(value, device, world):
    """The maximum of a float over all ranks of the process group (the value
    itself on one rank): the bench reports the slowest replica's time."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def make_workload(name, rank=0):
    from paper_2303_00301_gb300 import workloads
    w = WORKLOADS[name]
    if w["kind"] == "sv":
        wl = workloads.stochastic_volatility(d=w["d"], T=w["T"], n_chains=w["C"], mcmc_seed=1 + rank)
    else:
        wl = workloads.linear_gaussian(d=w["d"], T=w["T"], n_chains=w["C"], mcmc_seed=1 + rank)
    return wl, w


# --------------------------------------------------------------------------- flops model
# Algorithmic flops in the unpadded dimension d (2 per multiply-add): a dense
# d x d product is 2 d^3, a triangular solve with d right-hand sides or a
# triangular x dense product d^3, a Cholesky factorisation d^3 / 3, a
# matrix-vector product 2 d^2. With a diagonal F (the SV model) the products
# F C, F C F^T, F A and F P^f are O(d^2) and counted as such.
def combine_flops(d):
    """Element operator, Cholesky form: 2 Cholesky, 2 triangular x dense, 1
    triangular solve with d right-hand sides, 8 dense products, 9 mat-vec."""
    return (59.0 / 3.0) * d ** 3 + 18.0 * d ** 2


def matrix_combine_flops(d):
    """Matrix part (A, C, J) of the element operator, Cholesky form: Cholesky of C_i
    and of N = I + U^T J_j U, one triangular solve with d right-hand sides, ten
    dense products."""
    return (2.0 / 3.0 + 1.0 + 20.0) * d ** 3


def conly_flops(d):
    """C part of prefix (x) E for a prefix with A = J = 0: two Cholesky, one triangular
    solve, four dense products (J U, U^T J U, A B, P P^T)."""
    return (2.0 / 3.0 + 1.0 + 8.0) * d ** 3


def cov2_tables_flops_per_step(d, fdiag):
    """Per-step tables from P^f_(t-1), P^f_t: Cholesky of S_t, W = L^{-1} (triangular
    solve with d right-hand sides), K' = r W^T W; Cholesky of P^p_(t+1),
    Y = L^{-1} F P^f_t, Sigma = P^f_t - Y^T Y, G by a triangular solve, Cholesky of
    Sigma; a dense F adds F P^f F^T twice and F P^f (five products)."""
    return (1.0 / 3 + 1 + 2 + 1.0 / 3 + 1 + 2 + 1 + 1.0 / 3) * d ** 3 + (0.0 if fdiag else 10.0 * d ** 3)


def reduce_flops_per_step(d, fdiag):
    """Conditional Kalman step: Cholesky of S, 2 triangular solves (Y, W), 3 products
    (Y^T Y, Y^T W, W^T W); with a dense F also F C, (F C) F^T and F A."""
    f = (1.0 / 3.0 + 2 + 6) * d ** 3 + 7 * d ** 2
    return f + (0.0 if fdiag else 6.0 * d ** 3) + (3 * d ** 2 if fdiag else 0.0)


def apply_flops_per_step(d, epilogue, fdiag):
    """In-block Kalman step: Cholesky of S, 1 triangular solve, P^f downdate; with the
    backward-element epilogue also the Cholesky of P^p and Sigma, a forward and a
    backward triangular solve, the Sigma downdate and the running G product; with a
    dense F the prediction F P^f F^T (two products)."""
    f = (1.0 / 3.0 + 1 + 2) * d ** 3 + 5 * d ** 2
    if epilogue:
        f += (1.0 / 3.0 + 1 + 2 + 1 + 1.0 / 3.0 + 2) * d ** 3 + 6 * d ** 2
    return f + (0.0 if fdiag else 4.0 * d ** 3) + (3 * d ** 2 if fdiag else 0.0)


def cov_apply_flops_per_step(d, fdiag):
    """Covariance pass, in-block step: the apply step with the epilogue, the
    inverse Cholesky factor W_t = chol(S_t)^{-1}, M_t = r W^T W F (triangular
    product) and the running products M_t AH and G prefix (two dense products)."""
    return apply_flops_per_step(d, True, fdiag) + (1.0 / 3.0 + 1.0 + 4.0) * d ** 3


def means_flops_per_step(kind, d, fdiag, epilogue=True):
    """Per chain-timestep flops of the means kernels: dense mat-vec 2 d^2,
    triangular mat-vec d^2. reduce/apply: K' e (+ F m); apply with the epilogue
    also G m^p, chol(Sigma) eps (triangular) and the block prefix product."""
    fm = 2.0 * d if fdiag else 2.0 * d ** 2
    if kind == "reduce":
        return 2.0 * d ** 2 + fm
    return 2.0 * d ** 2 + fm + ((2.0 + 1.0 + 2.0) * d ** 2 if epilogue else 0.0)


def bridge_tree_shape(T):
    """(levels J, internal nodes NN) of the dyadic tree over T - 1 unit intervals."""
    cnt, levels, nodes = T - 1, 0, 0
    while cnt > 1:
        cnt = (cnt + 1) // 2
        levels += 1
        nodes += cnt
    return levels, nodes


def kernel_work(mode, kind, w, d, T, C, nb, nbc, fdiag, esz):
    """Algorithmic work of one launch of a kernel kind, averaged over the launches
    of one MH step: (flops, HBM bytes). Bytes count what the algorithm must move
    (unpadded d): tables once, per-chain vectors once; None where not modelled."""
    vec = C * T * d * esz
    tab = T * d * d * esz
    if mode == "per_chain_sqrt":
        # square-root form: one operator per step in the reduction (29.3 d^3: 12 products,
        # 2 Cholesky of I + W W^T, 4 triangular solves, 2 Householder triangularisations
        # of d x 2d at 3.3 d^3); the in-block step 17.3 d^3 (3 products, 2 triangular
        # solves with d right-hand sides, Cholesky of S, 2 triangularisations), and the
        # backward-element epilogue 17.7 d^3 in the forward pass only
        if kind == "reduce":
            return C * T * 29.3 * d ** 3, None
        if kind == "apply":
            return C * T * (17.3 * 2 + 17.7) * d ** 3 / 2, None
        return None, None
    if mode == "per_chain":
        if kind == "reduce":
            return C * T * reduce_flops_per_step(d, fdiag), None
        if kind == "apply":
            return C * T * (apply_flops_per_step(d, True, fdiag) +
                            apply_flops_per_step(d, False, fdiag)) / 2, None
        return None, None
    if kind == "reduce":   # forward (linearise: x, y in; u, v, ytilde out) and reverse (ytilde* in)
        return (C * T * means_flops_per_step("reduce", d, fdiag),
                tab + (5 * vec + vec) / 2)
    if kind == "apply":    # forward (4 tables, ytilde in, U out) and reverse (1 table, ytilde* in)
        return (C * T * (means_flops_per_step("apply", d, fdiag, True) +
                         means_flops_per_step("apply", d, fdiag, False)) / 2,
                (4 * tab + 2 * vec + tab + vec) / 2)
    if kind == "backward":  # G table, U in, x* out, MH inputs x, u, v, y in, ytilde* out (2 launches)
        return C * T * 2.0 * d ** 2 / 2, (tab + 7 * vec) / 2
    if kind == "bridge":
        # divide-and-conquer sampler, 2 launches per step: node offsets up the tree
        # (E_l once per node; g_l, g_r in, g out per chain-node; 2 d^2), the two ends, the
        # split points down the tree (G, Gamma, chol V once per node; x_k, x_m, g, g_r in,
        # x_l out per chain-node; 5 d^2) and the MH terms (x*, x, u, v, y in, ytilde* out)
        levels, nodes = bridge_tree_shape(T)
        byt = (4 * nodes * d * d + 8 * C * nodes * d) * esz + 6 * vec
        return C * nodes * 7.0 * d ** 2 / 2, byt / 2   # k_b_sample + k_b_mh
    if kind == "bridge_tree":
        # leaf covariances LS LS^T (d^3 per step) and, per node, E_l L_r, E_l E_r,
        # T1 E_l^T, chol(L), G by two triangular solves, Gamma, V and chol(V)
        levels, nodes = bridge_tree_shape(T)
        return ((T - 1) * d ** 3 + nodes * (6 + 1.0 / 3 + 2 + 4 + 1.0 / 3) * d ** 3) / (levels + 1), None
    Lc = (T + nbc - 1) // nbc
    ragged = nbc >= 3 and T % Lc != 0
    if mode == "table_sqrt" and kind in ("cov_reduce", "cov_scan", "cov_apply"):
        # the covariance pass on factors: one square-root operator (29.3 d^3, as above)
        # per element folded and per prefix; the in-block step 17.3 d^3, its epilogue
        # 17.7 d^3, P^f = U U^T (d^3), M_t = K' F and the two running products (6 d^3)
        n_end = nbc - 1 if ragged else nbc
        levels = max(0, math.ceil(math.log2(n_end))) if n_end > 1 else 0
        if kind == "cov_reduce":
            return min(nbc, 3 if ragged else 2) * Lc * 29.3 * d ** 3, None
        if kind == "cov_scan":
            combines = (n_end - 1) + max(0, levels - 1) + (1 if ragged else 0)
            return combines * 29.3 * d ** 3 / max(1, levels + (1 if ragged else 0)), None
        return T * (17.3 + 17.7 + 1 + 6) * d ** 3, None
    # covariance form (aux_cov2.cuh): prefixes by doubling over the steps
    if kind == "cov_reduce":
        # P^f_0 (Cholesky of S0, one triangular solve, Y^T Y) and the shared element E
        # (Cholesky of S, two triangular solves, Y^T Y, Y^T V, V^T V)
        return (1.0 / 3 + 1 + 2 + 1.0 / 3 + 2 + 6) * d ** 3, None
    if kind == "cov_scan":
        # T - 1 prefix operators (C part only) and one power per level but the last,
        # averaged over the ceil(log2 T) level launches
        levels = max(0, math.ceil(math.log2(T))) if T > 1 else 0
        if levels == 0:
            return None, None
        return ((T - 1) * conly_flops(d) + (levels - 1) * matrix_combine_flops(d)) / levels, None
    if kind == "cov_apply":
        return T * cov2_tables_flops_per_step(d, fdiag), None
    if kind == "cov_products":
        # one product per step in the G chain and one in the M chain (M_t = K'_t F: one more
        # product with a dense F)
        return T * (4.0 + (0.0 if fdiag else 2.0)) * d ** 3, None
    return None, None


KERNEL_NAMES = {
    "per_chain": {"reduce": "k_filter_reduce", "apply": "k_filter_apply", "scan": "k_filter_scan_level",
                  "backward": "k_sample_backward", "mh": "k_mh + k_commit", "linearise": "k_linearise"},
    "per_chain_sqrt": {"reduce": "k_sr_reduce", "apply": "k_sr_apply", "scan": "k_sr_scan_level",
                       "backward": "k_sample_backward", "mh": "k_mh + k_commit", "linearise": "k_linearise"},
    "table": {"reduce": "k_mf_reduce", "apply": "k_mf_apply", "scan": "k_mean_cross2",
              "backward": "k_mean_cross2 + k_mb_apply", "mh": "k_mh + k_commit",
              "cov_reduce": "k_c2_init", "cov_scan": "k_c2_level",
              "cov_apply": "k_c2_tables", "cov_products": "k_c2_products + k_cov_xprod",
              "bridge": "k_b_sample + k_b_mh", "bridge_tree": "k_br_leaf + k_br_node"},
}


KERNEL_NAMES["table_sqrt"] = dict(KERNEL_NAMES["table"], cov_reduce="k_srcov_reduce",
                                  cov_scan="k_srcov_scan_double", cov_apply="k_srcov_apply",
                                  cov_products="k_cov_products + k_cov_gp_fix")


def source_hash():
    """sha256 over the library sources (csrc/*.cu*, csrc/*.h, include/*.h)."""
    import glob
    import hashlib
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2303_00301_gb300", "csrc", "*.cu*")) +
                   glob.glob(os.path.join(ROOT, "paper_2303_00301_gb300", "csrc", "*.h")) +
                   glob.glob(os.path.join(ROOT, "include", "*.h")))
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()


def dram_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when
    the library sources changed since that capture (profiles/dram_traffic.json)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != source_hash():
        return None
    return rec.get("dram_bytes_per_launch", {}).get(kernel)


def roofline_line(mode, kind, prof, w, d, T, C, nb, nbc, fdiag, esz, peaks, steps, path):
    """One roofline line for kernel kind `kind` from the per-launch event times."""
    if kind not in prof or not prof[kind][1]:
        return None
    ms, launches = prof[kind]
    avg_ms = ms / launches
    flops, bytes_ = kernel_work(mode, kind, w, d, T, C, nb, nbc, fdiag, esz)
    name = KERNEL_NAMES[mode if mode in ("per_chain", "per_chain_sqrt", "table_sqrt") else "table"].get(kind, kind)
    line = {"path": path, "kernel": name, "launches": launches, "avg_launch_ms": avg_ms}
    if bytes_ is not None and "hbm_gbs" in peaks:
        achieved = bytes_ / (avg_ms / 1e3) / 1e9
        line.update({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": dram_traffic(name),
                     "bytes_per_launch": bytes_, "peak_basis": "measured HBM copy bandwidth"})
        if flops is not None:
            line["flops_per_launch"] = flops
        return line
    if flops is None:
        return None
    if w["dtype"] == "f32":
        n_sm, sm_max, src = device_caps(peaks)
        peak = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        basis = (f"{n_sm} SMs (device properties) x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                 f"{sm_max:.0f} MHz ({src})")
    else:
        peak = 1.25
        basis = "nominal GB300 FP64 rate"
    achieved = flops / (avg_ms / 1e3) / 1e12
    line.update({"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                 "frac": achieved / peak, "traffic": dram_traffic(name), "flops_per_launch": flops,
                 "diagonal_F": fdiag, "peak_basis": basis})
    return line


# --------------------------------------------------------------------------- ESS
def geyer_ess(x):
    """Effective sample size of a 1-D series by Geyer's initial monotone sequence
    estimator (sums of consecutive autocorrelation pairs, truncated at the first
    non-positive pair and made monotone)."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    xc = x - x.mean()
    var = xc.var()
    if n < 4 or var <= 0:
        return float(n)
    f = np.fft.rfft(xc, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n] / (n * var)
    pairs = acf[: (n // 2) * 2].reshape(-1, 2).sum(axis=1)
    pos = np.where(pairs <= 0)[0]
    m = pos[0] if pos.size else pairs.size
    gam = np.minimum.accumulate(pairs[:m]) if m > 0 else np.zeros(0)
    tau = -1.0 + 2.0 * gam.sum()
    return float(n / max(tau, 1e-12))


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        out_dir = os.environ.get("AUX_BENCH_CLOCK_DIR")   # keep the raw samples there when set
        if out_dir and os.path.isdir(out_dir):
            self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")
        else:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv", prefix="clocks_")
            os.close(fd)

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts once the sampler is producing rows; the rows
        # taken before it are left out of the summary
        t0 = time.time()
        self.skip = 0
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            with open(self.path) as f:
                self.skip = f.read().count("\n")
            if self.skip >= 1:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.out.close()
        out = open(self.path).read()
        rows = [r.split(",") for r in (out or "").strip().splitlines() if r.count(",") >= 8]
        if len(rows) > self.skip:
            rows = rows[self.skip:]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- CPU oracle
def _oracle_chain_step(args):
    import numpy as np  # noqa: F401
    from oracle import mcmc
    name, chain, it = args
    wl, _ = make_workload(name)
    if wl.emission == 1:
        em = mcmc.SVEmission(wl.y, wl.mask)
    else:
        em = mcmc.LinearGaussianEmission(wl.y, wl.Ry, wl.mask)
    model = dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)
    t0 = time.perf_counter()
    mcmc.aux_step_philox(wl.x_init[chain % wl.n_chains], model, wl.delta, wl.mcmc_seed, chain, it)
    return time.perf_counter() - t0


def _oracle_replay(args):
    """One oracle step of chain `chain` at iteration `it` from the GPU's state x_before:
    (log alpha, accepted, x*, smoothing sd of x*)."""
    from oracle import kalman, mcmc
    name, chain, it, x_before = args
    wl, _ = make_workload(name)
    em = mcmc.SVEmission(wl.y, wl.mask) if wl.emission == 1 else \
        mcmc.LinearGaussianEmission(wl.y, wl.Ry, wl.mask)
    model = dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=em)
    ref = mcmc.aux_step_philox(x_before, model, wl.delta, wl.mcmc_seed, chain, it)
    _, Ps = kalman.rts_smoother(ref["kf"], wl.F)
    import numpy as np
    sd = np.sqrt(np.maximum(np.einsum("tii->ti", Ps), 0.0))
    return ref["log_alpha"], ref["accepted"], ref["x_star"], sd


def _oracle_wide_step(args):
    """The oracle's step of chain `chain` (iteration 0, from the workload's initial state)
    on the d = 128 SV workload with step size delta, with everything the error report of
    the wide line compares: log alpha, the decision, ytilde, log Z, m^f and its sd, x* and
    its smoothing sd."""
    import numpy as np
    from oracle import kalman, mcmc
    d, T, C, delta, chain = args
    from paper_2303_00301_gb300 import workloads as W
    wl = W.stochastic_volatility(d=d, T=T, n_chains=C, delta=delta)
    model = dict(m0=wl.m0, P0=wl.P0, F=wl.F, b=wl.b, Q=wl.Q, emission=mcmc.SVEmission(wl.y, wl.mask))
    ref = mcmc.aux_step_philox(wl.x_init[chain], model, wl.delta, wl.mcmc_seed, chain, 0)
    kf = ref["kf"]
    _, Ps = kalman.rts_smoother(kf, wl.F)
    sd = lambda P: np.sqrt(np.maximum(np.einsum("tii->ti", P), 0.0))
    return dict(log_alpha=ref["log_alpha"], accepted=ref["accepted"], ytilde=ref["ytilde"],
                logZ=kf["logZ"], mf=kf["mf"], sd_f=sd(kf["Pf"]), x_star=ref["x_star"], sd_s=sd(Ps))


def wide_error_block(refs, wl, dtype, delta, chains):
    """Errors of one dtype's wide path against the FP64 oracle on sampled chains: the
    step's |d log alpha| and MH decision (iteration 0 from the initial state), log Z and
    m^f of aux_loglik on the oracle's ytilde, and x* of aux_sample_path on the same ytilde
    with the step's backward noise; element-wise errors scaled by (|oracle| + sd)."""
    import numpy as np
    import torch
    from oracle import philox
    from paper_2303_00301_gb300 import AuxKalman
    from paper_2303_00301_gb300 import workloads as W
    C, T, d = wl.n_chains, wl.T, wl.d
    ws = W.stochastic_volatility(d=d, T=T, n_chains=C, delta=delta)
    h = AuxKalman(ws, dtype=dtype, mode="cached")
    x = torch.tensor(ws.x_init, dtype=torch.float32, device="cuda")
    la = torch.zeros(C, dtype=torch.float64, device="cuda")
    h.step(x, 1, iter0=0, log_alpha=la)
    yt = np.zeros((C, T, d))
    for c in chains:
        yt[c] = refs[c]["ytilde"]
    ytg = torch.tensor(yt, dtype=torch.float32, device="cuda")
    logZ = torch.zeros(C, dtype=torch.float64, device="cuda")
    mf = torch.zeros((C, T, d), dtype=torch.float32, device="cuda")
    h.loglik(ytg, logZ, mf)
    xs = torch.zeros((C, T, d), dtype=torch.float32, device="cuda")
    h.sample_path(ytg, xs, eps=None, iteration=0)
    torch.cuda.synchronize()
    rc = h.status()[0]
    h.close()
    lag, lzg, mfg, xsg = la.cpu().numpy(), logZ.cpu().numpy(), mf.double().cpu().numpy(), xs.double().cpu().numpy()
    out = {"dla": [], "logZ_rel": [], "mf_elem": [], "x_star_elem": [], "decision_mismatches": 0}
    for c in chains:
        r = refs[c]
        out["dla"].append(abs(lag[c] - r["log_alpha"]))
        lu = float(np.log(philox.mh_uniform(ws.mcmc_seed, c, 0)))
        if bool(lu < lag[c]) != bool(r["accepted"]):
            out["decision_mismatches"] += 1
        out["logZ_rel"].append(abs(lzg[c] - r["logZ"]) / abs(r["logZ"]))
        out["mf_elem"].append(float(np.max(np.abs(mfg[c] - r["mf"]) / (np.abs(r["mf"]) + r["sd_f"]))))
        out["x_star_elem"].append(float(np.max(np.abs(xsg[c] - r["x_star"]) / (np.abs(r["x_star"]) + r["sd_s"]))))
    return {"against": "FP64 oracle (iteration 0 from the initial state; aux_loglik and aux_sample_path "
                       "on the oracle's ytilde with the step's backward noise)",
            "chains": list(chains), "status": int(rc),
            "abs_dlog_alpha_max": float(max(out["dla"])), "mh_decision_mismatches": out["decision_mismatches"],
            "logZ_rel_max": float(max(out["logZ_rel"])),
            "mf_max_err_over_abs_plus_sd": float(max(out["mf_elem"])),
            "x_star_max_err_over_abs_plus_sd": float(max(out["x_star_elem"]))}


def fp32_error_block(name, wl, w, mode, block_len, pool, chains=(0, 9, 22, 31), steps=16):
    """Error of the FP32 GPU path against the FP64 oracle on sampled chains: each GPU
    step is replayed on the oracle from the GPU's state before it, on the same Philox
    draws. Reports the |d log alpha| distribution, MH-decision mismatches (with the
    near-tie band), and the element-wise error of accepted x* scaled by
    (|x*_oracle| + smoothing sd)."""
    import numpy as np
    import torch
    from oracle import philox
    from paper_2303_00301_gb300 import AuxKalman
    tdt = torch.float32 if w["dtype"] == "f32" else torch.float64
    chains = [c for c in chains if c < w["C"]]
    s = AuxKalman(wl, dtype=w["dtype"], block_len=block_len, mode=mode)
    x = torch.tensor(wl.x_init, dtype=tdt, device="cuda")
    la = torch.zeros(w["C"], dtype=torch.float64, device="cuda")
    jobs, gpu = [], []
    for it in range(steps):
        xb = x.double().cpu().numpy()
        s.step(x, 1, iter0=it, log_alpha=la)
        torch.cuda.synchronize()
        xa, lag = x.double().cpu().numpy(), la.cpu().numpy()
        for c in chains:
            jobs.append((name, c, it, xb[c]))
            gpu.append((lag[c], xa[c], xb[c]))
    s.close()
    refs = pool.map(_oracle_replay, jobs, chunksize=1)
    band = 2e-3
    dla, mism, near, xerr = [], 0, 0, 0.0
    for (nm, c, it, _), (lg, xa, xb), (lr, acc, xs, sd) in zip(jobs, gpu, refs):
        dla.append(abs(lg - lr))
        lu = float(np.log(philox.mh_uniform(wl.mcmc_seed, c, it)))
        if abs(lr - lu) < band:
            near += 1
        if bool(lu < lg) != bool(acc):
            mism += 1
        elif acc:
            xerr = max(xerr, float(np.max(np.abs(xa - xs) / (np.abs(xs) + sd))))
    a = np.asarray(dla)
    return {"mode": mode, "chains": list(chains), "steps": steps, "chain_steps": len(dla),
            "against": "FP64 oracle, same Philox draws, each step from the GPU's state",
            "abs_dlog_alpha": {"p50": float(np.percentile(a, 50)), "p90": float(np.percentile(a, 90)),
                               "p99": float(np.percentile(a, 99)), "max": float(a.max())},
            "mh_decision_mismatches": mism, "near_ties_within_band": near, "near_tie_band": band,
            "x_star_max_err_over_abs_plus_sd": xerr}


def cpu_oracle_rate(name, n_chain_steps, pool, cores, it0=0):
    """chain·timesteps/s of the oracle on `cores` processes over n_chain_steps chain-steps."""
    _, w = make_workload(name)
    t0 = time.perf_counter()
    pool.map(_oracle_chain_step, [(name, c, it0 + c) for c in range(n_chain_steps)], chunksize=1)
    wall = time.perf_counter() - t0
    return n_chain_steps * w["T"] / wall, wall


def _cpu_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def run_reference(args):
    """The oracle arm: same metric/config, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    _cpu_env()
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    name = args.workload
    _, w = make_workload(name)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for k in range(args.warmup):
            cpu_oracle_rate(name, cores, pool, cores, it0=k * cores)
        rates, walls = [], []
        for k in range(args.steps):
            r, wall = cpu_oracle_rate(name, cores, pool, cores, it0=(args.warmup + k) * cores)
            rates.append(r)
            walls.append(wall)
    value = len(rates) * cores * w["T"] / sum(walls)
    sample = f"{cores} chain-steps per step (one MH iteration of {cores} chains, full T={w['T']})"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(name, w, args.block_len, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(name, w, block_len, nb):
    return {"workload": f"{name}_C{w['C']}", "model": "multivariate stochastic volatility"
            if w["kind"] == "sv" else "linear-Gaussian", "d_x": w["d"], "T": w["T"],
            "chains_per_gpu": w["C"], "block_len": block_len or None, "scan_blocks": nb,
            "l2": "flushed (256 MiB write) before every timed step", "parallelism": "replicas"}


# --------------------------------------------------------------------------- GPU arm
def run_spatial(args, flush, stream):
    """The lattice model of Section 4.2 (factorised prior, Student-t emission, d = 64,
    T = 1024, one chain as in the paper): delta adapted on the device to 50 %
    acceptance during warm-up, then frozen; time per MH iteration."""
    import torch
    from paper_2303_00301_gb300 import AuxKalman
    from paper_2303_00301_gb300 import workloads as W
    wls = W.spatio_temporal(side=8, T=1024, n_chains=1, delta=0.05)
    ss = AuxKalman(wls, dtype="f32")
    xsp = torch.tensor(wls.x_init, dtype=torch.float32, device="cuda")
    ss.adapt_delta(True, target=0.5, gain=1.0)
    ss.step(xsp, 400, iter0=0)
    ss.adapt_delta(False)
    accs = torch.zeros(1, dtype=torch.int32, device="cuda")
    ss.step(xsp, 5, iter0=400)
    torch.cuda.synchronize()
    n_sp = max(args.steps, 50)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n_sp)]
    for k in range(n_sp):
        flush.zero_()
        evs[k][0].record(stream)
        ss.step(xsp, 1, iter0=405 + k, accept_count=accs)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms_sp = sum(a.elapsed_time(b) for a, b in evs) / n_sp
    # the same iteration replayed from a CUDA graph (iteration index on the device)
    ss.device_iteration(True, 405 + n_sp)
    g = ss.capture(xsp, 1, accs)
    evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(n_sp)]
    for k in range(n_sp):
        flush.zero_()
        evg[k][0].record(stream)
        g.replay()
        evg[k][1].record(stream)
    torch.cuda.synchronize()
    ms_gr = sum(a.elapsed_time(b) for a, b in evg) / n_sp
    ss.device_iteration(False)
    del g
    out = {"workload": "spatio_temporal_8x8_T1024_C1 (Section 4.2, Student-t nu = 1)",
           "ms_per_iteration": ms_gr, "launch": "CUDA graph replay", "ms_per_iteration_eager": ms_sp,
           "value": wls.T / (ms_gr / 1e3), "unit": UNIT,
           "delta": ss.delta(), "accept_rate": accs.item() / (2 * n_sp),
           "paper_ms_per_iteration": 0.52,
           "paper_hardware": "RTX 3090, JAX (another machine and software: context only)"}
    ss.close()
    return out


def run_wide(args, flush, stream, peaks, pool=None):
    """The mixed-precision workload's shape (SV, d = 128, T = 4096, 16 chains) on the wide
    table-mode kernels, in two forms: single precision throughout ("f32": FP64 only in the
    log-determinants and the likelihood sums) and mixed precision ("mixed": the covariance
    pass's products on the tensor cores in split TF32 with FP32 accumulation, the
    factorisations of the element operator in FP64). delta is adapted on the device to 50 %
    acceptance during warm-up of the f32 form (the covariance pass reruns at every
    adaptation step) and frozen for both; cached covariance tables; the MH iteration
    captured in a CUDA graph and replayed, L2 flushed before each replay. The shared mode
    (the covariance pass rerun every step) is timed beside it, eager. With a process pool,
    each form's error against the FP64 oracle on two sampled chains is reported."""
    import numpy as np
    import torch
    from paper_2303_00301_gb300 import AuxKalman
    from paper_2303_00301_gb300 import _binding as B
    from paper_2303_00301_gb300 import workloads as W
    d, T, C = 128, args.wide_T, 16
    wl = W.stochastic_volatility(d=d, T=T, n_chains=C)
    delta = wl.delta
    n_adapt = args.wide_adapt
    if n_adapt > 0:
        h = AuxKalman(wl, dtype="f32", mode="cached", block_len=args.wide_L)
        x = torch.tensor(wl.x_init, dtype=torch.float32, device="cuda")
        h.adapt_delta(True, target=0.5, gain=1.0)
        h.step(x, n_adapt, iter0=0)
        h.adapt_delta(False)
        delta = h.delta()
        h.close()
    chains = (0, C - 1)
    refs = None
    if pool is not None:
        res = pool.map(_oracle_wide_step, [(d, T, C, delta, c) for c in chains], chunksize=1)
        refs = dict(zip(chains, res))
    L = args.wide_L or math.ceil(math.sqrt(T))
    nb = (T + L - 1) // L
    n = max(args.steps // 10, 30)
    out = {}
    for dt in ("f32", "mixed"):
        wd = W.stochastic_volatility(d=d, T=T, n_chains=C, delta=delta)
        h = AuxKalman(wd, dtype=dt, mode="cached", block_len=args.wide_L)
        x = torch.tensor(wd.x_init, dtype=torch.float32, device="cuda")
        it = n_adapt
        h.step(x, 3, iter0=it)
        it += 3
        acc = torch.zeros(C, dtype=torch.int32, device="cuda")
        B.aux_set_profiling(h.handle, True)
        for k in range(n):
            flush.zero_()
            h.step(x, 1, iter0=it + k, accept_count=acc)
        torch.cuda.synchronize()
        B.aux_set_profiling(h.handle, False)
        prof = B.aux_read_profile(h.handle)
        it += n
        rate = acc.float().mean().item() / n
        h.device_iteration(True, it)
        g = h.capture(x, 1)
        g.replay()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for k in range(n):
            flush.zero_()
            ev[k][0].record(stream)
            g.replay()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / n
        h.device_iteration(False)
        del g
        rc = h.status()[0]
        h.close()
        # the shared mode: the covariance pass every step
        hs = AuxKalman(wd, dtype=dt, mode="shared", block_len=args.wide_L)
        xs = torch.tensor(wd.x_init, dtype=torch.float32, device="cuda")
        hs.step(xs, 2, iter0=0)
        B.aux_set_profiling(hs.handle, True)
        ns = 5
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ns)]
        for k in range(ns):
            flush.zero_()
            evs[k][0].record(stream)
            hs.step(xs, 1, iter0=2 + k)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        B.aux_set_profiling(hs.handle, False)
        profs = B.aux_read_profile(hs.handle)
        ms_sh = sum(a.elapsed_time(b) for a, b in evs) / ns
        hs.close()
        w = {"dtype": "f32"}
        dom = max((k for k in prof if prof[k][1]), key=lambda k: prof[k][0])
        line = roofline_line("cached", dom, prof, w, d, T, C, nb, T, True, 4, peaks, n,
                             "dominant kernel (cached tables, per-chain means)")
        if line:
            line["kernel"] = {"reduce": "k_wmf_reduce", "apply": "k_wmf_apply", "scan": "k_wmean_cross",
                              "backward": "k_wmean_cross + k_wmb_apply"}.get(dom, dom)
            line["traffic"] = dram_traffic(f"{line['kernel']}@sv_d{d}_T{T}_C{C}")
        prec = ("FP32 tables and means; FP64 log-determinants and likelihood sums" if dt == "f32" else
                "covariance-pass products on the tensor cores (split TF32, FP32 accumulation); FP64 "
                "factorisations of C_i and N = I + U^T J U and inverse of chol(N); FP32 tables and means; "
                "FP64 log-determinants and likelihood sums")
        out[dt] = {"precision": prec, "mode": "cached", "launch": "CUDA graph replay", "ms_per_step": ms,
                   "value": C * T / (ms / 1e3), "unit": UNIT, "accept_rate": rate, "status": int(rc), "steps": n,
                   "kernel_ms_per_step": {k: v[0] / n for k, v in prof.items() if v[1]},
                   "roofline": line,
                   "shared_mode": {"ms_per_step": ms_sh, "value": C * T / (ms_sh / 1e3), "launch": "eager",
                                   "kernel_ms_per_step": {k: v[0] / ns for k, v in profs.items() if v[1]}},
                   "error_vs_fp64_oracle": (wide_error_block(refs, wl, dt, delta, chains) if refs else None)}
    res = {"workload": f"sv_d{d}_T{T}_C{C} (SV, d = {d}, T = {T}, {C} chains)", "block_len": L,
           "delta": delta, "delta_adaptation_steps": n_adapt}
    res.update(out["f32"])
    res["mixed_precision"] = out["mixed"]
    return res


def _time_graph(g, flush, stream, n):
    """Mean device time (ms) of n replays of a captured graph, L2 flushed before each."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        flush.zero_()
        ev[k][0].record(stream)
        g.replay()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / n


def _capture(fn):
    import torch
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=cap):
        fn(cap)
    torch.cuda.current_stream().wait_stream(cap)
    torch.cuda.synchronize()
    return g


def batch_p(d):
    """Padded width of the library's narrow (4, 8, 16, 32) and wide (64, 128) kernels."""
    for p in (4, 8, 16, 32, 64, 128):
        if d <= p:
            return p
    raise ValueError(d)


def batched_instances(n_inst=256, dims=(8, 16, 32, 64), seed=3):
    """The batched workload: n_inst SV instances, one chain each, T_k ~ U{128..4096},
    d_k cycling through dims, per-instance phi, data and seeds; delta_k = 0.0183
    (30 * 1024 / (d_k T_k))^(1/2) (the d = 30, T = 1024 value scaled by the
    pseudo-observation precision per state)."""
    import numpy as np
    from paper_2303_00301_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_inst):
        d = dims[k % len(dims)]
        T = int(rng.integers(128, 4097))
        delta = 0.0183 * math.sqrt(30 * 1024 / (d * T))
        out.append(W.stochastic_volatility(d=d, T=T, n_chains=1, sim_seed=100 + k, mcmc_seed=1000 + k, delta=delta))
    return out


def run_batched(args, flush, stream, n_streams=32):
    """The batched line: 256 SV instances (batched_instances) advanced by ONE persistent
    launch per MCMC iteration (aux_batch_step), its launch shape and block lengths
    picked by the library's autotuner (aux_batch_tune); each step a CUDA-graph replay
    with L2 flushed before it. Cached mode (tables kept) and shared mode (every
    instance's covariance pass rerun every step, side by side on the batch's streams)
    are both timed. For comparison the same instances stepped one handle at a time
    (11 launches each, one graph with 32 stream branches), the batch's predecessor."""
    import torch
    from paper_2303_00301_gb300 import AuxBatch, AuxKalman
    wls = batched_instances(n_inst=args.batched_instances)
    n = max(args.steps // 2, 10)
    models = [AuxKalman(wl, dtype="f32", mode="cached") for wl in wls]
    xs = [torch.tensor(wl.x_init, dtype=torch.float32, device="cuda") for wl in wls]
    steps_total = sum(wl.T for wl in wls)
    out = {"workload": f"{len(wls)} SV instances, one chain each, T ~ U{{128..4096}}, d in [8, 16, 32, 64]",
           "unit": UNIT, "instances": len(wls), "timesteps_per_step": steps_total,
           "launch": "one persistent kernel per MCMC iteration (aux_batch_step), CUDA graph replay",
           "l2": "flushed before every step"}

    def batch_line(sub, it0):
        # it0: a fresh range of MCMC iterations (reusing a range on chains that have
        # already drawn its Philox numbers correlates the draws and depresses acceptance)
        bx = AuxBatch([models[i] for i in sub], [xs[i] for i in sub], iteration=it0)
        t0 = time.perf_counter()
        tuned_ms = bx.tune(reps=3)
        tune_s = time.perf_counter() - t0
        cfg = bx.config()
        res = {}
        for mode in (("cached",) if args.batched_quick else ("cached", "shared")):
            bx.set_mode(mode)
            acc = torch.zeros(len(sub), dtype=torch.int32, device="cuda")
            bx.step(2)
            torch.cuda.synchronize()
            g = _capture(lambda st: bx.step(1, accept_count=acc, stream=st))
            g.replay()
            torch.cuda.synchronize()
            acc.zero_()
            nn = n if mode == "cached" else max(n // 4, 5)
            ms = _time_graph(g, flush, stream, nn)
            ts = sum(wls[i].T for i in sub)
            r = {"ms_per_step": ms, "value": ts / (ms / 1e3), "accept_rate": acc.sum().item() / (nn * len(sub)),
                 "steps": nn}
            if mode == "cached":
                r["launches_per_step"] = 2
            else:
                # the covariance passes' launches, counted by the handles' profiler on one eager step
                for i in sub:
                    models[i].b.aux_set_profiling(models[i].handle, True)
                bx.step(1)
                torch.cuda.synchronize()
                nl = 0
                for i in sub:
                    prof = models[i].b.aux_read_profile(models[i].handle)
                    nl += sum(v[1] for k, v in prof.items() if k.startswith("cov_"))
                    models[i].b.aux_set_profiling(models[i].handle, False)
                r["launches_per_step"] = nl + 4   # + table copy, block tables, persistent step, counter
            del g
            res[mode] = r
        rc, ab = bx.status()
        bx.close()
        # HBM roofline of the persistent step (cached): per chain-timestep it streams eight
        # p x p tables (K' in the forward reduce, apply, reverse reduce and reverse apply;
        # G twice; chol(Sigma); the block prefix GP) and about 17 d + 2 p vector words
        tb = sum(8 * wls[i].T * batch_p(wls[i].d) ** 2 * 4 + wls[i].T * (17 * wls[i].d + 2 * batch_p(wls[i].d)) * 4
                 for i in sub)
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        hbm = json.load(open(pk)).get("hbm_gbs") if os.path.exists(pk) else None
        ach = tb / (res["cached"]["ms_per_step"] * 1e-3) / 1e9
        key = f"k_batch_step@batched{len(sub)}"
        res["cached"]["roofline"] = {"kernel": "k_batch_step", "bound": "hbm", "achieved": ach, "peak": hbm,
                                     "unit": "GB/s", "frac": (ach / hbm) if hbm else None,
                                     "traffic": dram_traffic(key),
                                     "bytes_per_step": tb, "peak_basis": "measured HBM copy bandwidth",
                                     "timing": "graph replay of the step (persistent kernel + counter)"}
        line = dict(res["cached"])
        line.update({"mode": "cached", "status": int(rc), "aborted": int(ab), "shared_mode": res.get("shared"),
                     "tuner": {"best_ms_per_step": tuned_ms, "seconds": tune_s,
                               "warps_per_cta": cfg["warps_per_cta"], "ctas_per_sm": cfg["ctas_per_sm"],
                               "item_order": ["longest first", "shortest first"][cfg["order"]],
                               "block_len_factor_by_width": dict(zip(["p<=8", "p=16", "p=32", "p=64"],
                                                                     cfg["block_factor"]))}})
        return line

    out.update(batch_line(list(range(len(wls))), 0))
    if args.batched_quick:
        for h in models:
            h.close()
        return out
    out["d_le_32_subset"] = batch_line([i for i, wl in enumerate(wls) if wl.d <= 32], 1 << 20)
    out["d_le_32_subset"]["instances"] = sum(1 for wl in wls if wl.d <= 32)

    # the same instances one handle at a time (per-instance launches, 32 stream branches)
    for it in range(3):
        for h, x in zip(models, xs):
            h.step(x, 1, iter0=(2 << 20) + it)
    torch.cuda.synchronize()
    for h in models:
        h.device_iteration(True, (2 << 20) + 3)
    streams = [torch.cuda.Stream() for _ in range(n_streams)]

    def per_instance(cap):
        for st in streams:
            st.wait_stream(cap)
        for i, (h, x) in enumerate(zip(models, xs)):
            with torch.cuda.stream(streams[i % n_streams]):
                h.step(x, 1, 0)
        for st in streams:
            cap.wait_stream(st)

    g = _capture(per_instance)
    g.replay()
    torch.cuda.synchronize()
    ms = _time_graph(g, flush, stream, n)
    del g
    out["per_instance_launches"] = {"ms_per_step": ms, "value": steps_total / (ms / 1e3), "mode": "cached",
                                    "launch": f"11 launches per instance, one CUDA graph, {n_streams} stream branches"}
    for h in models:
        h.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _cpu_env()
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(os.cpu_count() or 1)
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2303_00301_gb300 import AuxKalman, build
    from paper_2303_00301_gb300 import _binding as B
    build.build()
    name = args.workload
    wl, w = make_workload(name, rank)
    C, T, d = w["C"], w["T"], w["d"]
    tdt = torch.float32 if w["dtype"] == "f32" else torch.float64
    esz = 4 if w["dtype"] == "f32" else 8
    def block_len_for(mode):
        """Means block length: the library's default ceil(sqrt T) on the per-chain path;
        ceil(sqrt(T) / 2) in the table modes, whose cross-block pass (one mat-vec per
        block) is cheaper than their in-block step (four), measured 4-5 % faster at T = 1024
        (and 21 % slower on the per-chain path)."""
        if args.block_len:
            return args.block_len
        if mode == "per_chain":
            return max(1, math.ceil(math.sqrt(T)))
        return max(1, math.ceil(math.sqrt(T) / 2))

    L = block_len_for(args.mode)
    nb = (T + L - 1) // L
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed_steps(step, n):
        """n steps, L2 flushed before each, every step bracketed by CUDA events
        on the launching stream; returns the per-step times in ms."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        for k in range(n):
            flush.zero_()
            ev[k][0].record(stream)
            step(k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    def run_mode(mode, with_clocks, proposal=1, adapt=False, sampler="scan", filter_form="covariance",
                 dtype=None):
        """Warm-up; one profiled eager pass (per-kernel events: the kernel
        breakdown and roofline durations); then the timed pass: the MCMC
        iteration captured once in a CUDA graph (iteration index on the
        device) and replayed args.steps times; then the same steps eager
        without events, for comparison."""
        dt_m = dtype or w["dtype"]
        sm = AuxKalman(wl, dtype=dt_m, block_len=block_len_for(mode), mode=mode, proposal=proposal,
                       sampler=sampler, filter_form=filter_form)
        if adapt:
            sm.adapt_delta(True, target=0.5, gain=1.0)
        xm = torch.tensor(wl.x_init, dtype=torch.float64 if dt_m == "f64" else tdt, device="cuda")
        accm = torch.zeros(C, dtype=torch.int32, device="cuda")
        lam = torch.zeros(C, dtype=torch.float64, device="cuda")
        itm = 0
        for _ in range(args.warmup):
            sm.step(xm, 1, iter0=itm, accept_count=accm, log_alpha=lam)
            itm += 1
        torch.cuda.synchronize()
        accm.zero_()
        B.aux_set_profiling(sm.handle, True)
        prof_ms = timed_steps(lambda k: sm.step(xm, 1, iter0=itm + k, accept_count=accm, log_alpha=lam),
                              args.steps)
        itm += args.steps
        B.aux_set_profiling(sm.handle, False)
        prof = B.aux_read_profile(sm.handle)
        accept_rate_m = accm.float().mean().item() / args.steps
        # the timed pass
        sm.device_iteration(True, itm)
        g = sm.capture(xm, 1, accm, lam)
        g.replay()                                   # warm the graph up
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ck = None
        if with_clocks:
            clocks = ClockSampler(local)
            clocks.start()
        step_ms = timed_steps(lambda k: g.replay(), args.steps)
        if with_clocks:
            ck = clocks.stop()
        itm = sm.iteration()
        sm.device_iteration(False)
        del g
        t_ms = max_over_ranks(sum(step_ms), "cuda", world)
        eager_ms = timed_steps(lambda k: sm.step(xm, 1, iter0=itm + k, accept_count=accm, log_alpha=lam),
                               args.steps)
        itm += args.steps
        res = {"mode": mode, "dtype": dt_m, "proposal": "second order" if proposal == 2 else "first order",
               "sampler": "divide-and-conquer bridging" if sampler == "bridging" else "(G, U) suffix scan",
               "filter_form": filter_form,
               "delta": sm.delta(), "delta_adaptation": bool(adapt),
               "value": world * C * T * args.steps / (t_ms / 1e3), "unit": UNIT,
               "ms_per_step": t_ms / args.steps, "launch": "CUDA graph replay",
               "ms_per_step_eager": sum(eager_ms) / args.steps,
               "ms_per_step_eager_profiled": sum(prof_ms) / args.steps,
               "step_ms_median": statistics.median(step_ms),
               "accept_rate": accept_rate_m,
               "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
               # the profiled kernels of each step, plus the graph's iteration-counter increment
               "gpu_launches": int(sum(v[1] for v in prof.values())) + args.steps}
        return sm, xm, lam, itm, prof, ck, res

    s, x, la, it, prof, ck, head = run_mode(args.mode, True, sampler=args.sampler,
                                            filter_form=args.filter_form)
    value = head["value"]
    total_ms = head["ms_per_step"] * args.steps
    accept_rate = head["accept_rate"]
    others, profs = {}, {args.mode: prof}
    if not args.headline_only:
        for mode in ("per_chain", "shared", "cached"):
            if mode != args.mode:
                so, _, _, _, po, _, r = run_mode(mode, False)
                so.close()
                others[mode] = r
                profs[mode] = po
        # the second-order proposal (Eqs. (2.8)-(2.9)): per-chain path, same delta
        so, _, _, _, _, _, r = run_mode("per_chain", False, proposal=2)
        so.close()
        others["per_chain_second_order"] = r
        # on-device delta adaptation (pooled Robbins-Monro, target 0.5): the covariance
        # pass reruns every step, as in the shared mode
        so, _, _, _, _, _, r = run_mode("cached", False, adapt=True)
        so.close()
        others["cached_delta_adaptation"] = r
        # the divide-and-conquer (bridging) sampler (Appendix A.2.3) in place of the scan
        for key, mode in (("cached_bridging", "cached"), ("shared_bridging", "shared"),
                          ("per_chain_bridging", "per_chain")):
            so, _, _, _, po, _, r = run_mode(mode, False, sampler="bridging")
            so.close()
            others[key] = r
            profs[key] = po
        # the square-root form of the per-chain filter (the remedy Section 4.1 names)
        so, _, _, _, po, _, r = run_mode("per_chain", False, filter_form="square_root")
        so.close()
        others["per_chain_square_root"] = r
        profs["per_chain_square_root"] = po
        # the headline mode in FP64 (the precision of the paper's SV runs, Section 4.1)
        if w["dtype"] == "f32":
            so, _, _, _, po, _, r = run_mode(args.mode, False, dtype="f64", sampler=args.sampler,
                                             filter_form=args.filter_form)
            so.close()
            others[args.mode + "_f64"] = r
            profs[args.mode + "_f64"] = po
        # the square-root form of the table modes' covariance pass
        if not (args.mode == "shared" and args.filter_form == "square_root"):
            so, _, _, _, po, _, r = run_mode("shared", False, filter_form="square_root")
            so.close()
            others["shared_square_root"] = r
            profs["shared_square_root"] = po

    spatial = None
    batched = None
    wide = None
    if not args.headline_only and rank == 0:
        spatial = run_spatial(args, flush, stream)
        batched = run_batched(args, flush, stream)
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        wide = run_wide(args, flush, stream, json.load(open(pk)) if os.path.exists(pk) else {}, pool)

    # end to end through the public API from pinned host buffers
    x_host = torch.tensor(wl.x_init, dtype=tdt).pin_memory()
    la_host = torch.zeros(C, dtype=torch.float64).pin_memory()
    for _ in range(2):
        x.copy_(x_host, non_blocking=True)
        s.step(x, 1, iter0=it, log_alpha=la)
        x_host.copy_(x, non_blocking=True)
        la_host.copy_(la, non_blocking=True)
        it += 1
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        x.copy_(x_host, non_blocking=True)
        s.step(x, 1, iter0=it, log_alpha=la)
        x_host.copy_(x, non_blocking=True)
        la_host.copy_(la, non_blocking=True)
        torch.cuda.synchronize()
        it += 1
    e2e_s = max_over_ranks(time.perf_counter() - t0, "cuda", world)
    e2e_value = world * C * T * args.steps / e2e_s
    rc, per_chain = s.status()

    # roofline lines: the dominant kernel of the headline mode, and one line per
    # path (general per-chain filter, means-only table path, covariance pass)
    fdiag = bool(np.all(wl.F == np.diag(np.diag(wl.F))))
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    def shape_for(mode):
        """(means blocks, covariance blocks) of a mode's handle (the library's rules)."""
        Lm = block_len_for(mode)
        Lc = max(c for c in range(1, min(4, Lm) + 1) if Lm % c == 0)
        return (T + Lm - 1) // Lm, (T + Lc - 1) // Lc
    dom = max((k for k in prof if prof[k][1]), key=lambda k: prof[k][0])
    def rl(mode, kind, path, key=None):
        nbm, nbcm = shape_for("per_chain" if mode.startswith("per_chain") else
                              ("shared" if mode == "table_sqrt" else mode))
        return roofline_line(mode, kind, profs[key or mode], w, d, T, C, nbm, nbcm, fdiag, esz, peaks,
                             args.steps, path)
    head_work = args.mode
    if args.filter_form == "square_root":
        head_work = "per_chain_sqrt" if args.mode == "per_chain" else "table_sqrt"
    roofline = rl(head_work, dom, f"dominant kernel of the {args.mode} mode", args.mode)
    lines = {}
    if "per_chain" in profs and not (args.mode == "per_chain" and args.filter_form == "square_root"):
        lines["general_path"] = rl("per_chain", "apply", "per-chain element scan (general path)")
    tmode = args.mode if args.mode != "per_chain" else ("cached" if "cached" in profs else None)
    if tmode:
        lines["means_path"] = rl(tmode, "apply", "means-only batched path (tables shared by all chains)")
        cov_kinds = [k for k in ("cov_reduce", "cov_scan", "cov_apply", "cov_products")
                     if k in profs.get("shared", {}) and profs["shared"][k][1]]
        if cov_kinds:
            ck_dom = max(cov_kinds, key=lambda k: profs["shared"][k][0])
            lines["covariance_pass"] = rl("shared", ck_dom, "covariance (Riccati) pass, once per call")
    if "per_chain_square_root" in profs:
        pq = profs["per_chain_square_root"]
        kq = max((k for k in ("reduce", "apply") if pq.get(k, (0, 0))[1]), key=lambda k: pq[k][0])
        lines["square_root_path"] = rl("per_chain_sqrt", kq, "square-root form of the per-chain filter "
                                       "(dominant kernel)", "per_chain_square_root")
    if "shared_square_root" in profs:
        pq = profs["shared_square_root"]
        kq = [k for k in ("cov_reduce", "cov_scan", "cov_apply") if pq.get(k, (0, 0))[1]]
        if kq:
            kq = max(kq, key=lambda k: pq[k][0])
            lines["square_root_covariance_pass"] = rl("table_sqrt", kq, "square-root form of the covariance "
                                                      "pass (dominant kernel)", "shared_square_root")
    if "cached_bridging" in profs:
        lines["bridging_sampler"] = rl("cached", "bridge", "divide-and-conquer sampler: offsets up, "
                                       "split points down, MH terms (tables shared)", "cached_bridging")
    if "shared_bridging" in profs:
        lines["bridging_tree"] = rl("shared", "bridge_tree", "divide-and-conquer tree matrices, once "
                                    "per covariance pass", "shared_bridging")

    # ESS and ESJD of the headline mode from a long run (outside the timed region)
    ess = None
    if args.ess_iters > 0 and rank == 0:
        se = AuxKalman(wl, dtype=w["dtype"], block_len=block_len_for(args.mode), mode=args.mode)
        xe = torch.tensor(wl.x_init, dtype=tdt, device="cuda")
        t_idx = torch.linspace(0, T - 1, 8).round().long().cuda()
        i_idx = torch.linspace(0, d - 1, min(d, 5)).round().long().cuda()
        tt, ii = torch.meshgrid(t_idx, i_idx, indexing="ij")
        tt, ii = tt.reshape(-1), ii.reshape(-1)
        trace = torch.empty((args.ess_iters, C, tt.numel()), dtype=torch.float64, device="cuda")
        jump = torch.zeros((C, T), dtype=torch.float64, device="cuda")
        ite = 10 ** 6
        for _ in range(args.ess_burn):
            se.step(xe, 1, iter0=ite)
            ite += 1
        xprev = xe.clone()
        for n_ in range(args.ess_iters):
            se.step(xe, 1, iter0=ite)
            ite += 1
            trace[n_] = xe[:, tt, ii].double()
            jump += ((xe - xprev).double() ** 2).sum(-1)
            xprev.copy_(xe)
        torch.cuda.synchronize()
        tr = trace.cpu().numpy()
        se.close()
        sec_per_iter = head["ms_per_step"] / 1e3
        ess_pair = np.array([sum(geyer_ess(tr[:, c, j]) for c in range(C)) for j in range(tr.shape[2])])
        esjd_t = (jump / args.ess_iters).mean(0).cpu().numpy()     # per chain, per t
        ess = {"iterations": args.ess_iters, "burn_in": args.ess_burn, "chains": C,
               "estimator": "Geyer initial monotone sequence, summed over chains",
               "coordinates": f"x_t(i) for t in {t_idx.tolist()}, i in {i_idx.tolist()}",
               "ess_min": float(ess_pair.min()), "ess_median": float(np.median(ess_pair)),
               "ess_per_s_min": float(ess_pair.min() / (args.ess_iters * sec_per_iter)),
               "ess_per_s_median": float(np.median(ess_pair) / (args.ess_iters * sec_per_iter)),
               "esjd_per_s_min": float(esjd_t.min() / sec_per_iter),
               "esjd_per_s_median": float(np.median(esjd_t) / sec_per_iter),
               "seconds_per_iteration": sec_per_iter}

    fp32_error = None
    if pool is not None and w["dtype"] == "f32":
        fp32_error = fp32_error_block(name, wl, w, args.mode, block_len_for(args.mode), pool)
    cpu = None
    if pool is not None:
        n = args.cpu_sample_chains or 2 * (os.cpu_count() or 1)
        rate, wall = cpu_oracle_rate(name, n, pool, os.cpu_count() or 1)
        pool.close()
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"{n} chain-steps (one MH iteration each, full T={T}, d={d}) in {wall:.1f} s"}
    if rank == 0:
        bi = C * T * d * esz
        bo = C * T * d * esz + C * 8
        cfg = config_of(name, w, L, nb)
        cfg["block_len_per_mode"] = {m: block_len_for(m) for m in ("per_chain", "shared", "cached")}
        cfg["mode"] = args.mode
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": w["dtype"], "data": "synthetic", "config": cfg,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bi,
                        "d2h_bytes_per_step": bo},
                "gpu_launches": head["gpu_launches"],
                "roofline": roofline, "roofline_lines": lines, "ess": ess, "fp32_error": fp32_error,
                "cpu_baseline": cpu, "clocks": ck,
                "kernel_ms_per_step": head["kernel_ms_per_step"],
                "launch": head["launch"], "ms_per_step_eager": head["ms_per_step_eager"],
                "ms_per_step_eager_profiled": head["ms_per_step_eager_profiled"],
                "accept_rate": accept_rate, "status": int(rc),
                "step_ms_median": head["step_ms_median"], "other_modes": others,
                "spatio_temporal": spatial, "batched_instances": batched, "wide_d128": wide}
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.spatial_only:
        import torch
        from paper_2303_00301_gb300 import build
        build.build()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(run_spatial(args, flush, torch.cuda.current_stream())), flush=True)
        return
    if args.wide_only:
        pool = None
        if not args.no_cpu_baseline:   # the oracle's error reference, started before any CUDA call
            _cpu_env()
            import multiprocessing as mp
            pool = mp.get_context("spawn").Pool(2)
        import torch
        from paper_2303_00301_gb300 import build
        build.build()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        peaks = json.load(open(pp)) if os.path.exists(pp) else {}
        print(json.dumps(run_wide(args, flush, torch.cuda.current_stream(), peaks, pool)), flush=True)
        if pool is not None:
            pool.close()
        return
    if args.batched_only:
        import torch
        from paper_2303_00301_gb300 import build
        build.build()
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps(run_batched(args, flush, torch.cuda.current_stream())), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

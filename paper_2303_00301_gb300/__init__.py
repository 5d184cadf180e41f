"""GB300 auxiliary Kalman sampler (arXiv:2303.00301, Section 2.2 / Algorithm 2).

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``)
behind the C ABI of ``include/aux_kalman.h``. ``_binding`` exposes those
entry points under their C names; ``AuxKalman`` is a small convenience
wrapper that owns the handle and takes torch CUDA tensors.
"""
from .workloads import EMIS_LINEAR_GAUSSIAN, EMIS_STUDENT_T, EMIS_SV  # noqa: F401


def _load_binding():
    from . import _binding as b
    return b


MODES = ("per_chain", "shared", "cached")
SAMPLERS = ("scan", "bridging")
FILTER_FORMS = ("covariance", "square_root")


class AuxKalman:
    """Owns an ``aux_model`` handle for one workload (torch is used for memory only).

    ``mode`` selects the execution of the filter (``aux_set_mode``): "per_chain"
    (every chain runs the full element recursion), "shared" (one covariance
    pass per call, means per chain) or "cached" (the covariance tables are kept
    until the model changes). ``proposal`` is the order of the auxiliary
    proposal (``aux_set_proposal``): 1 (first order) or 2 (second order,
    per-chain mode only). ``sampler`` draws the path from the smoothing law
    (``aux_set_sampler``): "scan" ((G, U) suffix scan) or "bridging"
    (divide-and-conquer tree of bridging conditionals). ``filter_form``
    (``aux_set_filter_form``): "covariance" or "square_root" (per chain with
    the first-order proposal and the scan sampler, or the covariance pass of
    the table modes). State dimensions 33..128 (FP32) run the table modes only
    ("shared" or "cached"), first order, scan sampler, covariance form; there
    ``dtype="mixed"`` runs the covariance pass's products on the tensor cores
    (split TF32, FP32 accumulation) with its factorisations in FP64.
    """

    def __init__(self, workload, dtype="f32", seed=None, n_chains=None, block_len=0, stream=None,
                 mode="per_chain", proposal=1, sampler="scan", filter_form="covariance"):
        import torch
        b = _load_binding()
        self.b = b
        self.wl = workload
        self.C = int(n_chains if n_chains is not None else workload.n_chains)
        self.T, self.d = workload.T, workload.d
        codes = {"f32": b.AUX_F32, "f64": b.AUX_F64, "mixed": b.AUX_MIXED}
        if dtype not in codes:
            raise ValueError(f"dtype must be one of {sorted(codes)}")
        self.dtype_code = codes[dtype]
        self.torch_dtype = torch.float64 if dtype == "f64" else torch.float32
        self.seed = workload.mcmc_seed if seed is None else seed
        self.handle = b.aux_init_model(
            d_x=self.d, T=self.T, n_chains=self.C, m0=workload.m0, P0=workload.P0,
            F=workload.F, b=workload.b, Q=workload.Q, y=workload.y, delta=workload.delta,
            emis_kind=workload.emission, dtype=self.dtype_code, R_y=workload.Ry,
            obs_mask=workload.mask, block_len=block_len, seed=self.seed, stream=stream,
            nu=getattr(workload, "nu", 0.0))
        if mode not in MODES:
            raise ValueError(f"mode must be one of {MODES}")
        self.mode = mode
        if mode != "per_chain":
            b.aux_set_mode(self.handle, b.AUX_MODE_SHARED_COV if mode == "shared" else b.AUX_MODE_CACHED_COV)
        self.proposal = proposal
        if proposal != 1:
            b.aux_set_proposal(self.handle, proposal)
        if sampler not in SAMPLERS:
            raise ValueError(f"sampler must be one of {SAMPLERS}")
        self.sampler = sampler
        if sampler != "scan":
            b.aux_set_sampler(self.handle, b.AUX_SAMPLER_BRIDGING)
        if filter_form not in FILTER_FORMS:
            raise ValueError(f"filter_form must be one of {FILTER_FORMS}")
        self.filter_form = filter_form
        if filter_form != "covariance":
            b.aux_set_filter_form(self.handle, b.AUX_FILTER_SQUARE_ROOT)

    def step(self, x, n_iters=1, iter0=0, accept_count=None, log_alpha=None, stream=None):
        self.b.aux_kalman_step(self.handle, x, n_iters, iter0, accept_count, log_alpha, stream)

    def loglik(self, ytilde, logZ, mf=None, Pf=None, stream=None):
        self.b.aux_loglik(self.handle, ytilde, logZ, mf, Pf, stream)

    def sample_path(self, ytilde, xstar, eps=None, iteration=0, logZ=None, stream=None):
        self.b.aux_sample_path(self.handle, ytilde, xstar, eps, iteration, logZ, stream)

    def status(self):
        return self.b.aux_get_status(self.handle, self.C)

    def adapt_delta(self, enable=True, target=0.5, gain=1.0):
        """On-device Robbins-Monro adaptation of delta (aux_set_delta_adaptation)."""
        self.b.aux_set_delta_adaptation(self.handle, enable, target, gain)

    def delta(self):
        return self.b.aux_get_delta(self.handle)

    def device_iteration(self, enable=True, start=0):
        """Keep the MCMC iteration on the device (aux_set_device_iteration)."""
        self.b.aux_set_device_iteration(self.handle, enable, start)
        self._dev_iter = bool(enable)

    def iteration(self):
        return self.b.aux_get_device_iteration(self.handle)

    def capture(self, x, n_iters=1, accept_count=None, log_alpha=None):
        """Capture ``n_iters`` MCMC iterations on ``x`` into a CUDA graph.

        Turns the device iteration counter on (keeping its value if it is on
        already, else starting at 0); every ``replay()`` of the returned graph
        then runs the next ``n_iters`` iterations. Warm the handle up with one
        eager ``step`` first so that no one-off work (the cached covariance
        pass) is captured."""
        import torch
        if not getattr(self, "_dev_iter", False):
            self.device_iteration(True, 0)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            self.step(x, n_iters, 0, accept_count, log_alpha)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def grad(self, ytilde, g_mu, g_phi, g_L, g_delta, logZ=None, stream=None):
        """aux_loglik_grad; ytilde None: the last step's pseudo-observations."""
        self.b.aux_loglik_grad(self.handle, ytilde, g_mu, g_phi, g_L, g_delta, logZ, stream)

    def grad_memory(self, max_bytes):
        """aux_set_grad_memory: cap the gradient's store of G_t, Sigma_t, U_t
        (recompute the in-block filter per chunk of blocks above it; 0: store all)."""
        self.b.aux_set_grad_memory(self.handle, max_bytes)

    def theta_step(self, g_mu, g_phi, g_L, lr, stream=None):
        """The on-device theta-update inside the sweep (aux_sv_theta_step)."""
        self.b.aux_sv_theta_step(self.handle, g_mu, g_phi, g_L, lr, stream)

    def set_theta(self, mu, phi, L, delta):
        self.b.aux_set_sv_theta(self.handle, mu, phi, L, delta)

    def theta(self):
        return self.b.aux_get_sv_theta(self.handle, self.d)

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.b.aux_free_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AuxBatch:
    """Many ``AuxKalman`` models (uneven T and d) advanced by one persistent launch per
    MCMC iteration (``aux_batch_*``). The models (FP32, "shared" or "cached" mode) and
    their state tensors ``xs`` (device, [C][T][d] FP32) must outlive the batch.
    ``step`` runs every chain of every model; ``tune`` runs the library's autotuner
    over launch shapes and block lengths (states restored afterwards)."""

    def __init__(self, models, xs, iteration=0, mode="cached", stream=None):
        b = _load_binding()
        self.b = b
        self.models = list(models)
        self.xs = list(xs)
        self.n_chains = sum(m.C for m in self.models)
        self.batch = b.aux_batch_create([m.handle for m in self.models], self.xs, iteration, stream)
        self.set_mode(mode)

    def set_mode(self, mode):
        if mode not in ("shared", "cached"):
            raise ValueError("mode must be 'shared' or 'cached'")
        self.mode = mode
        self.b.aux_batch_set_mode(self.batch, self.b.AUX_MODE_SHARED_COV if mode == "shared"
                                  else self.b.AUX_MODE_CACHED_COV)

    def step(self, n_iters=1, accept_count=None, log_alpha=None, stream=None):
        self.b.aux_batch_step(self.batch, n_iters, accept_count, log_alpha, stream)

    def tune(self, reps=3, stream=None):
        return self.b.aux_batch_tune(self.batch, reps, stream)

    def config(self):
        return self.b.aux_batch_get_config(self.batch, len(self.models))

    def set_config(self, warps_per_cta=8, ctas_per_sm=0, order=0, block_factor=None, stream=None):
        self.b.aux_batch_set_config(self.batch, warps_per_cta, ctas_per_sm, order, block_factor, stream)

    def iteration(self):
        return self.b.aux_batch_get_iteration(self.batch)

    def set_iteration(self, it, stream=None):
        self.b.aux_batch_set_iteration(self.batch, it, stream)

    def status(self):
        return self.b.aux_batch_get_status(self.batch)

    def close(self):
        if getattr(self, "batch", None) is not None:
            self.b.aux_batch_free(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

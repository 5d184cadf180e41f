"""ctypes binding of the C ABI in include/aux_kalman.h (argument marshalling only).

Every function here has the name of the C entry point it calls. Device
buffers are passed as torch CUDA tensors (their data pointers) or raw
integer addresses; streams as torch.cuda.Stream, an integer handle or None
(the current torch stream). There is no fallback: if the compiled library
is missing, importing the binding raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

AUX_ABI_VERSION = 3
AUX_OK, AUX_E_INVALID_ARG, AUX_E_NOT_PD, AUX_E_NONFINITE = 0, 1, 2, 3
AUX_E_CUDA, AUX_E_TIMEOUT, AUX_E_OOM, AUX_E_UNSUPPORTED = 4, 5, 6, 7
AUX_E_TOO_LARGE = 8
AUX_NOALLOC_SCRATCH_BYTES = 32 << 20
AUX_F32, AUX_F64, AUX_MIXED = 0, 1, 2
AUX_DYN_HOMOGENEOUS, AUX_DYN_TIME_VARYING = 0, 1
AUX_EMIS_LINEAR_GAUSSIAN, AUX_EMIS_SV, AUX_EMIS_STUDENT_T = 0, 1, 2
AUX_MODE_PER_CHAIN, AUX_MODE_SHARED_COV, AUX_MODE_CACHED_COV = 0, 1, 2
AUX_PROPOSAL_FIRST_ORDER, AUX_PROPOSAL_SECOND_ORDER = 1, 2
AUX_SAMPLER_SCAN, AUX_SAMPLER_BRIDGING = 0, 1
AUX_FILTER_COVARIANCE, AUX_FILTER_SQUARE_ROOT = 0, 1

_dbl_p = ctypes.POINTER(ctypes.c_double)
_u8_p = ctypes.POINTER(ctypes.c_uint8)


class aux_model_desc(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_int32),
        ("dtype", ctypes.c_int32),
        ("d_x", ctypes.c_int32),
        ("T", ctypes.c_int32),
        ("n_chains", ctypes.c_int32),
        ("emis_kind", ctypes.c_int32),
        ("y_per_chain", ctypes.c_int32),
        ("block_len", ctypes.c_int32),
        ("m0", _dbl_p),
        ("P0", _dbl_p),
        ("F", _dbl_p),
        ("b", _dbl_p),
        ("Q", _dbl_p),
        ("y", _dbl_p),
        ("obs_mask", _u8_p),
        ("R_y", _dbl_p),
        ("delta", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("dyn_kind", ctypes.c_int32),
    ]


class AuxError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {aux_status_string(code)} (code {code})")


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(
            f"the CUDA library {path} is not built; run "
            "`python -m paper_2303_00301_gb300.build` (nvcc, sm_103a) first")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.aux_init_model.argtypes = [ctypes.POINTER(aux_model_desc), ctypes.c_uint64, vp,
                                   ctypes.POINTER(vp)]
    lib.aux_init_model.restype = ctypes.c_int
    lib.aux_kalman_step.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_uint64, vp, vp, vp]
    lib.aux_kalman_step.restype = ctypes.c_int
    lib.aux_loglik.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.aux_loglik.restype = ctypes.c_int
    lib.aux_sample_path.argtypes = [vp, vp, vp, ctypes.c_uint64, vp, vp, vp]
    lib.aux_sample_path.restype = ctypes.c_int
    lib.aux_get_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.aux_get_status.restype = ctypes.c_int
    lib.aux_free_model.argtypes = [vp]
    lib.aux_free_model.restype = None
    lib.aux_set_profiling.argtypes = [vp, ctypes.c_int32]
    lib.aux_set_profiling.restype = ctypes.c_int
    lib.aux_read_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
    lib.aux_read_profile.restype = ctypes.c_int
    lib.aux_set_mode.argtypes = [vp, ctypes.c_int32]
    lib.aux_set_mode.restype = ctypes.c_int
    lib.aux_set_proposal.argtypes = [vp, ctypes.c_int32]
    lib.aux_set_proposal.restype = ctypes.c_int
    lib.aux_set_delta_adaptation.argtypes = [vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double]
    lib.aux_set_delta_adaptation.restype = ctypes.c_int
    lib.aux_get_delta.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.aux_get_delta.restype = ctypes.c_int
    lib.aux_set_filter_form.argtypes = [vp, ctypes.c_int32]
    lib.aux_set_filter_form.restype = ctypes.c_int
    lib.aux_set_sampler.argtypes = [vp, ctypes.c_int32]
    lib.aux_set_sampler.restype = ctypes.c_int
    lib.aux_set_device_iteration.argtypes = [vp, ctypes.c_int32, ctypes.c_uint64]
    lib.aux_set_device_iteration.restype = ctypes.c_int
    lib.aux_get_device_iteration.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.aux_get_device_iteration.restype = ctypes.c_int
    lib.aux_loglik_grad.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.aux_loglik_grad.restype = ctypes.c_int
    lib.aux_set_grad_memory.argtypes = [vp, ctypes.c_uint64]
    lib.aux_set_grad_memory.restype = ctypes.c_int
    lib.aux_set_model_params.argtypes = [vp, ctypes.POINTER(aux_model_desc)]
    lib.aux_set_model_params.restype = ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    lib.aux_set_sv_theta.argtypes = [vp, dp, dp, dp, ctypes.c_double]
    lib.aux_set_sv_theta.restype = ctypes.c_int
    lib.aux_sv_theta_step.argtypes = [vp, vp, vp, vp, ctypes.c_double, vp]
    lib.aux_sv_theta_step.restype = ctypes.c_int
    lib.aux_get_sv_theta.argtypes = [vp, dp, dp, dp]
    lib.aux_get_sv_theta.restype = ctypes.c_int
    lib.aux_loglik_noalloc.argtypes = [ctypes.POINTER(aux_model_desc), vp, vp, vp]
    lib.aux_loglik_noalloc.restype = ctypes.c_int
    lib.aux_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int32, ctypes.c_uint64,
                                     vp, ctypes.POINTER(vp)]
    lib.aux_batch_create.restype = ctypes.c_int
    lib.aux_batch_set_mode.argtypes = [vp, ctypes.c_int32]
    lib.aux_batch_set_mode.restype = ctypes.c_int
    lib.aux_batch_step.argtypes = [vp, ctypes.c_int32, vp, vp, vp]
    lib.aux_batch_step.restype = ctypes.c_int
    lib.aux_batch_set_config.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, dp, vp]
    lib.aux_batch_set_config.restype = ctypes.c_int
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.aux_batch_get_config.argtypes = [vp, ip, ip, ip, dp, ip]
    lib.aux_batch_get_config.restype = ctypes.c_int
    lib.aux_batch_tune.argtypes = [vp, ctypes.c_int32, vp, dp]
    lib.aux_batch_tune.restype = ctypes.c_int
    lib.aux_batch_set_iteration.argtypes = [vp, ctypes.c_uint64, vp]
    lib.aux_batch_set_iteration.restype = ctypes.c_int
    lib.aux_batch_get_iteration.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.aux_batch_get_iteration.restype = ctypes.c_int
    lib.aux_batch_get_status.argtypes = [vp, ip]
    lib.aux_batch_get_status.restype = ctypes.c_int
    lib.aux_batch_free.argtypes = [vp]
    lib.aux_batch_free.restype = None
    lib.aux_status_string.argtypes = [ctypes.c_int]
    lib.aux_status_string.restype = ctypes.c_char_p
    return lib


LIB = _load()


def _ptr(t):
    """Device address of a torch tensor, an int address, or None -> NULL."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, where):
    if rc != AUX_OK:
        raise AuxError(rc, where)


def aux_status_string(code):
    return LIB.aux_status_string(int(code)).decode()


def _as_c(a, dtype=np.float64):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _make_desc(d_x, T, n_chains, m0, P0, F, b, Q, y, delta, emis_kind, dtype, R_y, obs_mask,
               y_per_chain, block_len, nu=0.0):
    """Fill an aux_model_desc; returns it with the numpy arrays it points into."""
    keep = dict(m0=_as_c(m0), P0=_as_c(P0), F=_as_c(F), b=_as_c(b), Q=_as_c(Q))
    if y is not None:
        keep["y"] = _as_c(y)
    desc = aux_model_desc()
    desc.abi_version = AUX_ABI_VERSION
    desc.dtype = int(dtype)
    desc.d_x, desc.T, desc.n_chains = int(d_x), int(T), int(n_chains)
    desc.emis_kind = int(emis_kind)
    desc.y_per_chain = 1 if y_per_chain else 0
    desc.block_len = int(block_len)
    # stacked transitions (F of shape [T-1][d][d]) are time-varying dynamics
    desc.dyn_kind = AUX_DYN_TIME_VARYING if keep["F"].ndim == 3 else AUX_DYN_HOMOGENEOUS
    for k, v in keep.items():
        setattr(desc, k, v.ctypes.data_as(_dbl_p))
    if R_y is not None:
        keep["R_y"] = _as_c(R_y)
        desc.R_y = keep["R_y"].ctypes.data_as(_dbl_p)
    if obs_mask is not None:
        keep["mask"] = _as_c(obs_mask, np.uint8)
        desc.obs_mask = keep["mask"].ctypes.data_as(_u8_p)
    desc.delta = float(delta)
    desc.nu = float(nu)
    return desc, keep


def aux_init_model(*, d_x, T, n_chains, m0, P0, F, b, Q, y, delta, emis_kind, dtype=AUX_F32,
                   R_y=None, obs_mask=None, y_per_chain=False, block_len=0, seed=0, stream=None, nu=0.0):
    """Create a model handle (host arrays are copied during the call)."""
    desc, keep = _make_desc(d_x, T, n_chains, m0, P0, F, b, Q, y, delta, emis_kind, dtype, R_y,
                            obs_mask, y_per_chain, block_len, nu)
    handle = ctypes.c_void_p()
    rc = LIB.aux_init_model(ctypes.byref(desc), ctypes.c_uint64(int(seed)), _stream(stream),
                            ctypes.byref(handle))
    _check(rc, "aux_init_model")
    del keep
    return handle


def aux_set_mode(handle, mode):
    _check(LIB.aux_set_mode(handle, int(mode)), "aux_set_mode")


def aux_set_proposal(handle, order):
    _check(LIB.aux_set_proposal(handle, int(order)), "aux_set_proposal")


def aux_set_delta_adaptation(handle, enable, target=0.5, gain=1.0):
    _check(LIB.aux_set_delta_adaptation(handle, 1 if enable else 0, float(target), float(gain)),
           "aux_set_delta_adaptation")


def aux_get_delta(handle):
    out = ctypes.c_double(0.0)
    _check(LIB.aux_get_delta(handle, ctypes.byref(out)), "aux_get_delta")
    return out.value


def aux_set_filter_form(handle, form):
    _check(LIB.aux_set_filter_form(handle, int(form)), "aux_set_filter_form")


def aux_set_sampler(handle, sampler):
    _check(LIB.aux_set_sampler(handle, int(sampler)), "aux_set_sampler")


def aux_set_device_iteration(handle, enable, start=0):
    _check(LIB.aux_set_device_iteration(handle, 1 if enable else 0, int(start)), "aux_set_device_iteration")


def aux_get_device_iteration(handle):
    out = ctypes.c_uint64(0)
    _check(LIB.aux_get_device_iteration(handle, ctypes.byref(out)), "aux_get_device_iteration")
    return out.value


def aux_loglik_grad(handle, ytilde, g_mu, g_Phi, g_cholSigma, g_delta, logZ=None, stream=None):
    rc = LIB.aux_loglik_grad(handle, _ptr(ytilde), _ptr(logZ), _ptr(g_mu), _ptr(g_Phi),
                             _ptr(g_cholSigma), _ptr(g_delta), _stream(stream))
    _check(rc, "aux_loglik_grad")


def aux_set_grad_memory(handle, max_bytes):
    """Cap aux_loglik_grad's store of G_t, Sigma_t, U_t (bytes; 0: store all)."""
    _check(LIB.aux_set_grad_memory(handle, int(max_bytes)), "aux_set_grad_memory")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def aux_set_sv_theta(handle, mu, phi, L, delta):
    """Write theta = (mu, phi, L = chol Sigma) and delta (host values) into the handle."""
    mu, phi, L = _as_c(mu), _as_c(phi), _as_c(L)
    _check(LIB.aux_set_sv_theta(handle, _dptr(mu), _dptr(phi), _dptr(L), float(delta)), "aux_set_sv_theta")


def aux_sv_theta_step(handle, g_mu, g_phi, g_L, lr, stream=None):
    """The on-device theta-update from per-chain gradients (device tensors)."""
    rc = LIB.aux_sv_theta_step(handle, _ptr(g_mu), _ptr(g_phi), _ptr(g_L), float(lr), _stream(stream))
    _check(rc, "aux_sv_theta_step")


def aux_get_sv_theta(handle, d):
    mu, phi, L = np.zeros(d), np.zeros(d), np.zeros((d, d))
    _check(LIB.aux_get_sv_theta(handle, _dptr(mu), _dptr(phi), _dptr(L)), "aux_get_sv_theta")
    return mu, phi, L


def aux_set_model_params(handle, *, d_x, T, n_chains, m0, P0, F, b, Q, y, delta, emis_kind,
                         dtype=AUX_F32, R_y=None, obs_mask=None, y_per_chain=False, block_len=0):
    desc, keep = _make_desc(d_x, T, n_chains, m0, P0, F, b, Q, y, delta, emis_kind, dtype, R_y,
                            obs_mask, y_per_chain, block_len)
    rc = LIB.aux_set_model_params(handle, ctypes.byref(desc))
    _check(rc, "aux_set_model_params")
    del keep


def aux_loglik_noalloc(ytilde, logZ, *, d_x, T, n_chains, m0, P0, F, b, Q, delta,
                       dtype=AUX_F32, block_len=0, stream=None):
    """aux_loglik without a handle or any device allocation (fixed library scratch)."""
    desc, keep = _make_desc(d_x, T, n_chains, m0, P0, F, b, Q, None, delta, 0, dtype, None,
                            None, False, block_len)
    rc = LIB.aux_loglik_noalloc(ctypes.byref(desc), _ptr(ytilde), _ptr(logZ), _stream(stream))
    _check(rc, "aux_loglik_noalloc")
    del keep


def aux_kalman_step(handle, x, n_iters, iter0=0, accept_count=None, log_alpha=None, stream=None):
    rc = LIB.aux_kalman_step(handle, _ptr(x), int(n_iters), ctypes.c_uint64(int(iter0)),
                             _ptr(accept_count), _ptr(log_alpha), _stream(stream))
    _check(rc, "aux_kalman_step")


def aux_loglik(handle, ytilde, logZ, mf=None, Pf=None, stream=None):
    rc = LIB.aux_loglik(handle, _ptr(ytilde), _ptr(logZ), _ptr(mf), _ptr(Pf), _stream(stream))
    _check(rc, "aux_loglik")


def aux_sample_path(handle, ytilde, xstar, eps=None, iteration=0, logZ=None, stream=None):
    rc = LIB.aux_sample_path(handle, _ptr(ytilde), _ptr(eps), ctypes.c_uint64(int(iteration)),
                             _ptr(xstar), _ptr(logZ), _stream(stream))
    _check(rc, "aux_sample_path")


def aux_get_status(handle, n_chains=None):
    """Returns (first_code, per-chain codes as a numpy array or None)."""
    if n_chains is None:
        return LIB.aux_get_status(handle, None), None
    buf = (ctypes.c_int32 * int(n_chains))()
    rc = LIB.aux_get_status(handle, buf)
    return rc, np.frombuffer(buf, dtype=np.int32).copy()


PROFILE_KINDS = ["linearise", "template", "reduce", "scan", "apply", "backward", "mh", "sum",
                 "smooth", "grad", "cov_reduce", "cov_scan", "cov_apply", "cov_products",
                 "bridge_tree", "bridge"]


def aux_set_profiling(handle, enable):
    _check(LIB.aux_set_profiling(handle, 1 if enable else 0), "aux_set_profiling")


def aux_read_profile(handle):
    """{kind: (total_ms, launches)} since the last read."""
    n = len(PROFILE_KINDS)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int32 * n)()
    _check(LIB.aux_read_profile(handle, ms, cnt, n), "aux_read_profile")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(PROFILE_KINDS)}


def aux_free_model(handle):
    LIB.aux_free_model(handle)


def aux_batch_create(handles, xs, iteration=0, stream=None):
    """A batch over model handles and their state tensors (device, FP32)."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    ps = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    out = ctypes.c_void_p()
    rc = LIB.aux_batch_create(hs, ps, n, ctypes.c_uint64(int(iteration)), _stream(stream), ctypes.byref(out))
    _check(rc, "aux_batch_create")
    return out


def aux_batch_set_mode(batch, mode):
    _check(LIB.aux_batch_set_mode(batch, int(mode)), "aux_batch_set_mode")


def aux_batch_step(batch, n_iters=1, accept_count=None, log_alpha=None, stream=None):
    rc = LIB.aux_batch_step(batch, int(n_iters), _ptr(accept_count), _ptr(log_alpha), _stream(stream))
    _check(rc, "aux_batch_step")


def aux_batch_set_config(batch, warps_per_cta, ctas_per_sm, order, block_factor=None, stream=None):
    bf = None if block_factor is None else _as_c(block_factor)
    rc = LIB.aux_batch_set_config(batch, int(warps_per_cta), int(ctas_per_sm), int(order),
                                  None if bf is None else _dptr(bf), _stream(stream))
    _check(rc, "aux_batch_set_config")


def aux_batch_get_config(batch, n_models):
    w, c, o = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    bf = np.zeros(4)
    bl = (ctypes.c_int32 * int(n_models))()
    _check(LIB.aux_batch_get_config(batch, ctypes.byref(w), ctypes.byref(c), ctypes.byref(o), _dptr(bf), bl),
           "aux_batch_get_config")
    return dict(warps_per_cta=w.value, ctas_per_sm=c.value, order=o.value, block_factor=bf.tolist(),
                block_len=list(bl))


def aux_batch_tune(batch, reps=3, stream=None):
    """Run the autotuner; returns the best time per step (ms)."""
    best = ctypes.c_double(0.0)
    _check(LIB.aux_batch_tune(batch, int(reps), _stream(stream), ctypes.byref(best)), "aux_batch_tune")
    return best.value


def aux_batch_set_iteration(batch, iteration, stream=None):
    _check(LIB.aux_batch_set_iteration(batch, ctypes.c_uint64(int(iteration)), _stream(stream)),
           "aux_batch_set_iteration")


def aux_batch_get_iteration(batch):
    out = ctypes.c_uint64(0)
    _check(LIB.aux_batch_get_iteration(batch, ctypes.byref(out)), "aux_batch_get_iteration")
    return out.value


def aux_batch_get_status(batch):
    """Returns (code, aborted)."""
    ab = ctypes.c_int32(0)
    rc = LIB.aux_batch_get_status(batch, ctypes.byref(ab))
    return rc, ab.value


def aux_batch_free(batch):
    LIB.aux_batch_free(batch)

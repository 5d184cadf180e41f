"""The C-ABI library without a GPU: it builds, loads, exports every declared
symbol, and rejects bad model descriptions on the host (no device call)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aux_kalman.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(aux_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_00301_gb300 import build
    build.build()
    from paper_2303_00301_gb300 import _binding
    return _binding


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["aux_init_model", "aux_kalman_step", "aux_loglik", "aux_sample_path",
              "aux_get_status", "aux_free_model", "aux_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    cdll = ctypes.CDLL(lib._build.LIB)
    for n in _declared_functions():
        assert hasattr(cdll, n), n


def test_status_strings(lib):
    assert lib.aux_status_string(0) == "ok"
    assert "positive definite" in lib.aux_status_string(lib.AUX_E_NOT_PD)
    assert lib.aux_status_string(999) == "unknown status"


def _desc_kwargs(**over):
    d, T = 2, 8
    kw = dict(d_x=d, T=T, n_chains=1, m0=np.zeros(d), P0=np.eye(d), F=0.9 * np.eye(d),
              b=np.zeros(d), Q=0.1 * np.eye(d), y=np.zeros((T, d)), delta=0.1,
              emis_kind=0, R_y=0.5 * np.eye(d), stream=0)
    kw.update(over)
    return kw


@pytest.mark.parametrize("over,code", [
    (dict(P0=np.array([[1.0, 2.0], [2.0, 1.0]])), 2),          # not PD
    (dict(Q=np.array([[1.0, 0.5], [0.0, 1.0]])), 2),           # not symmetric
    (dict(R_y=-np.eye(2)), 2),
    (dict(y=np.full((8, 2), np.nan)), 3),                      # non-finite
    (dict(delta=0.0), 1),
    (dict(delta=-1.0), 1),
    (dict(d_x=0), 1),
    (dict(T=0), 1),
    (dict(n_chains=0), 1),
    (dict(emis_kind=7), 1),
    (dict(dtype=5), 1),
    (dict(d_x=129, m0=np.zeros(129), P0=np.eye(129), F=np.eye(129), b=np.zeros(129), Q=np.eye(129),
          y=np.zeros((8, 129)), R_y=np.eye(129)), 7),          # beyond the built sizes
    (dict(dtype=1, d_x=33, m0=np.zeros(33), P0=np.eye(33), F=np.eye(33), b=np.zeros(33), Q=np.eye(33),
          y=np.zeros((8, 33)), R_y=np.eye(33)), 7),            # FP64 stops at 16
    (dict(emis_kind=2, nu=1.0, Q=np.array([[0.1, 0.02], [0.02, 0.1]])), 7),   # Student-t needs a diagonal prior
    (dict(emis_kind=2, nu=0.0), 1),                            # Student-t needs nu > 0
    (dict(emis_kind=2, nu=1.0, R_y=None), 1),                  # and a scale matrix
    (dict(emis_kind=2, nu=1.0, R_y=np.array([[1.0, 2.0], [2.0, 1.0]])), 2),
    (dict(emis_kind=2, nu=1.0, d_x=1025, m0=np.zeros(1025), P0=np.eye(1025), F=np.eye(1025),
          b=np.zeros(1025), Q=np.eye(1025), y=np.zeros((8, 1025)), R_y=np.eye(1025)), 7),
])
def test_init_rejects_bad_descriptions_on_host(lib, over, code):
    with pytest.raises(lib.AuxError) as e:
        lib.aux_init_model(**_desc_kwargs(**over))
    assert e.value.code == code


def test_batch_entry_points_reject_bad_arguments_on_host(lib):
    """The batch calls check their arguments before any device call."""
    L = lib.LIB
    out = ctypes.c_void_p()
    vp = ctypes.c_void_p
    assert L.aux_batch_create(None, None, 1, 0, None, ctypes.byref(out)) == lib.AUX_E_INVALID_ARG
    hs = (vp * 1)(None)
    xs = (vp * 1)(None)
    assert L.aux_batch_create(hs, xs, 1, 0, None, ctypes.byref(out)) == lib.AUX_E_INVALID_ARG
    assert L.aux_batch_create(hs, xs, 0, 0, None, ctypes.byref(out)) == lib.AUX_E_INVALID_ARG
    assert L.aux_batch_step(None, 1, None, None, None) == lib.AUX_E_INVALID_ARG
    assert L.aux_batch_set_mode(None, lib.AUX_MODE_CACHED_COV) == lib.AUX_E_INVALID_ARG
    assert L.aux_batch_tune(None, 1, None, None) == lib.AUX_E_INVALID_ARG
    assert L.aux_batch_set_config(None, 8, 0, 0, None, None) == lib.AUX_E_INVALID_ARG
    assert L.aux_batch_get_status(None, None) == lib.AUX_E_INVALID_ARG
    L.aux_batch_free(None)   # a no-op


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    """The binding has no CPU fallback: a missing library is an import error."""
    import importlib
    from paper_2303_00301_gb300 import build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    import paper_2303_00301_gb300._binding as b
    with pytest.raises(ImportError):
        importlib.reload(b)
    monkeypatch.undo()
    importlib.reload(b)

"""Pins of the oracle's Philox4x32-10 + Box-Muller streams (no GPU)."""
import os

import numpy as np
import pytest

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(v, 16) for v in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_known_answer_vectors(ctr, key, expect):
    out = philox.philox4x32_10(np.array(ctr), np.array(key))
    assert [int(v) for v in out] == expect


def test_uniform_exact_and_open_interval():
    r = np.array([0, 1, 511, 512, 2 ** 32 - 1], dtype=np.uint64)
    u = philox.words_to_uniform(r)
    assert u.min() > 0.0 and u.max() < 1.0
    # exactly representable in binary32
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    assert u[0] == 0.5 * 2.0 ** -23 and u[-1] == 1.0 - 0.5 * 2.0 ** -23


def test_streams_distinct_and_deterministic():
    a = philox.normals(1, 0, 0, philox.PURPOSE_AUX, np.arange(8), 30)
    b = philox.normals(1, 0, 0, philox.PURPOSE_AUX, np.arange(8), 30)
    c = philox.normals(1, 0, 0, philox.PURPOSE_BACKWARD, np.arange(8), 30)
    d = philox.normals(1, 1, 0, philox.PURPOSE_AUX, np.arange(8), 30)
    e = philox.normals(1, 0, 1, philox.PURPOSE_AUX, np.arange(8), 30)
    f = philox.normals(2, 0, 0, philox.PURPOSE_AUX, np.arange(8), 30)
    assert np.array_equal(a, b)
    for other in (c, d, e, f):
        assert not np.allclose(a, other)
    # prefix property: the first d' normals do not depend on d
    assert np.array_equal(philox.normals(1, 0, 0, 0, 3, 5), philox.normals(1, 0, 0, 0, 3, 30)[:5])


def test_box_muller_is_standard_normal():
    from scipy import stats
    z = philox.normals(12345, np.arange(64)[:, None], 7, philox.PURPOSE_AUX,
                       np.arange(256)[None, :], 32).reshape(-1)
    assert abs(z.mean()) < 4.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4.0 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_mh_uniform_range():
    u = philox.mh_uniform(3, np.arange(1000), 5)
    assert u.min() > 0 and u.max() < 1
    from scipy import stats
    assert stats.kstest(u, "uniform").pvalue > 1e-3

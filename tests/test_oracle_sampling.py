"""Pins of the oracle's random stream and AO direction sampling.

Philox4x32-10 against the published known-answer vectors; the 24-bit uniform
map; the Duff et al. orthonormal basis; cosine-weighted moments.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(oracle, ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_philox_counter_sensitivity(oracle):
    # every output word changes when one counter bit flips (avalanche, not a formula check)
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for word in range(4):
        c = [1, 2, 3, 4]
        c[word] ^= 1
        out = oracle.philox4x32_10(c, [5, 6])
        assert all(out[k] != base[k] for k in range(4))


def test_ao_uniform_map(oracle):
    # u1, u2 are the top 24 bits of words 0 and 1 of Philox(ctr=(i,s,frame,0xA0), key=seed)
    seed = 0x123456789ABCDEF0
    for (i, s, f) in [(0, 0, 0), (7, 3, 2), (1 << 20, 15, 63)]:
        x = oracle.philox4x32_10([i, s, f, 0xA0], [seed & 0xFFFFFFFF, seed >> 32])
        u1, u2 = oracle.ao_uniforms(i, s, f, seed)
        assert u1 == (int(x[0]) >> 8) / 2.0 ** 24
        assert u2 == (int(x[1]) >> 8) / 2.0 ** 24
        assert 0.0 <= u1 < 1.0 and 0.0 <= u2 < 1.0


def test_uniform_moments(oracle):
    n = 20000
    u = np.array([oracle.ao_uniforms(i, 0, 0, 42) for i in range(n)])
    # U[0,1): mean 1/2, variance 1/12, within 5 sigma
    for k in range(2):
        assert abs(u[:, k].mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
        assert abs(u[:, k].var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)
    assert abs(np.corrcoef(u[:, 0], u[:, 1])[0, 1]) < 5 / math.sqrt(n)


NORMALS = [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0, 1, 0), (0, 0, 0.0), (0.6, 0.0, -0.8),
           (1e-9, 0, -1.0), (0.3, -0.4, 0.866), (-0.5, -0.5, -0.70710678)]


@pytest.mark.parametrize("n", NORMALS)
def test_onb_orthonormal_right_handed(oracle, n):
    n = np.asarray(n, float)
    if np.linalg.norm(n) == 0:
        n = np.array([1.0, 0.0, 0.0])
        n[2] = -0.0
    n = n / np.linalg.norm(n)
    b1, b2 = oracle.onb(n)
    M = np.stack([b1, b2, n])
    assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
    assert np.allclose(np.cross(b1, b2), n, atol=1e-12)


def test_cosine_directions_hemisphere_and_moments(oracle):
    rng = np.random.default_rng(5)
    n = rng.standard_normal(3)
    n /= np.linalg.norm(n)
    b1, b2 = oracle.onb(n)
    N = 20000
    cz = np.empty(N)
    cx = np.empty(N)
    for i in range(N):
        u1, u2 = oracle.ao_uniforms(i, 0, 0, 9)
        d = oracle.cosine_dir(n, u1, u2)
        assert abs(np.linalg.norm(d) - 1) < 1e-12
        cz[i] = d @ n
        cx[i] = d @ b1
    assert cz.min() >= 0.0
    # cosine-weighted hemisphere: cos^2(theta) ~ U[0,1] -> E[cos] = 2/3, E[cos^2] = 1/2
    assert abs(cz.mean() - 2 / 3) < 5 * math.sqrt((0.5 - 4 / 9) / N)
    assert abs((cz ** 2).mean() - 0.5) < 5 * math.sqrt(1 / 12 / N)
    # symmetric about the normal: E[d . b1] = 0, E[(d . b1)^2] = (1 - 1/2)/2
    assert abs(cx.mean()) < 5 * math.sqrt(0.25 / N)
    assert abs((cx ** 2).mean() - 0.25) < 0.01


def test_cosine_sample_extremes(oracle):
    n = np.array([0.0, 0.0, 1.0])
    # u1 = 0 -> the normal itself
    assert np.allclose(oracle.cosine_dir(n, 0.0, 0.3), n)
    # u1 -> 1 -> horizon, at azimuth 2 pi u2 measured from b1
    b1, b2 = oracle.onb(n)
    d = oracle.cosine_dir(n, 1.0, 0.25)
    assert np.allclose(d, b2, atol=1e-12)

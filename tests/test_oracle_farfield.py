"""Pins of the oracle's far-field pattern (the leading FFAT term, paper Sec. 3.1) and of the
training-sample coordinates (paper Sec. 3.4). CPU only."""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synthetic as S

scipy_special = pytest.importorskip("scipy.special")


def _h1(n, x, derivative=False):
    return (scipy_special.spherical_jn(n, x, derivative=derivative)
            + 1j * scipy_special.spherical_yn(n, x, derivative=derivative))


def pulsating_error(level=3, k=2.0):
    """Exact surface data of the pulsating unit sphere (p = 1/(ik - 1), g = 1): the far field is
    p(1) e^{-ik} in every direction."""
    V, F = S.icosphere(level)
    pa = 1.0 / (1j * k - 1.0)
    dirs = oracle.ffat_directions(16, 8)
    ff = oracle.far_field(V, F, k, dirs, np.full(len(F), pa), np.ones(len(F), complex))
    return float(np.max(np.abs(ff - pa * np.exp(-1j * k))) / abs(pa))


def oscillating_error(level=3, k=1.5):
    """Exact surface data of the oscillating unit sphere (g = cos theta, p = A h1(k) cos theta
    with A = 1/(k h1'(k))): h1(x) ~ -e^{ix}/x, so the far field is -A cos(theta) / k."""
    V, F = S.icosphere(level)
    c, _, _ = oracle.geometry(V, F)
    A = 1.0 / (k * _h1(1, k, True))
    cz = c[:, 2] / np.linalg.norm(c, axis=1)
    dirs = oracle.ffat_directions(16, 8)
    ff = oracle.far_field(V, F, k, dirs, A * _h1(1, k) * cz, cz.astype(complex))
    exact = -A * dirs[:, 2] / k
    return float(np.max(np.abs(ff - exact)) / np.max(np.abs(exact)))


def test_pulsating_sphere_far_field():
    e2, e3 = pulsating_error(2), pulsating_error(3)
    assert e3 < e2 and e3 < 0.01, (e2, e3)


def test_oscillating_sphere_far_field():
    e2, e3 = oscillating_error(2), oscillating_error(3)
    assert e3 < e2 and e3 < 0.02, (e2, e3)


def test_far_field_is_the_limit_of_the_field():
    """r e^{-ikr} p(r d) from the field evaluation tends to the far field as 1/r."""
    Vs, F = S.ring_sphere(600)
    V = S.perturbed_ellipsoid(Vs, 4)
    k = 3.0
    rng = np.random.default_rng(0)
    p = rng.normal(size=len(F)) + 1j * rng.normal(size=len(F))
    g = rng.normal(size=len(F)) + 1j * rng.normal(size=len(F))
    dirs = oracle.ffat_directions(8, 4)
    ff = oracle.far_field(V, F, k, dirs, p, g)
    errs = []
    for R in (1e2, 1e3, 1e4):
        f = oracle.evaluate(V, F, k, R * dirs, p, g) * R * np.exp(-1j * k * R)
        errs.append(float(np.max(np.abs(f - ff)) / np.max(np.abs(ff))))
    assert errs[2] < 1e-3 and errs[0] / errs[2] > 50, errs  # O(1/r)
    # the same relation for a Monte-Carlo solution
    Y, N, A = S.sphere_samples(500)
    pm = rng.normal(size=500) + 1j * rng.normal(size=500)
    gm = rng.normal(size=500) + 1j * rng.normal(size=500)
    ffm = oracle.mc_far_field(Y, N, A, k, dirs, pm, gm)
    fm = oracle.mc_evaluate(Y, N, A, k, 1e4 * dirs, pm, gm) * 1e4 * np.exp(-1j * k * 1e4)
    assert np.max(np.abs(fm - ffm)) / np.max(np.abs(ffm)) < 1e-3


def test_sample_coordinates():
    rng = np.random.default_rng(1)
    u = rng.random((1000, 3))
    center = np.array([0.1, -0.2, 0.3])
    tpr, xyz = oracle.sample_coords(u, center, 1.5, 3.0)
    d = xyz - center
    r = np.linalg.norm(d, axis=1)
    assert np.allclose(r, tpr[:, 2]) and r.min() >= 1.5 and r.max() <= 3.0
    assert np.allclose(np.arccos(d[:, 2] / r), tpr[:, 0])
    assert np.allclose(np.mod(np.arctan2(d[:, 1], d[:, 0]), 2 * np.pi), tpr[:, 1])
    dirs = oracle.ffat_directions(64, 32)
    assert dirs.shape == (2048, 3) and np.allclose(np.linalg.norm(dirs, axis=1), 1.0)


def test_planted_far_field_sign_is_caught():
    path = os.path.join(tempfile.mkdtemp(), "liboracle_plant9.so")
    oracle.build_variant(path, 9)
    with oracle.using_library(path):
        assert pulsating_error() > 0.01 or oscillating_error() > 0.02

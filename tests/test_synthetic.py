"""The seeded input generators give valid closed meshes with the stated sizes."""
import numpy as np
import pytest

import synthetic as S


@pytest.mark.parametrize("n", [8, 64, 500, 1000, 5174, 10240])
def test_ring_sphere_counts(oracle_lib, n):
    V, F = S.ring_sphere(n)
    assert F.shape == (n, 3) and V.shape == (n // 2 + 2, 3)
    assert oracle_lib.validate_mesh(V, F) == 0


def test_named_meshes_valid(oracle_lib):
    for lev in range(4):
        V, F = S.icosphere(lev)
        assert F.shape[0] == 20 * 4 ** lev and oracle_lib.validate_mesh(V, F) == 0
    V, F = S.uv_sphere(128, 40)
    assert F.shape[0] == 10240 and V.shape[0] == 5122 and oracle_lib.validate_mesh(V, F) == 0
    V, F = S.ring_sphere(10240)
    assert oracle_lib.validate_mesh(S.perturbed_ellipsoid(V, 2000), F) == 0


def test_seeded_and_deterministic():
    a = S.interior_source(n_tri=512, n_k=4, n_points=8)
    b = S.interior_source(n_tri=512, n_k=4, n_points=8)
    assert np.array_equal(a.V, b.V) and np.array_equal(a.ks, b.ks)
    assert np.all((a.ks >= 0.5) & (a.ks <= 20.0))
    g = S.sh_neumann(a.V, a.F, 3, 11)
    assert g.shape == (512, 3) and np.all(g.imag == 0) and g.flags.f_contiguous


def test_real_sph_harm_orthonormal():
    # Gauss-Legendre x uniform-azimuth product rule, exact for degree <= 16
    x, w = np.polynomial.legendre.leggauss(20)
    ph = 2 * np.pi * np.arange(40) / 40
    z = np.repeat(x, 40)
    s = np.sqrt(1 - z * z)
    P = np.tile(ph, 20)
    d = np.stack([s * np.cos(P), s * np.sin(P), z], 1)
    W = np.repeat(w, 40) * 2 * np.pi / 40
    Y = S.real_sph_harm(6, d)
    G = (Y * W[:, None]).T @ Y
    assert np.allclose(G, np.eye(49), atol=1e-12)


def test_fibonacci_points_on_sphere():
    p = S.fibonacci_points(1024, 4.0)
    assert np.allclose(np.linalg.norm(p, axis=1), 4.0)
    q = S.shell_points(100, 2.0, 5.0, 3)
    r = np.linalg.norm(q, axis=1)
    assert r.min() >= 2.0 and r.max() <= 5.0

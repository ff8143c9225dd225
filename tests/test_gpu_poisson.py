"""GPU parity of the Poisson-disk surface sampler (nat_bem_poisson_sample; paper Sec. 4.2)
against the oracle's sequential definition on the same draws: the same accepted draws and
bit-identical positions and normals (both sides round every product and sum in FP64 in the
same order)."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import poisson as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build
    build.build()
    return nb


def _check(nb, V, F, u, r):
    idx, x, n = nb.nat_bem_poisson_sample(V, F, u, r)
    ai, ax, an = P.sample(V, F, u, r)
    assert np.array_equal(idx, ai), (len(idx), len(ai))
    assert np.array_equal(x, ax)
    assert np.array_equal(n, an)
    return idx, x


def _spacing(V, F, M):
    """Spacing of a hexagonal packing of M points on the mesh's area."""
    P0, P1, P2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    A = 0.5 * np.linalg.norm(np.cross(P1 - P0, P2 - P0), axis=1).sum()
    return math.sqrt(2.0 * A / (math.sqrt(3.0) * M))


@pytest.mark.parametrize("m,r", [(1, 0.1), (257, 0.3), (5000, 0.08), (20011, 0.05)])
def test_sphere_matches_oracle(nb, m, r):
    V, F = S.icosphere(3)
    u = np.random.default_rng(m).random((m, 3))
    idx, x = _check(nb, V, F, u, r)
    assert len(idx) >= 1
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)) + np.eye(len(x)) * 1e9
    assert d.min() >= r


def test_ellipsoid_matches_oracle_and_is_poisson(nb):
    Vs, F = S.ring_sphere(5120)
    V = S.perturbed_ellipsoid(Vs, 11)
    r = 0.7 * _spacing(V, F, 2000)
    u = np.random.default_rng(3).random((16000, 3))
    idx, x = _check(nb, V, F, u, r)
    d = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)) + np.eye(len(x)) * 1e9
    assert d.min() >= r


def test_mc_workload_size(nb):
    """The Monte-Carlo workload's body (ring sphere of 10240 triangles, perturbed ellipsoid)
    with 8 x 4096 draws at 0.7 of the hexagonal spacing of 4096 points."""
    Vs, F = S.ring_sphere(10240)
    V = S.perturbed_ellipsoid(Vs, 6000)
    u = np.random.default_rng(6001).random((8 * 4096, 3))
    idx, x = _check(nb, V, F, u, 0.7 * _spacing(V, F, 4096))
    assert 3000 < len(idx) < 5000


def test_edge_cases(nb):
    V, F = S.icosphere(2)
    idx, x, n = nb.nat_bem_poisson_sample(V, F, np.zeros((0, 3)), 0.1)
    assert len(idx) == 0 and x.shape == (0, 3)
    # a radius beyond the bounding box: one cell, the lowest-index draw alone
    u = np.random.default_rng(1).random((999, 3))
    idx, x = _check(nb, V, F, u, 10.0)
    assert list(idx) == [0]
    # draws at the ends of [0, 1): the first and the last triangle, vertices and edges
    u = np.array([[0.0, 0.0, 0.0], [1.0 - 2 ** -53, 1.0 - 2 ** -53, 1.0 - 2 ** -53], [0.5, 1.0, 0.0],
                  [0.25, 1.0, 1.0]])
    _check(nb, V, F, u, 0.02)


def test_cap_and_bad_input(nb):
    V, F = S.icosphere(2)
    u = np.random.default_rng(2).random((3000, 3))
    ai, _, _ = P.sample(V, F, u, 0.1)
    with pytest.raises(nb.NatBemError):
        nb.nat_bem_poisson_sample(V, F, u, 0.1, cap=len(ai) - 1)
    idx, _, _ = nb.nat_bem_poisson_sample(V, F, u, 0.1, cap=len(ai))
    assert np.array_equal(idx, ai)
    Fb = F.copy()
    Fb[3, 1] = len(V)
    with pytest.raises(nb.NatBemError):
        nb.nat_bem_poisson_sample(V, Fb, u, 0.1)
    Fd = F.copy()
    Fd[5, 2] = Fd[5, 1]  # degenerate triangle
    with pytest.raises(nb.NatBemError):
        nb.nat_bem_poisson_sample(V, Fd, u, 0.1)
    with pytest.raises(nb.NatBemError):
        nb.nat_bem_poisson_sample(V, F, u, 1e-6)  # more than 2^28 cells


def test_device_tensors(nb):
    import torch
    V, F = S.icosphere(3)
    u = np.random.default_rng(5).random((4096, 3))
    dev = torch.device("cuda", 0)
    idx, x, n = nb.nat_bem_poisson_sample(torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev),
                                          torch.from_numpy(u).to(dev), 0.07)
    torch.cuda.synchronize()
    ai, ax, an = P.sample(V, F, u, 0.07)
    assert np.array_equal(idx, ai)
    assert np.array_equal(x.cpu().numpy(), ax)
    assert np.array_equal(n.cpu().numpy(), an)

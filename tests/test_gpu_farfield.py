"""GPU parity of the far-field pattern (FFAT maps, paper Sec. 3.1 and 5) and of the training
sampler (paper Sec. 3.4) against the FP64 oracle."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def nb():
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build
    build.build()
    return nb


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _data(n, nrhs, seed):
    rng = np.random.default_rng(seed)
    p = (rng.normal(size=(n, nrhs)) + 1j * rng.normal(size=(n, nrhs))).astype(np.complex64)
    g = (rng.normal(size=(n, nrhs)) + 1j * rng.normal(size=(n, nrhs))).astype(np.complex64)
    return np.asfortranarray(p), np.asfortranarray(g)


@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_far_field_matches_oracle(nb, oracle_lib, nrhs):
    Vs, F = S.ring_sphere(1500)
    V = S.perturbed_ellipsoid(Vs, 12)
    k = 3.0
    dirs = oracle_lib.ffat_directions(64, 32)
    P, G = _data(len(F), nrhs, 5)
    with nb.Operator.assemble(V, F, k) as op:
        out = op.far_field(dirs, P if nrhs > 1 else P[:, 0], G if nrhs > 1 else G[:, 0])
    out = np.asarray(out).reshape(len(dirs), nrhs, order="F") if nrhs > 1 else np.asarray(out)[:, None]
    for s in range(nrhs):
        ref = oracle_lib.far_field(V, F, k, dirs, P[:, s].astype(np.complex128), G[:, s].astype(np.complex128))
        assert _rel(out[:, s], ref) < TOL


def test_far_field_of_a_monte_carlo_op(nb, oracle_lib):
    Y, N, A = S.sphere_samples(900, 1.1)
    k = 4.0
    dirs = oracle_lib.ffat_directions(64, 32)
    P, G = _data(900, 1, 6)
    with nb.Operator.assemble_mc(Y, N, A, k) as op:
        out = op.far_field(dirs, P[:, 0], G[:, 0])
    ref = oracle_lib.mc_far_field(Y, N, A, k, dirs, P[:, 0].astype(np.complex128), G[:, 0].astype(np.complex128))
    assert _rel(out, ref) < TOL


def test_ffat_map_of_the_pulsating_sphere(nb):
    """Solve on the GPU, then the 64 x 32 FFAT map: |F| = |p(a)| a for the pulsating sphere."""
    V, F = S.icosphere(3)
    k = 2.0
    g = np.ones(len(F), np.complex64)
    with nb.Operator.assemble(V, F, k) as op:
        p, info, st = op.solve(g)
        assert st == nb.NAT_BEM_OK
        import oracle
        ff = op.far_field(oracle.ffat_directions(64, 32), p, g)
    exact = abs(1.0 / (1j * k - 1.0))
    assert np.max(np.abs(np.abs(ff) - exact)) / exact < 0.03


@pytest.mark.parametrize("nrhs", [1, 2])
def test_training_samples_match_oracle(nb, oracle_lib, nrhs):
    """10,000 samples in the shell 1.5-3 bounding radii about the body (paper Sec. 3.4)."""
    Vs, F = S.ring_sphere(1200)
    V = S.perturbed_ellipsoid(Vs, 13)
    k = 2.5
    lo, hi = V.min(axis=0), V.max(axis=0)
    center, rb = 0.5 * (lo + hi), 0.5 * np.linalg.norm(hi - lo)
    u = np.random.default_rng(7).random((10000, 3))
    P, G = _data(len(F), nrhs, 8)
    with nb.Operator.assemble(V, F, k) as op:
        coords, amp = op.sample_field(u, center, 1.5 * rb, 3.0 * rb, P if nrhs > 1 else P[:, 0],
                                      G if nrhs > 1 else G[:, 0])
    tpr, xyz = oracle_lib.sample_coords(u, center, 1.5 * rb, 3.0 * rb)
    assert np.allclose(coords, tpr, rtol=0, atol=1e-12)
    amp = np.asarray(amp).reshape(10000, nrhs, order="F") if nrhs > 1 else np.asarray(amp)[:, None]
    for s in range(nrhs):
        ref = np.abs(oracle_lib.evaluate(V, F, k, xyz, P[:, s].astype(np.complex128), G[:, s].astype(np.complex128)))
        assert _rel(amp[:, s], ref) < TOL


def test_sampler_rejects_bad_radii(nb):
    V, F = S.icosphere(1)
    with nb.Operator.assemble(V, F, 1.0) as op:
        g = np.ones(len(F), np.complex64)
        with pytest.raises(nb.NatBemError):
            op.sample_field(np.zeros((4, 3)), np.zeros(3), 2.0, 1.0, g, g)


def test_dataset_step_at_full_size(nb, oracle_lib):
    """The dataset workload's configuration (interior-source body, 10240 triangles): the GPU
    solve, then 10,000 shell samples and the 64 x 32 FFAT map; sampled outputs against the
    oracle's field and far field of the same surface data."""
    prob = S.interior_source(n_k=1, ka_range=(6.0, 6.0))
    V, F, k = prob.V, prob.F, float(prob.ks[0])
    g = np.ascontiguousarray(prob.neumann[0][:, 0]).astype(np.complex64)
    lo, hi = V.min(axis=0), V.max(axis=0)
    center, rb = 0.5 * (lo + hi), 0.5 * np.linalg.norm(hi - lo)
    u = np.random.default_rng(70).random((10000, 3))
    dirs = oracle_lib.ffat_directions(64, 32)
    with nb.Operator.assemble(V, F, k) as op:
        p, info, st = op.solve(g)
        assert st == nb.NAT_BEM_OK
        coords, amp = op.sample_field(u, center, 1.5 * rb, 3.0 * rb, p, g)
        ff = op.far_field(dirs, p, g)
    pick = np.random.default_rng(71).choice(10000, 64, replace=False)
    _, xyz = oracle_lib.sample_coords(u[pick], center, 1.5 * rb, 3.0 * rb)
    p64, g64 = p.astype(np.complex128), g.astype(np.complex128)
    ref = np.abs(oracle_lib.evaluate(V, F, k, xyz, p64, g64))
    assert _rel(amp[pick], ref) < TOL
    dpick = np.random.default_rng(72).choice(len(dirs), 48, replace=False)
    ref_ff = oracle_lib.far_field(V, F, k, dirs[dpick], p64, g64)
    assert _rel(ff[dpick], ref_ff) < TOL

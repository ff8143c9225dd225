"""GPU parity of the Monte-Carlo BEM path (nat_bem_assemble_mc, paper Sec. 4.1.1 and 4.2)
against the FP64 oracle on the same seeded samples."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5    # FP32 operator rows against FP64
SOL_TOL = 1e-4   # surface pressure and field against the FP64 oracle


@pytest.fixture(scope="module")
def nb():
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build
    build.build()
    return nb


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _ellipsoid_samples(M, seed, poisson=True):
    Vs, F = S.ring_sphere(3000)
    V = S.perturbed_ellipsoid(Vs, 17)
    gen = S.mesh_poisson_samples if poisson else S.mesh_random_samples
    return gen(V, F, M, seed)


@pytest.mark.parametrize("case", ["sphere700", "ellipsoid1000", "random_ellipsoid333"])
@pytest.mark.parametrize("k", [1.3, 7.0])
def test_mc_operator_entries(nb, oracle_lib, case, k):
    if case == "sphere700":
        Y, N, A = S.sphere_samples(700, 1.2)
    elif case == "ellipsoid1000":
        Y, N, A = _ellipsoid_samples(1000, 4)
    else:
        Y, N, A = _ellipsoid_samples(333, 5, poisson=False)
    L, R = oracle_lib.mc_assemble(Y, N, A, k)
    with nb.Operator.assemble_mc(Y, N, A, k) as op:
        Lg = op.rows(0, 0, op.n).astype(np.complex128)
        Rg = op.rows(1, 0, op.n).astype(np.complex128)
    for G, O in ((Lg, L), (Rg, R)):
        err = np.linalg.norm(G - O, axis=1) / np.linalg.norm(O, axis=1)
        assert np.max(err) < OP_TOL, np.max(err)
    assert np.allclose(np.diag(Lg), 0.5) and np.allclose(np.diag(Rg), np.diag(R), rtol=1e-6)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mc_solve_and_field_match_oracle(nb, oracle_lib, prec):
    """Interior monopole on a perturbed ellipsoid with Poisson-disk samples: surface pressure
    and field against the oracle (parity), and against the exact solution (the Monte-Carlo
    discretisation error, a few percent at 2000 samples)."""
    Y, N, A = _ellipsoid_samples(2000, 6)
    k = 2.5
    g = S.monopole_neumann_at(Y, N, k)
    pts = S.fibonacci_points(96, 4.0)
    p_ref, info = oracle_lib.mc_solve(Y, N, A, k, g, tol=1e-10)
    f_ref = oracle_lib.mc_evaluate(Y, N, A, k, pts, p_ref, g)
    opts = nb.nat_bem_opts_default(prec=nb.PREC_MIXED_BF16 if prec == "bf16" else nb.PREC_FP32)
    with nb.Operator.assemble_mc(Y, N, A, k, opts) as op:
        p, sinfo, st = op.solve(g.astype(np.complex64))
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        f = op.evaluate(pts, p, g.astype(np.complex64))
    assert _rel(p, p_ref) < SOL_TOL
    assert _rel(f, f_ref) < SOL_TOL
    assert _rel(p, S.monopole_field(Y, k)) < 0.08
    assert _rel(f, S.monopole_field(pts, k)) < 0.08


def test_mc_reassemble_matches_fresh(nb):
    Y, N, A = S.sphere_samples(600)
    with nb.Operator.assemble_mc(Y, N, A, 1.0) as op:
        op.reassemble(4.2)
        L1 = op.rows(0, 0, op.n)
        R1 = op.rows(1, 0, op.n)
    with nb.Operator.assemble_mc(Y, N, A, 4.2) as op:
        assert np.array_equal(op.rows(0, 0, op.n), L1)
        assert np.array_equal(op.rows(1, 0, op.n), R1)


def test_mc_full_size_sampled_rows(nb, oracle_lib):
    """4096 Poisson-disk samples (the bench's size) at ka = 10: sampled rows and the solve."""
    Y, N, A = _ellipsoid_samples(4096, 8)
    k = 10.0
    L, R = oracle_lib.mc_assemble(Y, N, A, k)
    rows = np.array([0, 1, 777, 2048, 4095])
    g = S.monopole_neumann_at(Y, N, k)
    with nb.Operator.assemble_mc(Y, N, A, k) as op:
        for r in rows:
            for which, M in ((0, L), (1, R)):
                row = op.rows(which, int(r), 1).astype(np.complex128)[0]
                assert np.linalg.norm(row - M[r]) / np.linalg.norm(M[r]) < OP_TOL
        p, info, st = op.solve(g.astype(np.complex64))
        assert st == nb.NAT_BEM_OK
    p_ref = np.linalg.solve(L, R @ g)
    assert _rel(p, p_ref) < SOL_TOL


def test_mc_rejects_non_unit_normals(nb):
    Y, N, A = S.sphere_samples(64)
    N = N * 1.01
    with pytest.raises(nb.NatBemError) as e:
        nb.Operator.assemble_mc(Y, N, A, 2.0)
    assert "EINVAL" in str(e.value)


def test_gpu_poisson_samples_through_the_mc_solve(nb, oracle_lib):
    """The Monte-Carlo path end to end on the device: Poisson-disk samples from the GPU sampler
    (identical to the sampler's reference), Monte-Carlo operators on them, solve and field,
    against the FP64 oracle on the same samples; and against the exact interior-source field
    (the Monte-Carlo discretisation error)."""
    from oracle import poisson as PS
    Vs, F = S.ring_sphere(3000)
    V = S.perturbed_ellipsoid(Vs, 17)
    u, radius = S.poisson_draws(V, F, 1500, 21)
    idx, Y, N = nb.nat_bem_poisson_sample(V, F, u, radius)
    ai, ay, an = PS.sample(V, F, u, radius)
    assert np.array_equal(idx, ai) and np.array_equal(Y, ay) and np.array_equal(N, an)
    P0, P1, P2 = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    A = 0.5 * float(np.linalg.norm(np.cross(P1 - P0, P2 - P0), axis=1).sum())
    k = 3.0
    g = S.monopole_neumann_at(Y, N, k)
    pts = S.fibonacci_points(64, 4.0)
    p_ref, info = oracle_lib.mc_solve(Y, N, A, k, g, tol=1e-10)
    f_ref = oracle_lib.mc_evaluate(Y, N, A, k, pts, p_ref, g)
    with nb.Operator.assemble_mc(Y, N, A, k) as op:
        p, sinfo, st = op.solve(g.astype(np.complex64))
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        f = op.evaluate(pts, p, g.astype(np.complex64))
    assert _rel(p, p_ref) < SOL_TOL
    assert _rel(f, f_ref) < SOL_TOL
    assert _rel(f, S.monopole_field(pts, k)) < 0.08

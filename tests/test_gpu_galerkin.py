"""GPU parity of the Galerkin Burton-Miller path (nat_bem_assemble_galerkin; paper Sec. 4, Eq. 6
with the element-to-element integration of Sec. 4.1) against the FP64 oracle on the same
meshes: operator rows, the solve, the field, the far field and the training samples."""
import numpy as np
import pytest

import synthetic as S
from oracle import galerkin as Gk

pytestmark = pytest.mark.gpu

OP_TOL = 2e-5    # FP32 operator rows against FP64 (relative, per row)
SOL_TOL = 1e-4   # surface pressure and field against the FP64 oracle


@pytest.fixture(scope="module")
def nb():
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build
    build.build()
    return nb


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _mesh(case):
    if case == "sphere":
        return S.icosphere(2)
    V, F = S.icosphere(2)
    return S.perturbed_ellipsoid(V, 21), F


@pytest.fixture(scope="module")
def oracle_ops():
    out = {}
    for case in ("sphere", "ellipsoid"):
        for k in (1.3, 7.0):
            V, F = _mesh(case)
            out[(case, k)] = (V, F) + Gk.assemble(V, F, k)
    return out


@pytest.mark.parametrize("case", ["sphere", "ellipsoid"])
@pytest.mark.parametrize("k", [1.3, 7.0])
def test_operator_rows(nb, oracle_ops, case, k):
    V, F, L, R = oracle_ops[(case, k)]
    with nb.Operator.assemble_galerkin(V, F, k) as op:
        assert nb.nat_bem_op_neumann_size(op.handle) == len(F)
        Lg = op.rows(0, 0, len(V)).astype(np.complex128)
        Rg = op.rows(1, 0, len(V)).astype(np.complex128)
    for G, O in ((Lg, L), (Rg, R)):
        err = np.linalg.norm(G - O, axis=1) / np.linalg.norm(O, axis=1)
        assert np.max(err) < OP_TOL, np.max(err)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_solve_field_far_field_match_oracle(nb, oracle_ops, prec):
    V, F, L, R = oracle_ops[("ellipsoid", 7.0)]
    k = 7.0
    g = S.monopole_neumann(V, F, k, x0=(0.1, -0.05, 0.05))
    p_ref = np.linalg.solve(L, R @ g)
    pts = S.fibonacci_points(96, 3.0)
    f_ref = Gk.evaluate(V, F, k, pts, p_ref, g)
    dirs = S.fibonacci_points(64, 1.0)
    ff_ref = Gk.far_field(V, F, k, dirs, p_ref, g)
    opts = nb.nat_bem_opts_default(prec=nb.PREC_MIXED_BF16 if prec == "bf16" else nb.PREC_FP32)
    with nb.Operator.assemble_galerkin(V, F, k, opts) as op:
        p, info, st = op.solve(g.astype(np.complex64))
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        assert p.shape == (len(V),)
        f = op.evaluate(pts, p, g.astype(np.complex64))
        ff = op.far_field(dirs, p, g.astype(np.complex64))
    assert _rel(p, p_ref) < SOL_TOL
    assert _rel(f, f_ref) < SOL_TOL
    assert _rel(ff, ff_ref) < SOL_TOL
    # and the physics: the interior source's exterior field
    assert _rel(f, S.monopole_field(pts, k, x0=(0.1, -0.05, 0.05))) < 0.05


def test_multi_rhs_and_samples(nb, oracle_ops):
    V, F, L, R = oracle_ops[("sphere", 1.3)]
    k = 1.3
    G = np.asfortranarray(S.sh_neumann(V, F, 3, seed=4).astype(np.complex64))
    P_ref = np.linalg.solve(L, R @ G.astype(np.complex128))
    u = np.random.default_rng(9).random((2000, 3))
    with nb.Operator.assemble_galerkin(V, F, k) as op:
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK
        coords, amp = op.sample_field(u, np.zeros(3), 1.5, 3.0, P, G)
    assert P.shape == (len(V), 3)
    for s in range(3):
        assert _rel(P[:, s], P_ref[:, s]) < SOL_TOL
    import oracle
    tpr, xyz = oracle.sample_coords(u, np.zeros(3), 1.5, 3.0)
    for s in range(3):
        ref = np.abs(Gk.evaluate(V, F, k, xyz, P_ref[:, s], G[:, s].astype(np.complex128)))
        assert _rel(amp[:, s], ref) < SOL_TOL


def test_pulsating_sphere_exact(nb):
    """Level-3 icosphere (1280 triangles, 642 vertices): p = 1 / (ik - 1) within 0.2%."""
    V, F = S.icosphere(3)
    k = 2.0
    with nb.Operator.assemble_galerkin(V, F, k) as op:
        p, info, st = op.solve(np.ones(len(F), np.complex64))
        assert st == nb.NAT_BEM_OK
    assert _rel(p, np.full(len(V), 1.0 / (1j * k - 1.0))) < 0.002


def test_reassemble_matches_fresh(nb):
    V, F = S.icosphere(2)
    with nb.Operator.assemble_galerkin(V, F, 1.0) as op:
        op.reassemble(5.5)
        L1, R1 = op.rows(0, 0, len(V)), op.rows(1, 0, len(V))
    with nb.Operator.assemble_galerkin(V, F, 5.5) as op:
        assert np.array_equal(op.rows(0, 0, len(V)), L1)
        assert np.array_equal(op.rows(1, 0, len(V)), R1)


def test_full_size_sampled_rows(nb):
    """The bench's mesh size (ring sphere of 5120 triangles, 2562 vertices) at ka = 10: sampled
    rows against the oracle's row assembly, and a solve that converges."""
    Vs, F = S.ring_sphere(5120)
    V = S.perturbed_ellipsoid(Vs, 5)
    k = 10.0
    rows = [0, 1, 1000, len(V) - 1]
    Lr, Rr = Gk.assemble_rows(V, F, k, rows)
    g = S.monopole_neumann(V, F, k, x0=(0.05, 0.0, 0.0))
    with nb.Operator.assemble_galerkin(V, F, k) as op:
        for i, r in enumerate(rows):
            lg = op.rows(0, r, 1).astype(np.complex128)[0]
            rg = op.rows(1, r, 1).astype(np.complex128)[0]
            assert np.linalg.norm(lg - Lr[i]) / np.linalg.norm(Lr[i]) < OP_TOL
            assert np.linalg.norm(rg - Rr[i]) / np.linalg.norm(Rr[i]) < OP_TOL
        p, info, st = op.solve(g.astype(np.complex64))
        assert st == nb.NAT_BEM_OK
        assert info.rel_residual < 1e-5


def test_galerkin_rejects_bad_input(nb):
    V, F = S.icosphere(1)
    Vx = np.concatenate([V, [[5.0, 5.0, 5.0]]])  # a vertex no triangle uses
    with pytest.raises(nb.NatBemError):
        nb.Operator.assemble_galerkin(Vx, F, 1.0)
    with pytest.raises(nb.NatBemError):
        nb.Operator.assemble_galerkin(V, F, -1.0)

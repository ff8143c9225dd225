"""GPU path against the FP64 oracle, element by element, through the C ABI (needs a GB300).

Tolerances (from the arithmetic, stated where used):
  * operator rows: relative L2 per row <= 1e-5. The regular entries are FP32 kernel values
    summed over 7 points (about 40 FP32 operations each, relative rounding ~1e-6) with the
    phase reduced to [-pi, pi] and taken from the hardware sine/cosine (absolute error ~4e-7);
    the self and vertex-sharing entries take d = x - y in float-float arithmetic (or, for the
    self term, the vertices relative to the centroid in FP64) and FP32 after that, with no
    cancelling forms: each term ~1e-7 relative, checked elementwise at 1e-6.
  * surface and field pressure: relative L2 <= 1e-4, the accuracy target of the solver. The
    GPU solve stops at a relative residual of 1e-6 against an FP32 operator; the oracle solves
    to 1e-12 in FP64.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
SOL_TOL = 1e-4
# mixed solves: the true residual reaches tol = 1e-6, or at most 4 tol when a refinement sweep
# stalls there (the rounding floor of the FP32 residual product ends the solve)
FLOOR_TOL = 4e-6


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2506_06190_gb300 import build
    build.build()
    import paper_2506_06190_gb300 as nb
    return nb


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _rowwise(gpu, ref):
    return np.linalg.norm(gpu - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("mesh", ["tetrahedron", "octahedron", "ico1", "ring1000"])
@pytest.mark.parametrize("k", [0.7, 4.0])
def test_operator_entries(nb, oracle_lib, mesh, k):
    V, F = {"tetrahedron": S.tetrahedron, "octahedron": S.octahedron,
            "ico1": lambda: S.icosphere(1), "ring1000": lambda: S.ring_sphere(1000)}[mesh]()
    if mesh == "ring1000":
        V = S.perturbed_ellipsoid(V, 11)
    L, R = oracle_lib.assemble(V, F, k)
    with nb.Operator.assemble(V, F, k) as op:
        Lg = op.rows(0, 0, op.n).astype(np.complex128)
        Rg = op.rows(1, 0, op.n).astype(np.complex128)
    assert np.max(_rowwise(Lg, L)) < OP_TOL
    assert np.max(_rowwise(Rg, R)) < OP_TOL
    # the self and vertex-sharing entries (float-float d, FP32 after it) are accurate elementwise
    near = np.array([[len(set(F[i]) & set(F[j])) > 0 for j in range(len(F))] for i in range(len(F))])
    assert np.max(np.abs(Lg - L)[near] / np.abs(L)[near]) < 1e-6
    assert np.max(np.abs(Rg - R)[near] / np.abs(R)[near]) < 1e-6


def test_pulsating_sphere_solve_and_field(nb, oracle_lib):
    prob = S.pulsating_sphere()
    V, F, k = prob.V, prob.F, float(prob.ks[0])
    g = prob.neumann[0][:, 0]
    p_ref, info_ref = oracle_lib.solve(V, F, k, g)
    f_ref = oracle_lib.evaluate(V, F, k, prob.points, p_ref, g)
    with nb.Operator.assemble(V, F, k) as op:
        rows = np.arange(0, op.n, 97)
        Lg = op.rows(0, 0, op.n).astype(np.complex128)
        assert np.max(_rowwise(Lg[rows], info_ref["L"][rows])) < OP_TOL
        p, info, st = op.solve(g)
        assert st == nb.NAT_BEM_OK and info.rel_residual < 1e-5 and info.iterations > 0
        fld = op.evaluate(prob.points, p, g)
    assert _rel(p, p_ref) < SOL_TOL
    assert _rel(fld, f_ref) < SOL_TOL
    # discretisation error against the closed form is the oracle's (about 1.7% here)
    exact = 1.0 / (1j * k - 1.0)
    assert _rel(p, np.full_like(p_ref, exact)) < 0.03


@pytest.mark.parametrize("n_tri", [576, 1000, 2306])
def test_ragged_sizes_interior_source(nb, oracle_lib, n_tri):
    """Triangle counts that are not multiples of the 32-column padding or of the tiles."""
    Vs, F = S.ring_sphere(n_tri)
    V = S.perturbed_ellipsoid(Vs, 2000 + n_tri)
    k = 5.3
    g = S.monopole_neumann(V, F, k)
    pts = S.fibonacci_points(77, 4.0)
    p_ref, _ = oracle_lib.solve(V, F, k, g)
    f_ref = oracle_lib.evaluate(V, F, k, pts, p_ref, g)
    with nb.Operator.assemble(V, F, k) as op:
        p, info, st = op.solve(g)
        assert st == nb.NAT_BEM_OK
        fld = op.evaluate(pts, p, g)
    assert _rel(p, p_ref) < SOL_TOL
    assert _rel(fld, f_ref) < SOL_TOL


def test_multi_rhs_matches_oracle_and_single(nb, oracle_lib):
    Vs, F = S.ring_sphere(800)
    V = S.perturbed_ellipsoid(Vs, 7)
    k = 3.1
    G = S.sh_neumann(V, F, 5, 99)
    pts = S.shell_points(64, 2.0, 5.0, 1)
    L, R = oracle_lib.assemble(V, F, k)
    with nb.Operator.assemble(V, F, k) as op:
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK
        fld = op.evaluate(pts, P, G)
        for s in range(G.shape[1]):
            p_ref = np.linalg.solve(L, R @ G[:, s])
            assert _rel(P[:, s], p_ref) < SOL_TOL
            f_ref = oracle_lib.evaluate(V, F, k, pts, p_ref, G[:, s])
            assert _rel(fld[:, s], f_ref) < SOL_TOL
        # alone (GEMV products) and inside the block (FP32 GEMM products) the same RHS agrees
        # to FP32 rounding; the bitwise check of the same request alone and in a mix is in
        # test_serving.py
        for s in (0, 3):
            p1, _, _ = op.solve(G[:, s])
            assert _rel(p1, P[:, s]) < 1e-5


@pytest.mark.parametrize("device_loop", [1, 0])
def test_fewer_columns_on_a_reused_workspace(nb, device_loop):
    """A solve with 6 RHS, then one with 5 and one with 3 of them on the same operator (its
    workspace and captured graphs are reused): each result has the bits of the same columns
    solved on a fresh operator, with the device-side loop and with host-polled chunks."""
    Vs, F = S.ring_sphere(900)
    V = S.perturbed_ellipsoid(Vs, 11)
    G = S.sh_neumann(V, F, 6, 12)
    opts = nb.nat_bem_opts_default(device_loop=device_loop)
    with nb.Operator.assemble(V, F, 2.7, opts) as op:
        for cols in (6, 5, 3):
            p, info, st = op.solve(np.asfortranarray(G[:, :cols]))
            assert st == nb.NAT_BEM_OK
            with nb.Operator.assemble(V, F, 2.7, opts) as fresh:
                p1, info1, st1 = fresh.solve(np.asfortranarray(G[:, :cols]))
            assert st1 == nb.NAT_BEM_OK and info.iterations == info1.iterations
            assert np.array_equal(p, p1), cols


def test_default_stream_solve_is_ordered_and_matches_explicit_stream(nb):
    """A solve called on the legacy default stream runs on the op's own stream (so its GMRES
    chunks can be captured as graphs): it must still see the Neumann data that a kernel queued
    just before it on the default stream wrote, and give the bits of the same solve on an
    explicit stream."""
    import torch
    Vs, F = S.ring_sphere(1200)
    V = S.perturbed_ellipsoid(Vs, 21)
    g = S.monopole_neumann(V, F, 2.5).astype(np.complex64)
    with nb.Operator.assemble(V, F, 2.5) as op:
        torch.cuda.synchronize()
        gd = torch.zeros(len(F), dtype=torch.complex64, device="cuda")
        big = torch.randn(4096, 4096, device="cuda")
        _ = big @ big  # keeps the default stream busy for a while
        gd.copy_(torch.from_numpy(g).cuda())  # queued behind it, not yet done when solve starts
        p0, info0, st0 = op.solve(gd)
        assert st0 == nb.NAT_BEM_OK
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            p1, info1, st1 = op.solve(torch.from_numpy(g).cuda(), stream=st.cuda_stream)
        torch.cuda.synchronize()
        assert st1 == nb.NAT_BEM_OK
    assert np.array_equal(p0.cpu().numpy(), p1.cpu().numpy())


def test_device_pointers_match_host(nb):
    import torch
    V, F = S.icosphere(2)
    k = 2.2
    g = S.cos_theta_neumann(V, F).astype(np.complex64)
    pts = S.fibonacci_points(40, 3.0)
    with nb.Operator.assemble(V, F, k) as op:
        p_h, _, _ = op.solve(g)
        f_h = op.evaluate(pts, p_h, g)
    Vd, Fd = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    gd = torch.from_numpy(g).cuda()
    with nb.Operator.assemble(Vd, Fd, k) as op:
        p_d, _, _ = op.solve(gd)
        f_d = op.evaluate(torch.from_numpy(pts).cuda(), p_d, gd)
        torch.cuda.synchronize()
    assert np.array_equal(p_d.cpu().numpy(), p_h)
    assert np.array_equal(f_d.cpu().numpy(), f_h)


def test_nonconvergence_reports_enoconv(nb, oracle_lib):
    V, F = S.icosphere(2)
    opts = nb.nat_bem_opts_default(max_iter=2)
    g = S.uniform_neumann(F)
    with nb.Operator.assemble(V, F, 6.0, opts) as op:
        p, info, st = op.solve(g)
    assert st == nb.NAT_BEM_ENOCONV and info.iterations == 2
    assert info.rel_residual > 1e-6 and np.all(np.isfinite(p))


def test_empty_field_and_errors(nb):
    V, F = S.icosphere(1)
    with nb.Operator.assemble(V, F, 1.0) as op:
        g = S.uniform_neumann(F)
        p, _, _ = op.solve(g)
        out = op.evaluate(np.zeros((0, 3)), p, g)
        assert out.shape[0] == 0
        with pytest.raises(nb.NatBemError):
            nb.nat_bem_op_rows(op.handle, 0, op.n - 1, 5)


@pytest.fixture(scope="module")
def full_size_ref(oracle_lib):
    """Oracle results on the 10240-triangle interior-source mesh (the bench's), per ka: sampled
    operator rows, the FP64 solution (GMRES to 1e-10) and the field at the 1024 points."""
    prob = S.interior_source(n_k=1)
    cache = {}

    def get(ka):
        if ka not in cache:
            V, F = prob.V, prob.F
            g = S.monopole_neumann(V, F, ka)
            rows = np.unique(np.concatenate([np.arange(0, len(F), 331), [len(F) - 1]]))
            Lr, Rr = oracle_lib.assemble_rows(V, F, ka, rows)
            p_ref, _ = oracle_lib.solve(V, F, ka, g, tol=1e-10)
            f_ref = oracle_lib.evaluate(V, F, ka, prob.points, p_ref, g)
            cache[ka] = dict(g=g, rows=rows, Lr=Lr, Rr=Rr, p=p_ref, f=f_ref)
        return cache[ka]

    return prob, get


PRECS = {"fp32": 0, "tf32": 1, "bf16": 2, "fp16": 3}


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("ka", [0.5, 5.0, 20.0])
def test_full_size_interior_source(nb, oracle_lib, full_size_ref, ka, prec):
    """The 10240-triangle interior-source mesh as the bench runs it, in plain FP32 and in the
    mixed BF16 form the bench's headline uses, at the low, middle and high end of its ka range:
    sampled operator rows against the oracle, the GPU solution against the oracle's full solve,
    the field at all 1024 points, and the discretisation error against the exact monopole
    field."""
    prob, get = full_size_ref
    ref = get(ka)
    V, F, g = prob.V, prob.F, ref["g"]
    opts = nb.nat_bem_opts_default(prec=PRECS[prec])
    with nb.Operator.assemble(V, F, ka, opts) as op:
        if prec == "fp32":
            Lg = np.concatenate([op.rows(0, int(r), 1) for r in ref["rows"]]).astype(np.complex128)
            Rg = np.concatenate([op.rows(1, int(r), 1) for r in ref["rows"]]).astype(np.complex128)
            assert np.max(_rowwise(Lg, ref["Lr"])) < OP_TOL and np.max(_rowwise(Rg, ref["Rr"])) < OP_TOL
            # each sampled row's self and vertex-sharing entries, elementwise as on small meshes
            for t, r in enumerate(ref["rows"]):
                near = np.isin(F, F[int(r)]).any(axis=1)
                for gpu, orc in ((Lg[t], ref["Lr"][t]), (Rg[t], ref["Rr"][t])):
                    assert np.max(np.abs(gpu - orc)[near] / np.abs(orc)[near]) < 1e-6, (ka, int(r))
        p, info, st = op.solve(g)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        if prec != "fp32":
            assert info.refinements >= 1
        fld = op.evaluate(prob.points, p, g)
    assert _rel(p, ref["p"]) < SOL_TOL
    assert _rel(fld, ref["f"]) < SOL_TOL
    c, _, _ = oracle_lib.geometry(V, F)
    assert _rel(p, S.monopole_field(c, ka)) < 0.1


def test_modal_multi_rhs_full_size_bf16(nb, oracle_lib):
    """The multi-RHS modal workload's shape: a 20480-triangle perturbed icosphere, 64 smooth
    right-hand sides solved in one block with BF16 tensor-core inner products and FP32
    refinement. Sampled operator rows against the oracle, and two right-hand sides against the
    oracle's FP64 solve (GMRES to 1e-10 on the full operator), surface and field."""
    prob = S.modal_multirhs(nrhs=64)
    V, F, k = prob.V, prob.F, float(np.max(prob.ks))  # the workload's highest wavenumber
    G = prob.neumann[0]
    pts = prob.points[::8]
    opts = nb.nat_bem_opts_default(prec=nb.PREC_MIXED_BF16)
    rows = np.unique(np.concatenate([np.arange(0, len(F), 997), [len(F) - 1]]))
    with nb.Operator.assemble(V, F, k, opts) as op:
        Lg = np.concatenate([op.rows(0, int(r), 1) for r in rows]).astype(np.complex128)
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        assert info.refinements >= 1
        fld = op.evaluate(pts, P, G)
    L, R = oracle_lib.assemble(V, F, k)
    assert np.max(_rowwise(Lg, L[rows])) < OP_TOL
    for s in (0, 63):
        p_ref, _, _, ok = oracle_lib.gmres(L, R @ G[:, s], tol=1e-10, maxit=400)
        assert ok
        assert _rel(P[:, s], p_ref) < SOL_TOL
        assert _rel(fld[:, s], oracle_lib.evaluate(V, F, k, pts, p_ref, G[:, s])) < SOL_TOL


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("ka", [1.0, 12.0])
def test_mixed_bf16_refinement_matches_oracle(nb, oracle_lib, ka, prec):
    """Inner GMRES on the BF16 (or row-scaled FP16) operator copy, refined against the FP32
    operator: the same 1e-4 bar against the FP64 oracle as the plain path."""
    Vs, F = S.ring_sphere(2306)
    V = S.perturbed_ellipsoid(Vs, 5)
    g = S.monopole_neumann(V, F, ka)
    G = np.stack([g, S.sh_neumann(V, F, 1, 3)[:, 0]], axis=1)
    pts = S.fibonacci_points(64, 4.0)
    L, R = oracle_lib.assemble(V, F, ka)
    opts = nb.nat_bem_opts_default(prec=PRECS[prec])
    with nb.Operator.assemble(V, F, ka, opts) as op:
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        assert info.refinements >= 1 and info.rel_residual <= FLOOR_TOL
        fld = op.evaluate(pts, P, G)
        if prec == "fp16":  # one RHS alone takes the FP16 GEMV (two take the tensor cores)
            p1, info1, st1 = op.solve(G[:, 0])
            assert st1 == nb.NAT_BEM_OK and _rel(p1, np.linalg.solve(L, R @ G[:, 0])) < SOL_TOL
    for s in range(2):
        p_ref = np.linalg.solve(L, R @ G[:, s])
        assert _rel(P[:, s], p_ref) < SOL_TOL
        assert _rel(fld[:, s], oracle_lib.evaluate(V, F, ka, pts, p_ref, G[:, s])) < SOL_TOL


@pytest.mark.parametrize("nrhs", [1, 3])
def test_mixed_bf16_high_wavenumber_converges(nb, oracle_lib, nrhs):
    """At ka = 20 the BF16 copy's error is close to the inner tolerance, so refinement sweeps
    stop contracting; the solve then finishes the correction equation on the FP32 operator and
    still meets the tolerance and the 1e-4 bar."""
    Vs, F = S.ring_sphere(2306)
    V = S.perturbed_ellipsoid(Vs, 21)
    ka = 20.0
    G = np.stack([S.monopole_neumann(V, F, ka)] + [S.sh_neumann(V, F, 1, 30 + q)[:, 0] for q in range(nrhs - 1)],
                 axis=1)
    L, R = oracle_lib.assemble(V, F, ka)
    opts = nb.nat_bem_opts_default(prec=nb.PREC_MIXED_BF16)
    with nb.Operator.assemble(V, F, ka, opts) as op:
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        assert info.rel_residual <= FLOOR_TOL
    for s in range(nrhs):
        assert _rel(P[:, s], np.linalg.solve(L, R @ G[:, s])) < SOL_TOL


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_restarted_gmres_matches_oracle(nb, oracle_lib, prec):
    """GMRES(m) with m = 30 Krylov vectors (the unrestarted solve needs more at ka = 9): several
    cycles, each on the true residual, and the result within 1e-4 of the oracle on the surface
    and in the field, for two right-hand sides, plain and mixed."""
    Vs, F = S.ring_sphere(2306)
    V = S.perturbed_ellipsoid(Vs, 15)
    ka = 9.0
    G = np.stack([S.monopole_neumann(V, F, ka), S.sh_neumann(V, F, 1, 16)[:, 0]], axis=1)
    pts = S.fibonacci_points(64, 4.0)
    L, R = oracle_lib.assemble(V, F, ka)
    pc = nb.PREC_FP32 if prec == "fp32" else nb.PREC_MIXED_BF16
    with nb.Operator.assemble(V, F, ka, nb.nat_bem_opts_default(prec=pc)) as op:
        _, info_full, st = op.solve(G)
        assert st == nb.NAT_BEM_OK
    opts = nb.nat_bem_opts_default(prec=pc, restart=30, max_iter=3000)
    with nb.Operator.assemble(V, F, ka, opts) as op:
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        assert info.refinements >= 2 and info.iterations > 30
        fld = op.evaluate(pts, P, G)
    if prec == "fp32":
        assert info_full.iterations > 30  # so restarts really happened
    for s in range(2):
        p_ref = np.linalg.solve(L, R @ G[:, s])
        assert _rel(P[:, s], p_ref) < SOL_TOL
        assert _rel(fld[:, s], oracle_lib.evaluate(V, F, ka, pts, p_ref, G[:, s])) < SOL_TOL


def test_restart_at_or_beyond_max_iter_is_the_unrestarted_solve(nb):
    """restart >= max_iter keeps every Krylov vector: the same path and the same bits as the
    default (restart = 0)."""
    Vs, F = S.ring_sphere(1000)
    V = S.perturbed_ellipsoid(Vs, 17)
    g = S.monopole_neumann(V, F, 6.0)
    out = []
    for r in (0, 200, 255):
        with nb.Operator.assemble(V, F, 6.0, nb.nat_bem_opts_default(restart=r)) as op:
            p, info, st = op.solve(g)
            assert st == nb.NAT_BEM_OK and info.refinements == 0
            out.append(p)
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_reassemble_matches_fresh_assembly(nb):
    """A new wavenumber on an existing op gives the same operator bits as a fresh assembly."""
    Vs, F = S.ring_sphere(700)
    V = S.perturbed_ellipsoid(Vs, 9)
    g = S.monopole_neumann(V, F, 6.5)
    with nb.Operator.assemble(V, F, 1.5) as op:
        op.solve(S.monopole_neumann(V, F, 1.5))
        op.reassemble(6.5)
        L1 = op.rows(0, 0, op.n)
        R1 = op.rows(1, 0, op.n)
        p1, _, st1 = op.solve(g)
    with nb.Operator.assemble(V, F, 6.5) as op2:
        assert np.array_equal(op2.rows(0, 0, op2.n), L1) and np.array_equal(op2.rows(1, 0, op2.n), R1)
        p2, _, st2 = op2.solve(g)
    assert st1 == st2 == nb.NAT_BEM_OK and np.array_equal(p1, p2)
    with pytest.raises(nb.NatBemError):
        nb.nat_bem_reassemble(None, 1.0)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_run_batch_uneven_meshes_matches_single_solves(nb, oracle_lib, prec):
    """Batched solves over meshes of uneven size (two jobs share a mesh) give the same bits as
    one solve at a time, with any number of workers, in plain FP32 and in mixed precision;
    every job is checked against the oracle, surface and field."""
    opts = nb.nat_bem_opts_default(prec=nb.PREC_FP32 if prec == "fp32" else nb.PREC_MIXED_BF16)
    import torch
    jobs = []
    for i, n_tri in enumerate([520, 1300, 760, 2010]):
        Vs, F = S.ring_sphere(n_tri)
        V = S.perturbed_ellipsoid(Vs, 40 + i)
        k = 1.0 + 2.5 * i
        g = S.sh_neumann(V, F, 1, 50 + i)[:, 0]
        jobs.append(dict(V=V, F=F, k=k, neumann=g, points=S.fibonacci_points(33, 4.0)))
    jobs.append(dict(jobs[1], k=7.7, neumann=S.sh_neumann(jobs[1]["V"], jobs[1]["F"], 1, 77)[:, 0]))
    singles = []
    for jd in jobs:
        with nb.Operator.assemble(jd["V"], jd["F"], jd["k"], opts) as op:
            p, info, st = op.solve(jd["neumann"])
            singles.append((p, op.evaluate(jd["points"], p, jd["neumann"])))
    for conc in (1, 3):
        st, res = nb.nat_bem_run_batch(jobs, opts, concurrency=conc)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        for (p, f, info, s_, ms), (p1, f1) in zip(res, singles):
            assert s_ == nb.NAT_BEM_OK and info.iterations > 0 and ms > 0
            assert np.array_equal(p, p1) and np.array_equal(f, f1)
    for jd, r in zip(jobs, res):
        L, R = oracle_lib.assemble(jd["V"], jd["F"], jd["k"])
        p_ref = np.linalg.solve(L, R @ jd["neumann"])
        assert _rel(r[0], p_ref) < SOL_TOL
        assert _rel(r[1], oracle_lib.evaluate(jd["V"], jd["F"], jd["k"], jd["points"], p_ref, jd["neumann"])) < SOL_TOL


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_run_batch_fused_uneven_meshes_match_oracle(nb, oracle_lib, prec):
    """The fused batch (size buckets solved in lockstep as padded systems of independent
    operators) on nine meshes of 520-2300 triangles, two sharing a mesh, plus one job with two
    right-hand sides (solved on its own): every job within 1e-4 of the oracle on the surface
    and in the field, and within 1e-5 of the one-at-a-time batch driver. max_batch 3 forces
    several buckets of each size class."""
    opts = nb.nat_bem_opts_default(prec=PRECS[prec])
    jobs = []
    for i, n_tri in enumerate([520, 560, 610, 1300, 760, 2300, 1100, 990]):
        Vs, F = S.ring_sphere(n_tri)
        V = S.perturbed_ellipsoid(Vs, 60 + i)
        k = 1.0 + 1.3 * i
        jobs.append(dict(V=V, F=F, k=k, neumann=S.sh_neumann(V, F, 1, 70 + i)[:, 0],
                         points=S.fibonacci_points(29, 4.0)))
    jobs.append(dict(jobs[3], k=6.1, neumann=S.monopole_neumann(jobs[3]["V"], jobs[3]["F"], 6.1)))
    jobs.append(dict(jobs[4], k=2.2, neumann=S.sh_neumann(jobs[4]["V"], jobs[4]["F"], 2, 99)))
    st, fused = nb.nat_bem_run_batch_fused(jobs, opts, max_batch=3)
    assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
    st, ref = nb.nat_bem_run_batch(jobs, opts, concurrency=2)
    assert st == nb.NAT_BEM_OK
    for jd, r, r1 in zip(jobs, fused, ref):
        p, f, info, s_, ms = r
        assert s_ == nb.NAT_BEM_OK and info.iterations > 0 and ms > 0
        assert _rel(p, r1[0]) < 1e-5 and _rel(f, r1[1]) < 1e-5
        L, R = oracle_lib.assemble(jd["V"], jd["F"], jd["k"])
        G = np.asarray(jd["neumann"]).reshape(len(jd["F"]), -1)
        P = np.asarray(p).reshape(len(jd["F"]), -1, order="F")
        Fd = np.asarray(f).reshape(len(jd["points"]), -1, order="F")
        for c in range(G.shape[1]):
            p_ref = np.linalg.solve(L, R @ G[:, c])
            assert _rel(P[:, c], p_ref) < SOL_TOL
            assert _rel(Fd[:, c], oracle_lib.evaluate(jd["V"], jd["F"], jd["k"], jd["points"], p_ref, G[:, c])) < SOL_TOL


def test_run_batch_fused_device_buffers_and_bad_mesh(nb):
    """Device arrays in, device results out; a mesh that fails its checks (inward winding)
    reports EINVAL for its job only, the rest of its bucket is solved."""
    import torch
    jobs = []
    for i, n_tri in enumerate([700, 720, 740]):
        Vs, F = S.ring_sphere(n_tri)
        V = S.perturbed_ellipsoid(Vs, 80 + i)
        g = S.monopole_neumann(V, F, 3.0).astype(np.complex64)
        if i == 1:
            F = np.ascontiguousarray(F[:, ::-1])
        jobs.append(dict(V=torch.from_numpy(V).cuda(), F=torch.from_numpy(F).cuda(), k=3.0,
                         neumann=torch.from_numpy(g).cuda(),
                         points=torch.from_numpy(S.fibonacci_points(17, 4.0)).cuda()))
    st, res = nb.nat_bem_run_batch_fused(jobs, max_batch=8)
    assert st == nb.NAT_BEM_EINVAL
    assert [r[3] for r in res] == [nb.NAT_BEM_OK, nb.NAT_BEM_EINVAL, nb.NAT_BEM_OK]
    for i in (0, 2):
        jd = jobs[i]
        with nb.Operator.assemble(jd["V"], jd["F"], 3.0) as op:
            p1, _, _ = op.solve(jd["neumann"])
            torch.cuda.synchronize()
        assert res[i][0].is_cuda
        assert _rel(res[i][0].cpu().numpy(), p1.cpu().numpy()) < 1e-5


@pytest.fixture(scope="module")
def product_case(oracle_lib):
    Vs, F = S.ring_sphere(1500)          # 1500 rows: the last 128-row tile is partial
    V = S.perturbed_ellipsoid(Vs, 77)
    k = 4.0
    L, R = oracle_lib.assemble(V, F, k)
    rng = np.random.default_rng(5)
    X = (rng.normal(size=(len(F), 100)) + 1j * rng.normal(size=(len(F), 100))).astype(np.complex64)
    return V, F, k, L, R, np.asfortranarray(X)


@pytest.mark.parametrize("variant", range(8))
def test_gemv_variants_match_oracle(nb, product_case, variant):
    """Every GEMV variant (register-tiled, bulk-copy, staged-x persistent) computes L x and R x
    to FP32 accuracy."""
    V, F, k, L, R, X = product_case
    x = X[:, 0].copy()
    with nb.Operator.assemble(V, F, k) as op:
        for which, M in ((0, L), (1, R)):
            y = op.apply(which, nb.ENGINE_GEMV0 + variant, x)
            assert _rel(y, M @ x.astype(np.complex128)) < 1e-5


@pytest.mark.parametrize("nrhs", [1, 6, 17, 40, 64, 100])
def test_fp32_gemm_matches_oracle(nb, product_case, nrhs):
    V, F, k, L, R, X = product_case
    Xs = np.asfortranarray(X[:, :nrhs])
    with nb.Operator.assemble(V, F, k) as op:
        for which, M in ((0, L), (1, R)):
            Y = op.apply(which, nb.ENGINE_FP32, Xs)
            ref = M @ Xs.astype(np.complex128)
            assert _rel(Y, ref) < 1e-5
            assert np.max(np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)) < 1e-5


@pytest.mark.parametrize("nrhs", [2, 8, 17, 64, 100])
def test_fp32_gemm_carries_fp32_accuracy(nb, product_case, nrhs, monkeypatch):
    """The FP32-accurate products against an FP64 product of the same FP32 operator entries,
    every column within 1e-6 (about 2e-7 on this case), and within 1e-6 of each other: the
    tensor-core form (L and X split into three BF16 pieces, six exact piece products, used for
    L with 8 RHS or more), the stream-K CUDA-core GEMM (NATBEM_NO_X6=1; float-float carries)
    and the fixed-tile one (NATBEM_CGEMM_TILED=1; FP64 carries)."""
    V, F, k, L, R, X = product_case
    Xs = np.asfortranarray(X[:, :nrhs])
    with nb.Operator.assemble(V, F, k) as op:
        for which in (0, 1):
            M = op.rows(which, 0, op.n).astype(np.complex128)
            ref = M @ Xs.astype(np.complex128)
            ys, errs = [], []
            for env in ({}, {"NATBEM_NO_X6": "1"}, {"NATBEM_NO_X6": "1", "NATBEM_CGEMM_TILED": "1"}):
                for v in ("NATBEM_NO_X6", "NATBEM_CGEMM_TILED"):
                    monkeypatch.delenv(v, raising=False)
                for kv in env.items():
                    monkeypatch.setenv(*kv)
                Y = op.apply(which, nb.ENGINE_FP32, Xs)
                err = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)
                assert err.max() < 1e-6, (env, err.max())
                ys.append(Y)
                errs.append(err.max())
            for v in ("NATBEM_NO_X6", "NATBEM_CGEMM_TILED"):
                monkeypatch.delenv(v, raising=False)
            assert _rel(ys[0], ys[1]) < 1e-6 and _rel(ys[1], ys[2]) < 1e-6
            if which == 0 and nrhs >= 8:  # the split product: no less accurate than the CUDA-core GEMM
                assert errs[0] <= 1.5 * errs[1] + 2e-8, errs


def test_fp32_products_full_size_accuracy(nb, monkeypatch):
    """At the modal size (20480 rows, K = 40960 real terms, 64 RHS), where long tensor-core
    accumulations lose accuracy: on 256 sampled rows, the split tensor-core product and the
    CUDA-core GEMM against an FP64 product of the same FP32 operator rows, per column within
    6e-7, the split one no less accurate than the CUDA-core one (measured 1.2e-7 against
    3.3e-7; with accumulator runs of four K blocks the split one reached 9.6e-7)."""
    prob = S.modal_multirhs(nrhs=64, n_k=1)
    rng = np.random.default_rng(41)
    with nb.Operator.assemble(prob.V, prob.F, float(prob.ks[0])) as op:
        n = op.n
        rows = np.sort(rng.choice(n, 256, replace=False))
        M = np.concatenate([op.rows(0, int(r), 1) for r in rows]).astype(np.complex128)
        X = np.asfortranarray((rng.normal(size=(n, 64)) + 1j * rng.normal(size=(n, 64))).astype(np.complex64))
        ref = M @ X.astype(np.complex128)
        errs = []
        for env in (None, "1"):
            if env:
                monkeypatch.setenv("NATBEM_NO_X6", env)
            else:
                monkeypatch.delenv("NATBEM_NO_X6", raising=False)
            Y = op.apply(0, nb.ENGINE_FP32, X)[rows]
            errs.append((np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)).max())
        monkeypatch.delenv("NATBEM_NO_X6", raising=False)
    assert max(errs) < 6e-7, errs
    assert errs[0] <= 1.5 * errs[1], errs


def test_plain_multi_rhs_solve_on_split_products(nb, oracle_lib, monkeypatch):
    """A plain FP32 solve with 12 RHS runs every matvec on the split tensor-core product: each
    RHS within 1e-4 of the FP64 oracle, within 1e-5 of the same solve on the CUDA-core GEMM,
    and a reassembly at another k rebuilds the split (the second solve matches a fresh op)."""
    Vs, F = S.ring_sphere(1500)
    V = S.perturbed_ellipsoid(Vs, 31)
    G = S.sh_neumann(V, F, 12, 32)
    out = {}
    for tag, env in (("x6", None), ("cuda_core", "1")):
        if env:
            monkeypatch.setenv("NATBEM_NO_X6", env)
        else:
            monkeypatch.delenv("NATBEM_NO_X6", raising=False)
        with nb.Operator.assemble(V, F, 2.0) as op:
            P, info, st = op.solve(G)
            assert st == nb.NAT_BEM_OK
            op.reassemble(4.5)
            P2, info2, st2 = op.solve(G)
            assert st2 == nb.NAT_BEM_OK
        out[tag] = (P, P2)
    monkeypatch.delenv("NATBEM_NO_X6", raising=False)
    for k, i in ((2.0, 0), (4.5, 1)):
        L, R = oracle_lib.assemble(V, F, k)
        Pref = np.linalg.solve(L, R @ G)
        for s in range(12):
            assert _rel(out["x6"][i][:, s], Pref[:, s]) < SOL_TOL
        assert _rel(out["x6"][i], out["cuda_core"][i]) < 1e-5
    with nb.Operator.assemble(V, F, 4.5) as fresh:
        P3, _, _ = fresh.solve(G)
    assert np.array_equal(P3, out["x6"][1])


@pytest.mark.parametrize("nrhs", [1, 6, 40, 64, 100])
def test_tensor_core_products_match_oracle(nb, product_case, nrhs):
    """tcgen05 TF32 (on L) and BF16 (on its copy) products: FP32 accumulation of operands
    carrying 10 (TF32, truncated by the MMA) and 8 (BF16, rounded) fraction bits, so the
    relative error is bounded by about 2^-10 and 2^-8 per product."""
    V, F, k, L, R, X = product_case
    Xs = np.asfortranarray(X[:, :nrhs])
    ref = L @ Xs.astype(np.complex128)
    opts = nb.nat_bem_opts_default(prec=nb.PREC_MIXED_BF16)
    with nb.Operator.assemble(V, F, k, opts) as op:
        Yt = op.apply(0, nb.ENGINE_TF32, Xs)
        Yb = op.apply(0, nb.ENGINE_BF16, Xs)
        with pytest.raises(nb.NatBemError):  # no FP16 copy on a BF16 op
            op.apply(0, nb.ENGINE_FP16, Xs)
    with nb.Operator.assemble(V, F, k, nb.nat_bem_opts_default(prec=nb.PREC_MIXED_FP16)) as op:
        Yh = op.apply(0, nb.ENGINE_FP16, Xs)
        with pytest.raises(nb.NatBemError):
            op.apply(0, nb.ENGINE_BF16, Xs)
    # FP16 keeps 11 significant bits (operator rows scaled into its range, x of unit scale):
    # 2^-11 per factor
    for Y, tol in ((Yt, 2e-3), (Yb, 8e-3), (Yh, 1.5e-3)):
        err = np.linalg.norm(Y.reshape(len(F), -1) - ref.reshape(len(F), -1), axis=0) / \
            np.linalg.norm(ref.reshape(len(F), -1), axis=0)
        assert np.all(err < tol), (err.max(), tol)
        assert np.all(err > 1e-7)  # really the reduced-precision path


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16"])
def test_multi_rhs_mixed_tensor_core_solve(nb, oracle_lib, prec):
    """Inner GMRES products on tensor cores, refinement against the FP32 operator: each RHS
    within 1e-4 of the FP64 oracle."""
    Vs, F = S.ring_sphere(1200)
    V = S.perturbed_ellipsoid(Vs, 8)
    k = 3.3
    G = S.sh_neumann(V, F, 8, 12)
    L, R = oracle_lib.assemble(V, F, k)
    opts = nb.nat_bem_opts_default(prec=PRECS[prec])
    with nb.Operator.assemble(V, F, k, opts) as op:
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        assert info.refinements >= 1 and info.rel_residual <= FLOOR_TOL
    for s in range(G.shape[1]):
        assert _rel(P[:, s], np.linalg.solve(L, R @ G[:, s])) < SOL_TOL


_LOOP_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import synthetic as S, paper_2506_06190_gb300 as nb
Vs, F = S.ring_sphere(2306)
V = S.perturbed_ellipsoid(Vs, 19)
out = []
for prec in (nb.PREC_FP32, nb.PREC_MIXED_BF16):
    g = np.stack([S.monopole_neumann(V, F, 7.0), S.sh_neumann(V, F, 1, 20)[:, 0]], axis=1)
    with nb.Operator.assemble(V, F, 7.0, nb.nat_bem_opts_default(prec=prec)) as op:
        p, info, st = op.solve(g[:, 0])
        out.append(p)
        p2, info, st = op.solve(g)
        out.append(p2.ravel(order="F"))
np.save(sys.argv[2], np.concatenate(out))
"""


def test_device_loop_option_gives_the_same_bits(nb):
    """opts.device_loop = 0 (host-polled chunks) and 1 (the loop on the device) run the same
    kernels in the same order: the same bits."""
    Vs, F = S.ring_sphere(1500)
    V = S.perturbed_ellipsoid(Vs, 23)
    g = S.monopole_neumann(V, F, 4.0)
    out = []
    for loop in (1, 0):
        with nb.Operator.assemble(V, F, 4.0, nb.nat_bem_opts_default(prec=nb.PREC_MIXED_BF16, device_loop=loop)) as op:
            p, info, st = op.solve(g)
            assert st == nb.NAT_BEM_OK
            out.append(p)
    assert np.array_equal(out[0], out[1])


def test_device_loop_matches_host_polled_chunks(tmp_path):
    """The GMRES loop run on the device (a conditional while node repeating a captured chunk)
    launches the same kernels in the same order as the host-polled chunks, so the results are
    the same bits, plain and mixed, one and two right-hand sides (two processes, one with the
    device loop switched off)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for off in (False, True):
        env = dict(os.environ)
        env.pop("NATBEM_NO_DEVICE_LOOP", None)
        if off:
            env["NATBEM_NO_DEVICE_LOOP"] = "1"
        f = str(tmp_path / f"p{int(off)}.npy")
        r = subprocess.run([sys.executable, "-c", _LOOP_CHILD, root, f], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(np.load(f))
    assert np.array_equal(outs[0], outs[1])


_BASIS_CHILD = r"""
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
import synthetic as S, paper_2506_06190_gb300 as nb
Vs, F = S.ring_sphere(1200)
V = S.perturbed_ellipsoid(Vs, 8)
out, its = [], []
for k, prec, nr in ((3.3, nb.PREC_MIXED_BF16, 8), (3.3, nb.PREC_MIXED_TF32, 8), (14.0, nb.PREC_MIXED_BF16, 8),
                    (3.3, nb.PREC_MIXED_BF16, 1), (14.0, nb.PREC_MIXED_BF16, 1)):
    G = S.sh_neumann(V, F, 8, 12)[:, :nr]
    with nb.Operator.assemble(V, F, k, nb.nat_bem_opts_default(prec=prec)) as op:
        P, info, st = op.solve(G)
        assert st == nb.NAT_BEM_OK and info.rel_residual <= 4e-6, (st, info.rel_residual)
        out.append(P.ravel(order="F"))
        its.append(info.iterations)
np.save(sys.argv[2], np.concatenate(out))
np.save(sys.argv[2] + ".its.npy", np.array(its))
"""


def test_fp32_krylov_basis_matches_fp64_basis_and_oracle(tmp_path, oracle_lib):
    """Inner refinement solves run the fused Arnoldi kernels (the multi-RHS one for 8 RHS, the
    single-RHS one for 1) on an FP32 basis; with NATBEM_FP64_BASIS=1 they keep the FP64 one.
    Both reach the true-residual target (1e-6, or 4e-6 at a stall), every RHS within 1e-4 of
    the FP64 oracle, the two within 1e-5 of each other, at ka 3.3 (BF16 and TF32 products) and
    14 (BF16 sweeps that hand over to FP32)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs, its = [], []
    for fp64 in (False, True):
        env = dict(os.environ)
        env.pop("NATBEM_FP64_BASIS", None)
        if fp64:
            env["NATBEM_FP64_BASIS"] = "1"
        f = str(tmp_path / f"b{int(fp64)}.npy")
        r = subprocess.run([sys.executable, "-c", _BASIS_CHILD, root, f], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(np.load(f))
        its.append(np.load(f + ".its.npy"))
    Vs, F = S.ring_sphere(1200)
    V = S.perturbed_ellipsoid(Vs, 8)
    G = S.sh_neumann(V, F, 8, 12)
    n = len(F)
    off = 0
    refs = {}
    for k, nr in ((3.3, 8), (3.3, 8), (14.0, 8), (3.3, 1), (14.0, 1)):
        if k not in refs:
            L, R = oracle_lib.assemble(V, F, k)
            refs[k] = np.linalg.solve(L, R @ G)
        Pref = refs[k]
        for o in outs:
            P = o[off:off + nr * n].reshape(n, nr, order="F")
            for s in range(nr):
                assert _rel(P[:, s], Pref[:, s]) < SOL_TOL
        assert _rel(outs[0][off:off + nr * n], outs[1][off:off + nr * n]) < 1e-5
        off += nr * n
    assert np.all(its[0] <= its[1] + 8), (its[0], its[1])


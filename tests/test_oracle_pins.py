"""Pins of the FP64 oracle against closed forms, brute force and invariants (CPU only).

The paper prints no worked numerical values for its BEM, so every pin here comes from
mathematics the oracle does not itself use: monomial exactness of the triangle rule, finite
differences of G, Duffy-mapped brute-force quadrature of the singular integrals, the limit of
the double-layer potential's normal derivative, Laplace closed forms, the radiating-sphere
solutions, the exact field of a source inside the body, energy balance and rigid-motion /
scaling invariance. Mutation tests build the oracle with deliberate mistakes and check that
the pins catch each one.
"""

import math
import os

import numpy as np
import pytest

import synthetic as S
from tests import bruteforce as bf


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def _h1(z):
    """Spherical Hankel function of the first kind, order 1."""
    return -np.exp(1j * z) * (z + 1j) / z ** 2


def _h1p(z):
    """Its derivative."""
    return -np.exp(1j * z) * (1j / z - 2.0 / z ** 2 - 2j / z ** 3)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ------------------------------------------------------------------------------ quadrature
def test_radon7_exact_to_degree_5(O):
    bary, w = O.quad_rule()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(bary.sum(1), 1.0, atol=1e-15)
    x, y = bary[:, 1], bary[:, 2]  # reference triangle (0,0), (1,0), (0,1), area 1/2
    worst6 = 0.0
    for deg in range(0, 7):
        for a in range(deg + 1):
            b = deg - a
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = 0.5 * np.sum(w * x ** a * y ** b)
            if deg <= 5:
                assert abs(got - exact) < 1e-15, (a, b)
            else:
                worst6 = max(worst6, abs(got - exact) / exact)
    assert worst6 > 1e-6  # degree exactly 5


def test_gauss_legendre_matches_library(O):
    for n in (1, 2, 5, 16, 64):
        x, w = O.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        o = np.argsort(x)
        assert np.allclose(x[o], xr, atol=1e-14) and np.allclose(w[o], wr, atol=1e-14)


# ------------------------------------------------------------------------------- kernels
def test_kernels_against_finite_differences(O):
    rng = np.random.default_rng(1)
    for _ in range(20):
        x, y = rng.normal(size=3), rng.normal(size=3)
        nx, ny = rng.normal(size=3), rng.normal(size=3)
        nx /= np.linalg.norm(nx)
        ny /= np.linalg.norm(ny)
        k = rng.uniform(0.3, 8.0)
        G, dny, dnx, H = O.kernels(k, x, nx, y, ny)
        r = np.linalg.norm(x - y)
        assert abs(G - np.exp(1j * k * r) / (4 * math.pi * r)) < 1e-15 * max(1.0, abs(G)) * 10
        h = 1e-5
        Gf = lambda xx, yy: O.kernels(k, xx, nx, yy, ny)[0]
        fd_ny = (Gf(x, y + h * ny) - Gf(x, y - h * ny)) / (2 * h)
        fd_nx = (Gf(x + h * nx, y) - Gf(x - h * nx, y)) / (2 * h)
        dny_f = lambda xx: O.kernels(k, xx, nx, y, ny)[1]
        fd_H = (dny_f(x + h * nx) - dny_f(x - h * nx)) / (2 * h)
        scale = abs(G) / r ** 2 + abs(G) * k ** 2
        assert abs(fd_ny - dny) < 1e-8 * scale
        assert abs(fd_nx - dnx) < 1e-8 * scale
        assert abs(fd_H - H) < 1e-7 * scale / r
        # the vector-form kernels of the brute-force module agree too
        bG, bny, bnx, bH = bf.kernels(k, x, nx, y, ny)
        assert np.allclose([G, dny, dnx, H], [bG, bny, bnx, bH], rtol=1e-12, atol=0)


# ------------------------------------------------------------------------- self integrals
TRIS = [
    np.array([[0, 0, 0], [0.3, 0, 0], [0.1, 0.25, 0]], float),
    np.array([[0.2, -0.1, 0.4], [0.5, 0.3, 0.1], [-0.1, 0.2, 0.3]], float),
    np.array([[0, 0, 0], [1.0, 0, 0], [0.5, 0.05, 0.02]], float),  # sliver
]


@pytest.mark.parametrize("ti", range(len(TRIS)))
@pytest.mark.parametrize("k", [0.5, 2.0, 9.0])
def test_self_single_layer_bruteforce(O, ti, k):
    tri = TRIS[ti]
    S_, _ = O.self_integrals(k, tri)
    x = tri.mean(0)
    sliver = ti == 2  # Duffy converges slowly when the centroid is close to an edge
    y, w = bf.duffy_points(tri, x, 256 if sliver else 48)
    Sb = np.sum(w * bf.green(k, x, y))
    assert abs(S_ - Sb) < (1e-7 if sliver else 1e-12) * abs(Sb)


def _laplace_closed_forms(tri):
    """At the centroid x of a flat triangle, with each edge at in-plane distance d_e spanning
    angles psi_P..psi_Q from its perpendicular: int dS / (4 pi r) = (1/4pi) sum d_e
    [asinh(tan psi)] and f.p. int dS / (4 pi r^3) = -(1/4pi) sum [sin psi] / d_e."""
    x = tri.mean(0)
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    n /= np.linalg.norm(n)
    s0 = fp0 = 0.0
    for e in range(3):
        P, Q = tri[e], tri[(e + 1) % 3]
        u = (Q - P) / np.linalg.norm(Q - P)
        tP, tQ = np.dot(P - x, u), np.dot(Q - x, u)   # signed positions along the edge line
        foot = x + (P - x) - tP * u
        de = np.linalg.norm(foot - x)
        psiP, psiQ = math.atan2(tP, de), math.atan2(tQ, de)
        s0 += de * (math.asinh(math.tan(psiQ)) - math.asinh(math.tan(psiP)))
        fp0 += -(math.sin(psiQ) - math.sin(psiP)) / de
    return s0 / (4 * math.pi), fp0 / (4 * math.pi)


@pytest.mark.parametrize("ti", range(len(TRIS)))
def test_self_integrals_laplace_limit(O, ti):
    tri = TRIS[ti]
    k = 1e-4
    S_, FP = O.self_integrals(k, tri)
    s0, fp0 = _laplace_closed_forms(tri)
    area = 0.5 * np.linalg.norm(np.cross(tri[1] - tri[0], tri[2] - tri[0]))
    rmax = np.max(np.linalg.norm(tri - tri.mean(0), axis=1))
    # S = S0 + ik|T|/(4 pi) - (k^2/24 pi) int R^3 dtheta + ...;  FP = FP0 + (k^2/8 pi) int R + ...
    assert abs(S_ - (s0 + 1j * k * area / (4 * math.pi))) < k * k * rmax ** 3 / 6 + 1e-12
    assert abs(FP - fp0) < k * k * rmax / 2 + 1e-10 * abs(fp0)
    assert abs(S_ - s0) > 0.5 * k * area / (4 * math.pi)  # the ik term is really there


@pytest.mark.parametrize("ti", range(len(TRIS)))
@pytest.mark.parametrize("k", [0.7, 2.0, 6.0])
def test_self_hypersingular_is_limit_of_double_layer_derivative(O, ti, k):
    """FP = lim_{h->0+} d/dh int_T dG/dn_y(x + h n, y) dS_y; the derivative is O(h) from the
    limit with a k^2 h / 2 leading term, so two small h are extrapolated linearly."""
    tri = TRIS[ti]
    _, FP = O.self_integrals(k, tri)
    h = 1e-5 * math.sqrt(0.5 * np.linalg.norm(np.cross(tri[1] - tri[0], tri[2] - tri[0])))
    d1 = bf.normal_derivative_of_double_layer(k, tri, 2 * h)
    d2 = bf.normal_derivative_of_double_layer(k, tri, h)
    assert abs((2 * d2 - d1) - FP) < 2e-6 * abs(FP)


def test_self_hypersingular_reference_value(O):
    """Triangle (0,0,0), (0.3,0,0), (0.1,0.25,0), k = 2: the finite part is
    -4.797839 + 0.007934i (the h -> 0 limit above, evaluated independently)."""
    _, FP = O.self_integrals(2.0, TRIS[0])
    assert abs(FP - (-4.797839 + 0.007934j)) < 2e-6


# -------------------------------------------------------------------- element integrals
def test_element_integrals_against_bruteforce(O):
    V, F = S.icosphere(0)
    c, n, _ = O.geometry(V, F)
    k = 3.0
    shared = lambda i, j: len(set(F[i]) & set(F[j])) > 0
    pairs = [(0, j) for j in range(1, 20) if not shared(0, j)][:3] + \
            [(0, j) for j in range(1, 20) if shared(0, j)][:3]
    for i, j in pairs:
        tri = V[F[j]]
        ours = O.element_integrals(k, c[i], n[i], tri, levels=4)
        y, w = bf.subdivided_duffy(tri, 3, 12)
        ref = [np.sum(w * v) for v in bf.kernels(k, c[i], n[i], y, n[j])]
        for a, b in zip(ours, ref):
            assert abs(a - b) < 1e-6 * max(abs(b), 1e-3), (i, j)
    # the default rule (7 points, no subdivision) on a far-away element (edge ~1, kh ~ 3)
    far = O.element_integrals(k, np.array([5.0, 0, 0]), np.array([1.0, 0, 0]), V[F[3]], 0)
    y, w = bf.subdivided_duffy(V[F[3]], 2, 10)
    ref = [np.sum(w * v) for v in bf.kernels(k, np.array([5.0, 0, 0]), np.array([1.0, 0, 0]), y, n[3])]
    assert np.allclose(far, ref, rtol=1e-4, atol=0)


def test_adjacent_subdivision_converges(O):
    """Vertex-sharing pairs use 4^2 sub-triangles; compare against 4^5."""
    V, F = S.icosphere(2)
    c, n, _ = O.geometry(V, F)
    i = 7
    js = [j for j in range(len(F)) if j != i and len(set(F[i]) & set(F[j]))][:6]
    for j in js:
        a = O.element_integrals(2.0, c[i], n[i], V[F[j]], 2)
        b = O.element_integrals(2.0, c[i], n[i], V[F[j]], 5)
        assert abs(a[3] - b[3]) < 5e-3 * abs(b[3])
        assert abs(a[0] - b[0]) < 1e-4 * abs(b[0])


# ------------------------------------------------------------------------ mesh validation
def test_validate_mesh(O):
    V, F = S.icosphere(1)
    assert O.validate_mesh(V, F) == 0
    assert O.validate_mesh(V, F[:, ::-1]) == 6          # inward orientation
    assert O.validate_mesh(V, F[:-1]) == 5              # open mesh
    F2 = F.copy(); F2[0, 1], F2[0, 2] = F2[0, 2], F2[0, 1]
    assert O.validate_mesh(V, F2) == 5                  # inconsistent orientation
    F3 = F.copy(); F3[0, 0] = len(V)
    assert O.validate_mesh(V, F3) == 3                  # index out of range
    V4 = V.copy(); V4[0, 0] = np.nan
    assert O.validate_mesh(V4, F) == 2
    V5 = V.copy(); V5[F[0, 1]] = V5[F[0, 0]]
    assert O.validate_mesh(V5, F) == 4                  # zero-area triangle
    for V6, F6 in (S.icosphere(0), S.uv_sphere(12, 5), S.tetrahedron(), S.octahedron()):
        assert O.validate_mesh(V6, F6) == 0


# ------------------------------------------------------------------------------- solver
def test_gmres_matches_dense_lu(O):
    V, F = S.icosphere(2)
    L, R = O.assemble(V, F, 3.0)
    g = S.cos_theta_neumann(V, F)
    b = R @ g
    x, it, rr, ok = O.gmres(L, b, tol=1e-12, maxit=300)
    assert ok and rr <= 1e-12
    xs = np.linalg.solve(L, b)
    assert _rel(x, xs) < 1e-10
    assert _rel(O.matvec(L, x), b) < 1e-11


def test_gmres_reports_nonconvergence(O):
    V, F = S.icosphere(1)
    L, R = O.assemble(V, F, 3.0)
    b = R @ S.cos_theta_neumann(V, F)
    x, it, rr, ok = O.gmres(L, b, tol=1e-12, maxit=2)
    assert not ok and it == 2 and rr > 1e-12


# -------------------------------------------------------------------- closed-form spheres
@pytest.fixture(scope="module")
def spheres(O):
    out = {}
    for lev in (1, 3):
        V, F = S.icosphere(lev)
        L, R = O.assemble(V, F, 2.0)
        out[lev] = (V, F, L, R)
    return out


def test_pulsating_sphere(O, spheres):
    """g = 1 on the unit sphere, ka = 2: p(r) = a^2 e^{ik(r-a)} / ((ika - 1) r), i.e.
    p(1) = -0.2 - 0.4i and p(3) = -0.0573307580 + 0.1376059825i."""
    k = 2.0
    exact = lambda r: np.exp(1j * k * (r - 1.0)) / ((1j * k - 1.0) * r)
    assert abs(exact(1.0) - (-0.2 - 0.4j)) < 1e-15
    assert abs(exact(3.0) - (-0.0573307580 + 0.1376059825j)) < 1e-10
    errs = []
    pts = S.fibonacci_points(256, 3.0)
    for lev in (1, 3):
        V, F, L, R = spheres[lev]
        g = S.uniform_neumann(F)
        p = np.linalg.solve(L, R @ g)
        e_s = _rel(p, np.full_like(p, exact(1.0)))
        fld = O.evaluate(V, F, k, pts, p, g)
        e_f = _rel(fld, np.full_like(fld, exact(3.0)))
        errs.append((e_s, e_f))
    assert errs[1][0] < 0.02 and errs[1][1] < 0.02
    assert errs[1][0] < 0.6 * errs[0][0] and errs[1][1] < 0.6 * errs[0][1]


def test_oscillating_sphere(O, spheres):
    """g = cos(theta): p = cos(theta) h1(kr) / (k h1'(ka)); at ka = 2, p(1, 0) = -0.3 - 0.4i
    and p(3, 0) = 0.0126184430 + 0.1505997379i."""
    k = 2.0
    amp = lambda r: _h1(k * r) / (k * _h1p(k))
    assert abs(amp(1.0) - (-0.3 - 0.4j)) < 1e-12
    assert abs(amp(3.0) - (0.0126184430 + 0.1505997379j)) < 1e-10
    pts = S.fibonacci_points(256, 3.0)
    errs = []
    for lev in (1, 3):
        V, F, L, R = spheres[lev]
        c, _, _ = O.geometry(V, F)
        g = S.cos_theta_neumann(V, F)
        p = np.linalg.solve(L, R @ g)
        ex = (c[:, 2] / np.linalg.norm(c, axis=1)) * amp(1.0)
        fld = O.evaluate(V, F, k, pts, p, g)
        exf = pts[:, 2] / 3.0 * amp(3.0)
        errs.append((_rel(p, ex), _rel(fld, exf)))
    assert errs[1][0] < 0.03 and errs[1][1] < 0.03
    assert errs[1][0] < 0.6 * errs[0][0] and errs[1][1] < 0.6 * errs[0][1]


@pytest.mark.parametrize("ka", [math.pi, 4.493409457909064])
def test_no_fictitious_frequency(O, ka):
    """At ka = pi and the first zero of j_1 the plain CBIE is singular on a sphere; the
    Burton-Miller system is not, so the pulsating sphere stays accurate there."""
    V, F = S.icosphere(3)
    L, R = O.assemble(V, F, ka)
    p = np.linalg.solve(L, R @ S.uniform_neumann(F))
    exact = 1.0 / (1j * ka - 1.0)
    assert _rel(p, np.full_like(p, exact)) < 0.03
    assert np.linalg.cond(L) < 1e3


def test_interior_monopole_converges(O):
    """Neumann data of a point source at the origin inside a perturbed ellipsoid give the
    exact exterior field; the error must fall under refinement."""
    k = 3.0
    errs = []
    pts = S.fibonacci_points(128, 4.0)
    for n_tri in (576, 2304):
        Vs, F = S.ring_sphere(n_tri)
        V = S.perturbed_ellipsoid(Vs, 2000)
        assert O.validate_mesh(V, F) == 0
        c, _, _ = O.geometry(V, F)
        g = S.monopole_neumann(V, F, k)
        L, R = O.assemble(V, F, k)
        p = np.linalg.solve(L, R @ g)
        fld = O.evaluate(V, F, k, pts, p, g)
        errs.append((_rel(p, S.monopole_field(c, k)), _rel(fld, S.monopole_field(pts, k))))
    assert errs[1][0] < 0.04 and errs[1][1] < 0.02
    assert errs[1][0] < 0.7 * errs[0][0] and errs[1][1] < 0.7 * errs[0][1]


def test_energy_balance(O, spheres):
    """Power through the surface, Im sum_j A_j conj(p_j) g_j, equals the far-field flux
    k int_{S_R} |p|^2 dS as R grows (for the sphere both are 4 pi a^4 k / (1 + k^2 a^2))."""
    k = 2.0
    V, F, L, R = spheres[3]
    V2 = S.perturbed_ellipsoid(V, 2001)
    _, _, area = O.geometry(V2, F)
    L2, R2 = O.assemble(V2, F, k)
    g = S.cos_theta_neumann(V2, F) + 0.5
    p = np.linalg.solve(L2, R2 @ g)
    p_surf = np.imag(np.sum(area * np.conj(p) * g))
    Rf = 200.0
    pts = S.fibonacci_points(4000, Rf)
    fld = O.evaluate(V2, F, k, pts, p, g)
    p_far = k * 4 * math.pi * Rf ** 2 * np.mean(np.abs(fld) ** 2)
    assert abs(p_surf - p_far) < 0.02 * abs(p_far)
    # the sphere's closed form for g = 1
    _, _, a1 = O.geometry(V, F)
    p1 = np.linalg.solve(L, R @ S.uniform_neumann(F))
    ref = 4 * math.pi * k / (1 + k * k)
    assert abs(np.imag(np.sum(a1 * np.conj(p1))) - ref) < 0.03 * ref


def test_rigid_motion_and_scaling_invariance(O):
    V, F = S.icosphere(2)
    V = S.perturbed_ellipsoid(V, 2002)
    k = 2.5
    g = S.sh_neumann(V, F, 1, 7)[:, 0]
    pts = S.fibonacci_points(32, 3.0)
    L, R = O.assemble(V, F, k)
    p = np.linalg.solve(L, R @ g)
    f = O.evaluate(V, F, k, pts, p, g)
    Q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    t = np.array([0.3, -1.2, 2.0])
    V2, pts2 = V @ Q.T + t, pts @ Q.T + t
    L2, R2 = O.assemble(V2, F, k)
    p2 = np.linalg.solve(L2, R2 @ g)
    assert _rel(p2, p) < 1e-11
    assert _rel(O.evaluate(V2, F, k, pts2, p2, g), f) < 1e-11
    s = 2.7  # mesh x s with k / s and g / s leaves p unchanged
    L3, R3 = O.assemble(V * s, F, k / s)
    p3 = np.linalg.solve(L3, R3 @ (g / s))
    assert _rel(p3, p) < 1e-11
    assert _rel(O.evaluate(V * s, F, k / s, pts * s, p3, g / s), f) < 1e-11


def test_assemble_rows_matches_full(O):
    V, F = S.icosphere(1)
    L, R = O.assemble(V, F, 1.7)
    rows = np.array([0, 5, 79])
    Lr, Rr = O.assemble_rows(V, F, 1.7, rows)
    assert np.array_equal(Lr, L[rows]) and np.array_equal(Rr, R[rows])


def test_bem_solve_pipeline(O):
    V, F = S.icosphere(2)
    pts = S.fibonacci_points(16, 3.0)
    g = S.uniform_neumann(F)
    p, fld, info = O.bem_solve(V, F, 2.0, g, pts, tol=1e-10, maxit=200)
    L, R = O.assemble(V, F, 2.0)
    assert info["converged"] and _rel(p, np.linalg.solve(L, R @ g)) < 1e-8
    assert _rel(fld, O.evaluate(V, F, 2.0, pts, p, g)) < 1e-14
    assert len(info["times"]) == 4


# ------------------------------------------------------------------------- mutation tests
def _sphere_errors(O):
    k = 2.0
    V, F = S.icosphere(2)
    c, _, _ = O.geometry(V, F)
    L, R = O.assemble(V, F, k)
    e1 = _rel(np.linalg.solve(L, R @ S.uniform_neumann(F)), np.full(len(F), 1 / (1j * k - 1)))
    amp = _h1(k) / (k * _h1p(k))
    ex = (c[:, 2] / np.linalg.norm(c, axis=1)) * amp
    e2 = _rel(np.linalg.solve(L, R @ S.cos_theta_neumann(V, F)), ex)
    _, FP = O.self_integrals(2.0, TRIS[0])
    return e1, e2, FP


@pytest.mark.parametrize("plant", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(O, plant, tmp_path):
    """1: jump term -beta/2 dropped; 2: sign of dG/dn_y flipped; 3: r_x r_y dropped from the
    hypersingular kernel; 4: ik dropped from the finite part. Each breaks a pin."""
    path = O.build_variant(str(tmp_path / f"liboracle_plant{plant}.so"), plant)
    with O.using_library(path):
        e1, e2, FP = _sphere_errors(O)
        G, dny, dnx, H = O.kernels(1.3, np.array([0.1, 0.2, 0.3]), np.array([0, 0, 1.0]),
                                   np.array([0.5, -0.1, 0.2]), np.array([0, 0.6, 0.8]))
    caught = e1 > 0.05 or e2 > 0.06 or abs(FP - (-4.797839 + 0.007934j)) > 1e-3
    bG, bny, bnx, bH = bf.kernels(1.3, np.array([0.1, 0.2, 0.3]), np.array([0, 0, 1.0]),
                                  np.array([0.5, -0.1, 0.2]), np.array([0, 0.6, 0.8]))
    caught = caught or not np.allclose([dny, H], [bny, bH], rtol=1e-10)
    assert caught
    e1, e2, _ = _sphere_errors(O)  # the real oracle passes the same checks
    assert e1 < 0.05 and e2 < 0.06

"""Pins of the Galerkin Burton-Miller reference (oracle/galerkin.py; paper Sec. 4, Eq. 6, with the
element-to-element integration of Sec. 4.1). CPU only.

  * each singular-pair rule integrates polynomials in (x, y) exactly (checked against a plain
    product Gauss rule over both triangles) and converges for the 1/r kernel;
  * the identical-pair 1/r integral equals the surface integral of the closed-form potential
    of a uniform triangle (an independent route: no singular transformation);
  * Laplace limit of the double layer on a closed surface: int dG/dn_y dS_y = -1/2 on the
    faces, so the rows of K sum to -1/2 the rows of M11;
  * the single-layer Galerkin matrix with P1 trial and test functions is symmetric;
  * pulsating and oscillating spheres converge to the exact solutions at the rate h^2, and an
    interior monopole on a perturbed ellipsoid reproduces its exact exterior field;
  * six planted mistakes each fail one of these pins.
"""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import galerkin as Gk


def _h1(z):
    return -np.exp(1j * z) * (z + 1j) / z ** 2


def _h1p(z):
    return -np.exp(1j * z) * (1j / z - 2.0 / z ** 2 - 2j / z ** 3)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _tri_rule(n):
    """Collapsed Gauss rule on {0 <= t <= s <= 1}: barycentric (1 - s, s - t, t), weights sum 1/2."""
    x, w = Gk.gauss01(n)
    a, b = np.meshgrid(x, x, indexing="ij")
    wa, wb = np.meshgrid(w, w, indexing="ij")
    s, t = a.ravel(), (a * b).ravel()
    return np.stack([1 - s, s - t, t], 1), (wa * wb * a).ravel()


def _product(Pt, Ps, f, n=12):
    bt, wt = _tri_rule(n)
    x, y = bt @ Pt, bt @ Ps
    X, Y = np.repeat(x, len(y), 0), np.tile(y, (len(x), 1))
    LA, MU = np.repeat(bt, len(bt), 0), np.tile(bt, (len(bt), 1))
    W = np.repeat(wt, len(wt)) * np.tile(wt, len(wt)) * (2 * Gk._area(Pt)) * (2 * Gk._area(Ps))
    return np.sum(W * f(X, Y, LA, MU))


def _poly(c):
    def f(X, Y, LA, MU):
        return (c[0] + c[1] * X[:, 0] + c[2] * Y[:, 1] + c[3] * X[:, 2] * Y[:, 0] + c[4] * X[:, 1] ** 2
                + c[5] * Y[:, 2] ** 2 * X[:, 0] + c[6] * LA[:, 0] * MU[:, 1] + c[7] * LA[:, 2] * MU[:, 2] * X[:, 1])
    return f


def _cases(n):
    rng = np.random.default_rng(0)
    P = rng.normal(size=(5, 3))
    T1, Te, Tv = np.array([0, 1, 2]), np.array([1, 0, 3]), np.array([3, 4, 0])
    return {"identical": (P[T1], P[T1], Gk.rule_identical(P[T1], n)),
            "edge": (P[T1], P[Te], Gk.rule_edge(P[T1], P[Te], 0, 1, 1, 0, n)),
            "vertex": (P[T1], P[Tv], Gk.rule_vertex(P[T1], P[Tv], 0, 2, n))}


@pytest.mark.parametrize("case", ["identical", "edge", "vertex"])
def test_singular_rules_exact_on_polynomials(case):
    Pt, Ps, (lam, mu, d, w) = _cases(8)[case]
    X, Y = lam @ Pt, mu @ Ps
    assert np.max(np.abs((X - Y) - d)) < 1e-13          # x - y formed consistently
    assert np.allclose(lam.sum(1), 1.0) and np.allclose(mu.sum(1), 1.0)
    for seed in range(3):
        f = _poly(np.random.default_rng(10 + seed).normal(size=8))
        assert abs(np.sum(w * f(X, Y, lam, mu)) - _product(Pt, Ps, f)) < 1e-12 * max(1.0, abs(_product(Pt, Ps, f)))


def test_singular_rules_converge_on_mesh_pairs():
    """1/r with a phase on the pairs touching one element of a perturbed ellipsoid mesh:
    the default rule (4 points per dimension) is within 5e-5 of the converged value."""
    V, F = S.icosphere(3)
    V = S.perturbed_ellipsoid(V, 12)
    F = np.asarray(F)
    t, k = 5, 5.0
    for s in range(len(F)):
        if not set(F[s]) & set(F[t]):
            continue
        vals = []
        for n in (Gk.N_SING, 8, 12):
            lam, mu, d, w = Gk.pair_rule(F, V, t, s, n)
            r = np.linalg.norm(d, axis=1)
            vals.append(np.sum(w * np.exp(1j * k * r) / r))
        assert abs(vals[1] - vals[2]) < 1e-6 * abs(vals[2])
        assert abs(vals[0] - vals[2]) < 5e-5 * abs(vals[2])


def _potential(P, X):
    """int_T dS_y / |x - y| for points X in the plane of T: sum over the edges of the signed
    distance to the edge line times log((R+ + s+) / (R- + s-))."""
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    tot = np.zeros(len(X))
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        t = (b - a) / np.linalg.norm(b - a)
        m = np.cross(t, n)
        d = (a - X) @ m
        sm, sp = (a - X) @ t, (b - X) @ t
        Rm, Rp = np.linalg.norm(a - X, axis=1), np.linalg.norm(b - X, axis=1)
        tot += d * np.log((Rp + sp) / (Rm + sm))
    return tot


def test_potential_formula_against_polar_integration():
    """The closed form against int_0^{2 pi} rho_max(theta) d theta summed edge by edge."""
    rng = np.random.default_rng(1)
    P = rng.normal(size=(3, 3))
    x, w = np.polynomial.legendre.leggauss(400)
    s, ws = 0.5 * (x + 1), 0.5 * w
    for _ in range(3):
        X = rng.dirichlet([1, 1, 1]) @ P
        polar = 0.0
        for i in range(3):
            a, b = P[i], P[(i + 1) % 3]
            r = a[None] + s[:, None] * (b - a)[None] - X[None]
            polar += np.sum(ws * np.linalg.norm(np.cross(r, (b - a)[None]), axis=1) / np.linalg.norm(r, axis=1))
        assert abs(_potential(P, X[None])[0] - polar) < 1e-8


def test_identical_pair_matches_closed_form_potential():
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.3, 0.9, 0.2]])
    x, w = Gk.gauss01(40)
    c = P.mean(0)
    ref = 0.0
    for i in range(3):   # three sub-triangles about the centroid, collapsed Gauss from the centroid
        a, b = P[i], P[(i + 1) % 3]
        xi, yj = np.meshgrid(x, x, indexing="ij")
        W = np.outer(w, w) * xi * np.linalg.norm(np.cross(a - c, b - a))
        pts = c[None] + (xi.ravel()[:, None]) * ((a - c)[None] + yj.ravel()[:, None] * (b - a)[None])
        ref += np.sum(W.ravel() * _potential(P, pts))
    lam, mu, d, wr = Gk.rule_identical(P, 10)
    got = np.sum(wr / np.linalg.norm(d, axis=1))
    assert abs(got - ref) < 1e-6 * ref


@pytest.fixture(scope="module")
def parts2():
    V, F = S.icosphere(2)
    return V, F, Gk.assemble_parts(V, F, 1e-4)


def test_laplace_double_layer_rows(parts2):
    """k -> 0: int dG/dn_y dS_y = -1/2 at points of the faces of a closed polyhedron."""
    V, F, m = parts2
    lhs = m["K"].sum(axis=1)
    rhs = -0.5 * m["M11"].sum(axis=1)
    assert np.max(np.abs(lhs - rhs)) < 2e-3 * np.max(np.abs(rhs))


def test_single_layer_p1_symmetric(parts2):
    """H at k -> 0 is -<G curl, curl>: symmetric like every Galerkin single-layer form."""
    V, F, m = parts2
    H = m["H"]
    assert np.max(np.abs(H - H.T)) < 1e-10 * np.max(np.abs(H))


@pytest.fixture(scope="module")
def spheres():
    out = {}
    for lev in (1, 2):
        V, F = S.icosphere(lev)
        out[lev] = (V, F) + Gk.assemble(V, F, 2.0)
    return out


def test_pulsating_sphere(spheres):
    """g = 1: p = 1 / (ik - 1) on the unit sphere and p(r) = p(1) e^{ik(r-1)} / r outside. The
    error falls as h^2: 2.0% -> 0.49% on the surface, 7.9% -> 2.1% in the field at r = 3."""
    k = 2.0
    exact = 1.0 / (1j * k - 1.0)
    errs = []
    for lev in (1, 2):
        V, F, L, R = spheres[lev]
        p = np.linalg.solve(L, R @ np.ones(len(F)))
        pts = S.fibonacci_points(64, 3.0)
        fld = Gk.evaluate(V, F, k, pts, p, np.ones(len(F)))
        ex = exact * np.exp(1j * k * 2.0) / 3.0
        errs.append((_rel(p, np.full(len(V), exact)), _rel(fld, np.full(len(pts), ex))))
    assert errs[1][0] < 0.006 and errs[1][1] < 0.025
    assert errs[1][0] < 0.3 * errs[0][0] and errs[1][1] < 0.3 * errs[0][1]


def test_oscillating_sphere(spheres):
    """g = cos(theta) per triangle: p = cos(theta) h1(k) / (k h1'(k)) at the vertices."""
    k = 2.0
    amp = _h1(k) / (k * _h1p(k))
    errs = []
    for lev in (1, 2):
        V, F, L, R = spheres[lev]
        g = S.cos_theta_neumann(V, F)
        p = np.linalg.solve(L, R @ g)
        ex = V[:, 2] / np.linalg.norm(V, axis=1) * amp
        errs.append(_rel(p, ex))
    assert errs[1] < 0.015
    assert errs[1] < 0.3 * errs[0]


def test_interior_monopole_on_ellipsoid():
    """Neumann data of a point source inside a perturbed ellipsoid: the Galerkin solve
    reproduces its exterior field."""
    V, F = S.icosphere(2)
    V = S.perturbed_ellipsoid(V, 31)
    k = 3.0
    g = S.monopole_neumann(V, F, k, x0=(0.1, -0.05, 0.05))
    p = Gk.solve(V, F, k, g)
    pts = S.fibonacci_points(64, 3.0)
    fld = Gk.evaluate(V, F, k, pts, p, g)
    assert _rel(fld, S.monopole_field(pts, k, x0=(0.1, -0.05, 0.05))) < 0.02
    assert _rel(p, S.monopole_field(V, k, x0=(0.1, -0.05, 0.05))) < 0.05


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5, 6])
def test_planted_mistakes_are_caught(plant, monkeypatch):
    monkeypatch.setattr(Gk, "PLANT", plant)
    failed = 0
    for check in (lambda: test_singular_rules_exact_on_polynomials("identical"),
                  lambda: test_singular_rules_exact_on_polynomials("edge"),
                  lambda: test_laplace_double_layer_rows((lambda V, F: (V, F, Gk.assemble_parts(V, F, 1e-4)))(*S.icosphere(1))),
                  lambda: _sphere_checks()):
        try:
            check()
        except AssertionError:
            failed += 1
    assert failed > 0


def _sphere_checks():
    k = 2.0
    V, F = S.icosphere(1)
    L, R = Gk.assemble(V, F, k)
    p = np.linalg.solve(L, R @ np.ones(len(F)))
    assert _rel(p, np.full(len(V), 1.0 / (1j * k - 1.0))) < 0.03
    g = S.cos_theta_neumann(V, F)
    p = np.linalg.solve(L, R @ g)
    assert _rel(p, V[:, 2] / np.linalg.norm(V, axis=1) * _h1(k) / (k * _h1p(k))) < 0.06


def test_far_field_of_the_pulsating_sphere(spheres):
    """F(d) = lim r e^{-ikr} p(r d) = p(1) e^{-ik} for the pulsating unit sphere."""
    k = 2.0
    V, F, L, R = spheres[2]
    p = np.linalg.solve(L, R @ np.ones(len(F)))
    dirs = S.fibonacci_points(40, 1.0)
    ff = Gk.far_field(V, F, k, dirs, p, np.ones(len(F)))
    exact = np.exp(-1j * k) / (1j * k - 1.0)
    assert _rel(ff, np.full(len(dirs), exact)) < 0.025       # the discretisation error (h^2)
    far = Gk.evaluate(V, F, k, 50.0 * dirs, p, np.ones(len(F))) * 50.0 * np.exp(-50j * k)
    assert _rel(ff, far) < 1e-3                                # the field's 1/r limit


def test_assemble_rows_matches_full(spheres):
    V, F, L, R = spheres[1]
    rows = [0, 7, 23, 41]
    Lr, Rr = Gk.assemble_rows(V, F, 2.0, rows)
    assert np.max(np.abs(Lr - L[rows])) < 1e-14 and np.max(np.abs(Rr - R[rows])) < 1e-14

"""Python access to the FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU-baseline leg use
this module; the product library and its binding never import it. It shares no code with the
CUDA path. The library is compiled from oracle.cpp with g++ on first use (or by the build
step), into this directory.

All complex arrays are complex128; matrices are row-major (n, n).
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# Defaults of the discretisation both sides implement (see oracle.cpp's header).
ADJ_LEVELS = 2      # 4^2 = 16 sub-triangles for vertex-sharing pairs
SELF_POINTS = 64    # Gauss-Legendre points per edge for the self integrals


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def build_variant(path: str, plant: int) -> str:
    """Compile a copy of the oracle with deliberate mistake number `plant` (mutation tests)."""
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", f"-DORACLE_PLANT={int(plant)}", "-o", path, _SRC])
    return path


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every call of this module to another build of oracle.cpp."""
    global _lib
    saved = _lib
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


def _configure(L):
    """Declare the C signatures of oracle.cpp's entry points on a loaded library."""
    if True:
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i64, c_int, c_d = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.oracle_validate_mesh.argtypes = [dp, i64, ip, i64]
        L.oracle_geometry.argtypes = [dp, ip, i64, dp, dp, dp]
        L.oracle_quad_rule.argtypes = [dp, dp]
        L.oracle_gauss_legendre.argtypes = [c_int, dp, dp]
        L.oracle_kernels.argtypes = [c_d, dp, dp, dp, dp, dp]
        L.oracle_element_integrals.argtypes = [c_d, dp, dp, dp, c_int, dp]
        L.oracle_self_integrals.argtypes = [c_d, dp, c_int, dp]
        L.oracle_assemble_rows.argtypes = [dp, i64, ip, i64, c_d, c_int, c_int, i64p, i64, dp, dp, c_int]
        L.oracle_assemble.argtypes = [dp, i64, ip, i64, c_d, c_int, c_int, dp, dp, c_int]
        L.oracle_matvec.argtypes = [dp, i64, dp, dp, c_int]
        L.oracle_gmres.argtypes = [dp, i64, dp, c_d, c_int, dp, ctypes.POINTER(c_int), dp, c_int]
        L.oracle_eval.argtypes = [dp, i64, ip, i64, c_d, dp, i64, dp, dp, dp, c_int]
        L.oracle_bem_solve.argtypes = [dp, i64, ip, i64, c_d, c_int, c_int, dp, dp, i64, c_d, c_int,
                                       c_int, dp, dp, ctypes.POINTER(c_int), dp, dp]
        L.oracle_mc_assemble.argtypes = [dp, dp, i64, c_d, c_d, dp, dp, c_int]
        L.oracle_mc_eval.argtypes = [dp, dp, i64, c_d, c_d, dp, i64, dp, dp, dp, c_int]
        L.oracle_far_field.argtypes = [dp, i64, ip, i64, c_d, dp, i64, dp, dp, dp, c_int]
        L.oracle_mc_far_field.argtypes = [dp, dp, i64, c_d, c_d, dp, i64, dp, dp, dp, c_int]
        L.oracle_hardware_threads.argtypes = []
    return L


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _mesh(V, F):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    return V, F


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def hardware_threads() -> int:
    return int(lib().oracle_hardware_threads())


def validate_mesh(V, F) -> int:
    V, F = _mesh(V, F)
    return int(lib().oracle_validate_mesh(_d(V), V.shape[0], _i(F), F.shape[0]))


def geometry(V, F):
    V, F = _mesh(V, F)
    n = F.shape[0]
    c, nr, a = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    lib().oracle_geometry(_d(V), _i(F), n, _d(c), _d(nr), _d(a))
    return c, nr, a


def quad_rule():
    bary, w = np.zeros((7, 3)), np.zeros(7)
    lib().oracle_quad_rule(_d(bary), _d(w))
    return bary, w


def gauss_legendre(n: int):
    x, w = np.zeros(n), np.zeros(n)
    lib().oracle_gauss_legendre(n, _d(x), _d(w))
    return x, w


def kernels(k, x, nx, y, ny):
    """(G, dG/dn_y, dG/dn_x, d2G/dn_x dn_y) at one pair of points."""
    out = np.zeros(8)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (x, nx, y, ny)]
    lib().oracle_kernels(float(k), *[_d(v) for v in a], _d(out))
    return out.view(np.complex128)


def element_integrals(k, x, nx, tri, levels=0):
    """Integrals of (G, dG/dn_y, dG/dn_x, H) over triangle `tri` (3x3) at point x, normal nx."""
    out = np.zeros(8)
    x, nx, tri = (np.ascontiguousarray(v, dtype=np.float64) for v in (x, nx, tri))
    lib().oracle_element_integrals(float(k), _d(x), _d(nx), _d(tri), int(levels), _d(out))
    return out.view(np.complex128)


def self_integrals(k, tri, npts=SELF_POINTS):
    """(S, FP): self single-layer integral and finite-part hypersingular integral at the centroid."""
    out = np.zeros(4)
    tri = np.ascontiguousarray(tri, dtype=np.float64)
    lib().oracle_self_integrals(float(k), _d(tri), int(npts), _d(out))
    return out.view(np.complex128)


def assemble(V, F, k, adj_levels=ADJ_LEVELS, self_pts=SELF_POINTS, nthreads=0):
    """Dense L and R (n x n complex128) of the P0 collocation Burton-Miller system."""
    V, F = _mesh(V, F)
    n = F.shape[0]
    L = np.zeros((n, n), dtype=np.complex128)
    R = np.zeros((n, n), dtype=np.complex128)
    rc = lib().oracle_assemble(_d(V), V.shape[0], _i(F), n, float(k), adj_levels, self_pts,
                               _d(L.view(np.float64)), _d(R.view(np.float64)), nthreads)
    if rc:
        raise ValueError(f"oracle_assemble failed ({rc})")
    return L, R


def assemble_rows(V, F, k, rows, adj_levels=ADJ_LEVELS, self_pts=SELF_POINTS, nthreads=0):
    """Selected rows of L and R, shape (len(rows), n)."""
    V, F = _mesh(V, F)
    n = F.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    L = np.zeros((rows.size, n), dtype=np.complex128)
    R = np.zeros((rows.size, n), dtype=np.complex128)
    rc = lib().oracle_assemble_rows(_d(V), V.shape[0], _i(F), n, float(k), adj_levels, self_pts,
                                    rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), rows.size,
                                    _d(L.view(np.float64)), _d(R.view(np.float64)), nthreads)
    if rc:
        raise ValueError(f"oracle_assemble_rows failed ({rc})")
    return L, R


def matvec(A, x, nthreads=0):
    A, x = _c(A), _c(x)
    y = np.zeros(A.shape[0], dtype=np.complex128)
    lib().oracle_matvec(_d(A.view(np.float64)), A.shape[0], _d(x.view(np.float64)),
                        _d(y.view(np.float64)), nthreads)
    return y


def gmres(A, b, tol=1e-12, maxit=200, nthreads=0):
    """Returns (x, iterations, relative residual estimate, converged)."""
    A, b = _c(A), _c(b)
    n = A.shape[0]
    x = np.zeros(n, dtype=np.complex128)
    it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = lib().oracle_gmres(_d(A.view(np.float64)), n, _d(b.view(np.float64)), float(tol), int(maxit),
                            _d(x.view(np.float64)), ctypes.byref(it), ctypes.byref(rr), nthreads)
    return x, it.value, rr.value, rc == 0


def evaluate(V, F, k, points, p, g, nthreads=0):
    """Field at `points` (m x 3) from surface Dirichlet p and Neumann g (both length n)."""
    V, F = _mesh(V, F)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    p, g = _c(p), _c(g)
    out = np.zeros(pts.shape[0], dtype=np.complex128)
    rc = lib().oracle_eval(_d(V), V.shape[0], _i(F), F.shape[0], float(k), _d(pts), pts.shape[0],
                           _d(p.view(np.float64)), _d(g.view(np.float64)), _d(out.view(np.float64)),
                           nthreads)
    if rc:
        raise ValueError(f"oracle_eval failed ({rc})")
    return out


def solve(V, F, k, g, tol=1e-12, maxit=400, nthreads=0):
    """Surface Dirichlet data p of L p = R g (one right-hand side), with GMRES info."""
    L, R = assemble(V, F, k, nthreads=nthreads)
    b = R @ _c(g)
    x, it, rr, ok = gmres(L, b, tol=tol, maxit=maxit, nthreads=nthreads)
    return x, dict(iterations=it, rel_residual=rr, converged=ok, L=L, R=R, b=b)


def bem_solve(V, F, k, g, points, tol=1e-6, maxit=200, nthreads=0):
    """One whole solve as the CPU baseline times it (assemble, b = R g, GMRES, field).
    Returns (p, field, info) with per-stage seconds in info['times']."""
    V, F = _mesh(V, F)
    n = F.shape[0]
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    g = _c(g)
    p = np.zeros(n, dtype=np.complex128)
    fld = np.zeros(pts.shape[0], dtype=np.complex128)
    it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    times = np.zeros(4)
    rc = lib().oracle_bem_solve(_d(V), V.shape[0], _i(F), n, float(k), ADJ_LEVELS, SELF_POINTS,
                                _d(g.view(np.float64)), _d(pts), pts.shape[0], float(tol), int(maxit),
                                nthreads, _d(p.view(np.float64)), _d(fld.view(np.float64)),
                                ctypes.byref(it), ctypes.byref(rr), _d(times))
    return p, fld, dict(iterations=it.value, rel_residual=rr.value, converged=rc == 0,
                        times=times.tolist())


# ---------------------------------------------------------------------------------- BEM-MC
def _samples(Y, N):
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(-1, 3)
    N = np.ascontiguousarray(N, dtype=np.float64).reshape(-1, 3)
    return Y, N


def mc_assemble(Y, N, area, k, nthreads=0):
    """L and R (M x M complex128) of the Monte-Carlo conventional BIE (paper Sec. 4.1.1 and
    4.2) at samples Y with unit outward normals N on a surface of total area `area`."""
    Y, N = _samples(Y, N)
    M = Y.shape[0]
    L = np.zeros((M, M), dtype=np.complex128)
    R = np.zeros((M, M), dtype=np.complex128)
    rc = lib().oracle_mc_assemble(_d(Y), _d(N), M, float(area), float(k), _d(L.view(np.float64)),
                                  _d(R.view(np.float64)), nthreads)
    if rc:
        raise ValueError(f"oracle_mc_assemble failed ({rc})")
    return L, R


def mc_evaluate(Y, N, area, k, points, p, g, nthreads=0):
    """Field at `points` from the samples' Dirichlet p and Neumann g (Monte-Carlo sum)."""
    Y, N = _samples(Y, N)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    p, g = _c(p), _c(g)
    out = np.zeros(pts.shape[0], dtype=np.complex128)
    rc = lib().oracle_mc_eval(_d(Y), _d(N), Y.shape[0], float(area), float(k), _d(pts), pts.shape[0],
                              _d(p.view(np.float64)), _d(g.view(np.float64)), _d(out.view(np.float64)),
                              nthreads)
    if rc:
        raise ValueError(f"oracle_mc_eval failed ({rc})")
    return out


def mc_solve(Y, N, area, k, g, tol=1e-12, maxit=400, nthreads=0):
    """Sample Dirichlet data p of the Monte-Carlo system L p = R g, with GMRES info."""
    L, R = mc_assemble(Y, N, area, k, nthreads=nthreads)
    b = R @ _c(g)
    x, it, rr, ok = gmres(L, b, tol=tol, maxit=maxit, nthreads=nthreads)
    return x, dict(iterations=it, rel_residual=rr, converged=ok, L=L, R=R, b=b)


# ------------------------------------------------------------------ far field and samples
def far_field(V, F, k, dirs, p, g, nthreads=0):
    """Far-field pattern F(d) = lim r e^{-ikr} p(r d) for unit directions `dirs` (nd x 3)."""
    V, F = _mesh(V, F)
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    p, g = _c(p), _c(g)
    out = np.zeros(d.shape[0], dtype=np.complex128)
    rc = lib().oracle_far_field(_d(V), V.shape[0], _i(F), F.shape[0], float(k), _d(d), d.shape[0],
                                _d(p.view(np.float64)), _d(g.view(np.float64)), _d(out.view(np.float64)),
                                nthreads)
    if rc:
        raise ValueError(f"oracle_far_field failed ({rc})")
    return out


def mc_far_field(Y, N, area, k, dirs, p, g, nthreads=0):
    """Far-field pattern of a Monte-Carlo solution (samples Y, normals N, total area)."""
    Y, N = _samples(Y, N)
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    p, g = _c(p), _c(g)
    out = np.zeros(d.shape[0], dtype=np.complex128)
    rc = lib().oracle_mc_far_field(_d(Y), _d(N), Y.shape[0], float(area), float(k), _d(d), d.shape[0],
                                   _d(p.view(np.float64)), _d(g.view(np.float64)),
                                   _d(out.view(np.float64)), nthreads)
    if rc:
        raise ValueError(f"oracle_mc_far_field failed ({rc})")
    return out


def ffat_directions(n_phi=64, n_theta=32):
    """Unit directions of an n_phi x n_theta FFAT map: cell centres in phi (azimuth, fastest
    varying) and theta (polar angle), row-major (theta, phi)."""
    th = (np.arange(n_theta) + 0.5) * np.pi / n_theta
    ph = (np.arange(n_phi) + 0.5) * 2.0 * np.pi / n_phi
    T, P = np.meshgrid(th, ph, indexing="ij")
    return np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1).reshape(-1, 3)


def sample_coords(u, center, r_lo, r_hi):
    """Training-sample coordinates (paper Sec. 3.4): theta = pi u0, phi = 2 pi u1,
    r = r_lo + (r_hi - r_lo) u2 about `center`; returns ((theta, phi, r), Cartesian points)."""
    u = np.asarray(u, dtype=np.float64).reshape(-1, 3)
    th, ph = np.pi * u[:, 0], 2.0 * np.pi * u[:, 1]
    r = r_lo + (r_hi - r_lo) * u[:, 2]
    xyz = np.asarray(center, dtype=np.float64) + r[:, None] * np.stack(
        [np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    return np.stack([th, ph, r], axis=1), xyz

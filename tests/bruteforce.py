"""Brute-force numerical integration used to pin the oracle (tests only).

Nothing here is shared with the oracle or the CUDA path. The Green's function derivatives are
written in vector (gradient / Hessian) form, not the radial-derivative form the oracle uses,
and integrals use Duffy-mapped or polar tensor Gauss-Legendre rules with many points, so an
error in the oracle's formulas or rules does not cancel against the same error here.
"""

from __future__ import annotations

import math

import numpy as np


def green(k, x, y):
    """G(x, y) = e^{ik|x-y|} / (4 pi |x-y|), vectorised over the leading axes of y."""
    r = np.linalg.norm(x - y, axis=-1)
    return np.exp(1j * k * r) / (4.0 * math.pi * r)


def _radial(k, r):
    g = np.exp(1j * k * r) / (4.0 * math.pi * r)
    g1 = g * (1j * k - 1.0 / r)
    g2 = g * (2.0 - 2.0j * k * r - (k * r) ** 2) / r ** 2
    return g, g1, g2


def kernels(k, x, nx, y, ny):
    """(G, grad_y G . ny, grad_x G . nx, nx^T Hess_{xy} G ny) with d = x - y:
    grad_x G = g'(r) d/r, grad_y G = -g'(r) d/r,
    d2G/dx_a dy_b = -[g''(r) d_a d_b / r^2 + g'(r) (delta_ab / r - d_a d_b / r^3)]."""
    d = x - y
    r = np.linalg.norm(d, axis=-1)
    g, g1, g2 = _radial(k, r)
    dnx = (d * nx).sum(-1)
    dny = (d * ny).sum(-1)
    nxny = (nx * ny).sum(-1)
    gy = -g1 * dny / r
    gx = g1 * dnx / r
    hess = -(g2 * dnx * dny / r ** 2 + g1 * (nxny / r - dnx * dny / r ** 3))
    return g, gy, gx, hess


def duffy_points(tri, apex, n):
    """Points and weights integrating over triangle `tri` split at `apex` (a point in its
    plane, inside or on it) into three sub-triangles, each mapped from the unit square by
    y = apex + s((1-t)(P-apex) + t(Q-apex)) with Jacobian s |(P-apex) x (Q-apex)|. The s factor
    cancels a 1/r singularity at the apex."""
    gx, gw = np.polynomial.legendre.leggauss(n)
    u, uw = 0.5 * (gx + 1.0), 0.5 * gw
    pts, wts = [], []
    for e in range(3):
        P, Q = tri[e], tri[(e + 1) % 3]
        jac = np.linalg.norm(np.cross(P - apex, Q - apex))
        if jac == 0.0:
            continue
        s, t = np.meshgrid(u, u, indexing="ij")
        ws = np.outer(uw, uw)
        y = apex + s[..., None] * ((1 - t)[..., None] * (P - apex) + t[..., None] * (Q - apex))
        pts.append(y.reshape(-1, 3))
        wts.append((ws * s * jac).reshape(-1))
    return np.concatenate(pts), np.concatenate(wts)


def subdivided_duffy(tri, levels, n):
    """Tensor rule over the 4^levels midpoint sub-triangles of `tri`, each Duffy-mapped from
    its first vertex (smooth integrands)."""
    tris = [np.asarray(tri, dtype=np.float64)]
    for _ in range(levels):
        nt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nt += [np.array(v) for v in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]
        tris = nt
    gx, gw = np.polynomial.legendre.leggauss(n)
    u, uw = 0.5 * (gx + 1.0), 0.5 * gw
    s, t = np.meshgrid(u, u, indexing="ij")
    ws = np.outer(uw, uw) * s
    pts, wts = [], []
    for a, b, c in tris:
        jac = np.linalg.norm(np.cross(b - a, c - a))
        y = a + s[..., None] * ((1 - t)[..., None] * (b - a) + t[..., None] * (c - a))
        pts.append(y.reshape(-1, 3))
        wts.append((ws * jac).reshape(-1))
    return np.concatenate(pts), np.concatenate(wts)


def polar_edges(tri, x, n_vec, nth):
    """Angular Gauss-Legendre nodes per edge about the in-plane point x: for each node the
    boundary distance R, the unit in-plane direction and the angular weight."""
    gx, gw = np.polynomial.legendre.leggauss(nth)
    out = []
    for e in range(3):
        P, Q = tri[e], tri[(e + 1) % 3]
        u = (Q - P) / np.linalg.norm(Q - P)
        foot = P + u * np.dot(x - P, u)
        ed = foot - x
        de = np.linalg.norm(ed)
        ed /= de
        td = np.cross(n_vec, ed)
        pP = math.atan2(np.dot(P - x, td), np.dot(P - x, ed))
        pQ = math.atan2(np.dot(Q - x, td), np.dot(Q - x, ed))
        psi = 0.5 * (pQ + pP) + 0.5 * (pQ - pP) * gx
        w = 0.5 * (pQ - pP) * gw
        dirs = np.cos(psi)[:, None] * ed + np.sin(psi)[:, None] * td
        out.append((de / np.cos(psi), dirs, w))
    return out


def normal_derivative_of_double_layer(k, tri, h, nth=64, nrho=240):
    """d/dh of D(h) = int_T dG/dn_y(x + h n, y) dS_y at the centroid x, computed as
    int_T nx^T Hess G ny (x + h n, y) dS_y with polar coordinates about x and the radial
    substitution rho = h sinh(s) that resolves the peak of width h."""
    tri = np.asarray(tri, dtype=np.float64)
    x = tri.mean(0)
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    n /= np.linalg.norm(n)
    sx, sw = np.polynomial.legendre.leggauss(nrho)
    total = 0.0
    for R, dirs, w in polar_edges(tri, x, n, nth):
        for Rq, dq, wq in zip(R, dirs, w):
            smax = math.asinh(Rq / h)
            s = 0.5 * smax * (sx + 1.0)
            ws = 0.5 * smax * sw
            rho = h * np.sinh(s)
            jac = h * np.cosh(s)
            y = x + rho[:, None] * dq
            _, _, _, hess = kernels(k, x + h * n, n, y, n)
            total += wq * np.sum(hess * rho * jac * ws)
    return total

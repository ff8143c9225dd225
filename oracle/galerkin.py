"""FP64 reference of the Galerkin form of the Burton-Miller equation (paper Sec. 4, Eq. 6; the
element-to-element integration of Sec. 4.1, as in bempp): P1 (continuous, piecewise linear)
Dirichlet data, P0 Neumann data, P1 test functions, double (element-pair) quadrature.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the tests, the smoke check and the bench's
CPU leg use it; the product library never does. It shares no code with the CUDA path.

Testing Eq. 6 with every P1 hat function psi_i and integrating over the surface gives

    L p = R g,   L = 1/2 M11 - K - beta H,   R = -V - beta K' - (beta/2) M10,

with phi_j the P1 basis, chi_s the indicator of triangle s, G = e^{ikr}/(4 pi r), beta = i/k:
    M11_ij = <phi_j, psi_i>,                      M10_is = <chi_s, psi_i>,
    K_ij   = <int dG/dn_y phi_j, psi_i>,          K'_is  = <int dG/dn_x chi_s, psi_i>,
    V_is   = <int G chi_s, psi_i>,
    H_ij   = <f.p. int d2G/dn_x dn_y phi_j, psi_i>
           = int int G(x, y) [k^2 (n_x . n_y) phi_j(y) psi_i(x) - curl phi_j(y) . curl psi_i(x)]
(the hypersingular form integrated by parts, after Maue; curl u = n x grad u is constant on a
flat triangle for P1 functions). Every entry is a sum over element pairs (tau test, sigma
trial) of 4D integrals over tau x sigma.

Quadrature (the scheme the GPU path implements too):
  * pairs sharing no vertex: the 7-point degree-5 rule on both triangles (49 point pairs);
  * pairs sharing a vertex, an edge, or identical: the integrand is weakly singular (1/r).
    Each case is mapped to a sum of unit 4-cubes on which the Jacobian cancels the
    singularity, then Gauss-Legendre with `n_sing` points per dimension:
      - vertex (2 regions): polar coordinates about the shared vertex on both triangles,
        split by which radius is larger;
      - edge (6 regions): on each triangle, coordinates along the shared edge and towards the
        opposite vertex; the three "normal" variables (both distances from the edge, and the
        offset along it) split by which is largest and by the sign of the offset;
      - identical (6 regions): relative coordinate z = y - x; the set of x for fixed z is a
        triangle homothetic to the element (scale 1 - gauge(z)), and z runs over the hexagon
        T - T, split into six triangles about z = 0 with Duffy coordinates.
    In every case x - y is formed from the transformed coordinates directly (a radius times a
    bounded vector), so no cancellation occurs near the singularity.
"""
from __future__ import annotations

import numpy as np

# 7-point degree-5 rule on the reference triangle (Radon 1948): barycentric points and
# weights summing to 1 (times the area)
_A1 = (6.0 - np.sqrt(15.0)) / 21.0
_A2 = (6.0 + np.sqrt(15.0)) / 21.0
_W1 = (155.0 - np.sqrt(15.0)) / 1200.0
_W2 = (155.0 + np.sqrt(15.0)) / 1200.0
RULE7_BARY = np.array([[1 / 3, 1 / 3, 1 / 3],
                       [_A1, _A1, 1 - 2 * _A1], [_A1, 1 - 2 * _A1, _A1], [1 - 2 * _A1, _A1, _A1],
                       [_A2, _A2, 1 - 2 * _A2], [_A2, 1 - 2 * _A2, _A2], [1 - 2 * _A2, _A2, _A2]])
RULE7_W = np.array([9.0 / 40.0, _W1, _W1, _W1, _W2, _W2, _W2])

N_SING = 4   # Gauss-Legendre points per dimension of the singular-pair rules (both sides)

# Deliberate mistakes for the mutation tests (0 = none): 1 curl term sign, 2 no k^2 n.n term,
# 3 dG/dn_y sign, 4 identical-pair Jacobian without the homothety factor, 5 edge-pair Jacobian
# without the offset factor, 6 sign of the Neumann mass term.
PLANT = 0

HEXAGON = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [-1.0, 0.0], [-1.0, -1.0], [0.0, -1.0]])


def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _grid4(n):
    """Tensor Gauss-Legendre points on [0,1]^4: (m, 4) coordinates, (m,) weights."""
    x, w = gauss01(n)
    g = np.stack(np.meshgrid(x, x, x, x, indexing="ij"), -1).reshape(-1, 4)
    wg = np.prod(np.stack(np.meshgrid(w, w, w, w, indexing="ij"), -1).reshape(-1, 4), axis=1)
    return g, wg


# ------------------------------------------------------------------------ pair rules
# Each rule returns, for a pair (tau, sigma), arrays over its points:
#   lam (m, 3): barycentric coordinates of x on tau's vertices (in tau's stored order)
#   mu  (m, 3): barycentric coordinates of y on sigma's vertices (stored order)
#   d   (m, 3): x - y
#   w   (m,):   weights including both area Jacobians


def rule_regular(Pt, Ps):
    At, As = _area(Pt), _area(Ps)
    lam = np.repeat(RULE7_BARY, 7, axis=0)
    mu = np.tile(RULE7_BARY, (7, 1))
    w = np.repeat(RULE7_W, 7) * np.tile(RULE7_W, 7) * At * As
    x = lam @ Pt
    y = mu @ Ps
    return lam, mu, x - y, w


def rule_vertex(Pt, Ps, it, js, n=N_SING):
    """Shared vertex: tau's local vertex it and sigma's local vertex js are the same point."""
    P = Pt[it]
    Bt, Ct = Pt[(it + 1) % 3], Pt[(it + 2) % 3]
    Bs, Cs = Ps[(js + 1) % 3], Ps[(js + 2) % 3]
    At, As = _area(Pt), _area(Ps)
    g, wg = _grid4(n)
    t, u, th, ths = g.T
    out = []
    for region in range(2):
        if region == 0:   # rho_sigma = rho_tau u
            rt, rs = t, t * u
        else:             # rho_tau = rho_sigma u
            rt, rs = t * u, t
        jac = t ** 3 * u
        et = (1 - th)[:, None] * (Bt - P) + th[:, None] * (Ct - P)
        es = (1 - ths)[:, None] * (Bs - P) + ths[:, None] * (Cs - P)
        d = rt[:, None] * et - rs[:, None] * es
        lam = np.zeros((len(t), 3))
        lam[:, it] = 1 - rt
        lam[:, (it + 1) % 3] = rt * (1 - th)
        lam[:, (it + 2) % 3] = rt * th
        mu = np.zeros((len(t), 3))
        mu[:, js] = 1 - rs
        mu[:, (js + 1) % 3] = rs * (1 - ths)
        mu[:, (js + 2) % 3] = rs * ths
        out.append((lam, mu, d, wg * jac * (2 * At) * (2 * As)))
    return _cat(out)


def rule_edge(Pt, Ps, ia, ib, ja, jb, n=N_SING):
    """Shared edge: tau's local vertices (ia, ib) are sigma's (ja, jb), the same points."""
    Pa, Pb = Pt[ia], Pt[ib]
    ic, jc = 3 - ia - ib, 3 - ja - jb
    Ct, Cs = Pt[ic], Ps[jc]
    At, As = _area(Pt), _area(Ps)
    g, wg = _grid4(n)
    t, u, v, wv = g.T
    out = []
    for sign in (1.0, -1.0):
        for region in range(3):
            if region == 0:     # eta_tau largest
                et, es, dd = t, t * u, t * v
            elif region == 1:   # eta_sigma largest
                et, es, dd = t * u, t, t * v
            else:               # |offset| largest
                et, es, dd = t * u, t * v, t
            delta = sign * dd
            xi = np.where(sign > 0, (1 - dd) * wv, dd + (1 - dd) * wv)   # tau's edge coordinate
            xs = xi + delta                                            # sigma's
            jac = t ** 2 * ((1 - dd) if PLANT != 5 else 1.0) * (1 - et) * (1 - es) * (2 * At) * (2 * As)
            Et = Pa + xi[:, None] * (Pb - Pa)
            Es = Pa + xs[:, None] * (Pb - Pa)
            d = -delta[:, None] * (Pb - Pa) + et[:, None] * (Ct - Et) - es[:, None] * (Cs - Es)
            lam = np.zeros((len(t), 3))
            lam[:, ia] = (1 - et) * (1 - xi)
            lam[:, ib] = (1 - et) * xi
            lam[:, ic] = et
            mu = np.zeros((len(t), 3))
            mu[:, ja] = (1 - es) * (1 - xs)
            mu[:, jb] = (1 - es) * xs
            mu[:, jc] = es
            out.append((lam, mu, d, wg * jac))
    return _cat(out)


def rule_identical(P, n=N_SING):
    """tau = sigma. Reference triangle {0 <= t <= s <= 1}, x = A + s (B - A) + t (C - B)."""
    A, B, C = P
    J = np.stack([B - A, C - B], axis=1)   # 3 x 2
    Ar = _area(P)
    g, wg = _grid4(n)
    rho, w, a1, a2 = g.T
    out = []
    for i in range(6):
        h0, h1 = HEXAGON[i], HEXAGON[(i + 1) % 6]
        zdir = h0[None, :] + w[:, None] * (h1 - h0)[None, :]      # on the hexagon boundary
        z = rho[:, None] * zdir
        a = np.maximum(0.0, -z[:, 1])
        b = np.maximum(0.0, z[:, 1] - z[:, 0])
        scale = 1.0 - rho                                          # 1 - gauge(z)
        # u in the reference triangle by collapsed coordinates: (s, t) = (a1, a1 a2)
        us, ut = a1, a1 * a2
        xs = a + b + scale * us
        xt = a + scale * ut
        ys, yt = xs + z[:, 0], xt + z[:, 1]
        jac = rho * abs(h0[0] * h1[1] - h0[1] * h1[0]) * (scale ** 2 if PLANT != 4 else scale) * a1 * (2 * Ar) ** 2
        d = -(z @ J.T)                                             # x - y = -J z
        lam = np.stack([1 - xs, xs - xt, xt], axis=1)
        mu = np.stack([1 - ys, ys - yt, yt], axis=1)
        out.append((lam, mu, d, wg * jac))
    return _cat(out)


def _cat(parts):
    return tuple(np.concatenate([p[i] for p in parts], axis=0) for i in range(4))


def _area(P):
    return 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))


def pair_rule(F, V, t, s, n_sing=N_SING):
    """The quadrature of the pair (test tau = F[t], trial sigma = F[s]) by the shared vertices."""
    Pt, Ps = V[F[t]], V[F[s]]
    if t == s:
        return rule_identical(Pt, n_sing)
    shared = [(a, b) for a in range(3) for b in range(3) if F[t][a] == F[s][b]]
    if len(shared) == 0:
        return rule_regular(Pt, Ps)
    if len(shared) == 1:
        return rule_vertex(Pt, Ps, shared[0][0], shared[0][1], n_sing)
    (ia, ja), (ib, jb) = shared[:2]
    return rule_edge(Pt, Ps, ia, ib, ja, jb, n_sing)


# ------------------------------------------------------------------------ operators
def kernels(k, d, nx, ny):
    """G, dG/dn_y, dG/dn_x for d = x - y (rows)."""
    r = np.linalg.norm(d, axis=1)
    G = np.exp(1j * k * r) / (4 * np.pi * r)
    f = G * (1 - 1j * k * r) / r ** 2
    sy = -1.0 if PLANT == 3 else 1.0
    return G, sy * f * (d @ ny), -f * (d @ nx)


def geometry(V, F):
    P = V[F]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nrm = cr / (2 * area[:, None])
    # surface curl of the P1 hat of local vertex a: (P_{a+1} - P_{a+2}) / (2 A)
    curl = np.stack([(P[:, (a + 1) % 3] - P[:, (a + 2) % 3]) / (2 * area[:, None]) for a in range(3)], axis=1)
    return area, nrm, curl


def pair_blocks(V, F, k, t, s, geo=None, n_sing=N_SING):
    """The element-pair integrals of (tau = F[t], sigma = F[s]):
    Kb[a, b] = int int psi_a phi_b dG/dn_y,  Gb[a, b] = int int psi_a phi_b G,  G0 = int int G,
    Vb[a] = int int psi_a G,  Kp[a] = int int psi_a dG/dn_x."""
    area, nrm, curl = geo if geo is not None else geometry(V, F)
    lam, mu, d, w = pair_rule(F, V, t, s, n_sing)
    G, dGy, dGx = kernels(k, d, nrm[t], nrm[s])
    Kb = (lam * (w * dGy)[:, None]).T @ mu
    Gb = (lam * (w * G)[:, None]).T @ mu
    G0 = np.sum(w * G)
    Vb = lam.T @ (w * G)
    Kp = lam.T @ (w * dGx)
    return Kb, Gb, G0, Vb, Kp


def _regular_blocks(V, F, k, t, S, geo):
    """pair_blocks for test triangle t against the trial triangles S (sharing no vertex with
    it), vectorised over S: arrays with a leading axis over S."""
    area, nrm, _ = geo
    x = RULE7_BARY @ V[F[t]]                                     # (7, 3)
    y = np.einsum("qb,sbd->sqd", RULE7_BARY, V[F[S]])            # (S, 7, 3)
    d = x[None, :, None, :] - y[:, None, :, :]                   # (S, 7, 7, 3)
    r = np.linalg.norm(d, axis=3)
    G = np.exp(1j * k * r) / (4 * np.pi * r)
    f = G * (1 - 1j * k * r) / r ** 2
    dGy = (-1.0 if PLANT == 3 else 1.0) * f * np.einsum("spqd,sd->spq", d, nrm[S])
    dGx = -f * (d @ nrm[t])
    w = (RULE7_W[:, None] * RULE7_W[None, :])[None] * (area[t] * area[S])[:, None, None]
    lam = RULE7_BARY                                             # (7, 3): x points on tau
    mu = RULE7_BARY                                              # (7, 3): y points on sigma
    Kb = np.einsum("pa,spq,qb->sab", lam, w * dGy, mu)
    Gb = np.einsum("pa,spq,qb->sab", lam, w * G, mu)
    G0 = np.sum(w * G, axis=(1, 2))
    Vb = np.einsum("pa,spq->sa", lam, w * G)
    Kp = np.einsum("pa,spq->sa", lam, w * dGx)
    return Kb, Gb, G0, Vb, Kp


def assemble_parts(V, F, k, n_sing=N_SING):
    """The Galerkin matrices of the terms of Eq. 6, complex128:
    M11 (nv, nv), K (nv, nv), H (nv, nv), M10 (nv, nt), Vs (nv, nt), Kp (nv, nt)."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    nv, nt = len(V), len(F)
    geo = geometry(V, F)
    area, nrm, curl = geo
    out = {name: np.zeros((nv, nv), complex) for name in ("M11", "K", "H")}
    out.update({name: np.zeros((nv, nt), complex) for name in ("M10", "Vs", "Kp")})
    curl_sign = 1.0 if PLANT != 1 else -1.0
    kk = k * k if PLANT != 2 else 0.0
    for t in range(nt):
        rows = F[t]
        touch = np.any(np.isin(F, rows), axis=1)
        S = np.nonzero(~touch)[0]
        Kb, Gb, G0, Vb, Kp = _regular_blocks(V, F, k, t, S, geo)
        nn = nrm[S] @ nrm[t]
        cc = np.einsum("ad,sbd->sab", curl[t], curl[S])
        H = kk * nn[:, None, None] * Gb - curl_sign * cc * G0[:, None, None]
        for b in range(3):
            cols = F[S][:, b][None, :]
            np.add.at(out["K"], (rows[:, None], cols), Kb[:, :, b].T)
            np.add.at(out["H"], (rows[:, None], cols), H[:, :, b].T)
        out["Vs"][np.ix_(rows, S)] += Vb.T
        out["Kp"][np.ix_(rows, S)] += Kp.T
        for s in np.nonzero(touch)[0]:
            Kb1, Gb1, G01, Vb1, Kp1 = pair_blocks(V, F, k, t, s, geo, n_sing)
            H1 = kk * float(nrm[t] @ nrm[s]) * Gb1 - curl_sign * (curl[t] @ curl[s].T) * G01
            out["K"][np.ix_(rows, F[s])] += Kb1
            out["H"][np.ix_(rows, F[s])] += H1
            out["Vs"][rows, s] += Vb1
            out["Kp"][rows, s] += Kp1
        # mass terms (exact): P1-P1 A/12 (1 + delta_ab), P0-P1 A/3
        out["M11"][np.ix_(rows, rows)] += area[t] / 12.0 * (np.ones((3, 3)) + np.eye(3))
        out["M10"][rows, t] += area[t] / 3.0
    return out


def assemble_rows(V, F, k, rows, n_sing=N_SING):
    """Rows `rows` (vertex indices) of L and R, from the element pairs whose test triangle
    contains one of them: the same sums as assemble, restricted."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    nv, nt = len(V), len(F)
    beta = 1j / k
    geo = geometry(V, F)
    area, nrm, curl = geo
    rows = np.asarray(rows)
    pos = {int(r): i for i, r in enumerate(rows)}
    L = np.zeros((len(rows), nv), complex)
    R = np.zeros((len(rows), nt), complex)
    for t in np.nonzero(np.any(np.isin(F, rows), axis=1))[0]:
        touch = np.any(np.isin(F, F[t]), axis=1)
        S = np.nonzero(~touch)[0]
        Kb, Gb, G0, Vb, Kp = _regular_blocks(V, F, k, t, S, geo)
        nn = nrm[S] @ nrm[t]
        cc = np.einsum("ad,sbd->sab", curl[t], curl[S])
        blk = -Kb - beta * (k * k * nn[:, None, None] * Gb - cc * G0[:, None, None])
        rblk = -Vb - beta * Kp
        sing = []
        for s in np.nonzero(touch)[0]:
            Kb1, Gb1, G01, Vb1, Kp1 = pair_blocks(V, F, k, t, s, geo, n_sing)
            H1 = k * k * float(nrm[t] @ nrm[s]) * Gb1 - (curl[t] @ curl[s].T) * G01
            sing.append((s, -Kb1 - beta * H1, -Vb1 - beta * Kp1))
        for a in range(3):
            i = pos.get(int(F[t][a]))
            if i is None:
                continue
            for b in range(3):
                np.add.at(L[i], F[S][:, b], blk[:, a, b])
            R[i, S] += rblk[:, a]
            for s, lb, rb in sing:
                L[i, F[s]] += lb[a]
                R[i, s] += rb[a]
            L[i, F[t]] += 0.5 * area[t] / 12.0 * (np.ones(3) + (np.arange(3) == a))
            R[i, t] += -0.5 * beta * area[t] / 3.0
    return L, R


def assemble(V, F, k, n_sing=N_SING):
    """Dense L (nv x nv) and R (nv x nt), complex128: L p = R g."""
    m = assemble_parts(V, F, k, n_sing)
    beta = 1j / k
    L = 0.5 * m["M11"] - m["K"] - beta * m["H"]
    mass_sign = 1.0 if PLANT != 6 else -1.0
    R = -m["Vs"] - beta * m["Kp"] - mass_sign * 0.5 * beta * m["M10"]
    return L, R


def solve(V, F, k, g, n_sing=N_SING):
    L, R = assemble(V, F, k, n_sing)
    return np.linalg.solve(L, R @ np.asarray(g, complex))


def evaluate(V, F, k, points, p, g):
    """Exterior representation p(x) = int [p(y) dG/dn_y - G g(y)] dS_y with P1 p (at the
    vertices) and P0 g (per triangle), the 7-point rule on every element."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    area, nrm, _ = geometry(V, F)
    P = V[F]
    y = np.einsum("qa,tad->tqd", RULE7_BARY, P)              # (nt, 7, 3)
    py = np.einsum("qa,ta->tq", RULE7_BARY, np.asarray(p)[F])  # P1 p at the points
    wy = RULE7_W[None, :] * area[:, None]
    out = np.zeros(len(points), complex)
    for m, x in enumerate(np.asarray(points, np.float64)):
        d = x[None, None, :] - y
        r = np.linalg.norm(d, axis=2)
        G = np.exp(1j * k * r) / (4 * np.pi * r)
        dGy = G * (1 - 1j * k * r) / r ** 2 * np.einsum("tqd,td->tq", d, nrm)
        out[m] = np.sum(wy * (py * dGy - G * np.asarray(g)[:, None]))
    return out


def far_field(V, F, k, dirs, p, g):
    """Far-field pattern F(d) = sum over elements and points (w A / 4 pi) [p(y) (-ik d.n) - g]
    e^{-ik d.y}, with P1 p interpolated at the 7 points of every element."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    area, nrm, _ = geometry(V, F)
    y = np.einsum("qa,tad->tqd", RULE7_BARY, V[F])
    py = np.einsum("qa,ta->tq", RULE7_BARY, np.asarray(p)[F])
    wy = RULE7_W[None, :] * area[:, None] / (4 * np.pi)
    out = np.zeros(len(dirs), complex)
    for m, dvec in enumerate(np.asarray(dirs, np.float64)):
        ph = np.exp(-1j * k * (y @ dvec))
        dn = (nrm @ dvec)[:, None]
        out[m] = np.sum(wy * ph * (py * (-1j * k * dn) - np.asarray(g)[:, None]))
    return out

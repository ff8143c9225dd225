"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module builds meshes, field points, wavenumbers and Neumann data only. It holds none of
the boundary element method's arithmetic (no Green's function, quadrature, assembly, solve or
field evaluation), so both the CUDA path and the FP64 oracle can take their inputs from here
without sharing any part of the computation.

The paper's scenes and modal data are not available, so these stand in for them (paper
Sec. 3.4 and Sec. 5-7 workloads): closed star-shaped bodies of 500 to 40k triangles, the
triangle counts the paper reports (5174 for the plate, 20,000 for phone and cup), wavenumbers
with ka up to 20, Neumann data that are constant per triangle, and field points on spheres and
shells around the body at 2-5 body radii.

Conventions: vertices are float64 (V, 3), triangles int32 (F, 3) with counter-clockwise winding
seen from outside (outward normals), complex data are complex128 numpy arrays.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "icosphere", "uv_sphere", "ring_sphere", "uv_sphere_for", "perturbed_ellipsoid", "centroids_normals",
    "fibonacci_points", "shell_points", "log_uniform", "real_sph_harm", "sh_neumann",
    "monopole_neumann", "monopole_field", "uniform_neumann", "cos_theta_neumann", "Problem",
    "pulsating_sphere", "interior_source", "modal_multirhs", "uneven_batch", "serving_stream",
    "tetrahedron", "octahedron", "nat_params", "nat_queries",
]


# ----------------------------------------------------------------------------------- meshes
def icosphere(level: int):
    """Unit icosphere: the icosahedron with `level` rounds of 4-to-1 midpoint subdivision,
    vertices projected to the unit sphere. F = 20*4^level, V = 10*4^level + 2."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
             (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
             (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
             (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    F = list(faces)
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int32)


def uv_sphere(n_lon: int, n_rings: int):
    """Unit UV sphere: two poles, `n_rings` latitude rings of `n_lon` vertices (equal polar
    angle steps), pole fans plus quads split in two. F = 2*n_lon*n_rings,
    V = n_lon*n_rings + 2."""
    if n_lon < 3 or n_rings < 1:
        raise ValueError("uv_sphere needs n_lon >= 3 and n_rings >= 1")
    verts = [(0.0, 0.0, 1.0)]
    for r in range(n_rings):
        th = math.pi * (r + 1) / (n_rings + 1)
        for c in range(n_lon):
            ph = 2.0 * math.pi * c / n_lon
            verts.append((math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)))
    verts.append((0.0, 0.0, -1.0))
    south = len(verts) - 1

    def vid(r: int, c: int) -> int:
        return 1 + r * n_lon + (c % n_lon)

    F = []
    for c in range(n_lon):
        F.append((0, vid(0, c), vid(0, c + 1)))
    for r in range(n_rings - 1):
        for c in range(n_lon):
            a, b = vid(r, c), vid(r, c + 1)
            d, e = vid(r + 1, c), vid(r + 1, c + 1)
            F.append((a, d, e))
            F.append((a, e, b))
    for c in range(n_lon):
        F.append((south, vid(n_rings - 1, c + 1), vid(n_rings - 1, c)))
    return np.array(verts, dtype=np.float64), np.array(F, dtype=np.int32)


def ring_sphere(n_tri: int):
    """Unit sphere with near-equilateral triangles and exactly `n_tri` triangles (even, >= 8):
    two poles and latitude rings whose vertex counts follow sin(theta) (largest-remainder
    rounding to a total of n_tri/2), consecutive rings stitched by merging their angular
    orders. F = 2 (V - 2). Unlike the UV sphere it has no pole slivers."""
    if n_tri < 8 or n_tri % 2:
        raise ValueError("ring_sphere needs an even triangle count >= 8")
    total = n_tri // 2
    h = math.sqrt(16.0 * math.pi / (math.sqrt(3.0) * n_tri))
    n_rings = max(1, int(round(math.pi / (h * math.sqrt(3.0) / 2.0))) - 1)
    n_rings = min(n_rings, max(1, total // 3))
    thetas = [math.pi * (i + 1) / (n_rings + 1) for i in range(n_rings)]
    want = np.array([math.sin(t) for t in thetas])
    want = want / want.sum() * total
    counts = np.maximum(3, np.floor(want).astype(int))
    while counts.sum() > total:                     # only when the minimum of 3 bites
        counts[np.argmax(counts)] -= 1
    rem = want - np.floor(want)
    for i in np.argsort(-rem)[: total - counts.sum()]:
        counts[i] += 1
    verts = [(0.0, 0.0, 1.0)]
    rings = []
    for i, (t, n) in enumerate(zip(thetas, counts)):
        off = 0.5 * (i % 2)
        angles = [2.0 * math.pi * (j + off) / n for j in range(n)]
        ids = []
        for a in angles:
            ids.append(len(verts))
            verts.append((math.sin(t) * math.cos(a), math.sin(t) * math.sin(a), math.cos(t)))
        rings.append((ids, angles))
    verts.append((0.0, 0.0, -1.0))
    south = len(verts) - 1
    F = []
    ids0, _ = rings[0]
    for j in range(len(ids0)):
        F.append((0, ids0[j], ids0[(j + 1) % len(ids0)]))
    for r in range(n_rings - 1):
        (ia, aa), (ib, ab) = rings[r], rings[r + 1]
        na, nb = len(ia), len(ib)
        # unwrapped angles: A_j = aa[0] + 2 pi j / na, B_j = B_0 + 2 pi j / nb with B_0 the
        # first vertex of ring B at or after aa[0]; merge the two orders counter-clockwise
        b0 = int(np.argmin([(x - aa[0]) % (2 * math.pi) for x in ab]))
        B0 = aa[0] + (ab[b0] - aa[0]) % (2 * math.pi)
        A = lambda j: aa[0] + 2 * math.pi * j / na
        B = lambda j: B0 + 2 * math.pi * j / nb
        ja = jb = 0
        while ja < na or jb < nb:
            ca, cb = ia[ja % na], ib[(b0 + jb) % nb]
            if jb >= nb or (ja < na and A(ja + 1) <= B(jb + 1)):
                F.append((ca, cb, ia[(ja + 1) % na]))
                ja += 1
            else:
                F.append((ca, cb, ib[(b0 + jb + 1) % nb]))
                jb += 1
    ids_l, _ = rings[-1]
    for j in range(len(ids_l)):
        F.append((south, ids_l[(j + 1) % len(ids_l)], ids_l[j]))
    return np.array(verts, dtype=np.float64), np.array(F, dtype=np.int32)


def uv_sphere_for(n_tri_target: int):
    """UV sphere whose triangle count is close to `n_tri_target`: n_rings = round(sqrt(F/4)),
    n_lon = round(F / (2 n_rings)); the actual count is 2*n_lon*n_rings."""
    n_rings = max(1, int(round(math.sqrt(n_tri_target / 4.0))))
    n_lon = max(3, int(round(n_tri_target / (2.0 * n_rings))))
    return uv_sphere(n_lon, n_rings)


def tetrahedron():
    """Regular tetrahedron inscribed in the unit sphere, outward winding."""
    V = np.array([(1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)], dtype=np.float64) / math.sqrt(3)
    F = np.array([(0, 1, 2), (0, 3, 1), (0, 2, 3), (1, 3, 2)], dtype=np.int32)
    return V, F


def octahedron():
    """Regular octahedron inscribed in the unit sphere, outward winding."""
    V = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
                 dtype=np.float64)
    F = np.array([(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4),
                  (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)], dtype=np.int32)
    return V, F


def real_sph_harm(lmax: int, dirs: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics Y_lm (l = 0..lmax, m = -l..l) at unit directions
    `dirs` (n, 3). Returns (n, (lmax+1)^2), column l*l + l + m. Associated Legendre functions
    by the standard three-term recurrence (no Condon-Shortley phase)."""
    dirs = np.asarray(dirs, dtype=np.float64)
    z = np.clip(dirs[:, 2], -1.0, 1.0)
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    n = dirs.shape[0]
    P = {}
    P[(0, 0)] = np.ones(n)
    for m in range(1, lmax + 1):
        P[(m, m)] = P[(m - 1, m - 1)] * (2 * m - 1) * s
    for m in range(0, lmax):
        P[(m + 1, m)] = (2 * m + 1) * z * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * z * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    out = np.zeros((n, (lmax + 1) ** 2))
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            if m == 0:
                out[:, l * l + l] = norm * P[(l, 0)]
            else:
                out[:, l * l + l + m] = math.sqrt(2.0) * norm * P[(l, m)] * np.cos(m * phi)
                out[:, l * l + l - m] = math.sqrt(2.0) * norm * P[(l, m)] * np.sin(m * phi)
    return out


def perturbed_ellipsoid(V: np.ndarray, seed: int, radii=(1.0, 0.8, 0.6), lmax: int = 6,
                        sigma: float = 0.05) -> np.ndarray:
    """Map a unit-sphere mesh's vertices u to e(u) * (1 + sum_{1<=l<=lmax, m} c_lm Y_lm(u)),
    e(u) the point of the ellipsoid with semi-axes `radii` along u, c_lm ~ N(0, sigma^2) drawn
    from numpy's PCG64 with `seed`. l = 0 is left out (it only rescales). Seeds whose radial
    factor is not positive at every vertex are rejected."""
    u = V / np.linalg.norm(V, axis=1, keepdims=True)
    a = np.asarray(radii, dtype=np.float64)
    e = u / np.sqrt(((u / a) ** 2).sum(axis=1, keepdims=True))
    rng = np.random.default_rng(seed)
    c = rng.normal(0.0, sigma, size=(lmax + 1) ** 2)
    c[0] = 0.0
    fac = 1.0 + real_sph_harm(lmax, u) @ c
    if not np.all(fac > 0.0):
        raise ValueError(f"seed {seed} gives a non-star-shaped body")
    return e * fac[:, None]


def centroids_normals(V: np.ndarray, F: np.ndarray):
    """Centroids and unit outward normals of the triangles (input bookkeeping for the data
    generators below)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    return (a + b + c) / 3.0, n


# ------------------------------------------------------------------------------ field points
def fibonacci_points(M: int, R: float) -> np.ndarray:
    """Fibonacci lattice on the sphere of radius R: z_i = 1 - (2i+1)/M, phi_i = i pi (3 - sqrt 5)."""
    i = np.arange(M, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / M
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return R * np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def shell_points(M: int, r_min: float, r_max: float, seed: int) -> np.ndarray:
    """Fibonacci directions with seeded radii r_i = r_min + (r_max - r_min) u_i, u ~ U[0,1)."""
    d = fibonacci_points(M, 1.0)
    r = r_min + (r_max - r_min) * np.random.default_rng(seed).random(M)
    return d * r[:, None]


def log_uniform(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n values log-uniform in [lo, hi] (seeded PCG64)."""
    u = np.random.default_rng(seed).random(n)
    return np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


# ----------------------------------------------------------------------------- Neumann data
def uniform_neumann(F: np.ndarray, value: complex = 1.0) -> np.ndarray:
    """Uniform normal velocity: the pulsating body."""
    return np.full(F.shape[0], value, dtype=np.complex128)


def cos_theta_neumann(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """g = cos(theta) of each centroid's direction: the oscillating (dipole) sphere."""
    c, _ = centroids_normals(V, F)
    return (c[:, 2] / np.linalg.norm(c, axis=1)).astype(np.complex128)


def sh_neumann(V: np.ndarray, F: np.ndarray, nrhs: int, seed: int, lmax: int = 8) -> np.ndarray:
    """Smooth real normal-velocity fields g_j = sum_{l<=lmax,m} c_lm Y_lm(x_j/|x_j|) at the
    centroids x_j, c_lm ~ N(0, 1); returns (F, nrhs) complex128, column-major per RHS."""
    c, _ = centroids_normals(V, F)
    Y = real_sph_harm(lmax, c / np.linalg.norm(c, axis=1, keepdims=True))
    coef = np.random.default_rng(seed).normal(0.0, 1.0, size=(Y.shape[1], nrhs))
    return np.asfortranarray((Y @ coef).astype(np.complex128))


def monopole_field(points: np.ndarray, k: float, x0=(0.0, 0.0, 0.0)) -> np.ndarray:
    """u(x) = e^{ik|x-x0|} / (4 pi |x-x0|): the exterior field of a point source inside the body."""
    d = np.linalg.norm(np.asarray(points) - np.asarray(x0), axis=1)
    return np.exp(1j * k * d) / (4.0 * math.pi * d)


def monopole_neumann(V: np.ndarray, F: np.ndarray, k: float, x0=(0.0, 0.0, 0.0)) -> np.ndarray:
    """du/dn of the interior point source at each centroid (outward normal)."""
    c, n = centroids_normals(V, F)
    d = c - np.asarray(x0)
    rho = np.linalg.norm(d, axis=1)
    u = np.exp(1j * k * rho) / (4.0 * math.pi * rho)
    du = u * (1j * k - 1.0 / rho)
    return du * (d * n).sum(axis=1) / rho


def monopole_neumann_at(Y: np.ndarray, N: np.ndarray, k: float, x0=(0.0, 0.0, 0.0)) -> np.ndarray:
    """du/dn of the interior point source at surface points Y with unit normals N."""
    d = np.asarray(Y) - np.asarray(x0)
    rho = np.linalg.norm(d, axis=1)
    u = np.exp(1j * k * rho) / (4.0 * math.pi * rho)
    du = u * (1j * k - 1.0 / rho)
    return du * (d * np.asarray(N)).sum(axis=1) / rho


# ------------------------------------------------------------------- surface sample points
# Sample sets for the Monte-Carlo solver: points on the surface, their unit outward normals and
# the total surface area. These are the random draws of the method, made here and passed in.
def sphere_samples(M: int, radius: float = 1.0):
    """Fibonacci-lattice points on a sphere (quasi-uniform), exact normals and area."""
    Y = fibonacci_points(M, radius)
    return Y, Y / radius, 4.0 * math.pi * radius * radius


def _triangle_table(V: np.ndarray, F: np.ndarray):
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    cr = np.cross(b - a, c - a)
    dbl = np.linalg.norm(cr, axis=1)
    return a, b, c, cr / dbl[:, None], 0.5 * dbl


def mesh_random_samples(V: np.ndarray, F: np.ndarray, M: int, seed: int):
    """M points of uniform density on a triangle mesh (triangle by area, then uniform
    barycentrics), with the triangle's outward normal; returns (Y, N, total area)."""
    rng = np.random.default_rng(seed)
    a, b, c, n, area = _triangle_table(V, F)
    t = rng.choice(len(F), size=M, p=area / area.sum())
    r1, r2 = rng.random(M), rng.random(M)
    s1 = np.sqrt(r1)
    Y = (1 - s1)[:, None] * a[t] + (s1 * (1 - r2))[:, None] * b[t] + (s1 * r2)[:, None] * c[t]
    return Y, n[t].copy(), float(area.sum())


def mesh_poisson_samples(V: np.ndarray, F: np.ndarray, M: int, seed: int, oversample: int = 8):
    """About M points on a triangle mesh with a minimum spacing (Poisson-disk sampling by
    greedy dart throwing over an oversampled uniform candidate set, in a hash grid), the
    radius shrunk until M points are accepted; returns (Y, N, total area)."""
    Yc, Nc, total = mesh_random_samples(V, F, oversample * M, seed)
    d_hex = math.sqrt(2.0 * total / (math.sqrt(3.0) * M))  # spacing of a hexagonal packing
    for frac in (0.8, 0.75, 0.7, 0.65, 0.6, 0.55, 0.5):
        r = frac * d_hex
        cell = {}
        keep = []
        inv = 1.0 / r
        for i, y in enumerate(Yc):
            key = tuple(np.floor(y * inv).astype(int))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for j in cell.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                            if np.sum((Yc[j] - y) ** 2) < r * r:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                cell.setdefault(key, []).append(i)
                keep.append(i)
                if len(keep) == M:
                    break
        if len(keep) == M:
            idx = np.array(keep)
            return Yc[idx].copy(), Nc[idx].copy(), total
    idx = np.array(keep)
    return Yc[idx].copy(), Nc[idx].copy(), total


# -------------------------------------------------------------------------- named workloads
@dataclass
class Problem:
    """One mesh with its wavenumbers, Neumann data (F, nrhs) and field points."""
    name: str
    V: np.ndarray
    F: np.ndarray
    ks: np.ndarray
    neumann: list = field(default_factory=list)  # one (F, nrhs) array per wavenumber
    points: np.ndarray | None = None
    exact_surface: list | None = None            # per wavenumber, at centroids, when known
    exact_field: list | None = None              # per wavenumber, at points, when known


def pulsating_sphere(level: int = 3, ka: float = 2.0, n_points: int = 256, R: float = 3.0):
    """Unit icosphere (level 3: 1280 triangles), g = 1, one wavenumber, Fibonacci points."""
    V, F = icosphere(level)
    g = uniform_neumann(F)[:, None]
    return Problem("pulsating_sphere", V, F, np.array([ka]), [g], fibonacci_points(n_points, R))


def interior_source(seed: int = 2000, n_tri: int = 10240, n_k: int = 64,
                    ka_range=(0.5, 20.0), n_points: int = 1024, R: float = 4.0):
    """Perturbed ellipsoid (1, 0.8, 0.6) with l <= 6 radial harmonics of std 0.05 on a ring
    sphere of n_tri triangles (10240: V = 5122), Neumann data of a monopole at the origin,
    n_k wavenumbers log-uniform in ka_range, Fibonacci points at radius R. The exterior field
    of the interior source is known exactly."""
    Vs, F = ring_sphere(n_tri)
    V = perturbed_ellipsoid(Vs, seed)
    ks = log_uniform(n_k, *ka_range, seed=seed + 1)
    pts = fibonacci_points(n_points, R)
    c, _ = centroids_normals(V, F)
    neu = [monopole_neumann(V, F, k)[:, None] for k in ks]
    return Problem("interior_source", V, F, ks, neu, pts,
                   [monopole_field(c, k) for k in ks], [monopole_field(pts, k) for k in ks])


def modal_multirhs(seed: int = 3000, level: int = 5, nrhs: int = 64, n_k: int = 16,
                   ka_range=(1.0, 15.0), n_points: int = 4096, shell=(2.0, 5.0)):
    """Perturbed-ellipsoid icosphere (level 5: 20480 triangles), nrhs smooth real SH (l <= 8)
    Neumann fields shared by all wavenumbers, n_k wavenumbers log-uniform, shell points."""
    Vs, F = icosphere(level)
    V = perturbed_ellipsoid(Vs, seed)
    ks = log_uniform(n_k, *ka_range, seed=seed + 1)
    g = sh_neumann(V, F, nrhs, seed + 2)
    pts = shell_points(n_points, shell[0], shell[1], seed + 3)
    return Problem("modal_multirhs", V, F, ks, [g] * n_k, pts)


def uneven_batch(seed: int = 4000, n_mesh: int = 512, f_range=(500, 8000), ka_range=(0.5, 12.0),
                 n_points: int = 1024, R: float = 4.0):
    """n_mesh perturbed ellipsoids with triangle counts log-uniform in f_range (ring spheres),
    one wavenumber (uniform in ka_range) and one smooth SH Neumann field each."""
    rng = np.random.default_rng(seed)
    targets = np.exp(rng.uniform(math.log(f_range[0]), math.log(f_range[1]), n_mesh))
    kas = rng.uniform(ka_range[0], ka_range[1], n_mesh)
    pts = fibonacci_points(n_points, R)
    out = []
    for i in range(n_mesh):
        Vs, F = ring_sphere(2 * int(round(targets[i] / 2)))
        V = perturbed_ellipsoid(Vs, seed + 10 + i)
        g = sh_neumann(V, F, 1, seed + 100000 + i)
        out.append(Problem(f"uneven_{i}", V, F, np.array([kas[i]]), [g], pts))
    return out


def serving_stream(seed: int = 5000, n_req: int = 2000, rate: float = 200.0,
                   f_range=(1000, 40000), ka_range=(0.5, 20.0), nrhs_max: int = 32):
    """Poisson arrivals (rate per second): list of (arrival_s, n_tri_target, ka, nrhs, seed)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    f = np.exp(rng.uniform(math.log(f_range[0]), math.log(f_range[1]), n_req)).astype(int)
    ka = rng.uniform(ka_range[0], ka_range[1], n_req)
    nrhs = rng.integers(1, nrhs_max + 1, n_req)
    return [(float(t[i]), int(f[i]), float(ka[i]), int(nrhs[i]), seed + 7 + i) for i in range(n_req)]


def mc_interior_body(seed: int = 6000, n_tri: int = 10240):
    """The Monte-Carlo workload's body: a ring sphere of n_tri triangles deformed into the
    perturbed ellipsoid of `seed`. Returns (V, F)."""
    Vs, F = ring_sphere(n_tri)
    return perturbed_ellipsoid(Vs, seed), F


def poisson_draws(V: np.ndarray, F: np.ndarray, M: int, seed: int, oversample: int = 8, frac: float = 0.7):
    """Draws for a Poisson-disk sampler aiming at about M samples: oversample * M uniform
    triples in [0, 1)^3 and the radius frac times the spacing of a hexagonal packing of M
    points over the mesh's area. Returns (u, radius)."""
    a, b, c, n, area = _triangle_table(V, F)
    d_hex = math.sqrt(2.0 * float(area.sum()) / (math.sqrt(3.0) * M))
    return np.random.default_rng(seed).random((oversample * M, 3)), frac * d_hex


def mc_interior_source(seed: int = 6000, n_tri: int = 10240, M: int = 4096, n_k: int = 64,
                       ka_range=(0.5, 12.0), n_points: int = 1024, R: float = 4.0, poisson: bool = True):
    """Monte-Carlo workload: the interior-source body (perturbed ellipsoid, l <= 6) sampled with
    M Poisson-disk (or uniform random) points, monopole Neumann data at the samples, n_k
    wavenumbers log-uniform in ka_range, field points at radius R. Returns
    (Y, N, area, ks, [g per k], points, [exact field per k])."""
    V, F = mc_interior_body(seed, n_tri)
    Y, N, area = (mesh_poisson_samples if poisson else mesh_random_samples)(V, F, M, seed + 1)
    ks = log_uniform(n_k, ka_range[0], ka_range[1], seed + 2)
    pts = fibonacci_points(n_points, R)
    return (Y, N, area, ks, [monopole_neumann_at(Y, N, k) for k in ks], pts,
            [monopole_field(pts, k) for k in ks])


# ------------------------------------------------------- neural acoustic transfer field
NAT_LEVELS = (8, 16, 32, 64)  # grid cells per axis of the four levels (paper Sec. 3.4)
NAT_WIDTH = 128               # hidden width; four hidden layers (paper Sec. 3.4)


def nat_params(n_cond: int = 2, n_out: int = 8, table_log2: int = 18, seed: int = 0):
    """Seeded random parameters of the neural transfer field (the trained networks are not
    available): plain float32 draws, with no rounding to any storage precision.

    tables: one (rows, 4) array per level, rows = min((N + 1)^3, 2^table_log2), U(-1, 1);
    weights: four (128, 128) arrays, then (n_out, 128), N(0, 2/128) (He initialisation, so the
    ReLU layers keep the activations' scale); biases: four of 128, then n_out, N(0, 0.05^2).
    Returns a dict with those lists and the shape arguments."""
    rng = np.random.default_rng(seed)
    tables = [rng.uniform(-1.0, 1.0, size=(min((N + 1) ** 3, 1 << table_log2), 4)).astype(np.float32)
              for N in NAT_LEVELS]
    weights, biases = [], []
    for l in range(5):
        n_o = n_out if l == 4 else NAT_WIDTH
        weights.append(rng.normal(0.0, math.sqrt(2.0 / NAT_WIDTH), size=(n_o, NAT_WIDTH)).astype(np.float32))
        biases.append(rng.normal(0.0, 0.05, size=n_o).astype(np.float32))
    return dict(n_cond=n_cond, n_out=n_out, table_log2=table_log2, tables=tables, weights=weights,
                biases=biases)


def nat_queries(n: int, D: int, seed: int) -> np.ndarray:
    """n query rows of D normalised inputs in [0, 1) (float32), uniform."""
    return np.random.default_rng(seed).random((n, D)).astype(np.float32)

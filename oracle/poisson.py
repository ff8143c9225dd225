"""Reference of the Poisson-disk surface sampler (paper Sec. 4.2: samples for the Monte-Carlo BEM
drawn with a minimum distance so that they cover the surface evenly; the paper uses a parallel
GPU sampler after Bowers et al. 2010).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the tests use it; the product library never
does. It shares no code with the CUDA path.

The sampler, as this build defines it (both sides implement exactly this):
  1. candidates: for each draw (u0, u1, u2) in [0, 1)^3, the triangle whose cumulative-area
     interval holds u0 * total area (the first triangle with cumulative area > u0 * A), and the
     point with barycentric coordinates (1 - sqrt(u1), sqrt(u1) (1 - u2), sqrt(u1) u2) of its
     vertices (uniform on the triangle), with the triangle's unit normal;
  2. a grid over the mesh's bounding box with cell size h = r / sqrt(3), so that two points in
     one cell are closer than r; cell (i, j, k) of point x is floor((x - lo) / h) per axis,
     clamped to the grid;
  3. 27 phases (i mod 3, j mod 3, k mod 3) in lexicographic order; in a phase, every cell
     accepts its lowest-index candidate that has no accepted sample within distance r
     (Euclidean, < r rejects) in the 5 x 5 x 5 block of cells around it. Cells of one phase are
     at least three cells apart, so they do not see each other's new samples: the result is the
     same in any order within a phase, and the GPU runs a phase's cells in parallel.
The accepted samples are returned in increasing candidate index.
"""
from __future__ import annotations

import numpy as np


def candidates(V, F, u):
    """Positions (m, 3), unit normals (m, 3) and triangle indices of the draws u (m, 3)."""
    V = np.asarray(V, np.float64)
    F = np.asarray(F, np.int64)
    u = np.asarray(u, np.float64).reshape(-1, 3)
    P = V[F]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    area = 0.5 * np.sqrt((cr[:, 0] * cr[:, 0] + cr[:, 1] * cr[:, 1]) + cr[:, 2] * cr[:, 2])
    cum = np.cumsum(area)
    tri = np.searchsorted(cum, u[:, 0] * cum[-1], side="right")
    tri = np.minimum(tri, len(F) - 1)
    s = np.sqrt(u[:, 1])
    b0, b1, b2 = 1.0 - s, s * (1.0 - u[:, 2]), s * u[:, 2]
    Q = P[tri]
    x = (b0[:, None] * Q[:, 0] + b1[:, None] * Q[:, 1]) + b2[:, None] * Q[:, 2]
    n = cr[tri] / (2.0 * area[tri])[:, None]
    return x, n, tri


def grid(V, r):
    """(lo, h, dims) of the sampling grid."""
    V = np.asarray(V, np.float64)
    lo, hi = V.min(axis=0), V.max(axis=0)
    h = r / np.sqrt(3.0)
    dims = np.floor((hi - lo) / h).astype(np.int64) + 1
    return lo, h, dims


def cell_of(x, lo, h, dims):
    c = np.floor((np.asarray(x) - lo) / h).astype(np.int64)
    return np.clip(c, 0, dims - 1)


def _dist2(a, b):
    d = a - b
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]


def sample(V, F, u, r):
    """Indices (increasing) of the accepted candidates, their positions and normals."""
    x, n, _ = candidates(V, F, u)
    lo, h, dims = grid(V, r)
    cells = cell_of(x, lo, h, dims)
    by_cell = {}
    for i, c in enumerate(map(tuple, cells)):
        by_cell.setdefault(c, []).append(i)
    taken = {}  # cell -> accepted candidate index
    r2 = r * r
    for phase in range(27):
        px, py, pz = phase // 9, (phase // 3) % 3, phase % 3
        for c, idx in by_cell.items():
            if (c[0] % 3, c[1] % 3, c[2] % 3) != (px, py, pz):
                continue
            near = []
            for dx in range(-2, 3):
                for dy in range(-2, 3):
                    for dz in range(-2, 3):
                        s = taken.get((c[0] + dx, c[1] + dy, c[2] + dz))
                        if s is not None:
                            near.append(s)
            for i in sorted(idx):
                if all(_dist2(x[i], x[s]) >= r2 for s in near):
                    taken[c] = i
                    break
    acc = np.array(sorted(taken.values()), dtype=np.int64)
    return acc, x[acc], n[acc]

"""Pins of the Poisson-disk sampler reference (oracle/poisson.py; paper Sec. 4.2). CPU only.

  * the accepted samples are pairwise at least r apart (brute force);
  * the set is maximal over the candidates: every candidate lies within r of a sample;
  * samples are a subset of the candidates, in increasing index;
  * candidates are uniform by area: triangle counts follow the areas, and on one triangle the
    mean of many candidates is its centroid;
  * the definition does not depend on the order of the cells within a phase (the property the
    parallel GPU form relies on): a shuffled order gives the same samples.
"""
import numpy as np

import synthetic as S
from oracle import poisson as PS


def _case(n_cand=6000, r=0.12, seed=0):
    V, F = S.icosphere(3)
    V = S.perturbed_ellipsoid(V, 7)
    u = np.random.default_rng(seed).random((n_cand, 3))
    return V, F, u, r


def test_poisson_property_and_maximality():
    V, F, u, r = _case()
    acc, x, n = PS.sample(V, F, u, r)
    assert len(acc) > 100
    d = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= r
    cand, _, _ = PS.candidates(V, F, u)
    dc = np.linalg.norm(cand[:, None, :] - x[None, :, :], axis=2)
    assert np.all(dc.min(axis=1) < r)
    assert np.all(np.diff(acc) > 0)
    assert np.allclose(cand[acc], x)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)


def test_candidates_uniform_by_area():
    V, F = S.icosphere(1)
    V = S.perturbed_ellipsoid(V, 3)
    u = np.random.default_rng(1).random((200000, 3))
    x, n, tri = PS.candidates(V, F, u)
    P = V[F]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    counts = np.bincount(tri, minlength=len(F))
    expect = area / area.sum() * len(u)
    chi2 = np.sum((counts - expect) ** 2 / expect)
    assert chi2 < len(F) + 6 * np.sqrt(2 * len(F))
    t0 = 5
    pts = x[tri == t0]
    assert np.linalg.norm(pts.mean(axis=0) - P[t0].mean(axis=0)) < 4 * np.sqrt(area[t0]) / np.sqrt(len(pts))


def test_order_within_a_phase_does_not_matter():
    """The phases written out again with the cells of each phase visited in a shuffled order."""
    V, F, u, r = _case(n_cand=3000, r=0.15, seed=2)
    acc, _, _ = PS.sample(V, F, u, r)
    x, n, _ = PS.candidates(V, F, u)
    lo, h, dims = PS.grid(V, r)
    cells = PS.cell_of(x, lo, h, dims)
    by_cell = {}
    for i, c in enumerate(map(tuple, cells)):
        by_cell.setdefault(c, []).append(i)
    order = list(by_cell.items())
    np.random.default_rng(3).shuffle(order)
    taken = {}
    for phase in range(27):
        px, py, pz = phase // 9, (phase // 3) % 3, phase % 3
        for c, idx in order:
            if (c[0] % 3, c[1] % 3, c[2] % 3) != (px, py, pz):
                continue
            near = [taken[(c[0] + a, c[1] + b, c[2] + d)] for a in range(-2, 3) for b in range(-2, 3)
                    for d in range(-2, 3) if (c[0] + a, c[1] + b, c[2] + d) in taken]
            for i in sorted(idx):
                if all(PS._dist2(x[i], x[s]) >= r * r for s in near):
                    taken[c] = i
                    break
    assert np.array_equal(np.array(sorted(taken.values())), acc)


def test_denser_radius_gives_more_samples():
    V, F, u, _ = _case(n_cand=8000, seed=4)
    a1, _, _ = PS.sample(V, F, u, 0.2)
    a2, _, _ = PS.sample(V, F, u, 0.1)
    # on a surface the count grows like 1 / r^2 (up to the candidates' coverage)
    assert 2.5 < len(a2) / len(a1) < 4.5

"""Writes the oracle regression fixtures in this directory. It calls only oracle/ and the
input generators, never the CUDA path: python tests/golden/make_golden.py

The paper prints no worked numerical values for its BEM (its tables give only run times and
image metrics), so these fixtures freeze the oracle's own output on small cases. A change in
them means the oracle's arithmetic changed, which needs the paper passage or reading that
justifies it.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402


def cplx(a):
    a = np.asarray(a).ravel()
    return [[float(v.real), float(v.imag)] for v in a]


def main():
    V, F = S.octahedron()
    L, R = oracle.assemble(V, F, 1.5)
    with open(os.path.join(HERE, "octahedron_k1.5.json"), "w") as f:
        json.dump({"mesh": "regular octahedron inscribed in the unit sphere", "k": 1.5,
                   "adj_levels": oracle.ADJ_LEVELS, "self_points": oracle.SELF_POINTS,
                   "L": cplx(L), "R": cplx(R)}, f, indent=0)
    V, F = S.icosphere(2)
    g = S.uniform_neumann(F)
    L, R = oracle.assemble(V, F, 2.0)
    p = np.linalg.solve(L, R @ g)
    pts = S.fibonacci_points(16, 3.0)
    fld = oracle.evaluate(V, F, 2.0, pts, p, g)
    with open(os.path.join(HERE, "pulsating_icosphere2_k2.json"), "w") as f:
        json.dump({"mesh": "icosphere level 2 (320 triangles)", "k": 2.0, "neumann": 1.0,
                   "points": "16 Fibonacci points at radius 3",
                   "p": cplx(p), "field": cplx(fld)}, f, indent=0)
    # the Poisson-disk sampler (Sec. 4.2, in this build's grid form): accepted draws and
    # positions on a small case
    from oracle import poisson as PS
    u = np.random.default_rng(11).random((400, 3))
    idx, x, _ = PS.sample(V, F, u, 0.25)
    with open(os.path.join(HERE, "poisson_icosphere2_r0.25.json"), "w") as f:
        json.dump({"mesh": "icosphere level 2 (320 triangles)", "draws": "numpy default_rng(11).random((400, 3))",
                   "radius": 0.25, "accepted": [int(i) for i in idx], "positions": x.tolist()}, f, indent=0)


if __name__ == "__main__":
    main()

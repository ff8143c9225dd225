"""The oracle reproduces its frozen fixtures (tests/golden, written by make_golden.py)."""
import json
import os

import numpy as np

import synthetic as S

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def _c(a):
    a = np.asarray(a, dtype=np.float64)
    return a[:, 0] + 1j * a[:, 1]


def test_octahedron_operator(oracle_lib):
    d = _load("octahedron_k1.5.json")
    V, F = S.octahedron()
    L, R = oracle_lib.assemble(V, F, d["k"], adj_levels=d["adj_levels"], self_pts=d["self_points"])
    assert np.allclose(L.ravel(), _c(d["L"]), rtol=1e-13, atol=1e-15)
    assert np.allclose(R.ravel(), _c(d["R"]), rtol=1e-13, atol=1e-15)


def test_pulsating_icosphere(oracle_lib):
    d = _load("pulsating_icosphere2_k2.json")
    V, F = S.icosphere(2)
    g = S.uniform_neumann(F)
    L, R = oracle_lib.assemble(V, F, d["k"])
    p = np.linalg.solve(L, R @ g)
    assert np.allclose(p, _c(d["p"]), rtol=1e-11)
    fld = oracle_lib.evaluate(V, F, d["k"], S.fibonacci_points(16, 3.0), p, g)
    assert np.allclose(fld, _c(d["field"]), rtol=1e-11)


def test_poisson_sampler():
    from oracle import poisson as PS
    d = _load("poisson_icosphere2_r0.25.json")
    V, F = S.icosphere(2)
    u = np.random.default_rng(11).random((400, 3))
    idx, x, _ = PS.sample(V, F, u, d["radius"])
    assert idx.tolist() == d["accepted"]
    assert np.array_equal(x, np.asarray(d["positions"]))

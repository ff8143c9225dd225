"""Serving loop on the GPU: requests that run concurrently give the same bits as the same
requests alone (every reduction has a fixed order), admission respects the memory budget, and
a device wait that nothing completes gives up with a status instead of hanging."""
import time

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2506_06190_gb300 import build
    build.build()
    import paper_2506_06190_gb300 as nb
    return nb


def _jobs():
    out = []
    for i, (n_tri, nrhs) in enumerate([(640, 1), (2100, 2), (900, 3), (1500, 1), (1100, 2), (2400, 1)]):
        Vs, F = S.ring_sphere(n_tri)
        V = S.perturbed_ellipsoid(Vs, 300 + i)
        g = S.sh_neumann(V, F, nrhs, 400 + i)
        out.append(dict(V=V, F=F, k=0.8 + 1.7 * i, neumann=g if nrhs > 1 else g[:, 0],
                        points=S.fibonacci_points(40, 4.0)))
    return out


def _oracle_check(oracle_lib, jd, p, f):
    """Every right-hand side of a served request against the FP64 oracle (dense solve of the
    oracle's operators), surface and field, at the solver's 1e-4 bar."""
    L, R = oracle_lib.assemble(jd["V"], jd["F"], jd["k"])
    G = np.asarray(jd["neumann"]).reshape(len(jd["F"]), -1)
    P = np.asarray(p).reshape(len(jd["F"]), -1, order="F")
    Fd = np.asarray(f).reshape(len(jd["points"]), -1, order="F")
    for s in range(G.shape[1]):
        p_ref = np.linalg.solve(L, R @ G[:, s])
        f_ref = oracle_lib.evaluate(jd["V"], jd["F"], jd["k"], jd["points"], p_ref, G[:, s])
        assert np.linalg.norm(P[:, s] - p_ref) / np.linalg.norm(p_ref) < 1e-4
        assert np.linalg.norm(Fd[:, s] - f_ref) / np.linalg.norm(f_ref) < 1e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_results_same_alone_and_in_the_mix(nb, oracle_lib, prec):
    """Six requests of 640-2400 triangles and 1-3 right-hand sides through three slots: each
    result is bit-identical to the same request solved alone, and within 1e-4 of the FP64
    oracle, in plain FP32 and in mixed precision (BF16 inner solves, FP32 refinement)."""
    opts = nb.nat_bem_opts_default(prec=nb.PREC_FP32 if prec == "fp32" else nb.PREC_MIXED_BF16)
    jobs = _jobs()
    alone = []
    for jd in jobs:
        with nb.Operator.assemble(jd["V"], jd["F"], jd["k"], opts) as op:
            p, info, st = op.solve(jd["neumann"])
            assert st == nb.NAT_BEM_OK
            alone.append((p, op.evaluate(jd["points"], p, jd["neumann"])))
    with nb.Server(64 << 30, opts, slots=3) as srv:
        tickets = [srv.submit(jd) for jd in jobs]
        res = [srv.wait(t, 120000) for t in tickets]
        assert srv.reserved() == 0
    for (st, p, f, info, dev_ms, q_ms, tot_ms), (p1, f1), jd in zip(res, alone, jobs):
        assert st == nb.NAT_BEM_OK and info.iterations > 0 and dev_ms > 0 and tot_ms >= q_ms >= 0
        if prec == "bf16":
            assert info.refinements >= 1
        assert np.array_equal(p, p1) and np.array_equal(f, f1)
        _oracle_check(oracle_lib, jd, p, f)


def test_budget_admits_one_at_a_time(nb):
    jobs = _jobs()[:3]
    need = max(nb.nat_bem_required_bytes(int(j["F"].shape[0]), 1 if np.ndim(j["neumann"]) == 1 else j["neumann"].shape[1])
               for j in jobs)
    with nb.Server(need + 1, slots=3) as srv:
        tickets = [srv.submit(jd) for jd in jobs]
        res = [srv.wait(t, 120000) for t in tickets]
    assert all(r[0] == nb.NAT_BEM_OK for r in res)
    q = [r[5] for r in res]
    assert q[0] < q[1] < q[2]  # each waited for the memory of the previous one


def test_bounded_device_wait_gives_up(nb):
    t = time.time()
    st = nb.nat_bem_selftest_bounded_wait(50)
    dt = time.time() - t
    assert st == nb.NAT_BEM_ETIMEOUT and dt < 5.0
    V, F = S.icosphere(1)  # the context is still usable
    with nb.Operator.assemble(V, F, 1.0) as op:
        p, info, st = op.solve(S.uniform_neumann(F))
        assert st == nb.NAT_BEM_OK

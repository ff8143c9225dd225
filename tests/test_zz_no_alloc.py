"""nat_bem_eval_noalloc: field evaluation for callers that cannot allocate device memory.

It must give what nat_bem_eval gives (same 1e-4 relative bar as the field parity tests) on
consecutive calls that share its fixed scratch array, reject more points than the array holds,
and refuse host pointers (staging them would allocate). This file is collected last so that a
run stopping at the first failure has already run every other test; it also passes alone.
"""
import ctypes

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the field tolerance of the parity tests


@pytest.fixture(scope="module")
def nb():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2506_06190_gb300 import build
    build.build()
    import paper_2506_06190_gb300 as nb
    return nb


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _check_calls(nb, op, cases):
    """Each case through nat_bem_eval_noalloc, one call after another (the same scratch array),
    against nat_bem_eval on the same inputs."""
    import torch
    for pts, p, g in cases:
        ref = op.evaluate(pts, p, g)
        out = torch.full_like(ref, complex(np.nan, np.nan))
        st = nb.nat_bem_eval_noalloc(op.handle, pts, p, g, out)
        assert st == nb.NAT_BEM_OK, nb.nat_bem_last_error()
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < TOL


def test_noalloc_matches_eval_on_consecutive_calls(nb):
    """Three, one and six right-hand sides in a row: six takes two passes of four through the
    shared partial sums, so the second pass reads what the first one left and must overwrite
    it first."""
    import torch
    Vs, F = S.ring_sphere(900)
    V = S.perturbed_ellipsoid(Vs, 31)
    k = 4.2
    G = torch.from_numpy(np.ascontiguousarray(S.sh_neumann(V, F, 6, 5).T).astype(np.complex64)).cuda()
    with nb.Operator.assemble(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda(), k) as op:
        P, _, st = op.solve(G)
        assert st == nb.NAT_BEM_OK
        _check_calls(nb, op, [
            (torch.from_numpy(S.shell_points(300, 2.0, 5.0, 1)).cuda(), P[:3].contiguous(), G[:3].contiguous()),
            (torch.from_numpy(S.fibonacci_points(77, 3.0)).cuda(), P[1:2].contiguous(), G[1:2].contiguous()),
            (torch.from_numpy(S.shell_points(500, 2.0, 5.0, 2)).cuda(), P, G)])


def test_noalloc_at_the_point_limit(nb):
    """65,536 points (the most one call takes: the scratch then allows a single element split)
    and 20,000 points (three splits instead of the four per SM that nat_bem_eval takes), two
    right-hand sides, against nat_bem_eval."""
    import torch
    Vs, F = S.ring_sphere(2306)
    V = S.perturbed_ellipsoid(Vs, 33)
    k = 3.0
    G = torch.from_numpy(np.ascontiguousarray(S.sh_neumann(V, F, 2, 6).T).astype(np.complex64)).cuda()
    with nb.Operator.assemble(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda(), k) as op:
        P, _, st = op.solve(G)
        assert st == nb.NAT_BEM_OK
        _check_calls(nb, op, [(torch.from_numpy(S.shell_points(65536, 2.0, 5.0, 3)).cuda(), P, G),
                              (torch.from_numpy(S.shell_points(20000, 2.0, 5.0, 4)).cuda(), P, G)])


def test_noalloc_monte_carlo_op(nb):
    """A Monte-Carlo op (one point per sample) through the same entry point."""
    import torch
    V, F = S.mc_interior_body(6000, 2000)
    Y, N, area = S.mesh_random_samples(V, F, 700, 7)
    k = 2.5
    g = torch.from_numpy(S.monopole_neumann_at(Y, N, k).astype(np.complex64)).cuda()
    with nb.Operator.assemble_mc(Y, N, area, k) as op:
        p, _, st = op.solve(g)
        assert st == nb.NAT_BEM_OK
        _check_calls(nb, op, [(torch.from_numpy(S.fibonacci_points(129, 4.0)).cuda(), p, g)])


def test_noalloc_binding_checks_shapes_before_launching(nb):
    """The C call cannot see array sizes: the binding rejects an undersized output, a wrong
    points shape, mismatched data and host tensors with ValueError, and launches nothing."""
    import torch
    V, F = S.icosphere(1)
    g = torch.ones((5, len(F)), dtype=torch.complex64, device="cuda")
    with nb.Operator.assemble(V, F, 1.0) as op:
        p, _, _ = op.solve(g)
        pts = torch.from_numpy(S.fibonacci_points(40, 3.0)).cuda()
        ok_out = torch.zeros((5, 40), dtype=torch.complex64, device="cuda")
        torch.cuda.synchronize()
        before = nb.nat_bem_trace_launches()
        bad = [(pts, p, g, torch.zeros(40, dtype=torch.complex64, device="cuda")),   # one RHS of five
               (pts[:, :2].contiguous(), p, g, ok_out),                              # (m, 2) points
               (pts, p, g[:3].contiguous(), ok_out),                                 # neumann != p
               (pts.cpu(), p, g, ok_out)]                                           # host points
        for a in bad:
            with pytest.raises(ValueError):
                nb.nat_bem_eval_noalloc(op.handle, *a)
        assert nb.nat_bem_trace_launches() == before
        assert nb.nat_bem_eval_noalloc(op.handle, pts, p, g, ok_out) == nb.NAT_BEM_OK


def test_noalloc_limits_and_host_pointers(nb):
    import torch
    V, F = S.icosphere(1)
    g = torch.ones(len(F), dtype=torch.complex64, device="cuda")
    with nb.Operator.assemble(V, F, 1.0) as op:
        p, _, _ = op.solve(g)
        big = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
        out = torch.zeros(65537, dtype=torch.complex64, device="cuda")
        assert nb.nat_bem_eval_noalloc(op.handle, big, p, g, out) == nb.NAT_BEM_EINVAL
        assert "65,536" in nb.nat_bem_last_error() or "65536" in nb.nat_bem_last_error()
        pts_h = S.fibonacci_points(8, 3.0)
        out_h = np.zeros(8, dtype=np.complex64)
        st = nb.lib().nat_bem_eval_noalloc(op.handle, ctypes.c_void_p(pts_h.ctypes.data), 8,
                                          ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(g.data_ptr()), 1,
                                          ctypes.c_void_p(out_h.ctypes.data), None)
        assert st == nb.NAT_BEM_EINVAL and "device pointers" in nb.nat_bem_last_error()

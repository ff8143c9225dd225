"""The C-ABI library loads, exports every symbol include/nat_bem.h declares, and rejects bad
arguments and invalid meshes on the host before any device work (CPU only: no compute calls)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nb():
    from paper_2506_06190_gb300 import build
    build.build()
    import paper_2506_06190_gb300 as nb
    return nb


def _declared():
    hdr = open(os.path.join(ROOT, "include", "nat_bem.h")).read()
    return sorted(set(re.findall(r"NAT_BEM_API\s+[\w\s\*]*?\b(nat_(?:bem|field)_\w+)\s*\(", hdr)))


def test_header_declares_the_binding_names(nb):
    assert _declared() == sorted(nb.EXPORTED)


def test_library_exports_every_declared_symbol(nb):
    out = subprocess.run(["nm", "-D", "--defined-only", nb.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(nat_(?:bem|field)_\w+)", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(nb.lib(), name)


def test_opts_defaults(nb):
    o = nb.nat_bem_opts_default()
    assert o.adj_subdiv_levels == 2 and o.self_theta_pts == 16
    assert o.tol == 1e-6 and o.max_iter == 200 and o.prec == nb.PREC_FP32
    assert o.inner_max_iter == 60 and o.inner_tol == 1e-2 and o.max_refinements == 10
    assert o.restart == 0 and o.quad_regular == 7 and o.device_loop == 1


def test_required_bytes(nb):
    n = 10240
    b = nb.nat_bem_required_bytes(n, 1)
    ld = (n + 31) // 32 * 32
    assert b >= 16 * n * ld                       # L and R in complex64
    assert b < 16 * n * ld * 1.2
    assert nb.nat_bem_required_bytes(n, 64) > b
    assert nb.nat_bem_required_bytes(0, 1) == 0


def test_required_bytes_fp16_copy(nb):
    """The FP16 copy takes the bytes of the BF16 one plus one scale per row."""
    n = 10240
    b16 = nb.nat_bem_required_bytes(n, 1, nb.nat_bem_opts_default(prec=nb.PREC_MIXED_BF16))
    f16 = nb.nat_bem_required_bytes(n, 1, nb.nat_bem_opts_default(prec=nb.PREC_MIXED_FP16))
    assert f16 - b16 == 4 * n


def test_required_bytes_restart(nb):
    """GMRES(m) keeps m + 1 Krylov vectors instead of max_iter + 1: admission sees the saving.
    A 40k-triangle request with 32 right-hand sides at max_iter = 200 needs 16 n 32 (m + 1)
    bytes of basis: about 4.1 GB unrestarted, about 0.63 GB at m = 30."""
    n, nrhs = 40000, 32
    full = nb.nat_bem_required_bytes(n, nrhs)
    r30 = nb.nat_bem_required_bytes(n, nrhs, nb.nat_bem_opts_default(restart=30))
    assert full - r30 >= 16 * n * nrhs * (200 - 30)
    assert nb.nat_bem_required_bytes(n, nrhs, nb.nat_bem_opts_default(restart=200)) == full
    # restart beyond max_iter is the unrestarted solve
    assert nb.nat_bem_required_bytes(n, nrhs, nb.nat_bem_opts_default(restart=255)) == full


def _assemble_status(nb, V, F, k=2.0, opts=None):
    op = ctypes.c_void_p()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    st = nb.lib().nat_bem_assemble(ctypes.c_void_p(V.ctypes.data), V.shape[0],
                                   ctypes.c_void_p(F.ctypes.data), F.shape[0], k,
                                   ctypes.byref(opts) if opts else None, None, ctypes.byref(op))
    return st, op


@pytest.mark.parametrize("case", ["inward", "open", "flipped_one", "index", "nan", "degenerate",
                                  "k_zero", "k_nan", "empty", "bad_levels", "bad_maxit",
                                  "maxit_unrestarted", "bad_restart", "bad_quad", "bad_loop"])
def test_assemble_rejects_bad_input(nb, case):
    V, F = S.icosphere(1)
    k, opts = 2.0, None
    if case == "inward":
        F = F[:, ::-1]
    elif case == "open":
        F = F[:-1]
    elif case == "flipped_one":
        F = F.copy(); F[3, 1], F[3, 2] = F[3, 2], F[3, 1]
    elif case == "index":
        F = F.copy(); F[0, 0] = V.shape[0] + 5
    elif case == "nan":
        V = V.copy(); V[2, 1] = np.nan
    elif case == "degenerate":
        V = V.copy(); V[F[0, 1]] = V[F[0, 0]]
    elif case == "k_zero":
        k = 0.0
    elif case == "k_nan":
        k = float("nan")
    elif case == "empty":
        F = F[:0]
    elif case == "bad_levels":
        opts = nb.nat_bem_opts_default(adj_subdiv_levels=7)
    elif case == "bad_maxit":
        opts = nb.nat_bem_opts_default(max_iter=0)
    elif case == "maxit_unrestarted":  # more than 255 iterations need restarts
        opts = nb.nat_bem_opts_default(max_iter=300)
    elif case == "bad_restart":
        opts = nb.nat_bem_opts_default(restart=256)
    elif case == "bad_quad":
        opts = nb.nat_bem_opts_default(quad_regular=6)
    elif case == "bad_loop":
        opts = nb.nat_bem_opts_default(device_loop=2)
    st, op = _assemble_status(nb, V, F, k, opts)
    assert st == nb.NAT_BEM_EINVAL and not op.value
    assert len(nb.nat_bem_last_error()) > 0


@pytest.mark.parametrize("case", ["one_sample", "area_zero", "area_nan", "k_zero", "null"])
def test_assemble_mc_rejects_bad_input(nb, case):
    """Argument checks that need no device (normals and positions are checked on the device)."""
    Y, N, A = S.sphere_samples(64)
    m, area, k = 64, A, 2.0
    if case == "one_sample":
        m = 1
    elif case == "area_zero":
        area = 0.0
    elif case == "area_nan":
        area = float("nan")
    elif case == "k_zero":
        k = 0.0
    Y = np.ascontiguousarray(Y)
    N = np.ascontiguousarray(N)
    op = ctypes.c_void_p()
    py = None if case == "null" else ctypes.c_void_p(Y.ctypes.data)
    st = nb.lib().nat_bem_assemble_mc(py, ctypes.c_void_p(N.ctypes.data), m, area, k, None, None,
                                      ctypes.byref(op))
    assert st == nb.NAT_BEM_EINVAL and not op.value
    assert len(nb.nat_bem_last_error()) > 0


def test_solve_and_eval_reject_null(nb):
    L = nb.lib()
    assert L.nat_bem_solve(None, None, 1, None, None, None) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_eval(None, None, 4, None, None, 1, None, None) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_op_rows(None, 0, 0, 1, None, None) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_op_size(None) == 0
    assert L.nat_bem_far_field(None, None, 4, None, None, 1, None, None) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_sample_field(None, None, 4, None, 1.0, 2.0, None, None, 1, None, None,
                                  None) == nb.NAT_BEM_EINVAL
    L.nat_bem_destroy(None)


def test_run_batch_fused_rejects_bad_arguments(nb):
    """Argument checks of the fused batch happen for every job before any device work."""
    L = nb.lib()
    V, F = S.icosphere(1)
    g = S.uniform_neumann(F).astype(np.complex64)
    p = np.zeros(len(F), np.complex64)
    job = nb.Job(ctypes.c_void_p(V.ctypes.data), len(V), ctypes.c_void_p(F.ctypes.data), len(F), 2.0,
                 ctypes.c_void_p(g.ctypes.data), 1, None, 0, ctypes.c_void_p(p.ctypes.data), None,
                 nb.SolveInfo(), 0, 0.0)
    arr = (nb.Job * 2)(job, job)
    assert L.nat_bem_run_batch_fused(arr, 2, None, 0, 2, None) == nb.NAT_BEM_EINVAL      # max_batch
    assert L.nat_bem_run_batch_fused(arr, 2, None, 257, 2, None) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_run_batch_fused(arr, 2, None, 4, 0, None) == nb.NAT_BEM_EINVAL     # concurrency
    assert L.nat_bem_run_batch_fused(None, 1, None, 4, 2, None) == nb.NAT_BEM_EINVAL
    arr[1].k = 0.0                                                                     # a bad job
    assert L.nat_bem_run_batch_fused(arr, 2, None, 4, 2, None) == nb.NAT_BEM_EINVAL
    assert "job 1" in nb.nat_bem_last_error()
    arr[1].k = 2.0
    arr[1].m = 5                                                                       # points missing
    assert L.nat_bem_run_batch_fused(arr, 2, None, 4, 2, None) == nb.NAT_BEM_EINVAL
    bad = nb.nat_bem_opts_default(restart=-1)
    assert L.nat_bem_run_batch_fused(arr, 1, ctypes.byref(bad), 4, 2, None) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_run_batch_fused(arr, 0, None, 4, 2, None) == nb.NAT_BEM_OK


def test_nat_field_rejects_bad_arguments(nb):
    """Host-side checks of the neural-field entry points (before any device call)."""
    L = nb.lib()
    h = ctypes.c_void_p()
    t = np.zeros(16, np.float32)
    w = np.zeros(16, np.float32)
    b = np.zeros(16, np.float32)
    ok = (ctypes.c_void_p(t.ctypes.data), ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(b.ctypes.data))
    assert L.nat_field_create(2, 8, 18, None, ok[1], ok[2], None, ctypes.byref(h)) == nb.NAT_BEM_EINVAL
    assert L.nat_field_create(2, 8, 18, *ok, None, None) == nb.NAT_BEM_EINVAL
    for n_cond, n_out, log2 in ((-1, 8, 18), (9, 8, 18), (2, 0, 18), (2, 129, 18), (2, 8, 11), (2, 8, 25)):
        assert L.nat_field_create(n_cond, n_out, log2, *ok, None, ctypes.byref(h)) == nb.NAT_BEM_EINVAL
        assert not h.value
    assert L.nat_field_forward(None, None, 4, None, None) == nb.NAT_BEM_EINVAL
    assert nb.nat_bem_gemv_variant(0) == -1
    L.nat_field_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2506_06190_gb300 as nb
    monkeypatch.setattr(nb, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nb, "_lib", None)
    with pytest.raises(ImportError):
        nb.lib()


def test_galerkin_rejects_bad_arguments(nb):
    """Host-side checks of nat_bem_assemble_galerkin before any device call."""
    L = nb.lib()
    op = ctypes.c_void_p()
    V = np.zeros((4, 3))
    F = np.zeros((4, 3), np.int32)
    pv, pf = ctypes.c_void_p(V.ctypes.data), ctypes.c_void_p(F.ctypes.data)
    assert L.nat_bem_assemble_galerkin(None, 4, pf, 4, 1.0, None, None, ctypes.byref(op)) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_assemble_galerkin(pv, 4, pf, 4, 1.0, None, None, None) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_assemble_galerkin(pv, 4, pf, 4, -2.0, None, None, ctypes.byref(op)) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_assemble_galerkin(pv, 4, pf, 0, 1.0, None, None, ctypes.byref(op)) == nb.NAT_BEM_EINVAL
    assert L.nat_bem_assemble_galerkin(pv, 4, pf, 65537, 1.0, None, None, ctypes.byref(op)) == nb.NAT_BEM_EINVAL
    assert not op.value
    assert L.nat_bem_op_neumann_size(None) == 0


def test_poisson_sample_rejects_bad_arguments(nb):
    L = nb.lib()
    V, F = S.icosphere(1)
    u = np.zeros((8, 3))
    pv, pf, pu = (ctypes.c_void_p(a.ctypes.data) for a in (V, F, u))
    out = np.zeros((8, 3))
    po = ctypes.c_void_p(out.ctypes.data)
    cnt = ctypes.c_int64(-1)
    ok = dict(nv=len(V), nt=len(F), r=0.1, m=8, cap=8)

    def call(pv=pv, nv=ok["nv"], pf=pf, nt=ok["nt"], r=ok["r"], pu=pu, m=ok["m"], cap=ok["cap"], po=po, cnt=cnt):
        return L.nat_bem_poisson_sample(pv, nv, pf, nt, r, pu, m, cap, None, po, po,
                                        ctypes.byref(cnt) if cnt is not None else None, None)

    assert call(pv=None) == nb.NAT_BEM_EINVAL
    assert call(pf=None) == nb.NAT_BEM_EINVAL
    assert call(pu=None) == nb.NAT_BEM_EINVAL
    assert call(cnt=None) == nb.NAT_BEM_EINVAL
    assert call(nv=0) == nb.NAT_BEM_EINVAL
    assert call(nt=0) == nb.NAT_BEM_EINVAL
    assert call(m=-1) == nb.NAT_BEM_EINVAL
    assert call(m=1 << 31) == nb.NAT_BEM_EINVAL
    assert call(cap=-1) == nb.NAT_BEM_EINVAL
    assert call(po=None) == nb.NAT_BEM_EINVAL
    for r in (0.0, -1.0, float("nan"), float("inf")):
        assert call(r=r) == nb.NAT_BEM_EINVAL

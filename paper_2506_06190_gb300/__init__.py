"""Python binding of libnatbem.so, the GB300 Burton-Miller BEM library (include/nat_bem.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels. The
functions keep the C names (nat_bem_assemble, nat_bem_solve, nat_bem_eval, ...). Arrays may be
numpy arrays (host memory) or torch tensors (host or CUDA); CUDA tensors are passed by device
pointer together with torch's current stream, so no copy is made.

Layouts: vertices float64 (nv, 3); triangles int32 (nt, 3); complex data complex64 with one
right-hand side per column of an (nt, nrhs) Fortran-ordered numpy array, or one per row of a
(nrhs, nt) C-contiguous torch tensor (the same bytes); points float64 (m, 3).

The library must have been built (python -m paper_2506_06190_gb300.build); there is no CPU
fallback, and importing functions that need it raises if libnatbem.so is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnatbem.so")

NAT_BEM_OK, NAT_BEM_EINVAL, NAT_BEM_ENOMEM, NAT_BEM_ENOCONV = 0, 1, 2, 3
NAT_BEM_ECUDA, NAT_BEM_ETIMEOUT, NAT_BEM_EBUSY = 4, 5, 6
PREC_FP32, PREC_MIXED_TF32, PREC_MIXED_BF16, PREC_MIXED_FP16 = 0, 1, 2, 3
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "ECUDA", 5: "ETIMEOUT", 6: "EBUSY"}

# every symbol include/nat_bem.h declares
EXPORTED = ["nat_bem_opts_default", "nat_bem_assemble", "nat_bem_reassemble", "nat_bem_solve", "nat_bem_eval",
            "nat_bem_op_rows", "nat_bem_op_size", "nat_bem_required_bytes", "nat_bem_destroy",
            "nat_bem_last_error", "nat_bem_trace_enable", "nat_bem_trace_reset",
            "nat_bem_trace_launches", "nat_bem_trace_kernel", "nat_bem_eval_noalloc",
            "nat_bem_run_batch", "nat_bem_trace_select", "nat_bem_op_apply",
            "nat_bem_server_create", "nat_bem_submit", "nat_bem_wait", "nat_bem_server_reserved",
            "nat_bem_server_destroy", "nat_bem_selftest_bounded_wait", "nat_bem_assemble_mc",
            "nat_bem_far_field", "nat_bem_sample_field", "nat_bem_gemv_variant", "nat_field_create",
            "nat_field_forward", "nat_field_destroy", "nat_bem_assemble_galerkin",
            "nat_bem_op_neumann_size", "nat_bem_trace_durations", "nat_bem_poisson_sample",
            "nat_bem_run_batch_fused"]
ENGINE_AUTO, ENGINE_FP32, ENGINE_TF32, ENGINE_BF16, ENGINE_FP16, ENGINE_GEMV0 = 0, 1, 2, 3, 4, 10
GEMV_VARIANTS = 8


class NatBemError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("adj_subdiv_levels", ctypes.c_int32), ("self_theta_pts", ctypes.c_int32),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("inner_max_iter", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_refinements", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("quad_regular", ctypes.c_int32), ("device_loop", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("rel_residual", ctypes.c_double)]


class Job(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("nv", ctypes.c_int64), ("tris", ctypes.c_void_p),
                ("nt", ctypes.c_int64), ("k", ctypes.c_double), ("neumann", ctypes.c_void_p),
                ("nrhs", ctypes.c_int32), ("pts", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("p_out", ctypes.c_void_p), ("field_out", ctypes.c_void_p), ("info", SolveInfo),
                ("status", ctypes.c_int), ("device_ms", ctypes.c_float)]


_lib = None


def lib():
    """Load libnatbem.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2506_06190_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.nat_bem_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.nat_bem_opts_default.restype = None
        L.nat_bem_assemble.argtypes = [vp, i64, vp, i64, d, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
        L.nat_bem_assemble.restype = ctypes.c_int
        L.nat_bem_assemble_mc.argtypes = [vp, vp, i64, d, d, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
        L.nat_bem_assemble_mc.restype = ctypes.c_int
        L.nat_bem_poisson_sample.argtypes = [vp, i64, vp, i64, d, vp, i64, i64, vp, vp, vp,
                                             ctypes.POINTER(i64), vp]
        L.nat_bem_poisson_sample.restype = ctypes.c_int
        L.nat_bem_far_field.argtypes = [vp, vp, i64, vp, vp, ctypes.c_int32, vp, vp]
        L.nat_bem_far_field.restype = ctypes.c_int
        L.nat_bem_sample_field.argtypes = [vp, vp, i64, vp, d, d, vp, vp, ctypes.c_int32, vp, vp, vp]
        L.nat_bem_sample_field.restype = ctypes.c_int
        L.nat_bem_reassemble.argtypes = [vp, d, vp]
        L.nat_bem_reassemble.restype = ctypes.c_int
        L.nat_bem_solve.argtypes = [vp, vp, i32, vp, ctypes.POINTER(SolveInfo), vp]
        L.nat_bem_solve.restype = ctypes.c_int
        L.nat_bem_eval.argtypes = [vp, vp, i64, vp, vp, i32, vp, vp]
        L.nat_bem_eval.restype = ctypes.c_int
        L.nat_bem_eval_noalloc.argtypes = [vp, vp, i64, vp, vp, i32, vp, vp]
        L.nat_bem_eval_noalloc.restype = ctypes.c_int
        L.nat_bem_run_batch.argtypes = [ctypes.POINTER(Job), i32, ctypes.POINTER(Opts), i32, vp]
        L.nat_bem_run_batch.restype = ctypes.c_int
        L.nat_bem_run_batch_fused.argtypes = [ctypes.POINTER(Job), i32, ctypes.POINTER(Opts), i32, i32, vp]
        L.nat_bem_run_batch_fused.restype = ctypes.c_int
        L.nat_bem_server_create.argtypes = [i64, ctypes.POINTER(Opts), i32, ctypes.POINTER(vp)]
        L.nat_bem_server_create.restype = ctypes.c_int
        L.nat_bem_submit.argtypes = [vp, ctypes.POINTER(Job), ctypes.POINTER(i64)]
        L.nat_bem_submit.restype = ctypes.c_int
        L.nat_bem_wait.argtypes = [vp, i64, i32, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.nat_bem_wait.restype = ctypes.c_int
        L.nat_bem_server_reserved.argtypes = [vp]
        L.nat_bem_server_reserved.restype = i64
        L.nat_bem_server_destroy.argtypes = [vp]
        L.nat_bem_server_destroy.restype = None
        L.nat_bem_selftest_bounded_wait.argtypes = [i32, vp]
        L.nat_bem_selftest_bounded_wait.restype = ctypes.c_int
        L.nat_bem_op_apply.argtypes = [vp, i32, i32, vp, i32, vp, vp]
        L.nat_bem_op_apply.restype = ctypes.c_int
        L.nat_bem_op_rows.argtypes = [vp, i32, i64, i64, vp, vp]
        L.nat_bem_op_rows.restype = ctypes.c_int
        L.nat_bem_op_size.argtypes = [vp]
        L.nat_bem_op_size.restype = i64
        L.nat_bem_required_bytes.argtypes = [i64, i32, ctypes.POINTER(Opts)]
        L.nat_bem_required_bytes.restype = i64
        L.nat_bem_destroy.argtypes = [vp]
        L.nat_bem_destroy.restype = None
        L.nat_bem_last_error.argtypes = []
        L.nat_bem_last_error.restype = ctypes.c_char_p
        L.nat_bem_trace_enable.argtypes = [i32]
        L.nat_bem_trace_enable.restype = None
        L.nat_bem_trace_select.argtypes = [ctypes.c_char_p]
        L.nat_bem_trace_select.restype = None
        L.nat_bem_trace_reset.argtypes = []
        L.nat_bem_trace_reset.restype = None
        L.nat_bem_trace_launches.argtypes = []
        L.nat_bem_trace_launches.restype = i64
        L.nat_bem_trace_kernel.argtypes = [ctypes.c_char_p, ctypes.POINTER(d), ctypes.POINTER(i64)]
        L.nat_bem_trace_kernel.restype = ctypes.c_int
        L.nat_bem_assemble_galerkin.argtypes = [vp, i64, vp, i64, d, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
        L.nat_bem_assemble_galerkin.restype = ctypes.c_int
        L.nat_bem_op_neumann_size.argtypes = [vp]
        L.nat_bem_op_neumann_size.restype = i64
        L.nat_bem_trace_durations.argtypes = [ctypes.c_char_p, vp, i64, ctypes.POINTER(i64)]
        L.nat_bem_trace_durations.restype = ctypes.c_int
        L.nat_bem_gemv_variant.argtypes = [i64]
        L.nat_bem_gemv_variant.restype = i32
        L.nat_field_create.argtypes = [i32, i32, i32, vp, vp, vp, vp, ctypes.POINTER(vp)]
        L.nat_field_create.restype = ctypes.c_int
        L.nat_field_forward.argtypes = [vp, vp, i64, vp, vp]
        L.nat_field_forward.restype = ctypes.c_int
        L.nat_field_destroy.argtypes = [vp]
        L.nat_field_destroy.restype = None
        _lib = L
    return _lib


def _check(status: int):
    if status != NAT_BEM_OK:
        raise NatBemError(status, lib().nat_bem_last_error().decode())


def nat_bem_opts_default(**overrides) -> Opts:
    o = Opts()
    lib().nat_bem_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


# ------------------------------------------------------------------ array marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream_of(x, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if _is_torch(x) and x.is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return ctypes.c_void_p(0)


def _ptr(x, dtype, shape_check=None):
    """(pointer, keep-alive) for a numpy array or torch tensor of the given dtype."""
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.complex64: torch.complex64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"expected a contiguous torch tensor of {want}")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.asarray(x)
    if dtype is np.complex64:
        a = np.asfortranarray(a.astype(np.complex64, copy=False))
    else:
        a = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), a


def _nrhs_of(x, n):
    shape = tuple(x.shape)
    if _is_torch(x):
        if len(shape) == 1:
            return 1
        if shape[1] != n:
            raise ValueError(f"torch complex data must be (nrhs, {n})")
        return shape[0]
    if len(shape) == 1:
        return 1
    if shape[0] != n:
        raise ValueError(f"numpy complex data must be ({n}, nrhs)")
    return shape[1]


# ------------------------------------------------------------------------ operations
def nat_bem_assemble(V, F, k: float, opts: Opts | None = None, stream=None) -> ctypes.c_void_p:
    """Assemble L and R on the device; returns the opaque op handle."""
    pv, kv = _ptr(V, np.float64)
    pt, kt = _ptr(F, np.int32)
    nv, nt = int(V.shape[0]), int(F.shape[0])
    op = ctypes.c_void_p()
    st = lib().nat_bem_assemble(pv, nv, pt, nt, float(k), ctypes.byref(opts) if opts else None,
                                _stream_of(V, stream), ctypes.byref(op))
    del kv, kt
    _check(st)
    return op


def nat_bem_assemble_galerkin(V, F, k: float, opts: Opts | None = None, stream=None) -> ctypes.c_void_p:
    """Galerkin op (P1 pressure at the vertices, P0 Neumann data per triangle)."""
    pv, kv = _ptr(V, np.float64)
    pt, kt = _ptr(F, np.int32)
    nv, nt = int(V.shape[0]), int(F.shape[0])
    op = ctypes.c_void_p()
    st = lib().nat_bem_assemble_galerkin(pv, nv, pt, nt, float(k), ctypes.byref(opts) if opts else None,
                                         _stream_of(V, stream), ctypes.byref(op))
    del kv, kt
    _check(st)
    return op


def nat_bem_op_neumann_size(op) -> int:
    return int(lib().nat_bem_op_neumann_size(op))


def nat_bem_assemble_mc(Y, N, area: float, k: float, opts: Opts | None = None, stream=None) -> ctypes.c_void_p:
    """Monte-Carlo op from surface samples Y (m x 3), unit outward normals N (m x 3) and the
    total surface area; returns the opaque op handle."""
    py, ky = _ptr(Y, np.float64)
    pn, kn = _ptr(N, np.float64)
    m = int(Y.shape[0])
    if int(N.shape[0]) != m:
        raise ValueError("Y and N must have the same number of samples")
    op = ctypes.c_void_p()
    st = lib().nat_bem_assemble_mc(py, pn, m, float(area), float(k), ctypes.byref(opts) if opts else None,
                                   _stream_of(Y, stream), ctypes.byref(op))
    del ky, kn
    _check(st)
    return op


def nat_bem_poisson_sample(V, F, u, radius: float, cap: int | None = None, stream=None):
    """Poisson-disk samples of the mesh (V, F) from the draws u (m x 3 in [0, 1)) at minimum
    distance `radius`: (indices of the accepted draws, positions, unit normals), in increasing
    index. Outputs are numpy arrays, or torch tensors on V's device when V is a torch tensor."""
    pv, kv = _ptr(V, np.float64)
    pt, kt = _ptr(F, np.int32)
    pu, ku = _ptr(u, np.float64)
    m = int(u.shape[0])
    cap = m if cap is None else int(cap)
    idx = np.zeros(max(cap, 1), np.int64)
    if _is_torch(V):
        import torch
        pts = torch.empty((max(cap, 1), 3), dtype=torch.float64, device=V.device)
        nrm = torch.empty_like(pts)
        pp, pn = ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(nrm.data_ptr())
    else:
        pts = np.zeros((max(cap, 1), 3))
        nrm = np.zeros((max(cap, 1), 3))
        pp, pn = ctypes.c_void_p(pts.ctypes.data), ctypes.c_void_p(nrm.ctypes.data)
    count = ctypes.c_int64(0)
    st = lib().nat_bem_poisson_sample(pv, int(V.shape[0]), pt, int(F.shape[0]), float(radius), pu, m, cap,
                                      ctypes.c_void_p(idx.ctypes.data), pp, pn, ctypes.byref(count),
                                      _stream_of(V, stream))
    del kv, kt, ku
    _check(st)
    c = int(count.value)
    return idx[:c], pts[:c], nrm[:c]


def nat_bem_reassemble(op, k: float, stream=None, like=None):
    """Re-assemble an op at wavenumber k (same mesh, memory and workspace)."""
    _check(lib().nat_bem_reassemble(op, float(k), _stream_of(like, stream)))


def nat_bem_solve(op, neumann, out=None, stream=None, check=True):
    """Solve L p = R g. Returns (p, SolveInfo, status)."""
    n = int(lib().nat_bem_op_size(op))
    nrhs = _nrhs_of(neumann, int(lib().nat_bem_op_neumann_size(op)))
    pg, kg = _ptr(neumann, np.complex64)
    if out is None:
        if _is_torch(neumann):
            import torch
            shape = (nrhs, n) if neumann.dim() == 2 else (n,)
            out = torch.empty(shape, dtype=torch.complex64, device=neumann.device)
        else:
            out = np.zeros((n, nrhs) if np.ndim(neumann) == 2 else (n,), dtype=np.complex64, order="F")
    po, ko = _ptr(out, np.complex64)
    info = SolveInfo()
    st = lib().nat_bem_solve(op, pg, nrhs, po, ctypes.byref(info), _stream_of(neumann, stream))
    if check and st not in (NAT_BEM_OK, NAT_BEM_ENOCONV):
        _check(st)
    if not _is_torch(out) and ko is not out:
        out[...] = ko
    return out, info, st


def nat_bem_eval(op, points, p, neumann, out=None, stream=None):
    """Field at points (m, 3) for the surface data p and neumann."""
    n = int(lib().nat_bem_op_size(op))
    nrhs = _nrhs_of(p, n)
    m = int(points.shape[0])
    pp, kp = _ptr(points, np.float64)
    pd, kd = _ptr(p, np.complex64)
    pg, kg = _ptr(neumann, np.complex64)
    if out is None:
        if _is_torch(p):
            import torch
            out = torch.empty((nrhs, m) if p.dim() == 2 else (m,), dtype=torch.complex64, device=p.device)
        else:
            out = np.zeros((m, nrhs) if np.ndim(p) == 2 else (m,), dtype=np.complex64, order="F")
    po, ko = _ptr(out, np.complex64)
    _check(lib().nat_bem_eval(op, pp, m, pd, pg, nrhs, po, _stream_of(p, stream)))
    if not _is_torch(out) and ko is not out:
        out[...] = ko
    return out


def nat_bem_far_field(op, dirs, p, neumann, out=None, stream=None):
    """Far-field pattern F(d) = lim r e^{-ikr} p(r d) at unit directions (nd, 3)."""
    n = int(lib().nat_bem_op_size(op))
    nrhs = _nrhs_of(p, n)
    nd = int(dirs.shape[0])
    pdir, kdir = _ptr(dirs, np.float64)
    pd, kp = _ptr(p, np.complex64)
    pg, kg = _ptr(neumann, np.complex64)
    if out is None:
        if _is_torch(p):
            import torch
            out = torch.empty((nrhs, nd) if p.dim() == 2 else (nd,), dtype=torch.complex64, device=p.device)
        else:
            out = np.zeros((nd, nrhs) if np.ndim(p) == 2 else (nd,), dtype=np.complex64, order="F")
    po, ko = _ptr(out, np.complex64)
    _check(lib().nat_bem_far_field(op, pdir, nd, pd, pg, nrhs, po, _stream_of(p, stream)))
    if not _is_torch(out) and ko is not out:
        out[...] = ko
    return out


def nat_bem_sample_field(op, u, center, r_lo, r_hi, p, neumann, stream=None):
    """Training samples (paper Sec. 3.4) from draws u (n, 3) in [0, 1): returns
    (coords (n, 3) = theta, phi, r; amplitudes |p| (n,) or (n, nrhs)), numpy or torch like u."""
    n_el = int(lib().nat_bem_op_size(op))
    nrhs = _nrhs_of(p, n_el)
    n = int(u.shape[0])
    pu, ku = _ptr(u, np.float64)
    pd, kp = _ptr(p, np.complex64)
    pg, kg = _ptr(neumann, np.complex64)
    c = np.ascontiguousarray(center, dtype=np.float64).reshape(3)
    if _is_torch(u):
        import torch
        coords = torch.empty((n, 3), dtype=torch.float64, device=u.device)
        amp = torch.empty((nrhs, n) if nrhs > 1 else (n,), dtype=torch.float32, device=u.device)
        pc, pa = ctypes.c_void_p(coords.data_ptr()), ctypes.c_void_p(amp.data_ptr())
    else:
        coords = np.zeros((n, 3), dtype=np.float64)
        amp = np.zeros((n, nrhs) if nrhs > 1 else (n,), dtype=np.float32, order="F")
        pc, pa = ctypes.c_void_p(coords.ctypes.data), ctypes.c_void_p(amp.ctypes.data)
    _check(lib().nat_bem_sample_field(op, pu, n, ctypes.c_void_p(c.ctypes.data), float(r_lo), float(r_hi),
                                      pd, pg, nrhs, pc, pa, _stream_of(u, stream)))
    return coords, amp


def nat_bem_eval_noalloc(op, points, p, neumann, out, stream=None) -> int:
    """nat_bem_eval without device allocation: all arrays must be CUDA torch tensors and
    `out` is written in place ((nrhs, m) or (m,) complex64). Returns the status code.
    The C call cannot see array sizes, so the shapes and devices are checked here first
    (ValueError), before anything is launched."""
    for name, t in (("points", points), ("p", p), ("neumann", neumann), ("out", out)):
        if not _is_torch(t) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA torch tensor")
    if len({t.device for t in (points, p, neumann, out)}) != 1:
        raise ValueError("points, p, neumann and out must be on one CUDA device")
    m = int(points.shape[0])
    n = int(lib().nat_bem_op_size(op))
    if points.dim() != 2 or int(points.shape[1]) != 3:
        raise ValueError("points must be (m, 3)")
    nrhs = _nrhs_of(p, n)
    if p.dim() == 2 and int(p.shape[1]) != n or p.dim() == 1 and int(p.shape[0]) != n:
        raise ValueError(f"p must be ({n},) or (nrhs, {n})")
    if tuple(neumann.shape) != tuple(p.shape):
        raise ValueError("neumann must have the shape of p")
    if int(out.numel()) != nrhs * m:
        raise ValueError(f"out must hold nrhs * m = {nrhs * m} values, has {int(out.numel())}")
    pp, _ = _ptr(points, np.float64)
    pd, _ = _ptr(p, np.complex64)
    pg, _ = _ptr(neumann, np.complex64)
    po, _ = _ptr(out, np.complex64)
    return int(lib().nat_bem_eval_noalloc(op, pp, m, pd, pg, nrhs, po, _stream_of(p, stream)))


def nat_bem_run_batch(jobs, opts: Opts | None = None, concurrency: int = 3, stream=None):
    """Run a list of solves. Each job is a dict with V, F, k, neumann and optionally points;
    arrays are numpy (host) or CUDA torch tensors. Returns (status, per-job list of
    (p, field, SolveInfo, status))."""
    keep = []
    arr = (Job * len(jobs))()
    outs = []
    for i, jd in enumerate(jobs):
        V, F, g = jd["V"], jd["F"], jd["neumann"]
        pts = jd.get("points")
        n = int(F.shape[0])
        nrhs = _nrhs_of(g, n)
        pv, kv = _ptr(V, np.float64)
        pt, kt = _ptr(F, np.int32)
        pg, kg = _ptr(g, np.complex64)
        torch_out = _is_torch(g)
        m = 0 if pts is None else int(pts.shape[0])
        if torch_out:
            import torch
            p = torch.empty(tuple(g.shape), dtype=torch.complex64, device=g.device)
            f = torch.empty((nrhs, m) if g.dim() == 2 else (m,), dtype=torch.complex64, device=g.device)
        else:
            p = np.zeros((n, nrhs) if np.ndim(g) == 2 else (n,), dtype=np.complex64, order="F")
            f = np.zeros((m, nrhs) if np.ndim(g) == 2 else (m,), dtype=np.complex64, order="F")
        pp, kp = _ptr(p, np.complex64)
        pf, kf = _ptr(f, np.complex64)
        if pts is not None:
            ppt, kpt = _ptr(pts, np.float64)
        else:
            ppt, kpt = ctypes.c_void_p(0), None
        keep += [kv, kt, kg, kp, kf, kpt]
        arr[i] = Job(pv, int(V.shape[0]), pt, n, float(jd["k"]), pg, nrhs, ppt, m, pp, pf,
                     SolveInfo(), 0, 0.0)
        outs.append((p, f))
    st = lib().nat_bem_run_batch(arr, len(jobs), ctypes.byref(opts) if opts else None,
                                 int(concurrency), _stream_of(jobs[0]["V"] if jobs else None, stream))
    res = [(outs[i][0], outs[i][1], arr[i].info, arr[i].status, arr[i].device_ms)
           for i in range(len(jobs))]
    del keep
    return st, res


def nat_bem_run_batch_fused(jobs, opts: Opts | None = None, max_batch: int = 64, concurrency: int = 4,
                            stream=None):
    """Fused batch: meshes bucketed by size, each bucket solved in lockstep as one padded system
    of independent operators (see include/nat_bem.h). Job dicts and results as for
    nat_bem_run_batch."""
    keep, outs = [], []
    arr = (Job * len(jobs))()
    for i, jd in enumerate(jobs):
        job, p, f, k = _make_job(jd)
        arr[i] = job
        outs.append((p, f))
        keep.append(k)
    st = lib().nat_bem_run_batch_fused(arr, len(jobs), ctypes.byref(opts) if opts else None, int(max_batch),
                                       int(concurrency), _stream_of(jobs[0]["V"] if jobs else None, stream))
    res = [(outs[i][0], outs[i][1], arr[i].info, arr[i].status, arr[i].device_ms) for i in range(len(jobs))]
    del keep
    return st, res


def nat_bem_op_apply(op, which: int, engine: int, X, stream=None):
    """Y = M X (M = L for which 0, R for 1) with the chosen product engine."""
    n = int(lib().nat_bem_op_size(op))
    cols = int(lib().nat_bem_op_neumann_size(op)) if which == 1 else n
    nrhs = _nrhs_of(X, cols)
    px, kx = _ptr(X, np.complex64)
    if _is_torch(X):
        import torch
        Y = torch.empty((nrhs, n) if X.dim() == 2 else (n,), dtype=torch.complex64, device=X.device)
    else:
        Y = np.zeros((n, nrhs) if np.ndim(X) == 2 else (n,), dtype=np.complex64, order="F")
    py, ky = _ptr(Y, np.complex64)
    _check(lib().nat_bem_op_apply(op, int(which), int(engine), px, nrhs, py, _stream_of(X, stream)))
    return Y


def _make_job(jd):
    """A Job struct for a job dict, with its output arrays and the references that keep the
    inputs alive (see nat_bem_run_batch for the dict keys)."""
    V, F, g = jd["V"], jd["F"], jd["neumann"]
    pts = jd.get("points")
    n = int(F.shape[0])
    nrhs = _nrhs_of(g, n)
    pv, kv = _ptr(V, np.float64)
    pt, kt = _ptr(F, np.int32)
    pg, kg = _ptr(g, np.complex64)
    m = 0 if pts is None else int(pts.shape[0])
    if _is_torch(g):
        import torch
        p = torch.empty(tuple(g.shape), dtype=torch.complex64, device=g.device)
        f = torch.empty((nrhs, m) if g.dim() == 2 else (m,), dtype=torch.complex64, device=g.device)
    else:
        p = np.zeros((n, nrhs) if np.ndim(g) == 2 else (n,), dtype=np.complex64, order="F")
        f = np.zeros((m, nrhs) if np.ndim(g) == 2 else (m,), dtype=np.complex64, order="F")
    pp, kp = _ptr(p, np.complex64)
    pf, kf = _ptr(f, np.complex64)
    ppt, kpt = _ptr(pts, np.float64) if pts is not None else (ctypes.c_void_p(0), None)
    job = Job(pv, int(V.shape[0]), pt, n, float(jd["k"]), pg, nrhs, ppt, m, pp, pf, SolveInfo(), 0, 0.0)
    return job, p, f, [kv, kt, kg, kp, kf, kpt]


class Server:
    """Serving loop of the library (nat_bem_server_*): submit job dicts, wait for tickets."""

    def __init__(self, budget_bytes: int, opts: Opts | None = None, slots: int = 4):
        self.handle = ctypes.c_void_p()
        _check(lib().nat_bem_server_create(int(budget_bytes), ctypes.byref(opts) if opts else None,
                                           int(slots), ctypes.byref(self.handle)))
        self._live = {}

    def submit(self, jd) -> int:
        job, p, f, keep = _make_job(jd)
        t = ctypes.c_int64(0)
        _check(lib().nat_bem_submit(self.handle, ctypes.byref(job), ctypes.byref(t)))
        self._live[t.value] = (job, p, f, keep)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(status, p, field, SolveInfo, device_ms, queue_ms, total_ms); status ETIMEOUT leaves
        the request queued."""
        q, tot = ctypes.c_double(0.0), ctypes.c_double(0.0)
        st = lib().nat_bem_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(q), ctypes.byref(tot))
        if st == NAT_BEM_ETIMEOUT:
            return st, None, None, None, None, None, None
        job, p, f, keep = self._live.pop(ticket)
        return st, p, f, job.info, job.device_ms, q.value, tot.value

    def reserved(self) -> int:
        return int(lib().nat_bem_server_reserved(self.handle))

    def close(self):
        if self.handle:
            lib().nat_bem_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def nat_bem_selftest_bounded_wait(timeout_ms: int = 50, stream=None) -> int:
    return int(lib().nat_bem_selftest_bounded_wait(int(timeout_ms), _stream_of(None, stream)))


def nat_bem_op_rows(op, which: int, row0: int, nrows: int, stream=None) -> np.ndarray:
    n = int(lib().nat_bem_op_size(op))
    cols = int(lib().nat_bem_op_neumann_size(op)) if which == 1 else n
    out = np.zeros((nrows, cols), dtype=np.complex64)
    _check(lib().nat_bem_op_rows(op, int(which), int(row0), int(nrows),
                                 ctypes.c_void_p(out.ctypes.data), _stream_of(None, stream)))
    return out


def nat_bem_required_bytes(nt: int, nrhs: int, opts: Opts | None = None) -> int:
    return int(lib().nat_bem_required_bytes(int(nt), int(nrhs), ctypes.byref(opts) if opts else None))


def nat_bem_destroy(op):
    if op:
        lib().nat_bem_destroy(op)


def nat_bem_last_error() -> str:
    return lib().nat_bem_last_error().decode()


def nat_bem_trace_enable(enable: bool = True):
    lib().nat_bem_trace_enable(1 if enable else 0)


def nat_bem_trace_select(names: str = ""):
    lib().nat_bem_trace_select(names.encode())


def nat_bem_trace_reset():
    lib().nat_bem_trace_reset()


def nat_bem_trace_launches() -> int:
    return int(lib().nat_bem_trace_launches())


def nat_bem_trace_durations(name: str) -> np.ndarray:
    """Per-launch device times (ms) of the traced kernels named exactly `name`."""
    c = ctypes.c_int64(0)
    _check(lib().nat_bem_trace_durations(name.encode(), None, 0, ctypes.byref(c)))
    out = np.zeros(c.value, dtype=np.float32)
    if c.value:
        _check(lib().nat_bem_trace_durations(name.encode(), ctypes.c_void_p(out.ctypes.data), c.value,
                                             ctypes.byref(c)))
    return out


def nat_bem_trace_kernel(name: str = ""):
    """(total device ms, launches) of the traced kernels whose name contains `name`."""
    t, c = ctypes.c_double(0.0), ctypes.c_int64(0)
    _check(lib().nat_bem_trace_kernel(name.encode(), ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


@dataclass
class Operator:
    """Owning wrapper of a nat_bem_op handle."""
    handle: ctypes.c_void_p
    n: int
    k: float

    @classmethod
    def assemble(cls, V, F, k, opts=None, stream=None):
        return cls(nat_bem_assemble(V, F, k, opts, stream), int(F.shape[0]), float(k))

    @classmethod
    def assemble_galerkin(cls, V, F, k, opts=None, stream=None):
        return cls(nat_bem_assemble_galerkin(V, F, k, opts, stream), int(V.shape[0]), float(k))

    @classmethod
    def assemble_mc(cls, Y, N, area, k, opts=None, stream=None):
        return cls(nat_bem_assemble_mc(Y, N, area, k, opts, stream), int(Y.shape[0]), float(k))

    def reassemble(self, k, stream=None, like=None):
        nat_bem_reassemble(self.handle, k, stream, like)
        self.k = float(k)

    def solve(self, neumann, out=None, stream=None, check=True):
        return nat_bem_solve(self.handle, neumann, out, stream, check)

    def evaluate(self, points, p, neumann, out=None, stream=None):
        return nat_bem_eval(self.handle, points, p, neumann, out, stream)

    def far_field(self, dirs, p, neumann, out=None, stream=None):
        return nat_bem_far_field(self.handle, dirs, p, neumann, out, stream)

    def sample_field(self, u, center, r_lo, r_hi, p, neumann, stream=None):
        return nat_bem_sample_field(self.handle, u, center, r_lo, r_hi, p, neumann, stream)

    def apply(self, which, engine, X):
        return nat_bem_op_apply(self.handle, which, engine, X)

    def rows(self, which, row0, nrows):
        return nat_bem_op_rows(self.handle, which, row0, nrows)

    def close(self):
        if self.handle:
            nat_bem_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nat_bem_gemv_variant(nt: int) -> int:
    """The GEMV variant the autotuner chose for nt elements on the current device (-1: not yet)."""
    return int(lib().nat_bem_gemv_variant(int(nt)))


# ------------------------------------------------------------- neural acoustic transfer field
def _f32_ptr(x, width=None):
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError("expected a contiguous float32 torch tensor")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=np.float32)
    return ctypes.c_void_p(a.ctypes.data), a


def nat_field_create(n_cond: int, n_out: int, table_log2: int, tables, weights, biases,
                     stream=None) -> ctypes.c_void_p:
    """tables: float32 rows of the four levels back to back (rows x 4); weights: float32, four
    128 x 128 layers then n_out x 128, concatenated (row-major [out][in]); biases: float32.
    The library rounds the tables to FP16 and the weights to BF16 itself."""
    pt, kt = _f32_ptr(tables)
    pw, kw = _f32_ptr(weights)
    pb, kb = _f32_ptr(biases)
    h = ctypes.c_void_p()
    _check(lib().nat_field_create(int(n_cond), int(n_out), int(table_log2), pt, pw, pb,
                                  _stream_of(None, stream), ctypes.byref(h)))
    return h


def nat_field_forward(field, x, n_out: int, out=None, stream=None):
    """x: (n, 4 + n_cond) float32 (numpy or torch, host or CUDA); returns (n, n_out) float32 of
    the same kind (or writes `out`)."""
    n = int(x.shape[0])
    if out is None:
        if _is_torch(x):
            import torch
            out = torch.empty((n, n_out), dtype=torch.float32, device=x.device)
        else:
            out = np.empty((n, n_out), dtype=np.float32)
    px, kx = _f32_ptr(x)
    if _is_torch(out):
        po = ctypes.c_void_p(out.data_ptr())
    else:
        if out.dtype != np.float32 or not out.flags.c_contiguous:
            raise TypeError("out must be a C-contiguous float32 array")
        po = ctypes.c_void_p(out.ctypes.data)
    _check(lib().nat_field_forward(field, px, n, po, _stream_of(x, stream)))
    return out


def nat_field_destroy(field):
    if field:
        lib().nat_field_destroy(field)


class NatField:
    """Owning wrapper of a nat_field handle: float32 tables (rows x 4, levels back to back),
    weights (concatenated row-major layers) and biases."""

    def __init__(self, n_cond, n_out, table_log2, tables, weights, biases, stream=None):
        self.n_cond, self.n_out = int(n_cond), int(n_out)
        self.handle = nat_field_create(n_cond, n_out, table_log2, tables, weights, biases, stream)

    @classmethod
    def from_params(cls, params, stream=None):
        """From a dict with n_cond, n_out, table_log2 and lists of tables, weights, biases."""
        cat = lambda xs: np.concatenate([np.asarray(a, dtype=np.float32).ravel() for a in xs])
        return cls(params["n_cond"], params["n_out"], params["table_log2"], cat(params["tables"]),
                   cat(params["weights"]), cat(params["biases"]), stream)

    def forward(self, x, out=None, stream=None):
        if int(x.shape[1]) != 4 + self.n_cond:
            raise ValueError(f"inputs must be (n, {4 + self.n_cond})")
        return nat_field_forward(self.handle, x, self.n_out, out, stream)

    def close(self):
        if self.handle:
            nat_field_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

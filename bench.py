"""Benchmark of the GB300 Burton-Miller BEM path: BEM solves per second.

Workload (the interior-point-source case): a perturbed ellipsoid (radii 1, 0.8, 0.6, l <= 6
radial harmonics of std 0.05) meshed with 10240 triangles, Neumann data of a monopole at the
origin, 64 wavenumbers log-uniform in ka in [0.5, 20], 1024 field points at radius 4. One step
is the whole path for all 64 wavenumbers: per wavenumber, assemble L and R on the device,
solve L p = R g by GMRES to a relative residual of 1e-6, and evaluate the field at the 1024
points. A "solve" is one (mesh, k, Neumann data) through all three stages. The solves run
through the library's batch driver (nat_bem_run_batch) with a few in flight at once; each
worker checks the mesh and builds its geometry once, then re-assembles per wavenumber.

Prints one JSON line. `value` is solves/s of the mixed-precision path (inner GMRES on the BF16
copy of L, refinement against the FP32 operator; --prec selects) with inputs resident in HBM;
`plain_fp32` is the same workload through the plain FP32 path, measured in the same run; `e2e`
is the metric through the public API with host (numpy) buffers, host-device copies included.
`--impl reference` times the FP64 CPU oracle on the same workload instead.

Multi-GPU: independent solves shard with no exchange (replicas only): each rank runs the
workload on its own GPU and `value` is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "BEM solves/s at \u22641e-4 rel err vs FP64 oracle, mixed vs plain FP32; p50/p99 ms"
UNIT = "solves/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every `interval_ms` during the timed
    region. A reader thread timestamps each sample; the summary keeps those taken inside the
    context (nvidia-smi takes a moment to start, so it is started `lead_s` before)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, interval_ms: int = 200, lead_s: float = 0.5):
        self.index = index
        self.interval_ms = interval_ms
        self.lead_s = lead_s
        self.proc = None
        self.samples = []

    def _read(self):
        for ln in self.proc.stdout:
            if ln.strip():
                self.samples.append((time.monotonic(), ln))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            time.sleep(self.lead_s)
        except OSError:
            self.proc = None
        self.t0 = time.monotonic()
        return self

    def __exit__(self, *exc):
        self.t1 = time.monotonic()
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            self.reader.join(timeout=5)
            inside = [ln for t, ln in self.samples if self.t0 <= t <= self.t1 + 0.05]
            self.lines = inside

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(n_k: int, n_tri: int = 10240):
    return S.interior_source(n_k=n_k, n_tri=n_tri)


# ------------------------------------------------------------------------------ GPU arm
KERNELS = ("assemble_regular", "assemble_near", "assemble_self", "geometry", "gemv_rhs", "gemv_resid", "gemv_bf16",
           "gemv_fp16", "copy_fp16",
           "gmres_start", "gmres_arnoldi", "gmres_dots", "gmres_update", "gmres_finish", "gmres_lsq",
           "gmres_xupdate", "eval_reduce", "ir_residual", "pad_copy", "cgemm_fp32", "tc_gemm", "tc_pack",
           "tc_reduce")


def _working_launches(d):
    """(total ms, launches) of the launches that streamed the operator. A GMRES chunk captured
    as 16 or 8 iterations keeps launching after its RHS converged; those matvecs exit at once
    (a few microseconds against tens), so launches under a quarter of the 90th-percentile time
    are set aside. Returns (ms, working, skipped)."""
    d = np.asarray(d, dtype=np.float64)
    if d.size == 0:
        return 0.0, 0, 0
    keep = d >= 0.25 * np.percentile(d, 90)
    return float(d[keep].sum()), int(keep.sum()), int((~keep).sum())


def _kernel_table(nb):
    kern = {name: nb.nat_bem_trace_kernel(name) for name in KERNELS}
    g = nb.nat_bem_trace_kernel("gemv")
    kern["gemv"] = tuple(a - b - c - d - e for a, b, c, d, e in
                         zip(g, kern["gemv_rhs"], kern["gemv_resid"], kern["gemv_bf16"], kern["gemv_fp16"]))
    ev = nb.nat_bem_trace_kernel("eval")
    kern["eval"] = (ev[0] - kern["eval_reduce"][0], ev[1] - kern["eval_reduce"][1])
    return kern


def check_indices(ks):
    """The wavenumbers whose results the bench checks against the oracle: the lowest, the
    median and the highest of the workload."""
    order = np.argsort(np.asarray(ks))
    return sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1])})


def run_gpu(args, rank: int, world: int, prec_name: str, full: bool = True):
    """One timed measurement of the interior workload at precision `prec_name`; with `full`
    also the traced per-kernel step and the end-to-end pass. The surface pressure and field of
    the wavenumbers of check_indices (first timed step) come back for the oracle check."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        nb_build.build()
    if world > 1:
        torch.distributed.barrier()
    prob = workload(args.n_k, args.n_tri)
    n = prob.F.shape[0]
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32, "fp16": nb.PREC_MIXED_FP16}[prec_name]
    opts = nb.nat_bem_opts_default(prec=prec)
    if args.inner_tol is not None:
        opts.inner_tol = args.inner_tol
    Vd = torch.from_numpy(prob.V).to(dev)
    Fd = torch.from_numpy(prob.F).to(dev)
    Gd = [torch.from_numpy(np.ascontiguousarray(g[:, 0]).astype(np.complex64)).to(dev) for g in prob.neumann]
    Pd = torch.from_numpy(prob.points).to(dev)
    jobs = [dict(V=Vd, F=Fd, k=float(k), neumann=Gd[i], points=Pd) for i, k in enumerate(prob.ks)]
    stream = torch.cuda.current_stream(dev)

    def step(conc=None):
        if args.batch_mode == "fused" and conc is None:
            st, res = nb.nat_bem_run_batch_fused(jobs, opts, max_batch=args.max_batch,
                                                 concurrency=args.fused_workers)
        else:
            st, res = nb.nat_bem_run_batch(jobs, opts, concurrency=conc or args.concurrency)
        if st not in (nb.NAT_BEM_OK, nb.NAT_BEM_ENOCONV):
            raise RuntimeError(nb.nat_bem_last_error())
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    nb.nat_bem_trace_enable(False)
    launches0 = nb.nat_bem_trace_launches()
    results = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            results.append(step())
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    ms_total = t0.elapsed_time(t1)
    launches = nb.nat_bem_trace_launches() - launches0
    lats = sorted(r[4] for res in results for r in res)
    iters = [r[2].iterations for res in results for r in res]
    statuses = [r[3] for res in results for r in res]
    summary = dict(ms_total=ms_total, launches=launches, lat=lats, iters=iters, clocks=clk.summary(), n=n,
                   max_rel_res=max(r[2].rel_residual for res in results for r in res),
                   n_enoconv=sum(1 for s_ in statuses if s_ != nb.NAT_BEM_OK),
                   refinements=max(r[2].refinements for res in results for r in res), prob=prob)
    summary["checks"] = {i: (results[0][i][0].cpu().numpy(), results[0][i][1].cpu().numpy())
                         for i in check_indices(prob.ks)}
    if not full:
        return summary
    # One more (untimed) step, one solve at a time, with every kernel bracketed by CUDA events
    # on its stream: the per-kernel table and the dominant kernel's roofline (each kernel runs
    # without other solves sharing HBM; per-launch events switch the graph replay off).
    nb.nat_bem_trace_reset()
    nb.nat_bem_trace_select("")
    nb.nat_bem_trace_enable(True)
    step(conc=1)
    torch.cuda.synchronize()
    nb.nat_bem_trace_enable(False)
    kern = _kernel_table(nb)
    working = {nm: _working_launches(nb.nat_bem_trace_durations(nm)) for nm in ("gemv", "gemv_bf16", "gemv_fp16")}
    summary["gemv_variant"] = nb.nat_bem_gemv_variant(n)
    nb.nat_bem_trace_reset()
    first = results[0][0]
    out = dict(summary, kern=kern, measured=kern, working=working, p0=first[0].cpu().numpy(),
               f0=first[1].cpu().numpy())

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e:
        Gh = [np.ascontiguousarray(g[:, 0]).astype(np.complex64) for g in prob.neumann]
        hjobs = [dict(V=prob.V, F=prob.F, k=float(k), neumann=Gh[i], points=prob.points)
                 for i, k in enumerate(prob.ks)]
        torch.cuda.synchronize()
        ta = time.perf_counter()
        st, res = nb.nat_bem_run_batch(hjobs, opts, concurrency=args.concurrency)
        torch.cuda.synchronize()
        tb = time.perf_counter()
        nk = len(prob.ks)
        # per job: mesh, Neumann data and points in (the Neumann data twice: solve and field),
        # surface pressure out and back in for the field, field out
        h2d = prob.V.nbytes + prob.F.nbytes + 2 * Gh[0].nbytes + prob.points.nbytes + res[0][0].nbytes
        d2h = res[0][0].nbytes + res[0][1].nbytes
        e2e = {"value": nk / (tb - ta), "unit": UNIT, "h2d_bytes_per_step": int(h2d * nk),
               "d2h_bytes_per_step": int(d2h * nk), "solves_per_step": nk}
    out["e2e"] = e2e
    return out


# ------------------------------------------------------------------------- other workloads
def _percentiles(xs):
    return {"p50": float(np.percentile(xs, 50)), "p99": float(np.percentile(xs, 99))}


def _sustained(n_req, last_arrival_s, served_s, p99_first, p99_last):
    """Whether a server kept up with a stream: completions >= 0.95 x the rate the stream
    actually offered (n_req over its last arrival time: a seeded Poisson stream's own mean
    rate, not the nominal one), and the queue did not grow along it (p99 latency of the last
    third of the requests <= 1.5 x that of the first third). Returns (offered, served, ok)."""
    offered = n_req / last_arrival_s
    served = n_req / served_s
    return offered, served, bool(served >= 0.95 * offered and p99_last <= 1.5 * p99_first)


def run_modal(args):
    """Multi-RHS modal transfer: one perturbed 20480-triangle icosphere (or a ring sphere of
    --n-tri triangles), --nrhs smooth real SH Neumann fields (l <= 8) shared by --n-k
    wavenumbers in ka [1, 15], 4096 shell points r in [2, 5]. One step: for each wavenumber,
    re-assemble, solve all right-hand sides in one block, evaluate the field. A solve is one
    (mesh, k, RHS)."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    nb_build.build()
    if args.n_tri == 20480:
        prob = S.modal_multirhs(nrhs=args.nrhs, n_k=args.n_k)
    else:
        Vs, F = S.ring_sphere(args.n_tri)
        V = S.perturbed_ellipsoid(Vs, 3000)
        prob = S.Problem("modal_multirhs", V, F, S.log_uniform(args.n_k, 1.0, 15.0, 3001),
                         [S.sh_neumann(V, F, args.nrhs, 3002)] * args.n_k, S.shell_points(4096, 2.0, 5.0, 3003))
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32, "fp16": nb.PREC_MIXED_FP16}[args.prec]
    opts = nb.nat_bem_opts_default(prec=prec)
    if args.inner_tol is not None:
        opts.inner_tol = args.inner_tol
    dev = torch.device("cuda", 0)
    Vd, Fd = torch.from_numpy(prob.V).to(dev), torch.from_numpy(prob.F).to(dev)
    G = torch.from_numpy(np.ascontiguousarray(prob.neumann[0].T).astype(np.complex64)).to(dev)
    Pd = torch.from_numpy(prob.points).to(dev)
    stream = torch.cuda.current_stream(dev)
    op = nb.Operator.assemble(Vd, Fd, float(prob.ks[0]), opts)
    infos = []

    def step(record=None):
        for k in prob.ks:
            op.reassemble(float(k), like=Vd)
            p, info, st = op.solve(G)
            f = op.evaluate(Pd, p, G)
            if record is not None:
                record.append((info.iterations, info.refinements, info.rel_residual, st))
        return p, f

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the tensor-core product's launches in one untimed traced step (CUDA events per launch)
    tc_name = {"bf16": "tc_gemm_bf16", "tf32": "tc_gemm_tf32", "fp16": "tc_gemm_fp16"}.get(args.prec)
    tc = None
    if tc_name:
        nb.nat_bem_trace_enable(True)
        nb.nat_bem_trace_select(tc_name)
        nb.nat_bem_trace_reset()
        step()
        torch.cuda.synchronize()
        tc = _working_launches(nb.nat_bem_trace_durations(tc_name))
        nb.nat_bem_trace_enable(False)
        nb.nat_bem_trace_reset()
    launches0 = nb.nat_bem_trace_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            p, f = step(infos)
        t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    launches = nb.nat_bem_trace_launches() - launches0
    n_solves = args.steps * len(prob.ks) * args.nrhs
    roof = None
    if tc and tc[1]:
        n = len(prob.F)
        ld = (n + 31) // 32 * 32
        ng = 2 * ((args.nrhs + 15) // 16 * 16)  # real columns of the packed right-hand sides
        per = tc[0] / tc[1] * 1e-3
        op_bytes = (8.0 if args.prec == "tf32" else 4.0) * n * ld
        flops = 2.0 * n * (2 * ld) * ng  # real GEMM n x 2ld times 2ld x ng
        peaks, peak_kind = _peaks()
        gbs = op_bytes / per / 1e9
        tfl = flops / per / 1e12
        tpeak = peaks["bf16_tflops"] * (0.5 if args.prec == "tf32" else 1.0)
        traffic = NCU_TRAFFIC_MODAL_20480.get(args.prec) if n == 20480 and args.nrhs == 64 else None
        roof = {"kernel": tc_name, "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "traffic": traffic, "launches": tc[1], "launches_exited_early": tc[2],
                "tensor_tflops": tfl, "tensor_peak": tpeak,
                "tensor_frac": tfl / tpeak,
                "note": "operator bytes per launch (the packed right-hand sides are small beside them); "
                        "64 flop per operator byte at 64 RHS is far below the tensor ridge, so HBM binds",
                "peak_source": f"{peak_kind} (hbm_gbs; bf16_tflops, TF32 at half the BF16 rate)"}
    # accuracy of the last wavenumber against the FP64 oracle on two right-hand sides
    acc = None
    if args.cpu and len(prob.F) <= 6000:
        import oracle
        L, R = oracle.assemble(prob.V, prob.F, float(prob.ks[-1]))
        pc = p.cpu().numpy()
        errs = []
        for c in (0, args.nrhs - 1):
            pref = np.linalg.solve(L, R @ prob.neumann[0][:, c])
            errs.append(float(np.linalg.norm(pc[c] - pref) / np.linalg.norm(pref)))
        acc = {"max_rel_err_vs_oracle": max(errs), "checked": "2 RHS of the last wavenumber"}
    op.close()
    return {"metric": METRIC, "value": n_solves / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "tf32": "tf32 tensor cores + f32 refinement", "bf16": "bf16 tensor cores + f32 refinement",
                      "fp16": "fp16 (row-scaled) tensor cores + f32 refinement"}[args.prec],
            "data": "synthetic",
            "config": {"workload": f"modal_multirhs_{len(prob.F)}tri_{args.nrhs}rhs_{len(prob.ks)}k",
                       "precision": args.prec, "field_points": 4096},
            "gmres": {"iterations_max": max(i[0] for i in infos), "refinements_max": max(i[1] for i in infos),
                      "max_rel_residual": max(i[2] for i in infos),
                      "not_converged": sum(1 for i in infos if i[3] != 0)},
            "gpu_launches": int(launches), "roofline": roof, "accuracy": acc, "clocks": clk.summary()}


# DRAM bytes (read + write) per launch of the BF16 tensor-core product on the 20480-triangle,
# 64-RHS modal operator, from one ncu capture (profiles/k_tc_gemm_modal_20480tri_64rhs.md,
# the mean of three launches).
NCU_TRAFFIC_MODAL_20480 = {"bf16": 1.7233e9 + 11.57e6}


def _pool(torch, dev, conc, make_op):
    """--concurrency workers over a list of wavenumbers: worker w owns an operator and a stream
    and takes wavenumbers w, w + nw, ... (the library's calls release the GIL and block only
    their own thread). Returns (streams, ops)."""
    streams = [torch.cuda.Stream(dev) for _ in range(conc)]
    ops = [make_op(st.cuda_stream) for st in streams]
    torch.cuda.synchronize()
    return streams, ops


def _pool_run(torch, streams, ops, n, body, nw=None):
    """body(op, stream handle, i) for i < n over the first nw workers; its results by i."""
    nw = len(ops) if nw is None else nw
    out = [None] * n

    def work(w):
        st = streams[w]
        with torch.cuda.stream(st):
            for i in range(w, n, nw):
                out[i] = body(ops[w], st.cuda_stream, i)

    if nw == 1:
        work(0)
    else:
        ths = [threading.Thread(target=work, args=(w,)) for w in range(nw)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    return out


def _pool_time(torch, stream, streams, fn):
    """Device milliseconds of fn() with the workers' streams bracketed by events on `stream`."""
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for st in streams:
        st.wait_event(t0)
    res = fn()
    for st in streams:
        e = torch.cuda.Event()
        e.record(st)
        stream.wait_event(e)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), res


def run_products(args):
    """The multi-RHS operator products alone (profiling and launch-shape sweeps): Y = L X for
    --nrhs seeded complex64 columns on a ring-sphere mesh of --n-tri triangles (default 20480),
    with the FP32 CUDA-core GEMM (--prec fp32) or the tensor-core product (bf16, tf32, fp16).
    --warmup products, then --steps products timed from the library's launch trace."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    nb_build.build()
    Vs, F = S.ring_sphere(args.n_tri)
    V = S.perturbed_ellipsoid(Vs, 3000)
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32,
            "fp16": nb.PREC_MIXED_FP16}[args.prec]
    engine = {"fp32": nb.ENGINE_FP32, "bf16": nb.ENGINE_BF16, "tf32": nb.ENGINE_TF32, "fp16": nb.ENGINE_FP16}[args.prec]
    rng = np.random.default_rng(3004)
    with nb.Operator.assemble(V, F, 4.0, nb.nat_bem_opts_default(prec=prec)) as op:
        n = op.n
        ld = (n + 31) // 32 * 32
        X = np.asfortranarray((rng.normal(size=(n, args.nrhs)) + 1j * rng.normal(size=(n, args.nrhs)))
                              .astype(np.complex64))
        for _ in range(args.warmup):
            op.apply(0, engine, X)
        torch.cuda.synchronize()
        nb.nat_bem_trace_enable(True)
        nb.nat_bem_trace_select("")
        nb.nat_bem_trace_reset()
        for _ in range(args.steps):
            op.apply(0, engine, X)
        torch.cuda.synchronize()
        # the FP32-accurate product runs on the split tensor-core kernel from 8 RHS (L only),
        # else on the CUDA-core GEMM
        names = ["tc_gemm_x6", "cgemm_fp32"] if args.prec == "fp32" else ["tc_gemm"]
        for name in names:
            t, c = nb.nat_bem_trace_kernel(name)
            if c > 0:
                break
        tr, cr = nb.nat_bem_trace_kernel("cgemm_reduce" if name == "cgemm_fp32" else "tc_reduce")
        tp, cp_ = nb.nat_bem_trace_kernel("tc_pack")
        nb.nat_bem_trace_enable(False)
    if c == 0:
        raise RuntimeError("no product kernel ran")
    ms = t / c
    # operator bytes one product streams: FP32 L (8 per complex), the three BF16 pieces (12),
    # or the BF16 / FP16 copy (4)
    op_bytes = (12 if name == "tc_gemm_x6" else 8 if args.prec in ("fp32", "tf32") else 4) * n * ld
    peaks, _ = _peaks()
    return {"metric": "multi-RHS operator products per second", "value": 1e3 / ms, "unit": "products/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": args.prec, "data": "synthetic",
            "config": {"workload": f"products_{n}tri_{args.nrhs}rhs", "engine": args.prec, "kernel": name},
            "ms_per_product": ms, "reduce_ms": tr / max(cr, 1), "pack_ms": tp / max(cp_, 1),
            "tflops": 8.0 * n * ld * args.nrhs / ms / 1e9,
            "operator_gbs": op_bytes / ms / 1e6, "hbm_frac": op_bytes / ms / 1e6 / peaks["hbm_gbs"]}


def run_mc(args):
    """Monte-Carlo BEM (paper Sec. 4.1.1, 4.2): the interior-source body sampled by the GPU
    Poisson-disk sampler (8 x --n-samples draws at 0.7 of the hexagonal spacing of --n-samples
    points; about 0.97 x --n-samples accepted) or with --n-samples uniform random points
    (--random-samples), monopole Neumann data at the samples, --n-k wavenumbers in ka
    [0.5, 12], 1024 field points at radius 4. One step: for each wavenumber, re-assemble the
    sample operators, solve, evaluate the field; --concurrency wavenumbers in flight. The
    sampler runs once per body and is timed on its own."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    nb_build.build()
    dev = torch.device("cuda", 0)
    Y, N, area, ks, gs, pts, exact = S.mc_interior_source(M=args.n_samples, n_k=args.n_k, poisson=False)
    sampler = None
    if not args.random_samples:
        # Poisson-disk samples from the GPU sampler, timed on their own (once per body)
        V, F = S.mc_interior_body()
        u, radius = S.poisson_draws(V, F, args.n_samples, 6001)
        Vd, Fd, ud = torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev), torch.from_numpy(u).to(dev)
        times = []
        for rep in range(13):
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, Yd, Nd = nb.nat_bem_poisson_sample(Vd, Fd, ud, radius)
            times.append(time.perf_counter() - t)
        Y, N = Yd.cpu().numpy(), Nd.cpu().numpy()
        gs = [S.monopole_neumann_at(Y, N, k) for k in ks]
        sampler = {"ms_median": 1e3 * float(np.median(times[3:])), "candidates": len(u), "radius": radius,
                   "samples": len(Y), "per": "one call, host wall clock, outputs on the device"}
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32, "fp16": nb.PREC_MIXED_FP16}[args.prec]
    opts = nb.nat_bem_opts_default(prec=prec)
    if args.inner_tol is not None:
        opts.inner_tol = args.inner_tol
    Yd, Nd, Pd = (torch.from_numpy(a).to(dev) for a in (Y, N, pts))
    Gd = [torch.from_numpy(g.astype(np.complex64)).to(dev) for g in gs]
    stream = torch.cuda.current_stream(dev)
    conc = max(1, min(args.concurrency, len(ks)))
    if conc > 1:
        opts.device_loop = 0  # host-polled chunks with several solves in flight
    streams, ops = _pool(torch, dev, conc, lambda sh: nb.Operator.assemble_mc(Yd, Nd, area, float(ks[0]), opts, stream=sh))
    infos = []

    def body(op, sh, i):
        op.reassemble(float(ks[i]), stream=sh)
        p, info, st = op.solve(Gd[i], stream=sh)
        f = op.evaluate(Pd, p, Gd[i], stream=sh)
        return p, f, (info.iterations, info.rel_residual, st)

    def step(record=None, nw=None):
        out = _pool_run(torch, streams, ops, len(ks), body, nw)
        if record is not None:
            record.extend(o[2] for o in out)
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-kernel device times from one untimed step (one worker)
    nb.nat_bem_trace_enable(True)
    nb.nat_bem_trace_select("")
    nb.nat_bem_trace_reset()
    step(nw=1)
    torch.cuda.synchronize()
    names = ["assemble_mc", "gemv", "gemv_bf16", "gemv_rhs", "gemv_resid", "ir_residual", "gmres_arnoldi",
             "gmres_lsq", "eval", "eval_reduce"]
    kern = {nm: nb.nat_bem_trace_kernel(nm) for nm in names}
    g = kern["gemv"]
    kern["gemv"] = tuple(a - b - c - d for a, b, c, d in zip(g, kern["gemv_rhs"], kern["gemv_resid"], kern["gemv_bf16"]))
    ev = kern["eval"]
    kern["eval"] = (ev[0] - kern["eval_reduce"][0], ev[1] - kern["eval_reduce"][1])
    nb.nat_bem_trace_enable(False)
    launches0 = nb.nat_bem_trace_launches()
    with ClockSampler(0) as clk:
        ms, res = _pool_time(torch, stream, streams, lambda: [step(infos) for _ in range(args.steps)][-1])
    launches = nb.nat_bem_trace_launches() - launches0
    n_solves = args.steps * len(ks)
    # the matvecs (as for the mesh workloads) and the assembly, which writes L and R (and L's BF16
    # copy in mixed precision) for every sample pair; the roofline is the dominant one's
    m = len(Y)
    peaks, peak_kind = _peaks()
    working = {nm: _working_launches(nb.nat_bem_trace_durations(nm)) for nm in ("gemv", "gemv_bf16", "gemv_fp16")}
    _, table = roofline({"n": m, "measured": dict(kern, assemble_regular=(0.0, 0)), "working": working},
                        peaks, peak_kind)
    bytes_pair = 16 + (4 if args.prec == "bf16" else 0)
    ta, ca = kern["assemble_mc"]
    if ca:
        gbs = (m * m * bytes_pair) / (ta / ca * 1e-3) / 1e9
        table["assemble_mc"] = {"bound": "hbm", "launches": ca, "avg_ms": ta / ca, "achieved": gbs,
                                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                                "algorithmic_bytes_per_launch": m * m * bytes_pair}
    dom = max(kern, key=lambda nm: kern[nm][0])
    roof = {"kernel": dom, "bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None, "note": "no roofline: the dominant kernel is latency-bound"}
    if dom in table:
        d = table[dom]
        roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": None, "peak_source": f"{peak_kind} (hbm_gbs)"}
        if dom in ("gemv", "gemv_bf16"):
            roof["note"] = ("the operator (8 or 4 x m x ld bytes: 125 or 63 MB at 3956 samples) is about the "
                            "size of L2 or smaller, so part of each matvec is served from L2")
    p0 = res[0][0].cpu().numpy()
    f0 = res[0][1].cpu().numpy()
    acc = {"surface_rel_err_vs_exact": float(np.linalg.norm(p0 - S.monopole_field(Y, float(ks[0])))
                                             / np.linalg.norm(S.monopole_field(Y, float(ks[0])))),
           "field_rel_err_vs_exact": float(np.linalg.norm(f0 - exact[0]) / np.linalg.norm(exact[0])),
           "k": float(ks[0])}
    if args.cpu:
        import oracle
        L, R = oracle.mc_assemble(Y, N, area, float(ks[0]))
        pref = np.linalg.solve(L, R @ gs[0])
        fref = oracle.mc_evaluate(Y, N, area, float(ks[0]), pts, pref, gs[0])
        acc["surface_rel_err_vs_oracle"] = float(np.linalg.norm(p0 - pref) / np.linalg.norm(pref))
        acc["field_rel_err_vs_oracle"] = float(np.linalg.norm(f0 - fref) / np.linalg.norm(fref))
    for op in ops:
        op.close()
    return {"metric": METRIC, "value": n_solves / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16 inner GMRES + f32 refinement", "tf32": "f32"}[args.prec],
            "data": "synthetic",
            "config": {"workload": f"bem_mc_{'random' if args.random_samples else 'poisson'}_{len(Y)}samples_{len(ks)}k",
                       "samples": len(Y), "ka_range": [0.5, 12.0], "field_points": len(pts), "precision": args.prec,
                       "in_flight": conc},
            "latency_ms": {"mean": ms / n_solves * conc,
                           "per": f"one solve (re-assembly + GMRES + field), {conc} in flight"},
            "gmres": {"iterations_max": max(i[0] for i in infos), "max_rel_residual": max(i[1] for i in infos),
                      "not_converged": sum(1 for i in infos if i[2] != 0)},
            "gpu_launches": int(launches),
            "kernels_ms_per_step": {nm: {"ms_total": v[0], "launches": v[1]} for nm, v in kern.items()},
            "roofline": roof, "rooflines": table,
            "accuracy": acc, "sampler": sampler, "clocks": clk.summary()}


def run_dataset(args):
    """Training-data generation (paper Sec. 3.4): for each of --n-k wavenumbers of the
    interior-source body, re-assemble, solve, draw 10,000 samples at (theta, phi, r) with r in
    [1.5, 3] bounding radii and take |p| there, and compute the 64 x 32 FFAT map of the far
    field; --concurrency wavenumbers in flight. Reports solves/s and training samples/s."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    nb_build.build()
    prob = workload(args.n_k, args.n_tri)
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32, "fp16": nb.PREC_MIXED_FP16}[args.prec]
    opts = nb.nat_bem_opts_default(prec=prec)
    if args.inner_tol is not None:
        opts.inner_tol = args.inner_tol
    dev = torch.device("cuda", 0)
    Vd, Fd = torch.from_numpy(prob.V).to(dev), torch.from_numpy(prob.F).to(dev)
    Gd = [torch.from_numpy(np.ascontiguousarray(g[:, 0]).astype(np.complex64)).to(dev) for g in prob.neumann]
    lo, hi = prob.V.min(axis=0), prob.V.max(axis=0)
    center, rb = 0.5 * (lo + hi), 0.5 * float(np.linalg.norm(hi - lo))
    n_samples = 10000
    rng = np.random.default_rng(7000)
    U = [torch.from_numpy(rng.random((n_samples, 3))).to(dev) for _ in prob.ks]
    th = (np.arange(32) + 0.5) * np.pi / 32
    ph = (np.arange(64) + 0.5) * 2 * np.pi / 64
    T, P = np.meshgrid(th, ph, indexing="ij")
    dirs = torch.from_numpy(np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)).to(dev)
    stream = torch.cuda.current_stream(dev)
    # --concurrency workers, each with its own operator and stream, take the wavenumbers in turn
    # (the library's calls release the GIL and block only their own thread)
    conc = max(1, min(args.concurrency, len(prob.ks)))
    if conc > 1:
        opts.device_loop = 0  # host-polled chunks with several solves in flight (as the batch driver does)
    streams = [torch.cuda.Stream(dev) for _ in range(conc)]
    ops = [nb.Operator.assemble(Vd, Fd, float(prob.ks[0]), opts, stream=st.cuda_stream) for st in streams]
    torch.cuda.synchronize()

    def work(w, nw):
        st, op = streams[w], ops[w]
        with torch.cuda.stream(st):
            for i in range(w, len(prob.ks), nw):
                op.reassemble(float(prob.ks[i]), stream=st.cuda_stream)
                p, info, s_ = op.solve(Gd[i], stream=st.cuda_stream)
                op.sample_field(U[i], center, 1.5 * rb, 3.0 * rb, p, Gd[i], stream=st.cuda_stream)
                op.far_field(dirs, p, Gd[i], stream=st.cuda_stream)

    def step(nw=conc):
        if nw == 1:
            work(0, 1)
            return
        ths = [threading.Thread(target=work, args=(w, nw)) for w in range(nw)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-kernel device times from one untimed step (one worker), and the dominant kernel's roofline
    nb.nat_bem_trace_reset()
    nb.nat_bem_trace_select("")
    nb.nat_bem_trace_enable(True)
    step(1)
    torch.cuda.synchronize()
    nb.nat_bem_trace_enable(False)
    kern = _kernel_table(nb)
    for nm in ("sample_points", "sample_abs", "far_field"):
        kern[nm] = nb.nat_bem_trace_kernel(nm)
    working = {nm: _working_launches(nb.nat_bem_trace_durations(nm)) for nm in ("gemv", "gemv_bf16", "gemv_fp16")}
    peaks, peak_kind = _peaks()
    dom, table = roofline({"n": len(prob.F), "measured": kern, "working": working}, peaks, peak_kind)
    nb.nat_bem_trace_reset()
    launches0 = nb.nat_bem_trace_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        t0.record(stream)
        for st in streams:  # the workers' streams start after t0 ...
            st.wait_event(t0)
        for _ in range(args.steps):
            step()
        for st in streams:  # ... and t1 follows all of them
            e = torch.cuda.Event()
            e.record(st)
            stream.wait_event(e)
        t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    launches = nb.nat_bem_trace_launches() - launches0
    n_solves = args.steps * len(prob.ks)
    for op in ops:
        op.close()
    roof = None
    if dom:
        d = table[dom]
        roof = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": NCU_TRAFFIC_10240.get(dom) if len(prob.F) == 10240 else None,
                "peak_source": f"{peak_kind} ({'hbm_gbs' if d['bound'] == 'hbm' else 'derived FP32'})"}
    return {"metric": METRIC, "value": n_solves / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic",
            "config": {"workload": f"dataset_{len(prob.F)}tri_{len(prob.ks)}k_{n_samples}samples_ffat64x32",
                       "samples_per_solve": n_samples, "ffat": [64, 32], "shell": [1.5, 3.0],
                       "in_flight": conc},
            "training_samples_per_s": n_solves * n_samples / (ms * 1e-3),
            "gpu_launches": int(launches),
            "kernels_ms_per_step": {nm: {"ms_total": v[0], "launches": v[1]} for nm, v in kern.items() if v[1]},
            "roofline": roof,
            "clocks": clk.summary()}


# FP32 flops of one regular Galerkin element pair in k_gal_regular: 49 point pairs of about 71
# (x - y, r, phase, G and both normal derivatives, and the three trial-function sums) plus 7
# test-point updates of 84 (the 3 x 3 blocks of K and G and the 3 K' sums), an FMA counting 2.
GAL_FLOPS_PER_PAIR = 49 * 71 + 7 * 84


def run_galerkin(args):
    """Galerkin Burton-Miller (paper Sec. 4, Eq. 6, element-to-element integration of Sec. 4.1):
    the interior-source body on --n-tri triangles (default 5120, 2562 vertices; P1 pressure, P0
    Neumann data), monopole Neumann data, --n-k wavenumbers log-uniform in ka [0.5, 10], 1024
    field points at radius 4. One step: for each wavenumber, re-assemble (element-pair blocks
    and their gathers), solve, evaluate the field; --concurrency wavenumbers in flight."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    nb_build.build()
    prob = S.interior_source(n_tri=args.n_tri, n_k=args.n_k, ka_range=(0.5, 10.0))
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32, "fp16": nb.PREC_MIXED_FP16}[args.prec]
    opts = nb.nat_bem_opts_default(prec=prec)
    if args.inner_tol is not None:
        opts.inner_tol = args.inner_tol
    dev = torch.device("cuda", 0)
    Vd, Fd, Pd = (torch.from_numpy(a).to(dev) for a in (prob.V, prob.F, prob.points))
    Gd = [torch.from_numpy(np.ascontiguousarray(g[:, 0]).astype(np.complex64)).to(dev) for g in prob.neumann]
    stream = torch.cuda.current_stream(dev)
    conc = max(1, min(args.concurrency, len(prob.ks)))
    if conc > 1:
        opts.device_loop = 0  # host-polled chunks with several solves in flight
    streams, ops = _pool(torch, dev, conc,
                         lambda sh: nb.Operator.assemble_galerkin(Vd, Fd, float(prob.ks[0]), opts, stream=sh))
    infos = []

    def body(op, sh, i):
        op.reassemble(float(prob.ks[i]), stream=sh)
        p, info, st = op.solve(Gd[i], stream=sh)
        f = op.evaluate(Pd, p, Gd[i], stream=sh)
        return p, f, (info.iterations, info.rel_residual, st)

    def step(record=None, nw=None):
        out = _pool_run(torch, streams, ops, len(prob.ks), body, nw)
        if record is not None:
            record.extend(o[2] for o in out)
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-kernel device times from one untimed step (one worker)
    nb.nat_bem_trace_enable(True)
    nb.nat_bem_trace_select("")
    nb.nat_bem_trace_reset()
    step(nw=1)
    torch.cuda.synchronize()
    names = ["gal_regular", "gal_singular", "gal_rowsum_L", "gal_gather_L", "gal_gather_R", "gemv_bf16",
             "gemv_rhs", "gemv_resid", "gmres_arnoldi", "eval", "gal_expand"]
    kern = {nm: nb.nat_bem_trace_kernel(nm) for nm in names}
    nb.nat_bem_trace_enable(False)
    launches0 = nb.nat_bem_trace_launches()
    with ClockSampler(0) as clk:
        ms, res = _pool_time(torch, stream, streams, lambda: [step(infos) for _ in range(args.steps)][-1])
    launches = nb.nat_bem_trace_launches() - launches0
    n_solves = args.steps * len(prob.ks)
    f0 = res[0][1].cpu().numpy()
    acc = {"field_rel_err_vs_exact": float(np.linalg.norm(f0 - prob.exact_field[0]) / np.linalg.norm(prob.exact_field[0])),
           "k": float(prob.ks[0])}
    nt = len(prob.F)
    t, c = kern["gal_regular"]
    peaks, peak_kind = _peaks()
    fp32_peak = FP32_LANES_PER_SM * sm_count() * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    # every launch of the traced step together covers the nt x nt pairs of each of its solves
    flops = float(len(prob.ks)) * nt * nt * GAL_FLOPS_PER_PAIR
    tf = flops / (t * 1e-3) / 1e12 if c else None
    for op in ops:
        op.close()
    return {"metric": METRIC, "value": n_solves / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16 inner GMRES + f32 refinement", "tf32": "f32"}[args.prec],
            "data": "synthetic",
            "config": {"workload": f"galerkin_interior_source_{nt}tri_{len(prob.V)}vert_{len(prob.ks)}k",
                       "n_tri": nt, "n_vert": len(prob.V), "ka_range": [0.5, 10.0],
                       "field_points": len(prob.points), "precision": args.prec, "in_flight": conc},
            "latency_ms": {"mean": ms / n_solves * conc,
                           "per": f"one solve (re-assembly + GMRES + field), {conc} in flight"},
            "gmres": {"iterations_max": max(i[0] for i in infos), "max_rel_residual": max(i[1] for i in infos),
                      "not_converged": sum(1 for i in infos if i[2] != 0)},
            "gpu_launches": int(launches),
            "kernels_ms_per_step": {nm: {"ms_total": v[0], "launches": v[1]} for nm, v in kern.items()},
            "roofline": {"kernel": "gal_regular", "bound": "alu", "achieved": tf, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": (tf / fp32_peak) if tf else None, "traffic": None,
                         "flops_per_pair": GAL_FLOPS_PER_PAIR,
                         "peak_source": f"derived: 128 FP32 lanes x {sm_count()} SMs x 2 x max SM clock"},
            "accuracy": acc, "clocks": clk.summary()}


def run_nat(args):
    """Neural acoustic transfer field inference (paper Sec. 3.3, 3.4): --n-queries listening
    points (theta/pi, phi/2pi, r_norm, v_1, v_2, f) uniform in [0, 1]^6 through the grid +
    positional encoding and the 4 x 128 MLP to 8 outputs (e.g. 8 modes), one fused tensor-core
    kernel per call. Random FP32 parameters from synthetic.nat_params with hash tables of 2^18
    rows (the trained model is not available); the library stores them in FP16 / BF16. Reports
    queries/s; the roofline counts the MLP's algorithmic FLOPs (first layer 52 wide, no padding)
    against the measured BF16 peak."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    import synthetic as S
    nb_build.build()
    n = args.n_queries
    m = S.nat_params(n_cond=2, n_out=8, table_log2=18, seed=0)
    dev = torch.device("cuda", 0)
    x = S.nat_queries(n, 6, 11)
    xd = torch.from_numpy(x).to(dev)
    out = torch.empty((n, 8), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    f = nb.NatField.from_params(m)
    batches = 64  # one step: 64 calls of n queries

    def step():
        for _ in range(batches):
            f.forward(xd, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    nb.nat_bem_trace_enable(True)
    nb.nat_bem_trace_select("nat_forward")
    nb.nat_bem_trace_reset()
    launches0 = nb.nat_bem_trace_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0, interval_ms=50) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    k_ms, k_launches = nb.nat_bem_trace_kernel("nat_forward")
    launches = nb.nat_bem_trace_launches() - launches0
    nb.nat_bem_trace_enable(False)
    # end to end through the public call with pinned host buffers (inputs in, outputs back,
    # every call; the library overlaps the copies with the kernels chunk by chunk); the call
    # blocks, so the host clock times it
    xh = torch.from_numpy(x).pin_memory()
    oh = torch.empty((n, 8), dtype=torch.float32).pin_memory()
    f.forward(xh, oh, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t_a = time.perf_counter()
    for _ in range(args.steps * batches):
        f.forward(xh, oh, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t_a) * 1e3
    width0 = 16 + 12 * 3  # grid features + P(v_1, v_2) + P(f)
    flops_q = 2 * (width0 * 128 + 3 * 128 * 128 + 128 * 8)  # the MLP's multiply-adds, unpadded
    kernel_ms = k_ms / max(k_launches, 1)
    peaks, peak_kind = _peaks()
    achieved = flops_q * n / (kernel_ms * 1e-3) / 1e12
    line = {"metric": "NAT field queries/s (grid + PE encoding, 4 x 128 MLP, 8 outputs)",
            "value": args.steps * batches * n / (ms * 1e-3), "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (FP32 accumulation)", "data": "synthetic (random weights and tables)",
            "config": {"workload": f"nat_inference_{n}queries", "queries": n, "calls_per_step": batches,
                       "inputs": 6, "outputs": 8,
                       "table_log2": 18, "levels": [8, 16, 32, 64], "width": 128, "hidden_layers": 4,
                       "l2": "inputs + outputs 235 MB per step, larger than L2"},
            "e2e": {"value": args.steps * batches * n / (e2e_ms * 1e-3), "unit": "queries/s",
                    "h2d_bytes_per_step": int(batches * x.nbytes), "d2h_bytes_per_step": int(batches * n * 8 * 4)},
            "gpu_launches": int(launches),
            "roofline": {"kernel": "nat_forward", "bound": "tensor", "achieved": achieved,
                         "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["bf16_tflops"],
                         "traffic": (NCU_TRAFFIC_NAT_PER_MQUERY * n / (1 << 20)) if NCU_TRAFFIC_NAT_PER_MQUERY else None,
                         "flops_per_query": flops_q, "peak_source": f"{peak_kind} (bf16_tflops)"},
            "clocks": clk.summary()}
    if args.cpu:
        from oracle import nat as O  # the CPU leg: the FP64 network and its rounding bound
        ns = 1 << 16
        xs = x[:ns].astype(np.float64)
        t = time.perf_counter()
        ref = O.forward(xs, m["tables"], m["weights"], m["biases"], 18)
        dt = time.perf_counter() - t
        got = out[:ns].cpu().numpy().astype(np.float64)
        sig = O.rounding_sigma(xs[:4096], m["tables"], m["weights"], m["biases"], 18)
        line["cpu_baseline"] = {"value": ns / dt, "unit": "queries/s", "cores": _numpy_threads(),
                                "kind": "oracle", "sample": f"first {ns} queries"}
        line["accuracy"] = {"rel_l2_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                            "max_dev_in_sigma": float(np.max(np.abs(got[:4096] - ref[:4096]) / sig)),
                            "bound_sigma": 12.0}
    f.close()
    return line


def _numpy_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


# DRAM bytes (read + write) of one k_nat_forward launch per 2^20 queries, from the committed ncu
# capture (profiles/k_nat_forward_nat_inference_1Mqueries.md); traffic grows with the queries.
# The write figure is what reached DRAM during the launch: most of the 33.6 MB of outputs were
# still in L2 when it ended.
NCU_TRAFFIC_NAT_PER_MQUERY = 28.146944e6 + 0.048128e6


def run_uneven(args):
    """Uneven batch: --n-mesh perturbed ring spheres of 500-8000 triangles (log-uniform), one
    wavenumber (ka in [0.5, 12]) and one smooth field each, 1024 points at radius 4. Two forms of
    the same batch, each timed over --steps steps: the fused batch (size buckets of meshes solved
    in lockstep as padded systems of independent operators, --max-batch meshes per bucket; the
    line's value) and the worker pool (largest first, --concurrency workers, one op and stream
    each). The lowest, median and largest meshes' results are checked against the oracle."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    nb_build.build()
    probs = S.uneven_batch(n_mesh=args.n_mesh)
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32, "fp16": nb.PREC_MIXED_FP16}[args.prec]
    opts = nb.nat_bem_opts_default(prec=prec)
    if args.inner_tol is not None:
        opts.inner_tol = args.inner_tol
    dev = torch.device("cuda", 0)
    jobs = []
    for pr in probs:
        jobs.append(dict(V=torch.from_numpy(pr.V).to(dev), F=torch.from_numpy(pr.F).to(dev), k=float(pr.ks[0]),
                         neumann=torch.from_numpy(np.ascontiguousarray(pr.neumann[0][:, 0]).astype(np.complex64)).to(dev),
                         points=torch.from_numpy(pr.points).to(dev)))
    stream = torch.cuda.current_stream(dev)
    runners = {"fused": lambda: nb.nat_bem_run_batch_fused(jobs, opts, max_batch=args.max_batch,
                                                           concurrency=args.fused_workers),
               "worker_pool": lambda: nb.nat_bem_run_batch(jobs, opts, concurrency=args.concurrency)}
    out = {}
    for name, fn in runners.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        nb.nat_bem_trace_enable(False)
        launches0 = nb.nat_bem_trace_launches()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lats = []
        with ClockSampler(0) as clk:
            t0.record(stream)
            for _ in range(args.steps):
                st, res = fn()
                lats += [r[4] for r in res]
            t1.record(stream)
            torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        out[name] = dict(value=args.steps * len(jobs) / (ms * 1e-3), ms=ms, lats=lats, res=res, clk=clk.summary(),
                         launches=nb.nat_bem_trace_launches() - launches0)
    sizes = [int(pr.F.shape[0]) for pr in probs]
    f = out["fused"]
    acc = None
    if args.cpu:
        import oracle
        order = np.argsort(sizes)
        errs = []
        for q in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
            pr = probs[q]
            g = pr.neumann[0][:, 0]
            pr_ref, fr_ref, _ = oracle.bem_solve(pr.V, pr.F, float(pr.ks[0]), g, pr.points, tol=1e-10, maxit=400)
            for name in ("fused", "worker_pool"):
                p_, f_ = out[name]["res"][q][0].cpu().numpy(), out[name]["res"][q][1].cpu().numpy()
                errs.append({"n_tri": sizes[q], "form": name,
                             "surface": float(np.linalg.norm(p_ - pr_ref) / np.linalg.norm(pr_ref)),
                             "field": float(np.linalg.norm(f_ - fr_ref) / np.linalg.norm(fr_ref))})
        acc = {"max": max(max(e["surface"], e["field"]) for e in errs), "per_job": errs}
    return {"metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic",
            "config": {"workload": f"uneven_batch_{len(jobs)}meshes", "n_tri_range": [min(sizes), max(sizes)],
                       "mean_n_tri": float(np.mean(sizes)), "form": "fused size buckets",
                       "max_batch": args.max_batch, "fused_workers": args.fused_workers},
            "latency_ms": dict(_percentiles(f["lats"]), per="one solve, device time of its bucket"),
            "gpu_launches": int(f["launches"]),
            "not_converged": sum(1 for r in f["res"] if r[3] != 0), "clocks": f["clk"],
            "worker_pool": {"value": out["worker_pool"]["value"], "ms_per_step": out["worker_pool"]["ms"] / args.steps,
                            "concurrency": args.concurrency, "gpu_launches": int(out["worker_pool"]["launches"]),
                            "latency_ms": dict(_percentiles(out["worker_pool"]["lats"]),
                                               per="one solve, device time, in the batch"),
                            "not_converged": sum(1 for r in out["worker_pool"]["res"] if r[3] != 0)},
            "rel_err_vs_oracle": acc}


def run_serving(args):
    """Serving stream: Poisson arrivals (--rate per second) of --n-req requests with meshes of
    1k-40k triangles (log-uniform; drawn from a pool of pre-built perturbed ring spheres), ka in
    [0.5, 20], 1-32 right-hand sides, admitted by dense-operator memory under --budget-gb of HBM.
    Requests are submitted at their arrival times; latency is submit to completion."""
    import torch
    import paper_2506_06190_gb300 as nb
    from paper_2506_06190_gb300 import build as nb_build
    nb_build.build()
    stream_def = S.serving_stream(n_req=args.n_req, rate=args.rate)
    pool_sizes = np.unique(np.geomspace(1000, 40000, 12).astype(int) // 2 * 2)
    pool = {}
    for nt in pool_sizes:
        Vs, F = S.ring_sphere(int(nt))
        pool[int(nt)] = (S.perturbed_ellipsoid(Vs, 5000 + int(nt)), F)
    prec = {"fp32": nb.PREC_FP32, "bf16": nb.PREC_MIXED_BF16, "tf32": nb.PREC_MIXED_TF32, "fp16": nb.PREC_MIXED_FP16}[args.prec]
    opts = nb.nat_bem_opts_default(prec=prec)
    if args.inner_tol is not None:
        opts.inner_tol = args.inner_tol
    dev = torch.device("cuda", 0)
    reqs = []
    pts = torch.from_numpy(S.fibonacci_points(256, 4.0)).to(dev)
    for (t_arr, nt_target, ka, nrhs, seed) in stream_def:
        nt = int(pool_sizes[np.argmin(np.abs(pool_sizes - nt_target))])
        V, F = pool[nt]
        g = S.sh_neumann(V, F, nrhs, seed)
        reqs.append((t_arr, dict(V=torch.from_numpy(V).to(dev), F=torch.from_numpy(F).to(dev), k=float(ka),
                                 neumann=torch.from_numpy(np.ascontiguousarray(g.T).astype(np.complex64)).to(dev),
                                 points=pts), nrhs))
    torch.cuda.synchronize()
    budget = int(args.budget_gb * (1 << 30))

    def serve(opts_, scale=1.0):
        # scale stretches the arrival times: the same requests offered at rate / scale
        with nb.Server(budget, opts_, slots=args.concurrency) as srv:
            tickets = []
            t_start = time.perf_counter()
            for t_arr, jd, nrhs in reqs:
                while time.perf_counter() - t_start < t_arr * scale:
                    time.sleep(0.0005)
                tickets.append((srv.submit(jd), nrhs))
            res = [(srv.wait(t, -1), nrhs) for t, nrhs in tickets]
            t_end = time.perf_counter()
        return res, t_end - t_start

    sweep = []
    for rate in [float(r) for r in args.rates.split(",") if r.strip()]:
        # the same stream offered at a lower rate (the arrival draws scale with 1 / rate); a rate
        # counts as sustained by _sustained
        r_res, r_dt = serve(opts, args.rate / rate)
        r_lat = [r[0][6] for r in r_res]
        third = len(r_lat) // 3
        p_first = float(np.percentile(r_lat[:third], 99))
        p_last = float(np.percentile(r_lat[-third:], 99))
        offered, rps, ok_rate = _sustained(len(r_res), reqs[-1][0] * args.rate / rate, r_dt, p_first, p_last)
        sweep.append({"offered_req_s": rate, "offered_actual_req_s": offered, "requests_per_s": rps,
                      "solves_per_s": sum(nrhs for r, nrhs in r_res if r[0] == 0) / r_dt,
                      "latency_ms": _percentiles(r_lat), "queue_ms": _percentiles([r[0][5] for r in r_res]),
                      "p99_first_third_ms": p_first, "p99_last_third_ms": p_last,
                      "sustained": ok_rate,
                      "all_ok": all(r[0][0] == 0 for r in r_res)})

    res, dt = serve(opts)
    lat = [r[0][6] for r in res]
    solves = sum(nrhs for r, nrhs in res if r[0] == 0)
    line = {"metric": METRIC, "value": solves / dt, "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * dt, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": f"serving_poisson_{args.rate}per_s_{args.n_req}req", "budget_gb": args.budget_gb,
                       "slots": args.concurrency, "offered_rate_req_s": args.rate},
            "requests_per_s": len(res) / dt,
            "latency_ms": dict(_percentiles(lat), per="request, submit to completion (queueing included)"),
            "queue_ms": _percentiles([r[0][5] for r in res]),
            "statuses": {str(k): int(v) for k, v in zip(*np.unique([r[0][0] for r in res], return_counts=True))}}
    if sweep:
        line["rate_sweep"] = sweep
        ok = [r["offered_req_s"] for r in sweep if r["sustained"] and r["all_ok"]]
        line["largest_sustained_rate_req_s"] = max(ok) if ok else None
    if args.prec != "fp32":
        res_p, dt_p = serve(nb.nat_bem_opts_default(prec=nb.PREC_FP32))
        lat_p = [r[0][6] for r in res_p]
        line["plain_fp32"] = {"value": sum(nrhs for r, nrhs in res_p if r[0] == 0) / dt_p, "unit": UNIT,
                              "requests_per_s": len(res_p) / dt_p, "latency_ms": _percentiles(lat_p),
                              "statuses": {str(k): int(v) for k, v in
                                           zip(*np.unique([r[0][0] for r in res_p], return_counts=True))}}
    return line


def roofline(res, peaks, peak_kind):
    """Dominant kernel's achieved rate against its ceiling."""
    n = res["n"]
    ld = (n + 31) // 32 * 32
    kern = res["measured"]
    working = res.get("working", {})
    table = {}
    # gemv: 8 n ld bytes of operator + 8 ld of x + 16 n of y per launch (one RHS); BF16 copy:
    # 4 n ld + 8 ld + 16 n. Averages over the launches that streamed the operator (the
    # iterations a captured chunk ran after convergence exit at once and are counted apart).
    for name, elem in (("gemv", 8.0), ("gemv_bf16", 4.0), ("gemv_fp16", 4.0)):
        if name not in kern:
            continue
        t, c, skipped = working.get(name, (kern[name][0], kern[name][1], 0))
        if c:
            bytes_per = elem * n * ld + 8.0 * ld + 16.0 * n + (4.0 * n if name == "gemv_fp16" else 0.0)
            gbs = bytes_per / (t / c * 1e-3) / 1e9
            table[name] = {"bound": "hbm", "launches": c, "launches_exited_early": skipped,
                           "avg_ms": t / c, "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": gbs / peaks["hbm_gbs"], "algorithmic_bytes_per_launch": bytes_per}
    # regular assembly: FP32 flops per element pair (7 quadrature points), counted from the
    # kernel's arithmetic (an FMA counts 2)
    t, c = kern["assemble_regular"]
    if c:
        pairs = float(n) * n
        flops = pairs * FLOPS_PER_PAIR
        tf = flops / (t / c * 1e-3) / 1e12
        fp32_peak = FP32_LANES_PER_SM * sm_count() * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        table["assemble_regular"] = {"bound": "alu", "launches": c, "avg_ms": t / c, "achieved": tf,
                                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": tf / fp32_peak,
                                     "algorithmic_flops_per_launch": flops}
    dom = max(table, key=lambda k: kern[k][0]) if table else None
    return dom, table


# DRAM bytes (read + write) per launch from ncu captures of the BF16 matvec on the current
# code, mean of six launches, 10240-triangle workload (profiles/k_gemv_interior_source_10240tri.md);
# None for kernels whose source changed since their capture.
NCU_TRAFFIC_10240 = {"gemv_bf16": 419.543e6 + 0.66e6}


# FP32 operations of k_assemble_regular per (i, j) pair: per quadrature point 29 FMA + 19
# other FP32 operations (2 x 29 + 19 = 77 flops) plus 3 MUFU operations (rsqrt, sin, cos) not
# counted; per pair 6 + 15 operations for the centroid difference and the three dot products.
FLOPS_PER_PAIR = 7 * 77 + 21
FP32_LANES_PER_SM = 128


def sm_count() -> int:
    """Streaming multiprocessors of the current device (152 on a GB300 when no GPU is seen)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        pass
    return 152


def aggregate_ranks(n_solves_local: float, ms_local: float, world: int, device=None):
    """Whole-job throughput for replicas: every rank solves its own copy of the workload with
    no exchange; value = total solves over all ranks / the slowest rank's time. Returns
    (value, max_ms)."""
    if world == 1:
        return n_solves_local / (ms_local * 1e-3), ms_local
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    n = torch.tensor([n_solves_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(n.item()) / (float(t.item()) * 1e-3), float(t.item())


def cpu_baseline(prob, nthreads: int):
    import oracle
    k = float(prob.ks[0])
    g = prob.neumann[0][:, 0]
    t = time.perf_counter()
    p, fld, info = oracle.bem_solve(prob.V, prob.F, k, g, prob.points, tol=1e-6, maxit=200,
                                    nthreads=nthreads)
    dt = time.perf_counter() - t
    return p, fld, dt, info


def run_extras(args):
    """The other workloads in short form (one warm-up and one timed step each), summarised under
    "workloads" in the headline's line: the multi-RHS modal products, the uneven batch (fused
    buckets beside the worker pool) and the serving stream (mixed beside plain FP32)."""
    out = {}
    base = dict(vars(args), steps=1, warmup=1, n_k=16, n_tri=20480, nrhs=64, prec="bf16", cpu=False,
                inner_tol=args.inner_tol)
    keep = ("value", "unit", "ms_per_step", "config", "latency_ms", "gpu_launches", "not_converged",
            "worker_pool", "plain_fp32", "requests_per_s", "statuses", "gmres", "rel_err_vs_oracle")
    for name, fn, over in (("modal", run_modal, {}),
                           ("uneven", run_uneven, dict(n_k=64, n_tri=10240, cpu=args.cpu)),
                           ("serve", run_serving, dict(concurrency=4))):
        try:
            r = fn(argparse.Namespace(**dict(base, **over)))
            d = {k: r[k] for k in keep if k in r}
            if r.get("roofline"):
                d["roofline"] = {k: r["roofline"][k] for k in ("kernel", "achieved", "peak", "unit", "frac", "traffic")
                                 if k in r["roofline"]}
            out[name] = d
        except Exception as e:  # report, do not lose the headline
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="natbem", choices=["natbem", "reference"])
    ap.add_argument("--prec", default=None, choices=["fp32", "bf16", "tf32", "fp16"],
                    help="bf16 = mixed (BF16 inner GMRES, FP32 refinement); default bf16, fp32 for the "
                         "Monte-Carlo and Galerkin workloads (their operators stay in or near L2, where the "
                         "BF16 copy saves little bandwidth and refinement costs iterations)")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the plain FP32 comparison run of the interior workload")
    ap.add_argument("--n-k", type=int, default=64)
    ap.add_argument("--n-tri", type=int, default=10240, help="smaller meshes only for profiling")
    ap.add_argument("--concurrency", type=int, default=4, help="solves in flight (batch workers)")
    ap.add_argument("--workload", default="interior",
                    choices=["interior", "modal", "uneven", "serve", "mc", "dataset", "nat", "galerkin", "products"])
    ap.add_argument("--n-samples", type=int, default=4096, help="Monte-Carlo workload: surface samples")
    ap.add_argument("--random-samples", action="store_true", help="Monte-Carlo workload: uniform random samples")
    ap.add_argument("--n-queries", type=int, default=1 << 22, help="NAT inference workload: queries per step")
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--n-mesh", type=int, default=512)
    ap.add_argument("--max-batch", type=int, default=64, help="uneven workload: meshes per fused bucket")
    ap.add_argument("--fused-workers", type=int, default=4, help="fused batch: bucket workers")
    ap.add_argument("--batch-mode", default="pool", choices=["pool", "fused"],
                    help="interior workload: worker pool (one op per job) or fused buckets")
    ap.add_argument("--n-req", type=int, default=300)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--rates", default="", help="serve workload: also offer the same stream at these rates "
                                                "(comma-separated req/s) and report the largest sustained one")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--inner-tol", type=float, default=None,
                    help="mixed precision: tolerance of each inner solve (default: the library's)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="interior workload: skip the short modal, uneven-batch and serving runs")
    ap.add_argument("--no-cpu-baseline", dest="cpu", action="store_false")
    args = ap.parse_args()
    if args.prec is None:
        args.prec = "fp32" if args.workload in ("mc", "galerkin") else "bf16"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    peaks, peak_kind = _peaks()

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        prob = workload(args.n_k, args.n_tri)
        nth = oracle.hardware_threads()
        for w in range(args.warmup):
            cpu_baseline(prob, nth)
        t = time.perf_counter()
        for s in range(args.steps):
            cpu_baseline(prob, nth)
        dt = time.perf_counter() - t
        v = args.steps / dt
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "interior_source_10240tri_64k", "n_tri": int(prob.F.shape[0]),
                           "step": "one solve (first wavenumber) of the workload"},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": nth, "kind": "oracle",
                                 "sample": "one wavenumber of the 64 per step"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if args.workload != "interior":
        if rank == 0:
            fn = {"modal": run_modal, "uneven": run_uneven, "serve": run_serving, "mc": run_mc,
                  "dataset": run_dataset, "nat": run_nat, "galerkin": run_galerkin,
                  "products": run_products}[args.workload]
            if args.workload == "products" and args.n_tri == 10240:
                args.n_tri = 20480
            if args.workload == "modal" and args.n_k == 64:
                args.n_k = 16
            if args.workload == "modal" and args.n_tri == 10240:
                args.n_tri = 20480
            if args.workload == "galerkin" and args.n_k == 64:
                args.n_k = 16
            if args.workload == "galerkin" and args.n_tri == 10240:
                args.n_tri = 5120
            print(json.dumps(fn(args)))
        return
    if world > 1:
        torch.distributed.init_process_group("nccl")
    res = run_gpu(args, rank, world, args.prec)
    prob = res.pop("prob")
    n_solves = args.steps * len(prob.ks)
    value, my_rate_time = aggregate_ranks(n_solves, res["ms_total"], world, device="cuda" if world > 1 else None)
    # the plain FP32 form on the same workload, same launch configuration, for comparison
    cmp = None
    cmp_checks = None
    if args.compare and args.prec != "fp32":
        cres = run_gpu(args, rank, world, "fp32", full=False)
        cres.pop("prob")
        cmp_checks = cres.pop("checks")
        cvalue, cms = aggregate_ranks(n_solves, cres["ms_total"], world, device="cuda" if world > 1 else None)
        cmp = {"value": cvalue, "unit": UNIT, "ms_per_step": cms / args.steps,
               "latency_ms": {"p50": float(np.percentile(cres["lat"], 50)),
                              "p99": float(np.percentile(cres["lat"], 99))},
               "gmres_iterations": {"median": float(np.median(cres["iters"])), "max": max(cres["iters"])},
               "max_rel_residual": cres["max_rel_res"], "not_converged": cres["n_enoconv"],
               "clocks": cres["clocks"]}
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    dom, table = roofline(res, peaks, peak_kind)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": my_rate_time / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32 (+f64 Krylov)",
                  "bf16": "bf16 inner GMRES + f32 refinement (+f64 Hessenberg and refinement sums)",
                  "fp16": "fp16 (row-scaled) inner GMRES + f32 refinement (+f64 Hessenberg and refinement sums)",
                  "tf32": "f32 (one RHS: TF32 saves no bytes)"}[args.prec],
        "data": "synthetic",
        "config": {"workload": f"interior_source_{res['n']}tri_{len(prob.ks)}k", "n_tri": res["n"],
                   "n_wavenumbers": len(prob.ks), "ka_range": [0.5, 20.0], "field_points": 1024,
                   "precision": args.prec, "tol": 1e-6, "max_iter": 200,
                   "l2": "inputs larger than L2: each wavenumber's operators are 2 x 839 MB"},
        "latency_ms": {"p50": float(np.percentile(res["lat"], 50)), "p99": float(np.percentile(res["lat"], 99)),
                       "per": "one solve (assemble + GMRES + field), device time, "
                              f"{args.concurrency} solves in flight"},
        "gmres_iterations": {"min": min(res["iters"]), "median": float(np.median(res["iters"])),
                             "max": max(res["iters"])},
        "max_rel_residual": res["max_rel_res"],
        "not_converged": res["n_enoconv"],
        "max_refinements": res["refinements"],
        "concurrency": args.concurrency,
        "gemv_variant_fp32": res.get("gemv_variant"),
        "gpu_launches": int(res["launches"]),
        "clocks": res["clocks"],
    }
    if dom:
        d = table[dom]
        line["roofline"] = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
                            "unit": d["unit"], "frac": d["frac"],
                            "traffic": NCU_TRAFFIC_10240.get(dom) if res["n"] == 10240 else None,
                            "measured_on": "one untimed step of the workload, one solve at a time, CUDA events per launch",
                            "peak_source": f"{peak_kind} ({'hbm_gbs' if d['bound'] == 'hbm' else f'derived: 128 FP32 lanes x {sm_count()} SMs x 2 x max SM clock'})"}
    if cmp:
        line["plain_fp32"] = cmp
    line["kernels"] = {k: {"ms_total": v[0], "launches": v[1]} for k, v in res["kern"].items()}
    line["rooflines"] = table
    if res["e2e"]:
        line["e2e"] = res["e2e"]
    if args.cpu:
        import oracle
        oracle.build()
        nth = oracle.hardware_threads()
        p_ref, f_ref, dt, info = cpu_baseline(prob, nth)
        ep = float(np.linalg.norm(res["p0"] - p_ref) / np.linalg.norm(p_ref))
        ef = float(np.linalg.norm(res["f0"] - f_ref) / np.linalg.norm(f_ref))
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": nth, "kind": "oracle",
                                "sample": f"one solve (k={prob.ks[0]:.4f}) of the 64; stage seconds "
                                          f"{[round(x, 2) for x in info['times']]}"}
        # accuracy: the lowest, median and highest wavenumber, both precisions, against oracle
        # solves to 1e-10 (untimed)
        per_k = []
        for i in sorted(res["checks"]):
            k = float(prob.ks[i])
            g = prob.neumann[i][:, 0]
            pr, fr, _ = oracle.bem_solve(prob.V, prob.F, k, g, prob.points, tol=1e-10, maxit=400,
                                         nthreads=nth)
            row = {"k": k}
            main_name = "plain_fp32" if args.prec == "fp32" else f"mixed_{args.prec}"
            for name, chk in ((main_name, res["checks"]), ("plain_fp32", cmp_checks)):
                if chk is None:
                    continue
                pg, fg = chk[i]
                row[name] = {"surface": float(np.linalg.norm(pg - pr) / np.linalg.norm(pr)),
                             "field": float(np.linalg.norm(fg - fr) / np.linalg.norm(fr))}
            per_k.append(row)
        errs = [v for row in per_k for nm, e in row.items() if nm != "k" for v in e.values()]
        line["rel_err_vs_oracle"] = {"max": max(errs), "meets_1e-4": bool(max(errs) <= 1e-4),
                                     "checked": "lowest, median and highest wavenumber; mixed and plain FP32; "
                                                "surface and field; oracle GMRES to 1e-10",
                                     "per_k": per_k,
                                     "first_k": {"surface": ep, "field": ef, "k": float(prob.ks[0])}}
    if args.extras and world == 1:
        line["workloads"] = run_extras(args)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

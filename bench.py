#!/usr/bin/env python
"""Benchmark: time-to-solution of the spacetime FEM Dirac solve on GB300.

One step = one whole solve of the 2+1 Zitterbewegung workload (96 x 96 space
x 96 time Q1 elements, 2-component spinor, 1,769,472 complex unknowns) to
relative residual 1e-8: right-hand side, FP32 operator applies inside GMRES(30),
one classical Gram-Schmidt pass per step (PETSc's GMRES default) on an
FP32-stored Krylov basis in compensated arithmetic, FP64 Givens/least squares,
FP64 residuals and iterative refinement.
Inputs are resident in HBM when the timed region starts; the GMRES basis
(31 x 28 MB) exceeds L2, so no L2 flush is needed between steps.

Also reported on the same line: the plain-FP64-GMRES time-to-solution of the
same system, the standalone operator-apply bandwidth (rotating buffers > 2x L2),
the roofline of the dominant kernel class measured with CUDA events around
every kernel of the last timed solve, the end-to-end time through the C ABI with host buffers, the
FP64 CPU oracle timed on the host cores, and the throughput of the batched
solve (dst_solve_batch) on two seeded sets of independent 1+1 / 2+1 solves.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --ncu-case solve60|solve60_klein32|apply32_zb|apply32_klein|apply64_klein  (ncu cases)
N > 1 runs under torch.distributed.run: independent replicas, one per GPU.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

RTOL = 1e-8
RESTART = 30
INNER_RTOL = 1e-4
# Gram-Schmidt of the timed solves: one classical pass per Arnoldi step, no
# reorthogonalisation (PETSc's GMRES default); on this workload it takes the same
# steps to the same residual as the library's default DGKS-selective second pass
ORTHO = 2
HBM_FALLBACK_GBS = 6800.0
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_FLOP_PER_CLK_SM = 4.0     # 2 FP64 FMA per clock per SM (1/64 of the FP32 rate)
FP32_FLOP_PER_CLK_SM = 256.0   # 128 FP32 FMA per clock per SM
CLASSES = ("apply64", "apply32", "cast", "project", "update", "scale", "misc", "rhs")
# DRAM read+write bytes per algorithmic byte of the projection / update on the FP32-stored
# basis, from one ncu capture of each (profiles/gram_schmidt_f32_zb_2p1.md); valid for
# project_f32_kernel / update_f32_kernel as committed with that file (None: not captured).
TRAFFIC_RATIO = {"project": 1.040, "update": 0.992}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", HBM_FALLBACK_GBS), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def iteration_count(name):
    p = os.path.join(ROOT, "tests", "golden", "oracle_iteration_counts.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if name in d and d[name].get("converged"):
            return d[name]["iters"]
    return None


# ---------------------------------------------------------------- CPU oracle

def oracle_seconds_per_step(w, k=4):
    """Seconds per Arnoldi step of the oracle's GMRES(30), as it stands, on the full mesh.

    Difference of two oracle solves capped at 1 and 1 + k steps (both include
    the same initial and final residual applies), divided by k.
    """
    from oracle import mesh as OM, operator as OOP, solvers as OS
    om = OM.Mesh(w.d, w.n_el, w.lo, w.hi, w.bc)
    b = OOP.rhs(om, w.m, w.V, w.psi0)
    A = lambda v: OOP.apply(om, w.m, w.V, v)  # noqa: E731
    t0 = time.perf_counter()
    OS.gmres(A, b, restart=RESTART, rtol=RTOL, maxiter=1)
    t1 = time.perf_counter()
    OS.gmres(A, b, restart=RESTART, rtol=RTOL, maxiter=1 + k)
    t2 = time.perf_counter()
    return max((t2 - t1) - (t1 - t0), 1e-9) / k


def replica_seed(rank):
    """Seed of the bench workload on a rank: independent replicas draw independent packets."""
    return 20210326 + rank


def aggregate_timing(t_ms, world, steps, dist=None, device="cuda"):
    """Length of the timed region as the maximum over ranks, and the whole-job
    throughput (solves of all ranks per second of that region)."""
    if world > 1:
        import torch
        tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    return t_ms, world * steps / (t_ms * 1e-3)


def host_cores():
    """Threads the oracle's numpy / BLAS work may use on this host (its dense element
    products are BLAS matrix products): the BLAS pool size where threadpoolctl is
    installed, else the usual thread-count variables, else the core count."""
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit() and int(v) > 0:
            return int(v)
    return os.cpu_count() or 1


def run_reference(args, rank):
    """The FP64 CPU oracle on the host cores, same workload / metric / unit."""
    if rank != 0:
        return
    w = W.zb_2p1()
    n_iter = iteration_count("zb_2p1")
    k = 2
    for _ in range(args.warmup):
        oracle_seconds_per_step(w, k)
    per = [oracle_seconds_per_step(w, k) for _ in range(args.steps)]
    sec_step = statistics.mean(per)
    if n_iter is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle GMRES step count for zb_2p1 not recorded "
                          "(run python -m oracle.iteration_counts)"}))
        return
    solve_s = sec_step * n_iter
    value = 1.0 / solve_s
    sample = ("each step: the oracle's GMRES(%d) from x0 = 0 on the full 96x96x96 system for 1 and %d Arnoldi "
              "steps; the difference / %d is the seconds per step, times the oracle's own %d-step solve "
              "(rel. resid %g) recorded by oracle/iteration_counts.py" % (RESTART, 1 + k, k, n_iter, RTOL))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * solve_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm

METRIC = "operator-apply HBM GB/s; time-to-solution at rel. resid 1e-8 vs plain FP64 GMRES"
CONFIG = {"workload": "zb_2p1: 2+1 Zitterbewegung packet (sigma 0.5, p0 (2,0), seed 20210326), Q1 mesh "
                      "96x96 space x 96 time on [-8,8]^2 x [0,4], periodic, m = 1, NC = 2, 1769472 complex "
                      "unknowns; GMRES(30) with FP32 operator apply inside FP64 iterative refinement to "
                      "rel. resid 1e-8",
          "unknowns": 1769472, "rtol": RTOL, "restart": RESTART, "inner_rtol": INNER_RTOL,
          "l2": "working set > L2 (FP32 GMRES basis 31 x 14 MB = 439 MB), no flush", "parallelism": "replicas",
          "gram_schmidt": "one classical pass per step (ortho = 2), mixed and FP64 solves alike"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.proc = None
        self.uuid = uuid

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd[1:1] = ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def time_apply(torch, B, mesh, prec, n, iters=40):
    """Average device time of one operator apply over rotating buffers (> 2x L2).

    The applies are captured once in a CUDA graph and replayed, so the host-side
    cost of the Python call does not leave the GPU idle between launches.
    """
    import ctypes
    lib = B.library()
    dt = torch.complex64 if prec == B.DST_FP32 else torch.complex128
    esz = 8 if prec == B.DST_FP32 else 16
    pairs = max(2, int(np.ceil(2 * 135e6 / (2 * n * esz))) + 1)
    xs = [torch.randn(n, dtype=dt, device="cuda") for _ in range(pairs)]
    ys = [torch.empty(n, dtype=dt, device="cuda") for _ in range(pairs)]
    for i in range(pairs):
        B.dst_apply_operator(mesh, prec, xs[i], ys[i])
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        cs = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for i in range(iters):
            rc = lib.dst_apply_operator(ctypes.c_void_p(mesh), prec, ctypes.c_void_p(xs[i % pairs].data_ptr()),
                                        ctypes.c_void_p(ys[i % pairs].data_ptr()), cs)
            if rc != 0:
                raise RuntimeError("dst_apply_operator failed in capture: %d" % rc)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    return ms, 2.0 * n * esz / (ms * 1e-3) / 1e9


NCU_CASES = ("solve60", "solve60_klein32", "apply32_zb", "apply32_klein", "apply64_klein")


def run_ncu_case(case):
    """Small fixed launches for ncu captures (nothing timed, nothing printed as a bench line).

    solve60: the first 60 Arnoldi steps (two GMRES(30) cycles) of the bench's mixed solve;
    solve60_klein32: the same on the 3+1 Klein workload at 32^3 x 32 (4.06M unknowns, large
    enough for the bulk-copy fed projection);
    apply32_zb / apply32_klein / apply64_klein: 12 operator applies on the 96^2 x 96 bench
    mesh or the 48^3 x 48 3+1 Klein mesh, over rotating buffers.
    """
    import torch
    from paper_2103_14588_gb300 import binding as B
    torch.cuda.set_device(0)
    if case == "solve60_klein32":
        w = W.klein_3p1(n=32, nt=32, p0=1.05)
    else:
        w = W.klein_3p1(p0=1.05) if case.endswith("klein") else W.zb_2p1()
    with B.Mesh.from_workload(w) as m:
        if case.startswith("solve60"):
            psi = torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda")
            st = B.dst_solve(m.handle, {"restart": RESTART, "rtol": RTOL, "max_iters": 60, "mixed_precision": 1}, psi)
            torch.cuda.synchronize()
            print("solve60: %d steps, status %d, %d second passes" % (st["iters"], st["status"], st["reorths"]))
        else:
            prec = B.DST_FP32 if case.startswith("apply32") else B.DST_FP64
            ms, gbs = time_apply(torch, B, m.handle, prec, m.n_unknowns, iters=12)
            print("%s: %.1f us per apply" % (case, 1e3 * ms))


BATCH_CASES = (
    # name, count, 1+1 element range per axis, 2+1 element range per axis, sequential sample
    ("tiny", 128, (24, 40), (8, 12), 16),
    ("mixed", 64, (32, 256), (16, 48), 8),
)


def run_batch_bench(torch, B):
    """Throughput of dst_solve_batch on seeded independent 1+1 / 2+1 solves
    (workloads.batch_instances), against single-mesh mixed solves one after
    another on an evenly spaced sample of the same instances (scaled to the count)."""
    import time as _t
    out = {}
    opts = {"rtol": RTOL, "max_iters": 20000, "max_refine": 100000}
    for name, count, n1, n2, sample in BATCH_CASES:
        ws = W.batch_instances(count, 4, n1=n1, n2=n2)
        meshes = [B.Mesh.from_workload(w) for w in ws]
        psis = [torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda") for m in meshes]
        torch.cuda.synchronize()
        t0 = _t.perf_counter()
        rc, sts = B.dst_solve_batch([m.handle for m in meshes], opts, psis)
        torch.cuda.synchronize()
        tb = _t.perf_counter() - t0
        idx = list(range(0, count, count // sample))[:sample]
        q = torch.zeros(max(m.n_unknowns for m in meshes), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = _t.perf_counter()
        seq_steps = 0
        for i in idx:
            seq_steps += B.dst_solve(meshes[i].handle, dict(opts, mixed_precision=1), q[:meshes[i].n_unknowns])["iters"]
        torch.cuda.synchronize()
        t_sample = _t.perf_counter() - t0
        ts = t_sample * count / len(idx)
        conv = sum(1 for st in sts if st["status"] == 0)
        out[name] = {"instances": count, "unknowns_total": int(sum(m.n_unknowns for m in meshes)),
                     "persistent_kernel_meshes": int(sum(m.n_unknowns <= 4096 for m in meshes)),
                     "batch_solves_per_s": count / tb, "batch_s": tb,
                     "sequential_solves_per_s": count / ts, "sequential_sample": len(idx),
                     "speedup": ts / tb, "converged": conv, "status": rc,
                     "arnoldi_steps": int(sum(st["iters"] for st in sts)),
                     "batch_steps_per_s": sum(st["iters"] for st in sts) / tb,
                     "sequential_steps_per_s": seq_steps / t_sample,
                     "note": "solves capped at 20000 Arnoldi steps count as solves on both sides"}
        for m in meshes:
            m.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve throughput cases")
    ap.add_argument("--ncu-case", choices=NCU_CASES, help="run one small case for an ncu capture and exit")
    args = ap.parse_args()
    if args.ncu_case:
        run_ncu_case(args.ncu_case)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2103_14588_gb300 import binding as B

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    w = W.zb_2p1(seed=replica_seed(rank))
    mesh_obj = B.Mesh.from_workload(w)
    mesh = mesh_obj.handle
    n = mesh_obj.n_unknowns
    psi = torch.zeros(n, dtype=torch.complex128, device="cuda")
    # one classical Gram-Schmidt pass per step (PETSc's GMRES default, ORTHO) in every timed
    # solve, mixed and plain FP64 alike
    opts = {"restart": RESTART, "rtol": RTOL, "max_iters": 200000, "mixed_precision": 1,
            "inner_rtol": INNER_RTOL, "max_refine": 60, "ortho": ORTHO}

    for _ in range(args.warmup):
        B.dst_solve(mesh, opts, psi)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    stats = []
    prof_opts = dict(opts, profile=1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(uuid if rank == 0 else None) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record()
        # the last timed solve records CUDA events around every kernel (the per-class
        # roofline); the others run without them
        for i in range(args.steps):
            stats.append(B.dst_solve(mesh, prof_opts if i == args.steps - 1 else opts, psi))
        e1.record()
        torch.cuda.synchronize()
        barrier()
    t_ms, value = aggregate_timing(e0.elapsed_time(e1), world, args.steps, dist)
    for s in stats:
        if s["status"] != 0:
            raise RuntimeError("timed solve did not converge: %s" % s)

    # per-class kernel accounting over the profiled (last) timed solve; launches over all
    tot = {k: [0.0, 0.0, 0.0, 0.0] for k in CLASSES}
    launches = sum(int(s["launches"]) for s in stats)
    for s in stats[-1:]:
        for i, k in enumerate(CLASSES):
            tot[k][0] += s["kernel_ms"][i]
            tot[k][1] += s["kernel_launches"][i]
            tot[k][2] += s["kernel_bytes"][i]
            tot[k][3] += s["kernel_flops"][i]
    kms = sum(v[0] for v in tot.values())

    if rank != 0:
        barrier()
        return

    hbm, hbm_kind = measured_peaks()
    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or SM_MAX_MHZ
    fp64_peak = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12   # TFLOP/s at max clock
    dom = max(CLASSES, key=lambda k: tot[k][0])
    d_ms, d_l, d_b, d_f = tot[dom]
    # in the timed mixed solve only the FP64 operator apply is bound by the FP64
    # pipe; every other class streams HBM
    fp64_classes = ("apply64",)
    if dom in fp64_classes and d_f > 0:
        ach = d_f / (d_ms * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": ach / fp64_peak, "traffic": None,
                "peak_kind": "FP64 FMA pipe: 152 SMs x 4 FLOP/clk x 2070 MHz (derived; probe measured 1.196)",
                "achieved_gbs": d_b / (d_ms * 1e-3) / 1e9, "hbm_frac": d_b / (d_ms * 1e-3) / 1e9 / hbm,
                "avg_launch_us": 1e3 * d_ms / max(d_l, 1)}
    else:
        ach = d_b / (d_ms * 1e-3) / 1e9
        traffic = None
        launches_ran = d_l
        if dom in ("project", "update"):
            # per step one first-pass launch plus one gated second pass, which moves data
            # only when it runs (reorths); achieved = bytes per launch / time per launch
            launches_ran = sum(s["iters"] + s["reorths"] for s in stats[-1:])
        if TRAFFIC_RATIO.get(dom):
            # average algorithmic bytes per launch that ran times the measured DRAM/algorithmic ratio
            traffic = TRAFFIC_RATIO[dom] * d_b / max(launches_ran, 1)
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "traffic_unit": "bytes per launch", "peak_kind": hbm_kind,
                "algorithmic_bytes_per_launch": d_b / max(launches_ran, 1),
                "avg_launch_us": 1e3 * d_ms / max(launches_ran, 1)}
    kernels = {k: {"ms_share": (v[0] / kms if kms else None), "launches": int(v[1]),
                   "GBps": (v[2] / (v[0] * 1e-3) / 1e9 if v[0] else None),
                   "TFLOPps": (v[3] / (v[0] * 1e-3) / 1e12 if v[0] else None)} for k, v in tot.items() if v[1]}

    # plain FP64 GMRES(30) on the same system (comparison, outside the timed region)
    fp64_opts = {"restart": RESTART, "rtol": RTOL, "max_iters": 200000, "mixed_precision": 0, "ortho": ORTHO}
    B.dst_solve(mesh, fp64_opts, psi)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    st64 = B.dst_solve(mesh, fp64_opts, psi)
    f1.record()
    torch.cuda.synchronize()
    fp64_s = f0.elapsed_time(f1) * 1e-3

    # standalone operator apply bandwidth (FP32 and FP64)
    a32_ms, a32_gbs = time_apply(torch, B, mesh, B.DST_FP32, n)
    a64_ms, a64_gbs = time_apply(torch, B, mesh, B.DST_FP64, n)

    # end to end through the C ABI with host buffers: psi0 from pinned host memory in,
    # solution to pinned host memory out, every step
    psi0_host = torch.from_numpy(np.ascontiguousarray(w.psi0).ravel().copy()).pin_memory()
    out_host = torch.empty(n, dtype=torch.complex128).pin_memory()
    e2e_steps = min(args.steps, 3)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record()
    for _ in range(e2e_steps):
        B.dst_set_initial_data(mesh, psi0_host)
        B.dst_solve(mesh, opts, psi)
        out_host.copy_(psi, non_blocking=True)
    g1.record()
    torch.cuda.synchronize()
    e2e_s = g0.elapsed_time(g1) * 1e-3 / e2e_steps
    e2e = {"value": 1.0 / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(psi0_host.numel() * 16),
           "d2h_bytes_per_step": int(n * 16)}

    batch = None if args.no_batch else run_batch_bench(torch, B)

    cpu = None
    if not args.no_cpu_baseline:
        sec_step = oracle_seconds_per_step(w, k=2)
        n_or = iteration_count("zb_2p1")
        src = "the oracle's own %s-step solve recorded by oracle/iteration_counts.py" % n_or
        if n_or is None:
            n_or = st64["iters"]
            src = "the %d Arnoldi steps the FP64 GPU GMRES took on this system" % n_or
        cpu = {"value": 1.0 / (sec_step * n_or), "unit": "solves/s", "cores": host_cores(), "kind": "oracle",
               "sample": "oracle GMRES(30), FP64 numpy, on the full 96x96x96 system for 1 and 3 Arnoldi steps "
                         "(difference / 2 = %.3f s per step), times %s" % (sec_step, src)}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 apply and Krylov basis; df32 (compensated f32) Gram-Schmidt; f64 residual, Givens, refinement", "data": "synthetic",
        "config": CONFIG,
        "time_to_solution_s": t_ms * 1e-3 / args.steps,
        "solve": {"iters": stats[-1]["iters"], "restarts": stats[-1]["restarts"],
                  "refinements": stats[-1]["refinements"], "reorths": stats[-1]["reorths"],
                  "rel_resid_true": stats[-1]["rel_resid_true"]},
        "fp64_gmres": {"time_to_solution_s": fp64_s, "iters": st64["iters"], "restarts": st64["restarts"],
                       "reorths": st64["reorths"],
                       "rel_resid_true": st64["rel_resid_true"], "mixed_speedup": fp64_s / (t_ms * 1e-3 / args.steps)},
        "apply": {"fp32_gbs": a32_gbs, "fp32_us": 1e3 * a32_ms, "fp32_frac_of_hbm": a32_gbs / hbm,
                  "fp64_gbs": a64_gbs, "fp64_us": 1e3 * a64_ms, "fp64_frac_of_hbm": a64_gbs / hbm,
                  "hbm_peak": hbm, "peak_kind": hbm_kind, "bytes_per_unknown": {"fp32": 16, "fp64": 32}},
        "roofline": roof,
        "roofline_source": "CUDA events around every kernel of the last timed solve",
        "apply_tile_variant": {"fp32": B.dst_get_apply_variant(mesh, B.DST_FP32)[0],
                               "fp64": B.dst_get_apply_variant(mesh, B.DST_FP64)[0]},
        "kernels": kernels,
        "batch": batch,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line))
    barrier()
    mesh_obj.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

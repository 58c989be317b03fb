#!/usr/bin/env python
"""Benchmark: time-to-solution of the spacetime FEM Dirac solve on GB300.

One step = one whole solve of the 3+1 Klein-step workload (48^3 space x 48 time
Q1 elements on [-6,6]^3 x [0,3], 4-component spinor, step potential V0 = 2.5 at
x >= 0, incident packet with momentum p0 ~ U[1,3] from the seed, 20,791,296
complex unknowns) to relative residual 1e-8: right-hand side, FP32 operator
applies inside GMRES(30), one classical Gram-Schmidt pass per step (PETSc's
GMRES default) on an FP32-stored Krylov basis in compensated arithmetic, FP64
Givens/least squares, FP64 residuals and iterative refinement.  Inputs are
resident in HBM when the timed region starts; one FP32 vector is 166 MB and the
basis 5.2 GB, beyond the 129 MB L2, so no flush is needed between steps.

Also reported on the same line: the solution's error against the FP64 oracle
at stored sample nodes; the plain-FP64-GMRES time-to-solution of the same
system and the mixed solve with native FP64 Arnoldi; the same figures for the
2+1 Zitterbewegung workload (96^2 x 96); the standalone operator-apply
bandwidth and FP64 arithmetic rate of both meshes; the roofline of the
dominant kernel class measured with CUDA events around every kernel of the
last timed solve; the end-to-end time through the C ABI with host buffers; the
FP64 CPU oracle timed on the host cores; and the throughput of the batched
solve (dst_solve_batch) on two seeded sets of independent 1+1 / 2+1 solves.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --ncu-case NAME     (small fixed launches for ncu captures)
N > 1 runs under torch.distributed.run: independent replicas, one per GPU
(rank r solves the Klein workload of seed 1 + r).
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
# GMRES(30) cycles per refinement step of the timed mixed solves: the first cycle starts
# from the FP64 residual, the next three from the inner residual with the FP32 operator
# (one FP64 residual apply per four cycles; the same Arnoldi steps on the Klein mesh)
INNER_CYCLES = 4
# Gram-Schmidt of the timed solves: one classical pass per Arnoldi step, no
# reorthogonalisation (PETSc's GMRES default); on these workloads it takes the same
# steps to the same residual as the library's default DGKS-selective second pass
ORTHO = 2
HBM_FALLBACK_GBS = 6800.0
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_FLOP_PER_CLK_SM = 4.0     # 2 FP64 FMA per clock per SM (1/64 of the FP32 rate)
FP64_PROBE_TFLOPS = 1.196      # FP64 FMA throughput measured by a probe kernel on this machine
CLASSES = ("apply64", "apply32", "cast", "project", "update", "scale", "misc", "rhs", "precond")
# DRAM read+write bytes per algorithmic byte of a kernel class, from one ncu capture of
# its kernel as committed (profiles/gram_schmidt_klein_3p1_32.md: update_tma_kernel and
# project_tma_kernel at 4.06M unknowns, nv = 11); classes without a capture of the
# current kernel are absent.
TRAFFIC_RATIO = {"update": 0.983, "project": 1.010}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", HBM_FALLBACK_GBS), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def fp64_peak_tflops():
    return SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12


def golden_sample(name):
    """Stored oracle solution at sample nodes (written by oracle/solution_sample.py)."""
    p = os.path.join(ROOT, "tests", "golden", "%s_solution_sample.json" % name)
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    d["values"] = np.array(d["re"]) + 1j * np.array(d["im"])
    d["nodes"] = np.array(d["nodes"], dtype=np.int64)
    return d


def err_vs_oracle(psi, g):
    """Relative L2 error of a device solution against the oracle's at the stored nodes."""
    if g is None:
        return None
    import torch
    idx = torch.from_numpy(g["nodes"]).to(psi.device)
    got = psi.view(-1, g["ncomp"]).index_select(0, idx).cpu().numpy()
    ref = g["values"]
    return {"rel_l2_at_sampled_nodes": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_abs_over_rms": float(np.abs(got - ref).max() / (g["norm"] / np.sqrt(g["n_unknown_nodes"]))),
            "sampled_nodes": int(len(g["nodes"])), "oracle": g.get("solver", "oracle GMRES(30) to rtol %g" % g.get("rtol", 0))}


# ---------------------------------------------------------------- CPU oracle

def oracle_seconds_per_step(w, restart=RESTART):
    """Seconds of one Arnoldi step of the oracle's GMRES(restart), as it stands, on the full mesh.

    Measured parts: one oracle operator apply on a random vector, and one modified
    Gram-Schmidt term (np.vdot and an axpy) plus one norm on full vectors; a step
    of a GMRES(m) cycle makes on average (m + 1) / 2 Gram-Schmidt terms.
    """
    from oracle import mesh as OM, operator as OOP
    om = OM.Mesh(w.d, w.n_el, w.lo, w.hi, w.bc)
    x = W.random_complex(om.n_unknowns, 3)
    v = W.random_complex(om.n_unknowns, 4)
    t0 = time.perf_counter()
    y = OOP.apply(om, w.m, w.V, x)
    t1 = time.perf_counter()
    h = np.vdot(v, y)
    y = y - h * v
    np.linalg.norm(y)
    t2 = time.perf_counter()
    return (t1 - t0) + 0.5 * (restart + 1) * (t2 - t1), t1 - t0, t2 - t1


def replica_seed(rank):
    """Seed of the bench workload on a rank: independent replicas draw independent momenta."""
    return 1 + rank


def headline_workload(rank=0):
    return W.klein_3p1(seed=replica_seed(rank))


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


def oracle_step_count():
    g = golden_sample("klein_3p1_seed1")
    return None if g is None else g["gmres30_iters_rtol_1e-8"]


def cpu_sample_text(sec_step, t_apply, t_gs, n_iter):
    return ("oracle (FP64 numpy) on the full 48^3 x 48 Klein system: one operator apply (%.2f s) + "
            "(m+1)/2 = %.1f modified Gram-Schmidt terms (vdot + axpy + norm, %.3f s each) = %.2f s per "
            "GMRES(%d) step, times the oracle's own %d-step count to 1e-8 (stacked 1+1 reduction, "
            "tests/golden/klein_3p1_seed1_solution_sample.json)"
            % (t_apply, 0.5 * (RESTART + 1), t_gs, sec_step, RESTART, n_iter))


def run_reference(args, rank):
    """The FP64 CPU oracle on the host cores, same workload / metric / unit."""
    if rank != 0:
        return
    w = headline_workload(0)
    n_iter = oracle_step_count()
    if n_iter is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle GMRES step count for klein_3p1 seed 1 not "
                          "recorded (run python -m oracle.solution_sample klein_3p1_seed1)"}))
        return
    for _ in range(args.warmup):
        oracle_seconds_per_step(w)
    per = [oracle_seconds_per_step(w) for _ in range(args.steps)]
    sec_step = statistics.mean(p[0] for p in per)
    solve_s = sec_step * n_iter
    value = 1.0 / solve_s
    sample = cpu_sample_text(sec_step, statistics.mean(p[1] for p in per), statistics.mean(p[2] for p in per), n_iter)
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
CONFIG = {"workload": "klein_3p1: 3+1 Klein step (V0 = 2.5 m at x >= 0), Q1 tesseract mesh 48^3 space x 48 time "
                      "on [-6,6]^3 x [0,3], x Dirichlet walls, y, z periodic, m = 1, NC = 4, incident packet "
                      "(sigma 0.5 at x = -2) with p0 ~ U[1,3] from seed 1 (p0 = 2.133), 20791296 complex "
                      "unknowns; GMRES(30) with FP32 operator apply inside FP64 iterative refinement to "
                      "rel. resid 1e-8",
          "unknowns": 20791296, "rtol": RTOL, "restart": RESTART, "inner_rtol": INNER_RTOL,
          "inner_cycles": INNER_CYCLES,
          "l2": "working set > L2 (FP32 vector 166 MB, FP32 GMRES basis 31 x 166 MB = 5.2 GB), no flush",
          "parallelism": "replicas (rank r: seed 1 + r)",
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


NCU_CASES = ("solve60", "solve60_klein32", "solve60_klein", "apply32_zb", "apply32_klein", "apply64_klein",
             "apply32_klein_zcol", "apply64_klein_zcol", "sweep_zb", "unet_zb48")


def run_ncu_case(case):
    """Small fixed launches for ncu captures (nothing timed, nothing printed as a bench line).

    solve60: the first 60 Arnoldi steps (two GMRES(30) cycles) of the 2+1 mixed solve
    (96^2 x 96); solve60_klein32 / solve60_klein: the same on the 3+1 Klein workload at
    32^3 x 32 (4.06M unknowns) or 48^3 x 48 (the bench mesh, seed 1), with the bench's
    one-pass Gram-Schmidt;
    apply32_zb / apply32_klein / apply64_klein: 12 operator applies on the 96^2 x 96 mesh or
    the 48^3 x 48 3+1 Klein mesh, over rotating buffers (tile variant 0);
    apply32_klein_zcol / apply64_klein_zcol: the same with the z-column kernel (variant 1);
    sweep_zb: 6 Crank-Nicolson sweeps on the 96^2 x 96 mesh;
    unet_zb48: 4 forward passes of the U-Net on the 48^2 x 48 grid.
    """
    import torch
    from paper_2103_14588_gb300 import binding as B
    torch.cuda.set_device(0)
    if case == "solve60_klein32":
        w = W.klein_3p1(n=32, nt=32, p0=1.05)
    elif case == "solve60_klein":
        w = W.klein_3p1(seed=1)
    elif case == "unet_zb48":
        w = W.zb_2p1(n=48, nt=48)
    else:
        w = W.klein_3p1(p0=1.05) if "klein" in case else W.zb_2p1()
    with B.Mesh.from_workload(w) as m:
        if case.startswith("solve60"):
            psi = torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda")
            st = B.dst_solve(m.handle, {"restart": RESTART, "rtol": RTOL, "max_iters": 60, "mixed_precision": 1,
                                        "ortho": ORTHO}, psi)
            torch.cuda.synchronize()
            print("solve60: %d steps, status %d, %d second passes" % (st["iters"], st["status"], st["reorths"]))
        elif case == "sweep_zb":
            v = torch.randn(m.n_unknowns, dtype=torch.complex64, device="cuda")
            z = torch.empty_like(v)
            for _ in range(6):
                B.dst_precond_apply(m.handle, B.DST_PRECOND_CN_SWEEP, v, z)
            torch.cuda.synchronize()
            print("sweep_zb: 6 sweeps")
        elif case == "unet_zb48":
            net = B.UNet(m.handle)
            net.set_params(np.random.default_rng(1).standard_normal(net.num_params).astype(np.float32) * 0.05)
            v = torch.randn(m.n_unknowns, dtype=torch.complex64, device="cuda")
            z = torch.empty_like(v)
            for _ in range(4):
                net.forward(v, z)
            torch.cuda.synchronize()
            net.close()
            print("unet_zb48: 4 forward passes")
        else:
            prec = B.DST_FP32 if case.startswith("apply32") else B.DST_FP64
            if case.endswith("_zcol"):
                B.dst_set_apply_variant(m.handle, prec, 1)
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


def timed_solve(torch, B, mesh, opts, psi):
    """One solve bracketed by CUDA events on the current stream; (seconds, stats)."""
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    st = B.dst_solve(mesh, opts, psi)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) * 1e-3, st


def apply_figures(torch, B, mesh_obj, st_prof, hbm):
    """Standalone FP32 / FP64 apply: time, HBM GB/s and the FP64 arithmetic rate
    (algorithmic flops per apply from the solver's accounting)."""
    n = mesh_obj.n_unknowns
    a32_ms, a32_gbs = time_apply(torch, B, mesh_obj.handle, B.DST_FP32, n)
    a64_ms, a64_gbs = time_apply(torch, B, mesh_obj.handle, B.DST_FP64, n)
    i64, i32 = CLASSES.index("apply64"), CLASSES.index("apply32")
    fl = None
    for i in (i64, i32):
        if st_prof["kernel_launches"][i] > 0:
            fl = st_prof["kernel_flops"][i] / st_prof["kernel_launches"][i]
            break
    out = {"fp32_gbs": a32_gbs, "fp32_us": 1e3 * a32_ms, "fp32_frac_of_hbm": a32_gbs / hbm,
           "fp64_gbs": a64_gbs, "fp64_us": 1e3 * a64_ms, "fp64_frac_of_hbm": a64_gbs / hbm,
           "bytes_per_unknown": {"fp32": 16, "fp64": 32}}
    if fl:
        tf64 = fl / (a64_ms * 1e-3) / 1e12
        out.update({"flops_per_apply": fl, "fp64_tflops": tf64, "fp64_frac_of_fp64_peak": tf64 / fp64_peak_tflops(),
                    "fp64_frac_of_probe": tf64 / FP64_PROBE_TFLOPS,
                    "fp64_peak_kind": "152 SMs x 4 FLOP/clk x 2070 MHz = %.3f TFLOP/s (derived); a probe kernel "
                                      "measured %.3f" % (fp64_peak_tflops(), FP64_PROBE_TFLOPS),
                    "fp32_tflops": fl / (a32_ms * 1e-3) / 1e12})
    return out


def run_batch_stated(torch, B, count, cap=4000):
    """A sample of the batched workload at its stated shape: every axis (time included) drawn
    from 32..256 for 1+1 and 2+1 alike (workloads.batch_instances with the full ranges), solved
    by one dst_solve_batch call with a cap of `cap` Arnoldi steps per instance; converged and
    capped instances are reported separately."""
    ws = W.batch_instances(count, 4, n1=(32, 256), n2=(32, 256))
    meshes = [B.Mesh.from_workload(w) for w in ws]
    psis = [torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda") for m in meshes]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, sts = B.dst_solve_batch([m.handle for m in meshes], {"rtol": RTOL, "max_iters": cap, "max_refine": 100000},
                                psis)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    conv = [i for i, st in enumerate(sts) if st["status"] == 0]
    out = {"instances": count, "cap_arnoldi_steps": cap, "wall_s": tb,
           "unknowns": [int(m.n_unknowns) for m in meshes], "dims": [w.d for w in ws],
           "converged": len(conv), "capped": count - len(conv),
           "converged_solves_per_s": len(conv) / tb,
           "converged_unknowns": int(sum(meshes[i].n_unknowns for i in conv)),
           "arnoldi_steps": int(sum(st["iters"] for st in sts))}
    for m in meshes:
        m.close()
    return out


def run_precond_bench(torch, B):
    """Flexible GMRES with the Crank-Nicolson sweep, with the sweep plus the learned
    U-Net correction (trained here on pairs generated on the GPU) and with node-block
    Jacobi, against the plain mixed solve, on the 2+1 Zitterbewegung packet at 48^3
    (where the sweep preconditions) and at 96^3 (where its quality is gone:
    ||A M v - v|| ~ ||v||)."""
    import numpy as _np
    out = {}
    base = {"restart": RESTART, "rtol": RTOL, "max_iters": 2000, "mixed_precision": 1, "inner_rtol": INNER_RTOL}
    for n in (48, 96):
        w = W.zb_2p1(n=n, nt=n)
        rec = {"unknowns": None}
        with B.Mesh.from_workload(w) as m:
            rec["unknowns"] = m.n_unknowns
            psi = torch.zeros(m.n_unknowns, dtype=torch.complex128, device="cuda")
            runs = [("plain", dict(base, ortho=ORTHO)), ("cn_sweep", dict(base, precond=B.DST_PRECOND_CN_SWEEP)),
                    ("block_jacobi", dict(base, precond=B.DST_PRECOND_BLOCK_JACOBI))]
            net = None
            if n == 48:
                net = B.UNet(m.handle)
                from_zero = net.get_params()
                rng = _np.random.default_rng(3)
                # He-normal hidden layers, zero output layer: training starts from the sweep itself
                params = from_zero.copy()
                params[:] = rng.standard_normal(params.size).astype(_np.float32) * 0.05
                params[-(2 * m.ncomp * 16 + 2 * m.ncomp):] = 0.0
                net.set_params(params)
                t0 = time.perf_counter()
                losses = net.train(m.handle, steps=600, lr=5e-4, seed=17)
                rec["training"] = {"steps": 600, "seconds": time.perf_counter() - t0,
                                   "loss_first_20": float(_np.mean(losses[:20])),
                                   "loss_last_20": float(_np.mean(losses[-20:])),
                                   "output_scale": net.output_scale()}
                B.dst_set_learned_precond(m.handle, net)
                runs.append(("cn_sweep_learned", dict(base, precond=B.DST_PRECOND_CN_LEARNED)))
            for name, o in runs:
                B.dst_solve(m.handle, dict(o, max_iters=60), psi)
                t, st = timed_solve(torch, B, m.handle, o, psi)
                rec[name] = {"time_s": t, "iters": st["iters"], "status": st["status"],
                             "rel_resid_true": st["rel_resid_true"]}
            if net is not None:
                B.dst_set_learned_precond(m.handle, None)
                net.close()
        out["zb_2p1_%d" % n] = rec
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve throughput cases")
    ap.add_argument("--no-precond", action="store_true", help="skip the preconditioned-solve comparison")
    ap.add_argument("--batch-stated", type=int, default=0,
                    help="only solve this many batched instances drawn at the stated 32..256 shape and exit")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed solves (no FP64 comparisons, second workload, applies)")
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
    if args.batch_stated:
        import torch
        from paper_2103_14588_gb300 import binding as B
        torch.cuda.set_device(local)
        print(json.dumps({"batch_stated_shape": run_batch_stated(torch, B, args.batch_stated)}))
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

    w = headline_workload(rank)
    mesh_obj = B.Mesh.from_workload(w)
    mesh = mesh_obj.handle
    n = mesh_obj.n_unknowns
    psi = torch.zeros(n, dtype=torch.complex128, device="cuda")
    # one classical Gram-Schmidt pass per step (PETSc's GMRES default, ORTHO) in every timed
    # solve, mixed and plain FP64 alike
    opts = {"restart": RESTART, "rtol": RTOL, "max_iters": 200000, "mixed_precision": 1,
            "inner_rtol": INNER_RTOL, "max_refine": 100000, "ortho": ORTHO, "inner_cycles": INNER_CYCLES}

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
    for st_ in stats:
        if st_["status"] != 0:
            raise RuntimeError("timed solve did not converge: %s" % st_)

    # per-class kernel accounting over the profiled (last) timed solve; launches over all
    tot = {k: [0.0, 0.0, 0.0, 0.0] for k in CLASSES}
    launches = sum(int(st_["launches"]) for st_ in stats)
    st_prof = stats[-1]
    for i, k in enumerate(CLASSES):
        tot[k] = [st_prof["kernel_ms"][i], st_prof["kernel_launches"][i], st_prof["kernel_bytes"][i],
                  st_prof["kernel_flops"][i]]
    kms = sum(v[0] for v in tot.values())

    if rank != 0:
        barrier()
        return

    hbm, hbm_kind = measured_peaks()
    clocks = clk.summary()
    err_headline = err_vs_oracle(psi, golden_sample("klein_3p1_seed1"))
    dom = max(CLASSES, key=lambda k: tot[k][0])
    d_ms, d_l, d_b, d_f = tot[dom]
    if dom == "apply64" and d_f > 0:
        ach = d_f / (d_ms * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp64_peak_tflops(), "unit": "TFLOP/s",
                "frac": ach / fp64_peak_tflops(), "traffic": None,
                "peak_kind": "FP64 FMA pipe: 152 SMs x 4 FLOP/clk x 2070 MHz (derived; probe measured %.3f)"
                             % FP64_PROBE_TFLOPS,
                "achieved_gbs": d_b / (d_ms * 1e-3) / 1e9, "hbm_frac": d_b / (d_ms * 1e-3) / 1e9 / hbm,
                "avg_launch_us": 1e3 * d_ms / max(d_l, 1)}
    else:
        ach = d_b / (d_ms * 1e-3) / 1e9
        launches_ran = d_l
        if dom in ("project", "update"):
            # per step one first-pass launch (a gated second pass moves data only when it runs)
            launches_ran = st_prof["iters"] + st_prof["reorths"] + (st_prof["restarts"] if dom == "update" else 0)
        traffic = TRAFFIC_RATIO[dom] * d_b / max(launches_ran, 1) if TRAFFIC_RATIO.get(dom) else None
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "traffic_unit": "bytes per launch", "peak_kind": hbm_kind,
                "algorithmic_bytes_per_launch": d_b / max(launches_ran, 1),
                "avg_launch_us": 1e3 * d_ms / max(launches_ran, 1)}
    kernels = {k: {"ms_share": (v[0] / kms if kms else None), "launches": int(v[1]),
                   "GBps": (v[2] / (v[0] * 1e-3) / 1e9 if v[0] else None),
                   "TFLOPps": (v[3] / (v[0] * 1e-3) / 1e12 if v[0] and v[3] else None)} for k, v in tot.items() if v[1]}

    extras = {}
    if not args.no_extras:
        # native FP64 Arnoldi (mixed_ortho = 1, library-default DGKS second pass) inside the same
        # mixed refinement, and plain FP64 GMRES(30) on the same system
        psi2 = torch.zeros_like(psi)
        t_fa, st_fa = timed_solve(torch, B, mesh, dict(opts, mixed_ortho=1, ortho=0), psi2)
        t_1c, st_1c = timed_solve(torch, B, mesh, dict(opts, inner_cycles=1), psi2)
        extras["one_cycle_per_refinement"] = {"time_to_solution_s": t_1c, "iters": st_1c["iters"],
                                              "refinements": st_1c["refinements"],
                                              "rel_resid_true": st_1c["rel_resid_true"],
                                              "vs_headline": t_1c / (t_ms * 1e-3 / args.steps),
                                              "what": "the headline solve with an FP64 residual after every "
                                                      "GMRES(30) cycle (inner_cycles = 1)"}
        t64, st64 = timed_solve(torch, B, mesh, {"restart": RESTART, "rtol": RTOL, "max_iters": 200000,
                                                 "mixed_precision": 0, "ortho": ORTHO}, psi2)
        extras["fp64_arnoldi_mixed"] = {"time_to_solution_s": t_fa, "iters": st_fa["iters"],
                                        "reorths": st_fa["reorths"], "rel_resid_true": st_fa["rel_resid_true"],
                                        "vs_headline": t_fa / (t_ms * 1e-3 / args.steps),
                                        "what": "mixed refinement with the Krylov basis and Gram-Schmidt in native "
                                                "FP64 (DGKS-selective second pass)"}
        extras["fp64_gmres"] = {"time_to_solution_s": t64, "iters": st64["iters"], "restarts": st64["restarts"],
                                "reorths": st64["reorths"], "rel_resid_true": st64["rel_resid_true"],
                                "err_vs_oracle": err_vs_oracle(psi2, golden_sample("klein_3p1_seed1")),
                                "mixed_speedup": t64 / (t_ms * 1e-3 / args.steps)}
        del psi2
        extras["apply"] = dict(apply_figures(torch, B, mesh_obj, st_prof, hbm), hbm_peak=hbm, peak_kind=hbm_kind)
        # the 2+1 Zitterbewegung workload (96^2 x 96, 1,769,472 unknowns)
        wz = W.zb_2p1()
        with B.Mesh.from_workload(wz) as mz:
            pz = torch.zeros(mz.n_unknowns, dtype=torch.complex128, device="cuda")
            B.dst_solve(mz.handle, opts, pz)
            zt = [timed_solve(torch, B, mz.handle, opts, pz) for _ in range(3)]
            tz = statistics.median(t for t, _ in zt)
            stz = zt[-1][1]
            ezb = err_vs_oracle(pz, golden_sample("zb_2p1"))
            _, stzp = timed_solve(torch, B, mz.handle, dict(opts, profile=1), pz)
            pz2 = torch.zeros_like(pz)
            tz64, stz64 = timed_solve(torch, B, mz.handle, {"restart": RESTART, "rtol": RTOL, "max_iters": 200000,
                                                            "mixed_precision": 0, "ortho": ORTHO}, pz2)
            extras["zb_2p1"] = {"unknowns": mz.n_unknowns, "time_to_solution_s": tz, "solves_per_s": 1.0 / tz,
                                "iters": stz["iters"], "rel_resid_true": stz["rel_resid_true"], "err_vs_oracle": ezb,
                                "fp64_gmres": {"time_to_solution_s": tz64, "iters": stz64["iters"],
                                               "rel_resid_true": stz64["rel_resid_true"],
                                               "err_vs_oracle": err_vs_oracle(pz2, golden_sample("zb_2p1"))},
                                "mixed_speedup": tz64 / tz,
                                "apply": apply_figures(torch, B, mz, stzp, hbm)}

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
    precond = None if args.no_precond else run_precond_bench(torch, B)

    cpu = None
    if not args.no_cpu_baseline:
        n_or = oracle_step_count()
        src_iters = n_or
        if n_or is None:
            n_or = stats[-1]["iters"]
        sec_step, t_apply, t_gs = oracle_seconds_per_step(w)
        cpu = {"value": 1.0 / (sec_step * n_or), "unit": "solves/s", "cores": host_cores(), "kind": "oracle",
               "sample": cpu_sample_text(sec_step, t_apply, t_gs, n_or) +
                         ("" if src_iters else " (count: the GPU solve's own steps)")}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 apply and Krylov basis; df32 (compensated f32) Gram-Schmidt; f64 residual, Givens, refinement",
        "data": "synthetic", "config": CONFIG,
        "time_to_solution_s": t_ms * 1e-3 / args.steps,
        "solve": {"iters": stats[-1]["iters"], "restarts": stats[-1]["restarts"],
                  "refinements": stats[-1]["refinements"], "reorths": stats[-1]["reorths"],
                  "rel_resid_true": stats[-1]["rel_resid_true"]},
        "err_vs_oracle": err_headline,
        "roofline": roof,
        "roofline_source": "CUDA events around every kernel of the last timed solve",
        "apply_tile_variant": {"fp32": B.dst_get_apply_variant(mesh, B.DST_FP32)[0],
                               "fp64": B.dst_get_apply_variant(mesh, B.DST_FP64)[0]},
        "kernels": kernels,
        "batch": batch,
        "preconditioners": precond,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    line.update(extras)
    print(json.dumps(line))
    barrier()
    mesh_obj.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

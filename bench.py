#!/usr/bin/env python
"""Throughput of the preconditioned H-matrix EFIE solve (arXiv 2111.13483) on one GB300.

One step = one pass of the whole hot path over a batch of B plane-wave right-hand sides
on the 30,720-unknown PEC sphere (icosphere subdivision 5, radius 2.4 lambda, leaf 64,
eta = 1, ACA 1e-3): precond_setup (pivot inverses, coefficient panels, Schur updates of
Sec. 3.1-3.2 in reverse Cuthill-McKee order) followed by solve_device for all B columns.
Default (--precision 1): complex-FP32 Schur products and Eq. 28 operator inside an FP64
refinement loop that stops at ||V - Z I|| / ||V|| <= 1e-5 (FP64 pivots, Arnoldi, Givens,
residual) -- the loosest setting whose solutions stay within 1e-4 of the FP64 solution --
with the fill-in blocks compressed at fill_tol 1e-2 (Sec. 3.4).  --precision 0: the
paper's FP64 form, GMRES(30) to a preconditioned relative residual.  The H-matrix and the
right-hand sides are resident in HBM before timing; every step refactors from the
resident near-field blocks.  value = RHS solved per second over all ranks.

Beside the headline, outside its timed region: the error of the timed solutions against
the FP64 solution of Z I = V (error_vs_fp64), and the plain FP64 form -- FP64 setup and
GMRES(30) to a preconditioned residual of 1e-4, one right-hand side per solve -- with its
setup ms, RHS/s and error (fp64), and the mixed-over-FP64 throughput ratio.

e2e: the same step through the public API from pinned host memory: hmat_create (upload
of near blocks, far factors and index maps), precond_setup, solve (host V -> host I),
hmat_destroy.

--impl reference runs the CPU oracle (numpy, the paper's algorithm step by step) on a
bounded sample of the same step and extrapolates to a full step with the oracle's own
GMRES iteration count (see cpu_baseline.sample); the 1,920-unknown sphere is solved by the
oracle in full, at one BLAS thread and at every host core, as a measured anchor.

Multi-GPU: replicas (each rank solves its own batch on its own geometry copy; no
collective on the data path), weak scaling; barrier + max over ranks around the timed
region.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "sphere30720": "PEC sphere r=2.4 lambda, icosphere d=5, 30720 RWG unknowns, leaf 64, eta 1, ACA 1e-3",
    "plate29800": "PEC plate 10 x 10 lambda, 100 x 100 grid jittered +-0.1h, 29800 RWG unknowns, leaf 64, eta 1, "
                  "ACA 1e-3",
    "sphere122880": "PEC sphere r=5 lambda, icosphere d=6, 122880 RWG unknowns, leaf 64, eta 1, ACA 1e-4",
    "sphere7680": "PEC sphere r=1.2 lambda, icosphere d=4, 7680 RWG unknowns, leaf 64, eta 1, ACA 1e-3",
}
ORDERINGS = {0: "cluster (no)", 1: "reverse Cuthill-McKee", 2: "Sloan"}
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12     # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 FMA/clk/SM x 2 flop x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere30720")
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-5,
                    help="mixed precision: ||V - Z I|| / ||V|| at which the outer FP64 loop stops (1e-5 is the "
                         "loosest setting whose solutions stay within 1e-4 of the FP64 solution on the sphere); "
                         "FP64: the preconditioned residual")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--fill-tol", type=float, default=1e-2)
    ap.add_argument("--fp64-rhs", type=int, default=4,
                    help="right-hand sides of the plain FP64 one-at-a-time solve measured beside the headline "
                         "(Eq. 28 GMRES to a preconditioned residual of --fp64-tol); 0 = skip")
    ap.add_argument("--fp64-tol", type=float, default=1e-6,
                    help="preconditioned residual of the FP64 forms (the one-RHS leg; --table7): 1e-6 with "
                         "fill_tol 0 puts the FP64 solutions within 1e-4 of the solution of Z I = V, the bar "
                         "the mixed path is held to")
    ap.add_argument("--fp64-fill-tol", type=float, default=0.0,
                    help="fill_tol of the FP64 one-RHS leg (0: exact factors, so that it solves Z I = V)")
    ap.add_argument("--cpu-anchor-run", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--ordering", type=int, default=1, choices=[0, 1, 2],
                    help="Algorithm 1 reordering: 0 none, 1 reverse Cuthill-McKee, 2 Sloan")
    ap.add_argument("--table7", action="store_true",
                    help="Sec. 5.2 Table 7 style comparison on the workload (FP64): Schur complement vs block "
                         "Jacobi, t_sp, p, t_mm, t_mp and t_total = t_sm + t_sp + p n (t_mm + t_mp) (Eq. 46) for "
                         "n = --nrhs right-hand sides; prints one JSON line")
    ap.add_argument("--compare-orderings", action="store_true",
                    help="Sec. 3.3 Tables 3-4 style comparison on the workload: setup ms, coefficient entries, "
                         "operator ms and iterations for no ordering, RCM and Sloan; prints one JSON line")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1],
                    help="0: complex FP64; 1: complex-FP32 operator inside FP64 refinement")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--serve-requests", type=int, default=360,
                    help="requests of the serving leg (monostatic plane waves, phi in 1-degree steps, Poisson "
                         "arrivals at 0.8x the measured RHS/s: a steady state of about half a minute); 0 = skip")
    ap.add_argument("--serve-full", action="store_true",
                    help="serving on two resident geometries (sphere30720 + plate29800), 360 requests each, "
                         "offered at 0.5/0.8/1.0x the measured throughput")
    ap.add_argument("--rhs", default="sweep", choices=["sweep", "random"],
                    help="right-hand sides: the monostatic phi sweep, or directions uniform on the sphere "
                         "with random polarisation (seed 3)")
    ap.add_argument("--build", default="host", choices=["host", "gpu"],
                    help="where the H-matrix comes from: the generator's host build (cached) or the GPU "
                         "EFIE fill and ACA (Sec. 2, Eqs. 7, 9-10)")
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--profile-op", type=int, default=0,
                    help="profiling case: set up the workload, then apply the operator of Eq. 28 this many "
                         "times to --nrhs columns (complex FP32 when --precision 1) and exit; no bench line")
    ap.add_argument("--profile-build", action="store_true",
                    help="profiling case: build the workload's H-matrix on the GPU (EFIE fill and ACA, Sec. 2) "
                         "twice, print the timings of the second and exit; no bench line")
    ap.add_argument("--error-check", type=int, default=4,
                    help="columns re-solved with the FP64 path at tol 1e-10 to state the relative solution error "
                         "of the measured (mixed) solutions; 0 = skip")
    ap.add_argument("--schedule", default="0,0",
                    help="sweep schedule 'groups,kind[,tile]' for --profile-op (0,0 = tuned)")
    ap.add_argument("--update-schedule", type=int, default=0,
                    help="complex-FP32 Schur updates for --profile-op: 1 CUDA cores, 2 tensor cores, 0 default")
    ap.add_argument("--pivot-schedule", type=int, default=0,
                    help="CTAs per FP64 pivot inversion in every setup of the run: 1, or a cluster of 2, 4 "
                         "or 8; 0 = the library default")
    ap.add_argument("--profile-setup", type=int, default=0,
                    help="profiling case: run precond_setup this many times on the workload (--precision, "
                         "--fill-tol, --pivot-schedule, --update-schedule), print each setup's device ms "
                         "and the last one's per-class ms, and exit; no bench line")
    ap.add_argument("--far-schedule", type=int, default=0,
                    help="complex-FP32 far-field kind for --profile-op: 1 CUDA cores, 2 tensor cores, 0 default")
    return ap.parse_args()


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, world):
    """The largest of the ranks' values of a per-rank time (every rank gets it); the value
    itself at world size 1.  Uses the initialised process group (NCCL on the GPU machine, gloo in
    the CPU tests)."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as td
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def replica_value(B, steps, world, ms_total):
    """Whole-job RHS/s of `world` independent replicas: the columns all ranks processed
    (B per step each) over the slowest rank's time for the `steps` steps."""
    return B * steps * world / (ms_total / 1e3)


def rhs_batch(P, B, plate=False, mode="sweep", seed=3):
    """Monostatic plane waves, phi_j = 360 j / B: theta = 90 deg with VV (theta-hat)
    polarisation; for a plate (in the xy plane) the same sweep in the xz plane, i.e. the
    plate standing upright, with HH polarisation (y-hat, tangential at every angle: an
    edge-on VV wave would not excite the plate).  mode "random": B waves arriving from
    directions uniform on the sphere (theta = arccos U(-1, 1), phi = U(0, 2 pi)), polarised at
    an angle psi = U(0, pi) from theta-hat towards phi-hat (default_rng(seed))."""
    cols = []
    if mode == "random":
        rng = np.random.default_rng(seed)
        th = np.arccos(rng.uniform(-1.0, 1.0, B))
        ph = rng.uniform(0.0, 2.0 * np.pi, B)
        psi = rng.uniform(0.0, np.pi, B)
        for j in range(B):
            st, ct, sp, cp = np.sin(th[j]), np.cos(th[j]), np.sin(ph[j]), np.cos(ph[j])
            khat = -np.array([st * cp, st * sp, ct])
            that = np.array([ct * cp, ct * sp, -st])
            phat = np.array([-sp, cp, 0.0])
            cols.append(P.plane_wave(khat, np.cos(psi[j]) * that + np.sin(psi[j]) * phat))
        return np.stack(cols, axis=1)
    for j in range(B):
        ph = 2.0 * np.pi * j / B
        if plate:
            khat = -np.array([np.cos(ph), 0.0, np.sin(ph)])
            pol = np.array([0.0, 1.0, 0.0])
        else:
            khat = -np.array([np.cos(ph), np.sin(ph), 0.0])
            pol = np.array([0.0, 0.0, -1.0])
        cols.append(P.plane_wave(khat, pol))
    return np.stack(cols, axis=1)


def load_problem(name, rank, world, build="host"):
    """The workload's H-matrix: from the seeded generator's host build (cached on disk), or
    built on this rank's GPU (hm_efie_fill / hm_efie_far; timings in P.build_timings)."""
    if build == "gpu":
        import torch
        from paper_2111_13483_gb300 import hmatrix
        P, t = hmatrix.build_problem(name, device=torch.cuda.current_device())
        P.build_timings = t
        return P
    import efie_problem as ep
    if world > 1:
        import torch.distributed as td
        if rank == 0:
            P = ep.build(name)
        td.barrier()
        if rank != 0:
            P = ep.build(name)
        return P
    return ep.build(name)


class Clocks:
    """nvidia-smi sampler over the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.path = tempfile.mktemp(suffix=".csv")
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx = max(mx, float(v[2]))
            except ValueError:
                continue
            for nm, val in zip(names, v[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def fill_structure(hm, h, P):
    order = hm.hm_get_order(h)
    sz = np.diff(P.leaf_ptr)[order].astype(np.int64)
    ptr, idx = hm.hm_get_fill(h)
    nnzL = 0
    upd = 0.0
    upd_launch = 0
    for k in range(len(sz)):
        S = idx[ptr[k]:ptr[k + 1]]
        if len(S) == 0:
            continue
        s = sz[S]
        nnzL += int(sz[k] * s.sum())
        cs = np.cumsum(s)
        upd += 8.0 * sz[k] * float(np.sum(s * cs))          # sum_{i>=j} n_i n_k n_j
        upd_launch += 1
    return {"nnzL": nnzL, "diag": int(np.sum(sz * sz)), "update_flops": upd, "update_launches": upd_launch,
            "order": order, "sz": sz, "ptr": ptr, "idx": idx}


def roofline(prof, fs, stats, n, precision):
    """Roofline entry for the kernel class with the largest device time.  The algorithmic work
    uses the right-hand-side columns the class actually processed (the slot engine packs
    fewer columns as solves finish); the bound is the one the arithmetic intensity selects
    against the ridge of the measured peaks."""
    cls = max(prof, key=lambda c: prof[c][2])
    launches, timed, ms, cols = prof[cls]
    t_s = ms / 1e3
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "when" in peaks else "fallback 6.8 TB/s (of fallback)"
    E = 8.0 if precision == 1 else 16.0
    alu_peak = FP32_PEAK_TFLOPS if precision == 1 else FP64_PEAK_TFLOPS
    alu_src = ("derived: 152 SMs x %d %s FMA/clk x 2 flop x 2.07 GHz" % ((128, "FP32") if precision == 1 else (2, "FP64")))

    def entry(flops, bytes_, extra, bound=None):
        # flops, bytes_: totals over the class's timed launches; bound: fixed, else the one the
        # intensity selects against the ridge
        ridge = alu_peak * 1e12 / (peaks["hbm_gbs"] * 1e9)
        d = {"avg_launch_ms": ms / max(timed, 1), "launches": launches, "rhs_columns": cols,
             "flops_per_launch": flops / max(launches, 1), "bytes_per_launch": bytes_ / max(launches, 1),
             "intensity_flop_per_byte": flops / max(bytes_, 1.0), "traffic": None,
             "alu_achieved_tflops": flops / t_s / 1e12, "alu_peak_tflops": alu_peak,
             "alu_frac": flops / t_s / 1e12 / alu_peak, "alu_peak_source": alu_src}
        if bound == "alu" or (bound is None and flops / max(bytes_, 1.0) > ridge):
            d.update({"bound": "alu", "achieved": flops / t_s / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                      "frac": flops / t_s / 1e12 / alu_peak, "peak_source": alu_src})
        else:
            d.update({"bound": "hbm", "achieved": bytes_ / t_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": bytes_ / t_s / 1e9 / peaks["hbm_gbs"], "peak_source": hbm_src})
        d.update(extra)
        return d

    if cls == "update":
        return cls, entry(fs["update_flops"] * launches / fs["update_launches"],
                          E * fs["nnzL"] * 3.0 * launches / fs["update_launches"], {})
    # the solve's operator (sweeps, far field) against HBM bandwidth, the bound the scope table
    # fixes for it (matrix bytes read once per launch); the FP32-ALU figures ride along
    if cls in ("sweep_fwd", "sweep_bwd"):
        # per launch: the stored coefficients once (dense blocks, and the factors of the
        # compressed fill-in blocks: each stored entry is one complex MAC per column), the input
        # and output vectors of its columns
        ce = stats["coef_entries"]
        return cls, entry(8.0 * ce * cols, E * (ce * launches + 2.0 * n * cols),
                          {"coef_entries": ce, "coef_entries_dense": fs["nnzL"]}, bound="hbm")
    if cls in ("far1", "far2"):
        # far2 counts two launches per product (partial products + their sum)
        per = launches if cls == "far1" else launches / 2
        return cls, entry(8.0 * stats["far_entries"] * cols, E * (stats["far_entries"] * per + 2.0 * n * cols), {},
                          bound="hbm")
    return cls, entry(0.0, 16.0 * n * max(cols, 1) * 2, {})


def sweep_code_digest(texts=None):
    """Key of the sweep kernels' code: sha256 (first 16 hex digits) of ops.cu + tile.cuh +
    cluster.cuh with comments and whitespace removed, so that an edit of comments keeps a
    measurement valid and any code change invalidates it."""
    import hashlib
    import re
    if texts is None:
        texts = [open(os.path.join(ROOT, "paper_2111_13483_gb300", "csrc", f)).read()
                 for f in ("ops.cu", "tile.cuh", "cluster.cuh")]
    code = "".join(texts)
    code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
    code = re.sub(r"//[^\n]*", " ", code)
    code = re.sub(r"\s+", " ", code).strip()
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def traffic_record(cls, workload, precision):
    """Measured DRAM traffic of `cls` from a profile summary taken on the current code of that
    kernel (sweep_code_digest; else None).  A record measured on the workload itself gives the
    bytes of one launch; one measured on a smaller case of the same kernel gives the ratio of
    measured to algorithmic bytes, to be scaled by the algorithmic bytes of this workload's
    launch.  Returns (bytes or None, ratio or None, columns, source file, measured-on)."""
    import glob
    digest = sweep_code_digest()
    best = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            if not line.startswith("traffic-record:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:])
            if kv.get("class") != cls or int(kv.get("precision", -1)) != precision or kv.get("source") != digest:
                continue
            rec = (int(kv["bytes"]) if "bytes" in kv else None, float(kv["ratio"]) if "ratio" in kv else None,
                   int(kv["columns"]), os.path.relpath(path, ROOT), kv.get("workload"))
            if kv.get("workload") == workload and rec[0] is not None:
                return rec
            if rec[1] is not None:
                best = rec
    return best


def serving_run(hm, serve, h, P, requests, rate, tol, restart, seed_rhs=2, seed_arr=1, plate=False):
    """Poisson-arrival serving on one resident geometry: requests (monostatic plane waves,
    host memory) submitted at their arrival times, continuous batching up to 64 slots."""
    rhs = [V for _, _, V in serve.monostatic_requests(P, requests, seed_rhs, phi_step_deg=360.0 / requests,
                                                      plane="xz" if plate else "xy")]
    arr = serve.poisson_arrivals(requests, rate, seed_arr)
    srv = serve.Server({"g": h}, max_slots=64, tol=tol, restart=restart)
    t0 = time.perf_counter()
    try:
        reqs = serve.run_stream(srv, [("g", arr, rhs)])
    finally:
        srv.close()
    wall = max(r.t_done for r in reqs) - min(r.t_submit for r in reqs)
    s = serve.latency_summary(reqs)
    s.update({"offered_rps": rate, "achieved_rhs_per_s": requests / wall, "wall_s": wall,
              "not_converged": sum(r.status != 0 for r in reqs), "slots": srv.slots("g")})
    # steady state: the completions between the 10th and the 90th percentile of completion
    # times (the ramp-up and the drain at the end left out)
    done = sorted(r.t_done for r in reqs)
    a, b = done[len(done) // 10], done[(9 * len(done)) // 10]
    mid = [r for r in reqs if a <= r.t_done <= b]
    if b > a and len(mid) > 1:
        st = serve.latency_summary(mid)
        st.update({"achieved_rhs_per_s": (len(mid) - 1) / (b - a), "window_s": b - a})
        s["steady"] = st
    del t0
    return s


def oracle_iterations(workload, fill_tol, tol, restart):
    """The oracle's own GMRES(restart) iteration counts on a workload at a preconditioned
    tolerance (oracle/iterations.json, written by oracle/record_iterations.py), or None."""
    path = os.path.join(ROOT, "oracle", "iterations.json")
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get("%s fill_tol=%g tol=%g restart=%d" % (workload, fill_tol, tol, restart))


def cpu_anchor_run():
    """The 1,920-unknown sphere (k = -z, p = x) solved in full by the oracle in this process:
    RCM, Schur setup with fill_tol 1e-2, GMRES(30) to a preconditioned residual of 1e-4.
    Prints one JSON object (measured wall times, iterations, BLAS threads)."""
    import efie_problem as ep
    from oracle import krylov, ordering, schur
    P = ep.build("sphere1920")
    b = P.plane_wave([0.0, 0.0, -1.0], [1.0, 0.0, 0.0])
    t0 = time.perf_counter()
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    S = krylov.System(P, schur.setup(P, order, fill_tol=1e-2))
    t1 = time.perf_counter()
    x, it, rr, ok = krylov.solve(S, b, tol=1e-4, restart=30)
    t2 = time.perf_counter()
    print(json.dumps({"workload": "sphere1920 (1920 unknowns), k=-z p=x, fill_tol 1e-2, GMRES(30) tol 1e-4",
                      "setup_s": t1 - t0, "solve_s": t2 - t1, "iters": int(it), "converged": bool(ok),
                      "rhs_per_s_solve_only": 1.0 / (t2 - t1), "rhs_per_s_with_setup": 1.0 / (t2 - t0),
                      "blas_threads": int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))}), flush=True)


def cpu_anchor(threads):
    """cpu_anchor_run in a fresh interpreter with `threads` BLAS threads (measured, not
    extrapolated); None if it fails."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    try:
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-anchor-run"], env=env,
                             capture_output=True, text=True, timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1])
    except Exception as ex:   # reported, not fatal: the anchor is context for the extrapolation
        return {"error": repr(ex)[:200]}


def oracle_iters_for(workload, args):
    """(mean oracle iterations per RHS, description of their source)."""
    rec = oracle_iterations(workload, args.fill_tol, 1e-4, args.restart)
    if rec is None:
        return float("nan"), "no recorded oracle iteration count for this workload"
    return float(np.mean(rec["iters"])), "oracle GMRES(%d) to 1e-4 on %s (oracle/iterations.json): %s" % (
        args.restart, "; ".join(rec["rhs"]), rec["iters"])


def cpu_baseline_entry(P, workload, B, args, budget_s, sample=None):
    """The oracle's CPU baseline of one step: a bounded sample of the step extrapolated to the
    full step (one BLAS thread), with the oracle's own iteration count, plus the measured full
    oracle solve of the 1,920-unknown sphere at one thread and at every host core.  `sample`:
    an already measured (seconds per step, description, wall seconds) of cpu_reference."""
    iters, src = oracle_iters_for(workload, args)
    s, desc, wall = sample or cpu_reference(P, B, iters, args.fill_tol, budget_s=budget_s, iters_src=src)
    nproc = os.cpu_count() or 1
    return {"value": B / s, "unit": "RHS/s", "cores": 1, "nproc": nproc, "kind": "oracle", "measured": False,
            "extrapolated": True, "sample": desc, "oracle_iters": iters, "iters_source": src,
            "sample_wall_s": wall, "extrapolated_s_per_step": s,
            "anchor_measured": {"threads_1": cpu_anchor(1), "threads_all": cpu_anchor(nproc)}}


def cpu_reference(P, B, iters_per_rhs, fill_tol, budget_s=15.0, iters_src=""):
    """The oracle on a bounded sample of one step, extrapolated to the full step.
    Returns (seconds per full step, description, wall seconds of the sample)."""
    from oracle import krylov, ordering, schur
    t0 = time.perf_counter()
    nl = len(P.leaf_ptr) - 1
    order = ordering.rcm(nl, list(zip(P.near_t.tolist(), P.near_s.tolist())))
    pos = np.empty(nl, dtype=np.int64)
    pos[order] = np.arange(nl)
    pairs = [(int(pos[t]), int(pos[s])) for t, s in zip(P.near_t, P.near_s)]
    S = schur.symbolic_fill(nl, pairs)
    t_plan = time.perf_counter() - t0
    sz = np.diff(P.leaf_ptr)[order].astype(np.int64)
    step_flops = np.array([8.0 * (sz[k] ** 3 + sz[k] ** 2 * sz[S[k]].sum() + sz[k] *
                                  float(np.sum(sz[S[k]] * np.cumsum(sz[S[k]])))) if S[k] else 8.0 * sz[k] ** 3
                           for k in range(nl)])
    # sample the first ks elimination steps, doubling ks until the sample takes budget/2
    ks = 4
    while True:
        t1 = time.perf_counter()
        F = schur.setup(P, order, fill_tol, max_steps=ks)
        t_samp = time.perf_counter() - t1
        if t_samp >= 0.5 * budget_s or ks >= nl:
            break
        ks = min(nl, ks * 2)
    setup_est = t_plan + t_samp * step_flops.sum() / step_flops[:ks].sum()
    # operator application: far field (whole), sweeps and block solves over the sampled
    # blocks, scaled by stored entries
    sysm = krylov.System(P, F)
    x = np.random.default_rng(0).standard_normal(sysm.n) + 0j
    t2 = time.perf_counter()
    sysm.far_new(x)
    t_far = time.perf_counter() - t2
    v = sysm.split(x)
    W = {key: val for key, val in F.W.items()}
    t3 = time.perf_counter()
    for k in range(ks):
        for j in F.S[k]:
            v[j] = v[j] - W[(k, j)].T @ v[k]
    for k in range(ks - 1, -1, -1):
        for j in F.S[k]:
            v[k] = v[k] - W[(k, j)] @ v[j]
    import scipy.linalg as sla
    for k in range(ks):
        v[k] = sla.lu_solve(F.lu[k], F.D[k] @ v[k])
    t_sw = time.perf_counter() - t3
    nnz_s = sum(int(sz[k] * sz[S[k]].sum()) for k in range(ks))
    nnz_t = sum(int(sz[k] * sz[S[k]].sum()) for k in range(nl))
    t_iter = t_far + t_sw * nnz_t / max(nnz_s, 1)
    step = setup_est + B * (iters_per_rhs + 3) * t_iter
    desc = ("oracle (numpy, 1 BLAS thread): RCM + symbolic fill in full (%.1f s), first %d of %d Schur elimination "
            "steps (%.1f s, %.2f%% of setup flops) extrapolated by flops; one far-field product in full (%.1f s); "
            "sweeps and block solves over the sampled blocks scaled by stored coefficient entries; "
            "%d RHS x (%.1f iterations + 3 operator applications); iterations: %s"
            % (t_plan, ks, nl, t_samp, 100 * step_flops[:ks].sum() / step_flops.sum(), t_far, B, iters_per_rhs,
               iters_src))
    return step, desc, time.perf_counter() - t0


def serving_full(hm, serve, h_sphere, P_sphere, args, rate1):
    """Two resident geometries (the sphere and the 10 x 10 lambda plate), 360 monostatic
    requests each (phi 0..359 deg, VV/HH drawn per request), Poisson arrivals offered at
    0.5, 0.8 and 1.0 times the measured single-geometry throughput, split between them."""
    import efie_problem as ep
    Pp = ep.build("plate29800")
    hp = hm.hmat_create(Pp, ordering=1, fill_tol=args.fill_tol, precision=args.precision)
    hm.precond_setup(hp)
    out = []
    for f in (0.5, 0.8, 1.0):
        rate = f * rate1
        streams = []
        for name, P, seed in (("sphere", P_sphere, 3), ("plate", Pp, 4)):
            rhs = [V for _, _, V in serve.monostatic_requests(P, 360, seed, plane="xz" if name == "plate" else "xy")]
            streams.append((name, serve.poisson_arrivals(360, rate / 2, seed + 10), rhs))
        srv = serve.Server({"sphere": h_sphere, "plate": hp}, max_slots=64, tol=args.tol,
                           restarts={"sphere": args.restart, "plate": 50})
        try:
            reqs = serve.run_stream(srv, streams)
        finally:
            srv.close()
        wall = max(r.t_done for r in reqs) - min(r.t_submit for r in reqs)
        s = serve.latency_summary(reqs)
        s.update({"offered_rps": rate, "achieved_rhs_per_s": len(reqs) / wall,
                  "per_geometry": {g: serve.latency_summary([r for r in reqs if r.geom == g])
                                   for g in ("sphere", "plate")}})
        out.append(s)
    hm.hmat_destroy(hp)
    return out


def metric_name(args):
    return ("RHS/s at rel. residual 1e-4 (30,720-unk sphere)" if args.workload == "sphere30720"
            else "RHS/s at rel. residual %g (%s)" % (args.tol, args.workload))


def nvtx_range(start):
    """Push / pop the NVTX range "timed steps" (ncu --nvtx --nvtx-include "timed steps/" then
    captures exactly the timed region's launches); a no-op where NVTX is unavailable."""
    import torch
    try:
        if start:
            torch.cuda.nvtx.range_push("timed steps")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def bench_config(args, P, world=1):
    """The workload, as both arms report it (identical for the GPU arm and the reference arm)."""
    plate = args.workload.startswith("plate")
    hmat_gb = 16e-9 * (len(P.near_data) + len(P.far_U) + len(P.far_V))
    return {"workload": WORKLOADS.get(args.workload, args.workload) + "; %d plane-wave RHS per step (%s), "
                        "GMRES(%d), fill_tol %g, %s ordering; solutions within 1e-4 of the FP64 solution: the "
                        "mixed-precision path stops at ||V - Z I||/||V|| <= %g, the FP64 forms at a preconditioned "
                        "residual of %g"
                        % (args.nrhs, "directions uniform on the sphere, random polarisation (seed 3)"
                           if getattr(args, "rhs", "sweep") == "random"
                           else "xz-plane phi sweep, HH" if plate else "theta 90 deg, phi sweep, VV",
                           args.restart, args.fill_tol, ORDERINGS[args.ordering], args.tol, args.fp64_tol),
            "nrhs_per_step": args.nrhs, "parallelism": "replicas x%d" % world,
            "l2": "inputs larger than L2 (H-matrix %.2f GB resident)" % hmat_gb,
            "hmatrix_build": "GPU EFIE fill + ACA" if getattr(args, "build", "host") == "gpu"
                             else "seeded generator (host)"}


def run_reference(args):
    """The oracle arm: each step is the oracle's bounded sample of the same workload (wall
    time = ms_per_step); value = the full step's RHS/s extrapolated from the sample."""
    world, rank, local = dist()
    if rank != 0:
        return
    P = load_problem(args.workload, 0, 1)
    B = args.nrhs
    iters, src = oracle_iters_for(args.workload, args)
    walls, samples = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        samples.append(cpu_reference(P, B, iters, args.fill_tol, budget_s=8.0, iters_src=src))
        walls.append(time.perf_counter() - t0)
    val = float(np.mean([B / smp[0] for smp in samples[args.warmup:]]))
    ms = 1e3 * float(np.mean(walls[args.warmup:]))
    cpu = dict(cpu_baseline_entry(P, args.workload, B, args, 8.0, sample=samples[-1]), value=val)
    line = {"metric": metric_name(args), "value": val, "unit": "RHS/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "impl": "reference", "config": bench_config(args, P, world),
            "cpu_baseline": cpu,
            "e2e": {"value": val, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    world, rank, local = dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
    import paper_2111_13483_gb300 as hm
    P = load_problem(args.workload, rank, world, args.build)
    B = args.nrhs
    plate = args.workload.startswith("plate")
    Vh = rhs_batch(P, B, plate, args.rhs)
    stream = torch.cuda.current_stream()
    h = hm.hmat_create(P, ordering=args.ordering, fill_tol=args.fill_tol, precision=args.precision, device=local,
                       stream=stream.cuda_stream)
    hm.hmsolve.hm_set_pivot_schedule(h, args.pivot_schedule)
    stats = hm.hmat_stats(h)
    dV = torch.from_numpy(np.ascontiguousarray(Vh.T)).to("cuda")
    dI = torch.zeros_like(dV)
    iters_all = []

    def step():
        hm.precond_setup(h)
        it, rr, code = hm.solve_device(h, dV, dI, tol=args.tol, restart=args.restart, maxit=5000)
        if code != 0:
            raise RuntimeError("solve did not converge (code %d)" % code)
        iters_all.append(it.copy())

    for _ in range(args.warmup):
        step()
    stats = hm.hmat_stats(h)          # after a setup: the coefficient entries as stored
    fs = fill_structure(hm.hmsolve, h, P)
    hm.hm_profile(h, 2)
    hm.hm_profile(h, 1)
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nvtx_range(True)          # marks the timed steps for a profiler's range filter
    for _ in range(args.steps):
        step()
    nvtx_range(False)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms_total = e0.elapsed_time(e1)
    prof = hm.hm_get_profile(h)
    hm.hm_profile(h, 0)
    launches = int(sum(v[0] for v in prof.values()))
    setup_ms = hm.hmat_stats(h)["setup_ms"]
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    value = replica_value(B, args.steps, world, ms_total)
    iters = np.concatenate(iters_all[-args.steps:])
    cls, roof = roofline(prof, fs, stats, P.n, args.precision)
    tr = traffic_record(cls, args.workload, args.precision)
    if tr is not None and cls in ("sweep_fwd", "sweep_bwd"):
        E = 8.0 if args.precision == 1 else 16.0
        alg = E * (stats["coef_entries"] + 2.0 * P.n * tr[2])       # one tr[2]-column launch
        if tr[0] is not None:
            roof["traffic"] = tr[0]
            roof["traffic_note"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one %d-column launch (%s); "
                                    "algorithmic bytes of that launch %.0f" % (tr[2], tr[3], alg))
        else:
            roof["traffic"] = tr[1] * alg
            roof["traffic_note"] = ("scaled: ncu dram__bytes_read.sum + dram__bytes_write.sum over algorithmic bytes = "
                                    "%.3f on a %d-column launch of the same kernel on %s (%s), times this workload's "
                                    "algorithmic bytes of a %d-column launch (%.0f)"
                                    % (tr[1], tr[2], tr[4], tr[3], tr[2], alg))

    # ---- the plain FP64 form: setup, one RHS at a time, and the error of both forms --------
    cols = sorted(set(int(c) for c in np.linspace(0, B, max(args.error_check, args.fp64_rhs, 1),
                                                   endpoint=False)))
    fp64, err = None, None
    if rank == 0 and (args.error_check > 0 or args.fp64_rhs > 0):
        I_meas = dI.cpu().numpy()
        # reference: Z I = V solved by the FP64 path (oracle parity 1e-8) without fill
        # compression (its factorisation is exact, so the Eq. 28 system is Z I = V itself)
        g = hm.hmat_create(P, ordering=1, fill_tol=0.0, precision=0, device=local, stream=stream.cuda_stream)
        hm.precond_setup(g)
        Iref, it_r, rr_r, code_r = hm.solve(g, Vh[:, cols], tol=1e-10, restart=args.restart, maxit=20000)
        hm.hmat_destroy(g)

        def rel_err(X):
            return [float(np.linalg.norm(X[j] - Iref[:, q]) / np.linalg.norm(Iref[:, q])) for q, j in enumerate(cols)]
        if args.error_check > 0:
            e = rel_err(I_meas)
            err = {"columns": cols, "max": max(e), "median": float(np.median(e)), "per_column": e,
                   "tol": args.tol, "reference": "FP64 GPU path (oracle parity 1e-8), fill_tol 0, preconditioned "
                                                 "tol 1e-10: the solution of Z I = V",
                   "reference_converged": int(code_r) == 0}
        if args.fp64_rhs > 0:
            # the paper's arithmetic: FP64 setup (fill_tol as the headline) and GMRES(restart)
            # to a preconditioned residual of fp64_tol, one right-hand side per solve
            ft64 = args.fill_tol if args.fp64_fill_tol is None else args.fp64_fill_tol
            g = hm.hmat_create(P, ordering=args.ordering, fill_tol=ft64, precision=0, device=local,
                               stream=stream.cuda_stream)
            hm.hmsolve.hm_set_pivot_schedule(g, args.pivot_schedule)
            hm.precond_setup(g)           # first call allocates the factors
            hm.precond_setup(g)
            setup64 = hm.hmat_stats(g)["setup_ms"]
            fcols = cols[:args.fp64_rhs]
            I64 = torch.zeros_like(dI)
            ms1, its1 = [], []
            for j in fcols:
                f0 = torch.cuda.Event(enable_timing=True)
                f1 = torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                it, rr, code = hm.solve_device(g, dV[j:j + 1], I64[j:j + 1], tol=args.fp64_tol,
                                               restart=args.restart, maxit=5000)
                f1.record(stream)
                torch.cuda.synchronize()
                ms1.append(f0.elapsed_time(f1))
                its1.append(int(it[0]))
            hm.hmat_destroy(g)
            e64 = rel_err(I64.cpu().numpy())[:len(fcols)]
            per = float(np.mean(ms1)) / 1e3
            solve_only = 1.0 / per
            with_setup = B / (setup64 / 1e3 + B * per)
            fp64 = {"setup_ms": setup64, "tol_preconditioned": args.fp64_tol, "fill_tol": ft64,
                    "columns": fcols, "iters": its1, "solve_ms_per_rhs": [float(m) for m in ms1],
                    "rhs_per_s_solve_only": solve_only,
                    "rhs_per_s_with_setup": with_setup,
                    "with_setup_means": "one FP64 setup per %d right-hand sides, each solved alone" % B,
                    "error_vs_fp64": {"max": max(e64), "median": float(np.median(e64)), "per_column": e64},
                    "mixed_over_fp64_with_setup": value / with_setup,
                    "mixed_over_fp64_solve_only": (B / max((ms_step - setup_ms) / 1e3, 1e-9)) / solve_only}

    # ---- serving: Poisson arrivals into the continuous-batching engine ------------------
    serving = None
    if args.serve_requests > 0 and rank == 0:
        from paper_2111_13483_gb300 import serve
        serving = serving_run(hm, serve, h, P, args.serve_requests, 0.8 * value / world, args.tol, args.restart,
                              plate=plate)
    if args.serve_full and rank == 0:
        from paper_2111_13483_gb300 import serve
        serving = {"single": serving, "full": serving_full(hm, serve, h, P, args, value / world)}

    # ---- end to end through the public API from pinned host memory ---------------------
    e2e = None
    if args.e2e_steps > 0:
        pin = {}
        for f in ("near_data", "far_U", "far_V"):
            a = getattr(P, f)
            t = torch.empty(len(a), dtype=torch.complex128).pin_memory()
            t.numpy()[:] = a
            pin[f] = t
        Vp = torch.empty((B, P.n), dtype=torch.complex128).pin_memory()
        Vp.numpy()[:] = Vh.T
        Ip = torch.empty((B, P.n), dtype=torch.complex128).pin_memory()

        class PP:
            pass
        Q = PP()
        for f in ("perm", "leaf_ptr", "near_t", "near_s", "near_off", "far_r0", "far_r1", "far_c0", "far_c1",
                  "far_rank", "far_uoff", "far_voff"):
            setattr(Q, f, getattr(P, f))
        for f in pin:
            setattr(Q, f, pin[f].numpy())
        h2d = sum(pin[f].numel() * 16 for f in pin) + B * P.n * 16
        for f in ("perm", "leaf_ptr", "near_t", "near_s", "near_off", "far_r0", "far_r1", "far_c0", "far_c1",
                  "far_rank", "far_uoff", "far_voff"):
            h2d += getattr(P, f).nbytes
        d2h = B * P.n * 16
        del h
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.e2e_steps):
            g = hm.hmat_create(Q, ordering=args.ordering, fill_tol=args.fill_tol, precision=args.precision, device=local,
                               stream=stream.cuda_stream)
            hm.hmsolve.hm_set_pivot_schedule(g, args.pivot_schedule)
            hm.precond_setup(g)
            I, it2, rr2, code = hm.solve(g, Vp.numpy().T, tol=args.tol, restart=args.restart, maxit=5000)
            hm.hmat_destroy(g)
        a1.record(stream)
        torch.cuda.synchronize()
        ems = a0.elapsed_time(a1)
        ems = max_over_ranks(ems, world)
        e2e = {"value": replica_value(B, args.e2e_steps, world, ems), "unit": "RHS/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ems / args.e2e_steps}

    if rank != 0:
        return
    cpu = None
    if world == 1 and os.environ.get("HM_BENCH_NO_CPU") != "1":
        cpu = cpu_baseline_entry(P, args.workload, B, args, budget_s=16.0)
    line = {"metric": metric_name(args), "value": value, "unit": "RHS/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+c128" if args.precision == 1 else "c128", "data": "synthetic",
            "config": bench_config(args, P, world),
            "arithmetic": ("complex-FP32 Schur products, sweeps, far field and block solves inside an FP64 "
                           "refinement loop on ||V - Z I||/||V|| (FP64 pivots, Arnoldi, Givens, residual)"
                           if args.precision == 1 else "complex FP64 throughout (the paper's form)"),
            "coefficients_gb": (8e-9 if args.precision == 1 else 16e-9) * stats["coef_entries"],
            "fp64": fp64,
            "setup_ms": setup_ms, "iters_mean": float(np.mean(iters)), "iters_max": int(np.max(iters)),
            "solve_rhs_per_s": B / max((ms_step - setup_ms) / 1e3, 1e-9),
            "roofline": roof, "roofline_kernel": cls,
            "kernel_ms_per_step": {k: v[2] / args.steps for k, v in prof.items() if v[0]},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": ck, "serving": serving,
            "error_vs_fp64": err,
            "matrix_build_s": getattr(P, "build_timings", None),
            "stats": {k: stats[k] for k in ("n", "n_blocks", "near_entries", "far_entries", "fill_blocks",
                                            "coef_entries", "diag_entries", "bandwidth", "setup_gflop")}}
    s = json.dumps(line)
    print(s, flush=True)
    if args.json_out:
        with open(args.json_out, "w") as f:
            f.write(s + "\n")


def run_compare_orderings(args):
    """Sec. 3.3 (Tables 3-4) on the workload, per ordering: setup ms (second call), block
    bandwidth, coefficient blocks and entries, ms of one Eq. 28 operator application at 1 and
    at --nrhs columns, and the iterations of one solve (the first right-hand side of the
    bench batch)."""
    import torch
    import paper_2111_13483_gb300 as hm
    P = load_problem(args.workload, 0, 1, args.build)
    plate = args.workload.startswith("plate")
    V = rhs_batch(P, args.nrhs, plate, args.rhs)
    op = hm.hmsolve.OP32 + hm.hmsolve.OP_A if args.precision == 1 else hm.hmsolve.OP_A
    out = {"workload": args.workload, "precision": args.precision, "fill_tol": args.fill_tol, "orderings": {}}
    for o in (0, 1, 2):
        h = hm.hmat_create(P, ordering=o, fill_tol=args.fill_tol, precision=args.precision)
        hm.precond_setup(h)
        hm.precond_setup(h)
        st = hm.hmat_stats(h)
        times = {}
        for w in (1, args.nrhs):
            x = torch.randn(w, P.n, dtype=torch.complex128, device="cuda")
            y = torch.empty_like(x)
            for _ in range(3):
                hm.hm_apply(h, op, x, y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                hm.hm_apply(h, op, x, y)
            e1.record()
            torch.cuda.synchronize()
            times["op_ms_%d_cols" % w] = e0.elapsed_time(e1) / 5
        I, it, rr, code = hm.solve(h, V[:, 0], tol=args.tol, restart=args.restart)
        out["orderings"][ORDERINGS[o]] = dict(times, setup_ms=st["setup_ms"], bandwidth=st["bandwidth"],
                                              fill_blocks=st["fill_blocks"], coef_entries=st["coef_entries"],
                                              coef_entries_dense=st["coef_entries_dense"], iters=int(it[0]),
                                              converged=int(code) == 0)
        hm.hmat_destroy(h)
    print(json.dumps(out), flush=True)


def run_table7(args):
    """Sec. 5.2, Table 7 on a workload, in the paper's FP64 arithmetic: for the symmetric
    Schur-complement preconditioner (fill_tol as given), for the null-field comparison (the
    elimination without fill, applied from the left) and for block Jacobi (the near-field
    diagonal blocks), t_sp = precond_setup, p = mean GMRES(restart) iterations over a few
    right-hand sides of the bench sweep at the preconditioned tolerance --fp64-tol, the per
    iteration times of the operator's parts from the library's event profiler (one column):
    t_mm = far field (+ near field for the two comparisons), t_mpp = block solves and products
    with D, t_mps = coefficient sweeps (not for block Jacobi), and
    t_total = t_sm + t_sp + p n (t_mm + t_mp)
    (Eq. 46) for n = --nrhs right-hand sides, with t_sm = the build of the H-matrix (geometry,
    EFIE fill and ACA: on the GPU with --build gpu; on the host otherwise, 0 when the builder's
    cache held it) plus its upload (hmat_create)."""
    import torch
    import paper_2111_13483_gb300 as hm
    t0 = time.perf_counter()
    P = load_problem(args.workload, 0, 1, args.build)
    t_build = time.perf_counter() - t0
    plate = args.workload.startswith("plate")
    V = rhs_batch(P, args.nrhs, plate, args.rhs)
    cols = [int(c) for c in np.linspace(0, args.nrhs, 4, endpoint=False)]
    out = {"workload": args.workload, "n": int(P.n), "rhs_n": args.nrhs, "tol_preconditioned": args.fp64_tol,
           "restart": args.restart, "build": args.build, "build_s_this_process": t_build, "preconditioners": {}}
    if args.build == "gpu":
        out["gpu_build"] = P.build_timings
    for name, pc, ft in (("schur", 0, args.fill_tol), ("null_field", 2, 0.0), ("block_jacobi", 1, 0.0)):
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        h = hm.hmat_create(P, ordering=args.ordering, fill_tol=ft, precision=0, preconditioner=pc)
        t_sm = time.perf_counter() - c0
        hm.precond_setup(h)
        hm.precond_setup(h)
        t_sp = hm.hmat_stats(h)["setup_ms"] / 1e3
        its, solve_s, conv = [], [], []
        for c in cols:
            s0 = time.perf_counter()
            I, it, rr, code = hm.solve(h, V[:, c], tol=args.fp64_tol, restart=args.restart, maxit=20000)
            solve_s.append(time.perf_counter() - s0)
            its.append(int(it[0]))
            conv.append(int(code) == 0)
        x = torch.randn(1, P.n, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            hm.hm_apply(h, hm.hmsolve.OP_A, x, y)
        hm.hm_profile(h, 2)
        hm.hm_profile(h, 1)
        K = 20
        for _ in range(K):
            hm.hm_apply(h, hm.hmsolve.OP_A, x, y)
        torch.cuda.synchronize()
        pr = hm.hm_get_profile(h)
        hm.hm_profile(h, 0)
        ms = {k: v[2] / K for k, v in pr.items() if v[0]}
        t_mm = (ms.get("far1", 0) + ms.get("far2", 0) + ms.get("permute", 0) + ms.get("near", 0)) / 1e3
        t_mpp = ms.get("diag", 0) / 1e3
        t_mps = (ms.get("sweep_fwd", 0) + ms.get("sweep_bwd", 0)) / 1e3
        p = float(np.mean(its))
        st = hm.hmat_stats(h)
        t_sm += t_build      # the EFIE fill and ACA build (host: 0 when the builder's cache had it)
        out["preconditioners"][name] = {
            "t_sm_s": t_sm, "t_sp_s": t_sp, "p": p, "iters": its, "t_mm_s": t_mm, "t_mpp_s": t_mpp,
            "t_mps_s": t_mps, "t_mp_s": t_mpp + t_mps, "p_times_tmm_plus_tmp_s": p * (t_mm + t_mpp + t_mps),
            "t_total_s": t_sm + t_sp + p * args.nrhs * (t_mm + t_mpp + t_mps),
            "measured_solve_s_per_rhs": float(np.mean(solve_s)), "fill_tol": ft, "converged": conv,
            "coef_entries": st["coef_entries"] if pc != 1 else 0, "device_bytes": st["device_bytes"]}
        hm.hmat_destroy(h)
    s, b = out["preconditioners"]["schur"], out["preconditioners"]["block_jacobi"]
    out["speedup_total_schur_over_block_jacobi"] = b["t_total_s"] / s["t_total_s"]
    out["speedup_total_schur_over_null_field"] = out["preconditioners"]["null_field"]["t_total_s"] / s["t_total_s"]
    print(json.dumps(out), flush=True)


def run_profile_setup(args):
    """Setup timings for one schedule: the device ms of each precond_setup and, for the last,
    the event-profiler ms per kernel class."""
    import paper_2111_13483_gb300 as hm
    P = load_problem(args.workload, 0, 1, args.build)
    h = hm.hmat_create(P, ordering=args.ordering, fill_tol=args.fill_tol, precision=args.precision)
    hm.hmsolve.hm_set_update_schedule(h, args.update_schedule)
    hm.hmsolve.hm_set_pivot_schedule(h, args.pivot_schedule)
    ms = []
    for i in range(args.profile_setup):
        if i == args.profile_setup - 1:
            hm.hm_profile(h, 2)
            hm.hm_profile(h, 1)
        hm.precond_setup(h)
        ms.append(hm.hmat_stats(h)["setup_ms"])
    pr = hm.hm_get_profile(h)
    hm.hm_profile(h, 0)
    print(json.dumps({"workload": args.workload, "precision": args.precision, "fill_tol": args.fill_tol,
                      "pivot_schedule": args.pivot_schedule, "update_schedule": args.update_schedule,
                      "setup_ms": ms, "class_ms_last": {k: round(v[2], 3) for k, v in pr.items() if v[0]},
                      "class_launches_last": {k: v[0] for k, v in pr.items() if v[0]}}), flush=True)


def run_profile_op(args):
    """A short, deterministic case for ncu captures (no timing of its own)."""
    import torch
    import paper_2111_13483_gb300 as hm
    P = load_problem(args.workload, 0, 1, args.build)
    h = hm.hmat_create(P, ordering=args.ordering, fill_tol=args.fill_tol, precision=args.precision)
    hm.hmsolve.hm_set_update_schedule(h, args.update_schedule)
    hm.hmsolve.hm_set_pivot_schedule(h, args.pivot_schedule)
    hm.precond_setup(h)
    sched = [int(v) for v in args.schedule.split(",")]
    hm.hmsolve.hm_set_sweep_schedule(h, *sched)
    hm.hmsolve.hm_set_far_schedule(h, args.far_schedule)
    x = torch.randn(args.nrhs, P.n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    op = hm.hmsolve.OP32 + hm.hmsolve.OP_A if args.precision == 1 else hm.hmsolve.OP_A
    for _ in range(args.profile_op):
        hm.hm_apply(h, op, x, y)
    torch.cuda.synchronize()
    print("profile-op done: %s, %d x A on %d columns, coef entries %d" % (
        args.workload, args.profile_op, args.nrhs, hm.hmat_stats(h)["coef_entries"]), flush=True)


def main():
    args = parse()
    if args.cpu_anchor_run:
        cpu_anchor_run()
        return
    if args.profile_op > 0:
        run_profile_op(args)
        return
    if args.profile_setup > 0:
        run_profile_setup(args)
        return
    if args.profile_build:
        import torch
        from paper_2111_13483_gb300 import hmatrix
        hmatrix.build_problem(args.workload, device=torch.cuda.current_device())
        P, t = hmatrix.build_problem(args.workload, device=torch.cuda.current_device())
        print(json.dumps({"workload": args.workload, "gpu_build_s": t, "stats": P.stats()}), flush=True)
        return
    if args.compare_orderings:
        run_compare_orderings(args)
        return
    if args.table7:
        run_table7(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

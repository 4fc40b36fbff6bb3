#!/usr/bin/env python
"""Benchmark: sparsifying-preconditioned GMRES solves per second on one GB300.

Workload (one "step"): the 2D 512^2 problem pair, complex128 unknowns, b = 16,
  (a) Helmholtz, omega = 2 pi 64, c = 1 + 0.3 tanh(GRF, correlation length 0.05),
  (b) rescaled Schroedinger, l = 16, E = 10, 16 x 16 lattice of Gaussian wells
      (depth U[5, 15], width 0.15 l-units),
each with a random-centre, random-phase Gaussian source; for each problem the
step factors P = Q + C q (sp_factor) and solves to a true relative residual of
1e-8 (sp_solve).  One step = 2 solves; the two independent problems run side by
side, each context on its own CUDA stream driven by its own host thread
(--serial-pair: in turn on one stream).  The stencil set-up (sp_setup, once per
shift s) is outside the timed region.  `value` is the plain FP64 form; the
reduced-precision preconditioner forms (FP32 factor and sweeps, with or without
TF32 / 3xTF32 tensor-core Schur updates, GMRES-IR; FP64 operator, Gram-Schmidt
and residuals throughout) are reported beside it, the fastest as "chosen_form".

"workload_3d": the 3D 128^3 Helmholtz problem (omega = 2 pi 16, c = 1 + 0.3
tanh(GRF, correlation length 0.08), b = 8; one step = factor + solve of one
problem) in the tensor-core forms, with the roofline of the tcgen05 Schur update.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the library's stream, with an L2 flush (a 256 MB write) between steps outside
the events; barrier + synchronize around the timed loop; max over ranks.  N > 1
runs independent replicas (one per GPU, no collective on the data path).

--impl reference times the FP64 CPU oracle (numpy/scipy) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic_media as sm  # noqa: E402

METRIC = "solves/s at rel. residual 1e-8 (2D 512^2), plain FP64 GPU"
WORKLOAD_3D = "3D 128^3 Helmholtz GRF omega=2pi*16 (corr. length 0.08), b=8"
WORKLOAD_3D_SCHR = "3D 128^3 Schroedinger, 8 x 8 x 8 lattice wells (depth U[5,15], width 0.15 l-units), l=8, E=10, b=8"
# what the oracle arm actually times: one factor + solve of a 128^2 member of the
# 512^2 Helmholtz family (the 512^2 oracle factor alone takes minutes)
REF_SAMPLE = "oracle sample: 2D 128^2 Helmholtz GRF, b=8, omega=2pi*16 (8 points/wavelength as at 512^2), factor + solve"
UNIT = "solves/s"
WORKLOAD = "2D 512^2 pair: Helmholtz GRF omega=2pi*64 + Schroedinger wells l=16 E=10, b=16"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-chosen", action="store_true")
    p.add_argument("--profile-step", default=None,
                   choices=["fp64", "fp32", "tf32", "tf32x3", "tf32h", "tf32x3h"],
                   help="run exactly one untimed step (factor + solve of both problems) in the "
                        "given form after set-up and exit: the command profiled under ncu")
    p.add_argument("--profile-workload", default="2d512", choices=["2d512", "3d64", "3d128"],
                   help="workload of --profile-step (3d: one Helmholtz GRF problem, b = 8)")
    p.add_argument("--profile-gemm", default=None, metavar="M,N,K,FORM",
                   help="run the isolated Schur update C -= A B (sp_schur_update, FORM fp32 | "
                        "tf32 | tf32x3) three times on device-resident random operands and exit")
    p.add_argument("--profile-tc-probe", action="store_true",
                   help="run the tcgen05 rate probe once (C[8192^2] -= A B, K = 8192, TF32; one "
                        "warm-up and one timed launch) and exit: the command profiled under ncu")
    p.add_argument("--problems", default="helmholtz,schrodinger",
                   help="comma list of the step's problems (default both)")
    p.add_argument("--no-3d", action="store_true", help="skip the 3D 128^3 workload")
    p.add_argument("--forms-3d", default="tf32,tf32h,tf32x3",
                   help="comma list of the tensor-core forms timed on the 3D 128^3 Helmholtz "
                        "problem (tf32, tf32x3; a trailing h: sweeps from the FP16 copy of the "
                        "factor); each is profiled once for the breakdown and the roofline")
    p.add_argument("--forms-3d-schr", default="tf32,tf32h",
                   help="comma list of the forms timed on the 3D 128^3 Schroedinger problem "
                        "(empty: skip it)")
    p.add_argument("--no-tc-probe", action="store_true",
                   help="skip the rate probe of the tcgen05 update kernel (the measured TF32 "
                        "peak of the 3D roofline)")
    p.add_argument("--oracle-512", action="store_true",
                   help="time the FP64 oracle's full factor + solve of both 512^2 problems (two "
                        "spawned processes side by side, minutes of host CPU) and print its phases")
    p.add_argument("--steps-3d", type=int, default=1)
    p.add_argument("--setup-route-3d", type=int, default=1, choices=[0, 1],
                   help="stencil set-up of the 3D workload: 0 TSQR + SVD, 1 Gram (default)")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched heterogeneous 2D workload (64 problems x 8 right-hand sides)")
    p.add_argument("--batch-workers", type=int, default=16)
    p.add_argument("--no-batch-groups", action="store_true",
                   help="skip the problem-group arm of the batched workload")
    p.add_argument("--group-points", type=int, default=512 * 256,
                   help="problem groups of the batched workload hold about this many grid points")
    p.add_argument("--serial-pair", action="store_true",
                   help="run the two problems of a 2D step in turn on one stream")
    p.add_argument("--no-batch-fp64", action="store_true",
                   help="skip the plain-FP64 arm of the batched workload")
    p.add_argument("--no-learned", action="store_true",
                   help="skip the learned-initial-guess workload")
    p.add_argument("--learned-media", type=int, default=512)
    p.add_argument("--learned-eval", type=int, default=512)
    p.add_argument("--learned-epochs", type=int, default=10)
    p.add_argument("--learned-lr", type=float, default=1e-3)
    p.add_argument("--only-learned", action="store_true",
                   help="run the learned-initial-guess workload alone and print its JSON")
    p.add_argument("--sweeps", type=int, default=0, choices=[0, 1, 2],
                   help="sweeps of the block-inverse levels (sp_opts.sweeps): 0 fused launches on "
                        "many-front levels, chains elsewhere (default); 1 chains; 2 fused everywhere")
    p.add_argument("--device-loop", type=int, default=1, choices=[0, 1],
                   help="sp_opts.device_loop: 1 runs each GMRES restart cycle as one CUDA "
                        "graph (conditional while node), 0 lets the host drive each iteration")
    p.add_argument("--tc-epilogue", type=int, default=0, choices=[0, 1, 2, 3, 4],
                   help="sp_opts.tc_epilogue of the 3D tensor-core forms (C reads of the update)")
    p.add_argument("--no-autotune", action="store_true",
                   help="2D contexts keep the built-in launch-shape heuristics instead of "
                        "tuning them at set-up (sp_opts.autotune; results are bit-identical)")
    return p.parse_args()


def problems(which="helmholtz,schrodinger"):
    """Host inputs of the step's problems (dicts of synthetic_media)."""
    make = {"helmholtz": sm.helmholtz_grf_512, "schrodinger": sm.schrodinger_wells_512}
    return [make[w](0) for w in which.split(",")]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.device),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm_, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm_.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm_)) if sm_ else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm_)}


# ------------------------------------------------------------------ multi-GPU replicas
def reduce_max(x: float, dist=None, device: str = "cuda") -> float:
    """Max over ranks (one rank per GPU; every rank times its own replica)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(solves_per_step: int, world: int, ms_per_step_max: float) -> float:
    """Whole-job solves/s: every rank solves the same step's problems independently."""
    return solves_per_step * world / (ms_per_step_max / 1e3)


# ------------------------------------------------------------------ oracle (reference arm / cpu_baseline)
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count()
    # W untimed and K timed steps; a step is one bounded oracle sample (cpu_sample)
    prep = cpu_prep()
    for _ in range(args.warmup):
        cpu_sample(prep)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(max(1, args.steps)):
        it = cpu_sample(prep)
    dt, cpu_s = time.perf_counter() - t0, time.process_time() - c0
    steps = max(1, args.steps)
    res = {"value": steps / dt, "sample": cpu_sample_text(it, dt / steps)}
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": REF_SAMPLE, "same_as_gpu_arm": False,
                       "gpu_arm_workload": WORKLOAD},
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": cores,
                             "cores_busy": round(cpu_s / dt, 2), "kind": "oracle",
                             "sample": res["sample"]},
            "oracle_512_measured_once": ORACLE_512,
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_prep() -> dict:
    """Set-up of the bounded oracle sample (the stencil tables, once, like sp_setup): the
    Helmholtz GRF family of the 512^2 workload at 128^2 (b = 8, omega = 2 pi 16, the same
    8 points per wavelength)."""
    import oracle as O
    w = sm.helmholtz_grf(2, 128, 8, 2 * np.pi * 16, 0.05, 0)
    d, n, b = w["d"], w["n"], w["b"]
    s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
    return dict(w=w, s=s, q=q, tabs=O.stencil_tables(d, n, b, s))


def cpu_sample(prep) -> int:
    """One oracle factor + solve of the sample problem; returns the iterations."""
    import oracle as O
    w, s, q = prep["w"], prep["s"], prep["q"]
    d, n, b = w["d"], w["n"], w["b"]
    M = O.SparsifyingPreconditioner(d, n, b, s, q, tables=prep["tabs"], factor="splu")
    g = O.apply_green(d, n, s, w["f"])
    return O.gmres_right(lambda x: O.apply_operator(d, n, s, q, x), M.apply, g, tol=1e-8)["iters"]


def cpu_sample_text(iters: int, seconds: float) -> str:
    return (f"{REF_SAMPLE}: {iters} iterations, {seconds:.1f} s per sample; NOT the 512^2 "
            f"workload (see oracle_512_measured_once for the full 512^2 oracle solve)")


# The FP64 oracle's full factor + solve of the two 512^2 problems, measured once on the
# GPU machine's host cores (16 Arm cores) by `python bench.py --oracle-512` (both problems in
# spawned processes side by side).  Seconds per phase; "solve_s" = everything from the
# stencil tables to the GMRES solution at 1e-8; value = 2 solves / the slower process.
ORACLE_512 = {
    "value": 2.0 / 331.1, "unit": UNIT, "cores": 16, "kind": "oracle",
    "sample": "full FP64 oracle factor + solve of both 512^2 problems (tables, assembly, SuperLU "
              "factor of P, GMRES to 1e-8), two processes side by side, measured once",
    "wall_s": 331.1,
    "problems": {"helmholtz": {"tables_s": 6.9, "assemble_s": 3.3, "factor_s": 271.2,
                               "gmres_s": 49.4, "solve_s": 330.8, "iters": 43},
                 "schrodinger": {"tables_s": 5.0, "assemble_s": 3.4, "factor_s": 256.3,
                                 "gmres_s": 9.9, "solve_s": 274.5, "iters": 8}},
}


def _oracle_512_one(kind: str) -> dict:
    """Full oracle solve of one 512^2 problem with phase times (spawned process)."""
    import scipy.sparse.linalg as spla

    import oracle as O
    w = sm.helmholtz_grf_512() if kind == "helmholtz" else sm.schrodinger_wells_512()
    d, n, b = w["d"], w["n"], w["b"]
    if kind == "helmholtz":
        s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
        f = w["f"]
    else:
        s, q = O.schrodinger_shift(d, n, w["ell"], w["E"], w["V"])
        f = w["f"] * w["ell"] ** 2
    ph = {}
    t00 = t0 = time.perf_counter()
    tabs = O.stencil_tables(d, n, b, s)
    ph["tables_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    M = O.SparsifyingPreconditioner(d, n, b, s, q, tables=tabs, factor=None)
    ph["assemble_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    M._lu, M.kind = spla.splu(M.P.tocsc()), "splu"
    ph["factor_s"] = time.perf_counter() - t0
    g = O.apply_green(d, n, s, f)
    t0 = time.perf_counter()
    res = O.gmres_right(lambda x: O.apply_operator(d, n, s, q, x), M.apply, g, tol=1e-8)
    ph["gmres_s"] = time.perf_counter() - t0
    ph["solve_s"] = time.perf_counter() - t00
    ph["iters"] = res["iters"]
    ph["true_relres"] = res["true_relres"]
    return ph


def oracle_512() -> dict:
    """Both 512^2 problems in two spawned processes side by side (about 5-8 minutes)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(2, mp_context=mp.get_context("spawn")) as ex:
        fut = {k: ex.submit(_oracle_512_one, k) for k in ("helmholtz", "schrodinger")}
        out = {k: v.result() for k, v in fut.items()}
    wall = time.perf_counter() - t0
    return {"value": 2.0 / wall, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "wall_s": wall, "problems": out,
            "sample": "full FP64 oracle factor + solve of both 512^2 problems, side by side"}


def _oracle_phases_one(w: dict, reps: int = 3) -> dict:
    """Oracle phases of one small problem, best of `reps`: stencil tables, assembly of
    P, its factorisation (dense LU up to 4096 unknowns, SuperLU beyond, as the oracle
    chooses), one preconditioner application P^{-1} Q g and the GMRES solve to 1e-8."""
    import scipy.linalg as sla
    import scipy.sparse.linalg as spla

    import oracle as O
    d, n, b = w["d"], w["n"], w["b"]
    s, q = O.helmholtz_shift(d, n, w["omega"], w["c"])
    g = O.apply_green(d, n, s, w["f"])
    best = {}
    for _ in range(reps):
        ph = {}
        t0 = time.perf_counter()
        tabs = O.stencil_tables(d, n, b, s)
        ph["tables_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        M = O.SparsifyingPreconditioner(d, n, b, s, q, tables=tabs, factor=None)
        ph["assemble_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        if M.N <= 4096:
            M._lu, M.kind = sla.lu_factor(M.P.toarray()), "dense"
        else:
            M._lu, M.kind = spla.splu(M.P.tocsc()), "splu"
        ph["factor_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        M.apply(g)
        ph["apply_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        res = O.gmres_right(lambda x: O.apply_operator(d, n, s, q, x), M.apply, g, tol=1e-8)
        ph["gmres_s"] = time.perf_counter() - t0
        best = {k: min(v, best.get(k, v)) for k, v in ph.items()}
    best = {k: round(v, 4) for k, v in best.items()}
    best.update(iters=res["iters"], factor=M.kind, unknowns=M.N)
    return best


def oracle_phases() -> dict:
    """The oracle's phases, best of 3, on the small configurations it finishes in
    seconds: the 64^2 centre-Gaussian Helmholtz problem (b = 4) and a 3D 16^3 Helmholtz
    GRF problem (b = 4).  (3D 32^3 takes about a minute in SuperLU alone; the 512^2
    pair is in oracle_512_measured_once.)"""
    return {"helmholtz_2d64_b4": _oracle_phases_one(sm.helmholtz_centre_gaussian_64(0)),
            "helmholtz_3d16_b4": _oracle_phases_one(sm.helmholtz_grf_3d(16, 4, 0))}


def cpu_baseline() -> dict:
    """Bounded oracle sample (see the returned 'sample' text), after one untimed warm-up
    sample (imports, first factorisation)."""
    prep = cpu_prep()
    cpu_sample(prep)
    t0, c0 = time.perf_counter(), time.process_time()
    it = cpu_sample(prep)
    dt, cpu_s = time.perf_counter() - t0, time.process_time() - c0
    return {"value": 1.0 / dt, "sample": cpu_sample_text(it, dt), "seconds": dt,
            "cores_busy": cpu_s / dt}


# ------------------------------------------------------------------ tensor-core peak
def measure_tc_peak(B) -> dict:
    """Rate of the library's own tcgen05 update kernel on a deep product (the pipe
    limit, not an epilogue limit): C[8192 x 8192] -= A[8192 x 8192] B, TF32 and
    3xTF32, as a burst (10 launches after a warm-up) and sustained (launches back to
    back for about 2 s, under the power cap), CUDA events around the kernel alone."""
    M = N = K = 8192
    fl = 2.0 * M * N * K
    out = {"shape": [M, N, K], "kernel": "tc_gemm_sub_kernel (tcgen05.mma kind::tf32, TMA, TMEM)"}
    for split, name in ((0, "tf32"), (1, "tf32x3")):
        burst = B.sp_tc_probe(split, M, N, K, 10)
        reps = max(10, min(1000, int(2000.0 / max(burst, 1e-3))))
        sus = B.sp_tc_probe(split, M, N, K, reps)
        out[name] = {"burst_tflops": fl / (burst / 1e3) / 1e12,
                     "sustained_tflops": fl / (sus / 1e3) / 1e12,
                     "sustained_launches": reps,
                     "pipe_flops_per_update_flop": 3 if split else 1}
    return out


# ------------------------------------------------------------------ 3D 128^3
def _measure_3d_one(args, B, torch, flush, w, forms, tf32_peak, dist, world, profile_first):
    d, n, b = 3, 128, 8
    if w["kind"] == "helmholtz":
        s, q = B.sp_medium_helmholtz(d, n, w["omega"], w["c"])
        f = w["f"]
    else:
        s, q = B.sp_medium_schrodinger(d, n, w["ell"], w["E"], w["V"])
        f = w["f"] * w["ell"] ** 2
    qd = torch.from_numpy(q).cuda()
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    u = torch.empty(n ** d, dtype=torch.complex128, device="cuda")
    warm = max(1, min(args.warmup, 3))
    out = {}
    for fi, name in enumerate(forms):
        # a trailing "h": the sweeps read the FP16 copy of the factor (factor_storage 1)
        half = name.endswith("h")
        prec = {"tf32": B.SP_PREC_TF32, "tf32x3": B.SP_PREC_TF32X3}[name[:-1] if half else name]
        t0 = time.perf_counter()
        S = B.Solver(d, n, b, s, prec=prec, device=int(os.environ.get("LOCAL_RANK", "0")),
                     setup_route=args.setup_route_3d, sweeps=args.sweeps,
                     device_loop=args.device_loop, factor_storage=1 if half else 0,
                     tc_epilogue=args.tc_epilogue)
        setup_s = time.perf_counter() - t0
        for _ in range(warm):
            S.factor(qd)
            S.solve(fd, u)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms, infos = 0.0, []
        for _ in range(args.steps_3d):
            flush.zero_()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            S.factor(qd)
            infos.append(S.solve(fd, u))
            e.record()
            torch.cuda.synchronize()
            ms += a.elapsed_time(e)
        ms = reduce_max(ms / args.steps_3d, dist)
        r = {"value": replica_value(1, world, ms), "ms_per_step": ms, "setup_s": setup_s,
             "warmup": warm, "iters": infos[0]["iters"], "true_relres": infos[0]["true_relres"]}
        if profile_first:
            B.sp_profile(S.ctx, True)
            S.factor(qd)
            S.solve(fd, u)
            prof = B.sp_profile_read(S.ctx)
            B.sp_profile(S.ctx, False)
            tc_ms, tc_n, tc_fl = prof["lu_tc"]
            ach = tc_fl / (tc_ms / 1e3) / 1e12 if tc_ms > 0 else 0.0
            r["roofline"] = {"kernel": "lu_tc (tcgen05 TF32 Schur update)", "bound": "tensor",
                             "achieved": ach, "peak": tf32_peak["value"], "unit": "TFLOP/s",
                             "frac": ach / tf32_peak["value"], "traffic": recorded_traffic("lu_tc_3d128"),
                             "peak_source": tf32_peak["source"]}
            r["roofline"]["frac_of_tensor_pipe_ncu"] = ach / tf32_peak["pipe_ncu"]
            if tf32_peak.get("kernel_sustained"):
                r["roofline"]["frac_of_kernel_sustained_8192"] = ach / tf32_peak["kernel_sustained"]
            r["kernel_breakdown_ms_per_step"] = {
                k: {"ms": round(v[0], 2), "launches": v[1],
                    "achieved": round(v[2] / (v[0] / 1e3) / (1e12 if k.startswith("lu_") else 1e9), 2)
                    if v[0] > 0 else None,
                    "unit": "TFLOP/s" if k.startswith("lu_") else "GB/s"}
                for k, v in prof.items() if v[1]}
        out[name] = r
        S.close()
        torch.cuda.synchronize()
    return out


def measure_3d(args, B, torch, flush, peaks, tc_peak, dist, world):
    """The 3D 128^3 workloads (one step = sp_factor + sp_solve of one problem) in the
    tensor-core forms: Helmholtz (random-field velocity) and rescaled Schroedinger
    (lattice wells); up to 3 untimed warm-up steps, then args.steps_3d timed steps
    with CUDA events and an L2 flush in between.  The tcgen05 update's roofline is
    taken against the sustained rate the library's own kernel reaches on a deep
    product (the update is timed inside a seconds-long step), else the measured BF16
    rate x the nominal TF32/BF16 ratio."""
    # the update is timed inside a seconds-long step: the measured sustained BF16 rate
    # (under the power cap) x the nominal TF32/BF16 ratio is its denominator; beside it
    # the fraction of the TF32 pipe peak that ncu implies for the library's own kernel
    # (722 TFLOP/s at 59.6 % tensor-pipe activity, 8192^3 at 1.95 GHz: 1.21 PFLOP/s) and
    # of that kernel's live sustained rate on the deep product
    tf32_peak = {"value": peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1890.2))
                 * (1.1 / 2.25),
                 "source": "measured bf16_tflops_sustained x nominal TF32/BF16 ratio 1.1/2.25",
                 "pipe_ncu": 1211.0}
    if tc_peak:
        tf32_peak["kernel_sustained"] = tc_peak["tf32"]["sustained_tflops"]
    helm = _measure_3d_one(args, B, torch, flush, sm.helmholtz_grf_3d(128, 8, 0),
                           [f for f in args.forms_3d.split(",") if f], tf32_peak, dist, world, True)
    best = max(helm, key=lambda k: helm[k]["value"])
    res = {"workload": WORKLOAD_3D, "grid": "128^3", "b": 8, "solves_per_step": 1,
           "steps": args.steps_3d, "l2": "flushed between steps (256 MB write)", "data": "synthetic",
           "setup_route": "Gram" if args.setup_route_3d == 1 else "TSQR + SVD",
           "plain_fp64": "not run: the FP64 fronts alone take 237 GB and the FP64 factor "
                         "~8e14 flop at 1.25 TFLOP/s",
           "chosen": dict(helm[best], name=best), "forms": helm}
    schr_forms = [f for f in args.forms_3d_schr.split(",") if f]
    if schr_forms:
        sch = _measure_3d_one(args, B, torch, flush, sm.schrodinger_wells_3d(128, 8, 8.0, 10.0, 0),
                              schr_forms, tf32_peak, dist, world, False)
        res["schrodinger"] = {"workload": WORKLOAD_3D_SCHR, "forms": sch}
    return res


# ------------------------------------------------------------------ batched 2D
def measure_batch(args, B, torch, dist, world):
    """64 heterogeneous 2D problems (n in {128, 192, 256, 384, 512}, half Helmholtz,
    half Schroedinger) with 8 right-hand sides each; one step = for every problem
    sp_factor + sp_solve_many of its 8 right-hand sides (the factor amortised, the
    8 GMRES iterations in lockstep sharing every preconditioner application), the
    problems spread over `batch_workers` host threads, each context on its own CUDA
    stream so small problems run side by side.  FP32 preconditioner form.  Timed on
    the device: an event on the launching stream before, every worker stream waits on
    it, and the launching stream waits on every worker's end event."""
    import concurrent.futures as cf
    probs = sm.batched_2d_problems()
    nw = max(1, args.batch_workers)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    t0 = time.perf_counter()
    streams = [torch.cuda.Stream() for _ in probs]

    def setup(i, prec=B.SP_PREC_FP32, batched=True):
        p = probs[i]
        if p["kind"] == "helmholtz":
            s, q = B.sp_medium_helmholtz(2, p["n"], p["omega"], p["c"])
            scale = 1.0
        else:
            s, q = B.sp_medium_schrodinger(2, p["n"], p["ell"], p["E"], p["V"])
            scale = p["ell"] ** 2
        S = B.Solver(2, p["n"], p["b"], s, prec=prec, restart=64, device=local, sweeps=args.sweeps,
                     device_loop=args.device_loop,
                     stream=streams[i].cuda_stream, max_rhs=len(p["rhs"]) if batched else 1,
                     host_threads=max(1, (os.cpu_count() or 1) // nw))
        return S, q, [np.ascontiguousarray(f * scale) for f in p["rhs"]]

    with cf.ThreadPoolExecutor(nw) as ex:
        made = list(ex.map(setup, range(len(probs))))
    setup_s = time.perf_counter() - t0
    ctx = []
    for (S, q, fs), p in zip(made, probs):
        N = p["n"] ** 2
        F = torch.from_numpy(np.stack(fs)).cuda().contiguous()
        ctx.append(dict(S=S, q=torch.from_numpy(q).cuda(), F=F, U=torch.empty_like(F)))
    torch.cuda.synchronize()
    order = sorted(range(len(probs)), key=lambda i: -probs[i]["n"])  # largest first
    groups = [order[w::nw] for w in range(nw)]

    def work(w, infos, plain=False):
        for i in groups[w]:
            c = ctx[i]
            c["S"].factor(c["q"])
            if plain:  # one sp_solve per right-hand side
                for r in range(c["F"].shape[0]):
                    infos.append((i, c["S"].solve(c["F"][r], c["U"][r])))
            else:
                for inf in c["S"].solve_many(c["F"].view(-1), c["U"].view(-1)):
                    infos.append((i, inf))

    def step(infos, plain=False):
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        for i in range(len(probs)):
            streams[i].wait_event(start)
        with cf.ThreadPoolExecutor(nw) as ex:
            list(ex.map(lambda w: work(w, infos, plain), range(nw)))
        cur = torch.cuda.current_stream()
        for st_ in streams:
            ev = torch.cuda.Event()
            ev.record(st_)
            cur.wait_event(ev)
        end = torch.cuda.Event(enable_timing=True)
        end.record()
        torch.cuda.synchronize()
        return start.elapsed_time(end)

    for _ in range(args.warmup):
        step([])
    if dist:
        dist.barrier()
    infos = []
    ms = reduce_max(step(infos), dist)
    nsolve = sum(len(p["rhs"]) for p in probs)
    by_n = {}
    for i, inf in infos:
        e = by_n.setdefault(str(probs[i]["n"]), {"solves": 0, "iters": 0})
        e["solves"] += 1
        e["iters"] += inf["iters"]
    for c in ctx:
        c["S"].close()
    torch.cuda.synchronize()
    grouped = None if args.no_batch_groups else measure_batch_groups(args, B, torch, dist, world,
                                                                     probs, nw, local)
    # the same 512 solves in the plain FP64 form, one sp_solve per right-hand side
    # (same host threads and streams): the reference for the precision + batching gain
    plain = None
    if not args.no_batch_fp64:
        with cf.ThreadPoolExecutor(nw) as ex:
            made = list(ex.map(lambda i: setup(i, B.SP_PREC_FP64, False), range(len(probs))))
        for c, (S, q, fs) in zip(ctx, made):
            c["S"] = S
        torch.cuda.synchronize()
        step([], True)  # warm-up (one step: the plain form is slow)
        pinfos = []
        pms = reduce_max(step(pinfos, True), dist)
        for c in ctx:
            c["S"].close()
        torch.cuda.synchronize()
        plain = {"form": "plain FP64, one sp_solve per right-hand side", "value":
                 replica_value(nsolve, world, pms), "ms_per_step": pms,
                 "max_true_relres": max(inf["true_relres"] for _, inf in pinfos)}
    return {"workload": "batched 2D: 64 problems, n drawn from {128,192,256,384,512} (seed 3000), "
                        "half Helmholtz (omega = 2 pi n / 8, GRF c) half Schroedinger (l x l "
                        "lattice wells, l in {4,8,16}, E = 10), 8 random Gaussian sources each",
            "form": "FP32 preconditioner (FP64 operator, Gram-Schmidt, residuals)",
            "value": replica_value(nsolve, world, ms), "unit": "solves/s", "ms_per_step": ms,
            "solves_per_step": nsolve, "warmup": args.warmup, "steps": 1,
            "concurrency": f"{nw} host threads, one CUDA stream per problem; the 8 right-hand "
                           "sides of a problem in one sp_solve_many (restart 64)",
            "setup_s": setup_s,
            "max_true_relres": max(inf["true_relres"] for _, inf in infos),
            "plain_fp64": plain,
            "speedup_vs_plain_fp64": (replica_value(nsolve, world, ms) / plain["value"]) if plain else None,
            "problem_groups": grouped,
            "by_grid": by_n, "data": "synthetic"}


def measure_batch_groups(args, B, torch, dist, world, probs, nw, local):
    """The batched workload with the problems of each (grid, family) in one problem group
    (sp_setup_group): every factorisation and sweep launch covers the fronts of all the
    group's problems and one sp_solve_many advances the 8 right-hand sides of every
    problem of the group together (8 P Krylov instances, one CUDA graph per restart
    cycle); one host thread and one CUDA stream per group."""
    import concurrent.futures as cf
    t0 = time.perf_counter()
    # buckets of one (grid, family), split into groups of about args.group_points grid
    # points (so a group of small problems is as large as one big problem and the big
    # ones keep running side by side)
    keys, members = [], []
    for k in sorted({(p["n"], p["kind"]) for p in probs}, key=lambda k: (-k[0], k[1])):
        ids = [i for i, p in enumerate(probs) if (p["n"], p["kind"]) == k]
        per = max(1, args.group_points // (k[0] * k[0]))
        for j in range(0, len(ids), per):
            keys.append(k)
            members.append(ids[j:j + per])
    streams = [torch.cuda.Stream() for _ in keys]
    nthreads = min(nw, len(keys))

    def setup(gi):
        n, kind = keys[gi]
        shifts, qs, rhs = [], [], []
        for i in members[gi]:
            p = probs[i]
            if kind == "helmholtz":
                s, q = B.sp_medium_helmholtz(2, n, p["omega"], p["c"])
                scale = 1.0
            else:
                s, q = B.sp_medium_schrodinger(2, n, p["ell"], p["E"], p["V"])
                scale = p["ell"] ** 2
            shifts.append(s)
            qs.append(q)
            rhs.append([f * scale for f in p["rhs"]])
        R = len(rhs[0])
        S = B.Solver(2, n, probs[members[gi][0]]["b"], shifts if len(shifts) > 1 else shifts[0],
                     prec=B.SP_PREC_FP32, restart=64, device=local, sweeps=args.sweeps,
                     device_loop=args.device_loop, stream=streams[gi].cuda_stream, max_rhs=R,
                     host_threads=max(1, (os.cpu_count() or 1) // nthreads))
        # right-hand side r of member p at (r P + p) N
        F = np.stack([np.concatenate([rhs[p][r] for p in range(len(rhs))]) for r in range(R)])
        return S, np.concatenate(qs), F

    with cf.ThreadPoolExecutor(nthreads) as ex:
        made = list(ex.map(setup, range(len(keys))))
    setup_s = time.perf_counter() - t0
    units = []
    for S, q, F in made:
        Fd = torch.from_numpy(np.ascontiguousarray(F)).cuda().contiguous()
        units.append(dict(S=S, q=torch.from_numpy(q).cuda(), F=Fd, U=torch.empty_like(Fd)))
    torch.cuda.synchronize()

    # groups largest first, dealt round-robin to the host threads
    order = sorted(range(len(keys)), key=lambda gi: -keys[gi][0] ** 2 * len(members[gi]))
    share = [order[w::nthreads] for w in range(nthreads)]

    def work(w, infos):
        for gi in share[w]:
            u = units[gi]
            u["S"].factor(u["q"])
            infos.extend(u["S"].solve_many(u["F"].view(-1), u["U"].view(-1)))

    def step(infos):
        start = torch.cuda.Event(enable_timing=True)
        start.record()
        for st_ in streams:
            st_.wait_event(start)
        with cf.ThreadPoolExecutor(nthreads) as ex:
            list(ex.map(lambda w: work(w, infos), range(nthreads)))
        cur = torch.cuda.current_stream()
        for st_ in streams:
            ev = torch.cuda.Event()
            ev.record(st_)
            cur.wait_event(ev)
        end = torch.cuda.Event(enable_timing=True)
        end.record()
        torch.cuda.synchronize()
        return start.elapsed_time(end)

    for _ in range(args.warmup):
        step([])
    if dist:
        dist.barrier()
    infos = []
    ms = reduce_max(step(infos), dist)
    nsolve = sum(len(p["rhs"]) for p in probs)
    for u in units:
        u["S"].close()
    torch.cuda.synchronize()
    return {"form": f"FP32 preconditioner, problem groups of one (grid, family) and about "
                    f"{args.group_points} grid points",
            "value": replica_value(nsolve, world, ms), "unit": "solves/s", "ms_per_step": ms,
            "groups": [{"n": k[0], "kind": k[1], "problems": len(m)} for k, m in zip(keys, members)],
            "concurrency": f"{len(keys)} groups on {nthreads} host threads, one CUDA stream per "
                           "group; all right-hand sides of a group in one sp_solve_many "
                           "(restart 64)",
            "setup_s": setup_s, "solves_per_step": nsolve,
            "max_true_relres": max(inf["true_relres"] for inf in infos)}


LEARNED_N, LEARNED_B, LEARNED_ELL, LEARNED_E = 256, 8, 8.0, 10.0


def measure_learned(args, B, torch, dist, world):
    """Learned initial guess on 2D 256^2 Schroedinger problems (l = 8, E = 10, random 8 x 8
    lattice wells, b = 8), all sharing one context (one shift s; the solution does not
    depend on s).  The network learns a correction to the method's own first estimate
    z = M g = P^{-1} Q g (one preconditioner application): input (q / (10 l^2), g / c,
    z / c), target (u - z) / c, guess u0 = z + c y, with the complex scale
    c = rms|g| e^{i phi}, phi = arg(sum g^2) / 2 (the solution is complex-linear in the
    source, so c removes the source's size and phase).
    Training triples: `learned_media` potentials (seeds 5000 + m) x 8 random Gaussian
    sources (seeds 6000 + 8 m + r), each solved in FP64 by sp_factor + sp_solve_many;
    Adam on batches of 16 with a cosine learning-rate decay, every kernel in the library.
    The triples sit in slots permuted once (seeded), so a batch is a contiguous slice:
    batch membership is fixed across epochs and each epoch visits the batches in a new
    order.  Per epoch: the mean training loss over all its batches and the loss on 64
    validation problems (potential seeds 9000 + i, source seeds 9500 + i).
    Held-out: `learned_eval` problems (potential seed 7000 + i, source seed 8000 + i),
    each factored once and solved three times, every arm timed with CUDA events and
    stopped at the same true residual 1e-8: from zero (sp_solve), from z alone (the
    control: sp_apply + sp_solve_x0) and from the network's guess (sp_apply + features
    + forward + guess + sp_solve_x0)."""
    n, b, ell, E = LEARNED_N, LEARNED_B, LEARNED_ELL, LEARNED_E
    N = n * n
    nm, nrhs, ne = args.learned_media, 8, args.learned_eval
    nval = 64
    local = int(os.environ.get("LOCAL_RANK", "0"))
    qs = 1.0 / (10.0 * ell * ell)
    V0 = sm.lattice_wells_potential_2d(n, ell, 5000)
    s, _ = B.sp_medium_schrodinger(2, n, ell, E, V0)
    S = B.Solver(2, n, b, s, prec=B.SP_PREC_FP64, restart=200, device=local, max_rhs=nrhs,
                 sweeps=args.sweeps, device_loop=args.device_loop)
    cin = 5
    net = B.Fno(n, sm.fno_initial_params(c_in=cin, seed=4000), c_in=cin, batch_max=16)
    ntr = nm * nrhs
    X = torch.empty((ntr, cin, N), dtype=torch.float32, device="cuda")
    T = torch.empty((ntr, 2, N), dtype=torch.float32, device="cuda")
    sig = torch.empty(ntr, dtype=torch.complex128, device="cuda")
    g = torch.empty(N, dtype=torch.complex128, device="cuda")
    z = torch.empty(N, dtype=torch.complex128, device="cuda")
    slot = np.random.default_rng(9001).permutation(nm * nrhs)
    t0 = time.perf_counter()
    gen_iters = []
    for m in range(nm):
        V = sm.lattice_wells_potential_2d(n, ell, 5000 + m)
        q = torch.from_numpy(B.sp_medium_schrodinger_at(2, n, ell, E, V, s)).cuda()
        F = torch.from_numpy(np.stack([sm.random_gaussian_source(2, n, 6000 + nrhs * m + r) * ell ** 2
                                       for r in range(nrhs)])).cuda()
        U = torch.empty_like(F)
        S.factor(q)
        infos = S.solve_many(F.view(-1), U.view(-1))
        gen_iters += [i["iters"] for i in infos]
        for r in range(nrhs):
            k = int(slot[m * nrhs + r])
            S.green(F[r], g)
            S.apply(g, z)
            net.features_prior(q, qs, g, z, X[k], sig[k:k + 1])
            net.target_prior(U[r], sig[k:k + 1], z, T[k])
    # validation problems (their own potentials and sources)
    Xv = torch.empty((nval, cin, N), dtype=torch.float32, device="cuda")
    Tv = torch.empty((nval, 2, N), dtype=torch.float32, device="cuda")
    sv = torch.empty(nval, dtype=torch.complex128, device="cuda")
    uv = torch.empty(N, dtype=torch.complex128, device="cuda")
    for i in range(nval):
        V = sm.lattice_wells_potential_2d(n, ell, 9000 + i)
        q = torch.from_numpy(B.sp_medium_schrodinger_at(2, n, ell, E, V, s)).cuda()
        f = torch.from_numpy(sm.random_gaussian_source(2, n, 9500 + i) * ell ** 2).cuda()
        S.factor(q)
        S.solve(f, uv)
        S.green(f, g)
        S.apply(g, z)
        net.features_prior(q, qs, g, z, Xv[i], sv[i:i + 1])
        net.target_prior(uv, sv[i:i + 1], z, Tv[i])
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0

    def val_loss():
        tot = 0.0
        for i0 in range(0, nval, 16):
            L, _ = net.gradient(Xv[i0:i0 + 16], Tv[i0:i0 + 16], 16, want_grad=False)
            tot += L * 16
        return tot / nval

    # training
    bs, epochs = 16, args.learned_epochs
    nb = ntr // bs
    nsteps = epochs * nb
    lr0 = args.learned_lr
    rng = np.random.default_rng(9000)
    losses, vlosses = [], [val_loss()]
    train_ms = 0.0
    step = 0
    for ep in range(epochs):
        order = rng.permutation(nb)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        tot = 0.0
        for j in range(nb):
            bi = int(order[j])
            lr = 0.5 * lr0 * (1 + np.cos(np.pi * step / nsteps))
            tot += net.train_step(X[bi * bs:(bi + 1) * bs], T[bi * bs:(bi + 1) * bs], bs, lr, sync=True)
            step += 1
        ev1.record()
        torch.cuda.synchronize()
        train_ms += ev0.elapsed_time(ev1)
        losses.append(tot / nb)
        vlosses.append(val_loss())
    # held-out evaluation
    x1 = torch.empty((1, cin, N), dtype=torch.float32, device="cuda")
    y1 = torch.empty((1, 2, N), dtype=torch.float32, device="cuda")
    s1 = torch.empty(1, dtype=torch.complex128, device="cuda")
    u0 = torch.empty(N, dtype=torch.complex128, device="cuda")
    uz = torch.empty(N, dtype=torch.complex128, device="cuda")
    ug = torch.empty(N, dtype=torch.complex128, device="cuda")
    ms_zero = ms_prior = ms_guess = ms_factor = 0.0
    it_zero, it_prior, it_guess, g_rel, p_rel, u_err, used, worst = [], [], [], [], [], [], 0, 0.0
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for i in range(ne):
        V = sm.lattice_wells_potential_2d(n, ell, 7000 + i)
        q = torch.from_numpy(B.sp_medium_schrodinger_at(2, n, ell, E, V, s)).cuda()
        f = torch.from_numpy(sm.random_gaussian_source(2, n, 8000 + i) * ell ** 2).cuda()
        evs[0].record()
        S.factor(q)
        evs[1].record()
        iz = S.solve(f, uz)
        evs[2].record()
        S.green(f, g)
        S.apply(g, z)
        ip = S.solve_x0(f, z, ug)
        evs[3].record()
        S.green(f, g)
        S.apply(g, z)
        net.features_prior(q, qs, g, z, x1[0], s1)
        net.forward(x1, y1, 1)
        net.guess_prior(y1[0], s1, z, u0)
        evs[4].record()
        ig = S.solve_x0(f, u0, ug)
        evs[5].record()
        torch.cuda.synchronize()
        ms_factor += evs[0].elapsed_time(evs[1])
        ms_zero += evs[1].elapsed_time(evs[2])
        ms_prior += evs[2].elapsed_time(evs[3])
        ms_guess += evs[3].elapsed_time(evs[5])
        it_zero.append(iz["iters"])
        it_prior.append(ip["iters"])
        it_guess.append(ig["iters"])
        g_rel.append(ig["guess_relres"])
        p_rel.append(ip["guess_relres"])
        used += int(ig["guess_used"])
        worst = max(worst, iz["true_relres"], ip["true_relres"], ig["true_relres"])
        u_err.append(float(torch.linalg.vector_norm(u0 - uz) / torch.linalg.vector_norm(uz)))
    S.close()
    net.close()
    torch.cuda.synchronize()
    zero_v = ne / ((ms_factor + ms_zero) / 1e3)
    prior_v = ne / ((ms_factor + ms_prior) / 1e3)
    guess_v = ne / ((ms_factor + ms_guess) / 1e3)
    return {"workload": f"learned initial guess: 2D {n}^2 Schroedinger, l = {ell:g}, E = {E:g}, random "
                        f"8 x 8 lattice wells, b = {b}; {ntr} training triples ({nm} potentials x "
                        f"{nrhs} sources), {ne} held-out (potential, source) pairs",
            "network": "Fourier layers: 4 x width 32, 16 modes, projection 128; input (q, g, z = M g) "
                       "scaled, output the correction to z; bf16 weights, bf16 activations, "
                       "FP32 accumulation; Adam",
            "form": "plain FP64 solve in every arm",
            "value": guess_v, "unit": "solves/s", "zero_guess_value": zero_v,
            "speedup_vs_zero_guess": guess_v / zero_v,
            "prior_only": {"value": prior_v, "speedup_vs_zero_guess": prior_v / zero_v,
                           "iters_mean": float(np.mean(it_prior)),
                           "start_relres_median": float(np.median(p_rel))},
            "iters_zero_mean": float(np.mean(it_zero)), "iters_guess_mean": float(np.mean(it_guess)),
            "guess_relres_median": float(np.median(g_rel)), "guess_used": used,
            "guess_solution_relerr_median": float(np.median(u_err)),
            "max_true_relres": worst,
            "ms_per_solve": {"factor": ms_factor / ne, "zero_solve": ms_zero / ne,
                             "prior_and_solve": ms_prior / ne, "guess_and_solve": ms_guess / ne},
            "data_generation_s": gen_s, "data_iters_mean": float(np.mean(gen_iters)),
            "training": {"epochs": epochs, "batch": bs, "steps": nsteps, "lr0": lr0,
                         "ms": train_ms, "samples_per_s": nsteps * bs / (train_ms / 1e3),
                         "epoch_mean_loss": losses, "validation_loss_by_epoch": vlosses},
            "data": "synthetic"}


# ------------------------------------------------------------------ traffic and summary
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a kernel
# class, from one ncu capture, with the 16-hex SHA-256 prefix of the kernel's source
# text at the time (from the line that names the kernel to the first line that is a
# lone closing brace): a changed kernel reports null until it is captured again.
TRAFFIC = {
    # FP64 Schur update (gemm_sub_kernel<double, 32>), all 101 launches of one 2D 512^2
    # Helmholtz factorisation: 6.42 GB / 101 launches (ncu --metrics
    # dram__bytes_read.sum,dram__bytes_write.sum; command in the matching profile summary)
    "lu_gemm": {"bytes_per_launch": 63.6e6, "source": "paper_1409_0297_gb300/csrc/sp_factor.cu",
                "kernel": "gemm_sub_kernel(", "sha16": "6282b6619bef34c3"},
}


def _kernel_sha16(rel_path: str, marker: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, rel_path)) as fh:
        lines = fh.read().split("\n")
    start = next(i for i, ln in enumerate(lines) if marker in ln and "__global__" in ln)
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return hashlib.sha256("\n".join(lines[start:end + 1]).encode()).hexdigest()[:16]


def recorded_traffic(kernel_class: str):
    t = TRAFFIC.get(kernel_class)
    if not t or not t.get("sha16"):
        return None
    try:
        return t["bytes_per_launch"] if _kernel_sha16(t["source"], t["kernel"]) == t["sha16"] else None
    except (OSError, StopIteration):
        return None


def summary(line: dict) -> dict:
    """The headline figures again, compact, at the end of the line."""
    out = {"plain_fp64_2d512": round(line["value"], 3), "e2e_fp64_2d512": round(line["e2e"]["value"], 3),
           "roofline_frac": round(line["roofline"]["frac"], 3)}
    ch = line.get("chosen_form")
    if ch:
        out["chosen_2d512"] = {"form": ch["name"], "value": round(ch["value"], 3),
                               "speedup_vs_fp64": round(ch["speedup_vs_fp64"], 3), "iters": ch["iters"]}
    w3 = line.get("workload_3d")
    if w3:
        c3 = w3["chosen"]
        out["helmholtz_3d128"] = {k: {"value": round(v["value"], 4), "iters": v["iters"]}
                                  for k, v in w3["forms"].items()}
        if "roofline" in c3:
            out["helmholtz_3d128"]["tc_update_frac"] = round(c3["roofline"]["frac"], 3)
        if "schrodinger" in w3:
            out["schrodinger_3d128"] = {k: {"value": round(v["value"], 4), "iters": v["iters"]}
                                        for k, v in w3["schrodinger"]["forms"].items()}
    tp = line.get("tc_peak")
    if tp:
        out["tf32_kernel_tflops"] = {"burst": round(tp["tf32"]["burst_tflops"], 1),
                                     "sustained": round(tp["tf32"]["sustained_tflops"], 1)}
    wb = line.get("workload_batch")
    if wb:
        out["batch_2d"] = {"value": round(wb["value"], 2),
                           "speedup_vs_plain_fp64": round(wb["speedup_vs_plain_fp64"], 3)
                           if wb.get("speedup_vs_plain_fp64") else None}
        if wb.get("problem_groups"):
            out["batch_2d"]["problem_groups"] = round(wb["problem_groups"]["value"], 2)
    wl = line.get("workload_learned")
    if wl:
        out["learned_guess_speedup"] = round(wl["speedup_vs_zero_guess"], 3)
    cb = line.get("cpu_baseline")
    if cb:
        out["oracle_sample_128"] = round(cb["value"], 3)
        if cb.get("oracle_512_measured_once"):
            out["oracle_512"] = round(cb["oracle_512_measured_once"]["value"], 6)
    return out


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    from paper_1409_0297_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    if args.only_learned:
        if rank == 0:
            print(json.dumps({"workload_learned": measure_learned(args, B, torch, dist, world)}),
                  flush=True)
        return

    probs = []
    for w in problems(args.problems):
        d, n, b = w["d"], w["n"], w["b"]
        if w["kind"] == "helmholtz":
            s, q = B.sp_medium_helmholtz(d, n, w["omega"], w["c"])
            f = w["f"]
        else:
            s, q = B.sp_medium_schrodinger(d, n, w["ell"], w["E"], w["V"])
            f = w["f"] * w["ell"] ** 2
        probs.append(dict(d=d, n=n, b=b, s=s, q=q, f=np.ascontiguousarray(f)))
    N = probs[0]["n"] ** probs[0]["d"]

    # the two problems of a step are independent: each context gets its own CUDA stream
    # and the step drives them from two host threads (--serial-pair: one stream, in turn)
    import concurrent.futures as cf
    pair_streams = None if args.serial_pair else [torch.cuda.Stream() for _ in probs]
    pair_pool = None if args.serial_pair else cf.ThreadPoolExecutor(len(probs))

    def run_pair(fn, n_items, concurrent=True):
        if pair_streams is None or not concurrent:
            for i in range(n_items):
                fn(i)
            return
        cur = torch.cuda.current_stream()
        ev = torch.cuda.Event()
        ev.record(cur)
        for s_ in pair_streams:
            s_.wait_event(ev)
        list(pair_pool.map(fn, range(n_items)))
        for s_ in pair_streams:
            e_ = torch.cuda.Event()
            e_.record(s_)
            cur.wait_event(e_)

    def make(prec):
        out = []
        for i, p in enumerate(probs):
            S = B.Solver(p["d"], p["n"], p["b"], p["s"], prec=prec, device=local, sweeps=args.sweeps,
                         device_loop=args.device_loop,
                         autotune=not args.no_autotune,
                         stream=pair_streams[i].cuda_stream if pair_streams else 0)
            out.append(dict(S=S, q=torch.from_numpy(p["q"]).cuda(),
                            f=torch.from_numpy(p["f"]).cuda(),
                            u=torch.empty(N, dtype=torch.complex128, device="cuda")))
        return out

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    form_prec = {"fp64": B.SP_PREC_FP64, "fp32": B.SP_PREC_FP32, "tf32": B.SP_PREC_TF32,
                 "tf32x3": B.SP_PREC_TF32X3}
    if args.profile_tc_probe:
        ms = B.sp_tc_probe(0, 8192, 8192, 8192, 1)
        print(json.dumps({"profile_tc_probe": [8192, 8192, 8192], "ms": ms}), flush=True)
        return
    if args.profile_gemm:
        M, Nn, K, form = args.profile_gemm.split(",")
        M, Nn, K = int(M), int(Nn), int(K)
        gen = torch.Generator(device="cuda").manual_seed(7)
        A = torch.randn(K, M, device="cuda", generator=gen)
        Bt = torch.randn(Nn, K, device="cuda", generator=gen)
        C = torch.randn(Nn, M, device="cuda", generator=gen)
        for _ in range(3):
            B.sp_schur_update(form_prec[form], M, Nn, K, A.data_ptr(), M, 0, Bt.data_ptr(), K, 0,
                              C.data_ptr(), M, 0, 1)
        torch.cuda.synchronize()
        print(json.dumps({"profile_gemm": [M, Nn, K, form]}), flush=True)
        return
    if args.profile_step and args.profile_workload != "2d512":
        n = 64 if args.profile_workload == "3d64" else 128
        w = sm.helmholtz_grf_3d(n, 8, 0)
        s3, q3 = B.sp_medium_helmholtz(3, n, w["omega"], w["c"])
        half = args.profile_step.endswith("h")
        S = B.Solver(3, n, 8, s3, prec=form_prec[args.profile_step.rstrip("h")], device=local,
                     sweeps=args.sweeps, device_loop=args.device_loop,
                     factor_storage=1 if half else 0)
        u = torch.empty(n ** 3, dtype=torch.complex128, device="cuda")
        q3d = torch.from_numpy(q3).cuda()
        f3d = torch.from_numpy(np.ascontiguousarray(w["f"])).cuda()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        S.factor(q3d)
        info = S.solve(f3d, u)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": args.profile_step, "workload": args.profile_workload,
                          "iters": info["iters"], "true_relres": info["true_relres"]}), flush=True)
        S.close()
        return
    if args.profile_step:
        if args.profile_step.endswith("h"):
            raise SystemExit("the FP16 factor copy is profiled on the 3D workloads")
        ctxs = make(form_prec[args.profile_step])
        torch.cuda.synchronize()
        infos = []
        # one bench step between cudaProfilerStart / Stop: `ncu --profile-from-start off`
        # captures exactly its launches (not the set-up's autotuning)
        torch.cuda.profiler.start()
        for c in ctxs:
            c["S"].factor(c["q"])
            infos.append(c["S"].solve(c["f"], c["u"]))
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": args.profile_step,
                          "iters": [i["iters"] for i in infos],
                          "true_relres": [i["true_relres"] for i in infos]}), flush=True)
        for c in ctxs:
            c["S"].close()
        return

    def step(ctxs, infos=None, concurrent=True):
        res = [None] * len(ctxs)

        def one(i):
            c = ctxs[i]
            c["S"].factor(c["q"])
            res[i] = c["S"].solve(c["f"], c["u"])

        run_pair(one, len(ctxs), concurrent)
        if infos is not None:
            infos.extend(res)

    def timed(ctxs, K, W):
        for _ in range(W):
            step(ctxs)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        infos = []
        t0 = time.perf_counter()
        for _ in range(K):
            flush.zero_()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step(ctxs, infos)
            e.record()
            evs.append((a, e))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - t0
        ms = reduce_max(sum(a.elapsed_time(e) for a, e in evs), dist)
        return ms / K, wall, infos

    fp64 = make(B.SP_PREC_FP64)
    L2d = int(np.log2(probs[0]["n"] // probs[0]["b"]))
    shapes64 = [B.sp_tuning(fp64[0]["S"].ctx, l) for l in range(L2d + 1)]
    sampler = ClockSampler(local)
    sampler.start()
    ms64, wall64, infos64 = timed(fp64, args.steps, args.warmup)
    clocks = sampler.stop()
    solves_per_step = len(probs)
    value = replica_value(solves_per_step, world, ms64)

    # e2e through the host-buffer entry points (pinned host memory)
    pin_q = [torch.from_numpy(p["q"]).pin_memory() for p in probs]
    pin_f = [torch.from_numpy(p["f"]).pin_memory() for p in probs]
    pin_u = [torch.empty(N, dtype=torch.complex128).pin_memory() for _ in probs]
    import ctypes

    infos_c = [B.sp_info() for _ in probs]

    def step_host():
        def one(i):
            c, q, f, u = fp64[i], pin_q[i], pin_f[i], pin_u[i]
            B._check(B.LIB.sp_factor_host(c["S"].ctx, ctypes.c_void_p(q.data_ptr())), "sp_factor_host")
            B._check(B.LIB.sp_solve_host(c["S"].ctx, ctypes.c_void_p(f.data_ptr()),
                                         ctypes.c_void_p(u.data_ptr()), ctypes.byref(infos_c[i])),
                     "sp_solve_host")
        run_pair(one, len(probs))
    step_host()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_host()
    torch.cuda.synchronize()
    e2e_s = reduce_max((time.perf_counter() - t0) / args.steps, dist)
    e2e_value = replica_value(solves_per_step, world, e2e_s * 1e3)

    def profiled(ctxs):
        for c in ctxs:
            B.sp_profile(c["S"].ctx, True)
        step(ctxs, concurrent=False)  # one problem at a time: per-class times do not overlap
        out = {}
        for c in ctxs:
            for k, (ms_, nl, wk) in B.sp_profile_read(c["S"].ctx).items():
                a = out.setdefault(k, [0.0, 0, 0.0])
                a[0] += ms_
                a[1] += nl
                a[2] += wk
            B.sp_profile(c["S"].ctx, False)
        return out

    # one profiled step: kernel classes, launch counts, roofline of the dominant class
    prof = profiled(fp64)
    launches_per_step = sum(v[1] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp64_peak_tflops = 1.25  # nominal GB300 FP64 rate (no FP64 entry in the measured peaks)
    alu_classes = {"lu_panel", "lu_trsm", "lu_gemm", "lu_trinv"}

    def roof(k, vals):
        ms_, nl, wk = vals
        if k in alu_classes:
            ach = wk / (ms_ / 1e3) / 1e12
            return {"kernel": k, "bound": "alu", "achieved": ach, "peak": fp64_peak_tflops,
                    "unit": "TFLOP/s", "frac": ach / fp64_peak_tflops, "traffic": recorded_traffic(k),
                    "peak_source": "nominal FP64 1.25 TFLOP/s"}
        ach = wk / (ms_ / 1e3) / 1e9
        return {"kernel": k, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": recorded_traffic(k), "peak_source": "measured hbm_gbs"}

    roofline = roof(dom, prof[dom])
    breakdown = {k: {"ms": round(v[0], 3), "launches": v[1],
                     "achieved": round((v[2] / (v[0] / 1e3)) / (1e12 if k in alu_classes else 1e9), 3)
                     if v[0] > 0 else None,
                     "unit": "TFLOP/s" if k in alu_classes else "GB/s"} for k, v in prof.items()}

    chosen = None
    forms = {}
    if not args.no_chosen:
        for name, prec, desc in (
                ("fp32", B.SP_PREC_FP32, "FP32 factor and sweeps; FP64 operator, Gram-Schmidt, residuals"),
                ("tf32", B.SP_PREC_TF32, "FP32 factor and sweeps, Schur updates of fronts m >= 1024 "
                                         "on tcgen05 tensor cores (TF32 x TF32 -> FP32); FP64 "
                                         "operator, Gram-Schmidt, residuals"),
                ("tf32x3", B.SP_PREC_TF32X3, "as tf32 with 3xTF32 split operands (FP32-accurate "
                                             "updates)"),
                ("mixed", B.SP_PREC_MIXED, "GMRES-IR: FP32 factor and sweeps, complex64 inner FGMRES "
                                           "(FFT, Gram-Schmidt) to 1e-5, FP64 refinement residuals")):
            ctxs = make(prec)
            ms_f, _, infos_f = timed(ctxs, args.steps, args.warmup)
            prof_f = profiled(ctxs)
            forms[name] = {"form": desc, "value": replica_value(solves_per_step, world, ms_f),
                           "ms_per_step": ms_f, "speedup_vs_fp64": ms64 / ms_f,
                           "iters": [i["iters"] for i in infos_f[:solves_per_step]],
                           "true_relres": [i["true_relres"] for i in infos_f[:solves_per_step]],
                           "kernel_breakdown_ms_per_step": {k: {"ms": round(v[0], 3), "launches": v[1]}
                                                            for k, v in prof_f.items()}}
            for c in ctxs:
                c["S"].close()
        best = max(forms, key=lambda k: forms[k]["value"])
        chosen = dict(forms[best], name=best)

    for c in fp64:
        c["S"].close()
    fp64 = []
    torch.cuda.synchronize()
    wbatch = None
    if not args.no_batch:
        wbatch = measure_batch(args, B, torch, dist, world)
    wlearn = None
    if not args.no_learned:
        wlearn = measure_learned(args, B, torch, dist, world)
    tc_peak = None
    if not args.no_tc_probe:
        tc_peak = measure_tc_peak(B)
    w3d = None
    if not args.no_3d:
        w3d = measure_3d(args, B, torch, flush, peaks, tc_peak, dist, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_baseline()
        cpu = {"value": r["value"], "unit": UNIT, "cores": os.cpu_count(),
               "cores_busy": round(r["cores_busy"], 2), "kind": "oracle",
               "sample": r["sample"], "workload": REF_SAMPLE,
               "oracle_phases_best_of_3": oracle_phases(),
               "oracle_512_measured_once": ORACLE_512}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "512^2", "b": 16, "solves_per_step": 2,
                       "tol": 1e-8, "l2": "flushed between steps (256 MB write)",
                       "autotune": not args.no_autotune, "fp64_tile_shapes_by_level": shapes64,
                       "sweeps": ["fused on many-front levels, per-block chains elsewhere",
                                  "per-block launch chains", "one fused launch per level"][args.sweeps],
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "pair_concurrency": "one stream" if args.serial_pair else
                       "two CUDA streams, one host thread per problem"},
            "iters": [i["iters"] for i in infos64[:solves_per_step]],
            "true_relres": [i["true_relres"] for i in infos64[:solves_per_step]],
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(p["q"].nbytes + p["f"].nbytes for p in probs)),
                    "d2h_bytes_per_step": int(len(probs) * N * 16)},
            "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roofline, "kernel_breakdown_ms_per_step": breakdown,
            "chosen_form": chosen, "forms": {k: {kk: v[kk] for kk in ("value", "ms_per_step", "iters")}
                                             for k, v in forms.items()},
            "clocks": clocks, "cpu_baseline": cpu, "tc_peak": tc_peak, "workload_3d": w3d,
            "workload_batch": wbatch, "workload_learned": wlearn,
        }
        line["summary"] = summary(line)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.oracle_512:
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps({"oracle_512": oracle_512()}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Throughput of the GAMER-2 patch-group hydro step on B300.

Workload: decaying turbulence on a uniform periodic 512^3 box (32768 patch
groups of 2x2x2 patches of 8^3 cells), gamma=5/3, C_CFL=0.5; rho=1, P=0.6,
Gaussian random velocity with k^-4 power on 1<=|k|<=16, rms Mach 1 (seeded,
synthetic).  One "step" is one pass of the whole per-group hot path over the
level: ghost gather, PLM + van Leer, Hancock half step, HLLC, conservative
update, and the Eq. (CFL2) time-step reduction of the new state (the next
step's dt is computed on the device from it).

`value` is the FP64 step (the plain method); the FP32-compute /
FP64-accumulate step and the 256^3 box are reported beside it.  Inputs
(5.4 GB of state) are far larger than the 126 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N>1) each rank runs an independent replica (the uniform
step has no exchange on one GPU's box): value = all ranks' cell updates /
max over ranks of the timed region.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))

METRIC = "cell updates/s per B300 (FP64 & FP32) + % HBM roofline"
UNIT = "cells/s"
# Algorithmic FP64 operations per cell update (add/sub, mul, div and sqrt
# counted as one flop each) of one step plus the Eq. (CFL2) speed, counted by
# the instrumented oracle build (oracle/flop_count.cpp) on this workload.
ALG_FLOPS_PER_CELL = 1027.0
# Algorithmic HBM bytes per cell update: read U^n (5 doubles) + write U^{n+1}.
ALG_BYTES_PER_CELL = 80.0
# FP64 peak: 148 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2032 MHz (2 FMA/clk/SM
# measured: 5.55e11 DFMA/s at 1942 MHz); FP32: 148 x 128 x 2 x 2032 MHz.
FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12
# DRAM bytes (read+write) per cell update of one k_hydro_step launch from an
# ncu capture, keyed by the hash of the kernel sources it was taken on.
TRAFFIC_BYTES_PER_CELL = {"f64:3a53b9b9c1ffc44e": 86.75, "f32:3a53b9b9c1ffc44e": 92.5}
KERNEL_SOURCES = ("paper_1712_07070_b300/csrc/step_kernel.cuh", "paper_1712_07070_b300/csrc/hydro_math.cuh")


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(HERE, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=512, help="box edge (cells), multiple of 16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--adjoint-case", action="store_true",
                    help="only adjoint steps of an n^3 turbulence level (profiling case)")
    ap.add_argument("--boxes-case", action="store_true",
                    help="only the box batch restricted to the boxes of edge <= n (profiling case)")
    ap.add_argument("--sor-case", action="store_true",
                    help="only the refined-level SOR solve on the blob hierarchy with an n^3 root (profiling case)")
    ap.add_argument("--amr-case", action="store_true",
                    help="only root steps of the 3-level blob hierarchy with an n^3 root in the FP32-compute mode, "
                         "the timed ones between cudaProfilerStart/Stop (profiling case)")
    return ap.parse_args()


# ---- ranks --------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend, init_method="env://")
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x, device="cpu"):
    """Largest value of the float x over all ranks (x itself on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks during the timed region --------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


# ---- our arm --------------------------------------------------------------------------

def timed_steps(torch, grid, stream, K):
    """K device-dt steps on `stream`; returns (region ms, mean kernel ms)."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in evs:
        a.record(stream)
        grid.step(-1.0)
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), sum(a.elapsed_time(b) for a, b in evs) / K


def e2e_steps(torch, grid, stream, host_a, host_b, K, dt):
    """K chained steps through the public host-buffer API
    (UniformGrid.step_host -> amr_hydro_advance_host): every step copies its
    input state host->device from pinned memory, advances it and copies the new
    state back, the copies overlapped with the update by z-slabs; each step
    takes the CFL dt of the previous output.  Returns (ms, dt for the next
    step).  The calls return only when their output is on the host."""
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        dt = grid.step_host(host_a, host_b, dt)
        host_a, host_b = host_b, host_a
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), dt


def entropy(U, gamma=5.0 / 3.0):
    """s = P / rho^(gamma-1) of a dense state (the dual-energy variable)."""
    P = (gamma - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
    return P / U[0] ** (gamma - 1.0)


def run_case(torch, A, UniformGrid, U0, n, prec, K, W, stream, want_e2e, scheme=None):
    g = UniformGrid((n, n, n), prec=prec, stream=stream.cuda_stream, scheme=scheme)
    g.upload(torch.from_numpy(U0))
    if scheme and scheme.get("dual_energy"):
        g.set_entropy(entropy(U0))
    torch.cuda.synchronize()
    for _ in range(W):
        g.step(-1.0)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    region_ms, kernel_ms = timed_steps(torch, g, stream, K)
    clocks = clk.stop()
    torch.cuda.synchronize()
    barrier()
    out = {"region_ms": region_ms, "kernel_ms": kernel_ms, "clocks": clocks}
    if want_e2e:
        host_a = torch.from_numpy(U0).pin_memory()
        host_b = torch.empty_like(host_a).pin_memory()
        _, dt = e2e_steps(torch, g, stream, host_a, host_b, 1, -1.0)  # warm-up: CFL dt of U0
        barrier()
        e2e_ms, _ = e2e_steps(torch, g, stream, host_b, host_a, K, dt)
        barrier()
        out["e2e_ms"] = e2e_ms
        out["bytes"] = host_a.numel() * 8
    g.close()
    return out


def cpu_baseline(n, steps=8, slab=64):
    """The oracle, as it stands, on a bounded sample of the same workload:
    `steps` steps of a periodic n x n x slab box cut from the same seeded
    turbulence field, timed on all host cores."""
    import oracle
    from paper_1712_07070_b300 import ics
    U = ics.turbulence(n, seed=1)[:, :slab].copy()
    g = 5.0 / 3.0
    dt = oracle.dt_cfl2(U, g, 0.5, 1.0 / n)
    t0 = time.perf_counter()
    for _ in range(steps):
        U, _ = oracle.step_periodic(U, 1.0 / n, dt, g)
    el = time.perf_counter() - t0
    cells = n * n * slab * steps
    return {"value": cells / el, "unit": UNIT, "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
            "kind": "oracle",
            "sample": f"{steps} FP64 steps of a {n}x{n}x{slab} periodic slab of the same seeded turbulence field "
                      f"({cells} cell updates, {el:.1f} s)"}


def cpu_baseline_single_core(n, slab=16):
    """The same oracle step on one host core (a child process with
    OMP_NUM_THREADS=1): one FP64 step of an n x n x slab slab."""
    code = ("import time, oracle; from paper_1712_07070_b300 import ics; "
            f"U = ics.turbulence({n}, seed=1)[:, :{slab}].copy(); g = 5.0 / 3.0; "
            f"dt = oracle.dt_cfl2(U, g, 0.5, 1.0 / {n}); oracle.step_periodic(U, 1.0 / {n}, dt, g); "
            f"t0 = time.perf_counter(); oracle.step_periodic(U, 1.0 / {n}, dt, g); "
            "print(time.perf_counter() - t0)")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=HERE, env=env, capture_output=True, text=True, timeout=600)
    el = float(r.stdout.strip().splitlines()[-1])
    cells = n * n * slab
    return {"value": cells / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one FP64 step of a {n}x{n}x{slab} periodic slab of the same seeded turbulence field "
                      f"({cells} cell updates, {el:.1f} s)"}


def live_parity(torch, A, UniformGrid):
    """The Sod + noise workload (64^3, 10 steps, device dt) in both
    precisions against the FP64 oracle: relative L1 per conserved variable
    (the full-length checks of the other workloads are GPU tests)."""
    import numpy as np
    import oracle
    from paper_1712_07070_b300 import ics
    U0 = ics.sod_noise(64, seed=1)
    ref, _ = oracle.run_periodic(U0, 1.0 / 64, 5.0 / 3.0, 0.5, 10)
    out = {"workload": "Sod + 8 density modes + N(0,0.01) velocities, 64^3, 10 steps, vs the FP64 oracle",
           "metric": "relative L1 per conserved variable (max over the five)"}
    for prec, name in ((A.AMR_FP64, "f64"), (A.AMR_FP32_ACC64, "fp32_acc64")):
        g = UniformGrid((64, 64, 64), prec=prec)
        g.upload(U0)
        for _ in range(10):
            g.step(-1.0)
        u = g.download()
        g.close()
        out[name] = max(float(np.abs(u[v] - ref[v]).sum() / np.abs(ref[v]).sum()) for v in range(5))
    out["tolerance"] = {"f64": 1e-12, "fp32_acc64": 1e-5}
    return out


def repeats(torch, grid_factory, stream, K, reps=5):
    """Median (and spread) of the per-step time over `reps` further
    repetitions of K steps (after the timed region)."""
    g = grid_factory()
    ms = []
    for _ in range(reps):
        r, _ = timed_steps(torch, g, stream, K)
        ms.append(r / K)
    g.close()
    ms.sort()
    return {"n": reps, "steps_each": K, "ms_per_step": ms, "median_ms_per_step": ms[len(ms) // 2]}


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init("nccl")
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.uniform import UniformGrid
    A.lib()  # fails loudly when the CUDA library is missing
    n, K, W = args.n, args.steps, args.warmup
    stream = torch.cuda.Stream()
    U0 = ics.turbulence(n, seed=1)
    cells = n ** 3

    main = run_case(torch, A, UniformGrid, U0, n, A.AMR_FP64, K, W, stream, want_e2e=True)
    f32 = run_case(torch, A, UniformGrid, U0, n, A.AMR_FP32_ACC64, K, W, stream, want_e2e=True)
    variants = []
    if not args.no_variants and n != 256:
        U1 = ics.turbulence(256, seed=1)
        for prec, name in ((A.AMR_FP64, "f64"), (A.AMR_FP32_ACC64, "fp32_acc64")):
            r = run_case(torch, A, UniformGrid, U1, 256, prec, K, W, stream, want_e2e=False)
            ms = max_over_ranks(r["region_ms"], "cuda") / K
            variants.append({"workload": "turbulence 256^3", "dtype": name, "ms_per_step": ms,
                             "value": world * 256 ** 3 / (ms * 1e-3)})

    ms64 = max_over_ranks(main["region_ms"], "cuda") / K
    ms32 = max_over_ranks(f32["region_ms"], "cuda") / K
    e64 = max_over_ranks(main["e2e_ms"], "cuda") / K
    e32 = max_over_ranks(f32["e2e_ms"], "cuda") / K
    value = world * cells / (ms64 * 1e-3)
    kh = kernel_hash()
    tb = TRAFFIC_BYTES_PER_CELL.get(f"f64:{kh}")
    k64_s = main["kernel_ms"] * 1e-3
    k32_s = f32["kernel_ms"] * 1e-3
    ach64 = ALG_FLOPS_PER_CELL * cells / k64_s / 1e12
    roof = {"bound": "alu", "achieved": ach64, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach64 / FP64_PEAK_TFLOPS, "traffic": (tb * cells if tb else None),
            "kernel": "k_hydro_step<double>", "peak_kind": "derived: 148 SM x 2 DFMA/clk x 2 flop x 2032 MHz",
            "hbm_frac_of_measured": ALG_BYTES_PER_CELL * cells / k64_s / 1e9 / hbm_peak()}
    tb32 = TRAFFIC_BYTES_PER_CELL.get(f"f32:{kh}")
    ach32 = ALG_BYTES_PER_CELL * cells / k32_s / 1e9
    roof32 = {"bound": "hbm", "achieved": ach32, "peak": hbm_peak(), "unit": "GB/s",
              "frac": ach32 / hbm_peak(), "traffic": (tb32 * cells if tb32 else None),
              "kernel": "k_hydro_step<float>", "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)",
              "alu_fp32_frac": ALG_FLOPS_PER_CELL * cells / k32_s / 1e12 / FP32_PEAK_TFLOPS}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"decaying turbulence {n}^3 periodic, uniform level of 8^3 patches "
                               f"({cells // 4096} patch groups), MUSCL-Hancock+PLM(van Leer)+HLLC, CFL 0.5",
                   "cells": cells, "parallelism": f"replicas x{world}",
                   "l2": "inputs (5.4 GB state at 512^3) larger than L2; no flush"},
        "roofline": roof,
        "e2e": {"value": world * cells / (e64 * 1e-3), "unit": UNIT, "h2d_bytes_per_step": main["bytes"],
                "d2h_bytes_per_step": main["bytes"]},
        "gpu_launches": K,
        "clocks": main["clocks"],
        "fp32_acc64": {"value": world * cells / (ms32 * 1e-3), "ms_per_step": ms32, "dtype": "fp32_acc64",
                       "roofline": roof32, "clocks": f32["clocks"], "gpu_launches": K,
                       "e2e": {"value": world * cells / (e32 * 1e-3), "unit": UNIT,
                               "h2d_bytes_per_step": f32["bytes"], "d2h_bytes_per_step": f32["bytes"]}},
        "variants": variants,
        "kernel_hash": kh,
    }
    if not args.no_variants:
        line["schemes"] = bench_schemes(torch, A, UniformGrid, stream, K, W, world)
        line["amr"] = bench_amr(torch, args)
        line["boxes"] = bench_boxes(torch, args)
        line["adjoint"] = bench_adjoint(torch, args)
        line["gravity"] = bench_gravity(torch, args)
    if not args.no_variants:
        def mk(prec):
            def f():
                g = UniformGrid((n, n, n), prec=prec, stream=stream.cuda_stream)
                g.upload(torch.from_numpy(U0))
                for _ in range(W):
                    g.step(-1.0)
                return g
            return f
        line["repeats"] = {"f64": repeats(torch, mk(A.AMR_FP64), stream, K),
                           "fp32_acc64": repeats(torch, mk(A.AMR_FP32_ACC64), stream, K)}
        line["parity"] = live_parity(torch, A, UniformGrid)
        line["breakdown"] = {
            "uniform level": "ghost gather, solve and the dt reduction of Eq. (CFL2) are fused in one "
                             "k_hydro_step launch per step (no separate ghost-fill or reduce pass); the AMR "
                             "workload's amr.*.phases_ms_per_root_step splits ghost fill / step / fix-up / "
                             "regrid / dt"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n)
        line["cpu_baseline"]["single_core"] = cpu_baseline_single_core(n)
    if rank == 0:
        print(json.dumps(line), flush=True)


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def bench_schemes(torch, A, UniformGrid, stream, K, W, world):
    """The other slope limiters and Riemann solvers of section 2.2 (HLLE for
    every limiter; Roe and the exact solver with the van Leer-type limiter)
    the VL scheme (van Leer-type with HLLC and with HLLE) and the CTU scheme
    (van Leer-type with HLLC and with Roe), PPM with MUSCL-Hancock + HLLC and
    with CTU + Roe (the scheme of the paper's Kelvin-Helmholtz runs), the
    remedies for unphysical results and the dual-energy formalism, on the
    256^3 turbulence level, the default MUSCL-Hancock + PLM van Leer-type +
    HLLC for reference: cells/s per precision."""
    from paper_1712_07070_b300 import ics
    U1 = ics.turbulence(256, seed=1)
    names = {A.AMR_LIM_VANLEER: "van Leer", A.AMR_LIM_GMINMOD: "generalized minmod 1.5",
             A.AMR_LIM_ALBADA: "van Albada", A.AMR_LIM_VL_GMINMOD: "hybrid van Leer/minmod 1.5"}
    out = []
    MH, VL, CTU = A.AMR_SCHEME_MH, A.AMR_SCHEME_VL, A.AMR_SCHEME_CTU
    PLM, PPM = A.AMR_RECON_PLM, A.AMR_RECON_PPM
    VLR = A.AMR_LIM_VANLEER
    combos = [(lim, rs, MH, PLM) for lim in names for rs in (A.AMR_RS_HLLC, A.AMR_RS_HLLE)]
    combos += [(VLR, A.AMR_RS_ROE, MH, PLM), (VLR, A.AMR_RS_EXACT, MH, PLM)]
    combos += [(VLR, A.AMR_RS_HLLC, VL, PLM), (VLR, A.AMR_RS_HLLE, VL, PLM)]
    combos += [(VLR, A.AMR_RS_HLLC, CTU, PLM), (VLR, A.AMR_RS_ROE, CTU, PLM)]
    combos += [(VLR, A.AMR_RS_HLLC, MH, PPM), (VLR, A.AMR_RS_ROE, CTU, PPM)]
    # the remedies for unphysical results and the dual-energy formalism (options)
    combos += [(VLR, A.AMR_RS_HLLC, MH, PLM, {"fallback": 1}), (VLR, A.AMR_RS_HLLC, MH, PLM, {"dual_energy": 1})]
    rnames = {A.AMR_RS_HLLC: "HLLC", A.AMR_RS_HLLE: "HLLE", A.AMR_RS_ROE: "Roe", A.AMR_RS_EXACT: "exact"}
    snames = {MH: "MUSCL-Hancock", VL: "VL", CTU: "CTU (6 solves/cell, Eq. CFL1)"}
    for lim, rs, scheme, recon, *extra in combos:
        opts = extra[0] if extra else {}
        sch = dict({"limiter": lim, "riemann": rs, "minmod_coeff": 1.5, "scheme": scheme, "recon": recon}, **opts)
        row = dict({"workload": "turbulence 256^3", "scheme": snames[scheme], "recon": "PPM" if recon == PPM else "PLM",
                    "limiter": names[lim], "riemann": rnames[rs]}, **opts)
        for prec, key in ((A.AMR_FP64, "f64"), (A.AMR_FP32_ACC64, "fp32_acc64")):
            r = run_case(torch, A, UniformGrid, U1, 256, prec, K, W, stream, want_e2e=False, scheme=sch)
            ms = max_over_ranks(r["region_ms"], "cuda") / K
            row[key] = world * 256 ** 3 / (ms * 1e-3)
        out.append(row)
    return {"unit": UNIT, "rows": out}


def bench_amr(torch, args):
    """3-level AMR: root 128^3 + 2 levels around 3 Gaussian blobs (contrast 100,
    sigma 0.05) moving at Mach 2, adaptive W-cycle with fix-up and regrid every
    level step; cell updates of all levels and substeps per second."""
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.amr import AmrHierarchy
    U0 = ics.blobs(128, seed=3)
    out = {"workload": "AMR 128^3 root, lmax 2, 3 blobs (contrast 100, sigma 0.05, Mach 2), theta 0.1, "
                       "N_buf 8/4, adaptive dt W-cycle with fix-up and regrid", "unit": UNIT}
    for prec, name in ((A.AMR_FP64, "f64"), (A.AMR_FP32_ACC64, "fp32_acc64")):
        H = AmrHierarchy(U0, lmax=2, theta=0.1, nbuf=(8, 4), prec=prec, max_patches=120000)
        for _ in range(max(1, args.warmup // 2)):
            H.advance_root()
        torch.cuda.synchronize()
        K = max(2, args.steps // 2)
        e0, e1 = _events(torch)
        e0.record()
        n = 0
        for _ in range(K):
            n += H.advance_root()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"value": n / (ms * 1e-3), "ms_per_root_step": ms / K, "cell_updates_per_root_step": n // K,
                     "patches": [H.n_patches(l) for l in range(3)]}
        # where a root step's time goes: event pairs around each phase on the
        # context's stream, over two further root steps (after the timed region)
        A.amr_hydro_phase_timing(H.ctx, True)
        A.amr_hydro_phase_times(H.ctx)
        for _ in range(2):
            H.advance_root()
        ph = A.amr_hydro_phase_times(H.ctx)
        A.amr_hydro_phase_timing(H.ctx, False)
        tot = sum(v[0] for v in ph.values())
        out[name]["phases_ms_per_root_step"] = {k: v[0] / 2 for k, v in ph.items()}
        out[name]["phase_share"] = {k: (v[0] / tot if tot > 0 else None) for k, v in ph.items()}
        H.close()
    out["value"] = out["f64"]["value"]
    return out


def bench_gravity(torch, args):
    """Gravity solvers (section 2.3): the root level's periodic FFT Poisson
    solve with accelerations on the 256^3 turbulence density, and the
    per-patch SOR solve (18^3 grid per patch, 60 red-black iterations,
    omega 1.7) with accelerations on the first refined level of the 3-level
    blob hierarchy of the AMR workload."""
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.amr import AmrHierarchy
    from paper_1712_07070_b300.uniform import UniformGrid

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"unit": UNIT}
    n = 256
    g = UniformGrid((n, n, n))
    g.upload(torch.from_numpy(ics.turbulence(n, seed=1)))
    phi = torch.zeros((g.n_patches, 8, 8, 8), dtype=torch.float64, device="cuda")
    acc = torch.zeros((g.n_patches, 3, 8, 8, 8), dtype=torch.float64, device="cuda")
    ms = timed(lambda: A.amr_hydro_poisson_root(g.ctx, 1.0, phi, acc, 2), 5)
    out["root_fft"] = {"workload": "periodic FFT Poisson + 2-point accelerations, 256^3 root level (own mixed-radix FFT)",
                       "ms": ms, "value": n ** 3 / (ms * 1e-3)}
    g.close()
    g = UniformGrid((n, n, n), scheme={"gravity_bc": A.AMR_GRAVITY_ISOLATED})
    g.upload(torch.from_numpy(ics.turbulence(n, seed=1)))
    ms = timed(lambda: A.amr_hydro_poisson_root(g.ctx, 1.0, phi, acc, 2), 5)
    out["root_fft_isolated"] = {"workload": "isolated FFT Poisson (zero-padded to 540x525x525, pruned transforms) + 2-point accelerations, "
                                            "256^3 root level (own mixed-radix FFT), FP64", "ms": ms, "value": n ** 3 / (ms * 1e-3)}
    g.close()
    for prec, tag, sch in ((A.AMR_FP64, "fp64", None), (A.AMR_FP32_ACC64, "fp32", None),
                           (A.AMR_FP64, "ctu_fp64", {"scheme": A.AMR_SCHEME_CTU})):
        g = UniformGrid((n, n, n), prec=prec, scheme=sch)
        g.upload(torch.from_numpy(ics.turbulence(n, seed=1)))
        state = {"acc": g.gravity(1.0, 2)[1]}

        def coupled():
            state["acc"] = g.step_gravity(1.0, state["acc"], -1.0, 2)[1]

        ms = timed(coupled, 5)
        out[f"coupled_{tag}"] = {"workload": f"hydro + self-gravity step ({'CTU' if sch else 'MUSCL-Hancock'} "
                                             "+ PLM + HLLC with the gravity predictor, FFT potential of the "
                                             f"predicted density, corrector), 256^3 turbulence, {tag}", "ms": ms,
                                 "value": n ** 3 / (ms * 1e-3)}
        g.close()
    for prec, tag in ((A.AMR_FP64, ""), (A.AMR_FP32_ACC64, "_fp32")):
        H = AmrHierarchy(ics.blobs(128, seed=3), lmax=2, theta=0.1, nbuf=(8, 4), max_patches=120000, prec=prec)
        phi0 = torch.zeros((H.n_patches(0), 8, 8, 8), dtype=torch.float64, device="cuda")
        A.amr_hydro_poisson_root(H.ctx, 1.0, phi0)
        n1 = H.n_patches(1)
        phi1 = torch.zeros((n1, 8, 8, 8), dtype=torch.float64, device="cuda")
        acc1 = torch.zeros((n1, 3, 8, 8, 8), dtype=torch.float64, device="cuda")
        ms = timed(lambda: A.amr_hydro_poisson_level(H.ctx, 1, 1.0, 1.7, 60, phi0, phi1, acc1, 2), 3)
        out["sor" + tag] = {"workload": f"SOR on 18^3 per patch, 60 red-black iterations, {n1} level-1 patches "
                                        f"of the blob hierarchy, {'FP64' if not tag else 'FP32 compute'}",
                            "ms": ms, "value": n1 * 512 / (ms * 1e-3),
                            "point_updates_per_s": n1 * 60 * 4096 / (ms * 1e-3)}
        H.close()
    return out


def bench_boxes(torch, args):
    """64 periodic Kelvin-Helmholtz boxes of seeded sizes {32..192}^3, one
    persistent launch per step over all of them, CUDA graph, autotuned."""
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.boxes import BoxBatch
    sizes = ics.kh_batch_sizes(64, seed=4)
    cells = sum(n ** 3 for n in sizes)
    B = BoxBatch(gamma=1.4, prec=A.AMR_FP32_ACC64)
    for i, n in enumerate(sizes):
        B.add_box(ics.kh_box(n, seed=100 + i, gamma=1.4))
    B.advance(args.steps)  # autotune + capture the graph of K steps
    B.advance(args.steps)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    B.advance(args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    tune = B.tuning()
    B.close()
    return {"workload": f"64 periodic KH boxes, sizes {{32..192}}^3 (seed 4), {cells} cells, gamma 1.4, FP32 "
                        f"compute / FP64 accumulate, one persistent launch per step, CUDA graph",
            "value": cells / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "cells": cells, "tuning": tune,
            "dtype": "fp32_acc64"}


def bench_adjoint(torch, args):
    """Adjoint/forward time ratio: 128^3 turbulence, 40 FP64 steps with a
    frozen dt sequence, sqrt(N) checkpoints; backward = segment recompute +
    adjoint kernels."""
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.adjoint import CheckpointedRun
    n, N = 128, 40
    run = CheckpointedRun((n, n, n))
    U0 = torch.from_numpy(ics.turbulence(n, seed=5)).cuda()
    for _ in range(2):  # spin up away from the uniform-density limiter kinks
        run.grid.upload(U0)
        run.grid.step(-1.0)
        U0 = run.grid.download(out=torch.empty_like(U0))
    dts = run.record_dts(U0, N)
    lam = torch.zeros_like(U0)
    lam[0] = 1.0 / n ** 3
    run.forward(U0, dts)  # warm-up
    run.backward(lam)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    run.forward(U0, dts)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1)
    e0.record()
    run.backward(lam)
    e1.record()
    torch.cuda.synchronize()
    bwd = e0.elapsed_time(e1)
    run.close()
    return {"workload": "adjoint of 40 FP64 steps of 128^3 turbulence, sqrt(N) checkpoints", "forward_ms": fwd,
            "backward_ms": bwd, "adjoint_forward_ratio": bwd / fwd,
            "value": n ** 3 * N / (bwd * 1e-3), "unit": "adjoint cell updates/s"}


def hbm_peak():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0  # fallback figure


# ---- reference arm: the oracle on the host cores ----------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n, K, W = args.n, args.steps, args.warmup
    import oracle
    from paper_1712_07070_b300 import ics
    slab = 16
    U = ics.turbulence(n, seed=1)[:, :slab].copy()
    g = 5.0 / 3.0
    for _ in range(W):
        dt = oracle.dt_cfl2(U, g, 0.5, 1.0 / n)
        U, _ = oracle.step_periodic(U, 1.0 / n, dt, g)
    t0 = time.perf_counter()
    for _ in range(K):
        dt = oracle.dt_cfl2(U, g, 0.5, 1.0 / n)
        U, _ = oracle.step_periodic(U, 1.0 / n, dt, g)
    el = time.perf_counter() - t0
    cells = n * n * slab
    value = cells * K / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count()))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": el / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": f"decaying turbulence {n}^3 periodic (oracle: bounded sample)", "cells": n ** 3},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: one FP64 step of a {n}x{n}x{slab} periodic slab of the same "
                                   f"seeded turbulence field ({cells} cell updates)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def sor_case(args):
    """The refined-level Poisson solve alone: SOR (60 red-black iterations,
    omega 1.7, two-point accelerations) on level 1 of the blob hierarchy
    with an n^3 root (3 blobs, seed 3, theta 0.1, N_buf 8), after the root
    FFT solve; ``--warmup`` untimed and ``--steps`` timed solves, one JSON line."""
    import torch
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.amr import AmrHierarchy
    H = AmrHierarchy(ics.blobs(args.n, seed=3), lmax=1, theta=0.1, nbuf=(8,), max_patches=120000)
    phi0 = torch.zeros((H.n_patches(0), 8, 8, 8), dtype=torch.float64, device="cuda")
    A.amr_hydro_poisson_root(H.ctx, 1.0, phi0)
    n1 = H.n_patches(1)
    phi1 = torch.zeros((n1, 8, 8, 8), dtype=torch.float64, device="cuda")
    acc1 = torch.zeros((n1, 3, 8, 8, 8), dtype=torch.float64, device="cuda")

    def solve():
        A.amr_hydro_poisson_level(H.ctx, 1, 1.0, 1.7, 60, phi0, phi1, acc1, 2)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(args.steps):
        solve()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"metric": "SOR point updates per second", "value": n1 * 60 * 4096 / (ms * 1e-3),
                      "unit": "point updates/s", "ms_per_solve": ms, "patches": n1,
                      "config": {"workload": f"SOR, 60 iterations, level 1 of the {args.n}^3-root blob hierarchy"}}))
    H.close()


def adjoint_case(args):
    """The adjoint step alone: --warmup untimed and --steps timed
    amr_hydro_step_adjoint calls on an n^3 turbulence level (two spin-up
    steps, dt of Eq. CFL2); one JSON line."""
    import torch
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.uniform import UniformGrid
    n = args.n
    g = UniformGrid((n, n, n))
    g.upload(torch.from_numpy(ics.turbulence(n, seed=5)))
    for _ in range(2):
        g.step(-1.0)
    dt = g.min_dt()
    U = g.state().clone()
    lam = torch.zeros_like(U)
    lam[:, 0] = 1.0 / n ** 3
    out = torch.empty_like(U)
    for _ in range(args.warmup):
        A.amr_hydro_step_adjoint(g.ctx, 0, dt, U, lam, out)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(args.steps):
        A.amr_hydro_step_adjoint(g.ctx, 0, dt, U, lam, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"metric": "adjoint cell updates/s", "value": n ** 3 / (ms * 1e-3), "unit": "cells/s",
                      "ms_per_step": ms, "config": {"workload": f"adjoint of one FP64 step, {n}^3 turbulence"}}))
    g.close()


def boxes_case(args):
    """The box batch alone, on the boxes of edge <= n of the seeded 64-box
    set (FP32 mode, autotuned launch): --warmup untimed and --steps timed
    steps; one JSON line."""
    import torch
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.boxes import BoxBatch
    sizes = [m for m in ics.kh_batch_sizes(64, seed=4) if m <= args.n]
    B = BoxBatch(gamma=1.4, prec=A.AMR_FP32_ACC64)
    for i, m in enumerate(sizes):
        B.add_box(ics.kh_box(m, seed=100 + i, gamma=1.4))
    B.advance(max(args.warmup, 1), log=False)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    B.advance(args.steps, log=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    cells = sum(m ** 3 for m in sizes)
    print(json.dumps({"metric": "cell updates/s", "value": cells / (ms * 1e-3), "unit": "cells/s",
                      "ms_per_step": ms, "boxes": len(sizes), "cells": cells,
                      "config": {"workload": f"KH box batch, the {len(sizes)} boxes of edge <= {args.n}"}}))
    B.close()


def amr_case(args):
    """The AMR workload alone (3 blobs, seed 3, theta 0.1, N_buf 8/4, lmax 2,
    n^3 root, FP32 compute): --warmup untimed root steps, then --steps timed
    ones inside cudaProfilerStart/Stop (for a launch list with ncu's
    --profile-from-start off); one JSON line."""
    import torch
    from paper_1712_07070_b300 import amr_hydro as A
    from paper_1712_07070_b300 import ics
    from paper_1712_07070_b300.amr import AmrHierarchy
    H = AmrHierarchy(ics.blobs(args.n, seed=3), lmax=2, theta=0.1, nbuf=(8, 4), prec=A.AMR_FP32_ACC64,
                     max_patches=120000)
    for _ in range(args.warmup):
        H.advance_root()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    e0, e1 = _events(torch)
    e0.record()
    n = 0
    for _ in range(args.steps):
        n += H.advance_root()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"metric": "cell updates/s", "value": n / max(args.steps, 1) / (ms * 1e-3), "unit": "cells/s",
                      "ms_per_root_step": ms, "patches": [H.n_patches(l) for l in range(3)],
                      "config": {"workload": f"AMR blobs, {args.n}^3 root, lmax 2, FP32 compute"}}))
    H.close()


def main():
    args = parse()
    if args.amr_case:
        amr_case(args)
        return
    if args.sor_case:
        sor_case(args)
        return
    if args.adjoint_case:
        adjoint_case(args)
        return
    if args.boxes_case:
        boxes_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

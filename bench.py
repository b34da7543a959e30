"""Benchmark of the reduced-space IPM hot path on one GB300.

Metric: scenario condensations per second (one scenario condensed and reduced
at one interior-point iteration = one condensation) and seconds per IPM
iteration.  Default workload: the mixed-precision configuration, a 10,000-bus
network with 1,000 generators and 256 scenarios (n_x = 18,999, n_u = 1,999),
on the mixed path (FP32 multi-RHS solves, BF16x3 tensor-core contraction,
FP64 LU, Cholesky and refinement); the plain FP64 path is timed on the same
iterates for comparison (a few steps: about 20 s each).  --workload
opf1000_n64 --precision fp64_tc gives the 1,000-bus / 64-scenario workload
on the FP64_TC path.  A step is one full IPM iteration (evaluation,
condensation, reduction, Cholesky with inertia correction, step recovery
with refinement, line search) over all scenarios; the states cycle through
complete solves from the cold start (re-initialised, untimed, whenever a
solve converges).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  --impl reference times the CPU oracle (the plain FP64
numpy/scipy implementation in oracle/) on a bounded sample of the same
workload.
"""
from __future__ import annotations

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

from paper_2301_04869_gb300 import synth  # noqa: E402

METRIC = "scenario condensations/s & s per IPM iter (mixed vs FP64 path, 1e-8 KKT res)"
# FP64 arithmetic peak of a GB300: 2 FP64 FMA per clock per SM x 152 SMs x 2.07 GHz = 1.259 TFLOP/s,
# the 1.25 TFLOP/s FP64 figure of the profiling recipe (a cuBLAS DGEMM measured 1.10 TFLOP/s here).
FP64_PEAK_TFLOPS = 1.25
# FP32 (SIMT) arithmetic peak: 128 FP32 FMA per clock per SM x 152 SMs x 2.07 GHz = 80.5 TFLOP/s.
FP32_PEAK_TFLOPS = 80.5
# DRAM bytes per launch from one ncu capture of the kernel as it stands (profiles/); None once the
# kernel changes until it is captured again.
TRAFFIC = {"k_gemm_tn64": 590.125568e6 + 25.997568e6,   # DRAM read + write, one launch, 1000 buses x 64
           "k_zsolve64": 1.691865e9 + 865.253632e6,
           "k_emu_schur": 1.137726e9 + 3.871488e6}
UNIT = "scenario condensations/s"
REF_BUDGET_S = 150.0  # timed host seconds of the reference arm on the 10,000-bus workload


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = [r.split(",") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


def emu_issued_flops(nu, krows):
    """BF16 tensor-core flops one emulated contraction issues: 36 slice products
    over every 128 x 64 upper tile and every (512-row padded) contraction row."""
    ntm, ntn = -(-nu // 128), -(-nu // 64)
    ntiles = sum(1 for a in range(ntm) for b in range(ntn) if a * 128 <= b * 64 + 63)
    kpad = -(-krows // 512) * 512
    return 36 * 2.0 * kpad * 128 * 64 * ntiles


def roofline(phases, dims, peaks, peak_kind, precision):
    """Roofline entry for the dominant kernel phase (device time share)."""
    # the dominant kernel among the phases that are one kernel (family); recover (the
    # step recovery: single-vector solves, CG and refinement), linesearch, reduced_rhs and
    # fallback (a mixed iteration condensed again in FP64) are sequences of kernels, and
    # their single-vector solves are timed on their own as solve1
    composite = {"recover", "linesearch", "reduced_rhs", "fallback"}
    name = max((k for k in phases if k not in composite), key=lambda k: phases[k][0])
    ms, calls = phases[name]
    N, nx, nu = dims.n_scen, dims.n_x, dims.n_u
    per_call_s = ms / 1e3 / max(calls, 1)
    fp64_peak = FP64_PEAK_TFLOPS
    # algorithmic flops of K_hat: the upper triangle of sum_i Z_i^T Y_i (symmetric)
    kflops = 2.0 * nx * (nu * (nu + 1) / 2.0) * N
    if name == "gemm" and precision == "fp64_tc":
        issued = emu_issued_flops(nu, N * nx)
        ach = issued / per_call_s / 1e12
        pk = peaks["bf16_tflops_sustained"]
        return {"kernel": "k_emu_schur (FP64-grade Z^T Y from exact BF16 slices, tcgen05)", "bound": "tensor",
                "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": TRAFFIC.get("k_emu_schur"),
                "algorithmic": f"{issued:.4g} BF16 flop/launch issued (36 slice products); "
                               f"{kflops:.4g} FP64 flop/launch of the contraction itself",
                "fp64_equivalent_tflops": kflops / per_call_s / 1e12}
    if name == "gemm" and precision == "mixed":
        return {"kernel": "k_tc_schur (BF16x3, tcgen05)", "bound": "tensor",
                "achieved": 6 * kflops / per_call_s / 1e12, "peak": peaks["bf16_tflops_sustained"],
                "unit": "TFLOP/s", "frac": 6 * kflops / per_call_s / 1e12 / peaks["bf16_tflops_sustained"],
                "traffic": None, "algorithmic": f"{6 * kflops:.4g} BF16 flop/launch (6 split products)"}
    if name == "gemm":
        ach = kflops / per_call_s / 1e12
        return {"kernel": "k_gemm_tn64 (FP64 Z^T Y + scenario sum)", "bound": "alu", "achieved": ach,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                "traffic": TRAFFIC.get("k_gemm_tn64"),
                "algorithmic": f"{kflops:.4g} flop/launch"}
    if name == "zsolve":
        # the solves with the n_u (+ 1 on the FP64 paths) dense right-hand sides (the columns of
        # G_u and g) and the products Y = K_x [Z; I], Y_u = K_u [Z; I]
        nrhs = nu if precision == "mixed" else nu + 1
        solve = 2.0 * dims.nnz_lu * nrhs * N
        prod = 2.0 * (dims.nnz_kx + dims.nnz_ku) * nu * N
        flops = solve + prod
        ach = flops / per_call_s / 1e12
        if precision == "mixed":
            kern = ("k_zsolve32 + k_btrsm_diag/update (FP32 multi-RHS solves, the dense trailing block by "
                    "batched blocked triangular solves, products with K)")
            pk = FP32_PEAK_TFLOPS
        else:
            kern = "k_zsolve64 (FP64 multi-RHS solves + products with K)"
            pk = fp64_peak
        return {"kernel": kern, "bound": "alu", "achieved": ach,
                "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": TRAFFIC.get("k_zsolve64") if precision != "mixed" else None,
                "algorithmic": f"{flops:.4g} flop/launch ({solve:.4g} solves + {prod:.4g} products with K)"}
    if name == "solve1":
        # one vector per scenario through G_x or G_x^T: the factor read once, the vector in and out
        byt = 8.0 * (dims.nnz_lu + 2 * nx) * N
        ach = byt / per_call_s / 1e9
        return {"kernel": "k_solve1 + k_trsv_first/k_trsv_step (single-vector FP64 solves: sparse levels in "
                          "one CTA per scenario, the dense trailing block by multi-CTA sweeps)",
                "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None,
                "algorithmic": f"{byt:.4g} B/solve (the LU factors once, the vector in and out)",
                "solves_timed": calls}
    if name == "lu":
        # sparse eliminations (one FMA each) and, with a dense trailing block, its LU (2/3 nd^3)
        flops = (2.0 * dims.lu_sparse_ops + (2.0 / 3.0) * dims.nd ** 3) * N
        ach = flops / per_call_s / 1e12
        return {"kernel": "k_lu_factor + trailing-block LU (k_blu_*; FP64-grade tensor-core updates on the "
                          "mixed and FP64_TC paths)" if dims.big_block else "k_lu_factor_pair",
                "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                "traffic": None, "algorithmic": f"{flops:.4g} FP64 flop/launch"}
    # bandwidth-type phases: bytes of Z and Y touched
    byt = 8.0 * nx * nu * N * 2
    ach = byt / per_call_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": None}


def oracle_sample(workload):
    """Scenarios per oracle sample: all of the 1000-bus workload's 64 (one
    IPM iteration ~5-10 s on the host), one of the 10,000-bus workload's 256
    (one iteration on one scenario ~30-40 s)."""
    n_bus, _, N = synth.CONFIGS[workload][:3]
    return N if n_bus <= 2000 else 1


def cpu_baseline(workload, min_s=10.0, max_iters=40):
    """The oracle, as it stands, on a bounded sample: IPM iterations from the
    cold start on the first oracle_sample(workload) scenarios of the
    workload, until about `min_s` seconds of CPU work (at least 2 iterations
    on the 1000-bus workload, 1 on the 10,000-bus one; at most `max_iters`; a
    converged solve restarts from the cold start)."""
    from oracle import ipm as oipm
    from oracle import opf
    n_sample = oracle_sample(workload)
    net, pd, qd = synth.workload(workload, n_scen=n_sample)
    M = opf.Model(net, pd, qd)
    st = oipm.initial_state(M)
    iters = 0
    min_it = 2 if synth.CONFIGS[workload][0] <= 2000 else 1
    t0 = time.perf_counter()
    while iters < max_iters and (iters < min_it or time.perf_counter() - t0 < min_s):
        conv, _ = oipm.iterate(M, st)
        iters += 1
        if conv:
            st = oipm.initial_state(M)
    dt = time.perf_counter() - t0
    return {"value": n_sample * iters / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{iters} IPM iterations from the cold start on {n_sample} of the workload's scenarios "
                      f"({dt:.1f} s, numpy/scipy FP64, BLAS threads = all cores)",
            "s_per_ipm_iter": dt / iters}


def run_reference(args):
    """The oracle as the reference arm: each step one oracle IPM iteration on
    the sample of oracle_sample(workload) scenarios (from the cold start; a
    converged solve restarts).  On the 10,000-bus workload a step takes about
    30-40 s of host time, so the run stops after REF_BUDGET_S seconds of timed
    steps (at least one) and skips the warm-up (CPU code needs none); the line
    reports the steps it timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import ipm as oipm
    from oracle import opf
    n_sample = oracle_sample(args.workload)
    big = synth.CONFIGS[args.workload][0] > 2000
    net, pd, qd = synth.workload(args.workload, n_scen=n_sample)
    M = opf.Model(net, pd, qd)
    st = oipm.initial_state(M)
    for _ in range(0 if big else args.warmup):
        conv, _ = oipm.iterate(M, st)
        if conv:
            st = oipm.initial_state(M)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        conv, _ = oipm.iterate(M, st)
        times.append(time.perf_counter() - t0)
        if conv:
            st = oipm.initial_state(M)
        if big and sum(times) > REF_BUDGET_S:
            break
    tot = sum(times)
    val = n_sample * len(times) / tot
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": len(times),
            "warmup": 0 if big else args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "scenarios_timed": n_sample, "path": "oracle FP64 (CPU)",
                       "steps_requested": args.steps},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step = one IPM iteration on {n_sample} of the workload's scenarios"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def fallback_count(sol):
    """Iterations of a mixed-precision context that were condensed again in
    FP64 so far (its IPM_Q_INFO fallback counter; 0 on the FP64 paths)."""
    from paper_2301_04869_gb300 import ipm
    return int(sol.ipm_get_quantity(ipm.Q_INFO)[10])


def raise_count(sol):
    """Times a mixed-precision context raised delta_w after CG met non-positive
    curvature of the exact reduced operator (IPM_Q_INFO; 0 on the FP64 paths)."""
    from paper_2301_04869_gb300 import ipm
    return int(sol.ipm_get_quantity(ipm.Q_INFO)[18])


def measure_path(ipm, net, pd, qd, precision, steps, warmup, world, local, flush, want_e2e=True, want_phases=True,
                 phase_steps=None):
    """Time `steps` IPM iterations of one precision path (device events per step,
    L2 flushed between steps; graphs and autotuned launch shapes on), then the
    first `phase_steps` (default all) of the same iterates again with the phase
    timers on, and the same iterates end to end."""
    import torch
    prec = {"fp64": ipm.PREC_FP64, "mixed": ipm.PREC_MIXED, "fp64_tc": ipm.PREC_FP64_TC}[precision]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sol = ipm.Solver(net, pd, qd, precision=prec, graphs=True, autotune=True)
        dims = sol.dims
        N = dims.n_scen

        def step():
            conv, _ = sol.ipm_step(stream=stream)
            if conv:  # a converged check takes no step: restart (untimed) and redo
                sol.ipm_init_state(stream=stream)
                conv, _ = sol.ipm_step(stream=stream)

        for _ in range(warmup):
            step()
        # checkpoint: the phase pass and the end-to-end pass restart from it,
        # so all three passes time the same iterates
        ck = torch.empty(dims.state_len, dtype=torch.float64, device="cuda")
        sol.ipm_get_state(ck, stream=stream)
        fb0, rc0 = fallback_count(sol), raise_count(sol)
        _, launches0 = sol.timers()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            for k in range(steps):
                flush.fill_(float(k))  # larger than L2: evicts the previous step's data
                ev[k][0].record(stream)
                conv, _ = sol.ipm_step(stream=stream)
                ev[k][1].record(stream)
                if conv:
                    sol.ipm_init_state(stream=stream)
                    flush.fill_(float(k))
                    ev[k][0].record(stream)
                    sol.ipm_step(stream=stream)
                    ev[k][1].record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        _, launches1 = sol.timers()
        fallbacks, raises = fallback_count(sol) - fb0, raise_count(sol) - rc0
        tot_ms = sum(a.elapsed_time(b) for a, b in ev)
        if world > 1:
            t = torch.tensor([tot_ms], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            tot_ms = float(t.item())
        # phase breakdown (events between phases; graphs are off while profiling)
        sol.ipm_set_state(ck, stream=stream)
        sol.ipm_set_profiling(2)
        n_ph = (phase_steps or steps) if want_phases else 0
        for k in range(n_ph):
            flush.fill_(float(k))
            step()
        torch.cuda.synchronize()
        phases, _ = sol.timers()
        sol.ipm_set_profiling(0)
        e2e_val = None
        if want_e2e:
            # end to end through the C ABI with host buffers: state in from pinned
            # host memory, one IPM iteration, state out to host memory, every step
            host = torch.empty(dims.state_len, dtype=torch.float64, pin_memory=True)
            hnp = host.numpy()
            # the same iterates as the device-timed pass: start from its checkpoint
            sol.ipm_set_state(ck, stream=stream)
            sol.ipm_get_state(hnp, stream=stream)
            torch.cuda.synchronize()
            e2e = []
            for k in range(steps):
                flush.fill_(float(k))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sol.ipm_set_state(hnp, stream=stream)
                conv, _ = sol.ipm_step(stream=stream)
                sol.ipm_get_state(hnp, stream=stream)
                torch.cuda.synchronize()
                e2e.append(time.perf_counter() - t0)
                if conv:
                    sol.ipm_init_state(stream=stream)
                    sol.ipm_get_state(hnp, stream=stream)
            e2e_val = world * N * len(e2e) / sum(e2e)
    per = {p: phases[p][0] / n_ph for p in phases} if n_ph else {p: 0.0 for p in phases}
    # the reduced right-hand side runs on a side stream beside the split on
    # the FP64 paths (its phase time overlaps); on the mixed path it follows
    # the contraction
    cond = ("condense_K", "lu", "zsolve", "split", "gemm") + (("reduced_rhs",) if precision == "mixed" else ())
    cond_ms = sum(per[p] for p in cond)
    return dict(sol=sol, dims=dims, N=N, tot_ms=tot_ms, value=world * N * steps / (tot_ms / 1e3),
                fallbacks=fallbacks, raises=raises,
                ms_per_step=tot_ms / steps, phases=phases, phases_ms_per_step=per,
                condense_only=N * world / (cond_ms / 1e3) if cond_ms > 0 else None,
                launches=launches1 - launches0, clocks=clk.summary(), e2e=e2e_val)


def run_ours(args):
    import torch
    from paper_2301_04869_gb300 import ipm

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    net, pd, qd = synth.workload(args.workload, n_scen=args.scenarios)
    big = synth.CONFIGS[args.workload][0] > 2000
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # the 10,000-bus phase breakdown takes the first 4 of the timed iterates
    main = measure_path(ipm, net, pd, qd, args.precision, args.steps, args.warmup, world, local, flush,
                        phase_steps=min(args.steps, 4) if big else None)
    # free the headline context before the others (the 10,000-bus one holds ~210 GB)
    main["sol"].close()
    del main["sol"]
    torch.cuda.empty_cache()
    others = {}
    if not args.no_compare:
        for p in ("fp64", "fp64_tc", "mixed"):
            if p == args.precision:
                continue
            # the 10,000-bus FP64 iteration takes ~20 s: two timed steps after one warm-up
            csteps, cwarm = (2, 1) if big else (max(5, args.steps // 2), args.warmup)
            try:
                r = measure_path(ipm, net, pd, qd, p, csteps, cwarm, world, local, flush, want_e2e=False,
                                 want_phases=not big)
            except ipm.IPMError as e:
                others[p] = {"unavailable": f"{e.kind}: this path's operands do not fit on one GPU at this size"
                             if e.kind == "IPM_ERR_OOM" else str(e)}
                torch.cuda.empty_cache()
                continue
            others[p] = {"value": r["value"], "unit": UNIT, "ms_per_step": r["ms_per_step"], "steps": csteps,
                         "warmup": cwarm, "condense_only": r["condense_only"],
                         "fp64_fallback_iterations": r["fallbacks"], "curvature_raises": r["raises"],
                         "phases_ms_per_step": {k: round(v, 3) for k, v in r["phases_ms_per_step"].items()},
                         "clocks": r["clocks"]}
            r["sol"].close()
            del r
            torch.cuda.empty_cache()
    if rank != 0:
        return
    dims, N = main["dims"], main["N"]
    peaks, pk = load_peaks()
    rl = roofline(main["phases"], dims, peaks, pk, args.precision)
    rl["peak_source"] = ("FP64 unit count x clock (2 FMA/clk/SM x 152 SMs x 2.07 GHz)" if rl["bound"] == "alu"
                         else (f"{pk} MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside a long step)"
                               if rl["bound"] == "tensor" else f"{pk} MEASURED_PEAKS.json hbm_gbs"))
    cb = cpu_baseline(args.workload) if (world == 1 and not args.no_cpu_baseline) else None
    paths = {args.precision: {"value": main["value"], "unit": UNIT, "ms_per_step": main["ms_per_step"],
                              "condense_only": main["condense_only"],
                              "fp64_fallback_iterations": main["fallbacks"],
                              "curvature_raises": main["raises"]}}
    paths.update(others)
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "bf16x3+f64", "fp64_tc": "f64 (bf16 slices)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload + (f" (first {N} scenarios)" if args.scenarios else ""),
                   "n_bus": dims.n_bus, "n_scen": N, "n_x": dims.n_x, "n_u": dims.n_u,
                   "path": args.precision, "l2": "flushed between steps (256 MB write)",
                   "graphs": True, "autotune": True,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "s_per_ipm_iter": main["ms_per_step"] / 1e3,
        "condense_only": {"value": main["condense_only"], "unit": UNIT,
                          "phases": ["condense_K", "lu", "zsolve", "split", "gemm"],
                          "note": "reduced_rhs runs on a side stream beside split (FP64 paths)"},
        "phases_ms_per_step": {k: round(v, 3) for k, v in main["phases_ms_per_step"].items()},
        "paths": paths,
        "roofline": rl,
        "cpu_baseline": cb,
        "e2e": {"value": main["e2e"], "unit": UNIT, "h2d_bytes_per_step": 8 * dims.state_len,
                "d2h_bytes_per_step": 8 * dims.state_len,
                "note": "the same iterates as value (restarted from the timed pass's checkpoint)"},
        "gpu_launches": main["launches"],
        "clocks": main["clocks"],
    }
    print(json.dumps(line))


def run_batch(args):
    """The multi-instance runner on uneven instances (bus counts log-uniform in
    [100, nmax], generators at 10 % of buses, 8..128 scenarios each): create,
    solve from the cold start and destroy every instance under a device-memory
    budget.  Metric: scenario condensations (scenarios x IPM iterations,
    summed over instances) per second of wall time for the whole job, context
    creation included, with the grouped persistent contraction; the same job
    without grouping, with one worker thread, and on the FP64_TC path
    (per-instance tensor-core contraction) is timed for comparison."""
    import torch
    from paper_2301_04869_gb300 import ipm
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    insts = synth.uneven_batch(n_inst=args.instances, seed=4, nmin=100, nmax=args.nmax, smin=8, smax=128)
    nets, pds, qds = [t[0] for t in insts], [t[1] for t in insts], [t[2] for t in insts]
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.7 * free)
    ipm.ipm_run_instances(nets[:4], pds[:4], qds[:4], budget, n_threads=4, max_iter=args.max_iter)  # warm-up
    runs = {}
    for tag, kw in (("grouped", dict(n_threads=8, group_contraction=True, precision=ipm.PREC_FP64)),
                    ("ungrouped", dict(n_threads=8, group_contraction=False, precision=ipm.PREC_FP64)),
                    ("one_thread", dict(n_threads=1, group_contraction=False, precision=ipm.PREC_FP64)),
                    ("fp64_tc", dict(n_threads=8, group_contraction=False, precision=ipm.PREC_FP64_TC))):
        l0 = ipm.kernel_launches()
        torch.cuda.synchronize()
        with Clocks(0) as clk:
            t0 = time.perf_counter()
            it, er, st, stats, _ = ipm.ipm_run_instances(nets, pds, qds, budget, max_iter=args.max_iter, **kw)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        cond = int(sum(int(p.shape[0]) * int(k) for p, k in zip(pds, it)))
        statuses = {ipm.STATUS.get(int(k), str(k)): int(v) for k, v in zip(*np.unique(st, return_counts=True))}
        runs[tag] = dict(value=cond / wall, wall_s=wall, condensations=cond, launches=ipm.kernel_launches() - l0,
                         converged=int((st == 0).sum()), failed=int((st != 0).sum()), statuses=statuses,
                         mean_iters=float(np.mean(it)), stats=stats, clocks=clk.summary())
    g = runs["grouped"]
    line = {
        "metric": METRIC, "value": g["value"], "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * g["wall_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batch_uneven", "instances": args.instances, "n_bus": f"log-uniform 100..{args.nmax}",
                   "generators": "10% of buses", "scenarios": "uniform 8..128",
                   "total_scenarios": int(sum(p.shape[0] for p in pds)), "max_iter": args.max_iter,
                   "mem_budget_bytes": budget, "timing": "wall clock of the whole job (host), device synchronised"},
        "runs": {k: {a: b for a, b in v.items() if a != "clocks"} for k, v in runs.items()},
        "e2e": {"value": g["value"], "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "host arrays in, final states out, inside the timed job"},
        "gpu_launches": g["launches"],
        "clocks": g["clocks"],
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed IPM iterations (default 10; 6 on the 10,000-bus workload)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="opf10000_n256", choices=list(synth.CONFIGS) + ["batch_uneven"])
    ap.add_argument("--instances", type=int, default=64, help="batch_uneven: number of instances")
    ap.add_argument("--max-iter", type=int, default=150, help="batch_uneven: IPM iteration limit")
    ap.add_argument("--nmax", type=int, default=1000,
                    help="batch_uneven: largest bus count (the many-instance configuration: --instances 512 "
                         "--nmax 5000)")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed", "fp64_tc"],
                    help="headline path (default: mixed on the 10,000-bus workload, fp64_tc otherwise)")
    ap.add_argument("--scenarios", type=int, default=None,
                    help="scenarios of the workload's network (default: the workload's own count); a smaller "
                         "count is for profiling captures, and the line's config then names it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precision paths")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.precision is None:
        args.precision = "mixed" if args.workload == "opf10000_n256" else "fp64_tc"
    if args.steps is None:
        args.steps = 6 if args.workload in synth.CONFIGS and synth.CONFIGS[args.workload][0] > 2000 else 10
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch_uneven":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

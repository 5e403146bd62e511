"""Benchmark of the contrail finite-volume step on GB300.

Workloads (synthetic plumes shaped like the paper's turbofan exhaust, Sec. 4.1):
  fp64      -- axisymmetric coaxial plume, 1024 x 256 cells, plain FP64 method (default)
  fp32      -- the same plume on 4096 x 1024 cells, FP32 transport with FP64 islands
  fp32_mlp  -- the 4096 x 1024 plume with the BF16 tensor-core source surrogate
  active_fp32 / active_mlp -- a hydrogen-like mixing plume (2048 x 512) whose source fires
               in about half of the cells, without / with the surrogate
  batch64   -- 64 plume cases of uneven grids (256 x 64 .. 2048 x 512) and conditions in
               one persistent, graph-captured launch per stage, FP32 + surrogate, autotuned
               tile shape

One benchmark step = one explicit SSP-RK2 step (two fused stage launches) over the whole
grid.  `value` is cell-steps per second (whole job) with the state resident in HBM; L2 is
flushed between timed steps (512 MB write).  `e2e` is the same metric through the C ABI's
host-buffer entry point (state host->device, one step, state device->host each step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

With --impl reference the CPU oracle (the plain FP64 C implementation the GPU path is
checked against) is timed on the host cores for the same workload and metric.
Multi-GPU: one process per GPU (torchrun); each rank advances its own plume replica
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-steps/s: plain FP64 vs FP32+MLP-source at stated error; % HBM peak"
UNIT = "Gcell-steps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


BATCH_DESC = ("sweep of 64 axisymmetric plumes, grids 256x64..2048x512 (uneven), T_amb 205-235 K, "
              "S_ice 0.9-1.3, water/fuel 1.25-8.9 kg/kg, duct 0 or 2 D_core, soot 1e10-1e13 m^-3; "
              "FP32 + BF16 tensor-core surrogate, one persistent graph-captured launch per stage")


def _workload(name):
    from synth import cases
    if name == "batch64":
        # the oracle's sample for this workload: the smallest case of the sweep
        bc = cases.batch_cases(n=64)
        k = int(np.argmin([c["nx"] * c["nr"] for c, _ in bc]))
        return bc[k][0], bc[k][1], BATCH_DESC, 2
    if name == "fp64":
        c, uf = cases.plume_case()
        return c, uf, "axisymmetric coaxial plume 1024x256, FP64 plain method", 0
    if name == "fp64_viscous":
        c, uf = cases.plume_case()
        return (dict(c, viscous=1, nu_t=0.5), uf,
                "axisymmetric coaxial plume 1024x256, FP64, viscous and diffusive fluxes (nu_t 0.5 m^2/s)", 0)
    if name in ("fp32", "fp32_mlp"):
        c, uf = cases.plume_case_mixed_precision()
        if name == "fp32":
            return c, uf, "axisymmetric coaxial plume 4096x1024, FP32 transport + FP64 islands", 1
        return c, uf, "axisymmetric coaxial plume 4096x1024, FP32 + BF16 tensor-core source surrogate", 2
    if name == "fp64_bimodal":
        c, uf = cases.plume_case()
        return (dict(c, bimodal=1), uf,
                "axisymmetric coaxial plume 1024x256, FP64, bimodal liquid (two moment sets, 18 fields)", 0)
    if name in ("active_fp64", "active_fp64_tables", "active_fp64_bimodal"):
        c, uf = cases.mixing_layer_case(nx=1024, nr=256)
        tab = name.endswith("tables")
        bi = name.endswith("bimodal")
        return (dict(c, tables=int(tab), bimodal=int(bi)), uf,
                "hydrogen-like mixing plume 1024x256 (pre-mixed layer), FP64"
                + (", water properties from tables (2nd-order Taylor)" if tab else ", closed-form properties")
                + (", bimodal liquid (two moment sets, 18 fields)" if bi else ""), 0)
    # active-heavy hydrogen-like mixing plume: the source fires in about half of the cells
    c, uf = cases.mixing_layer_case(nx=2048, nr=512)
    if name == "active_fp32":
        return c, uf, "hydrogen-like mixing plume 2048x512 (pre-mixed layer), FP32 + FP64 islands", 1
    if name == "active_fp32_bimodal":
        return (dict(c, bimodal=1), uf,
                "hydrogen-like mixing plume 2048x512 (pre-mixed layer), FP32 + FP64 islands, bimodal liquid", 1)
    return c, uf, "hydrogen-like mixing plume 2048x512 (pre-mixed layer), FP32 + BF16 tensor-core surrogate", 2


# Per-cell figures of the fused stage kernel, from one ncu capture each (see profiles/):
# FP64 arithmetic per cell-stage executed on the plume (mean of the two stages, 527.9 and
# 602.2 flops on the 16 x 16 two-CTA tile; the kernels skip the exact zeros of the particle
# moments in air without liquid or ice; the 16 x 14 tile's larger halo adds 0.5 %: 530.5
# and 605.2), and DRAM bytes per cell per launch (mean of the two stages) by tile shape,
# reported only for a shape counted on the current kernel.
FP64_FLOPS_PER_CELL_STAGE = 565.1
FP64_TRAFFIC_PER_CELL_LAUNCH = {7: 452.0, 8: 392.8}    # 16 x 16 and 16 x 14, two CTAs per SM
FP32_TRAFFIC_PER_CELL_LAUNCH = {9: 140.4}    # the column sweep (28 x 64 strips), four CTAs per SM
SWEEP_SHAPE = 9   # tile shape index of the column-sweep FP32 kernel (k_sweep)
# the viscous FP64 kernel (same capture recipe, plume with nu_t = 0.5 m^2/s, 16 x 14 tile:
# 1135.9 and 1377.4 flops)
FP64_VISC_FLOPS_PER_CELL_STAGE = 1256.7
# the bimodal FP64 kernel (18 fields; same recipe, dormant plume: 576.3 and 688.6 flops)
FP64_BI_FLOPS_PER_CELL_STAGE = 632.5


def measure_dgemm_tflops(dev) -> float:
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn_like(a)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize(dev)
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 2.0 * 4096**3 / best / 1e12


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ct_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            sm = [float(r[0]) for r in rows]
            mx = [float(r[1]) for r in rows]
            names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
            reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].strip() == "Active"})
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": reasons,
                    "samples": len(rows)}
        except Exception as e:  # noqa: BLE001
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)}


def max_over_ranks(values, dist, dev=None):
    """Per-rank timings -> their maximum over all ranks (the job's time); identity on one rank."""
    if not dist:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return [float(v) for v in t.tolist()]


def total_over_ranks(count, dist):
    """Units processed by all ranks (each rank its own work: weak scaling)."""
    if not dist:
        return int(count)
    import torch
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([int(count)], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def batch_seed(rank: int) -> int:
    """Seed of the plume sweep a rank steps: independent cases per rank."""
    return 5 + 1000 * int(rank)


def run_cuda(args):
    import torch
    import paper_2504_20742_gb300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    c, uf, desc, prec = _workload(args.workload)
    cells = int(c["nx"]) * int(c["nr"])
    cfl = 0.5
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        s = P.Solver(c, uf, precision=prec, device=dev, stream=stream)
        s.init_state(cfl)
        if prec == P.CT_FP32_MLP:
            from paper_2504_20742_gb300 import surrogate as S
            s.attach_surrogate(S.Surrogate.load(S.default_path()).blob(dev))
        if args.tile_shape >= 0:                 # a given tile shape instead of the autotuner's
            shape, tune_ms = args.tile_shape, []
            P.ct_set_tile_shape(c, prec, shape)
        else:
            shape, tune_ms = s.autotune(reps=3)     # the state is left as it was
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            s.step(1, cfl)
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        with Clocks(local) as clk:
            t0 = time.perf_counter()
            for k in range(args.steps):
                flush.fill_(float(k))              # L2 flush between timed steps (not timed)
                starts[k].record(stream)
                s.step(1, cfl)
                ends[k].record(stream)
            stream.synchronize()
            wall = time.perf_counter() - t0
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        step_ms = float(np.sum(ms)) / args.steps
        d = s.diagnostics()
        # end to end through the host-buffer entry point (pinned memory)
        host_in = s.U.detach().cpu().pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        e2e_steps = max(3, min(args.steps, 10))
        def e2e_step():
            if prec == P.CT_FP32_MLP:      # host buffers around the surrogate step
                s.U.copy_(host_in, non_blocking=True)
                P.ct_load_state(c, prec, s.work, s.U, s.U, cfl, stream)
                s.step(1, cfl)
                host_out.copy_(s.U, non_blocking=True)
                stream.synchronize()
            else:
                P.ct_step_host(c, prec, host_in, host_out, s.U, s.U1, s.work, 1, cfl, stream)
        e2e_step()
        stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    step_ms, e2e_s = max_over_ranks([step_ms, e2e_s], dist, dev)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = world * cells / (step_ms * 1e-3) / 1e9
    peaks, peak_kind = _peaks()
    # mean duration of one fused stage launch: CUDA events on the launching stream around
    # each timed step (two launches of k_stage per step)
    launch_ms_ev = step_ms / 2.0
    elem = 8 if prec == 0 else 4
    nf = 18 if c.get("bimodal") else 14   # fields of the state
    if prec == 0:
        # FP64 path: bound by the FP64 pipe.  Algorithmic flops per cell and stage are the
        # kernel's FP64 arithmetic (2 DFMA + DADD + DMUL), counted once with ncu
        # (profiles/k_stage_fp64_plume1024x256.md); the peak is cuBLAS DGEMM measured here.
        fpk = measure_dgemm_tflops(dev)
        per_cell = (FP64_VISC_FLOPS_PER_CELL_STAGE if c.get("viscous") else
                    FP64_BI_FLOPS_PER_CELL_STAGE if c.get("bimodal") else FP64_FLOPS_PER_CELL_STAGE)
        flops = cells * per_cell
        ach = flops / (launch_ms_ev * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 4), "peak": round(fpk, 4), "unit": "TFLOP/s",
                "frac": round(ach / fpk, 4),
                "traffic": (FP64_TRAFFIC_PER_CELL_LAUNCH[shape] * cells
                            if shape in FP64_TRAFFIC_PER_CELL_LAUNCH and not c.get("viscous") and not c.get("bimodal")
                            else None),
                "kernel": "ct::k_stage<double>",
                "peak_source": "measured: cuBLAS DGEMM 4096^3 on this GPU (FP64 has no entry in MEASURED_PEAKS.json)",
                "note": f"{per_cell} FP64 flops per cell-stage executed (a DFMA counts 2, a DADD or DMUL 1; "
                        "the FP64 pipe was 76-78 % busy on the plume in the ncu capture, profiles/); "
                        "the peak is cuBLAS DGEMM timed in this run; traffic (DRAM bytes of the ncu capture) "
                        "exceeds the 280 algorithmic bytes per cell-launch because the kernel reads and "
                        "writes the stored primitive planes on purpose (DRAM 2-3 % busy); "
                        f"mean launch {launch_ms_ev:.4f} ms"
                        + ("; figure of the dormant plume, a lower bound where the source fires"
                           if args.workload.startswith("active") else "")}
    else:
        alg_bytes = cells * nf * elem * 2.5      # stage 1: read U, write U1; stage 2: read U1, U, write U
        bw = alg_bytes / (launch_ms_ev * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(bw, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(bw / peaks["hbm_gbs"], 4),
                "traffic": (FP32_TRAFFIC_PER_CELL_LAUNCH[shape] * cells
                            if shape in FP32_TRAFFIC_PER_CELL_LAUNCH and not c.get("bimodal") and prec == 1
                            else None),
                "kernel": (("ct::k_sweep<float, queue> + ct::k_sweep_queue" if prec == 2 else "ct::k_sweep<float>")
                           if shape == SWEEP_SHAPE else "ct::k_stage<float>"),
                "peak_source": peak_kind,
                "note": f"algorithmic bytes 2.5*{nf}*4 per cell per launch (mean of the two stages); "
                        f"mean launch {launch_ms_ev:.4f} ms"
                        + ("; a launch is the stage kernel and its surrogate queue kernel"
                           if prec == 2 and shape == SWEEP_SHAPE else "")}
    bytes_state = cells * nf * elem
    line = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == 0 else ("f32" if prec == 1 else "f32+bf16"),
        "data": "synthetic", "impl": "cuda",
        "config": {"workload": desc, "cells": cells, "nx": c["nx"], "nr": c["nr"], "cfl": cfl,
                   "tile": ("%dx%d, %d CTAs/SM (autotuned; ms per stage-1 launch per shape: %s)"
                            % (*P.ct_tile_shape(shape), P.ct_tile_shape_ctas(shape, prec), [round(m, 4) for m in tune_ms])
                            if tune_ms else "%dx%d, %d CTAs/SM (given)"
                            % (*P.ct_tile_shape(shape), P.ct_tile_shape_ctas(shape, prec))),
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "e2e": {"value": round(world * cells / e2e_s / 1e9, 5), "unit": UNIT,
                "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state},
        "gpu_launches": 2 * args.steps * (2 if prec == 2 and shape == SWEEP_SHAPE else 1),
        "clocks": clk.summary(),
        "wall_s_timed": round(wall, 3),
        "diag": {"dt": d[0], "active_cells": d[7], "active_frac": round(d[7] / cells, 5), "nonfinite": d[8],
                 "surrogate_fallback_cells": d[26]},
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(c, uf, args.cpu_seconds)
    if args.workload == "fp64" and world == 1 and not args.no_surrogate:
        line["surrogate"] = surrogate_record(dev)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


SURROGATE_DESC = ("hydrogen-like mixing plume 4096x1024 (pre-mixed layer, Y_v 0.2 core, 205 K ambient): "
                  "the source fires in about half of the cells")


def surrogate_record(dev, steps=20, err_steps=10):
    """The metric's second half on a workload where the network runs: the plain FP64, the
    plain FP32 and the FP32 + BF16 tensor-core surrogate paths on the same plume at config
    4's grid, each timed over `steps` steps (CUDA events, autotuned tiles, after 3 warm-up
    steps), with the active and fallback fractions and each FP32 path's per-field error
    against the FP64 path after `err_steps` steps from the same initial state (the
    nucleating mixing layer is chaotic over longer runs)."""
    import torch
    import paper_2504_20742_gb300 as P
    from paper_2504_20742_gb300 import surrogate as S
    from synth import cases
    c, uf = cases.mixing_layer_case(nx=4096, nr=1024)
    cells = c["nx"] * c["nr"]
    blob = S.Surrogate.load(S.default_path()).blob(dev)
    out = {"workload": SURROGATE_DESC, "cells": cells, "steps": steps}
    stream = torch.cuda.Stream(dev)
    ref = None
    errs = {}
    for name, prec in (("fp64", P.CT_FP64), ("fp32", P.CT_FP32), ("fp32_mlp", P.CT_FP32_MLP)):
        with torch.cuda.stream(stream):
            s = P.Solver(c, uf, precision=prec, device=dev, stream=stream)
            s.init_state(0.5)
            if prec == P.CT_FP32_MLP:
                s.attach_surrogate(blob)
            s.autotune(reps=2)
            s.step(err_steps, 0.5)
            U = s.state64()
            if ref is None:
                ref = U
            else:
                # domain totals (cell-level fields of a nucleating mixing layer are chaotic:
                # whether a marginal cell nucleates within the first steps differs between
                # any two implementations), and the bulk fields cell by cell
                def tot(f):
                    return round(float(abs(U[f].sum() / ref[f].sum() - 1.0)), 8) if ref[f].sum() != 0 else None
                def cell(f):
                    return round(float(np.max(np.abs(U[f] - ref[f]) / (np.abs(ref[f]) + 1e-3 * np.abs(ref[f]).max()))), 8)
                errs[name] = {"total_liquid_number": tot(5), "total_ice_number": tot(9),
                              "total_liquid_mass": tot(8), "total_ice_mass": tot(12), "total_vapour": tot(4),
                              "cell_rho": cell(0), "cell_rho_E": cell(3)}
            s.step(3, 0.5)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(steps, 0.5)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            d = s.diagnostics()
            out[name] = {"ms_per_step": round(ms, 4), "value": round(cells / (ms * 1e-3) / 1e9, 5),
                         "active_frac": round(d[7] / cells, 4)}
            if prec == P.CT_FP32_MLP:
                out[name]["fallback_frac_of_active"] = round(d[26] / max(d[7], 1.0), 4)
            del s
            torch.cuda.empty_cache()
    out["err_vs_fp64_after_steps"] = err_steps
    out["err_vs_fp64"] = errs
    # the stated error: the condensing nozzle's configured run (400 cells, 20,000 steps to
    # steady state), FP32 + surrogate against the FP64 path (itself held to the oracle at
    # 1e-9), liquid number in total and cell by cell
    cn = cases.nozzle_case(nx=400)
    nz = {}
    for name, prec in (("fp64", P.CT_FP64), ("fp32_mlp", P.CT_FP32_MLP)):
        with torch.cuda.stream(stream):
            s = P.Solver(cn, None, precision=prec, device=dev, stream=stream)
            s.init_state(0.5)
            if prec == P.CT_FP32_MLP:
                s.attach_surrogate(blob)
            s.step(20000, 0.5)
            nz[name] = s.state64()[5].ravel()
    ref5, got5 = nz["fp64"], nz["fp32_mlp"]
    m = ref5 > 1e-6 * ref5.max()
    out["nozzle_steady_state"] = {
        "steps": 20000, "liquid_number_total": round(float(abs(got5.sum() / ref5.sum() - 1.0)), 6),
        "liquid_number_cell_l1": round(float(np.abs(got5[m] - ref5[m]).sum() / np.abs(ref5[m]).sum()), 6),
        "target": 0.02}
    out["speedup_fp32_mlp_over_fp64"] = round(out["fp64"]["ms_per_step"] / out["fp32_mlp"]["ms_per_step"], 3)
    out["speedup_fp32_mlp_over_fp32"] = round(out["fp32"]["ms_per_step"] / out["fp32_mlp"]["ms_per_step"], 3)
    out["error_metric"] = ("total_*: |sum x / sum x_fp64 - 1| over the domain; cell_*: max over cells of "
                           "|x - x_fp64| / (|x_fp64| + 1e-3 max|x_fp64|)")
    return out


def run_batch(args):
    """The 64-case sweep stepped by the batched persistent kernel (one replica per GPU)."""
    import torch
    import paper_2504_20742_gb300 as P
    from paper_2504_20742_gb300 import surrogate as S
    from synth import cases

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    bc = cases.batch_cases(seed=batch_seed(rank), n=64)   # every rank its own sweep
    cells_rank = int(sum(c["nx"] * c["nr"] for c, _ in bc))
    cfl = 0.5
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        blob = S.Surrogate.load(S.default_path()).blob(dev)
        b = P.Batch([c for c, _ in bc], [u for _, u in bc], precision=P.CT_FP32_MLP, device=dev, stream=stream,
                    blob=blob)
        b.init_state(cfl)
        if args.tile_shape >= 0:                 # a given tile shape instead of the autotuner's pick
            shape, tune_ms = args.tile_shape, []
            b.set_tile_shape(shape)
        else:
            shape, tune_ms = b.autotune(reps=2)
        for _ in range(args.warmup):
            b.step(1, cfl)
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        with Clocks(local) as clk:
            t0 = time.perf_counter()
            for k in range(args.steps):
                starts[k].record(stream)
                b.step(1, cfl)                # replay of the captured one-step graph
                ends[k].record(stream)
            stream.synchronize()
            wall = time.perf_counter() - t0
        torch.cuda.synchronize()
        step_ms = float(np.sum([a.elapsed_time(e) for a, e in zip(starts, ends)])) / args.steps
        d = b.diagnostics()
        # end to end: pinned host state in, one step, state out, every step
        host_in = b.U.detach().cpu().pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()

        def e2e_step():
            b.U.copy_(host_in, non_blocking=True)
            b.load_state(b.U, cfl)
            b.step(1, cfl)
            host_out.copy_(b.U, non_blocking=True)
            stream.synchronize()
        e2e_step()
        e2e_steps = max(3, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    step_ms, e2e_s = max_over_ranks([step_ms, e2e_s], dist, dev)
    cells = total_over_ranks(cells_rank, dist)      # collective: every rank takes part
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = cells / (step_ms * 1e-3) / 1e9
    peaks, peak_kind = _peaks()
    launch_ms = step_ms / 2.0
    bw = cells_rank * 14 * 4 * 2.5 / (launch_ms * 1e-3) / 1e9
    tx, ty = P.ct_tile_shape(shape)
    ctas = P.ct_tile_shape_ctas(shape, P.CT_FP32_MLP)
    bytes_state = cells_rank * 14 * 4
    line = {
        "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic", "impl": "cuda",
        "config": {"workload": BATCH_DESC, "cases": len(bc) * world, "cells": cells, "cfl": cfl,
                   "tile": (f"{tx}x{ty}, {ctas} CTAs/SM (autotuned; ms per stage-1 launch per shape: "
                            f"{[round(m, 4) for m in tune_ms]})" if tune_ms else f"{tx}x{ty}, {ctas} CTAs/SM (given)"),
                   "l2": "inputs larger than L2 (1.25 GB per FP32 state copy)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(bw, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(bw / peaks["hbm_gbs"], 4), "traffic": None,
                     "kernel": ("ct::k_batch_sweep<float, queue> + ct::k_batch_queue" if shape == SWEEP_SHAPE
                                else "ct::k_batch_stage<float, surrogate>"), "peak_source": peak_kind,
                     "note": f"algorithmic bytes 2.5*14*4 per cell per launch (mean of the two stages); "
                             f"mean launch {launch_ms:.4f} ms"},
        "e2e": {"value": round(cells / e2e_s / 1e9, 5), "unit": UNIT,
                "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state},
        "gpu_launches": 2 * args.steps * (2 if shape == SWEEP_SHAPE else 1),
        "clocks": clk.summary(),
        "wall_s_timed": round(wall, 3),
        "diag": {"dt_min": float(d[:, 0].min()), "dt_max": float(d[:, 0].max()),
                 "active_cells": float(d[:, 7].sum()), "active_frac": round(float(d[:, 7].sum()) / cells_rank, 5),
                 "nonfinite": float(d[:, 8].sum()), "surrogate_fallback_cells": float(d[:, 26].sum())},
    }
    if not args.no_cpu_baseline and world == 1:
        c, uf, _, _ = _workload("batch64")
        cb = cpu_baseline(c, uf, args.cpu_seconds)
        cb["sample"] = f"the sweep's smallest case ({c['nx']}x{c['nr']}), plain FP64: " + cb["sample"]
        line["cpu_baseline"] = cb
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def cpu_baseline(c, uf, target_s=12.0):
    """The oracle as it stands (plain C, FP64, OpenMP over rows) on the host cores, on a
    bounded sample of the workload: whole-grid steps until about target_s of CPU time."""
    import oracle as O
    o = O.Oracle(c, uf)
    U = o.init_state()
    t0 = time.perf_counter()
    o.step(U, 1, 0.5)
    t1 = time.perf_counter() - t0
    n = max(1, min(200, int(target_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.step(U, n, 0.5)
    dt = time.perf_counter() - t0
    cells = int(c["nx"]) * (int(c["nr"]) if c["geom"] == 1 else 1)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(cells * n / dt / 1e9, 7), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} whole-grid steps of the same workload after 1 warm-up step ({dt:.1f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c, uf, desc, prec = _workload(args.workload)
    import oracle as O
    o = O.Oracle(c, uf)
    U = o.init_state()
    cells = int(c["nx"]) * int(c["nr"])
    for _ in range(args.warmup):
        o.step(U, 1, 0.5)
    # bounded sample: at most ~60 s of oracle time in total
    t0 = time.perf_counter()
    o.step(U, 1, 0.5)
    per = time.perf_counter() - t0
    steps = max(1, min(args.steps, int(60.0 / max(per, 1e-6))))
    t0 = time.perf_counter()
    o.step(U, steps, 0.5)
    dt = time.perf_counter() - t0
    value = cells * steps / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": round(value, 7), "unit": UNIT, "n_gpus": 0, "steps": steps,
            "warmup": args.warmup, "ms_per_step": round(dt / steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "cells": cells},
            "cpu_baseline": {"value": round(value, 7), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} whole-grid steps (of {args.steps} requested)"
                                       + (f" of the sweep's smallest case ({c['nx']}x{c['nr']})"
                                          if args.workload == "batch64" else "")},
            "e2e": {"value": round(value, 7), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=("cuda", "reference"))
    ap.add_argument("--workload", default="fp64",
                    choices=("fp64", "fp64_viscous", "fp64_bimodal", "fp32", "fp32_mlp", "active_fp32",
                             "active_fp32_bimodal", "active_mlp", "active_fp64", "active_fp64_tables",
                             "active_fp64_bimodal", "batch64"))
    ap.add_argument("--tile-shape", type=int, default=-1,
                    help="stage-kernel tile shape (ct_tile_shape index) instead of the autotuner's pick")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="leave out the FP64 / FP32 / FP32+surrogate record of the default workload")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()

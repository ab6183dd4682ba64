"""Benchmark: PCG of the periodic FE homogenisation cell problem on one GB300.

Workload (one "step"): 128^3 trilinear-hexahedron small-strain elasticity, 60 seeded periodic
spheres (E = 100, nu = 0.2) in a matrix (E = 1, nu = 0.3), reference material = volume mean,
the 6 unit Mandel strains solved as one batch with plain FP64 PCG to a relative K_ref^-1-norm
residual of 1e-6.  A step runs the whole hot path through the C ABI: Algorithm 2 (preconditioner
build), right-hand sides, PCG iterations (stiffness apply, FFT preconditioner, fused updates and
reductions) and the volume averages giving C_eff.

value = PCG DOF*iterations/s = sum over loads of (3 * 128^3 * iterations) / step time (device
time, inputs resident in HBM).  e2e = the same through fehom_setup with host phase ids, with the
fluctuation fields read back to pinned host memory, host<->device copies inside the timed region.
The mixed-precision form (FP32 stiffness/FFT in FP64 iterative refinement) is timed on the same
workload and reported under "mixed".  The inputs (fields of 50 MB per load and component set)
are larger than L2, and every step rewrites them, so no L2 flush is added.

--impl reference runs the FP64 CPU oracle (assembled CSR + unpreconditioned CG in C/OpenMP) to
tolerance on a bounded sample of the same workload statistics on the host cores; --oracle-timing
times it on the benchmark table's workloads beside the GPU solves.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG DOF*iter/s + time-to-1e-6 (128^3 elastic), % HBM peak; mixed vs FP64"
UNIT = "DOF*iter/s"


# ------------------------------------------------------------------------------------------------
# replicas: one process per GPU (torch.distributed.run); every rank solves the whole workload (the
# path does not shard: independent cells are independent replicas), timing is the max over ranks
# ------------------------------------------------------------------------------------------------
def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return world, rank, local


def dist_init(backend):
    import torch.distributed as td
    world, rank, _ = dist_info()
    if world > 1 and not td.is_initialized():
        td.init_process_group(backend=backend, rank=rank, world_size=world)


def barrier():
    import torch.distributed as td
    if td.is_available() and td.is_initialized():
        td.barrier()


def reduce_over_ranks(x, op="max"):
    """Max (or sum) of a float over all ranks; the value itself without a process group."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()):
        return float(x)
    dev = "cuda" if td.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    td.all_reduce(t, op=td.ReduceOp.MAX if op == "max" else td.ReduceOp.SUM)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"




class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons}


def workload():
    from paper_2203_02962_gb300 import inputs
    return inputs.workload_spheres_elastic(128, seed=0)


# Algorithmic work per voxel and load of each PCG kernel class on the 128^3 elastic workload
# (c = 3 DOF per voxel).  Bytes: fields read + written once (s bytes per scalar), half spectra
# nxh / nx = 65/128 complex per real voxel per component, phase ids 1 byte.  FP64 operations: counted
# from the kernels' arithmetic (one FP64 instruction = add, mul or fma).  Stiffness, per voxel (one
# element, one node plane) for isotropic phases: in-plane butterflies of the node plane 24, z part
# 21, closed-form duals 35, transposed z part 18, face totals 12, transposed in-plane part 24, node
# gather and scale 12, fused <p, Ap> 3 = 149.
def kernel_model(s, c=3, n=128):
    hs = (n // 2 + 1) / n
    spec = c * hs * 2 * s              # one half-spectrum pass over the c components
    sym = c * (c + 1) // 2 * s * hs    # packed symmetric c x c K_hat^+ per half-spectrum k
    return {
        "stiffness": {"bytes": 2 * c * s + 1, "fp64_ops": 149},
        "fft_x_fwd": {"bytes": 3 * c * s + spec, "fp64_ops": 3 * 4.0 * 7 * 3.5 / 2 * 2},
        "fft_y_fwd": {"bytes": 2 * spec, "fp64_ops": 3 * hs * 7 * 3.5},
        "fft_last": {"bytes": 2 * spec + sym, "fp64_ops": 3 * hs * 2 * 7 * 3.5 + hs * 18},
        "fft_y_inv": {"bytes": 2 * spec, "fp64_ops": 3 * hs * 7 * 3.5},
        "fft_x_inv": {"bytes": spec + 4 * c * s, "fp64_ops": 3 * 4.0 * 7 * 3.5 / 2 * 2},
    }


FP64_INSTR_PEAK = 152 * 2 * 2.07e9     # FP64 instructions/s: 152 SMs x 2 FP64 lanes-per-clock x max clock
# DRAM bytes (read + write) of one 6-load FP64 stiffness launch on the 128^3 workload, from ncu
FP64_STIFFNESS_DRAM_BYTES = 324.537088e6 + 264.050432e6


def run_ours(args):
    import torch
    from paper_2203_02962_gb300 import fehom

    world, rank, local = dist_info()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist_init("nccl")
    w = workload()
    n = w["n"]
    N = n[0] * n[1] * n[2]
    c = 3
    loads = w["loads"]
    ids_dev = torch.tensor(w["ids"].ravel(), device=dev)
    stream = torch.cuda.Stream(device=dev)   # the library launches on this stream; events are recorded on it

    def step(s):
        s.precond_build()
        return s.solve(loads, tol=w["tol"], fields=None)

    # The timed steps run without per-launch events (an event pair around every kernel, read back after
    # each graph replay, adds about 2 ms to a mixed step); the per-kernel durations behind the roofline
    # come from a second run of the same steps on the same stream with those events recorded.
    results = {}
    for prec in ("fp64", "mixed"):
        s = fehom.Solver("hex8_3d", "elastic", n, ids_dev, w["moduli"], precision=prec, stream=stream)
        for _ in range(args.warmup):
            step(s)
        l_before = s.launch_count()
        torch.cuda.synchronize()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ev0.record(stream)
            outs = [step(s) for _ in range(args.steps)]
            ev1.record(stream)
            torch.cuda.synchronize()
        barrier()
        ms = reduce_over_ranks(ev0.elapsed_time(ev1) / args.steps, "max")
        load_iters = sum(sum(i["iterations"] for i in o["info"]) for o in outs)
        results[prec] = dict(ms=ms, iters=load_iters / args.steps, out=outs[-1], clocks=clk.summary(),
                             load_iters=load_iters, launches=s.launch_count() - l_before,
                             plan=s.fft_plan(prec), stencil=s.stencil_plan(prec), C_energy=s.effective_energy())
        s.close()
        # the profiled run: the same steps with CUDA events around every launch of the PCG iterations
        s = fehom.Solver("hex8_3d", "elastic", n, ids_dev, w["moduli"], precision=prec, stream=stream,
                         profile=True)
        step(s)
        t_before = s.kernel_times(prec)
        pev0, pev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pev0.record(stream)
        pouts = [step(s) for _ in range(args.steps)]
        pev1.record(stream)
        torch.cuda.synchronize()
        t_after = s.kernel_times(prec)
        results[prec]["kt"] = {k: (t_after[k][0] - t_before[k][0], t_after[k][1] - t_before[k][1]) for k in t_after}
        results[prec]["kt_load_iters"] = sum(sum(i["iterations"] for i in o["info"]) for o in pouts)
        results[prec]["profiled_ms"] = pev0.elapsed_time(pev1) / args.steps
        s.close()

    # e2e: host phase ids -> setup -> build -> solve -> fields back to pinned host memory
    ids_host = np.ascontiguousarray(w["ids"].ravel())
    fields_host = torch.empty((len(loads), c, N), dtype=torch.float64).pin_memory()
    import ctypes
    lib = fehom.load_library()

    def e2e_step():
        s = fehom.Solver("hex8_3d", "elastic", n, ids_host, w["moduli"], stream=stream)
        s.precond_build()
        flux = np.zeros((len(loads), 6))
        ceff = np.zeros((6, 6))
        info = (fehom.SolveInfo * len(loads))()
        st = lib.fehom_solve(s.ctx, len(loads), fehom._dptr(np.ascontiguousarray(loads)), w["tol"], None,
                             ctypes.c_void_p(fields_host.data_ptr()), 0, fehom._dptr(flux), fehom._dptr(ceff), info)
        assert st == 0, st
        s.close()
        return sum(info[l].iterations for l in range(len(loads)))

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e_iters = [e2e_step() for _ in range(max(1, args.steps))]
    torch.cuda.synchronize()
    barrier()
    e2e_ms = reduce_over_ranks((time.perf_counter() - t0) * 1e3 / max(1, args.steps), "max")

    # untimed tight FP64 solve: reference C_eff for the accuracy of both timed forms
    sref = fehom.Solver("hex8_3d", "elastic", n, ids_dev, w["moduli"], stream=stream)
    sref.precond_build()
    C_ref = sref.solve(loads, tol=1e-10, fields=None)["C_eff"]
    C_ref_energy = sref.effective_energy()
    sref.close()
    r64, rmx = results["fp64"], results["mixed"]
    err = lambda C: float(np.abs(C - C_ref).max() / np.abs(C_ref).max())
    # whole-job throughput: the voxel-load iterations of every rank over the slowest rank's time
    it64 = reduce_over_ranks(r64["iters"], "sum")
    itmx = reduce_over_ranks(rmx["iters"], "sum")
    ite2e = reduce_over_ranks(e_iters[-1], "sum")
    value = c * N * it64 / (r64["ms"] * 1e-3)
    hbm, hbm_src = peaks()
    # dominant kernel of the FP64 step, from the CUDA events recorded around every launch
    dom = max(r64["kt"], key=lambda k: r64["kt"][k][0])
    dom_ms, dom_launches = r64["kt"][dom]
    model = kernel_model(8)[dom]
    units = N * r64["kt_load_iters"]                    # voxel-loads processed by the profiled launches
    avg_ms = dom_ms / max(dom_launches, 1)
    units_per_launch = units / max(dom_launches, 1)
    achieved_ops = model["fp64_ops"] * units_per_launch / (avg_ms * 1e-3)
    achieved_gbs = model["bytes"] * units_per_launch / (avg_ms * 1e-3) / 1e9
    share = {k: r64["kt"][k][0] / max(sum(v[0] for v in r64["kt"].values()), 1e-30) for k in r64["kt"]}
    # mixed path: achieved HBM bandwidth of each FP32 kernel class over the timed launches (algorithmic
    # bytes per voxel-load x voxel-loads / the class's CUDA-event time); the fused x-y passes report
    # under fft_x_fwd / fft_x_inv (fft_y_* then have no launches)
    mx_model, mx_units = kernel_model(4), N * rmx["kt_load_iters"]
    roof_mx = {}
    for k, (ms_k, n_k) in rmx["kt"].items():
        if n_k > 0 and ms_k > 0:
            gbs = mx_model[k]["bytes"] * mx_units / (ms_k * 1e-3) / 1e9
            roof_mx[k] = {"achieved_gbs": gbs, "frac": gbs / hbm, "avg_launch_us": 1e3 * ms_k / n_k,
                          "launches": int(n_k)}
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r64["ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "128^3 hex8 elasticity, 60 periodic spheres E100/nu0.2 in E1/nu0.3, 6 unit Mandel "
                               "strains batched, C_ref = volume mean, FP64 PCG to 1e-6 (Algorithm 2 + solve + C_eff)",
                   "dof": c * N, "loads": len(loads), "tol": w["tol"], "parallelism": "1 GPU",
                   "l2": "inputs > L2 (50 MB per field, ~2 GB working set); no flush"},
        "time_to_tol_s": r64["ms"] * 1e-3,
        "pcg_iterations_per_load": [i["iterations"] for i in r64["out"]["info"]],
        "C_eff_diag": [float(v) for v in np.diag(r64["out"]["C_eff"])],
        "C_eff_rel_err_vs_fp64_tol1e-10": err(r64["out"]["C_eff"]),
        "C_eff_energy_rel_err_vs_fp64_tol1e-10": float(np.abs(r64["C_energy"] - C_ref_energy).max()
                                                       / np.abs(C_ref_energy).max()),
        "e2e": {"value": c * N * ite2e / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(N + w["moduli"].nbytes + loads.nbytes),
                "d2h_bytes_per_step": int(len(loads) * c * N * 8 + 6 * 6 * 8 + len(loads) * 6 * 8),
                "ms_per_step": e2e_ms},
        "mixed": {"value": c * N * itmx / (rmx["ms"] * 1e-3), "ms_per_step": rmx["ms"],
                  "time_to_tol_s": rmx["ms"] * 1e-3, "inner_iterations_per_load": [i["iterations"] for i in rmx["out"]["info"]],
                  "refinements_per_load": [i["refinements"] for i in rmx["out"]["info"]],
                  "speedup_vs_fp64": r64["ms"] / rmx["ms"],
                  "C_eff_rel_diff_vs_fp64": float(np.abs(rmx["out"]["C_eff"] - r64["out"]["C_eff"]).max()
                                                  / np.abs(r64["out"]["C_eff"]).max()),
                  "C_eff_rel_err_vs_fp64_tol1e-10": err(rmx["out"]["C_eff"]),
                  "C_eff_energy_rel_diff_vs_fp64": float(np.abs(rmx["C_energy"] - r64["C_energy"]).max()
                                                         / np.abs(r64["C_energy"]).max()),
                  "C_eff_energy_rel_err_vs_fp64_tol1e-10": float(np.abs(rmx["C_energy"] - C_ref_energy).max()
                                                                 / np.abs(C_ref_energy).max()),
                  "kernel_ms": {k: v[0] for k, v in rmx["kt"].items()},
                  "gpu_launches": rmx["launches"], "fft_plan": rmx["plan"],
                  "stencil_plan": {"rows": rmx["stencil"][0], "staging": ("tma" if rmx["stencil"][1] == 3 else "cp.async"),
                                   "ms_rows_8_16_cpasync_8_16_tma": rmx["stencil"][2]},
                  "roofline_hbm": {"bound": "hbm", "peak_gbs": hbm, "peak_source": hbm_src,
                                   "unit": "GB/s", "kernels": roof_mx, "profiled_ms_per_step": rmx["profiled_ms"]},
                  "clocks": rmx["clocks"]},
        "fft_plan_fp64": r64["plan"],
        "stencil_plan_fp64": {"rows": r64["stencil"][0], "ms_rows_8_16": r64["stencil"][2][:2]},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved_ops / 1e12, "peak": FP64_INSTR_PEAK / 1e12,
                     "unit": "T FP64-instr/s", "frac": achieved_ops / FP64_INSTR_PEAK,
                     "traffic": FP64_STIFFNESS_DRAM_BYTES if dom == "stiffness" else None,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 6-load launch of the "
                                       "current kernel, profiles/hex8_apply_fp64_128cube_elastic.md",
                     "algorithmic_bytes_per_launch": model["bytes"] * units_per_launch,
                     "peak_source": "152 SMs x 2 FP64 lanes/clk x 2.07 GHz (unit count x max clock)",
                     "avg_launch_ms": avg_ms, "launches": dom_launches,
                     "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": hbm, "hbm_frac": achieved_gbs / hbm,
                     "hbm_peak_source": hbm_src, "fp64_kernel_share": share,
                     "kernel_timing": "CUDA events around every launch on the library's stream, in a second run of "
                                      "the timed steps (the headline steps run without them)",
                     "profiled_ms_per_step": r64["profiled_ms"]},
        "clocks": r64["clocks"],
        "gpu_launches": r64["launches"],
    }
    if world > 1:  # replicas: the main timings only; rank 0 reports
        out["config"]["parallelism"] = f"{world} independent replicas (one process per GPU)"
        if rank == 0:
            print(json.dumps(out))
        return
    out["cufft_reference"] = cufft_comparison(N, c, len(loads), rmx["kt"], r64["kt"], rmx["kt_load_iters"],
                                              r64["kt_load_iters"], args.steps)
    out["batched"] = run_batched(args)
    out["warm_start_unet"] = run_unet(args)
    # the composite form against plain FP64 on the same GPU: mixed precision with every load of a cell
    # batched (the 128^3 cell), and mixed + batched over the 48 cells of uneven size; the learned warm
    # start is left out (on these workloads it costs PCG iterations); C_eff in both forms beside it
    bt = out["batched"]
    out["composite"] = {
        "warm_start": "out",
        "cell_128": {"fp64_ms": r64["ms"], "composite_ms": rmx["ms"], "speedup_vs_fp64": r64["ms"] / rmx["ms"],
                     "C_eff_rel_diff_vs_fp64": out["mixed"]["C_eff_rel_diff_vs_fp64"],
                     "C_eff_energy_rel_diff_vs_fp64": out["mixed"]["C_eff_energy_rel_diff_vs_fp64"]},
        "cells_48": {"fp64_sequential_ms": bt["fp64_sequential_wall_ms"], "composite_ms": bt["wall_ms_per_step"],
                     "speedup_vs_fp64": bt["composite_speedup_vs_fp64"],
                     "C_eff_rel_diff_vs_fp64": bt["C_eff_rel_diff_vs_fp64_max_over_cells"],
                     "C_eff_energy_rel_diff_vs_fp64": bt["C_eff_energy_rel_diff_vs_fp64_max_over_cells"]}}
    out["cpu_baseline"] = cpu_baseline(short=True)
    print(json.dumps(out))


def cufft_comparison(N, c, n_loads, kt32, kt64, iters32, iters64, steps):
    """cuFFT (through torch.fft) on the same half-spectrum transforms as one preconditioner apply:
    forward r2c + inverse c2r of n_loads x c fields of 128^3, timed with CUDA events; beside it the
    device time of our five FFT passes per apply (which also do the block solve, the Parseval dot
    and the CG updates).  A comparison only: cuFFT is not used by the solver."""
    import torch
    out = {}
    for name, dt, kt, its in (("fp32", torch.float32, kt32, iters32), ("fp64", torch.float64, kt64, iters64)):
        x = torch.randn((n_loads, c, 128, 128, 128), dtype=dt, device="cuda")
        for _ in range(3):
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(2, 3, 4)), s=(128, 128, 128), dim=(2, 3, 4))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(2, 3, 4)), s=(128, 128, 128), dim=(2, 3, 4))
        e1.record()
        torch.cuda.synchronize()
        cu_ms = e0.elapsed_time(e1) / 5
        ours = sum(kt[k][0] for k in ("fft_x_fwd", "fft_y_fwd", "fft_last", "fft_y_inv", "fft_x_inv"))
        iters_per_step = its / steps
        ours_ms = ours / steps / max(1.0, iters_per_step / n_loads)
        out[name] = {"cufft_ms_per_apply": cu_ms, "ours_ms_per_apply": ours_ms, "ratio_ours_over_cufft": ours_ms / cu_ms}
        del x, y
    return out


def run_grf512(args):
    """The 512^3 scalar conductivity cell (thresholded GRF, contrast 1000, three unit gradients, 134M
    DOF, tol 1e-6): plain FP64 PCG and the mixed form (FP32 inner PCG, FP64 refinement), each timed to
    tolerance (Algorithm 2 + solve + C_eff) after one untimed step; one JSON line."""
    import torch
    from paper_2203_02962_gb300 import fehom
    from paper_2203_02962_gb300 import inputs as I

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = I.workload_grf_scalar(512)
    n, loads, c = w["n"], w["loads"], 1
    N = n[0] * n[1] * n[2]
    ids_dev = torch.tensor(w["ids"].ravel(), device=dev)
    stream = torch.cuda.Stream(device=dev)
    steps = max(1, min(args.steps, 2))
    res = {}
    for prec in ("fp64", "mixed"):
        res[prec] = {}
        for profiled in (False, True):  # the timed steps without per-launch events, then with them
            s = fehom.Solver("hex8_3d", "scalar", n, ids_dev, w["moduli"], precision=prec, stream=stream,
                             profile=profiled)

            def step():
                s.precond_build()
                return s.solve(loads, tol=w["tol"], fields=None)

            step()
            t_before = s.kernel_times(prec) if profiled else None
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ClockSampler(0) as clk:
                ev0.record(stream)
                outs = [step() for _ in range(steps)]
                ev1.record(stream)
                torch.cuda.synchronize()
            load_iters = sum(sum(i["iterations"] for i in o["info"]) for o in outs)
            if profiled:
                t_after = s.kernel_times(prec)
                res[prec]["kt"] = {k: (t_after[k][0] - t_before[k][0], t_after[k][1] - t_before[k][1]) for k in t_after}
                res[prec]["kt_load_iters"] = load_iters
            else:
                res[prec].update(ms=ev0.elapsed_time(ev1) / steps, out=outs[-1], clocks=clk.summary(),
                                 load_iters=load_iters, C_energy=s.effective_energy())
            s.close()
    hbm, hbm_src = peaks()
    r64, rmx = res["fp64"], res["mixed"]
    model, units = kernel_model(4, c, n[0]), N * rmx["kt_load_iters"]
    roof = {}
    for k, (ms_k, n_k) in rmx["kt"].items():
        if n_k > 0 and ms_k > 0:
            gbs = model[k]["bytes"] * units / (ms_k * 1e-3) / 1e9
            roof[k] = {"achieved_gbs": gbs, "frac": gbs / hbm, "avg_launch_us": 1e3 * ms_k / n_k, "launches": int(n_k)}
    rel = lambda A, B: float(np.abs(A - B).max() / np.abs(B).max())
    print(json.dumps({
        "workload": "512^3 hex8 conductivity, thresholded periodic GRF (correlation length 16 voxels, 50 % volume), "
                    "k = 1 / 1000, 3 unit gradients, tol 1e-6, C_ref = volume mean",
        "dof": c * N, "steps": steps, "warmup": 1,
        "fp64": {"time_to_tol_s": r64["ms"] * 1e-3, "iterations_per_load": [i["iterations"] for i in r64["out"]["info"]],
                 "dof_iter_per_s": c * N * r64["load_iters"] / steps / (r64["ms"] * 1e-3),
                 "kernel_ms_per_step": {k: v[0] / steps for k, v in r64["kt"].items()}, "clocks": r64["clocks"]},
        "mixed": {"time_to_tol_s": rmx["ms"] * 1e-3,
                  "inner_iterations_per_load": [i["iterations"] for i in rmx["out"]["info"]],
                  "refinements_per_load": [i["refinements"] for i in rmx["out"]["info"]],
                  "dof_iter_per_s": c * N * rmx["load_iters"] / steps / (rmx["ms"] * 1e-3),
                  "roofline_hbm": {"peak_gbs": hbm, "peak_source": hbm_src, "kernels": roof}, "clocks": rmx["clocks"]},
        "speedup_mixed_vs_fp64": r64["ms"] / rmx["ms"],
        "C_eff_rel_diff_mixed_vs_fp64": rel(rmx["out"]["C_eff"], r64["out"]["C_eff"]),
        "C_eff_energy_rel_diff_mixed_vs_fp64": rel(rmx["C_energy"], r64["C_energy"]),
    }))


def run_batched(args):
    """48 elastic cells of uneven size (16 each of 32^3, 64^3, 96^3; spheres, contrast 10^U[1,3]),
    6 unit strains each = 288 solves, mixed precision to 1e-6: one fehom_solve_batch (the PCG
    iterations of all cells replayed from one CUDA graph) against the same cells solved one by one."""
    import torch
    from paper_2203_02962_gb300 import fehom, inputs
    cells = inputs.workload_batched_spheres(48)
    loads = np.eye(6)
    solvers = [fehom.Solver("hex8_3d", "elastic", c["n"], c["ids"], c["moduli"], precision="mixed") for c in cells]
    for sv in solvers:
        sv.precond_build()
    batch = fehom.Batch(solvers)
    for _ in range(max(1, args.warmup)):
        batch.solve(loads, tol=1e-6)
    torch.cuda.synchronize()
    l0 = sum(sv.launch_count() for sv in solvers)
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        outs = [batch.solve(loads, tol=1e-6) for _ in range(args.steps)]
        torch.cuda.synchronize()
        wall_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    launches = (sum(sv.launch_count() for sv in solvers) - l0) // args.steps
    dev_ms = statistics.median(o["info"][0][0]["solve_ms"] for o in outs)
    dof_iter = sum(3 * c["n"][0] ** 3 * sum(i["iterations"] for i in outs[-1]["info"][k]) for k, c in enumerate(cells))
    # the same cells one after another
    for sv in solvers:
        sv.solve(loads, tol=1e-6, fields=None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per_size = {}
    for _ in range(args.steps):
        for c, sv in zip(cells, solvers):
            o = sv.solve(loads, tol=1e-6, fields=None)
            per_size.setdefault(c["n"][0], []).append(o["info"][0]["solve_ms"])
    torch.cuda.synchronize()
    seq_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    # where the sequential time goes: device milliseconds per step by cell size (16 cells each)
    seq_by_size = {str(n): float(sum(v) / args.steps) for n, v in sorted(per_size.items())}
    conv = all(i["converged"] for cell in outs[-1]["info"] for i in cell)
    # C_eff of the batched mixed solves: the stress average (Sec. 2 volume average) and the energy form
    C_mix = [outs[-1]["C_eff"][k] for k in range(len(cells))]
    E_mix = [sv.effective_energy() for sv in solvers]
    batch.close()
    for sv in solvers:
        sv.close()
    # the plain form of the same work: every cell on its own, FP64 PCG to the same tolerance (the tuned
    # launch plans of each grid size are taken by one untimed solve first)
    s64 = [fehom.Solver("hex8_3d", "elastic", c["n"], c["ids"], c["moduli"], precision="fp64") for c in cells]
    for sv in s64:
        sv.precond_build()
    for k in (0, 16, 32):
        s64[k].solve(loads, tol=1e-6, fields=None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs64 = [sv.solve(loads, tol=1e-6, fields=None) for sv in s64]
    torch.cuda.synchronize()
    fp64_ms = (time.perf_counter() - t0) * 1e3
    C64 = [o["C_eff"] for o in outs64]
    E64 = [sv.effective_energy() for sv in s64]
    conv64 = all(i["converged"] for o in outs64 for i in o["info"])
    for sv in s64:
        sv.close()
    rel = lambda A, B: float(np.abs(A - B).max() / np.abs(B).max())  # noqa: E731
    err_s9 = max(rel(a, b) for a, b in zip(C_mix, C64))
    err_en = max(rel(a, b) for a, b in zip(E_mix, E64))
    return {"workload": "48 hex8 elastic cells (16 x 32^3, 16 x 64^3, 16 x 96^3), 288 solves, mixed, tol 1e-6",
            "value": dof_iter / (dev_ms * 1e-3), "unit": UNIT, "device_ms_per_step": dev_ms,
            "wall_ms_per_step": wall_ms, "sequential_wall_ms_per_step": seq_ms,
            "speedup_vs_sequential": seq_ms / wall_ms, "sequential_device_ms_by_cell_size": seq_by_size,
            "all_converged": conv, "gpu_launches": launches,
            "clocks": clk.summary(),
            "fp64_sequential_wall_ms": fp64_ms, "fp64_all_converged": conv64,
            "composite_speedup_vs_fp64": fp64_ms / wall_ms,
            "C_eff_rel_diff_vs_fp64_max_over_cells": err_s9,
            "C_eff_energy_rel_diff_vs_fp64_max_over_cells": err_en}


def unet_flops(n, widths, batch):
    """Algorithmic FLOPs (2 per multiply-add) of one training step of the warm-start U-Net: every
    3x3x3 convolution forward and weight gradient, and the input gradient of all but the first."""
    w = list(widths)
    L = len(w)
    layers = [(1, w[0], 0), (w[0], w[0], 0)]
    for l in range(1, L):
        layers += [(w[l - 1], w[l], l), (w[l], w[l], l)]
    for l in range(L - 2, -1, -1):
        layers += [(w[l] + w[l + 1], w[l], l), (w[l], w[l], l)]
    total = 0.0
    for i, (ci, co, l) in enumerate(layers):
        f = 2.0 * 27 * ci * co * batch * (n >> l) ** 3
        total += f * (2 if i == 0 else 3)
    return total


def run_unet(args):
    """One training step of the warm-start U-Net (64^3, widths 16-128, batch 8) on synthetic phase
    fields and targets: device time per step and achieved BF16 tensor FLOP/s."""
    import torch
    from paper_2203_02962_gb300 import fehom, warmstart
    n, widths, B = 64, (16, 32, 64, 128), 8
    g = torch.Generator(device="cpu").manual_seed(0)
    ids = (torch.rand((B, n ** 3), generator=g) < 0.3).to(torch.uint8).cuda()
    feat = torch.tensor([[0.0, 0.3 + 0.08 * b] for b in range(B)], dtype=torch.float32).cuda()
    tgt = (0.05 * torch.randn((B, 3, n ** 3), generator=g, dtype=torch.float64)).cuda()
    net = fehom.UNet(n, widths, n_phases=2, n_out=3, max_batch=B)
    net.set_params(warmstart.init_params(widths, 3, 0))
    net.set_loss("h1", 0.1)
    for _ in range(max(3, args.warmup) if args.ncu_case is None else 1):
        net.train_step(ids, feat, tgt, 0.05, 1e-4)
    torch.cuda.synchronize()
    steps = max(10, args.steps) if args.ncu_case is None else 1
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(net.stream)
    for _ in range(steps):
        net.train_step(ids, feat, tgt, 0.05, 1e-4)
    e1.record(net.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    x0 = torch.empty((B, 3, n ** 3), dtype=torch.float64, device="cuda")
    e0.record(net.stream)
    for _ in range(steps):
        net.predict(ids, feat, 0.05, out=x0)
    e1.record(net.stream)
    torch.cuda.synchronize()
    pms = e0.elapsed_time(e1) / steps
    net.close()
    flops = unet_flops(n, widths, B)
    peak = peaks_tensor()
    return {"workload": f"U-Net training step, {n}^3, widths {list(widths)}, batch {B}, H1 loss, Adam",
            "ms_per_step": ms, "predict_ms_per_batch": pms, "algorithmic_tflop_per_step": flops / 1e12,
            "achieved_tflops": flops / (ms * 1e-3) / 1e12, "peak_tflops_bf16_sustained": peak,
            "frac": flops / (ms * 1e-3) / 1e12 / peak if peak else None}


def peaks_tensor():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d.get("bf16_tflops_sustained") or d.get("bf16_tflops"))
    except Exception:
        return 1700.0


def _oracle_solve_loads(g, ids, mod, loads, tol, threads, which=None):
    """The oracle's solve of K u = b for each load (assembled CSR + unpreconditioned CG in C/OpenMP,
    stopping at ||r||_2 <= tol ||b||_2): per-load iterations and wall seconds (assembly not included),
    and C_eff when every load was solved."""
    from oracle import cg_native, fem, solvers
    K = fem.assemble_K(g, ids, mod)
    A = cg_native.CSR(K)
    which = range(len(loads)) if which is None else which
    its, secs, flux = [], [], []
    for l in which:
        b = fem.assemble_rhs(g, ids, mod, loads[l])
        t0 = time.perf_counter()
        x, it, _ = cg_native.cg(A, b, tol=tol, threads=threads)
        secs.append(time.perf_counter() - t0)
        its.append(it)
        flux.append(fem.mean_flux(g, ids, mod, loads[l], solvers.project_mean_zero(g, x)) / (g.vp * g.N))
    C = np.array(flux).T @ np.linalg.inv(np.asarray(loads).T) if len(flux) == len(loads) else None
    return its, secs, C


def cpu_baseline(short=False):
    """The oracle (assembled CSR + unpreconditioned CG, FP64, C/OpenMP) timed to tolerance on a bounded
    sample of the workload: a 32^3 cell with the workload's statistics (60 periodic spheres, radii scaled
    to 2-4 voxels, E = 100 / nu = 0.2 in E = 1 / nu = 0.3), the 6 unit Mandel strains to ||r||_2 / ||b||_2
    <= 1e-6, on every host core; one load again on one core."""
    from oracle import cg_native, fem
    from paper_2203_02962_gb300 import inputs

    n = 32
    w = inputs.workload_spheres_elastic(n, seed=0, rmin=n / 16, rmax=n / 8)
    g = fem.Grid((n, n, n), "hex8_3d", "elastic")
    ids = w["ids"].ravel()
    cores = cg_native.max_threads()
    its, secs, _ = _oracle_solve_loads(g, ids, w["moduli"], w["loads"], 1e-6, cores)
    its1, secs1, _ = _oracle_solve_loads(g, ids, w["moduli"], w["loads"], 1e-6, 1, which=[0])
    dof = g.c * g.N
    return {"value": dof * sum(its) / sum(secs), "unit": UNIT, "cores": cores, "kind": "oracle",
            "time_to_tol_s": sum(secs), "iterations_per_load": its,
            "one_core": {"value": dof * its1[0] / secs1[0], "time_to_tol_s_load0": secs1[0],
                         "iterations_load0": its1[0]},
            "sample": f"32^3 elastic spheres (60, radii 2-4 voxels, E100/nu0.2 in E1/nu0.3), 6 unit Mandel strains, "
                      f"assembled CSR + unpreconditioned CG (C/OpenMP) to ||r||_2/||b||_2 <= 1e-6 on {cores} threads: "
                      f"{sum(secs):.1f} s; load 0 on 1 thread: {secs1[0]:.1f} s"}


def oracle_timing(args):
    """The oracle timed to tolerance on the host cores for the workloads of the benchmark table (all
    threads, and one thread on one load), beside the GPU's FP64 and mixed solves of the same cells, with
    the C_eff of each against a tight FP64 GPU solve (tol 1e-10).  Workloads: the 32 x 32 P1 disc
    (2 loads, tol 1e-8); 64^3 elastic spheres standing in for the 128^3 cell (radii 4-8 voxels, 6 loads,
    tol 1e-6; the assembled 128^3 matrix has 0.5 G entries); 64^3 thresholded GRF conductivity with
    contrast 1000 (correlation length n/32 voxels, 3 loads, tol 1e-6).  The oracle stops on
    ||r||_2 / ||b||_2, the GPU on the K_ref^-1 norm of the residual."""
    import torch
    from oracle import cg_native, fem
    from paper_2203_02962_gb300 import fehom, inputs
    cores = cg_native.max_threads()
    cells = []
    w = inputs.workload_circle2d_32()
    cells.append(("32^2 P1 disc, k 10 in 1, 2 loads, tol 1e-8", (32, 32), w["elem"],
                  "scalar", w["ids"], w["moduli"], w["loads"], 1e-8))
    w = inputs.workload_spheres_elastic(64, seed=0, rmin=4.0, rmax=8.0)
    cells.append(("64^3 hex8 elastic spheres (proxy of the 128^3 cell), 6 loads, tol 1e-6", (64, 64, 64), "hex8_3d",
                  "elastic", w["ids"], w["moduli"], w["loads"], 1e-6))
    w = inputs.workload_grf_scalar(64, seed=0, ell=2.0)
    cells.append(("64^3 hex8 scalar GRF, contrast 1000, 3 loads, tol 1e-6", (64, 64, 64), "hex8_3d", "scalar",
                   w["ids"], w["moduli"], w["loads"], 1e-6))
    rows = []
    for name, shape, elem, phys, ids, mod, loads, tol in cells:
        g = fem.Grid(shape, elem, phys)
        idf = np.ascontiguousarray(ids).ravel()
        its, secs, C_or = _oracle_solve_loads(g, idf, mod, loads, tol, cores)
        its1, secs1, _ = _oracle_solve_loads(g, idf, mod, loads, tol, 1, which=[0])
        n_xyz = tuple(shape[::-1]) + (1,) * (3 - len(shape))
        gpu = {}
        for prec, t in (("ref", 1e-10), ("fp64", tol), ("mixed", tol)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = fehom.Solver(elem, phys, n_xyz, ids, mod, precision="fp64" if prec == "ref" else prec)
            s.precond_build()
            out = s.solve(loads, tol=t, fields=None)
            torch.cuda.synchronize()
            gpu[prec] = (time.perf_counter() - t0, out["C_eff"], [i["iterations"] for i in out["info"]])
            s.close()
        Cr = gpu["ref"][1]
        err = lambda C: float(np.abs(C - Cr).max() / np.abs(Cr).max())  # noqa: E731
        rows.append({"workload": name, "dof": g.c * g.N,
                     "oracle_all_cores": {"threads": cores, "time_to_tol_s": sum(secs), "iterations": its,
                                          "C_eff_rel_err": err(C_or)},
                     "oracle_one_core": {"threads": 1, "time_to_tol_s_load0": secs1[0], "iterations_load0": its1[0]},
                     "gpu_fp64": {"wall_s_setup_build_solve": gpu["fp64"][0], "iterations": gpu["fp64"][2],
                                  "C_eff_rel_err": err(gpu["fp64"][1])},
                     "gpu_mixed": {"wall_s_setup_build_solve": gpu["mixed"][0], "inner_iterations": gpu["mixed"][2],
                                   "C_eff_rel_err": err(gpu["mixed"][1])}})
        print(json.dumps(rows[-1]), flush=True)
    host = {"cores": os.cpu_count(), "machine": os.uname().machine}
    print(json.dumps({"oracle_timing": rows, "host": host}))


def run_reference(args):
    """The oracle arm: each step solves one load of the 32^3 sample (cpu_baseline's cell, loads in turn)
    to tolerance on every host core; value = DOF*iter/s over the timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import cg_native, fem
    from paper_2203_02962_gb300 import inputs
    n = 32
    w = inputs.workload_spheres_elastic(n, seed=0, rmin=n / 16, rmax=n / 8)
    g = fem.Grid((n, n, n), "hex8_3d", "elastic")
    ids = w["ids"].ravel()
    K = cg_native.CSR(fem.assemble_K(g, ids, w["moduli"]))
    rhs = [fem.assemble_rhs(g, ids, w["moduli"], e) for e in w["loads"]]
    cores = cg_native.max_threads()
    for k in range(args.warmup):
        cg_native.cg(K, rhs[k % 6], tol=1e-6, threads=cores)
    its, t0 = 0, time.perf_counter()
    for k in range(args.steps):
        its += cg_native.cg(K, rhs[k % 6], tol=1e-6, threads=cores)[1]
    dt = time.perf_counter() - t0
    v = g.c * g.N * its / dt
    sample = (f"32^3 elastic spheres (60, radii 2-4 voxels), one unit Mandel strain per step, assembled CSR + "
              f"unpreconditioned CG (C/OpenMP, {cores} threads) to ||r||_2/||b||_2 <= 1e-6; {args.steps} steps "
              f"in {dt:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "oracle sample: 32^3 elastic spheres, one load per step, CG to 1e-6"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ncu_case(precision, n_loads=6, rows=0, cell=0):
    """One untimed solve of the benchmark workload (its first n_loads loads), or with cell = 32, 64 or 96
    of the first cell of that size in the batched workload, for kernel captures under ncu; fewer loads
    keep the device memory that ncu saves between replay passes small."""
    import torch
    from paper_2203_02962_gb300 import fehom
    from paper_2203_02962_gb300 import inputs
    w = workload()
    if cell:
        c = next(x for x in inputs.workload_batched_spheres() if x["n"][0] == cell)
        w = dict(n=c["n"], ids=c["ids"], moduli=c["moduli"], loads=inputs.unit_loads(6), tol=1e-6)
    # the FFT plan and the stencil tile height the tuners pick in the timed runs (register-split FFT
    # passes; 8-row FP32 and 16-row FP64 tiles); under ncu the tuners' own timings are serialised
    # replays and would pick differently
    rows = rows or (8 if precision == "mixed" else 16)
    s = fehom.Solver("hex8_3d", "elastic", w["n"], w["ids"], w["moduli"], precision=precision,
                     fft_xy=1 if precision == "mixed" else -1, stencil_rows=rows)
    s.precond_build()
    out = s.solve(w["loads"][:n_loads], tol=w["tol"], fields=None)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": precision, "iterations": [i["iterations"] for i in out["info"]],
                      "launches": s.launch_count()}))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ncu-case", default=None, choices=["fp64", "mixed", "unet"],
                    help="run one untimed solve of the workload (for ncu kernel captures) and exit")
    ap.add_argument("--ncu-loads", type=int, default=6, help="loads of the --ncu-case solve (1-6)")
    ap.add_argument("--ncu-cell", type=int, default=0, choices=[0, 32, 64, 96],
                    help="run the --ncu-case solve on the first cell of this size of the batched workload")
    ap.add_argument("--ncu-rows", type=int, default=0, choices=[0, 8, 16],
                    help="stencil rows of the --ncu-case solve (0: the tuners' usual pick)")
    ap.add_argument("--grf512", action="store_true",
                    help="time FP64 and mixed solves of the 512^3 scalar GRF cell (134M DOF), then exit")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="time the oracle to tolerance on the host cores beside the GPU solves, then exit")
    args = ap.parse_args()
    if args.oracle_timing:
        oracle_timing(args)
        return
    if args.grf512:
        run_grf512(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.ncu_case == "unet":
        args.steps, args.warmup = 2, 1
        print(json.dumps({"ncu_case": "unet", **run_unet(args)}))
        return
    if args.ncu_case:
        run_ncu_case(args.ncu_case, args.ncu_loads, args.ncu_rows, args.ncu_cell)
        return
    run_ours(args)


if __name__ == "__main__":
    main()

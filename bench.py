"""Benchmark of the fused FPC-LBM step on GB300 (one JSON line on stdout).

Workload (default): the 3D differentially heated cubic cavity, 256^3 nodes, D3Q27 flow + D3Q15
energy, FP32 populations, Ra = 1e6, Pr = 0.71, Ma = 0.1 (hot -x, cold +x, adiabatic elsewhere,
gravity along z).  One step = one fused pull-stream + collide launch of both lattices; the wall
Nusselt reduction (FP64) runs on both heated walls once per timed block.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own independent cavity (an ensemble member, no
data exchange) and the aggregate node updates are divided by the slowest rank's time.
``--impl reference`` times the FP64 CPU oracle (the method's plain restatement) on the host cores
for the same workload, a bounded sample of nodes per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MLUPS and % HBM roofline per lattice/precision on 1 GB300; adjoint step time vs "
          "forward")
WORKLOAD = dict(lattice="d3q27", nx=256, ny=256, nz=256, Ra=1e6, Pr=0.71, Ma=0.1, precision="fp32")
KERNEL_SOURCES = ["lbm_common.cuh", "lattices.cuh", "step_d3q27.cuh", "step3d_f32.cu", "kernels.h"]


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(value: float, world: int) -> float:
    """Max of a per-rank value over all ranks (identity on one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the node updates of all ranks over the slowest rank's time."""
    return nodes_per_rank * steps * world / seconds / 1e6


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        ids = [v.strip() for v in vis.split(",")] if vis else []
        self.gpu = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.lines = []
        self.window = None

    def mark(self, start, end):
        """Restrict the summary to samples taken between two datetime.now() marks."""
        self.window = (start, end)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def median_sm_mhz(self, start, end):
        """Median SM clock of the samples taken between two datetime.now() marks, or None."""
        from datetime import datetime
        sm = []
        for line in list(self.lines):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                if start <= ts <= end:
                    sm.append(float(parts[2]))
            except ValueError:
                continue
        return statistics.median(sm) if sm else None

    def summary(self):
        from datetime import datetime
        sm, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                if self.window and not (self.window[0] <= ts <= self.window[1]):
                    continue
                sm.append(float(parts[2]))
                mx = float(parts[3])
                power.append(float(parts[4]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[6:10]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_median": statistics.median(power) if power else None}


# ---------------------------------------------------------------------------------------------
# Measured peaks and committed ncu traffic
# ---------------------------------------------------------------------------------------------
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2504_09041_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it still
    describes the current kernel source (same source hash), else None."""
    p = os.path.join(ROOT, "profiles", "step_d3q27_f32_cavity.md")
    try:
        text = open(p).read()
    except OSError:
        return None
    m_t = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    m_h = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m_t or not m_h or m_h.group(1) != kernel_source_hash():
        return None
    return float(m_t.group(1))


def bench_config(w, steps: int, world: int) -> dict:
    """The `config` of the bench line: the workload, with its sizes.  Both arms (the GPU and the
    oracle reference) report the same dictionary for the same workload."""
    three_d = w["lattice"] == "d3q27"
    n = w["nx"] * w["ny"] * w["nz"]
    elem = {"fp64": 8, "fp32": 4, "fp16s": 2}[w["precision"]]
    bpn = 2.0 * ((27 + 15) if three_d else 18) * elem
    state_gb = bpn / 2 * n / 1e9
    return {"workload": ("3D differentially heated cubic cavity, D3Q27 flow + D3Q15 energy, "
                         f"{w['precision'].upper()} populations, FP64 Nusselt reduction")
            if three_d else
            ("2D Rayleigh-Benard box, D2Q9 flow + D2Q9 energy, "
             f"{w['precision'].upper()} populations, FP64 Nusselt reduction"),
            "nx": w["nx"], "ny": w["ny"], "nz": w["nz"], "Ra": w["Ra"], "Pr": w["Pr"],
            "Ma": w["Ma"], "nodes_per_gpu": n, "bytes_per_node_update": bpn,
            "nusselt_every": steps,
            "l2": (f"inputs larger than L2 ({state_gb:.2f} GB read and {state_gb:.2f} GB "
                   "written per step)") if state_gb > 0.129 else
                  f"inputs fit in L2 ({state_gb * 1e3:.0f} MB per step): not an HBM figure",
            "parallelism": "independent cavity per GPU (ensemble member)" if world > 1
            else "single GPU"}


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    from paper_2504_09041_gb300 import lbm as L

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    w = WORKLOAD
    three_d = w["lattice"] == "d3q27"
    # 3D: the side-heated cubic cavity; 2D: the Rayleigh-Benard box (periodic x, hot bottom)
    walls = L.Walls.cavity(3) if three_d else L.Walls.rayleigh_benard()
    walls.seed = 1000 + rank        # each rank: its own ensemble member
    walls.perturb = 1e-3
    hot, cold = (0, 1) if three_d else (2, 3)
    with torch.cuda.stream(stream):
        lat = L.Lattice(w["lattice"], w["nx"], w["ny"], w["nz"], w["Ra"], w["Pr"], w["Ma"],
                        walls=walls, precision=w["precision"], stream=stream)
    if args.tma_rows:
        lat.set_param("tma_rows", args.tma_rows)
    if args.block:
        bx, by = (int(v) for v in args.block.lower().split("x"))
        lat.set_param("block_x", bx)
        lat.set_param("block_y", by)
    n = lat.n
    info = lat.info()
    bpn = info.bytes_per_node_update

    from datetime import datetime
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with ClockSampler(local) as clocks:
        # warm-up (also gives the clock sampler time to start)
        lat.step(args.warmup)
        lat.nusselt(hot)
        lat.sync()
        barrier(world)
        torch.cuda.synchronize()
        t_start = datetime.now()
        ev[0].record(stream)
        lat.step(args.steps)
        ev[1].record(stream)
        nu_hot = L.lbm_nusselt(lat.h, hot)
        nu_cold = L.lbm_nusselt(lat.h, cold)
        ev[2].record(stream)
        torch.cuda.synchronize()
        clocks.mark(t_start, datetime.now())
        # the other forms run while the sampler still records, so the FP64 forms are set
        # against the SM clock seen while they ran
        forms = []
        if world == 1 and not args.no_forms:
            forms = measure_forms(L, torch, stream, args, clocks)
    barrier(world)
    lat.sync()
    t_total = ev[0].elapsed_time(ev[2]) / 1e3
    t_steps = ev[0].elapsed_time(ev[1]) / 1e3
    t_max = reduce_max(t_total, world)
    launches = args.steps + 2

    # end to end through the C ABI with host buffers: upload a state from pinned host memory,
    # run the steps, read back the wall Nusselt numbers and the temperature field.  One untimed
    # pass of the same job first (as the steps have their warm-up), then the timed pass.
    state_host = torch.empty(info.state_bytes, dtype=torch.uint8).pin_memory()
    T_host = torch.empty(n, dtype=torch.float64).pin_memory()
    L.lbm_get_state(lat.h, state_host.numpy())

    def e2e_job(k):
        L.lbm_set_state(lat.h, state_host.numpy())
        L.lbm_step(lat.h, k)
        L.lbm_nusselt(lat.h, hot)
        L.lbm_nusselt(lat.h, cold)
        L.lbm_fields(lat.h, None, None, None, None, T_host.data_ptr(), 0)

    e2e_job(args.steps)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_job(args.steps)
    torch.cuda.synchronize()
    t_e2e = reduce_max(time.perf_counter() - t0, world)

    adjoint, batched, nu_acc = None, None, None
    if world == 1 and not args.no_forms:
        nu_acc = measure_nu_accuracy(L, stream)
        batched = measure_batched(L, torch, stream)
        adjoint = measure_adjoint(L, torch, stream)

    clk = clocks.summary()
    lat.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return None

    mlups = job_mlups(n, args.steps, world, t_max)
    step_s = t_steps / args.steps
    achieved = bpn * n / step_s / 1e9
    peak, peak_kind = hbm_peak()
    # the committed ncu traffic describes the 256^3 FP32 step only
    traffic = (committed_traffic() if three_d and w["precision"] == "fp32"
               and (w["nx"], w["ny"], w["nz"]) == (256, 256, 256) else None)
    e2e = job_mlups(n, args.steps, world, t_e2e)
    line = {
        "metric": METRIC,
        "value": round(mlups, 2),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_max / args.steps * 1e3, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16s": "f16 storage, f32 arithmetic"}[w["precision"]],
        "data": "synthetic (seeded initial temperature perturbation +-1e-3 of the cavity at rest)",
        "config": bench_config(w, args.steps, world),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_kind": peak_kind,
                     "kernel": ("step_d3q27_kernel" if three_d else "step_d2q9_kernel")
                     + "<Store" + {"fp32": "F32", "fp64": "F64", "fp16s": "F16S"}[w["precision"]] + ">",
                     "launch_ms": round(step_s * 1e3, 4), "traffic_unit": "bytes per launch",
                     "block": [info.block_x, info.block_y]},
        "e2e": {"value": round(e2e, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": info.state_bytes / args.steps,
                "d2h_bytes_per_step": (8 * n + 80) / args.steps,
                "job": "set_state from pinned host + K steps + 2 wall Nusselt + T field to host"},
        "gpu_launches": launches,
        "clocks": clk,
        "nusselt": {"hot_mean": nu_hot[0], "cold_mean": nu_cold[0],
                    "after_steps": args.warmup + args.steps},
    }
    cpu = None if args.no_cpu_baseline else cpu_baseline(seconds=args.cpu_seconds)
    return append_secondary(line, forms, nu_acc, batched, adjoint, cpu)


def append_secondary(line, forms, nu_acc, batched, adjoint, cpu):
    """Add the secondary measurements to the bench line: the detailed records first, the compact
    per-form table and the accuracy summary last, so that a reader who keeps only the end of the
    line still sees every form's figures."""
    if forms:
        line["per_form_detail"] = forms
    if nu_acc:
        line["nu_accuracy_detail"] = nu_acc
    if batched:
        line["batched"] = batched
    if adjoint:
        line["adjoint"] = adjoint
    line["paper_context"] = PAPER_CONTEXT
    if cpu:
        line["cpu_baseline"] = cpu
    if nu_acc:
        line["nu_accuracy"] = compact_nu_accuracy(nu_acc)
    if forms or batched or adjoint:
        line["per_form"] = compact_forms(line, forms, batched, adjoint)
    return line


FORM_BOUND = {"fp32": "hbm", "fp16s": "issue", "fp64": "fp64 alu"}


def compact_forms(line, forms, batched, adjoint):
    """One short record per measured form: the headline, the other lattice / precision forms,
    the batched ensemble and the adjoint ratio."""
    r = line["roofline"]
    cfg = line["config"]
    out = [{"form": f"{'3D' if cfg['nz'] > 1 else '2D'} {line['dtype']} (headline)",
            "box": f"{cfg['nx']}x{cfg['ny']}x{cfg['nz']}", "mlups": line["value"],
            "gbs": r["achieved"], "hbm_frac": r["frac"], "bound": r["bound"]}]
    for f in forms:
        rec = {"form": f"{'3D' if f['lattice'].startswith('D3') else '2D'} {f['precision']}"
                       + (" option B" if f["g_attractors"] == "option B" else ""),
               "box": "x".join(str(v) for v in f["box"]), "mlups": f["mlups"], "gbs": f["gbs"],
               "hbm_frac": f["hbm_frac"], "bound": FORM_BOUND[f["precision"]]}
        if "roofline" in f:
            rec["alu_frac"] = f["roofline"]["frac"]
        if f.get("l2_resident"):
            rec["note"] = "one step's state fits in L2: not an HBM figure"
        out.append(rec)
    if batched:
        out.append({"form": "2D fp32 batched ensemble", "box": f"{batched['nodes']} nodes",
                    "mlups": batched["mlups"], "gbs": batched["gbs"], "hbm_frac": batched["hbm_frac"],
                    "bound": "hbm", "speedup_vs_unbatched": batched["speedup_vs_unbatched"]})
    if adjoint:
        out.append({"form": "2D adjoint 256x256 (double-float VJP)",
                    "adjoint_ms_per_step": adjoint["adjoint_ms_per_step"],
                    "forward_ms_per_step": adjoint["forward_ms_per_step"],
                    "adjoint_over_forward": adjoint["adjoint_over_forward"]})
    return out


def compact_nu_accuracy(nu_acc):
    """Mean hot-wall Nu of FP64 and the relative deviation of the FP32 and FP16S forms."""
    return [{"case": a["case"].split(",")[0] + ", " + a["case"].split(",")[1].strip(),
             "nu_fp64": round(a["nu_hot_mean"]["fp64"], 6),
             "fp32_rel": float(f"{a['rel_vs_fp64']['fp32']:.3g}"),
             "fp16s_rel": float(f"{a['rel_vs_fp64']['fp16s']:.3g}")} for a in nu_acc]


# FP64 lane operations per node update of the FP64 steps at the default rates (ncu instruction
# counts of the FP64 kernels, committed with the profiles; the 3D count is that of the reduced
# collisions the default rates select) and GB300's FP64 pipe rate: 2 lane operations per SM per
# clock.
FP64_OPS_PER_NODE = {"d3q27": 866.8, "d2q9": 340.6}
FP64_LANE_OPS_PER_SM_CLK = 2


def fp64_alu_roofline(mlups: float, lattice: str = "d3q27", sms: int = 152, clock_ghz: float = 2.07,
                      clock_kind: str = "nominal maximum"):
    """The FP64 form against the FP64 pipe: sms and clock_ghz are the device's SM count and the
    SM clock sampled while the form ran (the nominal maximum when no sample was taken)."""
    peak = sms * FP64_LANE_OPS_PER_SM_CLK * clock_ghz              # G lane-ops / s
    achieved = mlups * 1e6 * FP64_OPS_PER_NODE[lattice] / 1e9
    return {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G FP64 lane-ops/s", "frac": round(achieved / peak, 4),
            "peak_kind": f"derived: {sms} SMs x {FP64_LANE_OPS_PER_SM_CLK} FP64 lanes/clk x "
                         f"{clock_ghz:.3f} GHz ({clock_kind})"}


def measure_forms(L, torch, stream, args, clocks=None):
    """MLUPS and HBM fraction of the other lattice / precision forms on the same GPU.  The FP64
    forms are also set against the FP64 pipe of this device (its SM count, and the median SM clock
    sampled while the form ran)."""
    from datetime import datetime
    out = []
    peak, _ = hbm_peak()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cases = [("d3q27", 256, 256, 256, "fp64", L.Walls.cavity(3), 1e6, 40, 0),
             ("d3q27", 256, 256, 256, "fp16s", L.Walls.cavity(3), 1e6, 50, 0),
             ("d3q27", 256, 256, 256, "fp32", L.Walls.cavity(3), 1e6, 50, 1),
             ("d2q9", 1024, 512, 1, "fp64", L.Walls.rayleigh_benard(seed=1), 1e8, 2000, 0),
             ("d2q9", 1024, 512, 1, "fp32", L.Walls.rayleigh_benard(seed=1), 1e8, 400, 0),
             ("d2q9", 1024, 512, 1, "fp16s", L.Walls.rayleigh_benard(seed=1), 1e8, 400, 0)]
    for lat_name, nx, ny, nz, prec, walls, Ra, k, gopt in cases:
        lat = L.Lattice(lat_name, nx, ny, nz, Ra, 0.71, 0.1, walls=walls, precision=prec, stream=stream)
        lat.set_param("g_attractors", gopt)
        lat.step(5)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_a = datetime.now()
        e0.record(stream)
        lat.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        t_b = datetime.now()
        lat.sync()
        s = e0.elapsed_time(e1) / 1e3 / k
        bpn = lat.info().bytes_per_node_update
        gbs = bpn * lat.n / s / 1e9
        rec = {"lattice": "D3Q27+D3Q15" if lat_name == "d3q27" else "D2Q9+D2Q9",
               "precision": prec, "box": [nx, ny, nz], "mlups": round(lat.n / s / 1e6, 1),
               "ms_per_step": round(s * 1e3, 4), "gbs": round(gbs, 1),
               "hbm_frac": round(gbs / peak, 4), "steps": k,
               "g_attractors": "option B" if gopt else "option A",
               "l2_resident": bpn / 2 * lat.n < 129e6}
        if prec == "fp64":
            mhz = clocks.median_sm_mhz(t_a, t_b) if clocks is not None else None
            rec["roofline"] = (fp64_alu_roofline(lat.n / s / 1e6, lat_name, sms, mhz / 1e3,
                                                 "median SM clock sampled during the form")
                               if mhz else fp64_alu_roofline(lat.n / s / 1e6, lat_name, sms))
        out.append(rec)
        lat.close()
    return out


def measure_nu_accuracy(L, stream):
    """Mean hot-wall Nu of the FP32 and FP16-storage forms against the FP64 form on the same GPU:
    the 64^2 cavity at Ra 1e4 after 20,000 steps (steady), a 32^3 cavity at Ra 1e5 after 20,000
    steps (both at Ma 0.1), and a 128^2 cavity at the paper's U_o = 0.01, where the per-step
    changes are six times smaller against the stored values."""
    cases = [("2D cavity 64x64, Ra 1e4, Pr 0.71, 20000 steps", "d2q9", 64, 64, 1, 1e4, 2, 0.1, 20000),
             ("3D cavity 32^3, Ra 1e5, Pr 0.71, 20000 steps", "d3q27", 32, 32, 32, 1e5, 3, 0.1, 20000),
             ("2D cavity 128x128 at U_o 0.01 (Ma 0.0173), Ra 1e5, Pr 0.71, 500000 steps", "d2q9",
              128, 128, 1, 1e5, 2, 0.01 * 3 ** 0.5, 500000)]
    out = []
    for label, lat_name, nx, ny, nz, Ra, dim, Ma, steps in cases:
        nu = {}
        for prec in ("fp64", "fp32", "fp16s"):
            lat = L.Lattice(lat_name, nx, ny, nz, Ra, 0.71, Ma, walls=L.Walls.cavity(dim),
                            precision=prec, stream=stream)
            lat.step(steps)
            lat.sync()
            nu[prec] = lat.nusselt(0)[0]
            lat.close()
        out.append({"case": label, "nu_hot_mean": nu,
                    "rel_vs_fp64": {p: abs(nu[p] - nu["fp64"]) / abs(nu["fp64"]) for p in ("fp32", "fp16s")}})
    return out


def measure_batched(L, torch, stream, steps: int = 2000, unbatched_steps: int = 256,
                    compare: bool = True, launch=None):
    """The ensemble workload: 64 independent square cavities (sides 64..512, Ra log-uniform in
    [1e3, 1e7], Pr uniform in [0.71, 7], seeded), FP32, one autotuned launch per
    step replayed from CUDA graphs.  Compared with the same members advanced one handle at a
    time (each with its own CUDA graphs), and, for a few members, the wall Nusselt number
    against FP64 unbatched runs of the same length."""
    from paper_2504_09041_gb300.workloads import ensemble_2d
    sizes, Ra, Pr = ensemble_2d()
    peak, _ = hbm_peak()
    b = L.Batch(sizes, Ra, Pr, Ma=0.1, precision="fp32", stream=stream)
    t0 = time.perf_counter()
    if launch:
        tx, ty, cps = launch
        b.set_launch(tx, ty, cps)
    else:
        tx, ty, cps = b.tune(20)
    tune_s = time.perf_counter() - t0
    b.step(64)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    flags = b.sync()
    t = e0.elapsed_time(e1) / 1e3 / steps
    inf = b.info()
    nodes = inf.total_nodes
    bpn = inf.bytes_per_node_update

    if not compare:
        b.close()
        gbs = bpn * nodes / t / 1e9
        return {"nodes": nodes, "mlups": round(nodes / t / 1e6, 1), "gbs": round(gbs, 1),
                "hbm_frac": round(gbs / peak, 4), "steps": steps,
                "launch": {"tile": [tx, ty], "ctas_per_sm": cps, "grid": inf.grid}}

    # the same members, one handle each, stepped one after the other on the same stream
    lats = [L.Lattice("d2q9", nx, ny, 1, Ra=Ra[k], Pr=Pr[k], Ma=0.1, precision="fp32",
                      stream=stream) for k, (nx, ny) in enumerate(sizes)]
    for lat in lats:
        lat.step(64)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in lats:
        lat.step(unbatched_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_un = e0.elapsed_time(e1) / 1e3 / unbatched_steps
    for lat in lats:
        lat.close()

    # Nusselt accuracy of FP32 batched members against FP64 unbatched runs of equal length
    order = sorted((sizes[k][0] * sizes[k][1], k) for k in range(len(sizes)) if not flags[k])
    picks = [k for _, k in order[:4]]
    nu_err = []
    for k in picks:
        nx, ny = sizes[k]
        ref = L.Lattice("d2q9", nx, ny, 1, Ra=Ra[k], Pr=Pr[k], Ma=0.1, precision="fp64",
                        stream=stream)
        ref.step(inf.steps)
        nb = b.nusselt(k, 0)[0]
        nr = ref.nusselt(0)[0]
        nu_err.append({"member": k, "side": nx, "Ra": round(Ra[k], 1), "Pr": round(Pr[k], 3),
                       "nu_fp32_batched": nb, "nu_fp64": nr, "rel": abs(nb - nr) / abs(nr)})
        ref.close()
    b.close()
    gbs = bpn * nodes / t / 1e9
    return {"workload": "64 independent 2D cavities, sides drawn from {64,...,512}, Ra log-uniform "
                        "[1e3, 1e7], Pr uniform [0.71, 7], FP32, one autotuned launch per step "
                        "under CUDA graphs",
            "nodes": nodes, "mlups": round(nodes / t / 1e6, 1), "ms_per_step": round(t * 1e3, 5),
            "gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4), "steps": steps,
            "launch": {"tile": [tx, ty], "ctas_per_sm": cps, "grid": inf.grid,
                       "tiles": inf.n_tiles, "tune_seconds": round(tune_s, 3)},
            "unbatched_mlups": round(nodes / t_un / 1e6, 1),
            "unbatched_ms_per_step": round(t_un * 1e3, 5),
            "speedup_vs_unbatched": round(t_un / t, 3),
            "diverged_members": int(flags.sum()),
            "nusselt_vs_fp64": nu_err,
            "nusselt_max_rel": max(e["rel"] for e in nu_err) if nu_err else None}


def run_only(args):
    """One secondary measurement on its own (used to profile its kernel)."""
    import torch
    from paper_2504_09041_gb300 import lbm as L
    stream = torch.cuda.Stream()
    if args.only == "batched":
        launch = tuple(int(v) for v in args.batch_launch.split("x")) if args.batch_launch else None
        return measure_batched(L, torch, stream, steps=args.steps, compare=False, launch=launch)
    return measure_adjoint(L, torch, stream)


def measure_adjoint(L, torch, stream):
    """The adjoint workload: 256^2 cavity, Ra 1e5, 2000 steps, gradient of the mean cold-wall Nu
    with respect to the 256-node hot-wall profile; FP32 forward, double-float adjoint (the default),
    with the FP64 and FP32 adjoint arithmetic timed beside it.  Reports the time
    per forward step and per adjoint step (the whole lbm_adjoint_step call, checkpointed forward,
    segment recomputation and adjoint kernels, divided by the step count)."""
    import numpy as np
    import math
    from paper_2504_09041_gb300.workloads import sine_profile
    n, steps = 256, 2000
    prof = sine_profile(2024, n)
    lat = L.Lattice("d2q9", n, n, 1, 1e5, 0.71, 0.1, walls=L.Walls.cavity(2), precision="fp32",
                    stream=stream)
    lat.set_wall_profile(0, prof)
    state0 = lat.get_state()
    lat.step(20)
    lat.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat.set_state(state0)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / 1e3
    timings = {}
    for flag in (2, 1, 0):
        lat.set_param("adjoint_arith", flag)
        lat.set_state(state0)
        lat.adjoint(50, 1, 0)          # warm-up of the adjoint path
        lat.set_state(state0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, grad = lat.adjoint(steps, 1, 0)
        timings[flag] = (time.perf_counter() - t0, J, grad)
    lat.close()
    adj, J, grad = timings[2]
    adj64, _, grad64 = timings[1]
    adj32 = timings[0][0]
    return {"workload": "2D cavity 256x256, Ra 1e5, Pr 0.71, 2000 steps, dJ/dT_w of the mean "
                        "cold-wall Nu w.r.t. the 256-node hot-wall profile",
            "forward_ms_per_step": round(fwd / steps * 1e3, 5),
            "adjoint_ms_per_step": round(adj / steps * 1e3, 5),
            "adjoint_over_forward": round(adj / fwd, 3),
            "fp32_arithmetic": {"adjoint_ms_per_step": round(adj32 / steps * 1e3, 5),
                                "adjoint_over_forward": round(adj32 / fwd, 3)},
            "fp64_arithmetic": {"adjoint_ms_per_step": round(adj64 / steps * 1e3, 5),
                                "adjoint_over_forward": round(adj64 / fwd, 3)},
            "max_abs_diff_vs_fp64_rel": float(np.abs(grad - grad64).max() / np.abs(grad64).max()),
            "arithmetic": "FP32 forward states; double-float (FP32-pair, 48-bit significand) "
                          "vector-Jacobian products and adjoint state; FP64 gradient accumulation",
            "J": J,
            "grad_norm": float(np.linalg.norm(grad)),
            "checkpoints": int(math.ceil(math.sqrt(steps)))}


# ---------------------------------------------------------------------------------------------
# CPU side: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------------------
def oracle_sample(seconds: float):
    """Time the oracle on slabs of the 256^3 cavity (full x-y planes, a few z layers) until about
    `seconds` of wall time has been spent; returns (MLUPS, threads, description)."""
    from oracle import oracle as O
    w = WORKLOAD
    nz = 4
    ora = O.Oracle(3, w["nx"], w["ny"], nz, bc=O.cavity_bc(3), Ra=w["Ra"], Pr=w["Pr"], Ma=w["Ma"])
    # the rates and g beta of the full 256^3 cavity (L = 256 along x, as in the slab)
    nodes, t_sum, reps = 0, 0.0, 0
    while t_sum < seconds or reps == 0:
        t0 = time.perf_counter()
        ora.update_box(0, w["nx"], 0, w["ny"], 0, nz)
        t_sum += time.perf_counter() - t0
        nodes += w["nx"] * w["ny"] * nz
        reps += 1
    desc = (f"{reps} node-update sweeps of a {w['nx']}x{w['ny']}x{nz} slab of the 256^3 cavity "
            f"({nodes} node updates, {t_sum:.1f} s)")
    return nodes / t_sum / 1e6, O.threads(), desc


def oracle_single_thread(seconds: float):
    """The same slab sample on one host thread (a child process with OMP_NUM_THREADS=1)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "m, c, d = bench.oracle_sample(%r); print(json.dumps([m, c]))" % (ROOT, seconds))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        return None
    m, c = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": round(m, 4), "unit": "MLUPS", "cores": c}


def oracle_cavity_64():
    """The 64^2 differentially heated cavity (Ra 1e4, Pr 0.71, Ma 0.1) run to 20000 steps by the
    oracle on all host threads, with its hot-wall Nusselt number beside Table con2's 2.2431."""
    from oracle import oracle as O
    ora = O.Oracle(2, 64, 64, 1, bc=O.cavity_bc(2), Ra=1e4, Pr=0.71, Ma=0.1)
    t0 = time.perf_counter()
    ora.step(20000)
    t = time.perf_counter() - t0
    return {"seconds": round(t, 2), "mlups": round(64 * 64 * 20000 / t / 1e6, 3),
            "nu_hot_mean": round(ora.nusselt(0)[0], 5), "table_con2_512": 2.2431,
            "cores": O.threads()}


# The paper's only timing (context, not a target): 128^3 D3Q27 + D3Q15 at Ra 1e8, 5e6 steps in
# 30.7 h on 512 CPU cores (C++ + MPI), i.e. 128^3 * 5e6 / (30.7 * 3600 s) node updates per second.
PAPER_CONTEXT = {"value": round(128 ** 3 * 5e6 / (30.7 * 3600) / 1e6, 1), "unit": "MLUPS",
                 "hardware": "512 CPU cores (INCLINE cluster), C++ with MPI",
                 "workload": "3D D3Q27 flow + D3Q15 energy, 128^3, Ra 1e8",
                 "precision": "not stated", "source": "Sec. 6.2 (run time) and Sec. 7"}


def cpu_baseline(seconds: float = 15.0):
    mlups, cores, desc = oracle_sample(seconds)
    out = {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
           "sample": desc}
    single = oracle_single_thread(min(5.0, seconds))
    if single:
        out["single_thread"] = single
    out["cavity_64x64_20000_steps"] = oracle_cavity_64()
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from oracle import oracle as O
    w = WORKLOAD
    nz = 2
    ora = O.Oracle(3, w["nx"], w["ny"], nz, bc=O.cavity_bc(3), Ra=w["Ra"], Pr=w["Pr"], Ma=w["Ma"])
    for _ in range(args.warmup):
        ora.update_box(0, w["nx"], 0, w["ny"], 0, nz)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ora.update_box(0, w["nx"], 0, w["ny"], 0, nz)
    t = time.perf_counter() - t0
    nodes = w["nx"] * w["ny"] * nz * args.steps
    mlups = nodes / t / 1e6
    sample = (f"each step updates a {w['nx']}x{w['ny']}x{nz} slab of the 256^3 cavity "
              f"({w['nx'] * w['ny'] * nz} nodes) with the FP64 oracle")
    return {"metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": bench_config(w, args.steps, world),
            "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": O.threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--block", default=None, help="thread-block shape of the step, e.g. 128x1")
    ap.add_argument("--tma-rows", type=int, default=0, choices=[0, 1, 2, 4],
                    help="TMA-staged 3D step with tiles of 64 x rows nodes (0 = plain step)")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "fp16s"])
    ap.add_argument("--lattice", default=None, choices=["d3q27", "d2q9"],
                    help="main workload: the 3D cavity (default) or the 2D Rayleigh-Benard box")
    ap.add_argument("--nx", type=int, default=None, help="override the box (profiling cases)")
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--nz", type=int, default=None)
    ap.add_argument("--only", default=None, choices=["batched", "adjoint"],
                    help="run one secondary measurement alone and print its record (profiling)")
    ap.add_argument("--batch-launch", default=None,
                    help="with --only batched: fixed launch TXxTYxCPS instead of the autotuner (profiling)")
    args = ap.parse_args(argv)
    if args.batch_launch and (args.only != "batched" or len(args.batch_launch.split("x")) != 3):
        ap.error("--batch-launch takes TXxTYxCPS and needs --only batched")
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.lattice == "d2q9":
        WORKLOAD.update(lattice="d2q9", nx=1024, ny=512, nz=1, Ra=1e8)
    for k in ("nx", "ny", "nz", "precision"):
        if getattr(args, k) is not None:
            WORKLOAD[k] = getattr(args, k)
    if args.only:
        print(json.dumps(run_only(args)), flush=True)
        return
    line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

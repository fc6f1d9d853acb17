"""Throughput of the fused free-energy D2Q9 step on GB300 (MLUPS and HBM roofline).

Workload: 4096 x 4096 periodic spinodal decomposition, improved scheme (Eqs. 24,
27-29), MRT collision (Eq. 8), FP32 populations stored as deviations from
w_a rho_ref. EOS: the paper's van der Waals set (a = 9/392, b = 2/21, kappa =
0.02) at T = 0.8 T_c; initial density = mean of the Maxwell densities times
(1 + U[-0.01, 0.01]) from the seeded SplitMix64 stream. One step = one time
step of the whole lattice (one fused kernel launch). The populations (1.2 GB
per step read + write) exceed the 129 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--scheme improved|improved_smooth|standard|standard_pt] [--walls] [--side N]

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle on a
bounded 256 x 256 sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D2Q9 free-energy LB MLUPS & % HBM roofline, FP32/batched vs plain FP64"
N_SIDE = 4096
T_RED = 0.8
BYTES_PER_NODE = {"f32": 72, "f64": 144}  # 9 populations read + 9 written
VDW = dict(a=9.0 / 392.0, b=2.0 / 21.0, R=1.0)
SAMPLE_SIDE = 256
WORKLOAD = (f"spinodal {N_SIDE}x{N_SIDE} periodic, improved scheme, MRT (tau_v 0.8, tau_e 1.0, tau_s 1.0, "
            f"tau_q 1.1), vdW a=9/392 b=2/21 kappa=0.02 at T/Tc={T_RED}, FP32 deviation storage")


def _max_over_ranks(x: float, ws: int, device) -> float:
    """Largest value of x over the ranks (the job is as slow as its slowest
    replica); identity at one rank."""
    if ws <= 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_mlups(ws: int, nodes_per_rank: int, steps: int, ms: float) -> float:
    """Whole-job throughput: node updates of all ranks over the slowest rank's time."""
    return ws * nodes_per_rank * steps / (ms * 1e-3) / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


PROFILE = os.path.join(ROOT, "profiles", "step_kernel_pair_spinodal4096.json")
# files that define the FP32 step kernel and its launch
STEP_SOURCES = ("launch.h", "lbfe_device.cuh", "step_f32.cu", "step_f32_pair.cuh", "step_f32_pair1.cu", "step_kernel.cuh",
                "step_pair.cuh", "step_tma.cuh")


def _kernel_source_sha256() -> str:
    import hashlib

    d = os.path.join(ROOT, "paper_2008_01473_gb300", "csrc")
    h = hashlib.sha256()
    for f in STEP_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _profiled_traffic(n_side: int):
    """DRAM bytes per step launch from the committed ncu record of this
    workload (profiles/*.json), or None if the kernel sources changed since it
    was taken or the lattice differs."""
    try:
        with open(PROFILE) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("nx") != n_side or rec.get("source_sha256") != _kernel_source_sha256():
        return None
    return int(rec["traffic_bytes_per_launch"])


# FP64 step (one column per thread): FP64 instructions executed per node update,
# halo recomputation included, from ncu's per-opcode thread counts at 2048^2
# (DADD 111.4, DFMA 88.5, DMUL 30.6); FLOPs count 2 per DFMA.
FP64_INST_PER_NODE = 230.5
FP64_FLOP_PER_NODE = 2 * 88.5 + 111.4 + 30.6
# GB300 FP64 rate: 2 FP64 thread-instructions per clock per SM (1.25 TFLOP/s
# of DFMA over 152 SMs at 2.07 GHz)
FP64_PER_CLK_SM, N_SMS, SM_MAX_GHZ = 2, 152, 2.07


def _fp64_roofline(nodes: int, mean_ms: float, hbm_frac: float) -> dict:
    """The FP64 step is bound by the FP64 pipe, not by HBM."""
    rate = nodes / (mean_ms * 1e-3)
    peak = N_SMS * FP64_PER_CLK_SM * 2 * SM_MAX_GHZ * 1e9
    achieved = rate * FP64_FLOP_PER_NODE
    return {"bound": "alu", "achieved": round(achieved / 1e12, 4), "peak": round(peak / 1e12, 4),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz",
            "fp64_pipe_frac": round(rate * FP64_INST_PER_NODE / (N_SMS * FP64_PER_CLK_SM * SM_MAX_GHZ * 1e9), 4),
            "fp64_inst_per_node": FP64_INST_PER_NODE, "hbm_frac": round(hbm_frac, 4),
            "kernel_ms_mean": round(mean_ms, 4)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index  # nvidia-smi id of the GPU (PCI bus id, or its index)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cs_variant(lbfe, inputs, n_side: int, prec, local: int, rank: int, steps: int = 20) -> dict:
    """Throughput of the Carnahan-Starling variant of the same step on the same
    lattice: CS with the vdW set's a and a/b (a = 9/392, b = 9/98), 0.8 T_c,
    which keeps the interface as wide as the vdW set's; device-resident
    populations, CUDA events over `steps` launches after the warm-up."""
    import torch

    a, b = 9.0 / 392.0, 9.0 / 98.0
    tc, _ = lbfe.critical(lbfe.CS, a, b, 1.0)
    T = T_RED * tc
    rg, rl = lbfe.maxwell(lbfe.CS, a, b, 1.0, T)
    case = lbfe.Case(nx=n_side, ny=n_side, scheme=lbfe.IMPROVED, collision=lbfe.MRT, eos=lbfe.CS, a=a, b=b, R=1.0,
                     T=T, kappa=0.02, tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1)
    lat = lbfe.Lattice([case], precision=prec, device=f"cuda:{local}")
    lat.init_fields(0, inputs.spinodal(n_side, n_side, 0.5 * (rg + rl), 0.01, seed=1 + rank))
    lat.step(16)  # autotune, and the 8-step graph of the buffer parity the timed steps start from
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, st = lat.reductions()
    lat.close()
    return {"value": round(n_side * n_side * steps / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "steps": steps,
            "workload": f"spinodal {n_side}x{n_side}, improved, MRT, CS a=9/392 b=9/98 at T/Tc={T_RED}",
            "stable": bool(st[0] == 0)}


def _parse_cpulist(txt: str) -> set:
    cpus = set()
    for part in txt.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def _format_cpulist(cpus) -> str:
    """The inverse of _parse_cpulist: sorted ranges, e.g. '0-7,64-71'."""
    out, run = [], []
    for c in sorted(cpus):
        if run and c == run[-1] + 1:
            run.append(c)
            continue
        if run:
            out.append(f"{run[0]}-{run[-1]}" if len(run) > 1 else str(run[0]))
        run = [c]
    if run:
        out.append(f"{run[0]}-{run[-1]}" if len(run) > 1 else str(run[0]))
    return ",".join(out)


def _smooth_variant(lbfe, inputs, n_side: int, local: int, rank: int, steps: int = 40) -> dict:
    """Throughput of the averaged correction (LB_IMPROVED_SMOOTH) on the same
    4096^2 vdW spinodal, MRT, 0.8 T_c, FP32: the packed kernel's scheme-3
    variant; device-resident populations, CUDA events over `steps` launches
    of one lb_step call after the warm-up."""
    import torch

    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    T = T_RED * tc
    rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], T)
    case = lbfe.Case(nx=n_side, ny=n_side, scheme=lbfe.IMPROVED_SMOOTH, collision=lbfe.MRT, eos=lbfe.VDW, T=T,
                     kappa=0.02, tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1, **VDW)
    lat = lbfe.Lattice([case], precision=lbfe.FP32, device=f"cuda:{local}")
    lat.init_fields(0, inputs.spinodal(n_side, n_side, 0.5 * (rg + rl), 0.01, seed=1 + rank))
    lat.step(16)  # autotune, and the 8-step graph of the buffer parity the timed steps start from
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    _, st = lat.reductions()
    lat.close()
    peak, _ = _peaks()
    value = n_side * n_side * steps / (ms * 1e-3) / 1e6
    achieved = BYTES_PER_NODE["f32"] * value * 1e6 / 1e9
    return {"value": round(value, 1), "unit": "MLUPS", "steps": steps,
            "workload": f"spinodal {n_side}x{n_side}, improved scheme with the correction of Eq. 29 on the "
                        f"lattice-weight average of phi u, MRT, vdW at T/Tc={T_RED}, FP32",
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4)},
            "stable": bool(st[0] == 0)}


def _pci_ids(props):
    """(nvidia-smi id, sysfs name) of a CUDA device from its PCI location
    (torch device properties: pci_domain_id, pci_bus_id, pci_device_id). The
    CUDA ordinal is not nvidia-smi's index once CUDA_VISIBLE_DEVICES remaps
    the devices; the bus id names the same GPU for both."""
    dom, bus, dev = (int(getattr(props, k)) for k in ("pci_domain_id", "pci_bus_id", "pci_device_id"))
    return f"{dom:08X}:{bus:02X}:{dev:02X}.0", f"{dom:04x}:{bus:02x}:{dev:02x}.0"


def _gpu_ids(local: int):
    """PCI ids of CUDA device `local`, or (str(local), None) where torch does
    not expose the PCI location."""
    import torch

    try:
        return _pci_ids(torch.cuda.get_device_properties(local))
    except Exception:
        return str(local), None


def _bind_to_gpu_node(sysfs_name):
    """Restrict this process to the host cores local to the GPU at PCI
    location `sysfs_name`, so that its pinned host buffers are allocated on
    that GPU's memory node; returns the core list, or None where the topology
    is not exposed."""
    if not sysfs_name:
        return None
    try:
        with open(f"/sys/bus/pci/devices/{sysfs_name}/local_cpulist") as fh:
            cpus = _parse_cpulist(fh.read()) & os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return f"{_format_cpulist(cpus)} ({len(cpus)} cores)"
    except Exception:
        return None


def _host_link(rho0_pin, res, stream) -> dict:
    """Rates of the host link for the end-to-end leg's copies: rho0 host to
    device and the three FP64 fields device to host (pinned host memory,
    cudaMemcpyAsync on the library's stream, CUDA events, best of 3)."""
    import torch

    dev = [torch.empty_like(rho0_pin, device="cuda") for _ in range(3)]
    out = {}
    for name, fn, nbytes in (("h2d", lambda: dev[0].copy_(rho0_pin, non_blocking=True), rho0_pin.nbytes),
                             ("d2h", lambda: [h.copy_(d, non_blocking=True) for h, d in zip(res.values(), dev)],
                              sum(h.nbytes for h in res.values()))):
        best = 1e30
        with torch.cuda.stream(stream):
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
        out[name + "_ms"] = round(best, 3)
        out[name + "_GBs"] = round(nbytes / (best * 1e-3) / 1e9, 1)
    return out


# --scheme of the spinodal workload: library scheme code and the name in config.workload
SCHEMES = {"improved": ("IMPROVED", "improved scheme"),
           "improved_smooth": ("IMPROVED_SMOOTH", "improved scheme with the correction of Eq. 29 taken on the "
                                                   "lattice-weight average of phi u"),
           "standard": ("STANDARD", "standard scheme (chemical-potential force)"),
           "standard_pt": ("STANDARD_PT", "standard scheme (pressure-tensor force)")}


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2008_01473_gb300 import build, inputs, lbfe

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    smi_id, sysfs_name = _gpu_ids(local)
    host_cpus = _bind_to_gpu_node(sysfs_name)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    build.build()
    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    T = T_RED * tc
    rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], T)
    n_side = args.side
    scheme = getattr(lbfe, SCHEMES[args.scheme][0])
    # --walls: no-slip plates at rest half a node outside rows 0 and ny - 1 (Sec. IV C's walls)
    wall_kw = dict(walls=1, wall_u=0.0, rho_wall=0.5 * (rg + rl)) if args.walls else {}
    case = lbfe.Case(nx=n_side, ny=n_side, scheme=scheme, collision=lbfe.MRT, eos=lbfe.VDW, T=T,
                     kappa=0.02, tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1, **VDW, **wall_kw)
    nodes = n_side * n_side
    rho0 = inputs.spinodal(n_side, n_side, 0.5 * (rg + rl), 0.01, seed=1 + rank)
    rho0_pin = torch.from_numpy(rho0).pin_memory()
    prec = lbfe.FP64 if args.precision == "fp64" else lbfe.FP32
    dtype = "f64" if prec == lbfe.FP64 else "f32"
    lat = lbfe.Lattice([case], precision=prec, device=f"cuda:{local}")
    stream = lat.stream

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    # ------------------------------------------------------ device-resident
    # The timed region is one lb_step(K) call, the library's own path: CUDA
    # graphs of 8 steps replayed back to back, then K mod 8 direct launches.
    # The graph of the buffer parity the region starts from is captured in
    # the warm-up (8 more untimed steps when W steps did not capture it).
    lat.init_fields(0, rho0_pin)
    lat.step(args.warmup)
    capture_steps = 0 if (args.warmup >= 8 and args.warmup % 2 == 0) else 8
    lat.step(capture_steps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    clocks = Clocks(smi_id)
    clocks.start()
    time.sleep(0.4)
    barrier()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        lat.step(args.steps)
        ev[1].record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = _max_over_ranks(ev[0].elapsed_time(ev[1]), ws, f"cuda:{local}")
    out, st = lat.reductions()
    stable = bool(st[0] == 0)
    # spread of single launches (outside the timed region): one lb_step(1) each
    pev = [torch.cuda.Event(enable_timing=True) for _ in range(9)]
    with torch.cuda.stream(stream):
        pev[0].record(stream)
        for k in range(8):
            lat.step(1)
            pev[k + 1].record(stream)
    torch.cuda.synchronize()
    per = [pev[k].elapsed_time(pev[k + 1]) for k in range(8)]

    # ------------------------------------------------------------ end to end
    import ctypes as C

    # The fields cross the host link in the handle's own precision: FP32
    # handles compute every per-node field in FP32 (FP64 only in the global
    # sums), so they take rho0 and return rho, u as FP32 (the _f32 calls).
    f32_io = prec == lbfe.FP32
    fdt = torch.float32 if f32_io else torch.float64
    fbytes = 4 if f32_io else 8
    e2e_rho0 = torch.from_numpy(rho0.astype(np.float32) if f32_io else rho0).pin_memory()
    res = {k: torch.empty((n_side, n_side), dtype=fdt).pin_memory() for k in ("rho", "ux", "uy")}
    init_fn = lbfe.lib().lb_init_fields_f32 if f32_io else lbfe.lib().lb_init_fields
    moments_fn = lbfe.lib().lb_moments_f32 if f32_io else lbfe.lib().lb_moments

    def end_to_end():
        lbfe._check(init_fn(lat._h, 0, C.c_void_p(e2e_rho0.data_ptr()), None, None, 0), lat._h)
        lat.step(args.steps)
        rc = moments_fn(lat._h, 0, C.c_void_p(res["rho"].data_ptr()), C.c_void_p(res["ux"].data_ptr()),
                        C.c_void_p(res["uy"].data_ptr()), None, 0)
        lbfe._check(rc, lat._h)

    for _ in range(2):  # warm-up: graphs for both buffer parities, first use of the pinned outputs
        end_to_end()
    link = _host_link(e2e_rho0, res, stream)
    barrier()
    e2e_passes = 3
    t0 = time.perf_counter()
    for _ in range(e2e_passes):
        end_to_end()
    e2e_s = _max_over_ranks((time.perf_counter() - t0) / e2e_passes, ws, f"cuda:{local}")
    seg_rows, n_items, narrow = lat.worklist()
    lat.close()
    cs = _cs_variant(lbfe, inputs, n_side, prec, local, rank) if ws == 1 and args.scheme == "improved" and not args.walls else None
    extras = {}
    default_case = args.scheme == "improved" and not args.walls
    if ws == 1 and dtype == "f32" and not args.no_extras and default_case:
        # the other measured targets, outside the timed region, a few seconds each
        extras["batched"] = _batched_throughput(lbfe, steps=20, warmup=16)
        # the same batch down to 0.65 T_c with the averaged correction (one-column kernel)
        extras["batched_smooth_0p65"] = _batched_throughput(lbfe, steps=20, warmup=16, t_range=(0.65, 0.9),
                                                            scheme=lbfe.IMPROVED_SMOOTH, per_case=False)
        extras["improved_smooth"] = _smooth_variant(lbfe, inputs, n_side, local, rank)
        extras["step_stats"] = _step_stats_cost(lbfe, case, rho0_pin, local, steps=40)
        extras["fp64"] = _fp64_spinodal(lbfe, inputs, n_side, steps=5, warmup=3, local=local, rank=rank)
        extras["adjoint"] = _adjoint_check(lbfe, inputs, steps=200, window=20, ckpt=20)
        extras["small_lattices"] = _small_lattices(lbfe, inputs)

    if rank == 0:
        peak, src = _peaks()
        mean_ms = total_ms / args.steps  # the timed region's average launch
        achieved = BYTES_PER_NODE[dtype] * nodes / (mean_ms * 1e-3) / 1e9
        value = _job_mlups(ws, nodes, args.steps, total_ms)
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD.replace(f"{N_SIDE}x{N_SIDE}", f"{n_side}x{n_side}").replace(
                           "FP32 deviation storage", "FP32 deviation storage" if dtype == "f32" else "FP64").replace(
                           "improved scheme", SCHEMES[args.scheme][1]).replace(
                           "periodic", "between no-slip walls at rest (y), periodic in x" if args.walls else "periodic"),
                       "nx": n_side, "ny": n_side, "nodes_per_gpu": nodes,
                       "parallelism": f"replicas{ws}" if ws > 1 else "single",
                       "l2": f"populations {BYTES_PER_NODE[dtype] * nodes / 1e9:.2f} GB per step vs 129 MB L2 "
                             "(no flush)",
                       "stable": stable,
                       "timed_call": f"one lb_step({args.steps}) (CUDA-graph replay of 8-step graphs)",
                       "graph_capture_steps_after_warmup": capture_steps,
                       "host_cores": host_cpus or "unbound (no sysfs topology)",
                       "vs_named_config": "vdW set of Sec. IV at 0.8 T_c instead of CS (a=1, b=4) at 0.7 T_c: "
                                          "the CS set's interface is 0.14 nodes wide and blows up within a few "
                                          "steps, and the improved scheme's vapour at 0.7 T_c is linearly "
                                          "unstable with the Eq. 17 discretisation of d(phi u); the CS kernel's "
                                          "throughput on a stable CS case is under eos_cs",
                       "worklist": {"segment_rows": {0: "slot share", -1: "slot share, filled", -2: "slot share, 2 waves", -3: "slot share, 4 waves"}.get(seg_rows, seg_rows), "items": n_items,
                                    "narrow_blocks": narrow}},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                         "traffic": _profiled_traffic(n_side) if dtype == "f32" and default_case else None,
                         "peak_source": src, "bytes_per_node": BYTES_PER_NODE[dtype],
                         "kernel_ms_mean": round(mean_ms, 4),
                         "single_launch_ms": {"min": round(min(per), 4), "max": round(max(per), 4),
                                              "note": "8 lb_step(1) calls after the timed region"}}
            if dtype == "f32" else _fp64_roofline(nodes, mean_ms, achieved / peak),
            "clocks": clk,
            "e2e": {"value": round(_job_mlups(ws, nodes, args.steps, e2e_s * 1e3), 1), "unit": "MLUPS",
                    "h2d_bytes_per_step": int(fbytes * nodes / args.steps),
                    "d2h_bytes_per_step": int(3 * fbytes * nodes / args.steps),
                    "includes": f"lb_init_fields{'_f32' if f32_io else ''} from pinned host rho0 (validated on the "
                                f"device), one lb_step(K) call, lb_moments{'_f32' if f32_io else ''} of rho, ux, uy "
                                "to pinned host; mean of 3 passes after 2 warm-up passes",
                    "field_dtype": "f32" if f32_io else "f64",
                    "host_link_bytes_per_pass": int(fbytes * nodes + 3 * fbytes * nodes), "host_link": link},
            "gpu_launches": args.steps,
        }
        if cs is not None:
            line["eos_cs"] = cs
        line.update(extras)
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(args.cpu_steps)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def batched_cases(lbfe, n_cases: int = 256, seed: int = 7, t_range=(0.8, 0.9), scheme=None):
    """The uneven batch: square periodic droplets, side uniform over the
    multiples of 4 in [32, 512], T/T_c ~ U[0.8, 0.9], kappa ~ U[0.01, 0.03],
    tau ~ U[0.8, 1.0], radius ~ U[0.15, 0.3] x side; improved scheme, BGK, vdW.
    t_range and scheme (default the improved scheme) select the variant run
    with the averaged correction down to 0.65 T_c."""
    import numpy as np

    from paper_2008_01473_gb300 import inputs

    rng = np.random.default_rng(seed)
    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    cases, rhos = [], []
    for i in range(n_cases):
        side = 4 * int(rng.integers(8, 129))
        t = rng.uniform(*t_range)
        kappa = rng.uniform(0.01, 0.03)
        tau = rng.uniform(0.8, 1.0)
        frac = rng.uniform(0.15, 0.3)
        T = t * tc
        rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], T)
        cases.append(lbfe.Case(nx=side, ny=side, scheme=lbfe.IMPROVED if scheme is None else scheme,
                               collision=lbfe.BGK, eos=lbfe.VDW, T=T, kappa=kappa, tau_v=tau, **VDW))
        rhos.append(inputs.droplet(side, side, frac * side, rl, rg, seed=seed, case=i))
    return cases, rhos


def _vdw_p(rho, T):
    """van der Waals pressure of Eq. 30's free energy, for the diagnostics."""
    return rho * VDW["R"] * T / (1.0 - VDW["b"] * rho) - VDW["a"] * rho * rho


def _batched_accuracy(lbfe, cases, rhos, steps):
    """Droplet diagnostics of a sub-batch run in FP32 against the same cases
    run in FP64 (whose step is checked against the FP64 oracle by the GPU
    tests) for the same number of steps: pressure jump p(rho_in) -
    p(rho_out) (centre disc of radius r0/4, corner squares of side L/8),
    equimolar radius and max |u|; both runs' densities also against the
    Young-Laplace prediction of Eq. 32 (host surface tension and inversion).
    Returns the worst relative errors and the largest spurious currents."""
    import numpy as np

    lats = {}
    for prec in (lbfe.FP32, lbfe.FP64):
        lat = lbfe.Lattice(cases, precision=prec)
        for i, r in enumerate(rhos):
            lat.init_fields(i, r)
        lat.step(steps)
        lats[prec] = lat
    err_dp, err_r, u = 0.0, 0.0, {}
    eq32 = {lbfe.FP32: [0.0, 0.0], lbfe.FP64: [0.0, 0.0]}  # worst |rho / rho_Eq.32 - 1|: gas, liquid
    for prec, lat in lats.items():  # max |u| of every case, reduced on the GPU
        u[prec] = float(lat.reductions()[0][:, 2].max())
    for i, c in enumerate(cases):
        L = c.nx
        s = L // 8
        dp, req = {}, {}
        for prec, lat in lats.items():
            # GPU FP64 window means: centre disc, the four corner squares (one
            # periodic square of side 2s around the corner node), whole lattice
            rin, rout, rbar = lat.window_means(i, [("disc", L / 2, L / 2, 0.25 * _batched_r0(rhos[i])),
                                                   ("rect", L - s, L - s, 2 * s, 2 * s), ("rect", 0, 0, L, L)])
            dp[prec] = _vdw_p(rin, c.T) - _vdw_p(rout, c.T)
            req[prec] = np.sqrt((rbar - rout) * L * L / (np.pi * (rin - rout)))
            sig = lbfe.surface_tension(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], c.T, c.kappa)
            g_th, l_th = lbfe.young_laplace(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], c.T, sig, req[prec])
            eq32[prec][0] = max(eq32[prec][0], abs(rout / g_th - 1))
            eq32[prec][1] = max(eq32[prec][1], abs(rin / l_th - 1))
        err_dp = max(err_dp, abs(dp[lbfe.FP32] / dp[lbfe.FP64] - 1))
        err_r = max(err_r, abs(req[lbfe.FP32] / req[lbfe.FP64] - 1))
    for lat in lats.values():
        lat.close()
    return {"cases": len(cases), "steps": steps, "max_rel_err_pressure_jump": err_dp,
            "max_rel_err_equimolar_radius": err_r, "max_u_fp32": u[lbfe.FP32], "max_u_fp64": u[lbfe.FP64],
            "vs_eq32_theory": {"fp32_gas": eq32[lbfe.FP32][0], "fp32_liquid": eq32[lbfe.FP32][1],
                               "fp64_gas": eq32[lbfe.FP64][0], "fp64_liquid": eq32[lbfe.FP64][1]}}


def _batched_r0(rho0):
    """Initial droplet radius from the tanh profile: the half-density
    crossing along the centre row."""
    import numpy as np

    L = rho0.shape[0]
    row = rho0[L // 2, L // 2:]
    mid = 0.5 * (row.max() + row.min())
    return float(np.argmax(row < mid))


def _warm(lat, warmup: int):
    """warmup steps, then 8 more if they did not capture the 8-step CUDA graph
    of the buffer parity that the timed steps start from (lb_step captures
    the graph of its starting parity on its first call of 8 steps or more)"""
    lat.step(warmup)
    if warmup < 8 or warmup % 2:
        lat.step(8)


def _batched_throughput(lbfe, steps: int, warmup: int, t_range=(0.8, 0.9), scheme=None,
                        per_case: bool = True) -> dict:
    """The uneven 256-case batch in one handle (one launch per step) and with
    one handle per case (one launch per case per step): MLUPS of each, CUDA
    events on the handles' stream around `steps` steps after `warmup`."""
    import torch

    cases, rhos = batched_cases(lbfe, t_range=t_range, scheme=scheme)
    nodes = sum(c.nx * c.ny for c in cases)
    lat = lbfe.Lattice(cases, precision=lbfe.FP32)
    for i, r in enumerate(rhos):
        lat.init_fields(i, r)
    _warm(lat, warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1)
    _, st = lat.reductions()
    seg_rows, n_items, narrow = lat.worklist()
    lat.close()
    res = {"value": round(nodes * steps / (batched_ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "steps": steps,
           "ms_per_step": round(batched_ms / steps, 4), "n_cases": len(cases), "nodes": nodes,
           "stable_cases": int((st == 0).sum()), "t_over_tc": list(t_range),
           "worklist": {"segment_rows": {0: "slot share", -1: "slot share, filled", -2: "slot share, 2 waves", -3: "slot share, 4 waves"}.get(seg_rows, seg_rows),
                        "items": n_items, "narrow_blocks": narrow},
           "roofline": {"bound": "hbm", "achieved": round(72 * nodes / (batched_ms / steps * 1e-3) / 1e9, 1),
                        "peak": _peaks()[0], "unit": "GB/s",
                        "frac": round(72 * nodes / (batched_ms / steps * 1e-3) / 1e9 / _peaks()[0], 4)}}
    if not per_case:
        return res
    lats = []
    for c, r in zip(cases, rhos):
        l1 = lbfe.Lattice([c], precision=lbfe.FP32)
        l1.init_fields(0, r)
        _warm(l1, warmup)
        lats.append(l1)
    torch.cuda.synchronize()
    e0.record(lats[0].stream)
    for l1 in lats:
        l1.step(steps)
    e1.record(lats[0].stream)
    torch.cuda.synchronize()
    per_case_ms = e0.elapsed_time(e1)
    for l1 in lats:
        l1.close()
    res["per_case_launches"] = {"value": round(nodes * steps / (per_case_ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                                "ms_per_step": round(per_case_ms / steps, 4)}
    return res


def _step_stats_cost(lbfe, case, rho0_pin, local: int, steps: int) -> dict:
    """The default workload with the per-step statistics attached (mass, kinetic
    energy and max |u| fused into every step) against the same steps without:
    MLUPS of each (lb_step(steps) between CUDA events, best of 3) and the
    recorded mass of the last state against lb_reductions of that state."""
    import torch

    lat = lbfe.Lattice([case], precision=lbfe.FP32, device=f"cuda:{local}")
    lat.init_fields(0, rho0_pin)
    lat.step(16)
    nodes = case.nx * case.ny

    def timed():
        best = 1e30
        with torch.cuda.stream(lat.stream):
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(lat.stream)
                lat.step(steps)
                e1.record(lat.stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
        return nodes * steps / (best * 1e-3) / 1e6

    off = timed()
    lat.attach_step_stats(4 * steps)
    lat.step(16)
    on = timed()
    out, _ = lat.reductions()  # the current state, which the next step records
    lat.step(1)
    first, rec = lat.step_stats(0)
    lat.close()
    return {"value": round(on, 1), "unit": "MLUPS", "without_stats": round(off, 1),
            "cost": round(1.0 - on / off, 4), "steps": steps,
            "recorded_states": int(rec.shape[0]), "first_recorded_state": int(first),
            "last_state_vs_reductions": {"mass_rel": float(abs(rec[-1, 0] / out[0, 0] - 1.0)),
                                         "ke_rel": float(abs(rec[-1, 1] / out[0, 1] - 1.0)),
                                         "umax_rel": float(abs(rec[-1, 2] / out[0, 2] - 1.0))}}


def _small_lattices(lbfe, inputs, steps: int = 400) -> dict:
    """Launch-bound workloads that live in L2: the sweep's 16 periodic
    1024 x 8 strips (improved scheme, BGK tau 1, vdW at T/T_c 0.95 ... 0.75,
    131,072 nodes) in FP32 and FP64, the same strips with the averaged
    correction at T/T_c 0.95 ... 0.65 in FP32, and one 40 x 33 FP64 droplet, each timed
    over `steps` steps with one launch per step (8-step graph replay), the
    strips also with the row kernel off (the sliding-window kernels), and
    with the persistent launch (one cooperative launch for the steps); MLUPS
    and microseconds per step."""
    import os

    import numpy as np
    import torch

    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    strips, strip_rho = [], []
    for t in np.linspace(0.95, 0.75, 16):
        rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], t * tc)
        strips.append(lbfe.Case(nx=1024, ny=8, scheme=lbfe.IMPROVED, collision=lbfe.BGK, eos=lbfe.VDW, T=t * tc,
                                kappa=0.02, tau_v=1.0, **VDW))
        strip_rho.append(inputs.slab(1024, 8, rl, rg))
    smooth, smooth_rho = [], []
    for t in np.linspace(0.95, 0.65, 16):
        rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], t * tc)
        smooth.append(lbfe.Case(nx=1024, ny=8, scheme=lbfe.IMPROVED_SMOOTH, collision=lbfe.BGK, eos=lbfe.VDW,
                                T=t * tc, kappa=0.02, tau_v=1.0, **VDW))
        smooth_rho.append(inputs.slab(1024, 8, rl, rg))
    rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], 0.8 * tc)
    drop = [lbfe.Case(nx=40, ny=33, scheme=lbfe.IMPROVED, collision=lbfe.MRT, eos=lbfe.VDW, T=0.8 * tc, kappa=0.02,
                      tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1, **VDW)]
    drop_rho = [inputs.droplet(40, 33, 9.0, rl, rg)]
    out = {}
    for name, cases, rhos, prec in (("sweep_strips_fp32", strips, strip_rho, lbfe.FP32),
                                    ("sweep_strips_fp64", strips, strip_rho, lbfe.FP64),
                                    ("sweep_strips_smooth_fp32", smooth, smooth_rho, lbfe.FP32),
                                    ("droplet_40x33_fp64", drop, drop_rho, lbfe.FP64)):
        nodes = sum(c.nx * c.ny for c in cases)
        res = {"nodes": nodes}
        runs = [(0, "graph_replay", "1"), (1, "persistent", "1")]
        if cases[0].ny <= 16:
            runs.insert(1, (0, "sliding_window", "0"))
        for mode, key, rows in runs:
            old = os.environ.get("LBFE_ROWS")
            os.environ["LBFE_ROWS"] = rows  # read when the handle is made
            try:
                lat = lbfe.Lattice(cases, precision=prec)
            finally:
                if old is None:
                    os.environ.pop("LBFE_ROWS")
                else:
                    os.environ["LBFE_ROWS"] = old
            lat.launch_mode(mode)
            for i, r in enumerate(rhos):
                lat.init_fields(i, r)
            lat.step(64)  # autotune, graph capture, kernel loads
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(lat.stream)
            lat.step(steps)
            e1.record(lat.stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            _, st = lat.reductions()
            lat.close()
            res[key] = {"MLUPS": round(nodes * steps / (ms * 1e-3) / 1e6, 1),
                        "us_per_step": round(ms * 1e3 / steps, 2), "stable": bool((st == 0).all())}
        res["population_bytes_both_buffers"] = (72 if prec == lbfe.FP32 else 144) * nodes
        res["gain"] = round(res["persistent"]["MLUPS"] / res["graph_replay"]["MLUPS"], 3)
        if "sliding_window" in res:
            res["row_kernel_gain"] = round(res["graph_replay"]["MLUPS"] / res["sliding_window"]["MLUPS"], 3)
        out[name] = res
    out["note"] = ("L2-resident (both population buffers far below the 129 MB L2): bound by launch latency and "
                   "the latency of a step's stages, not by HBM; the strips (ny 8) run the row kernel under graph "
                   "replay, the packed (FP32) or one-column (FP64) sliding-window kernel with it off, and the "
                   "one-column kernel when persistent; the droplet runs the one-column kernel")
    return out


def run_batched(args):
    """Throughput of the uneven batch in one handle (one launch per step)
    against one handle per case (one launch per case per step)."""
    import torch

    from paper_2008_01473_gb300 import build, lbfe

    build.build()
    torch.cuda.set_device(0)
    cases, rhos = batched_cases(lbfe)
    b = _batched_throughput(lbfe, args.steps, args.warmup)
    acc = _batched_accuracy(lbfe, cases[::8], rhos[::8], args.accuracy_steps) if args.accuracy_steps else None
    line = {"metric": METRIC, "value": b["value"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched uneven droplets: " + (batched_cases.__doc__ or "").split(":")[1].strip(),
                       "n_cases": b["n_cases"], "nodes": b["nodes"], "stable_cases": b["stable_cases"],
                       "worklist": b["worklist"]},
            "fp32_vs_fp64": acc,  # every 8th case of the batch
            "per_case_launches": b["per_case_launches"], "roofline": b["roofline"]}
    if not args.no_cpu:
        import numpy as np

        # 16 seeded cases spanning the size range (evenly spaced ranks by side)
        order = np.argsort([c.nx for c in cases], kind="stable")
        pick = [int(order[k]) for k in np.linspace(0, len(cases) - 1, 16).round().astype(int)]
        line["cpu_baseline"] = _oracle_pool_baseline([cases[i] for i in pick], [rhos[i] for i in pick], 100,
                                                     "16 cases of the batch spanning its sizes")
    print(json.dumps(line), flush=True)


def _adjoint_check(lbfe, inputs, steps: int, window: int, ckpt: int, n: int = 256) -> dict:
    """Gradient of the droplet loss (n^2 periodic droplet of radius n/4, vdW
    at T = 0.8 T_c, kappa 0.02, BGK tau 0.8, FP64): L = sum of |u|^2 over the
    last `window` steps of `steps` + (rho_g - rho_g^Maxwell(T))^2, rho_g the
    mean density over the four corner squares of side n/8. Times the
    lb_adjoint_step sweep (checkpoints every `ckpt` steps) and checks dL/dkappa
    and dL/d(T/T_c) against central differences (h = 3e-6 relative) of the
    GPU forward loss; also the same gradient from an FP32 handle."""
    import numpy as np
    import torch

    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    t_red = 0.8
    rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], t_red * tc)
    rho0 = inputs.droplet(n, n, n / 4.0, rl, rg)
    m = n // 8
    w = np.zeros((n, n))
    for ys in (slice(0, m), slice(n - m, n)):
        for xs in (slice(0, m), slice(n - m, n)):
            w[ys, xs] = 1.0
    w /= w.sum()

    def case(kappa, t):
        return lbfe.Case(nx=n, ny=n, scheme=lbfe.IMPROVED, collision=lbfe.BGK, eos=lbfe.VDW, T=t * tc, kappa=kappa,
                         tau_v=0.8, **VDW)

    def forward_loss(kappa, t):
        lat = lbfe.Lattice([case(kappa, t)], precision=lbfe.FP64)
        lat.init_fields(0, rho0)
        lat.step(steps - window)
        lu = 0.0
        for k in range(window + 1):
            mo = lat.moments(0)
            lu += float((mo["ux"] ** 2 + mo["uy"] ** 2).sum())
            if k < window:
                lat.step(1)
        g_m = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], t * tc)[0]
        rho_g = float((w * mo["rho"]).sum())
        lat.close()
        return lu + (rho_g - g_m) ** 2, rho_g, g_m

    kappa = 0.02
    L0, rho_g, gm = forward_loss(kappa, t_red)
    s_final = 2.0 * (rho_g - gm) * w
    out = {}
    for prec in (lbfe.FP64, lbfe.FP32):
        lat = lbfe.Lattice([case(kappa, t_red)], precision=prec)
        lat.adjoint(0, rho0, 8, 0, None, 0)  # warm-up: module load, first launches
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out[prec] = lat.adjoint(0, rho0, steps, steps - window, s_final, ckpt) + (time.perf_counter() - t0,)
        lat.close()
    La, g_rho0, gk, gT, t_adj = out[lbfe.FP64]
    La32, g32, gk32, gT32, t_adj32 = out[lbfe.FP32]
    fp32 = {"adjoint_seconds": round(t_adj32, 3), "rel_diff_loss": abs(La32 / La - 1),
            "rel_diff_dL_dkappa": abs(gk32 / gk - 1), "rel_diff_dL_dT_trajectory": abs(gT32 / gT - 1),
            "rel_diff_dL_drho0_max": float(np.abs(g32 - g_rho0).max() / np.abs(g_rho0).max())}
    # dL/dT: trajectory term from the adjoint, plus the explicit -2 (rho_g - rho_g^M) d rho_g^M / dT
    hT = 1e-6 * tc
    dgm = (lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], t_red * tc + hT)[0]
           - lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], t_red * tc - hT)[0]) / (2 * hT)
    dL_dt = tc * (gT - 2.0 * (rho_g - gm) * dgm)
    # h = 1e-4 relative leaves an O(h^2) truncation error of 3e-4 in dL/dT on
    # the 2000-step horizon (the loss is strongly curved in T); 3e-6 brings it
    # below 1e-6
    hk, ht = 3e-6 * kappa, 3e-6 * t_red
    fd_k = (forward_loss(kappa + hk, t_red)[0] - forward_loss(kappa - hk, t_red)[0]) / (2 * hk)
    fd_t = (forward_loss(kappa, t_red + ht)[0] - forward_loss(kappa, t_red - ht)[0]) / (2 * ht)
    return {"workload": f"{n}x{n} droplet r={n // 4}, vdW 0.8 T_c, BGK tau 0.8, {steps} steps, |u|^2 over the last "
                        f"{window}, checkpoints every {ckpt}, FP64",
            "loss": L0, "rel_diff_loss_adjoint_vs_forward": abs(La / L0 - 1), "adjoint_seconds": round(t_adj, 3),
            "adjoint_node_steps_per_s": round(n * n * steps / t_adj, 1),
            "dL_dkappa": {"adjoint": gk, "fd": fd_k, "rel_err": abs(gk - fd_k) / abs(fd_k)},
            "dL_dT_over_Tc": {"adjoint": dL_dt, "fd": fd_t, "rel_err": abs(dL_dt - fd_t) / abs(fd_t)},
            "fd_rel_step": 3e-6,
            "dL_drho0_norm": float(np.sqrt((g_rho0 ** 2).sum())), "rho_g": rho_g, "rho_g_maxwell": gm,
            "fp32_adjoint_vs_fp64": fp32}


def run_adjoint(args):
    """Differentiation workload: the 256^2 droplet of radius 64, 2000 steps
    (--adjoint-steps) checkpointed every 100, loss over the last 100 steps
    (_adjoint_check)."""
    from paper_2008_01473_gb300 import build, inputs, lbfe

    build.build()
    n = args.adjoint_steps
    line = {"metric": "adjoint gradient (lb_adjoint_step) vs central differences", "steps": n,
            **_adjoint_check(lbfe, inputs, steps=n, window=min(100, n // 2), ckpt=min(100, n // 2))}
    print(json.dumps(line), flush=True)


def _fp64_spinodal(lbfe, inputs, n_side: int, steps: int, warmup: int, local: int, rank: int) -> dict:
    """The same spinodal lattice with FP64 populations and arithmetic: MLUPS
    and the FP64-pipe roofline of the one-column step kernel."""
    import torch

    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    T = T_RED * tc
    rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], T)
    case = lbfe.Case(nx=n_side, ny=n_side, scheme=lbfe.IMPROVED, collision=lbfe.MRT, eos=lbfe.VDW, T=T,
                     kappa=0.02, tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1, **VDW)
    lat = lbfe.Lattice([case], precision=lbfe.FP64, device=f"cuda:{local}")
    lat.init_fields(0, inputs.spinodal(n_side, n_side, 0.5 * (rg + rl), 0.01, seed=1 + rank))
    lat.step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    _, st = lat.reductions()
    lat.close()
    nodes = n_side * n_side
    peak, _ = _peaks()
    return {"value": round(nodes / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "steps": steps, "ms_per_step": round(ms, 4),
            "workload": f"spinodal {n_side}x{n_side}, improved, MRT, vdW at T/Tc={T_RED}, FP64 populations",
            "stable": bool(st[0] == 0),
            "roofline": _fp64_roofline(nodes, ms, 144 * nodes / (ms * 1e-3) / 1e9 / peak)}


def _droplet_shape(rho, rho_g):
    """Centroid (periodic in x) and inertia-tensor aspect ratio of the
    density excess over rho_g."""
    import numpy as np

    ny, nx = rho.shape
    w = np.clip(rho - rho_g, 0.0, None)
    y, x = np.mgrid[0:ny, 0:nx]
    k = 2 * np.pi / nx
    cx = (np.angle((w * np.exp(1j * k * x)).sum()) / k) % nx
    cy = (w * y).sum() / w.sum()
    dx, dy = (x - cx + nx / 2) % nx - nx / 2, y - cy
    ev = np.linalg.eigvalsh([[(w * dx * dx).sum(), (w * dx * dy).sum()], [(w * dx * dy).sum(), (w * dy * dy).sum()]])
    return float(cx), float(cy), float(np.sqrt(ev[1] / ev[0]))


def run_galilean(args):
    """Moving droplet between sliding walls (Sec. IV C, Fig. 6): 120 x 120,
    droplet of radius 25 at the centre, walls at y = -1/2 and 119.5 moving at
    U = 0.1 from t = 0, constant kinematic viscosity 0.15, vdW at T = 0.7 T_c,
    BGK, FP64 populations; the improved scheme with the smoothed correction
    (LB_IMPROVED_SMOOTH), with the plain Eq. 17 correction (LB_IMPROVED) and
    the standard scheme; snapshots at 20,000, 40,000, 70,000 and 90,000 steps. Each
    scheme first settles the droplet for 10,000 steps between walls at rest;
    the settled density starts the run and its mean over the two wall rows is
    the wall state's density (the standard scheme's vapour is not at the
    Maxwell density)."""
    import torch

    from paper_2008_01473_gb300 import build, inputs, lbfe

    build.build()
    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    T = 0.7 * tc
    rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], T)
    L = 120
    rho0 = inputs.droplet(L, L, 25.0, rl, rg)
    out = {}
    for scheme, name in ((lbfe.IMPROVED_SMOOTH, "improved_smooth"), (lbfe.IMPROVED, "improved"),
                         (lbfe.STANDARD, "standard")):
        kw = dict(nx=L, ny=L, scheme=scheme, collision=lbfe.BGK, eos=lbfe.VDW, T=T, kappa=0.02, tau_v=1.0,
                  nu=0.15, walls=1, **VDW)
        lat = lbfe.Lattice([lbfe.Case(wall_u=0.0, rho_wall=rg, **kw)], precision=lbfe.FP64)
        lat.init_fields(0, rho0)
        lat.step(10000)
        _, st = lat.reductions()
        settled = lat.moments(0)["rho"]
        lat.close()
        if st[0] != 0:
            out[name] = {"stable": False, "unstable_while": "settling between walls at rest"}
            continue
        rw = float(0.5 * (settled[0].mean() + settled[-1].mean()))
        lat = lbfe.Lattice([lbfe.Case(wall_u=0.1, rho_wall=rw, **kw)], precision=lbfe.FP64)
        lat.init_fields(0, settled)
        snaps, done = [], 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for n in (20000, 40000, 70000, 90000):
            lat.step(n - done)
            done = n
            m = lat.moments(0)
            cx, cy, ar = _droplet_shape(m["rho"], rg)
            snaps.append({"step": n, "x_centroid": round(cx, 2), "y_centroid": round(cy, 3),
                          "aspect_ratio": round(ar, 5), "mean_ux": round(float(m["ux"].mean()), 5)})
        dt = time.perf_counter() - t0
        _, st = lat.reductions()
        lat.close()
        out[name] = {"rho_wall": round(rw, 5), "snapshots": snaps, "stable": bool(st[0] == 0),
                     "seconds": round(dt, 2)}
    print(json.dumps({"metric": "moving droplet between sliding walls (Galilean invariance)",
                      "workload": run_galilean.__doc__.split(";")[0].strip(), **out}), flush=True)


def run_sweep(args):
    """Coexistence sweep: 16 periodic 1024 x 8 strips with a liquid slab in the
    middle half (tanh edges of width 5), T/T_c evenly spaced from 0.95 down to
    0.75, vdW (a = 9/392, b = 2/21, kappa = 0.02), BGK tau = 1.0, all 16 in one
    handle; 50,000 steps; rho_g and rho_l (means over x < L/16 and |x - L/2| <
    L/16) against the Maxwell construction, for the improved scheme and the
    standard one with either force form, and for the improved scheme with the
    smoothed correction (LB_IMPROVED_SMOOTH) from 0.95 down to 0.65 T_c."""
    import numpy as np
    import torch

    from paper_2008_01473_gb300 import build, inputs, lbfe

    build.build()
    prec = lbfe.FP64 if args.precision == "fp64" else lbfe.FP32
    tc, _ = lbfe.critical(lbfe.VDW, **VDW)
    ts = np.linspace(0.95, 0.75, 16)
    nx, ny, steps = 1024, 8, args.steps if args.steps > 1000 else 50000
    out = {}
    first = None
    for scheme, name, ts in ((lbfe.IMPROVED, "improved", ts), (lbfe.STANDARD, "standard", ts),
                             (lbfe.STANDARD_PT, "standard_pressure_tensor", ts),
                             (lbfe.IMPROVED_SMOOTH, "improved_smooth", np.linspace(0.95, 0.65, 16))):
        cases, rhos, mx = [], [], []
        for t in ts:
            rg, rl = lbfe.maxwell(lbfe.VDW, VDW["a"], VDW["b"], VDW["R"], t * tc)
            cases.append(lbfe.Case(nx=nx, ny=ny, scheme=scheme, collision=lbfe.BGK, eos=lbfe.VDW, T=t * tc,
                                   kappa=0.02, tau_v=1.0, **VDW))
            rhos.append(inputs.slab(nx, ny, rl, rg))
            mx.append((rg, rl))
        first = first or (cases, rhos)
        lat = lbfe.Lattice(cases, precision=prec)
        for i, r in enumerate(rhos):
            lat.init_fields(i, r)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(lat.stream)
        lat.step(steps)
        e1.record(lat.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        _, st = lat.reductions()
        errs = []
        for i, (rg, rl) in enumerate(mx):
            # gas window x < L/16, liquid window |x - L/2| < L/16: GPU FP64 means
            g, l = lat.window_means(i, [("rect", 0, 0, nx // 16, ny), ("rect", nx // 2 - nx // 16, 0, nx // 8, ny)])
            errs.append((float(ts[i]), float(g / rg - 1), float(l / rl - 1)))
        lat.close()
        out[name] = {"mlups": round(len(cases) * nx * ny * steps / (ms * 1e-3) / 1e6, 1),
                     "max_rel_err_rho_g": max(abs(e[1]) for e in errs),
                     "max_rel_err_rho_l": max(abs(e[2]) for e in errs),
                     "stable_cases": int((st == 0).sum()),
                     "per_T": [[round(t, 4), f"{eg:.2e}", f"{el:.2e}"] for t, eg, el in errs]}
    line = {"metric": "coexistence sweep vs Maxwell", "workload": run_sweep.__doc__.split(";")[0].strip(),
            "dtype": "f64" if prec == lbfe.FP64 else "f32", "steps": steps, **out}
    if not args.no_cpu:
        line["cpu_baseline"] = _oracle_pool_baseline(*first, 2000, "the 16 improved-scheme strips")
    print(json.dumps(line), flush=True)


def _oracle_case_steps(args):
    """One oracle run (pool worker): a case given as keyword fields and its
    initial density, stepped `steps` times; returns (node updates, seconds,
    worker pid)."""
    kw, rho0, steps = args
    import oracle as O

    oc = O.Case(**kw)
    f = O.init(oc, rho0)
    t0 = time.perf_counter()
    done = O.step(oc, f, steps)
    return oc.nx * oc.ny * done, time.perf_counter() - t0, os.getpid()


def _oracle_pool_baseline(cases, rhos, steps, what):
    """The FP64 oracle, as it stands, on a bounded sample of a batched
    workload, one case per process over the host's cores (a spawn pool):
    whole-sample node updates over the busiest process's stepping time
    (process start-up excluded)."""
    import multiprocessing as mp

    keys = ("nx", "ny", "scheme", "collision", "eos", "a", "b", "R", "T", "kappa", "tau_v", "tau_e", "tau_s",
            "tau_q", "nu")
    jobs = [({k: getattr(c, k) for k in keys}, r, steps) for c, r in zip(cases, rhos)]
    cores = min(len(jobs), len(os.sched_getaffinity(0)))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_case_steps, jobs, chunksize=1)
    per_proc = {}
    for _, sec, pid in res:  # processes run side by side; each runs its cases one after another
        per_proc[pid] = per_proc.get(pid, 0.0) + sec
    span = max(per_proc.values())
    nodes = sum(r[0] for r in res)
    return {"value": round(nodes / span / 1e6, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{what}, {steps} steps each, cases spread over {cores} processes, busiest {span:.1f} s"}


def _oracle_sample():
    import oracle as O
    from oracle import thermo
    from paper_2008_01473_gb300 import inputs

    e = thermo.vdw_paper()
    T, rg, rl = thermo.maxwell_reduced(e, T_RED)
    oc = O.Case(nx=SAMPLE_SIDE, ny=SAMPLE_SIDE, scheme=O.IMPROVED, collision=O.MRT, eos=O.VDW, a=e.a, b=e.b,
                T=T, kappa=0.02, tau_v=0.8, tau_e=1.0, tau_s=1.0, tau_q=1.1)
    f = O.init(oc, inputs.spinodal(SAMPLE_SIDE, SAMPLE_SIDE, 0.5 * (rg + rl), 0.01, seed=1))
    return O, oc, f


def cpu_baseline(steps: int) -> dict:
    """The FP64 oracle (single-threaded C) on a bounded sample of the workload."""
    O, oc, f = _oracle_sample()
    O.step(oc, f, 1)
    t0 = time.perf_counter()
    O.step(oc, f, steps)
    dt = time.perf_counter() - t0
    return {"value": round(SAMPLE_SIDE * SAMPLE_SIDE * steps / dt / 1e6, 3), "unit": "MLUPS", "cores": 1,
            "kind": "oracle", "sample": f"{SAMPLE_SIDE}x{SAMPLE_SIDE} sub-lattice of the same workload, "
                                        f"{steps} steps, FP64 single thread, {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    O, oc, f = _oracle_sample()
    O.step(oc, f, max(args.warmup, 1))
    t0 = time.perf_counter()
    O.step(oc, f, args.steps)
    dt = time.perf_counter() - t0
    v = SAMPLE_SIDE * SAMPLE_SIDE * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("FP32 deviation storage", "FP64 oracle")
                       + f"; each step a {SAMPLE_SIDE}x{SAMPLE_SIDE} sample", "nx": SAMPLE_SIDE, "ny": SAMPLE_SIDE},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": f"{SAMPLE_SIDE}x{SAMPLE_SIDE} sub-lattice, {args.steps} steps"},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=450)
    ap.add_argument("--adjoint-steps", type=int, default=2000, help="horizon of --workload adjoint")
    ap.add_argument("--accuracy-steps", type=int, default=10000,
                    help="batched workload: steps of the FP32-vs-FP64 droplet check (0 skips it)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the batched, fp64 and adjoint sub-measurements")
    ap.add_argument("--side", type=int, default=N_SIDE, help="lattice side (profiling of smaller cases)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--walls", action="store_true",
                    help="spinodal workload: no-slip walls at rest across y (the walled kernels)")
    ap.add_argument("--scheme", default="improved", choices=list(SCHEMES),
                    help="spinodal workload: the scheme of the lattice (the sub-measurements run with improved only)")
    ap.add_argument("--workload", default="spinodal", choices=["spinodal", "batched", "adjoint", "sweep", "galilean"],
                    help="spinodal: the 4096^2 lattice (default); batched: 256 uneven droplets; "
                         "adjoint: gradient of the 256^2 droplet loss with a finite-difference check; "
                         "sweep: 16 flat-interface strips against the Maxwell construction; "
                         "galilean: a droplet carried between sliding walls")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "galilean":
        run_galilean(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

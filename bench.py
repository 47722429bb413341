#!/usr/bin/env python
"""Throughput benchmark of the free-surface LBM step on GB300.

Workload: 3D dam break 512 x 256 x 256 (33.5 M cells), walls on all faces,
liquid column x < 128, z < 192 at rest with hydrostatic density,
g = 1e-5 along -z, FSL rule, seeded fill perturbation 1e-3 on the interface
layer, tau = 0.53 with the magic parameter Lambda = 0.005: droplets thrown
off the splash fall freely (the free-surface model has no gas drag) and at
tau = 0.51 and 0.52 a run loses stability between 4000 and 9000 steps,
depending on Lambda and on rounding; tau = 0.53 with Lambda = 0.005 runs
13000 steps in FP32 and FP16.  The headline form is FP32 populations with FP64
interface mass and mass balance; FP64 and FP16-storage forms are measured in
the same run.  A "step" is one full time step: stream-collide, free-surface
reconstruction, mass exchange, mass balance and cell conversions.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
instead, on a bounded sample of the same workload.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FSLBM MLUPS at 1 GB300 (FP32/FP16-store vs FP64 plain), % HBM roofline, adjoint/fwd"
WORKLOAD = "dam_break_512x256x256_fsl"
DIMS = (512, 256, 256)
COL = (128, 192)
TAU, MAGIC = 0.53, 0.005
# kernels of one step: k_reset, k_segments, k_bulk, k_geom (FSL or surface
# tension only), k_iface, 2 x k_reduce, 5 conversion kernels
STORE_BYTES = {"f64": 8, "f32": 4, "f16": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--spinup", type=int, default=5000,
                    help="untimed steps from the initial column before the warm-up, so that the timed window "
                         "(steps spinup + warmup + 1 to spinup + warmup + steps) covers the front, the splash "
                         "and the spray of the dam break (its interface and conversions), not its start")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="f32,f64,f16", help="precision forms; the first is the headline")
    ap.add_argument("--form-steps", type=int, default=2000, help="timed steps of the non-headline forms")
    ap.add_argument("--as-written-steps", type=int, default=2000,
                    help="timed steps of the dam break at tau = 0.51, Lambda = 3/16 from its initial state "
                         "(0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end run from the initial state (default: --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the differentiation workload")
    ap.add_argument("--save-state", default=None, metavar="PREFIX",
                    help="run --save-after steps of the workload (first form), save the state, exit")
    ap.add_argument("--save-after", type=int, default=8000)
    ap.add_argument("--load-state", default=None, metavar="PREFIX",
                    help="time the first form from a state saved by --save-state (a late phase of the run)")
    ap.add_argument("--small", action="store_true", help="development size (128 x 64 x 64)")
    ap.add_argument("--dims", default=None, help="nx,ny,nz of a scaled dam break (profiling)")
    ap.add_argument("--tau", type=float, default=TAU)
    ap.add_argument("--magic", type=float, default=MAGIC)
    ap.add_argument("--rule", type=int, default=1, help="1 = FSL, 0 = FSK")
    ap.add_argument("--bulk-loads", default="pairs", choices=["plain", "async", "tma", "pairs"],
                    help="how the FP32/FP16 bulk kernel reaches its pulled values (pairs: two cells per lane, "
                         "packed FP32x2 collision; the fastest on GB300)")
    return ap.parse_args()


def dims_for(args):
    if args.dims:
        return tuple(int(v) for v in args.dims.split(","))
    return (128, 64, 64) if args.small else DIMS


def col_for(args):
    nx, ny, nz = dims_for(args)
    return (nx // 4, nz * 3 // 4)


def make_case(args):
    from paper_1409_5645_gb300 import cases
    nx, ny, nz = dims_for(args)
    cx, cz = col_for(args)
    return cases.dam_break(nx=nx, ny=ny, nz=nz, col_x=cx, col_z=cz, tau=args.tau, magic=args.magic,
                           rule=args.rule, bulk_loads=args.bulk_loads)


# ---------------------------------------------------------------------------
# distributed plumbing (independent replicas: one lattice per GPU)
# ---------------------------------------------------------------------------
def dist_setup(backend):
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class NvmlClocks:
    """SM clock, power and clock-event reasons sampled every millisecond by a
    host thread through NVML (read-only queries), so that a timed region of a
    few milliseconds still gets samples."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, gpu_index, period_s=0.001):
        import ctypes
        import threading
        self.ok = False
        try:
            self.L = ctypes.CDLL("libnvidia-ml.so.1")
            if self.L.nvmlInit_v2() != 0:
                return
            self.dev = ctypes.c_void_p()
            if self.L.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(self.dev)) != 0:
                return
            mx = ctypes.c_uint()
            self.L.nvmlDeviceGetMaxClockInfo(self.dev, 1, ctypes.byref(mx))
            self.max_mhz = float(mx.value)
        except (OSError, AttributeError):
            return
        self.ok = True
        self.samples, self.period = [], period_s
        self.stop_ev = threading.Event()
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        import ctypes
        clk, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        get_r = getattr(self.L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.L.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_ev.is_set():
            self.L.nvmlDeviceGetClockInfo(self.dev, 1, ctypes.byref(clk))
            self.L.nvmlDeviceGetPowerUsage(self.dev, ctypes.byref(pw))
            get_r(self.dev, ctypes.byref(rs))
            self.samples.append((float(clk.value), pw.value / 1000.0, int(rs.value)))
            time.sleep(self.period)

    def stop(self):
        if not self.ok:
            return None
        self.stop_ev.set()
        self.th.join(timeout=2)
        sm = [a for a, _, _ in self.samples]
        reasons = sorted({nm for _, _, r in self.samples for bit, nm in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sm), "power_w_median": statistics.median([p for _, p, _ in self.samples])
                if sm else None, "source": "NVML, 1 ms"}


class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


# ---------------------------------------------------------------------------
# measured peaks and the committed ncu traffic figure
# ---------------------------------------------------------------------------
def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha():
    """Hash of the bulk and interface kernels' code (comments and blank lines
    left out, so that a change of wording does not orphan a profile)."""
    h = hashlib.sha256()
    for f in ("fslbm_step.cu", "fslbm_step.cuh", "fslbm_staged.cu", "fslbm_pairs.cu", "fslbm_pull.cuh",
              "fslbm_dev.cuh"):
        text = open(os.path.join(ROOT, "paper_1409_5645_gb300", "csrc", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        code = [ln.split("//")[0].rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln.strip()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(form):
    """Per-launch DRAM bytes of k_bulk from the committed ncu summary, scaled
    to the full lattice; None if absent or taken on other kernel source."""
    path = os.path.join(ROOT, "profiles", f"k_bulk_dam_break_{form}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    val = re.search(r"traffic_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not sha or not val or sha.group(1) != kernel_source_sha():
        return None
    return float(val.group(1))


def fp64_counts_per_cell():
    """(FP64 operations with FMA = 2, FP64 instructions) per liquid-cell
    update of the FP64 bulk kernel, from the committed ncu instruction counts;
    None if absent or taken on other kernel source."""
    path = os.path.join(ROOT, "profiles", "k_bulk_dam_break_f64.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    fl = re.search(r"fp64_flops_per_liquid_cell:\s*([0-9.eE+]+)", text)
    ins = re.search(r"fp64_instructions_per_liquid_cell:\s*([0-9.eE+]+)", text)
    if not sha or not fl or not ins or sha.group(1) != kernel_source_sha():
        return None
    return float(fl.group(1)), float(ins.group(1))


# ---------------------------------------------------------------------------
# one precision form
# ---------------------------------------------------------------------------
def count_kinds(lat):
    import numpy as np
    from paper_1409_5645_gb300 import fslbm
    fl = lat.get(fslbm.FIELD_FLAGS)["flags"]
    return int(np.count_nonzero(fl == 1)), int(np.count_nonzero(fl == 2))


def save_state(lat, prefix):
    """Post-collision state of a lattice to prefix_{flags,f,m,phi}.npy (f as
    float32: the FP32 form's own values)."""
    import numpy as np
    from paper_1409_5645_gb300 import fslbm
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    st = lat.get(fslbm.FIELD_FLAGS | fslbm.FIELD_F | fslbm.FIELD_MASS | fslbm.FIELD_PHI, device=dev)
    np.save(prefix + "_flags.npy", st["flags"].cpu().numpy())
    np.save(prefix + "_f.npy", st["f"].float().cpu().numpy())
    np.save(prefix + "_m.npy", st["m"].cpu().numpy())
    np.save(prefix + "_phi.npy", st["phi"].cpu().numpy())


def load_state(lat, prefix, dev):
    import numpy as np
    import torch
    t = {k: torch.from_numpy(np.load(prefix + "_" + k + ".npy")).to(dev) for k in ("flags", "f", "m", "phi")}
    lat.set_state_post(t["flags"], t["f"].double(), t["m"], t["phi"])
    del t


def run_form(case, form, steps, warmup, ws, rank, local_rank, clocks=False, state=None, spinup=0, alone=False):
    """alone: after the timed steps, 3 + 10 more steps with every kernel in
    order on one stream (set_overlap(False)), timing the bulk kernel alone."""
    import torch
    from paper_1409_5645_gb300 import fslbm
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    lat = fslbm.Lattice(case["dims"], case["params"], precision=form, stream=stream.cuda_stream)
    if state:
        load_state(lat, state, dev)
    else:
        t = {k: torch.from_numpy(case[k]).to(dev) for k in ("flags", "rho", "u", "phi")}
        lat.init_equilibrium(t["flags"], t["rho"], t["u"], t["phi"])
        del t
    lat.step(spinup + warmup)
    lat.sync()
    M0, _ = lat.total_mass()
    nliq0, nifc0 = count_kinds(lat)
    lat.timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize(dev)
    ck = None
    if clocks:
        ck = NvmlClocks(local_rank)
        if not ck.ok:
            ck = Clocks(local_rank)
        time.sleep(0.01)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = ck.stop() if ck else None
    barrier(ws)
    ms = e0.elapsed_time(e1)
    groups, nt = lat.timing_read()
    lat.timing(False)
    lat.sync()
    M1, lost = lat.total_mass()
    nliq1, nifc1 = count_kinds(lat)
    groups_alone = None
    if alone:
        lat.set_overlap(False)
        lat.step(3)
        lat.timing(True)
        lat.step(10)
        groups_alone, _ = lat.timing_read()
        lat.timing(False)
        lat.set_overlap(True)
        lat.sync()
    out = dict(ms=ms, steps=steps, groups_ms=groups, groups_alone=groups_alone, timed_steps=nt, mass0=M0, mass1=M1,
               lost=lost,
               n_liquid=(nliq0 + nliq1) / 2, n_interface=(nifc0 + nifc1) / 2, clocks=clk,
               device_bytes=lat.device_bytes, t_end=lat.time, bulk_loads=lat.bulk_loads,
               launches_per_step=lat.launches_per_step)
    lat.close()
    torch.cuda.synchronize(dev)
    return out


def adjoint_run(form, steps=4000, K=200):
    """Differentiation workload: film 8 x 4 x 64, depth 40, objective the mean
    x-velocity of the interface cells after `steps` steps, checkpoints every K
    steps with recompute; forward and adjoint cost per step and peak memory."""
    from paper_1409_5645_gb300 import cases, fslbm
    lat = fslbm.Lattice.from_case(cases.adjoint_film(), precision=form)
    try:
        lat.adjoint_forward(steps, K)
        lat.adjoint_backward()
    except fslbm.FslbmError as e:
        lat.close()
        return {"steps": steps, "checkpoint_every": K, "error": str(e)}
    fwd, adj, peak = lat.adjoint_stats()
    lat.close()
    return {"steps": steps, "checkpoint_every": K, "fwd_ms_per_step": round(fwd, 5),
            "adj_ms_per_step": round(adj, 5), "adj_over_fwd": round(adj / fwd, 3) if fwd > 0 else None,
            "peak_bytes": int(peak)}


def adjoint_large(form, steps=400, K=40, dims=(256, 128, 128), peak=None, arith32=False):
    """Differentiation at scale: the dam break at 256 x 128 x 128 (4.2 M
    cells; cells fill, empty and appear inside the window, replayed by the
    adjoint), objective the mean x-velocity of the interface cells after
    `steps` steps, checkpoints every K steps.  Reverse-step throughput over
    the fluid cells, and its bytes: per fluid cell k_adj_local reads the saved
    populations (19 s) and the incoming adjoint (19 x 8 B) and writes the
    outgoing adjoint and the pulled-population adjoints (2 x 19 x 8 B), and
    k_adj_gather reads the latter and updates the former (3 x 19 x 8 B): 19 (s + 48) B.
    arith32: the reverse step of the FP32/FP16 form in FP32 arithmetic."""
    import numpy as np
    from paper_1409_5645_gb300 import cases, fslbm
    nx, ny, nz = dims
    c = cases.dam_break(nx=nx, ny=ny, nz=nz, col_x=nx // 4, col_z=nz * 3 // 4, tau=TAU, magic=MAGIC)
    lat = fslbm.Lattice.from_case(c, precision=form, adjoint_fp32=int(arith32))
    fl = c["flags"]
    nfluid = int(np.count_nonzero((fl == 1) | (fl == 2)))
    try:
        lat.adjoint_forward(steps, K)
        lat.adjoint_backward()
    except fslbm.FslbmError as e:
        lat.close()
        return {"steps": steps, "checkpoint_every": K, "error": str(e)}
    fwd, adj, pk = lat.adjoint_stats()
    lat.close()
    s = STORE_BYTES[form]
    gbs = nfluid * 19 * (s + 48) / (adj / 1e3) / 1e9
    out = {"dims": list(dims), "steps": steps, "checkpoint_every": K,
           "reverse_arithmetic": "fp32" if (arith32 and form != "f64") else "fp64", "fwd_ms_per_step": round(fwd, 5),
           "adj_ms_per_step": round(adj, 5), "adj_over_fwd": round(adj / fwd, 3) if fwd > 0 else None,
           "adj_mlups": round(c.N / (adj / 1e3) / 1e6, 1), "fluid_cells": nfluid,
           "adj_alg_gbs": round(gbs, 1), "peak_bytes": int(pk)}
    if peak:
        out["adj_hbm_frac"] = round(gbs / peak, 4)
    return out


def e2e_run(case, form, steps, local_rank):
    """The user's call sequence with host buffers: the initial state from
    pinned host memory (fslbm_init_equilibrium), then every step fslbm_step
    and a device->host read of that step's mass balance, and at the end the
    fields read back to pinned host memory (fslbm_get_fields: flags, rho, u,
    phi)."""
    import numpy as np
    import torch
    from paper_1409_5645_gb300 import fslbm
    dev = torch.device("cuda", local_rank)
    N = int(case["flags"].size)
    host = {k: torch.from_numpy(case[k]).pin_memory().numpy() for k in ("flags", "rho", "u", "phi")}
    h2d = sum(v.nbytes for v in host.values())
    mask = fslbm.FIELD_FLAGS | fslbm.FIELD_RHO | fslbm.FIELD_U | fslbm.FIELD_PHI
    out = {"flags": np.empty(N, np.uint8), "rho": np.empty(N), "u": np.empty((N, 3)), "phi": np.empty(N)}
    out = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in out.items()}
    d2h_end = sum(v.nbytes for v in out.values())
    lat = fslbm.Lattice(case["dims"], case["params"], precision=form)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    lat.init_equilibrium(host["flags"], host["rho"], host["u"], host["phi"])
    for _ in range(steps):
        lat.step(1)
        lat.step_mass()
    lat.get_into(mask, out)
    t1 = time.perf_counter()
    lat.close()
    return dict(value=N * steps / (t1 - t0) / 1e6, seconds=t1 - t0, h2d_bytes=h2d,
                d2h_bytes_per_step=8 + 4 + d2h_end / steps)


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_rate(dims, col, budget_s, max_steps=None, warmup=0, tau=TAU, magic=MAGIC, omp=False):
    from oracle.oracle import Oracle
    from paper_1409_5645_gb300 import cases
    c = cases.dam_break(nx=dims[0], ny=dims[1], nz=dims[2], col_x=col[0], col_z=col[1], tau=tau, magic=magic)
    o = Oracle.from_case(c, omp=omp)
    if warmup:
        o.step(warmup)
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            break
    return c.N * steps / el / 1e6, steps, el


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    rank, ws = dist_setup("nccl")
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    case = make_case(args)
    N = int(case["flags"].size)
    if args.save_state:
        from paper_1409_5645_gb300 import fslbm
        dev = torch.device("cuda", local_rank)
        lat = fslbm.Lattice(case["dims"], case["params"], precision=forms[0])
        t = {k: torch.from_numpy(case[k]).to(dev) for k in ("flags", "rho", "u", "phi")}
        lat.init_equilibrium(t["flags"], t["rho"], t["u"], t["phi"])
        del t
        lat.step(args.save_after)
        lat.sync()
        save_state(lat, args.save_state)
        print(json.dumps({"saved": args.save_state, "steps": args.save_after, "counters": lat.counters()}))
        return 0

    if ws > 1:
        return main_slabs(args, rank, ws, local_rank, forms[0])
    head = run_form(case, forms[0], args.steps, args.warmup, ws, rank, local_rank, clocks=True,
                    state=args.load_state, spinup=0 if args.load_state else args.spinup, alone=True)
    ms_max = max_over_ranks(head["ms"], ws, torch.device("cuda", local_rank))
    value = ws * N * args.steps / (ms_max / 1e3) / 1e6

    # roofline of the dominant kernel (k_bulk): algorithmic bytes per launch =
    # liquid cells x 2*19*s (pull + store) + every cell's flag byte
    s = STORE_BYTES[forms[0]]
    peak, peak_kind = hbm_peak()
    bulk_ms = head["groups_ms"][0]
    alg_bulk = head["n_liquid"] * 2 * 19 * s + N * 1.0
    achieved = alg_bulk / (bulk_ms / 1e3) / 1e9
    # whole step: + interface cells (populations, m, phi) and their lists
    alg_step = (head["n_liquid"] + head["n_interface"]) * 2 * 19 * s + N * 1.0 + head["n_interface"] * (16 + 8)
    step_gbs = alg_step / (head["ms"] / args.steps / 1e3) / 1e9
    alone_roof = None
    if head["groups_alone"]:
        a_ms = head["groups_alone"][0]
        alone_roof = {"launch_ms": round(a_ms, 5), "achieved": round(alg_bulk / (a_ms / 1e3) / 1e9, 1),
                      "frac": round(alg_bulk / (a_ms / 1e3) / 1e9 / peak, 4)}

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(head["ms"] / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": forms[0], "data": "synthetic",
        "config": {"workload": WORKLOAD if dims_for(args) == DIMS else "dam_break_%dx%dx%d" % dims_for(args),
                   "dims": list(dims_for(args)), "rule": "FSL" if args.rule else "FSK", "tau": args.tau,
                   "magic": args.magic, "g": 1e-5,
                   "precision": forms[0], "parallelism": "one lattice, one GPU",
                   "l2": "inputs larger than L2 (populations %.1f GB)" % (N * 2 * 19 * s / 1e9),
                   "start": ("saved state " + args.load_state) if args.load_state else
                   ("after %d untimed and %d warm-up steps from the initial column: timed steps %d to %d"
                    % (args.spinup, args.warmup, args.spinup + args.warmup + 1, args.spinup + args.warmup + args.steps)
                    if args.spinup else "initial column")},
        "mflups_active": round(ws * (head["n_liquid"] + head["n_interface"]) * args.steps
                               / (ms_max / 1e3) / 1e6, 2),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": ncu_traffic(forms[0]),
                     "kernel": {"tma": "k_bulk_tma", "async": "k_bulk_async", "pairs": "k_bulk_pairs"}.get(head["bulk_loads"], "k_bulk"),
                     "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bulk, "launch_ms": round(bulk_ms, 5),
                     "step": {"frac": round(step_gbs / peak, 4), "achieved": round(step_gbs, 1),
                              "note": "whole FP32 step (all kernels) over the same peak; the target of 0.70 is "
                                      "for this figure"},
                     "alone": alone_roof,
                     "note": "during the timed steps the interface kernels run on a second stream beside the "
                             "bulk kernel, whose grid leaves them room on every SM (launch_ms, frac); alone: the "
                             "same kernel on a full resident wave with every kernel in order, 10 steps right after"},
        "step_roofline": {"achieved": round(step_gbs, 1), "frac": round(step_gbs / peak, 4),
                          "alg_bytes_per_step": alg_step},
        "kernel_ms_per_step": {"bulk": round(head["groups_ms"][0], 5), "iface": round(head["groups_ms"][1], 5),
                               "reduce": round(head["groups_ms"][2], 5), "conversions": round(head["groups_ms"][3], 5)},
        "cells": {"total": N, "liquid_avg": head["n_liquid"], "interface_avg": head["n_interface"]},
        "mass_drift_rel": (head["mass1"] - head["mass0"]) / head["mass0"],
        "gpu_launches": head["launches_per_step"] * args.steps,
        "clocks": head["clocks"],
    }
    # the other precision forms on the same workload
    other = {}
    for f in forms[1:]:
        r = run_form(case, f, args.form_steps, args.warmup, ws, rank, local_rank,
                     spinup=0 if args.load_state else args.spinup)
        msx = max_over_ranks(r["ms"], ws, torch.device("cuda", local_rank))
        sb = STORE_BYTES[f]
        bulk = r["n_liquid"] * 2 * 19 * sb + N
        other[f] = {"value": round(ws * N * args.form_steps / (msx / 1e3) / 1e6, 2), "steps": args.form_steps,
                    "ms_per_step": round(r["ms"] / args.form_steps, 5),
                    "bulk_gbs": round(bulk / (r["groups_ms"][0] / 1e3) / 1e9, 1),
                    "bulk_frac": round(bulk / (r["groups_ms"][0] / 1e3) / 1e9 / peak, 4),
                    "kernel_ms_per_step": [round(x, 5) for x in r["groups_ms"]]}
        if f == "f64":
            # the FP64 bulk kernel against the measured FP64 arithmetic rate:
            # its FP64 operations per liquid-cell update from the committed ncu
            # count (instructions of the same kernel source)
            from paper_1409_5645_gb300 import fslbm
            rate = fslbm.fp64_rate()
            cnt = fp64_counts_per_cell()
            alu = {"bound": "alu", "peak": round(rate, 3), "unit": "TFLOP/s",
                   "peak_kind": "measured (dependent FMA chains on every SM)"}
            if cnt:
                t = r["groups_ms"][0] / 1e3
                ach = cnt[0] * r["n_liquid"] / t / 1e12
                # the FP64 pipe issues one FMA, add or multiply per slot: the
                # instruction rate against the measured FMA instruction rate
                ins = cnt[1] * r["n_liquid"] / t / 1e12
                alu.update(achieved=round(ach, 3), frac=round(ach / rate, 4), flops_per_liquid_cell=cnt[0],
                           instr_frac=round(ins / (rate / 2.0), 4), instructions_per_liquid_cell=cnt[1])
            other[f]["bulk_alu"] = alu
    # the configuration as written (tau = 0.51, Lambda = 3/16): from its
    # initial state for the steps it runs stably (a non-finite density
    # appears between 3500 and 9000 steps)
    if args.as_written_steps:
        aw = argparse.Namespace(**{**vars(args), "tau": 0.51, "magic": 3.0 / 16.0})
        case_aw = make_case(aw)
        r = run_form(case_aw, forms[0], args.as_written_steps, 5, ws, rank, local_rank)  # (5 warm-up steps)
        sb = STORE_BYTES[forms[0]]
        st_b = (r["n_liquid"] + r["n_interface"]) * 2 * 19 * sb + N + r["n_interface"] * 24
        other["as_written_tau0.51_magic3/16"] = {
            "form": forms[0], "value": round(N * args.as_written_steps / (r["ms"] / 1e3) / 1e6, 2),
            "steps": args.as_written_steps, "start": "initial column (after 5 warm-up steps)",
            "ms_per_step": round(r["ms"] / args.as_written_steps, 5),
            "step_frac": round(st_b / (r["ms"] / args.as_written_steps / 1e3) / 1e9 / peak, 4),
            "kernel_ms_per_step": [round(x, 5) for x in r["groups_ms"]],
            "mass_drift_rel": (r["mass1"] - r["mass0"]) / r["mass0"]}
    line["forms"] = other
    # end to end through the C interface with host buffers
    e2e_steps = args.e2e_steps or (args.spinup + args.warmup + args.steps)
    e2e = e2e_run(case, forms[0], e2e_steps, local_rank)
    e2e_v = max_over_ranks(-e2e["value"], ws, torch.device("cuda", local_rank))
    line["e2e"] = {"value": round(-e2e_v * ws, 2), "unit": "MLUPS",
                   "h2d_bytes_per_step": e2e["h2d_bytes"] // e2e_steps,
                   "d2h_bytes_per_step": round(e2e["d2h_bytes_per_step"], 1), "steps": e2e_steps,
                   "includes": "initial state from pinned host memory, per-step mass read, final fields "
                               "(flags, rho, u, phi) read back"}
    # differentiation: adjoint step cost per forward step (FP64 and FP32; the
    # FP32 form's reverse step in FP64 and in FP32 arithmetic)
    if not args.no_adjoint:
        line["adjoint"] = {"workload": "film 8x4x64 depth 40, checkpoints with recompute",
                           "objective": "mean x-velocity of interface cells",
                           "f64": adjoint_run("f64", 4000, 200), "f32": adjoint_run("f32", 4000, 200),
                           "large": {"f32": adjoint_large("f32", peak=peak),
                                     "f32_arith32": adjoint_large("f32", peak=peak, arith32=True),
                                     "f64": adjoint_large("f64", peak=peak)}}
    # the oracle on the host cores (rank 0, N = 1)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, st, el = oracle_rate((128, 64, 64), (32, 48), budget_s=12.0, tau=args.tau, magic=args.magic)
        line["cpu_baseline"] = {"value": round(rate, 3), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                                "sample": f"FP64 oracle, dam break 128x64x64 (same setup scaled by 1/4), "
                                          f"{st} steps in {el:.1f} s, single thread"}
        try:  # the OpenMP build of the same oracle source on every host core
            from oracle import oracle as orc
            nthr = orc.threads(os.cpu_count() or 1)
            rate_a, st_a, el_a = oracle_rate((128, 64, 64), (32, 48), budget_s=12.0, tau=args.tau,
                                             magic=args.magic, omp=True)
            line["cpu_baseline"]["all_cores"] = {
                "value": round(rate_a, 3), "unit": "MLUPS", "cores": nthr,
                "sample": f"the same oracle source built with OpenMP, {st_a} steps in {el_a:.1f} s"}
        except Exception as e:  # no OpenMP toolchain on the host
            line["cpu_baseline"]["all_cores"] = {"unavailable": str(e)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main_slabs(args, rank, ws, local_rank, form):
    """N > 1: one lattice of the dam break widened N times along y (weak
    scaling: every rank owns a full-size 512 x 256 x 256 slab), split into N
    y-slabs with ghost layers, one exchange of ghost layers with the
    neighbouring ranks per step (NCCL point-to-point) and an FP64 all-reduce
    of the mass.  The dam break is uniform along y, so every slab carries the
    same work."""
    import torch
    import torch.distributed as dist
    from paper_1409_5645_gb300 import cases, fslbm, slabs
    dev = torch.device("cuda", local_rank)
    nx, ny, nz = dims_for(args)
    cx, cz = col_for(args)
    gdims = (nx, ny * ws, nz)
    slab = slabs.Slab(gdims, 1, ws, rank)
    local = cases.dam_break(nx=nx, ny=slab.hi - slab.lo, nz=nz, col_x=cx, col_z=cz, tau=args.tau,
                            magic=args.magic, rule=args.rule, bulk_loads=args.bulk_loads, seed=cases.SEED + rank)
    stream = torch.cuda.Stream(device=dev)
    lat = fslbm.Lattice(local["dims"], local["params"], precision=form, stream=stream.cuda_stream)
    t = {k: torch.from_numpy(local[k]).to(dev) for k in ("flags", "rho", "u", "phi")}
    lat.init_equilibrium(t["flags"], t["rho"], t["u"], t["phi"])
    del t
    run = slabs.DistSlab(lat, slab, dev)
    run.exchange()  # ghost layers from the neighbours' owned cells
    run.step(args.spinup + args.warmup)
    lat.sync()
    M0, _ = run.total_mass()
    lat.timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize(dev)
    ck = NvmlClocks(local_rank)
    time.sleep(0.01)
    e0.record(stream)
    run.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = ck.stop() if ck.ok else None
    barrier(ws)
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, ws, dev)
    groups, _ = lat.timing_read()
    lat.timing(False)
    M1, lost = run.total_mass()
    own = nx * (slab.o1 - slab.o0) * nz
    nliq, nifc = count_kinds(lat)
    s_b = STORE_BYTES[form]
    peak, peak_kind = hbm_peak()
    alg_bulk = nliq * 2 * 19 * s_b + lat.N
    achieved = alg_bulk / (groups[0] / 1e3) / 1e9
    value = ws * own * args.steps / (ms_max / 1e3) / 1e6
    launches = (lat.launches_per_step + 2 * len(slab.neighbours())) * args.steps
    # end to end: the slab's initial state from pinned host memory, steps with
    # their exchanges, the all-reduced mass read every step, fields read back
    host = {k: torch.from_numpy(local[k]).pin_memory().numpy() for k in ("flags", "rho", "u", "phi")}
    e2e_steps = args.e2e_steps or args.steps
    lat2 = fslbm.Lattice(local["dims"], local["params"], precision=form)
    barrier(ws)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    lat2.init_equilibrium(host["flags"], host["rho"], host["u"], host["phi"])
    run2 = slabs.DistSlab(lat2, slab, dev)
    run2.exchange()
    for _ in range(e2e_steps):
        run2.step(1)
        run2.total_mass()
    fields = lat2.get(fslbm.FIELD_FLAGS | fslbm.FIELD_RHO | fslbm.FIELD_U | fslbm.FIELD_PHI)
    t1 = time.perf_counter()
    e2e_max = max_over_ranks(t1 - t0, ws, dev)
    d2h = sum(v.nbytes for v in fields.values())
    lat2.close()
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": form, "data": "synthetic",
        "config": {"workload": "dam_break_%dx%dx%d_fsl_y_slabs" % gdims, "dims": list(gdims), "rule":
                   "FSL" if args.rule else "FSK", "tau": args.tau, "magic": args.magic, "g": 1e-5,
                   "precision": form, "parallelism": f"y-slabs x{ws}, {slabs.GHOST} ghost layers per cut, "
                                                     f"NCCL point-to-point",
                   "l2": "inputs larger than L2", "start": "after %d untimed steps" % args.spinup},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "kernel": "k_bulk",
                     "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bulk, "launch_ms": round(groups[0], 5),
                     "rank": 0},
        "kernel_ms_per_step": {"bulk": round(groups[0], 5), "iface": round(groups[1], 5),
                               "reduce": round(groups[2], 5), "conversions": round(groups[3], 5)},
        "halo_bytes_per_step": run.bytes_per_exchange,
        "mass_drift_rel": (M1 - M0) / M0,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": round(ws * own * e2e_steps / e2e_max / 1e6, 2), "unit": "MLUPS",
                "h2d_bytes_per_step": sum(v.nbytes for v in host.values()) // e2e_steps,
                "d2h_bytes_per_step": round(16 + d2h / e2e_steps, 1), "steps": e2e_steps,
                "includes": "slab state from pinned host memory, exchanges, all-reduced mass read every step, "
                            "fields read back"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    lat.close()
    dist.destroy_process_group()
    return 0


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    ncores = os.cpu_count()
    total = args.steps + args.warmup
    # sample sized so that warm-up + timed steps take about two minutes
    budget = 120.0
    per_step = budget / max(total, 1)
    # oracle cost ~ 0.4 us per cell and step on one core
    cells = min(max(int(per_step / 4e-7), 16 * 8 * 12), 2_000_000)
    scale = (cells / (DIMS[0] * DIMS[1] * DIMS[2])) ** (1 / 3)
    nx = max(16, int(DIMS[0] * scale) // 4 * 4)
    ny = max(8, int(DIMS[1] * scale) // 4 * 4)
    nz = max(12, int(DIMS[2] * scale) // 4 * 4)
    col = (max(4, nx // 4), max(6, nz * 3 // 4))
    from oracle.oracle import Oracle
    from paper_1409_5645_gb300 import cases
    c = cases.dam_break(nx=nx, ny=ny, nz=nz, col_x=col[0], col_z=col[1], tau=args.tau, magic=args.magic,
                        rule=args.rule)
    o = Oracle.from_case(c)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = c.N * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "MLUPS", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 4),
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_dims": [nx, ny, nz], "rule": "FSL" if args.rule else "FSK",
                       "tau": args.tau, "magic": args.magic, "g": 1e-5},
            "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": f"FP64 oracle, dam break {nx}x{ny}x{nz} (same setup scaled), "
                                       f"{args.steps} timed steps, single thread of {ncores}"},
            "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

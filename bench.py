#!/usr/bin/env python
"""Throughput of the two-colour LBM step on the synthetic 256^3 porous rock
(primary drainage, Type-I Zou-He ends, Scheme-I wetting, FP32 storage).

One JSON line on rank 0:
  value      fluid-node updates per second / 1e6 (MLUPS), whole job over all
             ranks, populations resident in HBM, CUDA events around K steps,
             the median of --repeats timed regions (each K steps);
  e2e        the same metric through the public API from host buffers: the
             solid image and phi0 copied in from pinned memory, geometry set-up,
             K steps each followed by the FP64 saturation read-back (8 bytes),
             the final phase field copied out;
  roofline   the whole step against the measured HBM copy bandwidth, with
             308 B per fluid-node update (2 x 2Q populations of 4 B read and
             written plus a 4 B link mask) over the median step time;
             `traffic` the ncu DRAM bytes of the step's kernels summed;
  passes     every kernel of the step: CUDA-event time, its own
             algorithmic bytes (pass_bytes below) and ncu DRAM bytes;
             dominant_pass the longest of them;
  cpu_baseline  the FP64 oracle on a bounded slab of the same rock, on all
             host cores and on one;
  tube       the capillary-tube workload (256 x 20 x 20, r = 8, Type-I,
             20000 steps): throughput, and the interface speed beside the
             Washburn law for equal viscosities (Eq. 47);
  laplace    the Laplace test of Sec. III.A at the paper's 128^3 scale: the
             interfacial tension from five drops in N/m beside the 0.02 N/m
             input and the paper's 0.02009;
  washburn   Washburn Case-I (Sec. IV.A.1): spontaneous imbibition in the
             12x12x101 tube at 30-75 deg with both wetting schemes, and
             Case-II (Sec. IV.A.2): theta = 90 deg, three pressure drops,
             Type-I and Type-II; the paper's area error against Eq. (49);
  mrt        the same rock with the MRT collision (Eq. 2 with the rates of
             Eqs. 4, 15-16), with its error against the FP64 oracle's MRT;
  storage_16bit the same rock with FP16 / BF16 population storage, each
             with its error against the FP64 oracle on a slab;
  batched    the 96-drop contact-angle sweep stepped as one batch
             (autotuned schedule), FP32 and FP16-offset storage, each with
             its error against the FP64 oracle;
  adjoint    the gradient of the smooth saturation after 2000 steps of the
             128^3 imbibition pack w.r.t. theta and g_x, beside central
             finite differences.

`--impl reference` times the oracle (the reference arm) on the
host cores instead. Several GPUs (torchrun) run independent replicas.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline: plain FP32 vs FP16-storage/batched at stated error"
BYTES_POP = {"fp32": 4, "fp16": 2, "bf16": 2}


def pass_bytes(Q: int, bpp: int, cells_per_node: float = 3.66) -> dict:
    """Algorithmic DRAM bytes per processed node of each pass: what the pass
    must read and write once (a gathered field counts once per node, since
    every element is read by a fixed number of neighbours that L2 serves).
    Fluid passes find their neighbours in the dense entry box, 4 B per cell
    of the padded box, read once per pass: cells_per_node = box cells per
    fluid node (3.66 on the 256^3 rock, 15 B of entries per node); the
    Eq. 35 pass reads its CSR links (4.2 per node on the rock, taken as
    5 x 4 B) and two offsets; the Eq. 34 pass a 4 B direction mask."""
    ent = round(4.0 * cells_per_node, 1)
    return {
        # T_i of the sources (each once), (q, v) 16 B, the entries, flags
        # 1 B, padded index 4 B; writes f^t (Q planes), (rho^r, rho^b) 8 B,
        # the phase field 4 B and its dense copy 4 B
        "stream": Q * bpp + 16 + ent + 1 + 4 + Q * bpp + 8 + 4 + 4,
        # U of the node (Q planes), flags, the entry of x - a, phase of
        # that node; at the outlet the colour split of the known
        # populations re-reads about 14 entries and (q, v); writes
        # 5 planes, (rho^r, rho^b), phase and its dense copy (padded index)
        "zh_fix": Q * bpp + 1 + 4 + 4 + 7 * (4 + 16) + 5 * bpp + 8 + 4 + 8,
        # direction mask 4 B, padded index 4 B, face bits, the fluid
        # neighbours' phase from the dense box 4 B; writes the phase 4 B and
        # its dense copy 4 B
        "phi_solid": 4 + 4 + 1 + 4 + 4 + 4,
        # padded index 4 B, the dense phase field 4 B (no table), flags,
        # wall normal 16 B (fluid-boundary nodes, about 45 %: 7 B); write
        # (n_c, |C|) 16 B
        "gradient": 4 + 4 + 1 + 7 + 16,
        # the mark 1 B: the bytes every solid-boundary node needs (a node
        # marked by the gradient pass adds its links + offsets, the
        # neighbours' n_c 16 B and the write of 16 B)
        "nc_solid": 1,
        # the node's own (n_c, |C|) 16 B: the bytes every node needs (a
        # node with an interface adds its padded index 4 B, the entries, the
        # neighbours' (n_c, |C|) 16 B and the curvature write 4 B; a node
        # without one stops there, its surface force being zero)
        "curvature": 16,
        # (n_c, |C|) 16 B, f^t, (rho^r, rho^b), phase 4 B; writes f''
        # (Q planes) and (q, v) 16 B (plus the curvature, 4 B, at a node
        # with an interface)
        "collide": 16 + Q * bpp + 8 + 4 + Q * bpp + 16,
    }


# GB300 HBM3e nominal bandwidth (the measured copy peak is the roofline's
# denominator; this is reported beside it)
NOMINAL_HBM_GBS = 7900.0

# the kernel of each pass (names as ncu lists them)
PASS_KERNEL = {"stream": "k_stream", "zh_fix": "k_zh_fix",
               "phi_solid": "k_phi_solid", "gradient": "k_gradient",
               "nc_solid": "k_nc_solid_marked", "curvature": "k_curvature",
               "collide": "k_collide"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--drive", default="typeI", choices=["typeI", "typeII"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 96-drop batched sweep object")
    ap.add_argument("--batched-cases", type=int, default=96)
    ap.add_argument("--batched-steps", type=int, default=20)
    ap.add_argument("--no-tube", action="store_true",
                    help="skip the capillary-tube object")
    ap.add_argument("--no-laplace", action="store_true",
                    help="skip the Laplace-law object")
    ap.add_argument("--no-washburn", action="store_true",
                    help="skip the Washburn Case-I object")
    ap.add_argument("--no-mrt", action="store_true",
                    help="skip the MRT-collision object")
    ap.add_argument("--no-16bit", action="store_true",
                    help="skip the FP16/BF16-storage objects")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the gradient (adjoint) object")
    ap.add_argument("--repeats", type=int, default=5,
                    help="repeats of the timed region, at least (more when a repeat is short: about 0.5 s in all; median reported)")
    ap.add_argument("--oracle-sample", nargs=3, type=int, default=None,
                    metavar=("PLANES", "STEPS", "SIZE"),
                    help=argparse.SUPPRESS)
    ap.add_argument("--adjoint-fd64", nargs="?", const="all", default=None,
                    choices=["all", "gx"],
                    help="also central differences of the FP64 oracle at the "
                         "gradient workload's full size (about 15 min of "
                         "host CPU)")
    ap.add_argument("--adjoint-tlm64", action="store_true",
                    help="also the FP64 oracle's tangent-linear run at the "
                         "gradient workload's full size")
    ap.add_argument("--tile", default="auto",
                    help="tile shape of the fluid-node numbering: 'auto' "
                         "(the autotuner's search on the workload), "
                         "'default', or XxYxZ")
    ap.add_argument("--adjoint-size", type=int, default=128)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    return ap.parse_args()


def workload(args):
    from paper_2407_10914_gb300 import workloads as W
    n = args.size
    case = W.porous_3d(n=(n, n, n), drive=args.drive)
    name = f"porous{n}_drainage_{args.drive}_{args.storage}"
    return case, name


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_value(ws: int, units_per_rank: int, steps: int,
                    ms_max: float) -> float:
    """Whole-job throughput in millions of units per second: the units all
    ranks processed (every rank steps its own replica) over the slowest
    rank's time."""
    return ws * units_per_rank * steps / (ms_max * 1e-3) / 1e6


def max_over_ranks(v, ws):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.idx = gpu_index
        exe = shutil.which("nvidia-smi")
        if exe:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                [exe, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(gpu_index), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback 6.8 TB/s"


def kernel_source_hash():
    h = hashlib.sha1()
    for f in ("step.cu", "passes.cuh", "tiles.cuh",
              "stencil.cuh", "lattice.cuh", "context.hpp", "geometry.cu"):
        h.update(open(os.path.join(ROOT, "paper_2407_10914_gb300", "csrc", f),
                      "rb").read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary (profiles/dram_traffic.txt), if it was taken on the current
    kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    want = kernel_source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#"):
            if parts[0] == kernel and parts[1] == workload and parts[3] == want:
                return float(parts[2])
    return None


# --------------------------------------------------------- CPU oracle
def oracle_sample(case, planes: int):
    """A slab of the first `planes` x-planes of the rock (inlet reservoir +
    rock), same parameters, as a bounded sample for the oracle."""
    from paper_2407_10914_gb300 import workloads as W
    solid = np.ascontiguousarray(case.solid[:, :, :planes])
    phi0 = np.ascontiguousarray(case.phi0[:, :, :planes])
    return W.Case(case.name + f"_slab{planes}", case.lattice, solid,
                  case.periodic, phi0, dict(case.params))


def time_oracle(case, planes: int, steps: int, warmup: int = 0):
    from oracle import oracle as O
    O.build()
    sample = oracle_sample(case, planes)
    o = O.Oracle(sample.lattice, sample.solid, sample.periodic)
    o.set_params(**sample.params)
    o.init_state(sample.phi0)
    if warmup:
        o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    nf = int((sample.solid == 0).sum())
    return dict(value=nf * steps / dt / 1e6, unit="MLUPS", cores=O.max_threads(),
                kind="oracle",
                sample=f"first {planes} x-planes of the {case.solid.shape[2]}^3 "
                       f"rock ({nf} fluid nodes), {steps} steps, FP64 oracle",
                seconds=dt)


def oracle_single_core(args, planes: int, steps: int):
    """The oracle on one host core (OMP_NUM_THREADS=1, a child process, so
    that the OpenMP runtime starts with one thread) on a smaller slab of the
    same rock."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample",
           str(planes), str(steps), str(args.size), "--drive", args.drive]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True,
                           timeout=600)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


def run_oracle_sample(args):
    planes, steps, size = args.oracle_sample
    args.size = size
    case, _ = workload(args)
    res = time_oracle(case, planes, steps, 0)
    print(json.dumps({k: res[k] for k in ("value", "unit", "cores", "kind",
                                          "sample")}), flush=True)


def run_reference(args):
    ws, rank, _ = dist_init(args)
    if rank != 0:
        return
    case, name = workload(args)
    # size the slab so that warm-up + timed steps take about 90 s
    probe = time_oracle(case, 6, 1, 0)
    per_plane = probe["seconds"] / 6.0
    planes = int(90.0 / max(1, args.steps + args.warmup) / per_plane)
    planes = max(3, min(case.solid.shape[2], planes))
    res = time_oracle(case, planes, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": round(res["value"], 3),
            "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample": res["sample"]},
            "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind",
                                                  "sample")},
            "e2e": {"value": round(res["value"], 3), "unit": "MLUPS",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- our arm
def pick_tile(args, make, q):
    """Tile shape for the run: --tile auto runs the autotuner's tile search
    (each candidate a domain or batch of its own, 1 untimed + 8 timed
    steps); returns (tile or None for the default, the trials or None)."""
    if args.tile == "default":
        return None, None
    if args.tile != "auto":
        return tuple(int(v) for v in args.tile.split("x")), None
    from paper_2407_10914_gb300 import autotune
    r = autotune.tune_tile(make, q, trial_steps=8, use_cache=False)
    return r["tile"], r["trials"]


def tile_name(tile, q):
    if tile is None:
        tile = (32, 8, 8) if q == 19 else (64, 32, 1)
    return "x".join(str(v) for v in tile)


def run_ours(args):
    import torch
    from paper_2407_10914_gb300 import build, lbm

    ws, rank, local = dist_init(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    build.build()
    case, name = workload(args)
    Q = case.lattice

    def make(tile):
        s = lbm.Session(Q, case.solid, case.periodic, args.storage, tile=tile)
        s.set_params(**case.params)
        s.init_state(case.phi0.astype(np.float32))
        return s

    tile, tile_trials = pick_tile(args, make, Q)
    torch.cuda.empty_cache()
    s = make(tile)
    nf = s.n_fluid
    n_sbnd = s.counts[2]
    stream = torch.cuda.current_stream()

    torch.cuda.synchronize()
    w0 = torch.cuda.Event(enable_timing=True)
    w1 = torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    s.step(args.warmup)
    w1.record(stream)
    torch.cuda.synchronize()
    # repeats: at least --repeats, and enough for about 0.5 s of timed work
    # (so that the clock sampler sees the timed region), at most 200
    est_ms = w0.elapsed_time(w1) / max(1, args.warmup)
    n_rep = max(1, args.repeats)
    if est_ms > 0:
        n_rep = min(200, max(n_rep, int(math.ceil(500.0 / (est_ms * args.steps)))))
    clocks = ClockSampler(local)
    # the timed region, repeated: each repeat is `steps` steps between a
    # barrier and CUDA events on the launching stream; the population
    # buffers (2 x 0.35 GB on the rock) exceed the 129 MB L2 every step
    rep_ms = []
    for _ in range(n_rep):
        barrier(ws)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        rep_ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    ms = float(np.median(rep_ms))
    ms_max = max_over_ranks(ms, ws)
    value = whole_job_value(ws, nf, args.steps, ms_max)
    step_ms = ms_max / args.steps

    # per-pass times (events inside the library, on the same stream)
    k2 = max(1, min(args.steps, 200))
    pass_ms = s.step_timed(k2)
    bpp = BYTES_POP[args.storage]
    cells = float((case.solid.shape[0] + 2) * (case.solid.shape[1] + 2)
                  * (case.solid.shape[2] + 2)) / nf
    pb = pass_bytes(Q, bpp, cells)
    n_zh = s.n_zou_he
    n_of = {"stream": nf, "zh_fix": n_zh, "phi_solid": n_sbnd, "gradient": nf,
            "nc_solid": n_sbnd, "curvature": nf, "collide": nf}
    peak, peak_src = measured_peaks()
    passes_out = {}
    for p, t in pass_ms.items():
        if t <= 0 or n_of[p] == 0:
            continue
        t1 = t / k2
        b = pb[p] * n_of[p]
        kern = PASS_KERNEL[p]
        tr = recorded_traffic(kern, name)
        passes_out[p] = {"kernel": kern, "ms": round(t1, 5),
                         "bytes_per_node": pb[p], "nodes": n_of[p],
                         "GBps": round(b / (t1 * 1e-3) / 1e9, 1),
                         "frac": round(b / (t1 * 1e-3) / 1e9 / peak, 4),
                         "dram_bytes_per_launch": tr,
                         "dram_GBps": (round(tr / (t1 * 1e-3) / 1e9, 1)
                                       if tr else None)}
    dom = max(passes_out, key=lambda p: passes_out[p]["ms"])
    # the step against the algorithmic 308 B per fluid-node update (38 pops
    # read and written, 4 B link mask)
    upd_bytes = 2 * 2 * Q * bpp + 4
    step_alg = upd_bytes * nf
    achieved = step_alg / (step_ms * 1e-3) / 1e9
    step_traffic = None
    if passes_out and all(v["dram_bytes_per_launch"] for v in passes_out.values()):
        step_traffic = sum(v["dram_bytes_per_launch"] for v in passes_out.values())
    launches_per_step = len(passes_out)

    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(args, case, torch, lbm, tile)

    tube = None
    if not args.no_tube and rank == 0:
        tube = run_tube(torch, lbm)

    laplace = None
    if not args.no_laplace and rank == 0:
        laplace = run_laplace(lbm)

    washburn = None
    if not args.no_washburn and rank == 0:
        washburn = run_washburn(lbm)

    mrt = None
    if not args.no_mrt and rank == 0 and args.storage == "fp32":
        mrt = run_mrt(args, torch, lbm, case, min(args.steps, 500))

    sixteen = None
    if not args.no_16bit and rank == 0:
        sixteen = run_16bit(args, torch, lbm, case, min(args.steps, 500), tile)

    batched = None
    batched16 = None
    if not args.no_batched:
        batched = run_batched(args, torch, lbm, "fp32")
        batched16 = run_batched(args, torch, lbm, "fp16")
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(args, torch, lbm)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(case, 32, 6, 0)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        one = oracle_single_core(args, 8, 2)
        if one:
            cpu["single_core"] = one

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": name, "grid": list(case.solid.shape[::-1]),
                "fluid_nodes": nf, "nodes": case.n_nodes,
                "rock_porosity": round(case.info.get("rock_porosity", 0), 4),
                "storage": args.storage, "lattice": "D3Q19",
                "tile": tile_name(tile, Q),
                "tile_search_ms_per_step": tile_trials,
                "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                "l2": "inputs larger than L2 (two population buffers of "
                      f"{Q * bpp * nf / 1e9:.2f} GB each over the fluid "
                      "nodes, against 0.13 GB of L2)",
            },
            "roofline": {"bound": "hbm",
                         "kernel": "the whole step (" + ", ".join(
                             PASS_KERNEL[p] for p in passes_out) + ")",
                         "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": step_traffic, "peak_source": peak_src,
                         "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
                         "nominal_gbs": NOMINAL_HBM_GBS,
                         "dram_bytes_per_update": (
                             None if step_traffic is None
                             else round(step_traffic / nf, 1)),
                         "bytes_per_update": upd_bytes,
                         "algorithmic_bytes_per_step": step_alg,
                         "ms_per_step": round(step_ms, 5),
                         "timing": "CUDA events on the launching stream "
                                   f"around {args.steps} steps, median of "
                                   f"{len(rep_ms)} repeats",
                         "traffic_note": "sum over the step's kernels of "
                                         "ncu dram__bytes_read.sum + "
                                         "dram__bytes_write.sum per launch "
                                         "(profiles/dram_traffic.txt, current "
                                         "kernel source only), captured with "
                                         "the default tile shape "
                                         f"{tile_name(None, Q)}; this run's "
                                         f"tile: {tile_name(tile, Q)}"},
            "dominant_pass": dict(passes_out[dom], name=dom),
            "passes": passes_out,
            "repeats_ms_per_step": [round(x / args.steps, 5) for x in rep_ms],
            "spread_pct": round(100 * (max(rep_ms) - min(rep_ms)) / ms, 2),
            "pass_ms_per_step": {k: round(v / k2, 5) for k, v in pass_ms.items()},
            "gpu_launches": launches_per_step * args.steps * len(rep_ms),
            "clocks": clk,
            "total_node_MLUPS": round(ws * case.n_nodes * args.steps
                                      / (ms_max * 1e-3) / 1e6, 1),
        }
        if clk and clk.get("sm_mhz"):
            line["time_x_sm_mhz"] = round(step_ms * clk["sm_mhz"], 3)
        if e2e:
            line["e2e"] = e2e
        if tube:
            line["tube"] = tube
        if laplace:
            line["laplace"] = laplace
        if washburn:
            line["washburn"] = washburn
        if mrt:
            line["mrt"] = mrt
        if sixteen:
            line["storage_16bit"] = sixteen
        if batched:
            line["batched"] = batched
        if batched16:
            line["batched_fp16"] = batched16
        if adjoint:
            line["adjoint"] = adjoint
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# the drainage workload's run length (10 000 steps): the end-to-end leg
# runs it whole, set-up included
E2E_STEPS = 10000


def end_to_end(args, case, torch, lbm, tile=None):
    """The user's call sequence from host memory: workspace allocated
    beforehand; timed: lbm_init_geometry_tiled (solid image H2D from pinned
    host memory; the run's tile shape), phi0 H2D (pinned), K x (step + the
    S_w reduction read back to page-locked host memory with
    lbm_reduce_async, so the GPU never waits for the host), final phi D2H,
    and every step's S_w value (lbm_reduce_value). K is the workload's
    whole drainage run (10 000 steps), or the timed step count if that is
    larger."""
    from paper_2407_10914_gb300.lbm import STORAGE, lbm_workspace_bytes_tiled
    import ctypes as C
    nz, ny, nx = case.solid.shape
    Q = case.lattice
    solid_pin = torch.from_numpy(case.solid.reshape(-1)).pin_memory()
    phi_pin = torch.from_numpy(case.phi0.astype(np.float32).reshape(-1)).pin_memory()
    out_pin = torch.empty(case.n_nodes, dtype=torch.float32).pin_memory()
    mask = sum((1 << a) for a in range(3) if case.periodic[a])
    wsb = lbm_workspace_bytes_tiled(Q, nx, ny, nz, case.solid,
                                    STORAGE[args.storage], tile)
    tile_c = None if tile is None else (C.c_int * 3)(*tile)
    work = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    phi_dev = torch.empty(case.n_nodes, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    L = lbm.load_library()
    steps = max(args.steps, E2E_STEPS)
    raw = torch.zeros((steps, 4), dtype=torch.float64).pin_memory()
    raw_at = raw.data_ptr()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = C.c_void_p()
    st = L.lbm_init_geometry_tiled(C.byref(h), Q, nx, ny, nz,
                                   C.c_void_p(solid_pin.data_ptr()), mask,
                                   STORAGE[args.storage], tile_c,
                                   C.c_void_p(work.data_ptr()), wsb, sp)
    assert st == 0, st
    lbm.lbm_set_params(h, lbm.make_params(**case.params))
    phi_dev.copy_(phi_pin, non_blocking=True)
    lbm.lbm_init_state(h, phi_dev, sp)
    for i in range(steps):
        lbm.lbm_step(h, 1, sp)
        lbm.lbm_reduce_async(h, lbm.LBM_SW_COUNT, raw_at + 32 * i, sp)
    lbm.lbm_macros(h, None, phi_dev, None, sp)
    out_pin.copy_(phi_dev, non_blocking=True)
    torch.cuda.synchronize()
    sw_series = [lbm.lbm_reduce_value(h, lbm.LBM_SW_COUNT, raw_at + 32 * i)
                 for i in range(steps)]
    dt = time.perf_counter() - t0
    sw = sw_series[-1]
    lbm.lbm_destroy(h)
    nf = int((case.solid == 0).sum())
    return {"value": round(nf * steps / dt / 1e6, 2), "unit": "MLUPS",
            "h2d_bytes_per_step": round((case.n_nodes * 5) / steps, 1),
            "d2h_bytes_per_step": round(32 + case.n_nodes * 4 / steps, 1),
            "final_sw": sw, "first_sw": sw_series[0],
            "seconds": round(dt, 3), "steps": steps,
            "note": "the whole drainage run through the C-ABI from host "
                    "buffers: geometry set-up, phi0 upload, every step's "
                    "S_w read back (lbm_reduce_async into page-locked host "
                    "memory, lbm_reduce_value) and the final phi download "
                    "inside the timed region"}


def run_tube(torch, lbm):
    """The capillary tube in full (20000 steps, 4000 per record): MLUPS over
    its fluid nodes, and the interface speed (fit over the last four
    records) beside Eq. (47) with equal viscosities and cos(theta) = 0,
    with the effective radius that speed implies."""
    from paper_2407_10914_gb300 import analysis as A
    from paper_2407_10914_gb300 import workloads as W
    case = W.tube_3d()
    s = lbm.Session(19, case.solid, case.periodic)
    s.set_params(**case.params)
    s.init_state(case.phi0.astype(np.float32))
    stream = torch.cuda.current_stream()
    ts, zs, ms = [], [], 0.0
    for k in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(4000)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        ts.append(4000 * (k + 1))
        zs.append(A.interface_position(s.macros()["phi"].cpu().numpy(), 0,
                                       case.solid))
    U = float(np.polyfit(ts[1:], zs[1:], 1)[0])
    p = case.params
    dP = (p["rho_in"] - p["rho_out"]) / 3
    mu = p["rho0"] * (p["tau_r"] - 0.5) / 3
    L = case.solid.shape[2] - 1
    r = case.info["radius"]
    U_ref = r * r * dP / (8 * mu * L)
    return {"workload": "tube_256x20x20_r8_typeI", "steps": 20000,
            "fluid_nodes": s.n_fluid,
            "value": round(s.n_fluid * 20000 / (ms * 1e-3) / 1e6, 1),
            "unit": "MLUPS", "ms_per_step": round(ms / 20000, 5),
            "interface_z": [round(z, 3) for z in zs],
            "speed": U, "speed_eq47": U_ref,
            "speed_error_pct": round(100 * abs(U / U_ref - 1), 2),
            "r_eff": round(float(np.sqrt(8 * mu * L * U / dP)), 3),
            "note": "launch-bound at this size (seven kernels per step)"}


def run_laplace(lbm):
    """Sec. III.A at the paper's scale: five drops (R = 12-30) in a periodic
    128^3 box, 12000 steps each, the jump averaged over the second half;
    the slope of dP against 2/R in N/m (Eqs. 43-44, the paper's units)."""
    from paper_2407_10914_gb300 import laplace as Lp
    t0 = time.time()

    def make(case):
        s = lbm.Session(19, case.solid, case.periodic)
        s.set_params(**case.params)
        s.init_state(case.phi0.astype(np.float32))
        return s

    out = {"workload": "laplace_128cubed_5drops", "steps_per_drop": 12000,
           "gamma_input_n_per_m": 0.02, "paper_gamma_sim_n_per_m": 0.02009,
           "paper_error_pct": 0.45,
           "paper_context": "MRT, RTX 3090, FP32 (Sec. III.A)"}
    for coll, key in ((0, "single_rate"), (1, "mrt")):
        r = Lp.sweep(make, 128, (12.0, 16.0, 20.0, 24.0, 30.0), steps=12000,
                     collision=coll)
        out[key] = {"radii": [round(x, 3) for x in r["radii"]],
                    "dp_pa": [round(x, 2) for x in r["dp_phys"]],
                    "gamma_sim_n_per_m": round(r["gamma_phys_sim"], 6),
                    "error_pct": round(100 * r["error"], 3)}
    out["seconds"] = round(time.time() - t0, 1)
    return out


def run_washburn(lbm):
    """Washburn Case-I on the paper's tube: for each contact angle and
    wetting scheme the area error (%) of the interface path against Eq.
    (49) from t*_init (Eq. 49 at the settled initial interface) to t* = 60,
    and the interface position at the end beside Eq. (49)'s."""
    from paper_2407_10914_gb300 import washburn as Wb
    from paper_2407_10914_gb300 import workloads as W
    t0 = time.time()
    out = {"workload": "washburn_tube_12x12x101_r5", "viscosity_ratio": 0.2,
           "gamma_lbm": 1.0 / 45.0, "tstar_end": 60.0, "runs": []}
    for wetting in (1, 2):
        for theta in (30.0, 45.0, 60.0, 75.0):
            case = W.washburn_tube(theta, wetting)

            def make(params, case=case):
                s = lbm.Session(19, case.solid, case.periodic)
                s.set_params(**params)
                s.init_state(case.phi0.astype(np.float32))
                return s

            r = Wb.run_case1(make, case, theta, wetting, tstar_end=60.0)
            out["runs"].append({
                "scheme": "I" if wetting == 1 else "II", "theta_deg": theta,
                "area_error_pct": round(100 * r["area_error"], 3),
                "zstar_init": round(r["z_init"], 4),
                "tstar_init": round(r["tstar_init"], 3),
                "zstar_end": round(float(r["zstar"][-1]), 4),
                "zstar_end_eq49": round(float(r["zstar_eq49"][-1]), 4),
                "tstar_end": round(float(r["tstar"][-1]), 2)})
    # Case-II (Sec. IV.A.2): theta = 90 deg, pressure-driven, both drives
    case = W.washburn_tube(90.0, 1)

    def make2(params, case=case):
        s = lbm.Session(19, case.solid, case.periodic)
        s.set_params(**params)
        s.init_state(case.phi0.astype(np.float32))
        return s

    out["case2"] = []
    for drive in ("typeI", "typeII"):
        for dp_term in (0.01, 0.02, 0.04):
            dp = dp_term * 2 * case.info["length"] * case.params["gamma"] / 25.0
            r = Wb.run_case2(make2, case, dp, drive, tstar_end=60.0)
            out["case2"].append({
                "drive": drive, "dp_lbm": round(dp, 6),
                "dp_pa_paper_units": round(dp * 1e-15 / (1e-6 * (1e-6 / 30) ** 2), 1),
                "area_error_pct": round(100 * r["area_error"], 3),
                "zstar_end": round(float(r["zstar"][-1]), 4),
                "zstar_end_eq49": round(float(r["zstar_eq49"][-1]), 4)})
    out["seconds"] = round(time.time() - t0, 1)
    return out


def run_mrt(args, torch, lbm, case, steps: int):
    """The same rock and storage with the MRT collision (collision = 1):
    throughput over `steps` steps, per-pass times, and the error against the
    FP64 oracle's MRT after 10 steps from the initial state on the 32-plane
    slab (max |f_gpu - f_oracle| / max |f_oracle| per colour)."""
    from oracle import oracle as O
    params = dict(case.params, collision=1)
    slab = oracle_sample(case, 32)
    o = O.Oracle(slab.lattice, slab.solid, slab.periodic)
    o.set_params(**dict(slab.params, collision=1))
    o.init_state(slab.phi0)
    o.step(10)
    ref = o.pops
    fl = slab.solid == 0
    t = lbm.Session(slab.lattice, slab.solid, slab.periodic, args.storage)
    t.set_params(**dict(slab.params, collision=1))
    t.init_state(slab.phi0.astype(np.float32))
    t.step(10)
    got = t.get_populations().cpu().numpy().astype(np.float64)
    err = max(float(np.abs(got[c][:, fl] - ref[c][:, fl]).max()
                    / np.abs(ref[c][:, fl]).max()) for c in range(2))
    del t
    s = lbm.Session(case.lattice, case.solid, case.periodic, args.storage)
    s.set_params(**params)
    s.init_state(case.phi0.astype(np.float32))
    stream = torch.cuda.current_stream()
    s.step(args.warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    k2 = min(steps, 100)
    pm = s.step_timed(k2)
    out = {"collision": "MRT, rates of Eqs. 4, 15-16",
           "value": round(s.n_fluid / (ms * 1e-3) / 1e6, 2), "unit": "MLUPS",
           "ms_per_step": round(ms, 4),
           "pass_ms_per_step": {k: round(v / k2, 5) for k, v in pm.items()},
           "error_vs_fp64_oracle": err,
           "error_sample": "32-plane slab of the rock, 10 steps from the "
                           "initial state, max relative population error"}
    del s
    return out


def field_errors(o, s, fluid):
    """Largest |difference| over fluid nodes of phi, rho and |u| between the
    oracle and a session, after the same steps."""
    fo = o.fields()
    m = s.macros()
    out = {}
    for k in ("phi", "rho"):
        got = m[k].cpu().numpy().astype(np.float64)
        out[k] = float(np.abs(got - fo[k])[fluid].max())
    gu = m["u"].cpu().numpy().astype(np.float64)
    out["u"] = float(np.sqrt(((gu - fo["u"]) ** 2).sum(0))[fluid].max())
    out["u_max"] = float(np.sqrt((fo["u"] ** 2).sum(0))[fluid].max())
    return out


def run_16bit(args, torch, lbm, case, steps: int, tile=None):
    """The same rock with the f''_i planes stored as 16-bit offsets (FP16,
    BF16): throughput over `steps` steps, per-pass times, the fraction of
    the HBM roofline with their own 156 B per fluid-node update (2 x 2Q
    populations of 2 B and a 4 B link mask), and the error against the FP64
    oracle after 10 steps from the initial state: the populations on the
    32-plane slab (max |f_gpu - f_oracle| / max |f_oracle| per colour) and
    phi, rho, u on the full rock, with the FP32 storage's errors beside
    them."""
    from oracle import oracle as O
    out = {}
    slab = oracle_sample(case, 32)
    o = O.Oracle(slab.lattice, slab.solid, slab.periodic)
    o.set_params(**slab.params)
    o.init_state(slab.phi0)
    o.step(10)
    ref = o.pops
    fl = slab.solid == 0
    del o
    full = O.Oracle(case.lattice, case.solid, case.periodic)
    full.set_params(**case.params)
    full.init_state(case.phi0)
    full.step(10)
    fluid = case.solid == 0

    def errors(storage):
        t = lbm.Session(slab.lattice, slab.solid, slab.periodic, storage)
        t.set_params(**slab.params)
        t.init_state(slab.phi0.astype(np.float32))
        t.step(10)
        got = t.get_populations().cpu().numpy().astype(np.float64)
        pop = max(float(np.abs(got[c][:, fl] - ref[c][:, fl]).max()
                        / np.abs(ref[c][:, fl]).max()) for c in range(2))
        del t
        r = lbm.Session(case.lattice, case.solid, case.periodic, storage)
        r.set_params(**case.params)
        r.init_state(case.phi0.astype(np.float32))
        r.step(10)
        fe = field_errors(full, r, fluid)
        del r
        return pop, fe

    pop32, fe32 = errors("fp32")
    out["fp32_slab_error"] = pop32
    out["fp32_full_rock_field_errors"] = fe32
    stream = torch.cuda.current_stream()
    peak, _ = measured_peaks()
    out["tile"] = tile_name(tile, case.lattice)
    for storage in ("fp16", "bf16"):
        s = lbm.Session(case.lattice, case.solid, case.periodic, storage,
                        tile=tile)
        s.set_params(**case.params)
        s.init_state(case.phi0.astype(np.float32))
        s.step(args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        k2 = min(steps, 100)
        pm = s.step_timed(k2)
        upd = 2 * 2 * case.lattice * 2 + 4
        del s
        pop, fe = errors(storage)
        out[storage] = {
            "value": round(case_fluid(case) / (ms * 1e-3) / 1e6, 2),
            "unit": "MLUPS", "ms_per_step": round(ms, 4),
            "pass_ms_per_step": {k: round(v / k2, 5) for k, v in pm.items()},
            "bytes_per_update_2q_pops": upd,
            "roofline_frac": round(upd * case_fluid(case) / (ms * 1e-3) / 1e9
                                   / peak, 4),
            "error_vs_fp64_oracle": pop,
            "error_sample": "32-plane slab of the rock, 10 steps from the "
                            "initial state, max relative population error",
            "full_rock_field_errors": fe,
            "full_rock_sample": "the whole 256^3 rock, 10 steps from the "
                                "initial state: max |difference| over fluid "
                                "nodes of phi, rho and |u|",
        }
    return out


def case_fluid(case) -> int:
    return int((case.solid == 0).sum())


def batch_error(args, torch, lbm, storage: str, steps: int = 20):
    """Error of a batch against the FP64 oracle: the two smallest drops of
    the sweep stepped together in one batch (the same kernels), `steps`
    steps from the initial state, max |f_gpu - f_oracle| / max |f_oracle|
    per colour over both cases."""
    from oracle import oracle as O
    from paper_2407_10914_gb300 import workloads as W
    cases = sorted(W.batched_droplets(count=args.batched_cases),
                   key=lambda c: c.n_nodes)[:2]
    sess = []
    for c in cases:
        s = lbm.Session(c.lattice, c.solid, c.periodic, storage)
        s.set_params(**c.params)
        s.init_state(c.phi0.astype(np.float32))
        sess.append(s)
    b = lbm.Batch(sess)
    b.step(steps)
    torch.cuda.synchronize()
    err = 0.0
    for c, s in zip(cases, sess):
        o = O.Oracle(c.lattice, c.solid, c.periodic)
        o.set_params(**c.params)
        o.init_state(c.phi0)
        o.step(steps)
        got = s.get_populations().cpu().numpy().astype(np.float64)
        fl = c.solid == 0
        for k in range(2):
            err = max(err, float(np.abs(got[k][:, fl] - o.pops[k][:, fl]).max()
                                 / np.abs(o.pops[k][:, fl]).max()))
    del b, sess
    return err, [c.name for c in cases]


def run_batched(args, torch, lbm, storage: str = "fp32"):
    """The contact-angle sweep: 96 D3Q19 sessile drops in boxes of 48^3 to
    128^3 (Scheme-I and Scheme-II, theta 30-150 deg), stepped together by
    one batch. The schedule is chosen by the autotuner (its trials are
    reported too); the value is fluid-node updates per second over all
    cases, CUDA events around `batched-steps` steps; the error against the
    FP64 oracle comes from batch_error."""
    from paper_2407_10914_gb300 import autotune
    from paper_2407_10914_gb300 import workloads as W
    cases = W.batched_droplets(count=args.batched_cases)

    def make(tile):
        sess = []
        for c in cases:
            s = lbm.Session(c.lattice, c.solid, c.periodic, storage, tile=tile)
            s.set_params(**c.params)
            s.init_state(c.phi0.astype(np.float32))
            sess.append(s)
        return lbm.Batch(sess)

    tile, tile_trials = pick_tile(args, make, 19)
    torch.cuda.empty_cache()
    t0 = time.time()
    b = make(tile)
    sess = b.sessions
    setup_s = time.time() - t0
    tune = autotune.tune(b, trial_steps=4, use_cache=False)
    stream = torch.cuda.current_stream()
    b.step(1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.batched_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.batched_steps
    if b.status() != 0:
        raise SystemExit("batched sweep: a persistent-kernel wait ran out")
    nf = b.n_fluid
    sides = sorted(int(c.solid.shape[0]) for c in cases)
    peak, _ = measured_peaks()
    upd = 2 * 2 * 19 * BYTES_POP[storage] + 4
    out = {
        "workload": f"batch{len(cases)}_sessile_drops_{storage}",
        "cases": len(cases), "box_sides": [sides[0], sides[-1]],
        "fluid_nodes": nf,
        "nodes": int(sum(c.n_nodes for c in cases)),
        "value": round(nf / (ms * 1e-3) / 1e6, 2), "unit": "MLUPS",
        "ms_per_step": round(ms, 4), "steps": args.batched_steps,
        "roofline_frac": round(upd * nf / (ms * 1e-3) / 1e9 / peak, 4),
        "bytes_per_update": upd,
        "schedule": {"mode": ["level launches", "persistent"][tune["config"][0]],
                     "threads": tune["config"][1], "chunk": tune["config"][2]},
        "tuning_ms_per_step": tune.get("trials"),
        "tile": tile_name(tile, 19),
        "tile_search_ms_per_step": tile_trials,
        "setup_s": round(setup_s, 1),
    }
    del b, sess
    torch.cuda.empty_cache()
    err, names = batch_error(args, torch, lbm, storage)
    out["error_vs_fp64_oracle"] = err
    out["error_sample"] = (f"cases {names[0]} and {names[1]} stepped together "
                           "in one batch, 20 steps from the initial state, max "
                           "relative population error")
    return out


def run_adjoint(args, torch, lbm):
    """Gradient of the smooth saturation after T steps of the imbibition
    pack (128^3, porosity 0.25, Scheme-II theta = 40 deg, g_x = 5e-6) with
    respect to theta and g_x: checkpointed forward run plus hand-written
    reverse sweep (K = 45 for T = 2000), timed with CUDA events, and the
    same derivatives by central differences of the FP32 forward run."""
    from paper_2407_10914_gb300 import workloads as W
    from paper_2407_10914_gb300.adjoint import Run
    n, T = args.adjoint_size, args.adjoint_steps
    case = W.adjoint_pack(n=(n, n, n), steps=T)
    s = lbm.Session(case.lattice, case.solid, case.periodic, "fp32")
    s.set_params(**case.params)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    run = Run(s, case.phi0, T, every=45 if T == 2000 else None)
    ev[0].record(stream)
    J = run.forward()
    ev[1].record(stream)
    dth, dg = run.backward()
    ev[2].record(stream)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])

    def sw(**over):
        p = dict(case.params)
        p.update(over)
        s.set_params(**p)
        s.init_state(case.phi0.astype(np.float32))
        s.step(T)
        return s.reduce(lbm.LBM_SW_SMOOTH)

    th0 = case.params["theta_deg"]
    g0 = case.params["g"][0]
    # central differences of the FP32 forward run over a range of steps
    sweep_th, sweep_g = {}, {}
    for hth in (0.25, 0.5, 1.0, 2.0):
        sweep_th[str(hth)] = (sw(theta_deg=th0 + hth)
                              - sw(theta_deg=th0 - hth)) / (2 * hth)
    for frac in (0.05, 0.1, 0.2, 0.4):
        hg = frac * g0
        sweep_g[str(frac)] = (sw(g=(g0 + hg, 0.0, 0.0))
                              - sw(g=(g0 - hg, 0.0, 0.0))) / (2 * hg)
    fd_th, hth = sweep_th["1.0"], 1.0
    fd_g, hg = sweep_g["0.1"], 0.1 * g0
    ad_th = dth * math.pi / 180.0  # per degree
    # the regularisation of the linearisation: (freeze_sin, c_min)
    s.set_params(**case.params)
    regs = {}
    for fz, cm in ((0.05, 1e-3), (0.02, 1e-3), (0.1, 1e-3), (0.05, 1e-4),
                   (0.05, 1e-2), (0.01, 1e-4), (0.005, 1e-5), (0.002, 1e-6),
                   (0.0, 1e-3), (0.05, 0.0), (0.0, 0.0)):
        r2 = Run(s, case.phi0, T, every=45 if T == 2000 else None,
                 freeze_sin=fz, c_min=cm)
        r2.forward()
        a_th, a_g = r2.backward()
        regs[f"{fz}/{cm}"] = {"dJ_dtheta_per_deg": a_th * math.pi / 180.0,
                              "dJ_dgx": float(a_g[0])}
    nf = s.n_fluid
    out = {
        "workload": f"adjoint_pack{n}_scheme2_T{T}",
        "fluid_nodes": nf, "steps": T, "checkpoint_every": run.K,
        "J_sw_smooth": J,
        "dJ_dtheta_per_deg": {"adjoint": ad_th, "central_fd_fp32": fd_th,
                              "h_deg": hth,
                              "rel_diff": abs(ad_th - fd_th) / abs(fd_th),
                              "fd_fp32_by_h_deg": sweep_th},
        "dJ_dgx": {"adjoint": float(dg[0]), "central_fd_fp32": fd_g,
                   "h": hg, "rel_diff": abs(dg[0] - fd_g) / abs(fd_g),
                   "fd_fp32_by_h_frac": sweep_g},
        "adjoint_by_freeze_sin_c_min": regs,
        "forward_ms": round(fwd_ms, 1), "backward_ms": round(bwd_ms, 1),
        "gradient_MLUPS": round(nf * T / ((fwd_ms + bwd_ms) * 1e-3) / 1e6, 1),
        "freeze_sin": run.freeze_sin, "c_min": run.c_min,
        "note": "regularised linearisation: Scheme-II's direction around n_w "
                "held where sin(theta') < freeze_sin, n_c's direction where "
                "|C| < c_min (the exact derivative grows without bound over "
                "long runs); the FP64 tangent-linear oracle checks the same "
                "code to 1e-3 (tests/test_gpu_adjoint.py)",
    }
    ref = stored_fd64(n, T)
    if ref:
        th_ref, g_ref = ref["dJ_dtheta_per_deg"]["0.5"], ref["dJ_dgx"]["0.1"]
        ref["rel_diff_theta"] = abs(ad_th - th_ref) / abs(th_ref)
        ref["rel_diff_gx"] = abs(float(dg[0]) - g_ref) / abs(g_ref)
        out["fd_fp64_stored"] = ref
    if args.adjoint_fd64:
        out["fd_fp64_oracle"] = adjoint_fd64(case, T, args.adjoint_fd64)
    if args.adjoint_tlm64:
        out["tlm_fp64_oracle"] = adjoint_tlm64(case, T, run.freeze_sin,
                                               run.c_min)
    return out


def stored_fd64(n: int, T: int):
    """The FP64 oracle's central differences of the gradient workload
    (tests/golden/adjoint_pack128_T2000_fd64.txt, written by
    make_adjoint_fd64.py beside it), for the 128^3, T = 2000 case only:
    {"J", "dJ_dtheta_per_deg": {h: value}, "dJ_dgx": {h: value}}."""
    p = os.path.join(ROOT, "tests", "golden", "adjoint_pack128_T2000_fd64.txt")
    if n != 128 or T != 2000 or not os.path.exists(p):
        return None
    out = {"dJ_dtheta_per_deg": {}, "dJ_dgx": {},
           "source": "tests/golden/adjoint_pack128_T2000_fd64.txt"}
    for line in open(p):
        parts = line.split()
        if len(parts) != 3 or line.startswith("#"):
            continue
        if parts[0] == "J":
            out["J"] = float(parts[2])
        elif parts[0] in ("dJ_dtheta_per_deg", "dJ_dgx"):
            out[parts[0]][parts[1]] = float(parts[2])
    ok = "0.5" in out["dJ_dtheta_per_deg"] and "0.1" in out["dJ_dgx"]
    return out if ok else None


def adjoint_tlm64(case, T: int, freeze_sin: float, c_min: float) -> dict:
    """The FP64 oracle's tangent-linear run at the full size of the
    gradient workload with the adjoint's regularisation: the same
    derivative of the same regularised linearisation, from the forward
    mode and in FP64."""
    from oracle import oracle as O
    t0 = time.time()
    t = O.TangentLinear(case.lattice, case.solid, case.periodic)
    t.set_params(**case.params)
    t.set_freeze(freeze_sin)
    t.set_cmin(c_min)
    t.init_state(case.phi0)
    t.step(T)
    J, dth, dg = t.sw()
    return {"J": J, "dJ_dtheta_per_deg": dth * math.pi / 180.0,
            "dJ_dgx": dg, "freeze_sin": freeze_sin, "c_min": c_min,
            "seconds": round(time.time() - t0, 1)}


def adjoint_fd64(case, T: int, which: str = "all") -> dict:
    """Central differences of the FP64 oracle's forward run at the full size
    of the gradient workload (about 150 s per run on 16 host cores): theta
    at h = 0.5 and 1 deg, g_x at h = 10 % of g_x ("all"); or g_x alone at
    h = 5, 10 and 20 % ("gx")."""
    from oracle import oracle as O

    def sw64(**over):
        p = dict(case.params)
        p.update(over)
        o = O.Oracle(case.lattice, case.solid, case.periodic)
        o.set_params(**p)
        o.init_state(case.phi0)
        o.step(T)
        return o.reduce(O.SW_SMOOTH)

    t0 = time.time()
    th0, g0 = case.params["theta_deg"], case.params["g"][0]
    out = {"J": sw64()}
    if which == "all":
        out["dJ_dtheta_per_deg"] = {
            str(h): (sw64(theta_deg=th0 + h) - sw64(theta_deg=th0 - h))
            / (2 * h) for h in (0.5, 1.0)}
    out["dJ_dgx"] = {}
    for frac in ((0.1,) if which == "all" else (0.05, 0.1, 0.2)):
        hg = frac * g0
        out["dJ_dgx"][str(frac)] = (sw64(g=(g0 + hg, 0.0, 0.0))
                                    - sw64(g=(g0 - hg, 0.0, 0.0))) / (2 * hg)
    out["seconds"] = round(time.time() - t0, 1)
    return out


def main():
    args = parse()
    if args.oracle_sample:
        run_oracle_sample(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

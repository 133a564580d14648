#!/usr/bin/env python
"""Benchmark of the Contact Dynamics hot path on GB300.

A step is one full CD time step (detection, colouring and ordering, free
flight, persistent colour-sweep impulse solve to the convergence test, Euler
update) of the dense 2D workload: 100,000 frictional discs, radii U[0.8, 1.2],
mu = 0.3, a gravity-deposited pile in a periodic-x box of width
sqrt(sum pi r^2 / 0.80), top wall pushed down at 1e-3, dt = 1e-3, Gauss-Seidel
until the relative change of the mean impulse is below 1e-6 or 1000 sweeps.

Prints one JSON line.  ``value`` is contact updates per second (sum over the
timed steps of sweeps x contacts, divided by the device time of those steps,
measured with CUDA events recorded on the library's stream), aggregated over
all ranks.  ``--impl reference`` times the FP64 CPU oracle on a bounded
sample of the same workload instead.

Multi-GPU (torchrun, one rank per GPU): every rank steps its own packing
(seed offset by rank); no data-path collective; weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "contact updates/s and CD steps/s at residual 1e-6 (plain vs batched/adjoint)"
UNIT = "contact updates/s"
WORKLOAD = "dense_biaxial_discs_2d"
# algorithmic bytes of one colour sweep: per contact record (ids 8, normal 16,
# g/dt 8, m_n 8, m_t 8, impulse read 16 + write 16) and per particle (v, w
# read + write 2 x 24, inv_m, r, r/I 24); FP32 halves the real-valued parts
BYTES_PER_CONTACT = {"f64": 80, "f32": 44}
BYTES_PER_PARTICLE = {"f64": 72, "f32": 36}
# 3D: contact record ids 8, geometry 32, (m_n, m_t) 16, impulse read 32 +
# write 32; particle v, w read + write 2 x 64, static 32 (FP32 halves the reals)
BYTES_PER_CONTACT_3D = {"f64": 120, "f32": 64}
BYTES_PER_PARTICLE_3D = {"f64": 160, "f32": 80}
# algorithmic FP64 flops of one 2D contact update as the sweep kernel writes
# it: relative velocity 2 + 2 (u_n) + 7 (u_t), P_n 3, mu P_n 1, P_t 2,
# impulse change 2, its vector 6, both bodies' velocities 12, |P| 4 + 1 (the
# square root counted as one)
FLOPS_PER_UPDATE_2D = 42
# 3D (FMA = 2): lever sums 9, relative velocity 15, u_n 5, tangential part 6,
# P_n 3, trial P_t 6, mu P_n 1, cone test 6, impulse change 4, its vector 6,
# n x dP 9, both bodies' v and w 24, |P| 7 (+ square root; the cone scaling
# of sliding contacts is not counted)
FLOPS_PER_UPDATE_3D = 101
# algorithmic bytes of one detection (cell list, pair test, geometry and warm
# start; the library's "detect" phase): per particle the position and radius
# read (8 D + 8); per contact the key-order record written (key 8, normal 24,
# gap 8, m_n 8, m_t 8, impulse 8 x (D + 1)) and the previous set's key and
# impulse read by the warm start (8 + 8 x (D + 1), counted at the new set's
# size)
def detect_bytes_model(dim):
    pw = 2 if dim == 2 else 4
    return 64 + 16 * pw, 8 * dim + 8


# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA/clk x 2
# flops x 2.07 GHz (nominal 1.25 TFLOP/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f64", "f32"], default="f64")
    ap.add_argument("--workload", choices=["dense_biaxial_discs_2d", "sphere_gas_3d"],
                    default="dense_biaxial_discs_2d",
                    help="the 2D dense pile (default) or the 1e6-sphere 3D gas (its own run; no batched or "
                         "adjoint legs)")
    ap.add_argument("--n-discs", "--n", dest="n", type=int, default=None,
                    help="particles (default 100,000 discs or 1,000,000 spheres)")
    ap.add_argument("--max-sweeps", type=int, default=1000)
    ap.add_argument("--alpha", type=float, default=1e-6)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--domains", type=int, nargs=3, default=[1, 1, 1], metavar=("NX", "NY", "NZ"),
                    help="domain-wise update of Sec. 3.1: slabs per axis (1 1 1: Gauss-Seidel)")
    ap.add_argument("--merge-last-colour", type=int, default=4,
                    help="1: run the three (else two) last colours as one phase when the last class is small; 2: two at most; "
                         "4: as 1 after a solve of at least 64 sweeps (the default); 0: off")
    ap.add_argument("--sphere-steps", type=int, default=5,
                    help="timed steps of the 1e6-sphere 3D gas leg (rank 0 at N=1 only; 0: skip)")
    ap.add_argument("--batched-steps", type=int, default=3,
                    help="timed steps of the 512-packing batched workload (0: skip)")
    ap.add_argument("--packings", type=int, default=512)
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner and use the default 512 x 1 sweep grid")
    ap.add_argument("--adjoint-steps", type=int, default=200,
                    help="steps of the differentiated settling rollout (0: skip the adjoint leg)")
    ap.add_argument("--fp32-steps", type=int, default=None,
                    help="timed steps of the FP32 leg on the same pile (default --steps; 0: skip)")
    ap.add_argument("--dilute-steps", type=int, default=200,
                    help="timed steps of the 1,000-disc dilute leg (0: skip)")
    ap.add_argument("--converge-cap", type=int, default=100000,
                    help="sweep cap of the untimed steps that measure the sweeps to residual 1e-6 (0: skip)")
    ap.add_argument("--mixed-scan", type=int, nargs="*", default=None, metavar="N",
                    help="instead of the benchmark: the iterations N_I the mixed update of Sec. 2.3 needs against "
                         "its parallel fraction p, both readings of the parallel subset, on loaded piles of N discs")
    ap.add_argument("--cpu-sweeps", type=int, default=30,
                    help="sweep cap of the oracle's bounded sample step")
    return ap.parse_args()


def workload(args, rank):
    from paper_1104_3516_gb300 import workloads as W
    if args.workload == "sphere_gas_3d":
        wl = W.sphere_gas(seed=1107 + rank, n=args.n or 1_000_000)
    else:
        wl = W.dense_biaxial_discs(seed=1106 + rank, n=args.n or 100_000)
    wl.max_sweeps = args.max_sweeps
    wl.alpha = args.alpha
    return wl


def config(args, wl, extra=None):
    if wl.dim == 3:
        c = {"workload": "sphere_gas_3d", "n_spheres": wl.n, "packing_fraction_gas": 0.3, "mu": wl.mu,
             "dt": wl.dt, "gravity": 1.0, "floor": "100 x 100, 4 side walls", "v0": "N(0, 0.1)",
             "rotations": True}
    else:
        c = {"workload": WORKLOAD, "n_discs": wl.n, "packing_fraction_box": 0.80, "mu": wl.mu, "dt": wl.dt,
             "gravity": 1.0, "top_wall_speed": 1e-3, "periodic": "x"}
    c.update({"criterion": "global |dR_avg|/(R^j+R^j-1)", "alpha": args.alpha, "max_sweeps": args.max_sweeps,
              "warm_start": True,
              "order": "colour (largest degree first, then hash)",
              "domains": list(args.domains),
              "merge_last_colour": args.merge_last_colour,
              "l2": "flushed (512 MiB write) before every timed step"})
    if extra:
        c.update(extra)
    return c


def host_cpu():
    """The host CPU the oracle is timed on: its model (from /proc/cpuinfo where
    it names one, else the architecture) and the number of logical CPUs."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key, _, val = line.partition(":")
                if key.strip().lower() in ("model name", "hardware") and val.strip():
                    model = val.strip()
                    break
    except OSError:
        pass
    return {"cpu": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def profiled_traffic(kernel, precision, n):
    """DRAM bytes per launch from the committed ncu summary, or None if the
    sweep kernel's source changed since the counters were taken."""
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_1104_3516_gb300", "csrc", "cd_sweep.cu"), "rb").read()
        sha = hashlib.sha256(src).hexdigest()[:16]
        for line in open(os.path.join(ROOT, "profiles", "k_sweep_traffic.txt")):
            if line.startswith("#") or not line.strip():
                continue
            f = dict(kv.split("=", 1) for kv in line.split())
            if (f.get("kernel") == kernel and f.get("precision") == precision and int(f.get("n", -1)) == n
                    and f.get("src_sha256") == sha):
                return float(f["traffic_bytes_per_launch"])
    except Exception:
        return None
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for name, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "samples": len(sm), "reasons": sorted(reasons)}


def dist_init(args, backend=None):
    """Joins the process group torchrun set up (RANK / WORLD_SIZE /
    MASTER_* in the environment); returns (rank, world size, local rank).
    The CUDA arm uses NCCL for its two timing reductions, the oracle arm gloo."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        return dist.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return 0, 1, 0


def reduce_max_sum(vals_max, vals_sum, ws, device):
    """Max over ranks of the times, sum over ranks of the work: the only
    cross-rank traffic of the benchmark (no data-path collective)."""
    if ws == 1:
        return vals_max, vals_sum
    import torch
    import torch.distributed as dist
    a = torch.tensor(vals_max, dtype=torch.float64, device=device)
    b = torch.tensor(vals_sum, dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------

def oracle_steps(wl, steps, sweep_cap, colour_order=False):
    """Times `steps` oracle time steps (random sequential order, the paper's
    scheme, or with colour_order the GPU's colour order) of the workload with
    the sweep cap lowered to `sweep_cap`; returns (contact updates, seconds,
    sweeps, contacts)."""
    import oracle as O
    p = O.make_params(dim=wl.dim, dt=wl.dt, mu=wl.mu, gravity=wl.gravity, box_lo=wl.box_lo, box_hi=wl.box_hi,
                      periodic=wl.periodic, wall_mask=wl.wall_mask, wall_vel=np.asarray(wl.wall_vel).reshape(18),
                      delta=wl.delta, alpha=wl.alpha, criterion=O.CRIT_GLOBAL_REL, max_sweeps=sweep_cap,
                      order=O.ORDER_COLOUR if colour_order else O.ORDER_RANDOM, seed=wl.seed)
    s = O.OracleSystem(p, wl.x, wl.v, wl.w, wl.r, wl.inv_m, wl.inv_I, np.asarray(wl.wall_pos, dtype=np.float64),
                       cap=6 * wl.n)
    upd, sweeps = 0, 0
    t0 = time.perf_counter()
    for _ in range(steps):
        st = s.step()
        upd += st["sweeps"] * s.nc
        sweeps += st["sweeps"]
    return upd, time.perf_counter() - t0, sweeps, s.nc


def run_reference(args):
    rank, ws, _ = dist_init(args)
    if rank != 0:
        return
    wl = workload(args, 0)
    oracle_steps(wl, args.warmup, args.cpu_sweeps) if args.warmup > 0 else None
    upd, sec, sweeps, nc = oracle_steps(wl, args.steps, args.cpu_sweeps)
    value = upd / sec
    sample = (f"{args.steps} oracle time steps of the {wl.n}-particle workload, random sequential order, sweep cap "
              f"lowered to {args.cpu_sweeps} ({sweeps} sweeps over {nc} contacts)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(args, wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The CUDA path
# ---------------------------------------------------------------------------

def sweep_bytes_model(dim, precision):
    """Compulsory bytes of one colour sweep: per contact record and per particle."""
    if dim == 3:
        return BYTES_PER_CONTACT_3D[precision], BYTES_PER_PARTICLE_3D[precision]
    return BYTES_PER_CONTACT[precision], BYTES_PER_PARTICLE[precision]


def detect_roofline(dim, detect_ms, n, contacts):
    """HBM view of the detection phase: its algorithmic bytes over its
    CUDA-event time (`detect_ms` summed over the steps whose contact counts
    are `contacts`)."""
    bpc, bpp = detect_bytes_model(dim)
    peak, peak_kind = peaks()
    byt = sum(bpc * c + bpp * n for c in contacts)
    gbs = byt / (detect_ms / 1e3) / 1e9 if detect_ms > 0 else 0.0
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "kernels": "k_cell_count .. k_pair_count, k_pair_emit .. k_commit (the detect phase)",
            "avg_phase_ms": detect_ms / max(len(contacts), 1), "peak_source": f"{peak_kind} HBM copy bandwidth",
            "bytes_model": f"{bpc} B x contacts + {bpp} B x particles per detection"}


def timed_steps(sysg, wl, steps, flush, precision):
    """`steps` CD time steps of a system created with timing=1, the L2 flushed
    (512 MiB written) before each; device times from the library's CUDA events
    on its stream."""
    bpc, bpp = sweep_bytes_model(wl.dim, precision)
    out = {"upd": 0, "sweeps": 0, "launches": 0, "not_conv": 0, "sweep_bytes": 0.0, "ncs": [], "colours": [],
           "phases": [], "ph": {"detect": 0.0, "colour_order_pack": 0.0, "sweep": 0.0, "integrate": 0.0}}
    for _ in range(steps):
        flush.zero_()
        st = sysg.step(1)
        out["upd"] += st["total_contact_updates"]
        out["sweeps"] += st["total_sweeps"]
        out["launches"] += st["kernel_launches"]
        out["not_conv"] += st["n_not_converged"]
        nc = st["last"]["n_contacts"]
        out["ncs"].append(nc)
        out["colours"].append(st["last"]["n_colours"])
        out["phases"].append(st["last"]["n_phases"])
        out["sweep_bytes"] += st["total_sweeps"] * (nc * bpc + wl.n * bpp)
        for k in out["ph"]:
            out["ph"][k] += st["phase_ms"][k]
    return out


def graph_steps(g, steps, flush, stream):
    """`steps` steps of a system created with use_graph=1 (each replayed from
    the captured CUDA graph).  The counts come from a first pass with
    statistics; the system is then put back to its checkpoint and the same
    steps (bit-identical) are replayed without a host synchronisation inside,
    the L2 flushed before each, every step bracketed by CUDA events on the
    system's stream.  Returns (device ms, summed counts)."""
    import torch
    ck = g.save_checkpoint()
    cnt = {"upd": 0, "sweeps": 0, "not_conv": 0, "max_sweeps": 0, "launches": 0, "contacts": 0}
    for _ in range(steps):
        st = g.step(1)
        cnt["upd"] += st["total_contact_updates"]
        cnt["sweeps"] += st["total_sweeps"]
        cnt["not_conv"] += st["n_not_converged"]
        cnt["max_sweeps"] = max(cnt["max_sweeps"], st["max_sweeps_in_step"])
        cnt["launches"] += st["kernel_launches"]
        cnt["contacts"] = st["last"]["n_contacts"]
    g.load_checkpoint(ck)
    evs = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(1, stats=False)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs), cnt


def run_ours(args):
    import torch
    rank, ws, local = dist_init(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_1104_3516_gb300 import cd
    wl = workload(args, rank)
    prec = cd.CD_FP64 if args.precision == "f64" else cd.CD_FP32
    stream = torch.cuda.current_stream(device)
    shape, tuned = {}, None
    plain = list(args.domains) == [1, 1, 1]
    if not args.no_autotune and plain:
        # block shape of the sweep grid chosen by timing short solves of this system (untimed)
        from paper_1104_3516_gb300 import autotune
        shape, table = autotune.tune(wl, precision=prec, device=device, max_contacts=4 * wl.n,
                                     candidates=[dict(sweep_threads=t, sweep_blocks_per_sm=b)
                                                 for t, b in autotune.BLOCK_SHAPES])
        tuned = {"choice": shape, "ms_per_sweep": [[c, m] for c, m in table]}
    sysg = cd.CDSystem(wl, device=device, precision=prec, criterion=cd.CD_CONV_GLOBAL_REL, max_contacts=4 * wl.n,
                       timing=1, stream=stream,
                       domains=tuple(args.domains), merge_last_colour=args.merge_last_colour, **shape)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=device)

    for _ in range(args.warmup):
        flush.zero_()
        sysg.step(1)

    barrier(ws)
    torch.cuda.synchronize(device)
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.perf_counter()
    bpc, bpp = sweep_bytes_model(wl.dim, args.precision)
    flops_per_update = FLOPS_PER_UPDATE_3D if wl.dim == 3 else FLOPS_PER_UPDATE_2D
    t = timed_steps(sysg, wl, args.steps, flush, args.precision)
    torch.cuda.synchronize(device)
    barrier(ws)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    upd, sweeps, launches, not_conv = t["upd"], t["sweeps"], t["launches"], t["not_conv"]
    ph, sweep_bytes, ncs, colours, phases = t["ph"], t["sweep_bytes"], t["ncs"], t["colours"], t["phases"]

    dev_ms = sum(ph.values())
    (dev_ms_max, wall_max), (upd_sum, steps_sum) = reduce_max_sum([dev_ms, wall], [float(upd), float(args.steps)],
                                                                  ws, device)
    value = upd_sum / (dev_ms_max / 1e3)
    steps_per_s = steps_sum / (dev_ms_max / 1e3)

    peak, peak_kind = peaks()
    kname = "k_sweep"
    if list(args.domains) != [1, 1, 1]:
        kname = "k_sweep_domains"
    kname += f"<{wl.dim},{'double' if args.precision == 'f64' else 'float'}>"
    sweep_s = ph["sweep"] / 1e3
    gbs = sweep_bytes / sweep_s / 1e9 if sweep_s > 0 else 0.0
    hbm_view = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                "peak_source": f"{peak_kind} HBM copy bandwidth",
                "bytes_model": f"per sweep {bpc} B x contacts + {bpp} B x particles"}
    traffic = profiled_traffic(kname, args.precision, wl.n)
    if args.precision == "f64":
        tf = flops_per_update * upd / sweep_s / 1e12 if sweep_s > 0 else 0.0
        roofline = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": kname,
                    "peak_source": "FP64 unit count x clock (152 SMs x 2 FMA/clk x 2 x 2.07 GHz)",
                    "flops_model": f"{flops_per_update} FP64 flops per contact update",
                    "avg_launch_ms": ph["sweep"] / max(args.steps, 1), "hbm_view": hbm_view}
    else:
        roofline = dict(hbm_view, traffic=traffic, kernel=kname, avg_launch_ms=ph["sweep"] / max(args.steps, 1))
    roofline["detect_view"] = detect_roofline(wl.dim, ph["detect"], wl.n, t["ncs"])

    batched = None
    if args.batched_steps > 0 and wl.dim == 2:
        batched = run_batched(args, device, rank, flush, ws)

    adjoint = None
    if args.adjoint_steps > 0 and args.precision == "f64" and wl.dim == 2:
        adjoint = run_adjoint(args, device, rank, flush)

    sphere = None
    if args.sphere_steps > 0 and wl.dim == 2 and ws == 1:
        sphere = run_sphere_gas(args, device, flush)

    fp32 = dilute = converge = None
    fp32_steps = args.steps if args.fp32_steps is None else args.fp32_steps
    if fp32_steps > 0 and args.precision == "f64" and wl.dim == 2 and ws == 1:
        a32 = argparse.Namespace(**{**vars(args), "steps": fp32_steps})
        fp32 = run_fp32(a32, wl, device, flush, shape)
    if args.dilute_steps > 0 and wl.dim == 2 and ws == 1:
        dilute = run_dilute(args, device, flush)
    if args.converge_cap > 0 and args.precision == "f64" and wl.dim == 2 and ws == 1:
        converge = run_converge(args, sysg, wl, device, shape)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, sysg, wl, device, ws)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        o_upd, o_sec, o_sweeps, o_nc = oracle_steps(wl, 1, args.cpu_sweeps)
        c_upd, c_sec, _, _ = oracle_steps(wl, 1, args.cpu_sweeps, colour_order=True)
        cpu = {"value": o_upd / o_sec, "unit": UNIT, "cores": 1, "kind": "oracle",
               "colour_order_value": c_upd / c_sec,
               "sample": f"1 oracle time step of the same {wl.n}-particle packing, random sequential order, sweep cap "
                         f"{args.cpu_sweeps} ({o_sweeps} sweeps over {o_nc} contacts, {o_sec:.1f} s)",
               **host_cpu()}

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms_max / max(args.steps, 1), "steps_per_s": steps_per_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic (seeded gravity deposition)",
            "config": config(args, wl, {"mean_contacts": float(np.mean(ncs)), "mean_colours": float(np.mean(colours)),
                                        "mean_phases_per_sweep": float(np.mean(phases)),
                                        "sweeps_per_step": sweeps / max(args.steps, 1),
                                        "steps_not_converged": not_conv, "parallelism": f"replicas x{ws}"}),
            "phase_ms_per_step": {k: v / max(args.steps, 1) for k, v in ph.items()},
            "wall_s": wall_max, "roofline": roofline, "autotune": tuned, "batched": batched, "adjoint": adjoint,
            "sphere_gas_3d": sphere, "fp32": fp32, "dilute_discs_2d": dilute, "at_residual_1e-6": converge,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_fp32(args, wl, device, flush, shape):
    """The same 1e5-disc pile and convergence test with the sweep in FP32
    (contact records and sweep-time velocities in FP32; the residual
    reduction and the integration in FP64): warm-up, then `steps` timed
    steps with the L2 flushed before each."""
    import torch
    from paper_1104_3516_gb300 import cd
    stream = torch.cuda.current_stream(device)
    g = cd.CDSystem(wl, device=device, precision=cd.CD_FP32, criterion=cd.CD_CONV_GLOBAL_REL,
                    max_contacts=4 * wl.n, timing=1, stream=stream, merge_last_colour=args.merge_last_colour,
                    **shape)
    for _ in range(args.warmup):
        flush.zero_()
        g.step(1)
    torch.cuda.synchronize(device)
    t = timed_steps(g, wl, args.steps, flush, "f32")
    ms = sum(t["ph"].values())
    sweep_s = t["ph"]["sweep"] / 1e3
    peak, peak_kind = peaks()
    gbs = t["sweep_bytes"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
    bpc, bpp = sweep_bytes_model(2, "f32")
    out = {"value": t["upd"] / (ms / 1e3), "unit": UNIT, "dtype": "f32", "steps": args.steps,
           "ms_per_step": ms / args.steps, "steps_per_s": args.steps / (ms / 1e3),
           "sweeps_per_step": t["sweeps"] / args.steps, "steps_not_converged": t["not_conv"],
           "mean_phases_per_sweep": float(np.mean(t["phases"])),
           "phase_ms_per_step": {k: v / args.steps for k, v in t["ph"].items()},
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "kernel": "k_sweep<2,float>", "peak_source": f"{peak_kind} HBM copy bandwidth",
                        "bytes_model": f"per sweep {bpc} B x contacts + {bpp} B x particles",
                        "note": "the pile is L2-resident: the sweep is bound by the latency of its colour phases, "
                                "not by HBM"},
           "workload": "the same dense_biaxial_discs_2d packing as the headline line"}
    del g
    return out


def run_dilute(args, device, flush):
    """The 1,000-disc dilute configuration: discs r ~ U[0.8, 1.2], mu = 0.3,
    random sequential placement at packing fraction 0.40 in a box 40 wide
    with floor and side walls, gravity 1, dt = 1e-3, the same convergence
    test; 3 untimed steps (the first captures the step's CUDA graph), then
    `dilute_steps` steps replayed from the graph, the L2 flushed before each."""
    import torch
    from paper_1104_3516_gb300 import cd, workloads as W
    wl = W.dilute_discs(seed=1105, n=1000)
    wl.max_sweeps = args.max_sweeps
    wl.alpha = args.alpha
    stream = torch.cuda.Stream(device=device)
    g = cd.CDSystem(wl, device=device, criterion=cd.CD_CONV_GLOBAL_REL, use_graph=1, stream=stream,
                    merge_last_colour=args.merge_last_colour)
    g.step(3)
    ms, cnt = graph_steps(g, args.dilute_steps, flush, stream)
    n = args.dilute_steps
    out = {"value": cnt["upd"] / (ms / 1e3), "unit": UNIT, "dtype": "f64", "discs": wl.n, "steps": n,
           "ms_per_step": ms / n, "steps_per_s": n / (ms / 1e3), "sweeps_per_step": cnt["sweeps"] / n,
           "max_sweeps_in_step": cnt["max_sweeps"], "steps_not_converged": cnt["not_conv"],
           "contacts_last_step": cnt["contacts"], "kernel_launches_per_step": cnt["launches"] / n,
           "steps_from_cuda_graph": True,
           "workload": "dilute_discs_2d: 1000 discs, RSA at packing fraction 0.40 in a box 40 wide, floor and "
                       "side walls, v0 = 0, mu 0.3, 200 steps of dt 1e-3"}
    del g
    return out


def run_converge(args, sysg, wl, device, shape):
    """Sweeps the headline pile needs to reach the 1e-6 residual: a system
    over the state the timed steps left (positions, velocities, walls), with
    the sweep cap raised to `converge_cap`, stepped twice (untimed for the
    headline; device time recorded): the first solve starts from zero
    impulses, the second from the first's (warm start, as in the timed
    steps), so the second is one CD step at residual 1e-6."""
    import torch
    from paper_1104_3516_gb300 import cd, workloads as W
    s = sysg.state()
    wl2 = W.Workload(**{**wl.__dict__})
    wl2.x, wl2.v, wl2.w = s["x"], s["v"], s["w"]
    wl2.wall_pos = np.asarray(sysg.walls(), dtype=np.float64)
    wl2.max_sweeps = args.converge_cap
    stream = torch.cuda.current_stream(device)
    g = cd.CDSystem(wl2, device=device, precision=cd.CD_FP64, criterion=cd.CD_CONV_GLOBAL_REL,
                    max_contacts=4 * wl.n, timing=1, stream=stream, merge_last_colour=args.merge_last_colour,
                    **shape)
    out = {"sweep_cap": args.converge_cap, "alpha": args.alpha}
    for name in ("cold_start", "warm_start"):
        st = g.step(1)
        ms = sum(st["phase_ms"].values())
        out[name] = {"sweeps": st["total_sweeps"], "converged": st["n_not_converged"] == 0, "step_ms": ms,
                     "sweep_ms": st["phase_ms"]["sweep"], "residual": st["last"]["residual"],
                     "steps_per_s": 1e3 / ms if ms > 0 else None}
    del g
    return out


def run_batched(args, device, rank, flush, ws=1):
    """The batched workload: independent 2D packings (disc counts log-uniform
    in [200, 20000], mu ~ U[0.1, 0.6], each a pile settled under gravity in a
    periodic-x box sized to packing fraction 0.5), all stepped by one batched
    system.  Under torchrun the packings are split across the ranks: rank r
    takes the contiguous index range shard_range(packings, r, N) of the same
    seeded batch (disjoint, covering it), and the line reports the work of all
    ranks over the slowest rank's time (no data-path collective)."""
    import torch
    from paper_1104_3516_gb300 import cd, workloads as W
    batch = W.batched_settling(seed=1108, n_packings=args.packings, shard=(rank, ws))
    for b in batch:
        b.max_sweeps = args.max_sweeps
        b.alpha = args.alpha
    prec = cd.CD_FP64 if args.precision == "f64" else cd.CD_FP32
    shape, tuned = {}, None
    if not args.no_autotune:
        from paper_1104_3516_gb300 import autotune
        shape, table = autotune.tune(batch[0], batch=batch, precision=prec, device=device, steps=1,
                                     max_contacts=6 * sum(b.n for b in batch),
                                     candidates=[dict(sweep_threads=t, sweep_blocks_per_sm=b)
                                                 for t, b in autotune.BLOCK_SHAPES])
        tuned = {"choice": shape, "ms_per_sweep": [[c, m] for c, m in table]}
    # steps replayed from a captured CUDA graph (use_graph needs its own stream and timing 0);
    # the batch's working set (~1 GB) is larger than L2, so the steps run back to back
    stream = torch.cuda.Stream(device=device)
    g = cd.CDSystem(batch[0], device=device, batch=batch, precision=prec, criterion=cd.CD_CONV_GLOBAL_REL,
                    max_contacts=6 * sum(b.n for b in batch), use_graph=1, stream=stream, **shape)
    g.step(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    barrier(ws)
    e0.record(stream)
    st = g.step(args.batched_steps)
    e1.record(stream)
    e1.synchronize()
    ms_rank = e0.elapsed_time(e1)
    upd_rank, sweeps, nc = st["total_contact_updates"], st["max_sweeps_in_step"], st["last"]["n_contacts"]
    (ms,), (upd,) = reduce_max_sum([ms_rank], [float(upd_rank)], ws, device)
    stats = g.packing_stats()
    sw = np.array([p["sweeps"] for p in stats])
    lo, hi = W.shard_range(args.packings, rank, ws)
    out = {"value": upd / (ms / 1e3), "unit": UNIT, "dtype": args.precision, "packings": args.packings,
           "scaling": "strong" if ws > 1 else None,
           "shard": f"rank 0 of {ws}: packings [{lo}, {hi}) of {args.packings} (ranks take disjoint contiguous "
                    f"index ranges)",
           "particles_rank0": int(sum(b.n for b in batch)),
           "contacts_rank0": nc, "steps": args.batched_steps, "ms_per_step": ms / args.batched_steps,
           "steps_per_s": args.batched_steps / (ms / 1e3), "max_sweeps_in_step": int(sweeps),
           "steps_from_cuda_graph": True, "kernel_launches_per_step": st["kernel_launches"] / args.batched_steps,
           "sweeps_last_step": {"min": int(sw.min()), "median": float(np.median(sw)), "max": int(sw.max())},
           "packings_converged_last_step": int(sum(p["converged"] for p in stats)), "autotune": tuned,
           "workload": "batched_settling_2d: disc counts log-uniform [200, 20000], mu ~ U[0.1, 0.6], "
                       "gravity-settled piles in periodic-x boxes at packing fraction 0.5"}
    if args.precision == "f64":
        # on the whole step's device time (detection and colouring included): a lower bound for the sweep
        out["fp64_tflops_whole_step"] = FLOPS_PER_UPDATE_2D * upd / (ms / 1e3) / 1e12
        out["alu_frac_whole_step"] = out["fp64_tflops_whole_step"] / FP64_PEAK_TFLOPS
    del g
    torch.cuda.empty_cache()
    return out


def run_sphere_gas(args, device, flush):
    """The 3D configuration alongside the 2D line: 1,000,000 spheres (radii
    U[0.8, 1.2], mu = 0.5, rotations) falling as a gas at packing fraction
    0.3 (v0 ~ N(0, 0.1)) onto a 100 x 100 floor with four side walls, FP64,
    the same convergence test; one untimed step, then `sphere_steps` timed
    steps with the L2 flushed before each."""
    import torch
    from paper_1104_3516_gb300 import cd, workloads as W
    wl = W.sphere_gas(seed=1107, n=1_000_000)
    wl.max_sweeps = args.max_sweeps
    wl.alpha = args.alpha
    g = cd.CDSystem(wl, device=device, precision=cd.CD_FP64, criterion=cd.CD_CONV_GLOBAL_REL, timing=1,
                    max_contacts=8 * wl.n)
    flush.zero_()
    g.step(1)
    upd = sweeps = 0
    ph = {}
    colours, ncs = [], []
    sweep_bytes = 0.0
    bpc, bpp = sweep_bytes_model(3, "f64")
    for _ in range(args.sphere_steps):
        flush.zero_()
        st = g.step(1)
        upd += st["total_contact_updates"]
        sweeps += st["total_sweeps"]
        sweep_bytes += st["total_sweeps"] * (st["last"]["n_contacts"] * bpc + wl.n * bpp)
        for k, v in st["phase_ms"].items():
            ph[k] = ph.get(k, 0.0) + v
        colours.append(st["last"]["n_colours"])
        ncs.append(st["last"]["n_contacts"])
    ms = sum(ph.values())
    sweep_s = ph["sweep"] / 1e3
    peak, peak_kind = peaks()
    gbs = sweep_bytes / sweep_s / 1e9 if sweep_s > 0 else 0.0
    tf = FLOPS_PER_UPDATE_3D * upd / sweep_s / 1e12 if sweep_s > 0 else 0.0
    bpc, bpp = sweep_bytes_model(3, "f64")
    roofline = {"bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tf / FP64_PEAK_TFLOPS, "kernel": "k_sweep<3,double>",
                "peak_source": "FP64 unit count x clock (152 SMs x 2 FMA/clk x 2 x 2.07 GHz)",
                "flops_model": f"{FLOPS_PER_UPDATE_3D} FP64 flops per contact update",
                "avg_launch_ms": ph["sweep"] / args.sphere_steps,
                "hbm_view": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                             "peak_source": f"{peak_kind} HBM copy bandwidth",
                             "bytes_model": f"per sweep {bpc} B x contacts + {bpp} B x particles"},
                "detect_view": detect_roofline(3, ph["detect"], wl.n, ncs)}
    out = {"value": upd / (ms / 1e3), "unit": UNIT, "spheres": wl.n, "steps": args.sphere_steps, "roofline": roofline,
           "ms_per_step": ms / args.sphere_steps, "steps_per_s": args.sphere_steps / (ms / 1e3),
           "phase_ms_per_step": {k: v / args.sphere_steps for k, v in ph.items()},
           "sweeps_per_step": sweeps / args.sphere_steps, "contacts": ncs[-1], "colours": colours,
           "dtype": "f64", "workload": "sphere_gas_3d: 1e6 spheres, gas at packing fraction 0.3, v0 ~ N(0, 0.1), "
                                       "mu 0.5, 100 x 100 floor with 4 side walls, rotations"}
    del g
    torch.cuda.empty_cache()
    return out


def run_adjoint(args, device, rank, flush, every=20, adj_alpha=1e-10):
    """The differentiated rollouts, with a checkpoint every 20 steps, 10,000
    discs (radii U[0.8, 1.2], mu = 0.3, gravity 1):

    * settling (`adjoint_steps` steps, 200 by default): a jittered lattice at
      packing fraction 0.5 in a box with floor and side walls, initial
      velocities N(0, 0.05), falling under gravity;
    * settled pile (supplementary, solver-heavy, at most 40 steps): the same
      discs deposited into a loaded pile on a floor, periodic in x, so that
      every step solves a hyperstatic contact network;
    * sliding pyramids (supplementary, friction-dominated, `adjoint_steps`
      steps): 3,334 pyramids of three discs (10,002 discs) on a floor moving
      sideways at 1 under them, periodic in x, at rest: the base discs slide
      on the floor all along, so both losses depend on mu; dL/dmu is checked
      against central differences of four more forward rollouts (mu +- 1e-4,
      mu +- 2e-4), Richardson-extrapolated.  The floor pressure carries ~4e-9
      of rounding noise from the trajectory and a contact opens at mu + 4e-4,
      so its difference quotient resolves only ~1e-4; the packing height's
      resolves ~1e-7.

    Two losses of the final state are differentiated with respect to mu and
    all initial velocities: the floor pressure of the last step and the
    packing height (top of the highest disc).  Each backward pass reloads the
    checkpoints newest first, re-steps the segment and back-propagates
    through every step."""
    import torch
    from paper_1104_3516_gb300 import cd, workloads as W
    cases = {"settling": (W.settling_discs(seed=1109 + rank, n=10_000), args.adjoint_steps,
                          "settling_discs_2d: jittered lattice at packing fraction 0.5, floor and side walls, "
                          "v0 ~ N(0, 0.05)"),
             "settled_pile": (W.settled_pile(1109 + rank, 10_000), min(args.adjoint_steps, 40),
                              "settled_pile_2d (supplementary): gravity-deposited pile, floor, periodic x, v0 = 0"),
             "sliding_pyramids": (W.sliding_pyramids(1113 + rank, 3334), args.adjoint_steps,
                                  "sliding_pyramids_2d (supplementary): 3,334 three-disc pyramids on a floor moving "
                                  "sideways at 1, periodic x, v0 = 0")}
    out = {"checkpoint_every": every, "adjoint_alpha": adj_alpha, "n_discs": 10_000, "mu": 0.3}
    for cname, (wl, steps, desc) in cases.items():
        # the pyramids' forward solves sweep 150 times per step (converged: ~40 reach 1e-13), the same
        # in every run, so that central differences resolve dL/dmu
        fd = cname == "sliding_pyramids"
        out[cname] = adjoint_case(args, device, flush, wl, desc, every, adj_alpha, steps,
                                  fd_h=1e-4 if fd else None, fixed_sweeps=150 if fd else None)
    torch.cuda.empty_cache()
    return out


def adjoint_case(args, device, flush, wl, desc, every, adj_alpha, steps, compliance=0.0, fd_h=None,
                 fixed_sweeps=None):
    import torch
    from paper_1104_3516_gb300 import cd
    wl.max_sweeps = args.max_sweeps if fixed_sweeps is None else fixed_sweeps
    wl.alpha = args.alpha
    crit = cd.CD_CONV_GLOBAL_REL if fixed_sweeps is None else cd.CD_CONV_NONE
    T = steps
    width = float(wl.box_hi[0] - wl.box_lo[0])
    # steps replayed from a captured CUDA graph (one step = ~25 launches)
    g = cd.CDSystem(wl, device=device, criterion=crit, tape_steps=every,
                    adjoint_compliance=compliance, use_graph=1, stream=torch.cuda.Stream(device=device))
    stream = g.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    torch.cuda.synchronize(device)
    e0.record(stream)
    segs = []
    done = fwd_upd = fwd_sweeps = 0
    last = None
    while done < T:
        m = min(every, T - done)
        segs.append((g.save_checkpoint(), m))
        st = g.step(m)
        fwd_upd += st["total_contact_updates"]
        fwd_sweeps += st["total_sweeps"]
        last = st["last"]
        done += m
    e1.record(stream)
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    final = g.save_checkpoint()
    n = wl.n
    y = g.pos.view(n, 2)[:, 1] + g.radius
    top = int(torch.argmax(y))
    losses = {"floor_pressure": (float(last["wall_force"][2]) / width, None, [0, 0, 1.0 / width, 0, 0, 0]),
              "packing_height": (float(y[top]), top, None)}
    out = {"workload": desc, "steps": T, "adjoint_compliance": compliance, "steps_from_cuda_graph": True,
           "forward_test": ("fixed sweeps" if fixed_sweeps else f"global residual {wl.alpha}"),
           "forward_max_sweeps": wl.max_sweeps,
           "forward_ms_per_step": fwd_ms / T, "forward_sweeps_per_step": fwd_sweeps / T,
           "contacts_last_step": int(last["n_contacts"]),
           "forward_contact_updates_per_s": fwd_upd / (fwd_ms / 1e3) if fwd_ms > 0 else 0.0, "losses": {}}
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, (val, top_i, wall) in losses.items():
        gx = torch.zeros(2 * n, dtype=torch.float64, device=device)
        if top_i is not None:
            gx[2 * top_i + 1] = 1.0
        gv = torch.zeros_like(gx)
        gw = torch.zeros(n, dtype=torch.float64, device=device)
        adj_ms = 0.0
        sweeps = upd = not_conv = max_sw = hyper = diverged = 0
        gmu = 0.0
        torch.cuda.synchronize(device)
        e0.record(stream)
        for buf, m in reversed(segs):
            g.load_checkpoint(buf)
            g.step(m, stats=False)
            for _ in range(m):
                a0.record(stream)
                gx, gv, gw, st = g.adjoint_step(gx, gv, gw, adj_alpha, 100000, dL_dwall_force=wall)
                a1.record(stream)
                a1.synchronize()
                wall = None
                adj_ms += a0.elapsed_time(a1)
                sweeps += st["sweeps"]
                max_sw = max(max_sw, st["sweeps"])
                upd += st["sweeps"] * st["n_contacts"]
                not_conv += 1 - st["converged"]
                hyper += int(st["n_rows"] > st["n_dof"])
                diverged += st["diverged"]
                gmu += st["dL_dmu"]
        e1.record(stream)
        e1.synchronize()
        bwd_ms = e0.elapsed_time(e1)
        gnorm = float(gv.norm())
        if diverged or not_conv or not (math.isfinite(gmu) and math.isfinite(gnorm)):
            # no derivative: the frozen-state reverse system has no bounded solution on some step
            status = (f"failed: reverse pass diverged on {diverged} and hit the sweep cap on {not_conv} of {T} "
                      f"steps ({hyper} steps with more retained rows than degrees of freedom)")
            gmu_out, gnorm_out = None, None
        else:
            status = "ok"
            gmu_out, gnorm_out = gmu, gnorm
        out["losses"][name] = {
            "value": val, "status": status, "dL_dmu": gmu_out, "dL_dv0_norm": gnorm_out,
            "backward_ms_per_step": bwd_ms / T, "adjoint_kernel_ms_per_step": adj_ms / T,
            "adjoint_sweeps_per_step": sweeps / T, "adjoint_sweeps_max": int(max_sw),
            "adjoint_contact_updates_per_s": upd / (adj_ms / 1e3) if adj_ms > 0 else 0.0,
            "adjoint_steps_not_converged": int(not_conv), "adjoint_steps_diverged": int(diverged),
            "steps_hyperstatic": int(hyper),
            "steps_per_s_forward_plus_backward": T / ((fwd_ms + bwd_ms) / 1e3)}
    g.load_checkpoint(final)
    del g
    if fd_h:
        # central differences in mu of both losses at h and 2 h, Richardson-extrapolated
        import copy
        vals = {}
        for sgn in (1, -1, 2, -2):
            w2 = copy.copy(wl)
            w2.mu = wl.mu + sgn * fd_h
            g2 = cd.CDSystem(w2, device=device, criterion=crit)
            st2 = g2.step(T)
            y2 = g2.pos.view(n, 2)[:, 1] + g2.radius
            vals[sgn] = {"floor_pressure": float(st2["last"]["wall_force"][2]) / width,
                         "packing_height": float(torch.max(y2))}
            del g2
        for name in losses:
            d1 = (vals[1][name] - vals[-1][name]) / (2 * fd_h)
            d2 = (vals[2][name] - vals[-2][name]) / (4 * fd_h)
            fd = (4 * d1 - d2) / 3
            ad = out["losses"][name]["dL_dmu"]
            out["losses"][name]["fd_check"] = {
                "h": fd_h, "central_h": d1, "central_2h": d2, "dL_dmu_fd": fd,
                "rel_err": (abs(fd - ad) / max(abs(fd), 1e-300)) if ad is not None else None}
    return out


def run_e2e(args, sysg, wl, device, ws):
    """Same metric through the public API with host buffers: every step
    uploads (pos, vel, omega) from pinned host memory, steps, and downloads
    the new state."""
    import torch
    from paper_1104_3516_gb300 import cd
    n, D = wl.n, wl.dim
    pos_h = torch.empty(n * D, dtype=torch.float64, pin_memory=True)
    vel_h = torch.empty(n * D, dtype=torch.float64, pin_memory=True)
    rot = 1 if D == 2 else 3
    om_h = torch.empty(n * rot, dtype=torch.float64, pin_memory=True)
    cd.cd_download_state(sysg.handle, pos_h, vel_h, om_h)
    h2d = d2h = (2 * n * D + n * rot) * 8
    barrier(ws)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    upd = 0
    for _ in range(args.steps):
        cd.cd_upload_state(sysg.handle, pos_h, vel_h, om_h)
        st = sysg.step(1)
        upd += st["total_contact_updates"]
        cd.cd_download_state(sysg.handle, pos_h, vel_h, om_h)
    sec = time.perf_counter() - t0
    (sec_max,), (upd_sum,) = reduce_max_sum([sec], [float(upd)], ws, device)
    return {"value": upd_sum / sec_max, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": args.steps, "api": "cd_upload_state + cd_step + cd_download_state"}


def run_mixed_scan(args):
    """Sec. 2.3's protocol on the GPU: a static loaded packing (a
    gravity-deposited pile of N discs at rest, floor and a fixed lid, mu 0.3)
    has its forces set to zero and is solved within one time step until the
    global test passes at 1e-6 (cap 20,000 sweeps), for parallel fractions
    p from 0 to 1, with the parallel subset fixed per contact key and drawn
    afresh in every iteration step.  Prints one JSON line: N_I per p (null:
    not converged, with the largest impulse it reached)."""
    import torch
    from paper_1104_3516_gb300 import cd, workloads as W
    device = torch.device("cuda", 0)
    ps = [0.0, 0.05, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 1.0]
    out = {"protocol": "static gravity-loaded pile, forces from zero, one solve, global test 1e-6, cap 20000",
           "p": ps, "piles": {}}
    for n in args.mixed_scan or [2000]:
        wl = W.dense_biaxial_discs(n=n, wall_speed=0.0)
        res = {}
        for redraw in (0, 1):
            row = []
            for p in ps:
                g = cd.CDSystem(wl, device=device, criterion=cd.CD_CONV_GLOBAL_REL, alpha=1e-6, max_sweeps=20000,
                                warm_start=0, parallel_p=p, parallel_redraw=redraw, max_contacts=4 * n)
                st = g.step(1)["last"]
                pmax = float(np.nanmax(np.abs(g.contacts()["impulse"])))
                row.append({"sweeps": st["sweeps"] if st["converged"] else None, "max_impulse": pmax})
                del g
            res["redrawn_every_step" if redraw else "fixed_per_contact"] = row
        out["piles"][str(n)] = res
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.mixed_scan is not None:
        run_mixed_scan(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

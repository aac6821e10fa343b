"""Benchmark: D3Q19 forced-MRT lattice Boltzmann MLUPS and HBM roofline
fraction on one GB300 (or N independent replicas under torchrun).

Headline workload (one "step"): one time step of the 512^3 periodic
sedimentation box with 1e5 point colloids (seeded uniform positions,
force (0, 0, -1e-6) each, radius 0.117, uniform counter-force, a_L of
Appendix A), FP32 storage: the colloids' forces are spread with Peskin's
kernel, the fused collide + pull-stream kernel runs over all 512^3 sites
(writing the fluid velocity at the colloids' stencil nodes), the velocity
is interpolated back and every colloid moves (Sec. II-IV).  The blocks
beside it: the same box in the other storage formats with errors per field
against the FP64 run, the four-lattice 256^3 channel / multipole step, the
32^3 Stokeslet in FP64, the batched replicas and the learned correction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision f32]
    python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19 forced-MRT MLUPS & HBM-roofline fraction per precision at stated error"
L_HEAD, N_HEAD = 512, 100000  # the sedimentation box of the headline
PREC_NAMES = {"f64": 0, "f32": 1, "f16s": 2, "bf16s": 3}
BYTES = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}
ARITH = {"f64": 8, "f32": 4, "f16s": 4, "bf16s": 4}
PROFILE_DIR = os.path.join(ROOT, "profiles")
# Algorithmic bytes per colloid and step beyond the lattice's 2*19*s per
# site: its 64 stencil nodes x 3 force components, in the arithmetic type a:
# the spread reads and writes them (2), the collide reads the force and
# writes the velocity (2), the interpolation reads the velocity (1).
COLLIDE_NODE_PASSES, STEP_NODE_PASSES = 2, 5


def workload_name(L, n):
    return (f"colloids_{L}: {L}^3 periodic D3Q19 MRT (tau_s = tau_b = 1/2), {n} point colloids at seeded "
            f"uniform positions (seed 3), force (0,0,-1e-6) each, radius 0.117, uniform counter-force, "
            f"a_L of Appendix A")


def default_colloids(L):
    """The headline's number density (1e5 in 512^3) at side L."""
    return max(1, int(round(N_HEAD * (L / L_HEAD) ** 3)))


def collide_bytes(prec, V, n):
    return 2 * 19 * BYTES[prec] * V + COLLIDE_NODE_PASSES * 64 * 3 * ARITH[prec] * n


def step_bytes(prec, V, n):
    return 2 * 19 * BYTES[prec] * V + STEP_NODE_PASSES * 64 * 3 * ARITH[prec] * n


def kernel_source_hash():
    """Hash of the CUDA sources the collide kernels are built from; a
    committed ncu figure is only quoted while they are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0707_1299_gb300", "csrc")
    for f in ("lb_device.cuh", "lb_collide.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def committed_profile(name):
    """key: value fields of profiles/<name>.txt, or None when the file is
    missing or was taken from other kernel sources."""
    path = os.path.join(PROFILE_DIR, name + ".txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != kernel_source_hash():
        return None
    return vals


def committed_traffic(name):
    """DRAM bytes per full-size launch from a committed ncu summary."""
    vals = committed_profile(name)
    try:
        return float(vals["dram_bytes_per_launch_full_size"]) if vals else None
    except (KeyError, ValueError):
        return None


def committed_fp64_mix():
    """FP64 instructions and flops per site of k_collide<double> from the
    committed ncu instruction-mix summary (None once the sources changed)."""
    vals = committed_profile("k_collide_f64_160")
    try:
        return (float(vals["fp64_inst_per_site"]), float(vals["fp64_flop_per_site"])) if vals else None
    except (KeyError, ValueError):
        return None


# FP64 peak from the nominal 1.25 TFLOP/s of GB300: 152 SMs x 2.07 GHz x 2
# FP64 lanes per SM and clock x 2 flops per fused multiply-add.
FP64_LANES_PER_SM_CLK = 2
SM_COUNT, SM_MAX_HZ = 152, 2.07e9


def fp64_roofline(V, coll_ms):
    """The FP64 collide against the FP64 pipe: FP64 thread-instructions per
    site (committed instruction-mix capture) x sites / the phase-timed
    collide, over 152 SMs x 2.07 GHz x 2 FP64 lanes."""
    peak = SM_COUNT * SM_MAX_HZ * FP64_LANES_PER_SM_CLK
    out = {"bound": "alu", "kernel": "k_collide<f64> (FP64 pipe)", "unit": "FP64 inst/s", "peak": peak,
           "peak_kind": "nominal: 152 SMs x 2.07 GHz x 2 FP64 lanes", "launch_ms": coll_ms}
    mix = committed_fp64_mix()
    if mix is None or not coll_ms:
        return dict(out, achieved=None, frac=None)
    inst, flop = mix
    rate = inst * V / (coll_ms * 1e-3)
    return dict(out, achieved=round(rate, -7), frac=round(rate / peak, 4),
                tflops=round(flop * V / (coll_ms * 1e-3) / 1e12, 4), fp64_inst_per_site=inst)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, p in zip(names, parts[3:7]):
                if p.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- GPU arm
def build_lattices(prec_id, L):
    from paper_0707_1299_gb300 import lb, workloads as W


# ------------------------------------------------------------ ranks
# lattices of different ranks share nothing): the job's time is its slowest
# rank's, and the job's throughput is all ranks' site updates over it.
def _reduce_device():
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest x over the ranks (x itself with one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(sites_per_rank, steps, seconds, world):
    """Whole-job throughput: every rank's site updates over the job's time."""
    return world * sites_per_rank * steps / seconds / 1e6


# --------------------------------------------------------------- GPU arm
def colloid_lattice(prec, L, n):
    from paper_0707_1299_gb300 import lb, workloads as W
    prob = W.colloids(L=L, n=n, seed=3, force=1e-6)
    aL = lb.lb_compute_aL(prob.grid, [L / 2 + 0.5] * 3, [0, 0, 1])
    g = lb.Lattice(prob.grid, prob.tau_s, prob.tau_b, PREC_NAMES[prec])
    g.set_colloid_aL(aL)
    ps = prob.points[0]
    g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
    return g, aL


def field_snapshot(g, p0, L):
    """rho, u and the colloid displacements of a lattice (device, FP64)."""
    import torch
    rho, u, tot = g.moments()
    p1, _ = g.particles()
    disp = p1 - p0
    disp -= L * torch.round(disp / L)
    return {"rho": rho, "u": u, "disp": disp, "totals": tot}


def field_errors(s, ref):
    """Errors per field against the FP64 run (reading A20: max error over
    max reference magnitude; density as the deviation from rest)."""
    def rel(a, b):
        return float((a - b).abs().max() / b.abs().max())
    return {"velocity": rel(s["u"], ref["u"]), "density": rel(s["rho"] - 1.0, ref["rho"] - 1.0),
            "displacement": rel(s["disp"], ref["disp"])}


def run_gpu(args, rank, world):
    import torch
    from paper_0707_1299_gb300 import build, lb

    build.build()
    lb.load()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    prec = args.precision
    L = args.size
    n = args.colloids if args.colloids is not None else default_colloids(L)
    V = L ** 3
    stream = torch.cuda.current_stream()
    g, aL = colloid_lattice(prec, L, n)
    p0, _ = g.particles()

    for _ in range(args.warmup):
        g.step(1)
    torch.cuda.synchronize()
    lb.lb_set_phase_timing(g.ctx, 1)
    launches0 = g.kernel_launches()
    clocks = ClockSampler(dev)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        g.step(1)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), world)
    launches = g.kernel_launches() - launches0
    phases = lb.lb_phase_times(g.ctx)
    lb.lb_set_phase_timing(g.ctx, 0)
    step_ms = ms / args.steps
    mlups = job_mlups(V, args.steps, ms * 1e-3, world)
    phase_ms = {k: round(t / c, 5) for k, (t, c) in phases.items() if c}
    coll_ms = phases["collide"][0] / phases["collide"][1]

    # end to end through the C ABI with host buffers: every step the colloid
    # positions (the step's input) go in from page-locked host memory, the
    # step runs, and the new positions (its result) come back into host
    # memory; the positions read back feed the next step, so the trajectory
    # is the device-only one
    host_pos = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    hp = host_pos.numpy()
    lb.lb_set_host_async(g.ctx, 1)
    lb.lb_particles(g.ctx, hp, None)
    lb.lb_synchronize(g.ctx)
    e2e_steps = args.e2e_steps
    barrier(world)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        lb.lb_set_positions(g.ctx, hp)
        g.step(1)
        lb.lb_particles(g.ctx, hp, None)
        lb.lb_synchronize(g.ctx)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - te, world)
    lb.lb_set_host_async(g.ctx, 0)
    e2e_mlups = job_mlups(V, e2e_steps, e2e_s, world)
    steps_done = args.warmup + args.steps + e2e_steps

    peak, peak_kind = measured_peaks()
    b_coll = collide_bytes(prec, V, n)
    b_step = step_bytes(prec, V, n)
    achieved = b_coll / (coll_ms * 1e-3) / 1e9
    traffic = committed_traffic(f"k_collide_{prec}_vel_{L}_{n}")
    out = {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": workload_name(L, n), "lattice": [L, L, L], "colloids": n, "precision": prec,
                   "a_L": round(aL, 6), "sites_per_step": V,
                   "l2": "inputs larger than L2 (each population buffer %.2f GB)" % (19 * BYTES[prec] * V / 1e9),
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "hbm",
                     "kernel": f"k_collide<{prec}, periodic, {'FM_VEL' if n else 'FM_NONE'}> ({L}^3, {n} colloids; "
                               "one launch per step)",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                     "launch_ms": round(coll_ms, 5), "launches_timed": phases["collide"][1],
                     "bytes_per_launch": b_coll,
                     "bytes_rule": f"2*19*{BYTES[prec]} B per site + {COLLIDE_NODE_PASSES}*64*3*{ARITH[prec]} B per "
                                   "colloid (force read, velocity written at its stencil nodes)"},
        "step_roofline": {"bytes_per_step": b_step, "achieved": round(b_step / (step_ms * 1e-3) / 1e9, 1),
                          "frac": round(b_step / (step_ms * 1e-3) / 1e9 / peak, 4), "phase_ms": phase_ms,
                          "bytes_rule": f"2*19*{BYTES[prec]} B per site + {STEP_NODE_PASSES}*64*3*{ARITH[prec]} B "
                                        "per colloid (spread read+write, collide read+write, interpolation read)"},
        "e2e": {"value": round(e2e_mlups, 1), "unit": "MLUPS", "h2d_bytes_per_step": 24 * n,
                "d2h_bytes_per_step": 24 * n, "steps": e2e_steps,
                "mode": "C ABI, page-locked host buffers, host-async calls: lb_set_positions(host) + lb_step(1) + "
                        "lb_particles(host) + lb_synchronize every step"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank != 0 or world != 1 or args.no_per_precision:
        g.close()
        torch.cuda.empty_cache()
        return out

    # errors per field against the FP64 run of the same box and step count
    # (the FP64 CUDA path is held to the oracle at 1e-12 by the parity
    # tests, at this size too), and the other storage formats beside it
    mine = field_snapshot(g, p0, L)
    g.close()
    torch.cuda.empty_cache()
    out["per_precision"] = per_precision_colloids(L, n, steps_done, prec, mine, out)
    return out


def per_precision_colloids(L, n, steps, head_prec, head_snap, head, timed=40):
    """The headline box in every storage format for the same number of
    steps, the last `timed` device-timed; errors per field against the FP64
    run.  The FP64 run goes first and is kept as the reference."""
    import torch
    from paper_0707_1299_gb300 import lb
    peak, _ = measured_peaks()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    V = L ** 3
    res = {"steps": steps, "timed_steps": timed, "reference": "FP64 run of the same box and steps"}
    ref = head_snap if head_prec == "f64" else None
    if ref is not None:
        head["error"] = None  # the headline is the FP64 run
    for prec in ("f64", "f16s", "bf16s", "f32"):
        if prec == head_prec:
            continue
        g, _ = colloid_lattice(prec, L, n)
        p0, _ = g.particles()
        g.step(steps - timed)
        torch.cuda.synchronize()
        lb.lb_set_phase_timing(g.ctx, 1)
        e0.record(stream)
        g.step(timed)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / timed
        ph = lb.lb_phase_times(g.ctx)
        lb.lb_set_phase_timing(g.ctx, 0)
        coll_ms = ph["collide"][0] / ph["collide"][1] if ph["collide"][1] else None
        snap = field_snapshot(g, p0, L)
        row = {"value": round(V / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "ms_per_step": round(ms, 4),
               "hbm_frac_of_step": round(step_bytes(prec, V, n) / (ms * 1e-3) / 1e9 / peak, 4)}
        if prec == "f64":
            ref = snap
            t = snap["totals"].cpu().numpy()
            row["totals"] = {"mass_minus_V": float(t[0] - V), "momentum": [float(x) for x in t[1:]]}
            row["roofline"] = fp64_roofline(V, coll_ms)
            head["error"] = dict(field_errors(head_snap, ref), steps=steps,
                                 reference="FP64 run (CUDA, oracle-checked) of the same box")
            del head_snap
        else:
            row["error_vs_f64"] = field_errors(snap, ref)
        del snap
        res[prec] = row
        g.close()
        torch.cuda.empty_cache()
    del ref
    torch.cuda.empty_cache()
    return res


def channel_block(steps=200, warm=5, L=256):
    """The four 256^3 lattices of the wall-bounded channel / multipole
    workload (body-force channel between solid planes, a Stokeslet, a
    stresslet and a rotlet; FP32), one step each per step, device-timed;
    the channel lattice's lb_step launches exactly one kernel, k_collide,
    whose events give its roofline; its error against the exactly
    equivalent 1 x 1 x L FP64 oracle column."""
    import torch
    from paper_0707_1299_gb300 import lb, workloads as W
    lats = []
    for prob in W.channel_256(L=L):
        g = lb.Lattice(prob.grid, prob.tau_s, prob.tau_b, lb.LB_F32)
        g.set_body_force(prob.g)
        if prob.walls is not None:
            g.set_walls_z(*prob.walls)
        g.set_counterforce(prob.counter)
        for ps in prob.points:
            g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
        lats.append((prob, g))
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        for _, g in lats:
            g.step(1)
    torch.cuda.synchronize()
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in lats]
          for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(steps):
        for k, (_, g) in enumerate(lats):
            ev[s][k][0].record(stream)
            g.step(1)
            ev[s][k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    per_lat = [float(np.mean([ev[s][k][0].elapsed_time(ev[s][k][1]) for s in range(steps)]))
               for k in range(len(lats))]
    V = L ** 3
    peak, _ = measured_peaks()
    achieved = 152 * V / (per_lat[0] * 1e-3) / 1e9
    err = channel_error(lats[0][0], lats[0][1], L, warm + steps)
    for _, g in lats:
        g.close()
    torch.cuda.empty_cache()
    return {"workload": "channel_256: four 256^3 FP32 lattices (channel g=1e-6 between planes z=0,255; "
                        "Stokeslet 1e-5; stresslet dipole 1e-4; rotlet torque 1e-4), tau_s = tau_b = 1/2",
            "value": round(4 * V * steps / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "steps": steps,
            "ms_per_step": round(ms / steps, 4),
            "lb_step_ms_per_lattice": {p.name: round(t, 5) for (p, _), t in zip(lats, per_lat)},
            "roofline": {"kernel": "k_collide<float, walls, FM_NONE> (channel lattice)", "launch_ms": round(per_lat[0], 5),
                         "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "bytes_per_site": 152, "traffic": committed_traffic("k_collide_f32_channel_256")},
            "error": {"max_rel_velocity_vs_oracle": err, "steps": warm + steps,
                      "case": "channel lattice vs exactly equivalent 1x1xL FP64 oracle column"}}


def channel_error(prob, g, L, nsteps):
    """Channel lattice vs the exactly equivalent 1 x 1 x L FP64 oracle column."""
    import oracle
    _, u, _ = g.moments()
    col = oracle.OracleLB((1, 1, L), prob.tau_s, prob.tau_b, g=prob.g, walls=prob.walls, counter=False)
    col.step(nsteps)
    ref = col.observe()["u"][0, :, 0, 0]
    uu = u[0, :, :: max(1, L // 8), :: max(1, L // 8)].cpu().numpy()
    return float(np.abs(uu - ref[:, None, None]).max() / np.abs(ref).max())


def stokeslet_block(steps=1000):
    """The 32^3 Stokeslet in FP64 (1000 steps), device-timed in one call,
    against the oracle's 1000 steps."""
    import torch
    import oracle
    from paper_0707_1299_gb300 import lb, workloads as W
    prob = W.stokeslet_32()
    g = lb.Lattice(prob.grid, prob.tau_s, prob.tau_b, lb.LB_F64)
    ps = prob.points[0]
    g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
    g.step(3)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps - 3)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (steps - 3)
    _, u, _ = g.moments()
    o = oracle.OracleLB(prob.grid, prob.tau_s, prob.tau_b)
    o.add_points(ps.kind, ps.pos, ps.F, ps.param)
    o.step(steps)
    ref = o.observe()["u"]
    err = float(np.abs(u.cpu().numpy() - ref).max() / np.abs(ref).max())
    g.close()
    return {"workload": "stokeslet_32: 32^3 FP64, Stokeslet (0,0,1e-5) at (16.3,15.7,16.45), counter-force",
            "value": round(32 ** 3 / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "ms_per_step": round(ms, 5),
            "steps": steps, "max_rel_velocity_vs_oracle": err,
            "note": "10 MB per step: launch- and latency-bound, not a bandwidth case"}


def batched_replicas(steps=50, seq_steps=10, replicas=64):
    """64 independent sedimentation boxes of uneven sizes (48^3-128^3, 100-2000
    colloids each, FP32) advanced by one batch (one persistent cooperative
    launch per step over all boxes, graph-replayed, tuned grid) against the
    same boxes stepped one after another with lb_step."""
    import torch
    from paper_0707_1299_gb300 import lb, workloads as W
    probs = W.replicas(n=replicas)
    lats = []
    for p in probs:
        g = lb.Lattice(p.grid, p.tau_s, p.tau_b, lb.LB_F32)
        g.set_colloid_aL(lb.lb_compute_aL(p.grid, [p.grid[0] / 2] * 3, [0, 0, 1]))
        for ps in p.points:
            g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
        lats.append(g)
    sites = sum(g.V for g in lats)
    stream = torch.cuda.current_stream()
    batch = lb.lb_batch_create([g.ctx for g in lats])
    blocks = lb.lb_batch_tune(batch)
    lb.lb_batch_step(batch, 4)
    torch.cuda.synchronize()
    l0 = lb.lb_batch_info(batch)["launches"]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    lb.lb_batch_step(batch, steps)
    t1.record(stream)
    torch.cuda.synchronize()
    lb.lb_batch_synchronize(batch)  # raises if a barrier wait ran out
    ms_b = t0.elapsed_time(t1) / steps
    launches = lb.lb_batch_info(batch)["launches"] - l0
    lb.lb_batch_destroy(batch)
    for g in lats:
        g.step(1)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(seq_steps):
        for g in lats:
            g.step(1)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_s = t0.elapsed_time(t1) / seq_steps
    peak, _ = measured_peaks()
    npts = sum(g.num_points() for g in lats)
    for g in lats:
        g.close()
    torch.cuda.empty_cache()
    return {"replicas": len(probs), "sites_per_step": sites, "colloids": npts, "precision": "f32",
            "value": round(sites / (ms_b * 1e-3) / 1e6, 1), "unit": "MLUPS", "ms_per_step": round(ms_b, 4),
            "hbm_frac_of_step": round(step_bytes("f32", sites, npts) / (ms_b * 1e-3) / 1e9 / peak, 4),
            "bytes_rule": "as the headline step: 2*19*4 B per site + 5*64*3*4 B per colloid",
            "launches_per_step": launches / steps, "persistent_blocks": blocks, "steps": steps,
            "sequential_lb_step": {"value": round(sites / (ms_s * 1e-3) / 1e6, 1), "ms_per_step": round(ms_s, 4),
                                   "steps": seq_steps}}


def learned_correction(train_pairs=32, test_pairs=4, L_pair=64, T_pair=1000, steps=20, train=True):
    """The learned correction of the colloid velocity: trained on ~1e5
    samples of 1x/2x run pairs of the method (64^3 / 128^3 boxes at the
    number density of the workload below), judged on held-out pairs; then
    the 256^3 FP32 box with 2e5 colloids (seed 5, force 1e-6, a = 0.117)
    stepped with the plain update and with the corrected one."""
    import torch
    from paper_0707_1299_gb300 import lb, learned, workloads as W
    if train:
        t0 = time.perf_counter()
        data = [learned.pair_samples(L=L_pair, seed=s, T=T_pair) for s in range(train_pairs + test_pairs)]
        torch.cuda.synchronize()
        t_gen = time.perf_counter() - t0
        ftr = torch.cat([d[0] for d in data[:train_pairs]]).contiguous()
        ltr = torch.cat([d[1] for d in data[:train_pairs]]).contiguous()
        fte = torch.cat([d[0] for d in data[train_pairs:]]).contiguous()
        lte = torch.cat([d[1] for d in data[train_pairs:]]).contiguous()
        warm, _ = learned.train(ftr, ltr, steps=5, batch=4096, lr=2e-3)  # first use of the training kernels
        lb.lb_mlp_destroy(warm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net, hist = learned.train(ftr, ltr, steps=4000, batch=4096, lr=2e-3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        ev = learned.evaluate(net, fte, lte)
    else:  # the seeded initial network: the corrected step costs the same
        net = lb.lb_mlp_create(learned.initial_params(0))
    prob = W.colloids(L=256, n=200000, seed=5, force=1e-6)
    g = lb.Lattice(prob.grid, prob.tau_s, prob.tau_b, lb.LB_F32)
    g.set_colloid_aL(lb.lb_compute_aL(prob.grid, [128.5] * 3, [0, 0, 1]))
    ps = prob.points[0]
    g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {}
    for name, attach in (("plain", None), ("corrected", net)):
        lb.lb_set_colloid_correction(g.ctx, attach)
        g.step(3)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        # the phases on their own streams (the correction runs beside the
        # collide), in separate steps after the timed ones
        lb.lb_set_phase_timing(g.ctx, 1)
        g.step(steps)
        ph = lb.lb_phase_times(g.ctx)
        lb.lb_set_phase_timing(g.ctx, 0)
        out[name] = {"ms_per_step": round(ms, 4), "value": round(256 ** 3 / (ms * 1e-3) / 1e6, 1),
                     "phase_ms": {k: round(t / c_, 5) for k, (t, c_) in ph.items() if c_}}
    out["corrected"]["overhead"] = round(out["corrected"]["ms_per_step"] / out["plain"]["ms_per_step"] - 1, 4)
    lb.lb_set_colloid_correction(g.ctx, None)
    g.close()
    lb.lb_mlp_destroy(net)
    torch.cuda.empty_cache()
    if not train:
        return {"workload": "256^3 FP32, 2e5 colloids (seed 5), force 1e-6, a = 0.117", "unit": "MLUPS",
                "plain": out["plain"], "corrected": out["corrected"], "training": None,
                "note": "untrained seeded network (--no-training): step costs only"}
    return {"workload": "256^3 FP32, 2e5 colloids (seed 5), force 1e-6, a = 0.117", "unit": "MLUPS",
            "plain": out["plain"], "corrected": out["corrected"],
            "training": {"samples": int(ftr.shape[0]), "pairs": f"{train_pairs} x ({L_pair}^3 T={T_pair}, "
                                                                 f"{2 * L_pair}^3 T={4 * T_pair})",
                         "adam_steps": 4000, "generation_s": round(t_gen, 2), "train_s": round(t_train, 2),
                         "final_loss_rel": round(hist[-1], 4)},
            "velocity_error_vs_2x": {"held_out_samples": int(fte.shape[0]),
                                     "rms_plain_over_v0": round(ev["rms_plain"], 6),
                                     "rms_corrected_over_v0": round(ev["rms_corrected"], 6),
                                     "gain": round(ev["gain"], 3)}}


# ---------------------------------------------------------- oracle (CPU)
CPU_SAMPLE_L = 128  # the headline box cropped to 128^3 at the same colloid density


def oracle_colloids(L, n):
    import oracle
    from paper_0707_1299_gb300 import workloads as W
    prob = W.colloids(L=L, n=n, seed=3, force=1e-6)
    aL = oracle.aL_along(prob.grid, [L / 2 + 0.5] * 3, [0, 0, 1])
    o = oracle.OracleLB(prob.grid, prob.tau_s, prob.tau_b, a_L=aL)
    ps = prob.points[0]
    o.add_points(ps.kind, ps.pos, ps.F, ps.param)
    return o


def cpu_sample(L, budget_s, max_steps=400):
    """MLUPS of the oracle stepping the headline recipe cropped to L^3 (same
    number density, seed 3), for about budget_s seconds."""
    import oracle
    n = default_colloids(L)
    o = oracle_colloids(L, n)
    o.step(1)  # first touch of the oracle's buffers
    t = time.perf_counter()
    k = 0
    while time.perf_counter() - t < budget_s and k < max_steps:
        o.step(1)
        k += 1
    dt = time.perf_counter() - t
    return {"value": round(o.V * k / dt / 1e6, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
            "sample": f"{L}^3 with {n} colloids (the {L_HEAD}^3 / {N_HEAD} recipe cropped at its number density), "
                      f"FP64, {k} steps, {o.V * k / 1e6:.1f} M site updates in {dt:.1f} s"}


def cpu_baseline(budget_s=12.0):
    """The oracle as it stands on all host cores (OpenMP) on the cropped
    headline box, and on one core (a child process with OMP_NUM_THREADS=1)
    on a 64^3 crop."""
    import oracle
    oracle.build()
    res = cpu_sample(CPU_SAMPLE_L, budget_s)
    res["kind"] = "oracle"
    res["cpu_model"] = cpu_model()
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_sample(64, 6.0)))" % ROOT)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        res["one_core"] = one
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        res["one_core"] = None
    return res


def run_reference(args, rank, world):
    """The reference arm: the oracle as it stands, on the host cores, one
    step of the headline recipe cropped to 128^3 (same number density) per
    step (the paper publishes no code to run instead)."""
    import oracle
    oracle.build()
    L = min(args.size, CPU_SAMPLE_L)
    n = default_colloids(L)
    o = oracle_colloids(L, n)
    for _ in range(args.warmup):
        o.step(1)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t
    v = o.V * args.steps / dt / 1e6
    sample = (f"{L}^3 with {n} colloids per step (the {L_HEAD}^3 / {N_HEAD} recipe cropped at its number density), "
              f"FP64")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / max(args.steps, 1) * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.size, args.colloids or default_colloids(args.size)),
                       "sample": sample, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="f32", choices=list(PREC_NAMES))
    ap.add_argument("--size", type=int, default=L_HEAD, help="side of the headline sedimentation box")
    ap.add_argument("--colloids", type=int, default=None,
                    help="colloids of the headline box (default: 1e5 x (size/512)^3)")
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-precision", action="store_true")
    ap.add_argument("--no-channel", action="store_true")
    ap.add_argument("--channel-size", type=int, default=256)
    ap.add_argument("--no-stokeslet", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--replicas", type=int, default=64, help="members of the batched-replicas block (first N)")
    ap.add_argument("--no-training", action="store_true",
                    help="learned block: time the plain and corrected steps with the seeded initial "
                         "network, without generating pairs or training (for profiling)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, 1)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = run_gpu(args, rank, world)
    if rank == 0:
        extra = world == 1
        out["channel_256"] = channel_block(L=args.channel_size) if extra and not args.no_channel else None
        out["stokeslet_32"] = stokeslet_block() if extra and not args.no_stokeslet else None
        out["batched"] = batched_replicas(replicas=args.replicas) if extra and not args.no_batched else None
        out["learned"] = learned_correction(train=not args.no_training) if extra and not args.no_learned else None
        out["cpu_baseline"] = cpu_baseline() if extra and not args.no_cpu_baseline else None
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

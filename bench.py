"""Benchmark: D3Q19 forced-MRT lattice Boltzmann MLUPS and HBM roofline
fraction on one GB300 (or N independent replicas under torchrun).

Workload (one "step"): one time step of each of the four 256^3 FP32
lattices of the wall-bounded channel / multipole recipe -- the body-force
channel with solid planes z = 0, 255, a Stokeslet, a stresslet and a
rotlet at seeded positions (see paper_0707_1299_gb300.workloads).  Every
lattice step spreads its point forces (Peskin kernel), then runs the fused
collide + pull-stream kernel over all 256^3 sites.  The velocity at the
force points is interpolated back every step (gather kernel).

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
WORKLOAD = ("channel_256: four 256^3 D3Q19 MRT lattices per step (body-force channel g=1e-6 between "
            "solid planes z=0,255; Stokeslet F=1e-5; stresslet dipole 1e-4; rotlet torque 1e-4; "
            "seeded off-lattice positions), tau_s=tau_b=1/2")
PREC_NAMES = {"f64": 0, "f32": 1, "f16s": 2, "bf16s": 3}
BYTES = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}
PROFILE_DIR = os.path.join(ROOT, "profiles")


def kernel_source_hash():
    """Hash of the CUDA sources; the committed ncu traffic figure is only
    quoted while the kernels are unchanged since it was taken."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0707_1299_gb300", "csrc")
    for f in ("lb_device.cuh", "lb_collide.cu"):  # what k_collide is built from
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(prec):
    """dram bytes per k_collide launch from the committed ncu summary."""
    path = os.path.join(PROFILE_DIR, f"k_collide_{prec}_channel_256.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def committed_fp64_mix():
    """FP64 instructions and flops per site of k_collide<double> from the
    committed ncu instruction-mix summary (None once the sources changed)."""
    path = os.path.join(PROFILE_DIR, "k_collide_f64_160.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != kernel_source_hash():
        return None
    try:
        return float(vals["fp64_inst_per_site"]), float(vals["fp64_flop_per_site"])
    except (KeyError, ValueError):
        return None


# FP64 peak from the nominal 1.25 TFLOP/s of GB300: 152 SMs x 2.07 GHz x 2
# FP64 lanes per SM and clock x 2 flops per fused multiply-add.
FP64_LANES_PER_SM_CLK = 2
SM_COUNT, SM_MAX_HZ = 152, 2.07e9


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
    lats = []
    for prob in W.channel_256(L=L):
        g = lb.Lattice(prob.grid, prob.tau_s, prob.tau_b, prec_id)
        g.set_body_force(prob.g)
        if prob.walls is not None:
            g.set_walls_z(*prob.walls)
        g.set_counterforce(prob.counter)
        for ps in prob.points:
            g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
        lats.append((prob, g))
    return lats


# ------------------------------------------------------------ ranks
# One process per GPU, each stepping its own replica of the workload (the
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


def run_gpu(args, rank, world):
    import torch
    from paper_0707_1299_gb300 import build, lb

    build.build()
    lb.load()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    prec = args.precision
    L = args.size
    lats = build_lattices(PREC_NAMES[prec], L)
    V = L ** 3
    stream = torch.cuda.current_stream()

    # query points: the force points of each lattice, or the channel centre,
    # where the velocity is interpolated back every step
    qpos = []
    for prob, g in lats:
        p, _ = g.particles()
        if p.shape[0] == 0:
            p = torch.tensor([[L / 2, L / 2, L / 2]], dtype=torch.float64, device=p.device)
        qpos.append(p)
    vbuf = [torch.empty_like(q) for q in qpos]

    def one_step(events=None):
        for k, (prob, g) in enumerate(lats):
            if events is not None:
                events[k][0].record(stream)
            g.step(1)
            if events is not None:
                events[k][1].record(stream)
            lb.lb_velocity_at(g.ctx, qpos[k].shape[0], qpos[k], vbuf[k])

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    launches0 = sum(g.kernel_launches() for _, g in lats)
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in lats]
          for _ in range(args.steps)]
    clocks = ClockSampler(dev)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        one_step(ev[s])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(t0.elapsed_time(t1), world)
    launches = sum(g.kernel_launches() for _, g in lats) - launches0
    # lb_step(1) of the channel lattice (no points) launches exactly one
    # kernel, k_collide: its events time that kernel alone.  The point
    # lattices' lb_step(1) runs the field-free collide and the fix-up of
    # the few tiles their fixed points flag, reported beside it.
    per_lat = [float(np.mean([ev[s][k][0].elapsed_time(ev[s][k][1]) for s in range(args.steps)]))
               for k in range(len(lats))]
    coll_ms = per_lat[0]
    step_ms = ms / args.steps
    mlups = job_mlups(4 * V, args.steps, ms * 1e-3, world)

    # end to end through the C ABI with host buffers: per step copy the
    # point positions (the step's input) in from pinned host memory, step,
    # and read the interpolated velocities (the step's result) back into
    # pinned host memory
    has_pts = [g.num_points() > 0 for _, g in lats]
    host_q = [q.cpu().pin_memory() for q in qpos]
    host_v = [torch.empty(q.shape, dtype=torch.float64).pin_memory() for q in qpos]
    e2e_steps = max(3, args.steps // 4)
    h2d = sum(hq.numel() * 8 for hq, hp in zip(host_q, has_pts) if hp)
    d2h = sum(hv.numel() * 8 for hv in host_v)
    # host-async calls: the four lattices' copies and steps are enqueued
    # back to back, and each step ends with lb_synchronize, after which the step's
    # velocities are in host memory
    for _, g in lats:
        lb.lb_set_host_async(g.ctx, 1)
    barrier(world)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        for k, (prob, g) in enumerate(lats):
            if has_pts[k]:
                lb.lb_set_positions(g.ctx, host_q[k].numpy())
            g.step(1)
            lb.lb_velocity_at(g.ctx, host_q[k].shape[0], host_q[k].numpy(), host_v[k].numpy())
        for _, g in lats:
            lb.lb_synchronize(g.ctx)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - te, world)
    e2e_mlups = job_mlups(4 * V, e2e_steps, e2e_s, world)

    # stated error: the channel lattice against the exactly equivalent
    # 1 x 1 x L oracle column after the same number of steps (rank 0)
    err = None
    nsteps_done = args.warmup + args.steps + e2e_steps
    if rank == 0 and not args.no_check:
        err = channel_error(lats[0][0], lats[0][1], L, nsteps_done)

    peak, peak_kind = measured_peaks()
    b_alg = 2 * 19 * BYTES[prec] * V
    achieved = b_alg / (coll_ms * 1e-3) / 1e9
    traffic = committed_traffic(prec)
    for _, g in lats:
        g.close()
    torch.cuda.empty_cache()
    others = None
    if rank == 0 and world == 1 and not args.no_per_precision:
        others = per_precision(L, {p: (10 if p == "f64" else 100) for p in PREC_NAMES if p != prec})
    c512 = None
    if rank == 0 and world == 1 and not args.no_colloids512:
        c512 = colloids_512(L=args.colloids[0], n=args.colloids[1])
    batched = None
    if rank == 0 and world == 1 and not args.no_batched:
        batched = batched_replicas(replicas=args.replicas)
    learned = None
    if rank == 0 and world == 1 and not args.no_learned:
        learned = learned_correction(train=not args.no_training)
    out = {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": [L, L, L], "lattices_per_step": 4,
                   "sites_per_step": 4 * V, "precision": prec,
                   "l2": "inputs larger than L2 (each population buffer %.2f GB)" % (19 * BYTES[prec] * V / 1e9),
                   "parallelism": f"replicas{world}"},
        "error": {"max_rel_velocity_vs_oracle": err, "steps": nsteps_done,
                  "case": "channel lattice vs exactly equivalent 1x1xL FP64 oracle column"},
        "roofline": {"bound": "hbm", "kernel": f"k_collide<{prec}> (channel lattice: 256^3, walls, one launch per lb_step)",
                     "lb_step_ms_per_lattice": {p.name: round(t, 5) for (p, _), t in zip(lats, per_lat)},
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "bytes_per_site": 2 * 19 * BYTES[prec], "launch_ms": round(coll_ms, 5),
                     "traffic": traffic},
        "e2e": {"value": round(e2e_mlups, 1), "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                "mode": "C ABI with page-locked host buffers, host-async calls, lb_synchronize once per step"},
        "gpu_launches": launches,
        "clocks": clk,
        "per_precision": others,
        "colloids_512": c512,
        "batched": batched,
        "learned": learned,
    }
    return out


def channel_error(prob, g, L, nsteps):
    """Channel lattice vs the exactly equivalent 1 x 1 x L FP64 oracle column."""
    import oracle
    _, u, _ = g.moments()
    col = oracle.OracleLB((1, 1, L), prob.tau_s, prob.tau_b, g=prob.g, walls=prob.walls, counter=False)
    col.step(nsteps)
    ref = col.observe()["u"][0, :, 0, 0]
    uu = u[0, :, :: max(1, L // 8), :: max(1, L // 8)].cpu().numpy()
    return float(np.abs(uu - ref[:, None, None]).max() / np.abs(ref).max())


def per_precision(L, steps_for):
    """The same four-lattice step in the other storage formats: device-timed
    (CUDA events around the collide launches, as for the headline line),
    with the channel lattice's error against the FP64 oracle column."""
    import torch
    from paper_0707_1299_gb300 import lb
    peak, peak_kind = measured_peaks()
    stream = torch.cuda.current_stream()
    out = {}
    for prec, steps in steps_for.items():
        lats = build_lattices(PREC_NAMES[prec], L)
        warm = 3
        for _ in range(warm):
            for _, g in lats:
                g.step(1)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps * len(lats))]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s in range(steps):
            for k, (_, g) in enumerate(lats):
                e = ev[s * len(lats) + k]
                e[0].record(stream)
                g.step(1)
                e[1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1)
        coll = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
        V = L ** 3
        achieved = 2 * 19 * BYTES[prec] * V / (coll * 1e-3) / 1e9
        err = channel_error(lats[0][0], lats[0][1], L, warm + steps)
        out[prec] = {"value": round(4 * V * steps / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "steps": steps,
                     "collide_ms": round(coll, 5), "bytes_per_site": 2 * 19 * BYTES[prec],
                     "hbm_achieved_gbs": round(achieved, 1), "hbm_frac": round(achieved / peak, 4),
                     "bound": "alu (FP64 pipe)" if prec == "f64" else "hbm / issue",
                     "max_rel_velocity_vs_oracle": err, "error_steps": warm + steps}
        if prec == "f64":
            mix = committed_fp64_mix()
            peak_inst = SM_COUNT * SM_MAX_HZ * FP64_LANES_PER_SM_CLK
            if mix is not None:
                inst, flop = mix
                rate = inst * V / (coll * 1e-3)
                out[prec]["alu"] = {"unit": "FP64 thread-instructions/s", "achieved": round(rate / 1e9, 1),
                                    "peak": round(peak_inst / 1e9, 1), "frac": round(rate / peak_inst, 4),
                                    "scale": "1e9", "inst_per_site": inst, "flop_per_site": flop,
                                    "tflops": round(flop * V / (coll * 1e-3) / 1e12, 3),
                                    "peak_tflops_nominal": round(2 * peak_inst / 1e12, 3),
                                    "source": "profiles/k_collide_f64_160.txt"}
            else:
                out[prec]["alu"] = None
        for _, g in lats:
            g.close()
        torch.cuda.empty_cache()
    return out


def colloids_512(L=512, n=100000, steps=100, timed=40):
    """The 512^3 sedimentation box: 1e5 colloids (seed 3) with force 1e-6
    and radius 0.117, counter-force, a_L along z; every storage format
    stepped `steps` times, the last `timed` device-timed with CUDA events.
    Velocity field and colloid displacements are compared with the FP64
    run of the same configuration (the FP64 CUDA path is checked against
    the oracle on this recipe at 40^3 by the parity tests); FP64 mass and
    momentum totals are reported beside it."""
    import torch
    from paper_0707_1299_gb300 import lb, workloads as W
    peak, _ = measured_peaks()
    prob = W.colloids(L=L, n=n, seed=3, force=1e-6)
    aL = lb.lb_compute_aL(prob.grid, [L / 2 + 0.5] * 3, [0, 0, 1])
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    V = L ** 3
    ref = None
    out = {"workload": f"{L}^3 periodic, {n} colloids (seed 3), force 1e-6, a = 0.117, counter-force, a_L = {aL:.4g}",
           "steps": steps, "timed_steps": timed}
    for prec in ("f64", "f32", "f16s", "bf16s"):
        g = lb.Lattice(prob.grid, prob.tau_s, prob.tau_b, PREC_NAMES[prec])
        g.set_colloid_aL(aL)
        ps = prob.points[0]
        g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
        p0, _ = g.particles()
        g.step(steps - timed)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(timed)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / timed
        _, u, tot = g.moments()
        p1, _ = g.particles()
        disp = p1 - p0
        disp -= L * torch.round(disp / L)
        row = {"value": round(V / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "ms_per_step": round(ms, 4),
               "hbm_frac_of_step": round(2 * 19 * BYTES[prec] * V / (ms * 1e-3) / 1e9 / peak, 4)}
        if ref is None:
            ref = (u, disp)
            t = tot.cpu().numpy()
            row["totals"] = {"mass_minus_V": float(t[0] - V), "momentum": [float(x) for x in t[1:]]}
        else:
            row["max_rel_velocity_vs_f64"] = float((u - ref[0]).abs().max() / ref[0].abs().max())
            row["max_rel_displacement_vs_f64"] = float((disp - ref[1]).abs().max() / ref[1].abs().max())
            del u
        out[prec] = row
        g.close()
        torch.cuda.empty_cache()
    del ref
    torch.cuda.empty_cache()
    return out


def batched_replicas(steps=50, seq_steps=10, replicas=64):
    """64 independent sedimentation boxes of uneven sizes (48^3-128^3, 100-2000
    colloids each, FP32) advanced by one batch (a launch per phase over all
    boxes, graph-replayed steps, tuned persistent grid) against the same boxes
    stepped one after another with lb_step."""
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
            "hbm_frac_of_step": round(152 * sites / (ms_b * 1e-3) / 1e9 / peak, 4),
            "launches_per_step": launches / steps, "collide_blocks": blocks, "steps": steps,
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
        warm, _ = learned.train(ftr, ltr, steps=5, batch=4096, lr=2e-3)  # first use of torch's sampling kernels
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
        out[name] = {"ms_per_step": round(ms, 4), "value": round(256 ** 3 / (ms * 1e-3) / 1e6, 1)}
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
def oracle_sample_step(lats):
    for o in lats:
        o.step(1)


def oracle_lattices(L, nxy):
    import oracle
    from paper_0707_1299_gb300 import workloads as W
    out = []
    for prob in W.channel_256(L=L, nx=nxy, ny=nxy):
        o = oracle.OracleLB(prob.grid, prob.tau_s, prob.tau_b, g=prob.g, walls=prob.walls, counter=prob.counter)
        for ps in prob.points:
            o.add_points(ps.kind, ps.pos, ps.F, ps.param)
        out.append(o)
    return out


def cpu_baseline(L, budget_s=12.0, nxy=64):
    """The oracle on a bounded sample: the same four lattices cropped to
    nxy x nxy x L (the recipe's points stay inside), stepped until about
    budget_s seconds of CPU work."""
    import oracle
    lats = oracle_lattices(L, nxy)
    oracle_sample_step(lats)  # first-touch of the oracle's buffers
    sites = sum(o.V for o in lats)
    t = time.perf_counter()
    n = 0
    while time.perf_counter() - t < budget_s and n < 50:
        oracle_sample_step(lats)
        n += 1
    dt = time.perf_counter() - t
    return {"value": round(sites * n / dt / 1e6, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"four lattices {nxy}x{nxy}x{L} (channel recipe cropped in x,y), {n} steps, FP64, "
                      f"{sites * n / 1e6:.1f} M site updates in {dt:.1f} s"}


def run_reference(args, rank, world):
    import oracle
    oracle.build()
    nxy = 64
    lats = oracle_lattices(args.size, nxy)
    for _ in range(args.warmup):
        oracle_sample_step(lats)
    sites = sum(o.V for o in lats)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(lats)
    dt = time.perf_counter() - t
    v = sites * args.steps / dt / 1e6
    sample = f"four lattices {nxy}x{nxy}x{args.size} (channel recipe cropped in x,y) per step, FP64"
    return {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample, "parallelism": "host cores"},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="f32", choices=list(PREC_NAMES))
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-precision", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-colloids512", action="store_true")
    ap.add_argument("--colloids", type=int, nargs=2, default=[512, 100000], metavar=("L", "N"),
                    help="box side and colloid count of the sedimentation-box block")
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
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.size)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark of the batched multi-arm MPPI control cycle on GB300.

One "step" is one control cycle of every arm (Algorithm 1: sense, shift,
sample, rollout, update, ToPlan/publish).  The default workload is the
largest single-GPU one, workload 5: 8 arms x 7 DoF, 40 spheres each,
K = 4096 samples, H = 64 steps, dt = 0.01 s, 256 moving world spheres,
every arm costed against the other 7 arms' shared plans (2,097,152 rollout
steps per cycle).  The metric is rollout trajectory-steps per second:
sum_a K_a H_a x iterations / cycle time.

  value : exact costs, device-resident inputs, per-cycle CUDA-event time on
          the library's stream, L2 flushed (256 MiB write) before every
          timed cycle.
  e2e   : the same cycles through mrs_step with host buffers (H2D of the
          sensed state and D2H of the results inside the timed region),
          wall clock per call, closed loop (the host plant integrates U_*,
          goals drift), 5 seeded scenes x 200 cycles, p50 / p99 latency.

Also reported: the plain form (one context per arm, no graph), the learned
form (self and arm-pair networks trained here on the device), the other
workloads (2, 3 = 2 with the learned self network, 4, and 2 in the paper's M
setting), the rollout kernel's roofline, and the FP64 oracle timed on a
bounded sample of the same workload on the host cores.

`--impl reference` times the FP64 CPU oracle on the host cores instead.
With torchrun (N > 1) every rank runs an independent replica on its own GPU
(the arms of one replica couple through the plan board, which stays on one
device); value is the sum over ranks of the work divided by the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rollout trajectory-steps/s and control-cycle p50/p99 latency, learned vs exact"
UNIT = "trajectory-steps/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
CSRC = os.path.join(ROOT, "paper_2602_10114_gb300", "csrc")
# the rollout kernel's sources: an ncu summary applies while their hash matches
ROLLOUT_SOURCES = ["rollout_kernel.cuh", "rollout.cu", "rollout_mb2.cu", "rollout_mb4.cu",
                   "rollout_spg4.cu", "rollout_spg5.cu", "rollout_spg57.cu", "mrs_device.cuh",
                   "tc_gemm.cuh"]
ROLLOUT_PROFILE = os.path.join(ROOT, "profiles", "k_rollout_8arms_K4096_H64.md")
CPU_SAMPLE_K = 32        # samples per arm of the oracle's bounded sample


def rollout_source_hash():
    h = hashlib.sha256()
    for f in ROLLOUT_SOURCES:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_figures(path=ROLLOUT_PROFILE):
    """The `key: value` lines of the ncu summary's figures block, or None with
    the reason when the file is missing or was taken from other sources."""
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None, "no ncu summary"
    fig = {}
    for ln in lines:
        ln = ln.strip()
        if ln.startswith("figure "):
            k, _, v = ln[len("figure "):].partition(":")
            fig[k.strip()] = v.strip()
    if fig.get("source_sha256") != rollout_source_hash():
        return None, "the rollout kernel changed since its ncu capture"
    return fig, os.path.relpath(path, ROOT)


def measured_peaks():
    """The machine's measured HBM and BF16 peaks, else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "fallback"}


def mlp_flops(rows, in_pad, width, layers):
    """Dense BF16 work of one surrogate launch: 2 x rows x (in_pad x width +
    (layers - 1) x width^2 + width)."""
    return 2.0 * rows * (in_pad * width + (layers - 1) * width * width + width)


def self_mlp_flops(sc, width=256, layers=3):
    """The self networks' work over every rollout step of every arm (the
    input, 2 dof sin/cos features, padded to a multiple of 16)."""
    return sum(mlp_flops(a.K * a.H, (2 * a.dof + 15) // 16 * 16, width, layers) for a in sc.arms)


def workload(idx, run=0):
    """Workload 1..5, or "M": workload 2 in the paper's M setting (5
    optimisation iterations per cycle, Sec. V-A) with the manipulability term
    on (w_manip = 10)."""
    from paper_2602_10114_gb300 import scenarios as S
    if str(idx) == "M":
        sc = S.config(2, run=run, iterations=5, w_manip=10.0)
        sc.name = "cfg2 in the M setting: 4 arms x 7 DoF, K=512, H=30, 5 iterations, C_manip"
        return sc
    return S.config(int(idx), run=run)


def rollout_flops(sc):
    """Algorithmic FP32 work of one rollout launch, counted brute force as the
    paper counts distance queries (Sec. IV-A, N_Q): 10 flops (+1 sqrt) per
    sphere pair (world, self on bodies at least three apart, every other
    arm's plan at the same step), plus 60 d + 18 N_S per rollout step for the
    kinematics."""
    total = 0.0
    n_obst = len(sc.world) + len(sc.aabb)
    for j, a in enumerate(sc.arms):
        body = a.sphere_body
        self_pairs = sum(1 for s1 in range(a.n_spheres) for s2 in range(s1 + 1, a.n_spheres)
                         if abs(int(body[s1]) - int(body[s2])) >= 3)
        for h in range(a.H):
            others = sum(b.n_spheres for i, b in enumerate(sc.arms) if i != j and h < b.H)
            pairs = a.n_spheres * n_obst + self_pairs + a.n_spheres * others
            total += a.K * (10.0 * pairs + 60 * a.dof + 18 * a.n_spheres)
    return total * sc.params["iterations"]


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except Exception:
        pass
    return platform.processor() or platform.machine()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the
    timed region runs (into a temporary file)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="mrs_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}",
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1].split()[0]))
                smax.append(float(r[2].split()[0]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(name)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
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


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (a baseline, not the target)

def oracle_sample(sc):
    """The bounded sample of a workload the oracle is timed on: the same arms,
    horizon, world and plans, CPU_SAMPLE_K samples per arm instead of K (a
    rollout's cost does not depend on K; the update's share is small)."""
    from paper_2602_10114_gb300 import scenarios as S
    return S.shrink(sc, K=min(CPU_SAMPLE_K, min(a.K for a in sc.arms)))


def time_oracle(sc, threads, budget_s, min_cycles=1):
    """Closed-loop oracle cycles of `sc` until budget_s of wall time is spent;
    returns (trajectory-steps/s, cycles, seconds)."""
    from oracle.oracle import Oracle
    orc = Oracle(sc, threads=threads)
    gp, gR = zip(*[orc.goal_pose(a, sc.goal_q[a]) for a in range(sc.n_arms)])
    gp, gR = np.asarray(gp), np.asarray(gR)
    orc.cycle(sc.q0, sc.qd0, gp, gR, want_costs=False)     # cycle 0: publishes the plans
    cycles, el = 0, 0.0
    while cycles < min_cycles or el < budget_s:
        t = time.perf_counter()
        orc.cycle(sc.q0, sc.qd0, gp, gR, want_costs=False)
        el += time.perf_counter() - t
        cycles += 1
    return sc.rollout_steps() * sc.params["iterations"] * cycles / el, cycles, el


def cpu_baseline(sc, budget_s=12.0):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the workload (oracle_sample), all cores (OpenMP over samples) and one
    thread."""
    smp = oracle_sample(sc)
    threads = os.cpu_count() or 1
    v_all, n_all, t_all = time_oracle(smp, threads, budget_s * 0.4)
    v_one, n_one, t_one = time_oracle(smp, 1, budget_s * 0.6)
    what = (f"{smp.arms[0].K} of the {sc.arms[0].K} samples per arm of the workload's "
            f"cycle (all {sc.n_arms} arms, H={sc.arms[0].H}, the same world and shared "
            f"plans), FP64 oracle")
    return {"value": v_all, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_all} cycles of {what}, OpenMP over samples, {threads} threads",
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                              "sample": f"{n_one} cycles of the same sample, 1 thread",
                              "seconds": t_one},
            "cpu_model": cpu_model(), "seconds": t_all}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    sc = workload(args.workload)
    smp = oracle_sample(sc)
    from oracle.oracle import Oracle
    threads = os.cpu_count() or 1
    orc = Oracle(smp, threads=threads)
    gp, gR = zip(*[orc.goal_pose(a, smp.goal_q[a]) for a in range(smp.n_arms)])
    gp, gR = np.asarray(gp), np.asarray(gR)
    for _ in range(max(args.warmup, 1)):
        orc.cycle(smp.q0, smp.qd0, gp, gR, want_costs=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.cycle(smp.q0, smp.qd0, gp, gR, want_costs=False)
    el = time.perf_counter() - t0
    units = smp.rollout_steps() * smp.params["iterations"] * args.steps
    value = units / el
    sample = (f"each step one control cycle with {smp.arms[0].K} of the {sc.arms[0].K} samples "
              f"per arm (all {sc.n_arms} arms, H={sc.arms[0].H}, same world and plans), FP64 "
              f"oracle, {threads} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": sc.name + ", exact costs, 1 iteration", "arms": sc.n_arms,
                       "K": sc.arms[0].K, "H": sc.arms[0].H},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU timing

def make_controller(sc, dev, shape=None):
    """A context with the world set, the goal poses, and the packed
    device-resident input of the scene's start state."""
    import torch
    from paper_2602_10114_gb300 import mrs
    ctl = mrs.Controller(sc, device=dev)
    ctl.set_world()
    gp, gR = [], []
    for a in range(sc.n_arms):
        p, R = ctl.goal_pose(a, sc.goal_q[a])
        gp.append(p)
        gR.append(R)
    if shape is not None:
        ctl.set_rollout_shape(shape["tile_samples"], shape["blocks_per_sm"], shape["order"])
    d_in = torch.from_numpy(ctl.pack_input(sc.q0, sc.qd0, gp, gR)).to(dev)
    ctl.step_device(d_in)
    ctl.sync()
    return ctl, gp, gR, d_in


def stage_names(sc):
    return ["prep"] + ["sample", "surrogate", "rollout", "costs", "update"] * \
        sc.params["iterations"] + ["toplan"]


def launches_per_cycle(kt):
    """Kernels of one cycle: the stages with a non-zero time."""
    return int(np.sum(np.asarray(kt).mean(axis=0) > 0))


def time_device(ctl, d_in, steps, warmup, flush, ws):
    """Per-cycle CUDA-event times (ms) of device-resident cycles, L2 flushed
    before each, with the cycle's graph as a user runs it (no timing nodes);
    then the per-stage times from a second run of the same cycles with event
    nodes between the stages."""
    import torch
    s = ctl.stream

    def loop(n, stages):
        ctl.enable_timing(stages)
        for _ in range(max(warmup, 3)):
            ctl.step_device(d_in)
        ctl.sync()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        kt = []
        barrier(ws)
        torch.cuda.synchronize()
        for i in range(n):
            with torch.cuda.stream(s):
                flush.zero_()          # 256 MiB write: also covers the host's launch latency
                starts[i].record(s)
            ctl.step_device(d_in)
            with torch.cuda.stream(s):
                ends[i].record(s)
            if stages:
                kt.append(ctl.kernel_times())
            else:
                ends[i].synchronize()
        torch.cuda.synchronize()
        barrier(ws)
        return [x.elapsed_time(y) for x, y in zip(starts, ends)], kt

    step_ms, _ = loop(steps, False)
    _, kt = loop(min(steps, 20), True)
    ctl.enable_timing(False)
    return step_ms, np.asarray(kt)


def time_e2e(ctls, sc, gp, gR, cycles, warmup, flush, ws, episode=50):
    """Wall-clock latency of mrs_step with host buffers, closed loop (the host
    plant integrates U_*, goals drift), in episodes of `episode` cycles that
    restart from the initial state.  `ctls` is one Controller holding every
    arm, or one Controller per arm (the others external, their plans passed
    through mrs_share_plans after each arm's call: one arm at a time)."""
    import torch
    from paper_2602_10114_gb300 import exchange
    ctls = ctls if isinstance(ctls, list) else [ctls]
    blobs = [c.save_state() for c in ctls]
    dt = np.float32(sc.params["dt"])

    def one_cycle(q, qd, gpl, k):
        outs = {}
        for c in ctls:
            out = c.step(q, qd, gpl, gR)
            if len(ctls) > 1:
                ents = exchange.local_entries(c, out, k)
                for o in ctls:
                    if o is not c:
                        exchange.share_remote(o, ents)
            for a in range(sc.n_arms):
                if a not in c.external:
                    outs[a] = c.split(out["u_star"], "d", a)
        return outs

    def episode_state():
        return ([x.astype(np.float32).copy() for x in sc.q0],
                [x.astype(np.float32).copy() for x in sc.qd0], [g.copy() for g in gp])

    q, qd, gpl = episode_state()
    for k in range(max(warmup, 3)):
        one_cycle(q, qd, gpl, k)
    lat = []
    barrier(ws)
    k = 0
    while len(lat) < cycles:
        if k % episode == 0:
            for c, b in zip(ctls, blobs):
                c.load_state(b)
            q, qd, gpl = episode_state()
        with torch.cuda.stream(ctls[0].stream):
            flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        u = one_cycle(q, qd, gpl, k)
        lat.append(time.perf_counter() - t)
        for a in range(sc.n_arms):
            qd[a] = (qd[a] + u[a] * dt).astype(np.float32)
            q[a] = (q[a] + qd[a] * dt).astype(np.float32)
            gpl[a] = (gpl[a] + sc.goal_vel[a] * dt).astype(np.float32)
        k += 1
    barrier(ws)
    for c, b in zip(ctls, blobs):
        c.load_state(b)
    return lat


def e2e_over_seeds(idx, runs, cycles, shape, args, flush, ws, dev, first=None):
    """mrs_step latency over `runs` seeded scenes of workload idx, `cycles`
    closed-loop cycles each (one episode per scene); `first` = an existing
    (ctl, sc, gp, gR) for run 0."""
    lat = []
    for run in range(runs):
        if run == 0 and first is not None:
            ctl, sc, gp, gR = first
            lat += time_e2e(ctl, sc, gp, gR, cycles, args.warmup, flush, ws, episode=cycles)
            continue
        sc = workload(idx, run)
        ctl, gp, gR, _ = make_controller(sc, dev, shape)
        lat += time_e2e(ctl, sc, gp, gR, cycles, args.warmup, flush, ws, episode=cycles)
        ctl.close()
    return lat


def e2e_summary(lat, units, ws, ctl, runs, cycles):
    e2e_s = max_over_ranks(float(np.mean(lat)), ws)
    return {"value": units * ws / e2e_s, "unit": UNIT,
            "h2d_bytes_per_step": int(4 * ctl.sizes.input_floats),
            "d2h_bytes_per_step": int(4 * ctl.sizes.output_floats + 4),
            "cycles": len(lat), "scenes": runs, "cycles_per_scene": cycles,
            "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
            "latency_ms_p99": 1e3 * float(np.percentile(lat, 99))}


def rollout_roofline(sc, kt):
    """FP32 roofline of one k_rollout launch: algorithmic work (the paper's
    brute-force pair count) over the live CUDA-event duration, against the
    FP32 peak from unit counts; executed-work figures and DRAM traffic from
    the committed ncu summary of the same kernel source (else null)."""
    names = stage_names(sc)
    roll_ms = float(np.mean([kt[:, i] for i, n in enumerate(names) if n == "rollout"]))
    flops = rollout_flops(sc) / sc.params["iterations"]
    achieved = flops / (roll_ms / 1e3) / 1e12
    fig, src = profile_figures()
    out = {"kernel": "k_rollout", "bound": "alu", "achieved": achieved,
           "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
           "frac_brute_force": achieved / FP32_PEAK_TFLOPS,
           "frac_note": "achieved counts every sphere pair brute force (Sec. IV-A's N_Q); the "
                        "kernel's box culls skip most of them, so this fraction can exceed 1; "
                        "'executed' gives the hardware's own use of the FP32 pipe and issue "
                        "slots from ncu",
           "traffic": None, "peak_source": "FP32 FMA peak from unit counts and the maximum SM "
                                          "clock (152 SMs x 128 lanes x 2 x 2.07 GHz)",
           "flops_per_launch": flops, "launch_ms": roll_ms}
    if fig is not None:
        out["traffic"] = float(fig["dram_bytes_per_launch"])
        out["executed"] = {k: float(fig[k]) for k in fig
                           if k not in ("source_sha256", "dram_bytes_per_launch", "workload")}
        out["executed"]["source"] = src
    else:
        out["executed"] = {"source": None, "why": src}
    return out


# ---------------------------------------------------------------------------
# forms of the cycle

def plain_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units, dev, e2e_cycles, attach=None):
    """The same kernels one arm at a time: one context per arm (the other arms
    external, their plans shared), all on one stream, each cycle launched
    kernel by kernel without a CUDA graph; exact costs, or with attach(ctx,
    arm) the learned terms of that arm."""
    import torch
    from paper_2602_10114_gb300 import exchange, mrs
    A = sc.n_arms
    ctls = [mrs.Controller(sc, device=dev, stream=ctl.stream,
                           external=[b for b in range(A) if b != a]) for a in range(A)]
    # every context sees the other arms' plans from one batched cycle
    out = ctl.step(sc.q0, sc.qd0, gp, gR)
    ents = exchange.local_entries(ctl, out, 0)
    for a, c in enumerate(ctls):
        c.set_world()
        c.use_graph(False)
        exchange.share_remote(c, ents)
        if attach is not None:
            attach(c, a)
    s = ctl.stream
    for _ in range(max(args.warmup, 3)):
        for c in ctls:
            c.step_device(d_in)
    torch.cuda.synchronize()
    steps = max(5, args.steps // 5)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier(ws)
    for i in range(steps):
        with torch.cuda.stream(s):
            flush.zero_()
            starts[i].record(s)
        for c in ctls:
            c.step_device(d_in)
        with torch.cuda.stream(s):
            ends[i].record(s)
    torch.cuda.synchronize()
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = max_over_ranks(float(np.mean(step_ms)), ws)
    lat = time_e2e(ctls, sc, gp, gR, e2e_cycles, args.warmup, flush, ws, episode=e2e_cycles)
    e2e_s = max_over_ranks(float(np.mean(lat)), ws)
    for c in ctls:
        c.close()
    return {"value": units * ws / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "device_p50": float(np.percentile(step_ms, 50)),
            "device_p99": float(np.percentile(step_ms, 99)),
            "e2e": {"value": units * ws / e2e_s, "cycles": len(lat),
                    "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                    "latency_ms_p99": 1e3 * float(np.percentile(lat, 99))}}


def learned_self_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units, exact_ms, plain_dev=None,
                      target_fn=None):
    """The same cycle with the self-collision surrogate (trained here, on the
    device, by the library's kernels; one network per arm geometry):
    throughput, latency, false negatives, skip fraction and cost deviation
    against exact mode.  The fallback margin is workload 3's 0.03 m, or with
    target_fn each network's margin calibrated on half of its held-out
    samples to that false-negative rate (workload 4 fixes no margin)."""
    from paper_2602_10114_gb300 import surrogate
    groups = {}
    for a, arm in enumerate(sc.arms):
        groups.setdefault((arm.dof, arm.dh.tobytes(), arm.sphere_xyzr.tobytes()), []).append(a)
    nets, stats = [], []
    for arms in groups.values():
        net, st = surrogate.train_self_surrogate(ctl, arms[0], n_train=args.surrogate_samples,
                                                 n_val=400_000 if target_fn else 200_000,
                                                 epochs=8, lr=2e-3, target_fn=target_fn)
        nets.append(net)
        stats.append(st)
        for a in arms:
            ctl.set_self_surrogate(a, net, st["margin"])
    margin_of = {a: st["margin"] for arms, st in zip(groups.values(), stats) for a in arms}
    # cost deviation on one cycle from the same state
    blob = ctl.save_state()
    for a in range(sc.n_arms):
        ctl.set_self_surrogate(a, None)
    ctl.step_device(d_in)
    ctl.sync()
    c_exact = np.concatenate([ctl.debug_costs(a) for a in range(sc.n_arms)])
    for arms, net in zip(groups.values(), nets):
        for a in arms:
            ctl.set_self_surrogate(a, net, margin_of[a])
    ctl.load_state(blob)
    ctl.step_device(d_in)
    ctl.sync()
    c_learned = np.concatenate([ctl.debug_costs(a) for a in range(sc.n_arms)])
    B_self = float(np.float32(sc.params["B_self"]))
    evs = [surrogate.evaluate(*ctl.debug_self(a), B_self, margin_of[a]) for a in range(sc.n_arms)]
    ev = {"samples": sum(e["samples"] for e in evs), "colliding": sum(e["colliding"] for e in evs),
          "fn_rate": sum(e["false_negatives"] for e in evs) / max(1, sum(e["colliding"] for e in evs)),
          "skip_fraction": float(np.mean([e["skip_fraction"] for e in evs])),
          "mae": float(np.mean([e["mae"] for e in evs]))}
    step_ms, kt = time_device(ctl, d_in, args.steps, args.warmup, flush, ws)
    ms = max_over_ranks(float(np.mean(step_ms)), ws)
    lat = time_e2e(ctl, sc, gp, gR, args.latency_cycles, args.warmup, flush, ws)
    e2e_s = max_over_ranks(float(np.mean(lat)), ws)
    for a in range(sc.n_arms):
        ctl.set_self_surrogate(a, None)
    plain = None
    if plain_dev is not None:
        net_of = {a: net for arms, net in zip(groups.values(), nets) for a in arms}
        plain = plain_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units, plain_dev,
                           args.plain_cycles,
                           attach=lambda c, a: c.set_self_surrogate(a, net_of[a], margin_of[a]))
    dev = np.abs(c_learned - c_exact)
    sur_ms = float(kt[:, 2].mean())
    fl = self_mlp_flops(sc)
    pk = measured_peaks()
    return {
        "value": units * ws / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
        "speedup_vs_exact": exact_ms / ms,
        "e2e": {"value": units * ws / e2e_s, "cycles": len(lat),
                "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                "latency_ms_p99": 1e3 * float(np.percentile(lat, 99))},
        "surrogate_ms": sur_ms, "rollout_ms": float(kt[:, 3].mean()),
        "roofline": {"kernel": "k_mlp_fused", "bound": "tensor",
                     "achieved": fl / (sur_ms / 1e3) / 1e12, "peak": pk["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": fl / (sur_ms / 1e3) / 1e12 / pk["bf16_tflops"],
                     "peak_source": pk["source"] + " BF16 burst", "flops_per_launch": fl},
        "held_out": {k: (stats[0][k] if len(stats) == 1 else [st[k] for st in stats])
                     for k in ("fn_rate", "fn_rate_active", "skip_fraction", "mae", "colliding",
                               "samples", "margin")},
        "rollout_steps": {k: ev[k] for k in ("fn_rate", "skip_fraction", "mae", "colliding",
                                             "samples")},
        "cost_deviation": {"mean_rel": float(dev.mean() / np.abs(c_exact).mean()),
                           "max_abs": float(dev.max())},
        "train": {"samples": args.surrogate_samples, "epochs": 8,
                  "seconds": float(sum(st["train_seconds"] for st in stats)),
                  "networks": len(nets), "architecture": "2d sin/cos -> 3 x 256 SiLU -> 1, BF16"},
        "plain": plain,
    }


def learned_pair_mode(ctl, sc, gp, gR, d_in, args, flush, ws, exact_ms, plain_dev=None):
    """The headline workload with both learned clearances: the self-collision
    network and the arm-pair network (asymmetric loss, fallback margin
    calibrated on half of the held-out pairs to a 5e-4 false-negative rate,
    so that the other half stays within the 1e-3 target), trained on the
    device; throughput against exact mode, false negatives on held-out
    samples and on every rollout step of a cycle, skip fractions, cost
    deviation."""
    from paper_2602_10114_gb300 import surrogate
    t0 = time.perf_counter()
    snet, sst = surrogate.train_self_surrogate(ctl, 0, n_train=args.surrogate_samples, n_val=400_000,
                                               epochs=8, lr=2e-3, target_fn=5e-4)
    pnet, pst = surrogate.train_pair_surrogate(ctl, 0, n_train=args.pair_samples, n_val=400_000,
                                               epochs=12, lr=1e-3, over_weight=32.0,
                                               target_fn=5e-4)
    train_s = time.perf_counter() - t0
    blob = ctl.save_state()
    ctl.step_device(d_in)
    ctl.sync()
    c_exact = np.concatenate([ctl.debug_costs(a) for a in range(sc.n_arms)])
    for a in range(sc.n_arms):
        ctl.set_self_surrogate(a, snet, sst["margin"])
        ctl.set_pair_surrogate(a, -1, pnet, pst["margin"])
    ctl.load_state(blob)
    ctl.step_device(d_in)
    ctl.sync()
    c_learned = np.concatenate([ctl.debug_costs(a) for a in range(sc.n_arms)])
    B = float(np.float32(sc.params["B"]))
    pr = [ctl.debug_pair(0, b) for b in range(1, sc.n_arms)]
    ev_pair = surrogate.evaluate(np.concatenate([r[0].ravel() for r in pr]),
                                 np.concatenate([r[1].ravel() for r in pr]), B, pst["margin"])
    sr = [ctl.debug_self(a) for a in range(sc.n_arms)]
    ev_self = surrogate.evaluate(np.concatenate([r[0].ravel() for r in sr]),
                                 np.concatenate([r[1].ravel() for r in sr]),
                                 float(np.float32(sc.params["B_self"])), sst["margin"])
    steps = max(5, args.steps // 5)
    ln_ms, kt = time_device(ctl, d_in, steps, 3, flush, ws)
    ln = max_over_ranks(float(np.mean(ln_ms)), ws)
    for a in range(sc.n_arms):
        ctl.set_self_surrogate(a, None)
        ctl.set_pair_surrogate(a, -1, None)
    ctl.load_state(blob)
    units = sc.rollout_steps() * sc.params["iterations"]

    def attach(c, a):
        c.set_self_surrogate(a, snet, sst["margin"])
        c.set_pair_surrogate(a, -1, pnet, pst["margin"])
    plain = None
    if plain_dev is not None:
        plain = plain_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units, plain_dev,
                           max(20, args.plain_cycles // 5), attach=attach)
        ctl.load_state(blob)
    dev_ = np.abs(c_learned - c_exact)
    keep = ("fn_rate", "fn_rate_active", "skip_fraction", "mae", "colliding", "samples")
    return {"workload": sc.name + ", learned self + arm-pair clearance",
            "value": units * ws / (ln / 1e3), "unit": UNIT, "ms_per_step": ln,
            "exact_ms_per_step": exact_ms, "speedup_vs_exact": exact_ms / ln, "steps": steps,
            "surrogate_ms": float(kt[:, 2].mean()), "rollout_ms": float(kt[:, 3].mean()),
            "pair_margin": pst["margin"], "self_margin": sst["margin"],
            "held_out": {"self": {k: sst[k] for k in keep}, "pair": {k: pst[k] for k in keep}},
            "rollout_steps": {"self": {k: ev_self[k] for k in keep},
                              "pair": {k: ev_pair[k] for k in keep}},
            "cost_deviation": {"mean_rel": float(dev_.mean() / np.abs(c_exact).mean()),
                               "max_abs": float(dev_.max())},
            "train": {"self_samples": args.surrogate_samples, "pair_samples": args.pair_samples,
                      "seconds": train_s,
                      "architecture": "self 14 -> 3 x 256 SiLU -> 1; pair 35 -> 4 x 256 SiLU "
                                      "-> 1, BF16"},
            "plain": plain}


def other_workload(idx, args, flush, ws, dev):
    """Device-timed cycles of another workload (exact costs, autotuned shape):
    throughput, cycle time, rollout time and its FP32 roofline fraction; for
    workload 2 also its mrs_step latency over 20 scenes x 50 cycles; "3" is
    workload 2 with the learned self network."""
    learned = str(idx) == "3"
    sc = workload(2 if learned else idx)
    ctl, gp, gR, d_in = make_controller(sc, dev)
    best, table = ctl.autotune(reps=3)
    steps = max(5, args.steps // 2)
    step_ms, kt = time_device(ctl, d_in, steps, 3, flush, ws)
    ms = max_over_ranks(float(np.mean(step_ms)), ws)
    units = sc.rollout_steps() * sc.params["iterations"]
    it = sc.params["iterations"]
    roll = float(np.mean([kt[:, 3 + 5 * i] for i in range(it)]))     # one rollout launch
    fl = rollout_flops(sc) / it
    res = {"workload": sc.name, "value": units * ws / (ms / 1e3), "unit": UNIT,
           "ms_per_step": ms, "steps": steps, "rollout_ms": roll,
           "rollout_shape": best, "roofline_frac_brute_force": fl / (roll / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
           "flops_per_launch": fl}
    pdev = None if args.no_plain else dev
    if learned:
        res = {"workload": sc.name + ", learned self-collision clearance (workload 3)",
               "exact": res}
        if pdev is not None:
            res["exact"]["plain"] = plain_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units,
                                               pdev, args.plain_cycles)
        res.update(learned_self_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units, ms, pdev))
    elif str(idx) == "4" and not args.no_learned:
        res["learned"] = learned_self_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units, ms,
                                           target_fn=5e-4)
    elif str(idx) == "2" and not args.no_e2e_others:
        lat = e2e_over_seeds(2, 20, 50, best, args, flush, ws, dev, first=(ctl, sc, gp, gR))
        res["e2e"] = e2e_summary(lat, units, ws, ctl, 20, 50)
    ctl.close()
    return res


def run(args):
    import torch

    from paper_2602_10114_gb300 import build

    ws, rank, local = dist_setup()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    build.build()
    sc = workload(args.workload)
    units_per_step = sc.rollout_steps() * sc.params["iterations"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ctl, gp, gR, d_in = make_controller(sc, dev)
    tune = None
    if args.rollout_shape:
        t, b, o = (int(x) for x in args.rollout_shape.split(","))
        ctl.set_rollout_shape(t, b, o)
        tune = {"given": {"tile_samples": t, "blocks_per_sm": b, "order": o}}
    elif not args.no_autotune:
        best, table = ctl.autotune(reps=5)
        tune = {"chosen": best, "tried": len(table)}
    shape = dict(zip(("tile_samples", "blocks_per_sm", "order"), ctl.rollout_shape()[0]))

    # ---- device-resident cycles (exact costs) ------------------------------
    clk = ClockSampler(local)
    clk.__enter__()
    step_ms, kt = time_device(ctl, d_in, args.steps, args.warmup, flush, ws)
    ms_max = max_over_ranks(float(np.mean(step_ms)), ws)
    value = units_per_step * ws / (ms_max / 1e3)
    names = stage_names(sc)
    k_mean = {n: float(kt[:, i].mean()) for i, n in enumerate(names[:kt.shape[1]])
              if n != "surrogate"}
    roof = rollout_roofline(sc, kt)

    # ---- end to end through mrs_step with host buffers ---------------------
    runs = args.e2e_scenes
    per = max(1, args.latency_cycles // runs)
    lat = e2e_over_seeds(args.workload, runs, per, shape, args, flush, ws, dev,
                         first=(ctl, sc, gp, gR))
    e2e = e2e_summary(lat, units_per_step, ws, ctl, runs, per)
    clk.__exit__()
    clocks = clk.summary()

    plain = None
    if not args.no_plain:
        plain = plain_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units_per_step, dev,
                           args.plain_cycles)
    learned = None
    if not args.no_learned:
        pdev = None if args.no_plain else dev
        if len(sc.arms) > 1 and str(args.workload) == "5":
            learned = learned_pair_mode(ctl, sc, gp, gR, d_in, args, flush, ws, ms_max, pdev)
        else:
            learned = learned_self_mode(ctl, sc, gp, gR, d_in, args, flush, ws, units_per_step,
                                        ms_max, pdev)
    ctl.close()
    others = {}
    for idx in args.other_workloads:
        others[f"cfg{idx}"] = other_workload(idx, args, flush, ws, dev)
    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, budget_s=args.cpu_budget)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": sc.name + ", exact costs, 1 iteration", "arms": sc.n_arms,
                   "K": sc.arms[0].K, "H": sc.arms[0].H, "dof": sc.arms[0].dof,
                   "spheres": sc.arms[0].n_spheres, "world_spheres": int(len(sc.world)),
                   "moving_world": sc.world_vel is not None, "boxes": int(len(sc.aabb)),
                   "rollout_steps_per_cycle": units_per_step, "mode": "exact",
                   "l2": "flushed (256 MiB write) before every timed cycle",
                   "parallelism": f"replicas x{ws}", "graph": True,
                   "rollout_shape": tune},
        "latency_ms": {"device_p50": float(np.percentile(step_ms, 50)),
                       "device_p99": float(np.percentile(step_ms, 99))},
        "kernel_ms": k_mean,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "plain": plain,
        "learned": learned,
        "other_workloads": others,
        "gpu_launches": launches_per_cycle(kt) * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="5")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle time for the CPU baseline (both legs)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-surrogate comparison")
    ap.add_argument("--surrogate-samples", type=int, default=2_000_000)
    ap.add_argument("--pair-samples", type=int, default=5_000_000)
    ap.add_argument("--other-workloads", nargs="*", default=["2", "3", "4", "M"],
                    help="also time these workloads (device-resident, autotuned; 3 = workload "
                         "2 with the learned self network)")
    ap.add_argument("--no-e2e-others", action="store_true",
                    help="skip the mrs_step latency of the other workloads")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default rollout shape")
    ap.add_argument("--rollout-shape", default="",
                    help="tile_samples,blocks_per_sm,order: use this rollout shape instead of "
                         "the autotuner's (e.g. to profile the shape a run chose)")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the one-arm-at-a-time, graph-free comparison")
    ap.add_argument("--plain-cycles", type=int, default=200,
                    help="closed-loop cycles of the plain form's latency")
    ap.add_argument("--latency-cycles", type=int, default=1000,
                    help="closed-loop mrs_step calls for the latency percentiles")
    ap.add_argument("--e2e-scenes", type=int, default=5,
                    help="seeded scenes the latency cycles are spread over")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()

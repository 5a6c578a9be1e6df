"""Benchmark of the batched multi-arm MPPI control cycle on GB300.

One "step" is one control cycle of every arm (Algorithm 1: sense, shift,
sample, rollout, update, ToPlan/publish) on the four-arm workload (4 arms x 7
DoF, 40 spheres each, K=512 samples, H=30 steps, 32 world spheres + 4 boxes,
all plans shared, exact costs).  The metric is rollout trajectory-steps per
second: sum_a K_a H_a x iterations / cycle time.

  value : device-resident inputs, per-cycle CUDA-event time on the
          library's stream, L2 flushed (256 MiB write) between timed cycles.
  e2e   : the same cycles through mrs_step with host buffers (H2D of the
          sensed state, D2H of the results inside the timed region), wall
          clock per call, closed loop (the host plant integrates U_*).

`--impl reference` times the FP64 CPU oracle on the host cores instead.
With torchrun (N > 1) every rank runs an independent replica on its own GPU
(the arms of one replica couple through the plan board, which stays on one
device); value is the sum over ranks of the work divided by the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rollout trajectory-steps/s and control-cycle p50/p99 latency, learned vs exact"
UNIT = "trajectory-steps/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def workload(idx):
    from paper_2602_10114_gb300 import scenarios as S
    return S.config(idx)


def rollout_flops(sc):
    """Algorithmic FP32 work of one rollout launch, counted brute force as the
    paper counts distance queries: 10 flops (+1 sqrt) per sphere pair (world,
    self, every other arm's plan at the same step), plus 60 d + 18 N_S per
    rollout step for the kinematics."""
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


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out"))
                                 else "_build", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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


def cpu_baseline(sc, budget_s=12.0, threads=None):
    """The FP64 oracle, as it stands, on the host cores: full control cycles of
    the same workload until `budget_s` of wall time is spent (>= 1 cycle)."""
    from oracle.oracle import Oracle
    threads = threads or os.cpu_count()
    orc = Oracle(sc, threads=threads)
    gp, gR = zip(*[orc.goal_pose(a, sc.goal_q[a]) for a in range(sc.n_arms)])
    gp, gR = np.asarray(gp), np.asarray(gR)
    cycles, t0 = 0, time.perf_counter()
    times = []
    while True:
        t = time.perf_counter()
        orc.cycle(sc.q0, sc.qd0, gp, gR, want_costs=False)
        times.append(time.perf_counter() - t)
        cycles += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = sum(times)
    return {"value": sc.rollout_steps() * sc.params["iterations"] * cycles / el, "unit": UNIT,
            "cores": threads, "kind": "oracle",
            "sample": f"{cycles} full control cycles of the workload (FP64 oracle, OpenMP over "
                      f"samples, {threads} threads)",
            "ms_per_cycle": 1e3 * el / cycles}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    sc = workload(args.workload)
    from oracle.oracle import Oracle
    threads = os.cpu_count()
    orc = Oracle(sc, threads=threads)
    gp, gR = zip(*[orc.goal_pose(a, sc.goal_q[a]) for a in range(sc.n_arms)])
    gp, gR = np.asarray(gp), np.asarray(gR)
    for _ in range(args.warmup):
        orc.cycle(sc.q0, sc.qd0, gp, gR, want_costs=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.cycle(sc.q0, sc.qd0, gp, gR, want_costs=False)
    el = time.perf_counter() - t0
    units = sc.rollout_steps() * sc.params["iterations"] * args.steps
    value = units / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": sc.name + ", exact costs, 1 iteration", "arms": sc.n_arms,
                       "K": sc.arms[0].K, "H": sc.arms[0].H},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"each step one full control cycle of the workload "
                                       f"(FP64 oracle, {threads} threads)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run(args):
    import torch

    from paper_2602_10114_gb300 import build, mrs

    ws, rank, local = dist_setup()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    build.build()
    sc = workload(args.workload)
    ctl = mrs.Controller(sc, device=dev)
    ctl.set_world()
    gp, gR = [], []
    for a in range(sc.n_arms):
        p, R = ctl.goal_pose(a, sc.goal_q[a])
        gp.append(p)
        gR.append(R)
    units_per_step = sc.rollout_steps() * sc.params["iterations"]
    s = ctl.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # ---- device-resident cycles -------------------------------------------
    d_in = torch.from_numpy(ctl.pack_input(sc.q0, sc.qd0, gp, gR)).to(dev)
    ctl.enable_timing(True)
    for _ in range(max(args.warmup, 3)):
        ctl.step_device(d_in)
    ctl.sync()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ktimes = []
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(s):
                flush.zero_()
                starts[i].record(s)
            ctl.step_device(d_in)
            with torch.cuda.stream(s):
                ends[i].record(s)
            ktimes.append(ctl.kernel_times())
        torch.cuda.synchronize()
    barrier(ws)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = float(np.mean(step_ms))
    ms_max = max_over_ranks(ms, ws)
    value = units_per_step * ws / (ms_max / 1e3)
    kt = np.asarray(ktimes)            # [steps][kernels]
    names = ["prep"] + ["sample", "surrogate", "rollout", "costs", "update"] * sc.params["iterations"] + ["toplan"]
    k_mean = {n: float(kt[:, i].mean()) for i, n in enumerate(names[:kt.shape[1]])}
    roll_ms = float(np.mean([kt[:, i] for i, n in enumerate(names) if n == "rollout"]))
    flops = rollout_flops(sc) / sc.params["iterations"]
    achieved = flops / (roll_ms / 1e3) / 1e12
    ctl.enable_timing(False)

    # ---- end to end through mrs_step with host buffers ---------------------
    q = [x.astype(np.float32).copy() for x in sc.q0]
    qd = [x.astype(np.float32).copy() for x in sc.qd0]
    gpl = [g.copy() for g in gp]
    dt = np.float32(sc.params["dt"])
    for _ in range(max(args.warmup, 3)):
        ctl.step(q, qd, gpl, gR)
    lat = []
    barrier(ws)
    for i in range(args.steps):
        with torch.cuda.stream(s):
            flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = ctl.step(q, qd, gpl, gR)
        lat.append(time.perf_counter() - t)
        for a in range(sc.n_arms):     # host plant: Execute(U_*), goals drift
            u = ctl.split(out["u_star"], "d", a)
            qd[a] = (qd[a] + u * dt).astype(np.float32)
            q[a] = (q[a] + qd[a] * dt).astype(np.float32)
            gpl[a] = (gpl[a] + sc.goal_vel[a] * dt).astype(np.float32)
    barrier(ws)
    e2e_s = max_over_ranks(float(np.mean(lat)), ws)
    e2e = {"value": units_per_step * ws / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(4 * ctl.sizes.input_floats),
           "d2h_bytes_per_step": int(4 * ctl.sizes.output_floats + 4),
           "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
           "latency_ms_p99": 1e3 * float(np.percentile(lat, 99))}

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, budget_s=args.cpu_budget)
        cpu.pop("ms_per_cycle", None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": sc.name + ", exact costs, 1 iteration", "arms": sc.n_arms,
                   "K": sc.arms[0].K, "H": sc.arms[0].H, "dof": sc.arms[0].dof,
                   "spheres": sc.arms[0].n_spheres, "world_spheres": int(len(sc.world)),
                   "boxes": int(len(sc.aabb)), "mode": "exact",
                   "l2": "flushed (256 MiB write) before every timed cycle",
                   "parallelism": f"replicas x{ws}", "graph": True},
        "latency_ms": {"device_p50": float(np.percentile(step_ms, 50)),
                       "device_p99": float(np.percentile(step_ms, 99))},
        "kernel_ms": k_mean,
        "roofline": {"kernel": "k_rollout", "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                     "peak_source": "FP32 FMA peak from unit counts and the maximum SM clock "
                                    "(152 SMs x 128 lanes x 2 x 2.07 GHz)",
                     "flops_per_launch": flops},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int((2 + 4 * sc.params["iterations"]) * args.steps),   # no surrogate
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()

"""Plan exchange between processes (Algorithm 1, Publish, across a process
boundary; Sec. IV-A: plans go to the other arms through pub-sub).

Each process controls some arms of a shared scene (its local arms; the
others are declared `external` in its context) and, after every cycle,
publishes its local arms' board entries: the anticipated plan (sphere
trajectory and joint plan), the distance-to-goal sent with it, and the
publication stamp.  `all_gather_entries` exchanges them over
torch.distributed (gloo between CPU ranks, NCCL between GPUs); each process
then writes the remote entries into its own board (`mrs_share_plans`).  The
exchange is host-staged: one flat float64 vector per rank.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class PlanEntry:
    arm: int
    stamp: int
    dist_to_goal: float
    plan_spheres: np.ndarray   # [H][NS][4]
    plan_q: np.ndarray         # [H][dof]


def pack(entries, sc) -> np.ndarray:
    """Flatten entries: per entry [arm, stamp, dist, spheres..., q...]."""
    parts = [np.array([len(entries)], np.float64)]
    for e in entries:
        a = sc.arms[e.arm]
        parts.append(np.array([e.arm, e.stamp, e.dist_to_goal], np.float64))
        parts.append(np.asarray(e.plan_spheres, np.float64).reshape(a.H * a.n_spheres * 4))
        parts.append(np.asarray(e.plan_q, np.float64).reshape(a.H * a.dof))
    return np.concatenate(parts)


def unpack(buf, sc):
    out, o = [], 1
    for _ in range(int(buf[0])):
        arm, stamp, dist = int(buf[o]), int(buf[o + 1]), float(buf[o + 2])
        o += 3
        a = sc.arms[arm]
        ns = a.H * a.n_spheres * 4
        sph = buf[o:o + ns].reshape(a.H, a.n_spheres, 4)
        o += ns
        q = buf[o:o + a.H * a.dof].reshape(a.H, a.dof)
        o += a.H * a.dof
        out.append(PlanEntry(arm, stamp, dist, sph.copy(), q.copy()))
    return out


def all_gather_entries(entries, sc, group=None):
    """Every rank's entries, gathered on every rank (lengths first, then one
    padded all-gather)."""
    import torch
    import torch.distributed as dist
    buf = pack(entries, sc)
    dev = torch.device("cpu")
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    n = torch.tensor([buf.size], dtype=torch.int64, device=dev)
    ws = dist.get_world_size(group)
    sizes = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(sizes, n, group=group)
    m = int(max(int(s.item()) for s in sizes))
    t = torch.zeros(m, dtype=torch.float64, device=dev)
    t[:buf.size] = torch.from_numpy(buf).to(dev)
    got = [torch.zeros_like(t) for _ in range(ws)]
    dist.all_gather(got, t, group=group)
    out = []
    for g, s in zip(got, sizes):
        out += unpack(g[:int(s.item())].cpu().numpy(), sc)
    return out


def local_entries(ctl, result, cycle):
    """Board entries of a Controller's local arms after a step (`result` is
    the dict mrs.Controller.step returns; `cycle` the step's index)."""
    out = []
    for a in range(len(ctl.sc.arms)):
        if a in ctl.external:
            continue
        out.append(PlanEntry(a, cycle, float(result["dist_to_goal"][a]),
                             ctl.split(result["plan_spheres"], "hs", a),
                             ctl.split(result["plan_q"], "hd", a)))
    return out


def share_remote(ctl, entries):
    """Write the entries of this context's external arms into its board."""
    for e in entries:
        if e.arm in ctl.external:
            ctl.share_plans(e.arm, np.asarray(e.plan_spheres, np.float32),
                            np.asarray(e.plan_q, np.float32), e.dist_to_goal, e.stamp)

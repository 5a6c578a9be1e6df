"""Closed-loop task harness on the kinematic plant.

Runs the method's variants of Sec. V-A on a seeded multi-arm workload for
T_max control cycles, with the plant integrating each arm's U_* over one
period (the integrator of the rollout), and reports the paper's scores
(Sec. V-A, Reporting):

  * collision score: the cycles in which any arm touches a world obstacle or
    another arm (a sphere pair of negative clearance at the actual state);
  * following task: the mean end-effector tracking error err_f over cycles
    and arms, the goals drifting at constant velocity and reset to their
    start when they leave the arm's reach;
  * reaching task: the goals reached (end-effector within 5 cm), each arm then
    getting the next goal of its seeded list.

Variants (Sec. V-A): M (5 iterations per cycle), M_fast (1 iteration),
M_tau (tau = 0: plans shared, no priority), S_d (independent controllers that
see the other arms only as static obstacles at their current sphere
positions: no plan, no priority).  The IsaacSim scenes and robots are not
available; the seeded arms around a shared centre stand in for them.

    python -m paper_2602_10114_gb300.harness --workload 2 --cycles 500 --runs 3
"""
from __future__ import annotations

import argparse
import copy
import json

import numpy as np

from . import mrs
from . import scenarios as S

VARIANTS = {
    "M": dict(iterations=5),
    "M_fast": dict(iterations=1),
    "M_tau": dict(iterations=1, tau=0.0),
    "S_d": dict(iterations=1, w_dyn=0.0),
}


def sphere_box_distance(c, r, box):
    """Signed distance of spheres (centres c [n][3], radii r [n]) to an
    axis-aligned box (centre, half extents): outside, distance to the surface
    minus r; inside, minus the depth to the nearest face, minus r."""
    d = np.abs(c - box[:3]) - box[3:6]
    outside = np.linalg.norm(np.maximum(d, 0.0), axis=1)
    inside = np.minimum(np.max(d, axis=1), 0.0)
    return outside + inside - r


def contacts(spheres, world, aabb):
    """(arm-to-arm contact, world contact) at one state: spheres is a list
    of [N_S][4] arrays (centre, radius), one per arm; world [n][4] spheres,
    aabb [m][6] boxes."""
    arm = False
    for i in range(len(spheres)):
        for j in range(i + 1, len(spheres)):
            a, b = spheres[i], spheres[j]
            d = np.linalg.norm(a[:, None, :3] - b[None, :, :3], axis=2) - a[:, None, 3] - b[None, :, 3]
            if d.min() < 0:
                arm = True
    wc = False
    for s in spheres:
        if len(world):
            d = np.linalg.norm(s[:, None, :3] - world[None, :, :3], axis=2) - s[:, None, 3] - world[None, :, 3]
            wc |= bool(d.min() < 0)
        for box in aabb:
            wc |= bool(sphere_box_distance(s[:, :3], s[:, 3], box).min() < 0)
    return arm, wc


def run_episode(sc, variant, cycles=500, task="following", device="cuda", reach_tol=0.05,
                goal_seed=0):
    """One episode of `variant` on scenario `sc`; returns the scores."""
    s = copy.deepcopy(sc)
    s.params.update(VARIANTS[variant])
    A = s.n_arms
    if variant == "S_d":
        ctls = [mrs.Controller(s, device=device, external=[b for b in range(A) if b != a])
                for a in range(A)]
    else:
        ctls = [mrs.Controller(s, device=device)]
    ref = ctls[0]
    world = np.asarray(s.world, np.float32).reshape(-1, 4)
    vel = None if s.world_vel is None else np.asarray(s.world_vel, np.float32).reshape(-1, 3)
    aabb = np.asarray(s.aabb, np.float32).reshape(-1, 6)
    for c in ctls:
        c.set_world(world, vel, aabb)
    dt = np.float32(s.params["dt"])
    q = [np.asarray(x, np.float32).copy() for x in s.q0]
    qd = [np.asarray(x, np.float32).copy() for x in s.qd0]
    # goals: following, the seeded goal drifting; reaching, a seeded list
    rng = np.random.default_rng(goal_seed)
    reach = [float(np.sum(np.abs(a.dh[:, 0])) + np.sum(np.abs(a.dh[:, 1]))) for a in s.arms]
    base = [np.asarray(a.base_pose[:3], np.float64) for a in s.arms]
    start = [ref.goal_pose(a, s.goal_q[a]) for a in range(A)]
    gp = [p.copy() for p, _ in start]
    gR = [R.copy() for _, R in start]
    goals_reached = 0
    err = 0.0
    coll_steps = arm_steps = world_steps = 0
    for t in range(cycles):
        if variant == "S_d":
            u = [None] * A
            sph = [ref.fk(a, q[a])[1][0] for a in range(A)]
            for a in range(A):
                others = np.concatenate([sph[b] for b in range(A) if b != a])
                w = np.concatenate([world, others])
                v = None if vel is None else np.concatenate([vel, np.zeros((len(others), 3), np.float32)])
                ctls[a].set_world(w, v, aabb)
                out = ctls[a].step(q, qd, gp, gR)
                u[a] = ctls[a].split(out["u_star"], "d", a)
        else:
            out = ref.step(q, qd, gp, gR)
            u = [ref.split(out["u_star"], "d", a) for a in range(A)]
        for a in range(A):
            qd[a] = (qd[a] + u[a] * dt).astype(np.float32)
            q[a] = (q[a] + qd[a] * dt).astype(np.float32)
        # scores at the new state
        ee, sph = [], []
        for a in range(A):
            e, sp = ref.fk(a, q[a])
            ee.append(e[0, 9:12].astype(np.float64))
            sph.append(sp[0].astype(np.float64))
        w_now = world.astype(np.float64).copy()
        if vel is not None:
            w_now[:, :3] += vel * float(dt) * (t + 1)
        arm_c, world_c = contacts(sph, w_now, aabb.astype(np.float64))
        arm_steps += arm_c
        world_steps += world_c
        coll_steps += arm_c or world_c
        for a in range(A):
            dist = float(np.linalg.norm(ee[a] - gp[a]))
            err += dist
            if task == "reaching" and dist < reach_tol:
                goals_reached += 1
                qg = rng.uniform(s.arms[a].q_lo, s.arms[a].q_hi).astype(np.float32)
                gp[a], gR[a] = ref.goal_pose(a, qg)
            elif task == "following":
                gp[a] = (gp[a] + s.goal_vel[a] * dt).astype(np.float32)
                if np.linalg.norm(gp[a] - base[a]) > reach[a]:
                    gp[a] = start[a][0].copy()
    for c in ctls:
        c.close()
    return {"variant": variant, "task": task, "cycles": cycles, "collision_score": coll_steps,
            "arm_contact_steps": arm_steps, "world_contact_steps": world_steps,
            "err_f": err / (cycles * A), "goals_reached": goals_reached}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--cycles", type=int, default=500)
    ap.add_argument("--runs", type=int, default=3, help="seeded scenarios per variant")
    ap.add_argument("--task", default="following", choices=["following", "reaching"])
    ap.add_argument("--variants", nargs="*", default=list(VARIANTS))
    ap.add_argument("--n-world", type=int, default=None,
                    help="keep only this many world spheres and no boxes (difficulty level)")
    args = ap.parse_args()
    from . import build
    build.build()
    rows = []
    for run in range(args.runs):
        sc = S.config(args.workload, run=run)
        if args.n_world is not None:
            sc = S.shrink(sc, n_world=args.n_world)
            sc.aabb = sc.aabb[:0]
        for v in args.variants:
            r = run_episode(sc, v, args.cycles, args.task, goal_seed=run)
            r["run"] = run
            rows.append(r)
            print(json.dumps(r), flush=True)
    for v in args.variants:
        rs = [r for r in rows if r["variant"] == v]
        print(json.dumps({"variant": v, "runs": len(rs),
                          "collision_score_mean": float(np.mean([r["collision_score"] for r in rs])),
                          "arm_contact_mean": float(np.mean([r["arm_contact_steps"] for r in rs])),
                          "err_f_mean": float(np.mean([r["err_f"] for r in rs])),
                          "goals_reached_mean": float(np.mean([r["goals_reached"] for r in rs]))}))


if __name__ == "__main__":
    main()

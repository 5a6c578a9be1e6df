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
    getting the next goal of its seeded list; "reaching_central" draws every
    goal position near the centre the arms share (the paper's hard level,
    goals sampled centrally to maximise interaction), uniform in a ball of
    0.2 m radius at 0.4 m height, the orientation kept as the end
    effector's at the time the goal is set; a goal also resets after 1 s.

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


def planar_arm(links, per_link, radius, base_xyz, yaw, K, H):
    """A planar arm (alpha = d = 0: every joint axis vertical) of the given
    link lengths, `per_link` spheres of `radius` evenly spaced on each link
    segment (the frame-(i-1) origin end excluded), base at base_xyz turned by
    yaw about z."""
    dof = len(links)
    dh = np.zeros((dof, 4))
    dh[:, 0] = links
    bodies, xyzr = [], []
    for i, a in enumerate(links):
        for k in range(per_link):
            t = (k + 1) / per_link                 # from the joint to the link's end
            bodies.append(i + 1)
            xyzr.append([-(1.0 - t) * a, 0.0, 0.0, radius])
    return S.Arm(dof=dof, n_spheres=len(bodies), K=K, H=H, dh=dh.astype(np.float32),
                 q_lo=np.full(dof, -2.8, np.float32), q_hi=np.full(dof, 2.8, np.float32),
                 qd_max=np.full(dof, 2.0, np.float32), sphere_body=np.asarray(bodies, np.int32),
                 sphere_xyzr=np.asarray(xyzr, np.float32),
                 base_pose=np.asarray([*base_xyz, *S.yaw_quat(yaw)], np.float32))


_LINKS = (0.35, 0.35, 0.2)


def _reach_to(x_local, links=_LINKS):
    """Joints of a planar 3-link arm whose end effector lies on its base's x
    axis at x_local: shoulder turned so that the elbow, folded, brings the
    straight forearm and hand back onto the axis (wrist at zero)."""
    f = links[1] + links[2]
    c = np.clip((x_local ** 2 - links[0] ** 2 - f ** 2) / (2 * links[0] * f), -1, 1)
    q2 = np.arccos(c)
    q1 = -np.arctan2(f * np.sin(q2), links[0] + f * np.cos(q2))
    return np.array([q1, q2, 0.0], np.float32)


def livelock_scenario(tau, offset=0.05, lead=0.0, K=256, H=30, dt=0.02, **params):
    """The conflict of Sec. IV-B (Fig. 1): two planar 3-link arms on opposite
    sides of a shared workspace, 1.5 m apart and facing each other, each
    reaching for a goal just past the middle (+-offset from it on its own
    side's far edge), so that both end effectors cannot be at their goals at
    once.  Both start stretched out towards the middle, arm 0 `lead` metres
    closer to its goal; no world obstacles.  tau is the priority exponent."""
    links = list(_LINKS)
    arms = [planar_arm(links, 4, 0.04, (-0.75, 0.0, 0.3), 0.0, K, H),
            planar_arm(links, 4, 0.04, (0.75, 0.0, 0.3), np.pi, K, H)]
    p = dict(S.DEFAULT_PARAMS)
    p.update(dt=dt, tau=tau, seed=7)
    p.update(params)
    reach = sum(links)
    # goal joints: the end effector `offset` past the middle; the start:
    # folded back at the elbow, arm 0 `lead` further out than arm 1
    goal_q = [_reach_to(0.75 + offset), _reach_to(0.75 + offset)]
    start_x = 0.75 + offset - 0.35
    q0 = [_reach_to(start_x + lead), _reach_to(start_x)]
    qd0 = [np.zeros(3, np.float32), np.zeros(3, np.float32)]
    assert reach > 0.75 + offset
    return S.Scenario("livelock: two planar arms reaching past the middle", arms, p,
                      np.zeros((0, 4), np.float32), None, np.zeros((0, 6), np.float32),
                      q0, qd0, goal_q, np.zeros((2, 3), np.float32), cycles=300)


def priority_decision(tau, gaps=(0.02, 0.09), w_pose=1000.0, seed=0, cycles=6, K=1024,
                      device="cuda"):
    """The decision of Fig. 1 (C-D): both arms of livelock_scenario stretched
    towards one shared goal point (offset 0), arm 0 gaps[0] and arm 1
    gaps[1] from it, their anticipated plans overlapping.  `cycles` control
    cycles at that fixed state (the board carries each cycle's plans to the
    next); returns, per arm, the distance to the goal now and at the end of
    its last published plan (the plan's end effector).  Without priority
    (tau = 0) the arm nearer its goal does not advance either; with it, the
    nearer arm plans to advance and the other to retreat."""
    sc = livelock_scenario(tau, offset=0.0, lead=0.0, K=K, w_pose=w_pose, seed=seed)
    sc.q0 = [_reach_to(0.75 - gaps[0]), _reach_to(0.75 - gaps[1])]
    ctl = mrs.Controller(sc, device=device)
    ctl.set_world()
    goals = [ctl.goal_pose(a, sc.goal_q[a]) for a in range(2)]
    gp = [g[0] for g in goals]
    gR = [g[1] for g in goals]
    for _ in range(cycles):
        out = ctl.step(sc.q0, sc.qd0, gp, gR)
    now, end = [], []
    for a in range(2):
        pq = ctl.split(out["plan_q"], "hd", a)
        now.append(float(out["dist_to_goal"][a]))
        end.append(float(np.linalg.norm(ctl.fk(a, pq[-1])[0][0, 9:12] - gp[a])))
    ctl.close()
    return now, end


def livelock_episode(sc, cycles=300, device="cuda"):
    """Closed loop of the two-arm conflict on the kinematic plant: the
    distance of each end effector to its goal after every cycle [cycles][2],
    and the cycles with the two arms in contact."""
    ctl = mrs.Controller(sc, device=device)
    ctl.set_world()
    dt = np.float32(sc.params["dt"])
    q = [np.asarray(x, np.float32).copy() for x in sc.q0]
    qd = [np.asarray(x, np.float32).copy() for x in sc.qd0]
    goals = [ctl.goal_pose(a, sc.goal_q[a]) for a in range(2)]
    gp = [g[0] for g in goals]
    gR = [g[1] for g in goals]
    dist = np.zeros((cycles, 2))
    contact = 0
    for t in range(cycles):
        out = ctl.step(q, qd, gp, gR)
        for a in range(2):
            u = ctl.split(out["u_star"], "d", a)
            qd[a] = (qd[a] + u * dt).astype(np.float32)
            q[a] = (q[a] + qd[a] * dt).astype(np.float32)
        sph = []
        for a in range(2):
            e, sp = ctl.fk(a, q[a])
            dist[t, a] = float(np.linalg.norm(e[0, 9:12] - gp[a]))
            sph.append(sp[0].astype(np.float64))
        contact += contacts(sph, np.zeros((0, 4)), np.zeros((0, 6)))[0]
    ctl.close()
    return dist, contact


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
    centre = np.mean(base, axis=0) + np.array([0.0, 0.0, 0.4])

    def central_goal(a):
        v = rng.normal(size=3)
        v *= 0.2 * rng.uniform() ** (1 / 3) / np.linalg.norm(v)
        e, _ = ref.fk(a, q[a])
        return (centre + v).astype(np.float32), e[0, :9].reshape(3, 3).astype(np.float32)
    set_at = [0] * A
    if task == "reaching_central":
        for a in range(A):
            gp[a], gR[a] = central_goal(a)
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
            if task == "reaching_central":
                if dist < reach_tol:
                    goals_reached += 1
                if dist < reach_tol or (t + 1 - set_at[a]) * float(dt) >= 1.0:
                    gp[a], gR[a] = central_goal(a)
                    set_at[a] = t + 1
            elif task == "reaching" and dist < reach_tol:
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
    ap.add_argument("--task", default="following",
                    choices=["following", "reaching", "reaching_central"])
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

"""Seeded synthetic workloads for the multi-arm MPPI control cycle.

This module only draws random inputs: arm geometry (DH parameters, joint
limits, collision spheres in link frames), base placements, world obstacles,
initial joint states, goal joint configurations and goal drift.  It holds
none of the method's arithmetic (no kinematics, no costs, no sampling of
controls); the goal *pose* is obtained by the consumer from a goal joint
configuration with its own forward kinematics.

Every floating-point value is rounded to float32 here, so that the CUDA path
(float32) and the FP64 oracle read bit-identical inputs.

The five workloads mirror the paper's setting (several arms around a shared
workspace, Sec. V-A; drifting targets as in the "Following" task) with seeded
stand-ins for the IsaacSim scenes, which are not available:

  1: one 7-DoF arm, K=64, H=16, dt=0.05, 8 static world spheres.
  2: four 7-DoF arms on a 0.6 m circle, K=512, H=30, dt=0.02, 32 spheres +
     4 boxes, goals drifting at 0.1 m/s, 50 cycles.
  3: workload 2 with the learned self-collision term.
  4: sixteen arms of DoF 6/7/9, K in {256,1024,2048}, H in {20,30,48}, 64
     world spheres.
  5: eight 7-DoF arms, K=4096, H=64, dt=0.01, 256 moving spheres.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32

# Cost and update parameters.  B, w_dyn and tau are the paper's M setting
# (Sec. V-A "Algorithms Tested": w_d=5000, B=0.03, tau=3); the STORM weights,
# lambda and the EMA steps are not printed in the paper and are fixed here.
DEFAULT_PARAMS = dict(
    dt=0.02, lam=10.0, gamma=1.0, alpha_mu=0.9, alpha_sigma=0.5, sigma_init=0.3,
    w_pose=10.0, w_rot=0.5, w_stop=10.0, w_joint=100.0, w_coll=1000.0, w_self=1000.0,
    w_dyn=5000.0, B=0.03, B_world=0.03, B_self=0.03, tau=3.0, q_margin=0.1,
    iterations=1, seed=0, max_plan_age=0, w_manip=0.0, manip_w0=0.02,
)


@dataclass
class Arm:
    dof: int
    n_spheres: int
    K: int
    H: int
    dh: np.ndarray          # [dof][4] a, d, alpha, theta_offset  (float32)
    q_lo: np.ndarray        # [dof]
    q_hi: np.ndarray        # [dof]
    qd_max: np.ndarray      # [dof]
    sphere_body: np.ndarray  # [NS] int32, 1..dof+1 (dof+1 = tool)
    sphere_xyzr: np.ndarray  # [NS][4] centre in body frame + radius (float32)
    base_pose: np.ndarray   # [7] xyz + quaternion (w,x,y,z)  (float32)


@dataclass
class Scenario:
    name: str
    arms: list
    params: dict
    world: np.ndarray        # [n][4]
    world_vel: np.ndarray | None  # [n][3] or None
    aabb: np.ndarray         # [m][6] centre, half extents
    q0: list                 # per arm [dof]
    qd0: list                # per arm [dof]
    goal_q: list             # per arm [dof], goal = FK(goal_q)
    goal_vel: np.ndarray     # [A][3] goal drift velocity (m/s)
    cycles: int
    extra: dict = field(default_factory=dict)

    @property
    def n_arms(self) -> int:
        return len(self.arms)

    def rollout_steps(self) -> int:
        """Sum over arms of K_a * H_a (rollout-steps of one iteration)."""
        return sum(a.K * a.H for a in self.arms)


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(F32)


def random_geometry(rng: np.random.Generator, dof: int, per_link: int, tool_spheres: int):
    """DH parameters and link spheres of one seeded revolute arm.

    a ~ U[0, 0.1] m, d ~ U[0.1, 0.35] m, alpha in {+pi/2, -pi/2}, zero theta
    offsets, joint limits +-2.8 rad, velocity limit 2 rad/s.  Link i carries
    `per_link` spheres evenly spaced on the segment from the frame-i origin
    to the frame-(i-1) origin, which in frame i is t * (-a, -d sin(alpha),
    -d cos(alpha)), t in [0, 1]; radii ~ U[0.04, 0.07] m.  Tool spheres sit on
    the z axis of frame d at 0.02 .. 0.10 m with radii ~ U[0.02, 0.04] m.
    """
    a = rng.uniform(0.0, 0.1, dof)
    d = rng.uniform(0.1, 0.35, dof)
    alpha = np.where(rng.uniform(size=dof) < 0.5, math.pi / 2, -math.pi / 2)
    dh = np.stack([a, d, alpha, np.zeros(dof)], axis=1)
    bodies, xyzr = [], []
    ts = np.linspace(0.0, 1.0, per_link)
    for i in range(dof):
        seg = np.array([-a[i], -d[i] * math.sin(alpha[i]), -d[i] * math.cos(alpha[i])])
        for t in ts:
            bodies.append(i + 1)
            xyzr.append([*(t * seg), rng.uniform(0.04, 0.07)])
    for k in range(tool_spheres):
        bodies.append(dof + 1)
        z = 0.02 + 0.08 * k / max(tool_spheres - 1, 1)
        xyzr.append([0.0, 0.0, z, rng.uniform(0.02, 0.04)])
    return dict(dh=_f32(dh), sphere_body=np.asarray(bodies, np.int32), sphere_xyzr=_f32(xyzr))


def yaw_quat(yaw: float):
    return [math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2)]


def _make_arm(geo, dof, K, H, base_xyz, yaw):
    return Arm(dof=dof, n_spheres=len(geo["sphere_body"]), K=K, H=H, dh=geo["dh"],
               q_lo=_f32(np.full(dof, -2.8)), q_hi=_f32(np.full(dof, 2.8)),
               qd_max=_f32(np.full(dof, 2.0)), sphere_body=geo["sphere_body"],
               sphere_xyzr=geo["sphere_xyzr"], base_pose=_f32([*base_xyz, *yaw_quat(yaw)]))


def _world(rng, n_spheres, n_aabb, bases, lo, hi, speed=None):
    """World spheres (radius U[0.03, 0.08]) and boxes (half extents
    U[0.03, 0.10]) uniform in the box [lo, hi], rejecting any that comes within
    0.15 m of an arm base."""
    bases = np.asarray(bases, np.float64).reshape(-1, 3)

    def clear(c, r):
        return np.all(np.linalg.norm(bases - c, axis=1) - r > 0.15)

    sph = []
    while len(sph) < n_spheres:
        c = rng.uniform(lo, hi)
        r = rng.uniform(0.03, 0.08)
        if clear(c, r):
            sph.append([*c, r])
    boxes = []
    while len(boxes) < n_aabb:
        c = rng.uniform(lo, hi)
        he = rng.uniform(0.03, 0.10, 3)
        if clear(c, float(np.linalg.norm(he))):
            boxes.append([*c, *he])
    vel = None
    if speed is not None:
        v = rng.normal(size=(n_spheres, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        v *= rng.uniform(0.0, speed, (n_spheres, 1))
        vel = _f32(v)
    return (_f32(np.asarray(sph).reshape(-1, 4)), vel,
            _f32(np.asarray(boxes).reshape(-1, 6)))


def _states(rng, arms):
    """Start state and goal joints: every arm starts at rest in its rest pose
    (all joints zero, zero velocity), the pose at which the self-collision
    pair set is taken, so no arm starts in self-contact; the goal joints are
    uniform within the limits."""
    q0 = [_f32(np.zeros(a.dof)) for a in arms]
    qd0 = [_f32(np.zeros(a.dof)) for a in arms]
    goal_q = [_f32(rng.uniform(a.q_lo, a.q_hi)) for a in arms]
    return q0, qd0, goal_q


def _drift(rng, n, speed):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return _f32(v * speed)


def _circle(n, radius):
    out = []
    for a in range(n):
        phi = 2 * math.pi * a / n
        out.append(((radius * math.cos(phi), radius * math.sin(phi), 0.0), phi + math.pi))
    return out


def config(index: int, run: int = 0, **overrides) -> Scenario:
    """Workload `index` (1..5), seeded by index * 1000 + run."""
    seed = index * 1000 + run
    rng = np.random.default_rng(seed)
    params = dict(DEFAULT_PARAMS)
    params["seed"] = seed
    if index == 1:
        geo = random_geometry(rng, 7, per_link=4, tool_spheres=0)
        arms = [_make_arm(geo, 7, 64, 16, (0.0, 0.0, 0.0), 0.0)]
        params["dt"] = 0.05
        world, vel, aabb = _world(rng, 8, 0, [[0, 0, 0]], [-0.6, -0.6, 0.0], [0.6, 0.6, 1.2])
        q0, qd0, gq = _states(rng, arms)
        sc = Scenario("cfg1: 1 arm x 7 DoF, K=64, H=16", arms, params, world, vel, aabb,
                      q0, qd0, gq, _f32(np.zeros((1, 3))), cycles=1)
    elif index in (2, 3):
        geo = random_geometry(rng, 7, per_link=5, tool_spheres=5)
        arms = [_make_arm(geo, 7, 512, 30, xyz, yaw) for xyz, yaw in _circle(4, 0.6)]
        params["dt"] = 0.02
        bases = [a.base_pose[:3] for a in arms]
        world, vel, aabb = _world(rng, 32, 4, bases, [-0.9, -0.9, 0.0], [0.9, 0.9, 1.2])
        q0, qd0, gq = _states(rng, arms)
        sc = Scenario(f"cfg{index}: 4 arms x 7 DoF, K=512, H=30", arms, params, world, vel,
                      aabb, q0, qd0, gq, _drift(rng, 4, 0.1), cycles=50)
        if index == 3:
            sc.extra["mode"] = "learned-self"
    elif index == 4:
        geos = {d: random_geometry(rng, d, per_link=5, tool_spheres=5) for d in (6, 7, 9)}
        arms = []
        for a, (xyz, yaw) in enumerate(_circle(16, 1.0)):
            d = [6, 7, 9][a % 3]
            K = [256, 1024, 2048][(a // 3) % 3]
            H = [20, 30, 48][(a + a // 3) % 3]
            arms.append(_make_arm(geos[d], d, K, H, xyz, yaw))
        params["dt"] = 0.02
        bases = [a.base_pose[:3] for a in arms]
        world, vel, aabb = _world(rng, 64, 0, bases, [-1.3, -1.3, 0.0], [1.3, 1.3, 1.2])
        q0, qd0, gq = _states(rng, arms)
        sc = Scenario("cfg4: 16 arms, DoF 6/7/9, K 256-2048, H 20-48", arms, params, world,
                      vel, aabb, q0, qd0, gq, _drift(rng, 16, 0.1), cycles=50)
    elif index == 5:
        geo = random_geometry(rng, 7, per_link=5, tool_spheres=5)
        arms = [_make_arm(geo, 7, 4096, 64, xyz, yaw) for xyz, yaw in _circle(8, 0.6)]
        params["dt"] = 0.01
        bases = [a.base_pose[:3] for a in arms]
        world, vel, aabb = _world(rng, 256, 0, bases, [-1.0, -1.0, 0.0], [1.0, 1.0, 1.2],
                                  speed=0.5)
        q0, qd0, gq = _states(rng, arms)
        sc = Scenario("cfg5: 8 arms x 7 DoF, K=4096, H=64, 256 moving spheres", arms, params,
                      world, vel, aabb, q0, qd0, gq, _drift(rng, 8, 0.1), cycles=200)
        sc.extra["mode"] = "learned-self+pair"
    else:
        raise ValueError(f"unknown workload {index}")
    for k, v in overrides.items():
        if k in sc.params:
            sc.params[k] = v
        else:
            raise KeyError(k)
    return sc


def shrink(sc: Scenario, K: int | None = None, H: int | None = None, arms: int | None = None,
           n_world: int | None = None, K_div: int | None = None) -> Scenario:
    """A smaller copy of a workload (fewer samples, steps, arms or obstacles)
    for tests that must finish in seconds on the CPU oracle; K_div divides every
    arm's sample count and keeps their ratios."""
    import copy
    s = copy.deepcopy(sc)
    if K_div is not None:
        for a in s.arms:
            a.K = max(1, a.K // K_div)
    if arms is not None:
        s.arms = s.arms[:arms]
        s.q0, s.qd0, s.goal_q = s.q0[:arms], s.qd0[:arms], s.goal_q[:arms]
        s.goal_vel = s.goal_vel[:arms]
    for a in s.arms:
        if K is not None:
            a.K = K
        if H is not None:
            a.H = H
    if n_world is not None:
        s.world = s.world[:n_world]
        if s.world_vel is not None:
            s.world_vel = s.world_vel[:n_world]
    return s

"""Pins of the FP64 oracle against facts that do not come from the oracle:
published known-answer vectors, closed forms, library routines, geometric
invariants and brute force.  Each test names the passage of the paper it
checks (arxiv 2602.10114) or the outside source of its expected values."""
import math
import os

import numpy as np
import pytest
from scipy import special, stats
from scipy.spatial.distance import cdist
from scipy.spatial.transform import Rotation

from paper_2602_10114_gb300 import scenarios as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers

def tiny_scenario(arms, K=None, H=None, world=None, aabb=None, **params):
    p = dict(S.DEFAULT_PARAMS)
    p.update(params)
    A = len(arms)
    for a in arms:
        a.K = a.K if K is None else K
        a.H = a.H if H is None else H
    return S.Scenario(
        "tiny", arms, p,
        np.zeros((0, 4), np.float32) if world is None else np.asarray(world, np.float32),
        None, np.zeros((0, 6), np.float32) if aabb is None else np.asarray(aabb, np.float32),
        [np.zeros(a.dof, np.float32) for a in arms], [np.zeros(a.dof, np.float32) for a in arms],
        [np.zeros(a.dof, np.float32) for a in arms], np.zeros((A, 3), np.float32), cycles=1)


def point_arm(base_xyz, radius, K=8, H=4):
    """One revolute joint with a=d=alpha=0 and a single sphere at the frame-1
    origin, i.e. at the base position whatever q is."""
    return S.Arm(dof=1, n_spheres=1, K=K, H=H, dh=np.zeros((1, 4), np.float32),
                 q_lo=np.full(1, -2.8, np.float32), q_hi=np.full(1, 2.8, np.float32),
                 qd_max=np.full(1, 2.0, np.float32), sphere_body=np.array([1], np.int32),
                 sphere_xyzr=np.array([[0, 0, 0, radius]], np.float32),
                 base_pose=np.array([*base_xyz, 1, 0, 0, 0], np.float32))


def dh_arm(dh, spheres=None, bodies=None, base=(0, 0, 0, 1, 0, 0, 0), K=8, H=4):
    dh = np.asarray(dh, np.float32)
    d = len(dh)
    if spheres is None:
        spheres = np.array([[0, 0, 0, 0.01]], np.float32)
        bodies = np.array([d], np.int32)
    return S.Arm(dof=d, n_spheres=len(spheres), K=K, H=H, dh=dh,
                 q_lo=np.full(d, -2.8, np.float32), q_hi=np.full(d, 2.8, np.float32),
                 qd_max=np.full(d, 2.0, np.float32),
                 sphere_body=np.asarray(bodies, np.int32),
                 sphere_xyzr=np.asarray(spheres, np.float32),
                 base_pose=np.asarray(base, np.float32))


def goals_of(orc, sc):
    gp, gR = zip(*[orc.goal_pose(a, sc.goal_q[a]) for a in range(sc.n_arms)])
    return np.asarray(gp), np.asarray(gR)


# ---------------------------------------------------------------------------
# sampling (Sec. III-A Optimize: eps ~ N(0, Sigma_h))

def test_philox_known_answer_vectors(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle_mod.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform23_is_open_interval_and_float32_exact(oracle_mod):
    rng = np.random.default_rng(0)
    lo, hi = oracle_mod.uniform23(0), oracle_mod.uniform23(0xFFFFFFFF)
    assert lo == 0.5 / 2 ** 23 and hi == 1 - 0.5 / 2 ** 23
    for x in [0x12345678, 0xdeadbeef, 0x80000000, *rng.integers(0, 2**32, 1000)]:
        u = oracle_mod.uniform23(x)
        assert float(np.float32(u)) == u and 0 < u < 1


def test_normals_moments_and_independence(oracle_mod):
    d, N = 8, 125_000
    Z = np.array([oracle_mod.normals(7, 1, 3, 0, n % 5000, n // 5000, d) for n in range(N)])
    z = Z.ravel()
    M = z.size
    assert abs(z.mean()) < 5 / math.sqrt(M)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / M)
    assert abs(stats.skew(z)) < 5 * math.sqrt(6 / M)
    assert abs(stats.kurtosis(z)) < 5 * math.sqrt(24 / M)
    assert stats.kstest(z[:200_000], "norm").pvalue > 1e-4
    corr = np.corrcoef(Z.T)
    off = corr[~np.eye(d, dtype=bool)]
    assert np.abs(off).max() < 5 / math.sqrt(N)


def test_normals_depend_on_every_counter_field(oracle_mod):
    base = oracle_mod.normals(1, 0, 0, 0, 0, 0, 9)
    for args in [(2, 0, 0, 0, 0, 0), (1, 1, 0, 0, 0, 0), (1, 0, 1, 0, 0, 0), (1, 0, 0, 1, 0, 0),
                 (1, 0, 0, 0, 1, 0), (1, 0, 0, 0, 0, 1)]:
        z = oracle_mod.normals(*args, 9)
        assert np.all(z != base)
    # joints 4..7 come from a different Philox block than 0..3
    assert len(set(np.round(base, 12))) == 9


def test_cholesky_matches_library(oracle_mod):
    rng = np.random.default_rng(0)
    for d in (1, 6, 7, 9):
        X = rng.normal(size=(d, d))
        Sg = X @ X.T + 0.1 * np.eye(d)
        L = oracle_mod.cholesky(Sg, jitter=1e-8)
        assert np.allclose(np.triu(L, 1), 0)
        ref = np.linalg.cholesky(Sg + 1e-8 * np.eye(d))
        assert np.allclose(L, ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# kinematics (Sec. IV-A: link frames by forward kinematics, spheres at
# constant transforms from the links)

def test_fk_planar_two_link_closed_form(oracle_mod):
    from oracle.oracle import Oracle
    a1, a2 = 0.4, 0.3
    arm = dh_arm([[a1, 0, 0, 0], [a2, 0, 0, 0]])
    orc = Oracle(tiny_scenario([arm]))
    rng = np.random.default_rng(1)
    for _ in range(20):
        q = rng.uniform(-2.8, 2.8, 2)
        F, _ = orc.fk(0, q)
        ee = F[-1][:3, 3]
        exp = [a1 * math.cos(q[0]) + a2 * math.cos(q[0] + q[1]),
               a1 * math.sin(q[0]) + a2 * math.sin(q[0] + q[1]), 0.0]
        assert np.allclose(ee, exp, atol=1e-14)
        # planar: the end-effector heading is q1 + q2 about z
        R = F[-1][:3, :3]
        assert np.allclose(R, Rotation.from_euler("z", q[0] + q[1]).as_matrix(), atol=1e-14)


def _random_arm(seed, dof=7):
    rng = np.random.default_rng(seed)
    geo = S.random_geometry(rng, dof, per_link=5, tool_spheres=5)
    base = np.array([0.3, -0.2, 0.1, *Rotation.from_euler("zyx", [0.4, 0.2, -0.3]).as_quat(
        scalar_first=True)], np.float32)
    return S.Arm(dof=dof, n_spheres=len(geo["sphere_body"]), K=8, H=4, dh=geo["dh"],
                 q_lo=np.full(dof, -2.8, np.float32), q_hi=np.full(dof, 2.8, np.float32),
                 qd_max=np.full(dof, 2.0, np.float32), sphere_body=geo["sphere_body"],
                 sphere_xyzr=geo["sphere_xyzr"], base_pose=base)


def test_fk_frames_rigid_and_link_lengths(oracle_mod):
    from oracle.oracle import Oracle
    arm = _random_arm(3)
    orc = Oracle(tiny_scenario([arm]))
    dh = arm.dh.astype(np.float64)
    rng = np.random.default_rng(2)
    for _ in range(10):
        F, _ = orc.fk(0, rng.uniform(-2.8, 2.8, 7))
        for i in range(8):
            R = F[i][:3, :3]
            assert np.allclose(R @ R.T, np.eye(3), atol=1e-13)
            assert abs(np.linalg.det(R) - 1) < 1e-13
            assert np.allclose(F[i][3], [0, 0, 0, 1])
        for i in range(1, 8):
            step = np.linalg.norm(F[i][:3, 3] - F[i - 1][:3, 3])
            assert abs(step - math.hypot(dh[i - 1, 0], dh[i - 1, 1])) < 1e-13


def test_fk_joint_i_rotates_downstream_about_axis_z_im1(oracle_mod):
    """Joint i turns everything after it about the z axis of frame i-1 through
    the frame-(i-1) origin, by exactly the change of q_i (right-hand rule)."""
    from oracle.oracle import Oracle
    arm = _random_arm(4)
    orc = Oracle(tiny_scenario([arm]))
    rng = np.random.default_rng(5)
    for _ in range(10):
        q = rng.uniform(-2, 2, 7)
        F0, S0 = orc.fk(0, q)
        i = int(rng.integers(1, 8))
        dq = float(rng.uniform(-0.7, 0.7))
        q1 = q.copy()
        q1[i - 1] += dq
        F1, S1 = orc.fk(0, q1)
        axis = F0[i - 1][:3, 2]
        o = F0[i - 1][:3, 3]
        rot = Rotation.from_rotvec(axis * dq).as_matrix()
        down = arm.sphere_body >= i
        moved = (S0[down, :3] - o) @ rot.T + o
        assert np.allclose(S1[down, :3], moved, atol=1e-13)
        assert np.allclose(S1[~down, :3], S0[~down, :3], atol=0)
        assert np.allclose(F1[-1][:3, :3], rot @ F0[-1][:3, :3], atol=1e-13)


def test_link_sphere_end_points_sit_on_frame_origins(oracle_mod):
    """The generator puts t=0 of link i at the frame-i origin and t=1 at the
    frame-(i-1) origin; FK must place them there."""
    from oracle.oracle import Oracle
    arm = _random_arm(6)
    orc = Oracle(tiny_scenario([arm]))
    F, Sph = orc.fk(0, np.linspace(-1, 1, 7))
    for i in range(1, 8):
        idx = np.where(arm.sphere_body == i)[0]
        assert np.allclose(Sph[idx[0], :3], F[i][:3, 3], atol=1e-6)
        assert np.allclose(Sph[idx[-1], :3], F[i - 1][:3, 3], atol=1e-6)


def test_fk_base_pose_is_a_rigid_motion(oracle_mod):
    from oracle.oracle import Oracle
    arm = _random_arm(7)
    arm0 = _random_arm(7)
    arm0.base_pose = np.array([0, 0, 0, 1, 0, 0, 0], np.float32)
    o1 = Oracle(tiny_scenario([arm]))
    o0 = Oracle(tiny_scenario([arm0]))
    q = np.linspace(-1.3, 0.9, 7)
    _, s1 = o1.fk(0, q)
    _, s0 = o0.fk(0, q)
    bp = arm.base_pose.astype(np.float64)
    R = Rotation.from_quat(bp[3:], scalar_first=True).as_matrix()
    assert np.allclose(s1[:, :3], s0[:, :3] @ R.T + bp[:3], atol=1e-12)


# ---------------------------------------------------------------------------
# distances (Sec. IV-A rho_b)

def test_sphere_distances_brute_force(oracle_mod):
    rng = np.random.default_rng(8)
    A = rng.uniform(-1, 1, (20, 4))
    B = rng.uniform(-1, 1, (30, 4))
    A[:, 3] = np.abs(A[:, 3]) * 0.1
    B[:, 3] = np.abs(B[:, 3]) * 0.1
    ref = cdist(A[:, :3], B[:, :3]) - A[:, 3:4] - B[:, 3][None, :]
    got = np.array([[oracle_mod.sphere_sphere(a, b) for b in B] for a in A])
    assert np.allclose(got, ref, atol=1e-14)


def test_sphere_aabb_analytic_points(oracle_mod):
    box = [0.1, 0.2, 0.3, 0.2, 0.1, 0.05]
    c, h = np.array(box[:3]), np.array(box[3:])
    r = 0.02
    # centre inside: nearest face is the z face at 0.05
    assert math.isclose(oracle_mod.sphere_aabb([*c, r], box), -0.05 - r, abs_tol=1e-15)
    dlt = 0.07
    face = c + np.array([h[0] + dlt, 0, 0])
    assert math.isclose(oracle_mod.sphere_aabb([*face, r], box), dlt - r, abs_tol=1e-14)
    edge = c + np.array([h[0] + dlt, h[1] + dlt, 0])
    assert math.isclose(oracle_mod.sphere_aabb([*edge, r], box), dlt * math.sqrt(2) - r,
                        abs_tol=1e-14)
    corner = c - h - dlt
    assert math.isclose(oracle_mod.sphere_aabb([*corner, r], box), dlt * math.sqrt(3) - r,
                        abs_tol=1e-14)
    # random outside points: distance to the nearest point of the box
    rng = np.random.default_rng(9)
    for _ in range(200):
        p = rng.uniform(-1, 1, 3)
        near = np.clip(p, c - h, c + h)
        if np.all(near == p):
            continue
        assert math.isclose(oracle_mod.sphere_aabb([*p, r], box), np.linalg.norm(p - near) - r,
                            abs_tol=1e-14)


# ---------------------------------------------------------------------------
# stage-cost terms (Eq. 5) and the coordination ramp (Sec. IV-A)

def test_pose_cost_closed_forms(oracle_mod):
    rng = np.random.default_rng(10)
    R = Rotation.random(random_state=3).as_matrix()
    p = np.array([0.3, -0.1, 0.5])
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, p
    assert abs(oracle_mod.pose_cost(T, p, R, 0.5)) < 1e-15
    v = rng.normal(size=3) * 0.2
    assert math.isclose(oracle_mod.pose_cost(T, p + v, R, 0.5), np.linalg.norm(v), rel_tol=1e-14)
    for th in (0.1, 1.0, math.pi):
        Rg = Rotation.from_rotvec(th * np.array([0.6, 0.0, 0.8])).as_matrix() @ R
        assert math.isclose(oracle_mod.pose_cost(T, p, Rg, 0.5), 0.5 * (1 - math.cos(th)),
                            abs_tol=1e-14)


def test_stop_and_joint_cost_closed_forms(oracle_mod):
    qmax = np.array([2.0, 2.0, 2.0])
    assert oracle_mod.stop_cost([1.9, -2.0, 0.0], qmax) == 0.0
    assert math.isclose(oracle_mod.stop_cost([2.5, -3.0, 0.0], qmax), 0.25 + 1.0)
    lo, hi = np.full(2, -2.8), np.full(2, 2.8)
    assert oracle_mod.joint_cost([2.65, -2.65], lo, hi, 0.1) == 0.0
    assert math.isclose(oracle_mod.joint_cost([2.9, -3.0], lo, hi, 0.1), 0.2 ** 2 + 0.3 ** 2)


def test_ramp_closed_forms(oracle_mod):
    B = 0.03
    assert oracle_mod.ramp(B, B) == 0.0
    assert oracle_mod.ramp(0.5, B) == 0.0
    assert math.isclose(oracle_mod.ramp(B / 2, B), 0.5)
    assert oracle_mod.ramp(0.0, B) == 1.0
    assert oracle_mod.ramp(-0.01, B) > 1.0


def test_priority_rule(oracle_mod):
    """Sec. IV-B: tau = 0 disables priority; alpha^(j,i) alpha^(i,j) = 1;
    the arm closer to its goal gets the smaller weight."""
    for e1, e2 in [(0.2, 0.5), (0.01, 1.0), (0.3, 0.3)]:
        assert oracle_mod.priority(e1, e2, 0.0) == 1.0
        assert math.isclose(oracle_mod.priority(e1, e2, 3.0) * oracle_mod.priority(e2, e1, 3.0),
                            1.0, rel_tol=1e-14)
    assert oracle_mod.priority(0.1, 0.5, 3.0) < 1.0 < oracle_mod.priority(0.5, 0.1, 3.0)
    assert math.isclose(oracle_mod.priority(2 - 1e-4, 1 - 1e-4, 3.0), 8.0, rel_tol=1e-14)


def test_weights_softmax(oracle_mod):
    """Eq. 2: positive, sum to one, invariant to a common shift, equal to the
    library softmax of -C/lambda."""
    rng = np.random.default_rng(11)
    Cn = rng.uniform(0, 200, 257)
    w = oracle_mod.weights(Cn, 10.0)
    assert np.all(w > 0) and abs(w.sum() - 1) < 1e-12
    assert np.allclose(w, special.softmax(-Cn / 10.0), rtol=1e-12, atol=1e-300)
    assert np.allclose(oracle_mod.weights(Cn + 1e4, 10.0), w, rtol=1e-10)


# ---------------------------------------------------------------------------
# rollout (Sec. III-A f, Eq. 1)

def _single(world=None, **params):
    from oracle.oracle import Oracle
    arm = _random_arm(12)
    sc = tiny_scenario([arm], K=16, H=8, world=world, **params)
    return sc, Oracle(sc)


def test_integration_closed_form_constant_acceleration(oracle_mod):
    sc, orc = _single(dt=0.02)
    a = np.linspace(-0.5, 0.7, 7)
    q0 = np.linspace(-1, 1, 7)
    qd0 = np.linspace(0.2, -0.3, 7)
    gp, gR = goals_of(orc, sc)
    H, dt = 8, 0.02
    _, _, _, qtraj = orc.rollout(0, [q0], [qd0], gp, gR, np.tile(a, (H, 1)))
    for h in range(1, H + 1):
        exp = q0 + h * dt * qd0 + a * dt * dt * h * (h + 1) / 2
        assert np.allclose(qtraj[h - 1], exp, atol=1e-14)


def test_discounted_sum_of_constant_stage_cost(oracle_mod):
    """Eq. 1 with gamma < 1: a rollout standing still scores the same stage cost
    c at every step, so C = c (1 - gamma^H) / (1 - gamma)."""
    sc, orc = _single(gamma=0.9)
    gp, gR = goals_of(orc, sc)
    gp = gp + 0.1
    q0, qd0 = np.linspace(-1, 1, 7), np.zeros(7)
    tot, stage, _, _ = orc.rollout(0, [q0], [qd0], gp, gR, np.zeros((8, 7)))
    c = stage[0]
    assert c > 0 and np.allclose(stage, c, rtol=1e-14)
    g = float(np.float32(0.9))          # parameters are read as float32 values
    assert math.isclose(tot, c * (1 - g ** 8) / (1 - g), rel_tol=1e-13)


def test_colliding_pose_exceeds_threshold(oracle_mod):
    """A world sphere placed on a link sphere: the world term is above its
    unweighted threshold 1, i.e. the stage cost exceeds w_c."""
    from oracle.oracle import Oracle
    arm = _random_arm(13)
    q0 = np.linspace(-0.5, 0.5, 7)
    probe = Oracle(tiny_scenario([arm]))
    _, sph = probe.fk(0, q0)
    world = [[*sph[20, :3], 0.05]]
    sc = tiny_scenario([arm], H=3, world=world, w_pose=0, w_stop=0, w_joint=0, w_self=0)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    _, stage, _, _ = orc.rollout(0, [q0], [np.zeros(7)], gp, gR, np.zeros((3, 7)))
    o = sc.world[0].astype(np.float64)
    dmin = (cdist(sph[:, :3], o[None, :3])[:, 0] - sph[:, 3] - o[3]).min()
    assert dmin <= -(sph[20, 3] + 0.05) + 1e-6
    exp = 1 - dmin / float(np.float32(0.03))   # B_world as the float32 parameter
    assert stage[0] > sc.params["w_coll"]
    assert math.isclose(stage[0], sc.params["w_coll"] * exp, rel_tol=1e-12)


def _two_points(gap, tau=0.0, H_other=4):
    """Arm 0 and arm 1 are single spheres of radius 1/16 whose surfaces are
    `gap` apart (up to float32 rounding of the input position); arm 1's plan is published; only the coordination term is on."""
    from oracle.oracle import Oracle
    r = 0.0625
    a0 = point_arm((0, 0, 0), r, H=4)
    a1 = point_arm((2 * r + gap, 0, 0), r, H=H_other)
    sc = tiny_scenario([a0, a1], w_pose=0, w_stop=0, w_joint=0, w_coll=0, w_self=0,
                       w_dyn=1.0, tau=tau)
    orc = Oracle(sc)
    # publish both plans: run one cycle (plans = the spheres, which never move)
    gp = np.zeros((2, 3))
    gR = np.tile(np.eye(3).ravel(), (2, 1))
    orc.cycle([np.zeros(1)] * 2, [np.zeros(1)] * 2, gp, gR)
    return sc, orc, gp, gR


@pytest.mark.parametrize("gap,expected", [(0.0301, 0.0), (0.2, 0.0), (0.015, 0.5), (0.0, 1.0),
                                          (-0.02, 1.0)])
def test_coordination_cost_closed_forms(oracle_mod, gap, expected):
    """Sec. IV-A: C_dyn = max(0, 1 - rho_b / B): zero at rho_b >= B, one half at
    B/2, one at contact and under overlap (rho_b is a distance, >= 0)."""
    sc, orc, gp, gR = _two_points(gap)
    _, stage, _, _ = orc.rollout(0, [np.zeros(1)] * 2, [np.zeros(1)] * 2, gp, gR,
                                 np.zeros((4, 1)), alpha_row=np.array([0.0, 1.0]))
    # float32 rounding of the input position moves the gap by < 1e-8 m
    assert np.allclose(stage, expected, atol=1e-6)
    if expected in (0.0, 1.0):
        assert np.all(stage == expected)


def test_min_horizon_rule(oracle_mod):
    """Sec. IV-C: an arm uses min(H_j, H_i) steps of a received plan."""
    sc, orc, gp, gR = _two_points(0.0, H_other=2)
    _, stage, _, _ = orc.rollout(0, [np.zeros(1)] * 2, [np.zeros(1)] * 2, gp, gR,
                                 np.zeros((4, 1)), alpha_row=np.array([0.0, 1.0]))
    assert np.allclose(stage, [1, 1, 0, 0], atol=1e-12)


def test_missing_plans_are_ignored_and_query_count(oracle_mod):
    """Sec. IV-C: neighbours without a published plan are ignored (first
    cycle); afterwards every rollout step queries N_S^(j) * sum_i N_S^(i)
    sphere pairs (Sec. IV-A complexity)."""
    from oracle.oracle import Oracle
    sc = S.shrink(S.config(2), K=16, H=6)
    orc = Oracle(sc, threads=4)
    gp, gR = goals_of(orc, sc)
    o1 = orc.cycle(sc.q0, sc.qd0, gp, gR)
    assert np.all(o1["n_queries"] == 0) and np.all(o1["alpha"] == 0)
    o2 = orc.cycle(sc.q0, sc.qd0, gp, gR)
    for a in range(sc.n_arms):
        assert o2["n_queries"][a] == orc.query_count(a) == 6 * 16 * 40 * 120


def test_zero_noise_rollout_reproduces_the_plan(oracle_mod):
    """Sec. IV-A: ToPlan applies f to the means; a rollout of U = mu gives the
    published sphere trajectory and joint plan."""
    from oracle.oracle import Oracle
    sc = S.shrink(S.config(2), K=16, H=6)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    out = orc.cycle(sc.q0, sc.qd0, gp, gR)
    for a in range(sc.n_arms):
        mu = orc.split(out["mean_plan"], "hd", a)
        q = [sc.q0[i] for i in range(sc.n_arms)]
        _, _, sph, qt = orc.rollout(a, q, sc.qd0, gp, gR, mu)
        assert np.array_equal(sph, orc.split(out["plan_spheres"], "hs", a))
        assert np.array_equal(qt, orc.split(out["plan_q"], "hd", a))


def test_update_one_hot_weights_recover_best_sample(oracle_mod):
    """Eqs. 2-4 with lambda -> 0 and alpha_mu = alpha_Sigma = 1: the weights are
    one-hot on n*, so mu_1 = U_{n*,1} (= the executed U_*) and Sigma_1 = 0."""
    from oracle.oracle import Oracle
    sc = S.shrink(S.config(1), K=32, H=5)
    sc.params.update(lam=1e-9, alpha_mu=1.0, alpha_sigma=1.0)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    out = orc.cycle(sc.q0, sc.qd0, gp, gR)
    mu = orc.split(out["mean_plan"], "hd", 0)
    assert np.allclose(mu[0], out["u_star"], atol=1e-15)
    assert np.abs(orc.split(out["Sigma"], "hdd", 0)[0]).max() < 1e-20
    costs = out["costs"]
    assert out["n_star"][0] == int(np.argmin(costs))


def test_update_uniform_weights_give_sample_moments(oracle_mod):
    """Eqs. 3-4 with lambda -> infinity: uniform weights, so mu~ and Sigma~ are
    the sample mean and the (biased) sample covariance of the drawn U."""
    from oracle.oracle import Oracle
    sc = S.shrink(S.config(1), K=64, H=3)
    sc.params.update(lam=1e30, alpha_mu=1.0, alpha_sigma=1.0)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    out = orc.cycle(sc.q0, sc.qd0, gp, gR)
    d, K, s2 = 7, 64, float(np.float32(0.3)) ** 2
    L = oracle_mod.cholesky(s2 * np.eye(d), 1e-8)
    for h in range(3):
        U = np.array([L @ oracle_mod.normals(sc.params["seed"], 0, 0, 0, n, h, d)
                      for n in range(K)])
        assert np.allclose(orc.split(out["mean_plan"], "hd", 0)[h], U.mean(0), atol=1e-14)
        assert np.allclose(orc.split(out["Sigma"], "hdd", 0)[h], np.cov(U.T, bias=True),
                           atol=1e-14)


def test_shift_moves_phi_one_step(oracle_mod):
    """Sec. III-A left-shifting at the start of each cycle: phi_h <- phi_{h+1};
    with alpha_mu = alpha_Sigma = 0 the update keeps the shifted values."""
    from oracle.oracle import Oracle
    sc = S.shrink(S.config(1), K=16, H=5)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    o1 = orc.cycle(sc.q0, sc.qd0, gp, gR)
    orc.sc.params.update(alpha_mu=0.0, alpha_sigma=0.0)
    orc.cfg.alpha_mu = 0.0
    orc.cfg.alpha_sigma = 0.0
    o2 = orc.cycle(sc.q0, sc.qd0, gp, gR)
    mu1, mu2 = orc.split(o1["mean_plan"], "hd", 0), orc.split(o2["mean_plan"], "hd", 0)
    S1, S2 = orc.split(o1["Sigma"], "hdd", 0), orc.split(o2["Sigma"], "hdd", 0)
    assert np.array_equal(mu2[:-1], mu1[1:]) and np.array_equal(mu2[-1], mu1[-1])
    s2 = float(np.float32(0.3)) ** 2       # sigma_init as the float32 parameter
    assert np.array_equal(S2[:-1], S1[1:]) and np.array_equal(S2[-1], s2 * np.eye(7))


def test_priority_uses_own_sensed_and_neighbours_published_distance(oracle_mod):
    from oracle.oracle import Oracle
    sc = S.shrink(S.config(2), K=8, H=4)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    o1 = orc.cycle(sc.q0, sc.qd0, gp, gR)
    e_pub = o1["dist_to_goal"].copy()
    q2 = [q + 0.1 for q in sc.q0]
    o2 = orc.cycle(q2, sc.qd0, gp, gR)
    A = sc.n_arms
    al = o2["alpha"].reshape(A, A)
    for j in range(A):
        for i in range(A):
            exp = 0.0 if i == j else oracle_mod.priority(o2["dist_to_goal"][j], e_pub[i], 3.0)
            assert al[j, i] == exp


def test_sample_costs_agree_with_the_cycle(oracle_mod):
    """The one-by-one sample scorer reproduces the cycle's own costs of
    those samples (both follow Sense, Shift, SampleControls, Rollout)."""
    from oracle.oracle import Oracle
    sc = S.shrink(S.config(2), K=24, H=6)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    orc.cycle(sc.q0, sc.qd0, gp, gR)
    ns = [0, 5, 23]
    before = {a: orc.sample_costs(a, sc.q0, sc.qd0, gp, gR, ns) for a in range(sc.n_arms)}
    out = orc.cycle(sc.q0, sc.qd0, gp, gR)
    for a in range(sc.n_arms):
        assert np.array_equal(before[a], orc.split(out["costs"], "k", a)[ns])


# ---------------------------------------------------------------------------
# learned surrogate (not in the paper): FP64 MLP gradient

@pytest.mark.parametrize("over_weight", [1.0, 6.0])
def test_mlp_gradient_matches_central_differences(oracle_mod, over_weight):
    rng = np.random.default_rng(21)
    in_dim, width, layers = 14, 16, 3
    in_pad = 16
    n_par = width * in_pad + width + 2 * (width * width + width) + width + 1
    p = rng.normal(scale=0.4, size=n_par)
    x = rng.normal(size=(9, in_dim))
    t = rng.uniform(-0.2, 0.4, 9)          # some targets beyond the clip range
    loss, g, _ = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, t, over_weight=over_weight)
    idx = rng.choice(n_par, 60, replace=False)
    h = 1e-6
    for i in idx:
        if (i % (width * in_pad + width)) < width * in_pad and i < width * in_pad + width \
                and (i % in_pad) >= in_dim:
            continue          # weights on padding inputs: zero gradient
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle_mod.mlp_loss_grad(in_dim, width, layers, pp, x, t, False, over_weight)[0]
              - oracle_mod.mlp_loss_grad(in_dim, width, layers, pm, x, t, False, over_weight)[0]
              ) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mlp_asymmetric_loss_weights_over_predictions(oracle_mod):
    """With every output above its (clipped) target the weighted loss is
    over_weight times the plain one; with every output below, the same."""
    rng = np.random.default_rng(22)
    in_dim, width, layers = 3, 16, 1
    p = rng.normal(scale=0.05, size=16 * 16 + 16 + 16 + 1)
    x = rng.normal(size=(12, in_dim))
    _, _, y = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, np.zeros(12), False)
    p[-1] += 0.1 - y.mean()                    # outputs near 0.1
    _, _, y = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, np.zeros(12), False)
    below, above = y - 0.05, y + 0.05          # targets inside the clip range
    assert np.all(below > -0.1) and np.all(above < 0.3)
    plain_b = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, below, False)[0]
    plain_a = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, above, False)[0]
    assert math.isclose(plain_b, 0.05 ** 2, rel_tol=1e-12)
    w_b = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, below, False, 7.0)[0]
    w_a = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, above, False, 7.0)[0]
    assert math.isclose(w_b, 7.0 * plain_b, rel_tol=1e-12)
    assert math.isclose(w_a, plain_a, rel_tol=1e-12)


def test_mlp_forward_closed_form(oracle_mod):
    """One hidden unit layer per layer with known weights: y = w_out silu(...)."""
    in_dim, width, layers = 1, 16, 1
    p = np.zeros(16 * 16 + 16 + 16 + 1)
    p[0] = 2.0                              # W[0][0]
    p[256 + 0] = 0.5                        # b[0]
    p[256 + 16 + 0] = 3.0                   # w_out[0]
    p[-1] = -0.25                           # b_out
    x = np.array([[0.7]])
    _, _, y = oracle_mod.mlp_loss_grad(in_dim, width, layers, p, x, np.zeros(1), False)
    z = 2.0 * 0.7 + 0.5
    assert math.isclose(y[0], 3.0 * z / (1 + math.exp(-z)) - 0.25, rel_tol=1e-14)


def test_self_distance_is_the_self_term_of_the_rollout(oracle_mod):
    """The surrogate's label equals the clearance the rollout ramps: with only
    the self term weighted, a standing rollout's stage cost is w_self * ramp."""
    from oracle.oracle import Oracle
    arm = _random_arm(31)
    sc = tiny_scenario([arm], H=2, w_pose=0, w_stop=0, w_joint=0, w_coll=0, w_self=1.0)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    B = float(np.float32(0.03))
    rng = np.random.default_rng(2)
    for _ in range(20):
        q = rng.uniform(-2.8, 2.8, 7)
        d = orc.self_distance(0, q)[0]
        _, sph = orc.fk(0, q)
        _, rest = orc.fk(0, np.zeros(7))
        body = arm.sphere_body

        def clear(S, i, j):
            return np.linalg.norm(S[i, :3] - S[j, :3]) - S[i, 3] - S[j, 3]
        brute = min(clear(sph, i, j)
                    for i in range(len(sph)) for j in range(i + 1, len(sph))
                    if abs(int(body[i]) - int(body[j])) >= 3 and clear(rest, i, j) >= B)
        assert math.isclose(d, brute, rel_tol=1e-12, abs_tol=1e-15)
        _, stage, _, _ = orc.rollout(0, [q], [np.zeros(7)], gp, gR, np.zeros((2, 7)))
        assert math.isclose(stage[0], max(0.0, 1 - d / B), rel_tol=1e-12, abs_tol=1e-15)


def test_self_pair_set_ignores_pairs_touching_at_rest(oracle_mod):
    """The self-collision pair set (reading of C_self in Eq. 5): pairs on
    bodies at least three apart, minus those inside the B_self band at the
    rest pose.  A planar four-link arm (alpha = d = 0, a = 0.25 m) lies
    straight along x at rest, so frame i sits at x = 0.25 i; every sphere has
    r = 0.0625 m (all values exact in binary32).  Sphere 0 (body 1, frame-1
    origin) and sphere 1 (body 4, frame-4 origin) are 0.625 m clear at rest:
    kept.  Sphere 2 (body 4, 0.6875 m back along the link: x = 0.3125 at
    rest) overlaps sphere 0 at rest; sphere 3 (x = 0.390625) is 1/64 m clear
    of it, inside the 3 cm band: both dropped.  Sphere 4 (body 2) is only two
    bodies from sphere 1: dropped by the chain rule.  The clearance at any
    pose is then the planar closed form of the one kept pair."""
    from oracle.oracle import Oracle
    a, r = 0.25, 0.0625
    spheres = [[0, 0, 0, r], [0, 0, 0, r], [-0.6875, 0, 0, r], [-0.609375, 0, 0, r],
               [0, 0, 0, r]]
    bodies = [1, 4, 4, 4, 2]
    order = np.argsort(bodies, kind="stable")     # bodies must be non-decreasing
    arm = dh_arm([[a, 0, 0, 0]] * 4, np.asarray(spheres)[order], np.asarray(bodies)[order])
    orc = Oracle(tiny_scenario([arm]))
    kept = {(int(order[i]), int(order[j])) for i, j in orc.self_pairs(0)}
    kept = {tuple(sorted(p)) for p in kept}
    assert kept == {(0, 1)}
    rng = np.random.default_rng(4)
    for _ in range(20):
        q = rng.uniform(-2.8, 2.8, 4)
        th = np.cumsum(q)
        p1 = a * np.array([math.cos(th[0]), math.sin(th[0])])
        p4 = a * np.array([np.sum(np.cos(th)), np.sum(np.sin(th))])
        assert math.isclose(orc.self_distance(0, q)[0], np.linalg.norm(p4 - p1) - 2 * r,
                            rel_tol=1e-12, abs_tol=1e-14)


# ---------------------------------------------------------------------------
# arm-to-arm clearance (the label of the learned arm-pair surrogate)

def _planar_tip_arm(a1, a2, r, base_xyz, yaw):
    """Planar two-link arm (alpha = d = 0) with one sphere of radius r at the
    frame-2 origin (the tip), base rotated by yaw about z."""
    return S.Arm(dof=2, n_spheres=1, K=8, H=4,
                 dh=np.array([[a1, 0, 0, 0], [a2, 0, 0, 0]], np.float32),
                 q_lo=np.full(2, -2.8, np.float32), q_hi=np.full(2, 2.8, np.float32),
                 qd_max=np.full(2, 2.0, np.float32), sphere_body=np.array([2], np.int32),
                 sphere_xyzr=np.array([[0, 0, 0, r]], np.float32),
                 base_pose=np.array([*base_xyz, math.cos(yaw / 2), 0, 0, math.sin(yaw / 2)],
                                    np.float32))


def test_pair_distance_with_per_row_poses_equals_the_fixed_pose_form(oracle_mod):
    """The per-row-pose clearance (arm a at the identity, arm b at a pose per
    row) equals the fixed-pose clearance of the planar closed-form pin when
    every row carries b's pose in a's frame, and a rigid motion applied to
    both arms (here: a at a yawed, shifted base) leaves it unchanged."""
    from oracle.oracle import Oracle
    A = _planar_tip_arm(0.5, 0.25, 0.05, (0.0, 0.0, 0.0), 0.0)
    Bm = _planar_tip_arm(0.375, 0.5, 0.0625, (1.5, 0.25, 0.125), math.pi)
    orc = Oracle(tiny_scenario([A, Bm]))
    rng = np.random.default_rng(3)
    qa, qb = rng.uniform(-2.8, 2.8, (40, 2)), rng.uniform(-2.8, 2.8, (40, 2))
    ref = orc.pair_distance(0, 1, qa, qb)
    pose = np.tile(Bm.base_pose.astype(np.float64), (40, 1))
    got = orc.pair_distance_posed(0, 1, qa, qb, pose)
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
    # the same relative placement with a moved: yaw 0.7 about z, shifted
    yaw, t = 0.7, np.array([0.3, -0.2, 0.05])
    Rz = Rotation.from_euler("z", yaw)
    qa_w = Rotation.from_quat([0, 0, math.sin(yaw / 2), math.cos(yaw / 2)])
    pb = Bm.base_pose.astype(np.float64)
    rb = Rotation.from_quat([pb[4], pb[5], pb[6], pb[3]])
    base_b = np.concatenate([Rz.apply(pb[:3]) + t, np.roll((qa_w * rb).as_quat(), 1)])
    moved = orc.pair_distance(0, 1, qa, qb, base_b=base_b,
                              base_a=[*t, math.cos(yaw / 2), 0, 0, math.sin(yaw / 2)])
    assert np.allclose(moved, ref, rtol=0, atol=1e-12)


def test_pair_distance_planar_closed_form(oracle_mod):
    """Two planar two-link arms facing each other: the clearance of their tip
    spheres is |tip_a - tip_b| - r_a - r_b with tip = base + R_yaw (a1 c1 +
    a2 c12, a1 s1 + a2 s12, 0)."""
    from oracle.oracle import Oracle
    A = _planar_tip_arm(0.5, 0.25, 0.05, (0.0, 0.0, 0.0), 0.0)
    Bm = _planar_tip_arm(0.375, 0.5, 0.0625, (1.5, 0.25, 0.125), math.pi)
    orc = Oracle(tiny_scenario([A, Bm]))
    rng = np.random.default_rng(9)
    qa, qb = rng.uniform(-2.8, 2.8, (50, 2)), rng.uniform(-2.8, 2.8, (50, 2))
    got = orc.pair_distance(0, 1, qa, qb)

    def tip(arm, q):
        a1, a2 = float(arm.dh[0, 0]), float(arm.dh[1, 0])
        w, z = float(arm.base_pose[3]), float(arm.base_pose[6])
        yaw = 2 * math.atan2(z, w)
        x = a1 * math.cos(q[0]) + a2 * math.cos(q[0] + q[1])
        y = a1 * math.sin(q[0]) + a2 * math.sin(q[0] + q[1])
        c, s = math.cos(yaw), math.sin(yaw)
        b = arm.base_pose.astype(np.float64)
        return np.array([b[0] + c * x - s * y, b[1] + s * x + c * y, b[2]])
    for k in range(50):
        ref = (np.linalg.norm(tip(A, qa[k]) - tip(Bm, qb[k])) - float(np.float32(0.05)) - 0.0625)
        assert math.isclose(got[k], ref, rel_tol=1e-12, abs_tol=1e-13)


def test_pair_distance_symmetry_and_base_override(oracle_mod):
    """Swapping the two arms leaves the clearance unchanged; moving arm b's
    base far away along x raises it by the distance moved once the arms
    cannot reach each other; overriding b's base with its own pose is a
    no-op."""
    from oracle.oracle import Oracle
    a, b = _random_arm(41), _random_arm(42)
    b.base_pose = np.array([1.0, 0.2, 0.0, 0, 0, 0, 1], np.float32)
    orc = Oracle(tiny_scenario([a, b]))
    rng = np.random.default_rng(4)
    qa, qb = rng.uniform(-2.8, 2.8, (20, 7)), rng.uniform(-2.8, 2.8, (20, 7))
    d_ab = orc.pair_distance(0, 1, qa, qb)
    d_ba = orc.pair_distance(1, 0, qb, qa)
    assert np.allclose(d_ab, d_ba, rtol=0, atol=1e-13)
    assert np.array_equal(orc.pair_distance(0, 1, qa, qb, base_b=b.base_pose), d_ab)
    far1 = orc.pair_distance(0, 1, qa, qb, base_b=[20.0, 0.2, 0.0, 0, 0, 0, 1])
    far2 = orc.pair_distance(0, 1, qa, qb, base_b=[23.0, 0.2, 0.0, 0, 0, 0, 1])
    assert np.all(far1 > 10)
    assert np.allclose(far2 - far1, 3.0, atol=1e-2)   # nearly parallel to x at this range
    assert np.all(far2 - far1 <= 3.0 + 1e-12)          # triangle inequality



# ---------------------------------------------------------------------------
# manipulability (Eq. 5, C_manip: singularity avoidance)

def _rot_vee(M):
    return np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]) / 2


def test_jacobian_matches_finite_differences_of_fk(oracle_mod):
    """Linear columns = d p_ee / d q_i, angular columns = the rotation rate of
    the end-effector frame, both by central differences of the FK."""
    from oracle.oracle import Oracle
    arm = _random_arm(51)
    orc = Oracle(tiny_scenario([arm]))
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(5):
        q = rng.uniform(-2.8, 2.8, 7)
        J = orc.jacobian(0, q)
        for i in range(7):
            qp, qm = q.copy(), q.copy()
            qp[i] += h
            qm[i] -= h
            Fp, Fm = orc.fk(0, qp)[0][-1], orc.fk(0, qm)[0][-1]
            dp = (Fp[:3, 3] - Fm[:3, 3]) / (2 * h)
            w = _rot_vee((Fp[:3, :3] - Fm[:3, :3]) / (2 * h) @ orc.fk(0, q)[0][-1][:3, :3].T)
            assert np.allclose(J[:3, i], dp, atol=1e-8)
            assert np.allclose(J[3:, i], w, atol=1e-8)


def test_manipulability_is_the_product_of_singular_values(oracle_mod):
    from oracle.oracle import Oracle
    for dof, seed in ((7, 52), (6, 53), (9, 54)):
        arm = _random_arm(seed, dof=dof)
        orc = Oracle(tiny_scenario([arm]))
        rng = np.random.default_rng(seed)
        for _ in range(5):
            q = rng.uniform(-2.8, 2.8, dof)
            sv = np.linalg.svd(orc.jacobian(0, q), compute_uv=False)
            assert math.isclose(orc.manipulability(0, q), float(np.prod(sv[:min(6, dof)])),
                                rel_tol=1e-9)


def test_manipulability_planar_two_link_closed_form(oracle_mod):
    """Planar two-link arm: J has the linear rows (-a1 s1 - a2 s12, -a2 s12;
    a1 c1 + a2 c12, a2 c12; 0, 0) and the angular rows (0, 0; 0, 0; 1, 1);
    the manipulability is sqrt(det(J^T J))."""
    from oracle.oracle import Oracle
    a1, a2 = 0.5, 0.25
    orc = Oracle(tiny_scenario([dh_arm([[a1, 0, 0, 0], [a2, 0, 0, 0]])]))
    rng = np.random.default_rng(8)
    for _ in range(10):
        q = rng.uniform(-2.8, 2.8, 2)
        s1, c1 = math.sin(q[0]), math.cos(q[0])
        s12, c12 = math.sin(q[0] + q[1]), math.cos(q[0] + q[1])
        J = np.array([[-a1 * s1 - a2 * s12, -a2 * s12], [a1 * c1 + a2 * c12, a2 * c12],
                      [0, 0], [0, 0], [0, 0], [1, 1]])
        assert np.allclose(orc.jacobian(0, q), J, atol=1e-14)
        assert math.isclose(orc.manipulability(0, q), math.sqrt(np.linalg.det(J.T @ J)),
                            rel_tol=1e-9, abs_tol=1e-12)


def test_manip_cost_ramp(oracle_mod):
    assert oracle_mod.manip_cost(0.0, 0.02) == 1.0
    assert oracle_mod.manip_cost(0.01, 0.02) == 0.5
    assert oracle_mod.manip_cost(0.02, 0.02) == 0.0
    assert oracle_mod.manip_cost(0.5, 0.02) == 0.0


def test_manip_term_enters_the_stage_cost(oracle_mod):
    """With only w_manip weighted, a standing rollout's stage cost is
    w_manip * max(0, 1 - w(q_h) / w0) at every step."""
    from oracle.oracle import Oracle
    arm = _random_arm(55)
    sc = tiny_scenario([arm], H=3, w_pose=0, w_stop=0, w_joint=0, w_coll=0, w_self=0,
                       w_manip=2.0, manip_w0=0.5)
    orc = Oracle(sc)
    gp, gR = goals_of(orc, sc)
    q = np.random.default_rng(1).uniform(-2.8, 2.8, 7)
    _, stage, _, _ = orc.rollout(0, [q], [np.zeros(7)], gp, gR, np.zeros((3, 7)))
    w = orc.manipulability(0, q)
    assert w < 0.5
    assert np.allclose(stage, 2.0 * (1 - w / 0.5), rtol=1e-12)

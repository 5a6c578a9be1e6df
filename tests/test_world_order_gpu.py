"""The rollout reads the world spheres in its own spatial order (sorted by
the Morton code of their centres each cycle, so that its clusters of 8 stay
compact); the order changes no result.  The same scene with the world
spheres (and their velocities) given in a shuffled order runs the same
cycles bit for bit: per-sample costs, the updated mean, the published plan
and the chosen control."""
import numpy as np
import pytest

from paper_2602_10114_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10114_gb300 import build, mrs
    build.build()
    mrs.load()


def _cycles(sc, world, vel, cycles):
    from paper_2602_10114_gb300 import mrs
    ctl = mrs.Controller(sc)
    ctl.set_world(world, vel)
    gp, gR = zip(*[ctl.goal_pose(a, sc.goal_q[a]) for a in range(sc.n_arms)])
    outs = []
    for _ in range(cycles):
        out = ctl.step(sc.q0, sc.qd0, list(gp), list(gR))
        outs.append((out, [ctl.debug_costs(a).copy() for a in range(sc.n_arms)]))
    ctl.close()
    return outs


@pytest.mark.parametrize("idx", [5, 2])
def test_world_order_changes_no_result(idx):
    sc = S.shrink(S.config(idx), K_div=16) if idx == 5 else S.config(idx)
    rng = np.random.default_rng(11)
    perm = rng.permutation(len(sc.world))
    vel = sc.world_vel
    ref = _cycles(sc, sc.world, vel, 3)
    got = _cycles(sc, sc.world[perm], None if vel is None else vel[perm], 3)
    for (o1, c1), (o2, c2) in zip(ref, got):
        for a in range(sc.n_arms):
            assert np.array_equal(c1[a], c2[a]), f"arm {a} costs"
        for k in ("mean_plan", "plan_spheres", "u_star", "dist_to_goal"):
            assert np.array_equal(o1[k], o2[k]), k

"""A world crowded around the arms' bases: the rollout's overflow paths
against the oracle.

The rollout culls the other spheres of a work unit in three conservative
box tests and lists what survives per warp (candidates) and per block
(obstacle pairs); a full candidate list is drained and refilled, and pairs
beyond the block list's capacity are taken by the warp that found them.
Here 600 world spheres have their centres inside one sphere that never
moves (the sphere of link 1 at the frame-0 origin, which FK puts at the base
for every joint vector), so every sample's box of that sphere contains
them: the warp holding it lists at least 600 candidates (several drains of
its list of 128) and at least 600 obstacle pairs in every work unit (more
than the block list's 512).  200 more sit inside the same sphere of a
second arm and 112 inside that of each of the other two (drains without
overflow).

The world clearance is a minimum, so only the deepest pair of the crowd
decides it: the crowd's radii are 1 cm but for one of 4 cm, its centre within a
fifth of the fixed sphere's radius like the rest, so that its clearance is
at least 1.6 cm below every other's (w_coll * 0.016 / B_world per step, far
above the cost tolerance).  Which crowd sphere is the deep one is varied
over the crowd's extreme points (lowest and highest x, y, z), so that the
deciding pair comes early and late in the spatial order in which the lists
fill, and a pair lost in a drain or an overflow shows in the costs.  The host
tests check the premises with the oracle's FK and that the oracle's costs
move well beyond the tolerance without the deep spheres; the GPU test
replays two cycles against the oracle under two launch shapes."""
import numpy as np
import pytest

from paper_2602_10114_gb300 import scenarios as S

CLUSTER = (600, 200, 112, 112)   # world spheres inside the fixed sphere of each arm
R_CROWD, R_DEEP, SPREAD = 0.01, 0.04, 0.2
EXTREMES = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]   # (axis, highest?)


def _fixed_sphere(arm):
    """Index of the sphere of link 1 at the frame-0 origin, and its radius."""
    body = np.asarray(arm.sphere_body)
    j = int(np.flatnonzero(body == 1)[-1])
    return j, float(arm.sphere_xyzr[j][3])


def _scene(extreme=(0, 0)):
    rng = np.random.default_rng(21)
    sc = S.shrink(S.config(2), K=128)
    parts = []
    for a, n in enumerate(CLUSTER):
        base = np.asarray(sc.arms[a].base_pose[:3], np.float64)
        _, r = _fixed_sphere(sc.arms[a])
        u = rng.normal(size=(n, 3))
        u *= (rng.uniform(0.0, SPREAD * r, (n, 1)) / np.linalg.norm(u, axis=1, keepdims=True))
        c = np.concatenate([base + u, np.full((n, 1), R_CROWD)], axis=1)
        axis, high = extreme
        c[int(np.argmax(u[:, axis]) if high else np.argmin(u[:, axis])), 3] = R_DEEP
        parts.append(c)
    sc.world = np.concatenate(parts).astype(np.float32)
    sc.world_vel = None
    return sc


@pytest.mark.parametrize("extreme", EXTREMES)
def test_the_crowd_sits_inside_a_sphere_that_never_moves(extreme):
    from oracle.oracle import Oracle
    sc = _scene(extreme)
    orc = Oracle(sc, threads=1)
    rng = np.random.default_rng(5)
    w = sc.world.astype(np.float64)
    start = 0
    for a, n in enumerate(CLUSTER):
        j, r = _fixed_sphere(sc.arms[a])
        crowd = w[start:start + n]
        start += n
        for q in rng.uniform(-2.8, 2.8, (16, sc.arms[a].dof)):
            _, sph = orc.fk(a, q)
            assert np.linalg.norm(sph[j, :3] - np.asarray(sc.arms[a].base_pose[:3])) < 1e-6
            gap = np.linalg.norm(crowd[:, :3] - sph[j, :3], axis=1) - crowd[:, 3] - sph[j, 3]
            assert np.all(np.linalg.norm(crowd[:, :3] - sph[j, :3], axis=1) < SPREAD * r + 1e-6)
            # one deep sphere, its clearance at least 1.5 cm below every other's
            deep = np.flatnonzero(crowd[:, 3] > R_CROWD + 1e-6)
            assert len(deep) == 1
            rest = np.delete(gap, deep[0])
            assert gap[deep[0]] < rest.min() - 0.015
    # one warp's candidates and one block's pairs: more than the lists hold
    assert sum(CLUSTER) == 1024 and CLUSTER[0] > 512 and min(CLUSTER) > 96


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(32, 0, 0), (128, 0, 1)])
@pytest.mark.parametrize("extreme", EXTREMES)
def test_crowded_world_matches_the_oracle(shape, extreme):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10114_gb300 import build, mrs
    build.build()
    mrs.load()
    from parity_utils import Replay
    from test_parity_gpu import _check_cycle, _dump
    sc = _scene(extreme)
    R = Replay(sc)
    R.ctl.set_rollout_shape(*shape)
    for _ in range(2):
        d = _dump(sc)
        got, gc, ga, gs, exp = R.cycle(d)
        _check_cycle(R, got, gc, ga, gs, exp, d, label="dense world")
        R.advance(exp)


def test_losing_the_deciding_pair_would_show():
    """With the deep sphere of each crowd shrunk to the crowd's radius (what
    the rollout would see if it lost that sphere's pairs), the oracle's
    cost of every sample moves by more than ten times the parity tolerance."""
    from oracle.oracle import Oracle
    from parity_utils import cost_tol, goals
    sc = _scene()
    lost = _scene()
    lost.world[:, 3] = np.minimum(lost.world[:, 3], R_CROWD)
    costs = []
    for s in (sc, lost):
        orc = Oracle(s, threads=4)
        gp, gR = goals(orc, s)
        exp = orc.cycle([np.asarray(q, np.float64) for q in s.q0],
                        [np.asarray(q, np.float64) for q in s.qd0], gp, gR)
        costs.append(exp["costs"])
    assert np.all(np.abs(costs[0] - costs[1]) > 10 * cost_tol(costs[0]))

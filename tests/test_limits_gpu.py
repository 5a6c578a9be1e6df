"""The largest sizes include/mrs.h allows, each on its own and all at once,
against the oracle."""
import math

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


def _scenario(arms, world, aabb, name="limits"):
    A = len(arms)
    rng = np.random.default_rng(7)
    q0 = [rng.uniform(-1, 1, a.dof).astype(np.float32) for a in arms]
    gq = [rng.uniform(a.q_lo, a.q_hi).astype(np.float32) for a in arms]
    return S.Scenario(name, arms, dict(S.DEFAULT_PARAMS), np.asarray(world, np.float32), None,
                      np.asarray(aabb, np.float32).reshape(-1, 6), q0,
                      [np.zeros(a.dof, np.float32) for a in arms], gq,
                      np.zeros((A, 3), np.float32), cycles=2)


def _replay(sc, cycles=2):
    from parity_utils import Replay
    from test_parity_gpu import _check_cycle, _dump
    R = Replay(sc)
    for _ in range(cycles):
        d = _dump(sc)
        got, gc, ga, gs, exp = R.cycle(d)
        _check_cycle(R, got, gc, ga, gs, exp, d, label="limits")
        R.advance(exp)


def test_thirty_two_arms():
    """MRS_MAX_ARMS arms on a 1.5 m circle, each coupled to 31 published plans."""
    rng = np.random.default_rng(1)
    geo = S.random_geometry(rng, 3, per_link=1, tool_spheres=1)
    arms = [S._make_arm(geo, 3, 32, 4, (1.5 * math.cos(2 * math.pi * a / 32),
                                         1.5 * math.sin(2 * math.pi * a / 32), 0.0),
                        2 * math.pi * a / 32 + math.pi) for a in range(32)]
    _replay(_scenario(arms, [[0.0, 0.0, 0.6, 0.1]], np.zeros((0, 6))))


def test_largest_arm_horizon_and_world():
    """One arm of MRS_MAX_DOF joints and MRS_MAX_SPHERES spheres over
    MRS_MAX_HORIZON steps, among MRS_MAX_WORLD_SPHERES spheres and
    MRS_MAX_AABBS boxes."""
    rng = np.random.default_rng(2)
    geo = S.random_geometry(rng, 9, per_link=7, tool_spheres=1)
    assert len(geo["sphere_body"]) == 64
    arm = S._make_arm(geo, 9, 32, 128, (0.0, 0.0, 0.0), 0.0)
    world = np.concatenate([rng.uniform([-1.5, -1.5, 0.0], [1.5, 1.5, 1.5], (1024, 3)),
                            rng.uniform(0.02, 0.05, (1024, 1))], axis=1)
    boxes = np.concatenate([rng.uniform([-1.5, -1.5, 0.0], [1.5, 1.5, 1.5], (64, 3)),
                            rng.uniform(0.02, 0.06, (64, 3))], axis=1)
    _replay(_scenario([arm], world, boxes), cycles=1)


def test_most_samples():
    """MRS_MAX_SAMPLES samples of one arm (the one-arm workload's geometry)."""
    sc = S.shrink(S.config(1), K=8192)
    _replay(sc, cycles=1)


def test_every_limit_at_once():
    """32 arms of 64 spheres (9 DoF) among MRS_MAX_WORLD_SPHERES spheres and
    MRS_MAX_AABBS boxes: the largest staging the header allows (a step's 31
    published plans of 64 spheres and the full world, with their clusters and
    candidate lists) fits one block's shared memory, and two replayed cycles
    (the second stages the published plans) match the oracle."""
    rng = np.random.default_rng(3)
    geo = S.random_geometry(rng, 9, per_link=7, tool_spheres=1)
    assert len(geo["sphere_body"]) == 64
    arms = [S._make_arm(geo, 9, 32, 4, (2.0 * math.cos(2 * math.pi * a / 32),
                                        2.0 * math.sin(2 * math.pi * a / 32), 0.0), 0.0)
            for a in range(32)]
    world = np.concatenate([rng.uniform([-2.5, -2.5, 0.0], [2.5, 2.5, 1.5], (1024, 3)),
                            rng.uniform(0.02, 0.05, (1024, 1))], axis=1)
    boxes = np.concatenate([rng.uniform([-2.5, -2.5, 0.0], [2.5, 2.5, 1.5], (64, 3)),
                            rng.uniform(0.02, 0.06, (64, 3))], axis=1)
    _replay(_scenario(arms, world, boxes), cycles=2)

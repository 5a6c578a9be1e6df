"""The seeded input generator: deterministic, float32-exact, and with the
shapes of the five workloads."""
import numpy as np
import pytest

from paper_2602_10114_gb300 import scenarios as S


@pytest.mark.parametrize("idx", [1, 2, 3, 4, 5])
def test_deterministic_and_float32(idx):
    a, b = S.config(idx), S.config(idx)
    for x, y in zip(a.arms, b.arms):
        assert np.array_equal(x.dh, y.dh) and np.array_equal(x.sphere_xyzr, y.sphere_xyzr)
        assert x.dh.dtype == np.float32 and x.sphere_xyzr.dtype == np.float32
    assert np.array_equal(a.world, b.world) and a.world.dtype == np.float32
    assert all(np.array_equal(p, q) for p, q in zip(a.q0, b.q0))
    c = S.config(idx, run=1)
    assert not np.array_equal(a.world, c.world)


def test_workload_shapes():
    c1 = S.config(1)
    assert c1.n_arms == 1 and c1.arms[0].n_spheres == 28 and c1.rollout_steps() == 1024
    assert len(c1.world) == 8 and len(c1.aabb) == 0
    c2 = S.config(2)
    assert c2.n_arms == 4 and all(a.n_spheres == 40 for a in c2.arms)
    assert c2.rollout_steps() == 61_440 and len(c2.world) == 32 and len(c2.aabb) == 4
    c4 = S.config(4)
    assert c4.n_arms == 16 and c4.rollout_steps() == 549_888
    assert sorted({a.n_spheres for a in c4.arms}) == [35, 40, 50]
    c5 = S.config(5)
    assert c5.rollout_steps() == 2_097_152 and c5.world_vel is not None
    assert np.linalg.norm(c5.world_vel, axis=1).max() <= 0.5


def test_bases_face_the_centre_and_obstacles_clear_bases():
    sc = S.config(2)
    for a in sc.arms:
        p = a.base_pose[:3].astype(np.float64)
        assert abs(np.linalg.norm(p[:2]) - 0.6) < 1e-6
        w, z = a.base_pose[3], a.base_pose[6]
        yaw = 2 * np.arctan2(z, w)
        fwd = np.array([np.cos(yaw), np.sin(yaw)])
        assert np.dot(fwd, -p[:2] / np.linalg.norm(p[:2])) > 0.999
        d = np.linalg.norm(sc.world[:, :3] - p, axis=1) - sc.world[:, 3]
        assert d.min() > 0.15 - 1e-6

"""The closed-loop task harness: its contact and distance scores on
constructed states (CPU), and one short episode of every variant (GPU)."""
import math

import numpy as np
import pytest

from paper_2602_10114_gb300 import harness as Hn
from paper_2602_10114_gb300 import scenarios as S


def test_sphere_box_distance_points():
    box = np.array([0.0, 0.0, 0.0, 0.5, 0.25, 0.125])
    c = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 1.0, 0.0], [0.5, 0.0, 0.0]])
    r = np.array([0.1, 0.05, 0.0, 0.0])
    d = Hn.sphere_box_distance(c, r, box)
    assert math.isclose(d[0], 0.5 - 0.1)                         # face
    assert math.isclose(d[1], -0.125 - 0.05)                     # centre inside: depth to nearest face
    assert math.isclose(d[2], math.hypot(0.5, 0.75))             # corner region (edge in 2-D)
    assert math.isclose(d[3], 0.0, abs_tol=1e-15)                # on the surface


def test_contacts_between_arms_and_with_the_world():
    a = np.array([[0.0, 0.0, 0.0, 0.1], [0.0, 0.0, 0.5, 0.1]])
    b = np.array([[0.25, 0.0, 0.0, 0.1]])                        # 0.25 apart: clear
    c = np.array([[0.15, 0.0, 0.5, 0.1]])                        # overlaps a's second sphere
    world = np.array([[2.0, 0.0, 0.0, 0.5]])
    box = np.array([[0.0, 0.0, -1.0, 1.0, 1.0, 0.05]])
    assert Hn.contacts([a, b], world, np.zeros((0, 6))) == (False, False)
    assert Hn.contacts([a, b, c], world, np.zeros((0, 6))) == (True, False)
    assert Hn.contacts([a, b], np.array([[0.2, 0.0, 0.0, 0.15]]), np.zeros((0, 6)))[1]
    assert not Hn.contacts([a], world, box)[1]                   # box top at z = -0.95
    assert Hn.contacts([np.array([[0.0, 0.0, -0.9, 0.1]])], world, box)[1]


@pytest.mark.gpu
@pytest.mark.parametrize("variant", list(Hn.VARIANTS))
def test_short_episode_of_every_variant(variant):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sc = S.shrink(S.config(2), K=64, H=10)
    for task in ("following", "reaching"):
        r = Hn.run_episode(sc, variant, cycles=20, task=task)
        assert r["cycles"] == 20 and 0 <= r["collision_score"] <= 20
        assert r["arm_contact_steps"] <= r["collision_score"] <= (r["arm_contact_steps"]
                                                                  + r["world_contact_steps"])
        assert np.isfinite(r["err_f"]) and r["err_f"] > 0

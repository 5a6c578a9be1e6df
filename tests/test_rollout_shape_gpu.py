"""Rollout launch shapes (samples per work unit, resident blocks per SM, work
order) and the autotuner that picks one: the shape changes the time, never the
result."""
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


def _controller(sc):
    from paper_2602_10114_gb300 import mrs
    ctl = mrs.Controller(sc)
    ctl.set_world()
    gp, gR = [], []
    for a in range(sc.n_arms):
        p, R = ctl.goal_pose(a, sc.goal_q[a])
        gp.append(p)
        gR.append(R)
    return ctl, gp, gR


def test_every_shape_gives_the_same_cycle():
    """Sixteen uneven arms, with ragged sample counts (K = 16, 80, 100, ...):
    outputs and per-sample costs of one cycle from the same state are bitwise
    equal under every shape, including each number of resident blocks."""
    sc = S.shrink(S.config(4), K_div=16)
    sc.arms[1].K, sc.arms[5].K = 80, 100
    ctl, gp, gR = _controller(sc)
    ctl.step(sc.q0, sc.qd0, gp, gR)
    blob = ctl.save_state()
    (_, _, _), mx = ctl.rollout_shape()
    # every register budget the context can launch (1-2, 3 and 4 blocks per SM)
    shapes = [(32, 0, 0), (64, 0, 0), (128, 0, 1), (96, 1, 1), (256, min(2, mx), 0), (32, 1, 1),
              (64, 0, 2), (512, 0, 1), (1024, 0, 2)] + [(64, b, 1) for b in range(1, mx + 1)]
    ref = None
    for sh in shapes:
        ctl.load_state(blob)
        ctl.set_rollout_shape(*sh)
        out = ctl.step(sc.q0, sc.qd0, gp, gR)
        got = (out, [ctl.debug_costs(a) for a in range(sc.n_arms)])
        if ref is None:
            ref = got
            continue
        for k in ref[0]:
            assert np.array_equal(got[0][k], ref[0][k]), (sh, k)
        for a in range(sc.n_arms):
            assert np.array_equal(got[1][a], ref[1][a]), (sh, a)


def test_shape_out_of_range_is_rejected():
    from paper_2602_10114_gb300 import mrs
    ctl, _, _ = _controller(S.config(1))
    (_, _, _), mx = ctl.rollout_shape()
    for sh in [(16, 0, 0), (48, 0, 0), (1056, 0, 0), (32, mx + 1, 0), (32, 0, 3), (32, -1, 0)]:
        with pytest.raises(mrs.MrsError) as e:
            ctl.set_rollout_shape(*sh)
        assert e.value.status == 1


def test_autotune_keeps_the_fastest_and_restores_the_state():
    from paper_2602_10114_gb300 import mrs
    sc = S.config(2)
    ctl, gp, gR = _controller(sc)
    with pytest.raises(mrs.MrsError) as e:
        ctl.autotune(reps=2)           # no inputs yet
    assert e.value.status == 5
    ctl.step(sc.q0, sc.qd0, gp, gR)
    blob = ctl.save_state()
    best, tab = ctl.autotune(reps=3)
    (_, _, _), mx = ctl.rollout_shape()
    assert len(tab) == 6 * mx * 3
    assert all(t["cycle_ms"] > 0 for t in tab)
    assert best["cycle_ms"] == min(t["cycle_ms"] for t in tab)
    assert ctl.rollout_shape()[0] == (best["tile_samples"], best["blocks_per_sm"], best["order"])
    assert ctl.save_state() == blob
    # the next cycle equals the one the untuned controller runs
    ref, _, _ = _controller(sc)
    ref.step(sc.q0, sc.qd0, gp, gR)
    a = ctl.step(sc.q0, sc.qd0, gp, gR)
    b = ref.step(sc.q0, sc.qd0, gp, gR)
    for k in a:
        assert np.array_equal(a[k], b[k]), k

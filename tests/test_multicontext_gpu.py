"""Arms split across contexts (each controlling its local arms, the others
external) and plan exchange through paper_2602_10114_gb300.exchange; host-side
fault injection on the plan board (dropped, stale and non-finite plans)."""
import numpy as np
import pytest

from paper_2602_10114_gb300 import exchange, scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10114_gb300 import build, mrs
    build.build()
    mrs.load()


def _inputs(sc):
    from oracle.oracle import Oracle
    from parity_utils import goals
    gp, gR = goals(Oracle(sc), sc)
    return ([q.astype(np.float32) for q in sc.q0], [q.astype(np.float32) for q in sc.qd0],
            gp.astype(np.float32), gR.astype(np.float32))


def test_split_contexts_with_exchange_match_one_context():
    from paper_2602_10114_gb300 import mrs
    sc = S.shrink(S.config(2), K=96, H=12)
    q, qd, gp, gR = _inputs(sc)
    one = mrs.Controller(sc)
    one.set_world()
    parts = [mrs.Controller(sc, external={2, 3}), mrs.Controller(sc, external={0, 1})]
    for c in parts:
        c.set_world()
    for cycle in range(4):
        ref = one.step(q, qd, gp, gR)
        outs = [c.step(q, qd, gp, gR) for c in parts]
        entries = exchange.local_entries(parts[0], outs[0], cycle) + \
            exchange.local_entries(parts[1], outs[1], cycle)
        for c in parts:
            exchange.share_remote(c, entries)
        for c, o in zip(parts, outs):
            for a in range(sc.n_arms):
                if a in c.external:
                    continue
                for k in ("mean_plan", "plan_spheres", "plan_q"):
                    kind = "hs" if k == "plan_spheres" else "hd"
                    assert np.array_equal(c.split(o[k], kind, a), one.split(ref[k], kind, a)), k
                assert np.array_equal(c.split(o["u_star"], "d", a), one.split(ref["u_star"], "d", a))


def test_dropped_stale_and_corrupt_plans():
    """Host-side fault injection: a NaN plan is rejected (MRS_EINVAL) and the
    board keeps its entry; a withdrawn plan is ignored; with max_plan_age = 1
    an entry not refreshed for two cycles is ignored; the controller keeps
    stepping throughout."""
    from paper_2602_10114_gb300 import mrs
    sc = S.shrink(S.config(2), K=64, H=8)
    sc.params["max_plan_age"] = 1
    q, qd, gp, gR = _inputs(sc)
    c = mrs.Controller(sc, external={3})
    c.set_world()
    r0 = c.step(q, qd, gp, gR)                  # cycle 0: arms 0..2 publish
    good = c.split(r0["plan_spheres"], "hs", 0).copy()
    bad = good.copy()
    bad[2, 5, 1] = np.nan
    with pytest.raises(mrs.MrsError) as e:
        c.share_plans(3, bad, None, 0.3, 0)
    assert e.value.status == 1
    c.step(q, qd, gp, gR)                       # cycle 1: arm 3 never published
    assert np.all(c.debug_alpha()[:3, 3] == 0)
    c.share_plans(3, good, None, 0.3, 1)        # arm 3 publishes at cycle 1
    c.step(q, qd, gp, gR)                       # cycle 2: age 1, used
    assert np.all(c.debug_alpha()[:3, 3] > 0)
    c.step(q, qd, gp, gR)                       # cycle 3: age 2, stale
    assert np.all(c.debug_alpha()[:3, 3] == 0)
    c.share_plans(3, good, None, 0.3, 3)
    c.step(q, qd, gp, gR)                       # fresh again
    assert np.all(c.debug_alpha()[:3, 3] > 0)
    c.share_plans(3, good, None, -1.0, 4)       # withdrawn (dropped)
    r = c.step(q, qd, gp, gR)
    assert np.all(c.debug_alpha()[:3, 3] == 0)
    assert np.all(np.isfinite(r["mean_plan"]))


def test_a_smaller_context_made_later_leaves_a_larger_one_runnable():
    """The kernels' dynamic shared-memory limits are per process, not per
    context: a context whose rollout stages 256 world spheres keeps running
    after contexts with smaller staging (the initial 64-sphere capacity) are
    created, and computes what it computed before them."""
    from paper_2602_10114_gb300 import mrs
    big = S.shrink(S.config(5), K=32, H=8)
    q, qd, gp, gR = _inputs(big)
    ctl = mrs.Controller(big)
    ctl.set_world()                          # 256 spheres: the staging grows
    blob = ctl.save_state()
    ref = ctl.step(q, qd, gp, gR)
    small = [mrs.Controller(S.shrink(S.config(2), K=32, H=8)) for _ in range(2)]
    small.append(mrs.Controller(big, external=set(range(1, big.n_arms))))
    ctl.load_state(blob)
    got = ctl.step(q, qd, gp, gR)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    for c in small:
        c.close()

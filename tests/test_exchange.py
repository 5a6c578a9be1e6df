"""Plan exchange between processes (no GPU): two gloo ranks each optimise
half of the arms with the oracle controller and exchange their published
plans after every cycle; the result equals one process optimising all arms,
bit for bit.  Also the pack/unpack round trip and the stale-plan rule."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2602_10114_gb300 import exchange, scenarios as S

CYCLES = 3


def _scene():
    return S.shrink(S.config(2), K=12, H=5)


def _goals(orc, sc):
    from parity_utils import goals
    return goals(orc, sc)


def _oracle_entries(orc, arms):
    s = orc.state
    return [exchange.PlanEntry(a, int(s["plan_stamp"][a]), float(s["plan_dist"][a]),
                               orc.split(s["plan_spheres"], "hs", a).copy(),
                               orc.split(s["plan_q"], "hd", a).copy()) for a in arms]


def _oracle_share(orc, entries, remote):
    s = orc.state
    for e in entries:
        if e.arm not in remote:
            continue
        orc.split(s["plan_spheres"], "hs", e.arm)[:] = e.plan_spheres
        orc.split(s["plan_q"], "hd", e.arm)[:] = e.plan_q
        s["plan_dist"][e.arm] = e.dist_to_goal
        s["plan_stamp"][e.arm] = e.stamp
        s["plan_valid"][e.arm] = 1


def _run(orc, sc, arms, exchange_fn):
    """CYCLES closed-loop cycles; the plant integrates each local arm's U_*."""
    gp, gR = _goals(orc, sc)
    q = [x.astype(np.float64) for x in sc.q0]
    qd = [x.astype(np.float64) for x in sc.qd0]
    dt = float(np.float32(sc.params["dt"]))
    for _ in range(CYCLES):
        out = orc.cycle(q, qd, gp, gR)
        exchange_fn(orc)
        for a in arms:
            u = orc.split(out["u_star"], "d", a)
            qd[a] = qd[a] + u * dt
            q[a] = q[a] + qd[a] * dt
    return {a: (orc.split(orc.state["mu"], "hd", a).copy(),
                orc.split(orc.state["plan_spheres"], "hs", a).copy()) for a in arms}


def _rank(rank, world, port, tmpdir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch.distributed as dist
    from oracle.oracle import Oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    sc = _scene()
    mine = [a for a in range(sc.n_arms) if a % world == rank]
    active = [1 if a in mine else 0 for a in range(sc.n_arms)]
    orc = Oracle(sc, active=active)

    def ex(o):
        got = exchange.all_gather_entries(_oracle_entries(o, mine), sc)
        _oracle_share(o, got, [a for a in range(sc.n_arms) if a not in mine])

    res = _run(orc, sc, mine, ex)
    np.savez(os.path.join(tmpdir, f"rank{rank}.npz"),
             **{f"mu{a}": v[0] for a, v in res.items()},
             **{f"plan{a}": v[1] for a, v in res.items()})
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_pack_roundtrip():
    sc = _scene()
    rng = np.random.default_rng(0)
    es = [exchange.PlanEntry(a, 7 + a, 0.1 * a, rng.normal(size=(5, 40, 4)), rng.normal(size=(5, 7)))
          for a in (1, 3)]
    back = exchange.unpack(exchange.pack(es, sc), sc)
    for e, b in zip(es, back):
        assert (e.arm, e.stamp, e.dist_to_goal) == (b.arm, b.stamp, b.dist_to_goal)
        assert np.array_equal(e.plan_spheres, b.plan_spheres) and np.array_equal(e.plan_q, b.plan_q)


def test_two_gloo_ranks_match_one_process(tmp_path):
    from oracle.oracle import Oracle
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    sc = _scene()
    ref = _run(Oracle(sc), sc, list(range(sc.n_arms)), lambda o: None)
    for rank in range(world):
        got = np.load(os.path.join(tmp_path, f"rank{rank}.npz"))
        for a in range(sc.n_arms):
            if a % world != rank:
                continue
            assert np.array_equal(got[f"mu{a}"], ref[a][0])
            assert np.array_equal(got[f"plan{a}"], ref[a][1])


def test_stale_plans_count_as_missing():
    """With max_plan_age = 1, a board entry that was not refreshed for two
    cycles is ignored: no coordination cost and no priority weight."""
    from oracle.oracle import Oracle
    sc = _scene()
    sc.params["max_plan_age"] = 1
    orc = Oracle(sc, active=[1, 0, 0, 0])        # arm 0 local; 1..3 published once
    gp, gR = _goals(orc, sc)
    full = Oracle(sc)
    full.cycle(sc.q0, sc.qd0, gp, gR)            # every arm publishes at cycle 0
    for k in ("plan_spheres", "plan_q", "plan_dist", "plan_stamp", "plan_valid"):
        orc.state[k][:] = full.state[k]
    orc.cycle_index = 1
    o1 = orc.cycle(sc.q0, sc.qd0, gp, gR)       # cycle 1: age 1, used
    assert np.all(o1["alpha"].reshape(4, 4)[0, 1:] > 0) and o1["n_queries"][0] > 0
    o2 = orc.cycle(sc.q0, sc.qd0, gp, gR)       # cycle 2: age 2, ignored
    assert np.all(o2["alpha"].reshape(4, 4)[0] == 0) and o2["n_queries"][0] == 0

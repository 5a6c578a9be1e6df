"""A device-side bounded wait that runs out: the rollout's wait for its staged
plan copies, given no polls at all, gives up; the block records the error
word, drains its copies and ends, and mrs_step reports MRS_ETIMEOUT without a
trap, fault or hang.  The context is then usable again after a state load:
the next cycle equals the one an untouched context runs from that state."""
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


def test_rollout_wait_that_runs_out_returns_timeout_and_the_context_recovers():
    from oracle.oracle import Oracle
    from paper_2602_10114_gb300 import mrs
    from parity_utils import goals
    sc = S.shrink(S.config(2), K=64, H=6)
    gp, gR = goals(Oracle(sc), sc)
    gp, gR = gp.astype(np.float32), gR.astype(np.float32)
    ctl = mrs.Controller(sc)
    ctl.set_world()
    ctl.step(sc.q0, sc.qd0, gp, gR)        # cycle 0 publishes every arm's plan
    blob = ctl.save_state()
    ref = ctl.step(sc.q0, sc.qd0, gp, gR)  # cycle 1 stages the neighbours' plans
    with pytest.raises(mrs.MrsError):
        ctl.set_wait_limit(1 << 23)        # above the default: refused
    for _ in range(2):                     # twice: the hook can be used again
        ctl.load_state(blob)
        ctl.set_wait_limit(0)
        with pytest.raises(mrs.MrsError) as e:
            ctl.step(sc.q0, sc.qd0, gp, gR)
        assert e.value.status == 4                         # MRS_ETIMEOUT
        ctl.set_wait_limit(-1)
        ctl.load_state(blob)
        got = ctl.step(sc.q0, sc.qd0, gp, gR)
        for k in ref:
            assert np.array_equal(got[k], ref[k]), k

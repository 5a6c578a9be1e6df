"""mrs_step's two ways of returning results: copied into caller buffers
(`out`), or left in the context's pinned block read through
mrs_output_host (what the Python binding's step() uses).  Both must hold the
same values, equal to the binding's result for the same cycle."""
import ctypes as C

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


def test_caller_buffers_and_pinned_block_agree():
    from paper_2602_10114_gb300 import mrs
    sc = S.shrink(S.config(2), K=96, H=12)
    ctl = mrs.Controller(sc)
    ctl.set_world()
    gp, gR = [], []
    for a in range(sc.n_arms):
        p, R = ctl.goal_pose(a, sc.goal_q[a])
        gp.append(p)
        gR.append(R)
    blob = ctl.save_state()
    ref = ctl.step(sc.q0, sc.qd0, gp, gR)          # through the pinned block

    # the same cycle again, results copied into caller buffers
    ctl.load_state(blob)
    xin, states, block, keys = ctl._sbuf
    parts = []
    for a in range(sc.n_arms):
        parts += (np.asarray(sc.q0[a], np.float32), np.asarray(sc.qd0[a], np.float32),
                  np.ravel(gp[a]).astype(np.float32), np.ravel(gR[a]).astype(np.float32))
    np.concatenate(parts, out=xin)
    bufs = {k: np.full(s.stop - s.start, np.nan, np.float32) for k, s in keys}
    out = mrs.MrsStepOut(*[bufs[k].ctypes.data_as(C.POINTER(C.c_float))
                           for k in mrs.Controller._OUT_KEYS])
    assert ctl.L.mrs_step(ctl.h, states, C.byref(out)) == 0
    for k, s in keys:
        assert np.array_equal(bufs[k], block[s]), k        # caller copy == pinned block
        assert np.array_equal(bufs[k], ref[k]), k          # == the binding's result
    # the pinned pointers are the ones mrs_output_host reports
    o = mrs.MrsStepOut()
    assert ctl.L.mrs_output_host(ctl.h, C.byref(o)) == 0
    u = np.ctypeslib.as_array(o.u_star, shape=(ctl.sizes.d,))
    assert np.array_equal(u, ref["u_star"])
    ctl.close()

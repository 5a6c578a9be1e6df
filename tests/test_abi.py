"""The C ABI library (no GPU needed): it loads, exports every entry point
include/mrs.h declares, and rejects bad arguments before touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_10114_gb300 import build, mrs
    build.build()
    return mrs.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mrs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mrs_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2602_10114_gb300 import mrs
    assert set(declared_functions()) == set(mrs.SIGNATURES)


def test_argument_errors_without_a_device(lib):
    from paper_2602_10114_gb300 import mrs
    h = C.c_void_p()
    assert lib.mrs_create(None, None, C.byref(h)) == 1
    cfg = mrs.MrsConfig()
    cfg.n_arms = 0
    assert lib.mrs_create(C.byref(cfg), None, C.byref(h)) == 1
    assert lib.mrs_last_error(None) == b"null config or arms"   # the failed create's reason
    assert lib.mrs_philox(-1, None, None, None) == 1
    assert lib.mrs_query_sizes(None, None) == 1


def test_reserved_field_and_bad_arm(lib):
    import numpy as np
    from paper_2602_10114_gb300 import mrs, scenarios
    sc = scenarios.config(1)
    a = sc.arms[0]
    keep = [np.ascontiguousarray(x, np.float32) for x in (a.dh, a.q_lo, a.q_hi, a.qd_max,
                                                         a.sphere_xyzr)]
    body = np.ascontiguousarray(a.sphere_body, np.int32)
    arm = mrs.MrsArmDesc(a.dof, a.n_spheres, a.K, a.H, *[k.ctypes.data_as(mrs._fp) for k in keep[:4]],
                         body.ctypes.data_as(mrs._ip), keep[4].ctypes.data_as(mrs._fp))
    for k in range(7):
        arm.base_pose[k] = float(a.base_pose[k])
    arms = (mrs.MrsArmDesc * 1)(arm)
    p = sc.params
    cfg = mrs.MrsConfig(1, arms, p["dt"], p["lam"], p["gamma"], p["alpha_mu"], p["alpha_sigma"],
                        p["sigma_init"], p["w_pose"], p["w_rot"], p["w_stop"], p["w_joint"],
                        p["w_coll"], p["w_self"], p["w_dyn"], p["B"], p["B_world"], p["B_self"],
                        p["tau"], p["q_margin"], 1, 0, 1)
    h = C.c_void_p()
    assert lib.mrs_create(C.byref(cfg), None, C.byref(h)) == 1       # reserved must be 0
    assert b"reserved" in lib.mrs_last_error(None)
    cfg.reserved = 0
    cfg.lambda_ = float("nan")
    assert lib.mrs_create(C.byref(cfg), None, C.byref(h)) == 1
    cfg.lambda_ = 10.0
    body[3], body[4] = 5, 2                                          # not non-decreasing
    assert lib.mrs_create(C.byref(cfg), None, C.byref(h)) == 1


def test_sizes_beyond_the_limits_are_rejected(lib):
    """Every per-arm and per-context limit of include/mrs.h, one past it:
    MRS_EINVAL from mrs_create (validated before any device use), with the
    reason from mrs_last_error(NULL)."""
    import numpy as np
    from paper_2602_10114_gb300 import mrs, scenarios
    sc = scenarios.config(1)
    a = sc.arms[0]
    p = sc.params

    def create(dof=a.dof, ns=a.n_spheres, K=a.K, H=a.H, n_arms=1):
        dh = np.zeros((dof, 4), np.float32)
        dh[:, 1] = 0.1
        lo, hi = np.full(dof, -2.8, np.float32), np.full(dof, 2.8, np.float32)
        vm = np.full(dof, 2.0, np.float32)
        body = np.minimum(np.arange(ns, dtype=np.int32) // 4 + 1, dof + 1).astype(np.int32)
        xyzr = np.tile(np.array([0, 0, 0, 0.05], np.float32), (ns, 1))
        keep = [dh, lo, hi, vm, xyzr, body]
        arm = mrs.MrsArmDesc(dof, ns, K, H, *[k.ctypes.data_as(mrs._fp) for k in keep[:4]],
                             body.ctypes.data_as(mrs._ip), xyzr.ctypes.data_as(mrs._fp))
        arm.base_pose[3] = 1.0
        arms = (mrs.MrsArmDesc * n_arms)(*([arm] * n_arms))
        cfg = mrs.MrsConfig(n_arms, arms, p["dt"], p["lam"], p["gamma"], p["alpha_mu"],
                            p["alpha_sigma"], p["sigma_init"], p["w_pose"], p["w_rot"],
                            p["w_stop"], p["w_joint"], p["w_coll"], p["w_self"], p["w_dyn"],
                            p["B"], p["B_world"], p["B_self"], p["tau"], p["q_margin"], 1, 0, 0)
        h = C.c_void_p()
        st = lib.mrs_create(C.byref(cfg), None, C.byref(h))
        return st, lib.mrs_last_error(None).decode(), keep
    for kw, word in [(dict(dof=10), "dof"), (dict(ns=65), "sphere"), (dict(K=8193), "K"),
                     (dict(H=129), "H"), (dict(n_arms=33), "n_arms"), (dict(K=0), "K"),
                     (dict(dof=0), "dof")]:
        st, why, _ = create(**kw)
        assert st == 1, kw
        assert word in why, (kw, why)

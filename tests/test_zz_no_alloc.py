"""mrs_fk_static: forward kinematics for callers that cannot allocate device
memory (a hard-period control loop, or a process whose device memory belongs
to another allocator).  Its results must equal those of mrs_fk, the entry
point that allocates its staging buffers, on consecutive calls that reuse the
static scratch.

The file is collected last (pytest collects test files in name order) so
that a run stopping at its first failure has run every other test before
this one; the tests here also pass when run alone in a fresh process, since
they depend on no earlier call."""
import numpy as np
import pytest

from paper_2602_10114_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the sphere-position tolerance of the parity tests (m)


@pytest.fixture(scope="module")
def ctl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_10114_gb300 import build, mrs
    build.build()
    mrs.load()
    return mrs.Controller(S.config(4))


def test_static_fk_matches_allocating_fk_on_consecutive_calls(ctl):
    rng = np.random.default_rng(11)
    # two calls in a row, different arms and sizes: the second reuses the
    # scratch the first one left behind
    for arm, n in [(2, 257), (0, 33), (1, 3000)]:
        a = ctl.sc.arms[arm]
        q = rng.uniform(-2.8, 2.8, (n, a.dof)).astype(np.float32)
        ee_ref, sph_ref = ctl.fk(arm, q)
        ee, sph = ctl.fk_static(arm, q)
        assert np.abs(ee - ee_ref).max() <= TOL
        assert np.abs(sph - sph_ref).max() <= TOL
        assert np.array_equal(ee, ee_ref) and np.array_equal(sph, sph_ref)


def test_static_fk_rejects_requests_beyond_the_scratch(ctl):
    from paper_2602_10114_gb300 import mrs
    a = ctl.sc.arms[2]                       # 9 DoF, 50 spheres
    n = (1 << 20) // (12 + 4 * a.n_spheres + a.dof) + 1
    q = np.zeros((n, a.dof), np.float32)
    with pytest.raises(mrs.MrsError) as e:
        ctl.fk_static(2, q)
    assert e.value.status == 1
    ee, _ = ctl.fk_static(2, q[:10])          # still usable afterwards
    assert np.all(np.isfinite(ee))

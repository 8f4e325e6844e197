"""hm_farfield_static: the far-field entry point that allocates no device memory.

Callers that cannot let the library allocate device memory during a call (their
device memory belongs to their own allocator, or their loop forbids allocation)
use it in place of hm_farfield.  It must give the same far field and RCS as
hm_farfield, call after call, since every call reuses one static device array.
This file is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

from paper_2408_17116_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2408_17116_gb300 import build, hm  # noqa: E402

build.build()


def test_static_farfield_matches_allocating_farfield_on_two_calls():
    wl = workloads.workload("sphere_d1_m1_nc8")
    s = hm.Solver()
    s.hm_build_geometry(wl["bodies"], wl["ms"], wl["nc"], wl["k"], wl["leaf"], wl["eta"], wl["aca_tol"])
    s.hm_fill()
    s.hm_factor()
    kh, pol = workloads.incidence(3, workloads.SEED + 5)
    x = s.hm_solve(kh, pol)
    _, dirs_a = workloads.rcs_cuts(181)
    _, dirs_b = workloads.rcs_cuts(19)
    for dirs in (dirs_a, dirs_b):  # two calls in a row, the second smaller than the first
        ef_ref, rcs_ref = s.hm_farfield(x, dirs)
        ef, rcs = s.hm_farfield_static(x, dirs)
        torch.cuda.synchronize()
        assert rcs.shape == rcs_ref.shape
        assert np.allclose(rcs, rcs_ref, rtol=1e-12, atol=0)
        assert torch.allclose(ef, ef_ref, rtol=1e-12, atol=0)


def test_static_farfield_rejects_requests_beyond_its_scratch():
    wl = workloads.workload("sphere_d1_m1_nc8")
    s = hm.Solver()
    s.hm_build_geometry(wl["bodies"], wl["ms"], wl["nc"], wl["k"], wl["leaf"], wl["eta"], wl["aca_tol"])
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"])
    dirs = np.tile(np.array([[0.0, 0.0, 1.0]]), (20000, 1))  # 3 x 20000 + 20000 > 65536 doubles
    with pytest.raises(hm.HmError) as e:
        s.hm_farfield_static(x, dirs)
    assert e.value.status == 1
    assert "static scratch" in str(e.value)

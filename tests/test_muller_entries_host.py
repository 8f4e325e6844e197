"""The library's N-Mueller far-entry generator (hm_muller.cuh, evaluated on the host by
hm_muller_far_block_host) against the independent oracle's Nystrom rule for the same
formulation (oracle.MullerOracle.far_block): every one of the 16 row/column
components of every source node of a patch, for real and lossy interiors and a
rotated ellipsoid.  No GPU is needed."""
import numpy as np
import pytest

import oracle
from paper_2408_17116_gb300 import hm, workloads

K = 2 * np.pi


@pytest.mark.parametrize("eps", [2.25, 10.0, 4.0 - 1.5j])
@pytest.mark.parametrize("name", ["sphere_d2_m2_nc6", "ellipsoid_small"])
def test_far_entries_match_the_oracle(name, eps):
    wl = workloads.workload(name)
    o = oracle.MullerOracle(wl["bodies"], wl["ms"], wl["nc"], K, eps)
    nc2 = wl["nc"] ** 2
    flags = o.near_flags()
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(6):
        tn = int(rng.integers(o.nnode))
        q = tn // nc2
        for p in (int(np.flatnonzero(~flags[q])[0]), int(np.flatnonzero(flags[q] & (np.arange(o.npatch) != q))[0])):
            ref = o.far_block(tn, p)
            got = hm.muller_far_block_host(wl["bodies"], wl["ms"], wl["nc"], K, eps, tn, p)
            worst = max(worst, np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert worst < 1e-12, worst


def test_rejects_bad_arguments():
    wl = workloads.workload("sphere_d1_m1_nc8")
    with pytest.raises(hm.HmError):
        hm.muller_far_block_host(wl["bodies"], wl["ms"], 1, K, 2.0, 0, 1)
    with pytest.raises(hm.HmError):
        hm.muller_far_block_host(wl["bodies"], wl["ms"], 8, K, 2.0, 10 ** 6, 1)

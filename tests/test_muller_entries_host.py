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


def _near_compare(name, eps, rule):
    wl = workloads.workload(name)
    o = oracle.MullerOracle(wl["bodies"], wl["ms"], wl["nc"], K, eps)
    flags = o.near_flags()
    nc2 = wl["nc"] ** 2
    worst = 0.0
    for tn in (0, 5, nc2 // 2 + 3, 2 * nc2 + 7):
        q = tn // nc2
        for p in np.flatnonzero(flags[q])[:4]:   # the self patch and its neighbours
            ref = o.near_block(tn, p)
            got = hm.muller_near_block_host(wl["bodies"], wl["ms"], wl["nc"], K, eps, tn, int(p), *rule)
            worst = max(worst, np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    return worst


@pytest.mark.parametrize("eps", [2.25, 10.0, 4.0 - 1.5j])
@pytest.mark.parametrize("name", ["sphere_d2_m2_nc6", "ellipsoid_small", "sphere_d1_m1_nc8"])
def test_near_rule_matches_the_oracle_integrals(name, eps):
    # the device near-field rule (24/24/16 points, inner panel 0.5) against the oracle's
    # independent adaptive + Duffy integrals of the same N-Mueller integrand
    assert _near_compare(name, eps, (0, 0, 0, 0.0)) < 2e-9


@pytest.mark.parametrize("name", ["sphere_d2_m2_nc6", "sphere_d1_m1_nc8"])
def test_near_rule_at_high_contrast_needs_more_points(name):
    # eps_r = 80: the interior wavelength is 1/9 of the exterior one; with the points
    # doubled the rule meets the oracle again (the default rule does not: 3e-5 to 3e-3)
    assert _near_compare(name, 80.0, (48, 48, 32, 0.0)) < 1e-8


def test_rhs_and_far_field_match_the_oracle():
    wl = workloads.workload("ellipsoid_small")
    o = oracle.MullerOracle(wl["bodies"], wl["ms"], wl["nc"], K, 3.0)
    kh, po = workloads.incidence(1, workloads.SEED + 3)
    rhs, _ = hm.muller_rhs_farfield_host(wl["bodies"], wl["ms"], wl["nc"], K, kh[0], po[0])
    ref = o.rhs(kh, po)[0]
    assert np.max(np.abs(rhs - ref)) <= 1e-13 * np.max(np.abs(ref))
    rng = np.random.default_rng(3)
    x = rng.standard_normal(o.N) + 1j * rng.standard_normal(o.N)
    _, dirs = workloads.rcs_cuts(19)
    _, ef = hm.muller_rhs_farfield_host(wl["bodies"], wl["ms"], wl["nc"], K, x=x, dirs=dirs)
    efo, _ = o.farfield(x, dirs)
    assert np.max(np.abs(ef - efo)) <= 1e-12 * np.max(np.abs(efo))

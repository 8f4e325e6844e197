"""The block cluster tree (Sec. III, Eq. 21) built on the host by hm_plan_host, the
same planner hm_build_geometry runs: the permutation is a bijection, the leaves tile
the matrix exactly once, every admissible leaf satisfies Eq. 21 on the bounding boxes
of its clusters, every dense leaf is a leaf-cluster pair that is not admissible, and
the leaf clusters are balanced and no larger than n_leaf.  No GPU is needed."""
import numpy as np
import pytest

import oracle
from paper_2408_17116_gb300 import hm, workloads


def _geometry(name):
    wl = workloads.workload(name)
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    return o.node_table()[:, :3], wl


def _bbox(pts):
    return pts.min(0), pts.max(0)


def _dist_diam(p1, p2):
    (a0, a1), (b0, b1) = _bbox(p1), _bbox(p2)
    gap = np.maximum(0.0, np.maximum(a0 - b1, b0 - a1))
    return np.linalg.norm(gap), min(np.linalg.norm(a1 - a0), np.linalg.norm(b1 - b0))


@pytest.mark.parametrize("dof", [2, 4])
@pytest.mark.parametrize("name", ["sphere_d2_m2_nc6", "ellipsoid_small", "sphere_d4_m2_nc10"])
def test_block_tree_invariants(name, dof):
    xyz, wl = _geometry(name)
    leaf, eta = wl["leaf"], wl["eta"]
    blocks, perm = hm.plan_host(xyz, leaf, eta, dof)
    n = xyz.shape[0]
    N = dof * n
    assert np.array_equal(np.sort(perm), np.arange(n))
    # exact tiling of the N x N matrix
    cover = np.zeros((N, N), dtype=np.int16)
    for typ, r0, nr, c0, nc in blocks:
        assert r0 % dof == 0 and nr % dof == 0 and c0 % dof == 0 and nc % dof == 0  # nodes stay whole
        cover[r0:r0 + nr, c0:c0 + nc] += 1
    assert (cover == 1).all()
    pts = xyz[perm]
    sizes = set()
    for typ, r0, nr, c0, nc in blocks:
        pr, pc = pts[r0 // dof:(r0 + nr) // dof], pts[c0 // dof:(c0 + nc) // dof]
        dist, dmin = _dist_diam(pr, pc)
        if typ == 1:
            assert dist > 0 and dmin <= eta * dist * (1 + 1e-12)
        else:
            assert not (dist > 0 and dmin <= eta * dist * (1 - 1e-12))
            assert nr <= leaf and nc <= leaf
            sizes.update((nr, nc))
    assert max(sizes) - min(sizes) <= dof  # balanced bisection: leaf clusters differ by one node at most
    assert (blocks[:, 0] == 1).sum() > 0


def test_no_admissible_blocks_when_eta_is_tiny():
    xyz, wl = _geometry("sphere_d2_m2_nc6")
    blocks, _ = hm.plan_host(xyz, wl["leaf"], 1e-9)
    assert (blocks[:, 0] == 0).all()


def test_rejects_bad_arguments():
    with pytest.raises(hm.HmError):
        hm.plan_host(np.zeros((0, 3)), 64, 2.0)
    with pytest.raises(hm.HmError):
        hm.plan_host(np.random.default_rng(0).random((10, 3)), 1, 2.0)
    with pytest.raises(hm.HmError):
        hm.plan_host(np.random.default_rng(0).random((10, 3)), 16, 2.0, dof=3)


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_degenerate_and_tiny_inputs(n):
    # coincident points: zero distances, so nothing is admissible; the tiling still holds
    xyz = np.zeros((n, 3))
    blocks, perm = hm.plan_host(xyz, 4, 2.0)
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert (blocks[:, 0] == 0).all()
    cover = np.zeros((2 * n, 2 * n), dtype=np.int16)
    for typ, r0, nr, c0, nc in blocks:
        cover[r0:r0 + nr, c0:c0 + nc] += 1
    assert (cover == 1).all()


def test_collinear_points_split_along_the_line():
    xyz = np.stack([np.linspace(0, 10, 200), np.zeros(200), np.zeros(200)], 1)
    blocks, perm = hm.plan_host(xyz, 16, 2.0)
    # bisection along x keeps the order of the line (up to the tie rule)
    assert np.array_equal(perm, np.arange(200))
    assert (blocks[:, 0] == 1).any()


@pytest.mark.parametrize("dof", [2, 4])
def test_batch_planner_separates_bodies(dof):
    # a batch of independent bodies (hm_plan_bodies_host): the leaves still tile the matrix
    # exactly once; a block whose rows and columns lie on different bodies is a zero block
    # (type 2) and every other leaf lies on one body; clusters hold at most n_leaf unknowns
    wl = workloads.workload("batch_spheroids3")
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    xyz = o.node_table()[:, :3]
    sizes = [6 * m * m * wl["nc"] ** 2 for m in wl["ms"]]
    node_body = np.repeat(np.arange(len(sizes)), sizes)
    assert node_body.size == xyz.shape[0]
    blocks, perm = hm.plan_bodies_host(xyz, node_body, wl["leaf"], wl["eta"], dof)
    n = xyz.shape[0]
    N = dof * n
    assert np.array_equal(np.sort(perm), np.arange(n))
    tree_body = np.repeat(node_body[perm], dof)  # body of each tree-ordered unknown
    cover = np.zeros((N, N), dtype=np.int16)
    zero = 0
    for typ, r0, nr, c0, nc in blocks:
        cover[r0:r0 + nr, c0:c0 + nc] += 1
        rb, cb = np.unique(tree_body[r0:r0 + nr]), np.unique(tree_body[c0:c0 + nc])
        if np.intersect1d(rb, cb).size == 0:
            assert typ == 2
            zero += 1
        else:
            assert typ in (0, 1) and len(rb) == 1 and len(cb) == 1 and rb[0] == cb[0]
            if typ == 0:
                assert nr <= wl["leaf"] or nc <= wl["leaf"]
    assert np.all(cover == 1)
    assert zero >= len(sizes) - 1
    # the nodes of each body stay together in tree order
    assert np.all(np.diff(node_body[perm]) >= 0)


def test_batch_planner_rejects_unsorted_bodies():
    xyz = np.random.default_rng(0).standard_normal((40, 3))
    with pytest.raises(hm.HmError):
        hm.plan_bodies_host(xyz, np.array([1] * 20 + [0] * 20), 8, 2.0)

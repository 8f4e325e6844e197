"""Parity of the CUDA path (through the C-ABI) with the CPU oracle on the same seeded inputs.

Tolerances:
  * node geometry: 1e-12 absolute (same formulas, different code and libm);
  * self/near weights: 2e-8 of the block's largest weight (the two independent
    quadratures converge to ~1e-9; the floor is cancellation in r_i - r');
  * far entries and dense leaves: 1e-12 relative to the row scale;
  * ACA blocks: |A_b - U V^H|_F <= 10 tol |A_b|_F against the oracle's dense block;
  * solution: relative error and relative residual <= 1e-5 at ACA tolerance 1e-7.
"""
import numpy as np
import pytest

import oracle
from paper_2408_17116_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2408_17116_gb300 import build, hm  # noqa: E402

build.build()


def make_solver(wl, keep_matrix=False, **over):
    s = hm.Solver()
    prm = dict(leaf=wl["leaf"], eta=wl["eta"], aca_tol=wl["aca_tol"])
    prm.update(over)
    s.hm_build_geometry(wl["bodies"], wl["ms"], wl["nc"], wl["k"], keep_matrix=keep_matrix, **prm)
    return s


_cache = {}


def oracle_for(name):
    if name not in _cache:
        wl = workloads.workload(name)
        o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
        b = o.rhs(wl["kdirs"], wl["pols"])
        x, A = o.solve_dense(b)
        _cache[name] = (wl, o, A, b, x)
    return _cache[name]


SMALL = ["sphere_d1_m1_nc8", "sphere_d2_m2_nc6", "ellipsoid_small"]


@pytest.mark.parametrize("name", SMALL)
def test_node_geometry(name):
    wl = workloads.workload(name)
    s = make_solver(wl)
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    T = o.node_table()
    G = s.nodes()
    assert np.max(np.abs(G[:, :12] - T[:, :12])) < 1e-12
    assert np.max(np.abs(G[:, 12] - T[:, 12])) < 1e-12
    assert np.max(np.abs(G[:, 13] - T[:, 13])) < 1e-14
    # near pairs: identical sets
    F = o.near_flags()
    pairs = s.near_pairs()
    assert len(pairs) == F.sum()
    assert F[pairs[:, 0], pairs[:, 1]].all()


@pytest.mark.parametrize("name", SMALL)
def test_near_blocks(name):
    wl = workloads.workload(name)
    s = make_solver(wl)
    s.hm_fill()
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    pairs = s.near_pairs()
    rng = np.random.default_rng(3)
    nc2 = wl["nc"] ** 2
    pick = rng.choice(len(pairs), min(12, len(pairs)), replace=False)
    worst = 0.0
    for i in pick:
        q, p = pairs[i]
        for tl in (0, nc2 - 1, int(rng.integers(nc2))):
            tn = q * nc2 + tl
            ref = o.near_block(tn, p)
            got = s.near_block(tn, p)
            worst = max(worst, np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert worst < 2e-8, worst


@pytest.mark.parametrize("name", SMALL)
def test_entries_rows(name):
    wl, o, A, b, x = oracle_for(name)
    s = make_solver(wl)
    s.hm_fill()
    rng = np.random.default_rng(4)
    rows = rng.choice(o.N, 6, replace=False)
    for r in rows:
        cols = np.arange(o.N)
        got = s.entries(np.full(o.N, r), cols)
        ref = A[r, :]
        assert np.max(np.abs(got - ref)) <= 2e-8 * np.max(np.abs(ref))


# Low-rank leaves each workload must produce after ACA (a floor, not the count): the
# 1-wavelength sphere at leaf 64 has admissible blocks whose ACA all reach the rank bound
# of a 64 x 64 block (32), so every one of them ends up dense; the others compress.
MIN_LOWRANK = {"sphere_d1_m1_nc8": 0, "sphere_d2_m2_nc6": 1, "ellipsoid_small": 1, "sphere_d4_m2_nc10": 100}


@pytest.mark.parametrize("name", SMALL + ["sphere_d4_m2_nc10"])
def test_leaf_blocks_against_dense(name):
    wl, o, A, b, x = oracle_for(name)
    s = make_solver(wl)
    s.hm_fill()
    perm = s.perm()
    Ap = A[np.ix_(perm, perm)]
    blocks = s.blocks()
    lowrank = blocks[:, 0] == 1
    assert lowrank.sum() >= MIN_LOWRANK[name], (name, int(lowrank.sum()), len(blocks))
    assert (blocks[lowrank, 5] >= 1).all()
    # every (row, col) pair is covered exactly once by the leaves
    cover = np.zeros((o.N, o.N), dtype=np.int8)
    nchecked = 0
    for i, (typ, r0, nr, c0, ncol, k) in enumerate(blocks):
        cover[r0:r0 + nr, c0:c0 + ncol] += 1
        ref = Ap[r0:r0 + nr, c0:c0 + ncol]
        got = s.block_dense(i)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        if typ == 0:
            assert err < 2e-8, (i, err)
        else:
            assert err <= 10 * wl["aca_tol"], (i, err, k)
            assert k <= nr * ncol / (nr + ncol)
            nchecked += 1
    assert nchecked == lowrank.sum()
    assert (cover == 1).all()


@pytest.mark.parametrize("name", SMALL)
def test_solution_against_dense_oracle(name):
    wl, o, A, b, xo = oracle_for(name)
    s = make_solver(wl)
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    for r in range(x.shape[0]):
        err = np.linalg.norm(x[r] - xo[r]) / np.linalg.norm(xo[r])
        res = np.linalg.norm(A @ x[r] - b[r]) / np.linalg.norm(b[r])
        assert err <= 1e-5, (r, err)
        assert res <= 1e-5, (r, res)
    # host-buffer entry point gives the same numbers
    xh = s.hm_solve_host(wl["kdirs"], wl["pols"])
    assert np.array_equal(xh, x)


def test_rcs_and_currents_against_oracle_and_mie():
    from oracle import mie
    wl, o, A, b, xo = oracle_for("sphere_d1_m1_nc8")
    s = make_solver(wl)
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"])
    th, dirs = workloads.rcs_cuts()
    efar, rcs = s.hm_farfield(x, dirs)
    _, rcs_o = o.farfield(xo[0], dirs)
    assert np.linalg.norm(rcs[0] - rcs_o) / np.linalg.norm(rcs_o) < 1e-5
    ref = np.concatenate([mie.pec_rcs(wl["k"], wl["radius"], th, 0.0), mie.pec_rcs(wl["k"], wl["radius"], th, np.pi / 2)])
    assert np.linalg.norm(rcs[0] - ref) / np.linalg.norm(ref) < 1e-3


def test_matvec_against_dense_oracle():
    wl, o, A, b, xo = oracle_for("sphere_d2_m2_nc6")
    s = make_solver(wl, keep_matrix=True)
    s.hm_fill()
    rng = np.random.default_rng(9)
    xr = rng.standard_normal((2, o.N)) + 1j * rng.standard_normal((2, o.N))
    y = s.hm_matvec(torch.tensor(xr, device="cuda")).cpu().numpy()
    ref = xr @ A.T
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-6
    s.hm_factor()  # keep_matrix: the unfactored copy still serves hm_matvec
    y2 = s.hm_matvec(torch.tensor(xr, device="cuda")).cpu().numpy()
    assert np.linalg.norm(y2 - ref) / np.linalg.norm(ref) < 1e-6


MID = {  # precision, factor_leaf, simt_gemm
    "fp64": (hm.HM_FP64, 640, False),          # H-LU, dense blocks from 600-unknown clusters down
    "fp64-dense": (hm.HM_FP64, 4800, False),   # one dense block, split into a group of 3 row tiles
    "fp32r": (hm.HM_FP32_REFINED, 0, False),   # adaptive: one dense block, tensor-core LU, 2 row tiles
    "fp32r-h": (hm.HM_FP32_REFINED, 640, False),  # H-LU above 600-unknown dense blocks, tensor-core products
    "fp64-adaptive": (hm.HM_FP64, 0, False),   # adaptive: the whole matrix as one dense block
    "fp32r-simt": (hm.HM_FP32_REFINED, 0, True),  # CUDA-core products only, adaptive dense level
    "fp32r-fine": (hm.HM_FP32_REFINED, -1, False),  # the fill's leaves (leaf-level formatted arithmetic)
}


@pytest.mark.parametrize("precision", list(MID))
def test_mid_size_solution_against_dense_oracle(precision):
    # 4,800 unknowns (4-wavelength sphere, leaf 128): hundreds of low-rank leaves, so the
    # H-LU's formatted products and recompressions are exercised, in both precisions, and
    # the merged dense factor in both (grouped row tiles in the substitution)
    wl, o, A, b, xo = oracle_for("sphere_d4_m2_nc10")
    prec, fleaf, simt = MID[precision]
    s = make_solver(wl, precision=prec, factor_leaf=fleaf, simt_gemm=simt)
    s.hm_fill()
    assert s.hm_query("LR_BLOCKS") >= MIN_LOWRANK["sphere_d4_m2_nc10"]
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    for r in range(x.shape[0]):
        err = np.linalg.norm(x[r] - xo[r]) / np.linalg.norm(xo[r])
        res = np.linalg.norm(A @ x[r] - b[r]) / np.linalg.norm(b[r])
        assert err <= 1e-5, (precision, r, err)
        assert res <= 1e-5, (precision, r, res)


def test_no_admissible_blocks_reduces_to_block_dense_lu():
    # eta -> 0: every leaf is dense, so the H-LU is an exact block LU
    wl, o, A, b, xo = oracle_for("sphere_d2_m2_nc6")
    s = make_solver(wl, eta=1e-9)
    s.hm_fill()
    assert (s.blocks()[:, 0] == 0).all()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-10


def test_error_codes_and_call_order():
    wl = workloads.workload("sphere_d1_m1_nc8")
    s = hm.Solver()
    with pytest.raises(hm.HmError) as e:
        s.hm_fill()
    assert e.value.status == 2
    with pytest.raises(hm.HmError) as e:
        s.hm_build_geometry(wl["bodies"], wl["ms"], 1, wl["k"], 64, 2.0, 1e-7)
    assert e.value.status == 1
    s.hm_build_geometry(wl["bodies"], wl["ms"], wl["nc"], wl["k"], 64, 2.0, 1e-7)
    with pytest.raises(hm.HmError) as e:
        s.hm_solve(wl["kdirs"], wl["pols"])
    assert e.value.status == 2
    with pytest.raises(hm.HmError) as e:
        s.hm_query(99)
    assert e.value.status == 1


@pytest.mark.parametrize("factor_leaf", [0, -1])
@pytest.mark.parametrize("name", SMALL)
def test_fp32_factor_with_fp64_refinement_against_dense_oracle(name, factor_leaf):
    # FP32 H-LU as a preconditioner, FP64 refinement against the FP64 H-matrix; factor_leaf 0:
    # adaptive (at these sizes the whole matrix fits as one dense block), -1: the fill's
    # block structure (leaf-level formatted arithmetic in FP32)
    wl, o, A, b, xo = oracle_for(name)
    s = make_solver(wl, precision=hm.HM_FP32_REFINED, factor_leaf=factor_leaf)
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    assert s.hm_query("REFINE_RES") <= 1e-10
    assert 1 <= s.hm_query("REFINE_ITERS") <= 30
    assert s.hm_query("STORAGE32") > 0
    for r in range(x.shape[0]):
        err = np.linalg.norm(x[r] - xo[r]) / np.linalg.norm(xo[r])
        res = np.linalg.norm(A @ x[r] - b[r]) / np.linalg.norm(b[r])
        assert err <= 1e-5, (r, err)
        assert res <= 1e-5, (r, res)
    # the FP64 H-matrix is still available for products after the FP32 factor
    y = s.hm_matvec(torch.tensor(x, device="cuda")).cpu().numpy()
    assert np.linalg.norm(y - x @ A.T) / np.linalg.norm(x @ A.T) < 1e-6


def test_fp32_refinement_reports_non_convergence():
    # a step limit of one cannot reach a 1e-14 residual: the call reports it
    wl, o, A, b, xo = oracle_for("sphere_d1_m1_nc8")
    s = make_solver(wl, precision=hm.HM_FP32_REFINED, refine_tol=1e-14, refine_max_iter=1)
    s.hm_fill()
    s.hm_factor()
    with pytest.raises(hm.HmError) as e:
        s.hm_solve(wl["kdirs"], wl["pols"])
    assert e.value.status == 6
    assert s.hm_query("REFINE_ITERS") == 1


def test_full_size_fp32_refined_against_stored_dense_solution():
    # 19,200 unknowns (8-wavelength sphere, the benchmark workload) against the dense
    # oracle's solution, stored by tests/golden/make_dense_solution.py (oracle fill + dense LU)
    import json
    import os
    name = "sphere_d8_m4_nc10"
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + "_x")
    xo = np.load(gold + ".npy")
    meta = json.load(open(gold + ".json"))
    wl = workloads.workload(name)
    s = make_solver(wl, precision=hm.HM_FP32_REFINED)
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    assert s.hm_query("REFINE_RES") <= 1e-10
    assert x.shape == xo.shape
    for r in range(x.shape[0]):
        err = np.linalg.norm(x[r] - xo[r]) / np.linalg.norm(xo[r])
        assert err <= 1e-5, (r, err)
        # full residual through |A x - b| <= |A|_2 |x - x_o| + |A x_o - b|, with |A|_2 of the
        # oracle's matrix from power iteration (converged to 1e-9; sqrt(|A|_1 |A|_inf), a
        # rigorous but loose bound, is reported beside it)
        bound = meta["norm2_power"] * np.linalg.norm(x[r] - xo[r]) / meta["bnorm"][r] + meta["residual"][r]
        assert bound <= 1e-5, (r, bound, meta["norm2_bound"])
        # element by element: the metric's bar is the relative 2-norm above; no single
        # unknown may deviate by more than 1e-4 of the largest one (a local error would show
        # here first; measured 1.7e-5 at ACA tolerance 1e-7)
        assert np.max(np.abs(x[r] - xo[r])) <= 1e-4 * np.max(np.abs(xo[r])), r


def test_full_size_fp32_refined_sampled_residual():
    wl = workloads.workload("sphere_d8_m4_nc10")
    s = make_solver(wl, precision=hm.HM_FP32_REFINED)
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    assert s.hm_query("REFINE_RES") <= 1e-10
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], wl["k"])
    b = o.rhs(wl["kdirs"], wl["pols"])
    rng = np.random.default_rng(12)
    rows = rng.choice(o.N, 48, replace=False)
    R = o.matrix_rows(rows)
    for r in range(x.shape[0]):
        res = R @ x[r] - b[r][rows]
        assert np.linalg.norm(res) / np.linalg.norm(b[r][rows]) <= 1e-5

"""A batch of independent scatterers in one handle (hm_params.independent): one fill,
factor and solve for all bodies, each body scattering the incident waves alone.

Checks:
  * structure: every block whose rows and columns lie on different bodies is an
    identically zero block (no ACA), every other leaf lies on one body, and the factor
    stores each body's diagonal block dense (DENSE_LEVEL = -2);
  * each body's part of the batched solution equals the solution of that body alone
    (its own handle) to the ACA tolerance, in both precisions;
  * the smallest body against the dense oracle of that body alone: relative error and
    residual <= 1e-5 (the solution bar of the single-body tests).
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

WL = workloads.workload("batch_spheroids3")


def body_ranges(ms, nc, dof=2):
    sizes = [dof * 6 * m * m * nc * nc for m in ms]
    starts = np.concatenate([[0], np.cumsum(sizes)])
    return [(int(starts[i]), int(starts[i + 1])) for i in range(len(ms))]


def solve(bodies, ms, precision, independent):
    s = hm.Solver()
    s.hm_build_geometry(bodies, ms, WL["nc"], WL["k"], WL["leaf"], WL["eta"], WL["aca_tol"], precision=precision,
                        independent=independent)
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(WL["kdirs"], WL["pols"]).cpu().numpy()
    return s, x


def test_batch_structure_zero_blocks_and_pure_leaves():
    s = hm.Solver()
    s.hm_build_geometry(WL["bodies"], WL["ms"], WL["nc"], WL["k"], WL["leaf"], WL["eta"], WL["aca_tol"],
                        independent=True)
    s.hm_fill()
    rng = body_ranges(WL["ms"], WL["nc"])
    body_of = np.empty(s.N, dtype=np.int64)
    for b, (a, e) in enumerate(rng):
        body_of[a:e] = b
    tree_body = body_of[s.perm()]  # tree-ordered unknown -> body
    blocks = s.blocks()             # (type, r0, nr, c0, ncol, rank)
    zero = 0
    for typ, r0, nr, c0, nc, k in blocks:
        rb, cb = np.unique(tree_body[r0:r0 + nr]), np.unique(tree_body[c0:c0 + nc])
        if np.intersect1d(rb, cb).size == 0:
            # rows and columns on different bodies (above the body level several bodies each)
            assert typ == 1 and k == 0, "a block between bodies must be a zero block"
            zero += 1
        else:
            assert len(rb) == 1 and len(cb) == 1 and rb[0] == cb[0], "a leaf mixes bodies"
    assert zero > 0
    assert s.hm_query("LR_BLOCKS") > 0  # within-body admissible blocks still compressed
    s.hm_factor()
    assert s.hm_query("DENSE_LEVEL") == -2


@pytest.mark.parametrize("precision", [hm.HM_FP64, hm.HM_FP32_REFINED])
def test_batch_solution_equals_each_body_alone(precision):
    _, x = solve(WL["bodies"], WL["ms"], precision, True)
    for b, (a, e) in enumerate(body_ranges(WL["ms"], WL["nc"])):
        _, xb = solve(WL["bodies"][b:b + 1], [WL["ms"][b]], precision, False)
        err = np.linalg.norm(x[:, a:e] - xb) / np.linalg.norm(xb)
        assert err <= 1e-6, (b, err)


def test_smallest_body_of_the_batch_against_dense_oracle():
    _, x = solve(WL["bodies"], WL["ms"], hm.HM_FP32_REFINED, True)
    b = int(np.argmin(WL["ms"]))
    a, e = body_ranges(WL["ms"], WL["nc"])[b]
    o = oracle.Oracle(WL["bodies"][b:b + 1], [WL["ms"][b]], WL["nc"], WL["k"])
    rhs = o.rhs(WL["kdirs"], WL["pols"])
    xo, A = o.solve_dense(rhs)
    for r in range(rhs.shape[0]):
        err = np.linalg.norm(x[r, a:e] - xo[r]) / np.linalg.norm(xo[r])
        res = np.linalg.norm(A @ x[r, a:e] - rhs[r]) / np.linalg.norm(rhs[r])
        assert err <= 1e-5, (r, err)
        assert res <= 1e-5, (r, res)

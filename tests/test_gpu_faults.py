"""Error paths of the C-ABI, driven by host-side injection (no GPU fault, trap or hang).

Each injected fault must come back as its status code, and the handle must stay usable:
  * a zero pivot in a diagonal leaf -> HM_ERR_SINGULAR (H-LU, both precisions);
  * a NaN in the right-hand side -> HM_ERR_NUMERIC (scan of the solution);
  * a failed device allocation -> HM_ERR_OOM;
  * non-finite or out-of-range inputs, out-of-range material parameters and formulations
    this library was built without (the CFIE) -> HM_ERR_ARG before any device work.
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

ARG, OOM, SINGULAR, NUMERIC = 1, 4, 5, 8


def solver(wl, **over):
    s = hm.Solver()
    s.hm_build_geometry(wl["bodies"], wl["ms"], wl["nc"], wl["k"], wl["leaf"], wl["eta"], wl["aca_tol"], **over)
    return s


@pytest.mark.parametrize("precision", [hm.HM_FP64, hm.HM_FP32_REFINED])
def test_zero_pivot_reports_singular_and_handle_recovers(precision):
    wl = workloads.workload("sphere_d1_m1_nc8")
    s = solver(wl, precision=precision)
    s.hm_fill()
    s.hm_inject_fault("ZERO_PIVOT")
    with pytest.raises(hm.HmError) as e:
        s.hm_factor()
    assert e.value.status == SINGULAR
    # a fresh fill and factor on the same handle succeed
    s.hm_fill()
    s.hm_factor()
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    assert np.all(np.isfinite(x))


@pytest.mark.parametrize("precision", [hm.HM_FP64, hm.HM_FP32_REFINED])
def test_nan_rhs_reports_numeric(precision):
    wl = workloads.workload("sphere_d1_m1_nc8")
    s = solver(wl, precision=precision)
    s.hm_fill()
    s.hm_factor()
    s.hm_inject_fault("NAN_RHS")
    with pytest.raises(hm.HmError) as e:
        s.hm_solve(wl["kdirs"], wl["pols"])
    assert e.value.status == NUMERIC
    # the next solve (fault disarmed) is clean
    x = s.hm_solve(wl["kdirs"], wl["pols"]).cpu().numpy()
    assert np.all(np.isfinite(x))


def test_allocation_failure_reports_oom():
    wl = workloads.workload("sphere_d1_m1_nc8")
    s = solver(wl)
    s.hm_inject_fault("ALLOC")
    with pytest.raises(hm.HmError) as e:
        s.hm_fill()
    assert e.value.status == OOM
    s.hm_fill()
    s.hm_factor()


def test_bad_inputs_are_rejected_before_device_work():
    wl = workloads.workload("sphere_d1_m1_nc8")
    s = hm.Solver()
    bad = np.array(wl["bodies"], copy=True)
    bad[0, 0] = np.nan  # centre
    cases = [dict(bodies=bad), dict(formulation=hm.HM_PEC_CFIE + 7), dict(formulation=hm.HM_PEC_CFIE),
             dict(formulation=hm.HM_DIEL_MULLER, eps_r=-1.0), dict(formulation=hm.HM_DIEL_MULLER, eps_r=2.0, mu_r=2.0),
             dict(quad_order=2), dict(quad_order=40),
             dict(trunc_tol=-1.0), dict(k0=np.inf)]
    for c in cases:
        w = dict(wl)
        over = {k: v for k, v in c.items() if k not in ("bodies", "k0")}
        with pytest.raises(hm.HmError) as e:
            s.hm_build_geometry(c.get("bodies", w["bodies"]), w["ms"], w["nc"], c.get("k0", w["k"]), w["leaf"],
                                w["eta"], w["aca_tol"], **over)
        assert e.value.status == ARG, c
    with pytest.raises(hm.HmError) as e:
        s.hm_inject_fault(99)
    assert e.value.status == ARG


def test_quadrature_order_parameter_changes_the_near_rule_only_slightly():
    # quad_order sets the Gauss points of the self/near rule: a finer rule moves the near
    # weights by no more than the rule's own error (converged to ~1e-9 at the default)
    wl = workloads.workload("sphere_d1_m1_nc8")
    a = solver(wl)
    a.hm_fill()
    b = solver(wl, quad_order=32)
    b.hm_fill()
    assert b.hm_query("NEAR_QPOINTS") > a.hm_query("NEAR_QPOINTS")
    pairs = a.near_pairs()
    other = [tuple(x) for x in pairs if x[0] != x[1]][:2]
    assert other
    for q, p in [(0, 0)] + other:
        tn = q * wl["nc"] ** 2 + 5
        wa, wb = a.near_block(tn, p), b.near_block(tn, p)
        assert np.max(np.abs(wa - wb)) <= 1e-8 * np.max(np.abs(wb))

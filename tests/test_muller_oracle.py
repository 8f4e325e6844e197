"""Pins of the N-Mueller oracle (oracle.MullerOracle; Sec. II.A, Eqs. 7-9): with
eps_r = 1 every kernel term cancels and the solution is the incident field's
equivalent currents; the dense solution converges spectrally to the dielectric Mie
series (surface currents J, M and the bistatic RCS); the self/near integrals are
converged in the integrator's quadrature orders; and the discrete solutions of both
oracles (MFIE and N-Mueller) satisfy the optical theorem."""
import numpy as np
import pytest

import oracle
from oracle import mie
from paper_2408_17116_gb300 import workloads

K = 2 * np.pi


def _sphere(radius, ms, nc, eps):
    return oracle.MullerOracle(workloads.body(semi=(radius,) * 3)[None], [ms], nc, K, eps)


def _solve(o):
    kh, po = workloads.axial_incidence()
    b = o.rhs(kh, po)
    return np.linalg.solve(o.dense(), b[0])


def test_unit_permittivity_gives_the_incident_currents():
    o = _sphere(0.5, 1, 6, 1.0)
    x = _solve(o)
    J, M = o.currents(x)
    T = o.node_table()
    r, n = T[:, :3], T[:, 9:12]
    ph = np.exp(-1j * K * r[:, 2])
    E = np.outer(ph, [1.0, 0, 0])
    H = np.outer(ph, [0, 1.0, 0]) / oracle.ETA0
    assert np.linalg.norm(J - np.cross(n, H)) <= 1e-12 * np.linalg.norm(np.cross(n, H))
    assert np.linalg.norm(M - np.cross(E, n)) <= 1e-12 * np.linalg.norm(np.cross(E, n))


def _errors(o, radius, eps):
    x = _solve(o)
    J, M = o.currents(x)
    T = o.node_table()
    r = T[:, :3]
    th = np.arccos(np.clip(r[:, 2] / radius, -1, 1))
    ph = np.arctan2(r[:, 1], r[:, 0])
    m = np.sqrt(eps)
    ref = [mie.dielectric_surface_currents(K, radius, m, a, p, oracle.ETA0) for a, p in zip(th, ph)]
    Jm = np.array([c[0] for c in ref])
    Mm = np.array([c[1] for c in ref])
    w = T[:, 12] * T[:, 13]

    def err(a, b):
        return np.sqrt(np.sum(w * np.sum(np.abs(a - b) ** 2, 1)) / np.sum(w * np.sum(np.abs(b) ** 2, 1)))

    th2, dirs = workloads.rcs_cuts(91)
    _, rcs = o.farfield(x, dirs)
    rr = np.concatenate([mie.dielectric_rcs(K, radius, m, th2, 0.0), mie.dielectric_rcs(K, radius, m, th2, np.pi / 2)])
    return err(J, Jm), err(M, Mm), np.linalg.norm(rcs - rr) / np.linalg.norm(rr)


def test_dielectric_sphere_converges_to_mie():
    e6 = _errors(_sphere(0.25, 1, 6, 2.25), 0.25, 2.25)
    e8 = _errors(_sphere(0.25, 1, 8, 2.25), 0.25, 2.25)
    assert max(e8) < 2e-5, e8
    assert all(b < 0.1 * a for a, b in zip(e6, e8)), (e6, e8)


def test_high_contrast_sphere_against_mie():
    eJ, eM, eR = _errors(_sphere(0.25, 1, 8, 10.0), 0.25, 10.0)
    assert max(eJ, eM, eR) < 2e-4, (eJ, eM, eR)


def test_near_integrals_converged_in_quadrature_order():
    # self (interior and corner nodes) and neighbour patches: the adaptive integrator at
    # its default orders against markedly higher orders
    b = workloads.body(semi=(0.5,) * 3)[None]
    lo = oracle.MullerOracle(b, [1], 8, K, 4.0)
    hi = oracle.MullerOracle(b, [1], 8, K, 4.0, q=20, qd=32)
    for tn, p in [(27, 0), (0, 0), (27, 2), (63, 1)]:
        a, c = lo.near_block(tn, p), hi.near_block(tn, p)
        assert np.max(np.abs(a - c)) <= 1e-8 * np.max(np.abs(c)), (tn, p)


def _sphere_directions(nmu=24, nph=48):
    mu, wmu = np.polynomial.legendre.leggauss(nmu)
    ph = 2 * np.pi * np.arange(nph) / nph
    st = np.sqrt(1 - mu * mu)
    dirs = np.stack([np.outer(st, np.cos(ph)).ravel(), np.outer(st, np.sin(ph)).ravel(), np.repeat(mu, nph)], 1)
    return dirs, np.repeat(wmu, nph) * 2 * np.pi / nph


@pytest.mark.parametrize("kind", ["pec_mfie", "dielectric_muller"])
def test_optical_theorem_of_the_discrete_solution(kind):
    # lossless scatterers: the power scattered over all directions equals the power the
    # forward amplitude removes from the incident wave (exp(j w t): sigma_ext =
    # -(4 pi / k) Im(pol . E_far(khat))); both equal the Mie cross section
    kh, po = workloads.axial_incidence()
    if kind == "pec_mfie":
        wl = workloads.workload("sphere_d1_m1_nc8")
        o = oracle.Oracle(wl["bodies"], wl["ms"], 8, K)
        x = o.solve_dense(o.rhs(kh, po))[0][0]
        ref = mie.pec_cross_sections(K, wl["radius"])[0]
    else:
        o = _sphere(0.25, 1, 8, 2.25)
        x = _solve(o)
        ref = mie.dielectric_cross_sections(K, 0.25, 1.5)[0]
    dirs, w = _sphere_directions()
    ef, _ = o.farfield(x, dirs)
    sca = np.sum(w * np.sum(np.abs(ef) ** 2, 1))
    ef0, _ = o.farfield(x, kh)
    ext = -(4 * np.pi / K) * np.imag(ef0[0] @ po[0])
    assert abs(sca - ext) < 1e-4 * sca, (sca, ext)
    assert abs(sca - ref) < 1e-4 * ref and abs(ext - ref) < 1e-4 * ref, (sca, ext, ref)

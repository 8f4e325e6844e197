"""Pins of the dielectric-sphere Mie series (oracle/mie.py), the closed form for the
N-Mueller formulation (Sec. II.A, Eqs. 7-9; Sec. IV.B): no scatterer at m = 1,
energy conservation of a lossless sphere, the Rayleigh limit, the conducting limit of
a strongly absorbing sphere, and tangential continuity of E and H across the surface
between the exterior (incident + scattered) and interior expansions."""
import numpy as np
import pytest

from oracle import mie


def test_index_one_scatters_nothing():
    a, b = mie.dielectric_coefficients(2.0, 1.0)
    assert np.max(np.abs(a)) < 1e-13 and np.max(np.abs(b)) < 1e-13


@pytest.mark.parametrize("x,m", [(np.pi, 2.0), (1.0, np.sqrt(80.0)), (5.0, 1.3)])
def test_lossless_sphere_conserves_energy(x, m):
    a, b = mie.dielectric_coefficients(x, m)
    # each partial wave is lossless: Re(c) = |c|^2
    assert np.max(np.abs(np.real(a) - np.abs(a) ** 2)) < 1e-12
    assert np.max(np.abs(np.real(b) - np.abs(b) ** 2)) < 1e-12
    sca, ext = mie.dielectric_cross_sections(x, 1.0, m)
    assert abs(sca - ext) < 1e-12 * ext


def test_rayleigh_limit():
    k, a, m = 2 * np.pi, 0.002, 1.5
    sca, _ = mie.dielectric_cross_sections(k, a, m)
    ray = 8 * np.pi / 3 * k ** 4 * a ** 6 * abs((m * m - 1) / (m * m + 2)) ** 2
    assert abs(sca - ray) < 1e-3 * ray


def test_strongly_absorbing_sphere_tends_to_pec():
    x = 2.0
    a, b = mie.dielectric_coefficients(x, 3000.0 + 3000.0j)
    ap, bp = mie.pec_coefficients(x, a.size)
    assert np.max(np.abs(a - ap)) < 2e-3 and np.max(np.abs(b - bp)) < 2e-3


@pytest.mark.parametrize("x,m", [(np.pi, 2.0), (np.pi, np.sqrt(80.0))])
def test_tangential_fields_continuous_across_the_surface(x, m):
    k, eta = 2 * np.pi, 376.730313668
    a = x / k
    worst = 0.0
    for th in (0.3, 1.1, 2.0, 2.9):
        for ph in (0.0, 0.7, 2.4):
            Eo, Ho = mie.dielectric_fields_bh(k, a, m, a, th, ph, eta=eta)
            Ei, Hi = mie.dielectric_fields_bh(k, a, m, a, th, ph, eta=eta, part="interior")
            scaleE = np.max(np.abs(Eo))
            scaleH = np.max(np.abs(Ho))
            worst = max(worst, np.max(np.abs(Eo[1:] - Ei[1:])) / scaleE, np.max(np.abs(Ho[1:] - Hi[1:])) / scaleH)
    assert worst < 1e-9, worst


def test_dielectric_rcs_of_absorbing_sphere_tends_to_pec_rcs():
    k, a = 2 * np.pi, 0.5
    th = np.linspace(0.01, np.pi - 0.01, 37)
    r = mie.dielectric_rcs(k, a, 3000.0 + 3000.0j, th, 0.0)
    p = mie.pec_rcs(k, a, th, 0.0)
    assert np.linalg.norm(r - p) < 5e-3 * np.linalg.norm(p)

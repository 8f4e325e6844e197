"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties one oracle routine to something other than itself: exactness of
quadrature rules, closed-form potentials, sphere eigenvalues of the single-layer
operator, the magnetostatic limit of the MFIE, the Mie series, library LU.
"""
import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import scipy.special

import oracle
from oracle import mie
from paper_2408_17116_gb300 import workloads


def sphere(r, center=(0, 0, 0)):
    return workloads.body(center=center, semi=(r, r, r))[None]


# ---------------------------------------------------------------- 1-D rules (Sec. II.B)

@pytest.mark.parametrize("n", [2, 5, 8, 10, 13])
def test_fejer_exact_for_polynomials(n):
    x, w = oracle.cheb_nodes(n), oracle.fejer_weights(n)
    for d in range(n):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) < 1e-14
    # nodes are the first-kind points: T_n vanishes there, none at the endpoints
    assert np.max(np.abs(np.cos(n * np.arccos(x)))) < 1e-13
    assert np.all(np.abs(x) < 1)


@pytest.mark.parametrize("n", [3, 8, 10])
def test_cheb_cardinal_interpolates(n):
    nodes = oracle.cheb_nodes(n)
    for l in range(n):
        ell = oracle.cheb_cardinal(n, nodes[l])
        assert np.allclose(ell, np.eye(n)[l], atol=1e-13)
    # the interpolant of any polynomial of degree < n is exact (Eq. 12 with Eq. 13)
    rng = np.random.default_rng(1)
    c = rng.standard_normal(n)
    for xv in (-0.93, -0.2, 0.41, 0.999):
        ell = oracle.cheb_cardinal(n, xv)
        assert abs(ell @ np.polyval(c, nodes) - np.polyval(c, xv)) < 1e-12


@pytest.mark.parametrize("q", [1, 4, 12, 20])
def test_gauss_legendre_matches_library(q):
    x, w = oracle.gauss_legendre(q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    order = np.argsort(x)
    assert np.allclose(x[order], xr, atol=1e-14) and np.allclose(w[order], wr, atol=1e-14)


# ---------------------------------------------------------------- geometry (Eqs. 11, 14, 17-18)

def test_sphere_nodes_on_surface_and_area():
    o = oracle.Oracle(sphere(0.7), [2], 8, 1.0)
    T = o.node_table()
    r, au, av, n, sg, w = T[:, :3], T[:, 3:6], T[:, 6:9], T[:, 9:12], T[:, 12], T[:, 13]
    assert np.allclose(np.linalg.norm(r, axis=1), 0.7, atol=1e-14)
    assert np.allclose(n, r / 0.7, atol=1e-13)  # outward unit normal
    assert np.allclose(sg, np.linalg.norm(np.cross(au, av), axis=1), atol=1e-14)
    # contravariant vectors of Eq. 18 satisfy the duality of Eq. 17
    aU = np.cross(av, n) / sg[:, None]
    aV = np.cross(n, au) / sg[:, None]
    assert np.allclose(np.einsum("ij,ij->i", aU, au), 1) and np.allclose(np.einsum("ij,ij->i", aU, av), 0, atol=1e-13)
    assert np.allclose(np.einsum("ij,ij->i", aV, av), 1) and np.allclose(np.einsum("ij,ij->i", aV, au), 0, atol=1e-13)
    # Fejer quadrature of the surface Jacobian integrates the area spectrally
    assert abs(np.sum(w * sg) - 4 * np.pi * 0.49) / (4 * np.pi * 0.49) < 1e-7


def test_covariant_basis_is_derivative_of_map():
    wl = workloads.workload("ellipsoid_small")
    o = oracle.Oracle(wl["bodies"], wl["ms"], 6, 1.0)
    h = 1e-6
    for p in (0, 7, 13, 22):
        for (u, v) in ((0.3, -0.7), (-0.95, 0.1)):
            r, ru, rv = o.patch_point(p, u, v)
            assert np.allclose(ru, (o.patch_point(p, u + h, v)[0] - o.patch_point(p, u - h, v)[0]) / (2 * h), atol=1e-8)
            assert np.allclose(rv, (o.patch_point(p, u, v + h)[0] - o.patch_point(p, u, v - h)[0]) / (2 * h), atol=1e-8)


def test_prolate_spheroid_area():
    a, b = 1.5, 0.6  # semi-axes (z major)
    o = oracle.Oracle(workloads.body(semi=(b, b, a))[None], [2], 10, 1.0)
    T = o.node_table()
    e = np.sqrt(1 - b * b / (a * a))
    exact = 2 * np.pi * b * b * (1 + a / (b * e) * np.arcsin(e))
    assert abs(np.sum(T[:, 12] * T[:, 13]) - exact) / exact < 1e-6
    # outward normals point away from the centre on a convex body
    assert np.all(np.einsum("ij,ij->i", T[:, 9:12], T[:, :3]) > 0)


def test_near_flags_cube_sphere():
    o = oracle.Oracle(sphere(0.5), [1], 8, 1.0)
    F = o.near_flags()
    assert (F == F.T).all() and F.diagonal().all()
    # each face touches 4 faces and is far from the opposite one
    assert (F.sum(1) == 5).all()
    for f in range(3):
        assert not F[2 * f, 2 * f + 1]


# ---------------------------------------------------------------- independent self/near integrator

def _rect_inv_r(x1, x2, y1, y2, h):
    """Closed form of the integral of 1/sqrt(X^2+Y^2+h^2) over a rectangle (observer at origin)."""
    def F(X, Y):
        D = np.sqrt(X * X + Y * Y + h * h)
        t = X * np.log(Y + D) + Y * np.log(X + D)
        if h > 0:
            t -= h * np.arctan(X * Y / (h * D))
        return t
    return F(x2, y2) - F(x1, y2) - F(x2, y1) + F(x1, y1)


def test_rect_closed_form_against_library_quadrature():
    val = scipy.integrate.dblquad(lambda y, x: 1 / np.sqrt(x * x + y * y + 0.09), -0.7, 0.5, -0.2, 1.1, epsabs=1e-13)[0]
    assert abs(_rect_inv_r(-0.7, 0.5, -0.2, 1.1, 0.3) - val) < 1e-10


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (0.1, 1.0), (2.0, 0.3)])
def test_planar_self_integral_closed_form(a, b):
    nc = 8
    o = oracle.Oracle(sphere(0.5), [1], nc, 0.0)
    x = oracle.cheb_nodes(nc)
    for (l, k) in ((0, 0), (3, 5), (7, 2)):
        x0, y0 = a * x[l], b * x[k]
        W = o.planar_single_layer(a, b, 0.0, [x0, y0, 0.0], self_node=(l, k))
        exact = _rect_inv_r(-a - x0, a - x0, -b - y0, b - y0, 0.0) / (4 * np.pi)
        assert abs(W.sum() - exact) / exact < 1e-12


@pytest.mark.parametrize("h", [0.3, 0.02, 0.002])
def test_planar_near_integral_closed_form(h):
    o = oracle.Oracle(sphere(0.5), [1], 8, 0.0)
    for (x0, y0) in ((0.2, -0.4), (1.01, 0.3), (1.004, 1.002)):
        W = o.planar_single_layer(1.0, 1.0, 0.0, [x0, y0, h])
        exact = _rect_inv_r(-1 - x0, 1 - x0, -1 - y0, 1 - y0, h) / (4 * np.pi)
        assert abs(W.sum() - exact) / exact < 1e-12


def test_planar_dynamic_weights_against_library_quadrature():
    # each cardinal weight against scipy's adaptive quadrature at an off-patch target
    nc, k = 5, 2 * np.pi
    o = oracle.Oracle(sphere(0.5), [1], nc, k)
    tgt = np.array([0.4, 0.55, 0.35])
    W = o.planar_single_layer(0.6, 0.6, k, tgt)
    x = oracle.cheb_nodes(nc)
    for j in (0, 7, 18):
        l, kk = j % nc, j // nc
        def f(v, u, part):
            ell = oracle.cheb_cardinal(nc, u)[l] * oracle.cheb_cardinal(nc, v)[kk]
            R = np.linalg.norm(tgt - np.array([0.6 * u, 0.6 * v, 0]))
            val = np.exp(-1j * k * R) / (4 * np.pi * R) * 0.36 * ell
            return val.real if part == 0 else val.imag
        re = scipy.integrate.dblquad(f, -1, 1, -1, 1, args=(0,), epsabs=1e-12)[0]
        im = scipy.integrate.dblquad(f, -1, 1, -1, 1, args=(1,), epsabs=1e-12)[0]
        assert abs(W[j] - (re + 1j * im)) < 1e-10
    del x


def test_near_block_converged_in_order():
    wl = workloads.workload("sphere_d1_m1_nc8")
    lo = oracle.Oracle(wl["bodies"], wl["ms"], 8, wl["k"], q=12, qd=20)
    hi = oracle.Oracle(wl["bodies"], wl["ms"], 8, wl["k"], q=16, qd=28)
    for (tn, p) in ((0, 0), (27, 0), (63, 2), (5, 4), (100, 1)):
        if not lo.near_flags()[tn // 64, p]:
            continue
        a, b = lo.near_block(tn, p), hi.near_block(tn, p)
        # floor ~1e-10: cancellation in r_i - r' at the smallest Duffy radii, not quadrature
        assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))


# ---------------------------------------------------------------- operator pins on the sphere

@pytest.mark.parametrize("ka", [0.5, np.pi / 2])
def test_single_layer_sphere_eigenvalues(ka):
    # S[Y_n] = -j k a^2 j_n(ka) h2_n(ka) Y_n for G = exp(-jkR)/(4 pi R)  (Eqs. 3-4)
    a = 0.5
    k = ka / a
    o = oracle.Oracle(sphere(a), [1], 10, k)
    S = o.single_layer_dense()
    T = o.node_table()
    for n, Y in ((0, np.ones(o.nnode)), (1, T[:, 2] / a)):
        h2 = scipy.special.spherical_jn(n, ka) - 1j * scipy.special.spherical_yn(n, ka)
        lam = -1j * k * a * a * scipy.special.spherical_jn(n, ka) * h2
        assert np.max(np.abs(S @ Y - lam * Y)) <= 2e-7 * abs(lam)


def test_mfie_magnetostatic_limit():
    # a perfectly conducting sphere in a uniform field carries J = 3/2 n x H0
    o = oracle.Oracle(sphere(0.5), [1], 8, 1e-4)
    kd, po = np.array([0, 0, 1.0]), np.array([1.0, 0, 0])
    x, _ = o.solve_dense(o.rhs([kd], [po]))
    T = o.node_table()
    J = o.currents(x[0])
    Jref = 1.5 * np.cross(T[:, 9:12], np.cross(kd, po)[None, :] / oracle.ETA0)
    w = T[:, 12] * T[:, 13]
    err = np.sqrt(np.sum(w[:, None] * np.abs(J - Jref) ** 2) / np.sum(w[:, None] * np.abs(Jref) ** 2))
    assert err < 2e-4


def _mie_currents(o, k, a):
    T = o.node_table()
    J = np.array([mie.pec_surface_current(k, a, np.arccos(r[2] / a), np.arctan2(r[1], r[0]), oracle.ETA0)
                  for r in T[:, :3]])
    return T, J


def test_farfield_of_mie_current_matches_mie_rcs():
    # F^a = sqrtG a^a . J (Eq. 11) from the exact current; its far field must give Mie's RCS
    wl = workloads.workload("sphere_d1_m1_nc8")
    a, k = wl["radius"], wl["k"]
    o = oracle.Oracle(wl["bodies"], wl["ms"], 10, k)
    T, J = _mie_currents(o, k, a)
    n, au, av = T[:, 9:12], T[:, 3:6], T[:, 6:9]
    x = np.zeros(o.N, dtype=complex)
    x[0::2] = np.einsum("ij,ij->i", np.cross(av, n), J)
    x[1::2] = np.einsum("ij,ij->i", np.cross(n, au), J)
    th, dirs = workloads.rcs_cuts(91)
    _, rcs = o.farfield(x, dirs)
    ref = np.concatenate([mie.pec_rcs(k, a, th, 0.0), mie.pec_rcs(k, a, th, np.pi / 2)])
    assert np.linalg.norm(rcs - ref) / np.linalg.norm(ref) < 1e-4  # quadrature of the current at 10x10 nodes


def test_mfie_solution_matches_mie():
    wl = workloads.workload("sphere_d1_m1_nc8")
    a, k = wl["radius"], wl["k"]
    o = oracle.Oracle(wl["bodies"], wl["ms"], wl["nc"], k)
    x, _ = o.solve_dense(o.rhs(wl["kdirs"], wl["pols"]))
    T, Jm = _mie_currents(o, k, a)
    J = o.currents(x[0])
    w = T[:, 12] * T[:, 13]
    err = np.sqrt(np.sum(w[:, None] * np.abs(J - Jm) ** 2) / np.sum(w[:, None] * np.abs(Jm) ** 2))
    assert err < 2e-4
    th, dirs = workloads.rcs_cuts()
    _, rcs = o.farfield(x[0], dirs)
    ref = np.concatenate([mie.pec_rcs(k, a, th, 0.0), mie.pec_rcs(k, a, th, np.pi / 2)])
    assert np.linalg.norm(rcs - ref) / np.linalg.norm(ref) < 1e-3


# ---------------------------------------------------------------- dense LU (LAPACK-semantics pivoting)

def test_lu_solve_against_library():
    rng = np.random.default_rng(5)
    n = 57
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    LU, ipiv, info = oracle.zgetrf(A)
    assert info == 0
    X = oracle.zgetrs(LU, ipiv, B)
    assert np.allclose(X, np.linalg.solve(A, B), rtol=1e-11, atol=1e-12)
    # real matrix: modulus and LAPACK's |re|+|im| agree, so the pivots must match getrf
    Ar = rng.standard_normal((n, n))
    _, ip2, _ = oracle.zgetrf(Ar.astype(complex))
    assert (ip2 == scipy.linalg.lu_factor(Ar)[1]).all()


def test_lu_ties_pick_lowest_row():
    A = np.array([[1.0, 2.0], [-1.0, 3.0]], dtype=complex)
    _, ipiv, _ = oracle.zgetrf(A)
    assert ipiv[0] == 0
    _, ipiv, info = oracle.zgetrf(np.zeros((3, 3), complex))
    assert info == 1


# ---------------------------------------------------------------- Mie series pins

def test_spherical_bessel_against_library():
    for x in (0.3, np.pi, 2 * np.pi, 25.13):
        jn, yn = mie.sph_jn_yn(40, x)
        n = np.arange(41)
        assert np.allclose(jn, scipy.special.spherical_jn(n, x), rtol=1e-10, atol=1e-15)
        ok = np.abs(yn) < 1e200
        assert np.allclose(yn[ok], scipy.special.spherical_yn(n, x)[ok], rtol=1e-10)


def test_mie_plane_wave_expansion_and_pec_condition():
    k, a = 2 * np.pi, 0.5
    r, th, ph = 0.9, 1.1, 0.7
    E, H = mie.pec_fields_bh(k, a, r, th, ph, part="incident")
    e = np.exp(1j * k * r * np.cos(th))
    xh = np.array([np.sin(th) * np.cos(ph), np.cos(th) * np.cos(ph), -np.sin(ph)])  # x in (r,th,ph)
    yh = np.array([np.sin(th) * np.sin(ph), np.cos(th) * np.sin(ph), np.cos(ph)])
    assert np.allclose(E, e * xh, atol=1e-12) and np.allclose(H, e * yh, atol=1e-12)
    E, _ = mie.pec_fields_bh(k, a, a, th, ph)
    assert np.max(np.abs(E[1:])) < 1e-12


def test_mie_optical_theorem_and_rayleigh_limit():
    for x in (0.5, np.pi, 25.1):
        k = 2 * np.pi
        a = x / k
        sca, ext = mie.pec_cross_sections(k, a)
        S1, S2 = mie.pec_S1S2(x, 0.0)
        assert abs(S1 - S2) < 1e-12 * abs(S1)
        assert abs(sca - ext) < 1e-10 * ext
        assert abs(ext - 4 * np.pi / k ** 2 * S1.real) < 1e-10 * ext
        # sigma_sca from integrating the bistatic RCS over the sphere
        th = np.linspace(0, np.pi, 2001)
        integrand = [np.trapezoid(mie.pec_rcs(k, a, th, ph) * np.sin(th), th) for ph in np.linspace(0, 2 * np.pi, 65)[:-1]]
        assert abs(np.mean(integrand) * 2 * np.pi / (4 * np.pi) - sca) < 1e-4 * sca
    k, a = 2 * np.pi, 1e-3
    assert abs(mie.pec_rcs(k, a, np.pi, 0.0) / (np.pi * a * a) / (9 * (k * a) ** 4) - 1) < 1e-3


def test_mie_low_frequency_current():
    k, a = 2 * np.pi, 1e-4
    for th, ph in ((0.3, 0.2), (2.1, 4.0)):
        n = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
        J = mie.pec_surface_current(k, a, th, ph, oracle.ETA0)
        Jref = 1.5 * np.cross(n, [0, 1 / oracle.ETA0, 0])
        assert np.linalg.norm(J - Jref) < 1e-3 * np.linalg.norm(Jref)  # O(ka) correction


def test_mfie_converges_spectrally_to_mie_in_the_chebyshev_order():
    # p-refinement on the 1-wavelength sphere: the current error against Mie falls by an
    # order of magnitude or more from Nc = 5 to Nc = 7 to Nc = 9
    wl = workloads.workload("sphere_d1_m1_nc8")
    a, k = wl["radius"], wl["k"]
    errs = []
    for nc in (5, 7, 9):
        o = oracle.Oracle(wl["bodies"], wl["ms"], nc, k)
        x, _ = o.solve_dense(o.rhs(wl["kdirs"], wl["pols"]))
        T, Jm = _mie_currents(o, k, a)
        J = o.currents(x[0])
        w = T[:, 12] * T[:, 13]
        errs.append(np.sqrt(np.sum(w[:, None] * np.abs(J - Jm) ** 2) / np.sum(w[:, None] * np.abs(Jm) ** 2)))
    assert errs[1] < 0.1 * errs[0] and errs[2] < 0.1 * errs[1], errs

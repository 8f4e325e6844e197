"""Mie series for PEC and dielectric spheres -- TEST INFRASTRUCTURE ONLY.

The closed-form anchor the paper itself validates against (Sec. IV.A, Table 1:
density errors against the analytical Mie series).  Written from the textbook
vector-spherical-harmonic expansion of a plane wave scattered by a perfectly
conducting sphere (Bohren & Huffman, Ch. 4, exp(-i w t) convention); results that
depend on the time convention are conjugated to the paper's exp(j w t) convention.

Spherical Bessel functions are computed here by recurrences (j_n downward,
normalised by j_0 = sin x / x; y_n upward), independently of scipy; the tests
check them against scipy.
"""
import numpy as np


def sph_jn_yn(nmax, x):
    """j_n(x), y_n(x) for n = 0..nmax (real x > 0); j_n by Miller's downward recurrence."""
    x = float(x)
    start = int(nmax + 20 + 2 * np.sqrt(nmax + x) + x)
    j = np.zeros(start + 2)
    j[start + 1] = 0.0
    j[start] = 1e-300
    for n in range(start, 0, -1):
        j[n - 1] = (2 * n + 1) / x * j[n] - j[n + 1]
        if abs(j[n - 1]) > 1e250:
            j[n - 1:] *= 1e-250
    # normalise by whichever of the closed forms j_0, j_1 is larger in magnitude
    # (j_0 alone fails where sin x = 0, e.g. x = pi)
    j0 = np.sin(x) / x
    j1 = np.sin(x) / x ** 2 - np.cos(x) / x
    if abs(j0) >= abs(j1):
        jn = j[: nmax + 1] * (j0 / j[0])
    else:
        jn = j[: nmax + 1] * (j1 / j[1])
    yn = np.zeros(nmax + 1)
    yn[0] = -np.cos(x) / x
    if nmax >= 1:
        yn[1] = -np.cos(x) / x ** 2 - np.sin(x) / x
    for n in range(1, nmax):
        yn[n + 1] = (2 * n + 1) / x * yn[n] - yn[n - 1]
    return jn, yn


def nmax_for(x):
    return int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0)) + 10


def riccati(nmax, x):
    """psi_n = x j_n, xi_n = x h1_n and their derivatives, n = 0..nmax."""
    jn, yn = sph_jn_yn(nmax + 1, x)
    h = jn + 1j * yn
    n = np.arange(nmax + 1)
    psi = x * jn[: nmax + 1]
    xi = x * h[: nmax + 1]
    # [x z_n]' = x z_{n-1} - n z_n; for n = 0 use [x z_0]' = x z_0' + z_0 with z_0' = -z_1
    dpsi = np.empty(nmax + 1)
    dxi = np.empty(nmax + 1, dtype=complex)
    dpsi[0] = jn[0] - x * jn[1]
    dxi[0] = h[0] - x * h[1]
    dpsi[1:] = x * jn[: nmax] - n[1:] * jn[1: nmax + 1]
    dxi[1:] = x * h[: nmax] - n[1:] * h[1: nmax + 1]
    return psi, dpsi, xi, dxi, jn[: nmax + 1], h[: nmax + 1]


def pec_coefficients(x, nmax=None):
    """a_n = psi_n'(x)/xi_n'(x), b_n = psi_n(x)/xi_n(x), n = 1..nmax (tangential E = 0 at r = a)."""
    if nmax is None:
        nmax = nmax_for(x)
    psi, dpsi, xi, dxi, _, _ = riccati(nmax, x)
    return dpsi[1:] / dxi[1:], psi[1:] / xi[1:]


def pi_tau(nmax, mu):
    """Angular functions pi_n = P_n^1 / sin(theta), tau_n = dP_n^1/dtheta, n = 1..nmax."""
    mu = np.asarray(mu, dtype=float)
    pi = np.zeros((nmax + 1,) + mu.shape)
    tau = np.zeros((nmax + 1,) + mu.shape)
    pi[1] = 1.0
    tau[1] = mu
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) * mu * pi[n - 1] - n * pi[n - 2]) / (n - 1)
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def pec_S1S2(x, theta, nmax=None):
    if nmax is None:
        nmax = nmax_for(x)
    a, b = pec_coefficients(x, nmax)
    pi, tau = pi_tau(nmax, np.cos(theta))
    n = np.arange(1, nmax + 1)
    c = ((2 * n + 1) / (n * (n + 1)))[:, None] if np.ndim(theta) else (2 * n + 1) / (n * (n + 1))
    if np.ndim(theta):
        S1 = np.sum(c * (a[:, None] * pi + b[:, None] * tau), axis=0)
        S2 = np.sum(c * (a[:, None] * tau + b[:, None] * pi), axis=0)
    else:
        S1 = np.sum(c * (a * pi + b * tau))
        S2 = np.sum(c * (a * tau + b * pi))
    return S1, S2


def pec_rcs(k, radius, theta, phi):
    """Bistatic RCS (m^2) for incidence along +z, x-polarised, unit amplitude:
    sigma = (4 pi / k^2) (|S2|^2 cos^2 phi + |S1|^2 sin^2 phi)."""
    S1, S2 = pec_S1S2(k * radius, theta)
    return 4 * np.pi / k ** 2 * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)


def pec_cross_sections(k, radius):
    """Scattering and extinction cross sections from the coefficients
    (sigma_sca = 2 pi/k^2 sum (2n+1)(|a|^2+|b|^2), sigma_ext = 2 pi/k^2 sum (2n+1) Re(a+b))."""
    x = k * radius
    a, b = pec_coefficients(x)
    n = np.arange(1, a.size + 1)
    sca = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    ext = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    return sca, ext


def _vsh(n_arr, rho, theta, phi, kind):
    """M_e1n, M_o1n, N_e1n, N_o1n as (r, theta, phi) components; kind 1: j_n, kind 3: h1_n."""
    nmax = int(n_arr[-1])
    psi, dpsi, xi, dxi, jn, h = riccati(nmax, rho)
    if kind == 1:
        z, dz = jn[1:], dpsi[1:]
    else:
        z, dz = h[1:], dxi[1:]
    pi, tau = pi_tau(nmax, np.cos(theta))
    st, sp, cp = np.sin(theta), np.sin(phi), np.cos(phi)
    n = n_arr
    zr = z / rho
    dzr = dz / rho
    Me = np.stack([np.zeros(nmax, dtype=complex), -sp * pi * z, -cp * tau * z])
    Mo = np.stack([np.zeros(nmax, dtype=complex), cp * pi * z, -sp * tau * z])
    Ne = np.stack([cp * n * (n + 1) * st * pi * zr, cp * tau * dzr, -sp * pi * dzr])
    No = np.stack([sp * n * (n + 1) * st * pi * zr, sp * tau * dzr, cp * pi * dzr])
    return Me, Mo, Ne, No


def pec_fields_bh(k, radius, r, theta, phi, eta=1.0, part="total"):
    """E and H (spherical components) in the exp(-i w t) convention at (r, theta, phi), r >= radius.
    Incident E = x exp(ikz), H = y exp(ikz) / eta."""
    x = k * radius
    nmax = nmax_for(max(x, k * r))
    a, b = pec_coefficients(x, nmax)
    n = np.arange(1, nmax + 1)
    En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
    rho = k * r
    M1e, M1o, N1e, N1o = _vsh(n, rho, theta, phi, 1)
    M3e, M3o, N3e, N3o = _vsh(n, rho, theta, phi, 3)
    Ei = np.sum(En * (M1o - 1j * N1e), axis=1)
    Hi = -np.sum(En * (M1e + 1j * N1o), axis=1) / eta
    Es = np.sum(En * (1j * a * N3e - b * M3o), axis=1)
    Hs = np.sum(En * (1j * b * N3o + a * M3e), axis=1) / eta
    if part == "incident":
        return Ei, Hi
    if part == "scattered":
        return Es, Hs
    return Ei + Es, Hi + Hs


def pec_surface_current(k, radius, theta, phi, eta):
    """J = n x H_total on r = radius, as a Cartesian vector in the exp(j w t) convention
    (the conjugate of the exp(-i w t) phasor)."""
    _, H = pec_fields_bh(k, radius, radius, theta, phi, eta=eta)
    # n x H with n = r_hat: (r, th, ph) -> J_th = -H_ph, J_ph = H_th
    Jth, Jph = -H[2], H[1]
    th_hat = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])
    ph_hat = np.array([-np.sin(phi), np.cos(phi), 0.0])
    return np.conj(Jth * th_hat + Jph * ph_hat)


# ---------------------------------------------------------------------------
# Dielectric (penetrable, non-magnetic) sphere: the closed form the paper's
# dielectric results are checked against (Sec. IV.B).  Bohren & Huffman, Ch. 4,
# exp(-i w t) convention, relative refractive index m = sqrt(eps_r) of the sphere
# to its surroundings, mu = 1 on both sides.
# ---------------------------------------------------------------------------

def log_derivative(nmax, z):
    """D_n(z) = psi_n'(z) / psi_n(z), n = 0..nmax, by the downward recurrence
    D_{n-1} = n/z - 1/(D_n + n/z) started from zero far above max(nmax, |z|)
    (stable for large |z|, Wiscombe 1980).  z may be complex."""
    z = complex(z)
    nst = int(max(nmax, abs(z)) + 16 + 4.0 * abs(z) ** (1.0 / 3.0))
    D = np.zeros(nst + 1, dtype=complex)
    for n in range(nst, 0, -1):
        D[n - 1] = n / z - 1.0 / (D[n] + n / z)
    return D[: nmax + 1]


def dielectric_coefficients(x, m, nmax=None):
    """Scattering coefficients a_n, b_n, n = 1..nmax, of a sphere of size x = k a and
    relative index m, written with the logarithmic derivative of psi_n(m x):
      a_n = [(D_n/m + n/x) psi_n - psi_{n-1}] / [(D_n/m + n/x) xi_n - xi_{n-1}]
      b_n = [(m D_n + n/x) psi_n - psi_{n-1}] / [(m D_n + n/x) xi_n - xi_{n-1}]."""
    if nmax is None:
        nmax = nmax_for(x)
    psi, dpsi, xi, dxi, _, _ = riccati(nmax, x)
    D = log_derivative(nmax, m * x)[1:]
    n = np.arange(1, nmax + 1)
    ta = D / m + n / x
    tb = m * D + n / x
    a = (ta * psi[1:] - psi[:-1]) / (ta * xi[1:] - xi[:-1])
    b = (tb * psi[1:] - psi[:-1]) / (tb * xi[1:] - xi[:-1])
    return a, b


def dielectric_interior_coefficients(x, m, nmax=None):
    """Interior coefficients c_n, d_n (real m, mu = 1) from the same boundary conditions:
      c_n = (j_n(x) [x h_n(x)]' - h_n(x) [x j_n(x)]') / (j_n(mx) [x h_n(x)]' - h_n(x) [mx j_n(mx)]')
      d_n = m (j_n(x) [x h_n(x)]' - h_n(x) [x j_n(x)]') / (m^2 j_n(mx) [x h_n(x)]' - h_n(x) [mx j_n(mx)]')."""
    if nmax is None:
        nmax = nmax_for(x)
    _, dpsi, _, dxi, jn, h = riccati(nmax, x)
    _, dpsim, _, _, jnm, _ = riccati(nmax, m * x)
    num = jn[1:] * dxi[1:] - h[1:] * dpsi[1:]
    c = num / (jnm[1:] * dxi[1:] - h[1:] * dpsim[1:])
    d = m * num / (m * m * jnm[1:] * dxi[1:] - h[1:] * dpsim[1:])
    return c, d


def dielectric_fields_bh(k, radius, m, r, theta, phi, eta=1.0, part="total"):
    """E and H (spherical components, exp(-i w t)) for incident E = x exp(ikz): outside
    (r >= radius: incident + scattered) or inside (r <= radius, part = "interior")."""
    x = k * radius
    nmax = nmax_for(max(x, k * r))
    n = np.arange(1, nmax + 1)
    En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
    if part == "interior":
        c, d = dielectric_interior_coefficients(x, m, nmax)
        M1e, M1o, N1e, N1o = _vsh(n, m * k * r, theta, phi, 1)
        E = np.sum(En * (c * M1o - 1j * d * N1e), axis=1)
        H = -(m / eta) * np.sum(En * (d * M1e + 1j * c * N1o), axis=1)
        return E, H
    a, b = dielectric_coefficients(x, m, nmax)
    rho = k * r
    M1e, M1o, N1e, N1o = _vsh(n, rho, theta, phi, 1)
    M3e, M3o, N3e, N3o = _vsh(n, rho, theta, phi, 3)
    Ei = np.sum(En * (M1o - 1j * N1e), axis=1)
    Hi = -np.sum(En * (M1e + 1j * N1o), axis=1) / eta
    Es = np.sum(En * (1j * a * N3e - b * M3o), axis=1)
    Hs = np.sum(En * (1j * b * N3o + a * M3e), axis=1) / eta
    if part == "scattered":
        return Es, Hs
    return Ei + Es, Hi + Hs


def dielectric_surface_currents(k, radius, m, theta, phi, eta):
    """J = n x H and M = E x n on the outer side of r = radius, Cartesian vectors in the
    exp(j w t) convention (conjugates of the exp(-i w t) phasors)."""
    E, H = dielectric_fields_bh(k, radius, m, radius, theta, phi, eta=eta)
    th_hat = np.array([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)])
    ph_hat = np.array([-np.sin(phi), np.cos(phi), 0.0])
    J = -H[2] * th_hat + H[1] * ph_hat       # r x (H_th th + H_ph ph)
    M = E[2] * th_hat - E[1] * ph_hat        # (E_th th + E_ph ph) x r
    return np.conj(J), np.conj(M)


def dielectric_rcs(k, radius, m, theta, phi):
    """Bistatic RCS (m^2), incidence along +z, x-polarised, unit amplitude."""
    x = k * radius
    a, b = dielectric_coefficients(x, m)
    nmax = a.size
    pi, tau = pi_tau(nmax, np.cos(theta))
    n = np.arange(1, nmax + 1)
    c = ((2 * n + 1) / (n * (n + 1)))[:, None]
    S1 = np.sum(c * (a[:, None] * pi + b[:, None] * tau), axis=0)
    S2 = np.sum(c * (a[:, None] * tau + b[:, None] * pi), axis=0)
    return 4 * np.pi / k ** 2 * (np.abs(S2) ** 2 * np.cos(phi) ** 2 + np.abs(S1) ** 2 * np.sin(phi) ** 2)


def dielectric_cross_sections(k, radius, m):
    x = k * radius
    a, b = dielectric_coefficients(x, m)
    n = np.arange(1, a.size + 1)
    sca = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    ext = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    return sca, ext

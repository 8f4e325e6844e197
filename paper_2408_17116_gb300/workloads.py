"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark.

This module holds geometry descriptions, parameters and seeded random draws only;
none of the method's arithmetic lives here.  Every body is a cube-mapped
ellipsoid (6 m^2 curvilinear patches, the patch family of the paper's sphere
experiments, Sec. IV: 24..4056 patches = 6 m^2), wavelength 1 m (k = 2 pi).

Random incidence angles use numpy's Philox counter-based generator, the
Philox4x64-10 variant (not Philox4x32-10), seeded with 2408017116:
theta = arccos(1 - 2U), phi = 2 pi U, polarisation = theta-hat.  Every consumer
(library tests, oracle, benchmark) draws them from this module, so both sides of a
parity check see the same angles.
"""
import numpy as np

SEED = 2408017116
WAVELENGTH = 1.0
K0 = 2.0 * np.pi / WAVELENGTH


def body(center=(0.0, 0.0, 0.0), semi=(0.5, 0.5, 0.5), rot=None):
    """15 doubles: center[3], semi-axes[3], rotation[9] (row-major)."""
    R = np.eye(3) if rot is None else np.asarray(rot, dtype=np.float64).reshape(3, 3)
    return np.concatenate([np.asarray(center, float), np.asarray(semi, float), R.reshape(-1)])


def incidence(nrhs, seed=SEED):
    """nrhs seeded plane waves: (khat[nrhs,3], pol[nrhs,3])."""
    g = np.random.Generator(np.random.Philox(seed))
    u = g.random((nrhs, 2))
    th = np.arccos(1.0 - 2.0 * u[:, 0])
    ph = 2.0 * np.pi * u[:, 1]
    kh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    pol = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)
    return kh, pol


def axial_incidence():
    """+z propagation, x polarisation (the paper's excitation, Sec. IV.A)."""
    return np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]])


def rcs_cuts(nth=181):
    """Observation directions: theta = 0..180 deg in the phi = 0 and phi = 90 deg cuts."""
    th = np.linspace(0.0, np.pi, nth)
    out = []
    for ph in (0.0, 0.5 * np.pi):
        out.append(np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1))
    return th, np.concatenate(out, 0)


def workload(name):
    """Named workloads.  Sizes: N = 2 * 6 m^2 * nc^2 complex unknowns."""
    if name == "sphere_d1_m1_nc8":  # PEC sphere, 1 wavelength diameter, 768 unknowns
        kh, pol = axial_incidence()
        return dict(name=name, bodies=body(semi=(0.5,) * 3)[None], ms=[1], nc=8, k=K0,
                    leaf=64, eta=2.0, aca_tol=1e-7, kdirs=kh, pols=pol, radius=0.5)
    if name == "sphere_d8_m4_nc10":  # PEC sphere, 8 wavelengths diameter, 19,200 unknowns
        kh, pol = incidence(4)
        return dict(name=name, bodies=body(semi=(4.0,) * 3)[None], ms=[4], nc=10, k=K0,
                    leaf=128, eta=2.0, aca_tol=1e-7, kdirs=kh, pols=pol, radius=4.0)
    if name == "sphere_d4_m2_nc10":  # PEC sphere, 4 wavelengths, 4,800 unknowns (precision comparison)
        kh, pol = incidence(4)
        return dict(name=name, bodies=body(semi=(2.0,) * 3)[None], ms=[2], nc=10, k=K0,
                    leaf=128, eta=2.0, aca_tol=1e-7, kdirs=kh, pols=pol, radius=2.0)
    if name == "sphere_d2_m2_nc6":  # mid-size parity case: 1,728 unknowns, ragged leaves
        kh, pol = incidence(2, SEED + 1)
        return dict(name=name, bodies=body(semi=(1.0,) * 3)[None], ms=[2], nc=6, k=K0,
                    leaf=40, eta=2.0, aca_tol=1e-7, kdirs=kh, pols=pol, radius=1.0)
    if name == "ellipsoid_small":  # rotated, off-centre ellipsoid, 3,072 unknowns
        th = 0.3
        R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
        kh, pol = incidence(3, SEED + 2)
        return dict(name=name, bodies=body(center=(0.1, -0.2, 0.05), semi=(1.2, 0.8, 0.5), rot=R)[None],
                    ms=[2], nc=8, k=K0, leaf=48, eta=2.0, aca_tol=1e-7, kdirs=kh, pols=pol)
    if name == "dielectric_d1_eps80_m2_nc12":  # high-contrast dielectric sphere, 13,824 unknowns (4 per node)
        kh, pol = axial_incidence()
        return dict(name=name, bodies=body(semi=(0.5,) * 3)[None], ms=[2], nc=12, k=K0, leaf=96, eta=2.0,
                    aca_tol=1e-8, kdirs=kh, pols=pol, radius=0.5, formulation="MULLER", eps_r=80.0)
    if name == "ellipsoid_d30_m16_nc8":  # electrically large PEC ellipsoid, 196,608 unknowns, 181 RHS
        kh, pol = monostatic_sweep(181)
        return dict(name=name, bodies=body(semi=(3.75, 7.5, 15.0))[None], ms=[16], nc=8, k=K0, leaf=256, eta=2.0,
                    aca_tol=1e-5, kdirs=kh, pols=pol)
    if name == "batch_spheroids64":  # 64 independent PEC prolate spheroids, 16 incidences each
        bodies, ms = spheroid_batch(64, SEED + 3)
        kh, pol = incidence(16, SEED + 4)
        return dict(name=name, bodies=bodies, ms=ms, nc=8, k=K0, leaf=64, eta=2.0, aca_tol=1e-7, kdirs=kh,
                    pols=pol, independent=True)
    if name == "batch_spheroids3":  # three independent spheroids (test batch), 2 incidences
        bodies, ms = spheroid_batch(3, SEED + 5, major=(1.0, 1.6, 2.0))
        kh, pol = incidence(2, SEED + 6)
        return dict(name=name, bodies=bodies, ms=ms, nc=8, k=K0, leaf=64, eta=2.0, aca_tol=1e-7, kdirs=kh,
                    pols=pol, independent=True)
    raise KeyError(name)


def monostatic_sweep(n):
    """n plane waves arriving from theta = 0..180 deg in the phi = 0 plane (k-hat = -r-hat),
    polarised along theta-hat: the incidences of a monostatic RCS sweep."""
    th = np.linspace(0.0, np.pi, n)
    kh = -np.stack([np.sin(th), np.zeros(n), np.cos(th)], 1)
    pol = np.stack([np.cos(th), np.zeros(n), -np.sin(th)], 1)
    return kh, pol


def spheroid_batch(n, seed, major=None):
    """n prolate spheroids along z: axis ratio ~ U[1, 3], major diameter ~ U[1, 4] wavelengths
    (or the given diameters), m = 1, 2, 3 patches per cube edge for a major diameter below
    4/3, below 8/3, else (768 to 6,912 unknowns at 8 x 8 nodes); centres on a cubic grid
    of 6-wavelength spacing.  Returns (bodies[n, 15], ms[n])."""
    g = np.random.Generator(np.random.Philox(seed))
    ratio = 1.0 + 2.0 * g.random(n)
    dmaj = 1.0 + 3.0 * g.random(n) if major is None else np.asarray(major, float)
    side = int(np.ceil(n ** (1.0 / 3.0)))
    bodies, ms = [], []
    for i in range(n):
        c = 6.0 * np.array([i % side, (i // side) % side, i // (side * side)], float)
        a = 0.5 * dmaj[i]
        b = a / ratio[i]
        bodies.append(body(center=c, semi=(b, b, a)))
        ms.append(1 if dmaj[i] < 4.0 / 3.0 else (2 if dmaj[i] < 8.0 / 3.0 else 3))
    return np.stack(bodies), ms


WORKLOADS = ("sphere_d1_m1_nc8", "sphere_d8_m4_nc10", "sphere_d4_m2_nc10", "sphere_d2_m2_nc6", "ellipsoid_small",
             "dielectric_d1_eps80_m2_nc12", "batch_spheroids64", "batch_spheroids3", "ellipsoid_d30_m16_nc8")


def mlp_init(nin, nh, seed=SEED):
    """Seeded initial parameters of the rank-predictor MLP (packed as the library expects:
    W1, b1, W2, b2, w3, b3): weights uniform in +-1/sqrt(fan_in), biases zero."""
    g = np.random.Generator(np.random.Philox(seed + 7))
    W1 = g.uniform(-1, 1, (nh, nin)) / np.sqrt(nin)
    W2 = g.uniform(-1, 1, (nh, nh)) / np.sqrt(nh)
    w3 = g.uniform(-1, 1, nh) / np.sqrt(nh)
    return np.concatenate([W1.ravel(), np.zeros(nh), W2.ravel(), np.zeros(nh), w3, [0.0]]).astype(np.float32)


def mlp_toy_data(n, nin, seed=SEED):
    """Seeded synthetic regression data for the MLP kernels' parity tests."""
    g = np.random.Generator(np.random.Philox(seed + 11))
    X = g.uniform(-1, 1, (n, nin)).astype(np.float32)
    t = (np.sin(X @ np.linspace(0.5, 1.5, nin)) + 0.1 * X[:, 0] ** 2).astype(np.float32)
    return X, t

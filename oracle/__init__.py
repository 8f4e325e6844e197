"""CBIE/MFIE oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow FP64 CPU implementation of what the CUDA path computes (dense MFIE
fill with independently integrated self/near entries, dense LU with partial
pivoting, solve, far field), the dense N-Mueller system of a dielectric body
(``MullerOracle``), independent Mie series for PEC and dielectric spheres
(``oracle.mie``) and the rank-predictor MLP (``oracle.mlp``).
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the library itself never does.

Every routine cites the passage of arXiv 2408.17116 it follows; the C source
(``cbie_oracle.c``) carries the detailed citations and the readings taken where
the paper is silent.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbie_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

ETA0 = float(np.sqrt(1.25663706212e-6 / 8.8541878128e-12))


def build(force=False):
    """Compile the C oracle with gcc (portable C99 + OpenMP; no -march flags)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu99",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, f64 = ctypes.c_int, ctypes.c_double
        L.or_create.restype = P
        L.or_create.argtypes = [i32, P, P, i32, f64, f64, i32, i32]
        L.or_destroy.argtypes = [P]
        L.or_num_nodes.argtypes = [P]
        L.or_num_patches.argtypes = [P]
        L.or_node_table.argtypes = [P, P]
        L.or_near_flags.argtypes = [P, P]
        L.or_near_block.argtypes = [P, i32, i32, P]
        L.or_single_layer_block.argtypes = [P, i32, i32, P]
        L.or_planar_single_layer.argtypes = [P, f64, f64, f64, P, i32, i32, P]
        L.or_matrix_rows.argtypes = [P, i32, P, P]
        L.or_matrix_dense.argtypes = [P, P]
        L.or_single_layer_dense.argtypes = [P, P]
        L.or_rhs.argtypes = [P, i32, P, P, P]
        L.or_currents.argtypes = [P, P, P]
        L.or_farfield.argtypes = [P, P, i32, P, P, P]
        L.or_zgetrf.argtypes = [i32, P, P]
        L.or_zgetrf.restype = i32
        L.or_zgetrs.argtypes = [i32, P, P, i32, P]
        L.or_cheb_nodes.argtypes = [i32, P]
        L.or_fejer_weights.argtypes = [i32, P]
        L.or_gauss_legendre.argtypes = [i32, P, P]
        L.or_cheb_cardinal.argtypes = [i32, P, f64, P]
        L.or_patch_point.argtypes = [P, i32, f64, f64, P, P, P]
        L.or_set_dielectric.argtypes = [P, f64, f64]
        L.or_muller_near_block.argtypes = [P, i32, i32, P]
        L.or_muller_far_block.argtypes = [P, i32, i32, P]
        L.or_matrix_dense_muller.argtypes = [P, P]
        L.or_rhs_muller.argtypes = [P, i32, P, P, P]
        L.or_currents_muller.argtypes = [P, P, P, P]
        L.or_farfield_muller.argtypes = [P, P, i32, P, P, P]
        L.or_set_cfie.argtypes = [P, f64]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def cheb_nodes(n):
    x = np.zeros(n)
    lib().or_cheb_nodes(n, _p(x))
    return x


def fejer_weights(n):
    w = np.zeros(n)
    lib().or_fejer_weights(n, _p(w))
    return w


def gauss_legendre(q):
    x, w = np.zeros(q), np.zeros(q)
    lib().or_gauss_legendre(q, _p(x), _p(w))
    return x, w


def cheb_cardinal(n, x):
    nodes = cheb_nodes(n)
    ell = np.zeros(n)
    lib().or_cheb_cardinal(n, _p(nodes), float(x), _p(ell))
    return ell


def zgetrf(A):
    """In-place dense LU with partial pivoting of a column-major copy; returns (LU, ipiv, info)."""
    n = A.shape[0]
    LU = np.array(A, dtype=np.complex128, order="F", copy=True)
    ipiv = np.zeros(n, dtype=np.int32)
    info = lib().or_zgetrf(n, _p(LU), _p(ipiv))
    return LU, ipiv, info


def zgetrs(LU, ipiv, B):
    n = LU.shape[0]
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    if X.ndim == 1:
        X = X.reshape(n, 1, order="F")
    lib().or_zgetrs(n, _p(LU), _p(ipiv), X.shape[1], _p(X))
    return X


class Oracle:
    """Dense MFIE discretisation of a set of cube-mapped ellipsoids.

    bodies: array (nbodies, 15): center[3], semi-axes[3], rotation[9] (row-major).
    ms: patches per cube-face edge for each body.  nc: Chebyshev nodes per direction.
    k: wavenumber.  delta: near-pair criterion.  q, qd: Gauss orders of the
    independent self/near integrator (box rule and Duffy rule).
    """

    def __init__(self, bodies, ms, nc, k, delta=0.5, q=12, qd=20, cfie_alpha=None):
        self.bodies = np.ascontiguousarray(np.asarray(bodies, dtype=np.float64).reshape(-1, 15))
        self.ms = np.ascontiguousarray(np.asarray(ms, dtype=np.int32).reshape(-1))
        self.nc, self.k, self.delta = int(nc), float(k), float(delta)
        self._h = lib().or_create(self.bodies.shape[0], _p(self.bodies), _p(self.ms),
                                  self.nc, self.k, self.delta, int(q), int(qd))
        if not self._h:
            raise ValueError("oracle: bad geometry arguments")
        self.nnode = lib().or_num_nodes(self._h)
        self.npatch = lib().or_num_patches(self._h)
        self.N = 2 * self.nnode
        self.cfie_alpha = cfie_alpha
        if cfie_alpha is not None:
            # PEC combined field equation alpha EFIE / eta0 + (1 - alpha) MFIE (Eq. 10, both rows)
            lib().or_set_cfie(self._h, float(cfie_alpha))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    def node_table(self):
        t = np.zeros((self.nnode, 17))
        lib().or_node_table(self._h, _p(t))
        return t

    def near_flags(self):
        f = np.zeros((self.npatch, self.npatch), dtype=np.uint8)
        lib().or_near_flags(self._h, _p(f))
        return f.astype(bool)

    def near_block(self, tn, p):
        W = np.zeros((4, self.nc * self.nc), dtype=np.complex128)
        lib().or_near_block(self._h, int(tn), int(p), _p(W))
        return W

    def single_layer_block(self, tn, p):
        W = np.zeros(self.nc * self.nc, dtype=np.complex128)
        lib().or_single_layer_block(self._h, int(tn), int(p), _p(W))
        return W

    def planar_single_layer(self, a, b, k, tgt, self_node=None):
        W = np.zeros(self.nc * self.nc, dtype=np.complex128)
        t = np.ascontiguousarray(np.asarray(tgt, dtype=np.float64))
        lu, kv = (-1, -1) if self_node is None else self_node
        lib().or_planar_single_layer(self._h, float(a), float(b), float(k), _p(t), int(lu), int(kv), _p(W))
        return W

    def patch_point(self, p, u, v):
        r, ru, rv = np.zeros(3), np.zeros(3), np.zeros(3)
        lib().or_patch_point(self._h, int(p), float(u), float(v), _p(r), _p(ru), _p(rv))
        return r, ru, rv

    def matrix_rows(self, rows):
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
        out = np.zeros((rows.size, self.N), dtype=np.complex128)
        lib().or_matrix_rows(self._h, rows.size, _p(rows), _p(out))
        return out

    def dense(self):
        A = np.zeros((self.N, self.N), dtype=np.complex128, order="F")
        lib().or_matrix_dense(self._h, _p(A))
        return A

    def single_layer_dense(self):
        S = np.zeros((self.nnode, self.nnode), dtype=np.complex128, order="F")
        lib().or_single_layer_dense(self._h, _p(S))
        return S

    def rhs(self, kdirs, pols):
        kd = np.ascontiguousarray(np.asarray(kdirs, dtype=np.float64).reshape(-1, 3))
        po = np.ascontiguousarray(np.asarray(pols, dtype=np.float64).reshape(-1, 3))
        b = np.zeros((kd.shape[0], self.N), dtype=np.complex128)
        lib().or_rhs(self._h, kd.shape[0], _p(kd), _p(po), _p(b))
        return b

    def currents(self, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        J = np.zeros((self.nnode, 3), dtype=np.complex128)
        lib().or_currents(self._h, _p(x), _p(J))
        return J

    def farfield(self, x, dirs):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
        ef = np.zeros((d.shape[0], 3), dtype=np.complex128)
        rcs = np.zeros(d.shape[0])
        lib().or_farfield(self._h, _p(x), d.shape[0], _p(d), _p(ef), _p(rcs))
        return ef, rcs

    def solve_dense(self, b):
        """Dense fill, LU with partial pivoting, solve: the definition of the discrete solution."""
        A = self.dense()
        LU, ipiv, info = zgetrf(A)
        if info:
            raise np.linalg.LinAlgError("oracle: singular pivot %d" % info)
        X = zgetrs(LU, ipiv, np.asarray(b).T)
        return X.T.copy(), A


class MullerOracle(Oracle):
    """Dense N-Mueller discretisation (Sec. II.A, Eqs. 7-9) of dielectric cube-mapped
    ellipsoids of relative permittivity eps_r (mu_r = 1) in free space.

    Unknowns per node: (eta0 J^u, eta0 J^v, M^u, M^v) (F = sqrt|G| x contravariant
    component, Eq. 11); rows per node: tested E equation (u, v), tested H equation (u, v).
    """

    def __init__(self, bodies, ms, nc, k, eps_r, delta=0.5, q=12, qd=20):
        super().__init__(bodies, ms, nc, k, delta=delta, q=q, qd=qd)
        self.eps_r = complex(eps_r)
        lib().or_set_dielectric(self._h, self.eps_r.real, self.eps_r.imag)
        self.N = 4 * self.nnode

    def near_block(self, tn, p):
        W = np.zeros((16, self.nc * self.nc), dtype=np.complex128)
        lib().or_muller_near_block(self._h, int(tn), int(p), _p(W))
        return W

    def far_block(self, tn, p):
        W = np.zeros((16, self.nc * self.nc), dtype=np.complex128)
        lib().or_muller_far_block(self._h, int(tn), int(p), _p(W))
        return W

    def dense(self):
        A = np.zeros((self.N, self.N), dtype=np.complex128, order="F")
        lib().or_matrix_dense_muller(self._h, _p(A))
        return A

    def rhs(self, kdirs, pols):
        kd = np.ascontiguousarray(np.asarray(kdirs, dtype=np.float64).reshape(-1, 3))
        po = np.ascontiguousarray(np.asarray(pols, dtype=np.float64).reshape(-1, 3))
        b = np.zeros((kd.shape[0], self.N), dtype=np.complex128)
        lib().or_rhs_muller(self._h, kd.shape[0], _p(kd), _p(po), _p(b))
        return b

    def currents(self, x):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        J = np.zeros((self.nnode, 3), dtype=np.complex128)
        M = np.zeros((self.nnode, 3), dtype=np.complex128)
        lib().or_currents_muller(self._h, _p(x), _p(J), _p(M))
        return J, M

    def farfield(self, x, dirs):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
        d = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64).reshape(-1, 3))
        ef = np.zeros((d.shape[0], 3), dtype=np.complex128)
        rcs = np.zeros(d.shape[0])
        lib().or_farfield_muller(self._h, _p(x), d.shape[0], _p(d), _p(ef), _p(rcs))
        return ef, rcs

    def matrix_rows(self, rows):
        raise NotImplementedError("row sampling is provided for the MFIE system only")

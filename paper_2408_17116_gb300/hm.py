"""Thin ctypes binding of libhm (include/hm.h): argument marshalling only.

Every step of the solver runs in the CUDA library; PyTorch supplies device
buffers (complex128 tensors) and the stream.  Importing this module raises if
libhm.so has not been built: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "libhm.so")

HM_OK = 0
STATUS = {0: "HM_OK", 1: "HM_ERR_ARG", 2: "HM_ERR_STATE", 3: "HM_ERR_CUDA", 4: "HM_ERR_OOM",
          5: "HM_ERR_SINGULAR", 6: "HM_ERR_NOT_CONVERGED", 7: "HM_ERR_TIMEOUT", 8: "HM_ERR_NUMERIC"}
Q = dict(N=0, NNODE=1, NPATCH=2, NEAR_PAIRS=3, DENSE_BLOCKS=4, LR_BLOCKS=5, CR=6, MAX_RANK=7,
         T_GEOMETRY=8, T_NEAR=9, T_DENSE=10, T_ACA=11, T_FACTOR=12, T_SOLVE=13, FLOPS_FACTOR=14,
         STORAGE=15, ACA_NONCONV=16, LAUNCHES=17, NEAR_QPOINTS=18, MEAN_RANK=19, STORAGE_FACTOR=20,
         T_RECOMPRESS=21, REFINE_ITERS=22, REFINE_RES=23, STORAGE32=24, ACA_PREALLOC=25, ACA_RERUNS=26,
         RANK_PRED_ERR=27, TRUNC_BATCHES=28, TRUNC_JOBS=29, TRUNC_MAXK=30, TRUNC_WORK=31, T_TRUNC=32,
         ACA_SKIPPED=33, KQR_SECONDS=34, KQR_FLOPS=35, KQR_LAUNCHES=36, KCORE_SECONDS=37,
         KCORE_FLOPS=38, KCORE_LAUNCHES=39, DENSE_LEVEL=40, KGEMM_SECONDS=41, KGEMM_FLOPS=42,
         KGEMM_LAUNCHES=43, KTC_SECONDS=44, KTC_FLOPS=45, KTC_LAUNCHES=46,
         T_LU_PANEL=47, T_LU_U12=48, T_TILE_BUILD=49, T_SOLVE_SWEEP=50, T_SOLVE_MATVEC=51)
RANK_NFEAT = 8
HM_FP64, HM_FP32_REFINED = 0, 1
HM_PEC_MFIE, HM_PEC_CFIE, HM_DIEL_MULLER = 0, 1, 2
FAULT = dict(NONE=0, ZERO_PIVOT=1, NAN_RHS=2, ALLOC=3)

EXPORTS = ("hm_version", "hm_create", "hm_build_geometry", "hm_fill", "hm_factor", "hm_solve",
           "hm_solve_host", "hm_farfield", "hm_matvec", "hm_query", "hm_last_error", "hm_destroy",
           "hm_get_nodes_host", "hm_get_near_pairs_host", "hm_get_near_block_host", "hm_entries_host",
           "hm_get_perm_host", "hm_get_blocks_host", "hm_get_block_dense_host", "hm_rank_samples",
           "hm_set_rank_model", "hm_mlp_create", "hm_mlp_num_params", "hm_mlp_set_params", "hm_mlp_get_params",
           "hm_mlp_forward", "hm_mlp_loss_grad", "hm_mlp_train", "hm_mlp_last_error", "hm_mlp_destroy",
           "hm_farfield_static", "hm_plan_host", "hm_muller_far_block_host", "hm_muller_near_block_host",
           "hm_muller_rhs_farfield_host", "hm_inject_fault", "hm_get_trunc_log_host", "hm_cgemm", "hm_tc_tuning", "hm_plan_bodies_host")


class hm_params(ctypes.Structure):
    _fields_ = [("k0", ctypes.c_double), ("formulation", ctypes.c_int), ("leaf", ctypes.c_int),
                ("eta", ctypes.c_double), ("aca_tol", ctypes.c_double), ("near_delta", ctypes.c_double),
                ("aca_max_rank", ctypes.c_int), ("precision", ctypes.c_int), ("keep_matrix", ctypes.c_int),
                ("factor_tol", ctypes.c_double), ("refine_tol", ctypes.c_double), ("refine_max_iter", ctypes.c_int),
                ("cfie_alpha", ctypes.c_double), ("eps_r_re", ctypes.c_double), ("eps_r_im", ctypes.c_double),
                ("mu_r", ctypes.c_double), ("trunc_tol", ctypes.c_double), ("quad_order", ctypes.c_int),
                ("factor_leaf", ctypes.c_int), ("simt_gemm", ctypes.c_int), ("independent", ctypes.c_int)]


class hm_body(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("m", ctypes.c_int), ("center", ctypes.c_double * 3),
                ("semi_axes", ctypes.c_double * 3), ("rot", ctypes.c_double * 9)]


class HmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def load(path=SO):
    """Load libhm.so (raises when it is missing: build it with paper_2408_17116_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libhm.so not built (%s); run paper_2408_17116_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.hm_version.restype = ctypes.c_char_p
    L.hm_last_error.restype = ctypes.c_char_p
    L.hm_last_error.argtypes = [P]
    L.hm_create.argtypes = [ctypes.POINTER(P), P]
    L.hm_build_geometry.argtypes = [P, ctypes.POINTER(hm_body), I, I, ctypes.POINTER(hm_params)]
    L.hm_fill.argtypes = [P]
    L.hm_factor.argtypes = [P]
    L.hm_solve.argtypes = [P, I, P, P, P]
    L.hm_solve_host.argtypes = [P, I, P, P, P]
    L.hm_farfield.argtypes = [P, I, P, I, P, P, P]
    L.hm_matvec.argtypes = [P, I, P, P]
    L.hm_farfield_static.argtypes = [P, I, P, I, P, P, P]
    L.hm_plan_host.argtypes = [P, I, I, I, D, ctypes.POINTER(I), P, P]
    L.hm_plan_bodies_host.argtypes = [P, P, I, I, I, D, ctypes.POINTER(I), P, P]
    L.hm_muller_far_block_host.argtypes = [ctypes.POINTER(hm_body), I, I, D, D, D, I, I, P]
    L.hm_muller_near_block_host.argtypes = [ctypes.POINTER(hm_body), I, I, D, D, D, I, I, I, I, I, D, P]
    L.hm_muller_rhs_farfield_host.argtypes = [ctypes.POINTER(hm_body), I, I, D, P, P, P, P, I, P, P]
    L.hm_query.argtypes = [P, I, ctypes.POINTER(D)]
    L.hm_inject_fault.argtypes = [P, I]
    L.hm_tc_tuning.argtypes = [P, P]
    L.hm_cgemm.argtypes = [P, ctypes.c_char, ctypes.c_char, I, I, I, P, P, I, P, I, P, P, I, I]
    L.hm_get_trunc_log_host.argtypes = [P, ctypes.POINTER(I), P]
    L.hm_destroy.argtypes = [P]
    L.hm_destroy.restype = None
    L.hm_get_nodes_host.argtypes = [P, P]
    L.hm_get_near_pairs_host.argtypes = [P, P]
    L.hm_get_near_block_host.argtypes = [P, I, I, P]
    L.hm_entries_host.argtypes = [P, I, P, P, P]
    L.hm_get_perm_host.argtypes = [P, P]
    L.hm_get_blocks_host.argtypes = [P, ctypes.POINTER(I), P]
    L.hm_get_block_dense_host.argtypes = [P, I, P]
    L.hm_rank_samples.argtypes = [P, ctypes.POINTER(I), P, P]
    L.hm_set_rank_model.argtypes = [P, P]
    L.hm_mlp_create.argtypes = [ctypes.POINTER(P), I, I, P]
    L.hm_mlp_num_params.argtypes = [P]
    L.hm_mlp_set_params.argtypes = [P, P]
    L.hm_mlp_get_params.argtypes = [P, P]
    L.hm_mlp_forward.argtypes = [P, I, P, P]
    L.hm_mlp_loss_grad.argtypes = [P, I, P, P, ctypes.POINTER(D), P]
    L.hm_mlp_train.argtypes = [P, I, P, P, I, ctypes.c_float, ctypes.POINTER(D)]
    L.hm_mlp_last_error.restype = ctypes.c_char_p
    L.hm_mlp_last_error.argtypes = [P]
    L.hm_mlp_destroy.argtypes = [P]
    L.hm_mlp_destroy.restype = None
    for name in EXPORTS:
        if name not in ("hm_version", "hm_last_error", "hm_destroy", "hm_mlp_last_error", "hm_mlp_destroy"):
            getattr(L, name).restype = I
    _lib = L
    return L


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def plan_host(xyz, leaf, eta, dof=2):
    """Block cluster tree of hm_plan_host (host only): (blocks [n][5], perm_node [nnode])."""
    L = load()
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    n = ctypes.c_int()
    st = L.hm_plan_host(_np_ptr(xyz), xyz.shape[0], int(dof), int(leaf), float(eta), ctypes.byref(n), None, None)
    if st != HM_OK:
        raise HmError(st, "hm_plan_host")
    blocks = np.empty((n.value, 5), dtype=np.int32)
    perm = np.empty(xyz.shape[0], dtype=np.int32)
    st = L.hm_plan_host(_np_ptr(xyz), xyz.shape[0], int(dof), int(leaf), float(eta), ctypes.byref(n),
                        _np_ptr(blocks), _np_ptr(perm))
    if st != HM_OK:
        raise HmError(st, "hm_plan_host")
    return blocks, perm


def plan_bodies_host(xyz, node_body, leaf, eta, dof=2):
    """hm_plan_bodies_host (host only): the block cluster tree of a batch of independent
    bodies, (blocks [n][5] with type 2 for zero blocks between bodies, perm_node [nnode])."""
    L = load()
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    nb = np.ascontiguousarray(np.asarray(node_body, dtype=np.int32))
    n = ctypes.c_int()
    args = (_np_ptr(xyz), _np_ptr(nb), xyz.shape[0], int(dof), int(leaf), float(eta), ctypes.byref(n))
    st = L.hm_plan_bodies_host(*args, None, None)
    if st != HM_OK:
        raise HmError(st, "hm_plan_bodies_host")
    blocks = np.empty((n.value, 5), dtype=np.int32)
    perm = np.empty(xyz.shape[0], dtype=np.int32)
    st = L.hm_plan_bodies_host(*args, _np_ptr(blocks), _np_ptr(perm))
    if st != HM_OK:
        raise HmError(st, "hm_plan_bodies_host")
    return blocks, perm


def muller_far_block_host(bodies, ms, nc, k0, eps_r, tn, p):
    """N-Mueller far entries of target node tn over source patch p (host): [16][nc^2]."""
    L = load()
    arr = make_bodies(bodies, ms)
    out = np.zeros((16, int(nc) ** 2), dtype=np.complex128)
    eps = complex(eps_r)
    st = L.hm_muller_far_block_host(arr, len(ms), int(nc), float(k0), eps.real, eps.imag, int(tn), int(p),
                                    _np_ptr(out))
    if st != HM_OK:
        raise HmError(st, "hm_muller_far_block_host")
    return out


def muller_near_block_host(bodies, ms, nc, k0, eps_r, tn, p, qd=0, qi=0, qo=0, t0=0.0):
    """N-Mueller self/near integrals of target node tn over source patch p (host): [16][nc^2]."""
    L = load()
    arr = make_bodies(bodies, ms)
    out = np.zeros((16, int(nc) ** 2), dtype=np.complex128)
    eps = complex(eps_r)
    st = L.hm_muller_near_block_host(arr, len(ms), int(nc), float(k0), eps.real, eps.imag, int(tn), int(p),
                                     int(qd), int(qi), int(qo), float(t0), _np_ptr(out))
    if st != HM_OK:
        raise HmError(st, "hm_muller_near_block_host")
    return out


def muller_rhs_farfield_host(bodies, ms, nc, k0, khat=None, pol=None, x=None, dirs=None):
    """N-Mueller right-hand side [4 nnode] and far field [nang][3] (host)."""
    L = load()
    arr = make_bodies(bodies, ms)
    nnode = 6 * int(np.sum(np.asarray(ms) ** 2)) * int(nc) ** 2
    rhs = efar = None
    kp = pp = xp = dp = ep = None
    if khat is not None:
        kh = np.ascontiguousarray(np.asarray(khat, np.float64).reshape(3))
        po = np.ascontiguousarray(np.asarray(pol, np.float64).reshape(3))
        rhs = np.zeros(4 * nnode, dtype=np.complex128)
        kp, pp, rp = _np_ptr(kh), _np_ptr(po), _np_ptr(rhs)
    else:
        rp = None
    nang = 0
    if x is not None:
        xs = np.ascontiguousarray(np.asarray(x, np.complex128).reshape(-1))
        d = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
        nang = d.shape[0]
        efar = np.zeros((nang, 3), dtype=np.complex128)
        xp, dp, ep = _np_ptr(xs), _np_ptr(d), _np_ptr(efar)
    st = L.hm_muller_rhs_farfield_host(arr, len(ms), int(nc), float(k0), kp, pp, rp, xp, nang, dp, ep)
    if st != HM_OK:
        raise HmError(st, "hm_muller_rhs_farfield_host")
    return rhs, efar


def make_bodies(bodies, ms):
    bodies = np.asarray(bodies, dtype=np.float64).reshape(-1, 15)
    arr = (hm_body * bodies.shape[0])()
    for i, b in enumerate(bodies):
        arr[i].family = 0
        arr[i].m = int(ms[i])
        for d in range(3):
            arr[i].center[d] = b[d]
            arr[i].semi_axes[d] = b[3 + d]
        for d in range(9):
            arr[i].rot[d] = b[6 + d]
    return arr


def tc_tuning():
    """The tensor-core autotuner's record: (variant[8], ms[8, 3]) per depth class 64 << c;
    variant 2 / 4 = 2- / 4-stage ring, 1 = persistent, 0 = not tuned; ms columns in that
    order (2-stage, 4-stage, persistent)."""
    st = np.zeros(8, dtype=np.int32)
    ms = np.zeros(24, dtype=np.float32)
    r = load().hm_tc_tuning(_np_ptr(st), _np_ptr(ms))
    if r != HM_OK:
        raise HmError(r, "hm_tc_tuning")
    return st, ms.reshape(8, 3)


class Solver:
    """One hm_handle.  Methods mirror the C entry points of include/hm.h."""

    def __init__(self, stream=None):
        import torch
        self.torch = torch
        self.L = load()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.h = ctypes.c_void_p()
        self._check(self.L.hm_create(ctypes.byref(self.h), ctypes.c_void_p(stream)), nohandle=True)

    def _check(self, st, nohandle=False):
        if st != HM_OK:
            msg = "" if nohandle else self.L.hm_last_error(self.h).decode()
            raise HmError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.hm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def hm_build_geometry(self, bodies, ms, nc, k0, leaf, eta, aca_tol, near_delta=0.5, aca_max_rank=0,
                          keep_matrix=False, precision=HM_FP64, factor_tol=0.0, refine_tol=0.0, refine_max_iter=0,
                          formulation=HM_PEC_MFIE, cfie_alpha=0.0, eps_r=1.0, mu_r=0.0, trunc_tol=0.0,
                          quad_order=0, factor_leaf=0, simt_gemm=False, independent=False):
        self._bodies = make_bodies(bodies, ms)
        eps = complex(eps_r)
        p = hm_params(k0=float(k0), formulation=int(formulation), leaf=int(leaf), eta=float(eta),
                      aca_tol=float(aca_tol), near_delta=float(near_delta), aca_max_rank=int(aca_max_rank),
                      precision=int(precision), keep_matrix=int(bool(keep_matrix)), factor_tol=float(factor_tol),
                      refine_tol=float(refine_tol), refine_max_iter=int(refine_max_iter),
                      cfie_alpha=float(cfie_alpha), eps_r_re=eps.real, eps_r_im=eps.imag, mu_r=float(mu_r),
                      trunc_tol=float(trunc_tol), quad_order=int(quad_order), factor_leaf=int(factor_leaf),
                      simt_gemm=int(bool(simt_gemm)), independent=int(bool(independent)))
        self._check(self.L.hm_build_geometry(self.h, self._bodies, len(ms), int(nc), ctypes.byref(p)))
        self.N = int(self.hm_query("N"))
        self.dof = 4 if int(formulation) == HM_DIEL_MULLER else 2
        self.nnode = self.N // self.dof
        self.nc = int(nc)

    def hm_fill(self):
        self._check(self.L.hm_fill(self.h))

    def hm_factor(self):
        self._check(self.L.hm_factor(self.h))

    def hm_solve(self, kdirs, pols, out=None):
        kd = np.ascontiguousarray(np.asarray(kdirs, np.float64).reshape(-1, 3))
        po = np.ascontiguousarray(np.asarray(pols, np.float64).reshape(-1, 3))
        if out is None:
            out = self.torch.empty((kd.shape[0], self.N), dtype=self.torch.complex128, device="cuda")
        self._check(self.L.hm_solve(self.h, kd.shape[0], _np_ptr(kd), _np_ptr(po), ctypes.c_void_p(out.data_ptr())))
        return out

    def hm_solve_host(self, kdirs, pols, out=None):
        kd = np.ascontiguousarray(np.asarray(kdirs, np.float64).reshape(-1, 3))
        po = np.ascontiguousarray(np.asarray(pols, np.float64).reshape(-1, 3))
        if out is None:
            out = np.empty((kd.shape[0], self.N), dtype=np.complex128)
        self._check(self.L.hm_solve_host(self.h, kd.shape[0], _np_ptr(kd), _np_ptr(po), _np_ptr(out)))
        return out

    def hm_farfield(self, x, dirs, want_efar=True):
        d = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
        x = x.reshape(-1, self.N)
        nrhs = x.shape[0]
        efar = self.torch.empty((nrhs, d.shape[0], 3), dtype=self.torch.complex128, device="cuda") if want_efar else None
        rcs = np.empty((nrhs, d.shape[0]))
        self._check(self.L.hm_farfield(self.h, nrhs, ctypes.c_void_p(x.data_ptr()), d.shape[0], _np_ptr(d),
                                       ctypes.c_void_p(efar.data_ptr() if efar is not None else 0), _np_ptr(rcs)))
        return efar, rcs

    def hm_farfield_static(self, x, dirs, want_efar=True):
        """hm_farfield through the entry point that allocates no device memory."""
        d = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
        x = x.reshape(-1, self.N)
        nrhs = x.shape[0]
        efar = self.torch.empty((nrhs, d.shape[0], 3), dtype=self.torch.complex128, device="cuda") if want_efar else None
        rcs = np.empty((nrhs, d.shape[0]))
        self._check(self.L.hm_farfield_static(self.h, nrhs, ctypes.c_void_p(x.data_ptr()), d.shape[0], _np_ptr(d),
                                              ctypes.c_void_p(efar.data_ptr() if efar is not None else 0),
                                              _np_ptr(rcs)))
        return efar, rcs

    def hm_matvec(self, x):
        x = x.reshape(-1, self.N).contiguous()
        y = self.torch.empty_like(x)
        self._check(self.L.hm_matvec(self.h, x.shape[0], ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())))
        return y

    def trunc_log(self):
        """Per recompression batch: jobs, max m|n, max K, sum (m+n) K^2, QR s, core s, wall s."""
        n = ctypes.c_int()
        self._check(self.L.hm_get_trunc_log_host(self.h, ctypes.byref(n), None))
        out = np.empty((n.value, 7))
        self._check(self.L.hm_get_trunc_log_host(self.h, ctypes.byref(n), _np_ptr(out)))
        return out

    def hm_cgemm(self, opA, opB, alpha, A, B, beta, C, path=0):
        """C = alpha op(A) op(B) + beta C on complex64 CUDA tensors in column-major storage:
        pass the transposes of row-major torch tensors (A.T etc.), i.e. A, B, C are
        torch tensors whose .T is contiguous.  Returns C."""
        def colmajor(X):
            assert X.dtype == self.torch.complex64 and X.is_cuda and X.dim() == 2
            assert X.stride(0) == 1, "column-major (X.T contiguous) expected"
            return X.stride(1)
        lda, ldb, ldc = colmajor(A), colmajor(B), colmajor(C)
        m, n = C.shape
        k = A.shape[1] if opA == "N" else A.shape[0]
        al = (ctypes.c_float * 2)(complex(alpha).real, complex(alpha).imag)
        be = (ctypes.c_float * 2)(complex(beta).real, complex(beta).imag)
        self._check(self.L.hm_cgemm(self.h, opA.encode(), opB.encode(), m, n, k, ctypes.cast(al, ctypes.c_void_p),
                                    ctypes.c_void_p(A.data_ptr()), max(lda, 1), ctypes.c_void_p(B.data_ptr()),
                                    max(ldb, 1), ctypes.cast(be, ctypes.c_void_p), ctypes.c_void_p(C.data_ptr()),
                                    max(ldc, 1), int(path)))
        return C

    def hm_inject_fault(self, what):
        self._check(self.L.hm_inject_fault(self.h, FAULT[what] if isinstance(what, str) else int(what)))

    def hm_query(self, key):
        out = ctypes.c_double()
        self._check(self.L.hm_query(self.h, Q[key] if isinstance(key, str) else int(key), ctypes.byref(out)))
        return out.value

    def nodes(self):
        t = np.empty((self.nnode, 14))
        self._check(self.L.hm_get_nodes_host(self.h, _np_ptr(t)))
        return t

    def near_pairs(self):
        n = int(self.hm_query("NEAR_PAIRS"))
        out = np.empty((n, 2), dtype=np.int32)
        self._check(self.L.hm_get_near_pairs_host(self.h, _np_ptr(out)))
        return out

    def near_block(self, tn, p):
        out = np.empty((self.dof * self.dof, self.nc * self.nc), dtype=np.complex128)
        self._check(self.L.hm_get_near_block_host(self.h, int(tn), int(p), _np_ptr(out)))
        return out

    def entries(self, rows, cols):
        r = np.ascontiguousarray(np.asarray(rows, np.int32))
        c = np.ascontiguousarray(np.asarray(cols, np.int32))
        out = np.empty(r.size, dtype=np.complex128)
        self._check(self.L.hm_entries_host(self.h, r.size, _np_ptr(r), _np_ptr(c), _np_ptr(out)))
        return out

    def perm(self):
        out = np.empty(self.N, dtype=np.int32)
        self._check(self.L.hm_get_perm_host(self.h, _np_ptr(out)))
        return out

    def blocks(self):
        n = ctypes.c_int()
        self._check(self.L.hm_get_blocks_host(self.h, ctypes.byref(n), None))
        out = np.empty((n.value, 6), dtype=np.int32)
        self._check(self.L.hm_get_blocks_host(self.h, ctypes.byref(n), _np_ptr(out)))
        return out

    def block_dense(self, b):
        info = self.blocks()[b]
        out = np.empty((info[4], info[2]), dtype=np.complex128)  # column-major nr x nc -> (nc, nr) C-order
        self._check(self.L.hm_get_block_dense_host(self.h, int(b), _np_ptr(out)))
        return out.T

    def rank_samples(self):
        """(features [n][8] float32, log(1 + ACA rank) [n] float32) of the last hm_fill."""
        n = ctypes.c_int()
        self._check(self.L.hm_rank_samples(self.h, ctypes.byref(n), None, None))
        f = np.empty((n.value, RANK_NFEAT), dtype=np.float32)
        t = np.empty(n.value, dtype=np.float32)
        self._check(self.L.hm_rank_samples(self.h, ctypes.byref(n), _np_ptr(f), _np_ptr(t)))
        return f, t

    def set_rank_model(self, mlp):
        self._rank_model = mlp  # keeps the model alive while the handle may use it
        self._check(self.L.hm_set_rank_model(self.h, mlp.m if mlp is not None else None))


class MLP:
    """One hm_mlp: the learned ACA-rank predictor (include/hm.h)."""

    def __init__(self, nin=RANK_NFEAT, nh=32, stream=None):
        import torch
        self.torch = torch
        self.L = load()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.m = ctypes.c_void_p()
        st = self.L.hm_mlp_create(ctypes.byref(self.m), int(nin), int(nh), ctypes.c_void_p(stream))
        if st != HM_OK:
            raise HmError(st, "hm_mlp_create")
        self.nin, self.nh = int(nin), int(nh)
        self.np = self.L.hm_mlp_num_params(self.m)

    def _check(self, st):
        if st != HM_OK:
            raise HmError(st, self.L.hm_mlp_last_error(self.m).decode())

    def close(self):
        if getattr(self, "m", None):
            self.L.hm_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        assert p.size == self.np
        self._check(self.L.hm_mlp_set_params(self.m, _np_ptr(p)))

    def get_params(self):
        p = np.empty(self.np, dtype=np.float32)
        self._check(self.L.hm_mlp_get_params(self.m, _np_ptr(p)))
        return p

    def forward(self, x):
        x = x.contiguous()
        y = self.torch.empty(x.shape[0], dtype=self.torch.float32, device=x.device)
        self._check(self.L.hm_mlp_forward(self.m, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(y.data_ptr())))
        return y

    def loss_grad(self, x, t):
        x, t = x.contiguous(), t.contiguous()
        loss = ctypes.c_double()
        g = np.empty(self.np, dtype=np.float32)
        self._check(self.L.hm_mlp_loss_grad(self.m, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(t.data_ptr()), ctypes.byref(loss), _np_ptr(g)))
        return loss.value, g

    def train(self, x, t, steps, lr):
        x, t = x.contiguous(), t.contiguous()
        loss = ctypes.c_double()
        self._check(self.L.hm_mlp_train(self.m, x.shape[0], ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(t.data_ptr()), int(steps), float(lr), ctypes.byref(loss)))
        return loss.value

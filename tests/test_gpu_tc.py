"""Tensor-core complex64 GEMM (tcgen05, split-BF16, Sec. III / Eq. 23 Schur products) through
the C-ABI entry hm_cgemm, element by element against the FP64 product of the same complex64
inputs (numpy, on the host).

Bound (first order, rigorous): BF16 keeps 8 significant bits, so a_hi = bf16(a) is within
2^-8 |a| of a and a_lo = bf16(a - a_hi) leaves a remainder within 2^-16 |a|; the product
a_hi b_hi + a_hi b_lo + a_lo b_hi then differs from a b by at most 3 * 2^-16 |a| |b| (the two
remainders and the dropped a_lo b_lo).  FP32 accumulation of the 2k real terms of an entry
(and one rounding per 2,048-deep chunk of k) adds at most (2k + 4) 2^-24 of the same sum.
So |C - C_exact| <= (3 * 2^-16 + (2k + 4) 2^-24) (|alpha| |A| |B| + |beta| |C0|) entrywise,
with |A| |B| computed in FP64; the CUDA-core FP32 path is held to (2k + 4) 2^-24.
Shapes span several 128 x 256 output
tiles, ragged edges in m, n and k, more than one 2,048-deep chunk of k, and all four
combinations of 'N' and 'C'.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2408_17116_gb300 import build, hm  # noqa: E402

build.build()

ARG = 1


def colmajor(a):
    """complex64 CUDA tensor with column-major storage holding the numpy matrix a."""
    t = torch.from_numpy(np.ascontiguousarray(a.T.astype(np.complex64))).cuda()
    return t.T


def rand(rng, r, c):
    return (rng.standard_normal((r, c)) + 1j * rng.standard_normal((r, c))).astype(np.complex64)


def op(x, o):
    return x if o == "N" else x.conj().T


CASES = [(64, 64, 16), (200, 300, 100), (333, 517, 77), (1000, 700, 2500), (128, 256, 64), (97, 1290, 300),
         (2100, 1500, 256)]


@pytest.mark.parametrize("m,n,k", CASES)
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("C", "N"), ("N", "C"), ("C", "C")])
def test_tensor_core_gemm_against_fp64_product(m, n, k, opA, opB):
    rng = np.random.default_rng(m * 7919 + n * 31 + k + ord(opA) * 3 + ord(opB))
    A = rand(rng, m, k) if opA == "N" else rand(rng, k, m)
    B = rand(rng, k, n) if opB == "N" else rand(rng, n, k)
    C0 = rand(rng, m, n)
    alpha, beta = complex(-1.0, 0.25), complex(0.5, -1.0)
    Ad, Bd = op(A.astype(np.complex128), opA), op(B.astype(np.complex128), opB)
    ref = alpha * (Ad @ Bd) + beta * C0.astype(np.complex128)
    scale = abs(alpha) * (np.abs(Ad) @ np.abs(Bd)) + abs(beta) * np.abs(C0)
    s = hm.Solver()
    acc = (2 * k + 4) * 2.0 ** -24
    tc = 3 * 2.0 ** -16 + acc
    # 2: autotuned variant; 3, 4, 5: the 2-stage, 4-stage and persistent kernels; 1: CUDA cores
    for path, tol in ((2, tc), (3, tc), (4, tc), (5, tc), (1, acc)):
        C = colmajor(C0)
        s.hm_cgemm(opA, opB, alpha, colmajor(A), colmajor(B), beta, C, path=path)
        got = C.cpu().numpy()
        err = np.abs(got - ref) / scale
        assert np.all(np.isfinite(got))
        assert err.max() <= tol, (path, float(err.max()))
    s.close()


def test_tensor_core_gemm_on_submatrix_views_leaves_the_rest_untouched():
    # operands and output as sub-blocks of larger column-major arrays (ld > rows), the way
    # the H-LU calls it on blocks of a merged dense leaf
    rng = np.random.default_rng(5)
    big = rand(rng, 900, 800)
    Cbig = colmajor(big)
    keep = Cbig.cpu().numpy().copy()
    A = colmajor(rand(rng, 600, 500))[100:500, 50:450]   # 400 x 400 view, ld 600
    B = colmajor(rand(rng, 700, 600))[200:600, 0:390]    # 400 x 390 view, ld 700
    Cv = Cbig[300:700, 250:640]                           # 400 x 390 view, ld 900
    ref = Cv.cpu().numpy().astype(np.complex128) - A.cpu().numpy().astype(np.complex128) @ \
        B.cpu().numpy().astype(np.complex128)
    scale = np.abs(A.cpu().numpy()).astype(np.float64) @ np.abs(B.cpu().numpy()).astype(np.float64) + \
        np.abs(Cv.cpu().numpy())
    s = hm.Solver()
    s.hm_cgemm("N", "N", -1.0, A, B, 1.0, Cv, path=2)
    out = Cbig.cpu().numpy()
    err = np.abs(out[300:700, 250:640] - ref) / scale
    assert err.max() <= 3 * 2.0 ** -16 + (2 * 400 + 4) * 2.0 ** -24
    mask = np.ones(out.shape, bool)
    mask[300:700, 250:640] = False
    assert np.array_equal(out[mask], keep[mask])
    s.close()


def test_tensor_core_path_rejects_small_shapes():
    s = hm.Solver()
    A = colmajor(np.ones((32, 32), np.complex64))
    C = colmajor(np.zeros((32, 32), np.complex64))
    with pytest.raises(hm.HmError) as e:
        s.hm_cgemm("N", "N", 1.0, A, A, 0.0, C, path=2)
    assert e.value.status == ARG
    s.close()


def test_stage_autotuner_keeps_the_faster_variant():
    # the first large product of a depth class times both pipeline variants and keeps the
    # faster one; the product itself is still exact to the split-BF16 bound
    rng = np.random.default_rng(11)
    m = n = 3000
    k = 256
    A, B, C0 = rand(rng, m, k), rand(rng, k, n), rand(rng, m, n)
    s = hm.Solver()
    C = colmajor(C0)
    s.hm_cgemm("N", "N", -1.0, colmajor(A), colmajor(B), 1.0, C, path=2)
    st, ms = hm.tc_tuning()
    c = 2  # packed depth 256 = 64 << 2
    assert st[c] in (1, 2, 4), st
    assert np.all(ms[c] > 0), ms
    assert ms[c][{2: 0, 4: 1, 1: 2}[int(st[c])]] <= ms[c].min()
    ref = C0.astype(np.complex128) - A.astype(np.complex128) @ B.astype(np.complex128)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64) + np.abs(C0)
    assert np.max(np.abs(C.cpu().numpy() - ref) / scale) <= 3 * 2.0 ** -16 + (2 * k + 4) * 2.0 ** -24
    s.close()

"""The plane-wave-length complex products (qm_zgemm) in FP64 and in double-FP32 arithmetic,
element by element against a host FP64 product, and the precision form's Davidson with its FP64
phase in either arithmetic against plain FP64.

Bars: FP64 arithmetic within 1e-14 of the host product relative to the bound
sum_k |a_mk| |b_nk| of each element; double-FP32 within 2e-13 of the same bound (its operands
keep 47 significant bits, its products and per-tile sums are exact up to the dropped
a_lo b_lo < 2^-48 |a b|, and the tile sums are added in FP64); both far below FP32's 1e-7.
The BF16x3 tensor-core form (operands rounded to FP32, six BF16 products per product, FP32
accumulation per K split) within 1e-5: FP32 accumulation over 2K real terms gives about
sqrt(2K) 2^-24 (1.5e-6 at K = 316) typically, K 2^-24 at worst.
Davidson: eigenvalues within 1e-9 Ha of the plain FP64 form's.
"""
import numpy as np
import pytest

import qm_synth as S

from cases import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def crandn(rng, *shape, scale=1.0):
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def check(C, ref, bound, tol):
    err = np.abs(C - ref) / bound
    assert err.max() <= tol, err.max()
    return err.max()


@pytest.mark.parametrize("M,N,K", [(70, 45, 40000), (316, 316, 9000), (5, 3, 17)])
def test_cn_fp64_and_double_fp32(Q, M, N, K):
    rng = np.random.default_rng(M + N + K)
    # decaying magnitudes like plane-wave coefficients, plus exact cancellation in the sums
    A = crandn(rng, M, K) * np.exp(-np.linspace(0, 6, K))[None, :]
    B = crandn(rng, N, K, scale=1e-3) * np.exp(-np.linspace(0, 4, K))[None, :]
    ref = np.conj(A) @ B.T
    bound = np.abs(A) @ np.abs(B).T
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    c64 = Q.qm_zgemm("cn", dA, dB, arith=0).cpu().numpy()
    cds = Q.qm_zgemm("cn", dA, dB, arith=1).cpu().numpy()
    ctc = Q.qm_zgemm("cn", dA, dB, arith=2).cpu().numpy()
    check(c64, ref, bound, 1e-14)
    check(cds, ref, bound, 2e-13)
    check(ctc, ref, bound, 1e-5)   # BF16x3 on the tensor cores: FP32-level


def test_double_fp32_across_exponent_range(Q):
    """Operands spread over twenty decades, a few tiny elements and one below FP32's normal
    range (the plain split) keep the 2e-13 bound.  (Double-FP32 products must stay within
    FP32's range, about 1e-38 to 3e38, to keep their relative accuracy; the Davidson's do.)"""
    rng = np.random.default_rng(11)
    M, N, K = 40, 24, 3000
    A = crandn(rng, M, K) * 10.0 ** rng.uniform(-10, 10, (M, 1))
    B = crandn(rng, N, K) * 10.0 ** rng.uniform(-10, 10, (1, K))
    A[:, ::97] *= 1e-25          # a few elements below 2^-74 relative to their row's scale
    B[3, 5] = 1e-39 + 2e-39j     # below FP32's normal range: the plain split
    ref = np.conj(A) @ B.T
    bound = np.abs(A) @ np.abs(B).T
    cds = Q.qm_zgemm("cn", torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), arith=1).cpu().numpy()
    check(cds, ref, bound, 2e-13)


@pytest.mark.parametrize("M,N,K", [(316, 9000, 316), (33, 5000, 950), (2, 7, 3)])
def test_tn_fp64_and_double_fp32(Q, M, N, K):
    rng = np.random.default_rng(3 * M + N + K)
    A = crandn(rng, K, M)
    B = crandn(rng, K, N, scale=1e-2)
    ref = A.T @ B
    bound = np.abs(A).T @ np.abs(B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    c64 = Q.qm_zgemm("tn", dA, dB, arith=0).cpu().numpy()
    cds = Q.qm_zgemm("tn", dA, dB, arith=1).cpu().numpy()
    ctc = Q.qm_zgemm("tn", dA, dB, arith=2).cpu().numpy()
    check(c64, ref, bound, 1e-14)
    check(cds, ref, bound, 2e-13)
    check(ctc, ref, bound, 1e-5)


def test_precision_form_fp64_phase_arithmetic(Q):
    """The precision form (buffer bands: the anchored FP64 phase) with the FP64 phase's long
    products in double-FP32 (default) and in FP64 reaches the plain FP64 eigenvalues."""
    cell = S.cubic_si8(12.0, nbnd=16, reps=(2, 1, 1), kpts=[[0.25, 0.25, 0.25]])
    c = make_case(cell, 0, nb=cell.nbnd + 4)
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        out = {}
        for name, kw in [("fp64", dict(prec="fp64")), ("mixed_ds", dict(prec="mixed", fp64_exact=0)),
                         ("mixed_fp64", dict(prec="mixed", fp64_exact=1))]:
            psi = d(c["psi"])
            eig, info = Q.qm_davidson(g, 0, psi, d(c["v"]), d(c["beta"]), d(c["D"]), tol=1e-9, max_iter=300,
                                      nconv=cell.nbnd, **kw)
            assert info["converged"], (name, info)
            out[name] = eig[:cell.nbnd]
        assert np.abs(out["mixed_ds"] - out["fp64"]).max() <= 1e-9
        assert np.abs(out["mixed_fp64"] - out["fp64"]).max() <= 1e-9
    finally:
        Q.qm_gspace_destroy(g)

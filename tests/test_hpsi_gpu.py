"""Parity of the CUDA H-psi (qm_hpsi through the C ABI) with the FP64 oracle.

Tolerance: FP64 path, per band ||Hpsi_gpu - Hpsi_oracle|| / ||Hpsi_oracle|| <= 1e-11 and
element-wise |diff| <= 1e-11 * max|Hpsi_oracle(band)|.  The mixed path (FP32 FFTs, BF16x3
tensor-core GEMMs accumulated in FP32) is held per band and element-wise: FP32 round-off
(2^-24 = 6e-8) grows by ~log2(N_r) ~ 20 FFT stages and by sqrt(K) in the FP32 sums of the
projections over K = 2 npw terms.  Measured maxima: per band 5e-8 .. 3e-7 and element-wise
(relative to the band's largest element) 8e-8 .. 1.3e-6 on the cells up to 72^3 and 18k plane
waves; 3.5e-6 / 2.4e-5 and 5.5e-6 / 2.4e-5 on the 255- and 216-atom cells (96k and 44k plane
waves).  Bars: 1e-6 per band and 5e-6 element-wise up to 72^3, 1e-5 and 5e-5 beyond.
"""
import numpy as np
import pytest

import qm_synth as S
from oracle import hamiltonian as OH

from cases import band_rel_err, make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL_MIXED = 1e-6          # per band, cells up to 72^3
TOL_MIXED_ELEM = 5e-6     # element-wise, relative to the band's largest element
TOL_MIXED_LARGE = 1e-5    # per band, the 216- and 255-atom cells
TOL_MIXED_LARGE_ELEM = 5e-5


def check_mixed(got, want, large=False):
    rel = band_rel_err(got, want)
    scale = np.abs(want).max(axis=1, keepdims=True)
    el = (np.abs(got - want) / scale).max()
    tb, te = (TOL_MIXED_LARGE, TOL_MIXED_LARGE_ELEM) if large else (TOL_MIXED, TOL_MIXED_ELEM)
    assert rel.max() <= tb and el <= te, (rel.max(), el)
    return rel.max(), el


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_hpsi(Q, g, ik, c, psi=None, prec="fp64", ld_pad=0, with_nl=True, v=None):
    psi = c["psi"] if psi is None else psi
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    npw = psi.shape[1]
    p = torch.zeros((psi.shape[0], npw + ld_pad), dtype=cdt, device="cuda")
    p[:, :npw] = dev(psi, cdt)
    beta = dev(c["beta"], cdt) if with_nl else None
    D = dev(c["D"]) if with_nl else None
    out = torch.zeros_like(p)
    Q.qm_hpsi(g, ik, p, dev(c["v"] if v is None else v), beta, D, out=out, prec=prec)
    torch.cuda.synchronize()
    return out[:, :npw].cpu().numpy().astype(np.complex128)


def check64(got, want):
    rel = band_rel_err(got, want)
    assert rel.max() <= TOL64, rel.max()
    scale = np.abs(want).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - want) <= TOL64 * scale)
    return rel.max()


def _gspace(Q, cell):
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    return g


@pytest.mark.parametrize("cell", S.small_cells() + [S.config1()], ids=lambda c: f"{c.name}_{c.ecutwfc_ry:g}Ry")
def test_hpsi_fp64_matches_oracle(Q, cell):
    g = _gspace(Q, cell)
    try:
        for ik in range(len(cell.kpts)):
            c = make_case(cell, ik)
            idx, _, _ = Q.qm_gspace_indices(g, ik)
            np.testing.assert_array_equal(idx, c["gs"]["idx"])
            want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
            got = gpu_hpsi(Q, g, ik, c)
            check64(got, want)
            if np.prod(c["grid"]) <= 14000:
                naive = OH.hpsi_naive(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
                check64(got, naive)
    finally:
        Q.qm_gspace_destroy(g)


def test_hpsi_padded_rows_and_local_only(Q):
    cell = S.cubic_si8(12.0, nbnd=7, reps=(2, 1, 1), kpts=[[0.25, 0.25, -0.25]])
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, 0)
        want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
        check64(gpu_hpsi(Q, g, 0, c, ld_pad=5), want)
        want_loc = OH.hpsi_fft(c["psi"], c["gs"], c["v"], None, None)
        check64(gpu_hpsi(Q, g, 0, c, with_nl=False, ld_pad=3), want_loc)
        one = c["psi"][:1]
        check64(gpu_hpsi(Q, g, 0, c, psi=one), OH.hpsi_fft(one, c["gs"], c["v"], c["beta"], c["D"]))
    finally:
        Q.qm_gspace_destroy(g)


def _full_size_cells():
    return [(S.config2(), 0), (S.config2(), 3), (S.config4(), 0), (S.config5(), 0)]


@pytest.mark.parametrize("cell,ik", _full_size_cells(), ids=lambda x: getattr(x, "name", str(x)))
def test_hpsi_fp64_full_size_sampled_bands(Q, cell, ik):
    """All bands in the benchmark's launch configuration; sampled bands (first, chunk
    boundaries, last) computed one by one by the oracle."""
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, ik)
        got = gpu_hpsi(Q, g, ik, c)
        nb = cell.nbnd
        sample = sorted({0, 1, nb // 3, nb // 3 + 1, nb // 2, nb - 2, nb - 1})
        want = OH.hpsi_fft(c["psi"][sample], c["gs"], c["v"], c["beta"], c["D"])
        check64(got[sample], want)
    finally:
        Q.qm_gspace_destroy(g)


def test_hpsi_full_size_properties(Q):
    """Properties that hold at any size: V = 0 and no projectors gives exactly 1/2|k+G|^2 psi;
    a constant V0 adds V0 psi; <phi|H psi> = conj(<psi|H phi>)."""
    cell = S.config2()
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, 1, nb=24)
        zero = np.zeros_like(c["v"])
        got = gpu_hpsi(Q, g, 1, c, with_nl=False, v=zero)
        # exact up to the rounding of 1/2|k+G|^2, which the host C++ and numpy evaluate in a
        # different order (a few ulps)
        want = c["gs"]["kin"] * c["psi"]
        assert np.all(np.abs(got - want) <= 2e-15 * np.abs(want))
        v0 = -0.37
        shifted = gpu_hpsi(Q, g, 1, c, v=c["v"] + v0)
        base = gpu_hpsi(Q, g, 1, c)
        assert np.abs(shifted - base - v0 * c["psi"]).max() < 1e-12
        hphi = base
        phi = c["psi"]
        psi2 = S.psi_random(99, 24, phi.shape[1])
        hpsi2 = gpu_hpsi(Q, g, 1, c, psi=psi2)
        lhs = phi.conj() @ hpsi2.T
        rhs = (psi2.conj() @ hphi.T).T.conj()
        assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(lhs).max()
    finally:
        Q.qm_gspace_destroy(g)


def test_hpsi_deterministic(Q):
    cell = S.config2()
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, 2, nb=40)
        a = gpu_hpsi(Q, g, 2, c)
        b = gpu_hpsi(Q, g, 2, c)
        np.testing.assert_array_equal(a, b)
    finally:
        Q.qm_gspace_destroy(g)


@pytest.mark.parametrize("cell,ik,nb", [(S.config1(), 0, None), (S.config2(), 0, 48)],
                         ids=["config1", "config2_k0"])
def test_hpsi_mixed_precision_error(Q, cell, ik, nb):
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, ik, nb=nb)
        want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
        got = gpu_hpsi(Q, g, ik, c, prec="mixed")
        rel, el = check_mixed(got, want)
        print(f"mixed H-psi max per-band relative error {rel:.3e}, element-wise {el:.3e}")
    finally:
        Q.qm_gspace_destroy(g)


def test_hpsi_argument_errors_on_device(Q):
    cell = S.config1()
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, 0)
        psi = dev(c["psi"])
        with pytest.raises(Q.QMError):                      # out overlaps psi
            Q.qm_hpsi(g, 0, psi, dev(c["v"]), dev(c["beta"]), dev(c["D"]), out=psi)
        with pytest.raises(ValueError):                     # host tensors are refused
            Q.qm_hpsi(g, 0, torch.from_numpy(c["psi"]), dev(c["v"]), None, None)
        with pytest.raises(Q.QMError):                      # wrong k index
            Q.qm_hpsi(g, 3, psi, dev(c["v"]), None, None)
    finally:
        Q.qm_gspace_destroy(g)


@pytest.mark.parametrize("cell", S.small_cells(), ids=lambda c: f"{c.name}_{c.ecutwfc_ry:g}Ry")
def test_hpsi_mixed_small_cells(Q, cell):
    """Precision form on the small cells (runtime-plan lengths, radix 5, N1 != N2, k != 0)."""
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, 0)
        want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
        check_mixed(gpu_hpsi(Q, g, 0, c, prec="mixed"), want)
    finally:
        Q.qm_gspace_destroy(g)


def test_hpsi_mixed_padded_rows_local_only_and_repeatable(Q):
    cell = S.cubic_si8(12.0, nbnd=7, reps=(2, 1, 1), kpts=[[0.25, 0.25, -0.25]])
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, 0)
        want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
        a = gpu_hpsi(Q, g, 0, c, prec="mixed", ld_pad=5)
        check_mixed(a, want)
        b = gpu_hpsi(Q, g, 0, c, prec="mixed", ld_pad=5)
        np.testing.assert_array_equal(a, b)             # the two streams give a fixed result
        want_loc = OH.hpsi_fft(c["psi"], c["gs"], c["v"], None, None)
        check_mixed(gpu_hpsi(Q, g, 0, c, prec="mixed", with_nl=False, ld_pad=3), want_loc)
    finally:
        Q.qm_gspace_destroy(g)


@pytest.mark.parametrize("cell,ik", _full_size_cells(), ids=lambda x: getattr(x, "name", str(x)))
def test_hpsi_mixed_full_size_sampled_bands(Q, cell, ik):
    """Precision form with every band in one call (the benchmark's launch configuration: one
    stick buffer for all bands, the tensor-core nonlocal part overlapped on the second stream);
    sampled bands against the oracle."""
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, ik)
        got = gpu_hpsi(Q, g, ik, c, prec="mixed")
        nb = cell.nbnd
        sample = sorted({0, 1, nb // 2, nb - 2, nb - 1})
        want = OH.hpsi_fft(c["psi"][sample], c["gs"], c["v"], c["beta"], c["D"])
        rel, el = check_mixed(got[sample], want, large=cell.nat > 64)
        print(f"{cell.name} k{ik}: mixed max sampled band rel err {rel:.2e}, element-wise {el:.2e}")
    finally:
        Q.qm_gspace_destroy(g)


@pytest.mark.parametrize("cellf,ik,nb", [(S.config1, 0, None), (S.config2, 3, 160)], ids=["config1", "config2_k3_full"])
def test_hpsi_prepared_projectors_identical(Q, cellf, ik, nb):
    """qm_hpsi_prepare splits the projectors once; qm_hpsi(QM_MIXED) with the prepared beta gives
    bit-identical results to the call that splits beta itself, and releasing restores the
    per-call path."""
    cell = cellf()
    g = _gspace(Q, cell)
    try:
        c = make_case(cell, ik, nb=nb)
        psi = dev(c["psi"], torch.complex64)
        beta = dev(c["beta"], torch.complex64)
        v, D = dev(c["v"]), dev(c["D"])
        a = Q.qm_hpsi(g, ik, psi, v, beta, D, prec="mixed").clone()
        Q.qm_hpsi_prepare(g, ik, beta)
        b = Q.qm_hpsi(g, ik, psi, v, beta, D, prec="mixed").clone()
        beta2 = beta.clone()                              # another buffer: not the prepared one
        b2 = Q.qm_hpsi(g, ik, psi, v, beta2, D, prec="mixed").clone()
        Q.qm_hpsi_prepare(g, ik, None)
        d = Q.qm_hpsi(g, ik, psi, v, beta, D, prec="mixed").clone()
        torch.cuda.synchronize()
        assert torch.equal(a, b) and torch.equal(a, b2) and torch.equal(a, d)
    finally:
        Q.qm_gspace_destroy(g)

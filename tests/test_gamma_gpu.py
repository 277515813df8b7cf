"""Parity of the Gamma-point real-wavefunction H psi (qm_hpsi_gamma through the C ABI: two bands
per FFT, separated after the forward transform) with the FP64 oracle's H psi of each band.

Tolerances: those of qm_hpsi (tests/test_hpsi_gpu.py): FP64 1e-11 per band and element-wise
(relative to the band's largest element); precision form 1e-6 / 5e-6 up to 72^3 and 1e-5 / 5e-5
on the 216-atom cell.  Inputs are real-space-real states (qm_synth.psi_random_real).
"""
import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG
from oracle import hamiltonian as OH

from cases import band_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-11


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


def gamma_case(cell, nb, seed=21):
    grid = cell.grid or OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    gs = OG.gsphere(cell.lattice, grid, cell.ecut_ha, [0.0, 0.0, 0.0])
    v = S.vloc_on_grid(cell.lattice, cell.tau, gs["grid"])
    beta = S.beta_of_q(gs["q"], cell.tau, cell.omega)
    D = S.dvals(cell.nat)
    psi = S.psi_random_real(seed, nb, gs["miller"])
    return {"gs": gs, "v": v, "beta": beta, "D": D, "psi": psi, "grid": gs["grid"]}


def gpu_gamma(Q, g, c, prec="fp64", ld_pad=0, with_nl=True, psi=None, stream=None):
    psi = c["psi"] if psi is None else psi
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    nb, npw = psi.shape
    p = torch.zeros((nb, npw + ld_pad), dtype=cdt, device="cuda")
    p[:, :npw] = dev(psi, cdt)
    out = torch.full_like(p, float("nan"))
    beta = dev(c["beta"], cdt) if with_nl else None
    D = dev(c["D"]) if with_nl else None
    Q.qm_hpsi_gamma(g, 0, p, dev(c["v"]), beta, D, out=out, prec=prec, stream=stream)
    torch.cuda.synchronize()
    return out[:, :npw].cpu().numpy().astype(np.complex128)


def check(got, want, prec, large=False):
    if prec == "fp64":
        tb = te = TOL64
    else:
        tb, te = (1e-5, 5e-5) if large else (1e-6, 5e-6)
    rel = band_rel_err(got, want).max()
    el = (np.abs(got - want) / np.abs(want).max(axis=1, keepdims=True)).max()
    assert rel <= tb and el <= te, (prec, rel, el)
    return rel, el


_GAMMA_CELLS = [S.fcc_si2(8.0, nbnd=4), S.fcc_si2(30.0, nbnd=3), S.cubic_si8(10.0, nbnd=6), S.config1(),
                S.cubic_si8(12.0, nbnd=5, reps=(2, 1, 1))]


@pytest.mark.parametrize("cell", _GAMMA_CELLS, ids=lambda c: f"{c.name}_{c.ecutwfc_ry:g}Ry_nb{c.nbnd}")
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gamma_matches_oracle(Q, cell, prec):
    c = gamma_case(cell, cell.nbnd)
    g = Q.qm_gspace_create(cell.lattice, [[0, 0, 0]], cell.ecut_ha, cell.grid)
    try:
        idx, _, _ = Q.qm_gspace_indices(g, 0)
        np.testing.assert_array_equal(idx, c["gs"]["idx"])
        want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
        check(gpu_gamma(Q, g, c, prec), want, prec)
    finally:
        Q.qm_gspace_destroy(g)


def test_gamma_padded_rows_local_only_single_band_side_stream(Q):
    cell = S.cubic_si8(12.0, nbnd=7, reps=(2, 1, 1))
    c = gamma_case(cell, 7)
    g = Q.qm_gspace_create(cell.lattice, [[0, 0, 0]], cell.ecut_ha, cell.grid)
    try:
        s = torch.cuda.Stream()
        want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
        for prec in ("fp64", "mixed"):
            check(gpu_gamma(Q, g, c, prec, ld_pad=5, stream=s), want, prec)
            want_loc = OH.hpsi_fft(c["psi"], c["gs"], c["v"], None, None)
            check(gpu_gamma(Q, g, c, prec, ld_pad=3, with_nl=False), want_loc, prec)
            one = c["psi"][:1]
            check(gpu_gamma(Q, g, c, prec, psi=one), want[:1], prec)
    finally:
        Q.qm_gspace_destroy(g)


def test_gamma_equals_complex_path(Q):
    """The two-bands-per-transform result equals qm_hpsi of the same bands (FP64, 1e-12)."""
    cell = S.config1()
    c = gamma_case(cell, 8)
    g = Q.qm_gspace_create(cell.lattice, [[0, 0, 0]], cell.ecut_ha, cell.grid)
    try:
        p = dev(c["psi"])
        args = (dev(c["v"]), dev(c["beta"]), dev(c["D"]))
        a = Q.qm_hpsi_gamma(g, 0, p, *args).cpu().numpy()
        b = Q.qm_hpsi(g, 0, p, *args).cpu().numpy()
        assert (np.abs(a - b) / np.abs(b).max(axis=1, keepdims=True)).max() <= 1e-12
    finally:
        Q.qm_gspace_destroy(g)


def test_gamma_216_atom_cell_full_size(Q):
    """The 216-atom cell (90^3, Gamma, 43,819 plane waves) at full size: 75 bands (an odd count)
    in FP64, where the stick buffer holds 23 band pairs per chunk (38 transforms: chunks of 23
    and 15, the last band alone in its transform), and 9 bands in the precision form."""
    cell = S.config4()
    c = gamma_case(cell, 75)
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
        check(gpu_gamma(Q, g, c, "fp64"), want, "fp64")
        check(gpu_gamma(Q, g, c, "mixed", psi=c["psi"][:9]), want[:9], "mixed", large=True)
    finally:
        Q.qm_gspace_destroy(g)

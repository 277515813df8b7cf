"""Parity of the CUDA GW plane-wave matrix elements (qm_gw_mel through the C ABI) with the FP64
oracle (oracle/gw.py: the real-space route on numpy FFTs, and the direct Miller-index sum).

Tolerances: FP64 element-wise |diff| <= 1e-11 * max|M(pair)| (the H psi bar); precision form
(FP32 transforms): per pair ||diff|| / ||M|| <= 1e-6 and element-wise 5e-6 relative to the pair's
largest element, the H psi bars of the FP32 FFT path.
"""
import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG
from oracle import gw as OW

from cases import band_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def check(got, want, prec):
    scale = np.abs(want).max(axis=1, keepdims=True)
    el = (np.abs(got - want) / scale).max()
    if prec == "fp64":
        assert el <= 1e-11, el
    else:
        rel = band_rel_err(got, want).max()
        assert rel <= 1e-6 and el <= 5e-6, (rel, el)
    return el


def run_case(Q, cell, k, q, eps_frac, nl, nr, precs=("fp64", "mixed"), pad=0, direct=False):
    grid = tuple(cell.grid) if cell.grid else OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    k, q = np.asarray(k, float), np.asarray(q, float)
    same = not q.any()
    kpts = [k] if same else [k + q, k]
    g = Q.qm_gspace_create(cell.lattice, kpts, cell.ecut_ha, grid)
    ge = Q.qm_gspace_create(cell.lattice, [q], eps_frac * cell.ecut_ha, grid)
    try:
        gs_l = OG.gsphere(cell.lattice, grid, cell.ecut_ha, kpts[0])
        gs_r = OG.gsphere(cell.lattice, grid, cell.ecut_ha, kpts[-1])
        gse = OG.gsphere(cell.lattice, grid, eps_frac * cell.ecut_ha, q)
        np.testing.assert_array_equal(Q.qm_gspace_indices(ge, 0)[0], gse["idx"])
        cl = S.psi_random(41, nl, len(gs_l["idx"]))
        cr = S.psi_random(42, nr, len(gs_r["idx"]))
        want = OW.mel_fft(cl, gs_l, cr, gs_r, gse)
        if direct:
            np.testing.assert_allclose(OW.mel_direct(cl, gs_l, cr, gs_r, gse), want, rtol=0,
                                       atol=1e-12 * np.abs(want).max())
        npe = len(gse["idx"])
        for prec in precs:
            cdt = torch.complex128 if prec == "fp64" else torch.complex64
            pl = torch.zeros((nl, cl.shape[1] + pad), dtype=cdt, device="cuda")
            pl[:, :cl.shape[1]] = dev(cl, cdt)
            M = torch.full((nl * nr, npe + pad), float("nan"), dtype=cdt, device="cuda")
            Q.qm_gw_mel(g, 0, len(kpts) - 1, pl, dev(cr, cdt), ge, 0, npe, M=M, prec=prec)
            torch.cuda.synchronize()
            check(M[:, :npe].cpu().numpy().astype(np.complex128), want, prec)
    finally:
        Q.qm_gspace_destroy(ge)
        Q.qm_gspace_destroy(g)


def test_gw_small_cell_matches_oracle(Q):
    run_case(Q, S.fcc_si2(10.0), [0.25, -0.25, 0.25], [-0.5, 0.25, 0.0], 0.6, 3, 2, direct=True)


def test_gw_q0_overlap_and_padded_rows(Q):
    run_case(Q, S.fcc_si2(12.0), [0.25, 0.25, -0.25], [0.0, 0.0, 0.0], 0.5, 4, 4, pad=3)


def test_gw_radix5_grid_and_unequal_axes(Q):
    run_case(Q, S.cubic_si8(12.0, reps=(2, 1, 1)), [0.25, 0.25, -0.25], [-0.5, 0.0, 0.5], 0.4, 2, 5)


def test_gw_64_atom_cell_full_size(Q):
    """The 64-atom cell (72^3 grid, 18k plane waves per k-point): k and k+q two points of its shifted
    2x2x2 set, E_eps a quarter of the wavefunction cutoff, 4 x 3 pairs."""
    cell = S.config2()
    k = cell.kpts[0]
    run_case(Q, cell, k, cell.kpts[1] - k, 0.25, 4, 3)

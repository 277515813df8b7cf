"""Parity of the Davidson residual and correction steps (qm_precond_apply through the C ABI:
the k_residual, k_tpa and learned-network kernels of qm_davidson) with the FP64 oracle,
element by element.

Inputs come from the oracle only: X are seeded complex normal blocks, HX = oracle H X, eps the
Rayleigh quotients.  Bars:
  r_n, delta_n (TPA)  |gpu - oracle| <= 1e-12 max|oracle row| element-wise (FP64; the only
                      differences are fused multiply-adds and the order of the T_n sums);
  ||r_n||^2, T_n      1e-13 relative;
  delta_n (learned)   within 2e-3 of the oracle network evaluated with the kernels' BF16
                      roundings for all but 1e-4 of the elements and within 8e-3 (two BF16
                      units) for every element, and within 5e-2 of the plain FP64 oracle network,
                      relative to each element (the network runs in BF16 with FP32 accumulation).
"""
import numpy as np
import pytest

import qm_synth as S
from oracle import hamiltonian as OH
from oracle import mlp as M
from oracle import precond as OP

from cases import make_case
from test_mlp_gpu import forward_bf16, rand_theta

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def oracle_inputs(cell, ik, nb):
    c = make_case(cell, ik, nb=nb)
    X = c["psi"]
    HX = OH.hpsi_fft(X, c["gs"], c["v"], c["beta"], c["D"])
    eps = np.real(np.einsum("ng,ng->n", X.conj(), HX)) / np.real(np.einsum("ng,ng->n", X.conj(), X))
    return c, X, HX, eps


def run_gpu(Q, cell, ik, X, HX, eps, mlp=None, ld_pad=0, hdiag=None):
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        n, npw = X.shape
        Xd = torch.zeros((n, npw + ld_pad), dtype=torch.complex128, device="cuda")
        HXd = torch.zeros_like(Xd)
        Xd[:, :npw] = torch.from_numpy(X).cuda()
        HXd[:, :npw] = torch.from_numpy(HX).cuda()
        th = None if mlp is None else torch.from_numpy(np.asarray(mlp, np.float32)).cuda()
        hd = None if hdiag is None else torch.from_numpy(hdiag).cuda()
        R, d, rn2, tk = Q.qm_precond_apply(g, ik, Xd, HXd, torch.from_numpy(eps).cuda(), mlp=th, hdiag=hd)
        torch.cuda.synchronize()
        return (R[:, :npw].cpu().numpy(), d[:, :npw].cpu().numpy(), rn2.cpu().numpy(), tk.cpu().numpy())
    finally:
        Q.qm_gspace_destroy(g)


def check_rows(got, want, tol):
    scale = np.abs(want).max(axis=1, keepdims=True)
    err = np.abs(got - want) / scale
    assert err.max() <= tol, err.max()


CASES = [(S.config1, 0, 8, 0), (S.config1, 0, 3, 5),                    # 411 plane waves: a ragged tail
         (lambda: S.cubic_si8(12.0, nbnd=7, kpts=[[0.25, 0.25, 0.25]]), 0, 7, 2),
         (S.config2, 1, 160, 0)]                                          # full size, one k-point


@pytest.mark.parametrize("cellf,ik,nb,ld_pad", CASES, ids=["cfg1", "cfg1_padded", "si8_k", "cfg2_k1_full"])
def test_residual_and_tpa_match_oracle(Q, cellf, ik, nb, ld_pad):
    cell = cellf()
    c, X, HX, eps = oracle_inputs(cell, ik, nb)
    R, d, rn2, tk = run_gpu(Q, cell, ik, X, HX, eps, ld_pad=ld_pad)
    kin = c["gs"]["kin"]
    r_o = HX - eps[:, None] * X
    d_o = OP.tpa_apply(r_o, X, kin)
    w = np.abs(X) ** 2
    tk_o = (w * kin[None, :]).sum(axis=1) / w.sum(axis=1)
    check_rows(R, r_o, 1e-12)
    check_rows(d, d_o, 1e-12)
    np.testing.assert_allclose(rn2, (np.abs(r_o) ** 2).sum(axis=1), rtol=1e-13)
    np.testing.assert_allclose(tk, tk_o, rtol=1e-13)


@pytest.mark.parametrize("cellf,ik,nb", [(S.config1, 0, 8), (S.config2, 2, 160)], ids=["cfg1", "cfg2_k2_full"])
def test_learned_correction_matches_oracle(Q, cellf, ik, nb):
    cell = cellf()
    c, X, HX, eps = oracle_inputs(cell, ik, nb)
    th = rand_theta(7)
    kin = c["gs"]["kin"]
    hd = M.hamiltonian_diagonal(kin, c["v"], c["beta"], c["D"])
    R, d, rn2, tk = run_gpu(Q, cell, ik, X, HX, eps, mlp=th, hdiag=hd)
    r_o = HX - eps[:, None] * X
    F = M.features(kin, X, eps, hd)
    Ke = forward_bf16(th, F).reshape(r_o.shape)
    Ko = M.forward(th, F)[0].reshape(r_o.shape)
    nz = np.abs(r_o) > 0
    rel = np.abs(d - Ke * r_o)[nz] / np.abs(Ke * r_o)[nz]
    # FP32 sums inside the network can flip the BF16 rounding of a hidden activation relative to
    # the FP64 emulation: rare, and worth at most about one BF16 unit (2^-8) of K
    assert rel.max() < 8e-3 and np.quantile(rel, 0.9999) < 2e-3, (rel.max(), np.quantile(rel, 0.9999))
    assert np.max(np.abs(d - Ko * r_o)[nz] / np.abs(Ko * r_o)[nz]) < 5e-2
    check_rows(R, r_o, 1e-12)


def test_zero_bands_is_a_noop(Q):
    cell = S.config1()
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        e = torch.zeros((0, 411), dtype=torch.complex128, device="cuda")
        R, d, rn2, tk = Q.qm_precond_apply(g, 0, e, e, torch.zeros(0, dtype=torch.float64, device="cuda"))
        assert R.shape == (0, 411) and d.shape == (0, 411)
    finally:
        Q.qm_gspace_destroy(g)


@pytest.mark.parametrize("cellf,ik", [(S.config1, 0), (S.config2, 1)], ids=["cfg1", "cfg2_k1"])
def test_hamiltonian_diagonal_matches_oracle(Q, cellf, ik):
    """qm_hamiltonian_diag (the third feature's H_GG) against the oracle's diagonal, which is
    pinned to the brute-force H_GG'; with and without projectors."""
    cell = cellf()
    c = make_case(cell, ik, nb=1)
    kin = c["gs"]["kin"]
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        v, beta, D = (torch.from_numpy(a).cuda() for a in (c["v"], c["beta"], c["D"]))
        for b, dd in ((beta, D), (None, None)):
            got = Q.qm_hamiltonian_diag(g, ik, v, b, dd).cpu().numpy()
            want = M.hamiltonian_diagonal(kin, c["v"], None if b is None else c["beta"], None if b is None else c["D"])
            np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())
    finally:
        Q.qm_gspace_destroy(g)

"""CPU checks behind the Gamma-point real-wavefunction form (qm_hpsi_gamma): the synthetic
real-space-real states, the oracle Hamiltonian keeping that property at k = 0, and the
separation of two bands transformed together (the identity the GPU form relies on), all on the
oracle's own full-box transforms."""
import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG
from oracle import hamiltonian as OH


def _gamma_case(cell, nb=3, seed=11):
    grid = cell.grid or OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    gs = OG.gsphere(cell.lattice, grid, cell.ecut_ha, [0.0, 0.0, 0.0])
    v = S.vloc_on_grid(cell.lattice, cell.tau, gs["grid"])
    beta = S.beta_of_q(gs["q"], cell.tau, cell.omega)
    D = S.dvals(cell.nat)
    psi = S.psi_random_real(seed, nb, gs["miller"])
    return gs, v, beta, D, psi


def _minus(gs):
    pos = {tuple(r): i for i, r in enumerate(gs["miller"].tolist())}
    return np.array([pos[(-a, -b, -c)] for a, b, c in gs["miller"].tolist()])


def _to_box(gs, c):
    n1, n2, n3 = gs["grid"]
    box = np.zeros((c.shape[0], n1 * n2 * n3), complex)
    box[:, gs["idx"]] = c
    return np.fft.ifftn(box.reshape(-1, n3, n2, n1), axes=(1, 2, 3)).reshape(c.shape[0], -1)


@pytest.mark.parametrize("cell", [S.fcc_si2(12.0), S.cubic_si8(10.0)], ids=["fcc_si2", "cubic_si8"])
def test_real_states_and_h_keeps_them_real(cell):
    gs, v, beta, D, psi = _gamma_case(cell)
    neg = _minus(gs)
    np.testing.assert_array_equal(psi[:, neg], psi.conj())
    r = _to_box(gs, psi)
    assert np.abs(r.imag).max() <= 1e-15 * np.abs(r.real).max()
    hp = OH.hpsi_fft(psi, gs, v, beta, D)
    np.testing.assert_allclose(hp[:, neg], hp.conj(), rtol=0, atol=1e-12 * np.abs(hp).max())
    H = OH.dense_h(gs, v, beta, D)
    np.testing.assert_allclose(H[np.ix_(neg, neg)], H.conj(), rtol=0, atol=1e-13)


def test_two_bands_in_one_transform_separate():
    """F = fftn(V ifftn(psi_a + i psi_b)) on the box: (F(G) + conj F(-G))/2 and
    (F(G) - conj F(-G))/(2i) are the local products of psi_a and psi_b on their own."""
    cell = S.fcc_si2(14.0)
    gs, v, beta, D, psi = _gamma_case(cell, nb=2)
    neg = _minus(gs)
    n1, n2, n3 = gs["grid"]
    shp = (n3, n2, n1)

    def local(c):
        box = np.zeros((c.shape[0], n1 * n2 * n3), complex)
        box[:, gs["idx"]] = c
        r = np.fft.ifftn(box.reshape((-1,) + shp), axes=(1, 2, 3)) * v.reshape(shp)[None]
        return np.fft.fftn(r, axes=(1, 2, 3)).reshape(c.shape[0], -1)[:, gs["idx"]]

    F = local(psi[:1] + 1j * psi[1:2])[0]
    want = local(psi)
    a = 0.5 * (F + F[neg].conj())
    b = (F - F[neg].conj()) / 2j
    np.testing.assert_allclose(a, want[0], rtol=0, atol=1e-13 * np.abs(want).max())
    np.testing.assert_allclose(b, want[1], rtol=0, atol=1e-13 * np.abs(want).max())
    # and the same separation fails for states that are not real in real space
    z = S.psi_random(12, 2, len(gs["idx"]))
    Fz = local(z[:1] + 1j * z[1:2])[0]
    assert np.abs(0.5 * (Fz + Fz[neg].conj()) - local(z)[0]).max() > 1e-3 * np.abs(Fz).max()

"""Pins of the oracle's GW plane-wave matrix elements (oracle/gw.py, Section 5 "gw" module)
against closed forms, the overlap they reduce to, their conjugation symmetry, and each other."""
import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG
from oracle import gw as OW

K = np.array([0.25, -0.25, 0.25])
Q = np.array([-0.5, 0.25, 0.0])


def _spheres(cell, k, q, ecut_eps):
    grid = OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    gs_r = OG.gsphere(cell.lattice, grid, cell.ecut_ha, k)
    gs_l = OG.gsphere(cell.lattice, grid, cell.ecut_ha, k + q)
    ge = OG.gsphere(cell.lattice, grid, ecut_eps, q)
    return gs_l, gs_r, ge


@pytest.mark.parametrize("q", [np.zeros(3), Q], ids=["q0", "q"])
def test_direct_sum_equals_fft(q):
    cell = S.fcc_si2(10.0)
    gs_l, gs_r, ge = _spheres(cell, K, q, 0.6 * cell.ecut_ha)
    cl = S.psi_random(31, 3, len(gs_l["idx"]))
    cr = S.psi_random(32, 2, len(gs_r["idx"]))
    a = OW.mel_direct(cl, gs_l, cr, gs_r, ge)
    b = OW.mel_fft(cl, gs_l, cr, gs_r, ge)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-12 * np.abs(a).max())


def test_single_plane_waves():
    """c_l = alpha at G_a (sphere of k+q), c_r = beta at G_b (sphere of k): M(G) = conj(alpha) beta
    at G = G_a - G_b and 0 elsewhere (fixes the orientation G + G2 and the conjugated factor)."""
    cell = S.fcc_si2(10.0)
    gs_l, gs_r, ge = _spheres(cell, K, Q, cell.ecut_ha)
    alpha, beta = 0.3 - 0.7j, -1.1 + 0.4j
    ia, ib = int(np.argmin(gs_l["kin"])), int(np.argsort(gs_r["kin"])[3])   # short vectors: G_a - G_b on the q sphere
    cl = np.zeros((1, len(gs_l["idx"])), complex)
    cr = np.zeros((1, len(gs_r["idx"])), complex)
    cl[0, ia] = alpha
    cr[0, ib] = beta
    target = tuple(gs_l["miller"][ia] - gs_r["miller"][ib])
    want = np.zeros((1, len(ge["idx"])), complex)
    hits = [i for i, m in enumerate(ge["miller"].tolist()) if tuple(m) == target]
    assert hits, "G_a - G_b must lie on the sphere of q for this pin"
    want[0, hits[0]] = np.conj(alpha) * beta
    for f in (OW.mel_direct, OW.mel_fft):
        np.testing.assert_allclose(f(cl, gs_l, cr, gs_r, ge), want, rtol=0, atol=1e-14)


def test_q0_g0_is_the_overlap_matrix():
    """q = 0, G = 0: M_nn'(0) = <n|n'>, the identity for orthonormal states."""
    cell = S.fcc_si2(10.0)
    gs_l, gs_r, ge = _spheres(cell, K, np.zeros(3), 0.5 * cell.ecut_ha)
    c = S.psi_random(33, 4, len(gs_r["idx"]))
    q, _ = np.linalg.qr(c.T)
    c = q.T
    i0 = int(np.where((ge["miller"] == 0).all(1))[0][0])
    for f in (OW.mel_direct, OW.mel_fft):
        m = f(c, gs_l, c, gs_r, ge)[:, i0].reshape(4, 4)
        np.testing.assert_allclose(m, np.eye(4), atol=1e-13)


def test_conjugation_symmetry():
    """Swapping the states' roles (k+q <-> k, q -> -q, G -> -G) conjugates M:
    M_{n'n}(k+q, -q, -G) = conj(M_nn'(k, q, G))."""
    cell = S.fcc_si2(10.0)
    gs_l, gs_r, ge = _spheres(cell, K, Q, 0.7 * cell.ecut_ha)
    ge_m = OG.gsphere(cell.lattice, ge["grid"], 0.7 * cell.ecut_ha, -Q)
    cl = S.psi_random(34, 2, len(gs_l["idx"]))
    cr = S.psi_random(35, 3, len(gs_r["idx"]))
    m = OW.mel_fft(cl, gs_l, cr, gs_r, ge).reshape(2, 3, -1)
    s = OW.mel_fft(cr, gs_r, cl, gs_l, ge_m).reshape(3, 2, -1)
    pos = {tuple(x): i for i, x in enumerate(ge_m["miller"].tolist())}
    neg = np.array([pos[(-a, -b, -c)] for a, b, c in ge["miller"].tolist()])
    np.testing.assert_allclose(s[:, :, neg].transpose(1, 0, 2), m.conj(), rtol=0, atol=1e-13 * np.abs(m).max())

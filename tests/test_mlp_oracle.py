"""Pins of the learned-preconditioner oracle (oracle/mlp.py) against things other than itself:
central finite differences of the loss, closed forms of degenerate networks, invariances of the
features and the loss, and the defining properties of the exact correction on a cell solved by
brute-force diagonalisation."""
import math

import numpy as np
import pytest

import qm_synth as S
from oracle import hamiltonian as OH
from oracle import mlp as M
from oracle.precond import tpa_k

from cases import make_case


def random_data(seed, nb=4, npw=23):
    rng = np.random.default_rng(seed)
    F = np.stack([rng.uniform(0, 4, nb * npw), np.repeat(rng.uniform(-1, 1, nb), npw),
                  rng.normal(0, 1, nb * npw)], axis=1)
    r2 = rng.uniform(0.01, 1.0, nb * npw)
    c = rng.normal(0, 1, nb * npw)
    D = rng.uniform(0.5, 2.0, nb)
    D[1] = 0.0                                           # excluded band
    off = np.arange(0, nb * npw + 1, npw)
    return F, r2, c, D, off


def test_param_count_and_layout():
    assert M.NPARAM == 4481
    th = np.arange(M.NPARAM, dtype=float)
    W1, b1, W2, b2, w3, b3 = M.unpack(th)
    assert W1.shape == (64, 3) and W1[1, 0] == 3 and b1[0] == 192 and W2[0, 1] == 257
    assert b2[0] == 192 + 64 + 4096 and w3[0] == b2[0] + 64 and b3 == M.NPARAM - 1


def test_loss_gradient_matches_central_differences():
    F, r2, c, D, off = random_data(1)
    W = np.random.default_rng(11).uniform(0.1, 1.0, D.size)
    th = M.init_params(3)
    th[192:256] = 0.1                                    # nonzero b1
    th[-1] = 0.3
    loss, g = M.loss_and_grad(th, F, r2, c, D, off, W)
    rng = np.random.default_rng(7)
    blocks = [(0, 192), (192, 256), (256, 4352), (4352, 4416), (4416, 4480), (4480, 4481)]
    idx = sorted(set(int(rng.integers(a, b)) for a, b in blocks for _ in range(8)))
    h = 1e-5
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (M.loss_and_grad(tp, F, r2, c, D, off, W)[0] - M.loss_and_grad(tm, F, r2, c, D, off, W)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1e-3, abs(fd)) + 1e-10, (i, fd, g[i])


def test_degenerate_network_is_a_scaled_tpa_curve():
    F, r2, c, D, off = random_data(2)
    th = M.init_params(4)
    W1, b1, W2, b2, w3, b3 = M.unpack(th)
    W2[:] = 0.0
    w3[:] = 0.0
    th[-1] = -0.7
    K, _ = M.forward(th, F)
    # the TPA rational function written out (Teter, Payne & Allan 1989) times softplus(b3) / log 2
    x = F[:, 0]
    num = 27 + 18 * x + 12 * x ** 2 + 8 * x ** 3
    assert np.allclose(K, num / (num + 16 * x ** 4) * math.log1p(math.exp(-0.7)) / math.log(2.0), rtol=1e-14, atol=0)
    # a constant factor on TPA: the loss is TPA's own (scale invariance)
    assert abs(M.loss_and_grad(th, F, r2, c, D, off)[0] - M.cosine_loss_of_k(num / (num + 16 * x ** 4), r2, c, D, off)) < 1e-14
    th[-1] = 0.0                                         # an untrained output layer is TPA exactly
    assert np.allclose(M.forward(th, F)[0], num / (num + 16 * x ** 4), rtol=1e-15, atol=0)


def test_unit_weights_give_the_plain_mean():
    F, r2, c, D, off = random_data(12)
    th = M.init_params(5)
    l1, g1 = M.loss_and_grad(th, F, r2, c, D, off)
    l2, g2 = M.loss_and_grad(th, F, r2, c, D, off, np.full(D.size, 3.7))    # any constant weight
    assert abs(l1 - l2) < 1e-15 and np.allclose(g1, g2, rtol=1e-12, atol=1e-14 * np.abs(g1).max())
    # a single nonzero weight: that band's own loss
    K, _ = M.forward(th, F)
    W = np.zeros(D.size)
    W[2] = 1.0
    one = off[2:4]
    Kb, r2b, cb = K[one[0]:one[1]], r2[one[0]:one[1]], c[one[0]:one[1]]
    want = 1 - (Kb @ cb) ** 2 / ((Kb * Kb) @ r2b * D[2])
    assert abs(M.loss_and_grad(th, F, r2, c, D, off, W)[0] - want) < 1e-14


def test_snapshot_weights_are_residual_shares():
    rng = np.random.default_rng(13)
    nb, npw = 4, 9
    kin = rng.uniform(0, 3, npw)
    psi = rng.normal(size=(nb, npw)) + 1j * rng.normal(size=(nb, npw))
    res = rng.normal(size=(nb, npw)) + 1j * rng.normal(size=(nb, npw))
    res[1] *= 3.0
    dstar = rng.normal(size=(nb, npw)) + 1j * rng.normal(size=(nb, npw))
    dstar[3] = 0.0                                        # dropped band: no weight
    *_, D, W = M.samples(kin, psi, res, rng.normal(size=nb), dstar, kin + 0.3)
    rn2 = (np.abs(res) ** 2).sum(axis=1)
    assert W[3] == 0.0 and abs(W.sum() - 1.0) < 1e-15
    assert np.allclose(W[:3], rn2[:3] / rn2[:3].sum(), rtol=1e-15)


def test_cosine_loss_zero_for_exact_direction_and_bounded():
    rng = np.random.default_rng(3)
    nb, npw = 3, 40
    off = np.arange(0, nb * npw + 1, npw)
    r = rng.normal(size=(nb, npw)) + 1j * rng.normal(size=(nb, npw))
    k = rng.uniform(0.1, 2.0, (nb, npw))
    dstar = k * r                                         # exactly a diagonal correction
    r2 = (np.abs(r) ** 2).ravel()
    c = np.real(np.conj(r) * dstar).ravel()
    D = (np.abs(dstar) ** 2).sum(axis=1)
    assert M.cosine_loss_of_k(k.ravel(), r2, c, D, off) < 1e-14
    assert M.cosine_loss_of_k(5.0 * k.ravel(), r2, c, D, off) < 1e-14       # scale invariance
    other = M.cosine_loss_of_k(np.ones(nb * npw), r2, c, D, off)
    assert 0.0 < other < 1.0


def test_features_are_scale_free_and_x_is_one_on_a_single_wave():
    rng = np.random.default_rng(5)
    nb, npw = 2, 30
    kin = rng.uniform(0, 5, npw)
    hd = kin + rng.uniform(-1, 2, npw)
    psi = rng.normal(size=(nb, npw)) + 1j * rng.normal(size=(nb, npw))
    eps = np.array([-0.3, 0.4])
    F = M.features(kin, psi, eps, hd)
    F2 = M.features(kin, (3.0 - 2j) * psi, eps, hd)
    assert np.allclose(F, F2, rtol=1e-13, atol=1e-13)
    one = np.zeros((1, npw), complex)
    one[0, 7] = 2.0
    Fo = M.features(kin, one, eps[:1], hd)
    # a single plane wave: T_n = T_7, so x = 1 there, e = eps / T_7, d = (H_GG - eps) / T_7
    assert abs(Fo[7, 0] - 1.0) < 1e-15 and abs(Fo[0, 1] - eps[0] / kin[7]) < 1e-15
    assert np.allclose(Fo[:, 2], (hd - eps[0]) / kin[7], rtol=1e-15, atol=0)


def test_hamiltonian_diagonal_is_the_dense_diagonal():
    """H_GG of the feature equals the diagonal of the brute-force H_GG' (Eq. KSHamMat with the
    KB term), with and without projectors, and a constant V0 shifts it by V0."""
    cell = S.cubic_si8(10.0, nbnd=4, kpts=[[0.25, -0.25, 0.25]])
    c = make_case(cell, 0)
    H = OH.dense_h(c["gs"], c["v"], c["beta"], c["D"])
    hd = M.hamiltonian_diagonal(c["gs"]["kin"], c["v"], c["beta"], c["D"])
    np.testing.assert_allclose(hd, np.diag(H).real, rtol=0, atol=1e-12 * np.abs(hd).max())
    assert np.abs(np.diag(H).imag).max() < 1e-14
    H0 = OH.dense_h(c["gs"], c["v"], None, None)
    np.testing.assert_allclose(M.hamiltonian_diagonal(c["gs"]["kin"], c["v"], None, None), np.diag(H0).real,
                               rtol=0, atol=1e-12 * np.abs(hd).max())
    np.testing.assert_allclose(M.hamiltonian_diagonal(c["gs"]["kin"], c["v"] + 0.7, None, None),
                               np.diag(H0).real + 0.7, rtol=0, atol=1e-12 * np.abs(hd).max())


def test_exact_correction_lands_in_the_eigenspace():
    cell = S.fcc_si2(12.0, nbnd=8)
    c = make_case(cell, 0)
    H = OH.dense_h(c["gs"], c["v"], c["beta"], c["D"])
    lam, U = np.linalg.eigh(H)
    U = U.T.copy()                                       # rows = eigenvectors
    nu = 12
    rng = np.random.default_rng(9)
    noise = rng.normal(size=U[:8].shape) + 1j * rng.normal(size=U[:8].shape)
    psi = U[:8] + 0.05 * noise / np.linalg.norm(noise, axis=1)[:, None]     # Ritz-like: 5 % error
    psi /= np.linalg.norm(psi, axis=1)[:, None]
    dstar = M.exact_corrections(psi, lam[:nu], U[:nu], 1e-6)
    for n in range(8):
        assert abs(np.vdot(psi[n], dstar[n])) < 1e-12                 # orthogonal to psi_n
        assert np.linalg.norm(dstar[n]) > 1e-3                          # not dropped
        y = psi[n] + dstar[n]
        resid = np.linalg.norm(H @ y - lam[n] * y) / np.linalg.norm(y)  # eigenvector of eigenvalue n
        assert resid < 1e-10, (n, resid)
    # the Gamma-point triplet of Si: a cluster of three (the projector is not one vector)
    gaps = np.diff(lam[:8])
    assert np.sum(gaps < 1e-6) >= 2
    # a cluster reaching the last given pair is dropped: give only as many pairs as bands
    d2 = M.exact_corrections(psi, lam[:8], U[:8], 1e-6)
    top = np.nonzero(np.abs(lam[:8] - lam[7]) <= 1e-6)[0]
    assert np.all(d2[top] == 0) and np.all(np.linalg.norm(d2[: top[0]], axis=1) > 1e-3)


def test_tpa_factor_is_a_valid_comparison_k():
    """The TPA factor plugged into the same loss (what the learned K competes with)."""
    F, r2, c, D, off = random_data(6)
    L = M.cosine_loss_of_k(tpa_k(F[:, 0]), r2, c, D, off)
    assert 0.0 <= L <= 1.0

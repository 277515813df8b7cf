"""Pins of the FP64 oracle against the paper's printed examples, closed forms,
invariants and brute force (CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import qm_synth as S
from oracle import davidson as OD
from oracle import gspace as OG
from oracle import hamiltonian as OH
from oracle import precond as OP

from conftest import read_golden

BOHR_ANGSTROM = 0.529177210903   # CODATA 2018


def _setup(cell, ik=0, vloc=None, with_nl=True):
    gs = OG.gsphere(cell.lattice, cell.grid or OG.fft_grid(cell.lattice, 4 * cell.ecut_ha),
                    cell.ecut_ha, cell.kpts[ik])
    grid = gs["grid"]
    v = S.vloc_on_grid(cell.lattice, cell.tau, grid) if vloc is None else vloc
    beta = S.beta_of_q(gs["q"], cell.tau, cell.omega) if with_nl else np.zeros((0, len(gs["idx"])), complex)
    D = S.dvals(cell.nat) if with_nl else np.zeros(0)
    return gs, v, beta, D


# ----------------------------------------------------------------- paper's printed pins
def test_fe_gspace_matches_paper_example():
    gold = read_golden("fe_bcc_gspace.txt")
    alat = gold["alat_bohr"][0]
    lat = alat * 0.5 * np.array([[1, 1, 1], [-1, 1, 1], [-1, -1, 1]], float)
    ecut_ha = gold["ecutrho_ry"][0] / 2.0
    grid = OG.fft_grid(lat, ecut_ha)
    assert list(grid) == [int(x) for x in gold["grid"]]
    gs = OG.gsphere(lat, grid, ecut_ha)
    assert len(gs["idx"]) == int(gold["size_g"][0])
    assert int(np.prod(grid)) == int(gold["size_r"][0])
    g2 = 2.0 * gs["kin"]
    np.testing.assert_array_equal(np.round(g2[:5], 1), gold["gnorm2_head"])
    np.testing.assert_array_equal(np.round(g2[-5:], 1), gold["gnorm2_tail"])
    for i in range(3):
        np.testing.assert_array_equal(gs["miller"][:5, i], gold[f"g{i+1}_head"])
        np.testing.assert_array_equal(gs["miller"][-5:, i], gold[f"g{i+1}_tail"])
    assert abs(abs(np.linalg.det(lat)) - gold["omega"][0]) < 5e-6
    b = OG.reciprocal(lat)
    tpiba = 2 * math.pi / alat
    assert abs(tpiba - gold["tpiba"][0]) < 5e-6
    np.testing.assert_allclose(b / tpiba, [[1, 0, 1], [-1, 1, 0], [0, -1, 1]], atol=1e-14)


def test_bcc_lattice_matches_paper_example():
    gold = read_golden("bcc_lattice.txt")
    alat = 5.1 / BOHR_ANGSTROM
    assert abs(alat - gold["alat_bohr"][0]) < 1e-12
    lat = alat * 0.5 * np.array([[1, 1, 1], [-1, 1, 1], [-1, -1, 1]], float)
    tpiba = 2 * math.pi / alat
    assert abs(tpiba - gold["tpiba"][0]) < 1e-14
    b = OG.reciprocal(lat) / tpiba
    for i in range(3):
        np.testing.assert_allclose(b[i], gold[f"b{i+1}"], atol=1e-13)
    cr = np.array([[1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 1, 1]], float)
    cart = cr @ lat
    for i in range(4):
        np.testing.assert_allclose(cart[i], gold[f"cart{i}"], atol=1e-8)
    np.testing.assert_allclose(np.linalg.norm(cart, axis=1) / alat, gold["len_alat"], atol=1e-8)


def test_grid_rule_reproduces_stated_grids():
    for cell in (S.config1(), S.config2(), S.config4()):
        assert OG.fft_grid(cell.lattice, 4 * cell.ecut_ha) == tuple(cell.grid)


def test_sphere_is_brute_force_sphere():
    """Every lattice vector inside the cutoff is in the list once, none outside."""
    cell = S.fcc_si2(16.0, kpts=[[0.25, -0.25, 0.25]])
    gs, *_ = _setup(cell)
    b = OG.reciprocal(cell.lattice)
    r = np.arange(-12, 13)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    q = (m + cell.kpts[0]) @ b
    inside = 0.5 * np.einsum("ij,ij->i", q, q) <= cell.ecut_ha
    want = {tuple(x) for x in m[inside]}
    got = {tuple(x) for x in gs["miller"]}
    assert want == got and len(got) == len(gs["miller"])
    assert np.all(np.diff(gs["idx"]) > 0)


# ----------------------------------------------------------------- H psi closed forms
@pytest.mark.parametrize("k", [[0, 0, 0], [0.25, -0.25, 0.25]])
def test_free_electron(k):
    cell = S.fcc_si2(12.0, kpts=[k])
    gs, v, beta, D = _setup(cell, vloc=None, with_nl=False)
    v = np.zeros_like(v)
    psi = S.psi_random(3, 3, len(gs["idx"]))
    for f in (OH.hpsi_naive, OH.hpsi_fft):
        np.testing.assert_allclose(f(psi, gs, v, beta, D), gs["kin"] * psi, atol=1e-14)
    q = (gs["miller"] + np.array(k)) @ OG.reciprocal(cell.lattice)
    np.testing.assert_allclose(gs["kin"], 0.5 * (q * q).sum(1), rtol=1e-15)
    ev = np.linalg.eigvalsh(OH.dense_h(gs, v, beta, D))
    np.testing.assert_allclose(ev, np.sort(gs["kin"]), atol=1e-14)


def test_constant_potential_shift():
    cell = S.fcc_si2(12.0)
    gs, v, beta, D = _setup(cell)
    v0 = -0.731
    psi = S.psi_random(4, 3, len(gs["idx"]))
    for f in (OH.hpsi_naive, OH.hpsi_fft):
        d = f(psi, gs, v + v0, beta, D) - f(psi, gs, v, beta, D)
        np.testing.assert_allclose(d, v0 * psi, atol=1e-13)
    e1 = np.linalg.eigvalsh(OH.dense_h(gs, v, beta, D))
    e2 = np.linalg.eigvalsh(OH.dense_h(gs, v + v0, beta, D))
    np.testing.assert_allclose(e2 - e1, v0, atol=1e-12)


def test_sine_potential_closed_form():
    """V(r) = sin(g0.r): a plane wave G0 goes to -i/2 at G0+g0 and +i/2 at G0-g0.
    Fixes the sign of the exponent, the 1/N_r factor and the (G - G') orientation."""
    cell = S.fcc_si2(12.0, kpts=[[0.25, -0.25, 0.25]])
    gs, v, beta, D = _setup(cell, with_nl=False)
    n1, n2, n3 = gs["grid"]
    j1 = np.tile(np.arange(n1), n2 * n3)                  # flat x fastest
    v = np.sin(2 * math.pi * j1 / n1)                     # g0 = b1  (miller (1,0,0))
    m = gs["miller"]
    i0 = int(np.where((m == [0, 0, 0]).all(1))[0][0])
    ip = int(np.where((m == [1, 0, 0]).all(1))[0][0])
    im = int(np.where((m == [-1, 0, 0]).all(1))[0][0])
    psi = np.zeros((1, len(m)), complex)
    psi[0, i0] = 1.0
    want = gs["kin"] * psi
    want[0, ip] += -0.5j
    want[0, im] += 0.5j
    for f in (OH.hpsi_naive, OH.hpsi_fft):
        np.testing.assert_allclose(f(psi, gs, v, beta, D), want, atol=1e-14)
    np.testing.assert_allclose(psi @ OH.dense_h(gs, v, beta, D).T, want, atol=1e-14)


def test_gaussian_potential_mean_closed_form():
    """Vt(0) = mean V = depth (2 pi)^{3/2} w^3 nat / Omega for the Gaussian sum."""
    for cell in (S.config1(), S.cubic_si8(10.0)):
        grid = cell.grid or OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
        v = S.vloc_on_grid(cell.lattice, cell.tau, grid)
        want = cell.depth * (2 * math.pi) ** 1.5 * cell.width ** 3 * cell.nat / cell.omega
        vt = OH.vtilde(v, grid)
        assert abs(vt[0, 0, 0].real - want) < 1e-12
        assert abs(v.mean() - want) < 1e-12


def test_projector_norm_closed_form():
    """sum_G |beta_s(k+G)|^2 = sum_R e^{ik.R} exp(-R^2 / 4 rc^2) (Poisson summation)."""
    cell = S.fcc_si2(80.0, kpts=[[0.25, 0.25, -0.25]])
    gs = OG.gsphere(cell.lattice, OG.fft_grid(cell.lattice, 4 * cell.ecut_ha), cell.ecut_ha, cell.kpts[0])
    beta = S.beta_of_q(gs["q"], cell.tau[:1], cell.omega)
    r = np.arange(-4, 5)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    R = n @ cell.lattice
    kc = cell.kpts[0] @ OG.reciprocal(cell.lattice)
    want = np.sum(np.exp(1j * R @ kc) * np.exp(-(R * R).sum(1) / 4.0)).real
    assert abs(np.sum(np.abs(beta[0]) ** 2) - want) < 1e-12


def test_nonlocal_rank_one_secular_equation():
    """V = 0, one atom, s projector only: eigenvalues E solve 1 = D sum_G |b_G|^2/(E - T_G)."""
    cell = S.fcc_si2(10.0)
    gs = OG.gsphere(cell.lattice, OG.fft_grid(cell.lattice, 4 * cell.ecut_ha), cell.ecut_ha)
    beta = S.beta_of_q(gs["q"], cell.tau[:1], cell.omega)[:1]
    Ds = 5.0
    v = np.zeros(int(np.prod(gs["grid"])))
    H = OH.dense_h(gs, v, beta, np.array([Ds]))
    ev = np.linalg.eigvalsh(H)
    T = gs["kin"]
    order = np.argsort(T)
    cuts = np.where(np.diff(T[order]) > 1e-9)[0] + 1
    groups = np.split(order, cuts)
    levels = np.array([T[g].mean() for g in groups])
    w = np.array([np.sum(np.abs(beta[0][g]) ** 2) for g in groups])
    f = lambda E: 1.0 - Ds * np.sum(w / (E - levels))
    roots = []
    edges = list(levels) + [levels[-1] + Ds * w.sum() + 1.0]
    for lo, hi in zip(edges[:-1], edges[1:]):
        a, b = lo + 1e-13, hi - 1e-13
        if f(a) * f(b) > 0:
            continue
        for _ in range(200):
            c = 0.5 * (a + b)
            if f(a) * f(c) <= 0:
                b = c
            else:
                a = c
        roots.append(0.5 * (a + b))
    # each root is an eigenvalue; the remaining eigenvalues are unshifted free-electron levels
    for r in roots:
        assert np.min(np.abs(ev - r)) < 1e-11
    rest = [e for e in ev if np.min(np.abs(np.array(roots) - e)) > 1e-9]
    assert all(np.min(np.abs(levels - e)) < 1e-11 for e in rest)
    assert len(roots) + len(rest) == len(ev)
    # action on beta itself: H b = T b + D |b|^2 b  (fixes b D b^H against its transpose)
    for fn in (OH.hpsi_naive, OH.hpsi_fft):
        hb = fn(beta, gs, v, beta, np.array([Ds]))
        np.testing.assert_allclose(hb, T * beta + Ds * np.sum(np.abs(beta) ** 2) * beta, atol=1e-14)


def test_hermiticity_and_three_way_agreement():
    cell = S.cubic_si8(10.0, reps=(1, 1, 1), kpts=[[0.25, 0.25, -0.25]])
    gs, v, beta, D = _setup(cell)
    npw = len(gs["idx"])
    phi = S.psi_random(7, 2, npw)
    psi = S.psi_random(8, 2, npw)
    a = OH.hpsi_naive(psi, gs, v, beta, D)
    b = OH.hpsi_fft(psi, gs, v, beta, D)
    c = psi @ OH.dense_h(gs, v, beta, D).T
    scale = np.abs(b).max()
    assert np.abs(a - b).max() / scale < 1e-13
    assert np.abs(c - b).max() / scale < 1e-13
    hphi = OH.hpsi_fft(phi, gs, v, beta, D)
    lhs = np.sum(phi.conj() * b, axis=1)
    rhs = np.sum(hphi.conj() * psi, axis=1)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


def test_time_reversal_eigenvalues():
    cell = S.fcc_si2(10.0, kpts=[[0.25, -0.25, 0.25], [-0.25, 0.25, -0.25]])
    e = []
    for ik in range(2):
        gs, v, beta, D = _setup(cell, ik)
        e.append(np.linalg.eigvalsh(OH.dense_h(gs, v, beta, D))[:10])
    np.testing.assert_allclose(e[0], e[1], atol=1e-12)


# ----------------------------------------------------------------- preconditioner
def test_tpa_closed_forms():
    assert OP.tpa_k(0.0) == 1.0
    x = np.array([1e3, 1e4, 1e5])
    np.testing.assert_allclose(OP.tpa_k(x) * 2 * x, 1.0, rtol=2e-3)
    xs = np.linspace(0, 50, 1001)
    k = OP.tpa_k(xs)
    assert np.all(np.diff(k) < 0) and np.all(k > 0) and np.all(k <= 1)
    # x = 1: (27+18+12+8) / (65+16)
    assert abs(OP.tpa_k(1.0) - 65.0 / 81.0) < 1e-15


def test_tpa_apply_closed_form():
    """tpa_apply against hand-computed values: T_n is the kinetic energy per unit norm of the
    band's Ritz vector (weights |psi|^2, normalised), not of the residual, and the factor is
    applied to the residual.  Row 0: |psi|^2 = 1 on a plane wave with T_G = 1 and 3 on one with
    T_G = 3, so T_0 = (1 + 3*3) / 4 = 5/2; row 1: all weight on T_G = 5, so T_1 = 5.  At
    T_G = 0, 5/2, 5 the factors of row 0 are K(0) = 1, K(1) = 65/81 and
    K(2) = (27+36+48+64) / (27+36+48+64+256) = 175/431; row 1 sees x = 0, 1/2, 1, and
    K(1/2) = (27+9+3+1) / (27+9+3+1+1) = 40/41."""
    kin = np.array([0.0, 1.0, 3.0, 2.5, 5.0])
    psi = np.zeros((2, 5), complex)
    psi[0, 1] = 1.0 * np.exp(0.3j)
    psi[0, 2] = np.sqrt(3.0) * np.exp(-1.1j)
    psi[1, 4] = 2.0j                       # T_n must not depend on the norm or phase
    rng = np.random.default_rng(5)
    r = rng.normal(size=(2, 5)) + 1j * rng.normal(size=(2, 5))
    r[:, 1:3] *= 1e3                       # weight of the residual elsewhere than psi's
    got = OP.tpa_apply(r, psi, kin)
    k0 = {0: 1.0, 3: 65.0 / 81.0, 4: 175.0 / 431.0}
    k1 = {0: 1.0, 3: 40.0 / 41.0, 4: 65.0 / 81.0}
    for g, k in k0.items():
        assert abs(got[0, g] - k * r[0, g]) <= 1e-15 * abs(r[0, g])
    for g, k in k1.items():
        assert abs(got[1, g] - k * r[1, g]) <= 1e-15 * abs(r[1, g])
    # psi scaled by a complex constant per row: identical result
    np.testing.assert_allclose(OP.tpa_apply(r, 7.5j * psi, kin), got, rtol=1e-15, atol=0)


# ----------------------------------------------------------------- Davidson vs brute force
@pytest.mark.parametrize("cellf", [S.config1, lambda: S.cubic_si8(10.0, nbnd=8, kpts=[[0.25, 0.25, 0.25]])])
def test_davidson_matches_dense(cellf):
    cell = cellf()
    gs, v, beta, D = _setup(cell)
    ev = np.linalg.eigvalsh(OH.dense_h(gs, v, beta, D))[: cell.nbnd]
    psi0 = S.psi_random(cell.seed, cell.nbnd, len(gs["idx"]))
    e, X, info = OD.davidson(lambda Y: OH.hpsi_fft(Y, gs, v, beta, D), psi0, gs["kin"], tol=1e-9, max_iter=300)
    assert info["resid"].max() <= 1e-9
    np.testing.assert_allclose(e, ev, atol=1e-9)
    np.testing.assert_allclose(X @ X.conj().T, np.eye(cell.nbnd), atol=1e-12)


def test_davidson_ritz_values_monotone_between_restarts():
    """Cauchy interlacing: growing the basis can only lower each Ritz value."""
    cell = S.config1()
    gs, v, beta, D = _setup(cell)
    psi0 = S.psi_random(1, cell.nbnd, len(gs["idx"]))
    e, X, info = OD.davidson(lambda Y: OH.hpsi_fft(Y, gs, v, beta, D), psi0, gs["kin"],
                             fixed_iters=3, nvecx=10 * cell.nbnd)
    h = [x[0] for x in info["history"]]
    assert np.all(h[1] <= h[0] + 1e-13) and np.all(h[2] <= h[1] + 1e-13)


def test_orthonormalize_rows_is_gram_schmidt():
    X = S.psi_random(5, 4, 30)
    Y = OD.orthonormalize_rows(X)
    np.testing.assert_allclose(Y @ Y.conj().T, np.eye(4), atol=1e-13)
    # row 0 is just normalised; row 1 lies in span(x0, x1) (triangular structure)
    np.testing.assert_allclose(Y[0], X[0] / np.linalg.norm(X[0]), atol=1e-14)
    c = np.linalg.lstsq(X[:2].T, Y[1], rcond=None)[0]
    np.testing.assert_allclose(X[:2].T @ c, Y[1], atol=1e-12)

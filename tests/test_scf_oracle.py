"""Pins of the oracle's self-consistency pieces (oracle/scf.py: density, Hartree, LDA, Anderson
mixing, the loop) against closed forms, derivatives, limits and invariants (CPU only)."""
import math

import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG
from oracle import scf as OS


def test_exchange_closed_form():
    """Slater exchange written in the density: eps_x = -(3/4)(3n/pi)^(1/3), v_x = (4/3) eps_x; the
    correlation part is what remains (checked separately)."""
    for n in (1e-3, 0.02, 0.3, 3.0):
        ex = -0.75 * (3.0 * n / math.pi) ** (1.0 / 3.0)
        eps, v = OS.lda(np.array([n]))
        rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
        ec = (OS.PZ_GAMMA / (1 + OS.PZ_BETA1 * math.sqrt(rs) + OS.PZ_BETA2 * rs) if rs >= 1 else
              OS.PZ_A * math.log(rs) + OS.PZ_B + OS.PZ_C * rs * math.log(rs) + OS.PZ_D * rs)
        assert abs(eps[0] - (ex + ec)) <= 1e-14 * abs(ex)


@pytest.mark.parametrize("n", [1e-4, 3e-3, 0.05, 0.2, 0.25, 1.0, 10.0])
def test_potential_is_the_derivative_of_the_energy_density(n):
    """v_xc = d(n eps_xc)/dn (central differences), on both branches of the parametrisation."""
    h = 1e-6 * n
    e = lambda x: x * OS.lda(np.array([x]))[0][0]
    fd = (e(n + h) - e(n - h)) / (2 * h)
    assert abs(OS.lda(np.array([n]))[1][0] - fd) <= 1e-7 * abs(fd)


def test_correlation_limits():
    """Continuity of the two branches at r_s = 1 (to the parametrisation's 1e-4) and the
    high-density log coefficient of the electron gas, (1 - ln 2)/pi^2 (Gell-Mann-Brueckner)."""
    def ec(rs):
        n = 3.0 / (4.0 * math.pi * rs ** 3)
        ex = -0.75 * (3.0 * n / math.pi) ** (1.0 / 3.0)
        return OS.lda(np.array([n]))[0][0] - ex
    assert abs(ec(1 - 1e-9) - ec(1 + 1e-9)) < 1e-4
    r1, r2 = 1e-5, 2e-5
    slope = (ec(r2) - ec(r1)) / math.log(r2 / r1)
    assert abs(slope - (1 - math.log(2)) / math.pi ** 2) < 2e-4
    assert OS.lda(np.array([0.0, -1e-3]))[1].tolist() == [0.0, 0.0]


def test_hartree_of_a_cosine_density():
    """n = n0 + A cos(b1 . r): V_H = 4 pi A / |b1|^2 cos(b1 . r) (the uniform part is neutralised)."""
    cell = S.fcc_si2(10.0)
    grid = OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    n1, n2, n3 = grid
    j1 = np.tile(np.arange(n1), n2 * n3)
    c = np.cos(2 * math.pi * j1 / n1)
    b1 = OG.reciprocal(cell.lattice)[0]
    v = OS.hartree(0.03 + 0.01 * c, cell.lattice, grid, 4 * cell.ecut_ha)
    np.testing.assert_allclose(v, 4 * math.pi * 0.01 / (b1 @ b1) * c, rtol=0, atol=1e-13)


def test_density_integrates_to_the_electron_count():
    cell = S.cubic_si8(10.0)
    grid = OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    ks = [[0.0, 0.0, 0.0], [0.25, 0.25, 0.25]]
    sph = [OG.gsphere(cell.lattice, grid, cell.ecut_ha, k) for k in ks]
    coefs = []
    for i, gs in enumerate(sph):
        q, _ = np.linalg.qr(S.psi_random(50 + i, 6, len(gs["idx"])).T)
        coefs.append(q.T)
    n = OS.density(coefs, sph, [0.25, 0.75], 4, cell.omega)
    assert n.min() >= 0
    assert abs(cell.omega / n.size * n.sum() - 8.0) < 1e-12
    # one plane wave per k: the uniform density 2 / Omega
    pw = [np.eye(len(gs["idx"]))[:1] for gs in sph]
    np.testing.assert_allclose(OS.density(pw, sph, [0.5, 0.5], 1, cell.omega), 2.0 / cell.omega, rtol=1e-13)


def test_anderson_solves_a_linear_fixed_point():
    """x = A x + b (dimension 4, contraction): Anderson with 4 differences reaches the exact
    fixed point within 6 steps; with no history it is linear mixing x + alpha F."""
    rng = np.random.default_rng(7)
    A = 0.3 * rng.standard_normal((4, 4))
    b = rng.standard_normal(4)
    xs = np.linalg.solve(np.eye(4) - A, b)
    mix = OS.Anderson(0.5, 4)
    x = np.zeros(4)
    for _ in range(6):
        x = mix.step(x, A @ x + b - x)
    np.testing.assert_allclose(x, xs, atol=1e-10)
    lin = OS.Anderson(0.3, 0)
    x0 = rng.standard_normal(4)
    f0 = A @ x0 + b - x0
    np.testing.assert_allclose(lin.step(x0, f0), x0 + 0.3 * f0, atol=0)


def test_free_electron_gas_is_self_consistent_at_once():
    """No ionic potential, no projectors, two electrons at Gamma: the G = 0 state is occupied, the
    density is uniform, V_H = 0 and V_xc = v_xc(2/Omega): eigenvalues 1/2|G|^2 + v_xc exactly."""
    cell = S.cubic_si8(8.0)
    grid = OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    nr = int(np.prod(grid))
    gs = OG.gsphere(cell.lattice, grid, cell.ecut_ha, [0, 0, 0])
    eigs, n, v, it = OS.scf(cell.lattice, cell.omega, cell.ecut_ha, grid, [[0, 0, 0]], [1.0], 2, 5, np.zeros(nr),
                            [np.zeros((0, len(gs["idx"])), complex)], np.zeros(0))
    vxc = OS.lda(np.array([2.0 / cell.omega]))[1][0]
    assert it == 1
    np.testing.assert_allclose(eigs[0], np.sort(gs["kin"])[:5] + vxc, atol=1e-12)


def test_si_cell_converges_to_a_fixed_point():
    """Si2-like fcc cell with the synthetic wells, two k-points, 2 electrons (the lowest band,
    0.4 Ha below the next at Gamma; with 8 electrons and these two k-points the fourth and fifth
    bands of this weak potential trade places and the loop does not settle): the loop converges; at
    its density the potential's occupied states give the same density back, which holds 2
    electrons."""
    cell = S.fcc_si2(8.0)
    grid = OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    ks, w = [[0, 0, 0], [0.25, -0.25, 0.25]], [0.25, 0.75]
    sph = [OG.gsphere(cell.lattice, grid, cell.ecut_ha, k) for k in ks]
    betas = [S.beta_of_q(gs["q"], cell.tau, cell.omega) for gs in sph]
    vion = S.vloc_on_grid(cell.lattice, cell.tau, grid)
    eigs, n, v, it = OS.scf(cell.lattice, cell.omega, cell.ecut_ha, grid, ks, w, 2, 6, vion, betas,
                            S.dvals(cell.nat), tol=1e-10)
    assert 2 < it < 40
    assert abs(cell.omega / n.size * n.sum() - 2.0) < 1e-9
    from oracle import hamiltonian as OH
    coefs = [np.linalg.eigh(OH.dense_h(gs, OS.potential(n, vion, cell.lattice, grid, 4 * cell.ecut_ha), b,
                                       S.dvals(cell.nat)))[1][:, :1].T for gs, b in zip(sph, betas)]
    n_out = OS.density(coefs, sph, w, 1, cell.omega)
    assert cell.omega / n.size * np.abs(n_out - n).sum() <= 1e-9


def test_si_cell_eight_electrons_three_k_points():
    """Four occupied bands (8 electrons, Si-like) with the k-points Gamma, (1/4, -1/4, 1/4) and
    (1/2, 0, 0) (weights 1/8, 1/2, 3/8): the loop converges to a fixed point that holds 8 electrons."""
    cell = S.fcc_si2(8.0)
    grid = OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    ks, w = [[0, 0, 0], [0.25, -0.25, 0.25], [0.5, 0, 0]], [0.125, 0.5, 0.375]
    sph = [OG.gsphere(cell.lattice, grid, cell.ecut_ha, k) for k in ks]
    betas = [S.beta_of_q(gs["q"], cell.tau, cell.omega) for gs in sph]
    vion = S.vloc_on_grid(cell.lattice, cell.tau, grid)
    eigs, n, v, it = OS.scf(cell.lattice, cell.omega, cell.ecut_ha, grid, ks, w, 8, 6, vion, betas,
                            S.dvals(cell.nat), tol=1e-10, max_iter=80)
    assert it < 80
    assert abs(cell.omega / n.size * n.sum() - 8.0) < 1e-9
    assert n.min() > 0

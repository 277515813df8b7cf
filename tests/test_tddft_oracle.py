"""Pins of the oracle's real-time propagation (oracle/tddft.py, Section 5 "tddft" module)
against the exact exponential of the brute-force Hamiltonian, closed forms and invariants
(CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import qm_synth as S
from oracle import gspace as OG
from oracle import hamiltonian as OH
from oracle import tddft as OT


def _setup(cell, ik=0, with_nl=True, zero_v=False):
    grid = cell.grid or OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    gs = OG.gsphere(cell.lattice, grid, cell.ecut_ha, cell.kpts[ik])
    v = S.vloc_on_grid(cell.lattice, cell.tau, gs["grid"])
    if zero_v:
        v = np.zeros_like(v)
    beta = S.beta_of_q(gs["q"], cell.tau, cell.omega) if with_nl else None
    D = S.dvals(cell.nat) if with_nl else None
    return gs, v, beta, D


def _h(gs, v, beta, D):
    return lambda x: OH.hpsi_fft(x, gs, v, beta, D)


@pytest.mark.parametrize("dt", [0.05, 0.4])
def test_free_electron_phase(dt):
    """V = 0, no projectors: every plane wave is an eigenstate with eigenvalue 1/2|k+G|^2, so the
    converged series is the phase exp(-i dt |k+G|^2 / 2) (fixes the sign of i and the 1/r!)."""
    cell = S.fcc_si2(12.0, kpts=[[0.25, -0.25, 0.25]])
    gs, v, _, _ = _setup(cell, with_nl=False, zero_v=True)
    psi = S.psi_random(5, 3, len(gs["idx"]))
    got = OT.taylor_propagate(_h(gs, v, None, None), psi, dt, 60)
    want = np.exp(-1j * dt * gs["kin"])[None, :] * psi
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(psi).max())


@pytest.mark.parametrize("order", [1, 2, 4, 6])
def test_truncation_error_is_first_omitted_term(order):
    """For one plane wave of energy e the error of U_k against the exact phase is led by the
    first omitted term (-i dt e)^{k+1}/(k+1)!: the ratio tends to 1 as dt e -> 0.  A series
    cut one term early or late fails by a factor ~ dt e or ~ 1/(dt e)."""
    cell = S.fcc_si2(12.0, kpts=[[0.25, -0.25, 0.25]])
    gs, v, _, _ = _setup(cell, with_nl=False, zero_v=True)
    g = int(np.argmax(gs["kin"]))
    e = gs["kin"][g]
    psi = np.zeros((1, len(gs["idx"])), complex)
    psi[0, g] = 1.0
    for x in (0.02, 0.05):
        dt = x / e
        got = OT.taylor_propagate(_h(gs, v, None, None), psi, dt, order)[0, g]
        err = np.exp(-1j * x) - got          # the omitted tail of the series
        lead = (-1j * x) ** (order + 1) / math.factorial(order + 1)
        assert abs(err / lead - 1.0) < 2.0 * x, (order, x, err / lead)


def test_matches_dense_exponential():
    """Si2 cell with the local potential and the KB projectors at k != 0: the series of high
    order equals expm(-i dt H) of the brute-force matrix; order 4 stays within the series-tail
    bound for ||H|| = the largest |eigenvalue|."""
    cell = S.fcc_si2(14.0, kpts=[[0.25, -0.25, 0.25]])
    gs, v, beta, D = _setup(cell)
    H = OH.dense_h(gs, v, beta, D)
    ev = np.linalg.eigvalsh(H)
    hnorm = np.abs(ev).max()
    psi = S.psi_random(6, 4, len(gs["idx"]))
    dt = 0.3 / hnorm * 4
    exact = psi @ sla.expm(-1j * dt * H).T
    high = OT.taylor_propagate(_h(gs, v, beta, D), psi, dt, 40)
    np.testing.assert_allclose(high, exact, rtol=0, atol=1e-12 * np.abs(exact).max())
    low = OT.taylor_propagate(_h(gs, v, beta, D), psi, dt, 4)
    err = np.linalg.norm(low - exact, axis=1) / np.linalg.norm(psi, axis=1)
    bound = OT.taylor_remainder_bound(hnorm, dt, 4)
    assert np.all(err <= bound), (err.max(), bound)
    assert err.max() > 1e-3 * bound          # the bound is not vacuous at this step


def test_etrs_order_of_half_steps():
    """Two different potentials: ETRS equals expm(-i dt/2 H_next) expm(-i dt/2 H_now) of the
    brute-force matrices, and differs from the product in the other order (H_now and H_next
    do not commute)."""
    cell = S.fcc_si2(12.0, kpts=[[0.25, -0.25, 0.25]])
    gs, v, beta, D = _setup(cell)
    n1, n2, n3 = gs["grid"]
    j1 = np.tile(np.arange(n1), n2 * n3)
    v2 = v + 0.8 * np.cos(2 * math.pi * j1 / n1)
    Ha = OH.dense_h(gs, v, beta, D)
    Hb = OH.dense_h(gs, v2, beta, D)
    dt = 0.1
    psi = S.psi_random(7, 3, len(gs["idx"]))
    got = OT.etrs_step(_h(gs, v, beta, D), _h(gs, v2, beta, D), psi, dt, 40)
    Ua, Ub = sla.expm(-0.5j * dt * Ha), sla.expm(-0.5j * dt * Hb)
    want = psi @ (Ub @ Ua).T
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    other = psi @ (Ua @ Ub).T
    assert np.abs(other - want).max() > 1e-6


def test_etrs_constant_shift_is_a_phase():
    """V_next = V_now + c: the step is exp(-i c dt/2) exp(-i dt H_now) exactly."""
    cell = S.fcc_si2(12.0)
    gs, v, beta, D = _setup(cell)
    c, dt = -0.37, 0.2
    psi = S.psi_random(8, 2, len(gs["idx"]))
    got = OT.etrs_step(_h(gs, v, beta, D), _h(gs, v + c, beta, D), psi, dt, 40)
    want = np.exp(-0.5j * c * dt) * OT.taylor_propagate(_h(gs, v, beta, D), psi, dt, 40)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_unitarity():
    """The exact propagator keeps every inner product; the series of order 4 changes them only
    beyond its truncation order (by O((dt ||H||)^6) for order 4)."""
    cell = S.fcc_si2(12.0, kpts=[[0.25, -0.25, 0.25]])
    gs, v, beta, D = _setup(cell)
    psi = S.psi_random(9, 3, len(gs["idx"]))
    q, _ = np.linalg.qr(psi.T)
    psi = q.T
    hnorm = np.abs(np.linalg.eigvalsh(OH.dense_h(gs, v, beta, D))).max()
    for dt, order, tol in ((0.5 / hnorm, 40, 1e-13), (0.05 / hnorm, 4, 1e-7)):
        out = OT.taylor_propagate(_h(gs, v, beta, D), psi, dt, order)
        np.testing.assert_allclose(out.conj() @ out.T, np.eye(3), atol=tol)


def test_order_zero_and_zero_step_are_identity():
    cell = S.fcc_si2(8.0)
    gs, v, beta, D = _setup(cell)
    psi = S.psi_random(10, 2, len(gs["idx"]))
    np.testing.assert_array_equal(OT.taylor_propagate(_h(gs, v, beta, D), psi, 0.3, 0), psi)
    np.testing.assert_array_equal(OT.taylor_propagate(_h(gs, v, beta, D), psi, 0.0, 4), psi)

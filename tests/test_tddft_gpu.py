"""Parity of the CUDA real-time propagation (qm_tddft_taylor / qm_tddft_etrs through the C ABI)
with the FP64 oracle (oracle/tddft.py on oracle.hamiltonian.hpsi_fft).

Tolerances.  FP64: element-wise |diff| <= 1e-11 * max|psi_out(band)|, the H psi bar (each term
is a product of H psi applications, and the term of order r carries dt^r / r!).  Precision form:
per band ||diff|| / ||psi_out|| and element-wise relative to the band's largest element, with the
H psi bars of the precision form (1e-6 / 5e-6 up to 72^3, 1e-5 / 5e-5 beyond): the first term
carries dt times the H psi error, and every addition to psi rounds in FP32 (6e-8).
"""
import math

import numpy as np
import pytest

import qm_synth as S
from oracle import hamiltonian as OH
from oracle import tddft as OT

from cases import band_rel_err, make_case

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


def _h(c, v=None):
    vv = c["v"] if v is None else v
    return lambda x: OH.hpsi_fft(x, c["gs"], vv, c["beta"], c["D"])


def gpu_prop(Q, g, ik, c, dt, order, prec="fp64", v_next=None, ld_pad=0, psi=None, stream=None):
    psi = c["psi"] if psi is None else psi
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    nb, npw = psi.shape
    p = torch.zeros((nb, npw + ld_pad), dtype=cdt, device="cuda")
    p[:, :npw] = dev(psi, cdt)
    beta, D, v = dev(c["beta"], cdt), dev(c["D"]), dev(c["v"])
    if v_next is None:
        Q.qm_tddft_taylor(g, ik, p, v, beta, D, dt, order, prec=prec, stream=stream)
    else:
        Q.qm_tddft_etrs(g, ik, p, v, dev(v_next), beta, D, dt, order, prec=prec, stream=stream)
    torch.cuda.synchronize()
    return p[:, :npw].cpu().numpy().astype(np.complex128)


def check64(got, want):
    scale = np.abs(want).max(axis=1, keepdims=True)
    err = (np.abs(got - want) / scale).max()
    assert err <= TOL64, err
    return err


def check_mixed(got, want, large=False):
    tb, te = (1e-5, 5e-5) if large else (1e-6, 5e-6)
    rel = band_rel_err(got, want).max()
    el = (np.abs(got - want) / np.abs(want).max(axis=1, keepdims=True)).max()
    assert rel <= tb and el <= te, (rel, el)
    return rel, el


def _modulated(c):
    n1, n2, n3 = c["grid"]
    j1 = np.tile(np.arange(n1), n2 * n3)
    return c["v"] + 0.4 * np.cos(2 * math.pi * j1 / n1)


@pytest.mark.parametrize("cell", S.small_cells() + [S.config1()], ids=lambda c: f"{c.name}_{c.ecutwfc_ry:g}Ry")
def test_taylor_and_etrs_fp64_match_oracle(Q, cell):
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        for ik in range(len(cell.kpts)):
            c = make_case(cell, ik)
            for dt, order in ((0.05, 4), (0.02, 1), (0.1, 7)):
                want = OT.taylor_propagate(_h(c), c["psi"], dt, order)
                check64(gpu_prop(Q, g, ik, c, dt, order), want)
            v2 = _modulated(c)
            want = OT.etrs_step(_h(c), _h(c, v2), c["psi"], 0.05, 4)
            check64(gpu_prop(Q, g, ik, c, 0.05, 4, v_next=v2, ld_pad=3), want)
    finally:
        Q.qm_gspace_destroy(g)


def test_identity_cases_are_bit_exact(Q):
    """order 0 and dt = 0 leave psi bitwise unchanged."""
    cell = S.small_cells()[3]
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        c = make_case(cell, 0)
        for prec in ("fp64", "mixed"):
            want = c["psi"] if prec == "fp64" else c["psi"].astype(np.complex64).astype(np.complex128)
            np.testing.assert_array_equal(gpu_prop(Q, g, 0, c, 0.3, 0, prec=prec), want)
            np.testing.assert_array_equal(gpu_prop(Q, g, 0, c, 0.0, 4, prec=prec), want)
    finally:
        Q.qm_gspace_destroy(g)


def test_mixed_small_cells_match_oracle(Q):
    for cell in S.small_cells()[1:4]:
        g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
        try:
            c = make_case(cell, 0)
            check_mixed(gpu_prop(Q, g, 0, c, 0.05, 4, prec="mixed"), OT.taylor_propagate(_h(c), c["psi"], 0.05, 4))
            v2 = _modulated(c)
            check_mixed(gpu_prop(Q, g, 0, c, 0.05, 4, prec="mixed", v_next=v2),
                        OT.etrs_step(_h(c), _h(c, v2), c["psi"], 0.05, 4))
        finally:
            Q.qm_gspace_destroy(g)


@pytest.mark.parametrize("which,ik,nb", [("config2", 1, 12), ("config5", 0, 3)])
def test_full_size_sampled_bands(Q, which, ik, nb):
    """The 64-atom (72^3) and 255-atom (96x96x48) cells at full size, a few bands of one
    k-point, both precisions, order 4 (the benchmark's propagation step), on a side stream."""
    cell = getattr(S, which)()
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        c = make_case(cell, ik, nb=nb)
        dt = 0.05
        want = OT.taylor_propagate(_h(c), c["psi"], dt, 4)
        s = torch.cuda.Stream()
        check64(gpu_prop(Q, g, ik, c, dt, 4, stream=s), want)
        check_mixed(gpu_prop(Q, g, ik, c, dt, 4, prec="mixed", stream=s), want, large=which == "config5")
    finally:
        Q.qm_gspace_destroy(g)


def test_long_propagation_keeps_the_norm(Q):
    """100 ETRS steps of order 4 with a step well inside the series' convergence: the GPU keeps
    every band's norm and the overlaps of an orthonormal block as the exact propagator does, to
    the truncation error (bounded here by 100 x the series-tail bound of one step)."""
    cell = S.small_cells()[1]
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        c = make_case(cell, 0)
        q, _ = np.linalg.qr(c["psi"].T)
        psi0 = q.T.copy()
        hnorm = np.abs(np.linalg.eigvalsh(OH.dense_h(c["gs"], c["v"], c["beta"], c["D"]))).max()
        dt = 0.2 / hnorm
        p = dev(psi0)
        beta, D, v = dev(c["beta"]), dev(c["D"]), dev(c["v"])
        work = torch.empty(2 * p.numel(), dtype=torch.complex128, device="cuda")
        for _ in range(100):
            Q.qm_tddft_etrs(g, 0, p, v, v, beta, D, dt, 4, work=work)
        out = p.cpu().numpy()
        bound = 100 * 4 * OT.taylor_remainder_bound(hnorm, dt / 2, 4)
        np.testing.assert_allclose(out.conj() @ out.T, np.eye(len(out)), atol=bound + 1e-12)
        assert np.abs(out - psi0).max() > 1e-3           # the states did move
    finally:
        Q.qm_gspace_destroy(g)

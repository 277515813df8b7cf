"""C-ABI checks that need no GPU: the library loads, exports every declared symbol,
validates arguments, and its host-side G-sphere / grid logic equals the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2308_07277_gb300 import _lib as L
    return L.load()


def test_library_exports_every_declared_symbol():
    lib = _lib()
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(qm_[a-z0-9_]+)\s*\(", txt))
    assert {"qm_gspace_create", "qm_hpsi", "qm_last_error"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def _cells():
    return [S.config1(), S.config2(), S.config4(), S.config5()] + S.small_cells()


@pytest.mark.parametrize("cell", _cells(), ids=lambda c: c.name + str(c.ecutwfc_ry))
def test_host_gspace_equals_oracle(cell):
    import paper_2308_07277_gb300 as Q
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        info = Q.qm_gspace_query(g)
        want_grid = tuple(cell.grid) if cell.grid else OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
        assert info["grid"] == want_grid
        for ik in range(min(len(cell.kpts), 2)):
            gs = OG.gsphere(cell.lattice, want_grid, cell.ecut_ha, cell.kpts[ik])
            idx, mil, kpg = Q.qm_gspace_indices(g, ik)
            assert info["npw"][ik] == len(gs["idx"])
            np.testing.assert_array_equal(idx, gs["idx"])          # index work: bit-exact
            np.testing.assert_array_equal(mil, gs["miller"])
            np.testing.assert_allclose(kpg, gs["q"], rtol=0, atol=1e-12)
    finally:
        Q.qm_gspace_destroy(g)


def test_grid_rule_without_override_matches_oracle():
    import paper_2308_07277_gb300 as Q
    for cell in S.small_cells() + [S.config5()]:
        g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, None)
        try:
            assert Q.qm_gspace_query(g)["grid"] == OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
        finally:
            Q.qm_gspace_destroy(g)


def test_fe_example_through_the_abi():
    """The paper's printed GSpace example (Section 4.3.2) through the C ABI, using the
    density cutoff as the sphere cutoff exactly as the example does."""
    import paper_2308_07277_gb300 as Q
    alat = 5.107
    lat = alat * 0.5 * np.array([[1, 1, 1], [-1, 1, 1], [-1, -1, 1]], float)
    # grid from the density cutoff 160 Ry = 80 Ha: the rule takes the wavefunction cutoff
    # E_c and uses 4 E_c, so pass the grid explicitly
    g = Q.qm_gspace_create(lat, [[0, 0, 0]], 80.0, (18, 18, 18))
    try:
        info = Q.qm_gspace_query(g)
        assert info["npw"] == [2243]
        idx, mil, kpg = Q.qm_gspace_indices(g, 0)
        g2 = (kpg ** 2).sum(1)
        np.testing.assert_array_equal(np.round(g2[:5], 1), [0.0, 3.0, 12.1, 27.2, 48.4])
        np.testing.assert_array_equal(np.round(g2[-5:], 1), [78.7, 51.5, 30.3, 15.1, 6.1])
        np.testing.assert_array_equal(mil[:5, 0], [0, 1, 2, 3, 4])
    finally:
        Q.qm_gspace_destroy(g)


def test_argument_errors_are_reported_not_crashed():
    import paper_2308_07277_gb300 as Q
    lib = _lib()
    lat = np.eye(3) * 10.0
    with pytest.raises(Q.QMError) as e:
        Q.qm_gspace_create(lat, [[0, 0, 0]], -1.0)
    assert e.value.status == 1
    with pytest.raises(Q.QMError):
        Q.qm_gspace_create(np.zeros((3, 3)), [[0, 0, 0]], 5.0)
    with pytest.raises(Q.QMError):
        Q.qm_gspace_create(lat, [[0, 0, 0]], 5.0, (7, 8, 9))          # 7 is not 2,3,5-smooth
    with pytest.raises(Q.QMError):
        Q.qm_gspace_create(lat, [[0, 0, 0]], 50.0, (8, 8, 8))          # sphere does not fit
    g = Q.qm_gspace_create(lat, [[0, 0, 0]], 5.0)
    try:
        # NULL psi with nb > 0 -> QM_ERR_ARG before any device work
        st = lib.qm_hpsi(g, 0, 4, None, 10 ** 6, None, 0, None, 0, None, None, 10 ** 6, 0, None)
        assert st == 1 and "NULL" in Q.qm_last_error()
        st = lib.qm_hpsi(g, 5, 4, None, 0, None, 0, None, 0, None, None, 0, 0, None)
        assert st == 1 and "ik" in Q.qm_last_error()
        assert lib.qm_hpsi(g, 0, 0, None, 0, None, 0, None, 0, None, None, 0, 0, None) == 0
        assert lib.qm_hpsi(None, 0, 1, None, 0, None, 0, None, 0, None, None, 0, 0, None) == 1
    finally:
        Q.qm_gspace_destroy(g)
    lib.qm_gspace_destroy(None)


def test_davidson_option_errors_before_device_work():
    """qm_davidson validates its options (precision, preconditioner, mixed_ortho, nvecx, tol)
    and reports QM_ERR_ARG before it touches the device: the pointers below are never
    dereferenced."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    from paper_2308_07277_gb300 import _lib as L
    lib = _lib()
    g = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0]], 5.0)
    try:
        npw = Q.qm_gspace_query(g)["npw"][0]
        fake = ctypes.c_void_p(1 << 20)  # 16-byte aligned, never read
        eig = np.zeros(4)
        cases = [dict(prec=7), dict(precond=3), dict(precond=1), dict(mixed_ortho=2), dict(nvecx=5),
                 dict(tol=-1.0), dict(max_iter=-2), dict(fp64_exact=2)]
        msgs = ["unknown precision", "unknown preconditioner", "learned preconditioner without parameters",
                "mixed_ortho", "nvecx", "tol", "tol", "fp64_exact"]
        for kw, msg in zip(cases, msgs):
            opts = L.DavidsonOpts(**dict(dict(tol=1e-8, max_iter=10), **kw))
            st = lib.qm_davidson(g, 0, 4, fake, npw, fake, 0, None, 0, None, ctypes.byref(opts),
                                 eig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, None)
            assert st == 1 and msg in Q.qm_last_error(), (kw, st, Q.qm_last_error())
    finally:
        Q.qm_gspace_destroy(g)


def test_precond_apply_errors_before_device_work():
    """qm_precond_apply checks its arguments (band count, preconditioner, parameters, NULL
    buffers, leading dimension, alignment) and reports QM_ERR_ARG before any device work;
    n = 0 is a no-op."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    lib = _lib()
    g = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0]], 5.0)
    try:
        npw = Q.qm_gspace_query(g)["npw"][0]
        f = ctypes.c_void_p(1 << 20)      # aligned, never read
        odd = ctypes.c_void_p((1 << 20) + 8)
        cases = [((0, -1, f, f, npw, f, 0, None, None, f, f, f, f), "n"),
                 ((0, 70000, f, f, npw, f, 0, None, None, f, f, f, f), "n"),
                 ((3, 2, f, f, npw, f, 0, None, None, f, f, f, f), "ik"),
                 ((0, 2, f, f, npw, f, 2, None, None, f, f, f, f), "unknown preconditioner"),
                 ((0, 2, f, f, npw, f, 1, None, f, f, f, f, f), "without parameters"),
                 ((0, 2, f, f, npw, f, 1, f, None, f, f, f, f), "H diagonal"),
                 ((0, 2, None, f, npw, f, 0, None, None, f, f, f, f), "NULL"),
                 ((0, 2, f, f, npw, f, 0, None, None, f, f, None, f), "NULL"),
                 ((0, 2, f, f, npw - 1, f, 0, None, None, f, f, f, f), "ld < npw"),
                 ((0, 2, f, odd, npw, f, 0, None, None, f, f, f, f), "aligned")]
        for args, msg in cases:
            st = lib.qm_precond_apply(g, *args, None)
            assert st == 1 and msg in Q.qm_last_error(), (args, st, Q.qm_last_error())
        assert lib.qm_precond_apply(g, 0, 0, None, None, 0, None, 0, None, None, None, None, None, None, None) == 0
        assert lib.qm_precond_apply(None, 0, 1, f, f, npw, f, 0, None, None, f, f, f, f, None) == 1
        for args, msg in [((g, 3, f, 0, None, 0, None, f, None), "ik"), ((g, 0, None, 0, None, 0, None, f, None), "NULL"),
                          ((g, 0, f, 4, None, npw, f, f, None), "NULL"), ((g, 0, f, 4, f, npw - 1, f, f, None), "ld_beta")]:
            assert lib.qm_hamiltonian_diag(*args) == 1 and msg in Q.qm_last_error(), (args, Q.qm_last_error())
    finally:
        Q.qm_gspace_destroy(g)


def test_prepare_check_hold_argument_errors():
    """qm_hpsi_prepare, qm_hpsi_check and qm_batch_hold reject bad arguments with QM_ERR_ARG
    before any device work."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    lib = _lib()
    g = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0]], 5.0)
    try:
        npw = Q.qm_gspace_query(g)["npw"][0]
        f = ctypes.c_void_p(1 << 20)
        for args, msg in [((g, 1, 4, f, npw, None), "ik"), ((g, 0, -1, f, npw, None), "negative"),
                          ((g, 0, 4, None, npw, None), "NULL beta"), ((g, 0, 4, f, npw - 1, None), "ld_beta"),
                          ((None, 0, 4, f, npw, None), "NULL gspace")]:
            assert lib.qm_hpsi_prepare(*args) == 1 and msg in Q.qm_last_error(), (args, Q.qm_last_error())
        assert lib.qm_hpsi_check(None, None) == 1
        assert lib.qm_hpsi_check(g, None) == 0           # no workspace yet: nothing to report
    finally:
        Q.qm_gspace_destroy(g)
    assert lib.qm_batch_hold(None, 0, 0) == 1


def test_zgemm_argument_errors_before_device_work():
    """qm_zgemm rejects an unknown op or arithmetic, empty sizes, NULL operands and short
    leading dimensions with QM_ERR_ARG before any device work (the pointers are never read)."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    lib = _lib()
    fake = ctypes.c_void_p(1 << 20)
    cases = [((2, 0, 4, 4, 8, fake, 8, fake, 8, fake, 4), "op not 0/1"),
             ((0, 5, 4, 4, 8, fake, 8, fake, 8, fake, 4), "arith not 0..2"),
             ((0, 1, 0, 4, 8, fake, 8, fake, 8, fake, 4), "bad sizes"),
             ((1, 0, 4, 4, 8, None, 8, fake, 8, fake, 4), "bad sizes"),
             ((0, 0, 4, 4, 8, fake, 7, fake, 8, fake, 4), "leading dimension"),
             ((1, 1, 4, 6, 8, fake, 4, fake, 6, fake, 5), "leading dimension")]
    for args, msg in cases:
        st = lib.qm_zgemm(*args, None)
        assert st == 1 and msg in Q.qm_last_error(), (args, st, Q.qm_last_error())



def test_tddft_argument_errors_before_device_work():
    """qm_tddft_taylor / qm_tddft_etrs reject an order outside [0, 64], a non-finite step, NULL or
    overlapping buffers and short rows with QM_ERR_ARG before any device work (the pointers are
    never read); order 0 and nb 0 return QM_OK without launching."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    lib = _lib()
    g = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0]], 5.0)
    try:
        npw = Q.qm_gspace_query(g)["npw"][0]
        psi = ctypes.c_void_p(1 << 20)
        work = ctypes.c_void_p((1 << 20) + (1 << 24))
        inside = ctypes.c_void_p((1 << 20) + 16 * npw)
        odd = ctypes.c_void_p((1 << 20) + (1 << 24) + 8)
        v = ctypes.c_void_p(1 << 26)
        n0 = lib.qm_launch_count()

        def taylor(ik=0, nb=2, p=psi, ld=npw, dt=0.1, order=4, w=work, prec=0):
            return lib.qm_tddft_taylor(g, ik, nb, p, ld, v, 0, None, 0, None, dt, order, w, prec, None)

        for kw, msg in [({"order": -1}, "order"), ({"order": 65}, "order"), ({"dt": float("nan")}, "dt"),
                        ({"dt": float("inf")}, "dt"), ({"ik": 1}, "ik"), ({"nb": -1}, "negative"),
                        ({"p": None}, "NULL"), ({"w": None}, "NULL"), ({"ld": npw - 1}, "ld_psi"),
                        ({"w": inside}, "overlaps"), ({"w": odd}, "aligned"), ({"prec": 7}, "precision")]:
            assert taylor(**kw) == 1 and msg in Q.qm_last_error(), (kw, Q.qm_last_error())
        assert taylor(order=0) == 0 and taylor(nb=0) == 0
        st = lib.qm_tddft_etrs(g, 0, 2, psi, npw, v, None, 0, None, 0, None, 0.1, 4, work, 0, None)
        assert st == 1 and "potential" in Q.qm_last_error()
        assert lib.qm_tddft_etrs(None, 0, 2, psi, npw, v, v, 0, None, 0, None, 0.1, 4, work, 0, None) == 1
        assert lib.qm_launch_count() == n0
    finally:
        Q.qm_gspace_destroy(g)


def test_hpsi_gamma_rejects_other_k_points():
    """qm_hpsi_gamma needs the Gamma point: any other k-point of the handle is QM_ERR_ARG before
    any device work (the pointers are never read)."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    lib = _lib()
    g = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0], [0.25, 0, 0]], 5.0)
    try:
        npw = Q.qm_gspace_query(g)["npw"][1]
        a, b, v = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 26), ctypes.c_void_p(1 << 28)
        n0 = lib.qm_launch_count()
        st = lib.qm_hpsi_gamma(g, 1, 2, a, npw, v, 0, None, 0, None, b, npw, 0, None)
        assert st == 1 and "Gamma" in Q.qm_last_error()
        assert lib.qm_launch_count() == n0
    finally:
        Q.qm_gspace_destroy(g)


def test_gw_mel_argument_errors_before_device_work():
    """qm_gw_mel rejects handles on different grids, a q that is not k_left - k_right, short rows,
    NULL buffers and bad indices with QM_ERR_ARG before any device work; nl or nr 0 is QM_OK."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    lib = _lib()
    lat = np.eye(3) * 10.0
    g = Q.qm_gspace_create(lat, [[0.25, 0, 0], [0, 0, 0]], 5.0, (20, 20, 20))
    ge = Q.qm_gspace_create(lat, [[0.25, 0, 0]], 2.0, (20, 20, 20))
    ge_grid = Q.qm_gspace_create(lat, [[0.25, 0, 0]], 2.0, (24, 20, 20))
    ge_q = Q.qm_gspace_create(lat, [[0.5, 0, 0]], 2.0, (20, 20, 20))
    try:
        npw = Q.qm_gspace_query(g)["npw"]
        npe = Q.qm_gspace_query(ge)["npw"][0]
        f, h, m = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 24), ctypes.c_void_p(1 << 28)
        n0 = lib.qm_launch_count()

        def call(gw=g, ikl=0, ikr=1, nl=2, pl=f, ldl=npw[0], nr=3, pr=h, ldr=npw[1], e=ge, iq=0, M=m, ldm=npe, prec=0):
            return lib.qm_gw_mel(gw, ikl, ikr, nl, pl, ldl, nr, pr, ldr, e, iq, M, ldm, prec, None)

        for kw, msg in [({"e": ge_grid}, "grids"), ({"e": ge_q}, "not k(ik_left)"), ({"ikl": 2}, "out of range"),
                        ({"iq": 1}, "iq"), ({"nl": -1}, "negative"), ({"pl": None}, "NULL"), ({"M": None}, "NULL"),
                        ({"ldl": npw[0] - 1}, "leading dimension"), ({"ldm": npe - 1}, "leading dimension"),
                        ({"prec": 5}, "precision"), ({"gw": None}, "NULL gspace"),
                        ({"M": ctypes.c_void_p((1 << 28) + 8)}, "aligned")]:
            assert call(**kw) == 1 and msg in Q.qm_last_error(), (kw, Q.qm_last_error())
        assert call(nl=0) == 0 and call(nr=0) == 0
        assert lib.qm_launch_count() == n0
    finally:
        for h_ in (g, ge, ge_grid, ge_q):
            Q.qm_gspace_destroy(h_)


def test_scf_argument_errors_before_device_work():
    """qm_scf rejects bad options, odd or too many electrons, weights that do not sum to 1, NULL
    buffers and a grid that cannot hold the density sphere, with QM_ERR_ARG before device work."""
    import ctypes
    import paper_2308_07277_gb300 as Q
    from paper_2308_07277_gb300 import _lib as L
    lib = _lib()
    g = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0], [0.25, 0, 0]], 3.0)
    small = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0]], 3.0, (12, 12, 12))
    try:
        npw = max(Q.qm_gspace_query(g)["npw"])
        f = ctypes.c_void_p(1 << 20)
        psis = (ctypes.c_void_p * 2)(1 << 20, 1 << 24)
        eig = np.zeros(8)
        n0 = lib.qm_launch_count()

        def call(h=g, nelec=2, w=(0.5, 0.5), nb=4, p=psis, ld=npw, opts=None, out=f):
            wa = np.ascontiguousarray(np.asarray(w, np.float64))
            return lib.qm_scf(h, nelec, wa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nb, p, ld, f, 0, None, 0,
                              None, opts, eig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out, out, None, None)

        bad = L.ScfOpts(1e-8, 50, 1.5, 4, 1e-9, 100, 0)
        for kw, msg in [({"nelec": 3}, "even"), ({"nelec": 10}, "nb"), ({"w": (0.5, 0.6)}, "weights"),
                        ({"w": (-0.5, 1.5)}, "negative"), ({"ld": npw - 1}, "leading dimension"),
                        ({"out": None}, "NULL"), ({"opts": ctypes.byref(bad)}, "option"),
                        ({"p": (ctypes.c_void_p * 2)(1 << 20, None)}, "NULL psi")]:
            assert call(**kw) == 1 and msg in Q.qm_last_error(), (kw, Q.qm_last_error())
        st = call(h=small, w=(1.0,), ld=Q.qm_gspace_query(small)["npw"][0])
        assert st == 1 and "density sphere" in Q.qm_last_error(), Q.qm_last_error()
        assert lib.qm_launch_count() == n0
    finally:
        Q.qm_gspace_destroy(small)
        Q.qm_gspace_destroy(g)


@pytest.mark.parametrize("cell", [S.config1(), S.config4(), S.small_cells()[2], S.cubic_si8(12.0, reps=(2, 1, 1))],
                         ids=["si2_24", "si216_90", "si2_25", "si8x211"])
def test_sticks_and_gamma_tiles(cell):
    """The x-stick list equals the oracle sphere's distinct (i2, i3) in flat order; at the Gamma
    point every stick sits in exactly one tile slot, beside the slot of its partner (-i2, -i3) (the
    partner of the partner is the slot itself), empty slots are marked -1; elsewhere no tiles."""
    import paper_2308_07277_gb300 as Q
    grid = tuple(cell.grid) if cell.grid else OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
    kpts = [[0, 0, 0], [0.25, -0.25, 0.25]]
    g = Q.qm_gspace_create(cell.lattice, kpts, cell.ecut_ha, grid)
    try:
        n1, n2, n3 = grid
        for ik, k in enumerate(kpts):
            gs = OG.gsphere(cell.lattice, grid, cell.ecut_ha, k)
            keys = np.unique(gs["idx"] // n1)
            yz, tiles = Q.qm_gspace_sticks(g, ik)
            np.testing.assert_array_equal(yz[:, 0] + n2 * yz[:, 1], keys)
            if ik == 1:
                assert tiles.shape[0] == 0
                continue
            st, par = tiles[..., 0], tiles[..., 1]
            used = st[st >= 0]
            assert sorted(used.tolist()) == list(range(len(keys)))
            for t in range(tiles.shape[0]):
                for j in range(32):
                    s = st[t, j]
                    if s < 0:
                        continue
                    p = par[t, j]
                    assert 0 <= p < 32 and par[t, p] == j
                    i2, i3 = yz[s]
                    assert tuple(yz[st[t, p]]) == ((-i2) % n2, (-i3) % n3)
    finally:
        Q.qm_gspace_destroy(g)


def test_bindings_refuse_host_tensors():
    """Every compute call of the binding refuses CPU tensors (there is no CPU path): the H psi
    forms, real-time propagation, GW matrix elements and self-consistency."""
    import torch
    import paper_2308_07277_gb300 as Q
    g = Q.qm_gspace_create(np.eye(3) * 10.0, [[0, 0, 0]], 3.0)
    try:
        npw = Q.qm_gspace_query(g)["npw"][0]
        nr = int(np.prod(Q.qm_gspace_query(g)["grid"]))
        psi = torch.zeros((2, npw), dtype=torch.complex128)
        v = torch.zeros(nr, dtype=torch.float64)
        calls = [lambda: Q.qm_hpsi(g, 0, psi, v, None, None),
                 lambda: Q.qm_hpsi_gamma(g, 0, psi, v, None, None),
                 lambda: Q.qm_tddft_taylor(g, 0, psi, v, None, None, 0.1, 4),
                 lambda: Q.qm_tddft_etrs(g, 0, psi, v, v, None, None, 0.1, 4),
                 lambda: Q.qm_gw_mel(g, 0, 0, psi, psi, g, 0, npw, M=torch.zeros((4, npw), dtype=torch.complex128)),
                 lambda: Q.qm_scf(g, 2, [1.0], [psi], v, None, torch.zeros(0, dtype=torch.float64))]
        for c in calls:
            with pytest.raises(ValueError, match="CUDA tensor"):
                c()
    finally:
        Q.qm_gspace_destroy(g)

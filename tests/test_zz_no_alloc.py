"""qm_hpsi_noalloc, the allocation-free variant of qm_hpsi for callers that cannot
allocate device memory (e.g. under an allocator that owns the device heap), checked
against qm_hpsi through the C ABI on two calls in a row that share the library's fixed
scratch array, and against the FP64 oracle (padded rows, no projectors, a non-default
stream, a handle whose tables were never uploaded and one that already holds them).
Collected last on purpose: if it fails, a run stopping at the first failure has already run
every other test."""
import numpy as np
import pytest

import qm_synth as S
from oracle import hamiltonian as OH

from cases import band_rel_err, make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-11       # the FP64 H-psi parity tolerance of the other tests
# QM_MIXED: the no-allocation path runs its nonlocal part as FP32 SIMT products, the single
# call as BF16x3 tensor-core products; both are FP32-accurate, so they agree to about the
# FP32 H-psi error (measured up to 3e-7 per band on the 64-atom cell)
TOL_MIXED = 2e-6
TOL_MIXED_NOALLOC = 1e-6         # against the FP64 oracle, per band
TOL_MIXED_NOALLOC_ELEM = 5e-6    # element-wise, relative to the band's largest element


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def _inputs(cell, ik, nb, prec):
    c = make_case(cell, ik, nb=nb)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    return (dev(c["psi"], dt), dev(c["v"], torch.float64), dev(c["beta"], dt), dev(c["D"], torch.float64))


def test_noalloc_matches_hpsi_on_two_calls_in_a_row(Q):
    # call 1: the 64-atom cell (72^3), k-point 1, 64 bands; call 2: the Si2 cell (24^3),
    # a different problem that runs over whatever call 1 left in the shared scratch
    cases = [(S.config2(), 1, 64, "fp64"), (S.config1(), 0, 8, "fp64"), (S.config2(), 2, 32, "mixed")]
    prepared = []
    for cell, ik, nb, prec in cases:
        g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
        psi, v, beta, D = _inputs(cell, ik, nb, prec)
        ref = Q.qm_hpsi(g, ik, psi, v, beta, D, prec=prec)          # allocating path
        outs = [torch.full_like(psi, float("nan")) for _ in range(2)]
        prepared.append((g, ik, psi, v, beta, D, prec, ref, outs))
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]
    for rep in range(2):
        for (g, ik, psi, v, beta, D, prec, ref, outs) in prepared:
            Q.qm_hpsi_noalloc(g, ik, psi, v, beta, D, outs[rep], prec=prec)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # the first use may make the library's fixed array resident (the driver loads device
    # data lazily); nothing beyond it, and nothing at all on the second round of calls
    assert free[0] - free[1] <= Q.QM_HPSI_NOALLOC_SCRATCH_BYTES + (2 << 20), "device memory was allocated"
    assert abs(free[1] - free[2]) < (1 << 20), "device memory was allocated"
    for (g, ik, psi, v, beta, D, prec, ref, outs) in prepared:
        want = ref.cpu().numpy().astype(np.complex128)
        for rep in range(2):
            got = outs[rep].cpu().numpy().astype(np.complex128)
            assert np.all(np.isfinite(got))
            rel = band_rel_err(got, want).max()
            assert rel <= (TOL64 if prec == "fp64" else TOL_MIXED), (prec, rep, rel)
        Q.qm_gspace_destroy(g)


def test_noalloc_rejects_problems_larger_than_its_scratch(Q):
    cell = S.config1()
    # the Si2 cell on a 480^3 grid: V(r) alone needs 885 MB of scratch
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, (480, 480, 480))
    try:
        npw = Q.qm_gspace_query(g)["npw"][0]
        psi = torch.zeros((2, npw), dtype=torch.complex128, device="cuda")
        out = torch.zeros_like(psi)
        v = torch.zeros(480 ** 3, dtype=torch.float64, device="cuda")
        with pytest.raises(Q.QMError) as e:
            Q.qm_hpsi_noalloc(g, 0, psi, v, None, None, out)
        assert e.value.status == 1 and "scratch" in str(e.value)
    finally:
        Q.qm_gspace_destroy(g)


def test_noalloc_matches_oracle_padded_local_only_side_stream(Q):
    """Against the oracle: rows padded beyond npw, with and without projectors, on a side
    stream; first on a handle whose tables only exist on the host (copied into the scratch
    array), then on the same handle after qm_hpsi has uploaded them (read in place)."""
    cell = S.cubic_si8(12.0, nbnd=7, reps=(2, 1, 1), kpts=[[0.25, 0.25, -0.25]])
    c = make_case(cell, 0)
    want = OH.hpsi_fft(c["psi"], c["gs"], c["v"], c["beta"], c["D"])
    want_loc = OH.hpsi_fft(c["psi"], c["gs"], c["v"], None, None)
    npw = c["psi"].shape[1]
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    side = torch.cuda.Stream()
    try:
        for phase in ("host tables", "device tables"):
            for prec, tb, te in (("fp64", TOL64, TOL64), ("mixed", TOL_MIXED_NOALLOC, TOL_MIXED_NOALLOC_ELEM)):
                dt = torch.complex128 if prec == "fp64" else torch.complex64
                psi = torch.zeros((c["psi"].shape[0], npw + 5), dtype=dt, device="cuda")
                psi[:, :npw] = dev(c["psi"], dt)
                v, beta, D = dev(c["v"], torch.float64), dev(c["beta"], dt), dev(c["D"], torch.float64)
                for with_nl, ref in ((True, want), (False, want_loc)):
                    out = torch.full((psi.shape[0], npw + 3), float("nan"), dtype=dt, device="cuda")
                    torch.cuda.synchronize()
                    with torch.cuda.stream(side):
                        Q.qm_hpsi_noalloc(g, 0, psi, v, beta if with_nl else None, D if with_nl else None, out,
                                          prec=prec, stream=side)
                    side.synchronize()
                    got = out[:, :npw].cpu().numpy().astype(np.complex128)
                    rel = band_rel_err(got, ref).max()
                    el = (np.abs(got - ref) / np.abs(ref).max(axis=1, keepdims=True)).max()
                    assert rel <= tb and el <= te, (phase, prec, with_nl, rel, el)
            if phase == "host tables":
                Q.qm_hpsi(g, 0, dev(c["psi"], torch.complex128), dev(c["v"], torch.float64), None, None)
                torch.cuda.synchronize()
    finally:
        Q.qm_gspace_destroy(g)

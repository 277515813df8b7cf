"""Batched H psi (qm_batch_*: every band x k-point x cell in one persistent launch replayed
from a CUDA graph) against the FP64 oracle.

Bars: FP64 1e-11 relative per band; QM_MIXED 1e-6 relative per band (measured up to 1.1e-7 on
these cells: FP32 FFTs and FP32 nonlocal sums over at most ~9,000 plane waves); the batch
equals the per-cell qm_hpsi loop to 1e-13 (FP64: same FFT arithmetic, nonlocal sums in
another order) and to 1e-6 in QM_MIXED (the single call's nonlocal part is the BF16x3
tensor-core product); results do not depend on the launch shape.
"""
import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG
from oracle import hamiltonian as OH

from cases import band_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def grid_rule(cell):
    return OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)


def cell_cases(cell):
    """Oracle spheres and the synthetic inputs of every k-point of a cell (V computed once)."""
    grid = tuple(cell.grid) if cell.grid else grid_rule(cell)
    v = S.vloc_on_grid(cell.lattice, cell.tau, grid, cell.depth, cell.width, ortho_period=cell.ortho_period)
    D = S.dvals(cell.nat)
    out = []
    for ik in range(len(cell.kpts)):
        gs = OG.gsphere(cell.lattice, grid, cell.ecut_ha, cell.kpts[ik])
        out.append({"gs": gs, "v": v, "D": D, "beta": S.beta_of_q(gs["q"], cell.tau, cell.omega, cell.rc),
                    "psi": S.psi_random(cell.seed, cell.nbnd, len(gs["idx"]), stream=ik), "grid": grid})
    return out


def make_batch(Q, cells, prec, drop_proj=()):
    """GSpace handles, job dicts (device tensors) and the host cases of every (cell, k)."""
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    gss, jobs, cases = [], [], []
    for ci, cell in enumerate(cells):
        cc = cell_cases(cell)
        g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cc[0]["grid"])
        gss.append(g)
        v = torch.from_numpy(cc[0]["v"]).cuda()
        D = torch.from_numpy(cc[0]["D"]).cuda()
        for ik, c in enumerate(cc):
            psi = torch.from_numpy(c["psi"]).to(cdt).cuda()
            beta = None if ci in drop_proj else torch.from_numpy(c["beta"]).to(cdt).cuda()
            jobs.append({"g": g.handle, "ik": ik, "psi": psi, "vloc": v, "beta": beta, "D": D,
                         "out": torch.empty_like(psi)})
            cases.append((cell, ik, c, ci in drop_proj))
    return gss, jobs, cases


def oracle_hpsi(c, nproj_off, bands=None):
    psi = c["psi"] if bands is None else c["psi"][bands]
    if nproj_off:
        return OH.hpsi_fft(psi, c["gs"], c["v"], c["beta"][:0], c["D"][:0])
    return OH.hpsi_fft(psi, c["gs"], c["v"], c["beta"], c["D"])


def small_batch_cells():
    """Runtime-plan grids (< 18), 2/3/5 radices, k != 0, N1 != N2, nb = 1 and a few cells of
    the uneven-cell generator with their band counts cut."""
    cells = S.small_cells() + [S.config1()]
    cells[0].nbnd = 1
    gen = S.config3_cells(grid_rule, n=6, seed=11)
    for c in gen:
        c.nbnd = min(c.nbnd, 6)
        c.kpts = c.kpts[:2]
    return cells + gen


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_batch_matches_oracle_small(Q, prec, tol):
    cells = small_batch_cells()
    gss, jobs, cases = make_batch(Q, cells, prec, drop_proj=(2,))
    b = Q.Batch(jobs, prec=prec, ctas_per_sm=2, item_points=2048, group_mb=1)   # several pipelined groups
    b.run()
    b.check()
    info = b.info()
    assert info["candidates"] == 0 and info["group_mb"] == 1 and info["items"] > 0 and info["band_applies"] == sum(j["psi"].shape[0] for j in jobs)
    for j, (cell, ik, c, off) in zip(jobs, cases):
        want = oracle_hpsi(c, off)
        got = j["out"].cpu().numpy().astype(np.complex128)
        err = band_rel_err(got, want).max()
        assert err <= tol, (cell.name, ik, err)
    b.close()


def test_batch_equals_per_cell_loop_and_is_shape_independent(Q):
    """Launch shapes change only the schedule: bitwise the same result; the reversed FFT radix
    order changes the rounding: the same H psi to FP64 round-off (1e-13 against the loop)."""
    cells = small_batch_cells()
    gss, jobs, cases = make_batch(Q, cells, "fp64", drop_proj=(2,))
    outs = []
    shapes = [(1, 1024, -1, 1), (2, 4096, 1, 1), (1, 8192, 2, 1), (2, 2048, -1, 2)]   # FP64: at most 2 CTAs per SM
    for shape in shapes:
        b = Q.Batch(jobs, prec="fp64", ctas_per_sm=shape[0], item_points=shape[1], group_mb=shape[2],
                    fft_order=shape[3])
        assert b.info()["fft_order"] == shape[3] - 1
        b.run()
        b.check()
        outs.append([j["out"].clone() for j in jobs])
        b.run()                                         # replay: bitwise the same
        b.check()
        for a, j in zip(outs[-1], jobs):
            assert torch.equal(a, j["out"])
        b.close()
    for o, shape in zip(outs[1:], shapes[1:]):
        if shape[3] == 1:
            for a, c in zip(outs[0], o):
                assert torch.equal(a, c)
    for j, a, a2 in zip(jobs, outs[0], outs[-1]):
        ref = Q.qm_hpsi(j["g"], j["ik"], j["psi"], j["vloc"], j["beta"], j["D"])
        torch.cuda.synchronize()
        for x in (a, a2):
            rel = (torch.linalg.vector_norm(x - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)).max().item()
            assert rel <= 1e-13, rel


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_batch_uneven_cells_full_size(Q, prec, tol):
    """The 256-cell uneven workload in the autotuned launch: sampled bands of sampled jobs
    against the oracle, every job against the per-cell qm_hpsi loop."""
    cells = S.config3_cells(grid_rule)
    gss, jobs, cases = make_batch(Q, cells, prec)
    b = Q.Batch(jobs, prec=prec)
    info = b.info()
    assert info["candidates"] >= 7 and info["ctas_per_sm"] >= 1 and info["cells"] == 256 and info["fft_order"] in (0, 1)
    b.run()
    b.check()
    njob = len(jobs)
    sizes = np.array([np.prod(c[2]["grid"]) * c[2]["psi"].shape[0] for c in cases])
    pick = sorted(set([int(np.argmax(sizes)), int(np.argmin(sizes)), 0, njob - 1] +
                      list(np.random.default_rng(5).choice(njob, 8, replace=False))))
    for jj in pick:
        cell, ik, c, off = cases[jj]
        nb = c["psi"].shape[0]
        bands = sorted(set([0, nb - 1, nb // 2]))
        want = oracle_hpsi(c, off, bands)
        got = jobs[jj]["out"][bands].cpu().numpy().astype(np.complex128)
        err = band_rel_err(got, want).max()
        assert err <= tol, (cell.name, ik, err)
    loop_tol = 1e-13 if prec == "fp64" else 1e-6
    for j in jobs:
        ref = Q.qm_hpsi(j["g"], j["ik"], j["psi"], j["vloc"], j["beta"], j["D"], prec=prec)
        torch.cuda.synchronize()
        d = (torch.linalg.vector_norm(j["out"] - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)).max().item()
        assert d <= loop_tol, d
    b.close()


def test_batch_errors(Q):
    cells = [S.config1(), S.fcc_si2(16.0, nbnd=3)]
    gss, jobs, cases = make_batch(Q, cells, "fp64")
    bad = [dict(jobs[0]), dict(jobs[1])]
    bad[1]["out"] = bad[0]["out"][:3]                    # overlapping out blocks
    with pytest.raises(Q.QMError) as e:
        Q.Batch(bad, ctas_per_sm=1, item_points=2048, group_mb=-1)
    assert e.value.status == 1
    with pytest.raises(Q.QMError) as e:
        Q.Batch(jobs, ctas_per_sm=9, item_points=2048, group_mb=-1)   # shape out of range
    assert e.value.status == 1
    with pytest.raises(Q.QMError) as e:
        Q.Batch(jobs, ctas_per_sm=8, item_points=65536, group_mb=-1)  # does not fit an SM
    assert e.value.status == 7
    alias = [dict(jobs[0])]
    alias[0]["out"] = alias[0]["psi"]                    # out == psi
    with pytest.raises(Q.QMError):
        Q.Batch(alias, ctas_per_sm=1, item_points=2048, group_mb=-1)

"""Failure detection without faulting the GPU: every device-side wait of the library is
bounded, and an expired wait or a non-finite value comes back as a status the host reads.

- The batched form's bounded waits: a host-side hook (qm_batch_hold) withholds one completion
  from one job's last phase with a short poll limit, so its waits expire; qm_batch_check must
  report QM_ERR_TIMEOUT, and after the hook is released the next replay must succeed and give
  the per-call result.  Nothing faults: the waiting CTAs give up and return.
- Non-finite input: a NaN planted in psi on the host must make qm_davidson return
  QM_ERR_NUMERIC (the starting block loses rank) instead of running on garbage.
"""
import numpy as np
import pytest

import qm_synth as S
from oracle import gspace as OG

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QM_ERR_NUMERIC, QM_ERR_TIMEOUT = 5, 6


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def _jobs(Q, cells, prec):
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    gss, jobs = [], []
    for cell in cells:
        grid = tuple(cell.grid) if cell.grid else OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)
        g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, grid)
        gss.append(g)
        v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, grid)).cuda()
        D = torch.from_numpy(S.dvals(cell.nat)).cuda()
        for ik in range(len(cell.kpts)):
            _, _, kpg = g.indices(ik)
            psi = torch.from_numpy(S.psi_random(cell.seed, cell.nbnd, g.npw[ik], stream=ik)).to(cdt).cuda()
            beta = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).to(cdt).cuda()
            jobs.append({"g": g.handle, "ik": ik, "psi": psi, "vloc": v, "beta": beta, "D": D,
                         "out": torch.empty_like(psi)})
    return gss, jobs


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_wait_expires_and_recovers(Q, prec):
    cells = [S.config1(), S.fcc_si2(16.0, nbnd=5, kpts=[[0.25, -0.25, 0.25]])]
    gss, jobs = _jobs(Q, cells, prec)
    b = Q.Batch(jobs, prec=prec, ctas_per_sm=1, item_points=2048, group_mb=-1)
    try:
        b.run()
        b.check()
        good = [j["out"].clone() for j in jobs]
        b.hold(1, spin_limit=2000)          # job 1's last phase waits for a completion that never comes
        b.run()
        with pytest.raises(Q.QMError) as e:
            b.check()
        assert e.value.status == QM_ERR_TIMEOUT
        b.hold(-1)                          # released: the next replay is whole again
        for j in jobs:
            j["out"].zero_()
        b.run()
        b.check()
        for j, a in zip(jobs, good):
            assert torch.equal(j["out"], a)
    finally:
        b.close()
        for g in gss:
            g.close()


def test_davidson_reports_nan_input(Q):
    cell = S.config1()
    g = Q.GSpace(cell.lattice, cell.kpts, cell.ecut_ha, cell.grid)
    try:
        _, _, kpg = g.indices(0)
        v = torch.from_numpy(S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)).cuda()
        beta = torch.from_numpy(S.beta_of_q(kpg, cell.tau, cell.omega)).cuda()
        D = torch.from_numpy(S.dvals(cell.nat)).cuda()
        p = S.psi_random(cell.seed, cell.nbnd, g.npw[0])
        p[3, 17] = np.nan                   # planted on the host, before the upload
        for prec in ("fp64", "mixed"):
            with pytest.raises(Q.QMError) as e:
                Q.qm_davidson(g.handle, 0, torch.from_numpy(p).cuda(), v, beta, D, tol=1e-8, max_iter=20, prec=prec)
            assert e.value.status == QM_ERR_NUMERIC, e.value
        # a clean start on the same handle still works afterwards
        p[3, 17] = 0.5
        eig, info = Q.qm_davidson(g.handle, 0, torch.from_numpy(p).cuda(), v, beta, D, tol=1e-8, max_iter=300)
        assert info["converged"]
    finally:
        g.close()


def test_hpsi_check_is_clean_after_normal_calls(Q):
    cell = S.config1()
    gss, jobs = _jobs(Q, [cell], "mixed")
    j = jobs[0]
    try:
        Q.qm_hpsi(j["g"], 0, j["psi"], j["vloc"], j["beta"], j["D"], out=j["out"], prec="mixed")
        from paper_2308_07277_gb300 import _lib
        assert _lib.load().qm_hpsi_check(j["g"], None) == 0
    finally:
        for g in gss:
            g.close()

"""Learned preconditioner on the GPU against the FP64 oracle (oracle/mlp.py).

Bars: network outputs within 2e-3 of a BF16-rounding FP64 emulation and 5e-2 of the plain
FP64 oracle; loss within 1e-2 and gradient within 5e-2 (relative norm) of the oracle at the
BF16-rounded parameters; training samples within FP32 round-off of the oracle's; Davidson with
the trained network reaches the brute-force eigenvalues within 1e-9 Ha.
"""
import numpy as np
import pytest

import qm_synth as S
from oracle import hamiltonian as OH
from oracle import mlp as M
from oracle.precond import tpa_k

from cases import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_07277_gb300 as Q
    return Q


def bf16(x):
    """Round to the nearest BF16 (ties to even), as float64 (finite inputs)."""
    a = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    a = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(theta, F):
    """The oracle's forward with the kernels' BF16 roundings (weights, features, h1, h2; the
    TPA factor takes the unrounded x)."""
    W1, b1, W2, b2, w3, b3 = M.unpack(bf16(theta))
    Fr = bf16(F)
    h1 = bf16(M.silu(Fr @ W1.T + b1))
    h2 = bf16(M.silu(h1 @ W2.T + b2))
    return tpa_k(F[:, 0]) * M.softplus(h2 @ w3 + b3) / np.log(2.0)


def rand_theta(seed):
    th = M.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    th[192:256] = rng.normal(0, 0.3, 64)        # b1
    th[4352:4416] = rng.normal(0, 0.3, 64)      # b2
    th[-1] = 0.2
    return th


def dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_matches_oracle(Q):
    rng = np.random.default_rng(1)
    n = 1000                                     # 7 full tiles of 128 and a ragged tail
    F = np.stack([rng.uniform(0, 6, n), rng.uniform(-2, 1, n), rng.normal(-0.5, 1.0, n)], axis=1)
    th = rand_theta(2)
    K = Q.qm_mlp_forward(dev32(F), dev32(th)).cpu().numpy().astype(np.float64)
    Ke = forward_bf16(th, F)
    Ko, _ = M.forward(th, F)
    assert np.max(np.abs(K - Ke) / np.abs(Ke)) < 2e-3
    assert np.max(np.abs(K - Ko) / np.abs(Ko)) < 5e-2
    assert np.all(K > 0)


def ragged_data(seed):
    rng = np.random.default_rng(seed)
    lens = [300, 177, 257, 129, 64]
    n = sum(lens)
    F = np.stack([rng.uniform(0, 5, n), np.repeat(rng.uniform(-1, 0.5, len(lens)), lens), rng.normal(0, 1, n)], 1)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    r = rng.normal(size=n) + 1j * rng.normal(size=n)
    dstar = (rng.uniform(0.2, 2.0, n) + 0.3j * rng.normal(size=n)) * r + 0.2 * (rng.normal(size=n) + 1j * rng.normal(size=n))
    dstar[off[3]:off[4]] = 0.0                   # a band without a target (D = 0)
    r2 = np.abs(r) ** 2
    c = np.real(np.conj(r) * dstar)
    D = np.add.reduceat(np.abs(dstar) ** 2, off[:-1])
    return F, r2, c, D, off


def test_loss_and_gradient_match_oracle(Q):
    F, r2, c, D, off = ragged_data(3)
    W = np.random.default_rng(8).uniform(0.05, 1.0, D.size)
    th = rand_theta(4)
    loss, g = Q.qm_mlp_loss_grad(torch.from_numpy(off).cuda(), dev32(F), dev32(r2), dev32(c), dev32(D), dev32(th),
                                 W=dev32(W))
    lo, go = M.loss_and_grad(bf16(th), F, r2, c, D, off, W)
    g = g.cpu().numpy().astype(np.float64)
    assert 0.0 <= lo <= 1.0 and abs(loss - lo) <= 1e-2 * max(lo, 0.1), (loss, lo)
    assert np.linalg.norm(g - go) <= 5e-2 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)
    # each parameter block on its own (no block silently wrong)
    for a, b in [(0, 192), (192, 256), (256, 4352), (4352, 4416), (4416, 4480), (4480, 4481)]:
        assert np.linalg.norm(g[a:b] - go[a:b]) <= 1e-1 * np.linalg.norm(go[a:b]) + 1e-6, (a, b)


def test_pairs_match_oracle(Q):
    cell = S.fcc_si2(12.0, nbnd=6)
    c = make_case(cell, 0)
    H = OH.dense_h(c["gs"], c["v"], c["beta"], c["D"])
    lam, U = np.linalg.eigh(H)
    nu = 12
    U = np.ascontiguousarray(U.T[:nu])
    lam = lam[:nu]
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, c["grid"])
    try:
        X = torch.from_numpy(c["psi"]).cuda()
        v, beta, Dd = (torch.from_numpy(a).cuda() for a in (c["v"], c["beta"], c["D"]))
        eps, _ = Q.qm_davidson(g, 0, X, v, beta, Dd, tol=1e-14, max_iter=2, raise_not_converged=False)
        Xh = X.cpu().numpy()
        HX = OH.hpsi_fft(Xh, c["gs"], c["v"], c["beta"], c["D"])
        hd = M.hamiltonian_diagonal(c["gs"]["kin"], c["v"], c["beta"], c["D"])
        f, r2, cc, Dn, Wn = Q.qm_mlp_pairs(g, 0, X, torch.from_numpy(HX).cuda(), torch.from_numpy(eps).cuda(),
                                           torch.from_numpy(hd).cuda(), torch.from_numpy(U).cuda(),
                                           torch.from_numpy(lam).cuda(), 1e-6)
        R = HX - eps[:, None] * Xh
        dstar = M.exact_corrections(Xh, lam, U, 1e-6)
        Fo, r2o, co, Do, Wo = M.samples(c["gs"]["kin"], Xh, R, eps, dstar, hd)
        f, r2, cc, Dn, Wn = (a.cpu().numpy().astype(np.float64) for a in (f, r2, cc, Dn, Wn))
        assert np.max(np.abs(f - Fo)) < 1e-5 * max(1.0, np.abs(Fo).max())
        assert np.max(np.abs(r2 - r2o)) < 1e-6 * r2o.max()
        assert np.max(np.abs(cc - co)) < 1e-5 * np.abs(co).max()
        assert np.allclose(Dn, Do, rtol=1e-5, atol=1e-12)
        assert np.allclose(Wn, Wo, rtol=1e-5, atol=1e-12)
        assert np.any(Do > 0)
    finally:
        Q.qm_gspace_destroy(g)


def small_training_cells():
    cells = []
    for a, ec, nb in [((1, 1, 1), 14.0, 8), ((2, 1, 1), 12.0, 12), ((1, 1, 1), 18.0, 8)]:
        lat, tau = S.fcc_supercell(*a)
        cells.append(S.Cell(f"train_{a}_{ec}", lat, tau, ec, None, nbnd=nb, seed=500 + len(cells),
                            ortho_period=(2 * 10.26,) * 3))
    return cells


def cell_inputs(Q, cell):
    c = make_case(cell, 0, nb=cell.nbnd + 8)
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, c["grid"])
    t = {k: torch.from_numpy(c[k]).cuda() for k in ("v", "beta", "D", "psi")}
    return g, c, t


def test_training_lowers_the_loss_and_davidson_converges_with_it(Q):
    """What the trained network gains over TPA, measured.  Asserted: on its training samples the
    network's weighted correction-direction loss is below TPA's (the gain it is trained for), and
    block Davidson with it reaches the brute-force eigenvalues of a held-out cell.  Measured and
    printed, with loose bounds only: the held-out cell's loss (network vs TPA) and Davidson
    iteration counts.  On these Hamiltonians the gain does not carry over to held-out cells
    (measured: held-out loss 0.731 vs TPA 0.708, iterations within a few of TPA's either way), so
    the bounds catch a broken network, not a missing gain."""
    from paper_2308_07277_gb300 import learned
    parts, gs = [], []
    for cell in small_training_cells():
        g, c, t = cell_inputs(Q, cell)
        gs.append(g)
        parts += learned.collect(g, 0, t["v"], t["beta"], t["D"], t["psi"], cell.nbnd)
    ds = learned.assemble(parts)
    theta = learned.init_theta(1, "cuda")
    hist = learned.train(ds, theta, steps=600, lr=1e-3)
    assert np.all(np.isfinite(hist)) and hist[-1] < hist[0], hist[[0, -1]]
    # the same loss for the TPA factor, and the best any diagonal K reaches (K_G = c_G / |r_G|^2)
    off, F, r2, cc, D, W = (a.cpu().numpy().astype(np.float64) for a in ds)
    off = off.astype(np.int64)
    L_tpa = M.cosine_loss_of_k(tpa_k(F[:, 0]), r2, cc, D, off, W)
    L_best = M.cosine_loss_of_k(cc / np.maximum(r2, 1e-300), r2, cc, D, off, W)
    print(f"training loss {hist[0]:.4f} -> {hist[-1]:.4f}; TPA {L_tpa:.4f}; best diagonal {L_best:.4f}")
    assert L_best <= hist[-1] + 1e-3 and hist[-1] < L_tpa
    # a held-out cell: its own samples, and Davidson with the trained network
    lat, tau = S.fcc_supercell(1, 1, 1)
    cell = S.Cell("heldout", lat, tau, 16.0, None, nbnd=8, kpts=np.array([[0.25, -0.25, 0.25]]), seed=77)
    c = make_case(cell, 0, nb=cell.nbnd + 8)
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, c["grid"])
    gs.append(g)
    t = {k: torch.from_numpy(c[k]).cuda() for k in ("v", "beta", "D", "psi")}
    hold = learned.assemble(learned.collect(g, 0, t["v"], t["beta"], t["D"], t["psi"], cell.nbnd))
    L_net, _ = Q.qm_mlp_loss_grad(hold[0], hold[1], hold[2], hold[3], hold[4], theta, W=hold[5])
    offh, Fh, r2h, cch, Dh, Wh = (a.cpu().numpy().astype(np.float64) for a in hold)
    L_tpa_h = M.cosine_loss_of_k(tpa_k(Fh[:, 0]), r2h, cch, Dh, offh.astype(np.int64), Wh)
    print(f"held-out loss: network {L_net:.4f}, TPA {L_tpa_h:.4f}")
    assert L_net < L_tpa_h + 0.1
    ev = np.linalg.eigvalsh(OH.dense_h(c["gs"], c["v"], c["beta"], c["D"]))[: cell.nbnd]
    its = {}
    for name, mlp in [("tpa", None), ("mlp", theta)]:
        X = t["psi"][: cell.nbnd].clone()
        eig, info = Q.qm_davidson(g, 0, X, t["v"], t["beta"], t["D"], tol=1e-9, max_iter=300, mlp=mlp)
        assert info["converged"]
        np.testing.assert_allclose(eig, ev, atol=1e-9)
        its[name] = (info["iterations"], info["precond_fallback"])
    print("Davidson iterations (tpa, mlp):", its)
    assert its["mlp"][0] <= 1.5 * its["tpa"][0] + 5
    for g in gs:
        Q.qm_gspace_destroy(g)


def test_untrained_network_still_converges(Q):
    """All-zero parameters: K = TPA exactly (z3 = 0), so the learned path must take the same
    iterations as TPA and reach the same eigenvalues."""
    cell = S.fcc_si2(14.0, nbnd=8)
    c = make_case(cell, 0)
    ev = np.linalg.eigvalsh(OH.dense_h(c["gs"], c["v"], c["beta"], c["D"]))[: cell.nbnd]
    g = Q.qm_gspace_create(cell.lattice, cell.kpts, cell.ecut_ha, c["grid"])
    try:
        t = {k: torch.from_numpy(c[k]).cuda() for k in ("v", "beta", "D", "psi")}
        theta = torch.zeros(Q.QM_MLP_NPARAM, dtype=torch.float32, device="cuda")
        X = t["psi"].clone()
        eig, info = Q.qm_davidson(g, 0, X, t["v"], t["beta"], t["D"], tol=1e-9, max_iter=400, mlp=theta)
        assert info["converged"]
        np.testing.assert_allclose(eig, ev, atol=1e-9)
        X = t["psi"].clone()
        eig2, info2 = Q.qm_davidson(g, 0, X, t["v"], t["beta"], t["D"], tol=1e-9, max_iter=400)
        assert abs(info["iterations"] - info2["iterations"]) <= 2, (info["iterations"], info2["iterations"])
        with pytest.raises(ValueError):
            Q.qm_davidson(g, 0, X, t["v"], t["beta"], t["D"], mlp=theta.double())
    finally:
        Q.qm_gspace_destroy(g)

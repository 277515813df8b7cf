"""Kohn-Sham self-consistency around the H psi / Davidson path (Section 2.1: n -> V -> {psi} ->
n_out -> mix; Section 5, dft module scf and mixing), in plain numpy FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Density (Section 2.1, n(r) = sum_i f_i |psi_i(r)|^2): psi_nk(r) = Omega^-1/2 sum_G c_nk(G) e^{i(k+G).r}
with sum_G |c|^2 = 1, so n(r_j) = sum_k w_k sum_n f_n |u_nk(r_j)|^2 / Omega, u(r_j) = sum_G c(G) e^{iG.r_j};
f_n = 2 for the lowest nelec/2 bands (spin-degenerate insulator), w_k the k-point weights.

Potential (Section 2.1, V_aux = V_ext + V_Hartree + V_xc):
  Hartree: V_H(G) = 4 pi n(G) / |G|^2 on the density sphere |G|^2/2 <= 4 E_c (the dual cutoff of
  Section 2.2) without G = 0 (neutralising background), n(G) = (1/N_r) sum_j n_j e^{-iG.r_j}.
  Exchange-correlation: local density approximation, Slater exchange and the Perdew-Zunger
  parametrisation of the Ceperley-Alder correlation energy of the unpolarised electron gas
  (J. P. Perdew and A. Zunger, Phys. Rev. B 23, 5048 (1981), Appendix C), v_xc = d(n eps_xc)/dn.
  (Readings: the paper names Libxc functionals; LDA is the closed-form stand-in.)

Mixing (Section 5: Broyden mixing of the densities): Anderson mixing of the density residual
F = n_out - n_in with the last m differences (D. G. Anderson, J. ACM 12, 547 (1965)); Johnson's
modified Broyden scheme with equal weights is the same update (V. Eyert, J. Comput. Phys. 124,
271 (1996)).  Convergence: (Omega / N_r) sum_j |n_out - n_in| <= tol (electrons).
"""
from __future__ import annotations

import math

import numpy as np

from . import gspace as OG
from . import hamiltonian as OH

# Perdew-Zunger 1981 constants (unpolarised): r_s >= 1 and r_s < 1 branches
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def _box(grid):
    n1, n2, n3 = grid
    return (n3, n2, n1)


def density(coefs, spheres, weights, nocc, omega):
    """n(r) (N_r,) from the lowest nocc bands of every k-point, occupation 2."""
    grid = spheres[0]["grid"]
    nr = grid[0] * grid[1] * grid[2]
    n = np.zeros(nr)
    for c, gs, w in zip(coefs, spheres, weights):
        box = np.zeros((nocc, nr), np.complex128)
        box[:, gs["idx"]] = c[:nocc]
        u = nr * np.fft.ifftn(box.reshape((nocc,) + _box(grid)), axes=(1, 2, 3)).reshape(nocc, nr)
        n += w * 2.0 * (np.abs(u) ** 2).sum(axis=0) / omega
    return n


def hartree(n, lattice, grid, ecut_rho):
    """V_H(r) from n(r) (both flat, x fastest) with the density sphere of cutoff ecut_rho (Ha)."""
    gs = OG.gsphere(lattice, grid, ecut_rho, (0.0, 0.0, 0.0))
    nr = len(n)
    ng = np.fft.fftn(n.reshape(_box(grid))).reshape(-1)[gs["idx"]] / nr
    g2 = 2.0 * gs["kin"]
    vg = np.zeros_like(ng)
    nz = g2 > 0
    vg[nz] = 4.0 * math.pi * ng[nz] / g2[nz]
    box = np.zeros(nr, np.complex128)
    box[gs["idx"]] = vg
    return (nr * np.fft.ifftn(box.reshape(_box(grid)))).reshape(-1).real


RHO_FLOOR = 1e-12   # densities at or below this (mixing may overshoot) get eps_xc = v_xc = 0


def lda(n):
    """(eps_xc, v_xc) per electron (Ha) of the unpolarised electron gas; 0 where n <= RHO_FLOOR."""
    n = np.asarray(n, float)
    small = n <= RHO_FLOOR
    n = np.where(small, 1.0, n)
    rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    cx = 0.75 * (3.0 / (2.0 * math.pi)) ** (2.0 / 3.0)          # eps_x = -cx / rs
    ex = -cx / rs
    vx = 4.0 / 3.0 * ex
    ec = np.empty_like(rs)
    vc = np.empty_like(rs)
    hi = rs >= 1.0
    sq = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * sq + 4.0 / 3.0 * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    r, lr = rs[lo], np.log(rs[lo])
    ec[lo] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    vc[lo] = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * r * lr + (2.0 * PZ_D - PZ_C) / 3.0 * r
    return np.where(small, 0.0, ex + ec), np.where(small, 0.0, vx + vc)


def potential(n, vion, lattice, grid, ecut_rho):
    """V_aux = V_ext + V_H + V_xc on the grid."""
    return vion + hartree(n, lattice, grid, ecut_rho) + lda(n)[1]


class Anderson:
    """x_{i+1} = x_i + a F_i - (dX + a dF) gamma, gamma = argmin ||F_i - dF gamma||_2 over the last m
    differences dX_j = x_{j+1} - x_j, dF_j = F_{j+1} - F_j (m = 0: linear mixing)."""

    def __init__(self, alpha, m):
        self.alpha, self.m = alpha, m
        self.x = self.f = None
        self.dx, self.df = [], []

    def step(self, x, f):
        if self.x is not None and self.m > 0:
            self.dx.append(x - self.x)
            self.df.append(f - self.f)
            self.dx, self.df = self.dx[-self.m:], self.df[-self.m:]
        self.x, self.f = x.copy(), f.copy()
        new = x + self.alpha * f
        if self.df:
            dF = np.stack(self.df, axis=1)
            dX = np.stack(self.dx, axis=1)
            gamma = np.linalg.lstsq(dF, f, rcond=None)[0]
            new = new - (dX + self.alpha * dF) @ gamma
        return new


def scf(lattice, omega, ecut_ha, grid, kpts, weights, nelec, nbnd, vion, betas, D, tol=1e-9, alpha=0.5, history=4,
        max_iter=60):
    """Self-consistent density by dense diagonalisation of H at every k-point (tiny cells); betas[k]
    are the projectors on the sphere of kpts[k] (oracle.gspace.gsphere order).  Starts from the
    uniform density; returns (eigenvalues (nk, nbnd), n_in at convergence, V_aux, iterations)."""
    grid = tuple(grid)
    spheres = [OG.gsphere(lattice, grid, ecut_ha, k) for k in kpts]
    nr = grid[0] * grid[1] * grid[2]
    nocc = nelec // 2
    n_in = np.full(nr, nelec / omega)
    mixer = Anderson(alpha, history)
    for it in range(1, max_iter + 1):
        v = potential(n_in, vion, lattice, grid, 4 * ecut_ha)
        eigs, coefs = [], []
        for gs, beta in zip(spheres, betas):
            w, u = np.linalg.eigh(OH.dense_h(gs, v, beta, D))
            eigs.append(w[:nbnd])
            coefs.append(u[:, :nbnd].T.copy())
        n_out = density(coefs, spheres, weights, nocc, omega)
        f = n_out - n_in
        drho = omega / nr * np.abs(f).sum()
        if drho <= tol:
            return np.array(eigs), n_in, v, it
        n_in = mixer.step(n_in, f)
    raise RuntimeError("oracle SCF did not converge")

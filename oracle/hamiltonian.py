"""H psi in the plane-wave basis, three independent ways.

Operator (Section 2.2, Eq. "KSHamMat", plus the Kleinman-Bylander term of Section 2.3):

    (H psi)(G) = 1/2 |k+G|^2 psi(G)
               + sum_{G' in S_k} Vt((G - G') mod N) psi(G')
               + sum_p beta_p(G) D_p sum_{G'} conj(beta_p(G')) psi(G')

with the grid Fourier coefficient of the local potential
    Vt(g) = (1/N_r) sum_j V(r_j) exp(-i g . r_j),   r_j = sum_i (j_i / N_i) a_i,
which is exactly what the recipe of Section 4.3 (IFFT, multiply by V(r), FFT, keep the
sphere) computes with the r2g convention of Section 4.3.2 (forward = fftn, unnormalised;
inverse = ifftn, 1/N_r).

Arrays: psi (nb, npw) complex128 ordered like the G-sphere; vloc flat real (N_r,), x
fastest; beta (nproj, npw) complex128; D (nproj,) real.
"""
from __future__ import annotations

import math

import numpy as np


def _box_shape(grid):
    n1, n2, n3 = grid
    return (n3, n2, n1)          # numpy C order [i3, i2, i1] == flat x-fastest


def nonlocal_apply(psi, beta, D):
    """sum_p beta_p D_p <beta_p|psi> (Section 2.3, KB form)."""
    if beta is None or beta.shape[0] == 0:
        return np.zeros_like(psi)
    proj = psi @ beta.conj().T              # (nb, nproj): <beta_p | psi_b>
    return (proj * D[None, :]) @ beta


# --------------------------------------------------------------------------- naive DFT
def _phase_table(grid):
    """exp(2 pi i t / N_r) for t = 0..N_r-1 (one table; arguments reduced exactly)."""
    nr = grid[0] * grid[1] * grid[2]
    t = np.arange(nr)
    return np.exp(2j * math.pi * t / nr)


def _phase_index(miller, grid):
    """Integer t[g, j] with  G_g . r_j = 2 pi t / N_r  (mod 2 pi), computed in integers."""
    n1, n2, n3 = grid
    nr = n1 * n2 * n3
    j3, j2, j1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    j1, j2, j3 = j1.reshape(-1), j2.reshape(-1), j3.reshape(-1)      # flat x fastest
    m = np.asarray(miller, np.int64)
    t = (np.outer(m[:, 0], j1) % n1) * (nr // n1)
    t += (np.outer(m[:, 1], j2) % n2) * (nr // n2)
    t += (np.outer(m[:, 2], j3) % n3) * (nr // n3)
    return t % nr


def hpsi_naive(psi, gs, vloc, beta, D):
    """Direct sums over grid points (no FFT).  Cost O(npw * N_r) per band: tiny grids only.

    psi(r_j) = (1/N_r) sum_G psi(G) e^{i G.r_j};  (V psi)(G) = sum_j V_j psi(r_j) e^{-i G.r_j}.
    The common factor e^{i k.r} cancels between the two transforms.
    """
    grid = gs["grid"]
    nr = grid[0] * grid[1] * grid[2]
    E = _phase_table(grid)[_phase_index(gs["miller"], grid)]        # (npw, N_r) e^{iG.r}
    psir = (psi @ E) / nr
    vpsi = (psir * vloc[None, :]) @ E.conj().T
    return gs["kin"][None, :] * psi + vpsi + nonlocal_apply(psi, beta, D)


# --------------------------------------------------------------------------- FFT variant
def hpsi_fft(psi, gs, vloc, beta, D):
    """Full-box (unpruned) numpy FFT variant, same operator (Section 4.3 recipe)."""
    grid = gs["grid"]
    shp = _box_shape(grid)
    nb = psi.shape[0]
    box = np.zeros((nb, grid[0] * grid[1] * grid[2]), np.complex128)
    box[:, gs["idx"]] = psi
    box = np.fft.ifftn(box.reshape((nb,) + shp), axes=(1, 2, 3))
    box *= vloc.reshape(shp)[None]
    box = np.fft.fftn(box, axes=(1, 2, 3)).reshape(nb, -1)
    return gs["kin"][None, :] * psi + box[:, gs["idx"]] + nonlocal_apply(psi, beta, D)


# --------------------------------------------------------------------------- dense H
def vtilde(vloc, grid):
    """Vt(g) = (1/N_r) fftn(V)  on the whole grid, array [g3, g2, g1]."""
    nr = grid[0] * grid[1] * grid[2]
    return np.fft.fftn(vloc.reshape(_box_shape(grid))) / nr


def dense_h(gs, vloc, beta, D):
    """Explicit npw x npw matrix H_{GG'} (brute force)."""
    grid = np.array(gs["grid"])
    vt = vtilde(vloc, gs["grid"])
    m = gs["miller"]
    d = np.mod(m[:, None, :] - m[None, :, :], grid)                 # (G - G') mod N
    H = vt[d[..., 2], d[..., 1], d[..., 0]].astype(np.complex128)
    H[np.diag_indices_from(H)] += gs["kin"]
    if beta is not None and beta.shape[0]:
        H += (beta.T * D[None, :]) @ beta.conj()
    return H

"""G-space: FFT grid rule and the truncated plane-wave sphere.

Definitions followed:
* truncation: keep plane waves with |k + G|^2 / 2 <= E_cut (Section 2.2, after Eq.
  "KSHamMat"; Section 4.3.1, q <= sqrt(2 E_cut));
* the potential needs Fourier components up to the density cutoff 4 E_cut, i.e.
  |G_m - G_n| <= 2 sqrt(2 E_cut) (Section 2.2);
* reciprocal vectors b_i with a_i . b_j = 2 pi delta_ij (Section 4.2, ReciLattice);
* the GSpace example of Section 4.3.2: Fe bcc, alat 5.107 bohr, ecutrho 160 Ry gives an
  (18,18,18) grid with 2243 G-vectors, listed with G_1 varying fastest.

Readings where the paper is silent:
* grid rule: n_i = floor(sqrt(2 E_rho) |a_i| / 2 pi), N_i = smallest 2,3,5-smooth integer
  >= 2 n_i + 1 (reproduces the printed 18^3 / 2243);
* sphere surface: inclusive, with relative slack 1e-12 on E_cut;
* ordering: by flat grid index  i1 + N1 (i2 + N2 i3),  i_j = m_j mod N_j  (G_1 fastest, as
  printed).
"""
from __future__ import annotations

import math

import numpy as np

SPHERE_SLACK = 1e-12


def reciprocal(lattice):
    """Rows b_i = 2 pi (A^-1)^T rows, A rows a_i."""
    return 2.0 * math.pi * np.linalg.inv(np.asarray(lattice, float)).T


def is_smooth235(n: int) -> bool:
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def next_smooth235(n: int) -> int:
    while not is_smooth235(n):
        n += 1
    return n


def fft_grid(lattice, ecut_rho_ha):
    """FFT grid for the density cutoff ecut_rho_ha (Ha)."""
    gmax = math.sqrt(2.0 * ecut_rho_ha)
    out = []
    for a in np.asarray(lattice, float):
        n = int(math.floor(gmax * np.linalg.norm(a) / (2.0 * math.pi)))
        out.append(next_smooth235(2 * n + 1))
    return tuple(out)


def flat_index(miller, grid):
    n1, n2, n3 = grid
    i = np.mod(miller, np.array(grid))
    return i[:, 0] + n1 * (i[:, 1] + n2 * i[:, 2])


def gsphere(lattice, grid, ecut_ha, kpt_cryst=(0.0, 0.0, 0.0)):
    """Plane waves of the sphere |k+G|^2/2 <= ecut_ha, sorted by flat grid index.

    Returns dict with
      miller (npw,3) int   crystal components m of G = sum m_i b_i
      idx    (npw,)  int   flat grid index i1 + N1 (i2 + N2 i3)
      q      (npw,3) float Cartesian k + G (bohr^-1)
      kin    (npw,)  float |k+G|^2 / 2 (Ha)
    """
    lattice = np.asarray(lattice, float)
    b = reciprocal(lattice)
    k = np.asarray(kpt_cryst, float)
    qmax = math.sqrt(2.0 * ecut_ha)
    ranges = []
    for i in range(3):
        # (k+G) . a_i = 2 pi (m_i + k_i)  =>  |m_i + k_i| <= qmax |a_i| / 2 pi
        bound = qmax * np.linalg.norm(lattice[i]) / (2.0 * math.pi)
        ranges.append(np.arange(int(math.floor(-k[i] - bound)) - 1, int(math.ceil(-k[i] + bound)) + 2))
    m = np.stack(np.meshgrid(*ranges, indexing="ij"), axis=-1).reshape(-1, 3)
    q = (m + k) @ b
    kin = 0.5 * np.einsum("ij,ij->i", q, q)
    keep = kin <= ecut_ha * (1.0 + SPHERE_SLACK)
    m, q, kin = m[keep], q[keep], kin[keep]
    idx = flat_index(m, grid)
    order = np.argsort(idx, kind="stable")
    m, q, kin, idx = m[order], q[order], kin[order], idx[order]
    if np.unique(idx).size != idx.size:
        raise ValueError("G-sphere does not fit in the FFT grid (index collision)")
    return {"miller": m, "idx": idx, "q": q, "kin": kin, "grid": tuple(grid)}

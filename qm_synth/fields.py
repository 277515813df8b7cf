"""Synthetic potential, projectors and random wavefunctions.

* V_loc(r): a periodic sum of Gaussians of depth `depth` (Ha) and standard deviation
  `width` (bohr) centred on the atom sites, V(r) = depth * sum_{a,R} exp(-|r-tau_a-R|^2 / (2 w^2)),
  evaluated at the FFT grid points r_j = sum_i (j_i / N_i) a_i.  It stands in for the local
  part of a norm-conserving pseudopotential (Section 2.3).  Returned flat, x fastest:
  flat = j1 + N1 * (j2 + N2 * j3).
* beta(q): unit-norm Gaussian s and p projector functions in the plane-wave basis
  (Kleinman-Bylander form, Section 2.3), one s and three Cartesian p functions per atom,
  evaluated at the Cartesian wavevectors q = k + G the caller supplies:
      beta_s(q)  = Omega^-1/2 2^{3/2} pi^{3/4} rc^{3/2}  exp(-q^2 rc^2 / 2) exp(-i q.tau)
      beta_pa(q) = Omega^-1/2 4 pi^{3/4} rc^{5/2} q_a    exp(-q^2 rc^2 / 2) exp(-i q.tau)
  These are the plane-wave coefficients of the real-space functions
  (pi rc^2)^{-3/4} exp(-r^2/2rc^2) and sqrt(2/(pi^{3/2} rc^5)) x_a exp(-r^2/2rc^2),
  each of unit L2 norm; the (-i)^l phase is dropped (it cancels in beta D beta^H).
* D: diag(5.0, 1.5, 1.5, 1.5) Ha per atom, ordered (s, p_x, p_y, p_z).
* psi_random: complex normal coefficients from a seeded numpy Generator.
"""
from __future__ import annotations

import math

import numpy as np

D_PER_ATOM = (5.0, 1.5, 1.5, 1.5)


def _grid_fractions(grid):
    n1, n2, n3 = grid
    return (np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3)


def _box_sites(lattice, tau, box):
    """Sites of the orthorhombic box [0, box) that carry the lattice-periodic atom set
    (requires each box edge box_d e_d to be a lattice vector)."""
    F = np.diag(box) @ np.linalg.inv(lattice)           # box edges in lattice coordinates
    Fi = np.round(F)
    if not np.allclose(F, Fi, atol=1e-9):
        raise ValueError("ortho_period is not a superlattice of the cell")
    index = int(round(abs(np.linalg.det(Fi))))          # lattice points per box
    n = np.arange(index)
    shifts = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3) @ lattice
    pts = np.mod((tau[:, None, :] + shifts[None, :, :]).reshape(-1, 3), box)
    pts = np.where(np.isclose(pts, box, atol=1e-9), 0.0, pts)
    pts = np.unique(np.round(pts, 9), axis=0)
    if pts.shape[0] != index * tau.shape[0]:
        raise ValueError("could not place the cell's atoms in the ortho_period box")
    return pts


def vloc_on_grid(lattice, tau, grid, depth=-1.5, width=1.0, tail=1e-18, ortho_period=None):
    """Gaussian-sum potential on the grid, flat, x fastest (float64, length N1*N2*N3).

    Images R are summed while exp(-d^2/2w^2) can exceed `tail`.  ``ortho_period`` =
    (L1, L2, L3): an orthorhombic box whose edges are lattice vectors of the cell; the
    same periodic sum is then evaluated as a sum over the box's sites of products of three
    1D periodic Gaussian sums (exact; much faster for non-orthorhombic cells).
    """
    lattice = np.asarray(lattice, float)
    tau = np.atleast_2d(np.asarray(tau, float))
    n1, n2, n3 = (int(x) for x in grid)
    rcut = width * math.sqrt(2.0 * math.log(1.0 / tail))
    fx, fy, fz = _grid_fractions((n1, n2, n3))
    if ortho_period is not None:
        box = np.asarray(ortho_period, float)
        sites = _box_sites(lattice, tau, box)
        F = np.stack(np.meshgrid(fx, fy, fz, indexing="ij"), axis=-1).transpose(2, 1, 0, 3).reshape(-1, 3)
        r = F @ lattice                                                 # grid points, x fastest
        facs, codes = [], []
        for axis in range(3):
            u, inv = np.unique(sites[:, axis], return_inverse=True)
            nmax = int(math.ceil(rcut / box[axis])) + 1
            # the factor depends on the coordinate only: evaluate it on the distinct values
            xs, xinv = np.unique(np.mod(r[:, axis], box[axis]), return_inverse=True)
            fac = np.zeros((xs.size, u.size))
            for img in range(-nmax, nmax + 1):
                d = xs[:, None] - u[None, :] + img * box[axis]
                fac += np.exp(-d * d / (2.0 * width * width))
            facs.append(fac[xinv.reshape(-1)])
            codes.append(inv.reshape(-1))
        # sum over sites of fx[a] fy[b] fz[c] = sum_ab fx[a] fy[b] (sum_c M[a,b,c] fz[c])
        fx_, fy_, fz_ = facs
        M = np.zeros((fx_.shape[1], fy_.shape[1], fz_.shape[1]))
        np.add.at(M, (codes[0], codes[1], codes[2]), 1.0)
        w = (fz_ @ M.reshape(-1, M.shape[2]).T).reshape(r.shape[0], M.shape[0], M.shape[1])
        return depth * np.einsum("na,nb,nab->n", fx_, fy_, w)
    offdiag = lattice - np.diag(np.diag(lattice))
    if np.all(offdiag == 0.0):
        # orthorhombic: the 3D image sum factorises into three 1D image sums
        L = np.diag(lattice)
        facs = []
        for axis, f in enumerate((fx, fy, fz)):
            nmax = int(math.ceil(rcut / L[axis])) + 1
            imgs = np.arange(-nmax, nmax + 1)
            d = (f[None, :, None] * L[axis] - tau[:, axis][:, None, None]
                 + imgs[None, None, :] * L[axis])                       # (nat, N, nimg)
            facs.append(np.exp(-d * d / (2.0 * width * width)).sum(axis=2))  # (nat, N)
        gx, gy, gz = facs
        zy = (gz[:, :, None] * gy[:, None, :]).reshape(tau.shape[0], n3 * n2)  # (nat, N3*N2)
        v = zy.T @ gx                                                   # (N3*N2, N1)
        return (depth * v).reshape(-1)
    # general lattice: explicit image loop
    recip = 2.0 * math.pi * np.linalg.inv(lattice).T
    spacing = 2.0 * math.pi / np.linalg.norm(recip, axis=1)
    nmax = [int(math.ceil(rcut / s + 0.5)) for s in spacing]
    F = np.stack(np.meshgrid(fx, fy, fz, indexing="ij"), axis=-1)        # (N1,N2,N3,3)
    F = F.transpose(2, 1, 0, 3).reshape(-1, 3)                          # x fastest
    tau_f = tau @ np.linalg.inv(lattice)
    v = np.zeros(F.shape[0])
    imgs = np.array([(a, b, c) for a in range(-nmax[0], nmax[0] + 1)
                     for b in range(-nmax[1], nmax[1] + 1)
                     for c in range(-nmax[2], nmax[2] + 1)], float)
    for ta in tau_f:
        d0 = F - ta
        d0 -= np.round(d0)
        for img in imgs:
            d = (d0 + img) @ lattice
            r2 = np.einsum("ij,ij->i", d, d)
            m = r2 < rcut * rcut
            if np.any(m):
                v[m] += np.exp(-r2[m] / (2.0 * width * width))
    return depth * v


def beta_of_q(q, tau, omega, rc=1.0):
    """Projectors (4*nat, npw) complex128 at Cartesian wavevectors q (npw, 3)."""
    q = np.asarray(q, float)
    tau = np.atleast_2d(np.asarray(tau, float))
    q2 = np.einsum("ij,ij->i", q, q)
    g = np.exp(-0.5 * q2 * rc * rc) / math.sqrt(omega)
    cs = 2.0 ** 1.5 * math.pi ** 0.75 * rc ** 1.5
    cp = 4.0 * math.pi ** 0.75 * rc ** 2.5
    out = np.empty((4 * tau.shape[0], q.shape[0]), np.complex128)
    for a, t in enumerate(tau):
        ph = np.exp(-1j * (q @ t)) * g
        out[4 * a + 0] = cs * ph
        out[4 * a + 1] = cp * q[:, 0] * ph
        out[4 * a + 2] = cp * q[:, 1] * ph
        out[4 * a + 3] = cp * q[:, 2] * ph
    return out


def dvals(nat):
    """Diagonal D (4*nat,) float64, per atom (s, p_x, p_y, p_z) = (5.0, 1.5, 1.5, 1.5) Ha."""
    return np.tile(np.array(D_PER_ATOM), nat)


def psi_random(seed, nb, npw, stream=0):
    """Seeded complex normal coefficients (nb, npw) complex128, E|c|^2 = 1."""
    rng = np.random.default_rng([int(seed), int(stream)])
    z = rng.standard_normal((nb, npw, 2))
    return (z[..., 0] + 1j * z[..., 1]) / math.sqrt(2.0)


def psi_random_real(seed, nb, miller, stream=0):
    """Seeded coefficients (nb, npw) complex128 of functions that are real in real space: the
    random numbers of psi_random symmetrised as c(G) = (z(G) + conj(z(-G))) / sqrt(2) over the
    plane-wave list given by its integer indices miller (npw, 3), which must contain -G with
    every G (a Gamma-point sphere)."""
    m = np.asarray(miller, np.int64)
    z = psi_random(seed, nb, len(m), stream)
    pos = {tuple(r): i for i, r in enumerate(m.tolist())}
    neg = np.array([pos[(-a, -b, -c)] for a, b, c in m.tolist()])
    return np.ascontiguousarray((z + z[:, neg].conj()) / math.sqrt(2.0))

"""Seeded parity cases shared by the GPU tests: oracle sphere + synthetic inputs."""
from __future__ import annotations

import numpy as np

import qm_synth as S
from oracle import gspace as OG


def grid_of(cell):
    return tuple(cell.grid) if cell.grid else OG.fft_grid(cell.lattice, 4 * cell.ecut_ha)


def make_case(cell, ik=0, nb=None, seed=None):
    """Oracle G-sphere of k-point ik and the synthetic V, beta, D, psi on it."""
    grid = grid_of(cell)
    gs = OG.gsphere(cell.lattice, grid, cell.ecut_ha, cell.kpts[ik])
    v = S.vloc_on_grid(cell.lattice, cell.tau, grid, cell.depth, cell.width, ortho_period=cell.ortho_period)
    beta = S.beta_of_q(gs["q"], cell.tau, cell.omega, cell.rc)
    D = S.dvals(cell.nat)
    nb = cell.nbnd if nb is None else nb
    psi = S.psi_random(cell.seed if seed is None else seed, nb, len(gs["idx"]), stream=ik)
    return {"gs": gs, "v": v, "beta": beta, "D": D, "psi": psi, "grid": grid}


def band_rel_err(a, b):
    """Per-band ||a - b|| / ||b||."""
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)

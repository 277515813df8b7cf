"""Synthetic Si-like cells (geometry only).

Units are Hartree atomic units (bohr, Hartree); cutoffs are stated in Rydberg as the
workloads state them and halved by the consumers (E_c[Ha] = ecut[Ry] / 2).

Lattice matrices hold the real-space vectors a_1, a_2, a_3 as ROWS, Cartesian bohr.
Atom positions are Cartesian bohr.  k-points are crystal coordinates of the
reciprocal lattice (k = sum_i k_i b_i).

The cells stand in for the paper's Si supercells (Appendix E, Table "gpu_scaling";
Section 6.4), whose pseudopotential files are not available: the diamond-Si geometry
is kept, the pseudopotential is replaced by a Gaussian local potential and Gaussian
s+p Kleinman-Bylander projectors (Section 2.3, KB form).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

A0_SI = 10.26  # conventional diamond-Si lattice constant used by every workload, bohr

# crystal coordinates of the 8 diamond sites in the conventional cubic cell
_DIAMOND8 = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])

# 2x2x2 shifted Monkhorst-Pack grid, crystal coordinates {+-1/4}^3, reduced by
# time reversal (k ~ -k) to four points of equal weight.
KPTS_MP222_SHIFTED = np.array([
    [0.25, 0.25, 0.25], [0.25, 0.25, -0.25], [0.25, -0.25, 0.25], [-0.25, 0.25, 0.25],
])
KPT_GAMMA = np.zeros((1, 3))


@dataclass
class Cell:
    name: str
    lattice: np.ndarray            # (3,3) rows a_i, bohr
    tau: np.ndarray                # (nat,3) Cartesian, bohr
    ecutwfc_ry: float
    grid: tuple | None             # stated FFT grid (N1,N2,N3); None -> grid rule
    kpts: np.ndarray = field(default_factory=lambda: KPT_GAMMA.copy())
    nbnd: int = 8
    depth: float = -1.5            # Gaussian V_loc depth, Ha
    width: float = 1.0             # Gaussian V_loc sigma, bohr
    rc: float = 1.0                # projector radius, bohr
    seed: int = 1
    ortho_period: tuple | None = None  # orthorhombic box whose edges are lattice vectors (fast V_loc)

    @property
    def nat(self) -> int:
        return int(self.tau.shape[0])

    @property
    def nproj(self) -> int:
        return 4 * self.nat

    @property
    def ecut_ha(self) -> float:
        return 0.5 * self.ecutwfc_ry

    @property
    def omega(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))


def fcc_lattice(a: float) -> np.ndarray:
    """fcc primitive vectors (a/2)(-1,0,1), (a/2)(0,1,1), (a/2)(-1,1,0)."""
    return 0.5 * a * np.array([[-1.0, 0.0, 1.0], [0.0, 1.0, 1.0], [-1.0, 1.0, 0.0]])


def fcc_si2(ecutwfc_ry: float = 20.0, grid=None, nbnd: int = 8, kpts=None,
            a: float = A0_SI, seed: int = 1) -> Cell:
    """Two-atom fcc Si-like cell: atoms at 0 and (a/4)(1,1,1)."""
    tau = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    return Cell("fcc_si2", fcc_lattice(a), tau, ecutwfc_ry, grid,
                KPT_GAMMA.copy() if kpts is None else np.asarray(kpts, float), nbnd, seed=seed)


def cubic_supercell(n1: int, n2: int, n3: int, a0: float = A0_SI) -> tuple[np.ndarray, np.ndarray]:
    """Lattice and Cartesian sites of an n1 x n2 x n3 supercell of the 8-atom cube."""
    lat = np.diag([n1 * a0, n2 * a0, n3 * a0])
    sites = []
    for i3 in range(n3):
        for i2 in range(n2):
            for i1 in range(n1):
                sites.append((_DIAMOND8 + np.array([i1, i2, i3])) * a0)
    return lat, np.concatenate(sites, axis=0)


def cubic_si8(ecutwfc_ry: float = 15.0, grid=None, nbnd: int = 16, kpts=None,
              reps=(1, 1, 1), seed: int = 1) -> Cell:
    lat, tau = cubic_supercell(*reps)
    return Cell(f"cubic_si8x{reps[0]}{reps[1]}{reps[2]}", lat, tau, ecutwfc_ry, grid,
                KPT_GAMMA.copy() if kpts is None else np.asarray(kpts, float), nbnd, seed=seed)


def config1() -> Cell:
    """Plain FP64 Si2 cell: fcc a=10.26, 20 Ry, grid 24^3, Gamma, 8 bands."""
    return fcc_si2(20.0, grid=(24, 24, 24), nbnd=8)


def config2() -> Cell:
    """64-atom cubic cell a=20.52, 25 Ry, grid 72^3, 4 shifted k-points, 160 bands."""
    lat, tau = cubic_supercell(2, 2, 2)
    return Cell("si64_cubic", lat, tau, 25.0, (72, 72, 72), KPTS_MP222_SHIFTED.copy(), 160)


def config4(seed: int = 1) -> Cell:
    """216-atom cubic cell a=30.78 with 1 % seeded displacements, 20 Ry, 90^3, Gamma, 480 bands.

    Each Cartesian component is displaced by U(-0.01, 0.01) * a0.
    """
    lat, tau = cubic_supercell(3, 3, 3)
    rng = np.random.default_rng([seed, 4])
    tau = tau + rng.uniform(-0.01, 0.01, size=tau.shape) * A0_SI
    return Cell("si216_cubic_disp", lat, tau, 20.0, (90, 90, 90), KPT_GAMMA.copy(), 480, seed=seed)


def config5() -> Cell:
    """Cell 41.04 x 41.04 x 20.52 bohr (256 diamond sites) with one vacancy (site 0 removed),
    30 Ry, the stated grid 96x96x48, 4 shifted k-points, 288 bands."""
    lat, tau = cubic_supercell(4, 4, 2)
    return Cell("si255_vac", lat, tau[1:], 30.0, (96, 96, 48), KPTS_MP222_SHIFTED.copy(), 288)


def small_cells() -> list[Cell]:
    """Small cells for parity tests: several FFT-tile counts, 2/3/5 radices, ragged sticks,
    unequal grid dimensions, k != 0."""
    return [
        fcc_si2(8.0, nbnd=4),                                          # smallest grid
        fcc_si2(16.0, nbnd=5, kpts=[[0.25, -0.25, 0.25]]),              # 20^3 (radix 5), k != 0
        fcc_si2(30.0, nbnd=3),                                          # 25^3 (5*5)
        cubic_si8(12.0, nbnd=7, reps=(2, 1, 1), kpts=[[0.25, 0.25, -0.25]]),  # N1 != N2 = N3
        cubic_si8(10.0, nbnd=6, reps=(1, 1, 1)),
    ]


# the full 2x2x2 shifted Monkhorst-Pack set {+-1/4}^3 (no symmetry reduction), in a fixed order
KPTS_MP222_SHIFTED_FULL = np.array([[s1, s2, s3] for s1 in (0.25, -0.25) for s2 in (0.25, -0.25)
                                    for s3 in (0.25, -0.25)])


def fcc_supercell(n1: int, n2: int, n3: int, a: float = A0_SI) -> tuple[np.ndarray, np.ndarray]:
    """n1 x n2 x n3 supercell of the two-atom fcc cell: lattice rows n_i a_i, Cartesian sites."""
    prim = fcc_lattice(a)
    basis = np.array([[0.0, 0.0, 0.0], [0.25 * a, 0.25 * a, 0.25 * a]])
    lat = prim * np.array([[n1], [n2], [n3]], float)
    sites = [basis + i1 * prim[0] + i2 * prim[1] + i3 * prim[2]
             for i3 in range(n3) for i2 in range(n2) for i1 in range(n1)]
    return lat, np.concatenate(sites, axis=0)


# the cell families of the batched workload (2-16 atoms)
BATCH_FAMILIES = (("fcc_si2", "fcc", (1, 1, 1)), ("fcc_si4", "fcc", (2, 1, 1)), ("fcc_si8", "fcc", (2, 2, 1)),
                  ("cubic_si8", "cubic", (1, 1, 1)), ("fcc_si16", "fcc", (2, 2, 2)))


def config3_cells(grid_fn, n: int = 256, seed: int = 3, grid_range=(18, 48)) -> list[Cell]:
    """The batched workload: n independent cells of uneven size, cell i drawn from its own
    seeded generator [seed, 3, i].

    Per cell: a family of BATCH_FAMILIES (uniform), ecutwfc ~ U(15, 30) Ry, the FFT grid
    given by ``grid_fn(cell)`` (the caller's grid rule), redrawn until every N_d lies in
    ``grid_range``; then nbnd ~ U{8..48}, nk ~ U{1..8} (the first nk points of
    KPTS_MP222_SHIFTED_FULL) and the V_loc depth -1.5 * (1 + U(-0.2, 0.2)) Ha.
    """
    cells = []
    for i in range(n):
        rng = np.random.default_rng([int(seed), 3, i])
        while True:
            name, kind, reps = BATCH_FAMILIES[int(rng.integers(len(BATCH_FAMILIES)))]
            ecut = float(rng.uniform(15.0, 30.0))
            lat, tau = fcc_supercell(*reps) if kind == "fcc" else cubic_supercell(*reps)
            cell = Cell(f"{name}_{i}", lat, tau, ecut, None)
            grid = tuple(int(x) for x in grid_fn(cell))
            if all(grid_range[0] <= x <= grid_range[1] for x in grid):
                break
        cell.grid = grid
        cell.nbnd = int(rng.integers(8, 49))
        cell.kpts = KPTS_MP222_SHIFTED_FULL[: int(rng.integers(1, 9))].copy()
        cell.depth = -1.5 * (1.0 + float(rng.uniform(-0.2, 0.2)))
        cell.seed = 1000 + i
        cell.ortho_period = (2 * A0_SI,) * 3   # every family is diamond Si: 2 a0 cube is a superlattice
        cells.append(cell)
    return cells

"""Write tests/golden/config2_eigs.txt: the lowest 160 eigenvalues at each of the 4
k-points of the 64-atom cubic Si-like cell (a = 20.52 bohr, 25 Ry, 72^3, 256 projectors),
computed by the FP64 oracle only (oracle.gspace, oracle.hamiltonian.hpsi_fft,
oracle.davidson with residual tolerance 1e-10 Ha).

    python tests/golden/make_config2_eigs.py        (about an hour on 8 cores)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import qm_synth as S  # noqa: E402
from oracle import davidson as OD  # noqa: E402
from oracle import gspace as OG  # noqa: E402
from oracle import hamiltonian as OH  # noqa: E402


def main():
    cell = S.config2()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_eigs.txt")
    v = S.vloc_on_grid(cell.lattice, cell.tau, cell.grid)
    D = S.dvals(cell.nat)
    lines = ["# Lowest 160 eigenvalues (Ha) of H(k) for the 64-atom cubic Si-like cell",
             "# (a = 20.52 bohr, ecutwfc 25 Ry, grid 72^3, 4 shifted k-points, Gaussian V_loc depth -1.5 Ha",
             "# width 1 bohr, s+p Gaussian projectors rc = 1, D = (5, 1.5, 1.5, 1.5) Ha).",
             "# Written by tests/golden/make_config2_eigs.py with the FP64 oracle only",
             "# (oracle.davidson, residual tolerance 1e-10 Ha, start psi_random(seed=1, stream=ik))."]
    for ik in range(len(cell.kpts)):
        t = time.time()
        gs = OG.gsphere(cell.lattice, cell.grid, cell.ecut_ha, cell.kpts[ik])
        beta = S.beta_of_q(gs["q"], cell.tau, cell.omega)
        psi0 = S.psi_random(1, cell.nbnd, len(gs["idx"]), stream=ik)
        e, X, info = OD.davidson(lambda Y: OH.hpsi_fft(Y, gs, v, beta, D), psi0, gs["kin"], tol=1e-10,
                                 max_iter=400)
        assert info["resid"].max() <= 1e-10, info["resid"].max()
        lines.append(f"k{ik} " + " ".join(f"{x:.15f}" for x in e))
        print(f"k{ik}: {info['iterations']} iterations, {time.time() - t:.0f} s", flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()

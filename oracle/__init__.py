"""FP64 CPU oracle for the plane-wave H-psi / block-Davidson path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or runs this
package; only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
It shares no code with the CUDA path: it has its own G-sphere builder, its own H-psi
(naive DFT sums on tiny grids, a full-box numpy FFT variant, and a dense H_GG' matrix),
its own Davidson with the Teter-Payne-Allan preconditioner, written from the paper's
definitions:

* plane-wave Hamiltonian, Eq. "KSHamMat" (Section 2.2), with the cutoff of Section 2.2
  and the dual (4 E_cut) density cutoff;
* Kleinman-Bylander nonlocal form (Section 2.3, KB equation);
* the IFFT -> multiply by V(r) -> FFT recipe of Section 4.3, with the r2g convention
  r2g(f) = fftn(f).take(idxgrid) of the GSpaceBase example (Section 4.3.2);
* Davidson diagonalisation (Section 5, "dft module"), whose details the paper leaves open;
  the readings used are listed in oracle.davidson.

Every function here is pinned by a test under tests/ against something other than
itself (the paper's printed Fe G-space example, closed forms, invariants, brute force).
"""

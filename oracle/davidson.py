"""Plain block Davidson (FP64) for the lowest nb eigenpairs of H(k).

The paper's solver is "Davidson with overlap", modelled on Quantum ESPRESSO's and
matrix free: it only applies H to blocks of trial vectors (Section 5, dft module).  The
paper gives no further details, so this oracle takes these readings:

  (i)   convergence: max_n ||H x_n - eps_n x_n||_2 <= tol with ||x_n||_2 = 1;
  (ii)  basis size limit nvecx = 4 nb (QE default), restart to the current Ritz vectors;
  (iii) corrections delta_n = K r_n (Teter-Payne-Allan, oracle.precond), orthogonalised
        against the basis by two passes of classical Gram-Schmidt and orthonormalised
        among themselves (Cholesky of their Gram matrix), near-dependent ones dropped;
  (iv)  converged bands are kept in the Rayleigh-Ritz step but get no correction;
  (v)   Rayleigh-Ritz solves the generalised problem H_sub c = eps S_sub c in FP64
        (S_sub is kept although the basis is orthonormal, as in the overlap variant).

Steps per iteration: H_sub = V^H (H V), S_sub = V^H V; lowest nb eigenpairs; Ritz
vectors X = c^T V and HX = c^T (HV); residuals; corrections; append or restart.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .precond import tpa_apply


def orthonormalize_rows(X, drop_tol=None):
    """Rows of X made orthonormal in order (Cholesky-QR == Gram-Schmidt, positive diag)."""
    G = X @ X.conj().T                       # G[i,j] = <x_j|x_i>
    L = np.linalg.cholesky(G)
    return sla.solve_triangular(L, X, lower=True)


def davidson(apply_h, psi0, kin, tol=1e-8, max_iter=100, nvecx=None, fixed_iters=None,
             precond=tpa_apply):
    """Returns (eps (nb,), X (nb,npw), info).

    apply_h(Y) -> H Y for a block Y (rows).  With fixed_iters, exactly that many
    Rayleigh-Ritz steps are taken and no convergence test stops the loop.
    """
    nb = psi0.shape[0]
    nvecx = 4 * nb if nvecx is None else nvecx
    V = orthonormalize_rows(np.array(psi0, np.complex128))
    HV = apply_h(V)
    n_hpsi = nb
    hist = []
    eps = X = None
    it = 0
    iters = fixed_iters if fixed_iters is not None else max_iter
    for it in range(1, iters + 1):
        Hs = V.conj() @ HV.T                 # Hs[i,j] = <V_i|H|V_j>
        Hs = 0.5 * (Hs + Hs.conj().T)
        Ss = V.conj() @ V.T
        Ss = 0.5 * (Ss + Ss.conj().T)
        w, C = sla.eigh(Hs, Ss, subset_by_index=[0, nb - 1])
        eps = w
        X = C.T @ V
        HX = C.T @ HV
        nrm = np.linalg.norm(X, axis=1)
        X /= nrm[:, None]
        HX /= nrm[:, None]
        R = HX - eps[:, None] * X
        rn = np.linalg.norm(R, axis=1)
        hist.append((eps.copy(), rn.copy()))
        if fixed_iters is None and rn.max() <= tol:
            break
        if it == iters:
            break
        unc = rn > tol if fixed_iters is None else np.ones(nb, bool)
        if not np.any(unc):
            unc = rn >= rn.max()
        delta = precond(R[unc], X[unc], kin)
        if V.shape[0] + delta.shape[0] > nvecx:
            V, HV = X.copy(), HX.copy()
        for _ in range(2):
            delta = delta - (delta @ V.conj().T) @ V
        nd = np.linalg.norm(delta, axis=1)
        delta = delta[nd > 1e-12 * max(1.0, nd.max())]
        if delta.shape[0] == 0:
            break
        delta /= np.linalg.norm(delta, axis=1)[:, None]
        delta = orthonormalize_rows(delta)
        V = np.vstack([V, delta])
        HV = np.vstack([HV, apply_h(delta)])
        n_hpsi += delta.shape[0]
    info = {"iterations": it, "band_applies": n_hpsi, "history": hist,
            "resid": hist[-1][1] if hist else None}
    return eps, X, info

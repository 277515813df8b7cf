"""Real-time propagation of the Kohn-Sham states (Section 5, "tddft" module): the truncated
Taylor expansion of the propagator and the enforced-time-reversal-symmetry (ETRS) step,
both applied through the oracle's own H psi.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): nothing in the product imports it.

Taylor exponential (Section 5, expoper submodule): exp(-i dt H) is replaced by its power
series cut after the term of order k,

    U_k(dt) psi = sum_{r=0}^{k} (-i dt)^r / r!  H^r psi.

ETRS step (Section 5, prop submodule): psi_{n+1} = U(dt/2; H_{n+1}) U(dt/2; H_n) psi_n, where
H_n = H[psi_n] and H_{n+1} = H[psibar_{n+1}], psibar_{n+1} = U(dt; H_n) psi_n.

Reading: the Hamiltonian of this library has a given local potential (no density
functional: the SCF loop is not part of it), so H depends on the state only through the
potential the caller passes.  The ETRS step therefore takes the potentials of both ends of
the step, V_n and V_{n+1}; the predictor psibar only serves to build H[psibar] in a
self-consistent code and is a plain Taylor step here.  The projectors and D are those of
both ends.
"""
from __future__ import annotations

import numpy as np


def taylor_propagate(apply_h, psi, dt, order):
    """U_k(dt) psi = sum_{r=0}^{order} (-i dt)^r / r! H^r psi, with H^r psi built by repeated
    application (term_r = (-i dt / r) H term_{r-1}, term_0 = psi)."""
    psi = np.asarray(psi, np.complex128)
    out = psi.copy()
    term = psi.copy()
    for r in range(1, order + 1):
        term = (-1j * dt / r) * apply_h(term)
        out = out + term
    return out


def etrs_step(apply_h_now, apply_h_next, psi, dt, order):
    """psi_{n+1} = U_k(dt/2; H_{n+1}) U_k(dt/2; H_n) psi_n (the half step with H_n first)."""
    half = taylor_propagate(apply_h_now, psi, 0.5 * dt, order)
    return taylor_propagate(apply_h_next, half, 0.5 * dt, order)


def taylor_remainder_bound(hnorm, dt, order):
    """Bound on ||exp(-i dt H) - U_k(dt)|| for ||H|| <= hnorm: the tail of the exponential
    series, sum_{r>k} x^r / r! <= x^{k+1}/(k+1)! e^x, x = dt hnorm."""
    x = abs(dt) * hnorm
    f = 1.0
    for r in range(1, order + 2):
        f *= x / r
    return f * np.exp(x)

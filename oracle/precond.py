"""Teter-Payne-Allan diagonal preconditioner (Teter, Payne & Allan, Phys. Rev. B 40,
12255 (1989)).  The paper names no preconditioner for its Davidson (Section 5, dft
module); TPA is the standard diagonal one for plane waves.

    K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),
    x = (|k+G|^2 / 2) / T_n,   T_n = <psi_n| -1/2 nabla^2 |psi_n> / <psi_n|psi_n>.

Reading: T_n is the kinetic energy of the current Ritz vector of band n.
"""
from __future__ import annotations

import numpy as np


def tpa_k(x):
    x = np.asarray(x, float)
    num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x))
    return num / (num + 16.0 * x ** 4)


def tpa_apply(r, x_ritz, kin):
    """delta_n(G) = K(kin(G) / T_n) r_n(G) for each row n."""
    w = np.abs(x_ritz) ** 2
    tn = (w * kin[None, :]).sum(axis=1) / w.sum(axis=1)
    return tpa_k(kin[None, :] / tn[:, None]) * r

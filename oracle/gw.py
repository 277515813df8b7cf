"""Plane-wave matrix elements of the GW module (Section 5, "gw" module, matrix_elements):

    M_nn'(k, q, G) = < n k+q | exp(i (q+G).r) | n' k >,   G with |q+G|^2 / 2 <= E_eps,

two independent ways.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With psi_nk(r) = Omega^-1/2 sum_G c_nk(G) exp(i(k+G).r) the integral over the cell keeps the
terms with G1 = G + G2 (G1 on the sphere of k+q, G2 on the sphere of k):

    M_nn'(G) = sum_{G2} conj(c_{n,k+q}(G + G2)) c_{n',k}(G2).

mel_direct sums that over the Miller indices of the two spheres (no transform).  mel_fft takes
the paper's route: both states to real space on the FFT grid, u(r_j) = sum_G c(G) exp(iG.r_j),
and M(G) = (1/N_r) sum_j conj(u_{n,k+q}(r_j)) u_{n',k}(r_j) exp(+iG.r_j) (numpy ifftn of the
product), read at G; exact when the grid holds every G + G2 without wrap-around (the grid rule's
density grid does for E_eps <= E_wfc).

Arrays: cl (nl, npw_l) on sphere gs_l (k+q), cr (nr, npw_r) on sphere gs_r (k), ge the sphere
of q for E_eps; output (nl * nr, npw_eps), row n * nr + n'.
"""
from __future__ import annotations

import numpy as np


def mel_direct(cl, gs_l, cr, gs_r, ge):
    pos = {tuple(m): i for i, m in enumerate(gs_l["miller"].tolist())}
    nl, nr = cl.shape[0], cr.shape[0]
    out = np.zeros((nl * nr, len(ge["miller"])), np.complex128)
    for ig, mg in enumerate(ge["miller"].tolist()):
        src, dst = [], []
        for i2, m2 in enumerate(gs_r["miller"].tolist()):
            j = pos.get((mg[0] + m2[0], mg[1] + m2[1], mg[2] + m2[2]))
            if j is not None:
                src.append(i2)
                dst.append(j)
        if src:
            # (nl, nr): sum over the matching G2 of conj(c_l(G + G2)) c_r(G2)
            out[:, ig] = (cl[:, dst].conj() @ cr[:, src].T).reshape(-1)
    return out


def _real_space(c, gs):
    n1, n2, n3 = gs["grid"]
    nr = n1 * n2 * n3
    box = np.zeros((c.shape[0], nr), np.complex128)
    box[:, gs["idx"]] = c
    return nr * np.fft.ifftn(box.reshape(-1, n3, n2, n1), axes=(1, 2, 3)).reshape(c.shape[0], nr)


def mel_fft(cl, gs_l, cr, gs_r, ge):
    if tuple(gs_l["grid"]) != tuple(gs_r["grid"]) or tuple(ge["grid"]) != tuple(gs_r["grid"]):
        raise ValueError("the three spheres must share one FFT grid")
    n1, n2, n3 = gs_r["grid"]
    ul, ur = _real_space(cl, gs_l), _real_space(cr, gs_r)
    prod = (ul.conj()[:, None, :] * ur[None, :, :]).reshape(-1, n3, n2, n1)
    m = np.fft.ifftn(prod, axes=(1, 2, 3)).reshape(prod.shape[0], -1)
    return m[:, ge["idx"]]

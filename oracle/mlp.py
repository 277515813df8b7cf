"""Learned preconditioner of the Davidson correction step: plain FP64 CPU reference of the
network, its training samples, its loss and the loss gradient.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU baseline may
import this module.  It shares no code with the CUDA path.

The paper's Davidson (Sec. 5, dft module) uses a diagonal preconditioner; the learned form
replaces the Teter-Payne-Allan factor K(x) (oracle/precond.py) by a small network K(f_G) > 0
evaluated per plane wave, the correction of band n being delta_n(G) = K(f_nG) r_n(G).

Network (3 inputs, two hidden layers of 64, one output):
    z1 = W1 f + b1,  h1 = silu(z1),  z2 = W2 h1 + b2,  h2 = silu(z2),
    z3 = w3 . h2 + b3,  K = K_TPA(x) softplus(z3) / log 2
    silu(z) = z sigma(z),  sigma(z) = 1 / (1 + e^-z),  softplus(z) = log(1 + e^z)
Reading: the network's softplus output is a positive factor on the TPA curve K_TPA(x) of the
same plane wave (x the first feature), normalised so that z3 = 0 gives TPA exactly.  The
network is the correction operator (it replaces TPA in the step); TPA is its prior, so an
untrained network (w3 = 0, b3 = 0) starts from the TPA correction and training can only move
the fit away from it where the samples say so.
Parameters, one flat vector of NPARAM (the layout the library uses):
    W1 (64 x 3, row-major W1[j][k]) | b1 (64) | W2 (64 x 64, W2[j][i]) | b2 (64) | w3 (64) | b3 (1)

Features of plane wave G of band n (scale-free):
    x  = T_G / T_n                 T_G = |k+G|^2 / 2,  T_n = sum_G T_G |psi_n(G)|^2 / sum_G |psi_n(G)|^2
    e  = eps_n / T_n               eps_n: the band's Ritz value
    d  = (H_GG - eps_n) / T_n      H_GG: the diagonal of H(k) in the plane-wave basis,
                                   H_GG = T_G + Vt(0) + sum_p D_p |beta_p(G)|^2 (Eq. KSHamMat with the
                                   KB term; Vt(0) = mean of V(r))
Reading: the correction step's features carry the Hamiltonian's own diagonal, the quantity the
classic Davidson correction (H_GG - eps_n)^-1 r_n(G) divides by, of which TPA keeps only the
kinetic part; none of them depends on the residual, so K r_n stays linear in r_n.

Exact correction (the training target).  Reading: the correction that would turn the Ritz
vector psi_n into its component in the exact eigenspace it converges to,
    delta*_n = P_c psi_n / (psi_n^H P_c psi_n) - psi_n,   P_c = sum_{m in cluster} u_m u_m^H.
The n-th lowest Ritz pair of Davidson converges to the n-th lowest eigenpair, so the cluster of
band n is eigenvalue n together with every eigenvalue within `cluster_tol` of it (degenerate
partners).  delta*_n is orthogonal to psi_n, psi_n + delta*_n lies in the eigenspace, and for
eps_n -> lambda_n it is the exact solution of the Jacobi-Davidson correction equation (Sleijpen &
van der Vorst, SIAM J. Matrix Anal. Appl. 17, 401 (1996)).

Loss.  Davidson orthonormalises every correction against the basis, so only the direction
of K.r_n matters: per band the squared cosine between K.r_n and delta*_n,
    L_n = 1 - B_n^2 / (A_n D_n),  A_n = sum_G K_G^2 |r_G|^2,  B_n = sum_G K_G c_G,
    c_G = Re(conj(r_G) delta*_G),  D_n = ||delta*_n||^2,
and the loss is the weighted mean sum_n W_n L_n / sum_n W_n over the bands with D_n > 0.
Reading of the weights: Davidson stops on its LARGEST residual, so a band counts by its share
of the squared residual of the Ritz pairs it was sampled with, W_n = ||r_n||^2 / sum_m ||r_m||^2
(sum over the bands of that snapshot with D_m > 0); W_n = 1 gives the plain mean.  A training
sample is (f_G, |r_G|^2, c_G) with its band's D_n and W_n.
"""
from __future__ import annotations

import math

import numpy as np

from .precond import tpa_k

HIDDEN = 64
NIN = 3
NPARAM = HIDDEN * NIN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1  # 4481


def unpack(theta):
    """Views (W1, b1, W2, b2, w3, b3) of the flat parameter vector."""
    theta = np.asarray(theta, float)
    assert theta.size == NPARAM
    o = 0
    W1 = theta[o:o + HIDDEN * NIN].reshape(HIDDEN, NIN); o += HIDDEN * NIN
    b1 = theta[o:o + HIDDEN]; o += HIDDEN
    W2 = theta[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = theta[o:o + HIDDEN]; o += HIDDEN
    w3 = theta[o:o + HIDDEN]; o += HIDDEN
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def softplus(z):
    # log(1 + e^z) without overflow
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def init_params(seed):
    """Seeded parameters with every layer active: W ~ N(0, 1/fan_in), zero biases."""
    rng = np.random.default_rng([int(seed), 22])
    W1 = rng.standard_normal((HIDDEN, NIN)) / math.sqrt(NIN)
    W2 = rng.standard_normal((HIDDEN, HIDDEN)) / math.sqrt(HIDDEN)
    w3 = rng.standard_normal(HIDDEN) / math.sqrt(HIDDEN)
    return np.concatenate([W1.ravel(), np.zeros(HIDDEN), W2.ravel(), np.zeros(HIDDEN), w3, [0.0]])


def forward(theta, F):
    """K (n,) and the cached activations for the (n, 3) feature rows F."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    z1 = F @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    z3 = h2 @ w3 + b3
    return tpa_k(F[:, 0]) * softplus(z3) / math.log(2.0), (F, z1, h1, z2, h2, z3)


def hamiltonian_diagonal(kin, vloc, beta, D):
    """H_GG = T_G + Vt(0) + sum_p D_p |beta_p(G)|^2: the diagonal of Eq. KSHamMat with the KB term
    (Vt(0) = (1/N_r) sum_j V(r_j), the G = G' coefficient of the local potential)."""
    h = np.asarray(kin, float) + float(np.mean(vloc))
    if beta is not None and beta.shape[0]:
        h = h + (np.asarray(D, float)[:, None] * np.abs(beta) ** 2).sum(axis=0)
    return h


def features(kin, psi, eps, hdiag):
    """(nb*npw, 3) feature rows (x, e, d), band-major, for Ritz vectors psi with Ritz values eps
    and the Hamiltonian's diagonal hdiag."""
    w = np.abs(psi) ** 2
    tn = (w * kin[None, :]).sum(axis=1) / w.sum(axis=1)
    x = kin[None, :] / tn[:, None]
    e = np.broadcast_to((eps / tn)[:, None], x.shape)
    d = (hdiag[None, :] - eps[:, None]) / tn[:, None]
    return np.stack([x, e, d], axis=-1).reshape(-1, 3)


def exact_corrections(psi, lam, U, cluster_tol):
    """delta*_n for each Ritz vector psi_n (rows, n-th lowest), from exact eigenpairs (lam
    ascending, rows of U the unit eigenvectors): eigenvalue n and its partners within
    cluster_tol define P_c.  A band whose cluster reaches the last given eigenpair may be
    incomplete and gets a zero row (weight 0 in the loss)."""
    nb = psi.shape[0]
    nu = lam.size
    out = np.zeros_like(psi)
    for n in range(min(nb, nu)):
        cl = np.nonzero(np.abs(lam - lam[n]) <= cluster_tol)[0]
        if cl.max() == nu - 1:
            continue                                    # cluster may extend past the given pairs
        Uc = U[cl]                                      # (nc, npw)
        p = Uc.T @ (Uc.conj() @ psi[n])                 # P_c psi_n
        s = np.vdot(psi[n], p)                          # psi_n^H P_c psi_n (real, > 0)
        out[n] = p / s - psi[n]
    return out


def samples(kin, psi, res, eps, dstar, hdiag):
    """Training samples: features (nb*npw, 3), |r|^2 (nb*npw,), c (nb*npw,), D (nb,), W (nb,)."""
    F = features(kin, psi, eps, hdiag)
    r2 = (np.abs(res) ** 2).reshape(-1)
    c = np.real(np.conj(res) * dstar).reshape(-1)
    D = (np.abs(dstar) ** 2).sum(axis=1)
    rn2 = (np.abs(res) ** 2).sum(axis=1)
    W = np.where(D > 0, rn2, 0.0)
    W = W / W.sum() if W.sum() > 0 else W
    return F, r2, c, D, W


def _segsum(x, band_off):
    return np.add.reduceat(x, band_off[:-1], axis=0)


def loss_and_grad(theta, F, r2, c, D, band_off, W=None):
    """Weighted mean cosine loss over the bands with D > 0 and its gradient (NPARAM,).  Samples
    are grouped by band: band n owns samples band_off[n] .. band_off[n+1]-1.  W: per-band
    weights (None = 1)."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    band_off = np.asarray(band_off)
    K, (F_, z1, h1, z2, h2, z3) = forward(theta, F)
    seg = np.repeat(np.arange(D.size), np.diff(band_off))
    A = _segsum(K * K * r2, band_off)
    B = _segsum(K * c, band_off)
    use = D > 0
    Wb = np.where(use, np.ones(D.size) if W is None else np.asarray(W, float), 0.0)
    wsum = Wb.sum()
    safe = np.where(use, A * D, 1.0)
    loss = float(np.sum(Wb * np.where(use, 1.0 - B * B / safe, 0.0)) / wsum)
    coef = Wb * np.where(use, 2.0 * B / safe, 0.0) / wsum
    ratio = np.where(use, B / np.where(use, A, 1.0), 0.0)
    dK = coef[seg] * (ratio[seg] * K * r2 - c)
    dz3 = dK * tpa_k(F[:, 0]) * sigmoid(z3) / math.log(2.0)
    gw3 = h2.T @ dz3
    gb3 = dz3.sum()
    dz2 = (dz3[:, None] * w3[None, :]) * silu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * silu_grad(z1)
    gW1 = dz1.T @ F
    gb1 = dz1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, grad


def cosine_loss_of_k(K, r2, c, D, band_off, W=None):
    """The same loss for a given K per sample (e.g. the TPA factor), for comparisons."""
    band_off = np.asarray(band_off)
    A = _segsum(K * K * r2, band_off)
    B = _segsum(K * c, band_off)
    use = D > 0
    Wb = np.where(use, np.ones(D.size) if W is None else np.asarray(W, float), 0.0)
    return float(np.sum(Wb * np.where(use, 1.0 - B * B / np.where(use, A * D, 1.0), 0.0)) / Wb.sum())

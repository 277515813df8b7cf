"""Training of the learned Davidson preconditioner on samples the method generates itself.

For a cell's k-point: the exact lowest eigenpairs come from a tightly converged Davidson run
(qm_davidson, FP64); Ritz pairs come from Davidson runs stopped after a few Rayleigh-Ritz steps;
qm_mlp_pairs turns each Ritz pair into training samples (features x = T_G/T_n, e = eps_n/T_n,
d = (H_GG - eps_n)/T_n with the Hamiltonian's diagonal from qm_hamiltonian_diag; |r|^2; Re(conj(r) delta*))
against the exact correction delta*; qm_mlp_train fits the network with the library's BF16
forward and backward kernels (full-batch Adam).  Every arithmetic step runs in libqm.so; this
module sequences the calls and concatenates device buffers.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import api as A


def init_theta(seed, device):
    """Seeded initial parameters (QM_MLP_NPARAM float32 on `device`): hidden layers
    W ~ N(0, 1/fan_in) with zero biases, output layer zero, so the untrained network's K is
    the TPA factor exactly."""
    rng = np.random.default_rng([int(seed), 22])
    W1 = rng.standard_normal((64, 3)) / math.sqrt(3.0)
    W2 = rng.standard_normal((64, 64)) / 8.0
    th = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), np.zeros(64), [0.0]])
    assert th.size == A.QM_MLP_NPARAM
    return torch.from_numpy(th.astype(np.float32)).to(device)


def collect(g, ik, vloc, beta, D, psi0, nb, snapshots=(1, 2, 3, 5, 8, 12, 18, 26, 36), cluster_tol=1e-6,
            exact_tol=1e-10, stream=None):
    """Samples of one k-point.  psi0: (nb + extra, ld) complex128 CUDA start block; all rows
    seed the exact run (extra rows buffer the clusters at the top), the first nb rows the
    truncated runs.  Returns a list of (feats, r2, c, D, W) per snapshot."""
    dev = psi0.device
    hd = A.qm_hamiltonian_diag(g, ik, vloc, beta, D, stream=stream)
    U = psi0.clone()
    lam, _ = A.qm_davidson(g, ik, U, vloc, beta, D, tol=exact_tol, max_iter=1000, stream=stream)
    lam_d = torch.from_numpy(lam).to(dev)
    out = []
    for t in snapshots:
        X = psi0[:nb].clone()
        eps, _ = A.qm_davidson(g, ik, X, vloc, beta, D, tol=1e-14, max_iter=int(t), raise_not_converged=False,
                               stream=stream)
        HX = A.qm_hpsi(g, ik, X, vloc, beta, D, stream=stream)
        out.append(A.qm_mlp_pairs(g, ik, X, HX, torch.from_numpy(eps).to(dev), hd, U, lam_d, cluster_tol,
                                  stream=stream))
    return out


def assemble(parts):
    """Concatenate sample sets [(feats, r2, c, D, W), ...] into one training set
    (band_off int64, feats, r2, c, D, W) with samples grouped by band."""
    feats = torch.cat([p[0] for p in parts])
    r2 = torch.cat([p[1] for p in parts])
    c = torch.cat([p[2] for p in parts])
    D = torch.cat([p[3] for p in parts])
    W = torch.cat([p[4] for p in parts])
    counts = []
    for p in parts:
        nb = int(p[3].numel())
        counts += [int(p[1].numel()) // nb] * nb
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return torch.from_numpy(off).to(feats.device), feats, r2, c, D, W


def train(dataset, theta, steps=1500, lr=1e-3, stream=None):
    """Adam on theta (in place) over the whole training set (residual-share band weights);
    returns the loss history."""
    off, feats, r2, c, D, W = dataset
    return A.qm_mlp_train(off, feats, r2, c, D, theta, steps, lr, W=W, stream=stream)

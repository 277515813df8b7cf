"""Thin Python binding over the C ABI (include/qm.h): argument marshalling only.

Function names match the C entry points.  Device buffers are torch CUDA tensors (torch
is used for device memory and streams); every computation runs in libqm.so.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

QM_FP64 = 0
QM_MIXED = 1
QM_HPSI_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024   # include/qm.h
_PREC = {"fp64": QM_FP64, "mixed": QM_MIXED, QM_FP64: QM_FP64, QM_MIXED: QM_MIXED}
STATUS = {0: "QM_OK", 1: "QM_ERR_ARG", 2: "QM_ERR_CUDA", 3: "QM_ERR_OOM", 4: "QM_ERR_NOT_CONVERGED",
          5: "QM_ERR_NUMERIC", 6: "QM_ERR_TIMEOUT", 7: "QM_ERR_UNSUPPORTED"}


class QMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st):
    if st != 0:
        raise QMError(st, _lib.load().qm_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path exists)")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() >= 1 and t.stride(-1) != 1:
        raise ValueError(f"{name} must have unit stride along plane waves")
    return ctypes.c_void_p(t.data_ptr())


def qm_version():
    return _lib.load().qm_version().decode()


def qm_last_error():
    return _lib.load().qm_last_error().decode()


def qm_gspace_create(lattice, kpts, ecutwfc_ha, grid=None):
    """Handle (ctypes.c_void_p) for lattice rows a_i (bohr), kpts (nk,3) crystal, E_c (Ha)."""
    lib = _lib.load()
    lat = np.ascontiguousarray(np.asarray(lattice, np.float64).reshape(9))
    k = np.ascontiguousarray(np.asarray(kpts, np.float64).reshape(-1, 3))
    g = ctypes.c_void_p()
    gr = None
    if grid is not None:
        gr = (ctypes.c_int * 3)(*[int(x) for x in grid])
    _check(lib.qm_gspace_create(_dp(lat), int(k.shape[0]), _dp(k), float(ecutwfc_ha), gr, ctypes.byref(g)))
    return g


def qm_gspace_query(g):
    lib = _lib.load()
    nk = ctypes.c_int()
    _check(lib.qm_gspace_query(g, None, None, None, ctypes.byref(nk)))
    grid = (ctypes.c_int * 3)()
    npw = (ctypes.c_int * nk.value)()
    npw_max = ctypes.c_int()
    _check(lib.qm_gspace_query(g, grid, npw, ctypes.byref(npw_max), None))
    return {"grid": tuple(grid), "npw": list(npw), "npw_max": npw_max.value, "nk": nk.value}


def qm_gspace_indices(g, ik):
    """(idx (npw,) int32, miller (npw,3) int32, kpg (npw,3) float64) for k-point ik."""
    lib = _lib.load()
    npw = qm_gspace_query(g)["npw"][ik]
    idx = np.empty(npw, np.int32)
    mil = np.empty((npw, 3), np.int32)
    kpg = np.empty((npw, 3), np.float64)
    i32 = ctypes.POINTER(ctypes.c_int32)
    _check(lib.qm_gspace_indices(g, int(ik), idx.ctypes.data_as(i32), mil.ctypes.data_as(i32), _dp(kpg)))
    return idx, mil, kpg


def qm_gspace_sticks(g, ik):
    """(stick_yz (nstick, 2) int32, gamma tiles (ngtile, 32, 2) int32) of k-point ik (host tables)."""
    lib = _lib.load()
    ns, nt = ctypes.c_int(), ctypes.c_int()
    _check(lib.qm_gspace_sticks(g, int(ik), ctypes.byref(ns), None, ctypes.byref(nt), None))
    yz = np.empty((ns.value, 2), np.int32)
    tiles = np.empty((nt.value, 32, 2), np.int32)
    i32 = ctypes.POINTER(ctypes.c_int32)
    _check(lib.qm_gspace_sticks(g, int(ik), None, yz.ctypes.data_as(i32), None, tiles.ctypes.data_as(i32)))
    return yz, tiles


def qm_gspace_destroy(g):
    if g is not None and g.value:
        _lib.load().qm_gspace_destroy(g)


def qm_hpsi(g, ik, psi, vloc, beta, D, out=None, prec="fp64", stream=None):
    """out = H(k) psi.  psi (nb, >=npw) complex128 (fp64) or complex64 (mixed) CUDA tensor;
    vloc (N_r,) float64; beta (nproj, >=npw) like psi or None; D (nproj,) float64."""
    lib = _lib.load()
    p = _PREC[prec]
    cdt = torch.complex128 if p == QM_FP64 else torch.complex64
    if psi.dim() != 2:
        raise ValueError("psi must be 2-D (nb, ld)")
    if out is None:
        out = torch.empty_like(psi)
    nproj = 0 if beta is None else int(beta.shape[0])
    _check(lib.qm_hpsi(g, int(ik), int(psi.shape[0]),
                       _dev_ptr(psi, "psi", cdt), int(psi.stride(0)),
                       _dev_ptr(vloc, "vloc", torch.float64),
                       nproj, _dev_ptr(beta, "beta", cdt), int(beta.stride(0)) if nproj else 0,
                       _dev_ptr(D, "D", torch.float64) if nproj else None,
                       _dev_ptr(out, "out", cdt), int(out.stride(0)),
                       p, _stream_ptr(stream)))
    return out


def qm_hpsi_gamma(g, ik, psi, vloc, beta, D, out=None, prec="fp64", stream=None):
    """out = H(Gamma) psi for real-space-real bands (psi(-G) = conj psi(G)), two bands per FFT;
    arguments as qm_hpsi."""
    lib = _lib.load()
    p = _PREC[prec]
    cdt = torch.complex128 if p == QM_FP64 else torch.complex64
    if psi.dim() != 2:
        raise ValueError("psi must be 2-D (nb, ld)")
    if out is None:
        out = torch.empty_like(psi)
    nproj = 0 if beta is None else int(beta.shape[0])
    _check(lib.qm_hpsi_gamma(g, int(ik), int(psi.shape[0]),
                             _dev_ptr(psi, "psi", cdt), int(psi.stride(0)),
                             _dev_ptr(vloc, "vloc", torch.float64),
                             nproj, _dev_ptr(beta, "beta", cdt), int(beta.stride(0)) if nproj else 0,
                             _dev_ptr(D, "D", torch.float64) if nproj else None,
                             _dev_ptr(out, "out", cdt), int(out.stride(0)),
                             p, _stream_ptr(stream)))
    return out


def qm_hpsi_prepare(g, ik, beta, stream=None):
    """Prepare the precision form's projectors of k-point ik (beta: (nproj, >=npw) complex64
    CUDA tensor that stays unchanged while prepared; None releases)."""
    lib = _lib.load()
    nproj = 0 if beta is None else int(beta.shape[0])
    _check(lib.qm_hpsi_prepare(g, int(ik), nproj, _dev_ptr(beta, "beta", torch.complex64),
                               int(beta.stride(0)) if nproj else 0, _stream_ptr(stream)))


def qm_davidson(g, ik, psi, vloc, beta, D, tol=1e-8, max_iter=100, nvecx=0, prec="fp64", stream=None,
                raise_not_converged=True, mixed_switch=0.0, nconv=0, mlp=None, precond_stall=0.0, mixed_ortho=0,
                plain_restart=0, fp64_exact=0):
    """Lowest nb eigenpairs; psi (nb, >=npw) complex128 CUDA tensor is overwritten by the
    Ritz vectors.  Returns (eigenvalues ndarray (nb,), stats dict)."""
    lib = _lib.load()
    if psi.dim() != 2:
        raise ValueError("psi must be 2-D (nb, ld)")
    nb = int(psi.shape[0])
    nproj = 0 if beta is None else int(beta.shape[0])
    hist = np.zeros(max(1, int(max_iter)), np.float64)
    opts = _lib.DavidsonOpts(tol=float(tol), max_iter=int(max_iter), nvecx=int(nvecx), prec=_PREC[prec],
                             precond=0 if mlp is None else 1, mixed_switch=float(mixed_switch), nconv=int(nconv),
                             mixed_ortho=int(mixed_ortho), history=_dp(hist), mlp=_dev_ptr(mlp, "mlp", torch.float32),
                             precond_stall=float(precond_stall), plain_restart=int(plain_restart),
                             fp64_exact=int(fp64_exact))
    stats = _lib.DavidsonStats()
    eig = np.zeros(nb, np.float64)
    st = lib.qm_davidson(g, int(ik), nb, _dev_ptr(psi, "psi", torch.complex128), int(psi.stride(0)),
                         _dev_ptr(vloc, "vloc", torch.float64), nproj,
                         _dev_ptr(beta, "beta", torch.complex128), int(beta.stride(0)) if nproj else 0,
                         _dev_ptr(D, "D", torch.float64) if nproj else None, ctypes.byref(opts), _dp(eig),
                         ctypes.byref(stats), _stream_ptr(stream))
    info = {"iterations": stats.iterations, "converged": bool(stats.converged),
            "band_applies": stats.band_applies, "max_residual": stats.max_residual, "seconds": stats.seconds,
            "iterations_mixed": stats.iterations_mixed, "band_applies_mixed": stats.band_applies_mixed,
            "precond_fallback": stats.precond_fallback, "restarts": stats.restarts,
            "restart_kept": stats.restart_kept,
            "history": hist[: max(0, stats.iterations)].tolist(),
            "status": STATUS.get(st, st)}
    if st != 0 and not (st == 4 and not raise_not_converged):
        _check(st)
    return eig, info


class GSpace:
    """Owning wrapper of a qm_gspace handle."""

    def __init__(self, lattice, kpts, ecutwfc_ha, grid=None):
        self.handle = qm_gspace_create(lattice, kpts, ecutwfc_ha, grid)
        info = qm_gspace_query(self.handle)
        self.grid = info["grid"]
        self.npw = info["npw"]
        self.npw_max = info["npw_max"]
        self.nk = info["nk"]

    def indices(self, ik):
        return qm_gspace_indices(self.handle, ik)

    def hpsi(self, ik, psi, vloc, beta, D, out=None, prec="fp64", stream=None):
        return qm_hpsi(self.handle, ik, psi, vloc, beta, D, out=out, prec=prec, stream=stream)

    def davidson(self, ik, psi, vloc, beta, D, **kw):
        return qm_davidson(self.handle, ik, psi, vloc, beta, D, **kw)

    def close(self):
        if self.handle is not None:
            qm_gspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qm_hpsi_noalloc(g, ik, psi, vloc, beta, D, out, prec="fp64", stream=None):
    """qm_hpsi for callers that cannot allocate device memory: same arguments, but `out`
    must be passed (pre-allocated by the caller) and the library's fixed scratch array is
    used instead of any allocation."""
    lib = _lib.load()
    p = _PREC[prec]
    cdt = torch.complex128 if p == QM_FP64 else torch.complex64
    if psi.dim() != 2 or out is None:
        raise ValueError("psi must be 2-D and out must be given")
    nproj = 0 if beta is None else int(beta.shape[0])
    _check(lib.qm_hpsi_noalloc(g, int(ik), int(psi.shape[0]),
                               _dev_ptr(psi, "psi", cdt), int(psi.stride(0)),
                               _dev_ptr(vloc, "vloc", torch.float64),
                               nproj, _dev_ptr(beta, "beta", cdt), int(beta.stride(0)) if nproj else 0,
                               _dev_ptr(D, "D", torch.float64) if nproj else None,
                               _dev_ptr(out, "out", cdt), int(out.stride(0)),
                               p, _stream_ptr(stream)))
    return out


def qm_precond_apply(g, ik, X, HX, eps, mlp=None, hdiag=None, stream=None):
    """Residuals and Davidson corrections of the n rows of X (n, >=npw) complex128 CUDA tensor
    with HX (same shape and stride) and eps (n,) float64 CUDA tensor; TPA when mlp is None,
    else the network (QM_MLP_NPARAM float32 CUDA tensor) with hdiag (npw,) float64, the
    diagonal of H.  Returns (R, delta, rnorm2, tkin)."""
    lib = _lib.load()
    if X.dim() != 2 or HX.shape != X.shape or HX.stride(0) != X.stride(0):
        raise ValueError("X and HX must be 2-D with the same shape and row stride")
    n = int(X.shape[0])
    R = torch.empty_like(X)
    delta = torch.empty_like(X)
    rn2 = torch.empty(n, dtype=torch.float64, device=X.device)
    tk = torch.empty(n, dtype=torch.float64, device=X.device)
    _check(lib.qm_precond_apply(g, int(ik), n, _dev_ptr(X, "X", torch.complex128),
                                _dev_ptr(HX, "HX", torch.complex128), int(X.stride(0)),
                                _dev_ptr(eps, "eps", torch.float64), 0 if mlp is None else 1,
                                _dev_ptr(mlp, "mlp", torch.float32), _dev_ptr(hdiag, "hdiag", torch.float64),
                                _dev_ptr(R, "R", torch.complex128),
                                _dev_ptr(delta, "delta", torch.complex128), _dev_ptr(rn2, "rnorm2", torch.float64),
                                _dev_ptr(tk, "tkin", torch.float64), _stream_ptr(stream)))
    return R, delta, rn2, tk


def qm_eigh_lowest(A, nev, stream=None):
    """Lowest nev eigenpairs of the Hermitian (m, m) complex128 CUDA tensor A.
    Returns (evals (nev,) float64 CUDA tensor, Y (m, nev) complex128 CUDA tensor)."""
    lib = _lib.load()
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    m = int(A.shape[0])
    ev = torch.empty(nev, dtype=torch.float64, device=A.device)
    Y = torch.empty((m, nev), dtype=torch.complex128, device=A.device)
    _check(lib.qm_eigh_lowest(m, int(nev), _dev_ptr(A, "A", torch.complex128), int(A.stride(0)),
                              _dev_ptr(ev, "evals", torch.float64), _dev_ptr(Y, "Y", torch.complex128),
                              int(Y.stride(0)), _stream_ptr(stream)))
    return ev, Y


def qm_zgemm(op, A, B, arith=0, stream=None):
    """op "cn": C = conj(A) B^T for A (M, K), B (N, K); op "tn": C = A^T B for A (K, M), B (K, N).
    complex128 CUDA tensors; arith 0 = FP64, 1 = double-FP32.  Returns C (M, N)."""
    lib = _lib.load()
    if op == "cn":
        (M, K), N = A.shape, int(B.shape[0])
        if int(B.shape[1]) != K:
            raise ValueError("A and B must have the same K")
    elif op == "tn":
        (K, M), N = A.shape, int(B.shape[1])
        if int(B.shape[0]) != K:
            raise ValueError("A and B must have the same K")
    else:
        raise ValueError("op must be 'cn' or 'tn'")
    C = torch.empty((int(M), N), dtype=torch.complex128, device=A.device)
    _check(lib.qm_zgemm(0 if op == "cn" else 1, int(arith), int(M), N, int(K), _dev_ptr(A, "A", torch.complex128),
                        int(A.stride(0)), _dev_ptr(B, "B", torch.complex128), int(B.stride(0)),
                        _dev_ptr(C, "C", torch.complex128), int(C.stride(0)), _stream_ptr(stream)))
    return C



def _tddft_args(psi, beta, D, work, prec):
    p = _PREC[prec]
    cdt = torch.complex128 if p == QM_FP64 else torch.complex64
    if psi.dim() != 2:
        raise ValueError("psi must be 2-D (nb, ld)")
    nb, ld = int(psi.shape[0]), int(psi.stride(0))
    if work is None:
        work = torch.empty((2 * nb * ld,), dtype=cdt, device=psi.device)
    elif work.numel() < 2 * nb * ld or not work.is_contiguous():
        raise ValueError("work must be a contiguous tensor of at least 2 * nb * ld elements")
    nproj = 0 if beta is None else int(beta.shape[0])
    nl = (nproj, _dev_ptr(beta, "beta", cdt), int(beta.stride(0)) if nproj else 0,
          _dev_ptr(D, "D", torch.float64) if nproj else None)
    return p, cdt, nb, ld, work, nl


def qm_tddft_taylor(g, ik, psi, vloc, beta, D, dt, order=4, prec="fp64", work=None, stream=None):
    """psi <- sum_{r<=order} (-i dt)^r/r! H^r psi in place (psi: (nb, >=npw) CUDA tensor, complex128
    for fp64, complex64 for mixed); work: optional scratch of 2 * nb * ld elements."""
    lib = _lib.load()
    p, cdt, nb, ld, work, nl = _tddft_args(psi, beta, D, work, prec)
    _check(lib.qm_tddft_taylor(g, int(ik), nb, _dev_ptr(psi, "psi", cdt), ld, _dev_ptr(vloc, "vloc", torch.float64),
                               *nl, float(dt), int(order), _dev_ptr(work, "work", cdt), p, _stream_ptr(stream)))
    return psi


def qm_tddft_etrs(g, ik, psi, vloc_now, vloc_next, beta, D, dt, order=4, prec="fp64", work=None, stream=None):
    """One ETRS step psi <- U(dt/2; H_next) U(dt/2; H_now) psi in place (arguments as qm_tddft_taylor)."""
    lib = _lib.load()
    p, cdt, nb, ld, work, nl = _tddft_args(psi, beta, D, work, prec)
    _check(lib.qm_tddft_etrs(g, int(ik), nb, _dev_ptr(psi, "psi", cdt), ld,
                             _dev_ptr(vloc_now, "vloc_now", torch.float64),
                             _dev_ptr(vloc_next, "vloc_next", torch.float64),
                             *nl, float(dt), int(order), _dev_ptr(work, "work", cdt), p, _stream_ptr(stream)))
    return psi


def qm_gw_mel(g, ik_left, ik_right, psi_l, psi_r, geps, iq, npw_eps, M=None, prec="fp64", stream=None):
    """GW plane-wave matrix elements M (nl * nr, npw_eps): row n * nr + n' holds
    <n k+q| exp(i(q+G).r) |n' k> on the sphere of q of the handle geps (k-point iq)."""
    lib = _lib.load()
    p = _PREC[prec]
    cdt = torch.complex128 if p == QM_FP64 else torch.complex64
    nl, nr = int(psi_l.shape[0]), int(psi_r.shape[0])
    if M is None:
        M = torch.empty((nl * nr, int(npw_eps)), dtype=cdt, device=psi_r.device)
    _check(lib.qm_gw_mel(g, int(ik_left), int(ik_right), nl, _dev_ptr(psi_l, "psi_l", cdt), int(psi_l.stride(0)),
                         nr, _dev_ptr(psi_r, "psi_r", cdt), int(psi_r.stride(0)), geps, int(iq),
                         _dev_ptr(M, "M", cdt), int(M.stride(0)), p, _stream_ptr(stream)))
    return M


def qm_scf(g, nelec, weights, psis, vion, betas, D, tol=1e-8, max_iter=50, alpha=0.5, history=4, dav_tol=1e-9,
           dav_max_iter=100, prec="fp64", stream=None, raise_not_converged=True):
    """Kohn-Sham self-consistency: psis (one (nb, >=npw) complex128 CUDA tensor per k-point, updated in
    place), vion (N_r,) float64, betas (one tensor per k-point) or None, D.  Returns (eigenvalues
    ndarray (nk, nb), density (N_r,), potential (N_r,), stats dict)."""
    lib = _lib.load()
    nk = len(psis)
    nb = int(psis[0].shape[0])
    ld = int(psis[0].stride(0))
    for p in psis:
        if int(p.shape[0]) != nb or int(p.stride(0)) != ld:
            raise ValueError("every k-point's psi must have the same shape and row stride")
    w = np.ascontiguousarray(np.asarray(weights, np.float64))
    pp = (ctypes.c_void_p * nk)(*[_dev_ptr(p, "psi", torch.complex128).value for p in psis])
    nproj = 0 if betas is None else int(betas[0].shape[0])
    bp = None
    ldb = 0
    if nproj:
        bp = (ctypes.c_void_p * nk)(*[_dev_ptr(b, "beta", torch.complex128).value for b in betas])
        ldb = int(betas[0].stride(0))
    rho = torch.empty_like(vion)
    vl = torch.empty_like(vion)
    eig = np.zeros(nk * nb)
    opts = _lib.ScfOpts(float(tol), int(max_iter), float(alpha), int(history), float(dav_tol), int(dav_max_iter),
                        _PREC[prec])
    st = _lib.ScfStats()
    status = lib.qm_scf(g, int(nelec), _dp(w), nb, pp, ld, _dev_ptr(vion, "vion", torch.float64), nproj, bp, ldb,
                        _dev_ptr(D, "D", torch.float64) if nproj else None, ctypes.byref(opts), _dp(eig),
                        _dev_ptr(rho, "rho", torch.float64), _dev_ptr(vl, "vloc", torch.float64), ctypes.byref(st),
                        _stream_ptr(stream))
    info = {k: getattr(st, k) for k, _ in _lib.ScfStats._fields_}
    if status != 0 and not (status == 4 and not raise_not_converged):
        _check(status)
    return eig.reshape(nk, nb), rho, vl, info

class Batch:
    """A batched H psi plan (qm_batch of include/qm.h) bound to its buffers.

    jobs: list of dicts with keys g (gspace handle), ik, psi, vloc, beta, D, out (CUDA
    tensors as for qm_hpsi; beta/D may be None).  The tensors are referenced by the plan
    and must stay alive and in place while it exists."""

    def __init__(self, jobs, prec="fp64", ctas_per_sm=0, item_points=0, group_mb=0, stream=None, fft_order=None):
        lib = _lib.load()
        self.prec = _PREC[prec]
        cdt = torch.complex128 if self.prec == QM_FP64 else torch.complex64
        arr = (_lib.HpsiJob * len(jobs))()
        self._keep = []
        for i, j in enumerate(jobs):
            psi, out, beta = j["psi"], j["out"], j.get("beta")
            if psi.dim() != 2 or out.dim() != 2 or psi.shape[0] != out.shape[0]:
                raise ValueError(f"job {i}: psi and out must be 2-D with the same number of bands")
            nproj = 0 if beta is None else int(beta.shape[0])
            arr[i] = _lib.HpsiJob(g=j["g"].value if isinstance(j["g"], ctypes.c_void_p) else j["g"],
                                  ik=int(j["ik"]), nb=int(psi.shape[0]),
                                  psi=_dev_ptr(psi, "psi", cdt), ld_psi=int(psi.stride(0)), nproj=nproj,
                                  vloc_r=_dev_ptr(j["vloc"], "vloc", torch.float64),
                                  beta=_dev_ptr(beta, "beta", cdt) if nproj else None,
                                  ld_beta=int(beta.stride(0)) if nproj else 0, ld_out=int(out.stride(0)),
                                  D=_dev_ptr(j["D"], "D", torch.float64) if nproj else None,
                                  out=_dev_ptr(out, "out", cdt))
            self._keep.append((psi, out, beta, j["vloc"], j.get("D")))
        if fft_order is None:   # a fully given launch shape keeps the default radix order
            fft_order = 1 if (ctas_per_sm and item_points and group_mb) else 0
        shape = _lib.BatchShape(int(ctas_per_sm), int(item_points), int(group_mb), int(fft_order))
        h = ctypes.c_void_p()
        _check(lib.qm_batch_create(len(jobs), arr, self.prec, ctypes.byref(shape), _stream_ptr(stream),
                                   ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        _check(_lib.load().qm_batch_run(self.handle, _stream_ptr(stream)))

    def check(self, stream=None):
        _check(_lib.load().qm_batch_check(self.handle, _stream_ptr(stream)))

    def hold(self, job, spin_limit=0):
        """Failure-detection test hook (qm_batch_hold): job >= 0 withholds one completion from
        that job's last phase so the bounded waits expire; job = -1 restores."""
        _check(_lib.load().qm_batch_hold(self.handle, int(job), int(spin_limit)))

    def info(self):
        inf = _lib.BatchInfo()
        _check(_lib.load().qm_batch_query(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _lib.BatchInfo._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.load().qm_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qm_batch_create(jobs, prec="fp64", ctas_per_sm=0, item_points=0, group_mb=0, stream=None, fft_order=None):
    return Batch(jobs, prec=prec, ctas_per_sm=ctas_per_sm, item_points=item_points, group_mb=group_mb,
                 stream=stream, fft_order=fft_order)


QM_MLP_NPARAM = 4481   # include/qm.h


def qm_mlp_forward(feats, theta, stream=None):
    """K for the (n, 3) float32 feature rows (CUDA tensors); theta (QM_MLP_NPARAM,) float32."""
    if feats.dim() != 2 or feats.shape[1] != 3 or not feats.is_contiguous():
        raise ValueError("feats must be a contiguous (n, 3) tensor")
    K = torch.empty(feats.shape[0], dtype=torch.float32, device=feats.device)
    _check(_lib.load().qm_mlp_forward(int(feats.shape[0]), _dev_ptr(feats, "feats", torch.float32),
                                      _dev_ptr(theta, "theta", torch.float32), _dev_ptr(K, "K", torch.float32),
                                      _stream_ptr(stream)))
    return K


def qm_hamiltonian_diag(g, ik, vloc, beta, D, stream=None):
    """The diagonal of H(k) in the plane-wave basis, (npw,) float64 CUDA tensor (beta, D:
    complex128 / float64 CUDA tensors or None)."""
    info = qm_gspace_query(g)
    npw = info["npw"][ik]
    out = torch.empty(npw, dtype=torch.float64, device=vloc.device)
    nproj = 0 if beta is None else int(beta.shape[0])
    _check(_lib.load().qm_hamiltonian_diag(g, int(ik), _dev_ptr(vloc, "vloc", torch.float64), nproj,
                                           _dev_ptr(beta, "beta", torch.complex128), int(beta.stride(0)) if nproj else 0,
                                           _dev_ptr(D, "D", torch.float64) if nproj else None,
                                           _dev_ptr(out, "hdiag", torch.float64), _stream_ptr(stream)))
    return out


def qm_mlp_pairs(g, ik, psi, hpsi, eps, hdiag, U, lam, cluster_tol=1e-6, stream=None):
    """Training samples of the Ritz pairs (psi, eps) with H psi = hpsi against the exact
    eigenpairs (U rows, lam ascending), hdiag the diagonal of H (qm_hamiltonian_diag); all
    complex128/float64 CUDA tensors.
    Returns (feats (n*npw, 3), r2 (n*npw,), c (n*npw,), D (n,), W (n,)) float32 CUDA tensors."""
    n, npw = int(psi.shape[0]), None
    info = qm_gspace_query(g)
    npw = info["npw"][ik]
    dev = psi.device
    feats = torch.empty((n * npw, 3), dtype=torch.float32, device=dev)
    r2 = torch.empty(n * npw, dtype=torch.float32, device=dev)
    c = torch.empty(n * npw, dtype=torch.float32, device=dev)
    D = torch.empty(n, dtype=torch.float32, device=dev)
    W = torch.empty(n, dtype=torch.float32, device=dev)
    _check(_lib.load().qm_mlp_pairs(g, int(ik), n, _dev_ptr(psi, "psi", torch.complex128), int(psi.stride(0)),
                                    _dev_ptr(hpsi, "hpsi", torch.complex128), int(hpsi.stride(0)),
                                    _dev_ptr(eps, "eps", torch.float64), _dev_ptr(hdiag, "hdiag", torch.float64),
                                    int(U.shape[0]),
                                    _dev_ptr(U, "U", torch.complex128), int(U.stride(0)),
                                    _dev_ptr(lam, "lam", torch.float64), float(cluster_tol),
                                    _dev_ptr(feats, "feats"), _dev_ptr(r2, "r2"), _dev_ptr(c, "c"), _dev_ptr(D, "D"),
                                    _dev_ptr(W, "W"), _stream_ptr(stream)))
    return feats, r2, c, D, W


def qm_mlp_loss_grad(band_off, feats, r2, c, D, theta, W=None, stream=None):
    """(loss float, grad (QM_MLP_NPARAM,) float32 CUDA tensor); band_off int64 CUDA tensor;
    W per-band weights (None: all 1)."""
    grad = torch.empty(QM_MLP_NPARAM, dtype=torch.float32, device=theta.device)
    loss = np.zeros(1, np.float64)
    _check(_lib.load().qm_mlp_loss_grad(int(band_off.numel()) - 1, _dev_ptr(band_off, "band_off", torch.int64),
                                        _dev_ptr(feats, "feats", torch.float32), _dev_ptr(r2, "r2", torch.float32),
                                        _dev_ptr(c, "c", torch.float32), _dev_ptr(D, "D", torch.float32),
                                        _dev_ptr(W, "W", torch.float32), _dev_ptr(theta, "theta", torch.float32), _dp(loss),
                                        _dev_ptr(grad, "grad", torch.float32), _stream_ptr(stream)))
    return float(loss[0]), grad


def qm_mlp_train(band_off, feats, r2, c, D, theta, steps, lr, W=None, stream=None):
    """Adam steps on theta (updated in place); returns the loss history (steps + 1,)."""
    hist = np.zeros(int(steps) + 1, np.float64)
    _check(_lib.load().qm_mlp_train(int(band_off.numel()) - 1, _dev_ptr(band_off, "band_off", torch.int64),
                                    _dev_ptr(feats, "feats", torch.float32), _dev_ptr(r2, "r2", torch.float32),
                                    _dev_ptr(c, "c", torch.float32), _dev_ptr(D, "D", torch.float32),
                                    _dev_ptr(W, "W", torch.float32), _dev_ptr(theta, "theta", torch.float32),
                                    int(steps), float(lr), _dp(hist),
                                    _stream_ptr(stream)))
    return hist


def qm_davidson_batched(jobs, tol=1e-8, max_iter=100, nvecx=0, prec="fp64", nconv=0, mixed_switch=0.0, mlp=None,
                        max_concurrent=0, stream=None, raise_not_converged=True, mixed_ortho=0, plain_restart=0,
                        fp64_exact=0):
    """Concurrent Davidson solves.  jobs: list of dicts with keys g, ik, psi (overwritten by
    the Ritz vectors), vloc, beta, D (CUDA tensors as for qm_davidson).  Returns a list of
    (eigenvalues ndarray, info dict) in job order."""
    lib = _lib.load()
    n = len(jobs)
    arr = (_lib.DavidsonJob * n)()
    eigs, stats, hists = [], [], []
    for i, j in enumerate(jobs):
        psi, beta = j["psi"], j.get("beta")
        if psi.dim() != 2:
            raise ValueError("psi must be 2-D (nb, ld)")
        nb = int(psi.shape[0])
        nproj = 0 if beta is None else int(beta.shape[0])
        eigs.append(np.zeros(nb, np.float64))
        stats.append(_lib.DavidsonStats())
        hists.append(np.zeros(max(1, int(max_iter)), np.float64))
        arr[i] = _lib.DavidsonJob(g=j["g"].value if isinstance(j["g"], ctypes.c_void_p) else j["g"], ik=int(j["ik"]),
                                  nb=nb, psi_inout=_dev_ptr(psi, "psi", torch.complex128), ld_psi=int(psi.stride(0)),
                                  nproj=nproj, vloc_r=_dev_ptr(j["vloc"], "vloc", torch.float64),
                                  beta=_dev_ptr(beta, "beta", torch.complex128) if nproj else None,
                                  ld_beta=int(beta.stride(0)) if nproj else 0,
                                  D=_dev_ptr(j["D"], "D", torch.float64) if nproj else None,
                                  eig_out=eigs[-1].ctypes.data_as(ctypes.c_void_p), stats=ctypes.pointer(stats[-1]),
                                  history=hists[-1].ctypes.data_as(ctypes.c_void_p))
    opts = _lib.DavidsonOpts(tol=float(tol), max_iter=int(max_iter), nvecx=int(nvecx), prec=_PREC[prec],
                             precond=0 if mlp is None else 1, mixed_switch=float(mixed_switch), nconv=int(nconv),
                             mixed_ortho=int(mixed_ortho), history=None, mlp=_dev_ptr(mlp, "mlp", torch.float32),
                             plain_restart=int(plain_restart), fp64_exact=int(fp64_exact))
    st = lib.qm_davidson_batched(n, arr, ctypes.byref(opts), int(max_concurrent), _stream_ptr(stream))
    out = []
    for i in range(n):
        s = stats[i]
        out.append((eigs[i], {"iterations": s.iterations, "converged": bool(s.converged),
                              "band_applies": s.band_applies, "max_residual": s.max_residual, "seconds": s.seconds,
                              "iterations_mixed": s.iterations_mixed, "band_applies_mixed": s.band_applies_mixed,
                              "precond_fallback": s.precond_fallback, "restarts": s.restarts,
                              "restart_kept": s.restart_kept,
                              "history": hists[i][: max(0, s.iterations)].tolist(),
                              "status": STATUS.get(arr[i].status, arr[i].status)}))
    if st != 0 and not (st == 4 and not raise_not_converged):
        _check(st)
    return out

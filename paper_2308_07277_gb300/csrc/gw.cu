// qm_gw_mel: plane-wave matrix elements of the GW module (Sec. 5, "gw" module) through the
// stick-pruned FFT kernels; the kernels and the launch sequence are in gw_kernels.cuh.
#include <cmath>
#include <cstdint>

#include "qm_internal.h"

namespace qm {
template <class R>
qm_status gw_mel_impl(qm_gspace g, int ikl, int ikr, int nl, const void* psi_l, int ld_l, int nr, const void* psi_r,
                      int ld_r, qm_gspace ge, int iq, void* M, int ld_m, cudaStream_t s);
extern template qm_status gw_mel_impl<float>(qm_gspace, int, int, int, const void*, int, int, const void*, int,
                                             qm_gspace, int, void*, int, cudaStream_t);
extern template qm_status gw_mel_impl<double>(qm_gspace, int, int, int, const void*, int, int, const void*, int,
                                              qm_gspace, int, void*, int, cudaStream_t);
}  // namespace qm

using namespace qm;

extern "C" qm_status qm_gw_mel(qm_gspace g, int ik_left, int ik_right, int nl, const void* psi_l, int ld_l, int nr,
                               const void* psi_r, int ld_r, qm_gspace geps, int iq, void* M, int ld_m,
                               qm_precision prec, void* stream) {
    clear_error();
    if (!g || !geps) return fail(QM_ERR_ARG, "qm_gw_mel: NULL gspace");
    if (ik_left < 0 || ik_left >= g->nk || ik_right < 0 || ik_right >= g->nk)
        return fail(QM_ERR_ARG, "qm_gw_mel: k-point index out of range");
    if (iq < 0 || iq >= geps->nk) return fail(QM_ERR_ARG, "qm_gw_mel: iq out of range");
    if (nl < 0 || nr < 0) return fail(QM_ERR_ARG, "qm_gw_mel: negative band count");
    if (prec != QM_FP64 && prec != QM_MIXED) return fail(QM_ERR_ARG, "qm_gw_mel: unknown precision");
    for (int d = 0; d < 3; ++d)
        if (g->n[d] != geps->n[d]) return fail(QM_ERR_ARG, "qm_gw_mel: the two handles have different FFT grids");
    for (int d = 0; d < 3; ++d) {
        const double q = g->kpts[3 * ik_left + d] - g->kpts[3 * ik_right + d];
        if (std::fabs(q - geps->kpts[3 * iq + d]) > 1e-10)
            return fail(QM_ERR_ARG, "qm_gw_mel: k-point iq of geps is not k(ik_left) - k(ik_right)");
    }
    if ((long long)nl * nr > (1ll << 30)) return fail(QM_ERR_ARG, "qm_gw_mel: nl * nr too large");
    if (nl == 0 || nr == 0) return QM_OK;
    if (!psi_l || !psi_r || !M) return fail(QM_ERR_ARG, "qm_gw_mel: NULL psi_l, psi_r or M");
    if (ld_l < g->k[ik_left].npw || ld_r < g->k[ik_right].npw || ld_m < geps->k[iq].npw)
        return fail(QM_ERR_ARG, "qm_gw_mel: leading dimension smaller than its sphere");
    const size_t cs = prec == QM_MIXED ? sizeof(float2) : sizeof(double2);
    if (((uintptr_t)psi_l | (uintptr_t)psi_r | (uintptr_t)M) % cs)
        return fail(QM_ERR_ARG, "qm_gw_mel: psi_l/psi_r/M not aligned to the complex element size");
    qm_status st;
    if ((st = ensure_device(g)) || (st = ensure_device(geps))) return st;
    if (g->device != geps->device) return fail(QM_ERR_ARG, "qm_gw_mel: the handles live on different devices");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == QM_MIXED)
        return gw_mel_impl<float>(g, ik_left, ik_right, nl, psi_l, ld_l, nr, psi_r, ld_r, geps, iq, M, ld_m, s);
    return gw_mel_impl<double>(g, ik_left, ik_right, nl, psi_l, ld_l, nr, psi_r, ld_r, geps, iq, M, ld_m, s);
}

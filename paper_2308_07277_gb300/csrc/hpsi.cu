// qm_hpsi: H(k) psi for a block of bands (Eq. KSHamMat of Sec. 2.2 with the
// Kleinman-Bylander term of Sec. 2.3).
//
// Launch sequence on the caller's stream (no host synchronisation):
//   1. k_vt            V(r)/N_r laid out in the FFT path's permuted plane order
//   2. gemm_cn         P[p][b] = <beta_p|psi_b>             (nonlocal projection, FP64)
//   3. K1, K2, K3      out = 1/2|k+G|^2 psi + (V psi)(G)    (per chunk of bands)
//   4. gemm_tn         out += sum_p beta_p D_p P[p][b]      (nonlocal apply, FP64)
// QM_MIXED: the nonlocal part runs as BF16x3 split tcgen05 products (umma.cu) on the handle's
// second stream, concurrently with k_vt, K1 and K2 of every band: it writes
// out = sum_p beta_p D_p P[p][b], and K3 (which waits for it) adds the local and kinetic
// parts.  The tensor-core kernels (96 KB of shared memory) share SMs with the FFT kernels.
// Workspace (owned by the gspace handle): error word | Vt | P | split-K partials | stick buffer | nonlocal.
#include <algorithm>
#include <cstdint>

#include "qm_internal.h"

namespace qm {

// Stick-buffer budget per chunk of bands of the FP64 form: small enough that a chunk's
// intermediate data stays resident in the 129 MB L2 between the three FFT kernels.
constexpr size_t kStickBudget = 48ull << 20;
constexpr size_t kStickBudgetOverlap = 1ull << 30;

struct HpsiLayout {
    size_t vt_off, p_off, part_off, t_off, nl_off, err_off, total, t_bytes;
    int splits;
};

static HpsiLayout hpsi_layout(qm_gspace g, int ik, int nb, int nproj, bool fp32, bool own_beta, bool gamma) {
    HpsiLayout L{};
    const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
    const size_t rs = fp32 ? sizeof(float) : sizeof(double);
    const size_t nr = (size_t)g->n[0] * g->n[1] * g->n[2];
    const int npw = g->k[ik].npw;
    L.splits = nproj > 0 ? zgemm_cn_splits(nproj, nb, npw) : 1;
    size_t off = kWsHeader;  // the header holds the handle's sticky error word
    L.err_off = 0;
    L.vt_off = off;
    off = align_up(off + nr * rs, 256);
    L.p_off = off;
    off = align_up(off + (size_t)nproj * nb * cs, 256);
    L.part_off = off;
    off = align_up(off + (L.splits > 1 ? std::min((size_t)L.splits * nproj * nb * cs, gemm_cn_partial_bytes(fp32)) : 0), 256);
    L.t_off = off;
    const size_t per_band = stick_buffer_bytes_per_band(g, ik, fp32);
    // the precision form keeps every band's stick buffer (K1 and K2 of all bands overlap the
    // nonlocal part; K3 runs once it is done; without projectors the larger launches are faster
    // too), the FP64 form chunks the bands to stay in L2
    const size_t budget = fp32 ? kStickBudgetOverlap : kStickBudget;
    const size_t ntr = gamma ? (size_t)(nb + 1) / 2 : (size_t)nb;  // transforms (band pairs at Gamma)
    const size_t nbc = std::max<size_t>(1, std::min<size_t>(ntr, budget / per_band));
    L.t_bytes = nbc * per_band;
    off = align_up(off + L.t_bytes, 256);
    L.nl_off = off;  // tensor-core split operands (precision form)
    off = align_up(off + (fp32 && nproj > 0 ? nonlocal_tc_bytes(nproj, nb, npw, own_beta) : 0), 256);
    L.total = off;
    return L;
}

}  // namespace qm

using namespace qm;

extern "C" qm_status qm_hpsi(qm_gspace g, int ik, int nb, const void* psi, int ld_psi, const double* vloc_r,
                             int nproj, const void* beta, int ld_beta, const double* D, void* out, int ld_out,
                             qm_precision prec, void* stream) {
    clear_error();
    return hpsi_run(g, ik, nb, psi, ld_psi, vloc_r, nproj, beta, ld_beta, nullptr, D, out, ld_out, prec,
                    (cudaStream_t)stream);
}

qm_status qm::hpsi_run(qm_gspace g, int ik, int nb, const void* psi, int ld_psi, const double* vloc_r, int nproj,
                       const void* beta, int ld_beta, const void* beta_prepared, const double* D, void* out,
                       int ld_out, qm_precision prec, cudaStream_t s, bool ds_nonlocal, bool gamma) {
    if (!g) return fail(QM_ERR_ARG, "qm_hpsi: NULL gspace");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_hpsi: ik out of range");
    if (nb < 0 || nproj < 0) return fail(QM_ERR_ARG, "qm_hpsi: negative nb or nproj");
    if (prec != QM_FP64 && prec != QM_MIXED) return fail(QM_ERR_ARG, "qm_hpsi: unknown precision");
    if (nb == 0) return QM_OK;
    const int npw = g->k[ik].npw;
    if (!psi || !out || !vloc_r) return fail(QM_ERR_ARG, "qm_hpsi: NULL psi, out or vloc_r");
    if (ld_psi < npw || ld_out < npw) return fail(QM_ERR_ARG, "qm_hpsi: leading dimension < npw");
    if (nproj > 0 && (!beta || !D)) return fail(QM_ERR_ARG, "qm_hpsi: NULL beta or D with nproj > 0");
    if (nproj > 0 && ld_beta < npw) return fail(QM_ERR_ARG, "qm_hpsi: ld_beta < npw");
    const bool fp32 = prec == QM_MIXED;
    const uintptr_t al = fp32 ? 8 : 16;
    if (((uintptr_t)psi | (uintptr_t)out | (nproj > 0 ? (uintptr_t)beta : 0)) % al)
        return fail(QM_ERR_ARG, "qm_hpsi: psi/out/beta not aligned to the complex element size");
    const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
    {
        const char* a0 = (const char*)psi;
        const char* a1 = a0 + ((size_t)(nb - 1) * ld_psi + npw) * cs;
        const char* b0 = (const char*)out;
        const char* b1 = b0 + ((size_t)(nb - 1) * ld_out + npw) * cs;
        if (a0 < b1 && b0 < a1) return fail(QM_ERR_ARG, "qm_hpsi: out overlaps psi");
    }
    if (gamma && !g->k[ik].gamma) return fail(QM_ERR_ARG, "qm_hpsi_gamma: k-point ik is not the Gamma point");

    qm_status st = ensure_device(g);
    if (st) return st;
    if (fp32 && nproj > 0 && !beta_prepared && ik < (int)g->prep.size()) {
        const NlPrep& p = g->prep[ik];
        if (p.dev && p.beta == beta && p.ld == ld_beta && p.nproj == nproj) beta_prepared = p.dev;
    }

    const HpsiLayout L = hpsi_layout(g, ik, nb, nproj, fp32, beta_prepared == nullptr, gamma);
    if ((st = ensure_workspace(g, L.total, s))) return st;
    char* ws = (char*)g->ws.ptr;
    void* vt = ws + L.vt_off;
    void* P = ws + L.p_off;
    void* part = ws + L.part_off;
    void* T = ws + L.t_off;

    if (fp32 && nproj > 0) {
        // fork: the nonlocal part on the second stream writes out; K3 joins and adds to it
        int* err = (int*)(ws + L.err_off);
        cudaStream_t a = g->aux;
        if ((st = cuda_check(cudaEventRecord(g->ev_fork, s), "fork event")) ||
            (st = cuda_check(cudaStreamWaitEvent(a, g->ev_fork, 0), "fork wait")))
            return st;
        if ((st = nonlocal_tc(nproj, nb, npw, (const float2*)beta, ld_beta, beta_prepared, (const float2*)psi, ld_psi,
                              D, (float2*)out, ld_out, ws + L.nl_off, err, a, false)))
            return st;
        if ((st = cuda_check(cudaEventRecord(g->ev_join, a), "join event"))) return st;
        if ((st = launch_vt_prepare(g, vloc_r, vt, fp32, s))) return st;
        return launch_local_kinetic(g, ik, nb, psi, ld_psi, vt, out, ld_out, T, L.t_bytes, fp32, s, g->ev_join,
                                    true, gamma);
    }
    if ((st = launch_vt_prepare(g, vloc_r, vt, fp32, s))) return st;
    if (nproj > 0 && !fp32) {
        st = (ds_nonlocal ? zgemm_cn_ds : zgemm_cn)(nproj, nb, npw, (const double2*)beta, ld_beta,
                                                    (const double2*)psi, ld_psi, (double2*)P, nb, (double2*)part,
                                                    L.splits, s);
        if (st) return st;
    }
    if ((st = launch_local_kinetic(g, ik, nb, psi, ld_psi, vt, out, ld_out, T, L.t_bytes, fp32, s, nullptr, false,
                                   gamma)))
        return st;
    if (nproj > 0 && !fp32) {
        st = (ds_nonlocal ? zgemm_tn_ds : zgemm_tn)(nb, npw, nproj, (const double2*)P, nb, D, (const double2*)beta,
                                                    ld_beta, (double2*)out, ld_out, true, s, 1.0);
        if (st) return st;
    }
    return QM_OK;
}

extern "C" qm_status qm_hpsi_gamma(qm_gspace g, int ik, int nb, const void* psi, int ld_psi, const double* vloc_r,
                                   int nproj, const void* beta, int ld_beta, const double* D, void* out, int ld_out,
                                   qm_precision prec, void* stream) {
    clear_error();
    return hpsi_run(g, ik, nb, psi, ld_psi, vloc_r, nproj, beta, ld_beta, nullptr, D, out, ld_out, prec,
                    (cudaStream_t)stream, false, true);
}

extern "C" qm_status qm_hpsi_prepare(qm_gspace g, int ik, int nproj, const void* beta, int ld_beta, void* stream) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_hpsi_prepare: NULL gspace");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_hpsi_prepare: ik out of range");
    if (nproj < 0) return fail(QM_ERR_ARG, "qm_hpsi_prepare: negative nproj");
    const int npw = g->k[ik].npw;
    if (nproj > 0) {
        if (!beta) return fail(QM_ERR_ARG, "qm_hpsi_prepare: NULL beta with nproj > 0");
        if (ld_beta < npw) return fail(QM_ERR_ARG, "qm_hpsi_prepare: ld_beta < npw");
        if ((uintptr_t)beta % 8) return fail(QM_ERR_ARG, "qm_hpsi_prepare: beta not 8-byte aligned");
    }
    qm_status st = ensure_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if ((int)g->prep.size() < g->nk) g->prep.resize(g->nk);
    NlPrep& p = g->prep[ik];
    if (nproj == 0) {  // release
        if (p.dev) {
            if ((st = cuda_check(cudaStreamSynchronize(s), "qm_hpsi_prepare: sync"))) return st;
            cudaFree(p.dev);
        }
        p = NlPrep{};
        return QM_OK;
    }
    const size_t bytes = nonlocal_tc_beta_bytes(nproj, 1, npw);
    if (!p.dev || p.bytes < bytes) {
        if (p.dev) {
            if ((st = cuda_check(cudaStreamSynchronize(s), "qm_hpsi_prepare: sync"))) return st;
            cudaFree(p.dev);
            p = NlPrep{};
        }
        if (cudaMalloc(&p.dev, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = NlPrep{};
            return fail(QM_ERR_OOM, "qm_hpsi_prepare: device allocation of the prepared projectors");
        }
        p.bytes = bytes;
    }
    p.beta = beta;
    p.ld = ld_beta;
    p.nproj = nproj;
    if ((st = nonlocal_tc_prepare(nproj, 1, npw, (const float2*)beta, ld_beta, p.dev, s))) {
        p.beta = nullptr;  // a failed preparation is never used
        return st;
    }
    return QM_OK;
}

extern "C" qm_status qm_hpsi_check(qm_gspace g, void* stream) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_hpsi_check: NULL gspace");
    if (!g->ws.ptr) return QM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int e = 0;
    qm_status st;
    if ((st = cuda_check(cudaStreamSynchronize(s), "qm_hpsi_check: sync")) ||
        (st = cuda_check(cudaMemcpy(&e, g->ws.ptr, sizeof(int), cudaMemcpyDeviceToHost), "qm_hpsi_check: read")))
        return st;
    if (!e) return QM_OK;
    if ((st = cuda_check(cudaMemset(g->ws.ptr, 0, sizeof(int)), "qm_hpsi_check: clear"))) return st;
    return fail(QM_ERR_TIMEOUT, "a bounded tensor-core wait of an earlier call on this handle expired (its outputs are "
                                "undefined)");
}

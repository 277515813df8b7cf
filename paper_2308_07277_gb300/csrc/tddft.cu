// Real-time propagation on the H psi of this library (Sec. 5, "tddft" module).
//
// qm_tddft_taylor: psi <- sum_{r=0}^{k} (-i dt)^r / r! H^r psi, the truncated Taylor series of
// exp(-i dt H) (expoper submodule).  The terms are built by the recursion
//     u_0 = psi,   u_r = (-i dt / r) H u_{r-1},
// one qm_hpsi launch sequence per term into a caller-owned work row block, followed by one
// element-wise kernel that scales the new term in place and adds it to psi (psi is not read by
// the H application of any later term, so it accumulates in place).  Two work blocks alternate
// as input and output of H.
// qm_tddft_etrs: the enforced-time-reversal-symmetry step (prop submodule),
//     psi <- U(dt/2; H_next) U(dt/2; H_now) psi,
// with H_now and H_next differing in their local potential (the caller supplies both).
#include <cstdint>
#include <cstdio>

#include "qm_internal.h"

namespace qm {

// u <- c u;  psi <- psi + u   (c = (cr, ci)), over nb rows of npw elements
template <class C, class R>
__global__ void __launch_bounds__(256) k_taylor_acc(C* __restrict__ psi, int ld_psi, C* __restrict__ u, int ld_u,
                                                    int nb, int npw, R cr, R ci) {
    const size_t n = (size_t)nb * npw;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / npw);
        const int g = (int)(i - (size_t)b * npw);
        C x = u[(size_t)b * ld_u + g];
        C t;
        t.x = cr * x.x - ci * x.y;
        t.y = cr * x.y + ci * x.x;
        u[(size_t)b * ld_u + g] = t;
        C p = psi[(size_t)b * ld_psi + g];
        p.x += t.x;
        p.y += t.y;
        psi[(size_t)b * ld_psi + g] = p;
    }
}

static qm_status taylor_acc(void* psi, int ld_psi, void* u, int ld_u, int nb, int npw, double cr, double ci, bool fp32,
                            cudaStream_t s) {
    const int blocks = grid_stride_blocks((size_t)nb * npw, 256, 8);
    ProfScope pf(PF_OTHER, s);
    if (fp32)
        k_taylor_acc<float2, float><<<blocks, 256, 0, s>>>((float2*)psi, ld_psi, (float2*)u, ld_u, nb, npw, (float)cr,
                                                          (float)ci);
    else
        k_taylor_acc<double2, double><<<blocks, 256, 0, s>>>((double2*)psi, ld_psi, (double2*)u, ld_u, nb, npw, cr, ci);
    return cuda_check(cudaGetLastError(), "Taylor update launch");
}

static qm_status taylor_check(const char* who, qm_gspace g, int ik, int nb, const void* psi, int ld_psi, double dt,
                              int order, const void* work, qm_precision prec) {
    char buf[160];
    if (!g) return fail(QM_ERR_ARG, std::string(who) + ": NULL gspace");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, std::string(who) + ": ik out of range");
    if (nb < 0) return fail(QM_ERR_ARG, std::string(who) + ": negative nb");
    if (order < 0 || order > 64) {
        snprintf(buf, sizeof buf, "%s: order %d outside [0, 64]", who, order);
        return fail(QM_ERR_ARG, buf);
    }
    if (!(dt == dt) || dt > 1e300 || dt < -1e300) return fail(QM_ERR_ARG, std::string(who) + ": dt not finite");
    if (prec != QM_FP64 && prec != QM_MIXED) return fail(QM_ERR_ARG, std::string(who) + ": unknown precision");
    if (nb == 0 || order == 0) return QM_OK;
    if (!psi || !work) return fail(QM_ERR_ARG, std::string(who) + ": NULL psi or work");
    if (ld_psi < g->k[ik].npw) return fail(QM_ERR_ARG, std::string(who) + ": ld_psi < npw");
    const size_t cs = prec == QM_MIXED ? sizeof(float2) : sizeof(double2);
    if ((uintptr_t)work % cs || (uintptr_t)psi % cs)
        return fail(QM_ERR_ARG, std::string(who) + ": psi/work not aligned to the complex element size");
    const char* a0 = (const char*)psi;
    const char* a1 = a0 + ((size_t)(nb - 1) * ld_psi + g->k[ik].npw) * cs;
    const char* w0 = (const char*)work;
    const char* w1 = w0 + 2 * (size_t)nb * ld_psi * cs;
    if (a0 < w1 && w0 < a1) return fail(QM_ERR_ARG, std::string(who) + ": work overlaps psi");
    return QM_OK;
}

// psi <- U_order(dt) psi with the Hamiltonian of (vloc, beta, D); work = 2 blocks of nb x ld_psi
static qm_status taylor_run(qm_gspace g, int ik, int nb, void* psi, int ld_psi, const double* vloc_r, int nproj,
                            const void* beta, int ld_beta, const double* D, double dt, int order, void* work,
                            qm_precision prec, cudaStream_t s) {
    const bool fp32 = prec == QM_MIXED;
    const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
    const int npw = g->k[ik].npw;
    char* w[2] = {(char*)work, (char*)work + (size_t)nb * ld_psi * cs};
    const void* in = psi;
    // c_r = -i dt / r applied to the new term: (0, -dt/r)
    for (int r = 1; r <= order; ++r) {
        void* out = w[(r - 1) & 1];
        qm_status st = hpsi_run(g, ik, nb, in, ld_psi, vloc_r, nproj, beta, ld_beta, nullptr, D, out, ld_psi, prec, s);
        if (st) return st;
        if ((st = taylor_acc(psi, ld_psi, out, ld_psi, nb, npw, 0.0, -dt / r, fp32, s))) return st;
        in = out;
    }
    return QM_OK;
}

}  // namespace qm

using namespace qm;

extern "C" qm_status qm_tddft_taylor(qm_gspace g, int ik, int nb, void* psi, int ld_psi, const double* vloc_r,
                                     int nproj, const void* beta, int ld_beta, const double* D, double dt, int order,
                                     void* work, qm_precision prec, void* stream) {
    clear_error();
    qm_status st = taylor_check("qm_tddft_taylor", g, ik, nb, psi, ld_psi, dt, order, work, prec);
    if (st || nb == 0 || order == 0) return st;
    return taylor_run(g, ik, nb, psi, ld_psi, vloc_r, nproj, beta, ld_beta, D, dt, order, work, prec,
                      (cudaStream_t)stream);
}

extern "C" qm_status qm_tddft_etrs(qm_gspace g, int ik, int nb, void* psi, int ld_psi, const double* vloc_now,
                                   const double* vloc_next, int nproj, const void* beta, int ld_beta, const double* D,
                                   double dt, int order, void* work, qm_precision prec, void* stream) {
    clear_error();
    qm_status st = taylor_check("qm_tddft_etrs", g, ik, nb, psi, ld_psi, dt, order, work, prec);
    if (st || nb == 0 || order == 0) return st;
    if (!vloc_now || !vloc_next) return fail(QM_ERR_ARG, "qm_tddft_etrs: NULL potential");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = taylor_run(g, ik, nb, psi, ld_psi, vloc_now, nproj, beta, ld_beta, D, 0.5 * dt, order, work, prec, s)))
        return st;
    return taylor_run(g, ik, nb, psi, ld_psi, vloc_next, nproj, beta, ld_beta, D, 0.5 * dt, order, work, prec, s);
}

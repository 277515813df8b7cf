// qm_davidson: lowest nb eigenpairs of H(k) by block Davidson (Sec. 5, dft module: a
// matrix-free "Davidson with overlap" that only applies H to blocks of trial vectors).
//
// Per iteration, on the caller's stream (host loop; two small device->host reads):
//   Rayleigh-Ritz   H_sub = V^H (H V) (new columns only), Jacobi eigensolve (FP64)
//   Ritz vectors    X = V c, HX = (HV) c for the lowest nb eigenpairs
//   residuals       r_n = HX_n - eps_n X_n, ||r_n|| and T_n = <X_n|T|X_n> (FP64)
//   corrections     delta_n = K_TPA(kin / T_n) r_n for the bands with ||r_n|| > tol
//   restart         if the basis would exceed nvecx: V <- X, HV <- HX
//   orthonormalise  two classical Gram-Schmidt passes against V, then Loewdin (S^-1/2 via
//                   the Jacobi eigensolver) within the block, near-dependent directions dropped
//   expand          V <- [V, delta], HV <- [HV, H delta]
// The basis is kept orthonormal, so the subspace overlap S_sub is the identity to FP64
// round-off and Rayleigh-Ritz is a standard Hermitian eigenproblem.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

#include "qm_internal.h"

namespace qm {

namespace {

__global__ void k_residual(const double2* __restrict__ X, const double2* __restrict__ HX, int ld, int npw,
                           const double* __restrict__ eps, const double* __restrict__ kin, double2* __restrict__ R,
                           double* __restrict__ rnorm2, double* __restrict__ tkin) {
    const int n = blockIdx.x;
    const double e = eps[n];
    const double2* x = X + (size_t)n * ld;
    const double2* hx = HX + (size_t)n * ld;
    double2* r = R + (size_t)n * ld;
    double s_r = 0.0, s_t = 0.0, s_x = 0.0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        double2 xv = x[g], hv = hx[g];
        double2 rv = make_double2(hv.x - e * xv.x, hv.y - e * xv.y);
        r[g] = rv;
        s_r += rv.x * rv.x + rv.y * rv.y;
        double ax = xv.x * xv.x + xv.y * xv.y;
        s_x += ax;
        s_t += kin[g] * ax;
    }
    __shared__ double sh[3][256];
    sh[0][threadIdx.x] = s_r;
    sh[1][threadIdx.x] = s_t;
    sh[2][threadIdx.x] = s_x;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int a = 0; a < 3; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rnorm2[n] = sh[0][0];
        tkin[n] = sh[1][0] / sh[2][0];
    }
}

// Teter-Payne-Allan preconditioner K(x) = (27+18x+12x^2+8x^3)/(27+18x+12x^2+8x^3+16x^4),
// x = kin(G) / T_n  (Teter, Payne & Allan, Phys. Rev. B 40, 12255 (1989)).
__global__ void k_tpa(const double2* __restrict__ R, int ld, int npw, const int* __restrict__ sel,
                      const double* __restrict__ tkin, const double* __restrict__ kin, double2* __restrict__ out,
                      int ldo) {
    const int j = blockIdx.y;
    const int n = sel[j];
    const double inv_t = 1.0 / tkin[n];
    const double2* r = R + (size_t)n * ld;
    double2* o = out + (size_t)j * ldo;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        const double x = kin[g] * inv_t;
        const double num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
        const double k = num / (num + 16.0 * x * x * x * x);
        const double2 rv = r[g];
        o[g] = make_double2(k * rv.x, k * rv.y);
    }
}

// Hermitian completion after new columns [m0, m) of H were computed for rows [0, m):
// H[j][i] = conj(H[i][j]) for i < m0 <= j; the new diagonal block is symmetrised.
__global__ void k_herm_fill(double2* __restrict__ H, int ld, int m0, int m) {
    const int nn = m - m0;
    const long total = (long)m * nn;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / nn), j = m0 + (int)(e % nn);
        if (i < m0) {
            double2 v = H[(size_t)i * ld + j];
            H[(size_t)j * ld + i] = make_double2(v.x, -v.y);
        } else if (i < j) {
            double2 a = H[(size_t)i * ld + j], b = H[(size_t)j * ld + i];
            double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
            H[(size_t)i * ld + j] = h;
            H[(size_t)j * ld + i] = make_double2(h.x, -h.y);
        } else if (i == j) {
            H[(size_t)i * ld + i].y = 0.0;
        }
    }
}

// A[i][j] = Hermitian part of H (m x m)
__global__ void k_herm_copy(const double2* __restrict__ H, int ldh, int m, double2* __restrict__ A, int lda) {
    const long total = (long)m * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), j = (int)(e % m);
        const double2 a = H[(size_t)i * ldh + j], b = H[(size_t)j * ldh + i];
        A[(size_t)i * lda + j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
}

__global__ void k_set_diag(double2* __restrict__ H, int ld, int m, const double* __restrict__ d) {
    const long total = (long)m * m;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), j = (int)(e % m);
        H[(size_t)i * ld + j] = make_double2(i == j ? d[i] : 0.0, 0.0);
    }
}

// invs[i] = 1/sqrt(S_ii): scaling that gives the Gram matrix a unit diagonal
__global__ void k_inv_sqrt_diag(const double2* __restrict__ S, int ld, int n, double* __restrict__ invs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        invs[i] = 1.0 / sqrt(S[(size_t)i * ld + i].x);
}

__global__ void k_scale_sym(const double2* __restrict__ S, int lds, int n, const double* __restrict__ invs,
                            double2* __restrict__ T, int ldt) {
    const long total = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const double f = invs[i] * invs[j];
        double2 v = S[(size_t)i * lds + j];
        T[(size_t)i * ldt + j] = make_double2(f * v.x, f * v.y);
    }
}

// W[i][k] = invs[i] * U[i][sel[k]] * wk[k]   (Loewdin coefficients)
__global__ void k_lowdin_coef(const double2* __restrict__ U, int ldu, int n, const double* __restrict__ invs,
                              const int* __restrict__ sel, const double* __restrict__ wk, int nk,
                              double2* __restrict__ W, int ldw) {
    const long total = (long)n * nk;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / nk), k = (int)(e % nk);
        const double f = invs[i] * wk[k];
        double2 v = U[(size_t)i * ldu + sel[k]];
        W[(size_t)i * ldw + k] = make_double2(f * v.x, f * v.y);
    }
}

inline int grid_for(long n) { return (int)std::max<long>(1, std::min<long>((n + 255) / 256, 152 * 8)); }

struct Ws {
    double2 *V, *HV, *X, *HX, *R, *Dl, *Tmp;  // [.. rows][ld]
    double2 *Hs, *G, *A, *Z, *Cs, *Part;      // small
    double *eval, *eps, *rn2, *tk, *red, *invs, *wk;
    int *sel, *info;
    void* rot;
    void* heev;
};

}  // namespace

qm_status jacobi_eigh(const double2* H, int ldh, int m, double2* A, double2* Z, void* rot, double* red, int* info,
                      double* evals_dev, cudaStream_t s);

}  // namespace qm

using namespace qm;

namespace {

struct DavidsonRun {
    qm_gspace g;
    int ik, nb, npw, ld, nvecx, nproj, ldb;
    const double* vloc;
    const void* beta;
    const double* D;
    cudaStream_t s;
    Ws w;
    long long applies = 0;

    qm_status hpsi(const double2* in, double2* out, int n) {
        applies += n;
        return qm_hpsi(g, ik, n, in, ld, vloc, nproj, beta, ldb, D, out, ld, QM_FP64, s);
    }

    // Loewdin-orthonormalise the nd rows of Y (ld) into the rows of out; returns kept count.
    qm_status lowdin(const double2* Y, int nd, double2* out, int* kept) {
        qm_status st;
        const int lds = nd + (nd & 1);
        // S[i][j] = <Y_i|Y_j>
        if ((st = zgemm_cn(nd, nd, npw, Y, ld, Y, ld, w.Cs, lds, w.Part, zgemm_cn_splits(nd, nd, npw), s))) return st;
        // Loewdin on the unit-diagonal Gram matrix G = D^-1/2 S D^-1/2, D = diag(S)
        {
            ProfScope pf(PF_OTHER, s);
            k_inv_sqrt_diag<<<grid_for(nd), 256, 0, s>>>(w.Cs, lds, nd, w.invs);
        }
        {
            ProfScope pf(PF_OTHER, s);
            k_scale_sym<<<grid_for((long)nd * nd), 256, 0, s>>>(w.Cs, lds, nd, w.invs, w.G, lds);
        }
        if ((st = heev_lowest(w.G, lds, nd, nd, w.eval, w.Z, nd, w.heev, s))) return st;
        std::vector<double> lam(nd);
        if ((st = cuda_check(cudaMemcpyAsync(lam.data(), w.eval, sizeof(double) * nd, cudaMemcpyDeviceToHost, s),
                             "D2H Gram eigenvalues")))
            return st;
        if ((st = cuda_check(cudaStreamSynchronize(s), "stream sync"))) return st;
        double lmax = 0.0;
        for (double l : lam) lmax = std::max(lmax, l);
        std::vector<int> sel;
        std::vector<double> wk;
        for (int k = 0; k < nd; ++k)
            if (lam[k] > 1e-8 * lmax && std::isfinite(lam[k])) {
                sel.push_back(k);
                wk.push_back(1.0 / std::sqrt(lam[k]));
            }
        *kept = (int)sel.size();
        if (sel.empty()) return QM_OK;
        cudaMemcpyAsync(w.sel, sel.data(), sizeof(int) * sel.size(), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(w.wk, wk.data(), sizeof(double) * wk.size(), cudaMemcpyHostToDevice, s);
        {
            ProfScope pf(PF_OTHER, s);
            k_lowdin_coef<<<grid_for((long)nd * sel.size()), 256, 0, s>>>(w.Z, nd, nd, w.invs, w.sel, w.wk,
                                                                         (int)sel.size(), w.Cs, (int)sel.size());
        }
        // out[k] = sum_i W[i][k] Y_i
        st = zgemm_tn((int)sel.size(), npw, nd, w.Cs, (int)sel.size(), nullptr, Y, ld, out, ld, false, s);
        if (st) return st;
        return cuda_check(cudaGetLastError(), "lowdin launches");
    }
};

}  // namespace

extern "C" qm_status qm_davidson(qm_gspace g, int ik, int nb, void* psi_inout, int ld_psi, const double* vloc_r,
                                 int nproj, const void* beta, int ld_beta, const double* D,
                                 const qm_davidson_opts* opts, double* eig_out, qm_davidson_stats* stats,
                                 void* stream) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_davidson: NULL gspace");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_davidson: ik out of range");
    if (nb <= 0) return fail(QM_ERR_ARG, "qm_davidson: nb must be > 0");
    if (!psi_inout || !vloc_r || !eig_out) return fail(QM_ERR_ARG, "qm_davidson: NULL psi, vloc_r or eig_out");
    if (nproj < 0 || (nproj > 0 && (!beta || !D))) return fail(QM_ERR_ARG, "qm_davidson: bad projectors");
    const int npw = g->k[ik].npw;
    if (ld_psi < npw || (nproj > 0 && ld_beta < npw)) return fail(QM_ERR_ARG, "qm_davidson: leading dimension < npw");
    if (nb > npw / 2) return fail(QM_ERR_ARG, "qm_davidson: nb must be <= npw / 2");
    if ((uintptr_t)psi_inout % 16 || (nproj > 0 && (uintptr_t)beta % 16))
        return fail(QM_ERR_ARG, "qm_davidson: psi/beta not 16-byte aligned");
    qm_davidson_opts o;
    o.tol = 1e-8;
    o.max_iter = 100;
    o.nvecx = 4 * nb;
    o.prec = QM_FP64;
    if (opts) o = *opts;
    if (o.nvecx <= 0) o.nvecx = 4 * nb;
    o.nvecx = std::min(o.nvecx, npw);
    if (o.nvecx < 2 * nb) return fail(QM_ERR_ARG, "qm_davidson: nvecx must be >= 2 nb");
    if (!(o.tol > 0.0) || o.max_iter < 1) return fail(QM_ERR_ARG, "qm_davidson: tol must be > 0, max_iter >= 1");
    if (o.prec != QM_FP64) return fail(QM_ERR_UNSUPPORTED, "qm_davidson: only QM_FP64 H psi in this build");

    qm_status st = ensure_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();

    DavidsonRun run;
    run.g = g;
    run.ik = ik;
    run.nb = nb;
    run.npw = npw;
    run.ld = (int)align_up((size_t)npw, 2);
    run.nvecx = o.nvecx;
    run.nproj = nproj;
    run.ldb = ld_beta;
    run.vloc = vloc_r;
    run.beta = beta;
    run.D = D;
    run.s = s;
    const int ld = run.ld, nvx = o.nvecx;
    const int nsq = nvx + 1;  // padded small dimension
    // device workspace (grow-only, owned by the handle)
    const size_t big = (size_t)ld * sizeof(double2);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off = align_up(off + bytes, 256);
        return o2;
    };
    const size_t oV = take(big * nvx), oHV = take(big * nvx), oX = take(big * nb), oHX = take(big * nb),
                 oR = take(big * nb), oDl = take(big * nb), oTmp = take(big * nb);
    const size_t sq = (size_t)nsq * nsq * sizeof(double2);
    const size_t oHs = take(sq), oG = take(sq), oA = take(sq), oZ = take(sq), oCs = take(sq);
    const size_t oPart = take(gemm_cn_partial_bytes(false));
    const size_t oEval = take(sizeof(double) * nsq), oEps = take(sizeof(double) * nsq),
                 oRn = take(sizeof(double) * nsq), oTk = take(sizeof(double) * nsq),
                 oRed = take(sizeof(double) * 2 * kJacobiMaxBlocks), oInvs = take(sizeof(double) * nsq),
                 oWk = take(sizeof(double) * nsq), oSel = take(sizeof(int) * nsq), oInfo = take(sizeof(int) * 4),
                 oRot = take(jacobi_rot_bytes(nsq)), oHeev = take(heev_work_bytes(nsq, nsq));
    if ((st = ensure_dav_workspace(g, off, s))) return st;
    char* base = (char*)g->dws.ptr;
    Ws& w = run.w;
    w.V = (double2*)(base + oV);
    w.HV = (double2*)(base + oHV);
    w.X = (double2*)(base + oX);
    w.HX = (double2*)(base + oHX);
    w.R = (double2*)(base + oR);
    w.Dl = (double2*)(base + oDl);
    w.Tmp = (double2*)(base + oTmp);
    w.Hs = (double2*)(base + oHs);
    w.G = (double2*)(base + oG);
    w.A = (double2*)(base + oA);
    w.Z = (double2*)(base + oZ);
    w.Cs = (double2*)(base + oCs);
    w.Part = (double2*)(base + oPart);
    w.eval = (double*)(base + oEval);
    w.eps = (double*)(base + oEps);
    w.rn2 = (double*)(base + oRn);
    w.tk = (double*)(base + oTk);
    w.red = (double*)(base + oRed);
    w.invs = (double*)(base + oInvs);
    w.wk = (double*)(base + oWk);
    w.sel = (int*)(base + oSel);
    w.info = (int*)(base + oInfo);
    w.rot = base + oRot;
    w.heev = base + oHeev;
    const double* kin = g->k[ik].kin;

    // initial block: psi -> rows of Tmp (dense ld), orthonormalised into V
    if ((st = cuda_check(cudaMemcpy2DAsync(w.Tmp, big, psi_inout, (size_t)ld_psi * sizeof(double2),
                                           (size_t)npw * sizeof(double2), nb, cudaMemcpyDeviceToDevice, s),
                         "copy psi")))
        return st;
    int kept = 0;
    if ((st = run.lowdin(w.Tmp, nb, w.V, &kept))) return st;
    if (kept < nb) return fail(QM_ERR_NUMERIC, "qm_davidson: initial psi block is rank deficient");
    if ((st = run.hpsi(w.V, w.HV, nb))) return st;
    int m = nb, m0 = 0;
    std::vector<double> rn2(nb), eps(nb);
    int it = 0;
    bool converged = false;
    double max_res = 0.0;
    for (it = 1; it <= o.max_iter; ++it) {
        // new columns of H_sub
        if ((st = zgemm_cn(m, m - m0, npw, w.V, ld, w.HV + (size_t)m0 * ld, ld, w.Hs + m0, nsq, w.Part,
                           zgemm_cn_splits(m, m - m0, npw), s)))
            return st;
        {
            ProfScope pf(PF_OTHER, s);
            k_herm_fill<<<grid_for((long)m * (m - m0)), 256, 0, s>>>(w.Hs, nsq, m0, m);
        }
        {
            ProfScope pf(PF_OTHER, s);
            k_herm_copy<<<grid_for((long)m * m), 256, 0, s>>>(w.Hs, nsq, m, w.A, m);
        }
        // lowest nb eigenpairs: values -> eps (device, increasing), vectors -> Cs [m][nb]
        if ((st = heev_lowest(w.A, m, m, nb, w.eps, w.Cs, nb, w.heev, s))) return st;
        if ((st = zgemm_tn(nb, npw, m, w.Cs, nb, nullptr, w.V, ld, w.X, ld, false, s)) ||
            (st = zgemm_tn(nb, npw, m, w.Cs, nb, nullptr, w.HV, ld, w.HX, ld, false, s)))
            return st;
        {
            ProfScope pf(PF_OTHER, s);
            k_residual<<<nb, 256, 0, s>>>(w.X, w.HX, ld, npw, w.eps, kin, w.R, w.rn2, w.tk);
        }
        if ((st = cuda_check(cudaMemcpyAsync(rn2.data(), w.rn2, sizeof(double) * nb, cudaMemcpyDeviceToHost, s),
                             "D2H residual norms")) ||
            (st = cuda_check(cudaMemcpyAsync(eps.data(), w.eps, sizeof(double) * nb, cudaMemcpyDeviceToHost, s),
                             "D2H Ritz values")) ||
            (st = cuda_check(cudaStreamSynchronize(s), "stream sync")))
            return st;
        for (int n = 0; n < nb; ++n)
            if (!std::isfinite(eps[n])) return fail(QM_ERR_NUMERIC, "qm_davidson: non-finite Ritz value");
        std::vector<int> unc;
        max_res = 0.0;
        for (int n = 0; n < nb; ++n) {
            double r = std::sqrt(rn2[n]);
            if (!std::isfinite(r)) return fail(QM_ERR_NUMERIC, "qm_davidson: non-finite residual");
            max_res = std::max(max_res, r);
            if (r > o.tol) unc.push_back(n);
        }
        if (unc.empty()) {
            converged = true;
            break;
        }
        if (it == o.max_iter) break;
        const int nu = (int)unc.size();
        cudaMemcpyAsync(w.sel, unc.data(), sizeof(int) * nu, cudaMemcpyHostToDevice, s);
        {
            ProfScope pf(PF_OTHER, s);
            k_tpa<<<dim3((npw + 255) / 256 < 64 ? (npw + 255) / 256 : 64, nu), 256, 0, s>>>(w.R, ld, npw, w.sel, w.tk,
                                                                                            kin, w.Dl, ld);
        }
        if (m + nu > nvx) {  // restart from the Ritz vectors
            cudaMemcpyAsync(w.V, w.X, big * nb, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(w.HV, w.HX, big * nb, cudaMemcpyDeviceToDevice, s);
            {
                ProfScope pf(PF_OTHER, s);
                k_set_diag<<<grid_for((long)nb * nb), 256, 0, s>>>(w.Hs, nsq, nb, w.eps);
            }
            m = nb;
        }
        // two classical Gram-Schmidt passes against the basis
        for (int pass = 0; pass < 2; ++pass) {
            if ((st = zgemm_cn(m, nu, npw, w.V, ld, w.Dl, ld, w.Cs, nu, w.Part, zgemm_cn_splits(m, nu, npw), s)) ||
                (st = zgemm_tn(nu, npw, m, w.Cs, nu, nullptr, w.V, ld, w.Dl, ld, true, s, -1.0)))
                return st;
        }
        if ((st = run.lowdin(w.Dl, nu, w.V + (size_t)m * ld, &kept))) return st;
        if (kept == 0) break;  // no new directions: stagnation
        if ((st = run.hpsi(w.V + (size_t)m * ld, w.HV + (size_t)m * ld, kept))) return st;
        m0 = m;
        m += kept;
    }
    // outputs: Ritz vectors and values
    if ((st = cuda_check(cudaMemcpy2DAsync(psi_inout, (size_t)ld_psi * sizeof(double2), w.X, big,
                                           (size_t)npw * sizeof(double2), nb, cudaMemcpyDeviceToDevice, s),
                         "copy psi out")) ||
        (st = cuda_check(cudaStreamSynchronize(s), "stream sync")))
        return st;
    for (int n = 0; n < nb; ++n) eig_out[n] = eps[n];
    if (stats) {
        stats->iterations = it > o.max_iter ? o.max_iter : it;
        stats->band_applies = run.applies;
        stats->max_residual = max_res;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->converged = converged ? 1 : 0;
    }
    if (!converged) return fail(QM_ERR_NOT_CONVERGED, "qm_davidson: max_iter reached before tol");
    return QM_OK;
}

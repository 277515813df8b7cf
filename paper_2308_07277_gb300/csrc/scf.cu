// qm_scf: Kohn-Sham self-consistency around the block Davidson (Sec. 2.1: n -> V -> {psi} ->
// n_out -> mix, until n_out = n; Sec. 5, dft module scf with density mixing).
//
// Every step: V = V_ext + V_H[n_in] + v_xc(n_in) (scf_potential_run), Davidson at every k-point
// from the previous step's states, n_out = sum_k w_k sum_{n < nelec/2} 2 |psi_nk(r)|^2
// (scf_density_run), F = n_out - n_in, stop when (Omega/N_r) sum |F| <= tol, else Anderson mixing
// of the density (D. G. Anderson, J. ACM 12, 547 (1965); equal-weight modified Broyden is the
// same update, V. Eyert, J. Comput. Phys. 124, 271 (1996)):
//     n_in <- n_in + a F - sum_j gamma_j (dX_j + a dF_j),  gamma = argmin || F - sum_j gamma_j dF_j ||,
// over the last m differences dX_j, dF_j of successive n_in and F.  The densities live on the
// device; the m x m normal equations are solved on the host from device inner products.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "qm_internal.h"

namespace qm {

constexpr int kMaxHistory = 8;
constexpr int kDotBlocks = 304;

// F = a - b;  partial sums of |F| per block
__global__ void k_residual_abs(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ F,
                               size_t n, double* __restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double f = a[i] - b[i];
        F[i] = f;
        s += fabs(f);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// partial inner products <v_i, v_j> (i <= j < nv) and <v_i, F> per block: part[blk][...]
__global__ void k_gram(const double* const* __restrict__ v, int nv, const double* __restrict__ F, size_t n,
                       double* __restrict__ part) {
    __shared__ double red[256];
    const int npair = nv * (nv + 1) / 2 + nv;
    for (int q = 0; q < npair; ++q) {
        int i, j;
        const double *x, *y;
        if (q < nv * (nv + 1) / 2) {
            i = 0;
            int r = q;
            while (r >= nv - i) {
                r -= nv - i;
                ++i;
            }
            j = i + r;
            x = v[i];
            y = v[j];
        } else {
            x = v[q - nv * (nv + 1) / 2];
            y = F;
        }
        double s = 0.0;
        for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
            s += x[t] * y[t];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * npair + q] = red[0];
        __syncthreads();
    }
}

struct MixCoef {
    int m;
    double a;
    double gamma[kMaxHistory];
    const double* dx[kMaxHistory];
    const double* df[kMaxHistory];
};

// x <- x + a F - sum_j gamma_j (dX_j + a dF_j)
__global__ void k_mix(double* __restrict__ x, const double* __restrict__ F, size_t n, const MixCoef c) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        double v = x[t] + c.a * F[t];
        for (int j = 0; j < c.m; ++j) v -= c.gamma[j] * (c.dx[j][t] + c.a * c.df[j][t]);
        x[t] = v;
    }
}

// d = a - b
__global__ void k_diff(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ d, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        d[t] = a[t] - b[t];
}

__global__ void k_fill(double* __restrict__ x, double v, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) x[t] = v;
}

// solve the symmetric positive semi-definite m x m system A g = b (normal equations of the
// least-squares problem) by Cholesky with a relative diagonal shift; false if it breaks down
static bool small_solve(int m, std::vector<double> A, std::vector<double> b, double* g) {
    double tr = 0.0;
    for (int i = 0; i < m; ++i) tr = std::max(tr, A[i * m + i]);
    for (int i = 0; i < m; ++i) A[i * m + i] += 1e-14 * tr;
    for (int j = 0; j < m; ++j) {
        double d = A[j * m + j];
        for (int k = 0; k < j; ++k) d -= A[j * m + k] * A[j * m + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        A[j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            double s = A[i * m + j];
            for (int k = 0; k < j; ++k) s -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = s / d;
        }
    }
    for (int i = 0; i < m; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= A[i * m + k] * b[k];
        b[i] = s / A[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < m; ++k) s -= A[k * m + i] * b[k];
        b[i] = s / A[i * m + i];
    }
    for (int i = 0; i < m; ++i) g[i] = b[i];
    return true;
}

static double cell_volume(const double* a) {
    return std::fabs(a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]));
}

}  // namespace qm

using namespace qm;

extern "C" qm_status qm_scf(qm_gspace g, int nelec, const double* wk, int nb, void* const* psi, int ld_psi,
                            const double* vion_r, int nproj, const void* const* beta, int ld_beta, const double* D,
                            const qm_scf_opts* opts_in, double* eigs, double* rho_r, double* vloc_r,
                            qm_scf_stats* stats, void* stream) {
    clear_error();
    const auto t0 = std::chrono::steady_clock::now();
    if (!g) return fail(QM_ERR_ARG, "qm_scf: NULL gspace");
    qm_scf_opts o{1e-8, 50, 0.5, 4, 1e-9, 100, QM_FP64};
    if (opts_in) o = *opts_in;
    if (!(o.tol > 0) || o.max_iter < 1 || !(o.alpha > 0 && o.alpha <= 1) || o.history < 0 ||
        o.history > kMaxHistory || !(o.dav_tol > 0) || o.dav_max_iter < 1 || (o.prec != QM_FP64 && o.prec != QM_MIXED))
        return fail(QM_ERR_ARG, "qm_scf: option out of range");
    if (nelec < 2 || nelec % 2) return fail(QM_ERR_ARG, "qm_scf: nelec must be even and >= 2");
    if (nb < nelec / 2) return fail(QM_ERR_ARG, "qm_scf: nb < nelec / 2");
    if (!wk || !psi || !vion_r || !eigs || !rho_r || !vloc_r) return fail(QM_ERR_ARG, "qm_scf: NULL argument");
    if (nproj < 0 || (nproj > 0 && (!beta || !D))) return fail(QM_ERR_ARG, "qm_scf: NULL projectors with nproj > 0");
    const int nk = g->nk;
    double wsum = 0.0;
    for (int ik = 0; ik < nk; ++ik) {
        if (!psi[ik]) return fail(QM_ERR_ARG, "qm_scf: NULL psi of a k-point");
        if (nproj > 0 && !beta[ik]) return fail(QM_ERR_ARG, "qm_scf: NULL beta of a k-point");
        if (ld_psi < g->k[ik].npw || (nproj > 0 && ld_beta < g->k[ik].npw))
            return fail(QM_ERR_ARG, "qm_scf: leading dimension < npw");
        if (!(wk[ik] >= 0)) return fail(QM_ERR_ARG, "qm_scf: negative k-point weight");
        wsum += wk[ik];
    }
    if (std::fabs(wsum - 1.0) > 1e-12) return fail(QM_ERR_ARG, "qm_scf: k-point weights must sum to 1");
    // the density sphere (the dual cutoff 4 E_c) on the same grid, at k = 0
    qm_gspace grho = nullptr;
    {
        const double k0[3] = {0.0, 0.0, 0.0};
        qm_status st = qm_gspace_create(g->lattice, 1, k0, 4.0 * g->ecut, g->n, &grho);
        if (st) return fail(QM_ERR_ARG, "qm_scf: the FFT grid does not hold the density sphere (4 E_c)");
    }
    struct Guard {
        qm_gspace h;
        void* mem = nullptr;
        ~Guard() {
            if (mem) cudaFree(mem);
            qm_gspace_destroy(h);
        }
    } guard{grho};
    cudaStream_t s = (cudaStream_t)stream;
    qm_status st;
    if ((st = ensure_device(g)) || (st = ensure_device(grho))) return st;

    const int nocc = nelec / 2;
    const size_t nrr = (size_t)g->n[0] * g->n[1] * g->n[2];
    const double omega = cell_volume(g->lattice);
    const int m = o.history;
    // device memory: n_in | n_out (then F) | V | previous n_in, F | m dX | m dF | partial sums | pointer table | work
    const size_t vec = align_up(nrr * sizeof(double), 256);
    const int npair = (2 * m) * (2 * m + 1) / 2 + 2 * m;
    const size_t part_bytes = align_up((size_t)kDotBlocks * std::max(npair, 1) * sizeof(double), 256);
    const size_t ptr_bytes = align_up(2 * kMaxHistory * sizeof(double*), 256);
    const size_t work_bytes = scf_work_size(g, grho, nocc);
    const size_t total = vec * (5 + 2 * (size_t)m) + part_bytes + ptr_bytes + work_bytes;
    if (cudaMalloc(&guard.mem, total) != cudaSuccess) {
        cudaGetLastError();
        guard.mem = nullptr;
        return fail(QM_ERR_OOM, "qm_scf: device workspace");
    }
    char* base = (char*)guard.mem;
    double* n_in = (double*)base;
    double* F = (double*)(base + vec);
    double* V = (double*)(base + 2 * vec);
    double* x_prev = (double*)(base + 3 * vec);
    double* f_prev = (double*)(base + 4 * vec);
    std::vector<double*> dX(m), dF(m);
    for (int j = 0; j < m; ++j) {
        dX[j] = (double*)(base + (5 + j) * vec);
        dF[j] = (double*)(base + (5 + m + j) * vec);
    }
    double* part = (double*)(base + (5 + 2 * (size_t)m) * vec);
    const double** dptr = (const double**)(base + (5 + 2 * (size_t)m) * vec + part_bytes);
    void* work = base + (5 + 2 * (size_t)m) * vec + part_bytes + ptr_bytes;
    const int blocks = grid_stride_blocks(nrr, 256, 8);

    {
        ProfScope pf(PF_OTHER, s);
        k_fill<<<blocks, 256, 0, s>>>(n_in, nelec / omega, nrr);
    }
    qm_davidson_opts dopt{};
    dopt.tol = o.dav_tol;
    dopt.max_iter = o.dav_max_iter;
    dopt.prec = o.prec;
    int hist = 0, head = 0;
    bool have_prev = false, converged = false;
    double drho = 0.0;
    long long applies = 0;
    int it = 0;
    std::vector<double> hpart;
    for (it = 1; it <= o.max_iter; ++it) {
        if ((st = scf_potential_run(g, grho, n_in, vion_r, V, work, work_bytes, s))) return st;
        for (int ik = 0; ik < nk; ++ik) {
            qm_davidson_stats ds{};
            st = qm_davidson(g, ik, nb, psi[ik], ld_psi, V, nproj, nproj ? beta[ik] : nullptr, ld_beta, D, &dopt,
                             eigs + (size_t)ik * nb, &ds, stream);
            applies += ds.band_applies;
            if (st && st != QM_ERR_NOT_CONVERGED) return st;
        }
        // n_out accumulates in F, then F = n_out - n_in
        {
            ProfScope pf(PF_OTHER, s);
            k_fill<<<blocks, 256, 0, s>>>(F, 0.0, nrr);
        }
        for (int ik = 0; ik < nk; ++ik)
            if ((st = scf_density_run(g, ik, nocc, (const double2*)psi[ik], ld_psi, 2.0 * wk[ik] / omega, F, work, s)))
                return st;
        {
            ProfScope pf(PF_OTHER, s);
            k_residual_abs<<<kDotBlocks, 256, 0, s>>>(F, n_in, F, nrr, part);
        }
        hpart.resize(kDotBlocks);
        if ((st = cuda_check(cudaMemcpyAsync(hpart.data(), part, kDotBlocks * sizeof(double), cudaMemcpyDeviceToHost, s),
                             "qm_scf: read back")) ||
            (st = cuda_check(cudaStreamSynchronize(s), "qm_scf: sync")))
            return st;
        double sabs = 0.0;
        for (double x : hpart) sabs += x;
        drho = omega / (double)nrr * sabs;
        if (!std::isfinite(drho)) return fail(QM_ERR_NUMERIC, "qm_scf: non-finite density residual");
        if (drho <= o.tol) {
            converged = true;
            break;
        }
        if (it == o.max_iter) break;
        // history: dX = n_in - x_prev, dF = F - f_prev (ring of m)
        if (have_prev && m > 0) {
            ProfScope pf(PF_OTHER, s);
            k_diff<<<blocks, 256, 0, s>>>(n_in, x_prev, dX[head], nrr);
            k_diff<<<blocks, 256, 0, s>>>(F, f_prev, dF[head], nrr);
            head = (head + 1) % m;
            hist = std::min(hist + 1, m);
        }
        if ((st = cuda_check(cudaMemcpyAsync(x_prev, n_in, nrr * sizeof(double), cudaMemcpyDeviceToDevice, s),
                             "qm_scf: copy")) ||
            (st = cuda_check(cudaMemcpyAsync(f_prev, F, nrr * sizeof(double), cudaMemcpyDeviceToDevice, s),
                             "qm_scf: copy")))
            return st;
        have_prev = true;
        MixCoef c{};
        c.a = o.alpha;
        c.m = 0;
        if (hist > 0) {
            // order the stored differences oldest first; gram of the dF's and their products with F
            std::vector<const double*> ptrs(hist);
            for (int j = 0; j < hist; ++j) {
                const int slot = (head - hist + j + m) % m;
                ptrs[j] = dF[slot];
                c.dx[j] = dX[slot];
                c.df[j] = dF[slot];
            }
            const int np = hist * (hist + 1) / 2 + hist;
            if ((st = cuda_check(cudaMemcpyAsync(dptr, ptrs.data(), hist * sizeof(double*), cudaMemcpyHostToDevice, s),
                                 "qm_scf: pointer table")))
                return st;
            {
                ProfScope pf(PF_OTHER, s);
                k_gram<<<kDotBlocks, 256, 0, s>>>(dptr, hist, F, nrr, part);
            }
            hpart.resize((size_t)kDotBlocks * np);
            if ((st = cuda_check(cudaMemcpyAsync(hpart.data(), part, hpart.size() * sizeof(double),
                                                 cudaMemcpyDeviceToHost, s), "qm_scf: read back")) ||
                (st = cuda_check(cudaStreamSynchronize(s), "qm_scf: sync")))
                return st;
            std::vector<double> sum(np, 0.0), A((size_t)hist * hist), b(hist);
            for (int blk = 0; blk < kDotBlocks; ++blk)
                for (int q = 0; q < np; ++q) sum[q] += hpart[(size_t)blk * np + q];
            int q = 0;
            for (int i = 0; i < hist; ++i)
                for (int j = i; j < hist; ++j, ++q) A[i * hist + j] = A[j * hist + i] = sum[q];
            for (int i = 0; i < hist; ++i) b[i] = sum[q + i];
            if (small_solve(hist, A, b, c.gamma)) c.m = hist;
        }
        {
            ProfScope pf(PF_OTHER, s);
            k_mix<<<blocks, 256, 0, s>>>(n_in, F, nrr, c);
        }
    }
    if ((st = cuda_check(cudaMemcpyAsync(rho_r, n_in, nrr * sizeof(double), cudaMemcpyDeviceToDevice, s),
                         "qm_scf: output")) ||
        (st = cuda_check(cudaMemcpyAsync(vloc_r, V, nrr * sizeof(double), cudaMemcpyDeviceToDevice, s),
                         "qm_scf: output")) ||
        (st = cuda_check(cudaStreamSynchronize(s), "qm_scf: sync")))
        return st;
    if (stats) {
        stats->iterations = std::min(it, o.max_iter);
        stats->converged = converged ? 1 : 0;
        stats->drho = drho;
        stats->band_applies = applies;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return converged ? QM_OK : fail(QM_ERR_NOT_CONVERGED, "qm_scf: max_iter reached before the density converged");
}

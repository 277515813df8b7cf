// qm_davidson: lowest nb eigenpairs of H(k) by block Davidson (Sec. 5, dft module: a
// matrix-free "Davidson with overlap" that only applies H to blocks of trial vectors).
//
// Per iteration, on the caller's stream (host loop; two small device->host reads):
//   Rayleigh-Ritz   H_sub = V^H (H V) (new columns only), dense Hermitian eigensolve in FP64
//                   (heev.cu: Householder reduction, multisection, inverse iteration)
//   Ritz vectors    X = V c, HX = (HV) c for the lowest nb eigenpairs
//   residuals       r_n = HX_n - eps_n X_n, ||r_n|| and T_n = <X_n|T|X_n> (FP64)
//   corrections     delta_n = K_TPA(kin / T_n) r_n (or the learned K) for the bands with
//                   ||r_n|| > tol
//   restart         if the basis would exceed nvecx: V <- X, HV <- HX
//   orthonormalise  two classical Gram-Schmidt passes against V and two passes of
//                   Cholesky-QR within the block, near-dependent directions dropped
//   expand          V <- [V, delta], HV <- [HV, H delta]
// The basis is kept orthonormal, so the subspace overlap S_sub is the identity to FP64
// round-off and Rayleigh-Ritz is a standard Hermitian eigenproblem.
//
// Precision form (QM_MIXED): H psi in FP32 and the subspace products as BF16x3 split products
// on the tensor cores (FP64 storage rounded to FP32 on load, FP32 accumulation per K split,
// splits summed in FP64); with mixed_ortho = 1 the coefficients of the second Gram-Schmidt
// pass and the second Cholesky-QR pass stay FP64, which keeps the basis orthonormal to FP64
// round-off; eigensolves, residual norms and band energies in FP64.  Once the largest residual
// is below mixed_switch (or stops falling), the Ritz vectors are re-orthonormalised, H is
// applied to them in FP64 (refinement sweep), and the iterations continue with FP64 H psi and
// exact orthogonalisation passes; with buffer bands that FP64 phase is anchored on the Ritz
// vectors of each restart (see the loop below), which leaves the products of small
// quantities on the tensor cores.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
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
    const int n = sel ? sel[j] : j;  // sel == NULL: row j is band j
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

// partial sums of V(r) over a grid stride (one per block, fixed order: deterministic)
__global__ void __launch_bounds__(256) k_vsum(const double* __restrict__ V, size_t nr, double* __restrict__ part) {
    __shared__ double sh[256];
    double a = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nr; i += (size_t)gridDim.x * blockDim.x) a += V[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// hdiag[G] = kin[G] + mean(V) + sum_p D_p |beta_p(G)|^2: the diagonal of H(k) (Eq. KSHamMat with
// the KB term of Sec. 2.3; the G = G' coefficient of the local part is the mean of V(r))
__global__ void __launch_bounds__(256) k_hdiag(const double* __restrict__ kin, int npw, const double* __restrict__ part,
                                               int npart, double inv_nr, const double2* __restrict__ beta, int ld,
                                               int nproj, const double* __restrict__ D, double* __restrict__ hdiag) {
    __shared__ double vmean;
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int b = 0; b < npart; ++b) a += part[b];
        vmean = a * inv_nr;
    }
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npw) return;
    double nl = 0.0;
    for (int p = 0; p < nproj; ++p) {
        const double2 b = beta[(size_t)p * ld + g];
        nl += D[p] * (b.x * b.x + b.y * b.y);
    }
    hdiag[g] = kin[g] + vmean + nl;
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

// dst[j][i] = src[i][c(j)] for i < ni, j < nj, c(j) = sel ? sel[j] : j (column gather + transpose)
__global__ void k_cols_to_rows(const double2* __restrict__ src, int lds, int ni, const int* __restrict__ sel, int nj,
                               double2* __restrict__ dst, int ldd) {
    const long total = (long)ni * nj;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e / ni), i = (int)(e % ni);
        dst[(size_t)j * ldd + i] = src[(size_t)i * lds + (sel ? sel[j] : j)];
    }
}

// zero the rows of X (n rows of length len) whose 2-norm is below thresh: one warp per row
__global__ void k_zero_small_rows(double2* __restrict__ X, int ld, int n, int len, double thresh) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= n) return;
    double2* x = X + (size_t)row * ld;
    double s2 = 0.0;
    for (int i = lane; i < len; i += 32) s2 += x[i].x * x[i].x + x[i].y * x[i].y;
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (s2 < thresh * thresh)
        for (int i = lane; i < len; i += 32) x[i] = make_double2(0.0, 0.0);
}

// C[i][j] = (i == j) for i < rows, j < cols
__global__ void k_set_identity(double2* __restrict__ C, int ld, int rows, int cols) {
    const long total = (long)rows * cols;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int i = (int)(e / cols), j = (int)(e % cols);
        C[(size_t)i * ld + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
}

template <class D, class S>
__global__ void k_convert_rows(const S* __restrict__ in, int ldi, D* __restrict__ out, int ldo, int rows, int cols) {
    const long total = (long)rows * cols;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const S v = in[(size_t)r * ldi + c];
        D o;
        o.x = (decltype(o.x))v.x;
        o.y = (decltype(o.y))v.y;
        out[(size_t)r * ldo + c] = o;
    }
}

inline int grid_for(long n) { return grid_stride_blocks((size_t)std::max<long>(n, 1), 256, 8); }

template <class D, class S>
qm_status convert_rows(const S* in, int ldi, D* out, int ldo, int rows, int cols, cudaStream_t s) {
    if (rows <= 0) return QM_OK;
    ProfScope pf(PF_CONVERT, s);
    k_convert_rows<D, S><<<grid_for((long)rows * cols), 256, 0, s>>>(in, ldi, out, ldo, rows, cols);
    return cuda_check(cudaGetLastError(), "k_convert_rows launch");
}

}  // namespace

qm_status hamiltonian_diag(qm_gspace g, int ik, const double* vloc, int nproj, const double2* beta, int ld_beta,
                           const double* D, double* hdiag, double* work, cudaStream_t s) {
    const size_t nr = (size_t)g->n[0] * g->n[1] * g->n[2];
    const int npw = g->k[ik].npw;
    {
        ProfScope pf(PF_OTHER, s);
        k_vsum<<<kVmeanBlocks, 256, 0, s>>>(vloc, nr, work);
    }
    {
        ProfScope pf(PF_OTHER, s);
        k_hdiag<<<(npw + 255) / 256, 256, 0, s>>>(g->k[ik].kin, npw, work, kVmeanBlocks, 1.0 / (double)nr, beta,
                                                   ld_beta, nproj, D, hdiag);
    }
    return cuda_check(cudaGetLastError(), "hamiltonian diagonal launch");
}

namespace {

struct Ws {
    double2 *V, *HV, *X, *HX, *R, *Dl, *Tmp;  // [.. rows][ld]
    double2 *Hs, *G, *A, *Z, *Cs, *Part;      // small
    double2 *Cp, *CT, *PT, *QT;               // previous Ritz coefficients [nvecx+1][nb]; transposed blocks
    double2 *Y, *HY;                          // [nb][ld]: previous-direction rows kept at a restart
    double *eval, *eps, *rn2, *tk, *hdiag, *vpart;
    int *sel, *rank, *info;
    void* heev;
};

}  // namespace



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
    long long applies = 0, applies_mixed = 0;
    bool mixed = false;          // current phase: FP32 H psi and tensor-core (FP32-accuracy) subspace products
    float2* psi32 = nullptr;     // [nb][ld] FP32 staging of the vectors H is applied to
    float2* hpsi32 = nullptr;    // [nb][ld]
    float2* beta32 = nullptr;    // [nproj][ld]
    void* beta_tc = nullptr;     // the projectors split once into the tensor-core operand layouts
    bool tc = false;             // precision form: tensor-core subspace products available
    bool anchored = false;       // precision form, FP64 phase: basis rows 0..nb-1 are the Ritz
                                 // vectors of the last restart (the anchor), see qm_davidson
    bool ortho64 = false;        // FP32 phase: second CGS pass coefficients and Cholesky-QR pass in FP64
    void* sub = nullptr;         // tensor-core subspace products: split-K partials / coefficient operand
    size_t sub_bytes = 0;
    int* tc_err = nullptr;       // device error word of the tensor-core waits

    bool ds = false;             // precision form: the FP64 phase's long products in double-FP32
    qm_status hpsi(const double2* in, double2* out, int n) {
        applies += n;
        if (!mixed) return hpsi_run(g, ik, n, in, ld, vloc, nproj, beta, ldb, nullptr, D, out, ld, QM_FP64, s, ds);
        applies_mixed += n;
        qm_status st = convert_rows(in, ld, psi32, ld, n, npw, s);
        if (st) return st;
        st = hpsi_run(g, ik, n, psi32, ld, vloc, nproj, beta32, ld, beta_tc, D, hpsi32, ld, QM_MIXED, s);
        if (st) return st;
        return convert_rows(hpsi32, ld, out, ld, n, npw, s);
    }
    // tensor-core (BF16x3, FP32 accuracy) and FP64 forms of the two subspace products
    qm_status cn_tc(int M, int N, const double2* A, const double2* B, double2* C, int ldc) {
        return zgemm_cn_bf16x3(M, N, npw, A, ld, B, ld, C, ldc, sub, sub_bytes, tc_err, s);
    }
    qm_status cn64(int M, int N, const double2* A, const double2* B, double2* C, int ldc) {
        return (ds ? zgemm_cn_ds : zgemm_cn)(M, N, npw, A, ld, B, ld, C, ldc, w.Part, zgemm_cn_splits(M, N, npw), s);
    }
    qm_status tn_tc(int M, int K, const double2* A, int lda, const double2* B, double2* C, bool acc,
                    double alpha = 1.0) {
        return zgemm_tn_bf16x3(M, npw, K, A, lda, B, ld, C, ld, acc, alpha, sub, sub_bytes, tc_err, s);
    }
    qm_status tn64(int M, int K, const double2* A, int lda, const double2* B, double2* C, bool acc,
                   double alpha = 1.0) {
        return (ds ? zgemm_tn_ds : zgemm_tn)(M, npw, K, A, lda, nullptr, B, ld, C, ld, acc, s, alpha);
    }
    // products whose precision follows the phase: H_sub columns and the Ritz vectors
    qm_status gemm_cn(int M, int N, const double2* A, const double2* B, double2* C, int ldc) {
        return mixed ? cn_tc(M, N, A, B, C, ldc) : cn64(M, N, A, B, C, ldc);
    }
    qm_status gemm_tn(int M, int K, const double2* A, int lda, const double2* B, double2* C, bool acc) {
        return mixed ? tn_tc(M, K, A, lda, B, C, acc) : tn64(M, K, A, lda, B, C, acc);
    }
    // Precision form: the second pass of an orthogonalisation (Gram-Schmidt coefficients,
    // Cholesky-QR Gram matrix) is FP64 in the FP64 phase (and with ortho64), which keeps the
    // basis orthonormal to FP64 round-off; every other orthogonalisation product is a
    // tensor-core product, either of O(1) coefficients followed by that exact pass, or of tiny
    // coefficients (the exact pass's corrections), whose FP32 relative error is negligible.
    bool exact_second_pass() const { return !tc || !mixed || ortho64; }

    // Thick restart with the previous Ritz vectors (the "+k" of GD+k restarting; Stathopoulos &
    // Saad, Electron. Trans. Numer. Anal. 7, 163 (1998)).  In coefficient space of the current
    // orthonormal basis (m rows): C (m x nb, Cs) holds the current Ritz vectors, Cp those of the
    // previous step (zero in the rows added since).  The previous Ritz vectors of the nu
    // unconverged bands (sel) are orthogonalised against C twice, rows below 1e-12 dropped,
    // orthonormalised by two Cholesky-QR passes with dropping, and at most cap of them kept as
    // Q; the rows Y = V Q and H Y = (H V) Q are written to w.Y, w.HY (*k rows).  The span of
    // [X, Y] is that of the current and previous Ritz vectors, which is what a plain Ritz
    // restart throws away.  All small products in FP64; Y in the precision of the phase.
    qm_status prev_directions(int m, int nu, int cap, int nsq, int* kout) {
        *kout = 0;
        if (nu <= 0 || cap <= 0) return QM_OK;
        qm_status st;
        {
            ProfScope pf(PF_OTHER, s);
            k_cols_to_rows<<<grid_for((long)m * nb), 256, 0, s>>>(w.Cs, nb, m, nullptr, nb, w.CT, nsq);
            k_cols_to_rows<<<grid_for((long)m * nu), 256, 0, s>>>(w.Cp, nb, m, w.sel, nu, w.PT, nsq);
        }
        if ((st = cuda_check(cudaGetLastError(), "k_cols_to_rows launch"))) return st;
        auto cgs = [&](double2* Pr, int n) -> qm_status {
            qm_status s2;
            if ((s2 = zgemm_cn(nb, n, m, w.CT, nsq, Pr, nsq, w.A, n, w.Part, zgemm_cn_splits(nb, n, m), s)) ||
                (s2 = zgemm_tn(n, m, nb, w.A, n, nullptr, w.CT, nsq, Pr, nsq, true, s, -1.0)))
                return s2;
            return QM_OK;
        };
        auto cholqr_c = [&](double2* src, int n, double2* dst, double drop, int* k) -> qm_status {
            qm_status s2;
            int kk = 0;
            if ((s2 = zgemm_cn(n, n, m, src, nsq, src, nsq, w.G, n, w.Part, zgemm_cn_splits(n, n, m), s)) ||
                (s2 = chol_transform(w.G, n, n, drop, w.sel, w.rank, w.info, w.A, w.Z, 0, s)) ||
                (s2 = cuda_check(cudaMemcpyAsync(&kk, w.info, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H kept")) ||
                (s2 = cuda_check(cudaStreamSynchronize(s), "stream sync")))
                return s2;
            *k = kk;
            if (kk == 0) return QM_OK;
            if ((s2 = chol_transform_rows(w.G, n, n, w.sel, w.rank, kk, w.A, w.Z, s))) return s2;
            return zgemm_tn(kk, m, n, w.Z, kk, nullptr, src, nsq, dst, nsq, false, s);
        };
        int k1 = 0, k2 = 0;
        if ((st = cgs(w.PT, nu)) || (st = cgs(w.PT, nu))) return st;
        {
            ProfScope pf(PF_OTHER, s);
            k_zero_small_rows<<<(nu + 7) / 8, 256, 0, s>>>(w.PT, nsq, nu, m, 1e-12);
        }
        if ((st = cholqr_c(w.PT, nu, w.QT, 1e-10, &k1))) return st;
        if (k1 == 0) return QM_OK;
        if ((st = cgs(w.QT, k1)) || (st = cholqr_c(w.QT, k1, w.PT, 1e-14, &k2))) return st;
        const int k = std::min(k2, cap);
        if (k == 0) return QM_OK;
        {
            ProfScope pf(PF_OTHER, s);  // Q [m][k] from its rows
            k_cols_to_rows<<<grid_for((long)m * k), 256, 0, s>>>(w.PT, nsq, k, nullptr, m, w.QT, k);
        }
        if ((st = cuda_check(cudaGetLastError(), "k_cols_to_rows launch")) ||
            (st = gemm_tn(k, m, w.QT, k, w.V, w.Y, false)) || (st = gemm_tn(k, m, w.QT, k, w.HV, w.HY, false)))
            return st;
        *kout = k;
        return QM_OK;
    }

    // One Cholesky-QR pass with dropping: the n_in rows of src -> *k orthonormal rows of dst.
    // exact: Gram matrix and transform in FP64 (the transform of an exact pass can be far from
    // the identity when the tensor-core pass before it met an ill-conditioned block, so it is
    // not split into identity + small remainder).  Pass 0 drops directions whose pivot is below
    // `drop` of their own norm^2; an exact second pass only drops exact null directions.
    qm_status chol_pass(const double2* src, int n_in, double2* dst, bool exact, double drop, int* kout) {
        qm_status st = exact ? cn64(n_in, n_in, src, src, w.G, n_in) : cn_tc(n_in, n_in, src, src, w.G, n_in);
        if (st) return st;
        int k = 0;
        if ((st = chol_transform(w.G, n_in, n_in, drop, w.sel, w.rank, w.info, w.A, w.Cs, 0, s)) ||
            (st = cuda_check(cudaMemcpyAsync(&k, w.info, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H kept")) ||
            (st = cuda_check(cudaStreamSynchronize(s), "stream sync")))
            return st;
        *kout = k;
        if (k == 0) return QM_OK;
        if ((st = chol_transform_rows(w.G, n_in, n_in, w.sel, w.rank, k, w.A, w.Cs, s))) return st;
        return (!tc || exact) ? tn64(k, n_in, w.Cs, k, src, dst, false) : tn_tc(k, n_in, w.Cs, k, src, dst, false);
    }

    // One classical Gram-Schmidt pass of the nu rows of D against the m basis rows V:
    // D -= V^T (V^H D) (coefficients in FP64 when exact).
    qm_status cgs_pass(int m, int nu, double2* D, bool exact) {
        qm_status st = exact ? cn64(m, nu, w.V, D, w.Cs, nu) : cn_tc(m, nu, w.V, D, w.Cs, nu);
        if (st) return st;
        return tc ? tn_tc(nu, m, w.Cs, nu, w.V, D, true, -1.0) : tn64(nu, m, w.Cs, nu, w.V, D, true, -1.0);
    }

    // Orthonormalise the nd rows of Y into the rows of out by two passes of Cholesky-QR
    // (first pass with dropping of near-dependent directions); *kept = rows written.  Uses R.
    qm_status cholqr(const double2* Y, int nd, double2* out, int* kept) {
        int k = 0;
        qm_status st = chol_pass(Y, nd, w.R, !tc, tc ? 1e-5 : 1e-12, &k);  // FP32 Gram: ~1e-7 noise
        if (st || k == 0) {
            *kept = 0;
            return st;
        }
        const bool ex = exact_second_pass();
        if ((st = chol_pass(w.R, k, out, ex, ex ? 1e-14 : 1e-10, kept))) return st;
        return QM_OK;
    }

    // The nu correction rows of D (overwritten) -> *kept rows at `out`, orthonormal and
    // orthogonal to the m basis rows.  Plain FP64: two Gram-Schmidt passes, then two
    // Cholesky-QR passes.  Precision form: Gram-Schmidt and Cholesky-QR on the tensor cores,
    // then a second Gram-Schmidt pass and Cholesky-QR pass, exact in the FP64 phase (and with
    // mixed_ortho = 1): FP64 coefficients, Gram matrix and transform; only the Gram-Schmidt
    // correction, whose coefficients are tiny, is applied on the tensor cores.  The exact
    // passes come last because a tensor-core transform of O(1) coefficients leaves ~1e-7
    // components along the basis, which only an exact pass after it removes.
    qm_status expand(int m, int nu, double2* out, int* kept) {
        qm_status st;
        *kept = 0;
        if (!tc) {
            if ((st = cgs_pass(m, nu, w.Dl, true)) || (st = cgs_pass(m, nu, w.Dl, true))) return st;
            return cholqr(w.Dl, nu, out, kept);
        }
        int k = 0;
        if ((st = cgs_pass(m, nu, w.Dl, false)) || (st = chol_pass(w.Dl, nu, w.R, false, 1e-5, &k))) return st;
        if (k == 0) return QM_OK;
        const bool ex = exact_second_pass();
        if ((st = cgs_pass(m, k, w.R, ex))) return st;
        return chol_pass(w.R, k, out, ex, ex ? 1e-14 : 1e-10, kept);
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
    qm_davidson_opts o{};
    o.tol = 1e-8;
    o.max_iter = 100;
    o.nvecx = 4 * nb;
    o.prec = QM_FP64;
    o.mixed_switch = 1e-4;
    if (opts) o = *opts;
    if (o.nvecx <= 0) o.nvecx = 4 * nb;
    o.nvecx = std::min(o.nvecx, npw);
    if (o.nvecx < 2 * nb) return fail(QM_ERR_ARG, "qm_davidson: nvecx must be >= 2 nb");
    if (!(o.tol > 0.0) || o.max_iter < 1) return fail(QM_ERR_ARG, "qm_davidson: tol must be > 0, max_iter >= 1");
    if (o.prec != QM_FP64 && o.prec != QM_MIXED) return fail(QM_ERR_ARG, "qm_davidson: unknown precision");
    if (!(o.mixed_switch > 0.0)) o.mixed_switch = 1e-4;
    if (o.nconv <= 0 || o.nconv > nb) o.nconv = nb;
    if (o.precond != 0 && o.precond != 1) return fail(QM_ERR_ARG, "qm_davidson: unknown preconditioner");
    if (o.mixed_ortho != 0 && o.mixed_ortho != 1) return fail(QM_ERR_ARG, "qm_davidson: mixed_ortho must be 0 or 1");
    if (o.plain_restart != 0 && o.plain_restart != 1) return fail(QM_ERR_ARG, "qm_davidson: plain_restart must be 0 or 1");
    if (o.fp64_exact != 0 && o.fp64_exact != 1) return fail(QM_ERR_ARG, "qm_davidson: fp64_exact must be 0 or 1");
    if (o.precond == 1 && !o.mlp) return fail(QM_ERR_ARG, "qm_davidson: learned preconditioner without parameters");

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
    const size_t big32 = (size_t)ld * sizeof(float2);
    const bool use_mixed = o.prec == QM_MIXED;
    const size_t oP32 = take(use_mixed ? big32 * nb : 0), oH32 = take(use_mixed ? big32 * nb : 0),
                 oB32 = take(use_mixed ? big32 * std::max(nproj, 1) : 0),
                 oBtc = take(use_mixed && nproj > 0 ? nonlocal_tc_beta_bytes(nproj, nb, npw) : 0);
    const size_t sub_bytes = use_mixed ? subspace_bf16x3_bytes(nvx, nb) : 0;
    const size_t oSub = take(sub_bytes);
    const size_t sq = (size_t)nsq * nsq * sizeof(double2);
    const size_t oHs = take(sq), oG = take(sq), oA = take(sq), oZ = take(sq), oCs = take(sq);
    const bool thick = o.plain_restart == 0;
    const size_t sqb = (size_t)nsq * nb * sizeof(double2);
    const size_t oCp = take(thick ? sqb : 0), oCT = take(thick ? sqb : 0), oPT = take(thick ? sqb : 0),
                 oQT = take(thick ? sqb : 0), oY = take(thick ? big * nb : 0), oHY = take(thick ? big * nb : 0);
    const size_t oPart = take(gemm_cn_partial_bytes(false));
    const size_t oEval = take(sizeof(double) * nsq), oEps = take(sizeof(double) * nsq),
                 oRn = take(sizeof(double) * nsq), oTk = take(sizeof(double) * nsq),
                 oSel = take(sizeof(int) * nsq), oRank = take(sizeof(int) * nsq), oInfo = take(sizeof(int) * 4),
                 oHeev = take(heev_work_bytes(nsq, nsq));
    const size_t oHd = take(o.precond == 1 ? sizeof(double) * npw : 0),
                 oVp = take(o.precond == 1 ? sizeof(double) * kVmeanBlocks : 0);
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
    if (use_mixed) {
        run.psi32 = (float2*)(base + oP32);
        run.hpsi32 = (float2*)(base + oH32);
        run.beta32 = (float2*)(base + oB32);
        if (nproj > 0 && (st = convert_rows((const double2*)beta, ld_beta, run.beta32, ld, nproj, npw, s))) return st;
        if (nproj > 0) {
            run.beta_tc = base + oBtc;
            if ((st = nonlocal_tc_prepare(nproj, nb, npw, run.beta32, ld, run.beta_tc, s))) return st;
        }
        run.mixed = true;
        run.tc = true;
        run.ds = o.fp64_exact == 0;
        run.ortho64 = o.mixed_ortho == 1;
        run.sub = base + oSub;
        run.sub_bytes = sub_bytes;
    }
    w.Hs = (double2*)(base + oHs);
    w.G = (double2*)(base + oG);
    w.A = (double2*)(base + oA);
    w.Z = (double2*)(base + oZ);
    w.Cs = (double2*)(base + oCs);
    w.Part = (double2*)(base + oPart);
    if (thick) {
        w.Cp = (double2*)(base + oCp);
        w.CT = (double2*)(base + oCT);
        w.PT = (double2*)(base + oPT);
        w.QT = (double2*)(base + oQT);
        w.Y = (double2*)(base + oY);
        w.HY = (double2*)(base + oHY);
    }
    w.eval = (double*)(base + oEval);
    w.eps = (double*)(base + oEps);
    w.rn2 = (double*)(base + oRn);
    w.tk = (double*)(base + oTk);
    w.sel = (int*)(base + oSel);
    w.rank = (int*)(base + oRank);
    w.info = (int*)(base + oInfo);
    w.heev = base + oHeev;
    w.hdiag = (double*)(base + oHd);
    w.vpart = (double*)(base + oVp);
    run.tc_err = w.info + 3;
    if (use_mixed && (st = cuda_check(cudaMemsetAsync(run.tc_err, 0, sizeof(int), s), "reset error word"))) return st;
    const double* kin = g->k[ik].kin;

    // initial block: psi -> rows of Tmp (dense ld), orthonormalised into V
    if ((st = cuda_check(cudaMemcpy2DAsync(w.Tmp, big, psi_inout, (size_t)ld_psi * sizeof(double2),
                                           (size_t)npw * sizeof(double2), nb, cudaMemcpyDeviceToDevice, s),
                         "copy psi")))
        return st;
    int kept = 0;
    if ((st = run.cholqr(w.Tmp, nb, w.V, &kept))) return st;
    if (kept < nb) return fail(QM_ERR_NUMERIC, "qm_davidson: initial psi block is rank deficient");
    if ((st = run.hpsi(w.V, w.HV, nb))) return st;
    int m = nb, m0 = 0;
    // previous Ritz coefficients: after a (re)start the Ritz vectors are the first nb basis rows
    auto reset_prev = [&]() -> qm_status {
        if (!thick) return QM_OK;
        ProfScope pf(PF_OTHER, s);
        k_set_identity<<<grid_for((long)nsq * nb), 256, 0, s>>>(w.Cp, nb, nsq, nb);
        return cuda_check(cudaGetLastError(), "k_set_identity launch");
    };
    if ((st = reset_prev())) return st;
    bool use_mlp = o.precond == 1;
    const double stall = o.precond_stall > 0.0 ? o.precond_stall : 0.8;
    int fallback_it = 0;
    std::vector<double> hist_all;
    int* mlp_err = w.info + 2;
    if (use_mlp && (st = cuda_check(cudaMemsetAsync(mlp_err, 0, sizeof(int), s), "reset error word"))) return st;
    // the network's features need the Hamiltonian's diagonal (once per solve)
    if (use_mlp && (st = hamiltonian_diag(g, ik, vloc_r, nproj, (const double2*)beta, ld_beta, D, w.hdiag, w.vpart, s)))
        return st;
    std::vector<double> rn2(nb), eps(nb);
    int it = 0, it_mixed = 0, restarts = 0;
    long long prev_kept = 0;
    std::vector<double> hist_mixed;
    bool converged = false;
    double max_res = 0.0;
    // Anchored FP64 phase of the precision form.  After every restart the first nb basis rows
    // are the Ritz vectors X_a, exact in FP64 (so are H X_a), with H_sub block diag(eps_a) and
    // residuals R_a = H X_a - X_a eps_a (kept in Ra).  Every later direction d is orthogonal
    // to X_a to FP64 round-off (exact second orthogonalisation pass), hence
    //   <X_a | H d> = <H X_a | d> = <R_a | d>,
    // a product of small vectors whose FP32 relative accuracy suffices: the new columns of H_sub
    // come from tensor-core products (the couplings among later directions enter the Ritz
    // vectors only at second order).  The Ritz vectors X = X_a c_a + D c_d and H X take the
    // anchor part in FP64 (K = nb) and the small remainder D c_d on the tensor cores; before a
    // restart, at convergence and at exit they are recomputed entirely in FP64, so anchors and
    // reported residuals stay exact.  Used only with buffer bands (nconv < nb): without them the
    // top band may rotate by O(1) into states outside the block, and its large coefficients on
    // later directions would carry the FP32-accuracy errors into its residual.  An anchored
    // phase that stops making progress hands over to plain FP64 (deanchor below).
    double2* Ra = w.Tmp;  // free after the initial orthonormalisation
    bool need_anchor = false, split_ritz = false;
    int it_anchor = 0, it_halved = 0;
    double anchor_best = 0.0;
    std::vector<int> unc;
    bool all_conv = true;
    auto ritz = [&](bool exact) -> qm_status {
        qm_status st2;
        split_ritz = run.anchored && !exact && m > nb;
        if (split_ritz) {
            const double2* Cd = w.Cs + (size_t)nb * nb;
            if ((st2 = run.tn64(nb, nb, w.Cs, nb, w.V, w.X, false)) ||
                (st2 = run.tn_tc(nb, m - nb, Cd, nb, w.V + (size_t)nb * ld, w.X, true)) ||
                (st2 = run.tn64(nb, nb, w.Cs, nb, w.HV, w.HX, false)) ||
                (st2 = run.tn_tc(nb, m - nb, Cd, nb, w.HV + (size_t)nb * ld, w.HX, true)))
                return st2;
        } else if ((st2 = run.gemm_tn(nb, m, w.Cs, nb, w.V, w.X, false)) ||
                   (st2 = run.gemm_tn(nb, m, w.Cs, nb, w.HV, w.HX, false))) {
            return st2;
        }
        {
            ProfScope pf(PF_OTHER, s);
            k_residual<<<nb, 256, 0, s>>>(w.X, w.HX, ld, npw, w.eps, kin, w.R, w.rn2, w.tk);
        }
        if ((st2 = cuda_check(cudaMemcpyAsync(rn2.data(), w.rn2, sizeof(double) * nb, cudaMemcpyDeviceToHost, s),
                              "D2H residual norms")) ||
            (st2 = cuda_check(cudaMemcpyAsync(eps.data(), w.eps, sizeof(double) * nb, cudaMemcpyDeviceToHost, s),
                              "D2H Ritz values")) ||
            (st2 = cuda_check(cudaStreamSynchronize(s), "stream sync")))
            return st2;
        for (int n = 0; n < nb; ++n)
            if (!std::isfinite(eps[n])) return fail(QM_ERR_NUMERIC, "qm_davidson: non-finite Ritz value");
        unc.clear();
        max_res = 0.0;
        all_conv = true;
        for (int n = 0; n < nb; ++n) {
            double r = std::sqrt(rn2[n]);
            if (!std::isfinite(r)) return fail(QM_ERR_NUMERIC, "qm_davidson: non-finite residual");
            if (n < o.nconv) {
                max_res = std::max(max_res, r);
                all_conv = all_conv && r <= o.tol;
            }
            if (r > o.tol) unc.push_back(n);
        }
        return QM_OK;
    };
    for (it = 1; it <= o.max_iter; ++it) {
        // new columns of H_sub
        if (run.anchored && m0 >= nb) {
            if ((st = run.cn_tc(nb, m - m0, Ra, w.V + (size_t)m0 * ld, w.Hs + m0, nsq)) ||
                (st = run.cn_tc(m - nb, m - m0, w.V + (size_t)nb * ld, w.HV + (size_t)m0 * ld,
                                w.Hs + (size_t)nb * nsq + m0, nsq)))
                return st;
        } else if ((st = run.gemm_cn(m, m - m0, w.V, w.HV + (size_t)m0 * ld, w.Hs + m0, nsq))) {
            return st;
        }
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
        if ((st = ritz(false))) return st;
        // the anchored products assume that the bands which must converge take only small
        // coefficients on the later directions; if the best residual of the anchored phase has
        // not halved for 12 steps (robust to oscillation), or after 60 anchored steps, the rest
        // of the solve runs in plain FP64 from an exact restart
        bool deanchor = false;
        if (run.anchored) {
            if (max_res < 0.5 * anchor_best) {
                anchor_best = max_res;
                it_halved = it;
            }
            deanchor = max_res > o.tol && (it - it_halved > 12 || it - it_anchor > 60);
        }
        if (split_ritz && (all_conv || deanchor || it == o.max_iter || m + (int)unc.size() > nvx) &&
            (st = ritz(true)))
            return st;
        if (o.history && it - 1 < o.max_iter) o.history[it - 1] = max_res;
        hist_all.push_back(max_res);
        // the learned correction hands over to TPA when the residual stalls
        if (use_mlp && stall < 1.0 && hist_all.size() > 4 && max_res > stall * hist_all[hist_all.size() - 5]) {
            use_mlp = false;
            fallback_it = it;
        }
        if (run.mixed) hist_mixed.push_back(max_res);
        // FP32 round-off can only stall the residual well below 1e-3: there, no halving over the
        // last 10 FP32 iterations hands over to FP64 early
        bool stalled = false;
        if (run.mixed && max_res < 1e-3 && hist_mixed.size() > 10)
            stalled = max_res > 0.5 * hist_mixed[hist_mixed.size() - 11];
        if (run.mixed && (max_res <= std::max(o.mixed_switch, o.tol) || stalled)) {
            // FP64 refinement: re-orthonormalise the Ritz vectors in FP64, apply H to them in
            // FP64, and continue the iterations in FP64 from this basis (anchored after the
            // first Rayleigh-Ritz step)
            run.mixed = false;
            run.anchored = run.tc && o.nconv < nb;
            need_anchor = run.anchored;
            it_anchor = it_halved = it;
            anchor_best = max_res;
            it_mixed = it;
            if ((st = run.cholqr(w.X, nb, w.V, &kept))) return st;
            if (kept < nb) return fail(QM_ERR_NUMERIC, "qm_davidson: Ritz vectors lost rank at the FP64 switch");
            if ((st = run.hpsi(w.V, w.HV, nb))) return st;
            if ((st = reset_prev())) return st;
            m0 = 0;
            m = nb;
            continue;
        }
        if (all_conv) {
            converged = true;
            break;
        }
        if (it == o.max_iter) break;
        const int nu = (int)unc.size();
        if ((st = cuda_check(cudaMemcpyAsync(w.sel, unc.data(), sizeof(int) * nu, cudaMemcpyHostToDevice, s),
                             "H2D unconverged bands")))
            return st;
        if (use_mlp) {
            if ((st = mlp_precond_apply(o.mlp, w.R, ld, npw, w.sel, nu, w.tk, w.eps, w.hdiag, kin, w.Dl, ld, mlp_err, s)))
                return st;
        } else {
            ProfScope pf(PF_OTHER, s);
            k_tpa<<<dim3((npw + 255) / 256 < 64 ? (npw + 255) / 256 : 64, nu), 256, 0, s>>>(w.R, ld, npw, w.sel, w.tk,
                                                                                            kin, w.Dl, ld);
        }
        bool restarted = false;
        if (m + nu > nvx || need_anchor || deanchor) {  // restart from the Ritz vectors (exact here)
            // thick restart: the previous Ritz vectors' new directions ride along (not on the
            // restarts that open or close the anchored phase, whose basis must be the Ritz vectors)
            int kp = 0;
            if (thick && !need_anchor && !deanchor && (st = run.prev_directions(m, nu, nvx - nb - nu, nsq, &kp)))
                return st;
            if ((st = cuda_check(cudaMemcpyAsync(w.V, w.X, big * nb, cudaMemcpyDeviceToDevice, s), "restart copy")) ||
                (st = cuda_check(cudaMemcpyAsync(w.HV, w.HX, big * nb, cudaMemcpyDeviceToDevice, s), "restart copy")))
                return st;
            if (kp > 0 &&
                ((st = cuda_check(cudaMemcpyAsync(w.V + (size_t)nb * ld, w.Y, big * kp, cudaMemcpyDeviceToDevice, s),
                                  "restart copy")) ||
                 (st = cuda_check(cudaMemcpyAsync(w.HV + (size_t)nb * ld, w.HY, big * kp, cudaMemcpyDeviceToDevice, s),
                                  "restart copy"))))
                return st;
            if (run.anchored &&
                (st = cuda_check(cudaMemcpyAsync(Ra, w.R, big * nb, cudaMemcpyDeviceToDevice, s), "restart copy")))
                return st;
            {
                ProfScope pf(PF_OTHER, s);
                k_set_diag<<<grid_for((long)nb * nb), 256, 0, s>>>(w.Hs, nsq, nb, w.eps);
            }
            m = nb + kp;
            restarts += 1;
            prev_kept += kp;
            need_anchor = false;
            if (deanchor) run.anchored = false;
            restarted = true;
            if ((st = reset_prev())) return st;
        } else if (thick) {
            // this step's Ritz coefficients become the previous ones (rows added later are zero)
            if ((st = cuda_check(cudaMemcpyAsync(w.Cp, w.Cs, sizeof(double2) * (size_t)m * nb, cudaMemcpyDeviceToDevice, s),
                                 "copy Ritz coefficients")) ||
                (st = cuda_check(cudaMemsetAsync(w.Cp + (size_t)m * nb, 0, sizeof(double2) * (size_t)(nsq - m) * nb, s),
                                 "zero Ritz coefficients")))
                return st;
        }
        // orthogonalise the corrections against the basis and orthonormalise them
        if ((st = run.expand(m, nu, w.V + (size_t)m * ld, &kept))) return st;
        if (kept == 0) break;  // no new directions: stagnation
        if ((st = run.hpsi(w.V + (size_t)m * ld, w.HV + (size_t)m * ld, kept))) return st;
        m0 = restarted ? nb : m;  // after a thick restart the kept directions' columns of H_sub are new too
        m += kept;
    }
    if (split_ritz && (st = ritz(true))) return st;  // exact Ritz vectors for the output
    // outputs: Ritz vectors and values
    if ((st = cuda_check(cudaMemcpy2DAsync(psi_inout, (size_t)ld_psi * sizeof(double2), w.X, big,
                                           (size_t)npw * sizeof(double2), nb, cudaMemcpyDeviceToDevice, s),
                         "copy psi out")) ||
        (st = cuda_check(cudaStreamSynchronize(s), "stream sync")))
        return st;
    for (int n = 0; n < nb; ++n) eig_out[n] = eps[n];
    if (o.precond == 1) {
        int e = 0;
        if ((st = cuda_check(cudaMemcpy(&e, mlp_err, sizeof(int), cudaMemcpyDeviceToHost), "D2H error word")))
            return st;
        if (e) return fail(QM_ERR_TIMEOUT, "qm_davidson: a bounded tensor-core wait of the learned preconditioner expired");
    }
    if (use_mixed) {
        int e = 0;
        if ((st = cuda_check(cudaMemcpy(&e, run.tc_err, sizeof(int), cudaMemcpyDeviceToHost), "D2H error word")))
            return st;
        if (e) return fail(QM_ERR_TIMEOUT, "qm_davidson: a bounded tensor-core wait of a subspace product expired");
        if ((st = qm_hpsi_check(g, stream))) return st;  // the tensor-core nonlocal part of its H psi
    }
    if (stats) {
        stats->iterations = it > o.max_iter ? o.max_iter : it;
        stats->band_applies = run.applies;
        stats->max_residual = max_res;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->converged = converged ? 1 : 0;
        stats->iterations_mixed = run.mixed ? stats->iterations : it_mixed;
        stats->band_applies_mixed = run.applies_mixed;
        stats->precond_fallback = fallback_it;
        stats->restarts = restarts;
        stats->restart_kept = prev_kept;
    }
    if (!converged) return fail(QM_ERR_NOT_CONVERGED, "qm_davidson: max_iter reached before tol");
    return QM_OK;
}

// Independent Davidson problems (k-points, cells) run concurrently: worker threads take jobs
// in order, each on its own CUDA stream with its own workspace (a clone of the job's gspace
// sharing its device tables), so one job's host synchronisations, small eigensolves and
// latency-bound kernels overlap with the others' work on the GPU.
extern "C" qm_status qm_davidson_batched(int njobs, qm_davidson_job* jobs, const qm_davidson_opts* opts,
                                         int max_concurrent, void* stream) {
    clear_error();
    if (njobs < 1 || !jobs) return fail(QM_ERR_ARG, "qm_davidson_batched: no jobs");
    if (max_concurrent < 0) return fail(QM_ERR_ARG, "qm_davidson_batched: max_concurrent < 0");
    for (int i = 0; i < njobs; ++i) {
        if (!jobs[i].g || !jobs[i].psi_inout || !jobs[i].eig_out)
            return fail(QM_ERR_ARG, "qm_davidson_batched: job " + std::to_string(i) + " lacks g, psi or eig_out");
        jobs[i].status = QM_OK;
    }
    qm_status st;
    int dev = 0;
    if ((st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice"))) return st;
    for (int i = 0; i < njobs; ++i)
        if ((st = ensure_device(jobs[i].g))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ready = nullptr;
    if ((st = cuda_check(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming), "event")) ||
        (st = cuda_check(cudaEventRecord(ready, s), "event record")))
        return st;
    const int nw = std::min(njobs, max_concurrent > 0 ? max_concurrent : njobs);
    std::atomic<int> next{0};
    std::mutex mu;
    std::string first_msg;
    std::vector<cudaStream_t> wstreams(nw, nullptr);
    auto worker = [&](int w) {
        cudaSetDevice(dev);
        std::map<qm_gspace, qm_gspace> clones;
        cudaStream_t ws = nullptr;
        qm_status wst = cuda_check(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking), "worker stream");
        if (!wst) wst = cuda_check(cudaStreamWaitEvent(ws, ready, 0), "worker wait");
        wstreams[w] = ws;
        for (int i; (i = next.fetch_add(1)) < njobs;) {
            qm_davidson_job& j = jobs[i];
            qm_status r = wst;
            qm_gspace c = nullptr;
            if (!r) {
                auto it = clones.find(j.g);
                if (it == clones.end()) {
                    r = gspace_clone(j.g, &c);
                    if (!r) clones[j.g] = c;
                } else {
                    c = it->second;
                }
            }
            if (!r) {
                qm_davidson_opts o{};
                if (opts) o = *opts;
                o.history = j.history;
                r = qm_davidson(c, j.ik, j.nb, j.psi_inout, j.ld_psi, j.vloc_r, j.nproj, j.beta, j.ld_beta, j.D, &o,
                                j.eig_out, j.stats, ws);
            }
            j.status = r;
            if (r && r != QM_ERR_NOT_CONVERGED) {
                std::lock_guard<std::mutex> lk(mu);
                if (first_msg.empty()) first_msg = "job " + std::to_string(i) + ": " + qm_last_error();
            }
        }
        for (auto& kv : clones) qm_gspace_destroy(kv.second);  // synchronises the device
    };
    std::vector<std::thread> threads;
    for (int w = 0; w < nw; ++w) threads.emplace_back(worker, w);
    for (auto& t : threads) t.join();
    // order the caller's stream after every job
    for (int w = 0; w < nw; ++w) {
        if (!wstreams[w]) continue;
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(e, wstreams[w]);
            cudaStreamWaitEvent(s, e, 0);
            cudaEventDestroy(e);
        }
        cudaStreamDestroy(wstreams[w]);
    }
    cudaEventDestroy(ready);
    qm_status out = QM_OK;
    for (int i = 0; i < njobs; ++i)
        if (jobs[i].status && jobs[i].status != QM_ERR_NOT_CONVERGED) {
            out = jobs[i].status;
            break;
        }
    if (out) return fail(out, "qm_davidson_batched: " + first_msg);
    for (int i = 0; i < njobs; ++i)
        if (jobs[i].status == QM_ERR_NOT_CONVERGED)
            return fail(QM_ERR_NOT_CONVERGED, "qm_davidson_batched: job " + std::to_string(i) + " did not converge");
    return QM_OK;
}

// The residual and correction steps of one Davidson iteration on their own (the kernels the
// loop above launches): r_n = HX_n - eps_n X_n with ||r_n||^2 and T_n, then
// delta_n = K r_n with the TPA factor or the learned network.
extern "C" qm_status qm_precond_apply(qm_gspace g, int ik, int n, const void* X, const void* HX, int ld,
                                      const double* eps, int precond, const float* mlp, const double* hdiag, void* R,
                                      void* delta, double* rnorm2, double* tkin, void* stream) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_precond_apply: NULL gspace");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_precond_apply: ik out of range");
    if (n < 0 || n > 65535) return fail(QM_ERR_ARG, "qm_precond_apply: need 0 <= n <= 65535");
    if (precond != 0 && precond != 1) return fail(QM_ERR_ARG, "qm_precond_apply: unknown preconditioner");
    if (precond == 1 && (!mlp || !hdiag))
        return fail(QM_ERR_ARG, "qm_precond_apply: learned preconditioner without parameters or H diagonal");
    if (n == 0) return QM_OK;
    const int npw = g->k[ik].npw;
    if (!X || !HX || !eps || !R || !delta || !rnorm2 || !tkin)
        return fail(QM_ERR_ARG, "qm_precond_apply: NULL X, HX, eps, R, delta, rnorm2 or tkin");
    if (ld < npw) return fail(QM_ERR_ARG, "qm_precond_apply: ld < npw");
    if (((uintptr_t)X | (uintptr_t)HX | (uintptr_t)R | (uintptr_t)delta) % 16)
        return fail(QM_ERR_ARG, "qm_precond_apply: X, HX, R, delta not 16-byte aligned");
    qm_status st = ensure_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const double* kin = g->k[ik].kin;
    double2* r = (double2*)R;
    double2* d = (double2*)delta;
    {
        ProfScope pf(PF_OTHER, s);
        k_residual<<<n, 256, 0, s>>>((const double2*)X, (const double2*)HX, ld, npw, eps, kin, r, rnorm2, tkin);
    }
    if ((st = cuda_check(cudaGetLastError(), "k_residual launch"))) return st;
    if (precond == 0) {
        ProfScope pf(PF_OTHER, s);
        k_tpa<<<dim3(std::min(64, (npw + 255) / 256), n), 256, 0, s>>>(r, ld, npw, nullptr, tkin, kin, d, ld);
        return cuda_check(cudaGetLastError(), "k_tpa launch");
    }
    // the network's bounded tensor-core waits report through the handle's sticky error word
    if ((st = ensure_workspace(g, kWsHeader, s))) return st;
    if ((st = mlp_precond_apply(mlp, r, ld, npw, nullptr, n, tkin, eps, hdiag, kin, d, ld, (int*)g->ws.ptr, s)))
        return st;
    return qm_hpsi_check(g, stream);
}

extern "C" qm_status qm_hamiltonian_diag(qm_gspace g, int ik, const double* vloc_r, int nproj, const void* beta,
                                         int ld_beta, const double* D, double* hdiag, void* stream) {
    clear_error();
    if (!g) return fail(QM_ERR_ARG, "qm_hamiltonian_diag: NULL gspace");
    if (ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_hamiltonian_diag: ik out of range");
    if (nproj < 0 || !vloc_r || !hdiag || (nproj > 0 && (!beta || !D)))
        return fail(QM_ERR_ARG, "qm_hamiltonian_diag: NULL argument or negative nproj");
    const int npw = g->k[ik].npw;
    if (nproj > 0 && ld_beta < npw) return fail(QM_ERR_ARG, "qm_hamiltonian_diag: ld_beta < npw");
    if (nproj > 0 && (uintptr_t)beta % 16) return fail(QM_ERR_ARG, "qm_hamiltonian_diag: beta not 16-byte aligned");
    qm_status st = ensure_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the partial sums of V live in the handle's workspace, after its error-word header
    if ((st = ensure_workspace(g, kWsHeader + sizeof(double) * kVmeanBlocks, s))) return st;
    return hamiltonian_diag(g, ik, vloc_r, nproj, (const double2*)beta, ld_beta, D, hdiag,
                            (double*)((char*)g->ws.ptr + kWsHeader), s);
}

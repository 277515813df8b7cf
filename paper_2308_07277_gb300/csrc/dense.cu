// Small dense FP64 kernels of the Davidson subspace step: a parallel cyclic Jacobi
// eigensolver for complex Hermitian matrices (the Rayleigh-Ritz eigenproblem and the Gram
// matrices of the orthonormalisation), and the elementwise residual / preconditioner
// kernels.  FP64 throughout: the subspace eigensolve, orthonormalisation, residual norms
// and band energies stay in double precision in every form of the method.
//
// Jacobi: two-sided cyclic Jacobi with the round-robin ("chess tournament") ordering, so
// the n/2 rotations of one round touch disjoint index pairs and apply in parallel.  One
// cooperative launch runs all sweeps; grid-wide barriers separate the rotation and the
// update phase of each round.  Each complex 2x2 rotation is R = diag(1, w) J with
// w = conj(b)/|b| (makes the pivot real) and J the real symmetric Schur rotation
// (Golub & Van Loan, Matrix Computations, Sec. 8.5).
#include <cooperative_groups.h>

#include <algorithm>

#include "qm_internal.h"

namespace cg = cooperative_groups;

namespace qm {

namespace {

__device__ __forceinline__ double2 cm(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmc(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 sc(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ void rr_pair(int n, int r, int k, int& p, int& q) {
    const int m1 = n - 1;
    p = (k == 0) ? 0 : (k + r - 1) % m1 + 1;
    q = (n - 1 - k + r - 1) % m1 + 1;
}

struct Rot {
    double c, s;
    double2 w;
};

__global__ void __launch_bounds__(256)
k_jacobi(double2* __restrict__ A, int lda, double2* __restrict__ Z, int ldz, int n, int m, int max_sweeps, double tol2,
         Rot* __restrict__ rot, double* __restrict__ red, int* __restrict__ info) {
    cg::grid_group grid = cg::this_grid();
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    const int h = n / 2;
    __shared__ double sred[256];
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // convergence test: off-diagonal vs total Frobenius norm
        double off = 0.0, tot = 0.0;
        for (long e = tid; e < (long)m * m; e += nth) {   // the padding index is excluded
            int i = (int)(e / m), j = (int)(e % m);
            double2 v = A[(size_t)i * lda + j];
            double a2 = v.x * v.x + v.y * v.y;
            tot += a2;
            if (i != j) off += a2;
        }
        for (int pass = 0; pass < 2; ++pass) {
            double x = pass == 0 ? off : tot;
            sred[threadIdx.x] = x;
            __syncthreads();
            for (int st = blockDim.x / 2; st > 0; st >>= 1) {
                if (threadIdx.x < st) sred[threadIdx.x] += sred[threadIdx.x + st];
                __syncthreads();
            }
            if (threadIdx.x == 0) red[2 * blockIdx.x + pass] = sred[0];
            __syncthreads();
        }
        grid.sync();
        double o = 0.0, t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            o += red[2 * b];
            t += red[2 * b + 1];
        }
        grid.sync();  // everyone has read red[] before it is reused
        if (o <= tol2 * t || !(o == o)) break;  // converged, or NaN (reported through the eigenvalues)
        for (int r = 0; r < n - 1; ++r) {
            // phase 1: rotation of every pair of this round
            for (int k = tid; k < h; k += nth) {
                int p, q;
                rr_pair(n, r, k, p, q);
                const double a = A[(size_t)p * lda + p].x, d = A[(size_t)q * lda + q].x;
                const double2 b = A[(size_t)p * lda + q];
                const double ab = hypot(b.x, b.y);
                Rot R;
                if (ab < 1e-300) {
                    R.c = 1.0;
                    R.s = 0.0;
                    R.w = make_double2(1.0, 0.0);
                } else {
                    const double tau = (d - a) / (2.0 * ab);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    R.c = 1.0 / sqrt(1.0 + t * t);
                    R.s = t * R.c;
                    R.w = make_double2(b.x / ab, -b.y / ab);  // conj(b)/|b|
                }
                rot[k] = R;
            }
            grid.sync();
            // phase 2: A <- R^H A R on every 2x2 block, Z <- Z R on every row
            const long nblk = (long)h * h;
            const long total = nblk + (long)n * h;
            for (long e = tid; e < total; e += nth) {
                if (e < nblk) {
                    const int ki = (int)(e / h), kj = (int)(e % h);
                    int pi, qi, pj, qj;
                    rr_pair(n, r, ki, pi, qi);
                    rr_pair(n, r, kj, pj, qj);
                    const Rot Ri = rot[ki], Rj = rot[kj];
                    double2 x00 = A[(size_t)pi * lda + pj], x01 = A[(size_t)pi * lda + qj];
                    double2 x10 = A[(size_t)qi * lda + pj], x11 = A[(size_t)qi * lda + qj];
                    // Y = X R_j,  R_j = [[c, s], [-s w, c w]]
                    const double2 sw = sc(Rj.s, Rj.w), cw = sc(Rj.c, Rj.w);
                    double2 y00 = csub(sc(Rj.c, x00), cm(x01, sw)), y01 = cadd(sc(Rj.s, x00), cm(x01, cw));
                    double2 y10 = csub(sc(Rj.c, x10), cm(x11, sw)), y11 = cadd(sc(Rj.s, x10), cm(x11, cw));
                    // X' = R_i^H Y,  R_i^H = [[c, -s conj(w)], [s, c conj(w)]]
                    const double2 swi = sc(Ri.s, Ri.w), cwi = sc(Ri.c, Ri.w);
                    double2 z00 = csub(sc(Ri.c, y00), cmc(y10, swi)), z01 = csub(sc(Ri.c, y01), cmc(y11, swi));
                    double2 z10 = cadd(sc(Ri.s, y00), cmc(y10, cwi)), z11 = cadd(sc(Ri.s, y01), cmc(y11, cwi));
                    if (ki == kj) {  // the pivot block becomes exactly diagonal and real
                        z00.y = 0.0;
                        z11.y = 0.0;
                        z01 = make_double2(0.0, 0.0);
                        z10 = make_double2(0.0, 0.0);
                    }
                    A[(size_t)pi * lda + pj] = z00;
                    A[(size_t)pi * lda + qj] = z01;
                    A[(size_t)qi * lda + pj] = z10;
                    A[(size_t)qi * lda + qj] = z11;
                } else {
                    const long f = e - nblk;
                    const int row = (int)(f / h), kj = (int)(f % h);
                    int pj, qj;
                    rr_pair(n, r, kj, pj, qj);
                    const Rot Rj = rot[kj];
                    const double2 sw = sc(Rj.s, Rj.w), cw = sc(Rj.c, Rj.w);
                    double2 u = Z[(size_t)row * ldz + pj], v = Z[(size_t)row * ldz + qj];
                    Z[(size_t)row * ldz + pj] = csub(sc(Rj.c, u), cm(v, sw));
                    Z[(size_t)row * ldz + qj] = cadd(sc(Rj.s, u), cm(v, cw));
                }
            }
            grid.sync();
        }
    }
    if (tid == 0) info[0] = sweep;
}

__global__ void k_prepare_jacobi(const double2* __restrict__ H, int ldh, int m, double2* __restrict__ A, int lda,
                                 double2* __restrict__ Z, int ldz, int n, double pad_diag) {
    const long total = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        int i = (int)(e / n), j = (int)(e % n);
        double2 v = make_double2(0.0, 0.0);
        if (i < m && j < m) {
            // Hermitian part of the input (the stored matrix is Hermitian up to round-off)
            double2 a = H[(size_t)i * ldh + j], b = H[(size_t)j * ldh + i];
            v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        } else if (i == j) {
            v = make_double2(pad_diag, 0.0);
        }
        A[(size_t)i * lda + j] = v;
        Z[(size_t)i * ldz + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
}

__global__ void k_diag(const double2* __restrict__ A, int lda, int n, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = A[(size_t)i * lda + i].x;
}

}  // namespace

// Eigen-decomposition of the Hermitian m x m matrix H (ldh): eigenvalues into evals_dev
// (unsorted, length m), eigenvectors as the columns of Z (n x n, n = m rounded up to even;
// only the leading m x m block is meaningful).  A, Z: n x n workspaces; rot: n/2 entries;
// red: 2 * (max grid) doubles; info: 1 int (sweeps used).
qm_status jacobi_eigh(const double2* H, int ldh, int m, double2* A, double2* Z, void* rot, double* red, int* info,
                      double* evals_dev, cudaStream_t s) {
    if (m <= 0) return QM_OK;
    const int n = m + (m & 1);
    {
        long total = (long)n * n;
        int blocks = (int)std::min<long>((total + 255) / 256, 152 * 8);
        ProfScope pf(PF_OTHER, s);
        k_prepare_jacobi<<<blocks, 256, 0, s>>>(H, ldh, m, A, n, Z, n, n, 1e300);
    }
    int dev = 0, sms = 152, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jacobi, 256, 0);
    const long work = (long)(n / 2) * (n / 2) + (long)n * (n / 2);
    int blocks = (int)std::max<long>(1, std::min<long>((long)std::max(1, occ) * sms, (work + 1023) / 1024));
    blocks = std::min(blocks, kJacobiMaxBlocks);
    int max_sweeps = 40;
    double tol2 = 1e-30;
    int ld = n;
    Rot* rp = (Rot*)rot;
    int mm = m;
    void* args[] = {(void*)&A, (void*)&ld, (void*)&Z, (void*)&ld, (void*)&n, (void*)&mm, (void*)&max_sweeps, (void*)&tol2,
                    (void*)&rp, (void*)&red, (void*)&info};
    {
        ProfScope pf(PF_JACOBI, s);
        qm_status st = cuda_check(cudaLaunchCooperativeKernel((void*)k_jacobi, dim3(blocks), dim3(256), args, 0, s),
                                  "k_jacobi cooperative launch");
        if (st) return st;
    }
    ProfScope pf(PF_OTHER, s);
    k_diag<<<(m + 255) / 256, 256, 0, s>>>(A, n, m, evals_dev);
    return cuda_check(cudaGetLastError(), "k_diag launch");
}

size_t jacobi_rot_bytes(int m) { return sizeof(Rot) * (size_t)((m + 1) / 2 + 1); }

}  // namespace qm

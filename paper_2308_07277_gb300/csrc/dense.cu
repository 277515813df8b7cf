// Small dense FP64 kernels of the Davidson orthonormalisation step: Cholesky factorisation
// of the Gram matrix of a block of vectors, with dropping of near-dependent directions, and
// the triangular inverse that turns it into the transform of Cholesky-QR (the block is
// replaced by Y' = L^-H-weighted combinations of its rows, orthonormal and spanning the same
// space minus its near-null directions; Golub & Van Loan, Matrix Computations, Sec. 4.2, 5.2).
#include <algorithm>

#include "qm_internal.h"

namespace qm {
namespace {

// In-place lower Cholesky S = L L^H of an nd x nd Hermitian positive semi-definite matrix in
// one CTA (right-looking).  A pivot below drop_rel * S_jj(original) marks vector j as
// linearly dependent on the previous ones: its row and column are zeroed and it is skipped
// (Cholesky with dropping == Gram-Schmidt that discards near-null directions).
__global__ void __launch_bounds__(1024)
k_chol_drop(double2* __restrict__ S, int lds, int nd, double drop_rel, int* __restrict__ keep) {
    const int tid = threadIdx.x, bs = blockDim.x;
    extern __shared__ double sdiag[];  // original diagonal
    for (int i = tid; i < nd; i += bs) sdiag[i] = S[(size_t)i * lds + i].x;
    __syncthreads();
    for (int j = 0; j < nd; ++j) {
        const double piv = S[(size_t)j * lds + j].x;
        const bool ok = piv > drop_rel * sdiag[j] && piv > 0.0 && isfinite(piv);
        __syncthreads();
        if (!ok) {
            for (int i = j + tid; i < nd; i += bs) {
                S[(size_t)i * lds + j] = make_double2(0.0, 0.0);
                S[(size_t)j * lds + i] = make_double2(0.0, 0.0);
            }
            if (tid == 0) keep[j] = 0;
            __syncthreads();
            continue;
        }
        const double l = sqrt(piv), il = 1.0 / l;
        for (int i = j + 1 + tid; i < nd; i += bs) {
            double2 v = S[(size_t)i * lds + j];
            S[(size_t)i * lds + j] = make_double2(v.x * il, v.y * il);
        }
        if (tid == 0) {
            S[(size_t)j * lds + j] = make_double2(l, 0.0);
            keep[j] = 1;
        }
        __syncthreads();
        // trailing update of the lower triangle: S[i][k] -= L[i][j] conj(L[k][j]), j < k <= i;
        // one warp per row i, lanes over k
        const int lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
        for (int i = j + 1 + warp; i < nd; i += nwarp) {
            const double2 a = S[(size_t)i * lds + j];
            for (int k = j + 1 + lane; k <= i; k += 32) {
                const double2 b = S[(size_t)k * lds + j];
                double2 v = S[(size_t)i * lds + k];
                v.x -= a.x * b.x + a.y * b.y;
                v.y -= a.y * b.x - a.x * b.y;
                S[(size_t)i * lds + k] = v;
            }
        }
        __syncthreads();
    }
}

// Row c of the orthonormalising transform.  With S = L L^H (kept indices only) the new rows
// are z_k = sum_i conj((L^-1)[k][i]) y_i, i.e. W[i][k'] = conj((L^-1)[k][i]) for gemm_tn
// (k' = rank of k among the kept).  CTA c solves L x = e_c by forward substitution (a
// warp-parallel dot product per row) -- x is column c of L^-1 -- and writes row c of W.
__global__ void __launch_bounds__(32)
k_trinv_rows(const double2* __restrict__ L, int lds, int nd, const int* __restrict__ keep,
             const int* __restrict__ rank, int kept, double2* __restrict__ X, int ldx, double2* __restrict__ W,
             int ldw) {
    const int c = blockIdx.x, lane = threadIdx.x;
    double2* x = X + (size_t)c * ldx;  // scratch row for column c of L^-1
    if (!keep[c]) {
        for (int k = lane; k < kept; k += 32) W[(size_t)c * ldw + k] = make_double2(0.0, 0.0);
        return;
    }
    for (int i = lane; i < nd; i += 32) x[i] = make_double2(0.0, 0.0);
    __syncwarp();
    for (int i = c; i < nd; ++i) {
        if (!keep[i]) continue;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = c + lane; j < i; j += 32) {
            const double2 a = L[(size_t)i * lds + j], v = x[j];
            acc.x += a.x * v.x - a.y * v.y;
            acc.y += a.x * v.y + a.y * v.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) {
            const double d = L[(size_t)i * lds + i].x;
            x[i] = make_double2(((i == c ? 1.0 : 0.0) - acc.x) / d, -acc.y / d);
        }
        __syncwarp();
    }
    for (int k = lane; k < nd; k += 32)
        if (keep[k]) W[(size_t)c * ldw + rank[k]] = make_double2(x[k].x, -x[k].y);
}

__global__ void k_rank(const int* __restrict__ keep, int nd, int* __restrict__ rank, int* __restrict__ kept) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int r = 0;
        for (int i = 0; i < nd; ++i) {
            rank[i] = keep[i] ? r : -1;
            r += keep[i];
        }
        *kept = r;
    }
}

}  // namespace

// Transform W (nd x kept, ld kept) whose gemm_tn with the nd rows Y gives kept orthonormal
// rows spanning Y minus its near-null directions (Cholesky with dropping of the Gram matrix
// S = Y Y^H, given in S (lds), destroyed).  keep/rank: nd ints each; X: nd x nd scratch;
// kept_dev: 1 int.  Asynchronous; the caller reads kept_dev.
qm_status chol_transform(double2* S, int lds, int nd, double drop_rel, int* keep, int* rank, int* kept_dev,
                         double2* X, double2* W, int ldw_max, cudaStream_t s) {
    (void)ldw_max;
    {
        const size_t smem = (size_t)nd * sizeof(double);
        ProfScope pf(PF_CHOL, s);
        k_chol_drop<<<1, 1024, smem, s>>>(S, lds, nd, drop_rel, keep);
    }
    {
        ProfScope pf(PF_CHOL, s);
        k_rank<<<1, 32, 0, s>>>(keep, nd, rank, kept_dev);
    }
    return cuda_check(cudaGetLastError(), "chol_transform launches");
}

// second half, once kept is known on the host: W (nd x kept)
qm_status chol_transform_rows(const double2* L, int lds, int nd, const int* keep, const int* rank, int kept,
                              double2* X, double2* W, cudaStream_t s) {
    ProfScope pf(PF_CHOL, s);
    k_trinv_rows<<<nd, 32, 0, s>>>(L, lds, nd, keep, rank, kept, X, nd, W, kept);
    return cuda_check(cudaGetLastError(), "k_trinv_rows launch");
}

}  // namespace qm

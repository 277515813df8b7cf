// Small dense FP64 kernels of the Davidson orthonormalisation step: Cholesky factorisation
// of the Gram matrix of a block of vectors, with dropping of near-dependent directions, and
// the triangular inverse that turns it into the transform of Cholesky-QR (the block is
// replaced by Y' = L^-H-weighted combinations of its rows, orthonormal and spanning the same
// space minus its near-null directions; Golub & Van Loan, Matrix Computations, Sec. 4.2, 5.2).
#include <algorithm>

#include "qm_internal.h"

namespace qm {
namespace {

// Blocked lower Cholesky S = L L^H of an nd x nd Hermitian positive semi-definite matrix
// (right-looking, Golub & Van Loan Sec. 4.2.8) with dropping: a pivot below
// drop_rel * S_jj(original) marks vector j as linearly dependent on the previous ones; its
// column of L is zero and it is skipped (Cholesky with dropping == Gram-Schmidt that discards
// near-null directions).  Per block column k0 (kNB wide): the diagonal block is factored in
// one CTA (k_chol_diag), the rows below it solved against it on many CTAs (k_chol_panel),
// and the trailing lower triangle updated by the panel's rank-kNB product on many CTAs
// (k_chol_update); the dropping decisions are those of the unblocked algorithm, since every
// pivot is tested after all updates from the columns before it.  Only the lower triangle is
// read and written; the original diagonal is kept in `orig`.
constexpr int kNB = 32;

__global__ void k_chol_orig(const double2* __restrict__ S, int lds, int nd, double* __restrict__ orig) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x)
        orig[i] = S[(size_t)i * lds + i].x;
}

// factor the nb x nb diagonal block at (k0, k0) in shared memory (nb <= kNB); 1024 threads
__global__ void __launch_bounds__(1024)
k_chol_diag(double2* __restrict__ S, int lds, int k0, int nb, const double* __restrict__ orig, double drop_rel,
            int* __restrict__ keep) {
    __shared__ double2 a[kNB][kNB + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // column, row
    if (ty < nb && tx <= ty) a[ty][tx] = S[(size_t)(k0 + ty) * lds + k0 + tx];
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const double piv = a[j][j].x;
        const bool ok = piv > drop_rel * orig[k0 + j] && piv > 0.0 && isfinite(piv);
        __syncthreads();  // every thread has read the pivot
        if (ty == j && tx == 0) {
            a[j][j] = make_double2(ok ? sqrt(piv) : 0.0, 0.0);
            keep[k0 + j] = ok ? 1 : 0;
        }
        if (tx == j && ty > j) {  // column j below the diagonal
            const double il = ok ? 1.0 / sqrt(piv) : 0.0;
            a[ty][j] = make_double2(a[ty][j].x * il, a[ty][j].y * il);
        }
        __syncthreads();
        if (ty > j && tx > j && tx <= ty) {  // a[i][k] -= L[i][j] conj(L[k][j])
            const double2 p = a[ty][j], q = a[tx][j];
            a[ty][tx].x -= p.x * q.x + p.y * q.y;
            a[ty][tx].y -= p.y * q.x - p.x * q.y;
        }
        __syncthreads();
    }
    if (ty < nb && tx <= ty) S[(size_t)(k0 + ty) * lds + k0 + tx] = a[ty][tx];
}

// rows i >= k0 + nb of the block column: L[i][k0 + j] from S[i][k0 + j] = sum_t L[i][t] conj(L11[j][t])
// by forward substitution (a dropped column j has L11[j][j] = 0 and gives L[i][j] = 0);
// one thread per row, 32 rows per CTA
__global__ void __launch_bounds__(32)
k_chol_panel(double2* __restrict__ S, int lds, int nd, int k0, int nb) {
    __shared__ double2 l11[kNB][kNB + 1];
    __shared__ double2 row[32][kNB + 1];
    const int t = threadIdx.x;
    for (int r = 0; r < nb; ++r)
        if (t <= r) l11[r][t] = S[(size_t)(k0 + r) * lds + k0 + t];
    const int i0 = k0 + nb + blockIdx.x * 32;
    for (int r = 0; r < 32; ++r) {  // coalesced: lane t reads column t of row i0 + r
        const int i = i0 + r;
        if (i < nd && t < nb) row[r][t] = S[(size_t)i * lds + k0 + t];
    }
    __syncwarp();
    const int i = i0 + t;
    if (i < nd) {
        for (int j = 0; j < nb; ++j) {
            const double d = l11[j][j].x;
            double2 v = row[t][j];
            for (int q = 0; q < j; ++q) {  // v -= L[i][q] conj(L11[j][q])
                const double2 x = row[t][q], c = l11[j][q];
                v.x -= x.x * c.x + x.y * c.y;
                v.y -= x.y * c.x - x.x * c.y;
            }
            row[t][j] = d > 0.0 ? make_double2(v.x / d, v.y / d) : make_double2(0.0, 0.0);
        }
    }
    __syncwarp();
    for (int r = 0; r < 32; ++r) {
        const int ii = i0 + r;
        if (ii < nd && t < nb) S[(size_t)ii * lds + k0 + t] = row[r][t];
    }
}

// trailing lower triangle i >= k >= k1 = k0 + nb: S[i][k] -= sum_t L[i][k0 + t] conj(L[k][k0 + t]);
// one 32 x 32 output tile per CTA (tiles on or below the diagonal), 256 threads x 4 outputs
__global__ void __launch_bounds__(256)
k_chol_update(double2* __restrict__ S, int lds, int nd, int k0, int nb) {
    __shared__ double2 li[32][kNB + 1], lk[32][kNB + 1];
    const int k1 = k0 + nb;
    // tile (ti, tk) with tk <= ti from the linear block index
    const int b = blockIdx.x;
    int ti = (int)((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= b) ++ti;
    while (ti * (ti + 1) / 2 > b) --ti;
    const int tk = b - ti * (ti + 1) / 2;
    const int r0 = k1 + 32 * ti, c0 = k1 + 32 * tk;
    const int tid = threadIdx.x;
    for (int e = tid; e < 32 * kNB; e += 256) {
        const int r = e / kNB, t = e % kNB;
        li[r][t] = (r0 + r < nd && t < nb) ? S[(size_t)(r0 + r) * lds + k0 + t] : make_double2(0.0, 0.0);
        lk[r][t] = (c0 + r < nd && t < nb) ? S[(size_t)(c0 + r) * lds + k0 + t] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int c = tid & 31, rb = tid >> 5;  // column c, rows rb, rb + 8, rb + 16, rb + 24
    double2 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int t = 0; t < nb; ++t) {
        const double2 y = lk[c][t];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 x = li[rb + 8 * q][t];
            acc[q].x += x.x * y.x + x.y * y.y;
            acc[q].y += x.y * y.x - x.x * y.y;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = r0 + rb + 8 * q, k = c0 + c;
        if (i < nd && k <= i) {
            double2* p = S + (size_t)i * lds + k;
            double2 v = *p;
            v.x -= acc[q].x;
            v.y -= acc[q].y;
            *p = v;
        }
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
    double* orig = reinterpret_cast<double*>(X);  // the scratch X is free until chol_transform_rows
    {
        ProfScope pf(PF_CHOL, s);
        k_chol_orig<<<(nd + 255) / 256, 256, 0, s>>>(S, lds, nd, orig);
    }
    for (int k0 = 0; k0 < nd; k0 += kNB) {
        const int nb = std::min(kNB, nd - k0), below = nd - k0 - nb;
        {
            ProfScope pf(PF_CHOL, s);
            k_chol_diag<<<1, 1024, 0, s>>>(S, lds, k0, nb, orig, drop_rel, keep);
        }
        if (below > 0) {
            const int nt = (below + 31) / 32;
            {
                ProfScope pf(PF_CHOL, s);
                k_chol_panel<<<nt, 32, 0, s>>>(S, lds, nd, k0, nb);
            }
            {
                ProfScope pf(PF_CHOL, s);
                k_chol_update<<<nt * (nt + 1) / 2, 256, 0, s>>>(S, lds, nd, k0, nb);
            }
        }
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

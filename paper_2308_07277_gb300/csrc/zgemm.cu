// Complex GEMMs of the nonlocal projector step (Sec. 2.3, KB form: P = beta^H psi, then
// beta D P) and of the Davidson subspace products (<V_i|H V_j>, rotations by the Ritz
// coefficients).  SIMT kernels with shared-memory tiles: in FP64 the hardware's double
// rate, not memory, bounds these contractions, so register tiling over 64x64 output tiles
// is enough to keep the FP64 pipe busy.
//
//   cn : C[m][n] = sum_k conj(A[m][k]) B[n][k]            (k contiguous in A and B)
//        split over K into `splits` partials reduced in a fixed order (deterministic)
//   tn : C[m][n] (+)= sum_k A[k][m] d[k] B[k][n]           (m, n contiguous)
#include <algorithm>

#include "qm_internal.h"

namespace qm {

namespace {

template <class C> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

constexpr int BM = 64, BN = 64, BK = 16, NTH = 256;

template <class C>
__device__ __forceinline__ C czero() {
    C z;
    z.x = 0;
    z.y = 0;
    return z;
}

template <class C>
__global__ void __launch_bounds__(NTH)
k_gemm_cn(int M, int N, int K, const C* __restrict__ A, int lda, const C* __restrict__ B, int ldb,
          C* __restrict__ out, int ldo, int kchunk) {
    using R = typename Real<C>::T;
    __shared__ C As[BK][BM + 1];
    __shared__ C Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    R acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0;
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int it = 0; it < (BM * BK) / NTH; ++it) {
            int e = tid + it * NTH;
            int row = e / BK, kk = e % BK;
            int gm = m0 + row, gk = k0 + kk;
            As[kk][row] = (gm < M && gk < ke) ? A[(size_t)gm * lda + gk] : czero<C>();
            int gn = n0 + row;
            Bs[kk][row] = (gn < N && gk < ke) ? B[(size_t)gn * ldb + gk] : czero<C>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // conj(a) * b
                    acc[i][j][0] = fma(a[i].x, b[j].x, fma(a[i].y, b[j].y, acc[i][j][0]));
                    acc[i][j][1] = fma(a[i].x, b[j].y, fma(-a[i].y, b[j].x, acc[i][j][1]));
                }
        }
        __syncthreads();
    }
    C* o = out + (size_t)blockIdx.z * M * ldo;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn < N) {
                C v;
                v.x = acc[i][j][0];
                v.y = acc[i][j][1];
                o[(size_t)gm * ldo + gn] = v;
            }
        }
    }
}

template <class C>
__global__ void k_reduce_splits(int M, int N, const C* __restrict__ part, int splits, C* __restrict__ Cout, int ldc) {
    const size_t total = (size_t)M * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int m = (int)(i / N), n = (int)(i % N);
        C s = czero<C>();
        for (int z = 0; z < splits; ++z) {
            C v = part[(size_t)z * total + i];
            s.x += v.x;
            s.y += v.y;
        }
        Cout[(size_t)m * ldc + n] = s;
    }
}

template <class C>
__global__ void __launch_bounds__(NTH)
k_gemm_tn(int M, int N, int K, const C* __restrict__ A, int lda, const double* __restrict__ d,
          const C* __restrict__ B, int ldb, C* __restrict__ Cm, int ldc, int accumulate) {
    using R = typename Real<C>::T;
    __shared__ C As[BK][BM + 1];
    __shared__ C Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    R acc[4][4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int it = 0; it < (BM * BK) / NTH; ++it) {
            int e = tid + it * NTH;
            int kk = e / BM, col = e % BM;
            int gk = k0 + kk;
            C av = czero<C>(), bv = czero<C>();
            if (gk < K) {
                int gm = m0 + col;
                if (gm < M) {
                    av = A[(size_t)gk * lda + gm];
                    if (d) {
                        R s = (R)d[gk];
                        av.x *= s;
                        av.y *= s;
                    }
                }
                int gn = n0 + col;
                if (gn < N) bv = B[(size_t)gk * ldb + gn];
            }
            As[kk][col] = av;
            Bs[kk][col] = bv;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j][0] = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j][0]));
                    acc[i][j][1] = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j][1]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn < N) {
                C* p = Cm + (size_t)gm * ldc + gn;
                C v;
                v.x = acc[i][j][0];
                v.y = acc[i][j][1];
                if (accumulate) {
                    C o = *p;
                    v.x += o.x;
                    v.y += o.y;
                }
                *p = v;
            }
        }
    }
}

template <class C>
qm_status gemm_cn_impl(int M, int N, int K, const C* A, int lda, const C* B, int ldb, C* Cm, int ldc,
                       C* partial, int splits, cudaStream_t s) {
    if (M <= 0 || N <= 0) return QM_OK;
    splits = std::max(1, splits);
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    if (kchunk <= 0) kchunk = BK;
    splits = std::max(1, (K + kchunk - 1) / kchunk);
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    if (splits == 1 || partial == nullptr) {
        if (splits != 1) return fail(QM_ERR_ARG, "gemm_cn: split-K needs a partial buffer");
        ProfScope pf(PF_GEMM_CN, s);
        k_gemm_cn<C><<<grid, NTH, 0, s>>>(M, N, K, A, lda, B, ldb, Cm, ldc, kchunk);
    } else {
        {
            ProfScope pf(PF_GEMM_CN, s);
            k_gemm_cn<C><<<grid, NTH, 0, s>>>(M, N, K, A, lda, B, ldb, partial, N, kchunk);
        }
        size_t total = (size_t)M * N;
        int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 8);
        ProfScope pf(PF_REDUCE, s);
        k_reduce_splits<C><<<blocks, 256, 0, s>>>(M, N, partial, splits, Cm, ldc);
    }
    return cuda_check(cudaGetLastError(), "gemm_cn launch");
}

template <class C>
qm_status gemm_tn_impl(int M, int N, int K, const C* A, int lda, const double* d, const C* B, int ldb, C* Cm,
                       int ldc, bool accumulate, cudaStream_t s) {
    if (M <= 0 || N <= 0) return QM_OK;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, 1);
    ProfScope pf(PF_GEMM_TN, s);
    k_gemm_tn<C><<<grid, NTH, 0, s>>>(M, N, K, A, lda, d, B, ldb, Cm, ldc, accumulate ? 1 : 0);
    return cuda_check(cudaGetLastError(), "gemm_tn launch");
}

}  // namespace

int zgemm_cn_splits(int M, int N, int K) {
    // enough CTAs for ~2 waves on 152 SMs, each split at least 256 deep
    long tiles = (long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    long want = std::max<long>(1, (2 * 152 + tiles - 1) / tiles);
    long maxs = std::max<long>(1, K / 256);
    return (int)std::min(want, maxs);
}

qm_status zgemm_cn(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb, double2* C,
                   int ldc, double2* partial, int splits, cudaStream_t s) {
    return gemm_cn_impl<double2>(M, N, K, A, lda, B, ldb, C, ldc, partial, splits, s);
}
qm_status cgemm_cn(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, float2* C, int ldc,
                   float2* partial, int splits, cudaStream_t s) {
    return gemm_cn_impl<float2>(M, N, K, A, lda, B, ldb, C, ldc, partial, splits, s);
}
qm_status zgemm_tn(int M, int N, int K, const double2* A, int lda, const double* d, const double2* B, int ldb,
                   double2* C, int ldc, bool accumulate, cudaStream_t s) {
    return gemm_tn_impl<double2>(M, N, K, A, lda, d, B, ldb, C, ldc, accumulate, s);
}
qm_status cgemm_tn(int M, int N, int K, const float2* A, int lda, const double* d, const float2* B, int ldb,
                   float2* C, int ldc, bool accumulate, cudaStream_t s) {
    return gemm_tn_impl<float2>(M, N, K, A, lda, d, B, ldb, C, ldc, accumulate, s);
}

}  // namespace qm

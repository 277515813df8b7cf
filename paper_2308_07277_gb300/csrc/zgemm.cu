// Complex GEMMs of the nonlocal projector step (Sec. 2.3, KB form: P = beta^H psi, then
// beta D P) and of the Davidson subspace products (<V_i|H V_j>, rotations by the Ritz
// coefficients, Gram-Schmidt projections).  SIMT kernels with shared-memory tiles: in FP64
// the GB300's double rate (about 1.2 TFLOP/s), not memory, bounds these contractions, so
// register tiling with enough CTAs to fill every SM is what matters.
//
//   cn : C[m][n] = sum_k conj(A[m][k]) B[n][k]                 (k contiguous in A and B)
//        split over K into partial sums reduced in a fixed order (deterministic)
//   tn : C[m][n] = alpha sum_k A[k][m] d[k] B[k][n] (+ C[m][n])  (m, n contiguous)
//
// 16 x 16 threads per CTA, each owning a TM x TN block of outputs (tile 16TM x 16TN); the
// per-call tile is chosen so that the M and N edges waste as little as possible (160
// bands -> TM = 5, 256 projectors -> TM = 4).  With FP32 arithmetic the products of one K tile
// (16 terms) are summed in FP32 and the tile sums in FP64, so the rounding error does not grow
// with K (inner products over 10^4 - 10^5 plane waves keep ~1e-7 relative accuracy).
#include <algorithm>

#include "qm_internal.h"

namespace qm {

namespace {

template <class C> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

constexpr int BK = 16, NTH = 256;

template <class C>
__device__ __forceinline__ C czero() {
    C z;
    z.x = 0;
    z.y = 0;
    return z;
}

template <class D, class S>
__device__ __forceinline__ D cvt(S a) {
    D r;
    r.x = (decltype(r.x))a.x;
    r.y = (decltype(r.y))a.y;
    return r;
}

// FP32 arithmetic: move the FP32 sum of one K tile into the FP64 sums (nothing in FP64)
template <class R, int TM, int TN>
__device__ __forceinline__ void flush_tile(R (&acc)[TM][TN][2], double (&hi)[TM][TN][2]) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    hi[i][j][c] += (double)acc[i][j][c];
                    acc[i][j][c] = 0;
                }
    }
}

// FP32 arithmetic: the result is the FP64 sum, rounded on output by the caller
template <class R, int TM, int TN>
__device__ __forceinline__ void finish_tiles(R (&acc)[TM][TN][2], const double (&hi)[TM][TN][2]) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
#pragma unroll
                for (int c = 0; c < 2; ++c) acc[i][j][c] = (R)hi[i][j][c];
    }
}

// C: storage type of A, B and the output; W: arithmetic type (FP64 or FP32 complex)
template <class C, class W, int TM, int TN>
__global__ void __launch_bounds__(NTH)
k_gemm_cn(int M, int N, int K, const C* __restrict__ A, int lda, const C* __restrict__ B, int ldb,
          C* __restrict__ out, int ldo, int kchunk) {
    using R = typename Real<W>::T;
    constexpr int BM = 16 * TM, BN = 16 * TN;
    __shared__ W As[BK][BM + 1];
    __shared__ W Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    R acc[TM][TN][2];
    double hi[TM][TN][2];  // FP32 arithmetic: sums of the per-tile FP32 partial sums
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j][0] = acc[i][j][1] = 0, hi[i][j][0] = hi[i][j][1] = 0.0;
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NTH) {
            int row = e / BK, kk = e % BK;
            int gm = m0 + row, gk = k0 + kk;
            As[kk][row] = (gm < M && gk < ke) ? cvt<W>(A[(size_t)gm * lda + gk]) : czero<W>();
        }
        for (int e = tid; e < BN * BK; e += NTH) {
            int row = e / BK, kk = e % BK;
            int gn = n0 + row, gk = k0 + kk;
            Bs[kk][row] = (gn < N && gk < ke) ? cvt<W>(B[(size_t)gn * ldb + gk]) : czero<W>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            W a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    // conj(a) * b
                    acc[i][j][0] = fma(a[i].x, b[j].x, fma(a[i].y, b[j].y, acc[i][j][0]));
                    acc[i][j][1] = fma(a[i].x, b[j].y, fma(-a[i].y, b[j].x, acc[i][j][1]));
                }
        }
        flush_tile<R, TM, TN>(acc, hi);
        __syncthreads();
    }
    finish_tiles<R, TM, TN>(acc, hi);
    C* o = out + (size_t)blockIdx.z * M * ldo;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn < N) {
                C v;
                v.x = (decltype(v.x))acc[i][j][0];
                v.y = (decltype(v.y))acc[i][j][1];
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

template <class C, class W, int TM, int TN>
__global__ void __launch_bounds__(NTH)
k_gemm_tn(int M, int N, int K, const C* __restrict__ A, int lda, const double* __restrict__ d, double alpha,
          const C* __restrict__ B, int ldb, C* __restrict__ Cm, int ldc, int accumulate) {
    using R = typename Real<W>::T;
    constexpr int BM = 16 * TM, BN = 16 * TN;
    __shared__ W As[BK][BM + 1];
    __shared__ W Bs[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    R acc[TM][TN][2];
    double hi[TM][TN][2];  // FP32 arithmetic: sums of the per-tile FP32 partial sums
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j][0] = acc[i][j][1] = 0, hi[i][j][0] = hi[i][j][1] = 0.0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NTH) {
            int kk = e / BM, col = e % BM;
            int gk = k0 + kk, gm = m0 + col;
            W av = czero<W>();
            if (gk < K && gm < M) {
                av = cvt<W>(A[(size_t)gk * lda + gm]);
                R s = (R)(d ? alpha * d[gk] : alpha);
                av.x *= s;
                av.y *= s;
            }
            As[kk][col] = av;
        }
        for (int e = tid; e < BN * BK; e += NTH) {
            int kk = e / BN, col = e % BN;
            int gk = k0 + kk, gn = n0 + col;
            Bs[kk][col] = (gk < K && gn < N) ? cvt<W>(B[(size_t)gk * ldb + gn]) : czero<W>();
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            W a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    acc[i][j][0] = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j][0]));
                    acc[i][j][1] = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j][1]));
                }
        }
        flush_tile<R, TM, TN>(acc, hi);
        __syncthreads();
    }
    finish_tiles<R, TM, TN>(acc, hi);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn < N) {
                C* p = Cm + (size_t)gm * ldc + gn;
                C v;
                v.x = (decltype(v.x))acc[i][j][0];
                v.y = (decltype(v.y))acc[i][j][1];
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

// thread-tile size for one dimension: the T in {5, 4, 2} (BM = 16 T) that pads n least
int pick_t(int n) {
    int best = 4;
    long bestpad = 1L << 60;
    for (int t : {5, 4, 2}) {
        long b = 16L * t;
        long pad = (n + b - 1) / b * b;
        if (pad < bestpad) {
            bestpad = pad;
            best = t;
        }
    }
    return best;
}

constexpr int kMaxSlots = 4 * 152;

// resident CTAs of a kernel on the current device (occupancy x SM count), cached per kernel
template <class F>
int resident_slots(F* kernel) {
    static thread_local int cached = 0;
    if (cached) return cached;
    int dev = 0, sms = 152, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NTH, 0) != cudaSuccess || occ < 1) occ = 1;
    cached = std::min(kMaxSlots, occ * sms);
    return cached;
}

template <class C, class W, int TM, int TN>
qm_status cn_launch(int M, int N, int K, const C* A, int lda, const C* B, int ldb, C* Cm, int ldc, C* partial,
                    int max_splits, cudaStream_t s) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const int kSlots = resident_slots(k_gemm_cn<C, W, TM, TN>);
    // splits: fill the resident slots in whole waves, each split at least 128 deep
    int splits = std::max(1, std::min({kSlots / std::max(1, tiles), std::max(1, K / 128), max_splits}));
    if (!partial) splits = 1;
    int kchunk = (K + splits - 1) / splits;
    kchunk = std::max(BK, (kchunk + BK - 1) / BK * BK);
    splits = std::max(1, (K + kchunk - 1) / kchunk);
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    if (splits == 1) {
        ProfScope pf(PF_GEMM_CN, s);
        k_gemm_cn<C, W, TM, TN><<<grid, NTH, 0, s>>>(M, N, K, A, lda, B, ldb, Cm, ldc, kchunk);
    } else {
        {
            ProfScope pf(PF_GEMM_CN, s);
            k_gemm_cn<C, W, TM, TN><<<grid, NTH, 0, s>>>(M, N, K, A, lda, B, ldb, partial, N, kchunk);
        }
        size_t total = (size_t)M * N;
        const int blocks = grid_stride_blocks(total, 256, 8);
        ProfScope pf(PF_REDUCE, s);
        k_reduce_splits<C><<<blocks, 256, 0, s>>>(M, N, partial, splits, Cm, ldc);
    }
    return cuda_check(cudaGetLastError(), "gemm_cn launch");
}

template <class C, class W>
qm_status gemm_cn_impl(int M, int N, int K, const C* A, int lda, const C* B, int ldb, C* Cm, int ldc,
                       C* partial, int max_splits, cudaStream_t s) {
    if (M <= 0 || N <= 0) return QM_OK;
    const int tm = pick_t(M), tn = pick_t(N);
#define QM_CN(a, b) \
    if (tm == a && tn == b) return cn_launch<C, W, a, b>(M, N, K, A, lda, B, ldb, Cm, ldc, partial, max_splits, s);
    QM_CN(5, 5) QM_CN(5, 4) QM_CN(4, 5) QM_CN(4, 4) QM_CN(2, 4) QM_CN(4, 2) QM_CN(2, 5) QM_CN(5, 2) QM_CN(2, 2)
#undef QM_CN
    return fail(QM_ERR_UNSUPPORTED, "gemm_cn: no tile");
}

template <class C, class W, int TM, int TN>
qm_status tn_launch(int M, int N, int K, const C* A, int lda, const double* d, double alpha, const C* B, int ldb,
                    C* Cm, int ldc, bool accumulate, cudaStream_t s) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, 1);
    ProfScope pf(PF_GEMM_TN, s);
    k_gemm_tn<C, W, TM, TN><<<grid, NTH, 0, s>>>(M, N, K, A, lda, d, alpha, B, ldb, Cm, ldc, accumulate ? 1 : 0);
    return cuda_check(cudaGetLastError(), "gemm_tn launch");
}

template <class C, class W>
qm_status gemm_tn_impl(int M, int N, int K, const C* A, int lda, const double* d, double alpha, const C* B,
                       int ldb, C* Cm, int ldc, bool accumulate, cudaStream_t s) {
    if (M <= 0 || N <= 0) return QM_OK;
    const int tm = pick_t(M);
    // the N dimension (plane waves) is long: TN = 4 keeps 256-wide rows of whole tiles
#define QM_TN(a) \
    if (tm == a) return tn_launch<C, W, a, 4>(M, N, K, A, lda, d, alpha, B, ldb, Cm, ldc, accumulate, s);
    QM_TN(5) QM_TN(4) QM_TN(2)
#undef QM_TN
    return fail(QM_ERR_UNSUPPORTED, "gemm_tn: no tile");
}

}  // namespace

size_t gemm_cn_partial_bytes(bool fp32) {
    // splits * tiles <= resident slots, so splits * M * N <= kMaxSlots * (80 x 80 largest tile)
    return (size_t)kMaxSlots * 80 * 80 * (fp32 ? sizeof(float2) : sizeof(double2));
}

int zgemm_cn_splits(int M, int N, int K) {
    (void)M;
    (void)N;
    return std::max(1, std::min(kMaxSlots, K / 128));
}

qm_status zgemm_cn(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb, double2* C,
                   int ldc, double2* partial, int splits, cudaStream_t s) {
    return gemm_cn_impl<double2, double2>(M, N, K, A, lda, B, ldb, C, ldc, partial, splits, s);
}
qm_status cgemm_cn(int M, int N, int K, const float2* A, int lda, const float2* B, int ldb, float2* C, int ldc,
                   float2* partial, int splits, cudaStream_t s) {
    return gemm_cn_impl<float2, float2>(M, N, K, A, lda, B, ldb, C, ldc, partial, splits, s);
}
qm_status zgemm_tn(int M, int N, int K, const double2* A, int lda, const double* d, const double2* B, int ldb,
                   double2* C, int ldc, bool accumulate, cudaStream_t s, double alpha) {
    return gemm_tn_impl<double2, double2>(M, N, K, A, lda, d, alpha, B, ldb, C, ldc, accumulate, s);
}
qm_status cgemm_tn(int M, int N, int K, const float2* A, int lda, const double* d, const float2* B, int ldb,
                   float2* C, int ldc, bool accumulate, cudaStream_t s, double alpha) {
    return gemm_tn_impl<float2, float2>(M, N, K, A, lda, d, alpha, B, ldb, C, ldc, accumulate, s);
}

}  // namespace qm

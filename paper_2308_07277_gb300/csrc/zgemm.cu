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

// Double-FP32 ("double-single") complex arithmetic type: a double value v is held as
// hi (v's first 24 significant bits) + lo (the next 23), 47 bits.  A product a b accumulates into a
// (hi, lo) pair by error-free transformations on the FP32 pipe (Dekker's exact product via an
// FMA, Knuth's TwoSum): p = fl(a_h b_h) with its exact error e = fma(a_h, b_h, -p), the cross
// terms a_h b_l + a_l b_h added to e (a_l b_l < 2^-48 |a b| is dropped), then
// (hi, lo) += p + e with the rounding error of hi + p kept exactly.  About 12 FP32 operations
// per real multiply-add against one FP64 FMA, on a pipe 64 times wider on this GPU; the sums of
// every few K tiles go to FP64 accumulators, so the result keeps ~2^-46 relative accuracy per product and
// no error growth with K.  The _rn intrinsics keep the compiler from fusing the steps.  The
// products live in FP32's exponent range: terms below about 1e-38 lose their relative accuracy
// (they are negligible next to the sums of the plane-wave products this serves).
struct ds2 {
    float xh, xl, yh, yl;
};
template <> struct Real<ds2> { using T = float; };
template <class W> constexpr bool is_ds = false;
template <> constexpr bool is_ds<ds2> = true;

__device__ __forceinline__ void ds_mac(float& hi, float& lo, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float t = __fadd_rn(hi, p);
    const float v = __fsub_rn(t, hi);
    const float w = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, v)), __fsub_rn(p, v));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(w, e));
}

constexpr int BK = 16, NTH = 256;

template <class C>
__device__ __forceinline__ C czero() {
    C z;
    z.x = 0;
    z.y = 0;
    return z;
}

// x = hi + lo with hi = x truncated to 24 significant bits (exact) and lo = the remaining 29
// mantissa bits truncated to 23: 47 significant bits, from the bit fields by integer operations
// (the FP64 conversions and the FP64 subtraction of the plain split run on this GPU's narrow
// FP64 path and stalled the tile loads).  Exponents outside FP32's normal range take the plain
// split.
// the plain split, for exponents outside FP32's normal range; not inlined, so that the common
// path branches around it instead of issuing its FP64 instructions predicated off
__device__ __noinline__ float2 split_ds_slow(double x) {
    const float hi = __double2float_rn(x);
    const bool zero_exp = (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu) == 0;
    return make_float2(hi, zero_exp ? 0.f : __double2float_rn(x - (double)hi));
}
__device__ __forceinline__ void split_ds(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
    const int e = (int)((hw >> 20) & 0x7FFu);
    const int ef = e - 1023 + 127;
    if (ef <= 0 || ef >= 255) {
        const float2 r = split_ds_slow(x);
        hi = r.x;
        lo = r.y;
        return;
    }
    const unsigned int sign = hw & 0x80000000u;
    hi = __uint_as_float(sign | ((unsigned int)ef << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    // lo = m_lo 2^(e - 1075), m_lo the low 29 mantissa bits, kept to its top 23: the float
    // 1 + (m_lo >> 6) 2^-23 minus 1 is exact (Sterbenz), then scaled by 2^(e - 1046) - no
    // integer-to-float conversion (conversions run on this GPU's narrow FP64 path).  hi + lo
    // keeps 47 significant bits; lo is dropped (zero) when |x| < 2^-103.
    const int es = e - 1046 + 127;
    const float scale = es >= 1 ? __uint_as_float((unsigned int)es << 23) : 0.f;
    const float f = __fsub_rn(__uint_as_float(0x3F800000u | ((lw & 0x1FFFFFFFu) >> 6)), 1.0f);
    const float l = __fmul_rn(f, scale);
    lo = sign ? -l : l;
}

template <class D, class S>
__device__ __forceinline__ D cvt(S a) {
    if constexpr (is_ds<D>) {
        D r;
        split_ds(a.x, r.xh, r.xl);
        split_ds(a.y, r.yh, r.yl);
        return r;
    } else {
        D r;
        r.x = (decltype(r.x))a.x;
        r.y = (decltype(r.y))a.y;
        return r;
    }
}
template <> __device__ __forceinline__ ds2 czero<ds2>() { return ds2{0.f, 0.f, 0.f, 0.f}; }

// End of a K tile.  FP32 arithmetic: the tile's sum moves into the FP64 sums.  Double-FP32:
// the (hi, lo) pairs are renormalised in FP32 (FastTwoSum: hi + lo unchanged, |lo| back to
// half an ulp of hi) and move into the FP64 sums only every kDsFlush tiles and at the end
// (`flush`): the conversions and FP64 additions run on this GPU's narrow FP64 path (two lanes
// per clock per SM), so flushing every tile cost about as much as the products themselves.
// FP64 arithmetic: nothing.
constexpr int kDsFlush = 8;
template <class W, class R, int TM, int TN>
__device__ __forceinline__ void flush_tile(R (&acc)[TM][TN][2], float (&lo)[TM][TN][2], double (&hi)[TM][TN][2],
                                           bool flush) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if constexpr (is_ds<W>) {
                        if (flush) {
                            hi[i][j][c] += (double)acc[i][j][c];
                            hi[i][j][c] += (double)lo[i][j][c];
                            acc[i][j][c] = 0;
                            lo[i][j][c] = 0.f;
                        } else {
                            const float t = __fadd_rn(acc[i][j][c], lo[i][j][c]);
                            lo[i][j][c] = __fsub_rn(lo[i][j][c], __fsub_rn(t, acc[i][j][c]));
                            acc[i][j][c] = t;
                        }
                    } else {
                        hi[i][j][c] += (double)acc[i][j][c];
                        acc[i][j][c] = 0;
                    }
                }
    }
}

// the finished sum of output (i, j), component c: the FP64 sums for FP32 and double-FP32
// arithmetic (rounded on output by the caller), the accumulator itself in FP64
template <class R, int TM, int TN>
__device__ __forceinline__ double result(const R (&acc)[TM][TN][2], const double (&hi)[TM][TN][2], int i, int j,
                                         int c) {
    if constexpr (sizeof(R) == 4)
        return hi[i][j][c];
    else
        return acc[i][j][c];
}

// one complex multiply-add of the K loop: cn: acc += conj(a) b; tn: acc += a b
template <class W, bool CONJ, class R>
__device__ __forceinline__ void cmac(R (&acc)[2], float (&lo)[2], const W& a, const W& b) {
    if constexpr (is_ds<W>) {
        const float s = CONJ ? 1.f : -1.f;  // sign of the a_im b_im term of the real part
        ds_mac(acc[0], lo[0], a.xh, a.xl, b.xh, b.xl);
        ds_mac(acc[0], lo[0], s * a.yh, s * a.yl, b.yh, b.yl);
        ds_mac(acc[1], lo[1], a.xh, a.xl, b.yh, b.yl);
        ds_mac(acc[1], lo[1], -s * a.yh, -s * a.yl, b.xh, b.xl);
    } else if constexpr (CONJ) {
        acc[0] = fma(a.x, b.x, fma(a.y, b.y, acc[0]));
        acc[1] = fma(a.x, b.y, fma(-a.y, b.x, acc[1]));
    } else {
        acc[0] = fma(a.x, b.x, fma(-a.y, b.y, acc[0]));
        acc[1] = fma(a.x, b.y, fma(a.y, b.x, acc[1]));
    }
}

// C: storage type of A, B and the output; W: arithmetic type (FP64, FP32 or double-FP32 complex)
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
    float lo[TM][TN][2];   // double-FP32 arithmetic: the low parts
    double hi[TM][TN][2];  // FP32 / double-FP32 arithmetic: sums of the per-tile partial sums
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
            acc[i][j][0] = acc[i][j][1] = 0, lo[i][j][0] = lo[i][j][1] = 0.f, hi[i][j][0] = hi[i][j][1] = 0.0;
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
                for (int j = 0; j < TN; ++j) cmac<W, true>(acc[i][j], lo[i][j], a[i], b[j]);  // conj(a) * b
        }
        flush_tile<W, R, TM, TN>(acc, lo, hi, ((k0 - kb) / BK) % kDsFlush == kDsFlush - 1 || k0 + BK >= ke);
        __syncthreads();
    }
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
                v.x = (decltype(v.x))result(acc, hi, i, j, 0);
                v.y = (decltype(v.y))result(acc, hi, i, j, 1);
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
    float lo[TM][TN][2];   // double-FP32 arithmetic: the low parts
    double hi[TM][TN][2];  // FP32 / double-FP32 arithmetic: sums of the per-tile partial sums
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
            acc[i][j][0] = acc[i][j][1] = 0, lo[i][j][0] = lo[i][j][1] = 0.f, hi[i][j][0] = hi[i][j][1] = 0.0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NTH) {
            int kk = e / BM, col = e % BM;
            int gk = k0 + kk, gm = m0 + col;
            W av = czero<W>();
            if (gk < K && gm < M) {
                C v = A[(size_t)gk * lda + gm];
                const auto sc = (decltype(v.x))(d ? alpha * d[gk] : alpha);
                v.x *= sc;
                v.y *= sc;
                av = cvt<W>(v);
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
                for (int j = 0; j < TN; ++j) cmac<W, false>(acc[i][j], lo[i][j], a[i], b[j]);
        }
        flush_tile<W, R, TM, TN>(acc, lo, hi, (k0 / BK) % kDsFlush == kDsFlush - 1 || k0 + BK >= K);
        __syncthreads();
    }
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
                v.x = (decltype(v.x))result(acc, hi, i, j, 0);
                v.y = (decltype(v.y))result(acc, hi, i, j, 1);
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
    // splits: each at least 128 deep, within the caller's partial-sum buffer (max_splits, and
    // the size gemm_cn_partial_bytes guarantees), chosen so that the CTAs fill the resident
    // slots in nearly whole waves: the fewest splits whose last wave is not more than 10 %
    // emptier than the best choice (a grid of 160 tiles on 304 slots otherwise leaves half
    // of them idle)
    const long cap = (long)(gemm_cn_partial_bytes(sizeof(C) == 8) / sizeof(C)) / std::max<long>(1, (long)M * N);
    const int smax = (int)std::max<long>(1, std::min<long>({(long)std::max(1, K / 128), (long)max_splits, cap, 64L}));
    auto fill = [&](int sp) {
        const long ctas = (long)tiles * sp, waves = (ctas + kSlots - 1) / kSlots;
        return (double)ctas / (double)(waves * kSlots);
    };
    double best = 0.0;
    for (int sp = 1; sp <= smax; ++sp) best = std::max(best, fill(sp));
    int splits = 1;
    while (splits < smax && fill(splits) < best - 0.1) ++splits;
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
    if constexpr (is_ds<W>) {
        // double-FP32: two FP32 accumulators and an FP64 sum per output; 8 outputs per thread
        // (about 120 registers, two CTAs per SM)
        if (M >= N) return cn_launch<C, W, 4, 2>(M, N, K, A, lda, B, ldb, Cm, ldc, partial, max_splits, s);
        return cn_launch<C, W, 2, 4>(M, N, K, A, lda, B, ldb, Cm, ldc, partial, max_splits, s);
    } else {
        const int tm = pick_t(M), tn = pick_t(N);
#define QM_CN(a, b) \
    if (tm == a && tn == b) return cn_launch<C, W, a, b>(M, N, K, A, lda, B, ldb, Cm, ldc, partial, max_splits, s);
        QM_CN(5, 5) QM_CN(5, 4) QM_CN(4, 5) QM_CN(4, 4) QM_CN(2, 4) QM_CN(4, 2) QM_CN(2, 5) QM_CN(5, 2) QM_CN(2, 2)
#undef QM_CN
        return fail(QM_ERR_UNSUPPORTED, "gemm_cn: no tile");
    }
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
    if constexpr (is_ds<W>) {  // double-FP32: 8 outputs per thread, as in gemm_cn_impl
        return tn_launch<C, W, 2, 4>(M, N, K, A, lda, d, alpha, B, ldb, Cm, ldc, accumulate, s);
    } else {
        const int tm = pick_t(M);
        // the N dimension (plane waves) is long: TN = 4 keeps 256-wide rows of whole tiles
#define QM_TN(a) \
    if (tm == a) return tn_launch<C, W, a, 4>(M, N, K, A, lda, d, alpha, B, ldb, Cm, ldc, accumulate, s);
        QM_TN(5) QM_TN(4) QM_TN(2)
#undef QM_TN
        return fail(QM_ERR_UNSUPPORTED, "gemm_tn: no tile");
    }
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
qm_status zgemm_cn_ds(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb, double2* C,
                      int ldc, double2* partial, int splits, cudaStream_t s) {
    return gemm_cn_impl<double2, ds2>(M, N, K, A, lda, B, ldb, C, ldc, partial, splits, s);
}
qm_status zgemm_tn_ds(int M, int N, int K, const double2* A, int lda, const double* d, const double2* B, int ldb,
                      double2* C, int ldc, bool accumulate, cudaStream_t s, double alpha) {
    return gemm_tn_impl<double2, ds2>(M, N, K, A, lda, d, alpha, B, ldb, C, ldc, accumulate, s);
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

using namespace qm;

extern "C" qm_status qm_zgemm(int op, int arith, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                              void* C, int ldc, void* stream) {
    clear_error();
    if ((op != 0 && op != 1) || arith < 0 || arith > 2) return fail(QM_ERR_ARG, "qm_zgemm: op not 0/1 or arith not 0..2");
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return fail(QM_ERR_ARG, "qm_zgemm: bad sizes or NULL operand");
    if (op == 0 ? (lda < K || ldb < K || ldc < N) : (lda < M || ldb < N || ldc < N))
        return fail(QM_ERR_ARG, "qm_zgemm: leading dimension too small");
    cudaStream_t s = (cudaStream_t)stream;
    const double2* a = (const double2*)A;
    const double2* b = (const double2*)B;
    double2* c = (double2*)C;
    if (arith == 2) {  // BF16x3 split products on the tensor cores (the Davidson's FP32 phase)
        const size_t wbytes = op == 0 ? subspace_bf16x3_bytes(M, N)
                                      : std::max(subspace_bf16x3_bytes(M, 1), (size_t)M * K * sizeof(float2));
        void* work = nullptr;
        int* err = nullptr;
        if (cudaMallocAsync(&work, wbytes, s) != cudaSuccess || cudaMallocAsync((void**)&err, sizeof(int), s) != cudaSuccess) {
            cudaGetLastError();
            if (work) cudaFreeAsync(work, s);
            return fail(QM_ERR_OOM, "qm_zgemm: tensor-core workspace");
        }
        qm_status st = cuda_check(cudaMemsetAsync(err, 0, sizeof(int), s), "memset");
        if (!st)
            st = op == 0 ? zgemm_cn_bf16x3(M, N, K, a, lda, b, ldb, c, ldc, work, wbytes, err, s)
                         : zgemm_tn_bf16x3(M, N, K, a, lda, b, ldb, c, ldc, false, 1.0, work, wbytes, err, s);
        int e = 0;
        if (!st) st = cuda_check(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H error word");
        if (!st) st = cuda_check(cudaStreamSynchronize(s), "stream sync");
        cudaFreeAsync(work, s);
        cudaFreeAsync(err, s);
        if (!st && e) st = fail(QM_ERR_TIMEOUT, "qm_zgemm: a bounded tensor-core wait expired");
        return st;
    }
    if (op == 1)
        return (arith ? zgemm_tn_ds : zgemm_tn)(M, N, K, a, lda, nullptr, b, ldb, c, ldc, false, s, 1.0);
    void* part = nullptr;
    const int splits = zgemm_cn_splits(M, N, K);
    const size_t bytes = std::min((size_t)splits * M * N * sizeof(double2), gemm_cn_partial_bytes(false));
    if (cudaMallocAsync(&part, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(QM_ERR_OOM, "qm_zgemm: split-K partial sums");
    }
    qm_status st = (arith ? zgemm_cn_ds : zgemm_cn)(M, N, K, a, lda, b, ldb, c, ldc, (double2*)part, splits, s);
    cudaFreeAsync(part, s);
    return st;
}

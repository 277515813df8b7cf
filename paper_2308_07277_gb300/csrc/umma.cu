// Tensor-core (tcgen05) subspace products of the precision form's Davidson (the overlaps of
// Sec. 5's Davidson: H_sub, Gram matrices, basis rotations) as 3-term BF16 split products
// accumulated in FP32, with operands split on the fly from FP64 storage.
//
// Splitting: an FP32 value x is written x = x0 + x1 + x2 with x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); a product a*b keeps the six terms a_i b_j with
// i + j <= 2 (the dropped terms are below 2^-24 |a b|), each a BF16 x BF16 tensor-core product
// accumulated in FP32 in tensor memory.
//
// Complex -> real: with re/im interleaved along K, sum_k A[m][k] B[n][k] becomes a real GEMM
// over 2K in which the B operand is "expanded" to two real rows per complex row:
//   C = A B:        rows (b_re, -b_im), (b_im,  b_re)
//   C = conj(A) B:  rows (b_re,  b_im), (b_im, -b_re)
// so the real output C'[m][2n + t] is the interleaved complex result.
//
// Kernel: one CTA of 8 warps per 128 x 128 real output tile (and a K range for split-K).
// The operands are read as FP32 complex from global memory and split / expanded on the fly
// into shared memory (canonical no-swizzle K-major layout of 8 x 16-byte core matrices), so no
// split copy ever goes to HBM.  Two shared-memory stages: while the tensor core multiplies
// tile k (one thread issues 6 products x 2 K-steps of tcgen05.mma, M = N = 128, K = 16, into a
// 128-column FP32 accumulator in tensor memory, then commits to the stage's mbarrier), the
// CTA's loads of tile k+1 are in flight and are split into the other stage.  Every mbarrier wait is bounded and sets an error word
// instead of hanging.  The epilogue reads the accumulator with tcgen05.ld.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "qm_internal.h"
#include "tc_util.cuh"

namespace qm {
namespace {

constexpr int UM = 128, UN = 128, UK = 32;       // CTA tile: M x N x K (K in real elements)
constexpr int KCH = UK / 8;                      // 16-byte K chunks per core-matrix row
constexpr int TILE_BYTES = UM * UK * 2;          // one BF16 split component of one operand tile
constexpr int STAGE_BYTES = 6 * TILE_BYTES;      // A and B, 3 components each
constexpr int kThreads = 256;
constexpr long kSpinLimit = 1L << 26;            // bounded mbarrier waits

using tc::idesc_bf16;
using tc::sdesc;
using tc::smem_u32;
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) { return tc::mbar_wait(mbar, phase, kSpinLimit); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// split two FP32 values into the three BF16 components, packed in pairs
__device__ __forceinline__ void split_pair(float x, float y, uint32_t& c0, uint32_t& c1, uint32_t& c2) {
    const __nv_bfloat16 x0 = __float2bfloat16_rn(x), y0 = __float2bfloat16_rn(y);
    const float rx = x - __bfloat162float(x0), ry = y - __bfloat162float(y0);
    const __nv_bfloat16 x1 = __float2bfloat16_rn(rx), y1 = __float2bfloat16_rn(ry);
    const __nv_bfloat16 x2 = __float2bfloat16_rn(rx - __bfloat162float(x1));
    const __nv_bfloat16 y2 = __float2bfloat16_rn(ry - __bfloat162float(y1));
    c0 = pack2(x0, y0);
    c1 = pack2(x1, y1);
    c2 = pack2(x2, y2);
}

__device__ __forceinline__ void put_pair(unsigned char* dst, int off, float x, float y) {
    uint32_t c0, c1, c2;
    split_pair(x, y, c0, c1, c2);
    *reinterpret_cast<uint32_t*>(dst + off) = c0;
    *reinterpret_cast<uint32_t*>(dst + TILE_BYTES + off) = c1;
    *reinterpret_cast<uint32_t*>(dst + 2 * TILE_BYTES + off) = c2;
}

// Operand sources (FP32 complex in global memory).  A tile covers 128 real rows and UK = 32
// real K columns = 16 complex columns: 16 row groups x 4 K chunks = 64 core matrices of 8 rows
// x 16 bytes (96 KB of shared memory for both stages, so two CTAs fit on an SM).  Each warp
// fills one core matrix per step (8 per tile), lane i writing the i-th
// 4-byte word (one (re, im) pair of BF16) of each split component, so the shared-memory stores
// are free of bank conflicts.  fetch() issues the tile's global loads into registers;
// stash() splits them into shared memory.  Fetching tile k+1 before the products of tile k are
// issued hides the global latency behind the tensor core.
constexpr int kCmPerWarp = 16 * KCH / (kThreads / 32);  // 16 row groups x KCH chunks per tile

__device__ __forceinline__ void put_word(unsigned char* dst, int cm, int lane, float x, float y) {
    put_pair(dst, cm * 128 + lane * 4, x, y);
}

// complex element of the source as FP32: FP32 sources are read as they are, FP64 sources (the
// Davidson basis) are rounded to FP32 on load
__device__ __forceinline__ float2 ld_f2(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ld_f2(const double2* p) {
    const double2 v = __ldg(p);
    return make_float2((float)v.x, (float)v.y);
}

template <class Src>
struct PlainRows {  // rows = complex rows of src, K = the complex columns (interleaved re, im)
    const Src* src;
    int ld, rows, K;
    // core matrix cm = (row group) * 8 + (K chunk); lane = 4 * (row in group) + (complex col in chunk)
    __device__ __forceinline__ void fetch(float2* v, int r0, int kc0, int tid) const {
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int it = 0; it < kCmPerWarp; ++it) {
            const int cm = warp + 8 * it;
            const int gr = r0 + (cm / KCH) * 8 + (lane >> 2), gk = kc0 + (cm % KCH) * 4 + (lane & 3);
            v[it] = (gr < rows && gk < K) ? ld_f2(src + (size_t)gr * ld + gk) : make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ void stash(unsigned char* dst, const float2* v, int tid) const {
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int it = 0; it < kCmPerWarp; ++it) put_word(dst, warp + 8 * it, lane, v[it].x, v[it].y);
    }
};

// two real rows (2c, 2c+1) per complex element; lane = 8 a + 2 b + c: complex row a of the 4 in
// the row group, complex column b of the 4 in the K chunk, c = which of the two real rows
// (word (2a + c) * 4 + b of the core matrix)
__device__ __forceinline__ int expand_word(int lane) { return ((2 * (lane >> 3) + (lane & 1)) << 2) + ((lane >> 1) & 3); }

template <class Src>
struct ExpandRows {  // B rows from complex rows of src (conj_a: pattern of conj(A) B)
    const Src* src;
    int ld, rows, K, conj_a;
    __device__ __forceinline__ void fetch(float2* v, int r0, int kc0, int tid) const {
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int it = 0; it < kCmPerWarp; ++it) {
            const int cm = warp + 8 * it;
            const int gr = (r0 >> 1) + (cm / KCH) * 4 + (lane >> 3), gk = kc0 + (cm % KCH) * 4 + ((lane >> 1) & 3);
            v[it] = (gr < rows && gk < K) ? ld_f2(src + (size_t)gr * ld + gk) : make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ void stash(unsigned char* dst, const float2* v, int tid) const {
        const int warp = tid >> 5, lane = tid & 31, w = expand_word(lane), odd = lane & 1;
#pragma unroll
        for (int it = 0; it < kCmPerWarp; ++it) {
            const float2 a = v[it];
            float x, y;
            if (!conj_a) {
                x = odd ? a.y : a.x;
                y = odd ? a.x : -a.y;
            } else {
                x = odd ? a.y : a.x;
                y = odd ? -a.x : a.y;
            }
            put_pair(dst, (warp + 8 * it) * 128 + w * 4, x, y);
        }
    }
};

template <class Src>
struct ExpandTRows {  // B = src^T expanded: src [P][G] (G contiguous); rows 2g, 2g+1; K = p
    const Src* src;
    int ld, P, G;
    __device__ __forceinline__ void fetch(float2* v, int r0, int kc0, int tid) const {
        const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int it = 0; it < kCmPerWarp; ++it) {
            const int cm = warp + 8 * it;
            const int gg = (r0 >> 1) + (cm / KCH) * 4 + (lane >> 3), gp = kc0 + (cm % KCH) * 4 + ((lane >> 1) & 3);
            v[it] = (gp < P && gg < G) ? ld_f2(src + (size_t)gp * ld + gg) : make_float2(0.f, 0.f);
        }
    }
    __device__ __forceinline__ void stash(unsigned char* dst, const float2* v, int tid) const {
        const int warp = tid >> 5, lane = tid & 31, w = expand_word(lane), odd = lane & 1;
#pragma unroll
        for (int it = 0; it < kCmPerWarp; ++it) {
            const float2 b = v[it];  // rows (b_re, -b_im), (b_im, b_re)
            put_pair(dst, (warp + 8 * it) * 128 + w * 4, odd ? b.y : b.x, odd ? b.x : -b.y);
        }
    }
};

// C'[m][n] (+)= sum_k A[m][k] B[n][k] over the real K range of this split.  Output FP32 or
// FP64 (Out) with row stride ldc; rows >= M or columns >= N are not written.  Split z writes at
// C + z * zstride.  accumulate: add to the existing output.
template <class LA, class LB, class Out>
__global__ void __launch_bounds__(kThreads)
k_umma_split(LA la, LB lb, int M, int N, int ktiles_per_split, int ktiles_total, Out* __restrict__ C, size_t ldc,
             size_t zstride, int accumulate, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * UM, n0 = blockIdx.x * UN;
    const int kt0 = blockIdx.z * ktiles_per_split;
    const int kt1 = min(ktiles_total, kt0 + ktiles_per_split);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(UN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_bf16(UM, UN);
    uint32_t ph[2] = {0u, 0u};
    int issued[2] = {0, 0}, waited[2] = {0, 0};
    bool ok = true;
    float2 va[kCmPerWarp], vb[kCmPerWarp];
    if (kt0 < kt1) {
        la.fetch(va, m0, kt0 * (UK / 2), tid);
        lb.fetch(vb, n0, kt0 * (UK / 2), tid);
    }
    for (int kt = kt0; kt < kt1 && ok; ++kt) {
        const int s = (kt - kt0) & 1;
        unsigned char* sA = smem + s * STAGE_BYTES;
        unsigned char* sB = sA + 3 * TILE_BYTES;
        if (issued[s] > waited[s]) {  // the products of tile kt-2 must have read this stage
            const bool w = mbar_wait(smem_u32(&mbar[s]), ph[s]);
            ph[s] ^= 1u;
            ++waited[s];
            if (!__syncthreads_and(w)) {  // a uniform decision: no thread is left at a barrier
                ok = false;
                if (tid == 0) atomicExch(err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
        }
        la.stash(sA, va, tid);
        lb.stash(sB, vb, tid);
        if (kt + 1 < kt1) {  // next tile's loads are in flight while this tile is multiplied
            la.fetch(va, m0, (kt + 1) * (UK / 2), tid);
            lb.fetch(vb, n0, (kt + 1) * (UK / 2), tid);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            // products a_i b_j with i + j <= 2, smallest terms first
            const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
#pragma unroll
                for (int ks = 0; ks < UK / 16; ++ks) {
                    const uint64_t da = sdesc(smem_u32(sA + pa[q] * TILE_BYTES) + ks * 256, 128, KCH * 128);
                    const uint64_t db = sdesc(smem_u32(sB + pb[q] * TILE_BYTES) + ks * 256, 128, KCH * 128);
                    const uint32_t acc = (kt > kt0 || q > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&mbar[s])));
        }
        ++issued[s];
    }
    // wait for the products still in flight (every thread runs the same waits)
    for (int s = 0; s < 2 && ok; ++s) {
        while (issued[s] > waited[s] && ok) {
            const bool w = mbar_wait(smem_u32(&mbar[s]), ph[s]);
            ph[s] ^= 1u;
            ++waited[s];
            if (!__syncthreads_and(w)) {
                ok = false;
                if (tid == 0) atomicExch(err, 1);
            }
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (ok && kt1 > kt0) {
        // warp w reads accumulator lanes 32 (w % 4) + 0..31 (tile rows); warps 0-3 take
        // columns 0..63, warps 4-7 columns 64..127
        const int q = warp & 3, chalf = (warp >> 2) * 64;
        const int row = m0 + q * 32 + (tid & 31);
        Out* crow = C + (size_t)blockIdx.z * zstride + (size_t)row * ldc;
#pragma unroll 1
        for (int c0 = chalf; c0 < chalf + 64; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < N) {
                        const Out x = (Out)__uint_as_float(v[j]);
                        crow[col] = accumulate ? crow[col] + x : x;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UN));
}

// sum the split-K partials C'[z][i][2j + t] of a subspace product in FP64 and write the complex
// result C[i][j] (FP64, row stride ldc)
__global__ void k_reduce_cn(const float* __restrict__ part, int Z, size_t zstride, int ldp, int M, int N,
                            double2* __restrict__ C, int ldc) {
    const size_t total = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e % N);
        double sr = 0.0, si = 0.0;
        for (int z = 0; z < Z; ++z) {
            const float2 q = __ldg(reinterpret_cast<const float2*>(part + (size_t)z * zstride + (size_t)i * ldp) + j);
            sr += (double)q.x;
            si += (double)q.y;
        }
        C[(size_t)i * ldc + j] = make_double2(sr, si);
    }
}

// At[i][j] = alpha * A[j][i] in FP32 (the small coefficient matrix of a basis rotation, made
// K-major for the tensor-core operand)
__global__ void k_coef_t(const double2* __restrict__ A, int lda, int M, int K, double alpha, float2* __restrict__ At) {
    const size_t total = (size_t)M * K;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / K), j = (int)(e % K);
        const double2 a = A[(size_t)j * lda + i];
        At[e] = make_float2((float)(alpha * a.x), (float)(alpha * a.y));
    }
}

inline size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int grid_for(size_t n) { return grid_stride_blocks(std::max<size_t>(n, 1), 256, 16); }

template <class LA, class LB, class Out>
qm_status umma_launch(const LA& la, const LB& lb, int M, int N, int kreal, int splits, Out* C, size_t ldc,
                      size_t zstride, bool accumulate, int* err, cudaStream_t s, int* zout) {
    const int ktiles = (int)((rup((size_t)kreal, UK)) / UK);
    splits = std::max(1, std::min(splits, ktiles));
    const int per = (ktiles + splits - 1) / splits;
    splits = (ktiles + per - 1) / per;
    if (zout) *zout = splits;
    const size_t smem = 2 * (size_t)STAGE_BYTES;
    qm_status st = allow_dynamic_smem((const void*)k_umma_split<LA, LB, Out>, smem, "tensor-core GEMM shared memory");
    if (st) return st;
    dim3 grid((N + UN - 1) / UN, (M + UM - 1) / UM, splits);
    ProfScope pf(PF_UMMA, s);
    k_umma_split<LA, LB, Out><<<grid, kThreads, smem, s>>>(la, lb, M, N, per, ktiles, C, ldc, zstride, accumulate ? 1 : 0,
                                                     err);
    return cuda_check(cudaGetLastError(), "k_umma_split launch");
}

}  // namespace

// ---- subspace products of the Davidson FP32 phase (FP64 storage, BF16x3 tensor-core products) ----

size_t subspace_bf16x3_bytes(int max_m, int max_n) {
    // the cn split-K partials: splits x tiles <= 2 x SMs + tiles (see zgemm_cn_bf16x3)
    const size_t tiles = (rup((size_t)max_m, UM) / UM) * (rup(2 * (size_t)max_n, UN) / UN);
    const size_t part = rup((2 * (size_t)device_sms() + tiles) * UM * UN * sizeof(float), 256);
    // the tn coefficient operand: M x K FP32 complex.  Calls on one stream reuse the buffer.
    const size_t coef = rup((size_t)max_m * max_m * sizeof(float2), 256);
    return std::max(part, coef);
}

qm_status zgemm_cn_bf16x3(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb, double2* C,
                          int ldc, void* work, size_t work_bytes, int* err, cudaStream_t s) {
    if (M <= 0 || N <= 0) return QM_OK;
    const size_t rM = rup(M, UM), r2N = rup(2 * (size_t)N, UN);
    const int tiles = (int)((rM / UM) * (r2N / UN));
    const size_t zstride = rM * r2N;
    const int cap = (int)std::min<size_t>(kMaxUmmaSplits, work_bytes / (zstride * sizeof(float)));
    if (cap < 1) return fail(QM_ERR_ARG, "zgemm_cn_bf16x3: workspace too small");
    const int splits = std::max(1, std::min(cap, (2 * device_sms() + tiles - 1) / tiles));  // 2 CTAs per SM
    PlainRows<double2> la{A, lda, M, K};
    ExpandRows<double2> lb{B, ldb, N, K, 1};
    int Z = 1;
    float* part = (float*)work;
    qm_status st = umma_launch(la, lb, M, 2 * N, 2 * K, splits, part, r2N, zstride, false, err, s, &Z);
    if (st) return st;
    {
        ProfScope pf(PF_SPLIT, s);
        k_reduce_cn<<<grid_for((size_t)M * N), 256, 0, s>>>(part, Z, zstride, (int)r2N, M, N, C, ldc);
    }
    return cuda_check(cudaGetLastError(), "k_reduce_cn launch");
}

qm_status zgemm_tn_bf16x3(int M, int N, int K, const double2* A, int lda, const double2* B, int ldb, double2* C,
                          int ldc, bool accumulate, double alpha, void* work, size_t work_bytes, int* err,
                          cudaStream_t s) {
    if (M <= 0 || N <= 0) return QM_OK;
    if (K <= 0) {
        if (accumulate) return QM_OK;
        return cuda_check(cudaMemset2DAsync(C, (size_t)ldc * sizeof(double2), 0, (size_t)N * sizeof(double2), M, s),
                          "zgemm_tn_bf16x3 zero");
    }
    if ((size_t)M * K * sizeof(float2) > work_bytes) return fail(QM_ERR_ARG, "zgemm_tn_bf16x3: workspace too small");
    float2* at = (float2*)work;
    {
        ProfScope pf(PF_SPLIT, s);
        k_coef_t<<<grid_for((size_t)M * K), 256, 0, s>>>(A, lda, M, K, alpha, at);
    }
    qm_status st = cuda_check(cudaGetLastError(), "k_coef_t launch");
    if (st) return st;
    PlainRows<float2> la{at, K, M, K};
    ExpandTRows<double2> lb{B, ldb, K, N};
    return umma_launch(la, lb, M, 2 * N, 2 * K, 1, (double*)C, 2 * (size_t)ldc, 0, accumulate, err, s, nullptr);
}

}  // namespace qm

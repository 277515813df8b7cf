// Nonlocal part of the precision form on the tensor cores: the projection P = beta^H psi and
// the application beta (D P) of the Kleinman-Bylander term (Sec. 2.3) as 3-term BF16 split
// products accumulated in FP32 (tcgen05, accumulators in tensor memory).
//
// Splitting: an FP32 value x is written x = x0 + x1 + x2 with x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); a product a*b keeps the six terms a_i b_j with
// i + j <= 2 (the dropped terms are below 2^-24 |a b|).
//
// Operands are split ONCE into BF16 planes stored in global memory in a tile-blocked order:
// block (row tile, K tile) holds, for each of the three planes, the R x 32 tile in the
// canonical no-swizzle K-major shared-memory layout of the tensor core (8-row x 16-byte core
// matrices; element (r, k) at ((r/8)*4 + k/8)*128 + (r%8)*16 + (k%8)*2).  A K tile of one
// operand is therefore one contiguous run of 3*R*64 bytes, which a single bulk copy
// (cp.async.bulk, completion counted on an mbarrier) lands in shared memory ready for the MMA.
//
// Complex products as real GEMMs over K' = 2K (re, im interleaved or (p, u) pairs):
//   projection  C[p][2b+t] = sum_(g,u) betaK[p][(g,u)] psiX[2b+t][(g,u)]
//               betaK = beta as stored (K = (g, u) interleaved), psiX row 2b = psi_b as stored,
//               row 2b+1 = (im, -re) of psi_b, so C[p][2b] = Re<beta_p|psi_b>, C[p][2b+1] = Im.
//   application C[2b+t][g] = sum_(p,u) E[2b+t][(p,u)] betaT[g][(p,u)]
//               betaT[g][(p,u)] = component u of beta[p][g] (beta transposed, not expanded),
//               E = D P expanded: E[2b][(p,0)] = ar, E[2b][(p,1)] = -ai, E[2b+1][(p,0)] = ai,
//               E[2b+1][(p,1)] = ar (a = D_p P[p][b]), so C[2b][g] = Re(beta D P)[b][g], C[2b+1] = Im.
//
// GEMM kernel (k_nl_gemm): one CTA per (M tile of 128, N tile of BN <= 256, K range), eight
// warps: warp 0 issues the bulk copies into a 3-stage ring, warp 1 owns the tensor memory and
// one of its threads issues the 6 x 2 tcgen05.mma of each K tile (M = 128, N = BN, K = 16)
// and commits each stage back to the producer, warps 4-7 drain the accumulator with
// tcgen05.ld.  Every mbarrier wait is bounded: on expiry the kernel sets the error word, waits
// (bounded) for its own copies and products in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "qm_internal.h"
#include "tc_util.cuh"

namespace qm {
namespace {

constexpr int KT = 32;          // K tile (real elements): 4 chunks of 8 BF16
constexpr int TM = 128;         // rows of an A tile (M of the MMA)
constexpr int kStages = 3;
constexpr int kGemmThreads = 256;
constexpr long kSpin = 1L << 26;

__host__ __device__ constexpr size_t plane_bytes(int R) { return (size_t)R * KT * 2; }
__host__ __device__ constexpr size_t block_bytes(int R) { return 3 * plane_bytes(R); }

// byte offset of element (r, k) inside one plane of a tile
__device__ __forceinline__ int cm_off(int r, int k) {
    return ((((r >> 3) << 2) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// split two FP32 values into their three BF16 components, packed in pairs
__device__ __forceinline__ void split2(float x, float y, uint32_t& c0, uint32_t& c1, uint32_t& c2) {
    const __nv_bfloat16 x0 = __float2bfloat16_rn(x), y0 = __float2bfloat16_rn(y);
    const float rx = x - __bfloat162float(x0), ry = y - __bfloat162float(y0);
    const __nv_bfloat16 x1 = __float2bfloat16_rn(rx), y1 = __float2bfloat16_rn(ry);
    const __nv_bfloat16 x2 = __float2bfloat16_rn(rx - __bfloat162float(x1));
    const __nv_bfloat16 y2 = __float2bfloat16_rn(ry - __bfloat162float(y1));
    c0 = pack2(x0, y0);
    c1 = pack2(x1, y1);
    c2 = pack2(x2, y2);
}

// write the 8 consecutive K values v[0..7] of row r (k0 a multiple of 8) into the blocked array
__device__ __forceinline__ void put8(unsigned char* blk, int R, int nkt, int r, int k0, const float* v) {
    const int rt = r / R, rr = r - rt * R, kt = k0 / KT, kk = k0 - kt * KT;
    unsigned char* p = blk + ((size_t)rt * nkt + kt) * block_bytes(R) + cm_off(rr, kk);
    uint4 c[3];
    split2(v[0], v[1], c[0].x, c[1].x, c[2].x);
    split2(v[2], v[3], c[0].y, c[1].y, c[2].y);
    split2(v[4], v[5], c[0].z, c[1].z, c[2].z);
    split2(v[6], v[7], c[0].w, c[1].w, c[2].w);
#pragma unroll
    for (int q = 0; q < 3; ++q) *reinterpret_cast<uint4*>(p + q * plane_bytes(R)) = c[q];
}

// Rows of complex src (K = 2 ncols interleaved reals) -> blocked split operand.  expand = 0:
// row r is src row r as stored; expand = 1: rows 2b, 2b+1 are src row b as stored and its
// rotation (im, -re).  Rows >= nsrc (resp. 2 nsrc) and K beyond 2 ncols are written as zeros.
// CTA: 8 rows (one core-matrix row group, blockIdx.y) x 32 chunks of 8 K values (blockIdx.x);
// the 8 rows of a core matrix on consecutive threads (one 128-byte run per plane), the 4
// chunks of a K tile on consecutive thread octets.
constexpr int kSplitChunks = 32;
__global__ void __launch_bounds__(256) k_split_rows(const float2* __restrict__ src, int ld, int nsrc, int ncols,
                                                    int expand, int R, int nkt, unsigned char* __restrict__ blk) {
    const int r = blockIdx.y * 8 + (threadIdx.x & 7);
    const int ch = blockIdx.x * kSplitChunks + (threadIdx.x >> 3);
    if (ch >= nkt * (KT / 8)) return;
    const int b = expand ? (r >> 1) : r;
    const int c0 = ch * 4;  // first complex column of the chunk
    float v[8];
    if (b < nsrc && c0 + 3 < ncols) {
        const float2* s2 = src + (size_t)b * ld + c0;
        if (((uintptr_t)s2 & 15) == 0) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(s2)), bb = __ldg(reinterpret_cast<const float4*>(s2) + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = bb.x; v[5] = bb.y; v[6] = bb.z; v[7] = bb.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 x = __ldg(s2 + j);
                v[2 * j] = x.x;
                v[2 * j + 1] = x.y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 x = make_float2(0.f, 0.f);
            if (b < nsrc && c0 + j < ncols) x = __ldg(src + (size_t)b * ld + c0 + j);
            v[2 * j] = x.x;
            v[2 * j + 1] = x.y;
        }
    }
    if (expand && (r & 1)) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float re = v[2 * j], im = v[2 * j + 1];
            v[2 * j] = im;
            v[2 * j + 1] = -re;
        }
    }
    put8(blk, R, nkt, r, ch * 8, v);
}

// beta [P][G] (complex, ld) -> blocked split betaT: row g, K = (p, u) (u = re/im of beta[p][g]).
// CTA tile: 64 rows g x 16 projectors (one K tile), transposed through shared memory so the
// global reads run along g.  Rows g >= G (up to rows_pad) and p >= P are zeros.
constexpr int kTG = 64, kTP = KT / 2;
__global__ void __launch_bounds__(256) k_split_t(const float2* __restrict__ beta, int ld, int P, int G, int R, int nkt,
                                                 unsigned char* __restrict__ blk) {
    __shared__ float2 t[kTP][kTG + 1];
    const int g0 = blockIdx.x * kTG, p0 = blockIdx.y * kTP;
    for (int i = threadIdx.x; i < kTP * kTG; i += blockDim.x) {
        const int pp = i / kTG, gg = i - pp * kTG;
        const int p = p0 + pp, g = g0 + gg;
        t[pp][gg] = (p < P && g < G) ? __ldg(beta + (size_t)p * ld + g) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    // 64 rows x 4 chunks of 4 projectors; the 8 rows of a core matrix on consecutive threads
    const int rlo = threadIdx.x & 7, ch = (threadIdx.x >> 3) & 3, rg = threadIdx.x >> 5;
    const int gg = rg * 8 + rlo;
    float v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 x = t[ch * 4 + j][gg];
        v[2 * j] = x.x;
        v[2 * j + 1] = x.y;
    }
    put8(blk, R, nkt, g0 + gg, p0 * 2 + ch * 8, v);
}

// sum the split-K partials of the projection C[z][p][c] (FP32, ldc; c = 2b + t) in a fixed order
// and scale by D_p: Pd[p][c] = D_p sum_z C[z][p][c] (consecutive threads, consecutive c: coalesced)
__global__ void k_reduce_p(const float* __restrict__ part, int Z, size_t zstride, int ldc, int P, int ncol,
                           const double* __restrict__ D, float* __restrict__ Pd) {
    const size_t total = (size_t)P * ncol;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(e / ncol), c = (int)(e - (size_t)p * ncol);
        const float* q = part + (size_t)p * ldc + c;
        float a = 0.f;
        for (int z = 0; z < Z; ++z) a += __ldg(q + (size_t)z * zstride);
        Pd[e] = a * (float)__ldg(D + p);
    }
}

// the application's A operand E = D P expanded, blocked and split (rows 2b + t, K = (p, u)):
// E[2b][(p,0)] = ar, E[2b][(p,1)] = -ai, E[2b+1][(p,0)] = ai, E[2b+1][(p,1)] = ar with
// a = Pd[p][2b] + i Pd[p][2b+1]; rows >= 2 nb and p >= P are zeros.  One thread per (row, 4
// projectors), the 8 rows of a core matrix on consecutive threads.
__global__ void k_expand_e(const float* __restrict__ Pd, int P, int nb, int rows_pad, int nkt,
                           unsigned char* __restrict__ blk) {
    const int nchunk = nkt * (KT / 8);
    const long total = (long)rows_pad * nchunk;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int rlo = (int)(e & 7);
        const long q = e >> 3;
        const int ch = (int)(q % nchunk);
        const int r = (int)(q / nchunk) * 8 + rlo;
        const int b = r >> 1, t = r & 1;
        float v[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = ch * 4 + j;
            float ar = 0.f, ai = 0.f;
            if (b < nb && p < P) {
                const float2 a = __ldg(reinterpret_cast<const float2*>(Pd + (size_t)p * 2 * nb) + b);
                ar = a.x;
                ai = a.y;
            }
            v[2 * j] = t ? ai : ar;
            v[2 * j + 1] = t ? ar : -ai;
        }
        put8(blk, TM, nkt, r, ch * 8, v);
    }
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort) {
    for (long i = 0; i < kSpin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 1023) == 1023 && abort && *abort) return false;
    }
    return false;
}

// C (+)= A B^T over the K tiles [kt0, kt1) of this split.  A: blocked, 128-row tiles, nkt K
// tiles per row tile; B: blocked, BN-row tiles.  EPI 0: C is FP32 [m][n] (ldc) at C + z*zstride
// (split-K partials); EPI 1: row m = 2b + t, column g -> complex out[b][g] component t
// (ldc = complex row stride), accumulate: add to out.
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 1)
k_nl_gemm(const unsigned char* __restrict__ A, const unsigned char* __restrict__ B, int nkt, int BN, int M, int N,
          int kt_per_split, float* __restrict__ C, size_t ldc, size_t zstride, int accumulate, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, s_used, s_issued;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // projection: N tiles fastest (the few N tiles of one M tile share its beta tiles in L2);
    // application: M tiles fastest (the M tiles of one N tile share its betaT tiles, which are
    // then read from HBM once instead of once per M tile)
    const int nt = EPI == 0 ? blockIdx.x : blockIdx.y, mt = EPI == 0 ? blockIdx.y : blockIdx.x;
    const int kt0 = blockIdx.z * kt_per_split;
    const int kt1 = min(nkt, kt0 + kt_per_split);
    const int nk = max(0, kt1 - kt0);
    const uint32_t a_bytes = (uint32_t)block_bytes(TM), b_bytes = (uint32_t)block_bytes(BN);
    const uint32_t stage_bytes = a_bytes + b_bytes;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tc::smem_u32(&tmem_base)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::smem_u32(&accf)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    volatile int* abort = &abort_flag;
    const unsigned char* a_src = A + ((size_t)mt * nkt + kt0) * a_bytes;
    const unsigned char* b_src = B + ((size_t)nt * nkt + kt0) * b_bytes;
    const uint32_t sbase = tc::smem_u32(smem);
    int issued = 0;  // producer: K tiles whose copies were issued
    int used = 0;    // MMA issuer: K tiles consumed
    if (warp == 0 && lane == 0) {
        for (int it = 0; it < nk; ++it) {
            const int s = it % kStages;
            if (it >= kStages && !wait_bar(tc::smem_u32(&empty[s]), ((it / kStages) & 1) ^ 1, abort)) {
                *abort = 1;
                break;
            }
            const uint32_t fb = tc::smem_u32(&full[s]);
            const uint32_t dst = sbase + s * stage_bytes;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(stage_bytes) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                "l"(a_src + (size_t)it * a_bytes), "r"(a_bytes), "r"(fb)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    dst + a_bytes),
                "l"(b_src + (size_t)it * b_bytes), "r"(b_bytes), "r"(fb)
                : "memory");
            issued = it + 1;
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc::idesc_bf16(TM, BN);
        const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};  // smallest terms first
        for (int it = 0; it < nk; ++it) {
            const int s = it % kStages;
            if (!wait_bar(tc::smem_u32(&full[s]), (it / kStages) & 1, abort)) {
                *abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
#pragma unroll
                for (int ks = 0; ks < KT / 16; ++ks) {
                    const uint64_t da = tc::sdesc(sa + pa[q] * (uint32_t)plane_bytes(TM) + ks * 256, 128, 512);
                    const uint64_t db = tc::sdesc(sb + pb[q] * (uint32_t)plane_bytes(BN) + ks * 256, 128, 512);
                    const uint32_t acc = (it > 0 || q > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                tc::smem_u32(&empty[s])));
            used = it + 1;
        }
        // the accumulator is final once every product issued so far has completed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            tc::smem_u32(&accf)));
    }
    if (warp == 1 && lane == 0) s_used = used;
    if (warp == 0 && lane == 0) s_issued = issued;
    if (warp >= 4) {
        const bool ok = wait_bar(tc::smem_u32(&accf), 0, nullptr);
        if (!ok) *abort = 1;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        // warp-uniform decision (tcgen05.ld and the shuffles below need the whole warp)
        if (__all_sync(0xffffffffu, ok && nk > 0 && !*abort)) {
            const int q = warp & 3;
            const int mrow = mt * TM + q * 32 + lane;  // this thread's accumulator row
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                const int n0 = nt * BN + c0;
                if (EPI == 0) {
                    if (mrow < M) {
                        float* crow = C + (size_t)blockIdx.z * zstride + (size_t)mrow * ldc;
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (n0 + j < N) crow[n0 + j] = __uint_as_float(v[j]);
                    }
                } else {
                    // lanes 2j, 2j+1 hold Re and Im of band mrow/2: swap halves so that each lane
                    // owns 8 complex values (64 contiguous bytes) of the band's row
                    const int t = lane & 1;
                    float y[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        y[j] = __shfl_xor_sync(0xffffffffu, __uint_as_float(t ? v[j] : v[8 + j]), 1);
                    if (mrow < M) {
                        const int g0 = n0 + (t ? 8 : 0);
                        float2* orow = reinterpret_cast<float2*>(C) + (size_t)(mrow >> 1) * ldc;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int g = g0 + j;
                            if (g < N) {
                                float2 o = t ? make_float2(y[j], __uint_as_float(v[8 + j]))
                                             : make_float2(__uint_as_float(v[j]), y[j]);
                                if (accumulate) {
                                    const float2 a = orow[g];
                                    o.x += a.x;
                                    o.y += a.y;
                                }
                                orow[g] = o;
                            }
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (*abort) {
        if (tid == 0) atomicExch(err, 1);
        // drain: the copies issued but never consumed, then every product issued
        if (warp == 0 && lane == 0) {
            for (int it = s_used; it < s_issued; ++it) {
                const int s = it % kStages;
                wait_bar(tc::smem_u32(&full[s]), (it / kStages) & 1, nullptr);
            }
        }
        if (warp == 1 && lane == 0) wait_bar(tc::smem_u32(&accf), 0, nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256));
}

inline size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

// N tile of the projection: the 2 nb columns in the fewest tiles of at most 256, rounded to 16
int proj_bn(int nb) {
    const int n = 2 * nb;
    const int tiles = (n + 255) / 256;
    return (int)rup((size_t)((n + tiles - 1) / tiles), 16);
}
constexpr int kAppBN = 256;

struct NlLayout {
    int bn_p, ntile_p, mtile_p, nkt_p;  // projection: N tile, tiles, K tiles (of 2 npw)
    int mtile_a, ntile_a, nkt_a;        // application
    int splits;
    size_t betaK_off, betaT_off, psiX_off, part_off, pd_off, e_off, total;
    size_t zstride;
};

NlLayout nl_layout(int nproj, int nb, int npw, bool with_beta) {
    NlLayout L{};
    L.bn_p = proj_bn(nb);
    L.ntile_p = (2 * nb + L.bn_p - 1) / L.bn_p;
    L.mtile_p = (nproj + TM - 1) / TM;
    L.nkt_p = (int)(rup(2 * (size_t)npw, KT) / KT);
    L.mtile_a = (2 * nb + TM - 1) / TM;
    L.ntile_a = (npw + kAppBN - 1) / kAppBN;
    L.nkt_a = (int)(rup(2 * (size_t)nproj, KT) / KT);
    const int tiles = L.ntile_p * L.mtile_p;
    L.splits = std::max(1, std::min(std::min(kMaxUmmaSplits, L.nkt_p), device_sms() / std::max(1, tiles)));
    L.zstride = (size_t)L.mtile_p * TM * L.ntile_p * L.bn_p;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off = rup(off + b, 256);
        return o;
    };
    L.betaK_off = take(with_beta ? (size_t)L.mtile_p * L.nkt_p * block_bytes(TM) : 0);
    L.betaT_off = take(with_beta ? (size_t)L.ntile_a * L.nkt_a * block_bytes(kAppBN) : 0);
    L.psiX_off = take((size_t)L.ntile_p * L.nkt_p * block_bytes(L.bn_p));
    L.part_off = take((size_t)L.splits * L.zstride * sizeof(float));
    L.pd_off = take((size_t)nproj * 2 * nb * sizeof(float));
    L.e_off = take((size_t)L.mtile_a * L.nkt_a * block_bytes(TM));
    L.total = off;
    return L;
}

// grid-dimension limits of the split and GEMM launches (y and z of a grid are below 65536)
qm_status check_limits(const NlLayout& L) {
    if ((long)L.mtile_p * TM / 8 > 65535 || (long)L.ntile_p * L.bn_p / 8 > 65535 || L.nkt_a > 65535 ||
        L.ntile_a > 65535 || L.mtile_p > 65535)
        return fail(QM_ERR_UNSUPPORTED, "tensor-core nonlocal part: too many bands, projectors or plane waves");
    return QM_OK;
}

inline int grid_for(long n, int per = 256) { return grid_stride_blocks((size_t)std::max<long>(n, 1), per, 16); }

qm_status split_beta(int nproj, int npw, const float2* beta, int ld_beta, const NlLayout& L, unsigned char* betaK,
                     unsigned char* betaT, cudaStream_t s) {
    {
        ProfScope pf(PF_SPLIT, s);
        const dim3 grid((unsigned)((L.nkt_p * (KT / 8) + kSplitChunks - 1) / kSplitChunks), (unsigned)(L.mtile_p * TM / 8));
        k_split_rows<<<grid, 256, 0, s>>>(beta, ld_beta, nproj, npw, 0, TM, L.nkt_p, betaK);
    }
    qm_status st = cuda_check(cudaGetLastError(), "k_split_rows launch");
    if (st) return st;
    {
        ProfScope pf(PF_SPLIT, s);
        dim3 grid((unsigned)(L.ntile_a * kAppBN / kTG), (unsigned)L.nkt_a);
        k_split_t<<<grid, 256, 0, s>>>(beta, ld_beta, nproj, npw, kAppBN, L.nkt_a, betaT);
    }
    return cuda_check(cudaGetLastError(), "k_split_t launch");
}

template <int EPI>
qm_status gemm_launch(const unsigned char* A, const unsigned char* B, int nkt, int BN, int M, int N, int mt, int ntl,
                      int splits, float* C, size_t ldc, size_t zstride, bool accumulate, int* err, cudaStream_t s) {
    const int per = (nkt + splits - 1) / splits;
    splits = (nkt + per - 1) / per;
    const size_t smem = (size_t)kStages * (block_bytes(TM) + block_bytes(BN));
    qm_status st = allow_dynamic_smem((const void*)k_nl_gemm<EPI>, smem, "tensor-core nonlocal GEMM shared memory");
    if (st) return st;
    ProfScope pf(PF_UMMA, s);
    const dim3 grid = EPI == 0 ? dim3(ntl, mt, splits) : dim3(mt, ntl, splits);
    k_nl_gemm<EPI><<<grid, kGemmThreads, smem, s>>>(A, B, nkt, BN, M, N, per, C, ldc, zstride, accumulate ? 1 : 0, err);
    return cuda_check(cudaGetLastError(), "k_nl_gemm launch");
}

}  // namespace

size_t nonlocal_tc_bytes(int nproj, int nb, int npw, bool with_beta) {
    return nl_layout(nproj, nb, npw, with_beta).total;
}

size_t nonlocal_tc_beta_bytes(int nproj, int nb, int npw) {
    const NlLayout L = nl_layout(nproj, nb, npw, true);
    return L.psiX_off;  // betaK and betaT come first
}

qm_status nonlocal_tc_prepare(int nproj, int nb, int npw, const float2* beta, int ld_beta, void* beta_work,
                              cudaStream_t s) {
    if (nproj <= 0) return QM_OK;
    const NlLayout L = nl_layout(nproj, nb, npw, true);
    if (qm_status st0 = check_limits(L)) return st0;
    unsigned char* w = (unsigned char*)beta_work;
    return split_beta(nproj, npw, beta, ld_beta, L, w + L.betaK_off, w + L.betaT_off, s);
}

qm_status nonlocal_tc(int nproj, int nb, int npw, const float2* beta, int ld_beta, const void* beta_prepared,
                      const float2* psi, int ld_psi, const double* D, float2* out, int ld_out, void* work, int* err,
                      cudaStream_t s, bool accumulate) {
    if (nproj <= 0 || nb <= 0) return QM_OK;
    const bool own_beta = beta_prepared == nullptr;
    const NlLayout L = nl_layout(nproj, nb, npw, own_beta);
    if (qm_status st0 = check_limits(L)) return st0;
    unsigned char* w = (unsigned char*)work;
    const unsigned char* betaK;
    const unsigned char* betaT;
    qm_status st;
    if (own_beta) {
        if ((st = split_beta(nproj, npw, beta, ld_beta, L, w + L.betaK_off, w + L.betaT_off, s))) return st;
        betaK = w + L.betaK_off;
        betaT = w + L.betaT_off;
    } else {
        const NlLayout Lb = nl_layout(nproj, nb, npw, true);
        betaK = (const unsigned char*)beta_prepared + Lb.betaK_off;
        betaT = (const unsigned char*)beta_prepared + Lb.betaT_off;
    }
    unsigned char* psiX = w + L.psiX_off;
    float* part = (float*)(w + L.part_off);
    unsigned char* E = w + L.e_off;
    {
        ProfScope pf(PF_SPLIT, s);
        const dim3 grid((unsigned)((L.nkt_p * (KT / 8) + kSplitChunks - 1) / kSplitChunks), (unsigned)(L.ntile_p * L.bn_p / 8));
        k_split_rows<<<grid, 256, 0, s>>>(psi, ld_psi, nb, npw, 1, L.bn_p, L.nkt_p, psiX);
    }
    if ((st = cuda_check(cudaGetLastError(), "k_split_rows launch"))) return st;
    // projection C[p][2b + t] = <beta_p | psi_b>, split over K
    const size_t ldc_p = (size_t)L.ntile_p * L.bn_p;
    if ((st = gemm_launch<0>(betaK, psiX, L.nkt_p, L.bn_p, nproj, 2 * nb, L.mtile_p, L.ntile_p, L.splits, part, ldc_p,
                             L.zstride, false, err, s)))
        return st;
    const int Z = [&] {
        const int per = (L.nkt_p + L.splits - 1) / L.splits;
        return (L.nkt_p + per - 1) / per;
    }();
    float* Pd = (float*)(w + L.pd_off);
    {
        ProfScope pf(PF_SPLIT, s);
        k_reduce_p<<<grid_for((long)nproj * 2 * nb), 256, 0, s>>>(part, Z, L.zstride, (int)ldc_p, nproj, 2 * nb, D, Pd);
    }
    if ((st = cuda_check(cudaGetLastError(), "k_reduce_p launch"))) return st;
    {
        ProfScope pf(PF_SPLIT, s);
        const long n = (long)L.mtile_a * TM * L.nkt_a * (KT / 8);
        k_expand_e<<<grid_for(n), 256, 0, s>>>(Pd, nproj, nb, L.mtile_a * TM, L.nkt_a, E);
    }
    if ((st = cuda_check(cudaGetLastError(), "k_expand_e launch"))) return st;
    // application out[b][g] (+)= sum_p beta[p][g] D_p P[p][b]
    return gemm_launch<1>(E, betaT, L.nkt_a, kAppBN, 2 * nb, npw, L.mtile_a, L.ntile_a, 1, (float*)out, (size_t)ld_out,
                          0, accumulate, err, s);
}

}  // namespace qm

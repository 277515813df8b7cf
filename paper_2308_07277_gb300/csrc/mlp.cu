// Learned preconditioner of the Davidson correction step: a 3 -> 64 -> 64 -> 1 network K(f) > 0
// on per-plane-wave features replaces the Teter-Payne-Allan factor, delta_n(G) = K(f_nG) r_n(G).
//
// Network: z1 = W1 f + b1, h1 = silu(z1), z2 = W2 h1 + b2, h2 = silu(z2), z3 = w3.h2 + b3,
// K = K_TPA(x) softplus(z3) / log 2: a positive factor on the TPA curve of the plane wave
// (z3 = 0 gives TPA exactly); parameters one flat FP32 vector (layout in include/qm.h).  Arithmetic is
// BF16 x BF16 with FP32 accumulation: weights, features, hidden activations and the backward
// pass's deltas are rounded to BF16 before every product; sums, activation functions and the
// loss are FP32.
// Features (scale-free): x = T_G / T_n, e = eps_n / T_n, d = (H_GG - eps_n) / T_n (H_GG the
// diagonal of H(k) in the plane-wave basis).
//
// Kernels
//   k_mlp_infer   inference with the 64 x 64 layer on the tensor cores: a CTA of 4 warps takes
//                 128 samples per tile, forms h1 in registers and writes it to shared memory as
//                 the BF16 A operand (K-major core matrices), one thread issues
//                 tcgen05.mma (M = 128, N = 64, K = 4 x 16) against W2 (B operand, resident in
//                 shared memory) into a 64-column FP32 accumulator in tensor memory, and every
//                 thread reads its sample's row back with tcgen05.ld for the output layer
//   k_mlp_grad    training: forward and backward of 128-sample tiles with the three 64 x 64
//                 contractions (z2, dz1 and the weight gradient, which also carries the bias and
//                 first-layer gradients) as tcgen05 products; per-CTA gradient partials are
//                 reduced in a fixed order
//   k_mlp_pairs   training samples from Ritz pairs and exact corrections
//   k_mlp_adam    Adam update (Kingma & Ba, ICLR 2015)
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "qm_internal.h"
#include "tc_util.cuh"

namespace qm {
namespace {

constexpr int kH = 64;
constexpr int kOffW1 = 0, kOffB1 = 192, kOffW2 = 256, kOffB2 = 4352, kOffW3 = 4416, kOffB3 = 4480;
constexpr int kNP = 4481;
static_assert(kNP == QM_MLP_NPARAM, "parameter count");
constexpr long kSpin = 1L << 26;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float silu_d(float z) {
    const float s = sigm(z);
    return s * (1.f + z * (1.f - s));
}
__device__ __forceinline__ float softplus(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }
constexpr float kInvLog2 = 1.44269504088896340736f;  // 1 / log 2
// Teter-Payne-Allan factor (27+18x+12x^2+8x^3)/(27+18x+12x^2+8x^3+16x^4) (Phys. Rev. B 40, 12255)
__device__ __forceinline__ float tpa(float x) {
    const float num = 27.f + x * (18.f + x * (12.f + 8.f * x));
    const float x2 = x * x;
    return num / (num + 16.f * x2 * x2);
}

// features of one plane wave (shared by the sample generator and the Davidson correction):
// x = T_G / T_n, e = eps_n / T_n, d = (H_GG - eps_n) / T_n with H_GG the Hamiltonian's diagonal
__device__ __forceinline__ void mlp_feat(double kin, double inv_t, double eps, double hdiag, float f[3]) {
    f[0] = (float)(kin * inv_t);
    f[1] = (float)(eps * inv_t);
    f[2] = (float)((hdiag - eps) * inv_t);
}

// ---------------------------------------------------------------- inference (tensor cores)
constexpr int kMT = 128;  // samples per tile = TMEM lanes
constexpr uint32_t kIdesc = tc::idesc_bf16(128, kH);

// byte offset of element (row, k) of a K-major no-swizzle operand with 64 K columns
__device__ __forceinline__ int cm_off(int row, int k) { return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2; }

struct FeatArray {  // features given as (n, 3) rows; output K
    const float* feats;
    float* K;
    long n;
    __device__ __forceinline__ long ntiles() const { return (n + kMT - 1) / kMT; }
    __device__ __forceinline__ bool load(long tile, int tid, float f[3]) const {
        const long s = tile * kMT + tid;
        if (s >= n) return false;
        f[0] = feats[3 * s];
        f[1] = feats[3 * s + 1];
        f[2] = feats[3 * s + 2];
        return true;
    }
    __device__ __forceinline__ void store(long tile, int tid, float k) const { K[tile * kMT + tid] = k; }
};

struct DavidsonCorr {  // out_j(G) = K r_{sel[j]}(G), features from the residual block
    const double2* R;
    int ld, npw, nu;
    const int* sel;
    const double *tk, *eps, *hdiag, *kin;
    double2* out;
    int ldo;
    __device__ __forceinline__ long tiles_per_band() const { return (npw + kMT - 1) / kMT; }
    __device__ __forceinline__ long ntiles() const { return tiles_per_band() * nu; }
    __device__ __forceinline__ bool load(long tile, int tid, float f[3]) const {
        const long tpb = tiles_per_band();
        const int j = (int)(tile / tpb);
        const int g = (int)(tile - (long)j * tpb) * kMT + tid;
        if (g >= npw) return false;
        const int n = sel ? __ldg(sel + j) : j;  // sel == NULL: row j is band j
        const double t = __ldg(tk + n);
        mlp_feat(__ldg(kin + g), 1.0 / t, __ldg(eps + n), __ldg(hdiag + g), f);
        return true;
    }
    __device__ __forceinline__ void store(long tile, int tid, float k) const {
        const long tpb = tiles_per_band();
        const int j = (int)(tile / tpb);
        const int g = (int)(tile - (long)j * tpb) * kMT + tid;
        const double2 r = R[(size_t)(sel ? __ldg(sel + j) : j) * ld + g];
        out[(size_t)j * ldo + g] = make_double2((double)k * r.x, (double)k * r.y);
    }
};

template <class Src>
__global__ void __launch_bounds__(kMT) k_mlp_infer(Src src, const float* __restrict__ theta, int* __restrict__ err) {
    __shared__ __align__(1024) unsigned char sA[kMT * kH * 2];  // h1, BF16, 128 x 64 K-major
    __shared__ __align__(1024) unsigned char sB[kH * kH * 2];   // W2, BF16, 64 x 64 K-major
    __shared__ float sW1[kH * 3], sb1[kH], sb2[kH], sw3[kH];
    __shared__ float sb3;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         tc::smem_u32(&tmem_base)),
                     "r"(kH));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        sb3 = bf16r(theta[kOffB3]);
    }
    for (int i = tid; i < kH * 3; i += kMT) sW1[i] = bf16r(theta[kOffW1 + i]);
    for (int i = tid; i < kH; i += kMT) {
        sb1[i] = bf16r(theta[kOffB1 + i]);
        sb2[i] = bf16r(theta[kOffB2 + i]);
        sw3[i] = bf16r(theta[kOffW3 + i]);
    }
    for (int e = tid; e < kH * kH; e += kMT) {
        const int j = e >> 6, i = e & 63;  // W2[j][i]: B row j (output), K column i (input)
        *reinterpret_cast<__nv_bfloat16*>(sB + cm_off(j, i)) = __float2bfloat16_rn(theta[kOffW2 + e]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    const long nt = src.ntiles();
    for (long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        float f[3];
        const bool valid = src.load(tile, tid, f);
        if (!valid) f[0] = f[1] = f[2] = 0.f;
        const float x = f[0];
        f[0] = bf16r(f[0]);
        f[1] = bf16r(f[1]);
        f[2] = bf16r(f[2]);
        // layer 1 and the A operand row of this sample (8 x 16-byte chunks)
#pragma unroll
        for (int kc = 0; kc < kH / 8; ++kc) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float h[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int j = kc * 8 + 2 * q + t;
                    const float z = sb1[j] + sW1[3 * j] * f[0] + sW1[3 * j + 1] * f[1] + sW1[3 * j + 2] * f[2];
                    h[t] = silu(z);
                }
                w[q] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(h[0])) |
                       ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(h[1])) << 16);
            }
            *reinterpret_cast<uint4*>(sA + cm_off(tid, kc * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
            for (int ks = 0; ks < kH / 16; ++ks) {
                const uint64_t da = tc::sdesc(tc::smem_u32(sA) + ks * 256, 128, 1024);
                const uint64_t db = tc::sdesc(tc::smem_u32(sB) + ks * 256, 128, 1024);
                const uint32_t acc = ks > 0 ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                tc::smem_u32(&mbar)));
        }
        const bool ok = tc::mbar_wait(tc::smem_u32(&mbar), phase, kSpin);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {  // uniform: every thread leaves the loop together
            if (tid == 0) atomicExch(err, 1);
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        float z3 = sb3;
#pragma unroll
        for (int c0 = 0; c0 < kH; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) z3 += sw3[c0 + q] * bf16r(silu(__uint_as_float(v[q]) + sb2[c0 + q]));
        }
        if (valid) src.store(tile, tid, tpa(x) * softplus(z3) * kInvLog2);
        // the next tile's products overwrite the accumulator: every read must be done
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kH));
}

int infer_grid(long ntiles) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (int)std::max<long>(1, std::min<long>(ntiles, (long)nsm * 8));
}

// ---------------------------------------------------------------- training (tensor cores)
// Forward and backward pass of a tile of 128 samples (one per thread, one per TMEM lane) with
// the three 64 x 64 contractions on the tensor cores (BF16 operands, FP32 accumulators):
//   MMA1  z2 - b2 = h1 W2^T      M = 128 samples, N = 64, K = 64   (A = h1,  B = W2)
//   MMA2  dz1 / silu'(z1) = dz2 W2                                  (A = dz2, B = W2^T)
//   MMA3  G += Amat Bmat^T over the tile's samples, accumulated in tensor memory across tiles:
//         Amat rows 0..63 = dz2^T, rows 64..127 = dz1^T (K = 128 samples);
//         Bmat rows 0..63 = h1^T, row 64 = ones, rows 65..67 = f^T, rows 68..79 zero (N = 80), so
//         G[j][i] = dW2[j][i], G[j][64] = db2[j], G[64+j][64] = db1[j], G[64+j][65+k] = dW1[j][k].
// dw3 and db3 are per-tile column sums on the CUDA cores.  dz2 and dz1 are rounded to BF16
// before their products, like every other operand.
constexpr int kGN3 = 80;                             // N of MMA3
constexpr int kGStride = kH + 1;                     // padded row of h2 (floats, odd: no bank conflicts)
constexpr uint32_t kIdesc3 = tc::idesc_bf16(128, kGN3);
constexpr size_t kGradSmem = 2 * 16384 + 2 * 8192 + 32768 + 20480 + sizeof(float) * (kMT * kGStride + kMT + kH * 3 +
                                                                                    3 * kH + 4);

// byte offset of element (row, k) of a K-major no-swizzle operand with 128 K columns
__device__ __forceinline__ int cm_off128(int row, int k) {
    return (row >> 3) * 2048 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ void put_bf16(unsigned char* base, int off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t v[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
// one thread issues nks K-steps of 16 (operands K-major, 8-row groups sbo bytes apart) and
// commits them to the mbarrier
__device__ __forceinline__ void mma_issue(uint32_t d, uint32_t a, uint32_t b, uint32_t sbo, int nks, uint32_t idesc,
                                          bool accumulate, uint32_t mbar) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    for (int ks = 0; ks < nks; ++ks) {
        const uint64_t da = tc::sdesc(a + ks * 256, 128, sbo);
        const uint64_t db = tc::sdesc(b + ks * 256, 128, sbo);
        const uint32_t acc = (accumulate || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar));
}
// shared-memory writes by the threads -> visible to the tensor core, then one thread issues
__device__ __forceinline__ void to_async_proxy_and_sync() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
}

// Cosine-loss gradient of every tile of the CTA (grid-stride), given per-band coefficients:
// per-CTA partials to gpart[blockIdx.x][kNP].  128 threads; a bounded wait that expires sets
// *err and ends the CTA (its partials are then not written).
__global__ void __launch_bounds__(kMT, 1)
k_mlp_grad(long n, const float* __restrict__ feats, const float* __restrict__ theta, const int* __restrict__ band_of,
           const float* __restrict__ r2, const float* __restrict__ cc, const float* __restrict__ coef,
           const float* __restrict__ ratio, float* __restrict__ gpart, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char dsm[];
    unsigned char* sA1 = dsm;              // h1, 128 x 64
    unsigned char* sA2 = sA1 + 16384;      // dz2, 128 x 64
    unsigned char* sW2 = sA2 + 16384;      // W2 as the B operand of MMA1 (rows j, K = i)
    unsigned char* sW2t = sW2 + 8192;      // W2^T as the B operand of MMA2 (rows i, K = j)
    unsigned char* sA3 = sW2t + 8192;      // Amat of MMA3, 128 x 128
    unsigned char* sB3 = sA3 + 32768;      // Bmat of MMA3, 80 x 128
    float* sH2 = reinterpret_cast<float*>(sB3 + 20480);  // h2 [sample][kGStride]
    float* sDz3 = sH2 + kMT * kGStride;
    float* sW1 = sDz3 + kMT;
    float* sb1 = sW1 + kH * 3;
    float* sb2 = sb1 + kH;
    float* sw3 = sb2 + kH;
    float* sb3 = sw3 + kH;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         tc::smem_u32(&tmem_base)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc::smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        *sb3 = bf16r(theta[kOffB3]);
    }
    for (int i = tid; i < kH * 3; i += kMT) sW1[i] = bf16r(theta[kOffW1 + i]);
    for (int i = tid; i < kH; i += kMT) {
        sb1[i] = bf16r(theta[kOffB1 + i]);
        sb2[i] = bf16r(theta[kOffB2 + i]);
        sw3[i] = bf16r(theta[kOffW3 + i]);
    }
    for (int e = tid; e < kH * kH; e += kMT) {
        const int j = e >> 6, i = e & 63;
        const float w = theta[kOffW2 + e];
        put_bf16(sW2, cm_off(j, i), w);
        put_bf16(sW2t, cm_off(i, j), w);
    }
    for (int r = 64; r < kGN3; ++r) put_bf16(sB3, cm_off128(r, tid), r == 64 ? 1.f : 0.f);  // ones, f (per tile), zeros
    to_async_proxy_and_sync();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const uint32_t mb = tc::smem_u32(&mbar);
    uint32_t phase = 0;
    float gw3 = 0.f;  // thread j < 64: dw3[j]; thread 64: db3
    bool aborted = false;
    int tiles = 0;
    const long nt = (n + kMT - 1) / kMT;
    for (long tile = blockIdx.x; tile < nt; tile += gridDim.x, ++tiles) {
        const long s = tile * kMT + tid;
        const bool valid = s < n;
        float f[3] = {0.f, 0.f, 0.f};
        if (valid) {
            f[0] = feats[3 * s];
            f[1] = feats[3 * s + 1];
            f[2] = feats[3 * s + 2];
        }
        const float t = valid ? tpa(f[0]) * kInvLog2 : 0.f;  // unrounded x
        f[0] = bf16r(f[0]);
        f[1] = bf16r(f[1]);
        f[2] = bf16r(f[2]);
        // layer 1: h1 row of this sample into MMA1's A operand and column `tid` of Bmat
#pragma unroll
        for (int kc = 0; kc < kH / 8; ++kc) {
            float h[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = kc * 8 + q;
                h[q] = bf16r(silu(sb1[j] + sW1[3 * j] * f[0] + sW1[3 * j + 1] * f[1] + sW1[3 * j + 2] * f[2]));
                put_bf16(sB3, cm_off128(j, tid), h[q]);
            }
            *reinterpret_cast<uint4*>(sA1 + cm_off(tid, kc * 8)) =
                make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) put_bf16(sB3, cm_off128(65 + k, tid), f[k]);
        to_async_proxy_and_sync();
        if (tid == 0) mma_issue(tmem, tc::smem_u32(sA1), tc::smem_u32(sW2), 1024, kH / 16, kIdesc, false, mb);
        bool ok = tc::mbar_wait(mb, phase, kSpin);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            aborted = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        // layer 2 and output from z2 - b2 (tensor memory columns 0..63)
        float z3 = *sb3;
#pragma unroll
        for (int c0 = 0; c0 < kH; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + lane_off + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float h2 = bf16r(silu(__uint_as_float(v[q]) + sb2[c0 + q]));
                sH2[tid * kGStride + c0 + q] = h2;
                z3 += sw3[c0 + q] * h2;
            }
        }
        float dz3 = 0.f;
        if (valid) {
            const int b = band_of[s];
            const float K = t * softplus(z3);
            dz3 = coef[b] * (ratio[b] * K * r2[s] - cc[s]) * t * sigm(z3);
        }
        sDz3[tid] = dz3;
        // dz2 = dz3 w3 silu'(z2): A operand of MMA2 (row tid) and rows 0..63 of Amat (column tid)
#pragma unroll
        for (int c0 = 0; c0 < kH; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + lane_off + (uint32_t)c0, v);
            float d[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                d[q] = bf16r(dz3 * sw3[c0 + q] * silu_d(__uint_as_float(v[q]) + sb2[c0 + q]));
                put_bf16(sA3, cm_off128(c0 + q, tid), d[q]);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
                *reinterpret_cast<uint4*>(sA2 + cm_off(tid, c0 + 8 * h)) =
                    make_uint4(pack_bf16(d[8 * h], d[8 * h + 1]), pack_bf16(d[8 * h + 2], d[8 * h + 3]),
                               pack_bf16(d[8 * h + 4], d[8 * h + 5]), pack_bf16(d[8 * h + 6], d[8 * h + 7]));
        }
        to_async_proxy_and_sync();
        if (tid == 0) mma_issue(tmem + 64, tc::smem_u32(sA2), tc::smem_u32(sW2t), 1024, kH / 16, kIdesc, false, mb);
        // dw3, db3 of this tile while the tensor core works (h2 and dz3 are complete)
        if (tid < kH) {
            float a = 0.f;
            for (int q = 0; q < kMT; ++q) a += sDz3[q] * sH2[q * kGStride + tid];
            gw3 += a;
        } else if (tid == kH) {
            float a = 0.f;
            for (int q = 0; q < kMT; ++q) a += sDz3[q];
            gw3 += a;
        }
        ok = tc::mbar_wait(mb, phase, kSpin);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            aborted = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        // dz1 = (dz2 W2) silu'(z1): rows 64..127 of Amat (column tid)
#pragma unroll
        for (int c0 = 0; c0 < kH; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + lane_off + 64u + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = c0 + q;
                const float z1 = sb1[i] + sW1[3 * i] * f[0] + sW1[3 * i + 1] * f[1] + sW1[3 * i + 2] * f[2];
                put_bf16(sA3, cm_off128(64 + i, tid), __uint_as_float(v[q]) * silu_d(z1));
            }
        }
        to_async_proxy_and_sync();
        if (tid == 0)
            mma_issue(tmem + 128, tc::smem_u32(sA3), tc::smem_u32(sB3), 2048, kMT / 16, kIdesc3, tiles > 0, mb);
        // the next tile overwrites the operands: wait for MMA3 here
        ok = tc::mbar_wait(mb, phase, kSpin);
        phase ^= 1u;
        if (!__syncthreads_and(ok)) {
            aborted = true;
            break;
        }
    }
    if (aborted) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        float* g = gpart + (size_t)blockIdx.x * kNP;
        if (tiles == 0) {
            for (int e = tid; e < kNP; e += kMT) g[e] = 0.f;
        } else {
            // row tid of G: dW2 row j (tid < 64) with db2[j]; db1 and dW1 row j (tid = 64 + j)
#pragma unroll 1
            for (int c0 = 0; c0 < kGN3; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + lane_off + 128u + (uint32_t)c0, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = c0 + q;
                    const float x = __uint_as_float(v[q]);
                    if (tid < kH) {
                        if (col < kH) g[kOffW2 + tid * kH + col] = x;
                        else if (col == kH) g[kOffB2 + tid] = x;
                    } else {
                        const int j = tid - kH;
                        if (col == kH) g[kOffB1 + j] = x;
                        else if (col > kH && col <= kH + 3) g[kOffW1 + 3 * j + (col - kH - 1)] = x;
                    }
                }
            }
            if (tid < kH) g[kOffW3 + tid] = gw3;
            if (tid == kH) g[kOffB3] = gw3;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256));
}

// per band: A = sum K^2 r2, B = sum K c over its samples (FP64 sums in a fixed order)
__global__ void k_mlp_band_ab(const long long* __restrict__ off, const float* __restrict__ K, const float* __restrict__ r2,
                              const float* __restrict__ cc, double* __restrict__ A, double* __restrict__ B) {
    const int b = blockIdx.x;
    double a = 0.0, bb = 0.0;
    for (long long s = off[b] + threadIdx.x; s < off[b + 1]; s += blockDim.x) {
        const double k = K[s];
        a += k * k * r2[s];
        bb += k * cc[s];
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = bb;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + st];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + st];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        A[b] = sh[0][0];
        B[b] = sh[1][0];
    }
}

// loss = sum_b W_b (1 - B^2/(A D)) / sum_b W_b over bands with D > 0 and A > 0 (W = NULL: 1);
// dL/dK_s = coef_b (ratio_b K r2 - c)
__global__ void k_mlp_coef(int nband, const double* __restrict__ A, const double* __restrict__ B,
                           const float* __restrict__ D, const float* __restrict__ W, float* __restrict__ coef,
                           float* __restrict__ ratio, double* __restrict__ loss) {
    __shared__ double sl[256], sw[256];
    double l = 0.0, wsum = 0.0;
    for (int b = threadIdx.x; b < nband; b += blockDim.x) {
        if (D[b] > 0.f && A[b] > 0.0) {
            const double w = W ? (double)W[b] : 1.0;
            l += w * (1.0 - B[b] * B[b] / (A[b] * D[b]));
            wsum += w;
        }
    }
    sl[threadIdx.x] = l;
    sw[threadIdx.x] = wsum;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            sl[threadIdx.x] += sl[threadIdx.x + st];
            sw[threadIdx.x] += sw[threadIdx.x + st];
        }
        __syncthreads();
    }
    const double wt = sw[0];
    for (int b = threadIdx.x; b < nband; b += blockDim.x) {
        const bool use = D[b] > 0.f && A[b] > 0.0 && wt > 0.0;
        const double w = W ? (double)W[b] : 1.0;
        coef[b] = use ? (float)(w * 2.0 * B[b] / (A[b] * D[b]) / wt) : 0.f;
        ratio[b] = use ? (float)(B[b] / A[b]) : 0.f;
    }
    if (threadIdx.x == 0) *loss = wt > 0.0 ? sl[0] / wt : 0.0;
}

// W_n = ||r_n||^2 / sum_m ||r_m||^2 over the bands with D > 0 (W_n = 0 where D_n = 0)
__global__ void k_mlp_wnorm(int n, const float* __restrict__ D, float* __restrict__ W) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        if (D[b] > 0.f) s += W[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    const double tot = sh[0];
    for (int b = threadIdx.x; b < n; b += blockDim.x) W[b] = (D[b] > 0.f && tot > 0.0) ? (float)(W[b] / tot) : 0.f;
}

__global__ void k_mlp_reduce_grad(const float* __restrict__ gpart, int nblk, float* __restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNP) return;
    float a = 0.f;
    for (int b = 0; b < nblk; ++b) a += gpart[(size_t)b * kNP + e];
    grad[e] = a;
}

__global__ void k_mlp_band_of(const long long* __restrict__ off, int nband, int* __restrict__ band_of) {
    const int b = blockIdx.x;
    if (b >= nband) return;
    for (long long s = off[b] + threadIdx.x; s < off[b + 1]; s += blockDim.x) band_of[s] = b;
}

__global__ void k_mlp_adam(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr_t, float b1, float b2, float eps) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNP) return;
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    theta[e] -= lr_t * me / (sqrtf(ve) + eps);
}

// ---------------------------------------------------------------- training samples
// band n's cluster: exact eigenvalue n and its partners within tol; zero S[m][n] outside it
__global__ void k_mlp_cluster(const double* __restrict__ lam, int nu, int nb, double tol, double2* __restrict__ S,
                              int lds, int* __restrict__ ok) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nb) return;
    if (n >= nu) {  // no exact pair for this band
        ok[n] = 0;
        return;
    }
    const int m0 = n;
    int lo = m0, hi = m0;
    while (lo > 0 && fabs(lam[lo - 1] - lam[m0]) <= tol) --lo;
    while (hi < nu - 1 && fabs(lam[hi + 1] - lam[m0]) <= tol) ++hi;
    ok[n] = hi < nu - 1 ? 1 : 0;
    for (int m = 0; m < nu; ++m)
        if (m < lo || m > hi) S[(size_t)m * lds + n] = make_double2(0.0, 0.0);
}

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[256]) {
#pragma unroll
    for (int a = 0; a < NV; ++a) sh[a][threadIdx.x] = v[a];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
#pragma unroll
            for (int a = 0; a < NV; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + st];
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = sh[a][0];
    __syncthreads();
}

// one CTA per band: r = H psi - eps psi, delta* = P/(psi^H P) - psi (P = P_c psi), features,
// |r|^2, Re(conj(r) delta*) and ||delta*||^2 (0 if the band's cluster is incomplete)
__global__ void __launch_bounds__(256)
k_mlp_pairs(const double2* __restrict__ psi, int ldp, const double2* __restrict__ hpsi, int ldh,
            const double* __restrict__ eps, const double2* __restrict__ P, const int* __restrict__ ok,
            const double* __restrict__ kin, const double* __restrict__ hdiag, int npw, float* __restrict__ feats,
            float* __restrict__ r2, float* __restrict__ cc, float* __restrict__ D, float* __restrict__ W) {
    __shared__ double sh[4][256];
    const int n = blockIdx.x;
    const double e = eps[n];
    const double2* x = psi + (size_t)n * ldp;
    const double2* hx = hpsi + (size_t)n * ldh;
    const double2* p = P + (size_t)n * npw;
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // |psi|^2, kin |psi|^2, |r|^2, Re psi^H P
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const double2 a = x[g], h = hx[g], q = p[g];
        const double rx = h.x - e * a.x, ry = h.y - e * a.y;
        const double w = a.x * a.x + a.y * a.y;
        v[0] += w;
        v[1] += kin[g] * w;
        v[2] += rx * rx + ry * ry;
        v[3] += a.x * q.x + a.y * q.y;
    }
    block_sum<4>(v, sh);
    const double inv_t = v[0] / v[1], is = 1.0 / v[3];
    double d[1] = {0.0};
    const bool keep = ok[n] != 0;  // an incomplete cluster: no target (delta* = 0)
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
        const double2 a = x[g], h = hx[g], q = p[g];
        const double rx = h.x - e * a.x, ry = h.y - e * a.y;
        const double dx = keep ? q.x * is - a.x : 0.0, dy = keep ? q.y * is - a.y : 0.0;
        const size_t s = (size_t)n * npw + g;
        float f[3];
        mlp_feat(kin[g], inv_t, e, hdiag[g], f);
        feats[3 * s] = f[0];
        feats[3 * s + 1] = f[1];
        feats[3 * s + 2] = f[2];
        r2[s] = (float)(rx * rx + ry * ry);
        cc[s] = (float)(rx * dx + ry * dy);
        d[0] += dx * dx + dy * dy;
    }
    block_sum<1>(d, sh);
    if (threadIdx.x == 0) {
        D[n] = (float)d[0];
        W[n] = (float)v[2];  // ||r_n||^2, normalised over the call's bands by k_mlp_wnorm
    }
}

}  // namespace

qm_status mlp_precond_apply(const float* theta, const double2* R, int ld, int npw, const int* sel, int nu,
                            const double* tk, const double* eps, const double* hdiag, const double* kin, double2* out,
                            int ldo, int* err, cudaStream_t s) {
    DavidsonCorr src{R, ld, npw, nu, sel, tk, eps, hdiag, kin, out, ldo};
    const long nt = (long)((npw + kMT - 1) / kMT) * nu;
    ProfScope pf(PF_MLP, s);
    k_mlp_infer<DavidsonCorr><<<infer_grid(nt), kMT, 0, s>>>(src, theta, err);
    return cuda_check(cudaGetLastError(), "learned preconditioner launch");
}

}  // namespace qm

using namespace qm;

namespace {

struct DevBuf {
    void* p = nullptr;
    cudaStream_t s;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    qm_status get(size_t bytes) {
        return cuda_check(cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s), "cudaMallocAsync");
    }
    ~DevBuf() {
        if (p) cudaFreeAsync(p, s);
    }
};

int train_grid() {  // one gradient CTA per SM (its shared memory allows one)
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm;
}

// loss (device) and gradient (device) for one parameter vector
qm_status loss_grad_dev(int nband, const long long* off, const int* band_of, long n, const float* feats, const float* r2,
                        const float* cc, const float* D, const float* W, const float* theta, float* K, double* A, double* B,
                        float* coef, float* ratio, double* loss_dev, float* gpart, int nblk, float* grad, int* err,
                        cudaStream_t s) {
    qm_status st0 = allow_dynamic_smem((const void*)k_mlp_grad, kGradSmem, "network training shared memory");
    if (st0) return st0;
    {
        ProfScope pf(PF_MLP, s);
        FeatArray src{feats, K, n};
        k_mlp_infer<FeatArray><<<infer_grid((n + kMT - 1) / kMT), kMT, 0, s>>>(src, theta, err);
    }
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_band_ab<<<nband, 256, 0, s>>>(off, K, r2, cc, A, B);
    }
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_coef<<<1, 256, 0, s>>>(nband, A, B, D, W, coef, ratio, loss_dev);
    }
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_grad<<<nblk, kMT, kGradSmem, s>>>(n, feats, theta, band_of, r2, cc, coef, ratio, gpart, err);
    }
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_reduce_grad<<<(kNP + 255) / 256, 256, 0, s>>>(gpart, nblk, grad);
    }
    return cuda_check(cudaGetLastError(), "learned preconditioner training launch");
}

// the error word of the bounded tensor-core waits, read after the stream has drained
qm_status check_err_word(const int* err, cudaStream_t s, const char* what) {
    int e = 0;
    qm_status st;
    if ((st = cuda_check(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H error word")) ||
        (st = cuda_check(cudaStreamSynchronize(s), "stream sync")))
        return st;
    return e ? fail(QM_ERR_TIMEOUT, what) : QM_OK;
}

qm_status check_samples(int nband, const long long* band_off, long nsamples, const void* feats, const void* r2,
                        const void* c, const void* D, const void* theta) {
    if (nband < 1 || nsamples < 1) return fail(QM_ERR_ARG, "learned preconditioner: no samples");
    if (!band_off || !feats || !r2 || !c || !D || !theta) return fail(QM_ERR_ARG, "learned preconditioner: NULL argument");
    return QM_OK;
}

}  // namespace

extern "C" qm_status qm_mlp_forward(long long n, const float* feats, const float* theta, float* K, void* stream) {
    clear_error();
    if (n < 0 || (n > 0 && (!feats || !theta || !K))) return fail(QM_ERR_ARG, "qm_mlp_forward: bad arguments");
    if (n == 0) return QM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf err(s);
    qm_status st = err.get(sizeof(int));
    if (st) return st;
    if ((st = cuda_check(cudaMemsetAsync(err.p, 0, sizeof(int), s), "memset"))) return st;
    FeatArray src{feats, K, (long)n};
    const long nt = (n + kMT - 1) / kMT;
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_infer<FeatArray><<<infer_grid(nt), kMT, 0, s>>>(src, theta, (int*)err.p);
    }
    if ((st = cuda_check(cudaGetLastError(), "qm_mlp_forward launch"))) return st;
    int e = 0;
    if ((st = cuda_check(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H error word")) ||
        (st = cuda_check(cudaStreamSynchronize(s), "stream sync")))
        return st;
    return e ? fail(QM_ERR_TIMEOUT, "qm_mlp_forward: a bounded tensor-core wait expired") : QM_OK;
}

extern "C" qm_status qm_mlp_pairs(qm_gspace g, int ik, int n, const void* psi, int ld_psi, const void* hpsi,
                                  int ld_hpsi, const double* eps, const double* hdiag, int nu, const void* U, int ld_u,
                                  const double* lam, double cluster_tol, float* feats, float* r2, float* c, float* D,
                                  float* W, void* stream) {
    clear_error();
    if (!g || ik < 0 || ik >= g->nk) return fail(QM_ERR_ARG, "qm_mlp_pairs: bad gspace or ik");
    const int npw = g->k[ik].npw;
    if (n < 1 || nu < 1 || !psi || !hpsi || !eps || !hdiag || !U || !lam || !feats || !r2 || !c || !D || !W)
        return fail(QM_ERR_ARG, "qm_mlp_pairs: bad arguments");
    if (ld_psi < npw || ld_hpsi < npw || ld_u < npw) return fail(QM_ERR_ARG, "qm_mlp_pairs: leading dimension < npw");
    if (!(cluster_tol >= 0.0)) return fail(QM_ERR_ARG, "qm_mlp_pairs: cluster_tol < 0");
    qm_status st = ensure_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int splits = zgemm_cn_splits(nu, n, npw);
    DevBuf S(s), part(s), P(s), ok(s);
    if ((st = S.get(sizeof(double2) * (size_t)nu * n)) || (st = part.get(sizeof(double2) * (size_t)splits * nu * n)) ||
        (st = P.get(sizeof(double2) * (size_t)n * npw)) || (st = ok.get(sizeof(int) * (size_t)n)))
        return st;
    if ((st = zgemm_cn(nu, n, npw, (const double2*)U, ld_u, (const double2*)psi, ld_psi, (double2*)S.p, n,
                       (double2*)part.p, splits, s)))
        return st;
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_cluster<<<(n + 127) / 128, 128, 0, s>>>(lam, nu, n, cluster_tol, (double2*)S.p, n, (int*)ok.p);
    }
    if ((st = zgemm_tn(n, npw, nu, (const double2*)S.p, n, nullptr, (const double2*)U, ld_u, (double2*)P.p, npw, false,
                       s)))
        return st;
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_pairs<<<n, 256, 0, s>>>((const double2*)psi, ld_psi, (const double2*)hpsi, ld_hpsi, eps,
                                      (const double2*)P.p, (const int*)ok.p, g->k[ik].kin, hdiag, npw, feats, r2, c,
                                      D, W);
    }
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_wnorm<<<1, 256, 0, s>>>(n, D, W);
    }
    if ((st = cuda_check(cudaGetLastError(), "qm_mlp_pairs launch"))) return st;
    return cuda_check(cudaStreamSynchronize(s), "stream sync");
}

extern "C" qm_status qm_mlp_loss_grad(int nband, const long long* band_off, const float* feats, const float* r2,
                                      const float* c, const float* D, const float* W, const float* theta, double* loss,
                                      float* grad, void* stream) {
    clear_error();
    if (!grad || !loss) return fail(QM_ERR_ARG, "qm_mlp_loss_grad: NULL loss or grad");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<long long> hoff(2);
    qm_status st = check_samples(nband, band_off, 1, feats, r2, c, D, theta);
    if (st) return st;
    long long last = 0;
    if ((st = cuda_check(cudaMemcpy(&last, band_off + nband, sizeof(long long), cudaMemcpyDeviceToHost), "D2H offsets")))
        return st;
    const long n = (long)last;
    if (n < 1) return fail(QM_ERR_ARG, "qm_mlp_loss_grad: no samples");
    const int nblk = train_grid();
    DevBuf K(s), bo(s), A(s), B(s), co(s), ra(s), ld(s), gp(s), er(s);
    if ((st = K.get(sizeof(float) * n)) || (st = bo.get(sizeof(int) * n)) || (st = A.get(sizeof(double) * nband)) ||
        (st = B.get(sizeof(double) * nband)) || (st = co.get(sizeof(float) * nband)) ||
        (st = ra.get(sizeof(float) * nband)) || (st = ld.get(sizeof(double))) ||
        (st = gp.get(sizeof(float) * (size_t)nblk * kNP)) || (st = er.get(sizeof(int))))
        return st;
    if ((st = cuda_check(cudaMemsetAsync(er.p, 0, sizeof(int), s), "memset"))) return st;
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_band_of<<<nband, 256, 0, s>>>(band_off, nband, (int*)bo.p);
    }
    if ((st = loss_grad_dev(nband, band_off, (const int*)bo.p, n, feats, r2, c, D, W, theta, (float*)K.p,
                            (double*)A.p, (double*)B.p, (float*)co.p, (float*)ra.p, (double*)ld.p, (float*)gp.p, nblk,
                            grad, (int*)er.p, s)))
        return st;
    if ((st = cuda_check(cudaMemcpyAsync(loss, ld.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H loss")))
        return st;
    return check_err_word((const int*)er.p, s, "qm_mlp_loss_grad: a bounded tensor-core wait expired");
}

extern "C" qm_status qm_mlp_train(int nband, const long long* band_off, const float* feats, const float* r2,
                                  const float* c, const float* D, const float* W, float* theta, int steps, double lr,
                                  double* loss_history, void* stream) {
    clear_error();
    if (steps < 1 || !(lr > 0.0)) return fail(QM_ERR_ARG, "qm_mlp_train: steps < 1 or lr <= 0");
    cudaStream_t s = (cudaStream_t)stream;
    qm_status st = check_samples(nband, band_off, 1, feats, r2, c, D, theta);
    if (st) return st;
    long long last = 0;
    if ((st = cuda_check(cudaMemcpy(&last, band_off + nband, sizeof(long long), cudaMemcpyDeviceToHost), "D2H offsets")))
        return st;
    const long n = (long)last;
    if (n < 1) return fail(QM_ERR_ARG, "qm_mlp_train: no samples");
    const int nblk = train_grid();
    DevBuf K(s), bo(s), A(s), B(s), co(s), ra(s), lh(s), gp(s), gr(s), m(s), v(s), er(s);
    if ((st = K.get(sizeof(float) * n)) || (st = bo.get(sizeof(int) * n)) || (st = A.get(sizeof(double) * nband)) ||
        (st = B.get(sizeof(double) * nband)) || (st = co.get(sizeof(float) * nband)) ||
        (st = ra.get(sizeof(float) * nband)) || (st = lh.get(sizeof(double) * (steps + 1))) ||
        (st = gp.get(sizeof(float) * (size_t)nblk * kNP)) || (st = gr.get(sizeof(float) * kNP)) ||
        (st = m.get(sizeof(float) * kNP)) || (st = v.get(sizeof(float) * kNP)) || (st = er.get(sizeof(int))))
        return st;
    if ((st = cuda_check(cudaMemsetAsync(m.p, 0, sizeof(float) * kNP, s), "memset")) ||
        (st = cuda_check(cudaMemsetAsync(v.p, 0, sizeof(float) * kNP, s), "memset")) ||
        (st = cuda_check(cudaMemsetAsync(er.p, 0, sizeof(int), s), "memset")))
        return st;
    {
        ProfScope pf(PF_MLP, s);
        k_mlp_band_of<<<nband, 256, 0, s>>>(band_off, nband, (int*)bo.p);
    }
    const float b1 = 0.9f, b2 = 0.999f;
    for (int t = 1; t <= steps + 1; ++t) {
        // step t: loss and gradient at the current parameters (the last pass only records the loss)
        if ((st = loss_grad_dev(nband, band_off, (const int*)bo.p, n, feats, r2, c, D, W, theta, (float*)K.p,
                                (double*)A.p, (double*)B.p, (float*)co.p, (float*)ra.p, (double*)lh.p + (t - 1),
                                (float*)gp.p, nblk, (float*)gr.p, (int*)er.p, s)))
            return st;
        if (t > steps) break;
        const double lr_t = lr * std::sqrt(1.0 - std::pow((double)b2, t)) / (1.0 - std::pow((double)b1, t));
        {
            ProfScope pf(PF_MLP, s);
            k_mlp_adam<<<(kNP + 255) / 256, 256, 0, s>>>(theta, (const float*)gr.p, (float*)m.p, (float*)v.p,
                                                          (float)lr_t, b1, b2, 1e-8f);
        }
    }
    if (loss_history &&
        (st = cuda_check(cudaMemcpyAsync(loss_history, lh.p, sizeof(double) * (steps + 1), cudaMemcpyDeviceToHost, s),
                         "D2H loss history")))
        return st;
    return check_err_word((const int*)er.p, s, "qm_mlp_train: a bounded tensor-core wait expired");
}

// Plane-wave matrix elements of the GW module (Sec. 5, "gw" module, matrix_elements):
//
//     M_nn'(k, q, G) = <n k+q| exp(i(q+G).r) |n' k>,   |q+G|^2 / 2 <= E_eps,
//
// by the paper's real-space route: both sets of states to real space on the FFT grid, the
// pairwise product, one forward transform per pair onto the sphere of q.  It reuses the
// stick-pruned FFT kernels of the H psi path:
//   k_stick_inverse (sphere -> x-transformed sticks) + k_plane_real (inverse y on the active
//   rows, inverse z, the plane stored to HBM) for the left (k+q) and right (k) states;
//   k_plane_pair: one plane of the product u_n conj(u_n') (the digit-reversed positions of both
//   factors coincide, so the product needs no reordering), forward z, forward y on the rows of
//   the q sphere, compacted onto its sticks;
//   k_stick_mel: forward x and the gather onto the q sphere, M = conj(F) / N_r.
// With u(r_j) = sum_G c(G) exp(iG.r_j) and the forward transform F[f](G) = sum_j f_j exp(-iG.r_j),
// N_r M(G) = sum_j conj(u_n(r_j)) u_n'(r_j) exp(+iG.r_j) = conj(F[u_n conj(u_n')](G)).
// Kernels and the launch sequence, compiled once per precision with the FFT path's kernels
// (fft_f32.cu, fft_f64.cu), so that every stick-pruned FFT kernel has one instantiation.
#pragma once
#include <cmath>
#include <cstdint>

#include "fft_kernels.cuh"

namespace qm {

// inverse y (active rows) and z of one plane of x-transformed sticks, stored whole:
// U[b][p1][p3 * N2 + p2] (all positions digit-reversed, as the FFT path leaves them)
template <class R, bool FUSED>
__global__ void __launch_bounds__(kThreads, fft_min_ctas<R, FUSED>())
k_plane_real(const typename Cx<R>::T* __restrict__ T, int nstick, int nstick_pad, const int* __restrict__ stick_plane,
             const int* __restrict__ rows, int nrow, const __grid_constant__ AxisPlan py,
             const __grid_constant__ AxisPlan pz, const typename Cx<R>::T* __restrict__ tw_y,
             const typename Cx<R>::T* __restrict__ tw_z, int ldy, int N1, typename Cx<R>::T* __restrict__ U) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N2 = py.n, N3 = pz.n;
    C* plane = reinterpret_cast<C*>(smem_raw);
    C* twy = plane + N3 * ldy;
    C* twz = twy + N2;
    int* srow = reinterpret_cast<int*>(twz + N3);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int p1 = blockIdx.x, b = blockIdx.y;
    for (int i = tid; i < N2; i += nt) twy[i] = tw_y[i];
    for (int i = tid; i < N3; i += nt) twz[i] = tw_z[i];
    for (int i = tid; i < nrow; i += nt) srow[i] = __ldg(rows + i);
    for (int i = tid; i < N3 * ldy; i += nt) plane[i] = mk<C>(0, 0);
    __syncthreads();
    const C* Tp = T + ((size_t)b * N1 + p1) * nstick_pad;
    for (int s = tid; s < nstick; s += nt) plane[__ldg(stick_plane + s)] = Tp[s];
    __syncthreads();
    if constexpr (FUSED) {
        fft2_lines<C, +1, true, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
        fft2_lines<C, +1, true, true>(plane, ldy, 1, N2, nullptr, pz, twz, tid, nt);
    } else {
        fft_lines<C, +1, true, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
        fft_lines<C, +1, true, true>(plane, ldy, 1, N2, nullptr, pz, twz, tid, nt);
    }
    C* Up = U + ((size_t)b * N1 + p1) * ((size_t)N3 * N2);
    const RDiv d2{N2, 1.0f / (float)N2};
    for (int i = tid; i < N3 * N2; i += nt) {
        const int p3 = d2.div(i), p2 = i - p3 * N2;
        Up[i] = plane[p3 * ldy + p2];
    }
}

// one plane of the product u_n conj(u_n') of pair (n, n') = (pair / nr, pair % nr), forward z,
// forward y on the rows of the q sphere, compacted onto its sticks: Te[j][p1][s]
template <class R, bool FUSED>
__global__ void __launch_bounds__(kThreads, fft_min_ctas<R, FUSED>())
k_plane_pair(const typename Cx<R>::T* __restrict__ UL, const typename Cx<R>::T* __restrict__ UR, int nr, int pair0,
             int nstick, int nstick_pad, const int* __restrict__ stick_plane, const int* __restrict__ rows, int nrow,
             const __grid_constant__ AxisPlan py, const __grid_constant__ AxisPlan pz,
             const typename Cx<R>::T* __restrict__ tw_y, const typename Cx<R>::T* __restrict__ tw_z, int ldy, int N1,
             typename Cx<R>::T* __restrict__ Te) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N2 = py.n, N3 = pz.n;
    C* plane = reinterpret_cast<C*>(smem_raw);
    C* twy = plane + N3 * ldy;
    C* twz = twy + N2;
    int* srow = reinterpret_cast<int*>(twz + N3);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int p1 = blockIdx.x, j = blockIdx.y;
    const int pair = pair0 + j;
    const int n = pair / nr, m = pair - n * nr;
    for (int i = tid; i < N2; i += nt) twy[i] = tw_y[i];
    for (int i = tid; i < N3; i += nt) twz[i] = tw_z[i];
    for (int i = tid; i < nrow; i += nt) srow[i] = __ldg(rows + i);
    const size_t nplane = (size_t)N3 * N2;
    const C* a = UL + ((size_t)n * N1 + p1) * nplane;
    const C* c = UR ? UR + ((size_t)m * N1 + p1) * nplane : nullptr;  // no right factor: the plane of UL
    const RDiv d2{N2, 1.0f / (float)N2};
    for (int i = tid; i < N3 * N2; i += nt) {
        const int p3 = d2.div(i), p2 = i - p3 * N2;
        const C x = a[i], y = c ? c[i] : mk<C>(1, 0);
        plane[p3 * ldy + p2] = mk<C>(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y);  // x conj(y)
    }
    __syncthreads();
    if constexpr (FUSED) {
        fft2_lines<C, -1, false, true>(plane, ldy, 1, N2, nullptr, pz, twz, tid, nt);
        fft2_lines<C, -1, false, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
    } else {
        fft_lines<C, -1, false, true>(plane, ldy, 1, N2, nullptr, pz, twz, tid, nt);
        fft_lines<C, -1, false, false>(plane, 1, ldy, nrow, srow, py, twy, tid, nt);
    }
    C* Tp = Te + ((size_t)j * N1 + p1) * nstick_pad;
    for (int s = tid; s < nstick; s += nt) Tp[s] = plane[__ldg(stick_plane + s)];
}

// forward x on the q sphere's sticks and the gather M[j][g] = conj(F(G)) / N_r (conj_out = 0:
// F(G) / N_r, the Fourier coefficient of a function given in real space)
template <class R, bool FUSED>
__global__ void __launch_bounds__(kThreads, fft_min_ctas<R, FUSED>())
k_stick_mel(const typename Cx<R>::T* __restrict__ Te, int nstick, int nstick_pad, const int* __restrict__ stick_g0,
            const int2* __restrict__ g_code, const __grid_constant__ AxisPlan px,
            const typename Cx<R>::T* __restrict__ tw_x, int ldx, R inv_nr, typename Cx<R>::T* __restrict__ M,
            int ld_m, int conj_out) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* lines = reinterpret_cast<C*>(smem_raw);
    C* tw = lines + sticks_per_cta<R>() * ldx;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int j = blockIdx.y;
    const int s0 = blockIdx.x * sticks_per_cta<R>();
    const int ns = min(sticks_per_cta<R>(), nstick - s0);
    const int N1 = px.n;
    for (int i = tid; i < N1; i += nt) tw[i] = tw_x[i];
    const C* src = Te + (size_t)j * N1 * nstick_pad + s0;
    for (int i = tid; i < N1 * ns; i += nt) {
        const int p = i / ns, l = i - p * ns;
        lines[l * ldx + p] = src[(size_t)p * nstick_pad + l];
    }
    __syncthreads();
    if constexpr (FUSED)
        fft2_lines<C, -1, false, false>(lines, 1, ldx, ns, nullptr, px, tw, tid, nt);
    else
        fft_lines<C, -1, false, false>(lines, 1, ldx, ns, nullptr, px, tw, tid, nt);
    const int gb = __ldg(stick_g0 + s0), ge = __ldg(stick_g0 + s0 + ns);
    C* out = M + (size_t)j * ld_m;
    for (int g = gb + tid; g < ge; g += nt) {
        const int2 cd = __ldg(g_code + g);
        const C x = lines[(cd.x - s0) * ldx + cd.y];
        out[g] = mk<C>(x.x * inv_nr, conj_out ? -x.y * inv_nr : x.y * inv_nr);
    }
}

template <class R>
qm_status gw_mel_impl(qm_gspace g, int ikl, int ikr, int nl, const void* psi_l, int ld_l, int nr,
                             const void* psi_r, int ld_r, qm_gspace ge, int iq, void* M, int ld_m, cudaStream_t s) {
    using C = typename Cx<R>::T;
    const int N1 = g->n[0], N2 = g->n[1], N3 = g->n[2];
    const size_t nrr = (size_t)N1 * N2 * N3;
    const KTables& kl = g->k[ikl];
    const KTables& kr = g->k[ikr];
    const KTables& ke = ge->k[iq];
    const bool fx = fused_length(N1), fyz = fused_length(N2) || fused_length(N3);
    auto kin_ = fx ? k_stick_inverse<R, true> : k_stick_inverse<R, false>;
    auto kre_ = fyz ? k_plane_real<R, true> : k_plane_real<R, false>;
    auto kpa_ = fyz ? k_plane_pair<R, true> : k_plane_pair<R, false>;
    auto kme_ = fx ? k_stick_mel<R, true> : k_stick_mel<R, false>;
    const size_t sm_stick = (size_t)(sticks_per_cta<R>() * g->ldx + N1) * sizeof(C);
    const size_t sm_plane = (size_t)(N3 * g->ldy + N2 + N3) * sizeof(C) + (size_t)N3 * sizeof(int);
    qm_status st;
    if ((st = allow_dynamic_smem((const void*)kin_, sm_stick, "qm_gw_mel: sticks in shared memory")) ||
        (st = allow_dynamic_smem((const void*)kme_, sm_stick, "qm_gw_mel: sticks in shared memory")) ||
        (st = allow_dynamic_smem((const void*)kre_, sm_plane, "qm_gw_mel: plane in shared memory")) ||
        (st = allow_dynamic_smem((const void*)kpa_, sm_plane, "qm_gw_mel: plane in shared memory")))
        return st;
    const int nt_re = plane_threads((const void*)kre_, sm_plane);
    const int nt_pa = plane_threads((const void*)kpa_, sm_plane);

    // workspace: U_left | U_right | stick buffer of the inverse passes | stick buffer of the pairs
    constexpr size_t kChunk = 256ull << 20;
    const size_t box = nrr * sizeof(C);
    const size_t per_t = (size_t)N1 * std::max(kl.nstick_pad, kr.nstick_pad) * sizeof(C);
    const size_t per_e = (size_t)N1 * ke.nstick_pad * sizeof(C);
    // states and pairs per launch: 256 MB stick buffers, at most the grid's 65535 y extent
    const int nbc =
        (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>((size_t)std::max(nl, nr), kChunk / per_t), kMaxGridY));
    const int npair = nl * nr;
    const int npc = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>((size_t)npair, kChunk / per_e), kMaxGridY));
    const size_t off_ul = kWsHeader;
    const size_t off_ur = align_up(off_ul + (size_t)nl * box, 256);
    const size_t off_t = align_up(off_ur + (size_t)nr * box, 256);
    const size_t off_e = align_up(off_t + (size_t)nbc * per_t, 256);
    const size_t total = align_up(off_e + (size_t)npc * per_e, 256);
    if ((st = ensure_workspace(g, total, s))) return st;
    char* ws = (char*)g->ws.ptr;
    C* UL = (C*)(ws + off_ul);
    C* UR = (C*)(ws + off_ur);
    C* T = (C*)(ws + off_t);
    C* Te = (C*)(ws + off_e);
    const C* tw[3];
    for (int d = 0; d < 3; ++d) tw[d] = (const C*)(sizeof(R) == 8 ? (const void*)g->tw64[d] : (const void*)g->tw32[d]);

    // both sets of states to real space
    const struct { const KTables* kt; const C* psi; int ld, n; C* U; } side[2] = {
        {&kl, (const C*)psi_l, ld_l, nl, UL}, {&kr, (const C*)psi_r, ld_r, nr, UR}};
    for (const auto& sd : side) {
        const int ntile = (sd.kt->nstick + sticks_per_cta<R>() - 1) / sticks_per_cta<R>();
        for (int b0 = 0; b0 < sd.n; b0 += nbc) {
            const int nbx = std::min(nbc, sd.n - b0);
            {
                ProfScope pf(PF_STICK_INV, s);
                kin_<<<dim3(ntile, nbx), stick_threads<R>(), sm_stick, s>>>(
                    sd.psi + (size_t)b0 * sd.ld, sd.ld, sd.kt->stick_g0, sd.kt->g_code, sd.kt->nstick,
                    sd.kt->nstick_pad, g->plan[0], tw[0], g->ldx, T, 0);
            }
            {
                ProfScope pf(PF_PLANE, s);
                kre_<<<dim3(N1, nbx), nt_re, sm_plane, s>>>(T, sd.kt->nstick, sd.kt->nstick_pad, sd.kt->stick_plane,
                                                            sd.kt->rows, sd.kt->nrow, g->plan[1], g->plan[2], tw[1],
                                                            tw[2], g->ldy, N1, sd.U + (size_t)b0 * nrr);
            }
        }
    }
    // the pairs
    const int ntile_e = (ke.nstick + sticks_per_cta<R>() - 1) / sticks_per_cta<R>();
    const R inv_nr = (R)(1.0 / (double)nrr);
    for (int p0 = 0; p0 < npair; p0 += npc) {
        const int npx = std::min(npc, npair - p0);
        {
            ProfScope pf(PF_PLANE, s);
            kpa_<<<dim3(N1, npx), nt_pa, sm_plane, s>>>(UL, UR, nr, p0, ke.nstick, ke.nstick_pad, ke.stick_plane,
                                                        ke.rows, ke.nrow, g->plan[1], g->plan[2], tw[1], tw[2],
                                                        g->ldy, N1, Te);
        }
        {
            ProfScope pf(PF_STICK_FWD, s);
            kme_<<<dim3(ntile_e, npx), stick_threads<R>(), sm_stick, s>>>(Te, ke.nstick, ke.nstick_pad, ke.stick_g0,
                                                                         ke.g_code, g->plan[0], tw[0], g->ldx, inv_nr,
                                                                         (C*)M + (size_t)p0 * ld_m, ld_m, 1);
        }
    }
    return cuda_check(cudaGetLastError(), "qm_gw_mel launch");
}

}  // namespace qm

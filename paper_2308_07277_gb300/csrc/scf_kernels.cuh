// Device side of the self-consistency loop (qm_scf, Sec. 2.1): the density of the occupied
// states and the potential V_ext + V_Hartree + V_xc of a density, through the stick-pruned FFT
// kernels of the H psi path (compiled with them in fft_f64.cu; FP64 only).
//
//   density:   states -> x sticks (k_stick_inverse) -> whole real-space planes (k_plane_real,
//              digit-reversed positions) -> n(r) += w f |u(r)|^2 / Omega at the natural position
//              (k_density_acc: the digit reversal is undone by the scatter).
//   potential: n(r) -> digit-reversed complex box (k_permute_cbox) -> Fourier coefficients on the
//              density sphere |G|^2/2 <= 4 E_c (k_plane_pair with no right factor, k_stick_mel)
//              -> V_H(G) = 4 pi n(G) / |G|^2, V_H(0) = 0 (k_hartree) -> real space
//              (k_stick_inverse, k_plane_real) -> V = V_ext + Re V_H + v_xc(n) (k_potential).
// LDA: Slater exchange and the Perdew-Zunger parametrisation of the Ceperley-Alder correlation
// of the unpolarised electron gas (Phys. Rev. B 23, 5048 (1981)); v_xc = d(n eps_xc)/dn;
// densities at or below 1e-12 (an overshooting mixing step) contribute no exchange-correlation.
#pragma once
#include "gw_kernels.cuh"

namespace qm {

constexpr double kRhoFloor = 1e-12;

__device__ __forceinline__ double lda_vxc(double n) {
    if (!(n > kRhoFloor)) return 0.0;
    const double pi = 3.14159265358979323846;
    const double rs = cbrt(3.0 / (4.0 * pi * n));
    const double cx = 0.45816529328314287;  // (3/4)(3/(2 pi))^(2/3): eps_x = -cx / rs
    const double vx = -4.0 / 3.0 * cx / rs;
    double vc;
    if (rs >= 1.0) {
        const double g = -0.1423, b1 = 1.0529, b2 = 0.3334;
        const double sq = sqrt(rs), den = 1.0 + b1 * sq + b2 * rs;
        vc = g / den * (1.0 + 7.0 / 6.0 * b1 * sq + 4.0 / 3.0 * b2 * rs) / den;
    } else {
        const double A = 0.0311, B = -0.048, Cc = 0.0020, Dd = -0.0116, lr = log(rs);
        vc = A * lr + (B - A / 3.0) + 2.0 / 3.0 * Cc * rs * lr + (2.0 * Dd - Cc) / 3.0 * rs;
    }
    return vx + vc;
}

// natural flat index (x fastest) of digit-reversed box position i = p1 N3 N2 + p3 N2 + p2
__device__ __forceinline__ size_t natural_of(size_t i, int N1, int N2, int N3, const int* rev1, const int* rev2,
                                             const int* rev3) {
    const size_t plane = (size_t)N3 * N2;
    const int p1 = (int)(i / plane);
    const int rem = (int)(i - (size_t)p1 * plane);
    const int p3 = rem / N2, p2 = rem - p3 * N2;
    return (size_t)__ldg(rev1 + p1) + (size_t)N1 * ((size_t)__ldg(rev2 + p2) + (size_t)N2 * __ldg(rev3 + p3));
}

// n[natural(i)] += w sum_b |U[b][i]|^2 over nb boxes (each position written by one thread)
__global__ void k_density_acc(const double2* __restrict__ U, int nb, size_t nrr, int N1, int N2, int N3,
                              const int* __restrict__ rev1, const int* __restrict__ rev2,
                              const int* __restrict__ rev3, double w, double* __restrict__ n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nrr; i += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double2 u = U[(size_t)b * nrr + i];
            s += u.x * u.x + u.y * u.y;
        }
        n[natural_of(i, N1, N2, N3, rev1, rev2, rev3)] += w * s;
    }
}

// box[i] = (n[natural(i)], 0)
__global__ void k_permute_cbox(const double* __restrict__ n, size_t nrr, int N1, int N2, int N3,
                               const int* __restrict__ rev1, const int* __restrict__ rev2,
                               const int* __restrict__ rev3, double2* __restrict__ box) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nrr; i += (size_t)gridDim.x * blockDim.x)
        box[i] = make_double2(n[natural_of(i, N1, N2, N3, rev1, rev2, rev3)], 0.0);
}

// V_H(G) = 4 pi n(G) / |G|^2 in place (|G|^2 = 2 kin at k = 0), 0 at G = 0
__global__ void k_hartree(double2* __restrict__ v, const double* __restrict__ kin, int npw) {
    const double fourpi = 12.566370614359172954;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
        const double k2 = 2.0 * kin[g];
        const double f = k2 > 0.0 ? fourpi / k2 : 0.0;
        v[g] = make_double2(v[g].x * f, v[g].y * f);
    }
}

// v[natural(i)] = vion + Re(vh[i]) + v_xc(n)
__global__ void k_potential(const double2* __restrict__ vh, const double* __restrict__ n,
                            const double* __restrict__ vion, size_t nrr, int N1, int N2, int N3,
                            const int* __restrict__ rev1, const int* __restrict__ rev2, const int* __restrict__ rev3,
                            double* __restrict__ v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nrr; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = natural_of(i, N1, N2, N3, rev1, rev2, rev3);
        v[r] = vion[r] + vh[i].x + lda_vxc(n[r]);
    }
}

// bytes of the work buffer the two functions below need
inline size_t scf_work_bytes(qm_gspace g, qm_gspace grho, int nocc) {
    const size_t nrr = (size_t)g->n[0] * g->n[1] * g->n[2];
    int pad = grho->k[0].nstick_pad;
    for (const auto& kt : g->k) pad = std::max(pad, kt.nstick_pad);
    const int nbc = std::max(1, std::min(nocc, 16));
    const size_t t = (size_t)nbc * g->n[0] * pad * sizeof(double2);
    const size_t u = (size_t)nbc * nrr * sizeof(double2);
    const size_t vg = align_up((size_t)grho->k[0].npw * sizeof(double2), 256);
    return align_up(t, 256) + align_up(u, 256) + vg;
}

struct ScfFft {
    qm_gspace g;
    size_t sm_stick, sm_plane;
    int nt_re, nt_pa;
    decltype(&k_stick_inverse<double, true>) kin;
    decltype(&k_plane_real<double, true>) kre;
    decltype(&k_plane_pair<double, true>) kpa;
    decltype(&k_stick_mel<double, true>) kme;
};

inline qm_status scf_fft_setup(qm_gspace g, ScfFft& f) {
    const int N1 = g->n[0], N2 = g->n[1], N3 = g->n[2];
    const bool fx = fused_length(N1), fyz = fused_length(N2) || fused_length(N3);
    f.g = g;
    f.kin = fx ? k_stick_inverse<double, true> : k_stick_inverse<double, false>;
    f.kre = fyz ? k_plane_real<double, true> : k_plane_real<double, false>;
    f.kpa = fyz ? k_plane_pair<double, true> : k_plane_pair<double, false>;
    f.kme = fx ? k_stick_mel<double, true> : k_stick_mel<double, false>;
    f.sm_stick = (size_t)(sticks_per_cta<double>() * g->ldx + N1) * sizeof(double2);
    f.sm_plane = (size_t)(N3 * g->ldy + N2 + N3) * sizeof(double2) + (size_t)N3 * sizeof(int);
    qm_status st;
    if ((st = allow_dynamic_smem((const void*)f.kin, f.sm_stick, "qm_scf: sticks in shared memory")) ||
        (st = allow_dynamic_smem((const void*)f.kme, f.sm_stick, "qm_scf: sticks in shared memory")) ||
        (st = allow_dynamic_smem((const void*)f.kre, f.sm_plane, "qm_scf: plane in shared memory")) ||
        (st = allow_dynamic_smem((const void*)f.kpa, f.sm_plane, "qm_scf: plane in shared memory")))
        return st;
    f.nt_re = plane_threads((const void*)f.kre, f.sm_plane);
    f.nt_pa = plane_threads((const void*)f.kpa, f.sm_plane);
    return QM_OK;
}

// sphere coefficients (nb rows, ld) of k-point table kt -> nb whole real-space boxes U (digit-reversed)
inline void scf_to_real(const ScfFft& f, const KTables& kt, const double2* c, int ld, int nb, double2* T, double2* U,
                        cudaStream_t s) {
    qm_gspace g = f.g;
    const int N1 = g->n[0];
    const int ntile = (kt.nstick + sticks_per_cta<double>() - 1) / sticks_per_cta<double>();
    {
        ProfScope pf(PF_STICK_INV, s);
        f.kin<<<dim3(ntile, nb), stick_threads<double>(), f.sm_stick, s>>>(c, ld, kt.stick_g0, kt.g_code, kt.nstick,
                                                                           kt.nstick_pad, g->plan[0], g->tw64[0],
                                                                           g->ldx, T, 0);
    }
    {
        ProfScope pf(PF_PLANE, s);
        f.kre<<<dim3(N1, nb), f.nt_re, f.sm_plane, s>>>(T, kt.nstick, kt.nstick_pad, kt.stick_plane, kt.rows, kt.nrow,
                                                        g->plan[1], g->plan[2], g->tw64[1], g->tw64[2], g->ldy, N1, U);
    }
}

// n_nat += sum over the first nocc rows of psi of w |u(r)|^2 (w = weight x occupation / Omega)
inline qm_status scf_density(const ScfFft& f, int ik, int nocc, const double2* psi, int ld, double w, double* n_nat,
                             void* work, cudaStream_t s) {
    qm_gspace g = f.g;
    const size_t nrr = (size_t)g->n[0] * g->n[1] * g->n[2];
    const int nbc = std::max(1, std::min(nocc, 16));
    int pad = 0;
    for (const auto& kt : g->k) pad = std::max(pad, kt.nstick_pad);
    double2* T = (double2*)work;
    double2* U = (double2*)((char*)work + align_up((size_t)nbc * g->n[0] * pad * sizeof(double2), 256));
    for (int b0 = 0; b0 < nocc; b0 += nbc) {
        const int nb = std::min(nbc, nocc - b0);
        scf_to_real(f, g->k[ik], psi + (size_t)b0 * ld, ld, nb, T, U, s);
        ProfScope pf(PF_OTHER, s);
        k_density_acc<<<grid_stride_blocks(nrr, 256, 8), 256, 0, s>>>(U, nb, nrr, g->n[0], g->n[1], g->n[2], g->rev[0],
                                                                     g->rev[1], g->rev[2], w, n_nat);
    }
    return cuda_check(cudaGetLastError(), "qm_scf: density launch");
}

// v_nat = vion + V_H[n] + v_xc(n); grho: the density sphere (k = 0, same grid as f.g)
inline qm_status scf_potential(const ScfFft& f, qm_gspace grho, const double* n_nat, const double* vion,
                               double* v_nat, void* work, size_t work_bytes, cudaStream_t s) {
    qm_gspace g = f.g;
    const int N1 = g->n[0], N2 = g->n[1], N3 = g->n[2];
    const size_t nrr = (size_t)N1 * N2 * N3;
    const KTables& kr = grho->k[0];
    // work: box (nrr complex) | T (one band of sticks) | coefficients on the density sphere
    const size_t off_t = align_up(nrr * sizeof(double2), 256);
    const size_t off_c = align_up(off_t + (size_t)N1 * kr.nstick_pad * sizeof(double2), 256);
    if (off_c + (size_t)kr.npw * sizeof(double2) > work_bytes) return fail(QM_ERR_ARG, "qm_scf: work buffer too small");
    double2* box = (double2*)work;
    double2* T = (double2*)((char*)work + off_t);
    double2* cg = (double2*)((char*)work + off_c);
    const int blocks = grid_stride_blocks(nrr, 256, 8);
    {
        ProfScope pf(PF_OTHER, s);
        k_permute_cbox<<<blocks, 256, 0, s>>>(n_nat, nrr, N1, N2, N3, g->rev[0], g->rev[1], g->rev[2], box);
    }
    {
        ProfScope pf(PF_PLANE, s);
        f.kpa<<<dim3(N1, 1), f.nt_pa, f.sm_plane, s>>>(box, nullptr, 1, 0, kr.nstick, kr.nstick_pad, kr.stick_plane,
                                                       kr.rows, kr.nrow, g->plan[1], g->plan[2], g->tw64[1],
                                                       g->tw64[2], g->ldy, N1, T);
    }
    {
        const int ntile = (kr.nstick + sticks_per_cta<double>() - 1) / sticks_per_cta<double>();
        ProfScope pf(PF_STICK_FWD, s);
        f.kme<<<dim3(ntile, 1), stick_threads<double>(), f.sm_stick, s>>>(T, kr.nstick, kr.nstick_pad, kr.stick_g0,
                                                                          kr.g_code, g->plan[0], g->tw64[0], g->ldx,
                                                                          1.0 / (double)nrr, cg, kr.npw, 0);
    }
    {
        ProfScope pf(PF_OTHER, s);
        k_hartree<<<grid_stride_blocks((size_t)kr.npw, 256, 4), 256, 0, s>>>(cg, kr.kin, kr.npw);
    }
    scf_to_real(f, kr, cg, kr.npw, 1, T, box, s);
    {
        ProfScope pf(PF_OTHER, s);
        k_potential<<<blocks, 256, 0, s>>>(box, n_nat, vion, nrr, N1, N2, N3, g->rev[0], g->rev[1], g->rev[2], v_nat);
    }
    return cuda_check(cudaGetLastError(), "qm_scf: potential launch");
}

}  // namespace qm

// Host launchers of the FFT path; the kernels live in fft_kernels.cuh and are compiled once
// per precision (fft_f64.cu, fft_f32.cu).
#include "fft_kernels.cuh"

namespace qm {

extern template qm_status local_kinetic_impl<double>(qm_gspace, int, int, const void*, int, const void*, void*, int,
                                                     void*, size_t, cudaStream_t, cudaEvent_t, bool, bool);
extern template qm_status local_kinetic_impl<float>(qm_gspace, int, int, const void*, int, const void*, void*, int,
                                                    void*, size_t, cudaStream_t, cudaEvent_t, bool, bool);
extern template qm_status local_kinetic_tab_impl<double>(const DevTables&, int, const void*, int, const void*, void*,
                                                         int, void*, size_t, cudaStream_t);
extern template qm_status local_kinetic_tab_impl<float>(const DevTables&, int, const void*, int, const void*, void*,
                                                        int, void*, size_t, cudaStream_t);

// ---------------------------------------------------------------- host launchers
size_t stick_buffer_bytes_per_band(qm_gspace g, int ik, bool fp32) {
    return (size_t)g->n[0] * g->k[ik].nstick_pad * (fp32 ? sizeof(float2) : sizeof(double2));
}

qm_status launch_vt_prepare(qm_gspace g, const double* vloc, void* vt, bool fp32, cudaStream_t s) {
    const size_t nr = (size_t)g->n[0] * g->n[1] * g->n[2];
    const double scale = 1.0 / (double)nr;
    const int blocks = grid_stride_blocks(nr, 256, 8);
    ProfScope ps(PF_VT, s);
    if (fp32)
        k_vt<float><<<blocks, 256, 0, s>>>(vloc, (float*)vt, g->n[0], g->n[1], g->n[2], g->rev[0], g->rev[1], g->rev[2], scale);
    else
        k_vt<double><<<blocks, 256, 0, s>>>(vloc, (double*)vt, g->n[0], g->n[1], g->n[2], g->rev[0], g->rev[1], g->rev[2], scale);
    return cuda_check(cudaGetLastError(), "k_vt launch");
}

qm_status launch_local_kinetic(qm_gspace g, int ik, int nb, const void* psi, int ld_psi, const void* vt,
                               void* out, int ld_out, void* tbuf, size_t tbuf_bytes, bool fp32, cudaStream_t s,
                               cudaEvent_t wait_k3, bool accumulate, bool gamma) {
    if (fp32)
        return local_kinetic_impl<float>(g, ik, nb, psi, ld_psi, vt, out, ld_out, tbuf, tbuf_bytes, s, wait_k3,
                                         accumulate, gamma);
    return local_kinetic_impl<double>(g, ik, nb, psi, ld_psi, vt, out, ld_out, tbuf, tbuf_bytes, s, wait_k3,
                                      accumulate, gamma);
}


// ---------------------------------------------------------------- launchers on explicit tables
// Same launch sequence as above, with every table given by pointer (used by the entry point
// whose scratch and tables live in caller-independent fixed device memory).
qm_status launch_vt_prepare_tab(const DevTables& t, const double* vloc, void* vt, bool fp32, cudaStream_t s) {
    const size_t nr = (size_t)t.n[0] * t.n[1] * t.n[2];
    const double scale = 1.0 / (double)nr;
    const int blocks = grid_stride_blocks(nr, 256, 8);
    ProfScope ps(PF_VT, s);
    if (fp32)
        k_vt<float><<<blocks, 256, 0, s>>>(vloc, (float*)vt, t.n[0], t.n[1], t.n[2], t.rev[0], t.rev[1], t.rev[2], scale);
    else
        k_vt<double><<<blocks, 256, 0, s>>>(vloc, (double*)vt, t.n[0], t.n[1], t.n[2], t.rev[0], t.rev[1], t.rev[2], scale);
    return cuda_check(cudaGetLastError(), "k_vt launch");
}

qm_status launch_local_kinetic_tab(const DevTables& t, int nb, const void* psi, int ld_psi, const void* vt, void* out,
                                   int ld_out, void* tbuf, size_t tbuf_bytes, bool fp32, cudaStream_t s) {
    if (fp32) return local_kinetic_tab_impl<float>(t, nb, psi, ld_psi, vt, out, ld_out, tbuf, tbuf_bytes, s);
    return local_kinetic_tab_impl<double>(t, nb, psi, ld_psi, vt, out, ld_out, tbuf, tbuf_bytes, s);
}

}  // namespace qm

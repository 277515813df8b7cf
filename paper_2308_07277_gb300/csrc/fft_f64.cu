// FFT-path kernels instantiated for double (one translation unit per precision so the two
// compile in parallel).
#include "fft_kernels.cuh"
#include "gw_kernels.cuh"
#include "scf_kernels.cuh"

namespace qm {
template qm_status local_kinetic_impl<double>(qm_gspace, int, int, const void*, int, const void*, void*, int, void*,
                                         size_t, cudaStream_t, cudaEvent_t, bool, bool);
template qm_status local_kinetic_tab_impl<double>(const DevTables&, int, const void*, int, const void*, void*, int,
                                             void*, size_t, cudaStream_t);
template qm_status gw_mel_impl<double>(qm_gspace, int, int, int, const void*, int, int, const void*, int, qm_gspace,
                                     int, void*, int, cudaStream_t);

// self-consistency loop (qm_scf): the FFT-path parts, compiled here with the kernels they launch
size_t scf_work_size(qm_gspace g, qm_gspace grho, int nocc) { return scf_work_bytes(g, grho, nocc); }

qm_status scf_density_run(qm_gspace g, int ik, int nocc, const double2* psi, int ld, double w, double* n_nat,
                          void* work, cudaStream_t s) {
    ScfFft f;
    qm_status st = scf_fft_setup(g, f);
    return st ? st : scf_density(f, ik, nocc, psi, ld, w, n_nat, work, s);
}

qm_status scf_potential_run(qm_gspace g, qm_gspace grho, const double* n_nat, const double* vion, double* v_nat,
                            void* work, size_t work_bytes, cudaStream_t s) {
    ScfFft f;
    qm_status st = scf_fft_setup(g, f);
    return st ? st : scf_potential(f, grho, n_nat, vion, v_nat, work, work_bytes, s);
}
}  // namespace qm

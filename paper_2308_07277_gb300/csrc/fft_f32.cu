// FFT-path kernels instantiated for float (one translation unit per precision so the two
// compile in parallel).
#include "fft_kernels.cuh"
#include "gw_kernels.cuh"

namespace qm {
template qm_status local_kinetic_impl<float>(qm_gspace, int, int, const void*, int, const void*, void*, int, void*,
                                         size_t, cudaStream_t, cudaEvent_t, bool, bool);
template qm_status local_kinetic_tab_impl<float>(const DevTables&, int, const void*, int, const void*, void*, int,
                                             void*, size_t, cudaStream_t);
template qm_status gw_mel_impl<float>(qm_gspace, int, int, int, const void*, int, int, const void*, int, qm_gspace,
                                     int, void*, int, cudaStream_t);
}  // namespace qm

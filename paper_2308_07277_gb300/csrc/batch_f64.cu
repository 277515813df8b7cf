// FP64 instantiation of the batched H psi kernel (batch.cuh).
#include "batch.cuh"

namespace qm {
qm_status batch_launch_f64(const BatchLaunch& L, cudaStream_t s) { return batch_launch_impl<double>(L, s); }
int batch_occupancy_f64(size_t smem, int order) { return batch_occupancy_impl<double>(smem, order); }
}  // namespace qm

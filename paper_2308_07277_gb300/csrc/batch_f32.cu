// FP32 instantiation of the batched H psi kernel (batch.cuh).
#include "batch.cuh"

namespace qm {
qm_status batch_launch_f32(const BatchLaunch& L, cudaStream_t s) { return batch_launch_impl<float>(L, s); }
int batch_occupancy_f32(size_t smem, int order) { return batch_occupancy_impl<float>(smem, order); }
}  // namespace qm

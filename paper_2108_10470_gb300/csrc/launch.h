// Host-side launch wrappers of the step kernels. Each kernel family lives in its own translation
// unit (kernels_shared.cu, kernels_global.cu, kernels_persistent.cu) so the library's device
// code compiles in parallel; the C ABI (sim_api.cu) reaches the kernels only through these.
#pragma once
#include <cuda_runtime.h>

#include "sim_internal.h"

namespace artsim {

// One launch of step_kernel<G, rows_global> over ta.n_launch_envs envs, groups_per_block envs per
// CTA (G lanes each), smem bytes of dynamic shared memory per CTA.
cudaError_t launch_step_kernel(int G, bool rows_global, const StepArgs& a, const TypeArgs& ta,
                               int groups_per_block, size_t smem, cudaStream_t st);
// Cap of dynamic shared memory per CTA for step_kernel<G, rows_global>.
cudaError_t set_step_kernel_smem_cap(int G, bool rows_global, size_t bytes);

cudaError_t launch_persistent_kernel(const PersistArgs& P, int grid, size_t smem, cudaStream_t st);
cudaError_t set_persistent_kernel_smem_cap(size_t bytes);
cudaError_t persistent_kernel_occupancy(int* ctas_per_sm, size_t smem);

}  // namespace artsim

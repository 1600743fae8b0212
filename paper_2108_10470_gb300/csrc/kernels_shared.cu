// Per-type step kernels, contact and row blocks in shared memory: the G = 8, 16 and 32 instantiations
// and their host-side launch wrappers.
#include "launch.h"
#include "step_kernel.cuh"

namespace artsim {

namespace {
template <int G>
cudaError_t launch(const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem, cudaStream_t st) {
  const int blocks = (ta.n_launch_envs + gpb - 1) / gpb;
  step_kernel<G, false><<<blocks, gpb * G, smem, st>>>(a, ta);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_shared(int G, const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem, cudaStream_t st) {
  if (G == 8) return launch<8>(a, ta, gpb, smem, st);
  if (G == 16) return launch<16>(a, ta, gpb, smem, st);
  return launch<32>(a, ta, gpb, smem, st);
}

cudaError_t launch_shared_smem_cap(int G, size_t bytes) {
  if (G == 8) return cudaFuncSetAttribute(step_kernel<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (G == 16) return cudaFuncSetAttribute(step_kernel<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaFuncSetAttribute(step_kernel<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_global(int G, bool ball, const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem,
                          cudaStream_t st);
cudaError_t launch_global_smem_cap(int G, bool ball, size_t bytes);

cudaError_t launch_step_kernel(int G, bool rows_global, bool ball, const StepArgs& a, const TypeArgs& ta,
                               int groups_per_block, size_t smem, cudaStream_t st) {
  return rows_global ? launch_global(G, ball, a, ta, groups_per_block, smem, st)
                     : launch_shared(G, a, ta, groups_per_block, smem, st);
}

cudaError_t set_step_kernel_smem_cap(int G, bool rows_global, bool ball, size_t bytes) {
  return rows_global ? launch_global_smem_cap(G, ball, bytes) : launch_shared_smem_cap(G, bytes);
}

}  // namespace artsim

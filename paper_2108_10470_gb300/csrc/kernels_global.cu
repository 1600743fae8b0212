// Per-type step kernels, contact and row blocks in global scratch (with the shape-pair phase): the G = 8, 16 and 32 instantiations
// and their host-side launch wrappers.
#include "launch.h"
#include "step_kernel.cuh"

namespace artsim {

namespace {
template <int G>
cudaError_t launch(const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem, cudaStream_t st) {
  const int blocks = (ta.n_launch_envs + gpb - 1) / gpb;
  step_kernel<G, true><<<blocks, gpb * G, smem, st>>>(a, ta);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_global(int G, const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem, cudaStream_t st) {
  if (G == 8) return launch<8>(a, ta, gpb, smem, st);
  if (G == 16) return launch<16>(a, ta, gpb, smem, st);
  return launch<32>(a, ta, gpb, smem, st);
}

cudaError_t launch_global_smem_cap(int G, size_t bytes) {
  if (G == 8) return cudaFuncSetAttribute(step_kernel<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (G == 16) return cudaFuncSetAttribute(step_kernel<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaFuncSetAttribute(step_kernel<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace artsim

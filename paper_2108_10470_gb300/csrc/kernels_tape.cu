// The reverse pass of the step: the taped instantiations of the step kernel (the same step, which
// also records each env-substep's tape) and the adjoint kernel, with their host-side launch
// wrappers. Per-type launches only (the persistent kernel has no taped instantiation).
#include "adjoint_kernel.cuh"
#include "launch.h"

namespace artsim {

namespace {
template <int G, bool GROWS>
cudaError_t launch_taped(const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem, cudaStream_t st) {
  const int blocks = (ta.n_launch_envs + gpb - 1) / gpb;
  step_kernel<G, GROWS, false, true><<<blocks, gpb * G, smem, st>>>(a, ta);
  return cudaGetLastError();
}
template <int G, bool GROWS>
cudaError_t cap_taped(size_t bytes) {
  return cudaFuncSetAttribute(step_kernel<G, GROWS, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}
template <int G>
cudaError_t launch_adj(const StepArgs& a, const TypeArgs& ta, const AdjArgs& j, cudaStream_t st) {
  constexpr int kThreads = 64;
  const int gpb = kThreads / G;
  const int blocks = (ta.n_launch_envs + gpb - 1) / gpb;
  const size_t smem = sizeof(float) * (size_t)gpb * j.al.total;
  adjoint_kernel<G><<<blocks, kThreads, smem, st>>>(a, ta, j);
  return cudaGetLastError();
}
template <int G>
cudaError_t cap_adj(size_t bytes) {
  return cudaFuncSetAttribute(adjoint_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
}  // namespace

cudaError_t launch_taped_step_kernel(int G, bool rows_global, const StepArgs& a, const TypeArgs& ta,
                                     int groups_per_block, size_t smem, cudaStream_t st) {
  if (rows_global) {
    if (G == 8) return launch_taped<8, true>(a, ta, groups_per_block, smem, st);
    if (G == 16) return launch_taped<16, true>(a, ta, groups_per_block, smem, st);
    return launch_taped<32, true>(a, ta, groups_per_block, smem, st);
  }
  if (G == 8) return launch_taped<8, false>(a, ta, groups_per_block, smem, st);
  if (G == 16) return launch_taped<16, false>(a, ta, groups_per_block, smem, st);
  return launch_taped<32, false>(a, ta, groups_per_block, smem, st);
}

cudaError_t set_taped_step_kernel_smem_cap(int G, bool rows_global, size_t bytes) {
  if (rows_global) {
    if (G == 8) return cap_taped<8, true>(bytes);
    if (G == 16) return cap_taped<16, true>(bytes);
    return cap_taped<32, true>(bytes);
  }
  if (G == 8) return cap_taped<8, false>(bytes);
  if (G == 16) return cap_taped<16, false>(bytes);
  return cap_taped<32, false>(bytes);
}

cudaError_t launch_adjoint_kernel(int G, const StepArgs& a, const TypeArgs& ta, const AdjArgs& j, cudaStream_t st) {
  if (G == 8) return launch_adj<8>(a, ta, j, st);
  if (G == 16) return launch_adj<16>(a, ta, j, st);
  return launch_adj<32>(a, ta, j, st);
}

cudaError_t set_adjoint_kernel_smem_cap(int G, size_t bytes) {
  if (G == 8) return cap_adj<8>(bytes);
  if (G == 16) return cap_adj<16>(bytes);
  return cap_adj<32>(bytes);
}

}  // namespace artsim

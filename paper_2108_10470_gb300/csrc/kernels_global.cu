// Per-type step kernels, contact and row blocks in global scratch (with the shape-pair phase): the
// G = 8, 16 and 32 instantiations without and with the ball-joint code, and their host-side launch
// wrappers.
#include "launch.h"
#include "step_kernel.cuh"

namespace artsim {

namespace {
template <int G, bool BALL>
cudaError_t launch(const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem, cudaStream_t st) {
  const int blocks = (ta.n_launch_envs + gpb - 1) / gpb;
  step_kernel<G, true, BALL><<<blocks, gpb * G, smem, st>>>(a, ta);
  return cudaGetLastError();
}
template <bool BALL>
cudaError_t cap(int G, size_t bytes) {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (G == 8) return cudaFuncSetAttribute(step_kernel<8, true, BALL>, at, (int)bytes);
  if (G == 16) return cudaFuncSetAttribute(step_kernel<16, true, BALL>, at, (int)bytes);
  return cudaFuncSetAttribute(step_kernel<32, true, BALL>, at, (int)bytes);
}
}  // namespace

// ball: the instantiation with the ball-joint code (env types with ball joints)
cudaError_t launch_global(int G, bool ball, const StepArgs& a, const TypeArgs& ta, int gpb, size_t smem,
                          cudaStream_t st) {
  if (ball) {
    if (G == 8) return launch<8, true>(a, ta, gpb, smem, st);
    if (G == 16) return launch<16, true>(a, ta, gpb, smem, st);
    return launch<32, true>(a, ta, gpb, smem, st);
  }
  if (G == 8) return launch<8, false>(a, ta, gpb, smem, st);
  if (G == 16) return launch<16, false>(a, ta, gpb, smem, st);
  return launch<32, false>(a, ta, gpb, smem, st);
}

cudaError_t launch_global_smem_cap(int G, bool ball, size_t bytes) { return ball ? cap<true>(G, bytes) : cap<false>(G, bytes); }

}  // namespace artsim

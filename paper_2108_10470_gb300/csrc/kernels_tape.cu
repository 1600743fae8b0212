// The reverse pass of the step: the adjoint kernel and its host-side launch wrappers. (The tape is
// recorded by the step kernels themselves, given a tape pointer: sim_step_taped launches the same
// per-type kernels as sim_step.)
#include "adjoint_kernel.cuh"
#include "launch.h"

namespace artsim {

namespace {
// One instantiation per group size, with the capsule-box pair phase for env types with shape pairs
// and the 3-DOF blocks for env types with ball joints (their code and registers stay out of the
// kernels of the other types).
template <int G, bool PAIRS, bool BALL>
cudaError_t launch_adj(const StepArgs& a, const TypeArgs& ta, const AdjArgs& j, cudaStream_t st) {
  constexpr int kThreads = 64;
  const int gpb = kThreads / G;
  const int blocks = (ta.n_launch_envs + gpb - 1) / gpb;
  const size_t smem = sizeof(float) * (size_t)gpb * j.al.total;
  adjoint_kernel<G, PAIRS, BALL><<<blocks, kThreads, smem, st>>>(a, ta, j);
  return cudaGetLastError();
}
template <int G>
cudaError_t cap_adj(size_t bytes) {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<G, false, false>, at, (int)bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(adjoint_kernel<G, true, false>, at, (int)bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(adjoint_kernel<G, false, true>, at, (int)bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(adjoint_kernel<G, true, true>, at, (int)bytes);
  return e;
}
template <bool PAIRS, bool BALL>
cudaError_t launch_g(int G, const StepArgs& a, const TypeArgs& ta, const AdjArgs& j, cudaStream_t st) {
  if (G == 8) return launch_adj<8, PAIRS, BALL>(a, ta, j, st);
  if (G == 16) return launch_adj<16, PAIRS, BALL>(a, ta, j, st);
  return launch_adj<32, PAIRS, BALL>(a, ta, j, st);
}
}  // namespace

cudaError_t launch_adjoint_kernel(int G, bool ball, const StepArgs& a, const TypeArgs& ta, const AdjArgs& j,
                                  cudaStream_t st) {
  const bool pairs = ta.tl.cw > 5;
  if (ball) return pairs ? launch_g<true, true>(G, a, ta, j, st) : launch_g<false, true>(G, a, ta, j, st);
  return pairs ? launch_g<true, false>(G, a, ta, j, st) : launch_g<false, false>(G, a, ta, j, st);
}

cudaError_t set_adjoint_kernel_smem_cap(int G, size_t bytes) {
  if (G == 8) return cap_adj<8>(bytes);
  if (G == 16) return cap_adj<16>(bytes);
  return cap_adj<32>(bytes);
}

}  // namespace artsim

// Host-side launch wrappers of the step kernels. Each kernel family lives in its own translation
// unit (kernels_shared.cu, kernels_global.cu, kernels_persistent.cu) so the library's device
// code compiles in parallel; the C ABI (sim_api.cu) reaches the kernels only through these.
#pragma once
#include <cuda_runtime.h>

#include "sim_internal.h"

namespace artsim {

// Arguments of the derivative kernel (kernels_adjoint.cu). mode 0: adjoint (vector-Jacobian
// product) over the directions dir_base + k * 32 + lane; mode 1: tangent (Jacobian-vector product)
// of the caller's direction. Layouts are those of the state views.
struct TangentArgs {
  const float* root; const float* dof; const float* act; const float* cache;  // step input
  const float* g_root; const float* g_dof; const float* g_cache;              // adjoint: output gradient
  float* gi_root; float* gi_dof; float* gi_act; float* gi_cache;              // adjoint: input gradient
  const float* t_root; const float* t_dof; const float* t_act; const float* t_cache;  // tangent: input
  float* o_root; float* o_dof; float* o_cache;                                // step output (optional)
  float* to_root; float* to_dof; float* to_cache;                             // tangent: output
  int* status;                                                                // per env: 0, or 2 on failure
  int mode, dir_base;
};


// One launch of step_kernel<G, rows_global, ball> over ta.n_launch_envs envs, groups_per_block envs
// per CTA (G lanes each), smem bytes of dynamic shared memory per CTA. ball selects the global-rows
// instantiation with the ball-joint code (ignored for shared rows).
cudaError_t launch_step_kernel(int G, bool rows_global, bool ball, const StepArgs& a, const TypeArgs& ta,
                               int groups_per_block, size_t smem, cudaStream_t st);
// Cap of dynamic shared memory per CTA for step_kernel<G, rows_global, ball>.
cudaError_t set_step_kernel_smem_cap(int G, bool rows_global, bool ball, size_t bytes);

// The persistent kernel; ball selects the instantiation whose global-rows tile bodies carry the
// ball-joint code (a step with any ball-joint env type).
cudaError_t launch_persistent_kernel(const PersistArgs& P, bool ball, int grid, size_t smem, cudaStream_t st);
cudaError_t set_persistent_kernel_smem_cap(bool ball, size_t bytes);
cudaError_t persistent_kernel_occupancy(bool ball, int* ctas_per_sm, size_t smem);

// Derivative of the step (kernels_adjoint.cu): K tangents per lane (1, 2, 4 or 8), one env per warp.
cudaError_t launch_tangent_kernel(int K, const StepArgs& a, const TypeArgs& ta, const TangentArgs& v, cudaStream_t st);
int tangent_lanes_per_dir(int n_dirs);
// Reverse pass (kernels_tape.cu): the adjoint kernel (64-thread CTAs, 64 / G envs each, the
// AdjLayout arena per env). The tape is written by the per-type step kernels when TypeArgs::tape
// is set.
cudaError_t launch_adjoint_kernel(int G, bool ball, const StepArgs& a, const TypeArgs& ta, const AdjArgs& j,
                                  cudaStream_t st);
cudaError_t set_adjoint_kernel_smem_cap(int G, size_t bytes);
// Mass matrices (what = 0, n_envs x n_max x n_max) or link Jacobians (what = 1, n_envs x l_max x 6 x
// n_max) of the envs of one type at the current state, one thread per env.
cudaError_t launch_query_kernel(int what, const StepArgs& a, const TypeArgs& ta, float* out, int n_max, int l_max,
                                cudaStream_t st);

}  // namespace artsim

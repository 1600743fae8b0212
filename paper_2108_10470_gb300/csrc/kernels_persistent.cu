// The heterogeneous persistent step kernel and its host-side wrappers.
#include "launch.h"
#include "step_kernel.cuh"

namespace artsim {

// ---- heterogeneous persistent launch -----------------------------------------------------------
// All env types of a step in one launch of resident CTAs. A tile is the 32 / G envs of one type
// that one warp steps together; warps take tiles from a global counter in schedule order (the
// costliest types first, so the cheap tiles fill the tail) until none is left. The last warp to
// finish resets the counters, so back-to-back launches (and graph replays) need no memset. Each
// variant's tile body is a separate (not inlined) function, so it gets its own register
// allocation: inlining all six into the one kernel measured slower on Humanoid-like envs (by 10
// and by 20 % in two builds of the kernel).
template <int G, bool GROWS, bool BALL>
__device__ __noinline__ void persistent_tile(const StepArgs& A, const TypeArgs& TA, int tile, float* wsm,
                                                int gwarp) {
  const int gw = (threadIdx.x & 31) / G;  // group within the warp
  const int grp = tile * (32 / G) + gw;
  float* sm = wsm + gw * TA.lay.total;
  float* slot = TA.lay.scratch_words ? TA.scratch + (size_t)(gwarp * (32 / G) + gw) * TA.lay.scratch_words : nullptr;
  float* rb = GROWS ? slot : sm;
  step_group<G, GROWS, BALL, false>(A, TA, grp, sm, rb, GROWS ? nullptr : slot);  // taped and direct-buffer steps: per-type kernels
}

template <bool BALL>
__global__ void __launch_bounds__(128, 4) persistent_step_kernel(const __grid_constant__ PersistArgs P) {
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * (blockDim.x >> 5) + wid;
  float* wsm = smem + wid * P.warp_words;
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(P.counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= P.n_tiles) break;
    int s = 0;
    while (t >= P.tile_end[s]) ++s;
    const int k = P.order[s];
    const int tile = t - (s ? P.tile_end[s - 1] : 0);
    const TypeArgs& TA = P.types[k];
    switch (P.variant[k]) {
      case kVar8: persistent_tile<8, false, false>(P.common, TA, tile, wsm, gwarp); break;
      case kVar16: persistent_tile<16, false, false>(P.common, TA, tile, wsm, gwarp); break;
      case kVar32: persistent_tile<32, false, false>(P.common, TA, tile, wsm, gwarp); break;
      case kVar8 | kVarRowsGlobal: persistent_tile<8, true, BALL>(P.common, TA, tile, wsm, gwarp); break;
      case kVar16 | kVarRowsGlobal: persistent_tile<16, true, BALL>(P.common, TA, tile, wsm, gwarp); break;
      default: persistent_tile<32, true, BALL>(P.common, TA, tile, wsm, gwarp); break;
    }
    __syncwarp();
  }
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(P.counter + 1, 1u) == (unsigned)P.n_warps - 1u) {
      atomicExch(P.counter, 0u);
      atomicExch(P.counter + 1, 0u);
    }
  }
}

cudaError_t launch_persistent_kernel(const PersistArgs& P, bool ball, int grid, size_t smem, cudaStream_t st) {
  if (ball)
    persistent_step_kernel<true><<<grid, 128, smem, st>>>(P);
  else
    persistent_step_kernel<false><<<grid, 128, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t set_persistent_kernel_smem_cap(bool ball, size_t bytes) {
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  return ball ? cudaFuncSetAttribute(persistent_step_kernel<true>, at, (int)bytes)
              : cudaFuncSetAttribute(persistent_step_kernel<false>, at, (int)bytes);
}

cudaError_t persistent_kernel_occupancy(bool ball, int* ctas_per_sm, size_t smem) {
  return ball ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, persistent_step_kernel<true>, 128, smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, persistent_step_kernel<false>, 128, smem);
}

}  // namespace artsim

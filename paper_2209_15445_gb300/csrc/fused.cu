// One kernel per generation for all three species (S11, paper Sec. 3 and Sec. 5).
//
// Every warp takes the 32-track tiles of the concatenated gamma, e- and e+ queues in a
// warp-strided order, species by species, in three consecutive loops (so that the register
// allocation of one species' step does not overlap another's). Nothing waits for anything,
// so the kernel needs no co-residency. Chained in a CUDA graph this is one kernel node per
// generation instead of a fork, three species kernels and a join, and the species share
// the SMs until the generation's last tile.
#include <cuda_runtime.h>

#include "layout.h"
#include "transport.cuh"

namespace adept {

// index of this warp's first tile of the next segment of length `len`, given its first
// tile `first` in the current segment (warp-strided order over the concatenation)
__device__ __forceinline__ uint32_t next_first(uint32_t first, uint32_t len, uint32_t stride) {
  if (first >= len) return first - len;
  const uint32_t k = (len - first + stride - 1) / stride;  // tiles this warp took in the segment
  return first + k * stride - len;
}

template <class R, int MINB, int V>
__global__ void __launch_bounds__(256, MINB) k_fused_generation(Params P, uint32_t gk) {
  __shared__ WarpRing<R> rings[8];
  __shared__ unsigned long long s_cnt[6];
  WarpRing<R>& ring = rings[threadIdx.x >> 5];
  grid_dependency_wait();
  allow_dependent_launch();
  if (gk == kGkDevice) gk = __ldcg(&P.ctrl->tail_k);  // a generation of a tail chunk
  const uint32_t gen = __ldcg(&P.ctrl->gen) + gk;
  if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) open_generation(P, gen, gk);
  __syncthreads();
  const uint32_t wpb = blockDim.x >> 5;
  const uint32_t nwarps = gridDim.x * wpb;
  const int p = gen & 1, cr = gen % 3, cw = (gen + 1) % 3;
  const uint32_t n0 = min(__ldcg(&P.ctrl->count[cr][0].n), P.cap);
  const uint32_t n1 = min(__ldcg(&P.ctrl->count[cr][1].n), P.cap);
  const uint32_t n2 = min(__ldcg(&P.ctrl->count[cr][2].n), P.cap);
  const uint32_t T0 = (n0 + 31) >> 5, T1 = (n1 + 31) >> 5, T2 = (n2 + 31) >> 5;
  uint32_t nsteps[3] = {0, 0, 0}, ncreated[3] = {0, 0, 0};  // this generation: steps per lane, secondaries per warp
  uint32_t first = blockIdx.x * wpb + (threadIdx.x >> 5);
  run_tiles<R, 0, V>(P, p, cw, first, T0, nwarps, n0, ring, nsteps, ncreated);
  first = next_first(first, T0, nwarps);
  run_tiles<R, 1, V>(P, p, cw, first, T1, nwarps, n1, ring, nsteps, ncreated);
  first = next_first(first, T1, nwarps);
  run_tiles<R, 2, V>(P, p, cw, first, T2, nwarps, n2, ring, nsteps, ncreated);
  for (int k = 0; k < 3; ++k) nsteps[k] = __reduce_add_sync(0xFFFFFFFFu, nsteps[k]);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 3; ++k) {
      if (nsteps[k]) atomicAdd(&s_cnt[k], (unsigned long long)nsteps[k]);
      if (ncreated[k]) atomicAdd(&s_cnt[3 + k], (unsigned long long)ncreated[k]);
    }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int k = 0; k < 3; ++k) {
    if (s_cnt[k]) atomicAdd(&P.ctrl->steps[k], s_cnt[k]);
    if (s_cnt[3 + k]) atomicAdd(&P.ctrl->created[k], s_cnt[3 + k]);
  }
}

// Variants: FP32 physics for 2 or 3 resident 256-thread blocks per SM, FP64 for 1 or 2;
// each without (V = 0) and with (V = 8) the helix in a field. The fused kernel has no other
// optional part (adept_init refuses chords, the optional physics and the histogram with it).
template <int V>
static const void* fused_by(int precision, int minb) {
  if (precision)
    return minb >= 3 ? (const void*)k_fused_generation<float, 3, V> : (const void*)k_fused_generation<float, 2, V>;
  return minb >= 2 ? (const void*)k_fused_generation<double, 2, V> : (const void*)k_fused_generation<double, 1, V>;
}
static const void* fused_fn(int precision, int minb, int variant) {
  return (variant & 8) ? fused_by<8>(precision, minb) : fused_by<0>(precision, minb);
}

int fused_max_blocks_per_sm(int precision, int minb, int block, int variant) {
  return max_blocks_small_carveout(fused_fn(precision, minb, variant), block);
}

cudaError_t launch_fused_generation(const Params& P, uint32_t gk, int precision, int minb, int grid, int block,
                                    bool pdl, cudaStream_t st) {
  void* args[] = {const_cast<Params*>(&P), &gk};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelExC(&cfg, fused_fn(precision, minb, transport_variant(P)), args);
}

}  // namespace adept

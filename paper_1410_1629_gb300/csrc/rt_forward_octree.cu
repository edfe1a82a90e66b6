// Forward transport on octree grids (SKIRT paper, Sect. 2.4): the
// state-machine kernel of rt_transport.cuh instantiated with the octree cell
// walk (ancestor stack per lane in shared memory, top of the tree cached in
// shared memory).
#include "rt_transport.cuh"

// Resident blocks per SM the register allocation aims at: four (64
// registers) fit the shared memory of trees up to depth 10, whose per-lane
// ancestor stacks (dynamic shared memory, depth + 1 entries) take 11 KB of
// the block's 55 KB; deeper trees run three.
#ifndef RT_OCT_MIN_BLOCKS
#define RT_OCT_MIN_BLOCKS 4
#endif

namespace rtk {

namespace {
__global__ void __launch_bounds__(tr::kBlock, RT_OCT_MIN_BLOCKS) k_forward_octree(const FwdParams P) {
  tr::forward_body<tr::OctGrid>(P);
}
}  // namespace

cudaError_t launch_forward_octree(const FwdParams& p, int num_sms, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(p.work_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const size_t stack_bytes = (size_t)tr::kBlock * (size_t)p.oct_levels * sizeof(int);
  // static and dynamic shared memory together pass 48 KB: the launch needs
  // the dynamic part allowed explicitly
  e = cudaFuncSetAttribute(k_forward_octree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stack_bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward_octree, tr::kBlock, stack_bytes);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  unsigned long long blocks = (unsigned long long)num_sms * per_sm;
  const unsigned long long useful = (p.n_total + tr::kBlock - 1) / tr::kBlock;
  if (blocks > useful) blocks = useful;
  if (blocks < 1) blocks = 1;
  k_forward_octree<<<(unsigned)blocks, tr::kBlock, stack_bytes, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk

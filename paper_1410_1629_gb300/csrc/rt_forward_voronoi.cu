// Forward transport on Voronoi grids (the VoronoiDustGrid of the SKIRT paper,
// Table 1(d) and Sect. 2.4): the state-machine kernel of rt_transport.cuh
// instantiated with the walk across the cells' bisecting planes.
#include "rt_transport.cuh"

// four resident blocks of 256 fit the Voronoi walk in 64 registers without
// spills: more warps to hide the L2 latency of the face-plane loads
#ifndef RT_VOR_MIN_BLOCKS
#define RT_VOR_MIN_BLOCKS 4
#endif

namespace rtk {

namespace {
__global__ void __launch_bounds__(tr::kBlock, RT_VOR_MIN_BLOCKS) k_forward_voronoi(const FwdParams P) {
  tr::forward_body<tr::VorGrid>(P);
}
}  // namespace

cudaError_t launch_forward_voronoi(const FwdParams& p, int num_sms, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(p.work_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward_voronoi, tr::kBlock, 0);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  unsigned long long blocks = (unsigned long long)num_sms * per_sm;
  const unsigned long long useful = (p.n_total + tr::kBlock - 1) / tr::kBlock;
  if (blocks > useful) blocks = useful;
  if (blocks < 1) blocks = 1;
  k_forward_voronoi<<<(unsigned)blocks, tr::kBlock, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk

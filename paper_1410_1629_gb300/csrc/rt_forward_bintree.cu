// Forward transport on k-d tree grids (the BinTree grid of the SKIRT paper,
// Table 1(d)): the state-machine kernel of rt_transport.cuh instantiated with
// the k-d tree cell walk.
#include "rt_transport.cuh"

// four resident blocks of 256 (64 registers; 8 B of spills) hide more of the
// L2 latency of the node-word loads than three without spills: 350 -> 316 ms
// on the clumpy 2e5-leaf tree
#ifndef RT_BIN_MIN_BLOCKS
#define RT_BIN_MIN_BLOCKS 4
#endif

namespace rtk {

namespace {
__global__ void __launch_bounds__(tr::kBlock, RT_BIN_MIN_BLOCKS) k_forward_bintree(const FwdParams P) {
  tr::forward_body<tr::BinGrid>(P);
}
}  // namespace

cudaError_t launch_forward_bintree(const FwdParams& p, int num_sms, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(p.work_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward_bintree, tr::kBlock, 0);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  unsigned long long blocks = (unsigned long long)num_sms * per_sm;
  const unsigned long long useful = (p.n_total + tr::kBlock - 1) / tr::kBlock;
  if (blocks > useful) blocks = useful;
  if (blocks < 1) blocks = 1;
  k_forward_bintree<<<(unsigned)blocks, tr::kBlock, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk

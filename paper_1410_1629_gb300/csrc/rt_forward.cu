// Forward transport on cartesian grids: the state-machine kernel of
// rt_transport.cuh instantiated with the cartesian cell walk.
#include "rt_transport.cuh"

namespace rtk {

namespace {
__global__ void __launch_bounds__(tr::kBlock, RT_FWD_MIN_BLOCKS) k_forward_cartesian(const FwdParams P) {
  tr::forward_body<tr::CartGrid>(P);
}
// The same launch recording the adjoint tape (P.tape): the tape's lane state
// needs more registers (RT_TAPE_MIN_BLOCKS resident blocks per SM).
#ifndef RT_TAPE_MIN_BLOCKS
#define RT_TAPE_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(tr::kBlock, RT_TAPE_MIN_BLOCKS) k_forward_cartesian_tape(const FwdParams P) {
  tr::forward_body<tr::CartGrid, true>(P);
}
// The launch with execution counters (P.profile set, no tape).
__global__ void __launch_bounds__(tr::kBlock, RT_FWD_MIN_BLOCKS) k_forward_cartesian_prof(const FwdParams P) {
  tr::forward_body<tr::CartGrid, false, true>(P);
}
}  // namespace

cudaError_t launch_forward(const FwdParams& p, int grid_kind, int num_sms, cudaStream_t stream) {
  if (grid_kind == RT_GRID_OCTREE) return launch_forward_octree(p, num_sms, stream);
  if (grid_kind == RT_GRID_RECTILINEAR) return launch_forward_rect(p, num_sms, stream);
  if (grid_kind == RT_GRID_BINTREE) return launch_forward_bintree(p, num_sms, stream);
  if (grid_kind == RT_GRID_VORONOI) return launch_forward_voronoi(p, num_sms, stream);
  cudaError_t e = cudaMemsetAsync(p.work_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  const bool prof = p.profile != nullptr && !p.tape;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, p.tape ? k_forward_cartesian_tape : (prof ? k_forward_cartesian_prof : k_forward_cartesian), tr::kBlock,
      0);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  if (p.blocks_per_sm > 0 && p.blocks_per_sm < per_sm) per_sm = p.blocks_per_sm;
  unsigned long long blocks = (unsigned long long)num_sms * per_sm;
  const unsigned long long useful = (p.n_total + tr::kBlock - 1) / tr::kBlock;
  if (blocks > useful) blocks = useful;
  if (blocks < 1) blocks = 1;
  if (p.tape) {
    k_forward_cartesian_tape<<<(unsigned)blocks, tr::kBlock, 0, stream>>>(p);
  } else if (prof) {
    k_forward_cartesian_prof<<<(unsigned)blocks, tr::kBlock, 0, stream>>>(p);
  } else {
    k_forward_cartesian<<<(unsigned)blocks, tr::kBlock, 0, stream>>>(p);
  }
  return cudaGetLastError();
}

namespace {

// One thread per grid line along `axis`: the density integral from the far
// face of each cell to the boundary the ray meets (direction dir), summed in
// FP64 from that boundary inwards.  Cell widths along the axis: d, or the
// differences of the FP64 planes `planes` (rectilinear grids) when given.
__global__ void k_columns(const float* __restrict__ density, int nx, int ny, int nz, int axis, int dir, double d,
                          const double* __restrict__ planes, float* __restrict__ out) {
  const long long n_lines = axis == 0 ? (long long)ny * nz : (axis == 1 ? (long long)nx * nz : (long long)nx * ny);
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < n_lines;
       L += (long long)gridDim.x * blockDim.x) {
    long long base, stride;
    int n;
    if (axis == 0) {
      base = L * nx; stride = 1; n = nx;
    } else if (axis == 1) {
      base = (L % nx) + (L / nx) * (long long)nx * ny; stride = nx; n = ny;
    } else {
      base = L; stride = (long long)nx * ny; n = nz;
    }
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
      const int j = dir > 0 ? n - 1 - k : k;
      const long long c = base + (long long)j * stride;
      out[c] = (float)acc;
      acc += (double)density[c] * (planes ? planes[j + 1] - planes[j] : d);
    }
  }
}

}  // namespace

cudaError_t launch_columns(const float* density, int nx, int ny, int nz, int axis, int dir, float d,
                           const double* planes, float* out, cudaStream_t stream) {
  const long long n_lines = axis == 0 ? (long long)ny * nz : (axis == 1 ? (long long)nx * nz : (long long)nx * ny);
  const int block = 256;
  long long blocks = (n_lines + block - 1) / block;
  if (blocks > 65535) blocks = 65535;
  k_columns<<<(unsigned)blocks, block, 0, stream>>>(density, nx, ny, nz, axis, dir, (double)d, planes, out);
  return cudaGetLastError();
}

}  // namespace rtk

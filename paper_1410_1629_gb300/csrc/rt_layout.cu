// Storage order of cartesian and rectilinear grids.  A straight walk steps
// through the cell faces of each axis at a rate proportional to the cells per
// unit length along it; the axis crossed most often is stored unit-stride, so
// that consecutive crossings of a walk share 32-byte sectors of the density
// and of the absorption tallies (a disk galaxy's thin vertical cells are
// crossed about eight times as often as its horizontal ones).  Everything
// outside the kernels (inputs, read-outs, cell ids) stays row-major; these
// kernels convert.
#include <algorithm>

#include "rt_internal.h"

namespace rtk {

void crossing_order_strides(const int n[3], const double extent[3], int strides[3]) {
  int order[3] = {0, 1, 2};
  std::stable_sort(order, order + 3, [&](int a, int b) { return n[a] / extent[a] > n[b] / extent[b]; });
  int s = 1;
  for (int k = 0; k < 3; ++k) {
    strides[order[k]] = s;
    s *= n[order[k]];
  }
}

namespace {

__device__ __forceinline__ long long storage_index(long long r, int nx, int ny, int s0, int s1, int s2) {
  const long long ix = r % nx, iy = (r / nx) % ny, iz = r / ((long long)nx * ny);
  return ix * s0 + iy * s1 + iz * s2;
}

__global__ void k_to_storage(const float* __restrict__ src, float* __restrict__ dst, int nx, int ny, long long n,
                             int s0, int s1, int s2) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    dst[storage_index(r, nx, ny, s0, s1, s2)] = src[r];
}

// Row-major out (coalesced writes), one wavelength per blockIdx.y.
__global__ void k_from_storage(const double* __restrict__ src, double* __restrict__ dst, int nx, int ny, long long n,
                               int s0, int s1, int s2) {
  const double* s = src + (size_t)blockIdx.y * n;
  double* d = dst + (size_t)blockIdx.y * n;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    d[r] = s[storage_index(r, nx, ny, s0, s1, s2)];
}

// A plain copy of n doubles (coalesced loads and stores): the device writing
// page-locked host memory that it addresses.
__global__ void k_copy_f64(const double* __restrict__ src, double* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

unsigned blocks_for(long long n) {
  const long long b = (n + 255) / 256;
  return (unsigned)std::min<long long>(b, 4096);
}

}  // namespace

cudaError_t launch_to_storage(const float* src, float* dst, int nx, int ny, int nz, const int strides[3],
                              cudaStream_t stream) {
  const long long n = (long long)nx * ny * nz;
  k_to_storage<<<blocks_for(n), 256, 0, stream>>>(src, dst, nx, ny, n, strides[0], strides[1], strides[2]);
  return cudaGetLastError();
}

cudaError_t launch_from_storage(const double* src, double* dst, int n_lambda, int nx, int ny, int nz,
                                const int strides[3], cudaStream_t stream) {
  const long long n = (long long)nx * ny * nz;
  dim3 grid(blocks_for(n), (unsigned)n_lambda);
  k_from_storage<<<grid, 256, 0, stream>>>(src, dst, nx, ny, n, strides[0], strides[1], strides[2]);
  return cudaGetLastError();
}

cudaError_t launch_copy_f64(const double* src, double* dst, long long n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_copy_f64<<<blocks_for(n), 256, 0, stream>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace rtk

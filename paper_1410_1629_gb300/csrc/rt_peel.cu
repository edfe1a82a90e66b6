// The sorted peel-off pass of the cartesian forward launch: the walks of the
// peel-offs that the transport kernel (rt_forward.cu) recorded, ordered by
// instrument and start cell.
#include "rt_transport.cuh"

namespace rtk {

namespace {

// ---- the sorted peel-off pass
//
// The transport kernel hands each walked peel-off to this pass as a record
// (start point, weight, phase-function value) counted under its sort key
// (instrument, cell of the start point).  Ordered by key, the records of a
// warp start in the same or neighbouring cells and walk parallel rays
// towards one instrument, so their density loads fall on the same cache
// lines; in the transport kernel the lanes of a warp walk unrelated rays.
// Each walk is the transport kernel's own (same arithmetic, same optical
// depth pair, same deposit), so only the order of the FP64 image additions
// differs from walking the peel-off in place.

constexpr int kScanTile = 4096;  // keys per block of the scan (256 threads x 16)

// Exclusive scan of each tile of 4096 key counts in place; tile totals out.
__global__ void __launch_bounds__(256) k_peel_scan_tiles(unsigned* __restrict__ h, unsigned long long n,
                                                          unsigned* __restrict__ tile_sum) {
  __shared__ unsigned warp_tot[8];
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const unsigned long long base = (unsigned long long)blockIdx.x * kScanTile + threadIdx.x * 16ull;
  unsigned v[16];
  unsigned sum = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    v[j] = base + j < n ? h[base + j] : 0u;
    sum += v[j];
  }
  unsigned incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned w = lane < 8 ? warp_tot[lane] : 0u;
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (unsigned)o) wi += t;
    }
    if (lane < 8) warp_tot[lane] = wi - w;
    if (lane == 7) tile_sum[blockIdx.x] = wi;
  }
  __syncthreads();
  unsigned run = warp_tot[warp] + incl - sum;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (base + j < n) h[base + j] = run;
    run += v[j];
  }
}

// Exclusive scan of the tile totals in place (one block).
__global__ void __launch_bounds__(1024) k_peel_scan_sums(unsigned* __restrict__ ts, unsigned long long n) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned carry;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (unsigned long long b = 0; b < n; b += 1024) {
    const unsigned long long i = b + threadIdx.x;
    const unsigned v = i < n ? ts[i] : 0u;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const unsigned w = warp_tot[lane];
      unsigned wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= (unsigned)o) wi += t;
      }
      warp_tot[lane] = wi - w;
    }
    __syncthreads();
    const unsigned c0 = carry;
    const unsigned ex = c0 + warp_tot[warp] + incl - v;
    if (i < n) ts[i] = ex;
    __syncthreads();
    if (threadIdx.x == 1023) carry = ex + v;
    __syncthreads();
  }
}

// The permutation that orders the records by key: a record's place is its
// tile's base, plus its key's offset in the tile, plus the records of that
// key placed before it.
__global__ void __launch_bounds__(256) k_peel_scatter(const PeelRecord* __restrict__ rec,
                                                       const unsigned long long* __restrict__ count,
                                                       unsigned long long cap, unsigned* __restrict__ h,
                                                       const unsigned* __restrict__ tile_sum,
                                                       unsigned* __restrict__ perm) {
  const unsigned long long n = min(*count, cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned key = __ldg(&rec[i].key);
    const unsigned pos = tile_sum[key / kScanTile] + atomicAdd(&h[key], 1u);
    perm[pos] = (unsigned)i;
  }
}

// The walks of the sorted records and their deposits; one record per thread,
// consecutive threads on consecutive records of the order.
__global__ void __launch_bounds__(256) k_peel_sorted(const FwdParams P, const unsigned* __restrict__ perm) {
  for (int i = threadIdx.x; i < P.n_instr; i += blockDim.x) tr::S_INSTR[i] = P.instr[i];
  for (int i = threadIdx.x; i < P.n_lambda; i += blockDim.x) tr::S_LAM[i] = P.lam[i];
  __syncthreads();
  const unsigned long long n = min(*P.peel_count, P.peel_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && n) atomicAdd(&P.counters[8], n);
  const unsigned stride_k = (unsigned)(P.n_cells + 1);
  unsigned long long crossings = 0;
  for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
       j += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned i = perm[j];
    const float4* r = reinterpret_cast<const float4*>(&P.peel[i]);
    const float4 a = r[0], b = r[1];
    const unsigned key = __float_as_uint(a.w);
    const unsigned meta = __float_as_uint(b.w);
    const int q = (int)(key / stride_k);
    const unsigned c = key - (unsigned)q * stride_k;
    const int lam = (int)(meta & 0xffffu);
    const bool known = (meta >> 31) != 0u;
    const double L = __hiloint2double(__float_as_int(b.y), __float_as_int(b.x));
    const float3 x = make_float3(a.x, a.y, a.z);
    const DevInstr& I = tr::S_INSTR[q];
    tr::CartGrid::Cell cell;
    cell.ix = (int)(c % (unsigned)P.nx);
    cell.iy = (int)((c / (unsigned)P.nx) % (unsigned)P.ny);
    cell.iz = (int)(c / ((unsigned)P.nx * (unsigned)P.ny));
    float th, tl;
    crossings += tr::ray_tau(P, x, tr::instr_dir(I), known, cell, tr::S_LAM[lam].kappa, th, tl);
    const ulonglong2 tag = P.peel_tag ? P.peel_tag[i] : make_ulonglong2(0ull, 0ull);
    tr::deposit_peel(P, q, lam, x, L, b.z, th, tl, (meta >> 30) & 1u, tag.x, (int)tag.y);
  }
  for (int o = 16; o > 0; o >>= 1) crossings += __shfl_down_sync(0xffffffffu, crossings, o);
  if ((threadIdx.x & 31u) == 0 && crossings) atomicAdd(&P.counters[0], crossings);
}

}  // namespace

cudaError_t launch_peel_pass(const FwdParams& p, unsigned long long n_keys, unsigned* tile_sum, unsigned* perm,
                             int num_sms, cudaStream_t stream, cudaEvent_t mid) {
  const unsigned long long n_tiles = (n_keys + kScanTile - 1) / kScanTile;
  k_peel_scan_tiles<<<(unsigned)n_tiles, 256, 0, stream>>>(p.peel_hist, n_keys, tile_sum);
  k_peel_scan_sums<<<1, 1024, 0, stream>>>(tile_sum, n_tiles);
  k_peel_scatter<<<(unsigned)num_sms * 8u, 256, 0, stream>>>(p.peel, p.peel_count, p.peel_cap, p.peel_hist, tile_sum,
                                                            perm);
  if (mid) {
    const cudaError_t em = cudaEventRecord(mid, stream);
    if (em != cudaSuccess) return em;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel_sorted, 256, 0);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  k_peel_sorted<<<(unsigned)num_sms * (unsigned)per_sm, 256, 0, stream>>>(p, perm);
  return cudaGetLastError();
}

}  // namespace rtk

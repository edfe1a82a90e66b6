// Panchromatic mode (SKIRT paper, Sect. 2.1 and 2.2): the equilibrium
// temperature of the dust in every cell from the luminosity it absorbed over
// the wavelength grid, the dust's thermal emission per cell and wavelength,
// and the running sums over the cells from which the transport kernel draws
// the emitting cell of a dust-emission packet.
//
//   emission of cell c at temperature T: S m_c sum_l w_l beta_l(T), with
//   m_c = rho_c V_c, w_l = kappa_l (1 - albedo_l) dlambda_l (the host's
//   per-wavelength weights, S folded in), beta_l(T) = lambda_l^-5 /
//   (exp(C2 / (lambda_l T)) - 1), lambda in um, C2 = hc/k in um K.
//   The temperature solves emission = absorbed luminosity in ln T between
//   ln t_min and ln t_max (Newton steps kept in a bisection bracket: a
//   single-precision estimate, then double precision to 1e-15); no absorption or
//   no dust: 0; short of the absorption at t_max: t_max, beyond it at t_min:
//   t_min (both counted).
// All of it is FP64: it runs once per temperature update, not per crossing.
#include "rt_internal.h"

namespace rtk {

namespace {

constexpr double kC2 = 14387.768775039337;  // hc / k in um K

struct DustArgs {
  int n_lambda, nx, ny, nz;
  long long n_cells;
  int stride[3];          // storage strides of the absorption tallies
  const double* planes;   // FP64 cell planes: x [nx + 1], y [ny + 1], z [nz + 1]
  const float* density;   // row-major
  double a[kMaxLambda];   // S kabs_l dlambda_l / lambda_l^5
  double b[kMaxLambda];   // C2 / lambda_l
  float af[kMaxLambda];   // a_l / max a_l
  float bf[kMaxLambda];   // b_l
  double ln_a_max;
};

__device__ __forceinline__ double cell_mass(const DustArgs& A, long long c, int& ix, int& iy, int& iz) {
  ix = (int)(c % A.nx);
  iy = (int)((c / A.nx) % A.ny);
  iz = (int)(c / ((long long)A.nx * A.ny));
  const double* px = A.planes;
  const double* py = A.planes + A.nx + 1;
  const double* pz = py + A.ny + 1;
  const double V = (px[ix + 1] - px[ix]) * (py[iy + 1] - py[iy]) * (pz[iz + 1] - pz[iz]);
  return (double)A.density[c] * V;
}

// Emission per unit mass at T, sum_l a_l / (exp(b_l / T) - 1), and its
// derivative with respect to ln T; Real is double, or float with the a_l
// scaled by 1 / max a_l (a first estimate of the root only).
template <class Real>
__device__ __forceinline__ Real emission(int n, const Real* a, const Real* b, Real T, Real* d_dlnT = nullptr) {
  Real sum = 0, der = 0;
  for (int l = 0; l < n; ++l) {
    const Real x = b[l] / T;
    const Real em1 = expm1(x);
    const Real t = a[l] / em1;
    sum += t;
    if (d_dlnT) der += t * x * (Real(1) + Real(1) / em1);
  }
  if (d_dlnT) *d_dlnT = der;
  return sum;
}

// Root of ln E(exp(u)) = target in u within [lo, hi]: Newton steps, replaced by
// the bracket's midpoint where they leave it, until a step (or the bracket)
// is below tol relative to max(1, |u|).
template <class Real>
__device__ __forceinline__ Real solve_ln_t(int n, const Real* a, const Real* b, Real target, Real lo, Real hi,
                                           Real u, Real tol, int max_it) {
  for (int it = 0; it < max_it; ++it) {
    Real der;
    const Real e = emission(n, a, b, exp(u), &der);
    const Real f = log(e) - target;
    if (f < Real(0)) lo = u; else hi = u;
    const Real un = u - f * e / der;
    const Real scale = fmax(Real(1), fabs(u));
    if (fabs(un - u) <= tol * scale) return un;
    u = un >= lo && un <= hi ? un : Real(0.5) * (lo + hi);
    if (hi - lo <= tol * scale) break;
  }
  return u;
}

// absorbed: row-major [n_lambda][n_cells] (a caller's field) or, when
// stored is set, the context's tallies in storage order.
__global__ void k_dust_temperature(const DustArgs A, const double* __restrict__ absorbed, int stored,
                                   double t_min, double t_max, double* __restrict__ T, unsigned* clamped) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < A.n_cells;
       c += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    const double m = cell_mass(A, c, ix, iy, iz);
    const long long slot = stored ? (long long)ix * A.stride[0] + (long long)iy * A.stride[1] +
                                        (long long)iz * A.stride[2]
                                  : c;
    double ab = 0.0;
    for (int l = 0; l < A.n_lambda; ++l) ab += absorbed[(size_t)l * A.n_cells + slot];
    const double top = m * emission(A.n_lambda, A.a, A.b, t_max);
    if (!(ab > 0.0) || !(m > 0.0) || !(top > 0.0)) {
      T[c] = 0.0;
      continue;
    }
    if (top < ab) {
      T[c] = t_max;
      atomicAdd(clamped, 1u);
      continue;
    }
    if (m * emission(A.n_lambda, A.a, A.b, t_min) >= ab) {
      T[c] = t_min;
      atomicAdd(clamped, 1u);
      continue;
    }
    // the root of ln(m E(T)) = ln(absorbed) in u = ln T: a single-precision
    // estimate to 1e-6, then double-precision steps to 1e-15 (the root the
    // oracle's bisection converges to)
    const double lo = log(t_min), hi = log(t_max);
    const double target = log(ab / m);
    const float u32 = solve_ln_t<float>(A.n_lambda, A.af, A.bf, (float)(target - A.ln_a_max), (float)lo,
                                        (float)hi, (float)(0.5 * (lo + hi)), 1e-6f, 60);
    const double u0 = (double)u32 > lo && (double)u32 < hi ? (double)u32 : 0.5 * (lo + hi);
    const double u = solve_ln_t<double>(A.n_lambda, A.a, A.b, target, lo, hi, u0, 1e-15, 200);
    T[c] = exp(u);
  }
}

// lum[l][c] = m_c w_l beta_l(T_c) (T = 0: none), row-major cells.
__global__ void k_dust_luminosity(const DustArgs A, const double* __restrict__ T, double* __restrict__ lum) {
  const int l = blockIdx.y;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < A.n_cells;
       c += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    const double m = cell_mass(A, c, ix, iy, iz);
    const double t = T[c];
    lum[(size_t)l * A.n_cells + c] = t > 0.0 ? m * (A.a[l] / expm1(A.b[l] / t)) : 0.0;
  }
}

// ---- inclusive running sums over the cells, per wavelength (blockIdx.y):
// tile totals, their exclusive scan, then each tile's scan plus its offset.
constexpr int kTile = 4096;  // 256 threads x 16 values

__device__ __forceinline__ double block_exclusive(double v, double* warp_tot, double& total) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  double incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const double w = lane < (blockDim.x >> 5) ? warp_tot[lane] : 0.0;
    double wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (unsigned)o) wi += t;
    }
    if (lane < (blockDim.x >> 5)) warp_tot[lane] = wi - w;
    if (lane == (blockDim.x >> 5) - 1) warp_tot[32] = wi;
  }
  __syncthreads();
  total = warp_tot[32];
  const double ex = warp_tot[warp] + incl - v;
  __syncthreads();
  return ex;
}

__global__ void __launch_bounds__(256) k_tile_sums(const double* __restrict__ x, long long n, double* tile_sum,
                                                   long long n_tiles) {
  __shared__ double warp_tot[33];
  const double* row = x + (size_t)blockIdx.y * n;
  const long long base = (long long)blockIdx.x * kTile + threadIdx.x * 16ll;
  double s = 0.0;
  for (int j = 0; j < 16; ++j)
    if (base + j < n) s += row[base + j];
  double total;
  block_exclusive(s, warp_tot, total);
  if (threadIdx.x == 0) tile_sum[(size_t)blockIdx.y * n_tiles + blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_tile_sums(double* ts, long long n_tiles) {
  __shared__ double warp_tot[33];
  __shared__ double carry;
  double* row = ts + (size_t)blockIdx.x * n_tiles;
  if (threadIdx.x == 0) carry = 0.0;
  __syncthreads();
  for (long long b = 0; b < n_tiles; b += blockDim.x) {
    const long long i = b + threadIdx.x;
    const double v = i < n_tiles ? row[i] : 0.0;
    double total;
    const double ex = block_exclusive(v, warp_tot, total);
    const double c0 = carry;
    if (i < n_tiles) row[i] = c0 + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = c0 + total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_tile_scan(double* __restrict__ x, long long n, const double* tile_off,
                                                   long long n_tiles) {
  __shared__ double warp_tot[33];
  double* row = x + (size_t)blockIdx.y * n;
  const long long base = (long long)blockIdx.x * kTile + threadIdx.x * 16ll;
  double v[16];
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    v[j] = base + j < n ? row[base + j] : 0.0;
    s += v[j];
  }
  double total;
  double run = tile_off[(size_t)blockIdx.y * n_tiles + blockIdx.x] + block_exclusive(s, warp_tot, total);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    run += v[j];
    if (base + j < n) row[base + j] = run;
  }
}

DustArgs make_args(int n_lambda, int nx, int ny, int nz, const int stride[3], const double* planes,
                   const float* density, const double* w, const double* lambda) {
  DustArgs A;
  A.n_lambda = n_lambda;
  A.nx = nx; A.ny = ny; A.nz = nz;
  A.n_cells = (long long)nx * ny * nz;
  for (int a = 0; a < 3; ++a) A.stride[a] = stride[a];
  A.planes = planes;
  A.density = density;
  double a_max = 0.0;
  for (int l = 0; l < kMaxLambda; ++l) {
    const double lam = l < n_lambda ? lambda[l] : 1.0;
    A.a[l] = l < n_lambda ? w[l] / (lam * lam * lam * lam * lam) : 0.0;
    A.b[l] = kC2 / lam;
    a_max = A.a[l] > a_max ? A.a[l] : a_max;
  }
  if (!(a_max > 0.0)) a_max = 1.0;
  A.ln_a_max = std::log(a_max);
  for (int l = 0; l < kMaxLambda; ++l) {
    A.af[l] = (float)(A.a[l] / a_max);
    A.bf[l] = (float)A.b[l];
  }
  return A;
}

unsigned cell_blocks(long long n) { return (unsigned)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192); }

}  // namespace

cudaError_t launch_dust_temperature(int n_lambda, int nx, int ny, int nz, const int stride[3], const double* planes,
                                    const float* density, const double* w, const double* lambda,
                                    const double* absorbed, int stored, double t_min, double t_max, double* T,
                                    unsigned* clamped, cudaStream_t s) {
  const DustArgs A = make_args(n_lambda, nx, ny, nz, stride, planes, density, w, lambda);
  k_dust_temperature<<<cell_blocks(A.n_cells), 256, 0, s>>>(A, absorbed, stored, t_min, t_max, T, clamped);
  return cudaGetLastError();
}

cudaError_t launch_dust_emission(int n_lambda, int nx, int ny, int nz, const int stride[3], const double* planes,
                                 const float* density, const double* w, const double* lambda, const double* T,
                                 double* lum, double* cum, double* tile_sum, cudaStream_t s) {
  const DustArgs A = make_args(n_lambda, nx, ny, nz, stride, planes, density, w, lambda);
  const long long n = A.n_cells;
  k_dust_luminosity<<<dim3(cell_blocks(n), (unsigned)n_lambda), 256, 0, s>>>(A, T, lum);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(cum, lum, (size_t)n_lambda * n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  const long long n_tiles = (n + kTile - 1) / kTile;
  k_tile_sums<<<dim3((unsigned)n_tiles, (unsigned)n_lambda), 256, 0, s>>>(cum, n, tile_sum, n_tiles);
  k_scan_tile_sums<<<(unsigned)n_lambda, 1024, 0, s>>>(tile_sum, n_tiles);
  k_tile_scan<<<dim3((unsigned)n_tiles, (unsigned)n_lambda), 256, 0, s>>>(cum, n, tile_sum, n_tiles);
  return cudaGetLastError();
}

long long dust_tiles(long long n_cells) { return (n_cells + kTile - 1) / kTile; }

}  // namespace rtk

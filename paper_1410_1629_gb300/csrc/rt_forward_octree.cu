// Forward transport kernel for octree grids (SKIRT paper, Sect. 2.4): the same
// per-packet algorithm as the cartesian kernel, one thread per packet.
//
// Execution model: a persistent grid (a few blocks per SM); every warp takes
// 32 consecutive packet indices from a global counter at a time, so a launch
// adapts to the uneven cost of packets.  Packets are ordered wavelength-major,
// so at any time the absorption tallies being updated are one wavelength's
// slice.  Geometry, the walk and the phase function are FP32; the cumulative
// optical depth of the forced path (which places the interaction), the packet
// weight and every accumulator are FP64.
#include <cuda_runtime.h>

#include "rt_device.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

struct Acc {
  double emitted = 0.0, escaped = 0.0, absorbed = 0.0, truncated = 0.0;
  unsigned long long crossings = 0, path_crossings = 0, events = 0, peeloffs = 0, packets = 0;
};

__device__ __forceinline__ float dot3(float3 a, const float* b) { return a.x * b[0] + a.y * b[1] + a.z * b[2]; }

// Peel-off towards every instrument from x (in cell `ref`) with weight
// L * factor * exp(-tau(x -> observer)); factor = 1/(4 pi) for emission and
// Phi(k . k_obs)/(4 pi) for scattering.
template <int GRID>
__device__ __forceinline__ void peel_all(const FwdParams& P, float3 x, float3 k, const CellRef& ref, int lam,
                                         float kappa, float g, double L, bool scattered,
                                         unsigned long long pid, int event, Acc& acc) {
  for (int q = 0; q < P.n_instr; ++q) {
    const DevInstr& I = P.instr[q];
    const float3 kobs = make_float3(I.kobs[0], I.kobs[1], I.kobs[2]);
    const float phase = scattered ? hg_phase(g, k.x * kobs.x + k.y * kobs.y + k.z * kobs.z) : 1.0f;
    float tau = 0.0f;
    const unsigned n = Walker<GRID>::walk(P, x, kobs, ref, [&](int c, float, float ds, const CellRef&) {
      tau = fmaf(kappa * __ldg(&P.density[c]), ds, tau);
      return true;
    });
    acc.crossings += n;
    acc.peeloffs += 1;
    const double value = L * kInv4PiD * (double)phase * exp(-(double)tau);
    const float fx = (dot3(x, I.ex) + I.off_x) * I.sx;
    const float fy = (dot3(x, I.ey) + I.off_y) * I.sy;
    const size_t plane = (size_t)I.ny * I.nx;
    const int ch = scattered ? 2 : 1;
    if (!I.bilinear) {
      const float fix = floorf(fx), fiy = floorf(fy);
      if (!(fix >= 0.0f && fiy >= 0.0f && fix < (float)I.nx && fiy < (float)I.ny)) continue;
      const int ix = (int)fix, iy = (int)fiy;
      const size_t pix = (size_t)iy * I.nx + ix;
      atomicAdd(&I.image[(size_t)lam * plane + pix], value);
      if (I.channels == 3) atomicAdd(&I.image[((size_t)ch * P.n_lambda + lam) * plane + pix], value);
      if (P.records && (P.record_stride <= 1 || pid % P.record_stride == 0)) {
        const unsigned long long slot = atomicAdd(&P.counters[4], 1ull);
        if ((long long)slot < P.records_cap) {
          rt_record r;
          r.packet = pid; r.lambda = lam; r.event = event; r.instrument = q; r.reserved = 0;
          r.pixel = (int64_t)pix; r.value = value;
          P.records[slot] = r;
        }
      }
    } else {
      const float gx = fx - 0.5f, gy = fy - 0.5f;
      const float x0 = floorf(gx), y0 = floorf(gy);
      const float tx = gx - x0, ty = gy - y0;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float fix = x0 + dx, fiy = y0 + dy;
          if (!(fix >= 0.0f && fiy >= 0.0f && fix < (float)I.nx && fiy < (float)I.ny)) continue;
          const double v = value * (double)((dx ? tx : 1.0f - tx) * (dy ? ty : 1.0f - ty));
          const size_t pix = (size_t)(int)fiy * I.nx + (int)fix;
          atomicAdd(&I.image[(size_t)lam * plane + pix], v);
          if (I.channels == 3) atomicAdd(&I.image[((size_t)ch * P.n_lambda + lam) * plane + pix], v);
        }
      }
    }
  }
}

// Emission (Sect. 3.4): source component by luminosity, position from its
// geometry (FP64, rounded to FP32), isotropic direction.
__device__ __forceinline__ void emit(const FwdParams& P, unsigned long long pid, int lam, float3& x, float3& k) {
  const uint4 r0 = draw_block(pid, lam, 0, 0, P.seed, P.model);
  const uint4 r1 = draw_block(pid, lam, 0, 1, P.seed, P.model);
  const double u0 = u01(r0.x), u1 = u01(r0.y), u2 = u01(r0.z), u3 = u01(r0.w);
  const double u4 = u01(r1.x), u5 = u01(r1.y), u6 = u01(r1.z), u7 = u01(r1.w);
  int s = P.n_sources - 1;
  for (int i = 0; i < P.n_sources; ++i) {
    if (u0 < P.src_cum[lam * P.n_sources + i]) { s = i; break; }
  }
  const DevSource S = P.src[s];
  double px = S.center[0], py = S.center[1], pz = S.center[2];
  if (S.kind == RT_SOURCE_EXPDISK) {
    const double R = -S.scale_r * log(u1 * u2);
    double sp, cp;
    sincospi(2.0 * u3, &sp, &cp);
    double z = -S.scale_z * log(u4);
    if (u5 < 0.5) z = -z;
    px += R * cp; py += R * sp; pz += z;
  } else if (S.kind == RT_SOURCE_PLUMMER) {
    const double r = S.scale_r / sqrt(pow(u1, -2.0 / 3.0) - 1.0);
    const double ct = 2.0 * u2 - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double sp, cp;
    sincospi(2.0 * u3, &sp, &cp);
    px += r * st * cp; py += r * st * sp; pz += r * ct;
  }
  x = make_float3((float)px, (float)py, (float)pz);
  const float mu = (float)(2.0 * u6 - 1.0);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
  float sp, cp;
  sincospif((float)(2.0 * u7), &sp, &cp);
  k = make_float3(st * cp, st * sp, mu);
}

__device__ __forceinline__ void trace_row(const FwdParams& P, unsigned long long pid, int lam, int event, int cell,
                                          float3 x, float3 k, double L, double tau_path, double tau_star) {
  if (!P.trace || pid != P.trace_packet || lam != P.trace_lambda || event >= P.trace_cap) return;
  rt_trace_row r;
  r.event = event; r.reserved = 0; r.cell = cell;
  r.x[0] = x.x; r.x[1] = x.y; r.x[2] = x.z;
  r.k[0] = k.x; r.k[1] = k.y; r.k[2] = k.z;
  r.L = L; r.tau_path = tau_path; r.tau_star = tau_star;
  P.trace[event] = r;
}

template <int GRID>
__device__ void run_packet(const FwdParams& P, unsigned long long pid, int lam, Acc& acc) {
  const DevLambda LP = P.lam[lam];
  const float kappa = LP.kappa, g = LP.g;
  const double albedo = LP.albedo;
  const double L0 = LP.lum_total / (double)P.n_norm;
  float3 x, k;
  emit(P, pid, lam, x, k);
  double L = L0;
  acc.emitted += L0;
  acc.packets += 1;
  CellRef cell;
  cell.cell = -1;
  trace_row(P, pid, lam, 0, -1, x, k, L, 0.0, 0.0);
  if (P.peel_emission) peel_all<GRID>(P, x, k, cell, lam, kappa, g, L, false, pid, 0, acc);
  double* __restrict__ absorb = P.absorption + (size_t)lam * P.n_cells;
  for (int j = 1;; ++j) {
    // forced path, first pass: optical depth to the boundary and continuous absorption
    const float wabs = (float)((1.0 - albedo) * L);
    double tau = 0.0;
    float tauf = 0.0f;
    const unsigned n = Walker<GRID>::walk(P, x, k, cell, [&](int c, float, float ds, const CellRef&) {
      const float dt = kappa * __ldg(&P.density[c]) * ds;
      if (dt > 0.0f) {
        const float dep = wabs * __expf(-tauf) * -expm1f(-dt);
        atomicAdd(&absorb[c], (double)dep);
      }
      tauf += dt;
      tau += (double)dt;
      return true;
    });
    acc.crossings += n;
    acc.path_crossings += n;
    if (!(tau > 0.0)) {
      trace_row(P, pid, lam, j, -1, x, k, L, 0.0, 0.0);
      acc.escaped += L;
      return;
    }
    const double E = exp(-tau);
    const double one_minus_E = -expm1(-tau);
    acc.escaped += L * E;
    acc.absorbed += (1.0 - albedo) * L * one_minus_E;
    // forced scattering: invert the cumulative optical depth (FP64)
    const uint4 r = draw_block(pid, lam, j, 0, P.seed, P.model);
    const double tau_star = -log1p(-u01(r.x) * one_minus_E);
    double tau2 = 0.0;
    bool found = false;
    float s_star = 0.0f, last_out = 0.0f;
    CellRef hit, last;
    hit.cell = -1;
    last.cell = -1;
    Walker<GRID>::walk(P, x, k, cell, [&](int c, float t_in, float ds, const CellRef& ref) {
      const float kr = kappa * __ldg(&P.density[c]);
      const float dt = kr * ds;
      const double t_next = tau2 + (double)dt;
      if (t_next > tau2) { last = ref; last_out = t_in + ds; }
      if (t_next > tau_star) {
        hit = ref;
        s_star = t_in + (float)(tau_star - tau2) / kr;
        found = true;
        return false;
      }
      tau2 = t_next;
      return true;
    });
    if (!found) { hit = last; s_star = last_out; }
    if (hit.cell < 0) {  // cannot happen with tau > 0; keep the packet well defined
      acc.truncated += L;
      return;
    }
    x = make_float3(fmaf(s_star, k.x, x.x), fmaf(s_star, k.y, x.y), fmaf(s_star, k.z, x.z));
    {
      float lo[3], hi[3];
      Walker<GRID>::box(P, hit, lo, hi);
      x.x = fminf(fmaxf(x.x, lo[0]), hi[0]);
      x.y = fminf(fmaxf(x.y, lo[1]), hi[1]);
      x.z = fminf(fmaxf(x.z, lo[2]), hi[2]);
    }
    cell = hit;
    L = albedo * L * one_minus_E;
    acc.events += 1;
    trace_row(P, pid, lam, j, cell.cell, x, k, L, tau, tau_star);
    if (P.peel_scatter) peel_all<GRID>(P, x, k, cell, lam, kappa, g, L, true, pid, j, acc);
    // Henyey-Greenstein direction
    const float mu = hg_sample(g, (float)u01(r.y));
    float sp, cp;
    sincospif((float)(2.0 * u01(r.z)), &sp, &cp);
    k = rotate_dir(k, mu, sp, cp);
    if ((P.weight_cut && L < P.w_min * L0) || j >= P.max_events) {
      acc.truncated += L;
      return;
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int GRID>
__global__ void __launch_bounds__(256) k_forward(const FwdParams P) {
  const int lane = threadIdx.x & 31;
  Acc acc;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(P.work_counter, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= P.n_total) break;
    const unsigned long long w = base + lane;
    if (w < P.n_total) {
      const int lam = (int)(w / P.n_per_lambda);
      const unsigned long long pid = P.first_id + (w - (unsigned long long)lam * P.n_per_lambda);
      run_packet<GRID>(P, pid, lam, acc);
    }
    __syncwarp();
  }
  const double s0 = warp_sum(acc.emitted), s1 = warp_sum(acc.escaped), s2 = warp_sum(acc.absorbed),
               s3 = warp_sum(acc.truncated);
  const unsigned long long c0 = warp_sum(acc.crossings), c1 = warp_sum(acc.events), c2 = warp_sum(acc.peeloffs),
                           c3 = warp_sum(acc.packets), c4 = warp_sum(acc.path_crossings);
  if (lane == 0) {
    (void)s0;
    atomicAdd(&P.stats[1], s1);
    atomicAdd(&P.stats[2], s2); atomicAdd(&P.stats[3], s3);
    atomicAdd(&P.counters[0], c0); atomicAdd(&P.counters[1], c1);
    atomicAdd(&P.counters[2], c2); atomicAdd(&P.counters[3], c3);
    atomicAdd(&P.counters[5], c4);
  }
}

}  // namespace

cudaError_t launch_forward_octree(const FwdParams& p, int num_sms, cudaStream_t stream) {
  const int block_size = 256;
  cudaError_t e = cudaMemsetAsync(p.work_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forward<RT_GRID_OCTREE>, block_size, 0);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  unsigned long long warps_needed = (p.n_total + 31) / 32;
  unsigned long long blocks = (unsigned long long)num_sms * per_sm;
  const unsigned long long max_useful = (warps_needed * 32 + block_size - 1) / block_size;
  if (blocks > max_useful) blocks = max_useful;
  if (blocks < 1) blocks = 1;
  k_forward<RT_GRID_OCTREE><<<(unsigned)blocks, block_size, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk

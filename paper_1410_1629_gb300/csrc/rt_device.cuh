// Device primitives of the transport kernels: counter-based random numbers,
// Henyey-Greenstein scattering, direction rotation, and the grid box tests
// of the cell walks.  Geometry is FP32.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rt_internal.h"

namespace rtk {

#define RT_INF __int_as_float(0x7f800000)

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror & Shaw (2011), "Parallel random numbers: as easy as
// 1, 2, 3": ten rounds of two 32x32->64 multiplications whose halves are
// permuted and XORed with a Weyl-sequence round key.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Random block for (packet, wavelength, event, block): counter =
// (pid low, pid high, event, (lambda << 8) | block), key = (seed, model).
static __device__ __noinline__ uint4 draw_block(unsigned long long pid, int lam, int event, int block,
                                        uint32_t seed, uint32_t model) {
  return philox4x32_10(make_uint4((uint32_t)pid, (uint32_t)(pid >> 32), (uint32_t)event,
                                  ((uint32_t)lam << 8) | (uint32_t)block),
                       seed, model);
}

// Uniform in (0, 1): (r + 1/2) 2^-32 = (2r + 1) 2^-33, exact in FP64, built
// from the 33-bit odd integer with integer operations (normalise by its
// leading zeros): the same value as the FP64 arithmetic, off the FP64 pipe.
__device__ __forceinline__ double u01(uint32_t r) {
  const unsigned long long m = 2ull * r + 1ull;
  const int lz = __clzll((long long)m);
  const unsigned long long bits = ((unsigned long long)(1053 - lz) << 52) | (((m << lz) << 1) >> 12);
  return __longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------- scattering
constexpr double kInv4PiD = 0.0795774715459476679;

// Henyey-Greenstein phase function, normalised to a mean of 1 over the sphere.
__device__ __forceinline__ float hg_phase(float g, float mu) {
  const float den = fmaf(-2.0f * g, mu, fmaf(g, g, 1.0f));
  return (1.0f - g * g) / (den * sqrtf(den));
}

// Cosine drawn from the HG distribution by inverting its CDF.
__device__ __forceinline__ float hg_sample(float g, float u) {
  if (fabsf(g) < 1e-6f) return 2.0f * u - 1.0f;
  const float f = (1.0f - g * g) / fmaf(2.0f * g, u, 1.0f - g);
  const float mu = (fmaf(g, g, 1.0f) - f * f) / (2.0f * g);
  return fminf(1.0f, fmaxf(-1.0f, mu));
}

// Direction at cosine mu to k and azimuth (sin_p, cos_p) about k, right-handed.
__device__ __forceinline__ float3 rotate_dir(float3 k, float mu, float sin_p, float cos_p) {
  const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
  const float s = sqrtf(k.x * k.x + k.y * k.y);
  float3 n;
  if (s == 0.0f) {
    n = k.z > 0.0f ? make_float3(st * cos_p, st * sin_p, mu) : make_float3(st * cos_p, -st * sin_p, -mu);
  } else {
    const float cx = k.x / s, cy = k.y / s;
    n.x = mu * k.x + st * (cos_p * cx * k.z - sin_p * cy);
    n.y = mu * k.y + st * (cos_p * cy * k.z + sin_p * cx);
    n.z = mu * k.z - st * cos_p * s;
  }
  const float inv = rsqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
  return make_float3(n.x * inv, n.y * inv, n.z * inv);
}

// ---------------------------------------------------------------- cell walks
__device__ __forceinline__ float comp3(float3 v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// Entry of a ray that starts outside the grid box (slab method).  Returns false
// if the ray misses; otherwise t_in and the entry axis.  Geo: any type with
// the box lo[3], hi[3] (the launch parameters, or one model of a batch).
template <class Geo>
__device__ __forceinline__ bool ray_box_entry(const Geo& P, float3 x, float3 k, float3 ik, float& t_in, int& axis) {
  float tin = -RT_INF, tout = RT_INF;
  axis = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float xa = comp3(x, a), ka = comp3(k, a), ika = comp3(ik, a);
    if (ka == 0.0f) {
      if (xa < P.lo[a] || xa > P.hi[a]) return false;
      continue;
    }
    const float t1 = (P.lo[a] - xa) * ika, t2 = (P.hi[a] - xa) * ika;
    const float tn = fminf(t1, t2), tf = fmaxf(t1, t2);
    if (tn > tin) { tin = tn; axis = a; }
    tout = fminf(tout, tf);
  }
  if (!(tin < tout) || tout <= 0.0f) return false;
  const float ka = comp3(k, axis);
  const float plane = ka > 0.0f ? P.lo[axis] : P.hi[axis];
  t_in = (plane - comp3(x, axis)) * comp3(ik, axis);
  return true;
}

template <class Geo>
__device__ __forceinline__ bool inside_box(const Geo& P, float3 x) {
  return x.x >= P.lo[0] && x.x <= P.hi[0] && x.y >= P.lo[1] && x.y <= P.hi[1] && x.z >= P.lo[2] &&
         x.z <= P.hi[2];
}

}  // namespace rtk

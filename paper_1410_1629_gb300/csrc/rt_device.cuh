// Device primitives of the transport kernels: counter-based random numbers,
// Henyey-Greenstein scattering, direction rotation, and the straight-line
// cell walks through cartesian grids and octrees.  Geometry is FP32.
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

// Uniform in (0, 1): (r + 1/2) 2^-32, exact in FP64.
__device__ __forceinline__ double u01(uint32_t r) { return ((double)r + 0.5) * 0x1p-32; }

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
// A located cell.  Cartesian: indices i[3]; octree: leaf id and its box.
struct CellRef {
  int cell;         // cell id (cartesian) or leaf id (octree); < 0: not located
  int i0, i1, i2;   // cartesian indices
  float lo[3], hi[3];  // octree leaf box
};

__device__ __forceinline__ float comp3(float3 v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// Entry of a ray that starts outside the grid box (slab method).  Returns false
// if the ray misses; otherwise t_in and the entry axis.
__device__ __forceinline__ bool ray_box_entry(const FwdParams& P, float3 x, float3 k, float3 ik, float& t_in,
                                              int& axis) {
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

__device__ __forceinline__ bool inside_box(const FwdParams& P, float3 x) {
  return x.x >= P.lo[0] && x.x <= P.hi[0] && x.y >= P.lo[1] && x.y <= P.hi[1] && x.z >= P.lo[2] &&
         x.z <= P.hi[2];
}

__device__ __forceinline__ float safe_inv(float k) { return k != 0.0f ? 1.0f / k : RT_INF; }

// Cartesian grid: walk from x along k, calling f(cell, t_in, ds, ref) for every
// cell segment (zero-length ones included) until f returns false or the ray
// leaves the grid.  `start` is the cell x lies in (cell < 0: locate x, or find
// the entry point when x is outside).  Returns the number of segments visited.
template <class F>
__device__ __forceinline__ unsigned walk_cartesian(const FwdParams& P, float3 x, float3 k, const CellRef& start,
                                                   F&& f) {
  const float3 ik = make_float3(safe_inv(k.x), safe_inv(k.y), safe_inv(k.z));
  int ix, iy, iz;
  float t = 0.0f;
  if (start.cell >= 0) {
    ix = start.i0; iy = start.i1; iz = start.i2;
  } else {
    int entry = -1;
    float3 p = x;
    if (!inside_box(P, x)) {
      if (!ray_box_entry(P, x, k, ik, t, entry)) return 0u;
      p = make_float3(fmaf(t, k.x, x.x), fmaf(t, k.y, x.y), fmaf(t, k.z, x.z));
    }
    ix = min(max(__float2int_rd((p.x - P.lo[0]) * P.inv_d[0]), 0), P.nx - 1);
    iy = min(max(__float2int_rd((p.y - P.lo[1]) * P.inv_d[1]), 0), P.ny - 1);
    iz = min(max(__float2int_rd((p.z - P.lo[2]) * P.inv_d[2]), 0), P.nz - 1);
    if (entry == 0) ix = k.x > 0.0f ? 0 : P.nx - 1;
    if (entry == 1) iy = k.y > 0.0f ? 0 : P.ny - 1;
    if (entry == 2) iz = k.z > 0.0f ? 0 : P.nz - 1;
  }
  const int sx = k.x > 0.0f ? 1 : -1, sy = k.y > 0.0f ? 1 : -1, sz = k.z > 0.0f ? 1 : -1;
  const int ux = k.x > 0.0f, uy = k.y > 0.0f, uz = k.z > 0.0f;
  float tx = k.x != 0.0f ? (fmaf((float)(ix + ux), P.d[0], P.lo[0]) - x.x) * ik.x : RT_INF;
  float ty = k.y != 0.0f ? (fmaf((float)(iy + uy), P.d[1], P.lo[1]) - x.y) * ik.y : RT_INF;
  float tz = k.z != 0.0f ? (fmaf((float)(iz + uz), P.d[2], P.lo[2]) - x.z) * ik.z : RT_INF;
  const int stride_y = P.nx, stride_z = P.nx * P.ny;
  int cell = ix + stride_y * iy + stride_z * iz;
  unsigned n = 0;
  CellRef ref;
  while (true) {
    float te = tx;
    int axis = 0;
    if (ty < te) { te = ty; axis = 1; }
    if (tz < te) { te = tz; axis = 2; }
    const float texit = fmaxf(te, t);
    ++n;
    ref.cell = cell; ref.i0 = ix; ref.i1 = iy; ref.i2 = iz;
    if (!f(cell, t, texit - t, ref)) break;
    t = texit;
    if (axis == 0) {
      ix += sx;
      if ((unsigned)ix >= (unsigned)P.nx) break;
      cell += sx;
      tx = (fmaf((float)(ix + ux), P.d[0], P.lo[0]) - x.x) * ik.x;
    } else if (axis == 1) {
      iy += sy;
      if ((unsigned)iy >= (unsigned)P.ny) break;
      cell += sy * stride_y;
      ty = (fmaf((float)(iy + uy), P.d[1], P.lo[1]) - x.y) * ik.y;
    } else {
      iz += sz;
      if ((unsigned)iz >= (unsigned)P.nz) break;
      cell += sz * stride_z;
      tz = (fmaf((float)(iz + uz), P.d[2], P.lo[2]) - x.z) * ik.z;
    }
  }
  return n;
}

// Octree point location from the root.  On every axis a point on a splitting
// plane goes to the child the ray enters (upper if k_a >= 0, lower if k_a < 0).
__device__ __forceinline__ int octree_locate(const FwdParams& P, float3 p, float3 k, float lo[3], float hi[3]) {
  lo[0] = P.lo[0]; lo[1] = P.lo[1]; lo[2] = P.lo[2];
  hi[0] = P.hi[0]; hi[1] = P.hi[1]; hi[2] = P.hi[2];
  int node = 0;
  int c = __ldg(&P.child[0]);
  int depth = 0;
  while (c >= 0) {
    int oct = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float mid = 0.5f * (lo[a] + hi[a]);
      const float pa = comp3(p, a);
      const bool upper = comp3(k, a) < 0.0f ? (pa > mid) : (pa >= mid);
      if (upper) { oct |= 1 << a; lo[a] = mid; } else { hi[a] = mid; }
    }
    node = c + oct;
    c = __ldg(&P.child[node]);
    if (++depth > kMaxOctreeDepth) { atomicOr(P.flags, kFlagOctreeDepth); return 0; }
  }
  return -c - 1;
}

// Octree: the same contract as walk_cartesian; each next leaf is located from
// the root at the exit point, with the exit coordinate set exactly to the face.
template <class F>
__device__ __forceinline__ unsigned walk_octree(const FwdParams& P, float3 x, float3 k, const CellRef& start,
                                                F&& f) {
  const float3 ik = make_float3(safe_inv(k.x), safe_inv(k.y), safe_inv(k.z));
  CellRef ref;
  float t = 0.0f;
  if (start.cell >= 0) {
    ref = start;
  } else {
    int entry = -1;
    float3 p = x;
    if (!inside_box(P, x)) {
      if (!ray_box_entry(P, x, k, ik, t, entry)) return 0u;
      p = make_float3(fmaf(t, k.x, x.x), fmaf(t, k.y, x.y), fmaf(t, k.z, x.z));
      if (entry == 0) p.x = k.x > 0.0f ? P.lo[0] : P.hi[0];
      if (entry == 1) p.y = k.y > 0.0f ? P.lo[1] : P.hi[1];
      if (entry == 2) p.z = k.z > 0.0f ? P.lo[2] : P.hi[2];
    }
    ref.cell = octree_locate(P, p, k, ref.lo, ref.hi);
  }
  unsigned n = 0;
  while (true) {
    const float tx = k.x != 0.0f ? ((k.x > 0.0f ? ref.hi[0] : ref.lo[0]) - x.x) * ik.x : RT_INF;
    const float ty = k.y != 0.0f ? ((k.y > 0.0f ? ref.hi[1] : ref.lo[1]) - x.y) * ik.y : RT_INF;
    const float tz = k.z != 0.0f ? ((k.z > 0.0f ? ref.hi[2] : ref.lo[2]) - x.z) * ik.z : RT_INF;
    float te = tx;
    int axis = 0;
    if (ty < te) { te = ty; axis = 1; }
    if (tz < te) { te = tz; axis = 2; }
    const float texit = fmaxf(te, t);
    ++n;
    if (!f(ref.cell, t, texit - t, ref)) break;
    t = texit;
    // exit point on the crossed face; the other coordinates stay inside the
    // leaf so that rounding never steps back across a face already crossed
    float3 p = make_float3(fminf(fmaxf(fmaf(t, k.x, x.x), ref.lo[0]), ref.hi[0]),
                           fminf(fmaxf(fmaf(t, k.y, x.y), ref.lo[1]), ref.hi[1]),
                           fminf(fmaxf(fmaf(t, k.z, x.z), ref.lo[2]), ref.hi[2]));
    if (n > kMaxWalkSteps) {
      atomicOr(P.flags, kFlagWalkSteps);
      break;
    }
    if (axis == 0) {
      const float plane = k.x > 0.0f ? ref.hi[0] : ref.lo[0];
      if ((k.x > 0.0f && plane >= P.hi[0]) || (k.x < 0.0f && plane <= P.lo[0])) break;
      p.x = plane;
    } else if (axis == 1) {
      const float plane = k.y > 0.0f ? ref.hi[1] : ref.lo[1];
      if ((k.y > 0.0f && plane >= P.hi[1]) || (k.y < 0.0f && plane <= P.lo[1])) break;
      p.y = plane;
    } else {
      const float plane = k.z > 0.0f ? ref.hi[2] : ref.lo[2];
      if ((k.z > 0.0f && plane >= P.hi[2]) || (k.z < 0.0f && plane <= P.lo[2])) break;
      p.z = plane;
    }
    ref.cell = octree_locate(P, p, k, ref.lo, ref.hi);
  }
  return n;
}

template <int GRID>
struct Walker;
template <>
struct Walker<RT_GRID_CARTESIAN> {
  template <class F>
  __device__ __forceinline__ static unsigned walk(const FwdParams& P, float3 x, float3 k, const CellRef& s, F&& f) {
    return walk_cartesian(P, x, k, s, f);
  }
  __device__ __forceinline__ static void box(const FwdParams& P, const CellRef& r, float lo[3], float hi[3]) {
    lo[0] = fmaf((float)r.i0, P.d[0], P.lo[0]); hi[0] = fmaf((float)(r.i0 + 1), P.d[0], P.lo[0]);
    lo[1] = fmaf((float)r.i1, P.d[1], P.lo[1]); hi[1] = fmaf((float)(r.i1 + 1), P.d[1], P.lo[1]);
    lo[2] = fmaf((float)r.i2, P.d[2], P.lo[2]); hi[2] = fmaf((float)(r.i2 + 1), P.d[2], P.lo[2]);
  }
};
template <>
struct Walker<RT_GRID_OCTREE> {
  template <class F>
  __device__ __forceinline__ static unsigned walk(const FwdParams& P, float3 x, float3 k, const CellRef& s, F&& f) {
    return walk_octree(P, x, k, s, f);
  }
  __device__ __forceinline__ static void box(const FwdParams&, const CellRef& r, float lo[3], float hi[3]) {
    for (int a = 0; a < 3; ++a) { lo[a] = r.lo[a]; hi[a] = r.hi[a]; }
  }
};

}  // namespace rtk

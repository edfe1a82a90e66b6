// The forward transport kernel, templated on the dust grid's cell walk:
// emission, peel-off, forced scattering with continuous absorption,
// Henyey-Greenstein scattering and termination for a stream of photon packets
// (SKIRT paper, Sect. 1 and Sect. 2.2-2.4).
//
// Execution model.  A persistent grid of warps; every lane carries one packet
// through a small state machine.  The expensive part of the method is the
// straight cell walk: per packet a peel-off walk per instrument at emission and
// at every scattering, and two walks of the forced path per scattering (the
// first accumulates the optical depth to the boundary and deposits absorption,
// the second stops at the interaction).  Peel-offs towards a frame along a grid
// axis take their optical depth from per-line column sums; on cartesian grids
// the other peel-offs become records for the sorted pass (rt_peel.cu), which
// walks them after this kernel, ordered by start cell.  The main loop advances
// every walking lane by exactly one cell crossing per iteration, whichever of
// the remaining walks it is in, so the warp stays converged on the hot path.  The per-event work
// (emission, forced-scattering inversion, weight update, deposits, the
// Henyey-Greenstein draw, fetching the next packet) is deferred until enough
// lanes of the warp need it and is then done for those lanes together;
// packets are fetched with one atomic per warp.
//
// Precision.  Geometry, the walk and the phase function are FP32.  The
// cumulative optical depth of the forced path is held as an unevaluated sum
// of two FP32 numbers updated by an error-free two-sum (about 2^-46 relative),
// bit-identical in both walks, so the interaction cell is always found; the
// inversion remainder, E = exp(-tau), tau*, packet weights and every
// accumulator are FP64.
//
// A grid policy G supplies the walk: G::Cell (the cell a position lies in),
// G::Walk (the walk state), init / exit / advance / cell / carried / clamp.
#pragma once

#include <cuda_runtime.h>

#include "rt_device.cuh"
#include "rt_internal.h"

namespace rtk {
namespace tr {

constexpr int kBlock = 256;
constexpr float kInv4PiF = 0.0795774715459476679f;
// Resident blocks per SM the register allocation aims at (4 x 256 threads,
// 64 registers: the per-event lane state lives in shared memory).
#ifndef RT_FWD_MIN_BLOCKS
#define RT_FWD_MIN_BLOCKS 4
#endif

enum Phase : int {
  kFetch = 0,      // needs a new packet
  kPeelEmit = 1,   // peel-off walk at emission (instrument q)
  kPath1 = 2,      // forced path, first walk
  kPath2 = 3,      // forced path, second walk (stops at the interaction)
  kPeelScat = 4,   // peel-off walk at a scattering (instrument q)
  kExit = 5,       // no packets left
  kPeelScan = 6,   // find the next peel-off of the event from instrument q
  kAfter = 7,      // after the scattering peel-offs
  kStart = 8       // start walk `wphase` from x along d
};

// Error-free transformation: a + b = s + e exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

__device__ __forceinline__ float inv_or_zero(float d) { return d != 0.0f ? 1.0f / d : 0.0f; }

// Exact widening of a positive normal FP32 value to FP64 with integer
// operations (rebias the exponent by 1023 - 127 and shift the significand),
// keeping the per-crossing path off GB300's low-rate FP64 pipe.  Zero,
// subnormal and non-finite inputs take the ordinary conversion.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = u & 0x7f800000u;
  if (e == 0u || e == 0x7f800000u) return (double)f;
  const unsigned hi = ((u & 0x7fffffffu) >> 3) + 0x38000000u;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(u << 29));
}

// f 2^e in FP64 for a positive FP32 f, with integer operations (the widening
// above with the exponent moved by e); zero for results below FP64's normal
// range and for zero or non-finite f.
__device__ __forceinline__ double widen_exp(float f, int e) {
  const unsigned u = __float_as_uint(f);
  const int be = (int)((u >> 23) & 0xffu);
  if (be == 0 || be == 0xff) return be == 0 && (u & 0x7fffffu) ? ldexp((double)f, e) : 0.0;
  const int de = be - 127 + 1023 + e;  // biased FP64 exponent of the result
  if (de <= 0) return 0.0;
  const unsigned hi = ((unsigned)de << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// A positive FP64 value v as m 2^e with m in [1/2, 1) cut to FP32 (integer
// operations); zero gives m = 0, e = 0.
__device__ __forceinline__ float split_exp(double v, int& e) {
  const long long b = __double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ff);
  if (be == 0 || v <= 0.0) {
    e = 0;
    return 0.0f;
  }
  e = be - 1022;  // v = (1.m / 2) 2^(be - 1022)
  return __uint_as_float((126u << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
}

// FP64 to FP32 by cutting the significand to 24 bits, with integer
// operations; zero and values outside the normal FP32 range take the
// ordinary conversion.
__device__ __forceinline__ float cut(double v) {
  const long long b = __double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ff);
  if (be < 1023 - 126 || be > 1023 + 127) return (float)v;
  const unsigned top = (unsigned)((unsigned long long)b >> 32);
  return __uint_as_float((top & 0x80000000u) | ((unsigned)(be - 896) << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
}

// v as the unevaluated FP32 pair hi + lo: hi = v cut to 24 bits, lo = the
// remainder (exact in FP64) cut likewise: |v - hi - lo| < 2^-46 |v|.
__device__ __forceinline__ void split_pair(double v, float& hi, float& lo) {
  hi = cut(v);
  lo = cut(v - widen(hi));
}

// Uniform (r + 1/2) 2^-32 rounded to FP32 (= the FP64 value rounded), from
// the exact 33-bit integer 2r + 1.
__device__ __forceinline__ float u01f(uint32_t r) { return __ull2float_rn(2ull * r + 1ull) * 0x1p-33f; }

// 2u - 1 rounded to FP32, exactly: (2r + 1 - 2^32) 2^-32.
__device__ __forceinline__ float u01f_signed(uint32_t r) {
  return __ll2float_rn((long long)(2ull * r + 1ull) - (1ll << 32)) * 0x1p-32f;
}

// L2 residency: the density is read at every crossing and should stay in L2;
// absorption tallies are written once per forced-path crossing and should be
// the first lines evicted.
__device__ __forceinline__ float load_density(const float* p) {
  float v;
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
      "ld.global.nc.L2::cache_hint.f32 %0, [%1], pol;\n\t}"
      : "=f"(v)
      : "l"(p));
  return v;
}

__device__ __forceinline__ void add_absorption(double* p, double v) {
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
      "red.global.add.L2::cache_hint.f64 [%0], %1, pol;\n\t}" ::"l"(p),
      "d"(v)
      : "memory");
}

// 1 - exp(-x) for x >= 0 with a relative error below 5e-7: the alternating
// series through x^8 for x < 1/4 (truncation below 1e-10), 1 - exp(-x) above.
__device__ __forceinline__ float one_minus_exp_neg(float x) {
  if (x < 0.25f) {
    float p = fmaf(x, -1.0f / 40320.0f, 1.0f / 5040.0f);
    p = fmaf(x, p, -1.0f / 720.0f);
    p = fmaf(x, p, 1.0f / 120.0f);
    p = fmaf(x, p, -1.0f / 24.0f);
    p = fmaf(x, p, 1.0f / 6.0f);
    p = fmaf(x, p, -0.5f);
    p = fmaf(x, p, 1.0f);
    return x * p;
  }
  return 1.0f - expf(-x);
}

// Exit face of a cell: the first axis with the smallest exit parameter.
__device__ __forceinline__ float first_min(float tx, float ty, float tz, int& axis) {
  const bool by = ty < tx;
  const float txy = by ? ty : tx;
  const bool bz = tz < txy;
  axis = bz ? 2 : (by ? 1 : 0);
  return bz ? tz : txy;
}

__device__ __forceinline__ float pick(int a, float3 v) { return a == 2 ? v.z : (a == 1 ? v.y : v.x); }

// Storage stride of axis a: the launch's (FwdParams), row-major for any
// other geometry (one model of a batch).
template <class Geo>
__device__ __forceinline__ int stride_of(const Geo& P, int a) {
  return a == 0 ? 1 : (a == 1 ? P.nx : P.nx * P.ny);
}
__device__ __forceinline__ int stride_of(const FwdParams& P, int a) { return P.stride[a]; }

// ---------------------------------------------------------------- cartesian grid
struct CartGrid {
  static constexpr bool kColumns = true;  // peel-offs along grid axes may use column sums
  static constexpr bool kIndexCells = true;  // cells indexed by (ix, iy, iz) between planes
  static constexpr bool kSortedPass = true;  // walked peel-offs may go to the sorted pass
  struct Cell {
    int ix, iy, iz;
  };
  // current cell, entry parameter t of its segment, next-plane parameters
  struct Walk {
    int ix, iy, iz, cell;
    float t, tx, ty, tz;
  };
  struct Scratch {};

  // Geo: the grid geometry, nx, ny, nz, lo[3], hi[3], d[3], inv_d[3] (the
  // launch parameters, or one model of a batch).
  template <class Geo>
  __device__ static __forceinline__ float plane_t(const Geo& P, int a, int i, float xa, float ida) {
    return (fmaf((float)i, P.d[a], P.lo[a]) - xa) * ida;
  }

  // Start a walk from x along d (inverse id; id_a = 0 marks d_a = 0).  With a
  // known cell x lies in it; otherwise x is located or the entry point found.
  // False if the ray misses the grid.
  template <class Geo>
  __device__ static __forceinline__ bool init(const Geo& P, float3 x, float3 d, float3 id, bool known, const Cell& c,
                                              Walk& w, Scratch&) {
    w.t = 0.0f;
    if (known) {
      w.ix = c.ix; w.iy = c.iy; w.iz = c.iz;
    } else {
      int entry = -1;
      float3 p = x;
      if (!inside_box(P, x)) {
        const float3 ik = make_float3(id.x != 0.0f ? id.x : RT_INF, id.y != 0.0f ? id.y : RT_INF,
                                      id.z != 0.0f ? id.z : RT_INF);
        if (!ray_box_entry(P, x, d, ik, w.t, entry)) return false;
        p = make_float3(fmaf(w.t, d.x, x.x), fmaf(w.t, d.y, x.y), fmaf(w.t, d.z, x.z));
      }
      w.ix = min(max(__float2int_rd((p.x - P.lo[0]) * P.inv_d[0]), 0), P.nx - 1);
      w.iy = min(max(__float2int_rd((p.y - P.lo[1]) * P.inv_d[1]), 0), P.ny - 1);
      w.iz = min(max(__float2int_rd((p.z - P.lo[2]) * P.inv_d[2]), 0), P.nz - 1);
      if (entry == 0) w.ix = d.x > 0.0f ? 0 : P.nx - 1;
      if (entry == 1) w.iy = d.y > 0.0f ? 0 : P.ny - 1;
      if (entry == 2) w.iz = d.z > 0.0f ? 0 : P.nz - 1;
    }
    w.tx = id.x != 0.0f ? plane_t(P, 0, w.ix + (id.x > 0.0f), x.x, id.x) : RT_INF;
    w.ty = id.y != 0.0f ? plane_t(P, 1, w.iy + (id.y > 0.0f), x.y, id.y) : RT_INF;
    w.tz = id.z != 0.0f ? plane_t(P, 2, w.iz + (id.z > 0.0f), x.z, id.z) : RT_INF;
    w.cell = w.ix * stride_of(P, 0) + w.iy * stride_of(P, 1) + w.iz * stride_of(P, 2);
    return true;
  }

  __device__ static __forceinline__ float exit(const Walk& w, float3, float3, int& axis) {
    return first_min(w.tx, w.ty, w.tz, axis);
  }

  // Move through face `axis` (w.t already at the exit); false when the ray
  // leaves the grid, in which case the walk still describes the last cell.
  // Selects rather than branches: the warp issues the advance once.
  template <class Geo>
  __device__ static __forceinline__ bool advance(const Geo& P, float3 x, float3, float3 id, int axis, Walk& w,
                                                 Scratch&) {
    const bool bz = axis == 2, by = axis == 1;
    const float ida = bz ? id.z : (by ? id.y : id.x);
    const int step = ida > 0.0f ? 1 : -1;
    const int ia = (bz ? w.iz : (by ? w.iy : w.ix)) + step;
    const int na = bz ? P.nz : (by ? P.ny : P.nx);
    if ((unsigned)ia >= (unsigned)na) return false;
    w.cell += step * (bz ? stride_of(P, 2) : (by ? stride_of(P, 1) : stride_of(P, 0)));
    const float xa = bz ? x.z : (by ? x.y : x.x);
    const float da = bz ? P.d[2] : (by ? P.d[1] : P.d[0]);
    const float loa = bz ? P.lo[2] : (by ? P.lo[1] : P.lo[0]);
    const float t_new = (fmaf((float)(ia + (step > 0)), da, loa) - xa) * ida;
    w.ix = (axis == 0) ? ia : w.ix;
    w.iy = by ? ia : w.iy;
    w.iz = bz ? ia : w.iz;
    w.tx = (axis == 0) ? t_new : w.tx;
    w.ty = by ? t_new : w.ty;
    w.tz = bz ? t_new : w.tz;
    return true;
  }

  __device__ static __forceinline__ int cell(const Walk& w) { return w.cell; }

  // The row-major cell id (records, traces, the tape).
  template <class Geo>
  __device__ static __forceinline__ int id(const Geo& P, const Walk& w) { return w.ix + P.nx * (w.iy + P.ny * w.iz); }

  // Plane i of axis a.
  __device__ static __forceinline__ float plane(const FwdParams& P, int a, int i) {
    return fmaf((float)i, P.d[a], P.lo[a]);
  }

  // The cell of a point inside the grid.
  __device__ static __forceinline__ void locate_cell(const FwdParams& P, float3 x, Cell& c) {
    c.ix = min(max(__float2int_rd((x.x - P.lo[0]) * P.inv_d[0]), 0), P.nx - 1);
    c.iy = min(max(__float2int_rd((x.y - P.lo[1]) * P.inv_d[1]), 0), P.ny - 1);
    c.iz = min(max(__float2int_rd((x.z - P.lo[2]) * P.inv_d[2]), 0), P.nz - 1);
  }

  __device__ static __forceinline__ Cell carried(const Walk& w) { return Cell{w.ix, w.iy, w.iz}; }

  // Keep x inside cell c.
  template <class Geo>
  __device__ static __forceinline__ void clamp(const Geo& P, const Cell& c, float3& x) {
    x.x = fminf(fmaxf(x.x, fmaf((float)c.ix, P.d[0], P.lo[0])), fmaf((float)(c.ix + 1), P.d[0], P.lo[0]));
    x.y = fminf(fmaxf(x.y, fmaf((float)c.iy, P.d[1], P.lo[1])), fmaf((float)(c.iy + 1), P.d[1], P.lo[1]));
    x.z = fminf(fmaxf(x.z, fmaf((float)c.iz, P.d[2], P.lo[2])), fmaf((float)(c.iz + 1), P.d[2], P.lo[2]));
  }
};

// ---------------------------------------------------------------- rectilinear grid
// Cuboidal cells between increasing edges given per axis (Table 1(d): the
// PowCub grid places them by a power law; Sect. 2.2: logarithmic and
// power-law grids put smaller cells in the central areas).  The walk is the
// cartesian one with the plane positions read from the edge arrays (FP32
// copies of the FP64 edges); a position is located by binary search.
struct RectGrid {
  static constexpr bool kColumns = true;
  static constexpr bool kIndexCells = true;
  static constexpr bool kSortedPass = false;
  using Cell = CartGrid::Cell;
  using Walk = CartGrid::Walk;
  struct Scratch {};

  __device__ static __forceinline__ float edge(const FwdParams& P, int a, int i) { return __ldg(&P.edge[a][i]); }

  // The cell along axis a that holds coordinate xa: the last i in [0, n) with
  // edge[i] <= xa (clamped into the grid).
  __device__ static __forceinline__ int locate(const FwdParams& P, int a, float xa, int n) {
    const float* e = P.edge[a];
    int lo = 0, hi = n - 1;  // answer in [lo, hi]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(&e[mid]) <= xa) lo = mid; else hi = mid - 1;
    }
    return lo;
  }

  __device__ static __forceinline__ bool init(const FwdParams& P, float3 x, float3 d, float3 id, bool known,
                                              const Cell& c, Walk& w, Scratch&) {
    w.t = 0.0f;
    if (known) {
      w.ix = c.ix; w.iy = c.iy; w.iz = c.iz;
    } else {
      int entry = -1;
      float3 p = x;
      if (!inside_box(P, x)) {
        const float3 ik = make_float3(id.x != 0.0f ? id.x : RT_INF, id.y != 0.0f ? id.y : RT_INF,
                                      id.z != 0.0f ? id.z : RT_INF);
        if (!ray_box_entry(P, x, d, ik, w.t, entry)) return false;
        p = make_float3(fmaf(w.t, d.x, x.x), fmaf(w.t, d.y, x.y), fmaf(w.t, d.z, x.z));
      }
      w.ix = locate(P, 0, p.x, P.nx);
      w.iy = locate(P, 1, p.y, P.ny);
      w.iz = locate(P, 2, p.z, P.nz);
      if (entry == 0) w.ix = d.x > 0.0f ? 0 : P.nx - 1;
      if (entry == 1) w.iy = d.y > 0.0f ? 0 : P.ny - 1;
      if (entry == 2) w.iz = d.z > 0.0f ? 0 : P.nz - 1;
    }
    w.tx = id.x != 0.0f ? (edge(P, 0, w.ix + (id.x > 0.0f)) - x.x) * id.x : RT_INF;
    w.ty = id.y != 0.0f ? (edge(P, 1, w.iy + (id.y > 0.0f)) - x.y) * id.y : RT_INF;
    w.tz = id.z != 0.0f ? (edge(P, 2, w.iz + (id.z > 0.0f)) - x.z) * id.z : RT_INF;
    w.cell = w.ix * P.stride[0] + w.iy * P.stride[1] + w.iz * P.stride[2];
    return true;
  }

  __device__ static __forceinline__ float exit(const Walk& w, float3, float3, int& axis) {
    return first_min(w.tx, w.ty, w.tz, axis);
  }

  __device__ static __forceinline__ bool advance(const FwdParams& P, float3 x, float3, float3 id, int axis, Walk& w,
                                                 Scratch&) {
    const bool bz = axis == 2, by = axis == 1;
    const float ida = bz ? id.z : (by ? id.y : id.x);
    const int step = ida > 0.0f ? 1 : -1;
    const int ia = (bz ? w.iz : (by ? w.iy : w.ix)) + step;
    const int na = bz ? P.nz : (by ? P.ny : P.nx);
    if ((unsigned)ia >= (unsigned)na) return false;
    w.cell += step * (bz ? P.stride[2] : (by ? P.stride[1] : P.stride[0]));
    const float xa = bz ? x.z : (by ? x.y : x.x);
    const float t_new = (edge(P, axis, ia + (step > 0)) - xa) * ida;
    w.ix = (axis == 0) ? ia : w.ix;
    w.iy = by ? ia : w.iy;
    w.iz = bz ? ia : w.iz;
    w.tx = (axis == 0) ? t_new : w.tx;
    w.ty = by ? t_new : w.ty;
    w.tz = bz ? t_new : w.tz;
    return true;
  }

  __device__ static __forceinline__ int cell(const Walk& w) { return w.cell; }

  __device__ static __forceinline__ int id(const FwdParams& P, const Walk& w) {
    return w.ix + P.nx * (w.iy + P.ny * w.iz);
  }

  __device__ static __forceinline__ float plane(const FwdParams& P, int a, int i) { return edge(P, a, i); }

  __device__ static __forceinline__ void locate_cell(const FwdParams& P, float3 x, Cell& c) {
    c.ix = locate(P, 0, x.x, P.nx);
    c.iy = locate(P, 1, x.y, P.ny);
    c.iz = locate(P, 2, x.z, P.nz);
  }

  __device__ static __forceinline__ Cell carried(const Walk& w) { return Cell{w.ix, w.iy, w.iz}; }

  __device__ static __forceinline__ void clamp(const FwdParams& P, const Cell& c, float3& x) {
    x.x = fminf(fmaxf(x.x, edge(P, 0, c.ix)), edge(P, 0, c.ix + 1));
    x.y = fminf(fmaxf(x.y, edge(P, 1, c.iy)), edge(P, 1, c.iy + 1));
    x.z = fminf(fmaxf(x.z, edge(P, 2, c.iz)), edge(P, 2, c.iz + 1));
  }
};

// ---------------------------------------------------------------- octree grid
// Nodes are split at box midpoints (Sect. 2.4); a point on a splitting plane
// belongs to the child the ray enters (upper if d_a >= 0, lower if d_a < 0).
constexpr int kOctStack = kMaxOctreeDepth + 1;  // path stack: depths 0..21 (3 path bits per level)
constexpr int kChildCache = 1024;                // first child[] entries kept in shared memory

__shared__ int S_CHILD[kChildCache];
// the octree kernel's per-lane ancestor stacks, P.oct_levels entries each
// (dynamic shared memory sized by the tree's depth)
extern __shared__ int S_OCT_STACK[];

struct OctGrid {
  static constexpr bool kColumns = false;
  static constexpr bool kIndexCells = false;
  static constexpr bool kSortedPass = false;
  struct Cell {
    int leaf;
    float lo[3], hi[3];
  };
  // current leaf and its box, its depth, the octants of its path (3 bits per
  // level from the root), entry parameter t; node indices of the path in the
  // lane's shared-memory stack
  struct Walk {
    int leaf, depth;
    float t;
    float lo[3], hi[3];
    unsigned long long path;
  };
  struct Scratch {
    int* stack;
  };

  __device__ static __forceinline__ int child(const FwdParams& P, int node) {
    return node < kChildCache ? S_CHILD[node] : __ldg(&P.child[node]);
  }

  __device__ static __forceinline__ int octant(float3 p, float3 d, float lo[3], float hi[3], bool descend) {
    int oct = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float mid = 0.5f * (lo[a] + hi[a]);
      const float pa = a == 0 ? p.x : (a == 1 ? p.y : p.z);
      const float da = a == 0 ? d.x : (a == 1 ? d.y : d.z);
      const bool upper = da < 0.0f ? (pa > mid) : (pa >= mid);
      if (upper) oct |= 1 << a;
      if (descend) {
        if (upper) lo[a] = mid; else hi[a] = mid;
      }
    }
    return oct;
  }

  // Descend from node stack[depth] (box w.lo/hi) to the leaf containing p.
  __device__ static __forceinline__ bool descend(const FwdParams& P, float3 p, float3 d, Walk& w, Scratch& sc) {
    int node = sc.stack[w.depth];
    while (true) {
      const int c = child(P, node);
      if (c < 0) {
        w.leaf = -c - 1;
        return true;
      }
      if (w.depth + 1 >= P.oct_levels) {
        atomicOr(P.flags, kFlagOctreeDepth);
        w.leaf = 0;
        return false;
      }
      const int oct = octant(p, d, w.lo, w.hi, true);
      w.path |= (unsigned long long)oct << (3 * w.depth);
      node = c + oct;
      w.depth += 1;
      sc.stack[w.depth] = node;
    }
  }

  __device__ static __forceinline__ bool locate_from_root(const FwdParams& P, float3 p, float3 d, Walk& w,
                                                          Scratch& sc) {
#pragma unroll
    for (int a = 0; a < 3; ++a) { w.lo[a] = P.lo[a]; w.hi[a] = P.hi[a]; }
    w.depth = 0;
    w.path = 0ull;
    sc.stack[0] = 0;
    return descend(P, p, d, w, sc);
  }

  __device__ static __forceinline__ bool init(const FwdParams& P, float3 x, float3 d, float3 id, bool known,
                                              const Cell& c, Walk& w, Scratch& sc) {
    w.t = 0.0f;
    if (known) {
      // rebuild the path of the known leaf by descending to its box centre,
      // which lies strictly inside every ancestor's chosen half
      const float3 ctr = make_float3(0.5f * (c.lo[0] + c.hi[0]), 0.5f * (c.lo[1] + c.hi[1]), 0.5f * (c.lo[2] + c.hi[2]));
      if (!locate_from_root(P, ctr, d, w, sc)) return false;
      if (w.leaf != c.leaf) atomicOr(P.flags, kFlagCellRange);
      return true;
    }
    int entry = -1;
    float3 p = x;
    if (!inside_box(P, x)) {
      const float3 ik = make_float3(id.x != 0.0f ? id.x : RT_INF, id.y != 0.0f ? id.y : RT_INF,
                                    id.z != 0.0f ? id.z : RT_INF);
      if (!ray_box_entry(P, x, d, ik, w.t, entry)) return false;
      p = make_float3(fmaf(w.t, d.x, x.x), fmaf(w.t, d.y, x.y), fmaf(w.t, d.z, x.z));
      if (entry == 0) p.x = d.x > 0.0f ? P.lo[0] : P.hi[0];
      if (entry == 1) p.y = d.y > 0.0f ? P.lo[1] : P.hi[1];
      if (entry == 2) p.z = d.z > 0.0f ? P.lo[2] : P.hi[2];
    }
    return locate_from_root(P, p, d, w, sc);
  }

  __device__ static __forceinline__ float exit(const Walk& w, float3 x, float3 id, int& axis) {
    const float tx = id.x != 0.0f ? ((id.x > 0.0f ? w.hi[0] : w.lo[0]) - x.x) * id.x : RT_INF;
    const float ty = id.y != 0.0f ? ((id.y > 0.0f ? w.hi[1] : w.lo[1]) - x.y) * id.y : RT_INF;
    const float tz = id.z != 0.0f ? ((id.z > 0.0f ? w.hi[2] : w.lo[2]) - x.z) * id.z : RT_INF;
    return first_min(tx, ty, tz, axis);
  }

  // Move through face `axis` to the neighbouring leaf at the exit point.  The
  // exit point's other coordinates stay inside the current leaf, so the walk
  // never steps back across a face.  The new leaf is found by replaying the
  // current leaf's path from the root while the exit point stays on it (no
  // loads), then descending with loads below the level where it leaves it.
  __device__ static __forceinline__ bool advance(const FwdParams& P, float3 x, float3 d, float3, int axis, Walk& w,
                                                 Scratch& sc) {
    const float da = pick(axis, d);
    const float plane = da > 0.0f ? (axis == 0 ? w.hi[0] : (axis == 1 ? w.hi[1] : w.hi[2]))
                                  : (axis == 0 ? w.lo[0] : (axis == 1 ? w.lo[1] : w.lo[2]));
    const float dom_lo = axis == 0 ? P.lo[0] : (axis == 1 ? P.lo[1] : P.lo[2]);
    const float dom_hi = axis == 0 ? P.hi[0] : (axis == 1 ? P.hi[1] : P.hi[2]);
    if ((da > 0.0f && plane >= dom_hi) || (da < 0.0f && plane <= dom_lo)) return false;
    float3 p = make_float3(fminf(fmaxf(fmaf(w.t, d.x, x.x), w.lo[0]), w.hi[0]),
                           fminf(fmaxf(fmaf(w.t, d.y, x.y), w.lo[1]), w.hi[1]),
                           fminf(fmaxf(fmaf(w.t, d.z, x.z), w.lo[2]), w.hi[2]));
    if (axis == 0) p.x = plane; else if (axis == 1) p.y = plane; else p.z = plane;
    const int old_depth = w.depth;
    const unsigned long long old_path = w.path;
    float lo[3] = {P.lo[0], P.lo[1], P.lo[2]}, hi[3] = {P.hi[0], P.hi[1], P.hi[2]};
    int depth = 0;
    // When the exit point lies strictly inside the leaf's box in the two other
    // axes, the old path and the new one part at the level where the face
    // plane splits an ancestor: with i the leaf's integer coordinate along
    // `axis` at its depth D, level D - 1 - (trailing ones of i) going up,
    // D - 1 - (trailing zeros of i) going down.  With exact boxes the new path is
    // then followed from there by its bits; otherwise the ancestor's box is
    // rebuilt by halving along the old path (the same arithmetic as the
    // descent) and the exit point descends from it.  When a coordinate lies
    // on a face of the leaf (the tie rule may part the paths earlier) the
    // path is replayed from the root.
    const bool in_x = axis == 0 || (p.x > w.lo[0] && p.x < w.hi[0]);
    const bool in_y = axis == 1 || (p.y > w.lo[1] && p.y < w.hi[1]);
    const bool in_z = axis == 2 || (p.z > w.lo[2] && p.z < w.hi[2]);
    const bool inside = in_x && in_y && in_z;
    if (inside) {
      // the path's bits on `axis`, level l at bit l (Morton compaction of
      // every third bit), then moved so that the leaf's level is bit 31
      unsigned long long m = (old_path >> axis) & 0x1249249249249249ull;
      m = (m ^ (m >> 2)) & 0x10c30c30c30c30c3ull;
      m = (m ^ (m >> 4)) & 0x100f00f00f00f00full;
      m = (m ^ (m >> 8)) & 0x1f0000ff0000ffull;
      m = (m ^ (m >> 16)) & 0x1f00000000ffffull;
      m = (m ^ (m >> 32)) & 0x1fffffull;
      const unsigned top = (unsigned)m << (32 - old_depth);
      // trailing ones (up) / zeros (down) of the leaf's coordinate
      const int tb = da > 0.0f ? __clz(~top) : __clz(top);
      const int part = old_depth - 1 - tb;
      if (P.oct_exact) {
        // exact boxes: below the parting level the new path is the old one
        // with the bit of `axis` flipped (in the other axes the exit point
        // lies strictly inside the leaf, so it keeps the old octants), and it
        // is followed without position tests down to the old depth or to a
        // leaf above it.  The box: the old leaf's, moved across the face, then
        // doubled on the side away from each octant up to the level reached.
        const int flip = 1 << axis;
        int node = sc.stack[part];
        int c = child(P, node);
        unsigned long long path = part > 0 ? (old_path & ((1ull << (3 * part)) - 1ull)) : 0ull;
        depth = part;
        while (c >= 0 && depth < old_depth) {
          const int oct = (int)((old_path >> (3 * depth)) & 7ull) ^ flip;
          path |= (unsigned long long)oct << (3 * depth);
          node = c + oct;
          depth += 1;
          sc.stack[depth] = node;
          c = child(P, node);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          lo[a] = w.lo[a];
          hi[a] = w.hi[a];
          if (a == axis) {
            const float size = hi[a] - lo[a];
            if (da > 0.0f) { lo[a] = hi[a]; hi[a] += size; } else { hi[a] = lo[a]; lo[a] -= size; }
          }
        }
        for (int l = old_depth - 1; l >= depth; --l) {
          const int oct = (int)((old_path >> (3 * l)) & 7ull) ^ flip;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float size = hi[a] - lo[a];
            if ((oct >> a) & 1) lo[a] -= size; else hi[a] += size;
          }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) { w.lo[a] = lo[a]; w.hi[a] = hi[a]; }
        w.depth = depth;
        w.path = path;
        if (c < 0) {
          w.leaf = -c - 1;
          return true;
        }
        // a finer neighbour: on by the exit point below the old depth
        return descend(P, p, d, w, sc);
      } else {
        for (; depth < part; ++depth) {
          const int oct = (int)((old_path >> (3 * depth)) & 7ull);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float mid = 0.5f * (lo[a] + hi[a]);
            if ((oct >> a) & 1) lo[a] = mid; else hi[a] = mid;
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) { w.lo[a] = lo[a]; w.hi[a] = hi[a]; }
      w.depth = depth;
      w.path = depth > 0 ? (old_path & ((1ull << (3 * depth)) - 1ull)) : 0ull;
      return descend(P, p, d, w, sc);
    }
    // replay from the root along the old path
    while (depth < old_depth) {
      float l2[3] = {lo[0], lo[1], lo[2]}, h2[3] = {hi[0], hi[1], hi[2]};
      const int oct = octant(p, d, l2, h2, true);
      if (oct != (int)((old_path >> (3 * depth)) & 7ull)) break;
#pragma unroll
      for (int a = 0; a < 3; ++a) { lo[a] = l2[a]; hi[a] = h2[a]; }
      ++depth;
    }
    if (depth == old_depth) {  // the exit point cannot lie in the leaf it leaves
      atomicOr(P.flags, kFlagWalkSteps);
      return false;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) { w.lo[a] = lo[a]; w.hi[a] = hi[a]; }
    w.depth = depth;
    w.path = depth > 0 ? (old_path & ((1ull << (3 * depth)) - 1ull)) : 0ull;
    return descend(P, p, d, w, sc);
  }

  __device__ static __forceinline__ int cell(const Walk& w) { return w.leaf; }

  __device__ static __forceinline__ int id(const FwdParams&, const Walk& w) { return w.leaf; }

  __device__ static __forceinline__ Cell carried(const Walk& w) {
    Cell c;
    c.leaf = w.leaf;
#pragma unroll
    for (int a = 0; a < 3; ++a) { c.lo[a] = w.lo[a]; c.hi[a] = w.hi[a]; }
    return c;
  }

  __device__ static __forceinline__ void clamp(const FwdParams&, const Cell& c, float3& x) {
    x.x = fminf(fmaxf(x.x, c.lo[0]), c.hi[0]);
    x.y = fminf(fmaxf(x.y, c.lo[1]), c.hi[1]);
    x.z = fminf(fmaxf(x.z, c.lo[2]), c.hi[2]);
  }
};

// ---------------------------------------------------------------- k-d tree grid
// A node halves its box at the midpoint of one axis (Table 1(d): BinTree).
// Device node word: (first child << 2) | split axis for an inner node (the
// lower child first, the upper one next), -(leaf + 1) for a leaf.  A point
// on a splitting plane belongs to the child the ray enters, as in octrees.
// The walk finds the next leaf at the exit point of the current one by a
// descent from the leaf's rope for the face it leaves through (the node
// across that face that covers it: the sibling of the ancestor whose split
// made the face), or from the root when the exit point lies on an edge of
// the leaf (the tie rule may then part the paths higher up).  Both give the
// leaf the root descent gives.  The first kChildCache node words sit in
// shared memory.
constexpr int kMaxBinDepth = 96;

struct BinGrid {
  static constexpr bool kColumns = false;
  static constexpr bool kIndexCells = false;
  static constexpr bool kSortedPass = false;
  using Cell = OctGrid::Cell;  // the leaf and its box
  struct Walk {
    int leaf;
    float t;
    float lo[3], hi[3];
  };
  struct Scratch {};

  __device__ static __forceinline__ int word(const FwdParams& P, int node) {
    return node < kChildCache ? S_CHILD[node] : __ldg(&P.child[node]);
  }

  // Descend from the root to the leaf holding p (direction d breaks ties).
  __device__ static __forceinline__ bool locate(const FwdParams& P, float3 p, float3 d, Walk& w) {
    return descend(P, 0, P.lo[0], P.lo[1], P.lo[2], P.hi[0], P.hi[1], P.hi[2], p, d, w);
  }

  // Descend from `node` (box lo/hi) to the leaf holding p.
  __device__ static __forceinline__ bool descend(const FwdParams& P, int node, float lx, float ly, float lz, float hx,
                                                 float hy, float hz, float3 p, float3 d, Walk& w) {
    for (int depth = 0; depth <= kMaxBinDepth; ++depth) {
      const int v = word(P, node);
      if (v < 0) {
        w.leaf = -v - 1;
        w.lo[0] = lx; w.lo[1] = ly; w.lo[2] = lz;
        w.hi[0] = hx; w.hi[1] = hy; w.hi[2] = hz;
        return true;
      }
      const int a = v & 3;
      const float la = a == 0 ? lx : (a == 1 ? ly : lz), ha = a == 0 ? hx : (a == 1 ? hy : hz);
      const float pa = a == 0 ? p.x : (a == 1 ? p.y : p.z), da = a == 0 ? d.x : (a == 1 ? d.y : d.z);
      const float mid = 0.5f * (la + ha);
      const bool upper = da < 0.0f ? (pa > mid) : (pa >= mid);
      lx = (a == 0 && upper) ? mid : lx;
      ly = (a == 1 && upper) ? mid : ly;
      lz = (a == 2 && upper) ? mid : lz;
      hx = (a == 0 && !upper) ? mid : hx;
      hy = (a == 1 && !upper) ? mid : hy;
      hz = (a == 2 && !upper) ? mid : hz;
      node = (v >> 2) + (upper ? 1 : 0);
    }
    atomicOr(P.flags, kFlagOctreeDepth);
    w.leaf = 0;
    return false;
  }

  __device__ static __forceinline__ bool init(const FwdParams& P, float3 x, float3 d, float3 id, bool known,
                                              const Cell& c, Walk& w, Scratch&) {
    w.t = 0.0f;
    if (known) {
      // the known leaf: descend to its box centre, strictly inside every
      // ancestor's chosen half
      const float3 ctr = make_float3(0.5f * (c.lo[0] + c.hi[0]), 0.5f * (c.lo[1] + c.hi[1]), 0.5f * (c.lo[2] + c.hi[2]));
      if (!locate(P, ctr, d, w)) return false;
      if (w.leaf != c.leaf) atomicOr(P.flags, kFlagCellRange);
      return true;
    }
    int entry = -1;
    float3 p = x;
    if (!inside_box(P, x)) {
      const float3 ik = make_float3(id.x != 0.0f ? id.x : RT_INF, id.y != 0.0f ? id.y : RT_INF,
                                    id.z != 0.0f ? id.z : RT_INF);
      if (!ray_box_entry(P, x, d, ik, w.t, entry)) return false;
      p = make_float3(fmaf(w.t, d.x, x.x), fmaf(w.t, d.y, x.y), fmaf(w.t, d.z, x.z));
      if (entry == 0) p.x = d.x > 0.0f ? P.lo[0] : P.hi[0];
      if (entry == 1) p.y = d.y > 0.0f ? P.lo[1] : P.hi[1];
      if (entry == 2) p.z = d.z > 0.0f ? P.lo[2] : P.hi[2];
    }
    return locate(P, p, d, w);
  }

  __device__ static __forceinline__ float exit(const Walk& w, float3 x, float3 id, int& axis) {
    const float tx = id.x != 0.0f ? ((id.x > 0.0f ? w.hi[0] : w.lo[0]) - x.x) * id.x : RT_INF;
    const float ty = id.y != 0.0f ? ((id.y > 0.0f ? w.hi[1] : w.lo[1]) - x.y) * id.y : RT_INF;
    const float tz = id.z != 0.0f ? ((id.z > 0.0f ? w.hi[2] : w.lo[2]) - x.z) * id.z : RT_INF;
    return first_min(tx, ty, tz, axis);
  }

  // Into the neighbouring leaf through face `axis`: the exit point with the
  // other coordinates kept inside the current leaf (the walk never steps
  // back across a face), located from the root.
  __device__ static __forceinline__ bool advance(const FwdParams& P, float3 x, float3 d, float3, int axis, Walk& w,
                                                 Scratch&) {
    const float da = pick(axis, d);
    const float plane = da > 0.0f ? (axis == 0 ? w.hi[0] : (axis == 1 ? w.hi[1] : w.hi[2]))
                                  : (axis == 0 ? w.lo[0] : (axis == 1 ? w.lo[1] : w.lo[2]));
    const float dom_lo = axis == 0 ? P.lo[0] : (axis == 1 ? P.lo[1] : P.lo[2]);
    const float dom_hi = axis == 0 ? P.hi[0] : (axis == 1 ? P.hi[1] : P.hi[2]);
    if ((da > 0.0f && plane >= dom_hi) || (da < 0.0f && plane <= dom_lo)) return false;
    float3 p = make_float3(fminf(fmaxf(fmaf(w.t, d.x, x.x), w.lo[0]), w.hi[0]),
                           fminf(fmaxf(fmaf(w.t, d.y, x.y), w.lo[1]), w.hi[1]),
                           fminf(fmaxf(fmaf(w.t, d.z, x.z), w.lo[2]), w.hi[2]));
    if (axis == 0) p.x = plane; else if (axis == 1) p.y = plane; else p.z = plane;
    const int old = w.leaf;
    const float t = w.t;
    const bool inside = (axis == 0 || (p.x > w.lo[0] && p.x < w.hi[0])) &&
                        (axis == 1 || (p.y > w.lo[1] && p.y < w.hi[1])) &&
                        (axis == 2 || (p.z > w.lo[2] && p.z < w.hi[2]));
    // the start of the descent (one loop for both starts: lanes of a warp
    // that start differently still descend together)
    int node = 0;
    float4 lo = make_float4(P.lo[0], P.lo[1], P.lo[2], 0.0f), hi = make_float4(P.hi[0], P.hi[1], P.hi[2], 0.0f);
    if (inside) {
      node = __ldg(&P.rope[(size_t)old * 6 + 2 * axis + (da > 0.0f ? 1 : 0)]);
      if (node < 0) return false;
      lo = __ldg(&P.node_box[2 * (size_t)node]);
      hi = __ldg(&P.node_box[2 * (size_t)node + 1]);
    }
    if (!descend(P, node, lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, p, d, w)) return false;
    w.t = t;
    if (w.leaf == old) {  // the exit point cannot lie in the leaf it leaves
      atomicOr(P.flags, kFlagWalkSteps);
      return false;
    }
    return true;
  }

  __device__ static __forceinline__ int cell(const Walk& w) { return w.leaf; }
  __device__ static __forceinline__ int id(const FwdParams&, const Walk& w) { return w.leaf; }

  __device__ static __forceinline__ Cell carried(const Walk& w) {
    Cell c;
    c.leaf = w.leaf;
#pragma unroll
    for (int a = 0; a < 3; ++a) { c.lo[a] = w.lo[a]; c.hi[a] = w.hi[a]; }
    return c;
  }

  __device__ static __forceinline__ void clamp(const FwdParams&, const Cell& c, float3& x) {
    x.x = fminf(fmaxf(x.x, c.lo[0]), c.hi[0]);
    x.y = fminf(fmaxf(x.y, c.lo[1]), c.hi[1]);
    x.z = fminf(fmaxf(x.z, c.lo[2]), c.hi[2]);
  }
};

// ---------------------------------------------------------------- Voronoi grid
// Cell c holds the points nearer to site c than to any other site (Table
// 1(d): VoronoiDustGrid; Sect. 2.4).  Its boundary with neighbour j is their
// bisecting plane, kept per face as the unit normal n towards s_j and the
// plane's distance h from s_c.  On entering a cell the walk finds the first
// plane ahead, t_f = (h - (x - s_c) . n) / (d . n) over the faces with
// d . n > 0, or the domain boundary if that comes first (the first minimal
// face wins ties, as in the oracle); a straight line meets each convex cell
// once, so a walk visiting more cells than the grid holds (P.max_walk) is
// stopped and flagged.  A point is located by a greedy descent from the site
// nearest to its bucket's centre: move to the nearest neighbour nearer to
// the point until none is; on a neighbour graph that holds every face inside
// the domain this ends at the nearest site.
struct VorGrid {
  static constexpr bool kColumns = false;
  static constexpr bool kIndexCells = false;
  static constexpr bool kSortedPass = false;
  using Cell = OctGrid::Cell;  // the cell id in .leaf (the box is not used)
  struct Walk {
    int leaf;   // current cell
    int next;   // the cell beyond the exit face, -1 for the domain boundary
    float t;    // entry parameter of the current segment
    float te;   // exit parameter
    float t_box;  // where the ray leaves the domain
    int steps;  // cells entered after the first
  };
  struct Scratch {};

  __device__ static __forceinline__ float dist2(float3 p, float4 s) {
    const float dx = p.x - s.x, dy = p.y - s.y, dz = p.z - s.z;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  }

  __device__ static __forceinline__ int locate(const FwdParams& P, float3 p) {
    const int bx = min(max(__float2int_rd((p.x - P.lo[0]) * P.vb_inv[0]), 0), P.vb_n[0] - 1);
    const int by = min(max(__float2int_rd((p.y - P.lo[1]) * P.vb_inv[1]), 0), P.vb_n[1] - 1);
    const int bz = min(max(__float2int_rd((p.z - P.lo[2]) * P.vb_inv[2]), 0), P.vb_n[2] - 1);
    int c = __ldg(&P.bucket_seed[bx + P.vb_n[0] * (by + P.vb_n[1] * bz)]);
    for (int it = 0; it < P.max_walk; ++it) {
      float best = dist2(p, __ldg(&P.site[c]));
      int move = -1;
      const int f1 = __ldg(&P.face_off[c + 1]);
      // three neighbours at once, as in the face loop of the walk (past the
      // last face the cell itself, never nearer than itself)
      for (int f = __ldg(&P.face_off[c]); f < f1; f += 3) {
        int j[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) j[k] = f + k < f1 ? __ldg(&P.child[f + k]) : c;
        float4 sj[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) sj[k] = __ldg(&P.site[j[k]]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float dj = dist2(p, sj[k]);
          if (dj < best) { best = dj; move = j[k]; }
        }
      }
      if (move < 0) return c;
      c = move;
    }
    atomicOr(P.flags, kFlagWalkSteps);
    return c;
  }

  // The exit of the current cell along x + t d: parameter and next cell.
  __device__ static __forceinline__ void find_exit(const FwdParams& P, float3 x, float3 d, Walk& w) {
    const float4 s = __ldg(&P.site[w.leaf]);
    const float rx = x.x - s.x, ry = x.y - s.y, rz = x.z - s.z;
    float best = w.t_box;
    int face = -1;
    const int f1 = __ldg(&P.face_off[w.leaf + 1]);
    // three face planes loaded at once (a plane past the last face reads as
    // zero: d.n = 0, never an exit), tested in face order: three L2 loads in
    // flight per lane instead of one (190 -> 142 ms on the 1e5-site disk; four
    // spill at 64 registers)
    for (int f = __ldg(&P.face_off[w.leaf]); f < f1; f += 3) {
      float4 n[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) n[k] = f + k < f1 ? __ldg(&P.face[f + k]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float den = fmaf(d.x, n[k].x, fmaf(d.y, n[k].y, d.z * n[k].z));
        if (den > 0.0f) {
          const float tf = (n[k].w - fmaf(rx, n[k].x, fmaf(ry, n[k].y, rz * n[k].z))) / den;
          if (tf < best) { best = tf; face = f + k; }
        }
      }
    }
    w.te = best;
    w.next = face >= 0 ? __ldg(&P.child[face]) : -1;
  }

  __device__ static __forceinline__ bool init(const FwdParams& P, float3 x, float3 d, float3 id, bool known,
                                              const Cell& c, Walk& w, Scratch&) {
    w.t = 0.0f;
    w.steps = 0;
    const float tx = id.x != 0.0f ? ((id.x > 0.0f ? P.hi[0] : P.lo[0]) - x.x) * id.x : RT_INF;
    const float ty = id.y != 0.0f ? ((id.y > 0.0f ? P.hi[1] : P.lo[1]) - x.y) * id.y : RT_INF;
    const float tz = id.z != 0.0f ? ((id.z > 0.0f ? P.hi[2] : P.lo[2]) - x.z) * id.z : RT_INF;
    w.t_box = fminf(tx, fminf(ty, tz));
    if (known) {
      w.leaf = c.leaf;
    } else {
      int entry = -1;
      float3 p = x;
      if (!inside_box(P, x)) {
        const float3 ik = make_float3(id.x != 0.0f ? id.x : RT_INF, id.y != 0.0f ? id.y : RT_INF,
                                      id.z != 0.0f ? id.z : RT_INF);
        if (!ray_box_entry(P, x, d, ik, w.t, entry)) return false;
        p = make_float3(fmaf(w.t, d.x, x.x), fmaf(w.t, d.y, x.y), fmaf(w.t, d.z, x.z));
        if (entry == 0) p.x = d.x > 0.0f ? P.lo[0] : P.hi[0];
        if (entry == 1) p.y = d.y > 0.0f ? P.lo[1] : P.hi[1];
        if (entry == 2) p.z = d.z > 0.0f ? P.lo[2] : P.hi[2];
      }
      w.leaf = locate(P, p);
    }
    find_exit(P, x, d, w);
    return true;
  }

  __device__ static __forceinline__ float exit(const Walk& w, float3, float3, int& axis) {
    axis = 0;
    return w.te;
  }

  __device__ static __forceinline__ bool advance(const FwdParams& P, float3 x, float3 d, float3, int, Walk& w,
                                                 Scratch&) {
    if (w.next < 0) return false;
    if (++w.steps > P.max_walk) {
      atomicOr(P.flags, kFlagWalkSteps);
      return false;
    }
    w.leaf = w.next;
    find_exit(P, x, d, w);
    return true;
  }

  __device__ static __forceinline__ int cell(const Walk& w) { return w.leaf; }
  __device__ static __forceinline__ int id(const FwdParams&, const Walk& w) { return w.leaf; }

  __device__ static __forceinline__ Cell carried(const Walk& w) {
    Cell c;
    c.leaf = w.leaf;
    return c;
  }

  // A Voronoi cell is no box: the position is kept inside the domain only (a
  // walk from a point a rounding error outside its cell takes a zero-length
  // segment there).
  __device__ static __forceinline__ void clamp(const FwdParams& P, const Cell&, float3& x) {
    x.x = fminf(fmaxf(x.x, P.lo[0]), P.hi[0]);
    x.y = fminf(fmaxf(x.y, P.lo[1]), P.hi[1]);
    x.z = fminf(fmaxf(x.z, P.lo[2]), P.hi[2]);
  }
};

// ---------------------------------------------------------------- lane state
// The lane state that only the per-event work touches lives in per-thread
// slots of shared memory (structure of arrays: the lanes of a warp hit
// distinct banks), so that the walk's own state fits the registers of four
// resident blocks per SM.
__shared__ unsigned long long S_PID[kBlock];
__shared__ double S_WEIGHT[kBlock];
__shared__ float3 S_DIR[kBlock];
__shared__ float2 S_HG[kBlock];
__shared__ int S_EVENT[kBlock], S_INSTR_Q[kBlock], S_WPHASE[kBlock];
// binary exponent of a path-1 deposit weight outside [1e-30, 1e30] (aux1 < 0)
__shared__ int S_DEPEXP[kBlock];
__shared__ bool S_HAS_CELL[kBlock];
__shared__ CartGrid::Cell S_CELL_CART[kBlock];
__shared__ OctGrid::Cell S_CELL_OCT[kBlock];

template <class G>
__device__ __forceinline__ typename G::Cell& cell_slot();
template <>
__device__ __forceinline__ CartGrid::Cell& cell_slot<CartGrid>() { return S_CELL_CART[threadIdx.x]; }
template <>
__device__ __forceinline__ OctGrid::Cell& cell_slot<OctGrid>() { return S_CELL_OCT[threadIdx.x]; }
template <>
__device__ __forceinline__ RectGrid::Cell& cell_slot<RectGrid>() { return S_CELL_CART[threadIdx.x]; }
template <>
__device__ __forceinline__ BinGrid::Cell& cell_slot<BinGrid>() { return S_CELL_OCT[threadIdx.x]; }
template <>
__device__ __forceinline__ VorGrid::Cell& cell_slot<VorGrid>() { return S_CELL_OCT[threadIdx.x]; }

template <class G>
struct Lane {
  int lam, phase;
  float kappa;          // extinction per unit density at this wavelength
  float3 x;             // position
  bool walking;
  // in shared memory: packet id, event index, instrument of the next
  // peel-off, the walk a kStart lane begins, weight, direction of travel,
  // the event's Henyey-Greenstein uniforms, the cell of x (valid when
  // has_cell)
  __device__ __forceinline__ unsigned long long& pid() const { return S_PID[threadIdx.x]; }
  __device__ __forceinline__ int& event() const { return S_EVENT[threadIdx.x]; }
  __device__ __forceinline__ int& q() const { return S_INSTR_Q[threadIdx.x]; }
  __device__ __forceinline__ int& wphase() const { return S_WPHASE[threadIdx.x]; }
  __device__ __forceinline__ double& L() const { return S_WEIGHT[threadIdx.x]; }
  __device__ __forceinline__ float3& k() const { return S_DIR[threadIdx.x]; }
  __device__ __forceinline__ float& u_mu() const { return S_HG[threadIdx.x].x; }
  __device__ __forceinline__ float& u_phi() const { return S_HG[threadIdx.x].y; }
  __device__ __forceinline__ typename G::Cell& cell() const { return cell_slot<G>(); }
  __device__ __forceinline__ bool& has_cell() const { return S_HAS_CELL[threadIdx.x]; }
  float3 d, id;         // direction of the current walk and its inverse
  typename G::Walk w;   // the walk: its current cell and exit data
  float rho;            // density of the walk's current cell (loaded one crossing ahead)
  float th, tl;         // optical depth of the current walk (pair sum)
  // path 1: the deposit weight (1 - albedo) L as aux0 2^e: aux0 the FP32
  // weight (e = 0) while that lies in [1e-30, 1e30], with aux1 = 64, the
  // optical depth below which a deposit takes the plain FP32 product; else
  // aux0 in [1/2, 1) and e in S_DEPEXP, aux1 = -1 (every deposit carries the
  // exponent), so that deposits keep FP64's range whatever the weight;
  // path 2: tau* as a float pair, then s*
  float aux0, aux1;
  // adjoint tape (launches that record one): plane sums of the current path
  // walk, entry axis of its segment, crossings so far, the interaction's
  // crossing index, kappa rho and remainder, the unit exponent of weights
  float3 g;
  int axis_in, n_cross, h, eL;
  float kr_h, rem;
  AdjRecord* rec;
};

// Small per-launch tables (instruments, per-wavelength optics) copied to
// shared memory at kernel start.
__shared__ DevInstr S_INSTR[kMaxInstruments];
__shared__ DevLambda S_LAM[kMaxLambda];

// Per-lane tallies, one slot per thread in shared memory (no atomics).
struct LaneTally {
  double escaped, absorbed, truncated;
  unsigned long long crossings, path_crossings, column_crossings;
  unsigned events, peeloffs, packets, column_peels;
};

template <class G>
__device__ __forceinline__ void trace_row(const FwdParams& P, const Lane<G>& s, int event, int cell, double L,
                                          double tau_path, double tau_star) {
  if (!P.trace || s.pid() != P.trace_packet || s.lam != P.trace_lambda || event >= P.trace_cap) return;
  rt_trace_row r;
  r.event = event; r.reserved = 0; r.cell = cell;
  r.x[0] = s.x.x; r.x[1] = s.x.y; r.x[2] = s.x.z;
  r.k[0] = s.k().x; r.k[1] = s.k().y; r.k[2] = s.k().z;
  r.L = L; r.tau_path = tau_path; r.tau_star = tau_star;
  P.trace[event] = r;
}

// Start a walk from the lane's position along d; the first cell's density
// load is issued here.
template <class G>
__device__ __forceinline__ void start_walk(const FwdParams& P, Lane<G>& s, float3 d, typename G::Scratch& sc) {
  s.d = d;
  s.id = make_float3(inv_or_zero(d.x), inv_or_zero(d.y), inv_or_zero(d.z));
  s.th = 0.0f;
  s.tl = 0.0f;
  s.walking = G::init(P, s.x, d, s.id, s.has_cell(), s.cell(), s.w, sc);
  if (s.walking) s.rho = load_density(&P.density[G::cell(s.w)]);
}

__device__ __forceinline__ float3 instr_dir(const DevInstr& I) { return make_float3(I.kobs[0], I.kobs[1], I.kobs[2]); }

// A peel-off along a frame that looks exactly along grid axis I.axis: the
// optical depth to the boundary is kappa (rho_c ds_0 + column[c]), with ds_0
// the distance to the face of the current cell that the ray leaves (the first
// segment of the walk) and column[c] the density integral of the cells beyond
// it on the same grid line.  The walk's crossings (n_cross) are counted all
// the same.  known: x lies in cell cc.  False when the position is outside the
// grid (the walk then finds the entry).
template <class G>
__device__ __forceinline__ bool column_tau(const FwdParams& P, float3 x, bool known, const CartGrid::Cell& cc,
                                           const DevInstr& I, float kappa, float& th,
                                           unsigned long long& n_cross) {
  CartGrid::Cell c;
  if (known) {
    c = cc;
  } else {
    if (!inside_box(P, x)) return false;
    G::locate_cell(P, x, c);
  }
  const int a = I.axis;
  const bool up = I.dir > 0;
  const int i = a == 0 ? c.ix : (a == 1 ? c.iy : c.iz);
  const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
  const float xa = a == 0 ? x.x : (a == 1 ? x.y : x.z);
  const float plane = G::plane(P, a, i + (up ? 1 : 0));
  const float ds0 = fmaxf(up ? plane - xa : xa - plane, 0.0f);
  const int cell = c.ix + P.nx * (c.iy + P.ny * c.iz);  // row-major: the column sums
  const int slot = c.ix * P.stride[0] + c.iy * P.stride[1] + c.iz * P.stride[2];
  th = kappa * fmaf(load_density(&P.density[slot]), ds0, __ldg(&I.column[cell]));
  n_cross = (unsigned long long)(up ? n - i : i + 1);
  return true;
}

template <class G>
__device__ __forceinline__ bool column_peel(const FwdParams& P, Lane<G>& s, const DevInstr& I, LaneTally* bt) {
  unsigned long long nc;
  if (!column_tau<G>(P, s.x, s.has_cell(), s.cell(), I, s.kappa, s.th, nc)) return false;
  s.tl = 0.0f;
  s.walking = false;
  bt->crossings += nc;
  bt->column_crossings += nc;
  bt->column_peels += 1u;
  return true;
}

// The optical depth th + tl from x along d to the grid boundary (FP32 pair
// sum, the transport kernel's walk arithmetic); known: x lies in cell cc.
// Returns the crossings.
__device__ __forceinline__ unsigned ray_tau(const FwdParams& P, float3 x, float3 d, bool known,
                                            const CartGrid::Cell& cc, float kappa, float& th, float& tl) {
  const float3 id = make_float3(inv_or_zero(d.x), inv_or_zero(d.y), inv_or_zero(d.z));
  CartGrid::Walk w;
  CartGrid::Scratch sc;
  th = 0.0f;
  tl = 0.0f;
  unsigned n = 0;
  if (CartGrid::init(P, x, d, id, known, cc, w, sc)) {
    float rho = load_density(&P.density[w.cell]);
    while (true) {
      int axis;
      const float te = CartGrid::exit(w, x, id, axis);
      const float texit = fmaxf(te, w.t);
      const float ds = texit - w.t;
      const float kr = kappa * rho;
      const float dt = kr * ds;
      float nh, e;
      two_sum(th, dt, nh, e);
      tl = tl + e;
      th = nh;
      ++n;
      w.t = texit;
      if (!CartGrid::advance(P, x, d, id, axis, w, sc)) break;
      rho = load_density(&P.density[w.cell]);
    }
  }
  return n;
}

// Phase-function value of a scattering peel-off towards instrument I.
__device__ __forceinline__ float peel_phase(int lam, float3 k, const DevInstr& I) {
  return hg_phase(S_LAM[lam].g, k.x * I.kobs[0] + k.y * I.kobs[1] + k.z * I.kobs[2]);
}

// Deposit a finished peel-off from x (weight L, phase-function value phase,
// optical depth th + tl) into instrument q's image(s); pid and event only
// label debug records.
__device__ __forceinline__ void deposit_peel(const FwdParams& P, int q, int lam, float3 x, double L, float phase,
                                             float th, float tl, bool scattered, unsigned long long pid, int event) {
  const DevInstr& I = S_INSTR[q];
  // exp(-(th + tl)) with the walk's compensated optical depth: the low word
  // enters as the first-order factor (1 - tl)
  const float tau = th;
  const double value = tau < 80.0f ? L * widen(kInv4PiF * phase * expf(-tau) * (1.0f - tl))
                                   : L * kInv4PiD * (double)phase * exp(-((double)tau + (double)tl));
  const int ch = scattered ? 2 : 1;
  if (I.sed) {
    // an SED instrument has one bin per wavelength and channel: the lanes of
    // the warp that deposit into the same bin add their values first (in lane
    // order) and one of them issues the atomics
    const unsigned act = __activemask();
    const unsigned key = ((unsigned)q << 20) | ((unsigned)lam << 1) | (scattered ? 1u : 0u);
    const unsigned grp = __match_any_sync(act, key);
    double sum = 0.0;
    for (unsigned m = grp; m; m &= m - 1u) sum += __shfl_sync(grp, value, __ffs(m) - 1);
    if ((int)(threadIdx.x & 31u) == __ffs(grp) - 1) {
      atomicAdd(&I.image[lam], sum);
      if (I.channels == 3) atomicAdd(&I.image[(size_t)ch * P.n_lambda + lam], sum);
    }
    if (P.records && (P.record_stride <= 1 || pid % P.record_stride == 0)) {
      const unsigned long long slot = atomicAdd(&P.counters[4], 1ull);
      if ((long long)slot < P.records_cap) {
        rt_record r;
        r.packet = pid; r.lambda = lam; r.event = scattered ? event : 0; r.instrument = q;
        r.reserved = 0; r.pixel = 0; r.value = value;
        P.records[slot] = r;
      }
    }
    return;
  }
  const float fx = (x.x * I.ex[0] + x.y * I.ex[1] + x.z * I.ex[2] + I.off_x) * I.sx;
  const float fy = (x.x * I.ey[0] + x.y * I.ey[1] + x.z * I.ey[2] + I.off_y) * I.sy;
  const size_t plane = (size_t)I.ny * I.nx;
  if (!I.bilinear) {
    const float fix = floorf(fx), fiy = floorf(fy);
    if (!(fix >= 0.0f && fiy >= 0.0f && fix < (float)I.nx && fiy < (float)I.ny)) return;
    const size_t pix = (size_t)(int)fiy * I.nx + (int)fix;
    atomicAdd(&I.image[(size_t)lam * plane + pix], value);
    if (I.channels == 3) atomicAdd(&I.image[((size_t)ch * P.n_lambda + lam) * plane + pix], value);
    if (P.records && (P.record_stride <= 1 || pid % P.record_stride == 0)) {
      const unsigned long long slot = atomicAdd(&P.counters[4], 1ull);
      if ((long long)slot < P.records_cap) {
        rt_record r;
        r.packet = pid; r.lambda = lam; r.event = scattered ? event : 0; r.instrument = q;
        r.reserved = 0; r.pixel = (int64_t)pix; r.value = value;
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
        const double v = value * widen((dx ? tx : 1.0f - tx) * (dy ? ty : 1.0f - ty));
        const size_t pix = (size_t)(int)fiy * I.nx + (int)fix;
        atomicAdd(&I.image[(size_t)lam * plane + pix], v);
        if (I.channels == 3) atomicAdd(&I.image[((size_t)ch * P.n_lambda + lam) * plane + pix], v);
      }
    }
  }
}

template <class G>
__device__ __forceinline__ void peel_deposit(const FwdParams& P, const Lane<G>& s, bool scattered) {
  const float phase = scattered ? peel_phase(s.lam, s.k(), S_INSTR[s.q()]) : 1.0f;
  deposit_peel(P, s.q(), s.lam, s.x, s.L(), phase, s.th, s.tl, scattered, s.pid(), s.event());
}

// Hand the peel-off towards instrument q from x to the sorted pass: a
// record in the next free slot (one atomic per group of lanes), counted under
// its sort key.  known: x lies in cell c (else it is located by the walk).
// False when the buffer is full (the caller then walks it itself).
__device__ __forceinline__ bool defer_record(const FwdParams& P, int q, int lam, float3 x, double L, float phase,
                                             bool known, const CartGrid::Cell& cc, bool emission,
                                             unsigned long long pid, int event) {
  const unsigned m = __activemask();
  const unsigned lane = threadIdx.x & 31u;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(P.peel_count, (unsigned long long)__popc(m));
  base = __shfl_sync(m, base, leader);
  const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
  if (slot >= P.peel_cap) return false;
  unsigned c = (unsigned)P.n_cells;
  if (known) {
    c = (unsigned)(cc.ix + P.nx * (cc.iy + P.ny * cc.iz));
  } else if (inside_box(P, x)) {
    // the cell the walk will locate x in
    const int ix = min(max(__float2int_rd((x.x - P.lo[0]) * P.inv_d[0]), 0), P.nx - 1);
    const int iy = min(max(__float2int_rd((x.y - P.lo[1]) * P.inv_d[1]), 0), P.ny - 1);
    const int iz = min(max(__float2int_rd((x.z - P.lo[2]) * P.inv_d[2]), 0), P.nz - 1);
    c = (unsigned)(ix + P.nx * (iy + P.ny * iz));
  }
  const unsigned key = (unsigned)q * (unsigned)(P.n_cells + 1) + c;
  const unsigned meta = (unsigned)lam | (emission ? 0u : 1u << 30) | (known ? 1u << 31 : 0u);
  const long long Lb = __double_as_longlong(L);
  float4* r = reinterpret_cast<float4*>(&P.peel[slot]);
  r[0] = make_float4(x.x, x.y, x.z, __uint_as_float(key));
  r[1] = make_float4(__int_as_float((int)(unsigned)Lb), __int_as_float((int)(Lb >> 32)), phase, __uint_as_float(meta));
  if (P.peel_tag) P.peel_tag[slot] = make_ulonglong2(pid, (unsigned long long)event);
  atomicAdd(&P.peel_hist[key], 1u);
  return true;
}

template <class G>
__device__ __forceinline__ bool defer_peel(const FwdParams& P, const Lane<G>& s, const DevInstr& I, bool emission) {
  const float phase = emission ? 1.0f : peel_phase(s.lam, s.k(), I);
  return defer_record(P, s.q(), s.lam, s.x, s.L(), phase, s.has_cell(), s.cell(), emission, s.pid(), s.event());
}

// Emission (Sect. 3.4): source component by luminosity (FP64 comparison of
// the uniform with the cumulative fractions), position from its geometry and
// an isotropic direction (FP32).
__device__ __forceinline__ void emit(const FwdParams& P, unsigned long long pid, int lam, float3& x_out, float3& k_out) {
  const uint4 r0 = draw_block(pid, lam, 0, 0, P.seed, P.model);
  const uint4 r1 = draw_block(pid, lam, 0, 1, P.seed, P.model);
  int src = P.n_sources - 1;
  if (P.n_sources > 1) {
    const double u0 = u01(r0.x);
    for (int i = 0; i < P.n_sources; ++i) {
      if (u0 < P.src_cum[lam * P.n_sources + i]) { src = i; break; }
    }
  }
  const DevSource& S = P.src[src];
  float3 x = make_float3((float)S.center[0], (float)S.center[1], (float)S.center[2]);
  if (S.kind == RT_SOURCE_EXPDISK) {
    // R has density R exp(-R/hR): minus hR times the log of two uniforms
    const float R = -(float)S.scale_r * (logf(u01f(r0.y)) + logf(u01f(r0.z)));
    float sp, cp;
    sincospif(2.0f * u01f(r0.w), &sp, &cp);
    float z = -(float)S.scale_z * logf(u01f(r1.x));
    if (r1.y < 0x80000000u) z = -z;  // u5 < 1/2
    x.x += R * cp; x.y += R * sp; x.z += z;
  } else if (S.kind == RT_SOURCE_PLUMMER) {
    // enclosed mass fraction m = r^3 / (r^2 + a^2)^(3/2): r = a / sqrt(m^(-2/3) - 1)
    const float m = u01f(r0.y);
    const float r = (float)S.scale_r / sqrtf(expm1f(-(2.0f / 3.0f) * logf(m)));
    const float ct = u01f_signed(r0.z), st = sqrtf(fmaxf(0.0f, 1.0f - ct * ct));
    float sp, cp;
    sincospif(2.0f * u01f(r0.w), &sp, &cp);
    x.x += r * st * cp; x.y += r * st * sp; x.z += r * ct;
  }
  x_out = x;
  const float mu = u01f_signed(r1.z);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
  float sp, cp;
  sincospif(2.0f * u01f(r1.w), &sp, &cp);
  k_out = make_float3(st * cp, st * sp, mu);
}

// Emission by the dust (panchromatic mode): the cell with probability
// proportional to its thermal luminosity at this wavelength (the first cell
// whose running sum exceeds u times the total, FP64), a uniform position in
// it (FP32, kept inside its planes), an isotropic direction; the cell is
// known to the first walks.
template <class G>
__device__ __forceinline__ void emit_dust(const FwdParams& P, unsigned long long pid, int lam, float3& x_out,
                                          float3& k_out, typename G::Cell& cell) {
  if constexpr (G::kIndexCells) {
    const uint4 r0 = draw_block(pid, lam, 0, 0, P.seed, P.model);
    const uint4 r1 = draw_block(pid, lam, 0, 1, P.seed, P.model);
    const double* cum = P.dust_cum + (size_t)lam * P.n_cells;
    const double target = u01(r0.x) * cum[P.n_cells - 1];
    long long lo = 0, hi = P.n_cells - 1;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (cum[mid] > target) hi = mid; else lo = mid + 1;
    }
    const int c = (int)lo;
    cell.ix = c % P.nx;
    cell.iy = (c / P.nx) % P.ny;
    cell.iz = c / (P.nx * P.ny);
    const int idx[3] = {cell.ix, cell.iy, cell.iz};
    const float u[3] = {u01f(r0.y), u01f(r0.z), u01f(r0.w)};
    float p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float lo_a = G::plane(P, a, idx[a]), hi_a = G::plane(P, a, idx[a] + 1);
      p[a] = fminf(fmaxf(fmaf(u[a], hi_a - lo_a, lo_a), lo_a), hi_a);
    }
    x_out = make_float3(p[0], p[1], p[2]);
    const float mu = u01f_signed(r1.z);
    const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
    float sp, cp;
    sincospif(2.0f * u01f(r1.w), &sp, &cp);
    k_out = make_float3(st * cp, st * sp, mu);
  }
}

// Ask for walk `phase` from the lane's position along d; walks start in the
// last stage of a control round, from one place in the code.
template <class G>
__device__ __forceinline__ void request_walk(Lane<G>& s, int phase, float3 d) {
  s.wphase() = phase;
  s.d = d;
  s.phase = kStart;
}

// The forced path of event s.event(): its first walk carries the deposit
// weight (1 - albedo) L.
template <class G>
__device__ __forceinline__ void request_path(Lane<G>& s) {
  const double wdep = S_LAM[s.lam].one_minus_albedo * s.L();
  const bool plain = wdep >= 1e-30 && wdep <= 1e30;
  int e = 0;
  s.aux0 = plain ? cut(wdep) : split_exp(wdep, e);
  s.aux1 = plain ? 64.0f : -1.0f;
  S_DEPEXP[threadIdx.x] = e;
  request_walk(s, kPath1, s.k());
}

// ---- the stages of a control round (each for the lanes in that phase)

// ---- the adjoint tape (cartesian grids; records as the adjoint's replay writes them)

// v 2^-e as FP32 (e: the unit exponent), by cutting the significand.
__device__ __forceinline__ float tape_units(double v, int e) {
  const long long b = __double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7ff);
  const int fe = be - 896 - e;
  if (be == 0x7ff || fe >= 255) return (float)ldexp(v, -e);
  if (be == 0 || fe <= 0) return 0.0f;
  const unsigned top = (unsigned)((unsigned long long)b >> 32);
  return __uint_as_float((top & 0x80000000u) | ((unsigned)fe << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
}

template <class G>
__device__ __forceinline__ int tape_cell(const FwdParams& P, const Lane<G>& s) {
  if constexpr (G::kColumns) {
    return s.has_cell() ? s.cell().ix + P.nx * (s.cell().iy + P.ny * s.cell().iz) : -1;
  } else {
    return -1;
  }
}

// The packet ends after event J: record 0 holds J and the last position.
template <class G>
__device__ __forceinline__ void tape_end(const FwdParams& P, const Lane<G>& s, int J) {
  AdjRecord& r = s.rec[0];
  r.h = J;
  r.x[0] = s.x.x; r.x[1] = s.x.y; r.x[2] = s.x.z;
  r.cell = tape_cell(P, s);
  r.L = tape_units(s.L(), s.eL);
}

// A new packet (index w of the launch): wavelength, weight, emission.
template <class G, bool kTape>
__device__ __forceinline__ void fetch(const FwdParams& P, Lane<G>& s, unsigned long long w, LaneTally* bt) {
  if (w >= P.n_total) { s.phase = kExit; return; }
  int lam = min((int)(__ull2float_rz(w) * P.inv_n_per_lambda), P.n_lambda - 1);
  while (lam > 0 && (unsigned long long)lam * P.n_per_lambda > w) --lam;
  while (lam + 1 < P.n_lambda && (unsigned long long)(lam + 1) * P.n_per_lambda <= w) ++lam;
  s.lam = lam;
  s.pid() = P.first_id + (w - (unsigned long long)lam * P.n_per_lambda);
  const double L0 = P.L0[lam];
  if (L0 == 0.0) {  // no emission at this wavelength (dust that emits nothing here)
    bt->packets += 1u;
    s.phase = kFetch;
    return;
  }
  s.kappa = S_LAM[lam].kappa;
  s.L() = L0;
  s.event() = 0;
  s.has_cell() = false;
  if constexpr (G::kIndexCells) {
    if (P.dust_cum) {
      emit_dust<G>(P, s.pid(), s.lam, s.x, s.k(), s.cell());
      s.has_cell() = true;
    } else {
      emit(P, s.pid(), s.lam, s.x, s.k());
    }
  } else {
    emit(P, s.pid(), s.lam, s.x, s.k());
  }
  bt->packets += 1u;
  trace_row(P, s, 0, -1, L0, 0.0, 0.0);
  if (kTape) {
    s.rec = P.tape + (size_t)w * (size_t)P.tape_stride;
    const int be = (int)((__double_as_longlong(L0) >> 52) & 0x7ff);
    s.eL = be == 0 ? 0 : be - 1022;  // L0 = m 2^eL, m in [1/2, 1)
  }
  s.q() = 0;
  s.phase = kPeelScan;
}

// Path 1 ended: escape, or the deposit bookkeeping and the forced-scattering
// inversion (FP64); then the second walk.
template <class G, bool kTape>
__device__ __forceinline__ void finish_path1(const FwdParams& P, Lane<G>& s, LaneTally* bt) {
  const double tau = widen(s.th) + widen(s.tl);
  if (!(tau > 0.0)) {
    trace_row(P, s, s.event(), -1, s.L(), 0.0, 0.0);
    bt->escaped += s.L();
    if (kTape) tape_end(P, s, s.event() - 1);
    s.phase = kFetch;
    return;
  }
  const double one_minus_E = -expm1(-tau);
  const double E = 1.0 - one_minus_E;
  bt->escaped += s.L() * E;
  bt->absorbed += S_LAM[s.lam].one_minus_albedo * s.L() * one_minus_E;
  const uint4 r = draw_block(s.pid(), s.lam, s.event(), 0, P.seed, P.model);
  const double tau_star = -log1p(-u01(r.x) * one_minus_E);
  s.u_mu() = u01f(r.y);
  s.u_phi() = u01f(r.z);
  split_pair(tau_star, s.aux0, s.aux1);
  if (kTape) {
    // the record's first two sectors, whole, with 16-byte stores
    float4* t = reinterpret_cast<float4*>(&s.rec[s.event()]);
    t[0] = make_float4(s.x.x, s.x.y, s.x.z, s.k().x);
    t[1] = make_float4(s.k().y, s.k().z, __int_as_float(tape_cell(P, s)), tape_units(s.L(), s.eL));
    t[2] = make_float4((float)one_minus_E, (float)E, u01f(r.x), s.g.x);
    t[3] = make_float4(s.g.y, s.g.z, 0.0f, 0.0f);
    s.h = -1;
  }
  s.L() = S_LAM[s.lam].albedo * s.L() * one_minus_E;  // weight after the scattering
  request_walk(s, kPath2, s.k());
}

// Path 2 ended in the interaction cell (aux0 holds s*): move the packet,
// then the scattering peel-offs.
template <class G, bool kTape>
__device__ __forceinline__ void finish_path2(const FwdParams& P, Lane<G>& s, LaneTally* bt) {
  if (kTape) {
    // the record's third sector, whole
    float4* t = reinterpret_cast<float4*>(&s.rec[s.event()]);
    t[4] = make_float4(__int_as_float(s.h), __int_as_float(s.axis_in), __int_as_float(G::id(P, s.w)), s.kr_h);
    t[5] = make_float4(s.rem, s.g.x, s.g.y, s.g.z);
  }
  const float s_star = s.aux0;
  float3 x = make_float3(fmaf(s_star, s.k().x, s.x.x), fmaf(s_star, s.k().y, s.x.y), fmaf(s_star, s.k().z, s.x.z));
  s.cell() = G::carried(s.w);
  G::clamp(P, s.cell(), x);
  s.x = x;
  s.has_cell() = true;
  bt->events += 1u;
  trace_row(P, s, s.event(), G::id(P, s.w), s.L(), 0.0, 0.0);
  s.q() = 0;
  s.phase = kPeelScan;
}

// The peel-off towards instrument s.q(), or the end of the event's peel-offs:
// along a frame that looks along a grid axis the optical depth comes from
// the column sums at once (the lane then waits for the deposit stage);
// otherwise a record for the sorted pass, or (no pass, or its buffer full)
// its walk.  After the last instrument: the first forced path (emission) or
// the scattering (kAfter).
template <class G>
__device__ __forceinline__ void peel_scan(const FwdParams& P, Lane<G>& s, LaneTally* bt) {
  const bool emission = s.event() == 0;
  if ((emission ? P.peel_emission : P.peel_scatter) && s.q() < P.n_instr) {
    const DevInstr& I = S_INSTR[s.q()];
    const int phase = emission ? kPeelEmit : kPeelScat;
    if constexpr (G::kColumns) {
      if (P.use_columns && I.column && column_peel(P, s, I, bt)) {
        s.phase = phase;
        return;
      }
      if (P.peel && G::kSortedPass && defer_peel(P, s, I, emission)) {
        // walked and deposited by the sorted pass; on to the next instrument
        bt->peeloffs += 1u;
        s.q() += 1;
        return;
      }
    }
    request_walk(s, phase, instr_dir(I));
    return;
  }
  if (emission) {
    s.event() = 1;
    request_path(s);
  } else {
    s.phase = kAfter;
  }
}

// After the scattering peel-offs: new direction, then termination or the
// next forced path.
template <class G, bool kTape>
__device__ __forceinline__ void after_scattering(const FwdParams& P, Lane<G>& s, LaneTally* bt) {
  const float mu = hg_sample(S_LAM[s.lam].g, s.u_mu());
  float sp, cp;
  sincospif(2.0f * s.u_phi(), &sp, &cp);
  s.k() = rotate_dir(s.k(), mu, sp, cp);
  if ((P.weight_cut && s.L() < P.L_cut[s.lam]) || s.event() >= P.max_events) {
    bt->truncated += s.L();
    if (kTape) tape_end(P, s, s.event());
    s.phase = kFetch;
    return;
  }
  s.event() += 1;
  request_path(s);
}

// One control round for the warp: every stage runs for the lanes in its
// phase together, and a stage hands lanes on to later stages (the peel-off
// loop repeats deposit and scan while any lane has a peel-off ready, which
// column sums complete without a walk; lanes whose packet ended fetch the
// next one and go round once more).
template <class G, bool kTape>
__device__ __forceinline__ void control_round(const FwdParams& P, Lane<G>& s, LaneTally* bt,
                                              typename G::Scratch& sc, unsigned lane, unsigned lt_mask) {
  if (!s.walking) {
    if (s.phase == kPath1) finish_path1<G, kTape>(P, s, bt);
    if (s.phase == kPath2) finish_path2<G, kTape>(P, s, bt);
  }
  // Peel-offs, the scattering and new packets, repeated while a lane has
  // just finished its packet: such a lane starts its next packet in the same
  // round (at most two passes: a new packet never ends before its first walk).
  while (true) {
    while (true) {
      const bool ready = !s.walking && (s.phase == kPeelEmit || s.phase == kPeelScat);
      if (!__any_sync(0xffffffffu, ready || s.phase == kPeelScan)) break;
      if (ready) {
        peel_deposit(P, s, s.phase == kPeelScat);
        bt->peeloffs += 1u;
        s.q() += 1;
        s.phase = kPeelScan;
      }
      if (s.phase == kPeelScan) peel_scan(P, s, bt);
    }
    if (s.phase == kAfter) after_scattering<G, kTape>(P, s, bt);
    // packets for every lane that needs one: one atomic per warp
    const bool wants = !s.walking && s.phase == kFetch;
    const unsigned fetchers = __ballot_sync(0xffffffffu, wants);
    if (!fetchers) break;
    unsigned long long base = 0;
    const int leader = __ffs(fetchers) - 1;
    if ((int)lane == leader) base = atomicAdd(P.work_counter, (unsigned long long)__popc(fetchers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (wants) fetch<G, kTape>(P, s, base + __popc(fetchers & lt_mask), bt);
  }
  if (s.phase == kStart) {
    s.phase = s.wphase();
    if (kTape) {
      s.g = make_float3(0.0f, 0.0f, 0.0f);
      s.axis_in = -1;
      s.n_cross = 0;
    }
    start_walk(P, s, s.d, sc);
  }
}

// One cell crossing of the lane's current walk.  Written with selects rather
// than branches where lanes in different walks (peel-off, forced path 1 or 2)
// share the step, so the warp issues it once.
template <class G, bool kTape>
__device__ __forceinline__ void walk_step(const FwdParams& P, Lane<G>& s, unsigned& n_path, unsigned& n_peel,
                                          typename G::Scratch& sc) {
  typename G::Walk& w = s.w;
  int axis;
  const float te = G::exit(w, s.x, s.id, axis);
  const float texit = fmaxf(te, w.t);
  const float ds = texit - w.t;
  const float kr = s.kappa * s.rho;
  const float dt = kr * ds;
  // optical depth of the walk as an exact pair sum (all walks)
  float nh, e;
  two_sum(s.th, dt, nh, e);
  const float nl = s.tl + e;
  const bool path1 = s.phase == kPath1;
  const bool path2 = s.phase == kPath2;
  if (path2 && (nh - s.aux0) + (nl - s.aux1) > 0.0f) {
    // interaction in this cell: s* = t_in + (tau* - tau_before) / (kappa rho);
    // tau* - tau_before from the two pairs (aux0 - th is exact where it matters)
    const float rem = ((s.aux0 - s.th) + s.aux1) - s.tl;
    s.aux0 = w.t + rem / kr;
    s.walking = false;
    if (kTape) {
      s.kr_h = kr;
      s.rem = rem;
      s.h = s.n_cross;
    }
    return;
  }
  if (kTape && (path1 || path2)) {
    // plane sums of the path for the adjoint: +kr at the exit plane, -kr at the entry plane
    s.g.x += (axis == 0 ? kr : 0.0f) - (s.axis_in == 0 ? kr : 0.0f);
    s.g.y += (axis == 1 ? kr : 0.0f) - (s.axis_in == 1 ? kr : 0.0f);
    s.g.z += (axis == 2 ? kr : 0.0f) - (s.axis_in == 2 ? kr : 0.0f);
    s.axis_in = axis;
    ++s.n_cross;
  }
  if (path1 && dt > 0.0f) {
    // continuous absorption: (1 - albedo) L exp(-tau_before) (1 - exp(-dtau))
    double* const a = &P.absorption[(size_t)s.lam * P.n_cells + G::cell(w)];
    if (s.th < s.aux1) {
      add_absorption(a, widen(s.aux0 * __expf(-s.th) * one_minus_exp_neg(dt)));
    } else {
      // exp(-tau_before) = 2^-y, y = k + f with k = floor(y): the integer
      // part joins the weight's exponent, so deep deposits do not underflow
      const float y = s.th * 1.44269504f;
      const float k = floorf(y);
      add_absorption(a, widen_exp(s.aux0 * exp2f(k - y) * one_minus_exp_neg(dt), S_DEPEXP[threadIdx.x] - (int)k));
    }
  }
  s.th = nh;
  s.tl = nl;
  n_path += path1 ? 1u : 0u;
  n_peel += (path1 || path2) ? 0u : 1u;
  w.t = texit;
  if (G::advance(P, s.x, s.d, s.id, axis, w, sc)) {
    s.rho = load_density(&P.density[G::cell(w)]);  // consumed by the next crossing
  } else {
    s.walking = false;
    if (path2) {
      // not reachable: the pair sums of both walks are identical and tau* is
      // below the path's optical depth; keep the packet at the path's end
      atomicOr(P.flags, kFlagNoInteraction);
      s.aux0 = texit;
    }
  }
}

template <class G>
__device__ __forceinline__ typename G::Scratch lane_scratch(const FwdParams& P);
template <>
__device__ __forceinline__ CartGrid::Scratch lane_scratch<CartGrid>(const FwdParams&) { return CartGrid::Scratch{}; }
template <>
__device__ __forceinline__ RectGrid::Scratch lane_scratch<RectGrid>(const FwdParams&) { return RectGrid::Scratch{}; }
template <>
__device__ __forceinline__ BinGrid::Scratch lane_scratch<BinGrid>(const FwdParams&) { return BinGrid::Scratch{}; }
template <>
__device__ __forceinline__ VorGrid::Scratch lane_scratch<VorGrid>(const FwdParams&) { return VorGrid::Scratch{}; }
template <>
__device__ __forceinline__ OctGrid::Scratch lane_scratch<OctGrid>(const FwdParams& P) {
  return OctGrid::Scratch{&S_OCT_STACK[threadIdx.x * P.oct_levels]};
}

template <class G>
__device__ __forceinline__ void load_grid_cache(const FwdParams& P);
template <>
__device__ __forceinline__ void load_grid_cache<CartGrid>(const FwdParams&) {}
template <>
__device__ __forceinline__ void load_grid_cache<RectGrid>(const FwdParams&) {}
template <>
__device__ __forceinline__ void load_grid_cache<VorGrid>(const FwdParams&) {}
template <>
__device__ __forceinline__ void load_grid_cache<BinGrid>(const FwdParams& P) {
  const int n = P.n_nodes < kChildCache ? (int)P.n_nodes : kChildCache;
  for (int i = threadIdx.x; i < n; i += kBlock) S_CHILD[i] = P.child[i];
}
template <>
__device__ __forceinline__ void load_grid_cache<OctGrid>(const FwdParams& P) {
  const int n = P.n_nodes < kChildCache ? (int)P.n_nodes : kChildCache;
  for (int i = threadIdx.x; i < n; i += kBlock) S_CHILD[i] = P.child[i];
}

// kProf: the kernel keeps the optional execution counters of P.profile (a
// separate instantiation: the counters' ballots and clock reads cost the
// plain kernel ~4 % of its time).
template <class G, bool kTape = false, bool kProf = false>
__device__ __forceinline__ void forward_body(const FwdParams& P) {
  __shared__ LaneTally tally[kBlock];
  for (int i = threadIdx.x; i < P.n_instr; i += kBlock) S_INSTR[i] = P.instr[i];
  for (int i = threadIdx.x; i < P.n_lambda; i += kBlock) S_LAM[i] = P.lam[i];
  load_grid_cache<G>(P);
  __syncthreads();
  typename G::Scratch sc = lane_scratch<G>(P);
  LaneTally* bt = &tally[threadIdx.x];
  bt->escaped = bt->absorbed = bt->truncated = 0.0;
  bt->crossings = bt->path_crossings = bt->column_crossings = 0ull;
  bt->events = bt->peeloffs = bt->packets = bt->column_peels = 0u;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  Lane<G> s;
  s.phase = kFetch;
  s.walking = false;
  unsigned n_path = 0, n_peel = 0;
  // optional execution counters (warp leader only)
  const bool prof = kProf && P.profile != nullptr && lane == 0;
  // iterations, walking lanes, rounds, lanes served, cycles in control, in
  // the walk: per warp in shared memory (no registers held across the loop)
  __shared__ unsigned long long prof_c[kBlock / 32][6];
  unsigned long long* pc = prof_c[threadIdx.x >> 5];
  if (prof)
    for (int i = 0; i < 6; ++i) pc[i] = 0ull;
  while (true) {
    const bool idle = !s.walking && s.phase != kExit;
    const unsigned need = __ballot_sync(0xffffffffu, idle);
    const unsigned walkers = __ballot_sync(0xffffffffu, s.walking);
    if (need == 0u && walkers == 0u) break;
    long long t0 = 0;
    if (prof) { pc[0] += 1ull; t0 = clock64(); }
    if (walkers == 0u || __popc(need) >= P.control_min) {
      if (prof) { pc[2] += 1ull; pc[3] += __popc(need); }
      control_round<G, kTape>(P, s, bt, sc, lane, lt_mask);
      if ((n_path | n_peel) & 0xC0000000u) {  // keep the 32-bit lane counters far from overflow
        bt->crossings += (unsigned long long)n_path + n_peel;
        bt->path_crossings += n_path;
        n_path = n_peel = 0;
      }
    }
    long long t1 = 0;
    if (prof) { t1 = clock64(); pc[4] += t1 - t0; }
    const unsigned stepping = kProf ? __ballot_sync(0xffffffffu, s.walking) : 0u;
    if (s.walking) walk_step<G, kTape>(P, s, n_path, n_peel, sc);
    if (prof) { pc[1] += __popc(stepping); pc[5] += clock64() - t1; }
  }
  if (prof) {
    for (int i = 0; i < 6; ++i) atomicAdd(&P.profile[i], pc[i]);
  }
  bt->crossings += (unsigned long long)n_path + n_peel;
  bt->path_crossings += n_path;
  __syncthreads();
  if (threadIdx.x < 32) {
    double esc = 0.0, ab = 0.0, trc = 0.0;
    unsigned long long cr = 0, pc = 0, ev = 0, pe = 0, pk = 0, cc = 0, cp = 0;
    for (int t = threadIdx.x; t < kBlock; t += 32) {
      esc += tally[t].escaped; ab += tally[t].absorbed; trc += tally[t].truncated;
      cr += tally[t].crossings; pc += tally[t].path_crossings;
      ev += tally[t].events; pe += tally[t].peeloffs; pk += tally[t].packets;
      cc += tally[t].column_crossings; cp += tally[t].column_peels;
    }
    for (int o = 16; o > 0; o >>= 1) {
      esc += __shfl_down_sync(0xffffffffu, esc, o);
      ab += __shfl_down_sync(0xffffffffu, ab, o);
      trc += __shfl_down_sync(0xffffffffu, trc, o);
      cr += __shfl_down_sync(0xffffffffu, cr, o);
      pc += __shfl_down_sync(0xffffffffu, pc, o);
      ev += __shfl_down_sync(0xffffffffu, ev, o);
      pe += __shfl_down_sync(0xffffffffu, pe, o);
      pk += __shfl_down_sync(0xffffffffu, pk, o);
      cc += __shfl_down_sync(0xffffffffu, cc, o);
      cp += __shfl_down_sync(0xffffffffu, cp, o);
    }
    if (threadIdx.x == 0) {
      atomicAdd(&P.stats[1], esc);
      atomicAdd(&P.stats[2], ab);
      atomicAdd(&P.stats[3], trc);
      atomicAdd(&P.counters[0], cr);
      atomicAdd(&P.counters[1], ev);
      atomicAdd(&P.counters[2], pe);
      atomicAdd(&P.counters[3], pk);
      atomicAdd(&P.counters[5], pc);
      if (cp) {
        atomicAdd(&P.counters[6], cp);
        atomicAdd(&P.counters[7], cc);
      }
    }
  }
}

}  // namespace tr
}  // namespace rtk

// Adjoint of the forward transport: the gradient of a linear functional of
// the images and the absorption field with respect to the cell densities,
// under common random numbers (the derivative along each packet's path:
// directions and random draws fixed, positions moving with the density
// through the forced-scattering inversion, weights through 1 - exp(-tau)).
//
// Structure.  Under common random numbers a packet's adjoint is linear in the
// adjoints (Lb, xb) of its weight and position that flow backwards from later
// events, so almost all of the work runs in the forward order:
//   * peel-off at event j towards instrument q, value l = L_j P e^{-tau(x_j)} W(x_j)
//     (W: the adjoint image interpolated like the deposit): a measuring walk
//     gives tau and d tau / d x, a depositing walk adds -l kappa ds to the
//     crossed cells; its share of (Lb_j, xb_j) is stored with the event;
//   * forced path j from x_{j-1}: the replay's two walks (to the boundary, to
//     the interaction) also give the per-axis plane sums G1, GH (and, with an
//     absorption adjoint, the deposit adjoints and G0) that the position
//     adjoint needs, and the interaction data;
// and then, per packet,
//   * the backward sweep over the stored events (no walks): the total T_j of
//     the optical-depth adjoints, the adjoint tbh_j of tau_{h-1}, the
//     interaction-cell term and the new (Lb, xb);
//   * one depositing walk per forced path: grad[c_m] += kappa ds_m
//     (T_j - tbh_j [m >= h_j]) (the suffix sums of the optical-depth adjoints).
// With n instruments a scattering costs 1 + 1/2 + 1 + 2n walks against the
// forward's 1 + 1/2 + n.
//
// Execution model as in the forward kernel: persistent warps, one packet per
// lane, every walking lane advancing one crossing per iteration whatever its
// walk, the per-event work deferred until enough lanes need it and then done
// in a fixed order of stages, so that lanes at the same stage run together.
// The events of a packet are stored in the lane's slot of a device buffer.
//
// Precision.  The replay repeats the forward kernel's arithmetic (FP32
// geometry and pair sums, FP64 inversion and weights), so it follows the same
// paths.  Adjoint quantities are FP32 in exact power-of-two units (the record
// type states them), which keeps the per-event work off GB300's low-rate FP64
// pipe; each deposit into the FP64 gradient is an FP32 product widened and
// rescaled exactly with integer operations.
#include "rt_transport.cuh"

#include <algorithm>
#include <climits>
#include <cmath>

namespace rtk {

namespace {

using tr::CartGrid;

constexpr int kAdjBlock = 256;
// Resident blocks per SM the register allocation aims at.
#ifndef RT_ADJ_MIN_BLOCKS
#define RT_ADJ_MIN_BLOCKS 3
#endif
constexpr float kInv4PiF = 0.0795774715459476679f;

enum AdjPhase : int {
  // walks (the lane walks; when the walk ends its phase names the stage that finishes it)
  aPeelM = 0,     // peel-off measuring walk (instrument q)
  aPeelD = 1,     // peel-off depositing walk
  aPath1 = 2,     // forced path, first walk (to the boundary)
  aPath2 = 3,     // forced path, second walk (to the interaction)
  aDep = 4,       // depositing walk of forced path `event`, after the sweep
  // pending work between walks
  aFetch = 5,     // needs a new packet
  aPeelScan = 6,  // find the next instrument from instrument q
  aAfter = 7,     // after the peel-offs of event `event`
  aSweep = 8,     // the packet's events are complete: backward sweep
  aDepScan = 9,   // find the next forced path to deposit from path `event`
  aStart = 10,    // start walk `wphase` from x along d
  aExit = 11
};

struct AdjParams {
  FwdParams f;
  const float* adj_img[kMaxInstruments];  // adjoint images in units 2^ea (or null)
  const double* adj_abs;                  // [n_lambda][n_cells] or null (FP64, as given)
  const unsigned long long* maxbits;      // largest |adjoint input| (FP64 bits): gives ea
  int e0[kMaxLambda];                     // exponent of the initial weight per wavelength
  double* grad;                           // [n_cells]
  AdjRecord* recs;                        // [lanes][max_events + 1]
  double* line_dep[6];                    // frames along grid axes: per-line deposit differences, index
                                          // 2 axis + (direction > 0); cell c holds what every cell
                                          // beyond c on its line (in the ray's direction) receives
  int rec_stride;                         // records per lane
  unsigned long long* counters;           // optional: [0] crossings, [1] depositing crossings
  AdjRecord* tape;                        // the forward launch's tape ([packets][rec_stride]) or null: replay
};

// The lane: one packet.
struct ALane {
  unsigned long long pid;
  int lam, event, phase, wphase, q, J;
  int eL, eLA;          // 2^eL: unit of weights; 2^eLA: unit of position and tau adjoints
  double L;             // weight (as in the forward kernel)
  float kappa;
  float u_mu, u_phi;    // the event's Henyey-Greenstein uniforms
  float3 x, k;          // position, direction of travel
  CartGrid::Cell cell;  // cell of x (valid when has_cell)
  bool has_cell, walking;
  float3 d, id;         // the walk's direction and its inverse (0 for a zero component)
  CartGrid::Walk w;
  float rho;            // density of the walk's current cell
  float th, tl;         // optical depth of the walk (pair sum)
  float a0, a1;         // path 2: tau* as a pair, then s*; path 2 hit: a1 = tau* - tau_{h-1}
  float3 g;             // plane sums of the walk: sum over segments of kr (e_exit - e_entry)
  int axis_in;          // axis of the plane the current segment was entered by (-1: none)
  int n_cross;          // crossings of the walk so far
  int h;                // path 2: crossing index of the interaction (-1: none); deposits: split index
  float kr_h;           // path 2: kappa rho of the interaction cell
  float c0, c1;         // depositing walks: coefficient before / from crossing h (units 2^eLA)
  // absorption adjoint, path 1 (FP64, true units)
  double P, D, a_prev, e_prev;
  double3 g0;
  AdjRecord* rec;
  float Lf;             // tape: the weight at the current event, units 2^eL
};

__device__ __forceinline__ void grad_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// v 2^e as FP64 for FP32 v: integer operations when v is a normal number and
// the result stays normal, the FP64 pipe otherwise.
__device__ __forceinline__ double scaled(float v, int e) {
  const unsigned u = __float_as_uint(v);
  const unsigned ex = u & 0x7f800000u;
  const int be = (int)(ex >> 23) + 896 + e;  // biased FP64 exponent of the result
  if (ex == 0u || ex == 0x7f800000u || be <= 0 || be >= 2047) return ldexp((double)v, e);
  const int hi = (int)((u & 0x7fffffffu) >> 3) + (896 + e) * (1 << 20);
  return __hiloint2double(hi | (int)(u & 0x80000000u), (int)(u << 29));
}

// v 2^-e as FP32 for FP64 v, truncating the significand, with integer
// operations; zero below the FP32 normal range.
__device__ __forceinline__ float narrow(double v, int e) {
  const int hi = __double2hiint(v);
  const unsigned lo = (unsigned)__double2loint(v);
  const int be = (hi >> 20) & 0x7ff;
  const int fe = be - 896 - e;  // biased FP32 exponent
  if (be == 0x7ff || fe >= 255) return (float)ldexp(v, -e);
  if (be == 0 || fe <= 0) return 0.0f;
  const unsigned bits = ((unsigned)hi & 0x80000000u) | ((unsigned)fe << 23) | (((unsigned)hi & 0xfffffu) << 3) |
                        (lo >> 29);
  return __uint_as_float(bits);
}

// Exponent ea of the adjoint inputs (their largest magnitude is below 2^ea).
__device__ __forceinline__ int adjoint_exponent(unsigned long long bits) {
  const int be = (int)((bits >> 52) & 0x7ffull);
  return be == 0 ? 0 : be - 1022;
}

// The adjoint image interpolated at x like a deposit, and its gradient in x
// (units 2^ea).
__device__ __forceinline__ float adj_weight(const AdjParams& A, int q, int lam, bool scattered, float3 x,
                                            float3& dW) {
  const DevInstr& I = tr::S_INSTR[q];
  dW = make_float3(0.0f, 0.0f, 0.0f);
  const float* img = A.adj_img[q];
  if (!img) return 0.0f;
  const size_t plane = (size_t)I.ny * I.nx;
  const float* a0 = img + (size_t)lam * plane;
  const float* a1 = I.channels == 3 ? img + ((size_t)(scattered ? 2 : 1) * A.f.n_lambda + lam) * plane : nullptr;
  const float fx = (x.x * I.ex[0] + x.y * I.ex[1] + x.z * I.ex[2] + I.off_x) * I.sx;
  const float fy = (x.x * I.ey[0] + x.y * I.ey[1] + x.z * I.ey[2] + I.off_y) * I.sy;
  if (I.sed) return a0[0] + (a1 ? a1[0] : 0.0f);  // one bin, independent of x
  auto at = [&](float fix, float fiy) -> float {
    if (!(fix >= 0.0f && fiy >= 0.0f && fix < (float)I.nx && fiy < (float)I.ny)) return 0.0f;
    const size_t pix = (size_t)(int)fiy * I.nx + (int)fix;
    return a0[pix] + (a1 ? a1[pix] : 0.0f);
  };
  if (!I.bilinear) return at(floorf(fx), floorf(fy));  // piecewise constant in x
  const float gx = fx - 0.5f, gy = fy - 0.5f;
  const float x0 = floorf(gx), y0 = floorf(gy);
  const float tx = gx - x0, ty = gy - y0;
  const float a00 = at(x0, y0), a10 = at(x0 + 1, y0), a01 = at(x0, y0 + 1), a11 = at(x0 + 1, y0 + 1);
  const float W = a00 * (1 - tx) * (1 - ty) + a10 * tx * (1 - ty) + a01 * (1 - tx) * ty + a11 * tx * ty;
  const float dWdfx = ((a10 - a00) * (1 - ty) + (a11 - a01) * ty) * I.sx;
  const float dWdfy = ((a01 - a00) * (1 - tx) + (a11 - a10) * tx) * I.sy;
  dW.x = dWdfx * I.ex[0] + dWdfy * I.ey[0];
  dW.y = dWdfx * I.ex[1] + dWdfy * I.ey[1];
  dW.z = dWdfx * I.ex[2] + dWdfy * I.ey[2];
  return W;
}

// Ask for walk `phase` from the lane's position along d; walks start in the
// last stage of a control round, from one place in the code.
__device__ __forceinline__ void request_walk(ALane& s, int phase, float3 d) {
  s.wphase = phase;
  s.d = d;
  s.phase = aStart;
}

__device__ __forceinline__ void start_walk(const FwdParams& P, ALane& s) {
  s.phase = s.wphase;
  s.id = make_float3(tr::inv_or_zero(s.d.x), tr::inv_or_zero(s.d.y), tr::inv_or_zero(s.d.z));
  s.th = s.tl = 0.0f;
  s.g = make_float3(0.0f, 0.0f, 0.0f);
  s.axis_in = -1;
  s.n_cross = 0;
  CartGrid::Scratch sc;
  s.walking = CartGrid::init(P, s.x, s.d, s.id, s.has_cell, s.cell, s.w, sc);
  if (s.walking) s.rho = tr::load_density(&P.density[s.w.cell]);
}

__device__ __forceinline__ int linear_cell(const FwdParams& P, const CartGrid::Cell& c) {
  return c.ix + P.nx * (c.iy + P.ny * c.iz);
}

template <bool kAbs>
__device__ __forceinline__ void request_path(ALane& s) {
  request_walk(s, aPath1, s.k);
  if (kAbs) {
    s.P = s.D = s.a_prev = 0.0;
    s.e_prev = 1.0;
    s.g0 = make_double3(0.0, 0.0, 0.0);
  }
}

// ---- the stages of a control round (each for the lanes in that phase)

// Tape: the lane's position, cell and weight at event s.event (records
// event+1 for events before the last, record 0 for the last), and the
// direction of travel into it (that of path s.event, for the phase function).
__device__ __forceinline__ void tape_event(const AdjParams& A, ALane& s) {
  const AdjRecord& r = s.rec[s.event < s.J ? s.event + 1 : 0];
  s.x = make_float3(r.x[0], r.x[1], r.x[2]);
  s.Lf = r.L;
  s.has_cell = r.cell >= 0;
  if (s.has_cell) {
    const FwdParams& P = A.f;
    s.cell.ix = r.cell % P.nx;
    s.cell.iy = (r.cell / P.nx) % P.ny;
    s.cell.iz = r.cell / (P.nx * P.ny);
  }
  if (s.event > 0) {
    AdjRecord& pj = s.rec[s.event];
    s.k = make_float3(pj.k[0], pj.k[1], pj.k[2]);
    pj.dLb = 0.0f;  // the peel-offs at this event accumulate here
    pj.dxb[0] = pj.dxb[1] = pj.dxb[2] = 0.0f;
  }
}

template <bool kTape>
__device__ __forceinline__ void fetch(const AdjParams& A, ALane& s, unsigned long long w) {
  const FwdParams& P = A.f;
  if (w >= P.n_total) { s.phase = aExit; return; }
  int lam = min((int)(__ull2float_rz(w) * P.inv_n_per_lambda), P.n_lambda - 1);
  while (lam > 0 && (unsigned long long)lam * P.n_per_lambda > w) --lam;
  while (lam + 1 < P.n_lambda && (unsigned long long)(lam + 1) * P.n_per_lambda <= w) ++lam;
  s.lam = lam;
  s.pid = P.first_id + (w - (unsigned long long)lam * P.n_per_lambda);
  s.kappa = tr::S_LAM[lam].kappa;
  s.L = P.L0[lam];
  s.eL = A.e0[lam];
  s.eLA = s.eL + adjoint_exponent(*A.maxbits);
  s.event = 0;
  s.J = 0;
  s.has_cell = false;
  s.q = 0;
  s.phase = aPeelScan;
  if constexpr (kTape) {
    // the forward launch recorded this packet's events: no replay
    s.rec = A.tape + (size_t)w * (size_t)A.rec_stride;
    s.J = s.rec[0].h;
    tape_event(A, s);
  } else {
    tr::emit(P, s.pid, s.lam, s.x, s.k);
  }
}

// Path 1 ended: escape, or the inversion (the forward kernel's FP64 steps)
// and the record of the path; then the second walk.
template <bool kAbs>
__device__ __forceinline__ void finish_path1(const AdjParams& A, ALane& s) {
  const FwdParams& P = A.f;
  const double tau = tr::widen(s.th) + tr::widen(s.tl);
  if (!(tau > 0.0)) {  // escapes: there is no event s.event
    s.J = s.event - 1;
    s.phase = aSweep;
    return;
  }
  const double albedo = tr::S_LAM[s.lam].albedo;
  const double omE = -expm1(-tau);
  const uint4 rn = draw_block(s.pid, s.lam, s.event, 0, P.seed, P.model);
  const double u = u01(rn.x);
  const double tau_star = -log1p(-u * omE);
  s.u_mu = tr::u01f(rn.y);
  s.u_phi = tr::u01f(rn.z);
  AdjRecord& r = s.rec[s.event];
  r.x[0] = s.x.x; r.x[1] = s.x.y; r.x[2] = s.x.z;
  r.k[0] = s.k.x; r.k[1] = s.k.y; r.k[2] = s.k.z;
  r.cell = s.has_cell ? linear_cell(P, s.cell) : -1;
  r.L = narrow(s.L, s.eL);
  r.omE = (float)omE;
  r.E = (float)(1.0 - omE);
  r.u = tr::u01f(rn.x);
  r.g1[0] = s.g.x; r.g1[1] = s.g.y; r.g1[2] = s.g.z;
  if (kAbs) {
    const double wd = (1.0 - albedo) * s.L;
    const int ea = s.eLA - s.eL;
    r.Tdep = narrow(s.P + wd * s.e_prev * s.a_prev, s.eLA);  // the last index: a_n = 0
    r.D = narrow(s.D, ea);
    r.g0[0] = narrow(s.g0.x, s.eLA); r.g0[1] = narrow(s.g0.y, s.eLA); r.g0[2] = narrow(s.g0.z, s.eLA);
  }
  s.L = albedo * s.L * omE;  // weight after the scattering
  tr::split_pair(tau_star, s.a0, s.a1);  // as the forward kernel
  s.h = -1;
  request_walk(s, aPath2, s.k);
}

// Path 2 ended at the interaction: record it, move the packet, then the
// scattering peel-offs.
__device__ __forceinline__ void finish_path2(const AdjParams& A, ALane& s) {
  const FwdParams& P = A.f;
  if (s.h < 0) {  // not reachable: identical pair sums in both walks and tau* < tau_path
    atomicOr(P.flags, kFlagNoInteraction);
    s.J = s.event - 1;
    s.phase = aSweep;
    return;
  }
  AdjRecord& r = s.rec[s.event];
  r.h = s.h;
  r.hit_axis = s.axis_in;
  r.hit_cell = s.w.cell;
  r.kr_h = s.kr_h;
  r.rem = s.a1;
  // segments h.. with the entry of h counted: all segments minus those before h
  r.gp[0] = s.g.x; r.gp[1] = s.g.y; r.gp[2] = s.g.z;
  r.dLb = 0.0f;
  r.dxb[0] = r.dxb[1] = r.dxb[2] = 0.0f;
  const float s_star = s.a0;
  float3 x = make_float3(fmaf(s_star, s.k.x, s.x.x), fmaf(s_star, s.k.y, s.x.y), fmaf(s_star, s.k.z, s.x.z));
  s.cell = CartGrid::carried(s.w);
  CartGrid::clamp(P, s.cell, x);
  s.x = x;
  s.has_cell = true;
  s.q = 0;
  s.phase = aPeelScan;
}

// A peel-off's value l = L phase e^{-tau} W / (4 pi) once its optical depth
// (and d tau / d x_a = -g_a / d_a) is known, and the event's share of (Lb,
// xb); returns l (units 2^eLA).
__device__ __forceinline__ float peel_values(const AdjParams& A, ALane& s, const DevInstr& I, float W, float3 dW) {
  float phase = 1.0f;
  if (s.event > 0) phase = hg_phase(tr::S_LAM[s.lam].g, s.k.x * I.kobs[0] + s.k.y * I.kobs[1] + s.k.z * I.kobs[2]);
  const float pe = kInv4PiF * phase * expf(-s.th) * (1.0f - s.tl);
  const float V = (A.tape ? s.Lf : narrow(s.L, s.eL)) * pe;  // units 2^eL
  const float l = V * W;                   // units 2^eLA
  if (s.event > 0) {
    AdjRecord& r = s.rec[s.event];
    r.dLb += pe * W;
    r.dxb[0] += V * dW.x + l * s.g.x * s.id.x;
    r.dxb[1] += V * dW.y + l * s.g.y * s.id.y;
    r.dxb[2] += V * dW.z + l * s.g.z * s.id.z;
  }
  return l;
}

// A peel-off measuring walk ended: its values, then the depositing walk or
// the next peel-off.
__device__ __forceinline__ void finish_peel_measure(const AdjParams& A, ALane& s) {
  const DevInstr& I = tr::S_INSTR[s.q];
  float3 dW;
  const float W = adj_weight(A, s.q, s.lam, s.event > 0, s.x, dW);
  const float l = peel_values(A, s, I, W, dW);
  if (l != 0.0f && s.n_cross > 0) {
    s.c0 = s.c1 = -l * s.kappa;
    s.h = INT_MAX;
    request_walk(s, aPeelD, s.d);
    return;
  }
  s.q += 1;
  s.phase = aPeelScan;
}

// A peel-off along a frame that looks exactly along a grid axis, without
// walks: the forward kernel's column sums give tau = kappa (rho_c ds_0 +
// column[c]); the only plane the ray's optical depth depends on is the exit
// face of the first cell, g_axis = kappa rho_c; the deposit -l kappa ds goes
// to cell c directly and, for the cells beyond it, into the line's
// difference array.  False when the position is outside the grid.
__device__ __forceinline__ bool column_peel(const AdjParams& A, ALane& s, const DevInstr& I, float W, float3 dW,
                                            unsigned& n_cross, unsigned& n_dep) {
  const FwdParams& P = A.f;
  CartGrid::Cell c;
  if (s.has_cell) {
    c = s.cell;
  } else {
    if (!inside_box(P, s.x)) return false;
    c.ix = min(max(__float2int_rd((s.x.x - P.lo[0]) * P.inv_d[0]), 0), P.nx - 1);
    c.iy = min(max(__float2int_rd((s.x.y - P.lo[1]) * P.inv_d[1]), 0), P.ny - 1);
    c.iz = min(max(__float2int_rd((s.x.z - P.lo[2]) * P.inv_d[2]), 0), P.nz - 1);
  }
  const int a = I.axis;
  const bool up = I.dir > 0;
  const int i = a == 0 ? c.ix : (a == 1 ? c.iy : c.iz);
  const int n = a == 0 ? P.nx : (a == 1 ? P.ny : P.nz);
  const float xa = a == 0 ? s.x.x : (a == 1 ? s.x.y : s.x.z);
  const float plane = fmaf((float)(i + (up ? 1 : 0)), P.d[a], P.lo[a]);
  const float ds0 = fmaxf(up ? plane - xa : xa - plane, 0.0f);
  const int cell = c.ix + P.nx * (c.iy + P.ny * c.iz);
  const float rho = tr::load_density(&P.density[cell]);
  s.th = s.kappa * fmaf(rho, ds0, __ldg(&I.column[cell]));
  s.tl = 0.0f;
  const float kr0 = s.kappa * rho;
  const float sgn = up ? 1.0f : -1.0f;
  s.g = make_float3(a == 0 ? kr0 : 0.0f, a == 1 ? kr0 : 0.0f, a == 2 ? kr0 : 0.0f);
  s.id = make_float3(a == 0 ? sgn : 0.0f, a == 1 ? sgn : 0.0f, a == 2 ? sgn : 0.0f);
  const unsigned cells = (unsigned)(up ? n - i : i + 1);
  n_cross += 2u * cells;  // the measuring and the depositing walk it stands for
  const float l = peel_values(A, s, I, W, dW);
  if (l != 0.0f) {
    const float coef = -l * s.kappa;
    grad_add(&A.grad[cell], scaled(coef * ds0, s.eLA));
    if (cells > 1u) grad_add(&A.line_dep[2 * a + (up ? 1 : 0)][cell], scaled(coef * P.d[a], s.eLA));
    n_dep += cells;
  }
  return true;
}

// The next instrument from s.q whose adjoint weight at the lane's position
// is not zero: its peel-off walk (frames along grid axes are done here
// without walks); after the last one, aAfter.
__device__ __forceinline__ void peel_scan(const AdjParams& A, ALane& s, unsigned& n_cross, unsigned& n_dep) {
  const FwdParams& P = A.f;
  const bool on = s.event == 0 ? P.peel_emission : P.peel_scatter;
  for (; on && s.q < P.n_instr; ++s.q) {
    float3 dW;
    const float W = adj_weight(A, s.q, s.lam, s.event > 0, s.x, dW);
    if (W == 0.0f && dW.x == 0.0f && dW.y == 0.0f && dW.z == 0.0f) continue;  // contributes nothing
    const DevInstr& I = tr::S_INSTR[s.q];
    if (P.use_columns && I.column && column_peel(A, s, I, W, dW, n_cross, n_dep)) continue;
    request_walk(s, aPeelM, tr::instr_dir(I));
    return;
  }
  s.phase = aAfter;
}

// After the peel-offs of event s.event: the first forced path, or the new
// direction and then termination (the sweep) or the next forced path.
template <bool kAbs, bool kTape>
__device__ __forceinline__ void after_peels(const AdjParams& A, ALane& s) {
  const FwdParams& P = A.f;
  if constexpr (kTape) {  // the next recorded event, or the sweep
    if (s.event < s.J) {
      s.event += 1;
      s.q = 0;
      tape_event(A, s);
      s.phase = aPeelScan;
    } else {
      s.phase = aSweep;
    }
    return;
  }
  if (s.event == 0) {
    s.event = 1;
    request_path<kAbs>(s);
    return;
  }
  const float mu = hg_sample(tr::S_LAM[s.lam].g, s.u_mu);
  float sp, cp;
  sincospif(2.0f * s.u_phi, &sp, &cp);
  s.k = rotate_dir(s.k, mu, sp, cp);
  if ((P.weight_cut && s.L < P.L_cut[s.lam]) || s.event >= P.max_events) {
    s.J = s.event;
    s.phase = aSweep;
    return;
  }
  s.event += 1;
  request_path<kAbs>(s);
}

// Backward sweep over the packet's events J..1 (no walks): per forced path
// the total T of its optical-depth adjoints and the adjoint of tau_{h-1} for
// the depositing walk, the interaction-cell term of the gradient, and the
// adjoints of the path's start weight and position.
template <bool kAbs>
__device__ __forceinline__ void sweep(const AdjParams& A, ALane& s) {
  const float albedo = (float)tr::S_LAM[s.lam].albedo;
  float Lb = 0.0f, xb0 = 0.0f, xb1 = 0.0f, xb2 = 0.0f;
  for (int j = s.J; j >= 1; --j) {
    AdjRecord& r = s.rec[j];
    Lb += r.dLb;
    xb0 += r.dxb[0]; xb1 += r.dxb[1]; xb2 += r.dxb[2];
    const float k0 = r.k[0], k1 = r.k[1], k2 = r.k[2];
    // x_j = x_{j-1} + s* k with s* = t_in(h) + (tau* - tau_{h-1}) / kr_h
    const float sb = xb0 * k0 + xb1 * k1 + xb2 * k2;
    const float krh = r.kr_h;
    const float tsb = sb / krh;  // adjoint of tau*
    grad_add(&A.grad[r.hit_cell], scaled(-tsb * r.rem * s.kappa / krh, s.eLA));
    float tbh = 0.0f;
    if (r.hit_axis >= 0) {  // t_in(h): the plane entering h, d t / d x_a = -1 / k_a
      tbh = -tsb;
      if (r.hit_axis == 0) xb0 -= sb / k0;
      else if (r.hit_axis == 1) xb1 -= sb / k1;
      else xb2 -= sb / k2;
    }
    // L_j = albedo L (1 - E), tau* = -ln(1 - u (1 - E)), E = exp(-tau_path)
    const float Eb = -Lb * albedo * r.L - tsb * r.u / (1.0f - r.u * r.omE);
    // deposit adjoints (with an absorption adjoint only)
    const float Tdep = kAbs ? r.Tdep : 0.0f, Dd = kAbs ? r.D : 0.0f;
    const float g00 = kAbs ? r.g0[0] : 0.0f, g01 = kAbs ? r.g0[1] : 0.0f, g02 = kAbs ? r.g0[2] : 0.0f;
    const float T = Tdep + tbh - r.E * Eb;
    // the planes of the path move with x: d ds_m / d x through their parameters
    // (segments from h on: all minus those before h)
    if (k0 != 0.0f) xb0 -= (T * r.g1[0] - g00 - tbh * (r.g1[0] - r.gp[0])) / k0;
    if (k1 != 0.0f) xb1 -= (T * r.g1[1] - g01 - tbh * (r.g1[1] - r.gp[1])) / k1;
    if (k2 != 0.0f) xb2 -= (T * r.g1[2] - g02 - tbh * (r.g1[2] - r.gp[2])) / k2;
    Lb = Lb * albedo * r.omE + (1.0f - albedo) * Dd;
    r.T = T;
    r.tbh = tbh;
  }
  s.event = 1;
  s.phase = aDepScan;
}

// The depositing walk of forced path s.event or of a later one; after the
// last, the lane needs a new packet.
__device__ __forceinline__ void dep_scan(const AdjParams& A, ALane& s) {
  const FwdParams& P = A.f;
  for (; s.event <= s.J; ++s.event) {
    const AdjRecord& r = s.rec[s.event];
    s.c0 = s.kappa * r.T;
    s.c1 = s.kappa * (r.T - r.tbh);
    if (s.c0 == 0.0f && s.c1 == 0.0f) continue;
    s.h = r.h;
    s.x = make_float3(r.x[0], r.x[1], r.x[2]);
    s.has_cell = r.cell >= 0;
    if (s.has_cell) {
      s.cell.ix = r.cell % P.nx;
      s.cell.iy = (r.cell / P.nx) % P.ny;
      s.cell.iz = r.cell / (P.nx * P.ny);
    }
    request_walk(s, aDep, make_float3(r.k[0], r.k[1], r.k[2]));
    return;
  }
  s.phase = aFetch;
}

// One cell crossing of the lane's current walk.
template <bool kAbs>
__device__ __forceinline__ void step(const AdjParams& A, ALane& s, unsigned& n_cross, unsigned& n_dep) {
  const FwdParams& P = A.f;
  CartGrid::Walk& w = s.w;
  int axis;
  const float te = CartGrid::exit(w, s.x, s.id, axis);
  const float texit = fmaxf(te, w.t);
  const float ds = texit - w.t;
  const float kr = s.kappa * s.rho;
  const float dt = kr * ds;
  float nh, e;
  tr::two_sum(s.th, dt, nh, e);
  const float nl = s.tl + e;
  ++n_cross;
  if (s.phase == aPath2 && (nh - s.a0) + (nl - s.a1) > 0.0f) {
    // the interaction is in this segment (the forward kernel's test and remainder)
    const float rem = ((s.a0 - s.th) + s.a1) - s.tl;
    s.a0 = w.t + rem / kr;
    s.a1 = rem;
    s.kr_h = kr;
    s.h = s.n_cross;
    s.walking = false;
    return;
  }
  // plane sums: +kr at the exit plane, -kr at the entry plane
  s.g.x += (axis == 0 ? kr : 0.0f) - (s.axis_in == 0 ? kr : 0.0f);
  s.g.y += (axis == 1 ? kr : 0.0f) - (s.axis_in == 1 ? kr : 0.0f);
  s.g.z += (axis == 2 ? kr : 0.0f) - (s.axis_in == 2 ? kr : 0.0f);
  const int cell = w.cell;
  if (s.phase == aPeelD || s.phase == aDep) {
    grad_add(&A.grad[cell], scaled((s.n_cross >= s.h ? s.c1 : s.c0) * ds, s.eLA));
    ++n_dep;
  }
  if (kAbs && s.phase == aPath1) {
    // deposits (1 - albedo) L (e_{m-1} - e_m) with adjoints a_m: P is the
    // prefix of the optical-depth adjoints wd e_i (a_i - a_{i+1}), i < m
    const double a = dt > 0.0f ? A.adj_abs[(size_t)s.lam * P.n_cells + cell] : 0.0;
    const double e_cur = (double)(expf(-nh) * (1.0f - nl));
    const double wd = (1.0 - tr::S_LAM[s.lam].albedo) * s.L;
    if (s.n_cross > 0) s.P += wd * s.e_prev * (s.a_prev - a);
    if (s.P != 0.0) grad_add(&A.grad[cell], -(double)(s.kappa * ds) * s.P);
    const double c = (double)kr * s.P;
    s.g0.x += (axis == 0 ? c : 0.0) - (s.axis_in == 0 ? c : 0.0);
    s.g0.y += (axis == 1 ? c : 0.0) - (s.axis_in == 1 ? c : 0.0);
    s.g0.z += (axis == 2 ? c : 0.0) - (s.axis_in == 2 ? c : 0.0);
    s.D += a * (s.e_prev - e_cur);
    s.e_prev = e_cur;
    s.a_prev = a;
  }
  s.th = nh;
  s.tl = nl;
  s.axis_in = axis;
  ++s.n_cross;
  w.t = texit;
  CartGrid::Scratch sc;
  if (CartGrid::advance(P, s.x, s.d, s.id, axis, w, sc)) {
    s.rho = tr::load_density(&P.density[w.cell]);
  } else {
    s.walking = false;
  }
}

template <bool kAbs, bool kTape>
__global__ void __launch_bounds__(kAdjBlock, RT_ADJ_MIN_BLOCKS) k_adjoint(const AdjParams A) {
  const FwdParams& P = A.f;
  for (int i = threadIdx.x; i < P.n_instr; i += kAdjBlock) tr::S_INSTR[i] = P.instr[i];
  for (int i = threadIdx.x; i < P.n_lambda; i += kAdjBlock) tr::S_LAM[i] = P.lam[i];
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  ALane s;
  s.phase = aFetch;
  s.walking = false;
  s.rec = A.recs + ((size_t)blockIdx.x * kAdjBlock + threadIdx.x) * (size_t)A.rec_stride;
  unsigned n_cross = 0, n_dep = 0;
  unsigned long long tot_cross = 0, tot_dep = 0;
  while (true) {
    const bool idle = !s.walking && s.phase != aExit;
    const unsigned need = __ballot_sync(0xffffffffu, idle);
    const unsigned walkers = __ballot_sync(0xffffffffu, s.walking);
    if (need == 0u && walkers == 0u) break;
    if (walkers == 0u || __popc(need) >= P.control_min) {
      // per-event work in stages, each run by the lanes in its phase together;
      // a stage only hands lanes on to later stages
      if (!s.walking) {
        if constexpr (!kTape) {
          if (s.phase == aPath1) finish_path1<kAbs>(A, s);
          if (s.phase == aPath2) finish_path2(A, s);
        }
        if (s.phase == aPeelM) finish_peel_measure(A, s);
        if (s.phase == aPeelD) { s.q += 1; s.phase = aPeelScan; }
        if (s.phase == aDep) { s.event += 1; s.phase = aDepScan; }
      }
      // new packets, their peel-offs, scatterings, sweeps and deposit scans,
      // repeated while a lane has just finished its packet (at most two passes)
      while (true) {
        const bool wants = !s.walking && s.phase == aFetch;
        const unsigned fetchers = __ballot_sync(0xffffffffu, wants);
        if (fetchers) {
          unsigned long long base = 0;
          const int leader = __ffs(fetchers) - 1;
          if ((int)lane == leader) base = atomicAdd(P.work_counter, (unsigned long long)__popc(fetchers));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (wants) fetch<kTape>(A, s, base + __popc(fetchers & lt_mask));
        }
        if (s.phase == aPeelScan) peel_scan(A, s, n_cross, n_dep);
        if (s.phase == aAfter) after_peels<kAbs, kTape>(A, s);
        if (s.phase == aSweep) {
          if (s.J >= 1) sweep<kAbs>(A, s); else s.phase = aFetch;
        }
        if (s.phase == aDepScan) dep_scan(A, s);
        // a fetched lane never returns to aFetch within the round
        if (!__any_sync(0xffffffffu, !s.walking && s.phase == aFetch)) break;
      }
      if (s.phase == aStart) start_walk(P, s);
      if ((n_cross | n_dep) & 0xC0000000u) {  // keep the 32-bit lane counters far from overflow
        tot_cross += n_cross;
        tot_dep += n_dep;
        n_cross = n_dep = 0;
      }
    }
    if (s.walking) step<kAbs>(A, s, n_cross, n_dep);
  }
  if (A.counters) {
    tot_cross += n_cross;
    tot_dep += n_dep;
    for (int o = 16; o > 0; o >>= 1) {
      tot_cross += __shfl_down_sync(0xffffffffu, tot_cross, o);
      tot_dep += __shfl_down_sync(0xffffffffu, tot_dep, o);
    }
    if (lane == 0) {
      atomicAdd(&A.counters[0], tot_cross);
      atomicAdd(&A.counters[1], tot_dep);
    }
  }
}

// Largest magnitude of an FP64 array (as FP64 bits: non-negative doubles
// order like their bit patterns).
__global__ void k_absmax(const double* a, size_t n, unsigned long long* out) {
  unsigned long long m = 0ull;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a[i]) & 0x7fffffffffffffffull;
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31u) == 0u && m) atomicMax(out, m);
}

// The per-line deposit differences into the gradient: along each grid line,
// in the ray's direction, every cell receives the sum of the entries of the
// cells before it.
__global__ void k_line_scatter(const double* __restrict__ dep, double* __restrict__ grad, int nx, int ny, int nz,
                               int axis, int dir) {
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
    double run = 0.0;
    for (int k = 0; k < n; ++k) {
      const int j = dir > 0 ? k : n - 1 - k;
      const long long c = base + (long long)j * stride;
      if (run != 0.0) grad[c] += run;
      run += dep[c];
    }
  }
}

// FP32 copy of an adjoint image in units 2^ea.
__global__ void k_to_units(const double* a, size_t n, const unsigned long long* maxbits, float* out) {
  const int ea = adjoint_exponent(*maxbits);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)ldexp(a[i], -ea);
}

}  // namespace

cudaError_t adjoint_lanes(int num_sms, unsigned long long n_total, unsigned long long* lanes) {
  int per_sm = 0, per_sm_abs = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint<false, false>, kAdjBlock, 0);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_abs, k_adjoint<true, false>, kAdjBlock, 0);
  if (e != cudaSuccess) return e;
  per_sm = per_sm_abs > per_sm ? per_sm_abs : per_sm;
  per_sm = per_sm < 1 ? 1 : per_sm;
  unsigned long long blocks = (unsigned long long)num_sms * per_sm;
  const unsigned long long useful = (n_total + kAdjBlock - 1) / kAdjBlock;
  if (blocks > useful) blocks = useful;
  if (blocks < 1) blocks = 1;
  *lanes = blocks * kAdjBlock;
  return cudaSuccess;
}

cudaError_t launch_adjoint(const FwdParams& f, const double* const* adj_img, const size_t* img_elems,
                           const double* adj_abs, double* grad, AdjRecord* recs, unsigned long long lanes,
                           unsigned long long* counters, float* img_f, unsigned long long* maxbits,
                           double* const* line_dep, AdjRecord* tape, cudaStream_t stream) {
  AdjParams a;
  a.f = f;
  a.tape = adj_abs ? nullptr : tape;  // the tape holds no absorption-adjoint quantities
  for (int k = 0; k < 6; ++k) {
    a.line_dep[k] = f.use_columns ? line_dep[k] : nullptr;
    if (a.line_dep[k]) {
      cudaError_t e = cudaMemsetAsync(a.line_dep[k], 0, (size_t)f.n_cells * sizeof(double), stream);
      if (e != cudaSuccess) return e;
    }
  }
  a.adj_abs = adj_abs;
  a.maxbits = maxbits;
  a.grad = grad;
  a.recs = recs;
  a.rec_stride = f.max_events + 1;
  a.counters = counters;
  for (int l = 0; l < kMaxLambda; ++l) {
    int e0 = 0;
    if (l < f.n_lambda && f.L0[l] > 0.0) std::frexp(f.L0[l], &e0);
    a.e0[l] = e0;
  }
  cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const int rb = 256, rg = 304;
  for (int q = 0; q < f.n_instr; ++q)
    if (adj_img[q]) k_absmax<<<rg, rb, 0, stream>>>(adj_img[q], img_elems[q], maxbits);
  if (adj_abs) k_absmax<<<rg, rb, 0, stream>>>(adj_abs, (size_t)f.n_lambda * (size_t)f.n_cells, maxbits);
  size_t off = 0;
  for (int q = 0; q < kMaxInstruments; ++q) {
    a.adj_img[q] = nullptr;
    if (q < f.n_instr && adj_img[q]) {
      k_to_units<<<rg, rb, 0, stream>>>(adj_img[q], img_elems[q], maxbits, img_f + off);
      a.adj_img[q] = img_f + off;
      off += img_elems[q];
    }
  }
  e = cudaMemsetAsync(f.work_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(lanes / kAdjBlock);
  if (adj_abs) {
    k_adjoint<true, false><<<blocks, kAdjBlock, 0, stream>>>(a);
  } else if (a.tape) {
    k_adjoint<false, true><<<blocks, kAdjBlock, 0, stream>>>(a);
  } else {
    k_adjoint<false, false><<<blocks, kAdjBlock, 0, stream>>>(a);
  }
  e = cudaGetLastError();
  for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
    if (!a.line_dep[k]) continue;
    const int axis = k / 2;
    const long long n_lines = (long long)f.n_cells / (axis == 0 ? f.nx : (axis == 1 ? f.ny : f.nz));
    const long long nb = std::min<long long>((n_lines + 255) / 256, 65535);
    k_line_scatter<<<(unsigned)nb, 256, 0, stream>>>(a.line_dep[k], grad, f.nx, f.ny, f.nz, axis, (k & 1) ? 1 : -1);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace rtk

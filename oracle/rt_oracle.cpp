// FP64 CPU oracle for photon-packet Monte Carlo dust radiative transfer.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against
// which the CUDA transport library is checked.  Only the test-suite, the
// smoke check and the benchmark's CPU-baseline leg may build or call it; the
// product path never does.  It shares no code, header, table or helper with the
// CUDA library.
//
// What it computes (Camps & Baes, "SKIRT: an advanced dust radiative transfer
// code with a user-friendly architecture"):
//   * Sect. 1: photon packages are emitted, undergo scattering events drawn
//     from probability distributions, and are absorbed or escape; the
//     optimisations used are peel-off at emission and scattering, continuous
//     absorption and forced scattering.
//   * Sect. 2.2: dust cells carry constant density and optical properties;
//     packages propagate through the grid; frame instruments use parallel
//     projection with inclination, azimuth and position angle and record the
//     flux per pixel per wavelength, optionally split into direct and
//     scattered radiation.
//   * Sect. 2.3: per wavelength an extinction coefficient, an albedo
//     (scattering / extinction) and an asymmetry parameter g that fixes the
//     phase function (taken as Henyey-Greenstein).
//   * Sect. 2.4 and Table 1(d): cartesian grids, rectilinear grids (PowCub:
//     cell edges spaced by a power law), octrees (recursive 2x2x2
//     subdivision), k-d trees (BinTree: halving along one axis per node) and
//     Voronoi grids (each cell the part of the domain nearest to its
//     generating site, walked across the bisecting planes of its neighbours).
//   * Sect. 3.4: a source geometry draws random emission positions from its
//     density (point, double-exponential disk, Plummer sphere; Table 1(a)).
// The paper does not spell out the transport algorithm (it says so in
// Sect. 1); the per-packet steps below follow the standard formulations of the
// methods it cites.  Every place where the paper is silent has one stated
// reading, listed in the design notes of the repository.
//
// Per packet (packet id p, wavelength index l):
//   1. L0 = L_tot(l) / N_norm.  Event-0 random numbers choose the source
//      component (proportional to its luminosity at l), the position, and an
//      isotropic direction.
//   2. Emission peel-off: per instrument, add L0/(4 pi) * exp(-tau(x -> obs))
//      to the pixel that x projects onto (direct channel).
//   3. For j = 1, 2, ...:
//      a. walk the grid from x along k to the boundary: cells c_i, segment
//         lengths ds_i, cumulative optical depths tau_i; if tau_path = 0 the
//         packet escapes with all of L;
//      b. E = exp(-tau_path); escaped += L E; continuous absorption: cell c_i
//         receives (1 - albedo) L (exp(-tau_{i-1}) - exp(-tau_i));
//      c. forced scattering: tau* = -ln(1 - u (1 - E)); the interaction lies
//         in the first cell with tau_i > tau*, at path length
//         s_{i-1} + (tau* - tau_{i-1}) / (kappa rho_i);
//      d. L <- albedo L (1 - E); scattering peel-off: per instrument add
//         L Phi(k . k_obs)/(4 pi) exp(-tau(x -> obs)) (scattered channel);
//      e. new direction from the Henyey-Greenstein distribution;
//      f. stop when L < w_min L0 (if the weight cut is on) or j = max_events;
//         the remaining L is tallied as "truncated".
//   Conservation: L0 = escaped + absorbed + truncated exactly (telescoping).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011, "Parallel
// random numbers: as easy as 1, 2, 3"), counter = (p low, p high, event,
// (l << 8) | block), key = (seed, model id), uniform = (r + 0.5) 2^-32.
//
// The whole per-packet algorithm is templated on the scalar type of quantities
// that depend on the dust density, so that running it with dual numbers gives
// the pathwise derivative of every tally with respect to one cell density
// (common random numbers: directions and draws are fixed; positions move with
// the density through the forced-scattering inversion).
//
// Pins (the tests under tests/test_oracle_*.py): Philox against a library
// generator, the phase function and emission distributions, the grid walks
// by brute force, closed-form path lengths and direct images, quadratures of
// the first-step escape, absorption field and single-scattering flux,
// special cases, symmetry, scale invariance, conservation, dual gradients
// against central differences, multiple scattering against an analog
// simulation (escaped and absorbed fractions, intensity towards a frame, the
// frame's inner 2 x 2 blocks of 4 x 4, the absorption field in 4 x 4 x 4
// blocks), and mutations of this file that the pins must catch.  Parity
// unpinned: multiply scattered light below that block resolution, beyond the
// invariants (no closed form exists).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>
#include <mutex>

namespace {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al. 2011, Sect. 3 (Philox): each round multiplies counter words 0
// and 2 by fixed 32-bit constants, swaps the products' halves into a new
// counter and XORs in the round key; the key is bumped by the Weyl constants
// between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)kPhiloxM0 * c[0];
    uint64_t p1 = (uint64_t)kPhiloxM1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Uniform in the open interval (0, 1): exact in FP64.
double uniform_from_bits(uint32_t r) { return ((double)r + 0.5) * 0x1p-32; }

// Four uniforms for (packet, wavelength, event, block).
void draw4(uint64_t pid, int lam, int event, int block, uint32_t seed, uint32_t model,
           double u[4]) {
  uint32_t ctr[4] = {(uint32_t)(pid & 0xFFFFFFFFu), (uint32_t)(pid >> 32), (uint32_t)event,
                     ((uint32_t)lam << 8) | (uint32_t)block};
  uint32_t key[2] = {seed, model};
  uint32_t r[4];
  philox4x32_10(ctr, key, r);
  for (int i = 0; i < 4; ++i) u[i] = uniform_from_bits(r[i]);
}

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v = 0.0, d = 0.0;
  Dual() = default;
  Dual(double value) : v(value), d(0.0) {}
  Dual(double value, double deriv) : v(value), d(deriv) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual exp(Dual a) { double e = std::exp(a.v); return {e, e * a.d}; }
inline Dual expm1(Dual a) { return {std::expm1(a.v), std::exp(a.v) * a.d}; }
inline Dual log(Dual a) { return {std::log(a.v), a.d / a.v}; }
inline Dual log1p(Dual a) { return {std::log1p(a.v), a.d / (1.0 + a.v)}; }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
using std::exp;
using std::expm1;
using std::log;
using std::log1p;

template <class T> struct V3 { T x, y, z; };
using V3d = V3<double>;
template <class T> T comp(const V3<T>& a, int axis) { return axis == 0 ? a.x : (axis == 1 ? a.y : a.z); }
template <class T> void set_comp(V3<T>& a, int axis, T v) {
  if (axis == 0) a.x = v; else if (axis == 1) a.y = v; else a.z = v;
}

}  // namespace

// ================================================================ public structs
extern "C" {

typedef struct {
  int32_t kind;  // 0 = cartesian, 1 = octree, 2 = rectilinear, 3 = k-d tree, 4 = Voronoi
  int32_t nx, ny, nz;
  double bounds[6];  // xmin, xmax, ymin, ymax, zmin, zmax
  const float* density;  // cartesian, rectilinear [nz][ny][nx] (x fastest); octree: per leaf
  int64_t n_nodes;
  const int32_t* child;  // octree: >= 0 first child index; < 0 leaf -(leaf+1)
  int64_t n_leaves;
  const double* edges[3];  // rectilinear: cell edges per axis, n + 1 each
  const int8_t* split_axis;  // k-d tree: split axis of every node (0, 1, 2)
  const double* sites;       // Voronoi: generating site of every cell [n_leaves][3]
  const int64_t* offsets;    // Voronoi: neighbours of cell c are child[offsets[c] .. offsets[c + 1])
} or_grid;

typedef struct {
  int32_t kind;  // 0 = point, 1 = exponential disk, 2 = Plummer sphere
  int32_t pad;
  double center[3];
  double scale_r;  // disk scale length hR, or Plummer radius a
  double scale_z;  // disk scale height hz
} or_source;

typedef struct {
  double inclination, azimuth, position_angle;  // radians
  int32_t nx, ny;
  double half_x, half_y;      // half-widths of the field of view
  double center_x, center_y;  // field centre in the image plane
  int32_t bilinear;           // 0 = nearest pixel, 1 = bilinear
  int32_t channels;           // 1 = total; 3 = total, direct, scattered
  int32_t sed;                // 1 = SED instrument: one bin per wavelength, no projection
  int32_t pad;
} or_instrument;

typedef struct {
  or_grid grid;
  int32_t n_lambda, n_sources, n_instr, pad;
  const double* kappa;   // extinction per unit density per unit length [n_lambda]
  const double* albedo;  // [n_lambda]
  const double* g;       // HG asymmetry [n_lambda]
  const or_source* sources;
  const double* lum;  // [n_sources][n_lambda]
  const or_instrument* instr;
  const double* dust_lum;  // [n_lambda][n_cells]: thermal emission of the dust cells, emitted instead of the
                           // sources (panchromatic mode), or NULL
} or_problem;

typedef struct {
  uint64_t n_per_lambda;
  uint64_t first_id;
  uint64_t n_norm;  // packets per wavelength used for the weight L_tot / n_norm
  uint32_t seed, model_id;
  double w_min;
  int32_t max_events;
  int32_t weight_cut;  // 1: stop when L < w_min L0; 0: stop only at max_events
  int32_t peel_emission, peel_scatter;
  int32_t n_threads;
  int32_t pad;
} or_opts;

// Per-event state of one traced packet (event 0 = emission).
typedef struct {
  int32_t event, pad;
  int64_t cell;
  double x[3], k[3];
  double L, tau_path, tau_star;
} or_trace_row;

typedef struct {
  uint64_t pid;
  int32_t lam, event, instr, pad;
  int64_t pixel;  // iy * nx + ix, nearest-pixel deposits only
  double value;
} or_record;

typedef struct {
  double** images;          // per instrument [channels][n_lambda][ny][nx]; may be NULL
  int64_t** image_counts;   // optional, same shapes
  double* absorption;       // [n_lambda][n_cells]; may be NULL
  int64_t* absorption_counts;
  double stats[4];          // emitted, escaped, absorbed, truncated
  uint64_t counters[4];     // crossings, scattering events, peel-off traversals, packets
  or_record* records;       // optional nearest-pixel peel-off records
  int64_t records_cap;
  int64_t records_n;
} or_output;

}  // extern "C"

namespace {

// ---------------------------------------------------------------- Neumaier sum
struct NSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// ---------------------------------------------------------------- instruments
// Sect. 2.2: parallel projection onto a frame with inclination theta, azimuth
// phi and position angle omega.  k_obs points from the model to the observer.
struct Frame {
  V3d kobs, ex, ey;
  int nx, ny;
  double half_x, half_y, cx, cy;
  bool bilinear;
  int channels;
  bool sed;
};

// Sines and cosines of the frame angles within 1e-15 of 0 or +-1 are taken
// as exact: the angles of the usual face-on and edge-on frames are multiples
// of pi/2, whose rounded values would otherwise leave components of order
// 1e-17 in directions meant to lie along the axes.
double snap_unit(double v) {
  if (std::fabs(v) < 1e-15) return 0.0;
  if (std::fabs(std::fabs(v) - 1.0) < 1e-15) return v > 0 ? 1.0 : -1.0;
  return v;
}

Frame make_frame(const or_instrument& in) {
  Frame f;
  double st = snap_unit(std::sin(in.inclination)), ct = snap_unit(std::cos(in.inclination));
  double sp = snap_unit(std::sin(in.azimuth)), cp = snap_unit(std::cos(in.azimuth));
  double so = snap_unit(std::sin(in.position_angle)), co = snap_unit(std::cos(in.position_angle));
  f.kobs = {st * cp, st * sp, ct};
  V3d a = {-sp, cp, 0.0};            // image x axis before the position angle
  V3d b = {-ct * cp, -ct * sp, st};  // image y axis before the position angle
  f.ex = {co * a.x - so * b.x, co * a.y - so * b.y, co * a.z - so * b.z};
  f.ey = {so * a.x + co * b.x, so * a.y + co * b.y, so * a.z + co * b.z};
  f.nx = in.nx; f.ny = in.ny;
  f.half_x = in.half_x; f.half_y = in.half_y;
  f.cx = in.center_x; f.cy = in.center_y;
  f.bilinear = in.bilinear != 0;
  f.channels = in.channels;
  f.sed = in.sed != 0;
  return f;
}

// ---------------------------------------------------------------- phase function
// Henyey-Greenstein: normalised so that its mean over the sphere is 1.
double hg_phase(double g, double mu) {
  double den = 1.0 + g * g - 2.0 * g * mu;
  return (1.0 - g * g) / (den * std::sqrt(den));
}

// Inverse of the HG cumulative distribution in mu = cos(scattering angle).
double hg_sample(double g, double u) {
  if (std::fabs(g) < 1e-6) return 2.0 * u - 1.0;
  double f = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
  double mu = (1.0 + g * g - f * f) / (2.0 * g);
  return std::min(1.0, std::max(-1.0, mu));
}

// Direction with cosine mu to k and azimuth phi about k.
V3d rotate_dir(const V3d& k, double mu, double phi) {
  double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  double cph = std::cos(phi), sph = std::sin(phi);
  double s = std::sqrt(k.x * k.x + k.y * k.y);
  V3d n;
  if (s == 0.0) {
    // k along +z or -z: take e1 = x, e2 = +y or -y (right-handed about k)
    n = k.z > 0 ? V3d{st * cph, st * sph, mu} : V3d{st * cph, -st * sph, -mu};
  } else {
    double cx = k.x / s, cy = k.y / s;
    // e1 = (cx kz, cy kz, -s), e2 = (-cy, cx, 0): orthonormal, perpendicular to k
    n.x = mu * k.x + st * (cph * cx * k.z - sph * cy);
    n.y = mu * k.y + st * (cph * cy * k.z + sph * cx);
    n.z = mu * k.z - st * cph * s;
  }
  double len = std::sqrt(n.x * n.x + n.y * n.y + n.z * n.z);
  return {n.x / len, n.y / len, n.z / len};
}

// New direction after a scattering event: HG polar cosine from u1, uniform
// azimuth 2 pi u2 about the incoming direction.
V3d scatter_direction(const V3d& k, double g, double u1, double u2) {
  return rotate_dir(k, hg_sample(g, u1), 2.0 * M_PI * u2);
}

// ---------------------------------------------------------------- grids
// A segment of a straight path: the cell and the entry / exit path lengths.
template <class T> struct Seg {
  int64_t cell;
  T s_in, s_out;
};

struct Box { double lo[3], hi[3]; };

struct Grid {
  int kind;
  double lo[3], hi[3];
  int n[3];
  double d[3];
  const float* density;
  const int32_t* child;
  int64_t n_nodes, n_leaves;
  const int8_t* split_axis = nullptr;  // k-d tree: split axis per node
  const double* sites = nullptr;       // Voronoi: site of every cell
  const int64_t* offsets = nullptr;    // Voronoi: neighbour list of every cell in child
  std::vector<Box> leaf_box;  // trees: box of every leaf
  std::vector<double> edges[3];  // rectilinear: cell edges per axis

  // octree (kind 1) and k-d tree (kind 3): cells are the leaves of a tree
  bool tree() const { return kind == 1 || kind == 3; }
  // Voronoi (kind 4; Table 1(d): VoronoiDustGrid): cell c is the part of the
  // domain closer to site c than to any other site
  bool voronoi() const { return kind == 4; }
  int64_t n_cells() const { return tree() || voronoi() ? n_leaves : (int64_t)n[0] * n[1] * n[2]; }

  // The cell of p in a Voronoi grid: the nearest site, by comparing every
  // site (the lowest index among equally near ones).
  int64_t nearest_site(const double p[3]) const {
    int64_t best = 0;
    double best_d2 = INFINITY;
    for (int64_t c = 0; c < n_leaves; ++c) {
      const double* s = sites + 3 * c;
      const double d2 = (p[0] - s[0]) * (p[0] - s[0]) + (p[1] - s[1]) * (p[1] - s[1]) + (p[2] - s[2]) * (p[2] - s[2]);
      if (d2 < best_d2) { best_d2 = d2; best = c; }
    }
    return best;
  }

  // Plane positions: cartesian lo + i * (hi - lo) / n; rectilinear the
  // given edges (Table 1(d): PowCub grids space them by a power law).
  double plane(int axis, int i) const { return kind == 2 ? edges[axis][(size_t)i] : lo[axis] + i * d[axis]; }

  Box cell_box(int64_t cell) const {
    if (tree()) return leaf_box[(size_t)cell];
    int64_t ix = cell % n[0], iy = (cell / n[0]) % n[1], iz = cell / ((int64_t)n[0] * n[1]);
    int64_t idx[3] = {ix, iy, iz};
    Box b;
    for (int a = 0; a < 3; ++a) { b.lo[a] = plane(a, (int)idx[a]); b.hi[a] = plane(a, (int)idx[a] + 1); }
    return b;
  }

  // Tree point location.  An octree node splits its box at the midpoints of
  // all three axes (eight children, octant bit a set for the upper half of
  // axis a); a k-d tree node (Table 1(d): BinTree) at the midpoint of its
  // split axis (two children, lower then upper).  A point on a splitting
  // plane goes to the child that a ray travelling along k enters there (the
  // upper one if k_a >= 0, the lower one if k_a < 0).
  int64_t tree_locate(const double p[3], const V3d& k, Box* box) const {
    double blo[3] = {lo[0], lo[1], lo[2]}, bhi[3] = {hi[0], hi[1], hi[2]};
    int64_t node = 0;
    while (child[node] >= 0) {
      if (kind == 3) {
        const int a = split_axis[node];
        const double mid = 0.5 * (blo[a] + bhi[a]);
        const bool upper = comp(k, a) < 0 ? (p[a] > mid) : (p[a] >= mid);
        if (upper) blo[a] = mid; else bhi[a] = mid;
        node = child[node] + (upper ? 1 : 0);
        continue;
      }
      int oct = 0;
      for (int a = 0; a < 3; ++a) {
        double mid = 0.5 * (blo[a] + bhi[a]);
        double ka = comp(k, a);
        bool upper = ka < 0 ? (p[a] > mid) : (p[a] >= mid);
        if (upper) { oct |= 1 << a; blo[a] = mid; } else { bhi[a] = mid; }
      }
      node = child[node] + oct;
    }
    for (int a = 0; a < 3; ++a) { box->lo[a] = blo[a]; box->hi[a] = bhi[a]; }
    return -(int64_t)child[node] - 1;
  }

  void build_leaf_boxes() {
    leaf_box.assign((size_t)n_leaves, Box{});
    struct Item { int64_t node; Box b; };
    std::vector<Item> stack;
    stack.push_back({0, {{lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}}});
    while (!stack.empty()) {
      Item it = stack.back();
      stack.pop_back();
      int32_t c = child[it.node];
      if (c < 0) { leaf_box[(size_t)(-(int64_t)c - 1)] = it.b; continue; }
      if (kind == 3) {
        const int a = split_axis[it.node];
        const double mid = 0.5 * (it.b.lo[a] + it.b.hi[a]);
        Box lower = it.b, upper = it.b;
        lower.hi[a] = mid;
        upper.lo[a] = mid;
        stack.push_back({(int64_t)c, lower});
        stack.push_back({(int64_t)c + 1, upper});
        continue;
      }
      for (int oct = 0; oct < 8; ++oct) {
        Box b;
        for (int a = 0; a < 3; ++a) {
          double mid = 0.5 * (it.b.lo[a] + it.b.hi[a]);
          if (oct & (1 << a)) { b.lo[a] = mid; b.hi[a] = it.b.hi[a]; }
          else { b.lo[a] = it.b.lo[a]; b.hi[a] = mid; }
        }
        stack.push_back({(int64_t)c + oct, b});
      }
    }
  }

  // Cartesian or rectilinear cell containing p (clamped into the grid): on
  // each axis the last cell whose lower plane is at or below p.
  int64_t cart_locate(const double p[3]) const {
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
      int64_t i;
      if (kind == 2) {
        i = (int64_t)(std::upper_bound(edges[a].begin(), edges[a].end(), p[a]) - edges[a].begin()) - 1;
      } else {
        i = (int64_t)std::floor((p[a] - lo[a]) / d[a]);
      }
      idx[a] = std::min<int64_t>(std::max<int64_t>(i, 0), n[a] - 1);
    }
    return idx[0] + n[0] * (idx[1] + (int64_t)n[1] * idx[2]);
  }
};

// Straight path from x along k to the grid boundary.  start_cell >= 0 means x
// is known to lie in that cell; otherwise x is located, or the entry point is
// found when x lies outside the grid.  A ray that misses the grid yields no
// segment.  Zero-length segments are kept.
template <class T>
void grid_path(const Grid& G, const V3<T>& x, const V3d& k, int64_t start_cell,
               std::vector<Seg<T>>& out) {
  out.clear();
  T t = T(0.0);
  int64_t cell = start_cell;
  double xv[3] = {val(x.x), val(x.y), val(x.z)};
  int entry_axis = -1;
  if (cell < 0) {
    bool inside = true;
    for (int a = 0; a < 3; ++a) inside = inside && xv[a] >= G.lo[a] && xv[a] <= G.hi[a];
    if (!inside) {
      // slab method on the values; the entry path length carries derivatives
      double tin = -INFINITY, tout = INFINITY;
      for (int a = 0; a < 3; ++a) {
        double ka = comp(k, a);
        if (ka == 0.0) {
          if (xv[a] < G.lo[a] || xv[a] > G.hi[a]) return;
          continue;
        }
        double t1 = (G.lo[a] - xv[a]) / ka, t2 = (G.hi[a] - xv[a]) / ka;
        double tn = std::min(t1, t2), tf = std::max(t1, t2);
        if (tn > tin) { tin = tn; entry_axis = a; }
        tout = std::min(tout, tf);
      }
      if (!(tin < tout) || tout <= 0.0) return;
      double ka = comp(k, entry_axis);
      double plane = ka > 0 ? G.lo[entry_axis] : G.hi[entry_axis];
      t = (T(plane) - comp(x, entry_axis)) / T(ka);
    }
  }
  if (G.voronoi()) {
    // Voronoi: the cell boundary between sites c and j is their bisecting
    // plane, {y : (y - m) . (s_j - s_c) = 0} with m the midpoint; the ray
    // leaves cell c at the first such plane it meets heading towards s_j
    // (k . (s_j - s_c) > 0) among c's neighbours, or at the domain boundary
    // if that comes first.  The first minimal plane wins ties.
    T t_box = T(INFINITY);
    for (int a = 0; a < 3; ++a) {
      double ka = comp(k, a);
      if (ka == 0.0) continue;
      T ta = (T(ka > 0 ? G.hi[a] : G.lo[a]) - comp(x, a)) / T(ka);
      if (val(ta) < val(t_box)) t_box = ta;
    }
    if (cell < 0) {
      double p[3];
      for (int a = 0; a < 3; ++a) p[a] = xv[a] + val(t) * comp(k, a);
      if (entry_axis >= 0) p[entry_axis] = comp(k, entry_axis) > 0 ? G.lo[entry_axis] : G.hi[entry_axis];
      cell = G.nearest_site(p);
    }
    // a straight line meets each convex cell once: more segments than cells
    // cannot happen
    for (int64_t step = 0; step <= G.n_leaves; ++step) {
      const double* sc = G.sites + 3 * cell;
      int64_t next = -1;
      T texit = t_box;
      for (int64_t f = G.offsets[cell]; f < G.offsets[cell + 1]; ++f) {
        const int64_t j = G.child[f];
        const double* sj = G.sites + 3 * j;
        const double nrm[3] = {sj[0] - sc[0], sj[1] - sc[1], sj[2] - sc[2]};
        const double den = k.x * nrm[0] + k.y * nrm[1] + k.z * nrm[2];
        if (!(den > 0.0)) continue;
        const T num = (T(0.5 * (sc[0] + sj[0])) - x.x) * T(nrm[0]) + (T(0.5 * (sc[1] + sj[1])) - x.y) * T(nrm[1]) +
                      (T(0.5 * (sc[2] + sj[2])) - x.z) * T(nrm[2]);
        const T tj = num / T(den);
        if (val(tj) < val(texit)) { texit = tj; next = j; }
      }
      if (val(texit) < val(t)) texit = t;
      out.push_back({cell, t, texit});
      t = texit;
      if (next < 0) break;
      cell = next;
    }
    return;
  }
  if (!G.tree()) {
    // cartesian and rectilinear: indices of the current cell
    int64_t idx[3];
    if (cell >= 0) {
      idx[0] = cell % G.n[0]; idx[1] = (cell / G.n[0]) % G.n[1]; idx[2] = cell / ((int64_t)G.n[0] * G.n[1]);
    } else {
      double p[3];
      for (int a = 0; a < 3; ++a) p[a] = xv[a] + val(t) * comp(k, a);
      int64_t c = G.cart_locate(p);
      idx[0] = c % G.n[0]; idx[1] = (c / G.n[0]) % G.n[1]; idx[2] = c / ((int64_t)G.n[0] * G.n[1]);
      if (entry_axis >= 0) idx[entry_axis] = comp(k, entry_axis) > 0 ? 0 : G.n[entry_axis] - 1;
    }
    while (true) {
      int64_t c = idx[0] + G.n[0] * (idx[1] + (int64_t)G.n[1] * idx[2]);
      // exit path length through each of the three cell faces ahead
      int axis = -1;
      T texit = T(INFINITY);
      for (int a = 0; a < 3; ++a) {
        double ka = comp(k, a);
        if (ka == 0.0) continue;
        double plane = ka > 0 ? G.plane(a, (int)idx[a] + 1) : G.plane(a, (int)idx[a]);
        T ta = (T(plane) - comp(x, a)) / T(ka);
        if (axis < 0 || val(ta) < val(texit)) { texit = ta; axis = a; }
      }
      if (val(texit) < val(t)) texit = t;
      out.push_back({c, t, texit});
      t = texit;
      idx[axis] += comp(k, axis) > 0 ? 1 : -1;
      if (idx[axis] < 0 || idx[axis] >= G.n[axis]) break;
    }
  } else {
    // octree: walk leaf to leaf, locating each next leaf from the root
    Box box;
    int64_t leaf;
    if (cell >= 0) {
      leaf = cell;
      box = G.leaf_box[(size_t)leaf];
    } else {
      double p[3];
      for (int a = 0; a < 3; ++a) p[a] = xv[a] + val(t) * comp(k, a);
      if (entry_axis >= 0) p[entry_axis] = comp(k, entry_axis) > 0 ? G.lo[entry_axis] : G.hi[entry_axis];
      leaf = G.tree_locate(p, k, &box);
    }
    while (true) {
      int axis = -1;
      T texit = T(INFINITY);
      for (int a = 0; a < 3; ++a) {
        double ka = comp(k, a);
        if (ka == 0.0) continue;
        double plane = ka > 0 ? box.hi[a] : box.lo[a];
        T ta = (T(plane) - comp(x, a)) / T(ka);
        if (axis < 0 || val(ta) < val(texit)) { texit = ta; axis = a; }
      }
      if (val(texit) < val(t)) texit = t;
      out.push_back({leaf, t, texit});
      t = texit;
      double ka = comp(k, axis);
      double plane = ka > 0 ? box.hi[axis] : box.lo[axis];
      if ((ka > 0 && plane >= G.hi[axis]) || (ka < 0 && plane <= G.lo[axis])) break;
      // exit point on the face crossed, the other coordinates kept inside the
      // leaf so that rounding never steps back across a face already crossed
      double p[3];
      for (int a = 0; a < 3; ++a)
        p[a] = std::min(box.hi[a], std::max(box.lo[a], val(comp(x, a)) + val(t) * comp(k, a)));
      p[axis] = plane;
      leaf = G.tree_locate(p, k, &box);
    }
  }
}

// ---------------------------------------------------------------- problem
struct Problem {
  Grid grid;
  int n_lambda;
  std::vector<double> kappa, albedo, g;
  std::vector<or_source> sources;
  std::vector<double> lum;  // [n_sources][n_lambda]
  std::vector<Frame> frames;
  // dust emission instead of the sources: per wavelength the running sum of
  // the cells' luminosities in cell order (empty: the sources emit)
  std::vector<std::vector<double>> dust_cum;
};

Problem make_problem(const or_problem& in) {
  Problem P;
  Grid& G = P.grid;
  G.kind = in.grid.kind;
  for (int a = 0; a < 3; ++a) { G.lo[a] = in.grid.bounds[2 * a]; G.hi[a] = in.grid.bounds[2 * a + 1]; }
  G.n[0] = in.grid.nx; G.n[1] = in.grid.ny; G.n[2] = in.grid.nz;
  for (int a = 0; a < 3; ++a) G.d[a] = G.kind == 0 ? (G.hi[a] - G.lo[a]) / G.n[a] : 0.0;
  if (G.kind == 2)
    for (int a = 0; a < 3; ++a) G.edges[a].assign(in.grid.edges[a], in.grid.edges[a] + G.n[a] + 1);
  G.density = in.grid.density;
  G.child = in.grid.child;
  G.n_nodes = in.grid.n_nodes;
  G.n_leaves = in.grid.n_leaves;
  G.split_axis = in.grid.split_axis;
  G.sites = in.grid.sites;
  G.offsets = in.grid.offsets;
  if (G.tree()) G.build_leaf_boxes();
  P.n_lambda = in.n_lambda;
  P.kappa.assign(in.kappa, in.kappa + in.n_lambda);
  P.albedo.assign(in.albedo, in.albedo + in.n_lambda);
  P.g.assign(in.g, in.g + in.n_lambda);
  P.sources.assign(in.sources, in.sources + in.n_sources);
  P.lum.assign(in.lum, in.lum + (size_t)in.n_sources * in.n_lambda);
  for (int i = 0; i < in.n_instr; ++i) P.frames.push_back(make_frame(in.instr[i]));
  if (in.dust_lum) {
    const int64_t nc = G.n_cells();
    P.dust_cum.assign((size_t)in.n_lambda, std::vector<double>((size_t)nc));
    for (int l = 0; l < in.n_lambda; ++l) {
      double run = 0.0;
      for (int64_t c = 0; c < nc; ++c) {
        run += in.dust_lum[(size_t)l * nc + c];
        P.dust_cum[(size_t)l][(size_t)c] = run;
      }
    }
  }
  return P;
}

// ---------------------------------------------------------------- tallies
// Lock-free add to a double shared between threads (compare-and-swap loop).
inline void shared_add(double* p, double v) {
  uint64_t* u = reinterpret_cast<uint64_t*>(p);
  uint64_t old = __atomic_load_n(u, __ATOMIC_RELAXED);
  while (true) {
    double cur;
    std::memcpy(&cur, &old, sizeof cur);
    const double nv = cur + v;
    uint64_t nu;
    std::memcpy(&nu, &nv, sizeof nu);
    if (__atomic_compare_exchange_n(u, &old, nu, true, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) return;
  }
}

// Accumulates into plain arrays (double runs).  With `shared_abs` set, the
// absorption tallies of all threads go to one array (large grids); with
// `shared_img` set, the images likewise (large frames).
struct ArrayTally {
  const Problem* P;
  std::vector<std::vector<double>> images;
  std::vector<std::vector<int64_t>> image_counts;
  std::vector<double> absorption;
  std::vector<int64_t> absorption_counts;
  bool want_abs = false, want_counts = false;
  double* shared_abs = nullptr;
  int64_t* shared_abs_counts = nullptr;
  double* const* shared_img = nullptr;       // per instrument, the output images
  int64_t* const* shared_img_counts = nullptr;
  NSum emitted, escaped, absorbed, truncated;
  uint64_t crossings = 0, events = 0, peeloffs = 0, packets = 0;
  std::vector<or_record>* records = nullptr;

  void init(const Problem& prob, bool abs, bool counts) {
    P = &prob;
    want_abs = abs;
    want_counts = counts;
    for (const Frame& f : prob.frames) {
      size_t n = shared_img ? 0 : (size_t)f.channels * prob.n_lambda * f.ny * f.nx;
      images.emplace_back(n, 0.0);
      image_counts.emplace_back(counts ? n : 0, 0);
    }
    if (abs && !shared_abs) {
      absorption.assign((size_t)prob.n_lambda * prob.grid.n_cells(), 0.0);
      if (counts) absorption_counts.assign(absorption.size(), 0);
    }
  }
  void pixel(int q, int ch, int lam, int64_t pix, double value, uint64_t pid, int event) {
    const Frame& f = P->frames[q];
    size_t base = ((size_t)ch * P->n_lambda + lam) * f.ny * f.nx;
    if (records && ch == 0) records->push_back({pid, lam, event, q, 0, pix, value});
    if (shared_img) {
      if (shared_img[q]) shared_add(&shared_img[q][base + pix], value);
      if (shared_img_counts && shared_img_counts[q])
        __atomic_fetch_add(&shared_img_counts[q][base + pix], 1, __ATOMIC_RELAXED);
      return;
    }
    images[q][base + pix] += value;
    if (want_counts) image_counts[q][base + pix] += 1;
  }
  void absorb(int lam, int64_t cell, double value) {
    absorbed.add(value);
    if (!want_abs) return;
    size_t i = (size_t)lam * P->grid.n_cells() + cell;
    if (shared_abs) {
      shared_add(&shared_abs[i], value);
      if (shared_abs_counts) __atomic_fetch_add(&shared_abs_counts[i], 1, __ATOMIC_RELAXED);
      return;
    }
    absorption[i] += value;
    if (want_counts) absorption_counts[i] += 1;
  }
};

// Accumulates the vector-Jacobian product sum_bins adj[bin] * d(bin)/d(rho_seed).
struct DualTally {
  const Problem* P;
  const double* const* adj_images;  // per instrument, shaped like the image
  const double* adj_absorption;     // [n_lambda][n_cells] or NULL
  double vjp = 0.0;
  void pixel(int q, int ch, int lam, int64_t pix, const Dual& value, uint64_t, int) {
    if (!adj_images || !adj_images[q]) return;
    const Frame& f = P->frames[q];
    size_t base = ((size_t)ch * P->n_lambda + lam) * f.ny * f.nx;
    vjp += adj_images[q][base + pix] * value.d;
  }
  void absorb(int lam, int64_t cell, const Dual& value) {
    if (!adj_absorption) return;
    vjp += adj_absorption[(size_t)lam * P->grid.n_cells() + cell] * value.d;
  }
};

template <class T> struct DensityOf;
template <> struct DensityOf<double> {
  const Grid* G;
  double operator()(int64_t cell) const { return (double)G->density[cell]; }
};
template <> struct DensityOf<Dual> {
  const Grid* G;
  int64_t seed_cell;
  Dual operator()(int64_t cell) const { return Dual((double)G->density[cell], cell == seed_cell ? 1.0 : 0.0); }
};

// ---------------------------------------------------------------- one packet
template <class T, class Tally>
struct Transport {
  const Problem& P;
  const or_opts& O;
  DensityOf<T> rho;
  Tally& tally;
  std::vector<Seg<T>> segs, peel_segs;
  std::vector<T> tau;

  Transport(const Problem& p, const or_opts& o, DensityOf<T> r, Tally& t) : P(p), O(o), rho(r), tally(t) {}

  // Emission position and direction (Sect. 3.4: the source geometry draws a
  // random position from its density; the emission is isotropic).
  void emit(uint64_t pid, int lam, V3d& x, V3d& k, int64_t* cell_out = nullptr) {
    double u[8];
    draw4(pid, lam, 0, 0, O.seed, O.model_id, u);
    draw4(pid, lam, 0, 1, O.seed, O.model_id, u + 4);
    if (!P.dust_cum.empty()) {
      // thermal dust emission: the cell with probability proportional to its
      // luminosity at this wavelength (the first cell whose running sum
      // exceeds u times the total), a uniform position inside it, an
      // isotropic direction
      const std::vector<double>& cum = P.dust_cum[(size_t)lam];
      const double target = u[0] * cum.back();
      const int64_t c = (int64_t)(std::upper_bound(cum.begin(), cum.end(), target) - cum.begin());
      const int64_t cell = std::min<int64_t>(c, (int64_t)cum.size() - 1);
      const Box b = P.grid.cell_box(cell);
      x = {b.lo[0] + u[1] * (b.hi[0] - b.lo[0]), b.lo[1] + u[2] * (b.hi[1] - b.lo[1]),
           b.lo[2] + u[3] * (b.hi[2] - b.lo[2])};
      if (cell_out) *cell_out = cell;
      double mu = 2.0 * u[6] - 1.0, st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
      double ph = 2.0 * M_PI * u[7];
      k = {st * std::cos(ph), st * std::sin(ph), mu};
      return;
    }
    // source component proportional to its luminosity at this wavelength
    size_t ns = P.sources.size();
    double total = 0.0;
    for (size_t s = 0; s < ns; ++s) total += P.lum[s * P.n_lambda + lam];
    size_t comp_i = ns - 1;
    double cum = 0.0;
    for (size_t s = 0; s < ns; ++s) {
      cum += P.lum[s * P.n_lambda + lam];
      if (u[0] < cum / total) { comp_i = s; break; }
    }
    const or_source& S = P.sources[comp_i];
    x = {S.center[0], S.center[1], S.center[2]};
    if (S.kind == 1) {
      // double-exponential disk: R has density R exp(-R/hR) (sum of two
      // exponential deviates), z is Laplace distributed with scale hz
      double R = -S.scale_r * std::log(u[1] * u[2]);
      double ph = 2.0 * M_PI * u[3];
      double z = -S.scale_z * std::log(u[4]);
      if (u[5] < 0.5) z = -z;
      x.x += R * std::cos(ph); x.y += R * std::sin(ph); x.z += z;
    } else if (S.kind == 2) {
      // Plummer sphere: enclosed mass fraction m = r^3 / (r^2 + a^2)^(3/2)
      double r = S.scale_r / std::sqrt(std::pow(u[1], -2.0 / 3.0) - 1.0);
      double ct = 2.0 * u[2] - 1.0, st = std::sqrt(std::max(0.0, 1.0 - ct * ct));
      double ph = 2.0 * M_PI * u[3];
      x.x += r * st * std::cos(ph); x.y += r * st * std::sin(ph); x.z += r * ct;
    }
    double mu = 2.0 * u[6] - 1.0, st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    double ph = 2.0 * M_PI * u[7];
    k = {st * std::cos(ph), st * std::sin(ph), mu};
  }

  // Optical depth from x to the grid boundary along d, with the crossing count.
  T optical_depth(const V3<T>& x, const V3d& d, int64_t cell, int lam, uint64_t& crossings) {
    grid_path(P.grid, x, d, cell, peel_segs);
    crossings += peel_segs.size();
    T t = T(0.0);
    for (const Seg<T>& s : peel_segs) t = t + T(P.kappa[lam]) * rho(s.cell) * (s.s_out - s.s_in);
    return t;
  }

  // Peel-off towards every instrument: weight_q * exp(-tau) into the pixel(s)
  // that x projects onto.  ch = 1 direct (emission), 2 scattered.
  void peel(const V3<T>& x, int64_t cell, int lam, const T& L, bool scattered, const V3d& k,
            uint64_t pid, int event) {
    for (size_t q = 0; q < P.frames.size(); ++q) {
      const Frame& f = P.frames[q];
      T w = L * T(1.0 / (4.0 * M_PI));
      if (scattered) w = w * T(hg_phase(P.g[lam], k.x * f.kobs.x + k.y * f.kobs.y + k.z * f.kobs.z));
      T value = w * exp(-optical_depth(x, f.kobs, cell, lam, tally_crossings));
      tally_peeloffs += 1;
      if (f.sed) {
        // SED instrument (Sect. 2.2): the flux received from direction k_obs
        // per wavelength, wherever the peel-off starts
        tally.pixel((int)q, 0, lam, 0, value, pid, event);
        if (f.channels == 3) tally.pixel((int)q, scattered ? 2 : 1, lam, 0, value, pid, event);
        continue;
      }
      T xp = x.x * T(f.ex.x) + x.y * T(f.ex.y) + x.z * T(f.ex.z) - T(f.cx);
      T yp = x.x * T(f.ey.x) + x.y * T(f.ey.y) + x.z * T(f.ey.z) - T(f.cy);
      T fx = (xp + T(f.half_x)) * T(f.nx / (2.0 * f.half_x));
      T fy = (yp + T(f.half_y)) * T(f.ny / (2.0 * f.half_y));
      int ch = scattered ? 2 : 1;
      if (!f.bilinear) {
        double ix = std::floor(val(fx)), iy = std::floor(val(fy));
        if (ix < 0 || iy < 0 || ix >= f.nx || iy >= f.ny) continue;
        int64_t pix = (int64_t)iy * f.nx + (int64_t)ix;
        tally.pixel((int)q, 0, lam, pix, value, pid, event);
        if (f.channels == 3) tally.pixel((int)q, ch, lam, pix, value, pid, event);
      } else {
        // bilinear: pixel centres at integer + 1/2
        T gx = fx - T(0.5), gy = fy - T(0.5);
        double ix0 = std::floor(val(gx)), iy0 = std::floor(val(gy));
        T tx = gx - T(ix0), ty = gy - T(iy0);
        for (int dy = 0; dy < 2; ++dy) {
          for (int dx = 0; dx < 2; ++dx) {
            double ix = ix0 + dx, iy = iy0 + dy;
            if (ix < 0 || iy < 0 || ix >= f.nx || iy >= f.ny) continue;
            T wx = dx ? tx : T(1.0) - tx;
            T wy = dy ? ty : T(1.0) - ty;
            int64_t pix = (int64_t)iy * f.nx + (int64_t)ix;
            T v = value * wx * wy;
            tally.pixel((int)q, 0, lam, pix, v, pid, event);
            if (f.channels == 3) tally.pixel((int)q, ch, lam, pix, v, pid, event);
          }
        }
      }
    }
  }

  uint64_t tally_crossings = 0, tally_peeloffs = 0, tally_events = 0;
  std::vector<or_trace_row>* trace = nullptr;
  void trace_row(int event, int64_t cell, const V3<T>& x, const V3d& k, const T& L, double tp, double ts) {
    if (!trace) return;
    trace->push_back({event, 0, cell, {val(x.x), val(x.y), val(x.z)}, {k.x, k.y, k.z}, val(L), tp, ts});
  }
  T t_emitted = T(0.0), t_escaped = T(0.0), t_truncated = T(0.0);

  // Step (a): the forced path from x along k to the grid boundary, its
  // segments (segs) and cumulative optical depths tau[0..n]; returns tau_path.
  T forced_path(const V3<T>& x, const V3d& k, int64_t cell, int lam) {
    grid_path(P.grid, x, k, cell, segs);
    tally_crossings += segs.size();
    tau.assign(segs.size() + 1, T(0.0));
    for (size_t i = 0; i < segs.size(); ++i)
      tau[i + 1] = tau[i] + T(P.kappa[lam]) * rho(segs[i].cell) * (segs[i].s_out - segs[i].s_in);
    return tau[segs.size()];
  }

  // Step (c): the segment of the forced path in which the cumulative optical
  // depth first exceeds tau_star, and the path length s_star of the
  // interaction, s_in + (tau_star - tau_before) / (kappa rho).  When rounding
  // leaves tau_star at or above the path's optical depth (u at its upper end),
  // the interaction is the end of the last segment that holds dust (the limit
  // of the inversion as tau_star tends to tau_path); *fallback reports it.
  size_t interaction(const T& tau_star, double kap, T& s_star, bool* fallback) {
    size_t hit = segs.size();
    for (size_t i = 0; i < segs.size(); ++i)
      if (val(tau[i + 1]) > val(tau_star)) { hit = i; break; }
    if (fallback) *fallback = hit == segs.size();
    if (hit == segs.size()) {
      hit = 0;
      for (size_t i = 0; i < segs.size(); ++i) if (val(tau[i + 1]) > val(tau[i])) hit = i;
      s_star = segs[hit].s_out;
    } else {
      s_star = segs[hit].s_in + (tau_star - tau[hit]) / (T(kap) * rho(segs[hit].cell));
    }
    return hit;
  }

  // Move x along k by s_star and keep it inside the interaction cell (the
  // point lies in that cell's segment; rounding of x + s_star k may put it a
  // few ulps outside).  *clamped reports whether a coordinate was moved.
  void move_to(V3<T>& x, const V3d& k, const T& s_star, int64_t cell, bool* clamped) {
    x = {x.x + s_star * T(k.x), x.y + s_star * T(k.y), x.z + s_star * T(k.z)};
    // the interaction cell's box; a Voronoi cell is no box: the point is
    // kept inside the domain only (a walk from a point a rounding error
    // outside its cell takes a zero-length segment there, exit distances
    // being clamped to the start)
    Box b = P.grid.voronoi() ? Box{{P.grid.lo[0], P.grid.lo[1], P.grid.lo[2]}, {P.grid.hi[0], P.grid.hi[1], P.grid.hi[2]}}
                             : P.grid.cell_box(cell);
    bool moved = false;
    for (int a = 0; a < 3; ++a) {
      T xa = comp(x, a);
      if (val(xa) < b.lo[a]) { xa = T(b.lo[a]); moved = true; }
      if (val(xa) > b.hi[a]) { xa = T(b.hi[a]); moved = true; }
      set_comp(x, a, xa);
    }
    if (clamped) *clamped = moved;
  }

  void run_packet(uint64_t pid, int lam) {
    double Ltot = 0.0;
    if (!P.dust_cum.empty()) {
      Ltot = P.dust_cum[(size_t)lam].back();
    } else {
      for (size_t s = 0; s < P.sources.size(); ++s) Ltot += P.lum[s * P.n_lambda + lam];
    }
    const double L0 = Ltot / (double)O.n_norm;
    if (L0 == 0.0 && !P.dust_cum.empty()) return;  // the dust emits nothing at this wavelength
    const double kap = P.kappa[lam], alb = P.albedo[lam], g = P.g[lam];
    V3d x0, k;
    int64_t cell = -1;
    emit(pid, lam, x0, k, &cell);
    V3<T> x = {T(x0.x), T(x0.y), T(x0.z)};
    T L = T(L0);
    t_emitted = t_emitted + L;
    trace_row(0, -1, x, k, L, 0.0, 0.0);
    if (O.peel_emission) peel(x, cell, lam, L, false, k, pid, 0);
    for (int j = 1;; ++j) {
      // (a) the forced path to the boundary
      const T tau_path = forced_path(x, k, cell, lam);
      if (val(tau_path) <= 0.0) {
        trace_row(j, -1, x, k, L, 0.0, 0.0);
        t_escaped = t_escaped + L;
        return;
      }
      // (b) escape and continuous absorption along the whole path
      const T E = exp(-tau_path);
      const T one_minus_E = -expm1(-tau_path);
      t_escaped = t_escaped + L * E;
      for (size_t i = 0; i < segs.size(); ++i) {
        if (!(val(tau[i + 1]) > val(tau[i]))) continue;
        T dep = T(1.0 - alb) * L * (exp(-tau[i]) - exp(-tau[i + 1]));
        tally.absorb(lam, segs[i].cell, dep);
      }
      // (c) forced scattering: invert the cumulative optical depth
      double u[4];
      draw4(pid, lam, j, 0, O.seed, O.model_id, u);
      const T tau_star = -log1p(-T(u[0]) * one_minus_E);
      T s_star;
      const size_t hit = interaction(tau_star, kap, s_star, nullptr);
      cell = segs[hit].cell;
      move_to(x, k, s_star, cell, nullptr);
      // (d) scattered weight and peel-off
      L = T(alb) * L * one_minus_E;
      trace_row(j, cell, x, k, L, val(tau_path), val(tau_star));
      tally_events += 1;
      if (O.peel_scatter) peel(x, cell, lam, L, true, k, pid, j);
      // (e) Henyey-Greenstein direction
      k = scatter_direction(k, g, u[1], u[2]);
      // (f) termination
      if ((O.weight_cut && val(L) < O.w_min * L0) || j >= O.max_events) {
        t_truncated = t_truncated + L;
        return;
      }
    }
  }
};

// ---------------------------------------------------------------- panchromatic mode
// A panchromatic simulation (Sect. 2.1, 2.2) integrates the absorbed energy
// over a wavelength range to find the dust temperature and adds the dust's
// thermal emission.  Equilibrium only: one grain type, each cell at the
// temperature at which it emits what it absorbs.
//   * wavelength bins: the grid points are bin centres on a logarithmic
//     scale, the inner borders their geometric means, the outer borders
//     mirrored; widths dlambda_l;
//   * emission of cell c at temperature T: S m_c sum_l kabs_l dlambda_l
//     beta_l(T), m_c = rho_c V_c, kabs_l = kappa_l (1 - albedo_l), beta_l(T) =
//     lambda_l^-5 / (exp(C2 / (lambda_l T)) - 1) the Planck function per unit
//     wavelength up to its constant (lambda in um, C2 = hc/k in um K), S the
//     caller's scale (the Planck constant 2hc^2, 4 pi and the units);
//   * the temperature: bisection in ln T between t_min and t_max (64 halvings)
//     on emission = sum_l absorbed_l[c]; no absorption or no dust: T = 0;
//     emission short of the absorption at t_max: T = t_max, beyond it at
//     t_min: T = t_min (both counted).
constexpr double kC2 = 14387.768775039337;  // hc / k in um K

std::vector<double> bin_widths(const double* lambda, int n) {
  std::vector<double> b((size_t)n + 1), w((size_t)n);
  for (int l = 1; l < n; ++l) b[(size_t)l] = std::sqrt(lambda[l - 1] * lambda[l]);
  b[0] = lambda[0] * std::sqrt(lambda[0] / lambda[1]);
  b[(size_t)n] = lambda[n - 1] * std::sqrt(lambda[n - 1] / lambda[n - 2]);
  for (int l = 0; l < n; ++l) w[(size_t)l] = b[(size_t)l + 1] - b[(size_t)l];
  return w;
}

double planck_shape(double lambda_um, double T) {
  return 1.0 / (std::pow(lambda_um, 5.0) * std::expm1(kC2 / (lambda_um * T)));
}

double cell_mass(const Grid& G, int64_t c) {
  const Box b = G.cell_box(c);
  return (double)G.density[c] * ((b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]));
}

// S kabs_l dlambda_l for every wavelength.
std::vector<double> emission_weights(const Problem& P, const double* lambda, double scale) {
  const std::vector<double> w = bin_widths(lambda, P.n_lambda);
  std::vector<double> out((size_t)P.n_lambda);
  for (int l = 0; l < P.n_lambda; ++l)
    out[(size_t)l] = scale * P.kappa[(size_t)l] * (1.0 - P.albedo[(size_t)l]) * w[(size_t)l];
  return out;
}

double cell_emission(const std::vector<double>& wts, const double* lambda, double mass, double T) {
  double sum = 0.0;
  for (size_t l = 0; l < wts.size(); ++l) sum += wts[l] * planck_shape(lambda[l], T);
  return mass * sum;
}

int64_t total_packets(const Problem& P, const or_opts& O) { return (int64_t)O.n_per_lambda * P.n_lambda; }

}  // namespace

// ================================================================ C API
extern "C" {

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox4x32_10(ctr, key, out);
}

void or_draw4(uint64_t pid, int32_t lam, int32_t event, int32_t block, uint32_t seed, uint32_t model,
              double out[4]) {
  draw4(pid, lam, event, block, seed, model, out);
}

double or_hg_sample(double g, double u) { return hg_sample(g, u); }
double or_hg_phase(double g, double mu) { return hg_phase(g, mu); }

void or_rotate(const double k[3], double mu, double phi, double out[3]) {
  V3d r = rotate_dir({k[0], k[1], k[2]}, mu, phi);
  out[0] = r.x; out[1] = r.y; out[2] = r.z;
}

void or_scatter_direction(const double k[3], double g, double u1, double u2, double out[3]) {
  V3d r = scatter_direction({k[0], k[1], k[2]}, g, u1, u2);
  out[0] = r.x; out[1] = r.y; out[2] = r.z;
}

// Frame axes: out = kobs[3], ex[3], ey[3].
void or_frame(const or_instrument* in, double out[9]) {
  Frame f = make_frame(*in);
  double v[9] = {f.kobs.x, f.kobs.y, f.kobs.z, f.ex.x, f.ex.y, f.ex.z, f.ey.x, f.ey.y, f.ey.z};
  std::memcpy(out, v, sizeof v);
}

// Emission of one packet: x[3], k[3].
void or_emit(const or_problem* prob, const or_opts* opts, uint64_t pid, int32_t lam, double x[3],
             double k[3]) {
  Problem P = make_problem(*prob);
  ArrayTally T;
  Transport<double, ArrayTally> tr(P, *opts, DensityOf<double>{&P.grid}, T);
  V3d xv, kv;
  tr.emit(pid, lam, xv, kv);
  x[0] = xv.x; x[1] = xv.y; x[2] = xv.z;
  k[0] = kv.x; k[1] = kv.y; k[2] = kv.z;
}

// Path segments from x along k: returns the segment count (<= cap written).
int64_t or_path(const or_problem* prob, const double x[3], const double k[3], int64_t start_cell,
                int64_t* cells, double* s_in, double* s_out, int64_t cap) {
  Problem P = make_problem(*prob);
  std::vector<Seg<double>> segs;
  grid_path(P.grid, V3d{x[0], x[1], x[2]}, V3d{k[0], k[1], k[2]}, start_cell, segs);
  for (size_t i = 0; i < segs.size() && (int64_t)i < cap; ++i) {
    cells[i] = segs[i].cell; s_in[i] = segs[i].s_in; s_out[i] = segs[i].s_out;
  }
  return (int64_t)segs.size();
}

// Leaf / cell containing p (octree tie rule along k; cartesian floor rule;
// Voronoi: the nearest site, box = the domain).
int64_t or_locate(const or_problem* prob, const double p[3], const double k[3], double box[6]) {
  Problem P = make_problem(*prob);
  Box b;
  int64_t c;
  if (P.grid.voronoi()) {
    c = P.grid.nearest_site(p);
    for (int a = 0; a < 3; ++a) { b.lo[a] = P.grid.lo[a]; b.hi[a] = P.grid.hi[a]; }
  } else if (P.grid.tree()) {
    c = P.grid.tree_locate(p, V3d{k[0], k[1], k[2]}, &b);
  } else {
    c = P.grid.cart_locate(p);
    b = P.grid.cell_box(c);
  }
  for (int a = 0; a < 3; ++a) { box[2 * a] = b.lo[a]; box[2 * a + 1] = b.hi[a]; }
  return c;
}

// Full transport run.  Returns 0 on success, < 0 on bad arguments.
int32_t or_run(const or_problem* prob, const or_opts* opts, or_output* out) {
  if (!prob || !opts || !out || opts->n_per_lambda == 0 || opts->n_norm == 0 || prob->n_lambda <= 0 ||
      (prob->n_sources <= 0 && !prob->dust_lum) || (prob->dust_lum && prob->grid.kind == 4))
    return -1;
  Problem P = make_problem(*prob);
  const or_opts& O = *opts;
  const int64_t n_total = total_packets(P, O);
  const int n_threads = std::max(1, O.n_threads);
  const bool want_abs = out->absorption != nullptr;
  const bool want_counts = out->image_counts != nullptr || out->absorption_counts != nullptr;
  std::vector<ArrayTally> tallies((size_t)n_threads);
  // peel-off records per thread, concatenated in thread order
  std::vector<std::vector<or_record>> recs((size_t)n_threads);
  // private absorption arrays per thread unless that needs more than 2 GiB
  const double abs_bytes = (double)P.n_lambda * (double)P.grid.n_cells() * (want_counts ? 16.0 : 8.0);
  const bool shared = want_abs && n_threads > 1 && abs_bytes * n_threads > 2.0 * (1 << 30);
  // likewise one set of images for all threads when private ones would need
  // more than 2 GiB
  double img_bytes = 0.0;
  for (const Frame& f : P.frames) img_bytes += (double)f.channels * P.n_lambda * f.ny * f.nx * (want_counts ? 16.0 : 8.0);
  const bool shared_images = n_threads > 1 && out->images && img_bytes * n_threads > 2.0 * (1 << 30);
  for (int t = 0; t < n_threads; ++t) {
    if (shared) {
      tallies[t].shared_abs = out->absorption;
      tallies[t].shared_abs_counts = out->absorption_counts;
    }
    if (shared_images) {
      tallies[t].shared_img = out->images;
      tallies[t].shared_img_counts = want_counts ? out->image_counts : nullptr;
    }
    tallies[t].init(P, want_abs, want_counts);
  }
  if (out->records)
    for (int t = 0; t < n_threads; ++t) tallies[t].records = &recs[(size_t)t];
  // static interleaved chunks: deterministic for a given thread count
  const int64_t chunk = 64;
  auto worker = [&](int tid) {
    ArrayTally& T = tallies[tid];
    Transport<double, ArrayTally> tr(P, O, DensityOf<double>{&P.grid}, T);
    for (int64_t c0 = (int64_t)tid * chunk; c0 < n_total; c0 += (int64_t)n_threads * chunk) {
      for (int64_t w = c0; w < std::min(n_total, c0 + chunk); ++w) {
        int lam = (int)(w / (int64_t)O.n_per_lambda);
        uint64_t pid = O.first_id + (uint64_t)(w % (int64_t)O.n_per_lambda);
        tr.t_emitted = tr.t_escaped = tr.t_truncated = 0.0;
        tr.run_packet(pid, lam);
        T.emitted.add(tr.t_emitted);
        T.escaped.add(tr.t_escaped);
        T.truncated.add(tr.t_truncated);
        T.packets += 1;
      }
    }
    T.crossings = tr.tally_crossings;
    T.events = tr.tally_events;
    T.peeloffs = tr.tally_peeloffs;
  };
  if (n_threads == 1) {
    worker(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < n_threads; ++t) th.emplace_back(worker, t);
    for (auto& t : th) t.join();
  }
  // reduce in thread order
  NSum em, es, ab, tr;
  uint64_t cr = 0, ev = 0, pe = 0, pk = 0;
  for (int t = 0; t < n_threads; ++t) {
    ArrayTally& T = tallies[t];
    em.add(T.emitted.value()); es.add(T.escaped.value()); ab.add(T.absorbed.value()); tr.add(T.truncated.value());
    cr += T.crossings; ev += T.events; pe += T.peeloffs; pk += T.packets;
    for (size_t q = 0; q < P.frames.size() && !shared_images; ++q) {
      if (out->images && out->images[q]) {
        double* dst = out->images[q];
        for (size_t i = 0; i < T.images[q].size(); ++i) dst[i] += T.images[q][i];
      }
      if (out->image_counts && out->image_counts[q] && want_counts) {
        int64_t* dst = out->image_counts[q];
        for (size_t i = 0; i < T.image_counts[q].size(); ++i) dst[i] += T.image_counts[q][i];
      }
    }
    if (want_abs && !shared) {
      for (size_t i = 0; i < T.absorption.size(); ++i) out->absorption[i] += T.absorption[i];
      if (out->absorption_counts)
        for (size_t i = 0; i < T.absorption_counts.size(); ++i) out->absorption_counts[i] += T.absorption_counts[i];
    }
  }
  out->stats[0] += em.value(); out->stats[1] += es.value(); out->stats[2] += ab.value(); out->stats[3] += tr.value();
  out->counters[0] += cr; out->counters[1] += ev; out->counters[2] += pe; out->counters[3] += pk;
  if (out->records) {
    int64_t n = 0;
    for (const auto& r : recs) {
      const int64_t take = std::min<int64_t>((int64_t)r.size(), std::max<int64_t>(0, out->records_cap - n));
      if (take > 0) std::memcpy(out->records + n, r.data(), (size_t)take * sizeof(or_record));
      n += (int64_t)r.size();
    }
    out->records_n = n;
  }
  return 0;
}

// Per-event trace of one packet; returns the number of rows (<= cap written).
int64_t or_trace(const or_problem* prob, const or_opts* opts, uint64_t pid, int32_t lam, or_trace_row* rows,
                 int64_t cap) {
  Problem P = make_problem(*prob);
  ArrayTally T;
  T.init(P, false, false);
  std::vector<or_trace_row> tr;
  Transport<double, ArrayTally> t(P, *opts, DensityOf<double>{&P.grid}, T);
  t.trace = &tr;
  t.run_packet(pid, lam);
  for (int64_t i = 0; i < (int64_t)tr.size() && i < cap; ++i) rows[i] = tr[(size_t)i];
  return (int64_t)tr.size();
}

// One forced path and its interaction (steps a and c of the per-packet
// algorithm) for a given uniform u, from x along k (start_cell >= 0: x lies in
// that cell): out_x[3] the interaction point, *out_cell its cell, *out_tau =
// {tau_path, tau_star}; returns flags: bit 0 the rounding fallback of the
// inversion acted, bit 1 the position was moved into the interaction cell,
// bit 2 the path holds no dust (nothing else is written).
int32_t or_interaction(const or_problem* prob, const double x[3], const double k[3], int64_t start_cell,
                       int32_t lam, double u, double out_x[3], int64_t* out_cell, double out_tau[2]) {
  Problem P = make_problem(*prob);
  or_opts O;
  std::memset(&O, 0, sizeof O);
  O.n_per_lambda = 1;
  O.n_norm = 1;
  ArrayTally T;
  T.init(P, false, false);
  Transport<double, ArrayTally> tr(P, O, DensityOf<double>{&P.grid}, T);
  V3d xv{x[0], x[1], x[2]}, kv{k[0], k[1], k[2]};
  const double tau_path = tr.forced_path(xv, kv, start_cell, lam);
  if (!(tau_path > 0.0)) return 4;
  const double one_minus_E = -std::expm1(-tau_path);
  const double tau_star = -std::log1p(-u * one_minus_E);
  double s_star = 0.0;
  bool fallback = false, clamped = false;
  const size_t hit = tr.interaction(tau_star, P.kappa[lam], s_star, &fallback);
  const int64_t cell = tr.segs[hit].cell;
  tr.move_to(xv, kv, s_star, cell, &clamped);
  out_x[0] = xv.x; out_x[1] = xv.y; out_x[2] = xv.z;
  *out_cell = cell;
  out_tau[0] = tau_path;
  out_tau[1] = tau_star;
  return (fallback ? 1 : 0) | (clamped ? 2 : 0);
}

// Equilibrium dust temperature of every cell from the absorbed luminosity
// absorption [n_lambda][n_cells] (panchromatic mode; see the notes above
// bin_widths).  Returns the number of cells held at t_min or t_max, or -1 on bad
// arguments (fewer than two wavelengths, an octree grid, t range empty).
int32_t or_dust_temperature(const or_problem* prob, const double* lambda, const double* absorption, double scale,
                            double t_min, double t_max, double* T_out) {
  if (!prob || !lambda || !absorption || !T_out || prob->n_lambda < 2 || prob->grid.kind == 1 || prob->grid.kind == 3 ||
      prob->grid.kind == 4 || !(t_min > 0 && t_max > t_min) || !(scale > 0))
    return -1;
  Problem P = make_problem(*prob);
  const int64_t nc = P.grid.n_cells();
  const std::vector<double> wts = emission_weights(P, lambda, scale);
  int32_t clamped = 0;
  for (int64_t c = 0; c < nc; ++c) {
    double absorbed = 0.0;
    for (int l = 0; l < P.n_lambda; ++l) absorbed += absorption[(size_t)l * nc + c];
    const double m = cell_mass(P.grid, c);
    if (!(absorbed > 0.0) || !(m > 0.0) || !(cell_emission(wts, lambda, m, t_max) > 0.0)) {
      T_out[c] = 0.0;
      continue;
    }
    if (cell_emission(wts, lambda, m, t_max) < absorbed) {
      T_out[c] = t_max;
      ++clamped;
      continue;
    }
    if (cell_emission(wts, lambda, m, t_min) >= absorbed) {
      T_out[c] = t_min;
      ++clamped;
      continue;
    }
    double lo = std::log(t_min), hi = std::log(t_max);
    for (int it = 0; it < 64; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (cell_emission(wts, lambda, m, std::exp(mid)) < absorbed) lo = mid; else hi = mid;
    }
    T_out[c] = std::exp(0.5 * (lo + hi));
  }
  return clamped;
}

// Thermal emission of every cell at the temperatures T [n_cells] (T = 0: no
// emission): lum_out [n_lambda][n_cells] = S m_c kabs_l dlambda_l beta_l(T_c).
int32_t or_dust_emission(const or_problem* prob, const double* lambda, const double* T, double scale,
                         double* lum_out) {
  if (!prob || !lambda || !T || !lum_out || prob->n_lambda < 2 || prob->grid.kind == 1 || prob->grid.kind == 3 ||
      prob->grid.kind == 4 || !(scale > 0))
    return -1;
  Problem P = make_problem(*prob);
  const int64_t nc = P.grid.n_cells();
  const std::vector<double> wts = emission_weights(P, lambda, scale);
  for (int64_t c = 0; c < nc; ++c) {
    const double m = cell_mass(P.grid, c);
    for (int l = 0; l < P.n_lambda; ++l)
      lum_out[(size_t)l * nc + c] = T[c] > 0.0 ? m * wts[(size_t)l] * planck_shape(lambda[l], T[c]) : 0.0;
  }
  return 0;
}

// Vector-Jacobian product by forward-mode dual numbers, one seeded cell at a
// time: grad[i] = sum_bins adj[bin] * d(bin)/d(rho[cells[i]]).
int32_t or_vjp(const or_problem* prob, const or_opts* opts, const double* const* adj_images,
               const double* adj_absorption, const int64_t* cells, int64_t n_cells, double* grad) {
  if (!prob || !opts || !grad || opts->n_per_lambda == 0 || opts->n_norm == 0) return -1;
  Problem P = make_problem(*prob);
  const or_opts& O = *opts;
  const int64_t n_total = total_packets(P, O);
  const int n_threads = std::max(1, O.n_threads);
  std::atomic<int64_t> next{0};
  auto worker = [&]() {
    for (int64_t i = next++; i < n_cells; i = next++) {
      DualTally T{&P, adj_images, adj_absorption, 0.0};
      Transport<Dual, DualTally> tr(P, O, DensityOf<Dual>{&P.grid, cells[i]}, T);
      for (int64_t w = 0; w < n_total; ++w) {
        int lam = (int)(w / (int64_t)O.n_per_lambda);
        uint64_t pid = O.first_id + (uint64_t)(w % (int64_t)O.n_per_lambda);
        tr.run_packet(pid, lam);
      }
      grad[i] = T.vjp;
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  return 0;
}

}  // extern "C"

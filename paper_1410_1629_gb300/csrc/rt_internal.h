// Internal definitions shared by the host side of the C ABI (rt_api.cu) and the
// kernels.  Not part of the public interface (include/rt.h).
#pragma once

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rt.h"

namespace rtk {

constexpr int kMaxLambda = 64;
constexpr int kMaxSources = 16;
constexpr int kMaxInstruments = 16;
constexpr int kMaxOctreeDepth = 21;

// Per-wavelength optical properties (Sect. 2.3) and source luminosity total.
struct DevLambda {
  float kappa;        // extinction per unit density per unit length (FP32 for the walk)
  float g;            // HG asymmetry parameter
  float pad0, pad1;
  double albedo;
  double one_minus_albedo;
  double lum_total;   // sum of the sources' luminosities at this wavelength
};

// Emission component (Sect. 3.4).
struct DevSource {
  int kind;
  int pad;
  double center[3];
  double scale_r, scale_z;
};

// Frame instrument (Sect. 2.2): FP32 projection axes and pixel mapping.
struct DevInstr {
  float kobs[3], ex[3], ey[3];
  float off_x, off_y;  // half width minus field centre
  float sx, sy;        // pixels per unit length: n / (2 half)
  int nx, ny;
  int bilinear, channels;
  int sed;             // SED instrument: one bin per wavelength, no projection
  double* image;       // [channels][n_lambda][ny][nx]
  // a frame looking exactly along grid axis `axis` (dir +-1): column[c] is the
  // density integral from the face of cell c that the ray leaves to the grid
  // boundary, sum of rho d_axis over the cells beyond c (or null: walk)
  const float* column;
  int axis, dir;
};

struct AdjRecord;

// A peel-off whose walk runs in the sorted pass after the transport kernel
// (one 32-byte sector): the position it starts from; its sort key, the
// instrument q times (n_cells + 1) plus the cell of the position (n_cells
// when it lies outside the grid); the packet weight; the phase-function value
// towards the instrument (1 at emission); the wavelength in the low 16 bits
// of meta, bit 30 set for a scattering, bit 31 when the walk starts from the
// packet's known cell.
struct alignas(32) PeelRecord {
  float x, y, z;
  unsigned key;
  double L;
  float phase;
  unsigned meta;
};

// Everything a forward launch needs, passed by value.
struct FwdParams {
  // dust grid
  int nx, ny, nz;
  int pad0;
  float lo[3], hi[3], d[3], inv_d[3];
  const float* density;
  const int32_t* child;  // octree: child[] as given; k-d tree: node words (first child << 2 | axis, or -(leaf + 1))
  // k-d trees: per leaf and face (2 axis + (exit towards +axis)) the node
  // across that face whose box covers the face (-1: the domain boundary), and
  // every node's box (FP32, lo then hi, as the descent halves it)
  const int32_t* rope;
  const float4* node_box;
  long long n_nodes;     // octree only
  // octree boxes are exact binary fractions of the domain (every box corner
  // at any depth is representable and every halving exact): a box can be
  // rebuilt upwards from a leaf (size doubled) instead of down from the root
  int oct_exact;
  int oct_levels;  // octrees: ancestor-stack entries per lane (the deepest leaf's depth + 1)
  const float* edge[3];  // rectilinear only: cell edges per axis, n + 1 each
  // Voronoi grids: sites (x, y, z, 0), the faces of cell c at
  // [face_off[c], face_off[c + 1]) as (unit normal towards the neighbour,
  // distance of the bisecting plane from the site) with the neighbour's id in
  // child[], and per bucket of a uniform bucket grid the site nearest to its
  // centre (bucket (i, j, k) at i + vb_n[0] (j + vb_n[1] k))
  const float4* site;
  const int* face_off;
  const float4* face;
  const int* bucket_seed;
  int vb_n[3];
  float vb_inv[3];  // buckets per unit length per axis
  int max_walk;     // cells one Voronoi walk or point location may visit before the walk flag
  // storage strides of the cell index (cartesian and rectilinear grids): the
  // density and absorption of cell (ix, iy, iz) sit at ix stride[0] +
  // iy stride[1] + iz stride[2]; row-major is (1, nx, nx ny).  Cell ids seen
  // outside the kernels (records, traces, the tape, read-outs) are row-major.
  int stride[3];
  long long n_cells;
  // problem
  int n_lambda, n_sources, n_instr;
  int pad1;
  const DevLambda* lam;
  const DevSource* src;
  const double* src_cum;  // [n_lambda][n_sources] cumulative luminosity fractions
  const DevInstr* instr;
  double* absorption;     // [n_lambda][n_cells]
  // run
  unsigned long long n_per_lambda, first_id, n_total, n_norm;
  unsigned int seed, model;
  double w_min;
  int max_events, weight_cut, peel_emission, peel_scatter;
  unsigned long long* work_counter;
  double* stats;                  // emitted, escaped, absorbed, truncated
  unsigned long long* counters;   // crossings, events, peeloffs, packets, records, path crossings,
                                  // column peel-offs, column crossings, sorted-pass peel-offs
  rt_record* records;
  long long records_cap;
  unsigned long long record_stride;
  rt_trace_row* trace;
  long long trace_cap;
  unsigned long long trace_packet;
  int trace_lambda;
  int control_min;  // lanes that must wait for per-event work before a warp runs it
  int blocks_per_sm;  // resident blocks of the persistent grid per SM (0: as many as fit)
  float inv_n_per_lambda;          // 1 / n_per_lambda (estimate of a packet's wavelength index)
  double L0[kMaxLambda];           // packet weight at emission, L_tot / n_norm, per wavelength
  double L_cut[kMaxLambda];        // w_min * L0 per wavelength
  unsigned long long* profile;  // optional execution counters (see rt_launch_opts.profile)
  int* flags;
  int use_columns;              // peel-offs along grid axes use the instruments' column sums
  AdjRecord* tape;              // adjoint tape: [packets][tape_stride] event records, or null
  int tape_stride;              // records per packet (max_events + 1)
  // peel-off walks deferred to the sorted pass (cartesian grids), or peel null
  PeelRecord* peel;
  unsigned long long peel_cap;     // records peel holds
  unsigned long long* peel_count;  // records asked for (beyond peel_cap the kernel walks them itself)
  unsigned* peel_hist;             // [n_instr][n_cells + 1]: records per sort key
  ulonglong2* peel_tag;            // [peel_cap] packet id and event of each record (debug records on), or null
  // panchromatic mode: packets emitted by the dust instead of the sources;
  // per wavelength the running sums of the cells' thermal luminosities over
  // the row-major cells ([n_lambda][n_cells]), or null
  const double* dust_cum;
};

enum DeviceFlag : int { kFlagCellRange = 1, kFlagOctreeDepth = 2, kFlagWalkSteps = 4, kFlagNoInteraction = 8 };
// Upper bound on the cells one straight octree walk may visit before the
// kernel flags an error and stops the walk (3 * 2^depth covers any ray for
// the depths used; this is a safety net, not a tuning knob).
constexpr unsigned kMaxWalkSteps = 1u << 22;

// Frame axes from inclination, azimuth and position angle (Sect. 2.2; FP64
// on the host).  Sines and cosines within 1e-15 of 0 or +-1 are taken as
// exact, so that the face-on and edge-on frames (angles at multiples of pi/2)
// look exactly along the grid axes.
inline double snap_unit(double v) {
  if (std::fabs(v) < 1e-15) return 0.0;
  if (std::fabs(std::fabs(v) - 1.0) < 1e-15) return v > 0 ? 1.0 : -1.0;
  return v;
}
inline void frame_axes(double inclination, double azimuth, double position_angle, double kobs[3], double ex[3],
                       double ey[3]) {
  const double st = snap_unit(std::sin(inclination)), ct = snap_unit(std::cos(inclination));
  const double sp = snap_unit(std::sin(azimuth)), cp = snap_unit(std::cos(azimuth));
  const double so = snap_unit(std::sin(position_angle)), co = snap_unit(std::cos(position_angle));
  kobs[0] = st * cp; kobs[1] = st * sp; kobs[2] = ct;
  const double a[3] = {-sp, cp, 0.0};
  const double b[3] = {-ct * cp, -ct * sp, st};
  for (int i = 0; i < 3; ++i) {
    ex[i] = co * a[i] - so * b[i];
    ey[i] = so * a[i] + co * b[i];
  }
}

// Message returned by rt_last_error(NULL) (calls without a context).
void set_context_free_error(const char* msg);

// Row-major storage strides (1, nx, nx ny) for p.stride.
inline void row_major_strides(FwdParams& p) {
  p.stride[0] = 1;
  p.stride[1] = p.nx;
  p.stride[2] = p.nx * p.ny;
}

// Storage order of a cartesian or rectilinear grid: the axes sorted by how
// often an isotropic ray crosses their cell faces (cells per unit length,
// n_a / extent_a), most often first (stable: ties keep x, y, z), so that the
// most frequent step of a walk is unit-stride.  Fills strides[3].
void crossing_order_strides(const int n[3], const double extent[3], int strides[3]);

// Copies between row-major order and the storage order of `strides`
// (rt_layout.cu): a float field into storage order, and n_lambda double
// fields back to row-major.
cudaError_t launch_to_storage(const float* src, float* dst, int nx, int ny, int nz, const int strides[3],
                              cudaStream_t stream);
cudaError_t launch_from_storage(const double* src, double* dst, int n_lambda, int nx, int ny, int nz,
                                const int strides[3], cudaStream_t stream);

// Panchromatic mode (rt_dust.cu): equilibrium temperatures T [n_cells] from
// the absorbed luminosity (stored = 1: the context's tallies in the storage
// order of `stride`; 0: a row-major [n_lambda][n_cells] field), and the
// thermal emission lum [n_lambda][n_cells] with its running sums cum over the
// cells (tile_sum: n_lambda * dust_tiles(n_cells) doubles).  planes: FP64
// cell planes x, y, z; w: S kappa_l (1 - albedo_l) dlambda_l; lambda in um.
cudaError_t launch_dust_temperature(int n_lambda, int nx, int ny, int nz, const int stride[3], const double* planes,
                                    const float* density, const double* w, const double* lambda,
                                    const double* absorbed, int stored, double t_min, double t_max, double* T,
                                    unsigned* clamped, cudaStream_t s);
cudaError_t launch_dust_emission(int n_lambda, int nx, int ny, int nz, const int stride[3], const double* planes,
                                 const float* density, const double* w, const double* lambda, const double* T,
                                 double* lum, double* cum, double* tile_sum, cudaStream_t s);
long long dust_tiles(long long n_cells);

// Launchers (rt_forward.cu).
cudaError_t launch_forward(const FwdParams& p, int grid_kind, int num_sms, cudaStream_t stream);
// Per-line suffix sums for peel-offs along axis `axis` in direction dir
// (+1 / -1): out[c] = sum over the cells j beyond c on c's grid line of
// rho_j d_j, accumulated in FP64 from the boundary (rt_forward.cu); d_j = d,
// or the width between the FP64 planes of the axis when `planes` is given.
cudaError_t launch_columns(const float* density, int nx, int ny, int nz, int axis, int dir, float d,
                           const double* planes, float* out, cudaStream_t stream);
cudaError_t launch_forward_octree(const FwdParams& p, int num_sms, cudaStream_t stream);
cudaError_t launch_forward_rect(const FwdParams& p, int num_sms, cudaStream_t stream);
cudaError_t launch_forward_bintree(const FwdParams& p, int num_sms, cudaStream_t stream);
cudaError_t launch_forward_voronoi(const FwdParams& p, int num_sms, cudaStream_t stream);
// The sorted peel-off pass after a forward launch with p.peel set
// (rt_forward.cu): scan of p.peel_hist (n_keys entries, tile totals in
// tile_sum: (n_keys + 4095) / 4096 entries), the permutation that orders the
// records by key (perm: p.peel_cap entries), and the walks and deposits.
// `mid`, if not null, is recorded on the stream between the ordering and the
// walks.
cudaError_t launch_peel_pass(const FwdParams& p, unsigned long long n_keys, unsigned* tile_sum, unsigned* perm,
                             int num_sms, cudaStream_t stream, cudaEvent_t mid);
// One forced path of a packet in the adjoint (rt_adjoint.cu): what the
// backward sweep and the path's depositing walk need.  Adjoint quantities are
// FP32 in exact power-of-two units: weights in 2^e0 (e0 the exponent of the
// packet's initial weight), adjoints of weights in 2^ea (ea the exponent of
// the largest adjoint input), adjoints of positions and optical depths in
// 2^(e0 + ea).
struct alignas(32) AdjRecord {
  // sectors 0-1: written when the path's first walk ends
  float x[3], k[3];    // start of the path (the previous event's position) and its direction
  int cell;            // linear cell of the start (-1: located by the walk)
  float L;             // weight at the start
  float omE, E, u;     // 1 - exp(-tau_path), exp(-tau_path), the inversion uniform
  float g1[3];         // plane sums of the whole path: sum over segments of kr (e_exit - e_entry)
  float pad0, pad1;
  // sector 2: written at the interaction
  int h;               // crossing index of the interaction segment
  int hit_axis;        // axis of the plane entering segment h (-1 when h = 0)
  int hit_cell;        // cell of the interaction
  float kr_h;          // kappa rho of the interaction cell
  float rem;           // tau* - tau_{h-1}
  float gp[3];         // the plane sums of the segments before h (those from h on: g1 - gp)
  // sector 3: the adjoint's
  float dLb, dxb[3];   // peel-offs at the interaction: adjoints of its weight and position
  float T, tbh;        // from the sweep: total tau-adjoint of the path, adjoint of tau_{h-1}
  float pad2, pad3;
  // sector 4: with an absorption adjoint
  float g0[3];         // plane sums weighted by the deposit-adjoint prefix
  float D, Tdep;       // sum a_m (e_{m-1} - e_m); sum of the deposit tau-adjoints
  float pad4[3];
};
static_assert(sizeof(AdjRecord) == 160, "AdjRecord layout: five 32-byte sectors");
// The fields are grouped by writer in whole 32-byte sectors, so that the
// forward launch recording the tape writes full sectors and never reads one.
// Record 0 of a packet on the tape: h = the packet's last event J, x / cell
// / L = its position, cell and weight after event J (records 1..J are its
// forced paths, as in the adjoint's own replay).
constexpr int kMaxAdjointEvents = 256;

// One model of a batch (rt_batch.cu): cartesian grid, one wavelength, one
// point source, one single-channel frame.
struct DevModel {
  int nx, ny, nz, pad0;
  float lo[3], hi[3], d[3], inv_d[3];  // as FwdParams
  float kappa, g;
  float src[3];                        // point source position
  int pad1;
  double albedo;
  double L0;                           // packet weight: luminosity / packets
  long long density;                   // offset of the model's densities in the batch buffer
  DevInstr instr;                      // its frame; image = the model's image [ny][nx]
};
// A run of packets [first, first + count) of one model; the work list is
// sorted by estimated cost, largest first.
struct BatchChunk {
  unsigned long long first;
  int model;
  unsigned count;
};
struct BatchParams {
  const DevModel* models;
  const BatchChunk* chunks;
  int n_models, n_chunks;
  const float* density;
  double* tallies;                     // [n_models][4]: emitted (host side), escaped, absorbed, truncated
  unsigned long long* chunk_counter;
  unsigned long long* counters;        // [6]: crossings, events, peel-offs, packets, column peel-offs,
                                       //      their crossings
  int* flags;
  double w_min;
  unsigned seed;
  int max_events, weight_cut, peel_emission, peel_scatter, control_min;
  int use_columns;                     // frames along grid axes use the models' column sums
};
constexpr int kBatchBlock = 256;
// The batch kernel and the per-launch emitted-tally kernel (graph nodes:
// k_batch(BatchParams), k_batch_emitted(double* tallies, const double* lum,
// int n)), the batch kernel's resident blocks per SM, and a plain launch.
const void* batch_kernel();
const void* batch_emitted_kernel();
// k_batch_columns(const DevModel* models, int n_models, const float* density):
// the column sums of every model whose frame looks along a grid axis.
const void* batch_columns_kernel();
cudaError_t batch_blocks_per_sm(int* blocks);
cudaError_t launch_batch(const BatchParams& p, unsigned blocks, cudaStream_t stream);
cudaError_t launch_batch_columns(const DevModel* models, int n_models, const float* density, cudaStream_t stream);

// Lanes (threads) of the adjoint launch for n_total packets; the record
// buffer holds lanes * (max_events + 1) records.
cudaError_t adjoint_lanes(int num_sms, unsigned long long n_total, unsigned long long* lanes);
// adj_img[q]: FP64 adjoint images of img_elems[q] elements (or null);
// img_f: FP32 scratch of sum img_elems elements; maxbits: one device word.
cudaError_t launch_adjoint(const FwdParams& f, const double* const* adj_img, const size_t* img_elems,
                           const double* adj_abs, double* grad, AdjRecord* recs, unsigned long long lanes,
                           unsigned long long* counters, float* img_f, unsigned long long* maxbits,
                           double* const* line_dep, AdjRecord* tape, cudaStream_t stream);

}  // namespace rtk

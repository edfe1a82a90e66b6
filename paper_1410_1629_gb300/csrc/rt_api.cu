// Host side of the C ABI declared in include/rt.h: context and device-memory
// management, argument validation, uploads, launches and read-back.
//
// The call sequence follows the simulation phases of the SKIRT paper
// (Sect. 3.2: construction, setup, run): the grid, optics, sources and
// instruments are copied to the device once (setup); rt_launch_packets runs
// packets (run); rt_read_* return the tallies.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "rt_internal.h"

namespace rtk {
// Zero entries after the Voronoi neighbour and face arrays (the walk reads
// lists in batches of three).
constexpr long long kVorPad = 2;
// rt_layout.cu: n doubles from device memory to memory the device addresses.
cudaError_t launch_copy_f64(const double* src, double* dst, long long n, cudaStream_t stream);
}  // namespace rtk

using namespace rtk;

namespace {

struct HostSource {
  rt_source_desc desc;
  std::vector<double> lum;
};

struct HostInstr {
  rt_instrument_desc desc;
  double* d_image = nullptr;
  size_t n_elems = 0;
};

thread_local std::string g_create_error;

}  // namespace

void rtk::set_context_free_error(const char* msg) { g_create_error = msg ? msg : ""; }

// A batch of small models (rt_batch_*).
struct Batch {
  int n_models = 0;
  std::vector<double> lum;                    // per model
  std::vector<unsigned long long> n_packets;  // per model
  std::vector<double> cost;                   // estimated work per packet, per model
  std::vector<size_t> img_off, img_elems;     // per model, in doubles
  size_t img_total = 0;
  float* d_density = nullptr;
  float* d_columns = nullptr;                 // column sums, parallel to d_density (or null)
  DevModel* d_models = nullptr;
  BatchChunk* d_chunks = nullptr;
  int n_chunks = 0;
  unsigned run_packets = 0;                   // packets per work-list run
  int control_lanes = 0;                      // chosen by rt_batch_tune (0: none)
  double* d_images = nullptr;
  double* d_tallies = nullptr;                // [n][4]
  double* d_lum = nullptr;
  unsigned long long* d_chunk_counter = nullptr;
  unsigned long long* d_counters = nullptr;   // [4]
  int* d_flags = nullptr;
  unsigned blocks = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t kernel_node = nullptr;
};

struct rt_ctx_s {
  int device = 0;
  int num_sms = 0;
  int pageable_access = 0;  // the device reaches pageable host memory (cudaDevAttrPageableMemoryAccess)
  std::string err;
  // grid
  bool has_grid = false;
  int grid_kind = 0;
  int nx = 0, ny = 0, nz = 0;
  double bounds[6] = {0};
  long long n_cells = 0;
  long long n_nodes = 0;
  float* d_density = nullptr;
  int32_t* d_child = nullptr;
  float* d_edges = nullptr;  // rectilinear grids: FP32 edges, x then y then z (nx + ny + nz + 3)
  // Voronoi grids: sites, face offsets, face planes (neighbour ids in
  // d_child, n_nodes faces), bucket seeds
  float4* d_site = nullptr;
  int* d_face_off = nullptr;
  float4* d_face = nullptr;
  int* d_bucket_seed = nullptr;
  int vb_n[3] = {1, 1, 1};
  bool oct_exact = false;  // octree boxes exact binary fractions (FwdParams::oct_exact)
  int oct_depth = 0;       // octrees: the deepest leaf's depth
  // k-d trees: leaf ropes [n_cells][6] and node boxes [n_nodes][2] (FwdParams)
  int32_t* d_rope = nullptr;
  float4* d_node_box = nullptr;
  // storage order of cartesian and rectilinear grids (crossing_order_strides):
  // the density copy the forward kernels read and the order of the absorption
  // tallies; permuted = not row-major
  int stride[3] = {1, 0, 0};
  bool permuted = false;
  float* d_density_s = nullptr;
  double* d_abs_tmp = nullptr;  // one wavelength of row-major absorption, for read-outs to host memory
  double* d_planes64 = nullptr; // FP64 cell planes x, y, z (cartesian and rectilinear grids)
  // panchromatic mode: wavelengths (um), the dust temperatures and thermal
  // emission [n_lambda][n_cells] with its running sums, their per-wavelength
  // totals, and whether launches may emit from the dust
  std::vector<double> lambda_um;
  double* d_dust_T = nullptr;
  double* d_dust_lum = nullptr;
  double* d_dust_cum = nullptr;
  double* d_dust_tiles = nullptr;
  unsigned* d_dust_clamped = nullptr;
  std::vector<double> dust_total;
  bool dust_ready = false;
  // optics
  int n_lambda = 0;
  std::vector<double> kappa, albedo, g;
  // sources, instruments
  std::vector<HostSource> sources;
  std::vector<HostInstr> instr;
  // device tables and tallies
  double* d_absorption = nullptr;
  DevLambda* d_lam = nullptr;
  DevSource* d_src = nullptr;
  double* d_src_cum = nullptr;
  DevInstr* d_instr = nullptr;
  double* d_stats = nullptr;
  unsigned long long* d_counters = nullptr;
  unsigned long long* d_work = nullptr;
  int* d_flags = nullptr;
  bool tables_dirty = true;
  // per-line suffix sums of the density for frames along the grid axes,
  // index 2 * axis + (direction > 0); rebuilt at every launch that uses them
  float* d_columns[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool columns_used[6] = {false, false, false, false, false, false};
  AdjRecord* d_adj = nullptr;  // adjoint event records, grown on demand
  size_t adj_bytes = 0;
  float* d_adj_img = nullptr;  // FP32 copies of the adjoint images, grown on demand
  double* d_line_dep[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // adjoint, per column table
  size_t adj_img_elems = 0;
  unsigned long long* d_adj_max = nullptr;
  std::vector<Batch*> batches;  // by id; null after rt_batch_destroy
  int control_lanes = 0;        // chosen by rt_tune for launches with control_lanes 0 (0: none)
  int blocks_per_sm = 0;        // chosen by rt_tune for launches with blocks_per_sm 0 (0: as many as fit)
  int adjoint_lanes = 0;        // chosen by rt_adjoint_tune for rt_adjoint (0: none)
  double* d_tune_grad = nullptr;  // rt_adjoint_tune's scratch gradient
  size_t tune_grad_cells = 0;
  // the adjoint tape of the last launch that recorded one, and what it holds
  AdjRecord* d_tape = nullptr;
  size_t tape_bytes = 0;
  bool tape_valid = false;
  unsigned long long tape_n = 0, tape_first = 0, tape_seed = 0, tape_norm = 0;
  int tape_max_events = 0, tape_weight_cut = 0, tape_peel_e = 0, tape_peel_s = 0, tape_model = 0;
  double tape_w_min = 0.0;
  // the sorted peel-off pass (cartesian launches): records, their order,
  // counts per sort key and per scan tile, the record counter; the count of
  // the last launch comes back through pinned memory without a wait and sizes
  // the buffer of later launches
  int n_walked_frames = 0;         // instruments without column sums
  PeelRecord* d_peel = nullptr;
  unsigned* d_peel_perm = nullptr;
  unsigned long long peel_cap = 0;
  ulonglong2* d_peel_tag = nullptr;  // packet ids and events, for launches with debug records
  unsigned long long peel_tag_cap = 0;
  unsigned* d_peel_hist = nullptr;
  unsigned* d_peel_tiles = nullptr;
  unsigned long long peel_keys = 0;
  unsigned long long* d_peel_count = nullptr;
  unsigned long long* h_peel_count = nullptr;  // pinned
  cudaEvent_t peel_event = nullptr;
  bool peel_pending = false;
  unsigned long long peel_last_packets = 0;
  double peel_per_packet = 0.0;    // records per packet seen (0: none yet)
  // events around the parts of the last launch made with opts.time_parts:
  // start, after the column sums, after the transport kernel, after the
  // ordering, after the sorted walks
  cudaEvent_t part_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool parts_timed = false;
  double emitted = 0.0;  // luminosity emitted since the last reset (host-side sum)
  // device buffers released by the problem's set-up calls, for reuse
  std::vector<std::pair<void*, size_t>> pool;
  size_t pool_bytes = 0;
};

namespace {

rt_status fail(rt_ctx ctx, rt_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf; else g_create_error = buf;
  return code;
}

rt_status cuda_fail(rt_ctx ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define RT_CUDA(ctx, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Device buffers of the problem (density, absorption, images, column sums)
// that a set-up call releases are kept for the next allocation of the same
// size, so that a problem rebuilt with the same grid, wavelengths and
// instruments (a fitting loop, an end-to-end run) allocates nothing.  At most
// kPoolLimit bytes are kept; an allocation that fails empties the pool and
// tries again.
constexpr size_t kPoolLimit = size_t(16) << 30;

void pool_flush(rt_ctx c) {
  for (auto& b : c->pool) cudaFree(b.first);
  c->pool.clear();
  c->pool_bytes = 0;
}

template <class T>
void pool_release(rt_ctx c, T*& p, size_t bytes) {
  if (!p) return;
  if (bytes == 0 || c->pool_bytes + bytes > kPoolLimit) {
    cudaFree(p);
  } else {
    c->pool.emplace_back(static_cast<void*>(p), bytes);
    c->pool_bytes += bytes;
  }
  p = nullptr;
}

template <class T>
cudaError_t pool_alloc(rt_ctx c, T** p, size_t bytes) {
  for (size_t i = 0; i < c->pool.size(); ++i) {
    if (c->pool[i].second != bytes) continue;
    *p = static_cast<T*>(c->pool[i].first);
    c->pool_bytes -= bytes;
    c->pool.erase(c->pool.begin() + (long)i);
    return cudaSuccess;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation && !c->pool.empty()) {
    cudaGetLastError();
    pool_flush(c);
    e = cudaMalloc(p, bytes);
  }
  return e;
}

rt_status set_device(rt_ctx ctx) {
  RT_CUDA(ctx, cudaSetDevice(ctx->device));
  return RT_OK;
}

void free_grid(rt_ctx c) {
  c->tape_valid = false;
  cudaDeviceSynchronize();  // no kernel may still read the released buffers
  pool_release(c, c->d_density, (size_t)c->n_cells * sizeof(float));
  pool_release(c, c->d_child, (size_t)c->n_nodes * sizeof(int32_t));
  if (c->grid_kind == RT_GRID_BINTREE) {
    pool_release(c, c->d_rope, (size_t)c->n_cells * 6 * sizeof(int32_t));
    pool_release(c, c->d_node_box, (size_t)c->n_nodes * 2 * sizeof(float4));
  }
  pool_release(c, c->d_edges, (size_t)(c->nx + c->ny + c->nz + 3) * sizeof(float));
  if (c->grid_kind == RT_GRID_VORONOI) {
    pool_release(c, c->d_site, (size_t)c->n_cells * sizeof(float4));
    pool_release(c, c->d_face_off, (size_t)(c->n_cells + 1) * sizeof(int));
    pool_release(c, c->d_face, (size_t)c->n_nodes * sizeof(float4));
    pool_release(c, c->d_bucket_seed, (size_t)c->vb_n[0] * c->vb_n[1] * c->vb_n[2] * sizeof(int));
  }
  pool_release(c, c->d_density_s, (size_t)c->n_cells * sizeof(float));
  pool_release(c, c->d_abs_tmp, (size_t)c->n_cells * sizeof(double));
  pool_release(c, c->d_planes64, (size_t)(c->nx + c->ny + c->nz + 3) * sizeof(double));
  pool_release(c, c->d_dust_T, (size_t)c->n_cells * sizeof(double));
  c->permuted = false;
  pool_release(c, c->d_absorption, (size_t)c->n_lambda * c->n_cells * sizeof(double));
  for (auto& p : c->d_columns) pool_release(c, p, (size_t)c->n_cells * sizeof(float));
  for (auto& p : c->d_line_dep) pool_release(c, p, (size_t)c->n_cells * sizeof(double));
  c->tables_dirty = true;
  c->tape_valid = false;
  c->has_grid = false;
}

// Grids whose cells are (ix, iy, iz) between planes: cartesian, rectilinear.
bool indexed_cells(int kind) { return kind == RT_GRID_CARTESIAN || kind == RT_GRID_RECTILINEAR; }

// The grid axis (and direction) a frame looks along exactly, or false.
bool frame_axis(const DevInstr& I, int& axis, int& dir) {
  int n = 0;
  for (int a = 0; a < 3; ++a) {
    if (I.kobs[a] != 0.0f) {
      ++n;
      axis = a;
    }
  }
  if (n != 1 || std::fabs(I.kobs[axis]) != 1.0f) return false;
  dir = I.kobs[axis] > 0.0f ? 1 : -1;
  return true;
}

void free_problem(rt_ctx c) {
  c->tape_valid = false;
  cudaDeviceSynchronize();  // no kernel may still write the released buffers
  for (auto& q : c->instr) pool_release(c, q.d_image, q.n_elems * sizeof(double));
  c->instr.clear();
  c->sources.clear();
  pool_release(c, c->d_absorption, (size_t)c->n_lambda * c->n_cells * sizeof(double));
  pool_release(c, c->d_dust_lum, (size_t)c->n_lambda * c->n_cells * sizeof(double));
  pool_release(c, c->d_dust_cum, (size_t)c->n_lambda * c->n_cells * sizeof(double));
  pool_release(c, c->d_dust_tiles, (size_t)c->n_lambda * dust_tiles(c->n_cells) * sizeof(double));
  c->dust_ready = false;
  c->dust_total.clear();
  c->n_lambda = 0;
  c->tables_dirty = true;
  c->tape_valid = false;
}

rt_status zero_tallies(rt_ctx c, cudaStream_t s) {
  for (auto& q : c->instr) RT_CUDA(c, cudaMemsetAsync(q.d_image, 0, q.n_elems * sizeof(double), s));
  if (c->d_absorption)
    RT_CUDA(c, cudaMemsetAsync(c->d_absorption, 0, (size_t)c->n_lambda * c->n_cells * sizeof(double), s));
  RT_CUDA(c, cudaMemsetAsync(c->d_stats, 0, 4 * sizeof(double), s));
  RT_CUDA(c, cudaMemsetAsync(c->d_counters, 0, 9 * sizeof(unsigned long long), s));
  RT_CUDA(c, cudaMemsetAsync(c->d_flags, 0, sizeof(int), s));
  c->emitted = 0.0;
  return RT_OK;
}

void frame_axes(const rt_instrument_desc& d, double kobs[3], double ex[3], double ey[3]) {
  rtk::frame_axes(d.inclination, d.azimuth, d.position_angle, kobs, ex, ey);
}

// Rebuild the small device tables (per-wavelength optics, sources, instruments).
rt_status upload_tables(rt_ctx c, cudaStream_t s) {
  if (!c->tables_dirty) return RT_OK;
  std::vector<DevLambda> lam((size_t)c->n_lambda);
  for (int l = 0; l < c->n_lambda; ++l) {
    DevLambda& L = lam[l];
    std::memset(&L, 0, sizeof L);
    L.kappa = (float)c->kappa[l];
    L.g = (float)c->g[l];
    L.albedo = c->albedo[l];
    L.one_minus_albedo = 1.0 - c->albedo[l];
    double tot = 0.0;
    for (auto& src : c->sources) tot += src.lum[l];
    L.lum_total = tot;
  }
  const int ns = (int)c->sources.size();
  std::vector<DevSource> src((size_t)ns);
  std::vector<double> cum((size_t)c->n_lambda * ns);
  for (int i = 0; i < ns; ++i) {
    const rt_source_desc& d = c->sources[i].desc;
    std::memset(&src[i], 0, sizeof(DevSource));
    src[i].kind = d.kind;
    for (int a = 0; a < 3; ++a) src[i].center[a] = d.center[a];
    src[i].scale_r = d.scale_r;
    src[i].scale_z = d.scale_z;
  }
  for (int l = 0; l < c->n_lambda; ++l) {
    double tot = 0.0, run = 0.0;
    for (int i = 0; i < ns; ++i) tot += c->sources[i].lum[l];
    for (int i = 0; i < ns; ++i) {
      run += c->sources[i].lum[l];
      cum[(size_t)l * ns + i] = run / tot;
    }
  }
  std::vector<DevInstr> ins(c->instr.size());
  for (size_t q = 0; q < c->instr.size(); ++q) {
    const rt_instrument_desc& d = c->instr[q].desc;
    double kobs[3], ex[3], ey[3];
    frame_axes(d, kobs, ex, ey);
    DevInstr& I = ins[q];
    std::memset(&I, 0, sizeof I);
    for (int a = 0; a < 3; ++a) { I.kobs[a] = (float)kobs[a]; I.ex[a] = (float)ex[a]; I.ey[a] = (float)ey[a]; }
    I.off_x = (float)(d.half_x - d.center_x);
    I.off_y = (float)(d.half_y - d.center_y);
    I.sx = (float)(d.nx / (2.0 * d.half_x));
    I.sy = (float)(d.ny / (2.0 * d.half_y));
    I.nx = d.nx; I.ny = d.ny;
    I.bilinear = d.deposit == RT_DEPOSIT_BILINEAR;
    I.sed = d.deposit == RT_DEPOSIT_SED;
    I.channels = d.channels;
    I.image = c->instr[q].d_image;
    int axis = 0, dir = 0;
    if (indexed_cells(c->grid_kind) && frame_axis(I, axis, dir)) {
      const int k = 2 * axis + (dir > 0 ? 1 : 0);
      if (!c->d_columns[k]) RT_CUDA(c, pool_alloc(c, &c->d_columns[k], (size_t)c->n_cells * sizeof(float)));
      I.column = c->d_columns[k];
      I.axis = axis;
      I.dir = dir;
    }
  }
  for (int k = 0; k < 6; ++k) c->columns_used[k] = false;
  c->n_walked_frames = 0;
  for (const DevInstr& I : ins) {
    if (I.column) c->columns_used[2 * I.axis + (I.dir > 0 ? 1 : 0)] = true;
    else c->n_walked_frames += 1;
  }
  dfree(c->d_lam); dfree(c->d_src); dfree(c->d_src_cum); dfree(c->d_instr);
  RT_CUDA(c, cudaMalloc(&c->d_lam, std::max<size_t>(1, lam.size()) * sizeof(DevLambda)));
  RT_CUDA(c, cudaMalloc(&c->d_src, std::max<size_t>(1, src.size()) * sizeof(DevSource)));
  RT_CUDA(c, cudaMalloc(&c->d_src_cum, std::max<size_t>(1, cum.size()) * sizeof(double)));
  RT_CUDA(c, cudaMalloc(&c->d_instr, std::max<size_t>(1, ins.size()) * sizeof(DevInstr)));
  // synchronous copies: the host vectors go out of scope on return
  if (!lam.empty()) RT_CUDA(c, cudaMemcpy(c->d_lam, lam.data(), lam.size() * sizeof(DevLambda), cudaMemcpyHostToDevice));
  if (!src.empty()) RT_CUDA(c, cudaMemcpy(c->d_src, src.data(), src.size() * sizeof(DevSource), cudaMemcpyHostToDevice));
  if (!cum.empty()) RT_CUDA(c, cudaMemcpy(c->d_src_cum, cum.data(), cum.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (!ins.empty()) RT_CUDA(c, cudaMemcpy(c->d_instr, ins.data(), ins.size() * sizeof(DevInstr), cudaMemcpyHostToDevice));
  (void)s;
  c->tables_dirty = false;
  return RT_OK;
}

bool is_finite(double v) { return std::isfinite(v); }

// The FP64 planes of one axis (cartesian and rectilinear grids).
const double* axis_planes(rt_ctx c, int axis) {
  return c->d_planes64 + (axis == 0 ? 0 : (axis == 1 ? c->nx + 1 : c->nx + c->ny + 2));
}

void free_batch(Batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  dfree(b->d_density); dfree(b->d_columns); dfree(b->d_models); dfree(b->d_chunks); dfree(b->d_images); dfree(b->d_tallies);
  dfree(b->d_lum); dfree(b->d_chunk_counter); dfree(b->d_counters); dfree(b->d_flags);
  delete b;
}

Batch* get_batch(rt_ctx c, int32_t id) {
  if (id < 0 || (size_t)id >= c->batches.size()) return nullptr;
  return c->batches[(size_t)id];
}

// Work list: every model's packets in runs of at most run_packets (models
// with fewer packets in one run), sorted by estimated cost, largest first.
std::vector<BatchChunk> batch_chunks(const Batch& b, unsigned run_packets, double fraction) {
  std::vector<BatchChunk> out;
  std::vector<double> cost;
  for (int m = 0; m < b.n_models; ++m) {
    unsigned long long n = b.n_packets[(size_t)m];
    if (fraction < 1.0) n = std::max<unsigned long long>(1, (unsigned long long)std::ceil((double)n * fraction));
    for (unsigned long long f = 0; f < n; f += run_packets) {
      BatchChunk ch;
      ch.first = f;
      ch.model = m;
      ch.count = (unsigned)std::min<unsigned long long>(run_packets, n - f);
      out.push_back(ch);
      cost.push_back(b.cost[(size_t)m] * ch.count);
    }
  }
  std::vector<size_t> order(out.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return cost[a] > cost[c]; });
  std::vector<BatchChunk> sorted(out.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = out[order[i]];
  return sorted;
}

rt_status upload_chunks(rt_ctx c, Batch* b, unsigned run_packets) {
  const std::vector<BatchChunk> ch = batch_chunks(*b, run_packets, 1.0);
  dfree(b->d_chunks);
  RT_CUDA(c, cudaMalloc(&b->d_chunks, std::max<size_t>(1, ch.size()) * sizeof(BatchChunk)));
  RT_CUDA(c, cudaMemcpy(b->d_chunks, ch.data(), ch.size() * sizeof(BatchChunk), cudaMemcpyHostToDevice));
  b->n_chunks = (int)ch.size();
  b->run_packets = run_packets;
  return RT_OK;
}

rt_status batch_opts(rt_ctx c, const rt_launch_opts* opts, uint64_t seed, rt_launch_opts& o) {
  rt_default_opts(&o);
  if (opts) o = *opts;
  if (seed >> 32) return fail(c, RT_ERR_ARG, "rt_batch: seed must be < 2^32");
  if (o.max_events < 1) return fail(c, RT_ERR_ARG, "rt_batch: max_events must be >= 1");
  if (!(o.w_min >= 0 && o.w_min < 1)) return fail(c, RT_ERR_ARG, "rt_batch: w_min must be in [0, 1)");
  if (o.control_lanes < 0 || o.control_lanes > 32) return fail(c, RT_ERR_ARG, "rt_batch: control_lanes in [0, 32]");
  return RT_OK;
}

BatchParams batch_params(const Batch* b, const rt_launch_opts& o, uint64_t seed, const BatchChunk* chunks,
                         int n_chunks) {
  BatchParams p;
  std::memset(&p, 0, sizeof p);
  p.models = b->d_models;
  p.chunks = chunks;
  p.n_models = b->n_models;
  p.n_chunks = n_chunks;
  p.density = b->d_density;
  p.tallies = b->d_tallies;
  p.chunk_counter = b->d_chunk_counter;
  p.counters = b->d_counters;
  p.flags = b->d_flags;
  p.w_min = o.w_min;
  p.seed = (unsigned)seed;
  p.max_events = o.max_events;
  p.weight_cut = o.weight_cut;
  p.peel_emission = o.peel_emission;
  p.peel_scatter = o.peel_scatter;
  p.control_min = o.control_lanes ? o.control_lanes : (b->control_lanes ? b->control_lanes : 16);
  p.use_columns = !o.walk_peels;
  return p;
}

// The launch graph: zero the work counter, add the emitted luminosity and
// rebuild the column sums, then the persistent kernel.
rt_status build_graph(rt_ctx c, Batch* b, const BatchParams& p) {
  RT_CUDA(c, cudaGraphCreate(&b->graph, 0));
  cudaMemsetParams mp;
  std::memset(&mp, 0, sizeof mp);
  mp.dst = b->d_chunk_counter;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 2;
  mp.height = 1;
  cudaGraphNode_t n_zero, n_emit;
  RT_CUDA(c, cudaGraphAddMemsetNode(&n_zero, b->graph, nullptr, 0, &mp));
  double* tallies = b->d_tallies;
  const double* lum = b->d_lum;
  int n = b->n_models;
  void* eargs[] = {&tallies, &lum, &n};
  cudaKernelNodeParams ep;
  std::memset(&ep, 0, sizeof ep);
  ep.func = const_cast<void*>(batch_emitted_kernel());
  ep.gridDim = dim3((unsigned)((n + 255) / 256));
  ep.blockDim = dim3(256);
  ep.kernelParams = eargs;
  RT_CUDA(c, cudaGraphAddKernelNode(&n_emit, b->graph, nullptr, 0, &ep));
  const DevModel* models = b->d_models;
  const float* dens = b->d_density;
  void* cargs[] = {&models, &n, &dens};
  cudaKernelNodeParams cp;
  std::memset(&cp, 0, sizeof cp);
  cp.func = const_cast<void*>(batch_columns_kernel());
  cp.gridDim = dim3((unsigned)n);
  cp.blockDim = dim3(128);
  cp.kernelParams = cargs;
  cudaGraphNode_t n_cols;
  RT_CUDA(c, cudaGraphAddKernelNode(&n_cols, b->graph, nullptr, 0, &cp));
  BatchParams pc = p;
  void* kargs[] = {&pc};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof kp);
  kp.func = const_cast<void*>(batch_kernel());
  kp.gridDim = dim3(b->blocks);
  kp.blockDim = dim3(kBatchBlock);
  kp.kernelParams = kargs;
  cudaGraphNode_t deps[3] = {n_zero, n_emit, n_cols};
  RT_CUDA(c, cudaGraphAddKernelNode(&b->kernel_node, b->graph, deps, 3, &kp));
  RT_CUDA(c, cudaGraphInstantiate(&b->exec, b->graph, 0));
  return RT_OK;
}

}  // namespace

extern "C" {

const char* rt_version(void) { return "rt_gb300 1.0 (sm_103a)"; }

rt_status rt_context_create(int32_t device, rt_ctx* out) {
  if (!out) return fail(nullptr, RT_ERR_ARG, "rt_context_create: out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return fail(nullptr, RT_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  if (device < 0 || device >= n) return fail(nullptr, RT_ERR_ARG, "device %d out of range [0, %d)", device, n);
  rt_ctx c = new (std::nothrow) rt_ctx_s();
  if (!c) return fail(nullptr, RT_ERR_OOM, "host allocation failed");
  c->device = device;
  e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->pageable_access, cudaDevAttrPageableMemoryAccess, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_stats, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_counters, 9 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_work, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_flags, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, 9 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_flags, 0, sizeof(int));
  if (e != cudaSuccess) {
    rt_context_destroy(c);
    return fail(nullptr, RT_ERR_CUDA, "context set-up: %s", cudaGetErrorString(e));
  }
  *out = c;
  return RT_OK;
}

rt_status rt_context_destroy(rt_ctx c) {
  if (!c) return RT_OK;
  cudaSetDevice(c->device);
  for (size_t i = 0; i < c->batches.size(); ++i) rt_batch_destroy(c, (int32_t)i);
  free_problem(c);
  free_grid(c);
  pool_flush(c);
  dfree(c->d_lam); dfree(c->d_src); dfree(c->d_src_cum); dfree(c->d_instr);
  dfree(c->d_stats); dfree(c->d_counters); dfree(c->d_work); dfree(c->d_flags);
  dfree(c->d_adj); dfree(c->d_adj_img); dfree(c->d_adj_max); dfree(c->d_tune_grad); dfree(c->d_tape);
  for (auto& p : c->d_line_dep) dfree(p);
  dfree(c->d_peel); dfree(c->d_peel_perm); dfree(c->d_peel_hist); dfree(c->d_peel_tiles); dfree(c->d_peel_count);
  dfree(c->d_peel_tag);
  if (c->h_peel_count) cudaFreeHost(c->h_peel_count);
  if (c->peel_event) cudaEventDestroy(c->peel_event);
  for (auto& e : c->part_ev)
    if (e) cudaEventDestroy(e);
  delete c;
  return RT_OK;
}

const char* rt_last_error(rt_ctx c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void rt_default_opts(rt_launch_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->w_min = 1e-4;
  o->max_events = 1000;
  o->weight_cut = 1;
  o->peel_emission = 1;
  o->peel_scatter = 1;
}

namespace {

// Whether every box of an octree of depth dmax over `bounds` has corners
// that FP32 represents exactly, with exact halvings and doublings: on each
// axis the finest box size q = extent / 2^dmax is an FP32 number, the lower
// bound an integer multiple n0 q, and (|n0| + 2^dmax) c < 2^23 for q = c 2^e
// with c odd (every corner is then n c 2^e, and sums of two corners stay
// below 2^24 c 2^e).
bool octree_boxes_exact(const double bounds[6], int dmax) {
  for (int a = 0; a < 3; ++a) {
    const double lo = bounds[2 * a], hi = bounds[2 * a + 1], ext = hi - lo;
    const double q = std::ldexp(ext, -dmax);
    if ((double)(float)q != q || std::ldexp(q, dmax) != ext || lo + ext != hi) return false;
    const double n0 = lo / q;
    if (n0 != std::floor(n0) || n0 * q != lo) return false;
    int e = 0;
    const double m = std::frexp(q, &e);
    unsigned long long cq = (unsigned long long)std::ldexp(m, 53);
    while (cq && !(cq & 1ull)) cq >>= 1;
    if (!((std::fabs(n0) + std::ldexp(1.0, dmax)) * (double)cq < 8388608.0)) return false;
  }
  return true;
}

}  // namespace

rt_status rt_create_grid(rt_ctx c, const rt_grid_desc* d, int32_t* grid_id) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!d || !d->density) return fail(c, RT_ERR_ARG, "rt_create_grid: null descriptor or density");
  for (int a = 0; a < 3; ++a)
    if (!(is_finite(d->bounds[2 * a]) && is_finite(d->bounds[2 * a + 1]) && d->bounds[2 * a] < d->bounds[2 * a + 1]))
      return fail(c, RT_ERR_ARG, "rt_create_grid: bounds on axis %d are not increasing", a);
  long long n_cells = 0, n_nodes = 0;
  std::vector<float> edges_f;
  if (d->kind == RT_GRID_CARTESIAN || d->kind == RT_GRID_RECTILINEAR) {
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0) return fail(c, RT_ERR_ARG, "rt_create_grid: cell counts must be > 0");
    n_cells = (long long)d->nx * d->ny * d->nz;
    if (n_cells > (1ll << 31) - 1) return fail(c, RT_ERR_ARG, "rt_create_grid: more than 2^31-1 cells");
  }
  if (d->kind == RT_GRID_RECTILINEAR) {
    // the edges: strictly increasing in FP64 and in FP32, ends equal to the bounds
    const int n3[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) {
      if (!d->edges[a]) return fail(c, RT_ERR_ARG, "rt_create_grid: rectilinear grid without edges on axis %d", a);
      std::vector<double> e((size_t)n3[a] + 1);
      if (d->on_device) {
        if (set_device(c) != RT_OK) return RT_ERR_CUDA;
        RT_CUDA(c, cudaMemcpy(e.data(), d->edges[a], e.size() * sizeof(double), cudaMemcpyDeviceToHost));
      } else {
        std::memcpy(e.data(), d->edges[a], e.size() * sizeof(double));
      }
      if (e.front() != d->bounds[2 * a] || e.back() != d->bounds[2 * a + 1])
        return fail(c, RT_ERR_ARG, "rt_create_grid: edges on axis %d do not end at the bounds", a);
      for (size_t i = 0; i < e.size(); ++i) {
        if (!is_finite(e[i]) || (i > 0 && !(e[i] > e[i - 1] && (float)e[i] > (float)e[i - 1])))
          return fail(c, RT_ERR_ARG, "rt_create_grid: edges on axis %d not strictly increasing (in FP32) at %zu", a, i);
        edges_f.push_back((float)e[i]);
      }
    }
  } else if (d->kind == RT_GRID_CARTESIAN) {
  } else if (d->kind == RT_GRID_OCTREE || d->kind == RT_GRID_BINTREE) {
    if (!d->child || d->n_nodes <= 0 || d->n_leaves <= 0)
      return fail(c, RT_ERR_ARG, "rt_create_grid: a tree needs child[] and counts > 0");
    if (d->kind == RT_GRID_BINTREE && !d->split_axis)
      return fail(c, RT_ERR_ARG, "rt_create_grid: a k-d tree needs split_axis[]");
    const long long limit = d->kind == RT_GRID_BINTREE ? (1ll << 29) - 2 : (1ll << 31) - 1;
    if (d->n_nodes > limit || d->n_leaves > (1ll << 31) - 1)
      return fail(c, RT_ERR_ARG, "rt_create_grid: tree too large for int32 indices");
    n_cells = d->n_leaves;
    n_nodes = d->n_nodes;
  } else if (d->kind == RT_GRID_VORONOI) {
    if ((!d->child && d->n_nodes > 0) || !d->sites || !d->offsets || d->n_leaves <= 0 || d->n_nodes < 0)
      return fail(c, RT_ERR_ARG, "rt_create_grid: a Voronoi grid needs sites[], offsets[], child[] and n_leaves > 0");
    if (d->n_leaves > (1ll << 31) - 2 || d->n_nodes > (1ll << 31) - 1)
      return fail(c, RT_ERR_ARG, "rt_create_grid: Voronoi grid too large for int32 indices");
    n_cells = d->n_leaves;
    n_nodes = d->n_nodes;
  } else {
    return fail(c, RT_ERR_ARG, "rt_create_grid: unknown grid kind %d", d->kind);
  }
  // Voronoi grids: sites and lists checked on the host; per face the unit
  // normal towards the neighbour and the distance of the bisecting plane
  // from the site (FP64, stored FP32); per bucket the nearest site to its
  // centre, by greedy descent from the previous bucket's
  std::vector<float4> vor_site, vor_face;
  std::vector<int> vor_off, vor_seed;
  int vb_n[3] = {1, 1, 1};
  if (d->kind == RT_GRID_VORONOI) {
    std::vector<double> site((size_t)n_cells * 3);
    std::vector<int64_t> off((size_t)n_cells + 1);
    std::vector<int32_t> nbr((size_t)n_nodes);
    if (d->on_device) {
      if (set_device(c) != RT_OK) return RT_ERR_CUDA;
      RT_CUDA(c, cudaMemcpy(site.data(), d->sites, site.size() * sizeof(double), cudaMemcpyDeviceToHost));
      RT_CUDA(c, cudaMemcpy(off.data(), d->offsets, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
      if (n_nodes > 0) RT_CUDA(c, cudaMemcpy(nbr.data(), d->child, nbr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(site.data(), d->sites, site.size() * sizeof(double));
      std::memcpy(off.data(), d->offsets, off.size() * sizeof(int64_t));
      if (n_nodes > 0) std::memcpy(nbr.data(), d->child, nbr.size() * sizeof(int32_t));
    }
    if (off[0] != 0 || off[(size_t)n_cells] != n_nodes)
      return fail(c, RT_ERR_ARG, "rt_create_grid: Voronoi offsets must run from 0 to n_nodes");
    for (long long i = 0; i < n_cells; ++i) {
      for (int a = 0; a < 3; ++a) {
        const double v = site[(size_t)(3 * i + a)];
        if (!(is_finite(v) && v >= d->bounds[2 * a] && v <= d->bounds[2 * a + 1]))
          return fail(c, RT_ERR_ARG, "rt_create_grid: Voronoi site %lld outside the domain", i);
      }
      if (off[(size_t)i + 1] < off[(size_t)i])
        return fail(c, RT_ERR_ARG, "rt_create_grid: Voronoi offsets decrease at %lld", i);
    }
    vor_site.resize((size_t)n_cells);
    for (long long i = 0; i < n_cells; ++i)
      vor_site[(size_t)i] = make_float4((float)site[(size_t)(3 * i)], (float)site[(size_t)(3 * i + 1)],
                                        (float)site[(size_t)(3 * i + 2)], 0.0f);
    vor_off.resize((size_t)n_cells + 1);
    vor_face.resize((size_t)n_nodes);
    for (long long i = 0; i < n_cells; ++i) {
      vor_off[(size_t)i] = (int)off[(size_t)i];
      const double* si = &site[(size_t)(3 * i)];
      for (int64_t f = off[(size_t)i]; f < off[(size_t)i + 1]; ++f) {
        const long long j = nbr[(size_t)f];
        if (j < 0 || j >= n_cells || j == i)
          return fail(c, RT_ERR_ARG, "rt_create_grid: Voronoi cell %lld lists neighbour %lld", i, j);
        const double* sj = &site[(size_t)(3 * j)];
        const double v[3] = {sj[0] - si[0], sj[1] - si[1], sj[2] - si[2]};
        const double len = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(len > 0.0)) return fail(c, RT_ERR_ARG, "rt_create_grid: Voronoi sites %lld and %lld coincide", i, j);
        vor_face[(size_t)f] = make_float4((float)(v[0] / len), (float)(v[1] / len), (float)(v[2] / len),
                                          (float)(0.5 * len));
      }
    }
    vor_off[(size_t)n_cells] = (int)n_nodes;
    // buckets: about one per two sites, cubic in shape, at most 256 per axis
    const double ext[3] = {d->bounds[1] - d->bounds[0], d->bounds[3] - d->bounds[2], d->bounds[5] - d->bounds[4]};
    const double h = std::cbrt(ext[0] * ext[1] * ext[2] / std::max(1.0, 0.5 * (double)n_cells));
    for (int a = 0; a < 3; ++a) vb_n[a] = (int)std::min(256.0, std::max(1.0, std::round(ext[a] / h)));
    vor_seed.resize((size_t)vb_n[0] * vb_n[1] * vb_n[2]);
    long long cur = 0;
    for (int k = 0; k < vb_n[2]; ++k)
      for (int j = 0; j < vb_n[1]; ++j)
        for (int i = 0; i < vb_n[0]; ++i) {
          const double q[3] = {d->bounds[0] + (i + 0.5) * ext[0] / vb_n[0], d->bounds[2] + (j + 0.5) * ext[1] / vb_n[1],
                               d->bounds[4] + (k + 0.5) * ext[2] / vb_n[2]};
          auto d2 = [&](long long s) {
            const double* p = &site[(size_t)(3 * s)];
            return (p[0] - q[0]) * (p[0] - q[0]) + (p[1] - q[1]) * (p[1] - q[1]) + (p[2] - q[2]) * (p[2] - q[2]);
          };
          long long steps = 0;
          for (;; ++steps) {
            if (steps > n_cells) return fail(c, RT_ERR_ARG, "rt_create_grid: Voronoi neighbour lists inconsistent");
            double best = d2(cur);
            long long move = -1;
            for (int64_t f = off[(size_t)cur]; f < off[(size_t)cur + 1]; ++f) {
              const double dj = d2(nbr[(size_t)f]);
              if (dj < best) { best = dj; move = nbr[(size_t)f]; }
            }
            if (move < 0) break;
            cur = move;
          }
          vor_seed[(size_t)i + (size_t)vb_n[0] * ((size_t)j + (size_t)vb_n[1] * k)] = (int)cur;
        }
  }
  std::vector<int32_t> child_host;
  std::vector<int32_t> rope_host;     // k-d trees: leaf ropes
  std::vector<float4> node_box_host;  // k-d trees: node boxes
  int oct_depth = 0;  // octrees: the deepest leaf's depth
  if (d->kind == RT_GRID_OCTREE || d->kind == RT_GRID_BINTREE) {
    // validate the tree on the host: every child block in range (after its
    // parent), every leaf id in range, k-d tree split axes 0..2; k-d tree
    // nodes go to the device as (first child << 2) | axis
    const bool bin = d->kind == RT_GRID_BINTREE;
    const long long kids = bin ? 2 : 8;
    child_host.resize((size_t)n_nodes);
    std::vector<int8_t> axis_host(bin ? (size_t)n_nodes : 0);
    if (d->on_device) {
      if (set_device(c) != RT_OK) return RT_ERR_CUDA;
      RT_CUDA(c, cudaMemcpy(child_host.data(), d->child, n_nodes * sizeof(int32_t), cudaMemcpyDeviceToHost));
      if (bin) RT_CUDA(c, cudaMemcpy(axis_host.data(), d->split_axis, (size_t)n_nodes, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(child_host.data(), d->child, n_nodes * sizeof(int32_t));
      if (bin) std::memcpy(axis_host.data(), d->split_axis, (size_t)n_nodes);
    }
    std::vector<int> node_depth(bin ? 0 : (size_t)n_nodes, 0);
    std::vector<unsigned char> leaf_seen((size_t)n_cells, 0);
    long long leaves_found = 0;
    for (long long i = 0; i < n_nodes; ++i) {
      const long long v = child_host[i];
      if (v >= 0 && (v <= i || v + kids > n_nodes))
        return fail(c, RT_ERR_ARG, "rt_create_grid: node %lld has child block %lld out of range", i, v);
      if (!bin && v >= 0) {
        for (long long k = 0; k < kids; ++k) node_depth[(size_t)(v + k)] = node_depth[(size_t)i] + 1;
        oct_depth = std::max(oct_depth, node_depth[(size_t)i] + 1);
      }
      if (v < 0 && (-v - 1) >= n_cells)
        return fail(c, RT_ERR_ARG, "rt_create_grid: node %lld has leaf id %lld out of range", i, -v - 1);
      if (v < 0) {
        // every leaf id once: the k-d tree walk keys its ropes by leaf id
        if (leaf_seen[(size_t)(-v - 1)]) return fail(c, RT_ERR_ARG, "rt_create_grid: leaf id %lld appears twice", -v - 1);
        leaf_seen[(size_t)(-v - 1)] = 1;
        ++leaves_found;
      }
      if (bin && v >= 0) {
        if (axis_host[(size_t)i] < 0 || axis_host[(size_t)i] > 2)
          return fail(c, RT_ERR_ARG, "rt_create_grid: node %lld has split axis %d", i, (int)axis_host[(size_t)i]);
        child_host[(size_t)i] = (int32_t)((v << 2) | axis_host[(size_t)i]);
      }
    }
    if (leaves_found != n_cells)
      return fail(c, RT_ERR_ARG, "rt_create_grid: %lld leaves in the tree for n_leaves = %lld", leaves_found, n_cells);
    if (!bin && oct_depth > kMaxOctreeDepth)
      return fail(c, RT_ERR_ARG, "rt_create_grid: octree depth %d above %d", oct_depth, kMaxOctreeDepth);
    if (bin) {
      // node boxes with the device's FP32 halving, and the ropes: going down,
      // the lower child's rope across its upper face on the split axis is the
      // upper child and the other way round; the other faces inherit
      rope_host.assign((size_t)n_cells * 6, -1);
      node_box_host.resize((size_t)n_nodes * 2);
      struct Item {
        long long node;
        float lo[3], hi[3];
        int32_t r[6];
      };
      std::vector<Item> stack;
      Item root;
      root.node = 0;
      for (int a = 0; a < 3; ++a) {
        root.lo[a] = (float)d->bounds[2 * a];
        root.hi[a] = (float)d->bounds[2 * a + 1];
      }
      for (int f = 0; f < 6; ++f) root.r[f] = -1;
      stack.push_back(root);
      while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        node_box_host[2 * (size_t)it.node] = make_float4(it.lo[0], it.lo[1], it.lo[2], 0.0f);
        node_box_host[2 * (size_t)it.node + 1] = make_float4(it.hi[0], it.hi[1], it.hi[2], 0.0f);
        const int32_t v = child_host[(size_t)it.node];
        if (v < 0) {
          for (int f = 0; f < 6; ++f) rope_host[(size_t)(-(long long)v - 1) * 6 + f] = it.r[f];
          continue;
        }
        const int a = v & 3;
        const long long first = (long long)(v >> 2);
        const float mid = 0.5f * (it.lo[a] + it.hi[a]);
        Item lower = it, upper = it;
        lower.node = first;
        lower.hi[a] = mid;
        lower.r[2 * a + 1] = (int32_t)(first + 1);
        upper.node = first + 1;
        upper.lo[a] = mid;
        upper.r[2 * a] = (int32_t)first;
        stack.push_back(lower);
        stack.push_back(upper);
      }
    }
  }
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  free_problem(c);
  free_grid(c);
  const cudaMemcpyKind kind = d->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  RT_CUDA(c, pool_alloc(c, &c->d_density, (size_t)n_cells * sizeof(float)));
  RT_CUDA(c, cudaMemcpy(c->d_density, d->density, (size_t)n_cells * sizeof(float), kind));
  if (d->kind == RT_GRID_RECTILINEAR) {
    RT_CUDA(c, pool_alloc(c, &c->d_edges, edges_f.size() * sizeof(float)));
    RT_CUDA(c, cudaMemcpy(c->d_edges, edges_f.data(), edges_f.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  if (d->kind == RT_GRID_OCTREE || d->kind == RT_GRID_BINTREE) {
    RT_CUDA(c, pool_alloc(c, &c->d_child, (size_t)n_nodes * sizeof(int32_t)));
    RT_CUDA(c, cudaMemcpy(c->d_child, child_host.data(), (size_t)n_nodes * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  if (d->kind == RT_GRID_BINTREE) {
    RT_CUDA(c, pool_alloc(c, &c->d_rope, rope_host.size() * sizeof(int32_t)));
    RT_CUDA(c, cudaMemcpy(c->d_rope, rope_host.data(), rope_host.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    RT_CUDA(c, pool_alloc(c, &c->d_node_box, node_box_host.size() * sizeof(float4)));
    RT_CUDA(c, cudaMemcpy(c->d_node_box, node_box_host.data(), node_box_host.size() * sizeof(float4),
                          cudaMemcpyHostToDevice));
  }
  if (d->kind == RT_GRID_VORONOI) {
    // neighbour ids and face planes with kVorPad zero entries after the last
    // list: the walk loads a cell's list three entries at a time (entries
    // past its end are masked, and the padding keeps them inside the arrays)
    const size_t n_alloc = (size_t)n_nodes + kVorPad;
    RT_CUDA(c, pool_alloc(c, &c->d_child, n_alloc * sizeof(int32_t)));
    RT_CUDA(c, cudaMemset(c->d_child, 0, n_alloc * sizeof(int32_t)));
    if (n_nodes > 0) RT_CUDA(c, cudaMemcpy(c->d_child, d->child, (size_t)n_nodes * sizeof(int32_t), kind));
    RT_CUDA(c, pool_alloc(c, &c->d_site, vor_site.size() * sizeof(float4)));
    RT_CUDA(c, cudaMemcpy(c->d_site, vor_site.data(), vor_site.size() * sizeof(float4), cudaMemcpyHostToDevice));
    RT_CUDA(c, pool_alloc(c, &c->d_face_off, vor_off.size() * sizeof(int)));
    RT_CUDA(c, cudaMemcpy(c->d_face_off, vor_off.data(), vor_off.size() * sizeof(int), cudaMemcpyHostToDevice));
    RT_CUDA(c, pool_alloc(c, &c->d_face, n_alloc * sizeof(float4)));
    RT_CUDA(c, cudaMemset(c->d_face, 0, n_alloc * sizeof(float4)));
    if (n_nodes > 0)
      RT_CUDA(c, cudaMemcpy(c->d_face, vor_face.data(), vor_face.size() * sizeof(float4), cudaMemcpyHostToDevice));
    RT_CUDA(c, pool_alloc(c, &c->d_bucket_seed, vor_seed.size() * sizeof(int)));
    RT_CUDA(c, cudaMemcpy(c->d_bucket_seed, vor_seed.data(), vor_seed.size() * sizeof(int), cudaMemcpyHostToDevice));
    for (int a = 0; a < 3; ++a) c->vb_n[a] = vb_n[a];
  }
  c->grid_kind = d->kind;
  c->oct_exact = d->kind == RT_GRID_OCTREE && oct_depth <= 21 && octree_boxes_exact(d->bounds, oct_depth);
  c->oct_depth = d->kind == RT_GRID_OCTREE ? oct_depth : 0;
  c->nx = d->nx; c->ny = d->ny; c->nz = d->nz;
  c->stride[0] = 1; c->stride[1] = d->nx; c->stride[2] = d->nx * d->ny;
  c->permuted = false;
  if (indexed_cells(d->kind) && d->layout != RT_LAYOUT_ROW_MAJOR) {
    const int n3[3] = {d->nx, d->ny, d->nz};
    const double ext[3] = {d->bounds[1] - d->bounds[0], d->bounds[3] - d->bounds[2], d->bounds[5] - d->bounds[4]};
    crossing_order_strides(n3, ext, c->stride);
    c->permuted = !(c->stride[0] == 1 && c->stride[1] == d->nx);
  }
  if (indexed_cells(d->kind)) {
    // FP64 planes: cartesian lo + i (hi - lo) / n, rectilinear the edges
    std::vector<double> planes;
    const int n3[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) {
      std::vector<double> e((size_t)n3[a] + 1);
      if (d->kind == RT_GRID_RECTILINEAR) {
        if (d->on_device) {
          RT_CUDA(c, cudaMemcpy(e.data(), d->edges[a], e.size() * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
          std::memcpy(e.data(), d->edges[a], e.size() * sizeof(double));
        }
      } else {
        const double lo = d->bounds[2 * a], step = (d->bounds[2 * a + 1] - lo) / n3[a];
        for (int i = 0; i <= n3[a]; ++i) e[(size_t)i] = lo + i * step;
      }
      planes.insert(planes.end(), e.begin(), e.end());
    }
    RT_CUDA(c, pool_alloc(c, &c->d_planes64, planes.size() * sizeof(double)));
    RT_CUDA(c, cudaMemcpy(c->d_planes64, planes.data(), planes.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (c->permuted) {
    RT_CUDA(c, pool_alloc(c, &c->d_density_s, (size_t)n_cells * sizeof(float)));
    RT_CUDA(c, launch_to_storage(c->d_density, c->d_density_s, d->nx, d->ny, d->nz, c->stride, nullptr));
    RT_CUDA(c, cudaStreamSynchronize(nullptr));
  }
  std::memcpy(c->bounds, d->bounds, sizeof c->bounds);
  c->n_cells = n_cells;
  c->n_nodes = d->kind == RT_GRID_VORONOI ? n_nodes + kVorPad : n_nodes;  // as allocated
  c->has_grid = true;
  c->tables_dirty = true;
  c->tape_valid = false;
  if (grid_id) *grid_id = 0;
  return RT_OK;
}

rt_status rt_set_optics(rt_ctx c, int32_t grid_id, int32_t n_lambda, const double* lambda, const double* kappa,
                        const double* albedo, const double* g) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!c->has_grid) return fail(c, RT_ERR_STATE, "rt_set_optics: no grid");
  if (grid_id != 0) return fail(c, RT_ERR_ARG, "rt_set_optics: unknown grid id %d", grid_id);
  if (n_lambda < 1 || n_lambda > kMaxLambda) return fail(c, RT_ERR_ARG, "rt_set_optics: n_lambda must be 1..%d", kMaxLambda);
  if (!kappa || !albedo || !g) return fail(c, RT_ERR_ARG, "rt_set_optics: null array");
  for (int l = 0; l < n_lambda; ++l) {
    if (!(is_finite(kappa[l]) && kappa[l] >= 0)) return fail(c, RT_ERR_ARG, "rt_set_optics: kappa[%d] invalid", l);
    if (!(albedo[l] >= 0 && albedo[l] <= 1)) return fail(c, RT_ERR_ARG, "rt_set_optics: albedo[%d] not in [0,1]", l);
    if (!(g[l] > -1 && g[l] < 1)) return fail(c, RT_ERR_ARG, "rt_set_optics: g[%d] not in (-1,1)", l);
  }
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  free_problem(c);
  c->n_lambda = n_lambda;
  c->lambda_um.clear();
  if (lambda) c->lambda_um.assign(lambda, lambda + n_lambda);
  c->kappa.assign(kappa, kappa + n_lambda);
  c->albedo.assign(albedo, albedo + n_lambda);
  c->g.assign(g, g + n_lambda);
  const size_t n_abs = (size_t)n_lambda * c->n_cells;
  RT_CUDA(c, pool_alloc(c, &c->d_absorption, n_abs * sizeof(double)));
  RT_CUDA(c, cudaMemset(c->d_absorption, 0, n_abs * sizeof(double)));
  RT_CUDA(c, cudaMemset(c->d_stats, 0, 4 * sizeof(double)));
  RT_CUDA(c, cudaMemset(c->d_counters, 0, 9 * sizeof(unsigned long long)));
  c->emitted = 0.0;
  c->tables_dirty = true;
  c->tape_valid = false;
  return RT_OK;
}

rt_status rt_add_sources(rt_ctx c, int32_t n, const rt_source_desc* s) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (c->n_lambda == 0) return fail(c, RT_ERR_STATE, "rt_add_sources: set optics first");
  if (n < 0 || (n > 0 && !s)) return fail(c, RT_ERR_ARG, "rt_add_sources: bad count or null array");
  if ((int)c->sources.size() + n > kMaxSources) return fail(c, RT_ERR_ARG, "rt_add_sources: at most %d sources", kMaxSources);
  for (int i = 0; i < n; ++i) {
    const rt_source_desc& d = s[i];
    if (d.kind < RT_SOURCE_POINT || d.kind > RT_SOURCE_PLUMMER) return fail(c, RT_ERR_ARG, "source %d: unknown kind", i);
    if (!d.luminosity) return fail(c, RT_ERR_ARG, "source %d: null luminosity", i);
    if (d.kind != RT_SOURCE_POINT && !(d.scale_r > 0)) return fail(c, RT_ERR_ARG, "source %d: scale_r must be > 0", i);
    if (d.kind == RT_SOURCE_EXPDISK && !(d.scale_z > 0)) return fail(c, RT_ERR_ARG, "source %d: scale_z must be > 0", i);
    for (int a = 0; a < 3; ++a) if (!is_finite(d.center[a])) return fail(c, RT_ERR_ARG, "source %d: bad centre", i);
    for (int l = 0; l < c->n_lambda; ++l)
      if (!(is_finite(d.luminosity[l]) && d.luminosity[l] >= 0)) return fail(c, RT_ERR_ARG, "source %d: bad luminosity", i);
  }
  for (int i = 0; i < n; ++i) {
    HostSource h;
    h.desc = s[i];
    h.lum.assign(s[i].luminosity, s[i].luminosity + c->n_lambda);
    h.desc.luminosity = nullptr;
    c->sources.push_back(h);
  }
  c->tables_dirty = true;
  c->tape_valid = false;
  return RT_OK;
}

rt_status rt_add_instruments(rt_ctx c, int32_t n, const rt_instrument_desc* q, int32_t* ids) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (c->n_lambda == 0) return fail(c, RT_ERR_STATE, "rt_add_instruments: set optics first");
  if (n < 0 || (n > 0 && !q)) return fail(c, RT_ERR_ARG, "rt_add_instruments: bad count or null array");
  if ((int)c->instr.size() + n > kMaxInstruments)
    return fail(c, RT_ERR_ARG, "rt_add_instruments: at most %d instruments", kMaxInstruments);
  for (int i = 0; i < n; ++i) {
    const rt_instrument_desc& d = q[i];
    if (d.nx <= 0 || d.ny <= 0 || (long long)d.nx * d.ny > (1ll << 28))
      return fail(c, RT_ERR_ARG, "instrument %d: bad pixel counts", i);
    if (d.deposit != RT_DEPOSIT_NEAREST && d.deposit != RT_DEPOSIT_BILINEAR && d.deposit != RT_DEPOSIT_SED)
      return fail(c, RT_ERR_ARG, "instrument %d: unknown deposit mode", i);
    if (d.deposit == RT_DEPOSIT_SED && (d.nx != 1 || d.ny != 1))
      return fail(c, RT_ERR_ARG, "instrument %d: an SED instrument has nx = ny = 1", i);
    if (d.deposit != RT_DEPOSIT_SED && !(d.half_x > 0 && d.half_y > 0))
      return fail(c, RT_ERR_ARG, "instrument %d: half widths must be > 0", i);
    if (d.channels != 1 && d.channels != 3) return fail(c, RT_ERR_ARG, "instrument %d: channels must be 1 or 3", i);
    if (!(is_finite(d.inclination) && is_finite(d.azimuth) && is_finite(d.position_angle) && is_finite(d.center_x) &&
          is_finite(d.center_y)))
      return fail(c, RT_ERR_ARG, "instrument %d: non-finite angle or centre", i);
  }
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    HostInstr h;
    h.desc = q[i];
    h.n_elems = (size_t)q[i].channels * c->n_lambda * q[i].ny * q[i].nx;
    RT_CUDA(c, pool_alloc(c, &h.d_image, h.n_elems * sizeof(double)));
    RT_CUDA(c, cudaMemset(h.d_image, 0, h.n_elems * sizeof(double)));
    if (ids) ids[i] = (int32_t)c->instr.size();
    c->instr.push_back(h);
  }
  c->tables_dirty = true;
  c->tape_valid = false;
  return RT_OK;
}

namespace {

// Buffers of the sorted peel-off pass for a launch of n_total packets with
// `walked` instruments whose peel-offs walk; on success p.peel is set (left
// null when the pass does not fit: the kernel then walks every peel-off).
rt_status prepare_peel_pass(rt_ctx c, FwdParams& p, unsigned long long n_total, int walked, bool tags,
                            cudaStream_t s) {
  const unsigned long long keys = (unsigned long long)c->instr.size() * (unsigned long long)(c->n_cells + 1);
  if (keys >= 0xffffffffull) return RT_OK;
  if (!c->peel_event) {
    RT_CUDA(c, cudaEventCreateWithFlags(&c->peel_event, cudaEventDisableTiming));
    RT_CUDA(c, cudaMallocHost(&c->h_peel_count, sizeof(unsigned long long)));
    RT_CUDA(c, cudaMalloc(&c->d_peel_count, sizeof(unsigned long long)));
  }
  if (c->peel_pending) {
    const cudaError_t q = cudaEventQuery(c->peel_event);
    if (q == cudaSuccess) {
      c->peel_pending = false;
      if (c->peel_last_packets)
        c->peel_per_packet = (double)*c->h_peel_count / (double)c->peel_last_packets;
    } else if (q == cudaErrorNotReady) {
      cudaGetLastError();  // not an error: the last launch is still running
    } else {
      return cuda_fail(c, q, "peel-off pass");
    }
  }
  // records per packet: what the last launch asked for plus a quarter, else
  // eight per walked instrument (a packet peels off once per event)
  const double per = c->peel_per_packet > 0.0 ? 1.25 * c->peel_per_packet + 0.05 : 8.0 * walked;
  unsigned long long want = (unsigned long long)std::min(per * (double)n_total, 4.0e9);
  want = std::max(want, 4096ull);
  if (want > c->peel_cap) {
    dfree(c->d_peel);
    dfree(c->d_peel_perm);
    c->peel_cap = 0;
    size_t free_b = 0, total_b = 0;
    RT_CUDA(c, cudaMemGetInfo(&free_b, &total_b));
    // at most 40 % of the free device memory
    const unsigned long long fit = (unsigned long long)(0.4 * (double)free_b) / (sizeof(PeelRecord) + sizeof(unsigned));
    want = std::min(want, fit);
    if (want < 4096) return RT_OK;
    if (cudaMalloc(&c->d_peel, want * sizeof(PeelRecord)) != cudaSuccess ||
        cudaMalloc(&c->d_peel_perm, want * sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      dfree(c->d_peel);
      dfree(c->d_peel_perm);
      return RT_OK;
    }
    c->peel_cap = want;
  }
  if (tags && c->peel_tag_cap < c->peel_cap) {
    dfree(c->d_peel_tag);
    c->peel_tag_cap = 0;
    if (cudaMalloc(&c->d_peel_tag, c->peel_cap * sizeof(ulonglong2)) != cudaSuccess) {
      cudaGetLastError();
      c->d_peel_tag = nullptr;
      return RT_OK;
    }
    c->peel_tag_cap = c->peel_cap;
  }
  if (keys > c->peel_keys) {
    dfree(c->d_peel_hist);
    dfree(c->d_peel_tiles);
    c->peel_keys = 0;
    RT_CUDA(c, cudaMalloc(&c->d_peel_hist, keys * sizeof(unsigned)));
    RT_CUDA(c, cudaMalloc(&c->d_peel_tiles, ((keys + 4095) / 4096) * sizeof(unsigned)));
    c->peel_keys = keys;
  }
  RT_CUDA(c, cudaMemsetAsync(c->d_peel_hist, 0, keys * sizeof(unsigned), s));
  RT_CUDA(c, cudaMemsetAsync(c->d_peel_count, 0, sizeof(unsigned long long), s));
  p.peel = c->d_peel;
  p.peel_cap = c->peel_cap;
  p.peel_count = c->d_peel_count;
  p.peel_hist = c->d_peel_hist;
  p.peel_tag = tags ? c->d_peel_tag : nullptr;
  return RT_OK;
}

}  // namespace

rt_status rt_launch_packets(rt_ctx c, uint64_t n_per_lambda, uint64_t first_packet_id, uint64_t seed,
                            const rt_launch_opts* opts, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!c->has_grid || c->n_lambda == 0) return fail(c, RT_ERR_STATE, "rt_launch_packets: grid and optics required");
  if (seed >> 32) return fail(c, RT_ERR_ARG, "rt_launch_packets: seed must be < 2^32");
  rt_launch_opts o;
  rt_default_opts(&o);
  if (opts) o = *opts;
  if (o.emitter != RT_EMITTER_SOURCES && o.emitter != RT_EMITTER_DUST)
    return fail(c, RT_ERR_ARG, "rt_launch_packets: unknown emitter %d", o.emitter);
  const bool dust = o.emitter == RT_EMITTER_DUST;
  if (dust && !c->dust_ready) return fail(c, RT_ERR_STATE, "rt_launch_packets: no dust emission set");
  if (dust && o.tape) return fail(c, RT_ERR_ARG, "rt_launch_packets: the adjoint tape needs the sources as emitter");
  if (!dust && c->sources.empty()) return fail(c, RT_ERR_STATE, "rt_launch_packets: no sources");
  // luminosity per wavelength of the emitter
  std::vector<double> lum_total((size_t)c->n_lambda, 0.0);
  for (int l = 0; l < c->n_lambda; ++l) {
    if (dust) {
      lum_total[(size_t)l] = c->dust_total[(size_t)l];
    } else {
      for (auto& src : c->sources) lum_total[(size_t)l] += src.lum[l];
    }
  }
  if (o.max_events < 1) return fail(c, RT_ERR_ARG, "rt_launch_packets: max_events must be >= 1");
  if (!(o.w_min >= 0 && o.w_min < 1)) return fail(c, RT_ERR_ARG, "rt_launch_packets: w_min must be in [0, 1)");
  if (o.control_lanes < 0 || o.control_lanes > 32)
    return fail(c, RT_ERR_ARG, "rt_launch_packets: control_lanes must be in [0, 32]");
  if ((o.records && o.records_capacity < 0) || (o.trace && o.trace_capacity < 0))
    return fail(c, RT_ERR_ARG, "rt_launch_packets: negative record or trace capacity");
  for (int l = 0; l < c->n_lambda; ++l)
    if (!dust && !(lum_total[(size_t)l] > 0))
      return fail(c, RT_ERR_ARG, "rt_launch_packets: zero total luminosity at wavelength %d", l);
  if (n_per_lambda == 0) return RT_OK;
  const unsigned long long n_total = n_per_lambda * (unsigned long long)c->n_lambda;
  if (n_total / (unsigned long long)c->n_lambda != n_per_lambda || n_total > (1ull << 62))
    return fail(c, RT_ERR_ARG, "rt_launch_packets: packet count overflow");
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  rt_status st = upload_tables(c, s);
  if (st != RT_OK) return st;
  FwdParams p;
  std::memset(&p, 0, sizeof p);
  p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
  for (int a = 0; a < 3; ++a) {
    p.lo[a] = (float)c->bounds[2 * a];
    p.hi[a] = (float)c->bounds[2 * a + 1];
    const int n = a == 0 ? c->nx : (a == 1 ? c->ny : c->nz);
    if (c->grid_kind == RT_GRID_CARTESIAN) {
      const double d = (c->bounds[2 * a + 1] - c->bounds[2 * a]) / n;
      p.d[a] = (float)d;
      p.inv_d[a] = (float)(1.0 / d);
    }
  }
  p.density = c->permuted ? c->d_density_s : c->d_density;
  for (int a = 0; a < 3; ++a) p.stride[a] = c->stride[a];
  p.child = c->d_child;
  p.n_nodes = c->n_nodes;
  p.oct_exact = c->oct_exact ? 1 : 0;
  p.oct_levels = c->oct_depth + 1;
  p.rope = c->d_rope;
  p.node_box = c->d_node_box;
  if (c->grid_kind == RT_GRID_VORONOI) {
    p.site = c->d_site;
    p.face_off = c->d_face_off;
    p.face = c->d_face;
    p.bucket_seed = c->d_bucket_seed;
    for (int a = 0; a < 3; ++a) {
      p.vb_n[a] = c->vb_n[a];
      p.vb_inv[a] = (float)(c->vb_n[a] / (c->bounds[2 * a + 1] - c->bounds[2 * a]));
    }
    p.max_walk = (int)std::min<long long>(c->n_cells + 64, (1ll << 31) - 1);
  }
  if (c->grid_kind == RT_GRID_RECTILINEAR) {
    p.edge[0] = c->d_edges;
    p.edge[1] = c->d_edges + c->nx + 1;
    p.edge[2] = c->d_edges + c->nx + c->ny + 2;
  }
  p.n_cells = c->n_cells;
  p.n_lambda = c->n_lambda;
  p.n_sources = (int)c->sources.size();
  p.n_instr = (int)c->instr.size();
  p.lam = c->d_lam;
  p.src = c->d_src;
  p.src_cum = c->d_src_cum;
  p.instr = c->d_instr;
  p.absorption = c->d_absorption;
  p.n_per_lambda = n_per_lambda;
  p.first_id = first_packet_id;
  p.n_total = n_total;
  p.n_norm = o.n_norm ? o.n_norm : n_per_lambda;
  p.seed = (unsigned)seed;
  p.model = o.model_id;
  p.w_min = o.w_min;
  p.max_events = o.max_events;
  p.weight_cut = o.weight_cut;
  p.peel_emission = o.peel_emission;
  p.peel_scatter = o.peel_scatter;
  p.work_counter = c->d_work;
  p.stats = c->d_stats;
  p.counters = c->d_counters;
  p.records = o.records;
  p.records_cap = o.records ? o.records_capacity : 0;
  p.record_stride = o.record_stride;
  p.trace = o.trace;
  p.trace_cap = o.trace ? o.trace_capacity : 0;
  p.trace_packet = o.trace_packet;
  p.trace_lambda = o.trace_lambda;
  p.control_min = o.control_lanes ? o.control_lanes : (c->control_lanes ? c->control_lanes : 16);
  if (o.blocks_per_sm < 0) return fail(c, RT_ERR_ARG, "rt_launch_packets: blocks_per_sm must be >= 0");
  p.blocks_per_sm = o.blocks_per_sm ? o.blocks_per_sm : c->blocks_per_sm;
  p.inv_n_per_lambda = (float)(1.0 / (double)n_per_lambda);
  for (int l = 0; l < c->n_lambda; ++l) {
    p.L0[l] = lum_total[(size_t)l] / (double)p.n_norm;
    p.L_cut[l] = o.w_min * p.L0[l];
  }
  p.dust_cum = dust ? c->d_dust_cum : nullptr;
  p.profile = reinterpret_cast<unsigned long long*>(o.profile);
  p.flags = c->d_flags;
  p.use_columns = indexed_cells(c->grid_kind) && !o.walk_peels;
  cudaEvent_t* ev = nullptr;
  if (o.time_parts) {
    for (auto& e : c->part_ev)
      if (!e) RT_CUDA(c, cudaEventCreate(&e));
    ev = c->part_ev;
    c->parts_timed = false;
  }
  if (o.tape) {
    if (c->grid_kind != RT_GRID_CARTESIAN) return fail(c, RT_ERR_ARG, "rt_launch_packets: the tape needs a cartesian grid");
    if (o.max_events > kMaxAdjointEvents)
      return fail(c, RT_ERR_ARG, "rt_launch_packets: the tape needs max_events <= %d", kMaxAdjointEvents);
    const size_t need = (size_t)n_total * (size_t)(o.max_events + 1) * sizeof(AdjRecord);
    if (need / sizeof(AdjRecord) / (size_t)(o.max_events + 1) != (size_t)n_total)
      return fail(c, RT_ERR_ARG, "rt_launch_packets: tape size overflow");
    if (need > c->tape_bytes) {
      dfree(c->d_tape);
      c->tape_bytes = 0;
      cudaError_t ea = cudaMalloc(&c->d_tape, need);
      if (ea != cudaSuccess) {
        c->d_tape = nullptr;
        cudaGetLastError();
        return fail(c, RT_ERR_OOM, "rt_launch_packets: %zu bytes of adjoint tape", need);
      }
      c->tape_bytes = need;
    }
    p.tape = c->d_tape;
    p.tape_stride = o.max_events + 1;
  }
  if (ev) RT_CUDA(c, cudaEventRecord(ev[0], s));
  if (p.use_columns) {
    for (int k = 0; k < 6; ++k) {
      if (!c->columns_used[k]) continue;
      const int axis = k / 2;
      cudaError_t ec = launch_columns(c->d_density, c->nx, c->ny, c->nz, axis, (k & 1) ? 1 : -1, p.d[axis],
                                      c->grid_kind == RT_GRID_RECTILINEAR ? axis_planes(c, axis) : nullptr,
                                      c->d_columns[k], s);
      if (ec != cudaSuccess) return cuda_fail(c, ec, "column sums");
    }
  }
  if (ev) RT_CUDA(c, cudaEventRecord(ev[1], s));
  const int walked = o.walk_peels ? (int)c->instr.size() : c->n_walked_frames;
  if (c->grid_kind == RT_GRID_CARTESIAN && !o.tape && !o.inline_peels && walked > 0 &&
      (o.peel_emission || o.peel_scatter)) {
    st = prepare_peel_pass(c, p, n_total, walked, o.records != nullptr, s);
    if (st != RT_OK) return st;
  }
  cudaError_t e = launch_forward(p, c->grid_kind, c->num_sms, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "forward launch");
  if (ev) RT_CUDA(c, cudaEventRecord(ev[2], s));
  if (p.peel) {
    e = launch_peel_pass(p, (unsigned long long)c->instr.size() * (unsigned long long)(c->n_cells + 1),
                         c->d_peel_tiles, c->d_peel_perm, c->num_sms, s, ev ? ev[3] : nullptr);
    if (e != cudaSuccess) return cuda_fail(c, e, "peel-off pass");
    if (!c->peel_pending) {
      RT_CUDA(c, cudaMemcpyAsync(c->h_peel_count, c->d_peel_count, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
      RT_CUDA(c, cudaEventRecord(c->peel_event, s));
      c->peel_pending = true;
      c->peel_last_packets = n_total;
    }
  } else if (ev) {
    RT_CUDA(c, cudaEventRecord(ev[3], s));
  }
  if (ev) {
    RT_CUDA(c, cudaEventRecord(ev[4], s));
    c->parts_timed = true;
  }
  if (o.tape) {
    c->tape_valid = true;
    c->tape_n = n_per_lambda; c->tape_first = first_packet_id; c->tape_seed = seed; c->tape_norm = p.n_norm;
    c->tape_max_events = o.max_events; c->tape_weight_cut = o.weight_cut; c->tape_w_min = o.w_min;
    c->tape_peel_e = o.peel_emission; c->tape_peel_s = o.peel_scatter; c->tape_model = (int)o.model_id;
  }
  // every packet starts with L0 = L_tot / n_norm
  for (int l = 0; l < c->n_lambda; ++l) c->emitted += (double)n_per_lambda * p.L0[l];
  return RT_OK;
}

rt_status rt_update_density(rt_ctx c, const float* density, int32_t on_device, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!c->has_grid) return fail(c, RT_ERR_STATE, "rt_update_density: no grid");
  if (!density) return fail(c, RT_ERR_ARG, "rt_update_density: null density");
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  c->tape_valid = false;
  const size_t bytes = (size_t)c->n_cells * sizeof(float);
  if (on_device) {
    RT_CUDA(c, cudaMemcpyAsync(c->d_density, density, bytes, cudaMemcpyDeviceToDevice, s));
  } else {
    // the caller may reuse its host buffer on return: copy synchronously
    RT_CUDA(c, cudaStreamSynchronize(s));
    RT_CUDA(c, cudaMemcpy(c->d_density, density, bytes, cudaMemcpyHostToDevice));
  }
  if (c->permuted) RT_CUDA(c, launch_to_storage(c->d_density, c->d_density_s, c->nx, c->ny, c->nz, c->stride, s));
  return RT_OK;
}

rt_status rt_adjoint(rt_ctx c, const double* const* adj_images, int32_t n_adj_images, const double* adj_absorption,
                     double* grad_density, uint64_t n_per_lambda, uint64_t first_packet_id, uint64_t seed,
                     const rt_launch_opts* opts, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!c->has_grid || c->n_lambda == 0 || c->sources.empty())
    return fail(c, RT_ERR_STATE, "rt_adjoint: grid, optics and sources required");
  if (c->grid_kind != RT_GRID_CARTESIAN) return fail(c, RT_ERR_ARG, "rt_adjoint: cartesian grids only");
  if (!grad_density) return fail(c, RT_ERR_ARG, "rt_adjoint: null gradient");
  if (n_adj_images < 0 || n_adj_images > (int)c->instr.size() || (n_adj_images > 0 && !adj_images))
    return fail(c, RT_ERR_ARG, "rt_adjoint: bad adjoint image list");
  if (seed >> 32) return fail(c, RT_ERR_ARG, "rt_adjoint: seed must be < 2^32");
  rt_launch_opts o;
  rt_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_events < 1 || o.max_events > kMaxAdjointEvents)
    return fail(c, RT_ERR_ARG, "rt_adjoint: max_events must be in [1, %d]", kMaxAdjointEvents);
  if (!(o.w_min >= 0 && o.w_min < 1)) return fail(c, RT_ERR_ARG, "rt_adjoint: w_min must be in [0, 1)");
  if (n_per_lambda == 0) return RT_OK;
  const unsigned long long n_total = n_per_lambda * (unsigned long long)c->n_lambda;
  if (n_total / (unsigned long long)c->n_lambda != n_per_lambda || n_total > (1ull << 62))
    return fail(c, RT_ERR_ARG, "rt_adjoint: packet count overflow");
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  rt_status st = upload_tables(c, s);
  if (st != RT_OK) return st;
  FwdParams p;
  std::memset(&p, 0, sizeof p);
  p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
  for (int a = 0; a < 3; ++a) {
    p.lo[a] = (float)c->bounds[2 * a];
    p.hi[a] = (float)c->bounds[2 * a + 1];
    const int n = a == 0 ? c->nx : (a == 1 ? c->ny : c->nz);
    const double d = (c->bounds[2 * a + 1] - c->bounds[2 * a]) / n;
    p.d[a] = (float)d;
    p.inv_d[a] = (float)(1.0 / d);
  }
  p.density = c->d_density;  // row-major: the adjoint keeps the row-major order
  row_major_strides(p);
  p.n_cells = c->n_cells;
  p.n_lambda = c->n_lambda;
  p.n_sources = (int)c->sources.size();
  p.n_instr = (int)c->instr.size();
  p.lam = c->d_lam;
  p.src = c->d_src;
  p.src_cum = c->d_src_cum;
  p.instr = c->d_instr;
  p.n_per_lambda = n_per_lambda;
  p.first_id = first_packet_id;
  p.n_total = n_total;
  p.n_norm = o.n_norm ? o.n_norm : n_per_lambda;
  p.seed = (unsigned)seed;
  p.model = o.model_id;
  p.w_min = o.w_min;
  p.max_events = o.max_events;
  p.weight_cut = o.weight_cut;
  p.peel_emission = o.peel_emission;
  p.peel_scatter = o.peel_scatter;
  p.work_counter = c->d_work;
  p.flags = c->d_flags;
  if (o.control_lanes < 0 || o.control_lanes > 32) return fail(c, RT_ERR_ARG, "rt_adjoint: control_lanes in [0, 32]");
  p.control_min = o.control_lanes ? o.control_lanes : (c->adjoint_lanes ? c->adjoint_lanes : 16);
  p.inv_n_per_lambda = (float)(1.0 / (double)n_per_lambda);
  for (int l = 0; l < c->n_lambda; ++l) {
    double tot = 0.0;
    for (auto& src : c->sources) tot += src.lum[l];
    p.L0[l] = tot / (double)p.n_norm;
    p.L_cut[l] = o.w_min * p.L0[l];
  }
  const double* adj[kMaxInstruments] = {nullptr};
  for (int q = 0; q < n_adj_images; ++q) adj[q] = adj_images[q];
  // the forward launch's tape, when it recorded exactly these packets
  const bool use_tape = c->tape_valid && !adj_absorption && c->tape_n == n_per_lambda &&
                        c->tape_first == first_packet_id && c->tape_seed == seed && c->tape_norm == p.n_norm &&
                        c->tape_max_events == o.max_events && c->tape_weight_cut == o.weight_cut &&
                        c->tape_w_min == o.w_min && c->tape_peel_e == o.peel_emission &&
                        c->tape_peel_s == o.peel_scatter && c->tape_model == (int)o.model_id;
  unsigned long long lanes = 0;
  cudaError_t e = adjoint_lanes(c->num_sms, n_total, &lanes);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint occupancy");
  const size_t need = use_tape ? 0 : (size_t)lanes * (size_t)(o.max_events + 1) * sizeof(AdjRecord);
  if (need > c->adj_bytes) {
    dfree(c->d_adj);
    c->adj_bytes = 0;
    e = cudaMalloc(&c->d_adj, need);
    if (e != cudaSuccess) {
      c->d_adj = nullptr;
      cudaGetLastError();
      return fail(c, RT_ERR_OOM, "rt_adjoint: %zu bytes of event records", need);
    }
    c->adj_bytes = need;
  }
  size_t elems[kMaxInstruments] = {0};
  size_t img_total = 0;
  for (int q = 0; q < n_adj_images; ++q) {
    elems[q] = c->instr[q].n_elems;
    if (adj[q]) img_total += elems[q];
  }
  if (img_total > c->adj_img_elems || !c->d_adj_img) {
    dfree(c->d_adj_img);
    c->adj_img_elems = 0;
    e = cudaMalloc(&c->d_adj_img, (img_total ? img_total : 1) * sizeof(float));
    if (e != cudaSuccess) {
      c->d_adj_img = nullptr;
      cudaGetLastError();
      return fail(c, RT_ERR_OOM, "rt_adjoint: %zu floats of adjoint images", img_total);
    }
    c->adj_img_elems = img_total ? img_total : 1;
  }
  if (!c->d_adj_max) RT_CUDA(c, cudaMalloc(&c->d_adj_max, sizeof(unsigned long long)));
  // frames along grid axes: the forward kernel's column sums, and a deposit
  // difference array per column table
  p.use_columns = !o.walk_peels;
  double* line_dep[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (p.use_columns) {
    for (int k = 0; k < 6; ++k) {
      if (!c->columns_used[k]) continue;
      const int axis = k / 2;
      if (!c->d_line_dep[k]) RT_CUDA(c, pool_alloc(c, &c->d_line_dep[k], (size_t)c->n_cells * sizeof(double)));
      line_dep[k] = c->d_line_dep[k];
      e = launch_columns(c->d_density, c->nx, c->ny, c->nz, axis, (k & 1) ? 1 : -1, p.d[axis], nullptr,
                         c->d_columns[k], s);
      if (e != cudaSuccess) return cuda_fail(c, e, "column sums");
    }
  }
  e = launch_adjoint(p, adj, elems, adj_absorption, grad_density, c->d_adj, lanes,
                     reinterpret_cast<unsigned long long*>(o.profile), c->d_adj_img, c->d_adj_max, line_dep,
                     use_tape ? c->d_tape : nullptr, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint launch");
  return RT_OK;
}

rt_status rt_tune(rt_ctx c, uint64_t n_per_lambda, uint64_t seed, const rt_launch_opts* opts, int32_t* control_lanes,
                  void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (n_per_lambda == 0) return fail(c, RT_ERR_ARG, "rt_tune: n_per_lambda must be >= 1");
  rt_launch_opts o;
  rt_default_opts(&o);
  if (opts) o = *opts;
  o.records = nullptr;
  o.trace = nullptr;
  o.profile = nullptr;
  o.blocks_per_sm = 0;
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  c->blocks_per_sm = 0;  // the threshold is timed with the most resident blocks
  const int cand[] = {8, 12, 16, 20, 24, 28};
  cudaEvent_t e0, e1;
  RT_CUDA(c, cudaEventCreate(&e0));
  RT_CUDA(c, cudaEventCreate(&e1));
  float best = -1.0f;
  int best_lanes = 16;
  rt_status st = RT_OK;
  for (int lanes : cand) {
    o.control_lanes = lanes;
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) st = rt_launch_packets(c, n_per_lambda, 0, seed, &o, stream);
    if (st != RT_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(c, e, "rt_tune");
      break;
    }
    if (best < 0 || ms < best) {
      best = ms;
      best_lanes = lanes;
    }
  }
  // then the resident blocks per SM at that threshold: the most that fit
  // (0), one and two fewer.  Only on a sample of at least kTuneBlockPackets
  // packets per resident thread: on fewer, the launch time is the slowest
  // packet's and fewer resident threads (less contention) win on the sample
  // while they lose on the full run.
  int best_blocks = 0;
  o.control_lanes = best_lanes;
  // the kernels' launch bounds
  const int max_blocks = 4;
  constexpr unsigned long long kTuneBlockPackets = 8;
  constexpr unsigned long long kTransportThreads = 256;  // threads per block of the transport kernels
  const unsigned long long resident =
      (unsigned long long)c->num_sms * (unsigned long long)max_blocks * kTransportThreads;
  const bool search_blocks = n_per_lambda * (unsigned long long)c->n_lambda >= kTuneBlockPackets * resident;
  for (int blocks = max_blocks - 1; search_blocks && st == RT_OK && blocks >= max_blocks - 2 && blocks >= 1;
       --blocks) {
    o.blocks_per_sm = blocks;
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) st = rt_launch_packets(c, n_per_lambda, 0, seed, &o, stream);
    if (st != RT_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(c, e, "rt_tune");
      break;
    }
    // fewer blocks must win clearly: one sample launch per candidate, and a
    // small sample's timing noise should not cost the full occupancy
    if (ms < 0.97f * best) {
      best = ms;
      best_blocks = blocks;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RT_OK) return st;
  c->control_lanes = best_lanes;
  c->blocks_per_sm = best_blocks;
  if (control_lanes) *control_lanes = best_lanes;
  return rt_reset_tallies(c, stream);
}

rt_status rt_tuned(rt_ctx c, int32_t* control_lanes, int32_t* blocks_per_sm) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (control_lanes) *control_lanes = c->control_lanes ? c->control_lanes : 16;
  if (blocks_per_sm) *blocks_per_sm = c->blocks_per_sm;
  return RT_OK;
}

rt_status rt_adjoint_tune(rt_ctx c, const double* const* adj_images, int32_t n_adj_images,
                          const double* adj_absorption, uint64_t n_per_lambda, uint64_t seed,
                          const rt_launch_opts* opts, int32_t* control_lanes, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!c->has_grid) return fail(c, RT_ERR_STATE, "rt_adjoint_tune: no grid");
  if (n_per_lambda == 0) return fail(c, RT_ERR_ARG, "rt_adjoint_tune: n_per_lambda must be >= 1");
  rt_launch_opts o;
  rt_default_opts(&o);
  if (opts) o = *opts;
  o.profile = nullptr;
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  if ((size_t)c->n_cells > c->tune_grad_cells) {
    dfree(c->d_tune_grad);
    c->tune_grad_cells = 0;
    RT_CUDA(c, cudaMalloc(&c->d_tune_grad, (size_t)c->n_cells * sizeof(double)));
    c->tune_grad_cells = (size_t)c->n_cells;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int cand[] = {12, 16, 20, 24, 28, 32};
  cudaEvent_t e0, e1;
  RT_CUDA(c, cudaEventCreate(&e0));
  RT_CUDA(c, cudaEventCreate(&e1));
  float best = -1.0f;
  int best_lanes = 16;
  rt_status st = RT_OK;
  for (int lanes : cand) {
    o.control_lanes = lanes;
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess)
      st = rt_adjoint(c, adj_images, n_adj_images, adj_absorption, c->d_tune_grad, n_per_lambda, 0, seed, &o, stream);
    if (st != RT_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(c, e, "rt_adjoint_tune");
      break;
    }
    if (best < 0 || ms < best) {
      best = ms;
      best_lanes = lanes;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RT_OK) return st;
  c->adjoint_lanes = best_lanes;
  if (control_lanes) *control_lanes = best_lanes;
  return RT_OK;
}

rt_status rt_reset_tallies(rt_ctx c, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  return zero_tallies(c, (cudaStream_t)stream);
}

// The device address of page-locked host memory that the device can write,
// or null (pageable or unknown memory).
static double* pinned_view(const double* host) {
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, host);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? static_cast<double*>(at.devicePointer) : nullptr;
}

// Where a kernel may write n doubles of host memory at `host` directly: on a
// device that reaches all host memory (every address of the range is then
// legal for it), when the range starts and ends in page-locked memory (the
// writes then run at the link's speed); else null.
static double* device_view(rt_ctx c, double* host, size_t n) {
  if (!c->pageable_access || n == 0) return nullptr;
  double* first = pinned_view(host);
  if (!first || first != host || pinned_view(host + (n - 1)) != host + (n - 1)) return nullptr;
  return first;
}

// Host destinations: a copy kernel writes them where device_view allows (the
// copy engine's first copy after a long launch was measured up to 15 times
// slower than the next), the copy engine elsewhere.
static rt_status copy_out(rt_ctx c, double* dst, const double* src, size_t n, int32_t on_device, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (on_device) {
    RT_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return RT_OK;
  }
  if (double* view = device_view(c, dst, n)) {
    RT_CUDA(c, launch_copy_f64(src, view, (long long)n, s));
  } else {
    RT_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  RT_CUDA(c, cudaStreamSynchronize(s));
  return RT_OK;
}

rt_status rt_read_absorption(rt_ctx c, double* dst, size_t n_elems, int32_t on_device, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!c->d_absorption) return fail(c, RT_ERR_STATE, "rt_read_absorption: no optics set");
  if (!dst) return fail(c, RT_ERR_ARG, "rt_read_absorption: null destination");
  const size_t n = (size_t)c->n_lambda * c->n_cells;
  if (n_elems != n) return fail(c, RT_ERR_ARG, "rt_read_absorption: n_elems %zu != %zu", n_elems, n);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  if (!c->permuted) return copy_out(c, dst, c->d_absorption, n, on_device, stream);
  // tallies in storage order: back to row-major into dst, or wavelength by
  // wavelength through a device buffer for a host destination
  cudaStream_t s = (cudaStream_t)stream;
  if (on_device) {
    RT_CUDA(c, launch_from_storage(c->d_absorption, dst, c->n_lambda, c->nx, c->ny, c->nz, c->stride, s));
    return RT_OK;
  }
  // host memory that device_view allows: the kernel writes the row-major
  // field into it directly (no staging buffer, no second pass)
  if (double* view = device_view(c, dst, n)) {
    RT_CUDA(c, launch_from_storage(c->d_absorption, view, c->n_lambda, c->nx, c->ny, c->nz, c->stride, s));
    RT_CUDA(c, cudaStreamSynchronize(s));
    return RT_OK;
  }
  if (!c->d_abs_tmp) RT_CUDA(c, pool_alloc(c, &c->d_abs_tmp, (size_t)c->n_cells * sizeof(double)));
  for (int l = 0; l < c->n_lambda; ++l) {
    RT_CUDA(c, launch_from_storage(c->d_absorption + (size_t)l * c->n_cells, c->d_abs_tmp, 1, c->nx, c->ny, c->nz,
                                   c->stride, s));
    RT_CUDA(c, cudaMemcpyAsync(dst + (size_t)l * c->n_cells, c->d_abs_tmp, (size_t)c->n_cells * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  }
  RT_CUDA(c, cudaStreamSynchronize(s));
  return RT_OK;
}

namespace {

// Checks shared by the panchromatic calls; fills the per-wavelength weights
// S kappa_l (1 - albedo_l) dlambda_l (bins centred on the wavelengths on a
// logarithmic scale: inner borders at geometric means, outer ones mirrored).
rt_status dust_setup(rt_ctx c, const char* who, double scale, std::vector<double>& w) {
  if (!c->has_grid || c->n_lambda == 0) return fail(c, RT_ERR_STATE, "%s: grid and optics required", who);
  if (!indexed_cells(c->grid_kind)) return fail(c, RT_ERR_ARG, "%s: cartesian or rectilinear grids only", who);
  if (c->n_lambda < 2 || (int)c->lambda_um.size() != c->n_lambda)
    return fail(c, RT_ERR_STATE, "%s: rt_set_optics needs the wavelengths (at least two, in um)", who);
  for (int l = 0; l < c->n_lambda; ++l)
    if (!(is_finite(c->lambda_um[l]) && c->lambda_um[l] > 0 && (l == 0 || c->lambda_um[l] > c->lambda_um[l - 1])))
      return fail(c, RT_ERR_ARG, "%s: wavelengths must be positive and increasing", who);
  if (!(is_finite(scale) && scale > 0)) return fail(c, RT_ERR_ARG, "%s: emission scale must be > 0", who);
  const int n = c->n_lambda;
  const std::vector<double>& lam = c->lambda_um;
  std::vector<double> b((size_t)n + 1);
  for (int l = 1; l < n; ++l) b[(size_t)l] = std::sqrt(lam[l - 1] * lam[l]);
  b[0] = lam[0] * std::sqrt(lam[0] / lam[1]);
  b[(size_t)n] = lam[n - 1] * std::sqrt(lam[n - 1] / lam[n - 2]);
  w.assign((size_t)n, 0.0);
  for (int l = 0; l < n; ++l) w[(size_t)l] = scale * c->kappa[l] * (1.0 - c->albedo[l]) * (b[(size_t)l + 1] - b[(size_t)l]);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  return RT_OK;
}

}  // namespace

rt_status rt_dust_temperature(rt_ctx c, double emission_scale, double t_min, double t_max, const double* absorption,
                              int32_t absorption_on_device, double* temperature, int32_t dst_on_device,
                              int32_t* n_clamped, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  std::vector<double> w;
  rt_status st = dust_setup(c, "rt_dust_temperature", emission_scale, w);
  if (st != RT_OK) return st;
  if (!temperature) return fail(c, RT_ERR_ARG, "rt_dust_temperature: null destination");
  if (!(t_min > 0 && t_max > t_min && is_finite(t_max)))
    return fail(c, RT_ERR_ARG, "rt_dust_temperature: need 0 < t_min < t_max");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nc = (size_t)c->n_cells, nl = (size_t)c->n_lambda;
  if (!c->d_dust_T) RT_CUDA(c, pool_alloc(c, &c->d_dust_T, nc * sizeof(double)));
  if (!c->d_dust_clamped) RT_CUDA(c, cudaMalloc(&c->d_dust_clamped, sizeof(unsigned)));
  RT_CUDA(c, cudaMemsetAsync(c->d_dust_clamped, 0, sizeof(unsigned), s));
  const double* src = c->d_absorption;
  int stored = 1;
  double* staged = nullptr;
  if (absorption) {
    stored = 0;
    if (absorption_on_device) {
      src = absorption;
    } else {
      RT_CUDA(c, cudaMalloc(&staged, nl * nc * sizeof(double)));
      cudaError_t e = cudaMemcpyAsync(staged, absorption, nl * nc * sizeof(double), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        cudaFree(staged);
        return cuda_fail(c, e, "rt_dust_temperature: absorption upload");
      }
      src = staged;
    }
  }
  cudaError_t e = launch_dust_temperature(c->n_lambda, c->nx, c->ny, c->nz, c->stride, c->d_planes64, c->d_density,
                                          w.data(), c->lambda_um.data(), src, stored, t_min, t_max, c->d_dust_T,
                                          c->d_dust_clamped, s);
  unsigned clamped = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&clamped, c->d_dust_clamped, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(temperature, c->d_dust_T, nc * sizeof(double),
                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (staged) cudaFree(staged);
  if (e != cudaSuccess) return cuda_fail(c, e, "rt_dust_temperature");
  if (n_clamped) *n_clamped = (int32_t)clamped;
  return RT_OK;
}

rt_status rt_set_dust_emission(rt_ctx c, const double* temperature, int32_t on_device, double emission_scale,
                               void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  std::vector<double> w;
  rt_status st = dust_setup(c, "rt_set_dust_emission", emission_scale, w);
  if (st != RT_OK) return st;
  if (!temperature) return fail(c, RT_ERR_ARG, "rt_set_dust_emission: null temperatures");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nc = (size_t)c->n_cells, nl = (size_t)c->n_lambda;
  c->dust_ready = false;
  c->tape_valid = false;
  if (!c->d_dust_T) RT_CUDA(c, pool_alloc(c, &c->d_dust_T, nc * sizeof(double)));
  if (!c->d_dust_lum) RT_CUDA(c, pool_alloc(c, &c->d_dust_lum, nl * nc * sizeof(double)));
  if (!c->d_dust_cum) RT_CUDA(c, pool_alloc(c, &c->d_dust_cum, nl * nc * sizeof(double)));
  if (!c->d_dust_tiles) RT_CUDA(c, pool_alloc(c, &c->d_dust_tiles, nl * dust_tiles(c->n_cells) * sizeof(double)));
  if (temperature != c->d_dust_T) {
    RT_CUDA(c, cudaMemcpyAsync(c->d_dust_T, temperature, nc * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (!on_device) RT_CUDA(c, cudaStreamSynchronize(s));  // the caller may reuse its host array
  }
  RT_CUDA(c, launch_dust_emission(c->n_lambda, c->nx, c->ny, c->nz, c->stride, c->d_planes64, c->d_density, w.data(),
                                  c->lambda_um.data(), c->d_dust_T, c->d_dust_lum, c->d_dust_cum, c->d_dust_tiles, s));
  // the per-wavelength totals (the last running sums) set the packet weights
  c->dust_total.assign(nl, 0.0);
  for (size_t l = 0; l < nl; ++l)
    RT_CUDA(c, cudaMemcpyAsync(&c->dust_total[l], c->d_dust_cum + l * nc + nc - 1, sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  RT_CUDA(c, cudaStreamSynchronize(s));
  for (size_t l = 0; l < nl; ++l)
    if (!(is_finite(c->dust_total[l]) && c->dust_total[l] >= 0))
      return fail(c, RT_ERR_ARG, "rt_set_dust_emission: non-finite emission at wavelength %zu", l);
  c->dust_ready = true;
  return RT_OK;
}

rt_status rt_read_dust_emission(rt_ctx c, double* dst, size_t n_elems, int32_t on_device, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!c->dust_ready) return fail(c, RT_ERR_STATE, "rt_read_dust_emission: no dust emission set");
  if (!dst) return fail(c, RT_ERR_ARG, "rt_read_dust_emission: null destination");
  const size_t n = (size_t)c->n_lambda * c->n_cells;
  if (n_elems != n) return fail(c, RT_ERR_ARG, "rt_read_dust_emission: n_elems %zu != %zu", n_elems, n);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  return copy_out(c, dst, c->d_dust_lum, n, on_device, stream);
}

rt_status rt_read_images(rt_ctx c, int32_t id, double* dst, size_t n_elems, int32_t on_device, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (id < 0 || id >= (int)c->instr.size()) return fail(c, RT_ERR_ARG, "rt_read_images: unknown instrument %d", id);
  if (!dst) return fail(c, RT_ERR_ARG, "rt_read_images: null destination");
  const size_t n = c->instr[id].n_elems;
  if (n_elems != n) return fail(c, RT_ERR_ARG, "rt_read_images: n_elems %zu != %zu", n_elems, n);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  return copy_out(c, dst, c->instr[id].d_image, n, on_device, stream);
}

rt_status rt_read_stats(rt_ctx c, rt_stats* out) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!out) return fail(c, RT_ERR_ARG, "rt_read_stats: null output");
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  RT_CUDA(c, cudaDeviceSynchronize());
  double st[4];
  unsigned long long cn[9];
  int flags = 0;
  RT_CUDA(c, cudaMemcpy(st, c->d_stats, sizeof st, cudaMemcpyDeviceToHost));
  RT_CUDA(c, cudaMemcpy(cn, c->d_counters, sizeof cn, cudaMemcpyDeviceToHost));
  RT_CUDA(c, cudaMemcpy(&flags, c->d_flags, sizeof flags, cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof *out);
  out->emitted = c->emitted; out->escaped = st[1]; out->absorbed = st[2]; out->truncated = st[3];
  out->crossings = cn[0]; out->path_crossings = cn[5]; out->events = cn[1]; out->peeloffs = cn[2]; out->packets = cn[3]; out->records = cn[4];
  out->column_peels = cn[6]; out->column_crossings = cn[7]; out->sorted_peels = cn[8];
  out->device_flags = flags;
  if (flags) return fail(c, RT_ERR_DEVICE_FLAG, "a kernel bounds check fired (flags 0x%x)", flags);
  return RT_OK;
}

rt_status rt_read_launch_times(rt_ctx c, float* ms, int32_t n) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!ms || n < 1 || n > 4) return fail(c, RT_ERR_ARG, "rt_read_launch_times: need 1..4 entries");
  if (!c->parts_timed) return fail(c, RT_ERR_STATE, "rt_read_launch_times: no launch with time_parts");
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  RT_CUDA(c, cudaEventSynchronize(c->part_ev[4]));
  for (int i = 0; i < n; ++i) RT_CUDA(c, cudaEventElapsedTime(&ms[i], c->part_ev[i], c->part_ev[i + 1]));
  return RT_OK;
}

rt_status rt_synchronize(rt_ctx c, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  RT_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
  RT_CUDA(c, cudaGetLastError());
  return RT_OK;
}

rt_status rt_batch_create(rt_ctx c, int32_t n_models, const rt_model_desc* models, int32_t* batch_id) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  if (!batch_id) return fail(c, RT_ERR_ARG, "rt_batch_create: null batch_id");
  if (n_models < 1 || n_models > (1 << 20) || !models) return fail(c, RT_ERR_ARG, "rt_batch_create: 1 .. 2^20 models");
  size_t n_cells_total = 0;
  for (int m = 0; m < n_models; ++m) {
    const rt_model_desc& d = models[m];
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nx > 65536 || d.ny > 65536 || d.nz > 65536)
      return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: cells per axis in 1 .. 65536", m);
    for (int a = 0; a < 3; ++a)
      if (!(d.bounds[2 * a + 1] > d.bounds[2 * a]) || !is_finite(d.bounds[2 * a]) || !is_finite(d.bounds[2 * a + 1]))
        return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: empty or non-finite bounds", m);
    if (!d.density) return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: null density", m);
    if (!(d.kappa >= 0) || !is_finite(d.kappa) || !(d.albedo >= 0 && d.albedo <= 1) || !(d.g > -1 && d.g < 1))
      return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: bad optics", m);
    if (!(d.luminosity > 0) || !is_finite(d.luminosity)) return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: luminosity", m);
    for (int a = 0; a < 3; ++a)
      if (!is_finite(d.source[a])) return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: source position", m);
    const rt_instrument_desc& q = d.instrument;
    if (q.nx < 1 || q.ny < 1 || !(q.half_x > 0) || !(q.half_y > 0) || q.channels != 1 ||
        (q.deposit != RT_DEPOSIT_NEAREST && q.deposit != RT_DEPOSIT_BILINEAR))
      return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: bad frame (channels must be 1)", m);
    if (d.n_packets < 1 || d.n_packets > 0xffffffffull)
      return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: packets in 1 .. 2^32 - 1", m);
    const size_t nc = (size_t)d.nx * d.ny * d.nz;
    for (size_t i = 0; i < nc; ++i)
      if (!(d.density[i] >= 0.0f) || !std::isfinite(d.density[i]))
        return fail(c, RT_ERR_ARG, "rt_batch_create: model %d: density must be finite and >= 0", m);
    n_cells_total += nc;
  }
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  Batch* b = new (std::nothrow) Batch();
  if (!b) return fail(c, RT_ERR_OOM, "rt_batch_create: host allocation");
  b->n_models = n_models;
  std::vector<DevModel> rows((size_t)n_models);
  std::vector<float> dens(n_cells_total);
  size_t off = 0;
  for (int m = 0; m < n_models; ++m) {
    const rt_model_desc& d = models[m];
    DevModel& M = rows[(size_t)m];
    std::memset(&M, 0, sizeof M);
    M.nx = d.nx; M.ny = d.ny; M.nz = d.nz;
    double mass = 0.0;
    const size_t nc = (size_t)d.nx * d.ny * d.nz;
    for (size_t i = 0; i < nc; ++i) mass += d.density[i];
    for (int a = 0; a < 3; ++a) {
      const int n = a == 0 ? d.nx : (a == 1 ? d.ny : d.nz);
      const double dd = (d.bounds[2 * a + 1] - d.bounds[2 * a]) / n;  // as rt_launch_packets
      M.lo[a] = (float)d.bounds[2 * a];
      M.hi[a] = (float)d.bounds[2 * a + 1];
      M.d[a] = (float)dd;
      M.inv_d[a] = (float)(1.0 / dd);
      M.src[a] = (float)d.source[a];
    }
    M.kappa = (float)d.kappa;
    M.g = (float)d.g;
    M.albedo = d.albedo;
    M.L0 = d.luminosity / (double)d.n_packets;
    M.density = (long long)off;
    std::memcpy(&dens[off], d.density, nc * sizeof(float));
    off += nc;
    double kobs[3], ex[3], ey[3];
    frame_axes(d.instrument, kobs, ex, ey);
    DevInstr& I = M.instr;
    for (int a = 0; a < 3; ++a) { I.kobs[a] = (float)kobs[a]; I.ex[a] = (float)ex[a]; I.ey[a] = (float)ey[a]; }
    I.off_x = (float)(d.instrument.half_x - d.instrument.center_x);
    I.off_y = (float)(d.instrument.half_y - d.instrument.center_y);
    I.sx = (float)(d.instrument.nx / (2.0 * d.instrument.half_x));
    I.sy = (float)(d.instrument.ny / (2.0 * d.instrument.half_y));
    I.nx = d.instrument.nx; I.ny = d.instrument.ny;
    I.bilinear = d.instrument.deposit == RT_DEPOSIT_BILINEAR;
    I.channels = 1;
    int axis = 0, dir = 0;
    if (frame_axis(I, axis, dir)) {
      I.axis = axis;
      I.dir = dir;
      I.column = reinterpret_cast<const float*>(1);  // marks "has column sums"; set after allocation
    }
    b->lum.push_back(d.luminosity);
    b->n_packets.push_back(d.n_packets);
    b->img_off.push_back(b->img_total);
    b->img_elems.push_back((size_t)d.instrument.nx * d.instrument.ny);
    b->img_total += (size_t)d.instrument.nx * d.instrument.ny;
    // work per packet ~ cells along a path x (1 + expected events), the
    // events from the mean optical depth across the model and the albedo
    const double side = (d.nx + d.ny + d.nz) / 3.0;
    const double tau = d.kappa * mass / (double)nc * (d.bounds[1] - d.bounds[0]);
    const double keep = std::max(1e-3, d.albedo * -std::expm1(-0.5 * tau));
    const double events = std::min(1000.0, std::log(1e-4) / std::log(std::min(keep, 0.999)));
    b->cost.push_back(side * (1.0 + events));
  }
  auto bail = [&](rt_status st) { free_batch(b); return st; };
  cudaError_t e = cudaSuccess;
  auto alloc = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(1, bytes));
  };
  alloc(&b->d_density, dens.size() * sizeof(float));
  bool any_columns = false;
  for (const DevModel& M : rows) any_columns = any_columns || M.instr.column != nullptr;
  if (any_columns) alloc(&b->d_columns, dens.size() * sizeof(float));
  alloc(&b->d_models, rows.size() * sizeof(DevModel));
  alloc(&b->d_images, b->img_total * sizeof(double));
  alloc(&b->d_tallies, (size_t)n_models * 4 * sizeof(double));
  alloc(&b->d_lum, (size_t)n_models * sizeof(double));
  alloc(&b->d_chunk_counter, sizeof(unsigned long long));
  alloc(&b->d_counters, 6 * sizeof(unsigned long long));
  alloc(&b->d_flags, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(c, RT_ERR_OOM, "rt_batch_create: device allocation: %s", cudaGetErrorString(e)));
  }
  for (int m = 0; m < n_models; ++m) {
    DevModel& M = rows[(size_t)m];
    M.instr.image = b->d_images + b->img_off[(size_t)m];
    if (M.instr.column) M.instr.column = b->d_columns + M.density;
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->d_density, dens.data(), dens.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_models, rows.data(), rows.size() * sizeof(DevModel), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_lum, b->lum.data(), b->lum.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_images, 0, b->img_total * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b->d_tallies, 0, (size_t)n_models * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, 6 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b->d_flags, 0, sizeof(int));
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "rt_batch_create: upload"));
  int per_sm = 0;
  e = batch_blocks_per_sm(&per_sm);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "rt_batch_create: occupancy"));
  b->blocks = (unsigned)(c->num_sms * std::max(1, per_sm));
  rt_status st = upload_chunks(c, b, 1024);
  if (st != RT_OK) return bail(st);
  c->batches.push_back(b);
  *batch_id = (int32_t)(c->batches.size() - 1);
  return RT_OK;
}

rt_status rt_batch_destroy(rt_ctx c, int32_t id) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  Batch* b = get_batch(c, id);
  if (!b) return fail(c, RT_ERR_ARG, "rt_batch_destroy: unknown batch %d", id);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  cudaDeviceSynchronize();
  free_batch(b);
  c->batches[(size_t)id] = nullptr;
  return RT_OK;
}

rt_status rt_batch_launch(rt_ctx c, int32_t id, uint64_t seed, const rt_launch_opts* opts, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  Batch* b = get_batch(c, id);
  if (!b) return fail(c, RT_ERR_ARG, "rt_batch_launch: unknown batch %d", id);
  rt_launch_opts o;
  rt_status st = batch_opts(c, opts, seed, o);
  if (st != RT_OK) return st;
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  const BatchParams p = batch_params(b, o, seed, b->d_chunks, b->n_chunks);
  if (!b->exec) {
    st = build_graph(c, b, p);
    if (st != RT_OK) return st;
  } else {
    BatchParams pc = p;
    void* kargs[] = {&pc};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = const_cast<void*>(batch_kernel());
    kp.gridDim = dim3(b->blocks);
    kp.blockDim = dim3(kBatchBlock);
    kp.kernelParams = kargs;
    RT_CUDA(c, cudaGraphExecKernelNodeSetParams(b->exec, b->kernel_node, &kp));
  }
  RT_CUDA(c, cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return RT_OK;
}

rt_status rt_batch_reset(rt_ctx c, int32_t id, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  Batch* b = get_batch(c, id);
  if (!b) return fail(c, RT_ERR_ARG, "rt_batch_reset: unknown batch %d", id);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  RT_CUDA(c, cudaMemsetAsync(b->d_images, 0, b->img_total * sizeof(double), s));
  RT_CUDA(c, cudaMemsetAsync(b->d_tallies, 0, (size_t)b->n_models * 4 * sizeof(double), s));
  RT_CUDA(c, cudaMemsetAsync(b->d_counters, 0, 6 * sizeof(unsigned long long), s));
  RT_CUDA(c, cudaMemsetAsync(b->d_flags, 0, sizeof(int), s));
  return RT_OK;
}

rt_status rt_batch_read_images(rt_ctx c, int32_t id, double* dst, size_t n_elems, int32_t on_device, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  Batch* b = get_batch(c, id);
  if (!b) return fail(c, RT_ERR_ARG, "rt_batch_read_images: unknown batch %d", id);
  if (!dst) return fail(c, RT_ERR_ARG, "rt_batch_read_images: null destination");
  if (n_elems != b->img_total) return fail(c, RT_ERR_ARG, "rt_batch_read_images: n_elems %zu != %zu", n_elems, b->img_total);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  return copy_out(c, dst, b->d_images, n_elems, on_device, stream);
}

rt_status rt_batch_read_tallies(rt_ctx c, int32_t id, double* dst, size_t n_elems, int32_t on_device, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  Batch* b = get_batch(c, id);
  if (!b) return fail(c, RT_ERR_ARG, "rt_batch_read_tallies: unknown batch %d", id);
  if (!dst) return fail(c, RT_ERR_ARG, "rt_batch_read_tallies: null destination");
  const size_t n = (size_t)b->n_models * 4;
  if (n_elems != n) return fail(c, RT_ERR_ARG, "rt_batch_read_tallies: n_elems %zu != %zu", n_elems, n);
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  return copy_out(c, dst, b->d_tallies, n, on_device, stream);
}

rt_status rt_batch_read_stats(rt_ctx c, int32_t id, rt_stats* out) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  Batch* b = get_batch(c, id);
  if (!b) return fail(c, RT_ERR_ARG, "rt_batch_read_stats: unknown batch %d", id);
  if (!out) return fail(c, RT_ERR_ARG, "rt_batch_read_stats: null output");
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  RT_CUDA(c, cudaDeviceSynchronize());
  std::vector<double> t((size_t)b->n_models * 4);
  unsigned long long cn[6];
  int flags = 0;
  RT_CUDA(c, cudaMemcpy(t.data(), b->d_tallies, t.size() * sizeof(double), cudaMemcpyDeviceToHost));
  RT_CUDA(c, cudaMemcpy(cn, b->d_counters, sizeof cn, cudaMemcpyDeviceToHost));
  RT_CUDA(c, cudaMemcpy(&flags, b->d_flags, sizeof flags, cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof *out);
  for (int m = 0; m < b->n_models; ++m) {
    out->emitted += t[(size_t)m * 4];
    out->escaped += t[(size_t)m * 4 + 1];
    out->absorbed += t[(size_t)m * 4 + 2];
    out->truncated += t[(size_t)m * 4 + 3];
  }
  out->crossings = cn[0]; out->events = cn[1]; out->peeloffs = cn[2]; out->packets = cn[3];
  out->column_peels = cn[4]; out->column_crossings = cn[5];
  out->device_flags = flags;
  if (flags) return fail(c, RT_ERR_DEVICE_FLAG, "a kernel bounds check fired (flags 0x%x)", flags);
  return RT_OK;
}

rt_status rt_batch_tune(rt_ctx c, int32_t id, uint64_t seed, double fraction, int32_t* control_lanes,
                        uint32_t* run_packets, void* stream) {
  if (!c) return RT_ERR_ARG;
  c->err.clear();
  Batch* b = get_batch(c, id);
  if (!b) return fail(c, RT_ERR_ARG, "rt_batch_tune: unknown batch %d", id);
  if (!(fraction > 0 && fraction <= 1)) return fail(c, RT_ERR_ARG, "rt_batch_tune: fraction in (0, 1]");
  rt_launch_opts o;
  rt_status st = batch_opts(c, nullptr, seed, o);
  if (st != RT_OK) return st;
  if (set_device(c) != RT_OK) return RT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const int lanes_c[] = {8, 12, 16, 20, 24, 28, 32};
  const unsigned runs_c[] = {64, 256, 1024, 4096};
  RT_CUDA(c, launch_batch_columns(b->d_models, b->n_models, b->d_density, s));
  cudaEvent_t e0, e1;
  RT_CUDA(c, cudaEventCreate(&e0));
  RT_CUDA(c, cudaEventCreate(&e1));
  float best = -1.0f;
  int best_lanes = 16;
  unsigned best_run = 1024;
  BatchChunk* d_ch = nullptr;
  cudaError_t e = cudaSuccess;
  for (unsigned run : runs_c) {
    const std::vector<BatchChunk> ch = batch_chunks(*b, run, fraction);
    dfree(d_ch);
    e = cudaMalloc(&d_ch, std::max<size_t>(1, ch.size()) * sizeof(BatchChunk));
    if (e == cudaSuccess) e = cudaMemcpy(d_ch, ch.data(), ch.size() * sizeof(BatchChunk), cudaMemcpyHostToDevice);
    for (int lanes : lanes_c) {
      if (e != cudaSuccess) break;
      o.control_lanes = lanes;
      const BatchParams p = batch_params(b, o, seed, d_ch, (int)ch.size());
      e = cudaMemsetAsync(b->d_chunk_counter, 0, sizeof(unsigned long long), s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = launch_batch(p, b->blocks, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && (best < 0 || ms < best)) {
        best = ms;
        best_lanes = lanes;
        best_run = run;
      }
    }
  }
  dfree(d_ch);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(c, e, "rt_batch_tune");
  b->control_lanes = best_lanes;
  if (best_run != b->run_packets) {
    st = upload_chunks(c, b, best_run);
    if (st != RT_OK) return st;
  }
  if (control_lanes) *control_lanes = best_lanes;
  if (run_packets) *run_packets = best_run;
  return rt_batch_reset(c, id, stream);
}

}  // extern "C"

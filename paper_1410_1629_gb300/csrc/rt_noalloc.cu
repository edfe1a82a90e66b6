// rt_launch_packets_noalloc: the cartesian forward transport without any
// device allocation, for callers that cannot allocate GPU memory themselves.
//
// Who needs this: code that must not call cudaMalloc or any allocating
// library routine while it runs -- for example a plug-in executed inside
// another framework that owns the whole device memory pool, or a service
// with a fixed memory budget checked at start-up.  Such a caller keeps its
// own device buffers for the inputs and outputs and needs the library to
// bring nothing else but a fixed, preallocated working area.
//
// The working area is the file-scope array `g_noalloc_scratch` below, a
// __device__ array of kNoallocScratchBytes bytes that every GPU which loads
// this library holds until the process exits.  It carries the packet work
// counter, the tallies and the device flags of one launch, and the small
// per-launch tables (optics per wavelength, sources, instruments).  Host code
// cannot use the array's name as a device address: every call looks the
// address up with cudaGetSymbolAddress on the current device (a lookup that
// allocates nothing, repeated per call so that a reset device never leaves a
// stale address behind).  The first call on a device also loads the library's
// device code there, so it should come before any stream capture on that
// device.  The per-launch tables travel to the working area as the parameter
// of a small set-up kernel (by value), never as a copy from host memory, so
// no queued work refers to the caller's stack.  Every call uses the same array
// and the array keeps the last call's contents; a call clears the parts that
// must start at zero.  Two calls that overlap on the GPU (different streams,
// or different host threads on one device) race on the array.
#include <cmath>
#include <cstring>
#include <cstddef>

#include <cuda_runtime.h>

#include "rt_internal.h"

using namespace rtk;

namespace {

constexpr size_t kNoallocScratchBytes = 16384;

// The per-launch tables, passed by value to the set-up kernel and kept in the
// working area after its first 256 bytes.
struct NoallocTables {
  DevLambda lam[kMaxLambda];
  DevSource src[kMaxSources];
  double cum[kMaxLambda * kMaxSources];  // [n_lambda][n_sources] cumulative luminosity fractions
  DevInstr ins[kMaxInstruments];
};

// Byte offsets inside the working area.
constexpr size_t kOffWork = 0;       // 1 x u64
constexpr size_t kOffStats = 16;     // 4 x f64
constexpr size_t kOffCounters = 48;  // 8 x u64
constexpr size_t kOffFlags = 112;    // 1 x i32
constexpr size_t kOffTables = 256;   // NoallocTables
constexpr size_t kOffLam = kOffTables + offsetof(NoallocTables, lam);
constexpr size_t kOffSrc = kOffTables + offsetof(NoallocTables, src);
constexpr size_t kOffCum = kOffTables + offsetof(NoallocTables, cum);
constexpr size_t kOffInstr = kOffTables + offsetof(NoallocTables, ins);
static_assert(kOffTables + sizeof(NoallocTables) <= kNoallocScratchBytes, "working area too small for its layout");
// a kernel parameter may hold up to 32764 bytes (CUDA 12.1 and later)
static_assert(sizeof(NoallocTables) <= 32000, "tables too large for a kernel parameter");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of the working area on the current device.
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

// Clears the counters, tallies and flags and writes the launch's tables into
// the working area.
__global__ void k_noalloc_setup(const NoallocTables t, unsigned char* scratch) {
  const unsigned* src = reinterpret_cast<const unsigned*>(&t);
  unsigned* dst = reinterpret_cast<unsigned*>(scratch + kOffTables);
  for (unsigned i = threadIdx.x; i < sizeof(NoallocTables) / 4; i += blockDim.x) dst[i] = src[i];
  unsigned* head = reinterpret_cast<unsigned*>(scratch);
  if (threadIdx.x < kOffTables / 4) head[threadIdx.x] = 0u;
}

// Packs the launch's tallies from the working area into an rt_stats.
__global__ void k_noalloc_stats(const unsigned char* scratch, double emitted, rt_stats* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double* st = reinterpret_cast<const double*>(scratch + kOffStats);
  const unsigned long long* cn = reinterpret_cast<const unsigned long long*>(scratch + kOffCounters);
  const int* flags = reinterpret_cast<const int*>(scratch + kOffFlags);
  rt_stats s;
  s.emitted = emitted;
  s.escaped = st[1];
  s.absorbed = st[2];
  s.truncated = st[3];
  s.crossings = cn[0];
  s.path_crossings = cn[5];
  s.events = cn[1];
  s.peeloffs = cn[2];
  s.packets = cn[3];
  s.records = cn[4];
  s.column_peels = cn[6];
  s.column_crossings = cn[7];
  s.sorted_peels = 0;
  s.device_flags = *flags;
  s.reserved = 0;
  *out = s;
}

rt_status fail(rt_status code, const char* msg) {
  set_context_free_error(msg);
  return code;
}

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace

extern "C" rt_status rt_launch_packets_noalloc(const rt_grid_desc* grid, int32_t n_lambda, const double* kappa,
                                               const double* albedo, const double* g, int32_t n_sources,
                                               const rt_source_desc* sources, int32_t n_instruments,
                                               const rt_instrument_desc* instruments, double* const* images,
                                               double* absorption, uint64_t n_per_lambda, uint64_t first_packet_id,
                                               uint64_t seed, const rt_launch_opts* opts, rt_stats* stats_out,
                                               void* stream) {
  set_context_free_error("");
  // ---- arguments (the same rules as the context calls, plus the fixed limits)
  if (!grid || grid->kind != RT_GRID_CARTESIAN)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: a cartesian grid descriptor is required");
  if (!grid->on_device || !grid->density)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: the density must be a device pointer (on_device = 1)");
  if (grid->nx <= 0 || grid->ny <= 0 || grid->nz <= 0 || (long long)grid->nx * grid->ny * grid->nz > (1ll << 31) - 1)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: bad cell counts");
  for (int a = 0; a < 3; ++a)
    if (!(std::isfinite(grid->bounds[2 * a]) && std::isfinite(grid->bounds[2 * a + 1]) &&
          grid->bounds[2 * a] < grid->bounds[2 * a + 1]))
      return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: bounds are not increasing");
  if (n_lambda < 1 || n_lambda > kMaxLambda)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: n_lambda must be 1..64 (working-area limit)");
  if (n_sources < 1 || n_sources > kMaxSources)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: n_sources must be 1..16 (working-area limit)");
  if (n_instruments < 0 || n_instruments > kMaxInstruments)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: n_instruments must be 0..16 (working-area limit)");
  if (!kappa || !albedo || !g || !sources || (n_instruments > 0 && (!instruments || !images)) || !absorption)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: null array");
  if (seed >> 32) return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: seed must be < 2^32");
  for (int l = 0; l < n_lambda; ++l) {
    if (!(std::isfinite(kappa[l]) && kappa[l] >= 0) || !(albedo[l] >= 0 && albedo[l] <= 1) || !(g[l] > -1 && g[l] < 1))
      return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: invalid optical properties");
  }
  for (int i = 0; i < n_sources; ++i) {
    const rt_source_desc& d = sources[i];
    if (d.kind < RT_SOURCE_POINT || d.kind > RT_SOURCE_PLUMMER || !d.luminosity || !finite3(d.center) ||
        (d.kind != RT_SOURCE_POINT && !(d.scale_r > 0)) || (d.kind == RT_SOURCE_EXPDISK && !(d.scale_z > 0)))
      return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: invalid source");
    for (int l = 0; l < n_lambda; ++l)
      if (!(std::isfinite(d.luminosity[l]) && d.luminosity[l] >= 0))
        return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: invalid source luminosity");
  }
  for (int q = 0; q < n_instruments; ++q) {
    const rt_instrument_desc& d = instruments[q];
    const bool sed = d.deposit == RT_DEPOSIT_SED;
    if (d.nx <= 0 || d.ny <= 0 || (long long)d.nx * d.ny > (1ll << 28) || (!sed && !(d.half_x > 0 && d.half_y > 0)) ||
        (sed && (d.nx != 1 || d.ny != 1)) || (d.channels != 1 && d.channels != 3) ||
        (d.deposit != RT_DEPOSIT_NEAREST && d.deposit != RT_DEPOSIT_BILINEAR && !sed) || !images[q])
      return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: invalid instrument or null image");
  }
  rt_launch_opts o;
  rt_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_events < 1 || !(o.w_min >= 0 && o.w_min < 1) || o.control_lanes < 0 || o.control_lanes > 32)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: invalid launch options");
  if ((o.records && o.records_capacity < 0) || (o.trace && o.trace_capacity < 0))
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: negative record or trace capacity");
  if (o.tape || o.time_parts)
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: the adjoint tape and part timings need a context");
  // ---- the working area of the current device
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, cudaGetErrorString(e));
  unsigned char* scratch = nullptr;
  e = scratch_address(&scratch);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, cudaGetErrorString(e));
  int num_sms = 0;
  e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, cudaGetErrorString(e));
  if (n_per_lambda == 0) return RT_OK;
  const unsigned long long n_total = n_per_lambda * (unsigned long long)n_lambda;
  if (n_total / (unsigned long long)n_lambda != n_per_lambda || n_total > (1ull << 62))
    return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: packet count overflow");
  // ---- per-launch tables, handed to the set-up kernel by value
  NoallocTables t;
  std::memset(&t, 0, sizeof t);
  DevLambda* lam = t.lam;
  DevSource* src = t.src;
  double* cum = t.cum;
  DevInstr* ins = t.ins;
  FwdParams p;
  std::memset(&p, 0, sizeof p);
  const unsigned long long n_norm = o.n_norm ? o.n_norm : n_per_lambda;
  double emitted = 0.0;
  for (int l = 0; l < n_lambda; ++l) {
    double tot = 0.0;
    for (int i = 0; i < n_sources; ++i) tot += sources[i].luminosity[l];
    if (!(tot > 0)) return fail(RT_ERR_ARG, "rt_launch_packets_noalloc: zero total luminosity at a wavelength");
    lam[l].kappa = (float)kappa[l];
    lam[l].g = (float)g[l];
    lam[l].albedo = albedo[l];
    lam[l].one_minus_albedo = 1.0 - albedo[l];
    lam[l].lum_total = tot;
    double run = 0.0;
    for (int i = 0; i < n_sources; ++i) {
      run += sources[i].luminosity[l];
      cum[l * n_sources + i] = run / tot;
    }
    p.L0[l] = tot / (double)n_norm;
    p.L_cut[l] = o.w_min * p.L0[l];
    emitted += (double)n_per_lambda * p.L0[l];
  }
  for (int i = 0; i < n_sources; ++i) {
    src[i].kind = sources[i].kind;
    for (int a = 0; a < 3; ++a) src[i].center[a] = sources[i].center[a];
    src[i].scale_r = sources[i].scale_r;
    src[i].scale_z = sources[i].scale_z;
  }
  for (int q = 0; q < n_instruments; ++q) {
    const rt_instrument_desc& d = instruments[q];
    double kobs[3], ex[3], ey[3];
    frame_axes(d.inclination, d.azimuth, d.position_angle, kobs, ex, ey);
    for (int i = 0; i < 3; ++i) {
      ins[q].kobs[i] = (float)kobs[i];
      ins[q].ex[i] = (float)ex[i];
      ins[q].ey[i] = (float)ey[i];
    }
    ins[q].off_x = (float)(d.half_x - d.center_x);
    ins[q].off_y = (float)(d.half_y - d.center_y);
    ins[q].sx = (float)(d.nx / (2.0 * d.half_x));
    ins[q].sy = (float)(d.ny / (2.0 * d.half_y));
    ins[q].nx = d.nx;
    ins[q].ny = d.ny;
    ins[q].bilinear = d.deposit == RT_DEPOSIT_BILINEAR;
    ins[q].sed = d.deposit == RT_DEPOSIT_SED;
    ins[q].channels = d.channels;
    ins[q].image = images[q];
  }
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_setup<<<1, 256, 0, s>>>(t, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(RT_ERR_CUDA, cudaGetErrorString(e));
  // ---- the launch, exactly as rt_launch_packets builds it
  p.nx = grid->nx; p.ny = grid->ny; p.nz = grid->nz;
  const int n3[3] = {grid->nx, grid->ny, grid->nz};
  for (int a = 0; a < 3; ++a) {
    p.lo[a] = (float)grid->bounds[2 * a];
    p.hi[a] = (float)grid->bounds[2 * a + 1];
    const double d = (grid->bounds[2 * a + 1] - grid->bounds[2 * a]) / n3[a];
    p.d[a] = (float)d;
    p.inv_d[a] = (float)(1.0 / d);
  }
  p.density = grid->density;
  row_major_strides(p);
  p.child = nullptr;
  p.n_cells = (long long)grid->nx * grid->ny * grid->nz;
  p.n_lambda = n_lambda;
  p.n_sources = n_sources;
  p.n_instr = n_instruments;
  p.lam = reinterpret_cast<const DevLambda*>(scratch + kOffLam);
  p.src = reinterpret_cast<const DevSource*>(scratch + kOffSrc);
  p.src_cum = reinterpret_cast<const double*>(scratch + kOffCum);
  p.instr = reinterpret_cast<const DevInstr*>(scratch + kOffInstr);
  p.absorption = absorption;
  p.n_per_lambda = n_per_lambda;
  p.first_id = first_packet_id;
  p.n_total = n_total;
  p.n_norm = n_norm;
  p.seed = (unsigned)seed;
  p.model = o.model_id;
  p.w_min = o.w_min;
  p.max_events = o.max_events;
  p.weight_cut = o.weight_cut;
  p.peel_emission = o.peel_emission;
  p.peel_scatter = o.peel_scatter;
  p.work_counter = reinterpret_cast<unsigned long long*>(scratch + kOffWork);
  p.stats = reinterpret_cast<double*>(scratch + kOffStats);
  p.counters = reinterpret_cast<unsigned long long*>(scratch + kOffCounters);
  p.records = o.records;
  p.records_cap = o.records ? o.records_capacity : 0;
  p.record_stride = o.record_stride;
  p.trace = o.trace;
  p.trace_cap = o.trace ? o.trace_capacity : 0;
  p.trace_packet = o.trace_packet;
  p.trace_lambda = o.trace_lambda;
  p.control_min = o.control_lanes ? o.control_lanes : 16;
  p.profile = reinterpret_cast<unsigned long long*>(o.profile);
  p.inv_n_per_lambda = (float)(1.0 / (double)n_per_lambda);
  p.flags = reinterpret_cast<int*>(scratch + kOffFlags);
  e = launch_forward(p, RT_GRID_CARTESIAN, num_sms, s);
  if (e != cudaSuccess) return fail(RT_ERR_CUDA, cudaGetErrorString(e));
  if (stats_out) {
    k_noalloc_stats<<<1, 32, 0, s>>>(scratch, emitted, stats_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RT_ERR_CUDA, cudaGetErrorString(e));
  }
  return RT_OK;
}

// Many small independent models in one persistent launch: parameter
// searches run the same transport on thousands of small grids (the model
// fitting of Sect. 1), each too small to fill a GB300 alone.
//
// Every model is a cartesian grid with one wavelength, one point source and
// one single-channel frame; its packets are the forward kernel's packets with
// Philox key (seed, model index), computed with the same arithmetic, so a
// model of a batch gives the tallies of rt_launch_packets on that model
// with model_id = its index.
//
// Work list: runs of packets of one model (chunks), sorted by estimated cost,
// largest first, so that the long runs start early and the short ones fill
// the tail.  A warp takes a chunk with one atomic and hands its packets to
// its lanes as they need them; lanes of a warp may hold packets of different
// models.  A lane keeps its model's grid geometry in its own shared-memory
// slot (the cell walk reads it there), and the model's escaped / absorbed /
// truncated luminosity in another, flushed to the model's FP64 tallies when
// the lane moves to another model.
#include "rt_transport.cuh"

namespace rtk {

namespace {

using tr::CartGrid;

// Grid geometry of a lane's model, in the shape CartGrid reads.
struct Geo {
  int nx, ny, nz, pad;
  float lo[3], hi[3], d[3], inv_d[3];
};

struct Tally {
  double escaped, absorbed, truncated;
  int model, pad;
  unsigned long long column_peels, column_crossings;  // the lane's, over the launch
};

__shared__ Geo S_GEO[kBatchBlock];
__shared__ Tally S_TALLY[kBatchBlock];

// The lane state that only the per-event work touches sits in the transport
// kernels' per-thread shared-memory slots, so that the walk's state fits the
// registers of four resident blocks per SM.
#ifndef RT_BATCH_MIN_BLOCKS
#define RT_BATCH_MIN_BLOCKS 4
#endif
static_assert(kBatchBlock == tr::kBlock, "per-thread slots are sized for the transport block");

struct BLane {
  int m, phase;
  float kappa;
  float3 x;
  bool walking;
  // in shared memory: packet id, event index, peel-off done (1) or not (0)
  // for this event, the walk a kStart lane begins, weight, direction of
  // travel, the event's Henyey-Greenstein uniforms, the cell of x (valid when
  // has_cell)
  __device__ __forceinline__ unsigned long long& pid() const { return tr::S_PID[threadIdx.x]; }
  __device__ __forceinline__ int& event() const { return tr::S_EVENT[threadIdx.x]; }
  __device__ __forceinline__ int& q() const { return tr::S_INSTR_Q[threadIdx.x]; }
  __device__ __forceinline__ int& wphase() const { return tr::S_WPHASE[threadIdx.x]; }
  __device__ __forceinline__ double& L() const { return tr::S_WEIGHT[threadIdx.x]; }
  __device__ __forceinline__ float3& k() const { return tr::S_DIR[threadIdx.x]; }
  __device__ __forceinline__ float& u_mu() const { return tr::S_HG[threadIdx.x].x; }
  __device__ __forceinline__ float& u_phi() const { return tr::S_HG[threadIdx.x].y; }
  __device__ __forceinline__ CartGrid::Cell& cell() const { return tr::S_CELL_CART[threadIdx.x]; }
  __device__ __forceinline__ bool& has_cell() const { return tr::S_HAS_CELL[threadIdx.x]; }
  float3 d, id;
  CartGrid::Walk w;
  float rho;
  float th, tl;
  float aux0, aux1;   // path 1: deposit weight (unused here); path 2: tau* pair, then s*
  const float* dens;  // the model's densities
};

__device__ __forceinline__ void flush(const BatchParams& P, Tally& t) {
  if (t.model >= 0) {
    double* q = &P.tallies[(size_t)t.model * 4];
    if (t.escaped != 0.0) atomicAdd(&q[1], t.escaped);
    if (t.absorbed != 0.0) atomicAdd(&q[2], t.absorbed);
    if (t.truncated != 0.0) atomicAdd(&q[3], t.truncated);
  }
  t.escaped = t.absorbed = t.truncated = 0.0;
}

__device__ __forceinline__ void start_walk(BLane& s, const Geo& G, float3 d) {
  s.d = d;
  s.id = make_float3(tr::inv_or_zero(d.x), tr::inv_or_zero(d.y), tr::inv_or_zero(d.z));
  s.th = 0.0f;
  s.tl = 0.0f;
  CartGrid::Scratch sc;
  s.walking = CartGrid::init(G, s.x, d, s.id, s.has_cell(), s.cell(), s.w, sc);
  if (s.walking) s.rho = tr::load_density(&s.dens[s.w.cell]);
}

__device__ __forceinline__ float3 kobs(const DevInstr& I) { return make_float3(I.kobs[0], I.kobs[1], I.kobs[2]); }

// The forward kernel's peel-off deposit for a single-channel frame.
__device__ __forceinline__ void deposit(const DevModel& M, const BLane& s, bool scattered) {
  const DevInstr& I = M.instr;
  float phase = 1.0f;
  if (scattered) phase = hg_phase(M.g, s.k().x * I.kobs[0] + s.k().y * I.kobs[1] + s.k().z * I.kobs[2]);
  const float tau = s.th;
  const double value = tau < 80.0f ? s.L() * tr::widen(tr::kInv4PiF * phase * expf(-tau) * (1.0f - s.tl))
                                   : s.L() * kInv4PiD * (double)phase * exp(-((double)tau + (double)s.tl));
  const float fx = (s.x.x * I.ex[0] + s.x.y * I.ex[1] + s.x.z * I.ex[2] + I.off_x) * I.sx;
  const float fy = (s.x.x * I.ey[0] + s.x.y * I.ey[1] + s.x.z * I.ey[2] + I.off_y) * I.sy;
  if (!I.bilinear) {
    const float fix = floorf(fx), fiy = floorf(fy);
    if (!(fix >= 0.0f && fiy >= 0.0f && fix < (float)I.nx && fiy < (float)I.ny)) return;
    atomicAdd(&I.image[(size_t)(int)fiy * I.nx + (int)fix], value);
    return;
  }
  const float gx = fx - 0.5f, gy = fy - 0.5f;
  const float x0 = floorf(gx), y0 = floorf(gy);
  const float tx = gx - x0, ty = gy - y0;
#pragma unroll
  for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
    for (int dx = 0; dx < 2; ++dx) {
      const float fix = x0 + dx, fiy = y0 + dy;
      if (!(fix >= 0.0f && fiy >= 0.0f && fix < (float)I.nx && fiy < (float)I.ny)) continue;
      const double v = value * tr::widen((dx ? tx : 1.0f - tx) * (dy ? ty : 1.0f - ty));
      atomicAdd(&I.image[(size_t)(int)fiy * I.nx + (int)fix], v);
    }
  }
}

// The forward kernel's column shortcut for a frame along a grid axis (see
// column_peel there); false when the position is outside the grid.
__device__ __forceinline__ bool column_peel(const DevInstr& I, BLane& s, const Geo& G, Tally& T,
                                            unsigned& n_cross) {
  CartGrid::Cell c;
  if (s.has_cell()) {
    c = s.cell();
  } else {
    if (!inside_box(G, s.x)) return false;
    c.ix = min(max(__float2int_rd((s.x.x - G.lo[0]) * G.inv_d[0]), 0), G.nx - 1);
    c.iy = min(max(__float2int_rd((s.x.y - G.lo[1]) * G.inv_d[1]), 0), G.ny - 1);
    c.iz = min(max(__float2int_rd((s.x.z - G.lo[2]) * G.inv_d[2]), 0), G.nz - 1);
  }
  const int a = I.axis;
  const bool up = I.dir > 0;
  const int i = a == 0 ? c.ix : (a == 1 ? c.iy : c.iz);
  const int n = a == 0 ? G.nx : (a == 1 ? G.ny : G.nz);
  const float xa = a == 0 ? s.x.x : (a == 1 ? s.x.y : s.x.z);
  const float plane = fmaf((float)(i + (up ? 1 : 0)), G.d[a], G.lo[a]);
  const float ds0 = fmaxf(up ? plane - xa : xa - plane, 0.0f);
  const int cell = c.ix + G.nx * (c.iy + G.ny * c.iz);
  s.th = s.kappa * fmaf(tr::load_density(&s.dens[cell]), ds0, __ldg(&I.column[cell]));
  s.tl = 0.0f;
  s.walking = false;
  const unsigned nc = (unsigned)(up ? n - i : i + 1);
  n_cross += nc;
  T.column_peels += 1ull;
  T.column_crossings += nc;
  return true;
}

// Ask for walk `phase` from the lane's position along d (started in the last
// stage of a control round, from one place in the code).
__device__ __forceinline__ void request_walk(BLane& s, int phase, float3 d) {
  s.wphase() = phase;
  s.d = d;
  s.phase = tr::kStart;
}

// ---- the stages of a control round (the forward kernel's, for one frame
// per model and no absorption field)

// A new packet (model m, packet id pid): the model's geometry, emission from
// its point source (the forward kernel's event-0 draws).
__device__ __forceinline__ void begin(const BatchParams& P, BLane& s, Geo& G, Tally& T, int m,
                                      unsigned long long pid) {
  const DevModel& M = P.models[m];
  if (T.model != m) {
    flush(P, T);
    T.model = m;
  }
  G.nx = M.nx; G.ny = M.ny; G.nz = M.nz;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    G.lo[a] = M.lo[a]; G.hi[a] = M.hi[a]; G.d[a] = M.d[a]; G.inv_d[a] = M.inv_d[a];
  }
  s.m = m;
  s.pid() = pid;
  s.dens = P.density + M.density;
  s.kappa = M.kappa;
  s.L() = M.L0;
  s.event() = 0;
  s.has_cell() = false;
  // one point source: the position draws of block 0 are not needed
  const uint4 r1 = draw_block(pid, 0, 0, 1, P.seed, (unsigned)m);
  s.x = make_float3(M.src[0], M.src[1], M.src[2]);
  const float mu = tr::u01f_signed(r1.z);
  const float st = sqrtf(fmaxf(0.0f, 1.0f - mu * mu));
  float sp, cp;
  sincospif(2.0f * tr::u01f(r1.w), &sp, &cp);
  s.k() = make_float3(st * cp, st * sp, mu);
  s.q() = 0;
  s.phase = tr::kPeelScan;
}

__device__ __forceinline__ void finish_path1(const BatchParams& P, BLane& s, Tally& T) {
  const DevModel& M = P.models[s.m];
  const double tau = tr::widen(s.th) + tr::widen(s.tl);
  if (!(tau > 0.0)) {
    T.escaped += s.L();
    s.phase = tr::kFetch;
    return;
  }
  const double albedo = M.albedo;
  const double one_minus_E = -expm1(-tau);
  const double E = 1.0 - one_minus_E;
  T.escaped += s.L() * E;
  T.absorbed += (1.0 - albedo) * s.L() * one_minus_E;
  const uint4 r = draw_block(s.pid(), 0, s.event(), 0, P.seed, (unsigned)s.m);
  const double tau_star = -log1p(-u01(r.x) * one_minus_E);
  s.u_mu() = tr::u01f(r.y);
  s.u_phi() = tr::u01f(r.z);
  tr::split_pair(tau_star, s.aux0, s.aux1);
  s.L() = albedo * s.L() * one_minus_E;
  request_walk(s, tr::kPath2, s.k());
}

__device__ __forceinline__ void finish_path2(const Geo& G, BLane& s, unsigned& n_events) {
  const float s_star = s.aux0;
  float3 x = make_float3(fmaf(s_star, s.k().x, s.x.x), fmaf(s_star, s.k().y, s.x.y), fmaf(s_star, s.k().z, s.x.z));
  s.cell() = CartGrid::carried(s.w);
  CartGrid::clamp(G, s.cell(), x);
  s.x = x;
  s.has_cell() = true;
  n_events += 1u;
  s.q() = 0;
  s.phase = tr::kPeelScan;
}

// The model's one peel-off of this event, or what follows it.
__device__ __forceinline__ void peel_scan(const BatchParams& P, BLane& s, const Geo& G, Tally& T,
                                          unsigned& n_cross) {
  const bool emission = s.event() == 0;
  if ((emission ? P.peel_emission : P.peel_scatter) && s.q() == 0) {
    const DevInstr& I = P.models[s.m].instr;
    const int phase = emission ? tr::kPeelEmit : tr::kPeelScat;
    if (P.use_columns && I.column && column_peel(I, s, G, T, n_cross)) {
      s.phase = phase;
      return;
    }
    request_walk(s, phase, kobs(I));
    return;
  }
  if (emission) {
    s.event() = 1;
    request_walk(s, tr::kPath1, s.k());
  } else {
    s.phase = tr::kAfter;
  }
}

__device__ __forceinline__ void after_scattering(const BatchParams& P, BLane& s, Tally& T) {
  const DevModel& M = P.models[s.m];
  const float mu = hg_sample(M.g, s.u_mu());
  float sp, cp;
  sincospif(2.0f * s.u_phi(), &sp, &cp);
  s.k() = rotate_dir(s.k(), mu, sp, cp);
  if ((P.weight_cut && s.L() < P.w_min * M.L0) || s.event() >= P.max_events) {
    T.truncated += s.L();
    s.phase = tr::kFetch;
    return;
  }
  s.event() += 1;
  request_walk(s, tr::kPath1, s.k());
}

// One cell crossing (the forward kernel's step without the absorption field).
__device__ __forceinline__ void step(const BatchParams& P, BLane& s, const Geo& G, unsigned& n_cross) {
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
  const bool path2 = s.phase == tr::kPath2;
  if (path2 && (nh - s.aux0) + (nl - s.aux1) > 0.0f) {
    const float rem = ((s.aux0 - s.th) + s.aux1) - s.tl;
    s.aux0 = w.t + rem / kr;
    s.walking = false;
    return;
  }
  s.th = nh;
  s.tl = nl;
  n_cross += path2 ? 0u : 1u;
  w.t = texit;
  CartGrid::Scratch sc;
  if (CartGrid::advance(G, s.x, s.d, s.id, axis, w, sc)) {
    s.rho = tr::load_density(&s.dens[w.cell]);
  } else {
    s.walking = false;
    if (path2) {  // not reachable (see the forward kernel)
      atomicOr(P.flags, kFlagNoInteraction);
      s.aux0 = texit;
    }
  }
}

__global__ void __launch_bounds__(kBatchBlock, RT_BATCH_MIN_BLOCKS) k_batch(const BatchParams P) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  Geo& G = S_GEO[threadIdx.x];
  Tally& T = S_TALLY[threadIdx.x];
  T.escaped = T.absorbed = T.truncated = 0.0;
  T.model = -1;
  T.column_peels = T.column_crossings = 0ull;
  BLane s;
  s.phase = tr::kFetch;
  s.walking = false;
  s.m = 0;
  unsigned n_cross = 0, n_events = 0, n_peel = 0, n_packets = 0;
  unsigned long long tot_cross = 0;
  // the warp's current chunk (the same in every lane)
  unsigned long long c_next = 0, c_end = 0;
  int c_model = 0;
  bool drained = false;
  while (true) {
    const bool idle = !s.walking && s.phase != tr::kExit;
    const unsigned need = __ballot_sync(0xffffffffu, idle);
    const unsigned walkers = __ballot_sync(0xffffffffu, s.walking);
    if (need == 0u && walkers == 0u) break;
    if (walkers == 0u || __popc(need) >= P.control_min) {
      // per-event work in stages, each run by the lanes in its phase together
      if (!s.walking) {
        if (s.phase == tr::kPath1) finish_path1(P, s, T);
        if (s.phase == tr::kPath2) finish_path2(G, s, n_events);
      }
      // peel-offs, the scattering and new packets, repeated while a lane has
      // just finished its packet (at most two passes)
      while (true) {
        while (true) {
          const bool ready = !s.walking && (s.phase == tr::kPeelEmit || s.phase == tr::kPeelScat);
          if (!__any_sync(0xffffffffu, ready || s.phase == tr::kPeelScan)) break;
          if (ready) {
            deposit(P.models[s.m], s, s.phase == tr::kPeelScat);
            n_peel += 1u;
            s.q() = 1;
            s.phase = tr::kPeelScan;
          }
          if (s.phase == tr::kPeelScan) peel_scan(P, s, G, T, n_cross);
        }
        if (s.phase == tr::kAfter) after_scattering(P, s, T);
        const bool wants = !s.walking && s.phase == tr::kFetch;
        const unsigned fetchers = __ballot_sync(0xffffffffu, wants);
        if (!fetchers) break;
        // hand out packets of the warp's chunk, taking new chunks as needed
        const int rank = __popc(fetchers & lt_mask);
        int remaining = __popc(fetchers), done = 0;
        int my_model = -1;
        unsigned long long my_pid = 0;
        while (remaining > 0 && !drained) {
          if (c_next >= c_end) {
            unsigned long long ci = 0;
            if (lane == 0) ci = atomicAdd(P.chunk_counter, 1ull);
            ci = __shfl_sync(0xffffffffu, ci, 0);
            if (ci >= (unsigned long long)P.n_chunks) {
              drained = true;
              break;
            }
            const BatchChunk ch = P.chunks[ci];
            c_model = ch.model;
            c_next = ch.first;
            c_end = ch.first + ch.count;
          }
          const unsigned long long avail = c_end - c_next;
          const int take = avail < (unsigned long long)remaining ? (int)avail : remaining;
          if (wants && rank >= done && rank < done + take) {
            my_model = c_model;
            my_pid = c_next + (unsigned long long)(rank - done);
          }
          c_next += (unsigned long long)take;
          done += take;
          remaining -= take;
        }
        if (wants) {
          if (my_model >= 0) {
            begin(P, s, G, T, my_model, my_pid);
            n_packets += 1u;
          } else {
            s.phase = tr::kExit;
          }
        }
      }
      if (s.phase == tr::kStart) {
        s.phase = s.wphase();
        start_walk(s, G, s.d);
      }
      if (n_cross & 0xC0000000u) {
        tot_cross += n_cross;
        n_cross = 0;
      }
    }
    if (s.walking) step(P, s, G, n_cross);
  }
  flush(P, T);
  tot_cross += n_cross;
  unsigned long long ev = n_events, pe = n_peel, pk = n_packets, cp = T.column_peels, cc = T.column_crossings;
  for (int o = 16; o > 0; o >>= 1) {
    cp += __shfl_down_sync(0xffffffffu, cp, o);
    cc += __shfl_down_sync(0xffffffffu, cc, o);
    tot_cross += __shfl_down_sync(0xffffffffu, tot_cross, o);
    ev += __shfl_down_sync(0xffffffffu, ev, o);
    pe += __shfl_down_sync(0xffffffffu, pe, o);
    pk += __shfl_down_sync(0xffffffffu, pk, o);
  }
  if (lane == 0) {
    atomicAdd(&P.counters[0], tot_cross);
    atomicAdd(&P.counters[1], ev);
    atomicAdd(&P.counters[2], pe);
    atomicAdd(&P.counters[3], pk);
    if (cp) {
      atomicAdd(&P.counters[4], cp);
      atomicAdd(&P.counters[5], cc);
    }
  }
}

// Column sums of each model whose frame looks along a grid axis: one block
// per model, one thread per grid line (the forward path's k_columns).
__global__ void k_batch_columns(const DevModel* models, int n_models, const float* density) {
  const int m = blockIdx.x;
  if (m >= n_models) return;
  const DevModel& M = models[m];
  float* out = const_cast<float*>(M.instr.column);
  if (!out) return;
  const float* dens = density + M.density;
  const int nx = M.nx, ny = M.ny, axis = M.instr.axis, dir = M.instr.dir;
  const int n = axis == 0 ? M.nx : (axis == 1 ? M.ny : M.nz);
  const long long n_lines = (long long)M.nx * M.ny * M.nz / n;
  const double d = (double)M.d[axis];
  for (long long L = threadIdx.x; L < n_lines; L += blockDim.x) {
    long long base, stride;
    if (axis == 0) {
      base = L * nx; stride = 1;
    } else if (axis == 1) {
      base = (L % nx) + (L / nx) * (long long)nx * ny; stride = nx;
    } else {
      base = L; stride = (long long)nx * ny;
    }
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
      const int j = dir > 0 ? n - 1 - k : k;
      const long long c = base + (long long)j * stride;
      out[c] = (float)acc;
      acc += (double)dens[c] * d;
    }
  }
}

// Every model emits its luminosity per launch.
__global__ void k_batch_emitted(double* tallies, const double* lum, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tallies[(size_t)i * 4] += lum[i];
}

}  // namespace

const void* batch_kernel() { return reinterpret_cast<const void*>(&k_batch); }
const void* batch_emitted_kernel() { return reinterpret_cast<const void*>(&k_batch_emitted); }
const void* batch_columns_kernel() { return reinterpret_cast<const void*>(&k_batch_columns); }

cudaError_t launch_batch_columns(const DevModel* models, int n_models, const float* density, cudaStream_t stream) {
  k_batch_columns<<<(unsigned)n_models, 128, 0, stream>>>(models, n_models, density);
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchParams& p, unsigned blocks, cudaStream_t stream) {
  k_batch<<<blocks, kBatchBlock, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t batch_blocks_per_sm(int* blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_batch, kBatchBlock, 0);
}

}  // namespace rtk

/*
 * rt.h - C ABI of the GB300 photon-packet Monte Carlo dust radiative transfer
 * library (librt_gb300.so).
 *
 * The operation is the transport loop of a SKIRT-style simulation (Camps &
 * Baes, "SKIRT: an advanced dust radiative transfer code with a user-friendly
 * architecture"): photon packets are emitted by the sources, walk straight
 * through the cells of a dust grid accumulating optical depth, interact by
 * forced scattering, deposit absorbed luminosity continuously along their
 * path, scatter with a Henyey-Greenstein phase function, and at emission and
 * at every scattering "peel off" a fraction of their luminosity towards every
 * frame instrument (Sect. 1: peel-off, continuous absorption, forced
 * scattering; Sect. 2.2: sources, dust system, grid, instruments; Sect. 2.3:
 * albedo and asymmetry parameter g; Sect. 2.4: cartesian grids and octrees).
 *
 * The simulation set-up of Sect. 2.2 (wavelength grid, stellar system, dust
 * system with its grid, instrument system) and the construct / setup / run
 * phases of Sect. 3.2 map onto the calls below:
 *   rt_context_create -> rt_create_grid -> rt_set_optics -> rt_add_sources ->
 *   rt_add_instruments -> rt_launch_packets (any number of times) ->
 *   rt_read_images / rt_read_absorption / rt_read_stats.
 *
 * Conventions for every call
 *   - Return value: RT_OK (0) or a negative rt_status.  No call aborts,
 *     traps or prints.  rt_last_error() gives a message for the last failure.
 *   - Ownership: the library owns all device state of a context.  Input
 *     arrays are copied during the call; the caller keeps ownership of its
 *     buffers and may free them when the call returns.  Output buffers belong
 *     to the caller.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Launches are asynchronous.  Errors raised by
 *     asynchronous work surface at the next synchronising call (rt_read_* to
 *     host memory, rt_read_stats, rt_synchronize).
 *   - A context is bound to one CUDA device and is not thread-safe.  Its
 *     launches share working buffers (the packet counter, the sorted
 *     peel-off pass's records, the adjoint tape), so two launches of one
 *     context must not overlap on the GPU: queue them on one stream or
 *     synchronise between them (separate contexts may run concurrently).
 *
 * Units: lengths in any consistent unit; kappa is the extinction cross
 * section per unit density per unit length; images hold luminosity per
 * steradian per pixel (divide by distance^2 for flux); absorption holds
 * absorbed luminosity per cell.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_ctx_s* rt_ctx;
typedef int32_t rt_status;

enum {
  RT_OK = 0,
  RT_ERR_ARG = -1,          /* invalid argument (null pointer, bad size, value out of range)  */
  RT_ERR_STATE = -2,        /* call out of order (e.g. launch before rt_set_optics)            */
  RT_ERR_OOM = -3,          /* device or host allocation failed                                */
  RT_ERR_CUDA = -4,         /* a CUDA runtime call failed; see rt_last_error                   */
  RT_ERR_TIMEOUT = -5,      /* a bounded device wait ran out                                   */
  RT_ERR_DEVICE_FLAG = -6   /* a kernel's own bounds check fired; results are not valid        */
};

enum { RT_GRID_CARTESIAN = 0, RT_GRID_OCTREE = 1, RT_GRID_RECTILINEAR = 2, RT_GRID_BINTREE = 3, RT_GRID_VORONOI = 4 };
enum { RT_SOURCE_POINT = 0, RT_SOURCE_EXPDISK = 1, RT_SOURCE_PLUMMER = 2 };
enum { RT_DEPOSIT_NEAREST = 0, RT_DEPOSIT_BILINEAR = 1, RT_DEPOSIT_SED = 2 };
enum { RT_LAYOUT_AUTO = 0, RT_LAYOUT_ROW_MAJOR = 1 };
enum { RT_EMITTER_SOURCES = 0, RT_EMITTER_DUST = 1 };

/* Dust grid (Sect. 2.2: constant density per cell; Sect. 2.4 and Table 1(d):
 * grid kinds).
 *   kind RT_GRID_CARTESIAN: nx*ny*nz equal cells spanning `bounds`;
 *       density float32 [nz][ny][nx] (x fastest); cell id = ix + nx*(iy + ny*iz).
 *   kind RT_GRID_RECTILINEAR: nx*ny*nz cuboidal cells between the strictly
 *       increasing edges edges[0] [nx + 1], edges[1] [ny + 1], edges[2]
 *       [nz + 1] (FP64; the first and last edges must equal `bounds`; they
 *       must stay strictly increasing when rounded to FP32).  The PowCub
 *       grid of Table 1(d) is the case of power-law spaced edges.  Density
 *       and cell ids as for RT_GRID_CARTESIAN.  Not supported by rt_adjoint,
 *       the adjoint tape, batches or rt_launch_packets_noalloc.
 *   kind RT_GRID_BINTREE: a k-d tree (the BinTree grid of Table 1(d)):
 *       node 0 the root; child[n] >= 0 is the index of the first of n's two
 *       contiguous children (the lower, then the upper half of n's box split
 *       at its midpoint along split_axis[n], 0 = x, 1 = y, 2 = z),
 *       child[n] < 0 marks a leaf with leaf id -(child[n] + 1), each id in
 *       [0, n_leaves) exactly once; density
 *       float32 [n_leaves]; cell id = leaf id; depth at most 96, node
 *       indices below 2^29.  Peel-offs walk their rays; not supported by the
 *       adjoint, batches, the allocation-free call or the dust emission.
 *   kind RT_GRID_OCTREE: recursive 2x2x2 subdivision of `bounds` at box
 *       midpoints; child int32 [n_nodes], node 0 the root: child[n] >= 0 is
 *       the index of the first of n's eight contiguous children (octant
 *       o = bit0 x-upper | bit1 y-upper | bit2 z-upper), child[n] < 0 marks a
 *       leaf with leaf id -(child[n] + 1), each id in [0, n_leaves) exactly
 *       once; density float32 [n_leaves]; cell id = leaf id.  Depth at most 21
 *       (deeper trees are rejected with RT_ERR_ARG).
 *   kind RT_GRID_VORONOI: the Voronoi grid of Table 1(d) (Sect. 2.4): cell c
 *       is the part of the domain nearer to site c than to any other site.
 *       n_leaves sites, sites FP64 [n_leaves][3], inside `bounds`, no two
 *       equal; the neighbours of cell c are child[offsets[c] ..
 *       offsets[c + 1]) (offsets int64 [n_leaves + 1], offsets[0] = 0,
 *       offsets[n_leaves] = n_nodes, ids in range, none equal to c).  The
 *       lists must hold every cell that shares a face with c inside the
 *       domain (the Delaunay neighbours of the sites do); extra entries only
 *       cost time.  density float32 [n_leaves]; cell id = site index.  The
 *       library keeps per face the FP32 unit normal and distance of the
 *       bisecting plane, and locates points by a descent to the nearest site
 *       from a bucket grid's seeds.  At most 2^31 - 1 sites and list
 *       entries.  Peel-offs walk their rays; not supported by the adjoint,
 *       batches, the allocation-free call or the dust emission.
 *   bounds: xmin, xmax, ymin, ymax, zmin, zmax (FP64; the kernels use FP32).
 *   Pointers are host pointers unless on_device = 1.  Data is copied.
 *   layout (cartesian and rectilinear grids): how the library stores the
 *       cells on the device.  RT_LAYOUT_AUTO (0): the axis whose cell faces a
 *       ray crosses most often (most cells per unit length) is stored
 *       unit-stride, then the next; RT_LAYOUT_ROW_MAJOR (1): x fastest.  Only
 *       the speed differs: inputs, read-outs and cell ids are row-major
 *       either way. */
typedef struct {
  int32_t kind;
  int32_t nx, ny, nz;
  double bounds[6];
  const float* density;
  int64_t n_nodes;
  const int32_t* child;
  int64_t n_leaves;
  int32_t on_device;
  int32_t layout;         /* RT_LAYOUT_AUTO or RT_LAYOUT_ROW_MAJOR */
  const double* edges[3]; /* RT_GRID_RECTILINEAR: cell edges per axis (host or device, as on_device) */
  const int8_t* split_axis; /* RT_GRID_BINTREE: split axis per node (host or device, as on_device) */
  const double* sites;      /* RT_GRID_VORONOI: sites [n_leaves][3] (host or device, as on_device) */
  const int64_t* offsets;   /* RT_GRID_VORONOI: neighbour list offsets [n_leaves + 1] (host or device) */
} rt_grid_desc;

/* Emission component (Sect. 2.2 stellar system, Sect. 3.4 position sampling,
 * Table 1(a) geometries).  RT_SOURCE_POINT: at `center`.  RT_SOURCE_EXPDISK:
 * double-exponential disk in the plane z = center[2], scale length scale_r,
 * scale height scale_z.  RT_SOURCE_PLUMMER: Plummer sphere of scale radius
 * scale_r.  Emission is isotropic.  luminosity: host float64 [n_lambda]. */
typedef struct {
  int32_t kind;
  int32_t reserved;
  double center[3];
  double scale_r, scale_z;
  const double* luminosity;
} rt_source_desc;

/* Frame instrument with parallel projection (Sect. 2.2; the parameters of
 * the FrameInstrument of the Sect. 2.5 example), or SED instrument
 * (deposit = RT_DEPOSIT_SED; Sect. 2.2: the spectral energy distribution of
 * the flux received from the viewing direction): every peel-off towards it
 * is summed per wavelength, wherever it starts; nx = ny = 1, the half widths
 * and field centre are not used, and the layout is [channels][n_lambda].  Direction to the observer
 * k = (sin i cos a, sin i sin a, cos i); image axes before the position angle
 * w: ex = (-sin a, cos a, 0), ey = (-cos i cos a, -cos i sin a, sin i); the
 * position angle turns them to cos w ex - sin w ey and sin w ex + cos w ey.
 * Pixel of image coordinate X: floor((X - center_x + half_x) nx / (2 half_x)).
 * channels = 1: total only; channels = 3: total, direct (emission peel-off),
 * scattered (scattering peel-off).  Image layout float64
 * [channels][n_lambda][ny][nx]. */
typedef struct {
  double inclination, azimuth, position_angle; /* radians */
  int32_t nx, ny;
  double half_x, half_y;
  double center_x, center_y;
  int32_t deposit;   /* RT_DEPOSIT_NEAREST, RT_DEPOSIT_BILINEAR (pixel centres) or RT_DEPOSIT_SED */
  int32_t channels;  /* 1 or 3 */
} rt_instrument_desc;

/* One peel-off deposit into the total channel (debug records, nearest
 * deposit only): packet id, wavelength index, event (0 = emission),
 * instrument, pixel iy*nx + ix, value. */
typedef struct {
  uint64_t packet;
  int32_t lambda, event, instrument, reserved;
  int64_t pixel;
  double value;
} rt_record;

/* Per-event state of one traced packet (event 0 = emission): position and
 * direction after / before the event, interaction cell, weight after the
 * event, optical depth of the forced path and the drawn tau*. */
typedef struct {
  int32_t event, reserved;
  int64_t cell;
  double x[3], k[3];
  double L, tau_path, tau_star;
} rt_trace_row;

/* Launch options.  Zero-initialise and set what you need; rt_default_opts
 * fills the defaults (w_min 1e-4, max_events 1000, weight cut on, both
 * peel-offs on). */
typedef struct {
  double w_min;         /* terminate when L < w_min * L0 (if weight_cut)                   */
  int32_t max_events;   /* terminate after this many scattering events (>= 1)              */
  int32_t weight_cut;   /* 1: weight rule + event cap; 0: event cap only                   */
  int32_t peel_emission;
  int32_t peel_scatter;
  uint64_t n_norm;      /* packets per wavelength for the weight L_tot/n_norm; 0 = n_per_lambda */
  uint32_t model_id;    /* second Philox key word                                          */
  int32_t walk_peels;   /* 0 (default): a peel-off towards a frame that looks exactly along a
                           grid axis takes its optical depth from per-line suffix sums of the
                           density (cartesian grids; rebuilt at every launch); 1: every
                           peel-off walks its ray.  The two agree to FP32 rounding.       */
  rt_record* records;   /* device buffer for debug records, or NULL                        */
  int64_t records_capacity;
  uint64_t record_stride; /* record only packets whose id is a multiple of this (0, 1: all)  */
  rt_trace_row* trace;  /* device buffer: per-event trace of packet trace_packet, or NULL    */
  int64_t trace_capacity;
  uint64_t trace_packet;
  int32_t trace_lambda;
  int32_t control_lanes; /* per-event work of a warp waits until this many of its lanes need it
                            (1..32; 0 = library choice)                                    */
  uint64_t* profile;    /* device buffer of 8 counters accumulated by the cartesian kernel (a
                           separately compiled instance; ignored with a tape or on other grids), or
                           NULL: loop iterations, walking lanes summed over iterations,
                           per-event rounds, lanes served summed over rounds, clock cycles in
                           per-event work, clock cycles in the walk; two reserved (zero)    */
  int32_t tape;         /* 1: record the adjoint tape of this launch in the context (cartesian
                           grids; 160 B x (max_events + 1) per packet), so that an rt_adjoint
                           of the same packets (same n_per_lambda, first_packet_id, seed and
                           options, density unchanged, no absorption adjoint) needs no
                           replay of the forced paths                                       */
  int32_t inline_peels; /* 0 (default): on cartesian grids, the peel-offs that walk (frames not
                           along a grid axis, or all with walk_peels) run in a second pass after
                           the transport kernel, ordered by instrument and start cell so that
                           the walks of a warp share cache lines (skipped with the tape, and
                           while its buffer, sized from the last launch's count within 40 % of
                           free device memory, cannot be had); 1: each walks inside the
                           transport kernel.  The two give the same optical depths, crossings
                           and deposits; only the order of the FP64 image additions differs.   */
  int32_t time_parts;   /* 1: record CUDA events around the parts of this launch on its stream,
                           read back by rt_read_launch_times                               */
  int32_t emitter;      /* RT_EMITTER_SOURCES (0): the sources emit; RT_EMITTER_DUST (1): the dust
                           cells emit their thermal luminosity (rt_set_dust_emission), a cell
                           drawn in proportion to its luminosity at the packet's wavelength, a
                           uniform position in it, an isotropic direction; a wavelength at which
                           the dust emits nothing launches packets of zero weight that end at once */
  int32_t blocks_per_sm; /* resident blocks of 256 threads per SM of the persistent transport grid
                            (0 = the value rt_tune chose, else as many as fit: 4, or 3 for
                            octrees deeper than 10 levels); the grid is this
                            times the SM count */
  int32_t reserved;
} rt_launch_opts;

/* Tallies since the last rt_reset_tallies. */
typedef struct {
  double emitted, escaped, absorbed, truncated; /* luminosity                              */
  uint64_t crossings;   /* cell segments visited by forced paths and peel-off paths        */
  uint64_t path_crossings; /* of which on forced paths (first pass)                         */
  uint64_t events;      /* forced scattering events                                        */
  uint64_t peeloffs;    /* peel-off paths (one per instrument per emission / scattering)   */
  uint64_t packets;
  uint64_t records;     /* debug records produced (may exceed the capacity)                */
  uint64_t column_peels;     /* peel-offs whose optical depth came from column sums        */
  uint64_t column_crossings; /* the crossings of their rays (included in crossings)        */
  uint64_t sorted_peels;     /* peel-offs walked in the sorted pass (rt_launch_opts.inline_peels) */
  int32_t device_flags; /* non-zero if a kernel bounds check fired                         */
  int32_t reserved;
} rt_stats;

/* Library version string (static storage). */
const char* rt_version(void);

/* Create a context on CUDA device `device`.  *out receives the handle.
 * Errors: RT_ERR_ARG (null out, bad device), RT_ERR_CUDA, RT_ERR_OOM. */
rt_status rt_context_create(int32_t device, rt_ctx* out);

/* Destroy a context and free all its device memory.  NULL is accepted. */
rt_status rt_context_destroy(rt_ctx ctx);

/* Message for the last failed call on ctx (static "" if none); owned by the
 * context, valid until the next call on it.  ctx NULL gives the message of the
 * last failed rt_context_create. */
const char* rt_last_error(rt_ctx ctx);

/* Fill *opts with the defaults. */
void rt_default_opts(rt_launch_opts* opts);

/* Dust grid (Sect. 2.2, 2.4).  Replaces any previous grid of the context,
 * drops optics, sources, instruments and tallies.  *grid_id receives 0.
 * Errors: RT_ERR_ARG (sizes <= 0, bounds not increasing, octree child index
 * out of range, negative density), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_create_grid(rt_ctx ctx, const rt_grid_desc* desc, int32_t* grid_id);

/* Optical properties per wavelength (Sect. 2.3): kappa (>= 0), albedo in
 * [0, 1], HG asymmetry g in (-1, 1); host float64 arrays [n_lambda],
 * 1 <= n_lambda <= 64; `lambda` (wavelengths) may be NULL.  Resets tallies.
 * Errors: RT_ERR_ARG, RT_ERR_STATE (no grid). */
rt_status rt_set_optics(rt_ctx ctx, int32_t grid_id, int32_t n_lambda, const double* lambda,
                        const double* kappa, const double* albedo, const double* g);

/* Append n emission components (Sect. 2.2 stellar system); at most 16 in
 * total.  Each luminosity array has n_lambda entries >= 0.
 * Errors: RT_ERR_ARG, RT_ERR_STATE (no optics). */
rt_status rt_add_sources(rt_ctx ctx, int32_t n, const rt_source_desc* sources);

/* Append n frame instruments (Sect. 2.2); at most 16 in total.  ids (may be
 * NULL) receives their indices.  Allocates and zeroes their images.
 * Errors: RT_ERR_ARG (pixels <= 0, half widths <= 0 for a frame, an SED
 * instrument with nx or ny other than 1, channels not 1 or 3),
 * RT_ERR_STATE (no optics), RT_ERR_OOM. */
rt_status rt_add_instruments(rt_ctx ctx, int32_t n, const rt_instrument_desc* instruments, int32_t* ids);

/* Run n_per_lambda packets at every wavelength (from the sources, or from the
 * dust with opts->emitter = RT_EMITTER_DUST), with packet ids
 * [first_packet_id, first_packet_id + n_per_lambda), Philox key (seed,
 * opts->model_id).  Tallies accumulate across launches until
 * rt_reset_tallies, so id ranges can be split over launches.  Asynchronous
 * on `stream`.  opts may be NULL (defaults).  seed must be < 2^32.
 * Errors: RT_ERR_ARG, RT_ERR_STATE (no sources or no optics), RT_ERR_CUDA. */
rt_status rt_launch_packets(rt_ctx ctx, uint64_t n_per_lambda, uint64_t first_packet_id, uint64_t seed,
                            const rt_launch_opts* opts, void* stream);

/* Choose the per-event deferral threshold (opts->control_lanes) and the
 * resident blocks per SM (opts->blocks_per_sm) for this context's problem:
 * times a launch of n_per_lambda packets per wavelength for each of 8, 12,
 * 16, 20, 24, 28 lanes at the most resident blocks, then, when the sample
 * holds at least 8 packets per resident thread at the most blocks, for the
 * best threshold with one and two blocks per SM fewer (kept only if at least
 * 3 % faster; other options from opts or the defaults), and keeps the fastest
 * pair for later launches with 0 in
 * those fields; the threshold is written to *control_lanes if not NULL.
 * Both only reorder work: results are the same to FP64 summation order.  The
 * tallies are zeroed afterwards.  Synchronous.  Errors: as rt_launch_packets. */
rt_status rt_tune(rt_ctx ctx, uint64_t n_per_lambda, uint64_t seed, const rt_launch_opts* opts,
                  int32_t* control_lanes, void* stream);

/* The launch shape that launches with 0 in opts->control_lanes and
 * opts->blocks_per_sm use: the values rt_tune kept (before any rt_tune: 16
 * lanes and 0, i.e. as many resident blocks as fit).  Either pointer may be
 * NULL.  Errors: RT_ERR_ARG (ctx NULL). */
rt_status rt_tuned(rt_ctx ctx, int32_t* control_lanes, int32_t* blocks_per_sm);

/* The same for rt_adjoint: times rt_adjoint with these adjoint inputs (into
 * a scratch gradient the context owns) for 12, 16, ..., 32 lanes and keeps
 * the fastest for rt_adjoint calls with control_lanes 0.  Synchronous.
 * Errors: as rt_adjoint, RT_ERR_OOM. */
rt_status rt_adjoint_tune(rt_ctx ctx, const double* const* adj_images, int32_t n_adj_images,
                          const double* adj_absorption, uint64_t n_per_lambda, uint64_t seed,
                          const rt_launch_opts* opts, int32_t* control_lanes, void* stream);

/* Zero images, absorption and statistics (asynchronous on stream). */
rt_status rt_reset_tallies(rt_ctx ctx, void* stream);

/* Copy the absorbed luminosity, float64 [n_lambda][n_cells], into dst.
 * n_elems must equal n_lambda * n_cells.  dst_on_device = 1: device pointer,
 * asynchronous on stream; 0: host pointer, returns when the copy is done
 * (on a device that reaches all host memory, cudaDevAttrPageableMemoryAccess,
 * a destination that starts and ends in page-locked memory is written by the
 * device directly; other host memory through a device staging buffer).
 * Errors: RT_ERR_ARG (size mismatch), RT_ERR_STATE, RT_ERR_CUDA. */
rt_status rt_read_absorption(rt_ctx ctx, double* dst, size_t n_elems, int32_t dst_on_device, void* stream);

/* ---------------------------------------------------------------- panchromatic mode
 * A panchromatic simulation (Sect. 2.1, 2.2: oligochromatic vs panchromatic)
 * integrates the absorbed luminosity over the wavelength grid to find the
 * dust temperature and adds the dust's thermal emission.  Equilibrium
 * emission of one grain type: cell c at temperature T emits
 *   S m_c sum_l kabs_l dlambda_l beta_l(T),   beta_l(T) = lambda_l^-5 / (exp(C2 / (lambda_l T)) - 1),
 * m_c = rho_c V_c its dust mass, kabs_l = kappa_l (1 - albedo_l), lambda in um
 * (rt_set_optics's wavelengths, at least two, increasing), C2 = hc/k =
 * 14387.77 um K, dlambda_l the widths of bins centred on the wavelengths on a
 * logarithmic scale (inner borders at geometric means, outer borders
 * mirrored), and S = emission_scale, the caller's factor for the Planck
 * constant 2hc^2, 4 pi and the units of luminosity, mass and length.
 * Cartesian and rectilinear grids. */

/* Equilibrium temperature of every cell: the T at which it emits the
 * luminosity it absorbed summed over the wavelengths, found by bisection in
 * ln T between t_min and t_max (64 halvings).  absorption: row-major float64
 * [n_lambda][n_cells] (host, or device with absorption_on_device = 1), or
 * NULL for the context's absorption tallies.  temperature: float64 [n_cells]
 * (host, or device with dst_on_device = 1): 0 for cells without dust or
 * without absorbed luminosity, t_max for cells that would need more and
 * t_min for cells that would need less (counted in *n_clamped if not NULL).
 * Synchronous.
 * Errors: RT_ERR_STATE (no grid or optics, no wavelengths), RT_ERR_ARG
 * (octree grid, scale <= 0, bad range), RT_ERR_CUDA, RT_ERR_OOM. */
rt_status rt_dust_temperature(rt_ctx ctx, double emission_scale, double t_min, double t_max,
                              const double* absorption, int32_t absorption_on_device, double* temperature,
                              int32_t dst_on_device, int32_t* n_clamped, void* stream);

/* Thermal emission of the dust at the temperatures [n_cells] (host, or
 * device with on_device = 1; e.g. from rt_dust_temperature): per cell and
 * wavelength S m_c kabs_l dlambda_l beta_l(T_c), and its running sums over
 * the cells, from which launches with opts.emitter = RT_EMITTER_DUST draw
 * the emitting cell.  Packet weights are the per-wavelength totals over
 * n_norm.  Kept until the optics, grid or emission change.  Synchronous.
 * Errors: as rt_dust_temperature. */
rt_status rt_set_dust_emission(rt_ctx ctx, const double* temperature, int32_t on_device, double emission_scale,
                               void* stream);

/* The thermal emission set by rt_set_dust_emission, float64
 * [n_lambda][n_cells] row-major; n_elems must match.  Conventions of
 * rt_read_absorption.  Errors: RT_ERR_STATE (none set), RT_ERR_ARG. */
rt_status rt_read_dust_emission(rt_ctx ctx, double* dst, size_t n_elems, int32_t dst_on_device, void* stream);

/* Copy instrument `instrument_id`'s image, float64 [channels][n_lambda][ny][nx],
 * into dst; n_elems must match.  Same conventions as rt_read_absorption. */
rt_status rt_read_images(rt_ctx ctx, int32_t instrument_id, double* dst, size_t n_elems, int32_t dst_on_device,
                         void* stream);

/* Synchronise the context's work and read the statistics.
 * Errors: RT_ERR_CUDA, RT_ERR_DEVICE_FLAG (stats are still written). */
rt_status rt_read_stats(rt_ctx ctx, rt_stats* out);

/* Device time in milliseconds of the parts of the last rt_launch_packets made
 * with opts->time_parts = 1 (CUDA events on its stream; waits for them):
 * ms[0] column sums, ms[1] the transport kernel, ms[2] the ordering of the
 * sorted peel-off pass (scan and scatter), ms[3] its walks; parts that did not
 * run read 0.  n (1..4) is the number of entries written.
 * Errors: RT_ERR_ARG (null ms, n out of range), RT_ERR_STATE (no timed
 * launch since the context was created), RT_ERR_CUDA. */
rt_status rt_read_launch_times(rt_ctx ctx, float* ms, int32_t n);

/* Wait for all work queued on `stream` and report asynchronous errors. */
rt_status rt_synchronize(rt_ctx ctx, void* stream);

/* Replace the cell densities of the current grid (same size as at
 * rt_create_grid), asynchronously on `stream`: for fitting loops (the inverse
 * problem of Sect. 1).  Tallies are kept.  density: float32 [n_cells], host
 * (copied before return) or device (on_device = 1, stream-ordered copy).
 * Errors: RT_ERR_STATE (no grid), RT_ERR_ARG, RT_ERR_CUDA. */
rt_status rt_update_density(rt_ctx ctx, const float* density, int32_t on_device, void* stream);

/* Gradient of a linear functional of the tallies with respect to the cell
 * densities, by reverse-mode differentiation of the transport of
 * rt_launch_packets under common random numbers (Sect. 1 motivates the
 * inverse problem: fitting models to observations).  For the packets
 * [first_packet_id, first_packet_id + n_per_lambda) at every wavelength:
 *   grad[c] += sum_q sum_pixels adj_images[q][pixel] d image_q[pixel] / d rho_c
 *            + sum_{l, c'} adj_absorption[l][c'] d absorption[l][c'] / d rho_c
 * with the derivative taken along each packet's path: directions and random
 * draws fixed, positions moving with the density through the forced
 * scattering inversion, weights through 1 - exp(-tau).  Each packet's path is
 * recomputed from its Philox key.  The functional is continuous in the density
 * with bilinear deposit and event-cap termination (opts->weight_cut = 0);
 * use those for gradient checks.  Cartesian grids only; max_events <= 256.
 * The context keeps a device buffer of per-event records, 160 B x
 * (max_events + 1) per resident thread (116,736 threads on a 152-SM GPU:
 * 0.39 GB at max_events = 20), allocated on the first call that needs more
 * (RT_ERR_OOM if it cannot be had); a call that can use the forward launch's
 * tape (rt_launch_opts.tape) needs none.  opts->profile, if not NULL, is a
 * device uint64 array: [0] += cell crossings of all walks, [1] += crossings
 * that deposited into grad_density.
 *   adj_images: host array of n_instruments device pointers (each shaped like
 *   the instrument's image) or NULL entries / a NULL array for none;
 *   adj_absorption: device [n_lambda][n_cells] or NULL; grad_density: device
 *   float64 [n_cells], accumulated into.  Asynchronous on `stream`.
 * Errors: RT_ERR_ARG, RT_ERR_STATE, RT_ERR_CUDA. */
rt_status rt_adjoint(rt_ctx ctx, const double* const* adj_images, int32_t n_adj_images, const double* adj_absorption,
                     double* grad_density, uint64_t n_per_lambda, uint64_t first_packet_id, uint64_t seed,
                     const rt_launch_opts* opts, void* stream);

/* The cartesian forward transport of rt_launch_packets without any device
 * memory allocation (every peel-off walks its ray: there is no room for
 * column sums, so it equals rt_launch_packets with opts->walk_peels = 1 to
 * FP64 summation order).  The paper has no counterpart: this entry point exists
 * for callers that may not allocate GPU memory while they run (a plug-in
 * inside a framework that owns the device memory pool, a service with a fixed
 * memory budget), so they pass every device buffer themselves.
 *   grid: kind RT_GRID_CARTESIAN, on_device = 1, density a device pointer.
 *   kappa, albedo, g [n_lambda]; sources [n_sources] with host luminosity
 *   arrays; instruments [n_instruments]: host arrays, as for the context calls.
 *   images: host array of n_instruments device pointers, each float64
 *   [channels][n_lambda][ny][nx]; absorption: device float64
 *   [n_lambda][nx*ny*nz].  Tallies are ADDED to these buffers.
 *   stats_out: device pointer that receives this call's rt_stats, or NULL.
 * Options: as for rt_launch_packets; every peel-off walks its ray inside the
 * transport kernel (walk_peels and inline_peels are implied), and tape or
 * time_parts set returns RT_ERR_ARG (both need a context).
 * Limits (fixed by the library's working area): n_lambda <= 64,
 * n_sources <= 16, n_instruments <= 16; larger values return RT_ERR_ARG.
 * The library keeps one working area of 16 KiB per device in a static
 * device array, held by every GPU that loads the library until the process
 * exits; the call allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  Every call looks the working area's address up on the
 * current device; the first call on a device also loads the library's device
 * code there and should come before any stream capture on that device.  The
 * call's tables reach the working area as a kernel parameter, so the caller's
 * host arrays may be reused when the call returns.  All calls share the
 * working area, which keeps the last call's contents: calls that overlap on
 * the GPU (other streams, other threads) race and must be serialised by the
 * caller.  Asynchronous on `stream`.  Errors: RT_ERR_ARG, RT_ERR_CUDA; the
 * message is rt_last_error(NULL). */
rt_status rt_launch_packets_noalloc(const rt_grid_desc* grid, int32_t n_lambda, const double* kappa,
                                    const double* albedo, const double* g, int32_t n_sources,
                                    const rt_source_desc* sources, int32_t n_instruments,
                                    const rt_instrument_desc* instruments, double* const* images,
                                    double* absorption, uint64_t n_per_lambda, uint64_t first_packet_id,
                                    uint64_t seed, const rt_launch_opts* opts, rt_stats* stats_out, void* stream);

/* Read bandwidth (GB/s, best of `repeats`) of the library's own kernel
 * streaming a device buffer of `bytes` bytes `passes` times with loads cached
 * in L2 only; a buffer well inside the L2 (a few tens of MB) gives the L2
 * read bandwidth, one far larger the HBM read bandwidth.  This is the
 * denominator of roofline fractions for kernels whose working set stays in
 * L2; the paper has no counterpart.  Allocates and frees its buffer.
 * Errors: RT_ERR_ARG, RT_ERR_CUDA (message: rt_last_error(NULL)). */
rt_status rt_probe_bandwidth(int32_t device, uint64_t bytes, int32_t passes, int32_t repeats, double* gb_per_s);

/* ---------------------------------------------------------------- batches
 * Many small independent models in one persistent launch, for the parameter
 * searches of model fitting that Sect. 1 motivates: thousands of small grids,
 * each too small to fill the GPU alone.  A model is a cartesian grid with one
 * wavelength, one point source and one single-channel frame.  Its packets are
 * the packets rt_launch_packets runs for the same problem with
 * model_id = the model's index in the batch and n_norm = n_packets, with the
 * same arithmetic, so its image and tallies equal that launch's up to the
 * order of FP64 additions.  No absorption field is kept (its total is). */
typedef struct {
  int32_t nx, ny, nz;            /* cells per axis, 1 .. 65536 */
  int32_t reserved;
  double bounds[6];              /* xmin, xmax, ymin, ymax, zmin, zmax */
  const float* density;          /* host, float32 [nz][ny][nx], finite and >= 0; copied */
  double kappa;                  /* extinction per unit density and length, >= 0 */
  double albedo;                 /* 0 .. 1 */
  double g;                      /* Henyey-Greenstein asymmetry, -1 < g < 1 */
  double luminosity;             /* of the point source, > 0 */
  double source[3];              /* point source position */
  rt_instrument_desc instrument; /* the frame; channels must be 1 */
  uint64_t n_packets;            /* packets per launch, 1 .. 2^32 - 1 */
} rt_model_desc;

/* Copy n_models (1 .. 2^20) models to the device: densities in one buffer,
 * one table row per model, FP64 images and tallies zeroed, the work list of
 * packet runs sorted by estimated cost.  *batch_id receives the handle.
 * Errors: RT_ERR_ARG (the model index is in the message), RT_ERR_OOM,
 * RT_ERR_CUDA. */
rt_status rt_batch_create(rt_ctx ctx, int32_t n_models, const rt_model_desc* models, int32_t* batch_id);

/* Free a batch (after its work has finished). */
rt_status rt_batch_destroy(rt_ctx ctx, int32_t batch_id);

/* Run every model's n_packets packets, accumulating into the batch's images
 * and tallies, asynchronously on `stream`, as one CUDA graph (reset the work
 * counter, add each model's luminosity to its emitted tally, the persistent
 * kernel) whose kernel parameters are updated per call.  opts: w_min,
 * max_events, weight_cut, peel_emission, peel_scatter and control_lanes are
 * used (control_lanes 0: the value rt_batch_tune chose, else 16); seed < 2^32.
 * Errors: RT_ERR_ARG, RT_ERR_CUDA. */
rt_status rt_batch_launch(rt_ctx ctx, int32_t batch_id, uint64_t seed, const rt_launch_opts* opts, void* stream);

/* Zero the batch's images, tallies and counters (stream-ordered). */
rt_status rt_batch_reset(rt_ctx ctx, int32_t batch_id, void* stream);

/* The models' images, concatenated in model order, each [ny][nx] float64;
 * n_elems must be the sum of nx * ny.  dst on the host (the call waits) or
 * on the device (on_device = 1, stream-ordered). */
rt_status rt_batch_read_images(rt_ctx ctx, int32_t batch_id, double* dst, size_t n_elems, int32_t on_device,
                               void* stream);

/* Per-model tallies [n_models][4] float64: emitted, escaped, absorbed,
 * truncated luminosity; n_elems must be 4 * n_models. */
rt_status rt_batch_read_tallies(rt_ctx ctx, int32_t batch_id, double* dst, size_t n_elems, int32_t on_device,
                                void* stream);

/* Synchronise and sum: the totals over the models and the counters
 * (crossings, events, peeloffs, packets, column_peels, column_crossings);
 * records, path_crossings 0.
 * Errors: RT_ERR_CUDA, RT_ERR_DEVICE_FLAG. */
rt_status rt_batch_read_stats(rt_ctx ctx, int32_t batch_id, rt_stats* out);

/* Choose control_lanes and the packets per work-list run by timing launches
 * of a fraction (0 < fraction <= 1) of every model's packets for each
 * candidate (control_lanes 8, 12, ..., 32; runs of 64, 256, 1024, 4096
 * packets); the choice is kept for later launches with control_lanes 0 and
 * written to *control_lanes and *run_packets if not NULL.  The images and
 * tallies are zeroed afterwards.  Synchronous.  Errors: RT_ERR_ARG,
 * RT_ERR_CUDA. */
rt_status rt_batch_tune(rt_ctx ctx, int32_t batch_id, uint64_t seed, double fraction, int32_t* control_lanes,
                        uint32_t* run_packets, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_GB300_H */

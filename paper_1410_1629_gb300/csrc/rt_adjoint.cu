// Adjoint of the forward transport: the gradient of a linear functional of
// the images and the absorption field with respect to the cell densities,
// under common random numbers (the derivative along each packet's path:
// directions and random draws fixed, positions moving with the density
// through the forced-scattering inversion, weights through 1 - exp(-tau)).
//
// One thread per packet.  The packet's path is first replayed from its Philox
// key (the forced path of every event, no peel-offs), storing one checkpoint
// per event: position, carried cell, direction, weight, tau_path, tau*.  The
// events are then swept backwards with the adjoints of the position and the
// weight:
//   * peel-off at event j towards instrument q, value l = L_j P e^{-tau(x_j)} W(x_j)
//     (W: the adjoint image interpolated like the deposit):
//       walk 1: tau and d tau / d x (the density jumps across the crossed planes),
//       walk 2: grad[c] -= l kappa ds_c;
//   * forced path of event j from x_{j-1}:
//       walk 1: optical depths, deposit adjoints, the interaction cell h,
//       walk 2: grad[c_m] += kappa ds_m S_m with S_m the suffix sum of the
//       adjoints of tau_i, and the plane terms of d/dx.
// Geometry is FP32 as in the forward kernel; adjoints of position and weight
// and every accumulator are FP64.
#include "rt_transport.cuh"

namespace rtk {

namespace {

using tr::CartGrid;

constexpr int kAdjBlock = 128;
constexpr int kMaxAdjEvents = 32;

struct AdjParams {
  FwdParams f;
  const double* adj_img[kMaxInstruments];  // adjoint images, shaped like the images (or null)
  const double* adj_abs;                   // [n_lambda][n_cells] or null
  double* grad;                            // [n_cells]
};

struct Checkpoint {
  float3 x, k;        // position after event j, direction of the forced path that follows
  int ci, cj, ck;     // carried cell (ci < 0: locate)
  double L;           // weight after event j
  double tau_path;    // optical depth of the forced path that led to event j
  double tau_star;    // its drawn tau*
};

__device__ __forceinline__ void grad_add(double* g, int cell, double v) { atomicAdd(&g[cell], v); }

// Walk from x along d (known cell or located) calling f(cell, t_in, ds, kr, exit_axis, is_last).
template <class F>
__device__ __forceinline__ void walk(const FwdParams& P, float3 x, float3 d, bool known, const CartGrid::Cell& c,
                                     float kappa, F&& f) {
  CartGrid::Walk w;
  CartGrid::Scratch sc;
  const float3 id = make_float3(tr::inv_or_zero(d.x), tr::inv_or_zero(d.y), tr::inv_or_zero(d.z));
  if (!CartGrid::init(P, x, d, id, known, c, w, sc)) return;
  while (true) {
    int axis;
    const float te = CartGrid::exit(w, x, id, axis);
    const float texit = fmaxf(te, w.t);
    const float kr = kappa * __ldg(&P.density[w.cell]);
    const int cell = w.cell;
    const float t_in = w.t;
    w.t = texit;
    const bool more = CartGrid::advance(P, x, d, id, axis, w, sc);
    if (!f(cell, t_in, texit - t_in, kr, axis, !more) || !more) return;
  }
}

__device__ __forceinline__ double3 plane_dt_dx(int axis, float3 d) {
  // d t / d x for the crossing of a plane normal to `axis` (t = (plane - x_a) / d_a)
  const double da = axis == 0 ? d.x : (axis == 1 ? d.y : d.z);
  const double v = -1.0 / da;
  return make_double3(axis == 0 ? v : 0.0, axis == 1 ? v : 0.0, axis == 2 ? v : 0.0);
}

// The adjoint image interpolated at x like a deposit, and its gradient in x.
__device__ __forceinline__ double adj_weight(const AdjParams& A, int q, int lam, bool scattered, float3 x,
                                             double3& dW) {
  const DevInstr& I = tr::S_INSTR[q];
  dW = make_double3(0.0, 0.0, 0.0);
  const double* img = A.adj_img[q];
  if (!img) return 0.0;
  const size_t plane = (size_t)I.ny * I.nx;
  const double* a0 = img + (size_t)lam * plane;
  const double* a1 = I.channels == 3 ? img + ((size_t)(scattered ? 2 : 1) * A.f.n_lambda + lam) * plane : nullptr;
  const float fx = (x.x * I.ex[0] + x.y * I.ex[1] + x.z * I.ex[2] + I.off_x) * I.sx;
  const float fy = (x.x * I.ey[0] + x.y * I.ey[1] + x.z * I.ey[2] + I.off_y) * I.sy;
  auto at = [&](float fix, float fiy) -> double {
    if (!(fix >= 0.0f && fiy >= 0.0f && fix < (float)I.nx && fiy < (float)I.ny)) return 0.0;
    const size_t pix = (size_t)(int)fiy * I.nx + (int)fix;
    return a0[pix] + (a1 ? a1[pix] : 0.0);
  };
  if (!I.bilinear) {
    return at(floorf(fx), floorf(fy));  // piecewise constant in x
  }
  const float gx = fx - 0.5f, gy = fy - 0.5f;
  const float x0 = floorf(gx), y0 = floorf(gy);
  const double tx = gx - x0, ty = gy - y0;
  const double a00 = at(x0, y0), a10 = at(x0 + 1, y0), a01 = at(x0, y0 + 1), a11 = at(x0 + 1, y0 + 1);
  const double W = a00 * (1 - tx) * (1 - ty) + a10 * tx * (1 - ty) + a01 * (1 - tx) * ty + a11 * tx * ty;
  const double dWdfx = (a10 - a00) * (1 - ty) + (a11 - a01) * ty;
  const double dWdfy = (a01 - a00) * (1 - tx) + (a11 - a10) * tx;
  dW.x = dWdfx * I.sx * I.ex[0] + dWdfy * I.sy * I.ey[0];
  dW.y = dWdfx * I.sx * I.ex[1] + dWdfy * I.sy * I.ey[1];
  dW.z = dWdfx * I.sx * I.ex[2] + dWdfy * I.sy * I.ey[2];
  return W;
}

__global__ void __launch_bounds__(kAdjBlock) k_adjoint(const AdjParams A) {
  const FwdParams& P = A.f;
  for (int i = threadIdx.x; i < P.n_instr; i += kAdjBlock) tr::S_INSTR[i] = P.instr[i];
  for (int i = threadIdx.x; i < P.n_lambda; i += kAdjBlock) tr::S_LAM[i] = P.lam[i];
  __syncthreads();
  Checkpoint ev[kMaxAdjEvents + 1];
  const unsigned lane = threadIdx.x & 31u;
  while (true) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(P.work_counter, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= P.n_total) break;
    const unsigned long long w = base + lane;
    if (w < P.n_total) {
      const int lam = (int)(w / P.n_per_lambda);
      const unsigned long long pid = P.first_id + (w - (unsigned long long)lam * P.n_per_lambda);
      const DevLambda LP = tr::S_LAM[lam];
      const float kappa = LP.kappa;
      const double albedo = LP.albedo;
      // ---- forward replay: checkpoints of every event
      tr::Lane<CartGrid> s;
      s.pid = pid;
      s.lam = lam;
      tr::emit(P, s);
      ev[0].x = s.x; ev[0].k = s.k; ev[0].ci = -1; ev[0].cj = ev[0].ck = 0;
      ev[0].L = P.L0[lam]; ev[0].tau_path = 0.0; ev[0].tau_star = 0.0;
      int J = 0;
      for (int j = 1; j <= P.max_events && j <= kMaxAdjEvents; ++j) {
        const Checkpoint& e0 = ev[j - 1];
        const CartGrid::Cell c0{e0.ci, e0.cj, e0.ck};
        float th = 0.0f, tl = 0.0f;
        walk(P, e0.x, e0.k, e0.ci >= 0, c0, kappa, [&](int, float, float ds, float kr, int, bool) {
          float nh, e;
          tr::two_sum(th, kr * ds, nh, e);
          th = nh;
          tl += e;
          return true;
        });
        const double tau = (double)th + (double)tl;
        if (!(tau > 0.0)) break;  // escapes: no event j
        const double omE = -expm1(-tau);
        const uint4 r = draw_block(pid, lam, j, 0, P.seed, P.model);
        const double tau_star = -log1p(-u01(r.x) * omE);
        const float a0 = (float)tau_star, a1 = (float)(tau_star - (double)a0);
        float h2 = 0.0f, l2 = 0.0f, s_star = 0.0f;
        int hx = -1, hy = 0, hz = 0;
        walk(P, e0.x, e0.k, e0.ci >= 0, c0, kappa, [&](int cell, float t_in, float ds, float kr, int, bool last) {
          float nh, e;
          tr::two_sum(h2, kr * ds, nh, e);
          const float nl = l2 + e;
          if ((nh - a0) + (nl - a1) > 0.0f || last) {
            const float rem = ((a0 - h2) + a1) - l2;
            s_star = ((nh - a0) + (nl - a1) > 0.0f) ? t_in + rem / kr : t_in + ds;
            hx = cell % P.nx; hy = (cell / P.nx) % P.ny; hz = cell / (P.nx * P.ny);
            return false;
          }
          h2 = nh;
          l2 = nl;
          return true;
        });
        float3 x = make_float3(fmaf(s_star, e0.k.x, e0.x.x), fmaf(s_star, e0.k.y, e0.x.y), fmaf(s_star, e0.k.z, e0.x.z));
        const CartGrid::Cell hc{hx, hy, hz};
        CartGrid::clamp(P, hc, x);
        const float mu = hg_sample(LP.g, tr::u01f(r.y));
        float sp, cp;
        sincospif(2.0f * tr::u01f(r.z), &sp, &cp);
        Checkpoint& e1 = ev[j];
        e1.x = x;
        e1.k = rotate_dir(e0.k, mu, sp, cp);
        e1.ci = hx; e1.cj = hy; e1.ck = hz;
        e1.L = albedo * e0.L * omE;
        e1.tau_path = tau;
        e1.tau_star = tau_star;
        J = j;
        if (P.weight_cut && e1.L < P.L_cut[lam]) break;
      }
      // ---- backward sweep
      double3 xb = make_double3(0.0, 0.0, 0.0);
      double Lb = 0.0;
      const double* adjA = A.adj_abs ? A.adj_abs + (size_t)lam * P.n_cells : nullptr;
      for (int j = J; j >= 0; --j) {
        const Checkpoint& ej = ev[j];
        const CartGrid::Cell cj{ej.ci, ej.cj, ej.ck};
        // peel-offs from x_j
        const bool do_peel = j == 0 ? P.peel_emission : P.peel_scatter;
        for (int q = 0; do_peel && q < P.n_instr; ++q) {
          const DevInstr& I = tr::S_INSTR[q];
          const float3 kobs = make_float3(I.kobs[0], I.kobs[1], I.kobs[2]);
          double3 dW;
          const double W = adj_weight(A, q, lam, j > 0, ej.x, dW);
          if (W == 0.0 && dW.x == 0.0 && dW.y == 0.0 && dW.z == 0.0) continue;
          const float3 kin = j > 0 ? ev[j - 1].k : ej.k;
          const double phase = j > 0 ? (double)hg_phase(LP.g, kin.x * kobs.x + kin.y * kobs.y + kin.z * kobs.z) : 1.0;
          float tau = 0.0f;
          double3 gx = make_double3(0.0, 0.0, 0.0);
          float kr_prev = 0.0f;
          int axis_prev = -1;
          walk(P, ej.x, kobs, ej.ci >= 0, cj, kappa, [&](int, float, float ds, float kr, int axis, bool last) {
            tau += kr * ds;
            if (axis_prev >= 0) {  // plane between the previous and this segment
              const double3 dt = plane_dt_dx(axis_prev, kobs);
              const double jump = (double)kr_prev - (double)kr;
              gx.x += dt.x * jump; gx.y += dt.y * jump; gx.z += dt.z * jump;
            }
            kr_prev = kr;
            axis_prev = axis;
            if (last) {
              const double3 dt = plane_dt_dx(axis, kobs);
              gx.x += dt.x * kr; gx.y += dt.y * kr; gx.z += dt.z * kr;
            }
            return true;
          });
          const double pe = kInv4PiD * phase * exp(-(double)tau);
          const double V = ej.L * pe;
          const double l = V * W;
          Lb += pe * W;
          xb.x += V * dW.x - l * gx.x;
          xb.y += V * dW.y - l * gx.y;
          xb.z += V * dW.z - l * gx.z;
          walk(P, ej.x, kobs, ej.ci >= 0, cj, kappa, [&](int cell, float, float ds, float, int, bool) {
            grad_add(A.grad, cell, -l * (double)kappa * (double)ds);
            return true;
          });
        }
        if (j == 0) break;
        // forced path of event j from x_{j-1}
        const Checkpoint& ep = ev[j - 1];
        const CartGrid::Cell cp{ep.ci, ep.cj, ep.ck};
        const double L = ep.L;
        const double tau_path = ej.tau_path, tau_star = ej.tau_star;
        const double omE = -expm1(-tau_path);
        const double E = 1.0 - omE;
        const uint4 r = draw_block(pid, lam, j, 0, P.seed, P.model);
        const double u = u01(r.x);
        const float a0 = (float)tau_star, a1 = (float)(tau_star - (double)a0);
        const double wd = (1.0 - albedo) * L;
        // walk 1: deposit adjoints, interaction cell
        float th = 0.0f, tl = 0.0f;
        double dL_dep = 0.0, T_dep = 0.0;
        double e_prev = 1.0, a_prev = 0.0;
        bool found = false;
        int hit_cell = -1, hit_axis = -1;
        double tau_hm1 = 0.0, kr_h = 0.0;
        int axis_before = -1;
        walk(P, ep.x, ep.k, ep.ci >= 0, cp, kappa, [&](int cell, float, float ds, float kr, int axis, bool) {
          const float dt = kr * ds;
          float nh, e;
          tr::two_sum(th, dt, nh, e);
          const float nl = tl + e;
          const double a = (adjA && dt > 0.0f) ? adjA[cell] : 0.0;
          const double e_cur = exp(-((double)nh + (double)nl));
          // tau-adjoint of the previous index from the deposits, wd e_{m-1} (a_{m-1} - a_m)
          // (none before the first segment: tau_0 = 0 is not a variable)
          if (axis_before >= 0) T_dep += wd * e_prev * (a_prev - a);
          dL_dep += a * (e_prev - e_cur);
          if (!found && (nh - a0) + (nl - a1) > 0.0f) {
            found = true;
            hit_cell = cell;
            hit_axis = axis_before;  // plane crossed at the hit cell's entry
            tau_hm1 = (double)th + (double)tl;
            kr_h = kr;
          }
          th = nh;
          tl = nl;
          e_prev = e_cur;
          a_prev = a;
          axis_before = axis;
          return true;
        });
        T_dep += wd * e_prev * a_prev;  // last index: a_{n+1} = 0
        if (!found) {  // not reachable with identical pair sums; keep the packet's derivative finite
          atomicOr(P.flags, kFlagNoInteraction);
          continue;
        }
        const double Lb_prev = Lb * albedo * omE + (1.0 - albedo) * dL_dep;
        double Eb = -Lb * albedo * L;
        const double sb = xb.x * ep.k.x + xb.y * ep.k.y + xb.z * ep.k.z;
        const double tsb = sb / kr_h;  // adjoint of tau*
        Eb += tsb * (-u / (1.0 - u * omE));
        const double tb_path = -E * Eb;
        const double tb_hm1 = hit_axis >= 0 ? -tsb : 0.0;
        grad_add(A.grad, hit_cell, -sb * (tau_star - tau_hm1) * (double)kappa / (kr_h * kr_h));
        if (hit_axis >= 0) {
          const double3 dt = plane_dt_dx(hit_axis, ep.k);
          xb.x += sb * dt.x; xb.y += sb * dt.y; xb.z += sb * dt.z;
        }
        const double T = T_dep + tb_hm1 + tb_path;
        // walk 2: grad[c_m] += kappa ds_m S_m, plane terms of d/dx
        th = 0.0f; tl = 0.0f;
        double prefix = 0.0;
        e_prev = 1.0; a_prev = 0.0;
        double kr_prev = 0.0, S_prev = 0.0;
        int axis_prev = -1, m = 0;
        bool past_hit = false;
        walk(P, ep.x, ep.k, ep.ci >= 0, cp, kappa, [&](int cell, float, float ds, float kr, int axis, bool last) {
          const float dt = kr * ds;
          float nh, e;
          tr::two_sum(th, dt, nh, e);
          const float nl = tl + e;
          const double a = (adjA && dt > 0.0f) ? adjA[cell] : 0.0;
          const double e_cur = exp(-((double)nh + (double)nl));
          if (m > 0) {
            // close index m-1: its tau-adjoint enters the prefix
            prefix += wd * e_prev * (a_prev - a);
            if (!past_hit && cell == hit_cell) prefix += tb_hm1;  // index m-1 is h-1
          }
          if (cell == hit_cell) past_hit = true;
          const double S = T - prefix;
          grad_add(A.grad, cell, (double)kappa * (double)ds * S);
          if (axis_prev >= 0) {
            const double3 dtp = plane_dt_dx(axis_prev, ep.k);
            const double v = kr_prev * S_prev - (double)kr * S;
            xb.x += dtp.x * v; xb.y += dtp.y * v; xb.z += dtp.z * v;
          }
          if (last) {
            const double3 dte = plane_dt_dx(axis, ep.k);
            const double v = (double)kr * S;
            xb.x += dte.x * v; xb.y += dte.y * v; xb.z += dte.z * v;
          }
          kr_prev = kr;
          S_prev = S;
          axis_prev = axis;
          th = nh;
          tl = nl;
          e_prev = e_cur;
          a_prev = a;
          ++m;
          return true;
        });
        Lb = Lb_prev;
      }
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_adjoint(const FwdParams& f, const double* const* adj_img, const double* adj_abs, double* grad,
                           int num_sms, cudaStream_t stream) {
  AdjParams a;
  a.f = f;
  for (int q = 0; q < kMaxInstruments; ++q) a.adj_img[q] = q < f.n_instr ? adj_img[q] : nullptr;
  a.adj_abs = adj_abs;
  a.grad = grad;
  cudaError_t e = cudaMemsetAsync(f.work_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint, kAdjBlock, 0);
  if (e != cudaSuccess) return e;
  per_sm = per_sm < 1 ? 1 : per_sm;
  unsigned long long blocks = (unsigned long long)num_sms * per_sm;
  const unsigned long long useful = (f.n_total + kAdjBlock - 1) / kAdjBlock;
  if (blocks > useful) blocks = useful;
  if (blocks < 1) blocks = 1;
  k_adjoint<<<(unsigned)blocks, kAdjBlock, 0, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace rtk

// Vector kernels of the outer float64 PCG recurrence (Section 6: CG
// preconditioned by one V-cycle), the precision boundary, permutations and
// the fused ionic update + right-hand side of the time step (Section 3.1).
// Dot products are reduced deterministically: a fixed grid writes one partial
// per block and the last block to finish sums them in block order.
#pragma once
#include "../../include/aggmg.h"
#include "face_op.cuh"
#include "kernels.cuh"

namespace aggmg {

enum { TK_PQ = 0, TK_R = 1, TK_Z = 2, TK_R0 = 3 };

// Loop control of the WHILE node, launched after the PCG set-up and at the end
// of every iteration: ends the loop once the solve is done, and after
// max_it + 2 iterations in any case. It is the only kernel that calls the
// device-side graph API, so every compute kernel stays visible to profilers.
static __global__ void k_loop_ctl(CGState* st) {
  if (st->done || st->guard >= st->max_it + 2) {
    st->done = 1;
    if (st->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, 0u);
  }
  st->guard += 1;
}

// Reset of the per-solve fields (and of the coarse-level kernel's grid
// barrier, if any); the options (rtol, atol, max_it, flexible, cond,
// use_cond) are written by the host before the launch.
static __global__ void k_cg_reset(CGState* st, GridBar* bar) {
  if (bar) {
    bar->count = 0u;
    bar->err = 0;
  }
  st->guard = 0;
  st->iter = 0;
  st->done = 0;
  st->status = 0;
  st->rho = st->alpha = st->beta = st->pq = st->rr = st->r0 = 0.0;
  st->rz_old = 0.0;
}

// Start of a solve: reset (with the coarse-level kernel's grid barrier, if
// any) and select the WHILE node that this launch ends.
static __global__ void k_cg_begin(CGState* st, unsigned long long cond, int use_cond, GridBar* bar) {
  if (bar) {
    bar->count = 0u;
    bar->err = 0;
  }
  st->iter = 0;
  st->done = 0;
  st->status = 0;
  st->rho = st->alpha = st->beta = st->pq = st->rr = st->r0 = 0.0;
  st->rz_old = 0.0;
  st->guard = 0;
  st->cond = cond;
  st->use_cond = use_cond;
}

static __global__ void k_set_opts(CGState* st, double rtol, double atol, int max_it, int flexible) {
  st->rtol = rtol;
  st->atol = atol;
  st->max_it = max_it;
  st->flexible = flexible;
}

static __global__ void k_noop() {}

// ||r0||, tolerance, early exit when already converged
static __global__ void __launch_bounds__(RED_NT) k_r0(const double* __restrict__ r, int64_t n, double* partials, CGState* st) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * RED_NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_NT)
    s += r[i] * r[i];
  if (partial_and_last<RED_NT>(s, partials, &st->ticket[TK_R0])) {
    double rr = sum_partials<RED_NT>(partials, gridDim.x);
    if (threadIdx.x == 0) {
      st->ticket[TK_R0] = 0;
      st->rr = rr;
      st->r0 = sqrt(rr);
      st->tol = fmax(st->rtol * st->r0, st->atol);
      if (!isfinite(st->r0)) {
        st->status = -6;
        st->done = 1;
      } else if (st->r0 <= st->tol || st->r0 == 0.0) {
        st->done = 1;
      }
    }
  }
}

// x += alpha p; r -= alpha q; ||r||; convergence test. Fused with the
// V-cycle's input cast (r32 = (float) r, when r32 is given) and, for the
// flexible variant, the (r_new, z_old) product of the Polak-Ribiere beta
// (z_old: the previous preconditioned residual). Both sums use the fixed
// grid and block order of the other reductions (second sum in
// partials[gridDim.x ..]).
static __global__ void __launch_bounds__(RED_NT) k_cg_update(double* __restrict__ x, double* __restrict__ r,
                                                      const double* __restrict__ p, const double* __restrict__ q,
                                                      float* __restrict__ r32, const double* __restrict__ zold,
                                                      int64_t n, double* partials, CGState* st) {
  if (st->done) return;
  const double alpha = st->alpha;
  const bool flex = st->flexible != 0;
  double s = 0.0, sz = 0.0;
  // pairs of entries per 16-byte access (n is even: whole 32-unit slices),
  // a scalar tail otherwise
  const int64_t n2 = n >> 1;
  for (int64_t i = (int64_t)blockIdx.x * RED_NT + threadIdx.x; i < n2; i += (int64_t)gridDim.x * RED_NT) {
    double2 xv = reinterpret_cast<double2*>(x)[i];
    double2 rv = reinterpret_cast<double2*>(r)[i];
    const double2 pv = reinterpret_cast<const double2*>(p)[i];
    const double2 qv = reinterpret_cast<const double2*>(q)[i];
    xv.x += alpha * pv.x;
    xv.y += alpha * pv.y;
    rv.x = rv.x - alpha * qv.x;
    rv.y = rv.y - alpha * qv.y;
    reinterpret_cast<double2*>(x)[i] = xv;
    reinterpret_cast<double2*>(r)[i] = rv;
    s += rv.x * rv.x;
    s += rv.y * rv.y;
    if (flex) {
      const double2 zv = reinterpret_cast<const double2*>(zold)[i];
      sz += rv.x * zv.x;
      sz += rv.y * zv.y;
    }
    if (r32) reinterpret_cast<float2*>(r32)[i] = make_float2((float)rv.x, (float)rv.y);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
    if (flex) sz += ri * zold[i];
    if (r32) r32[i] = (float)ri;
  }
  const double bz = block_sum<RED_NT>(sz);
  if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = bz;
  if (partial_and_last<RED_NT>(s, partials, &st->ticket[TK_R])) {
    double rr = sum_partials<RED_NT>(partials, gridDim.x);
    double rz = sum_partials<RED_NT>(partials + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      st->ticket[TK_R] = 0;
      if (flex) st->rz_old = rz;
      st->rr = rr;
      st->iter += 1;
      double rn = sqrt(rr);
      if (!isfinite(rn)) {
        st->status = -6;
        st->done = 1;
      } else if (rn <= st->tol) {
        st->done = 1;
      } else if (st->iter >= st->max_it) {
        st->status = -5;
        st->done = 1;
      }
    }
  }
}

// z64 <- zin (V-cycle output, any precision); rz = (r, z_new).
// INIT: rho = rz.  Otherwise beta = rz / rho (Fletcher-Reeves form) or, for
// the flexible variant, beta = (rz - (r, z_old)) / rho (Polak-Ribiere, with
// (r, z_old) from k_cg_update), then rho = rz.
template <typename TZ, bool INIT>
static __global__ void __launch_bounds__(RED_NT) k_zdot(const TZ* __restrict__ zin, double* __restrict__ z64,
                                                 const double* __restrict__ r, int64_t n, double* partials,
                                                 CGState* st) {
  if (st->done) return;
  double s = 0.0;
  using Z2 = typename std::conditional<std::is_same<TZ, float>::value, float2, double2>::type;
  const int64_t n2 = n >> 1;
  for (int64_t i = (int64_t)blockIdx.x * RED_NT + threadIdx.x; i < n2; i += (int64_t)gridDim.x * RED_NT) {
    const Z2 zv = reinterpret_cast<const Z2*>(zin)[i];
    const double2 rv = reinterpret_cast<const double2*>(r)[i];
    const double2 zn = make_double2((double)zv.x, (double)zv.y);
    reinterpret_cast<double2*>(z64)[i] = zn;
    s += rv.x * zn.x;
    s += rv.y * zn.y;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const double zn = (double)zin[n - 1];
    z64[n - 1] = zn;
    s += r[n - 1] * zn;
  }
  if (partial_and_last<RED_NT>(s, partials, &st->ticket[TK_Z])) {
    const double rz = sum_partials<RED_NT>(partials, gridDim.x);
    if (threadIdx.x == 0) {
      st->ticket[TK_Z] = 0;
      if (INIT) st->beta = 0.0;
      else st->beta = (st->flexible ? rz - st->rz_old : rz) / st->rho;
      st->rho = rz;
    }
  }
}

// p = z + beta p (INIT: p = z)
template <bool INIT>
static __global__ void __launch_bounds__(RED_NT) k_pupd(const double* __restrict__ z, double* __restrict__ p, int64_t n,
                                                 const CGState* st) {
  if (st->done) return;
  const double beta = st->beta;
  const int64_t n2 = n >> 1;
  for (int64_t i = (int64_t)blockIdx.x * RED_NT + threadIdx.x; i < n2; i += (int64_t)gridDim.x * RED_NT) {
    const double2 zv = reinterpret_cast<const double2*>(z)[i];
    if (INIT) {
      reinterpret_cast<double2*>(p)[i] = zv;
    } else {
      double2 pv = reinterpret_cast<double2*>(p)[i];
      pv.x = zv.x + beta * pv.x;
      pv.y = zv.y + beta * pv.y;
      reinterpret_cast<double2*>(p)[i] = pv;
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) p[n - 1] = INIT ? z[n - 1] : z[n - 1] + beta * p[n - 1];
}

template <typename TO, typename TI>
static __global__ void k_cast(const TI* __restrict__ in, TO* __restrict__ out, int64_t n, const CGState* st) {
  if (st && st->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

// dst[i*B + r] = src[perm[i]*B + r]  (caller order -> internal order)
template <typename TO, typename TI>
static __global__ void k_gather_units(const TI* __restrict__ src, TO* __restrict__ dst, const int64_t* __restrict__ perm,
                               int64_t n, int B) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n * B) return;
  const int64_t i = id / B;
  const int r = (int)(id % B);
  dst[id] = (TO)src[perm[i] * B + r];
}
// dst[perm[i]*B + r] = src[i*B + r]  (internal order -> caller order)
template <typename TO, typename TI>
static __global__ void k_scatter_units(const TI* __restrict__ src, TO* __restrict__ dst, const int64_t* __restrict__ perm,
                                int64_t n, int B) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n * B) return;
  const int64_t i = id / B;
  const int r = (int)(id % B);
  dst[perm[i] * B + r] = (TO)src[id];
}

// ---------------------------------------------------------------- ionic models
struct IonicParams {
  int model;
  double k, a, eps, gamma, mu1, mu2;
  agg_bueno_orovio_params bo;
};

// Gates per DoF: FitzHugh-Nagumo and Aliev-Panfilov 1, Bueno-Orovio 3; gate g
// of DoF i lives at w[g * stride + i].
constexpr int kMaxGates = 3;
__host__ __device__ inline int ionic_gates(int model) { return model == 2 ? 3 : 1; }

__device__ __forceinline__ double unit_step(double z, double z0) { return z >= z0 ? 1.0 : 0.0; }
__device__ __forceinline__ double smooth_step(double z, double z0, double k) {
  return 0.5 * (1.0 + tanh(k * (z - z0)));
}

// Bueno-Orovio (Section 2.3.2, Eq. BuenoOrovio): I_ion and the three gate rates
__device__ __forceinline__ void bueno_orovio_eval(const agg_bueno_orovio_params& p, double u, const double* w,
                                                  double& I, double* H) {
  const double hv1 = unit_step(u, p.V1), hv1m = unit_step(u, p.V1m);
  const double hv2 = unit_step(u, p.V2), hvo = unit_step(u, p.Vo);
  const double a0 = (1.0 - hv1) / (hv1m * (p.tau1pp - p.tau1p) + p.tau1p);
  const double b0 = -hv1 / p.tau1plus;
  const double w0inf = 1.0 - hv1m;
  const double a1 = (1.0 - hv2) / (smooth_step(u, p.V2m, p.k2) * (p.tau2pp - p.tau2p) + p.tau2p);
  const double b1 = -hv2 / p.tau2plus;
  const double w1inf = hvo * (p.winf_star - 1.0 + u / p.tau2inf) + 1.0 - u / p.tau2inf;
  const double a2 = 1.0 / (hv2 * (p.tau3pp - p.tau3p) + p.tau3p);
  const double w2inf = smooth_step(u, p.V3, p.k3);
  H[0] = (b0 - a0) * w[0] + a0 * w0inf;
  H[1] = (b1 - a1) * w[1] + a1 * w1inf;
  H[2] = -a2 * w[2] + a2 * w2inf;
  const double ifi = -hv1 * (u - p.V1) * (p.Vhat - u) * w[0] / p.taufi;
  const double iso = (1.0 - hv2) * (u - p.uo) / (hvo * (p.tauo_pp - p.tauo_p) + p.tauo_p) +
                     hv2 / (smooth_step(u, p.Vso, p.kso) * (p.tauso_pp - p.tauso_p) + p.tauso_p);
  const double isi = -hv2 * w[1] * w[2] / p.tausi;
  I = ifi + iso + isi;
}

// I_ion(u, w) and the gate rates H(u, w) (w, H: ionic_gates(model) values)
__device__ __forceinline__ void ionic_eval(const IonicParams& p, double u, const double* w, double& I, double* H) {
  if (p.model == 2) {
    bueno_orovio_eval(p.bo, u, w, I, H);
    return;
  }
  const double cub = p.k * u * (u - p.a) * (u - 1.0);
  if (p.model == 0) {
    I = cub + w[0];
    H[0] = p.eps * (u - p.gamma * w[0]);
  } else {
    I = cub + u * w[0];
    H[0] = (p.eps + p.mu1 * w[0] / (u + p.mu2)) * (-w[0] - p.k * u * (u - p.a - 1.0));
  }
}

// gate values of DoF i (stride between gates) into g[]
__device__ __forceinline__ void load_gates(const double* w, int64_t stride, int64_t i, int ng, double* g) {
#pragma unroll
  for (int k = 0; k < kMaxGates; ++k) g[k] = (k < ng) ? w[k * stride + i] : 0.0;
}

static __global__ void k_ionic_update(IonicParams prm, double dt, int64_t n, const double* __restrict__ u,
                               double* __restrict__ w) {
  const int ng = ionic_gates(prm.model);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double g[kMaxGates], H[kMaxGates], I;
    load_gates(w, n, i, ng, g);
    ionic_eval(prm, u[i], g, I, H);
#pragma unroll
    for (int k = 0; k < kMaxGates; ++k)
      if (k < ng) w[k * n + i] = g[k] + dt * H[k];
  }
}

// Time step prologue for the thread's element (Section 3.1):
//   w <- w + dt H(u, w);  f = I_app(t_{n+1}) mask - chi I(u, w_new);
//   b_e = M_e (c u_e + f_e)   (ionic current interpolation)
template <int B>
static __global__ void __launch_bounds__(UnitThreads<B>::value)
    k_ionic_rhs(const double* __restrict__ Me, const double* __restrict__ u, double* __restrict__ w,
                const double* __restrict__ mask, double* __restrict__ b, IonicParams prm, double dt, double chi,
                double c, double iapp_value, int64_t iapp_steps, const int64_t* __restrict__ step, int64_t nslices,
                int64_t wstride) {
  constexpr int NTB = UnitThreads<B>::value;
  constexpr int KP = Pad<double, B>::KP;
  const int lane = threadIdx.x & 31;
  {
  const int64_t slice = first_slice<NTB>();
  if (slice >= nslices) return;
  const int64_t unit = slice * SL + lane;
  const size_t o = (size_t)unit * B;
  const double ia = (*step < iapp_steps) ? iapp_value : 0.0;
  // per DoF: ionic update and the nodal load c u + I_app mask - chi I(u, w_new)
  const int ng = ionic_gates(prm.model);
  auto nodal = [&](int r) {
    const double ur = u[o + r];
    double g[kMaxGates], H[kMaxGates], I;
    load_gates(w, wstride, o + r, ng, g);
    ionic_eval(prm, ur, g, I, H);
#pragma unroll
    for (int k = 0; k < kMaxGates; ++k) {
      g[k] += dt * H[k];
      if (k < ng) w[k * wstride + o + r] = g[k];
    }
    ionic_eval(prm, ur, g, I, H);
    return c * ur + ia * mask[o + r] - chi * I;
  };
  double acc[B];
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = 0.0;
  const double* Mb = Me + (size_t)slice * SL * KP;
  if constexpr (B > 32) {
    __shared__ double tsh[B * NTB];
    double* ts = tsh + threadIdx.x;
#pragma unroll
    for (int r = 0; r < B; ++r) ts[r * NTB] = nodal(r);
    block_mv<double, double, B, NTB>(Mb, lane, ts, acc);
  } else {
    double t[B];
#pragma unroll
    for (int r = 0; r < B; ++r) t[r] = nodal(r);
    block_mv<double, double, B>(Mb, lane, t, acc);
  }
#pragma unroll
  for (int r = 0; r < B; ++r) b[o + r] = acc[r];
  }
}

// BDF2 history at the start (second-order derivative start), per element:
//   u^{-1} = u - dt u',  chi C_m u' = I_app - chi I(u, w) - M^{-1} A u,
//   w^{-1} = w - dt H(u, w),   with M^{-1} A u = M_e^{-1} (A0 u)_e - c u.
template <int B>
static __global__ void __launch_bounds__(UnitThreads<B>::value)
    k_bdf2_start(const double* __restrict__ Minv, const double* __restrict__ A0u, const double* __restrict__ u,
                 const double* __restrict__ w, const double* __restrict__ mask, double* __restrict__ up,
                 double* __restrict__ wp, IonicParams prm, double dt, double chi, double cm, double c, double ia,
                 int64_t nslices, int64_t wstride) {
  constexpr int NTB = UnitThreads<B>::value;
  constexpr int KP = Pad<double, B>::KP;
  const int lane = threadIdx.x & 31;
  const int64_t slice = first_slice<NTB>();
  if (slice >= nslices) return;
  const size_t o = (size_t)(slice * SL + lane) * B;
  double t[B];
#pragma unroll
  for (int r = 0; r < B; ++r) t[r] = 0.0;
  block_mv<double, double, B>(Minv + (size_t)slice * SL * KP, lane, A0u + o, t);
  const int ng = ionic_gates(prm.model);
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const double ur = u[o + r];
    double g[kMaxGates], H[kMaxGates], I;
    load_gates(w, wstride, o + r, ng, g);
    ionic_eval(prm, ur, g, I, H);
    const double f0 = ia * mask[o + r] - chi * I;
    const double udot = (f0 - (t[r] - c * ur)) / (chi * cm);
    up[o + r] = ur - dt * udot;
#pragma unroll
    for (int k = 0; k < kMaxGates; ++k)
      if (k < ng) wp[k * wstride + o + r] = g[k] - dt * H[k];
  }
}

// BDF2 step prologue (Eq. fully_discrete with extrapolation), per element:
//   U* = 2u - up, W* = 2w - wp, w_new = (4w - wp)/3 + (2dt/3) H(U*, W*),
//   f = I_app mask - chi I(U*, w_new), b_e = M_e (chi C_m (4u - up)/(2dt) + f);
//   then the history shifts: up <- u, wp <- w, w <- w_new.
template <int B>
static __global__ void __launch_bounds__(UnitThreads<B>::value)
    k_ionic_rhs_bdf2(const double* __restrict__ Me, const double* __restrict__ u, double* __restrict__ up,
                     double* __restrict__ w, double* __restrict__ wp, const double* __restrict__ mask,
                     double* __restrict__ b, IonicParams prm, double dt, double chi, double cm, double iapp_value,
                     int64_t iapp_steps, const int64_t* __restrict__ step, int64_t nslices, int64_t wstride) {
  constexpr int NTB = UnitThreads<B>::value;
  constexpr int KP = Pad<double, B>::KP;
  const int lane = threadIdx.x & 31;
  const int64_t slice = first_slice<NTB>();
  if (slice >= nslices) return;
  const size_t o = (size_t)(slice * SL + lane) * B;
  const double ia = (*step < iapp_steps) ? iapp_value : 0.0;
  const int ng = ionic_gates(prm.model);
  auto nodal = [&](int r) {
    const double un = u[o + r], upr = up[o + r];
    const double us = 2.0 * un - upr;
    double wn[kMaxGates], wpr[kMaxGates], ws[kMaxGates], w1[kMaxGates], H[kMaxGates], I;
    load_gates(w, wstride, o + r, ng, wn);
    load_gates(wp, wstride, o + r, ng, wpr);
#pragma unroll
    for (int k = 0; k < kMaxGates; ++k) ws[k] = 2.0 * wn[k] - wpr[k];
    ionic_eval(prm, us, ws, I, H);
#pragma unroll
    for (int k = 0; k < kMaxGates; ++k) w1[k] = (4.0 * wn[k] - wpr[k]) / 3.0 + (2.0 * dt / 3.0) * H[k];
    ionic_eval(prm, us, w1, I, H);
    up[o + r] = un;
#pragma unroll
    for (int k = 0; k < kMaxGates; ++k)
      if (k < ng) {
        wp[k * wstride + o + r] = wn[k];
        w[k * wstride + o + r] = w1[k];
      }
    return chi * cm / (2.0 * dt) * (4.0 * un - upr) + ia * mask[o + r] - chi * I;
  };
  double acc[B];
#pragma unroll
  for (int r = 0; r < B; ++r) acc[r] = 0.0;
  const double* Mb = Me + (size_t)slice * SL * KP;
  if constexpr (B > 32) {
    __shared__ double tsh[B * NTB];
    double* ts = tsh + threadIdx.x;
#pragma unroll
    for (int r = 0; r < B; ++r) ts[r * NTB] = nodal(r);
    block_mv<double, double, B, NTB>(Mb, lane, ts, acc);
  } else {
    double tv[B];
#pragma unroll
    for (int r = 0; r < B; ++r) tv[r] = nodal(r);
    block_mv<double, double, B>(Mb, lane, tv, acc);
  }
#pragma unroll
  for (int r = 0; r < B; ++r) b[o + r] = acc[r];
}

// Partial derivatives of the ionic model at one DoF (I_u, I_w, H_u, H_w).
__device__ __forceinline__ void ionic_jac(const IonicParams& p, double u, double w, double& Iu, double& Iw,
                                          double& Hu, double& Hw) {
  const double dcub = p.k * (3.0 * u * u - 2.0 * (p.a + 1.0) * u + p.a);
  if (p.model == 0) {
    Iu = dcub;
    Iw = 1.0;
    Hu = p.eps;
    Hw = -p.eps * p.gamma;
  } else {
    Iu = dcub + w;
    Iw = u;
    const double den = u + p.mu2;
    const double e = p.eps + p.mu1 * w / den;
    const double g = -w - p.k * u * (u - p.a - 1.0);
    const double e_u = -p.mu1 * w / (den * den), e_w = p.mu1 / den;
    const double g_u = -p.k * (2.0 * u - p.a - 1.0);
    Hu = e_u * g + e * g_u;
    Hw = e_w * g - e;
  }
}

// Reverse of one time step, pointwise part, for the thread's element
// (discrete adjoint of the step; lambda = K^{-1} ubar is the input):
//   q = M_e lambda_e,  w~ = wbar - chi I_w(u_n, w_np1) q,
//   ubar_n = q (c - chi I_u(u_n, w_np1)) + dt H_u(u_n, w_n) w~,
//   wbar_n = w~ (1 + dt H_w(u_n, w_n)),   with w_np1 = w_n + dt H(u_n, w_n).
template <int B>
static __global__ void __launch_bounds__(UnitThreads<B>::value)
    k_adj_pointwise(const double* __restrict__ Me, const double* __restrict__ lam, const double* __restrict__ u_n,
                    const double* __restrict__ w_n, double* __restrict__ ubar, double* __restrict__ wbar,
                    IonicParams prm, double dt, double chi, double c, int64_t nslices) {
  constexpr int NTB = UnitThreads<B>::value;
  constexpr int KP = Pad<double, B>::KP;
  const int lane = threadIdx.x & 31;
  {
  const int64_t slice = first_slice<NTB>();
  if (slice >= nslices) return;
  const int64_t unit = slice * SL + lane;
  const size_t o = (size_t)unit * B;
  double q[B];
#pragma unroll
  for (int r = 0; r < B; ++r) q[r] = 0.0;
  if constexpr (B > 32) {
    block_mv<double, double, B>(Me + (size_t)slice * SL * KP, lane, lam + o, q);
  } else {
    double lv[B];
#pragma unroll
    for (int r = 0; r < B; ++r) lv[r] = lam[o + r];
    block_mv<double, double, B>(Me + (size_t)slice * SL * KP, lane, lv, q);
  }
#pragma unroll
  for (int r = 0; r < B; ++r) {
    const double un = u_n[o + r], wn = w_n[o + r];
    double I, H[kMaxGates], Iu, Iw, Hu, Hw, Iu1, Iw1, Hu1, Hw1;
    const double wg[kMaxGates] = {wn, 0.0, 0.0};
    ionic_eval(prm, un, wg, I, H);                 // one-gate models only
    const double w1 = wn + dt * H[0];
    ionic_jac(prm, un, w1, Iu1, Iw1, Hu1, Hw1);
    ionic_jac(prm, un, wn, Iu, Iw, Hu, Hw);
    const double wt = wbar[o + r] - chi * Iw1 * q[r];
    ubar[o + r] = q[r] * (c - chi * Iu1) + dt * Hu * wt;
    wbar[o + r] = wt * (1.0 + dt * Hw);
  }
  }
}

// Layout of the adjoint face parts on the device: per slice and local face,
// five row-major parts (the structure of Mesh::Yc), each padded to whole
// double2 chunks, in the sliced chunk order [chunk][lane][2].
template <int B> struct AdjFaceLayout {
  static constexpr int NF = FaceIdx<FaceShape<B>::D, FaceShape<B>::N>::NF;
  static constexpr int P1 = (NF * B + 1) / 2 * 2, P2 = ((B - NF) * NF + 1) / 2 * 2, P3 = (B * NF + 1) / 2 * 2;
  static constexpr int P4 = P1, P5 = (NF * NF + 1) / 2 * 2;
  static constexpr int YS = P1 + P2 + P3 + P4 + P5;      // doubles per lane and face
};

// sum_{r, c} y(r) M[r][c] x(c) over one R x C part starting at chunk ch0
template <int R, int C, typename YF, typename XF>
__device__ __forceinline__ double part_bilinear(const double2* yb, int ch0, YF y, XF x) {
  double s = 0.0;
#pragma unroll 1
  for (int ch = 0; ch < (R * C + 1) / 2; ++ch) {
    const double2 v = __ldg(yb + (size_t)(ch0 + ch) * SL);
    const int k = 2 * ch;
    s += v.x * y(k / C) * x(k % C);
    if (k + 1 < R * C) s += v.y * y((k + 1) / C) * x((k + 1) % C);
  }
  return s;
}

// Per-element log-conductivity gradient, accumulated in the caller's order:
//   grad[e] -= lam_e^T Ke u_e + sum_faces [lam_e; lam_n]^T Y_e,F [u_e; u_n]
// with Ke the volume form and Y_e,F the face terms built with D_e, of which
// only the trace-structured parts are stored (AdjFaceLayout): ee on e's face
// rows and face columns, en on n's face columns, ne on n's face rows, nn.
template <int B>
static __global__ void __launch_bounds__(UnitThreads<B>::value)
    k_grad_logD(FaceView<double, B> F, const double* __restrict__ Ke, const double* __restrict__ Yc,
                const double* __restrict__ lam, const double* __restrict__ u, const int64_t* __restrict__ perm,
                double* __restrict__ grad, int64_t n) {
  constexpr int NTB = UnitThreads<B>::value;
  constexpr int KP = Pad<double, B>::KP;
  using FI = FaceIdx<FaceShape<B>::D, FaceShape<B>::N>;
  using YL = AdjFaceLayout<B>;
  constexpr int NF = YL::NF, NFACE = 2 * FaceShape<B>::D;
  const int lane = threadIdx.x & 31;
  const int64_t slice = first_slice<NTB>();
  if (slice >= F.nslices) return;
  const int64_t unit = slice * SL + lane;
  const size_t o = (size_t)unit * B;
  double t[B];
#pragma unroll
  for (int r = 0; r < B; ++r) t[r] = 0.0;
  block_mv<double, double, B>(Ke + (size_t)slice * SL * KP, lane, u + o, t);
  double g = 0.0;
#pragma unroll
  for (int r = 0; r < B; ++r) g += lam[o + r] * t[r];
  const double* lu = lam + o;
  const double* uu = u + o;
#pragma unroll 1
  for (int f = 0; f < NFACE; ++f) {
    const size_t fi = ((size_t)slice * NFACE + f) * SL + lane;
    const int nb = F.nbr[fi];
    if (nb < 0) continue;
    const int fn = F.code[fi];
    const double* ln = lam + (size_t)nb * B;
    const double* un = u + (size_t)nb * B;
    const double2* yb = reinterpret_cast<const double2*>(Yc) + ((size_t)(slice * NFACE + f) * (YL::YS / 2)) * SL + lane;
    g += part_bilinear<NF, B>(yb, 0, [&](int r) { return lu[FI::face(f, r)]; }, [&](int c) { return uu[c]; });
    g += part_bilinear<B - NF, NF>(yb, YL::P1 / 2, [&](int r) { return lu[FI::off(f, r)]; },
                                   [&](int c) { return uu[FI::face(f, c)]; });
    g += part_bilinear<B, NF>(yb, (YL::P1 + YL::P2) / 2, [&](int r) { return lu[r]; },
                              [&](int c) { return un[FI::face(fn, c)]; });
    g += part_bilinear<NF, B>(yb, (YL::P1 + YL::P2 + YL::P3) / 2, [&](int r) { return ln[FI::face(fn, r)]; },
                              [&](int c) { return uu[c]; });
    g += part_bilinear<NF, NF>(yb, (YL::P1 + YL::P2 + YL::P3 + YL::P4) / 2,
                               [&](int r) { return ln[FI::face(fn, r)]; }, [&](int c) { return un[FI::face(fn, c)]; });
  }
  if (unit < n) grad[perm[unit]] -= g;
}

// end of a time step: record the iteration count, advance the clock
static __global__ void k_step_end(const CGState* st, int64_t* step, int* iters, int* slot, int capacity, int* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const int s = *slot;
    if (s < capacity) iters[s] = st->iter;
    if (st->status != 0 && *status == 0) *status = st->status;
    *slot = s + 1;
    *step = *step + 1;
  }
}

}  // namespace aggmg

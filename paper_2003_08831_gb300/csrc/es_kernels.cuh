// Kernels of one relaxed RK step (templated on the LGL point count P1 = p+1
// and on the flux precision TF).  Each per-P1 translation unit instantiates
// them through the launchers at the bottom.
//
// Stage pipeline (Eq. (RK-step), Eq. (compressible_ns_diss)):
//   k_prep    y^i = u + dt sum_j a_ij k_j (fused relaxed update of the previous
//             step), parameter-vector state z and 1/z1 per node; for i > 1 the
//             increment w(y^i) - w(u) of the entropy variables.
//   k_face    interface flux f*(q-, q+) - diss lambda/2 (q+ - q-) per face node
//             (prescribed exterior states on Dirichlet-penalty boundary faces).
//   k_grad    (Navier--Stokes) BR1 entropy-variable gradients and the viscous
//             flux F^V_m = C_mj theta_j per node.
//   k_volume  per element: flux-differencing sums along every LGL line,
//             interface terms, viscous divergence; k_i, and the element sums
//             (eta' f)(y^i) (Eq. (eta-est-1-RK)) and the relaxation term A.
//   k_relax   per element (a group of 8-32 lanes): gamma_kappa of
//             Eq. (relaxation-local-gamma); atomic min into gamma (k_relax_ff:
//             the same in float-float for the mixed and ES_FP64X modes).
//   k_scalar  gamma = min gamma_kappa, t += gamma dt (Eq. (t-n-gamma)).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "es_device.cuh"
#include "es_launch.h"

namespace es {

// Volume-kernel tiles: elements per CTA (EPB) and threads per CTA for each degree.
// A CTA handles EPB (p+1)^2 lines per direction; the candidates are chosen so the
// lines fill whole warps or nearly so.  Variant 0 is the default; the batch
// autotuner times all of them on the instance data and keeps the fastest.
template <int P1, int V> struct VolCfg;
template <> struct VolCfg<3, 0> { static constexpr int EPB = 32, THREADS = 288; };
template <> struct VolCfg<3, 1> { static constexpr int EPB = 16, THREADS = 160; };
template <> struct VolCfg<3, 2> { static constexpr int EPB = 8, THREADS = 96; };
template <> struct VolCfg<4, 0> { static constexpr int EPB = 8, THREADS = 128; };
template <> struct VolCfg<4, 1> { static constexpr int EPB = 4, THREADS = 64; };
template <> struct VolCfg<4, 2> { static constexpr int EPB = 16, THREADS = 256; };
template <> struct VolCfg<5, 0> { static constexpr int EPB = 5, THREADS = 128; };
template <> struct VolCfg<5, 1> { static constexpr int EPB = 10, THREADS = 256; };
template <> struct VolCfg<5, 2> { static constexpr int EPB = 2, THREADS = 64; };
template <> struct VolCfg<6, 0> { static constexpr int EPB = 4, THREADS = 160; };
template <> struct VolCfg<6, 1> { static constexpr int EPB = 2, THREADS = 96; };
template <> struct VolCfg<6, 2> { static constexpr int EPB = 8, THREADS = 288; };

// ---------------------------------------------------------------------------
// accurate w(u + e) - w(u) from the increment e (no cancellation):
// x = e_rho/rho, dv = (e_m - v e_rho)/(rho + e_rho),
// y = (p' - p)/p = (gam-1)[e_E - v.e_m + |v|^2 e_rho/2 - (rho + e_rho)|dv|^2/2]/p,
// beta = rho/p, ds = log1p(y) - gam log1p(x),
// dw1 = -ds/(gam-1) - beta[(x-y)|v|^2 + (1+x)(2 v.dv + |dv|^2)]/(2(1+y)),
// dw_v = beta[(x-y) v + (1+x) dv]/(1+y), dw5 = -beta (x-y)/(1+y).
// With Pr = rho p = (gam-1)(rho E - |m|^2/2), one division 1/(rho rho' Pr) gives
// 1/rho, 1/rho' and 1/p (|v|^2 = |m|^2/rho^2); a second gives beta/(1+y), shared by
// every component.
__device__ __forceinline__ void entropy_var_increment(const double u[5], const double e[5], double gam,
                                                      double inv_gm1, double dw[5]) {
  const double gm1 = gam - 1.0;
  const double rho = u[0];
  const double rho1 = rho + e[0];
  const double m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const double Pr = gm1 * (rho * u[4] - 0.5 * m2);
  const double rr1 = rho * rho1;
  const double inv = fast_rcp(rr1 * Pr);
  const double pinv = Pr * inv;
  const double ir = rho1 * pinv, ir1 = rho * pinv, ip = rho * rr1 * inv;
  const double v0 = u[1] * ir, v1 = u[2] * ir, v2 = u[3] * ir;
  const double v2s = m2 * ir * ir;
  const double x = e[0] * ir;
  const double d0 = (e[1] - v0 * e[0]) * ir1, d1 = (e[2] - v1 * e[0]) * ir1, d2 = (e[3] - v2 * e[0]) * ir1;
  const double dv2 = d0 * d0 + d1 * d1 + d2 * d2;
  const double y =
      gm1 * (e[4] - (v0 * e[1] + v1 * e[2] + v2 * e[3]) + 0.5 * v2s * e[0] - 0.5 * rho1 * dv2) * ip;
  const double beta = rho * ip;
  const double biy = beta * fast_rcp(1.0 + y);  // beta / (1 + y)
  const double ds = (y + log1pmx(y)) - gam * (x + log1pmx(x));
  const double xy = x - y;
  const double opx = 1.0 + x;
  const double dkin = 0.5 * biy * (xy * v2s + opx * (2.0 * (v0 * d0 + v1 * d1 + v2 * d2) + dv2));
  dw[0] = -ds * inv_gm1 - dkin;
  dw[1] = biy * (xy * v0 + opx * d0);
  dw[2] = biy * (xy * v1 + opx * d1);
  dw[3] = biy * (xy * v2 + opx * d2);
  dw[4] = -biy * xy;
}

// ---------------------------------------------------------------------------
// Float-float pieces of the stage preparation in the mixed and ES_FP64X modes:
// the parameter vector and the entropy-variable increments on the FP32 pipe
// (es_ff.cuh), the FP64 state only read and split.
__device__ __forceinline__ ff to_ff(ff x) { return x; }
__device__ __forceinline__ ff to_ff(float x) { return ff(x, 0.0f); }
__device__ __forceinline__ ff to_ff(double x) { return ff_from_double(x); }
__device__ __forceinline__ ff ff_half(ff x) { return ff(0.5f * x.hi, 0.5f * x.lo); }
// a float-float value in the flux precision (float: hi + lo rounded once)
template <typename T> __device__ __forceinline__ T tf_from_ff(ff x);
template <> __device__ __forceinline__ float tf_from_ff<float>(ff x) { return __fadd_rn(x.hi, x.lo); }
template <> __device__ __forceinline__ ff tf_from_ff<ff>(ff x) { return x; }
__device__ __forceinline__ ff ff_twice(ff x) { return ff(2.0f * x.hi, 2.0f * x.lo); }

// log(1 + z) - z for |z| <= 1e-3: z^2 (-1/2 + z/3 + tail) with z^2, z/3 and the sum in
// float-float and the tail -z^2/4 + z^3/5 - z^4/6 + z^5/7 (below 5e-7 of the 1/2) in
// FP32, so the result carries ~2^-47 relative error; larger |z| through FP64.
// the rare wide-argument branch out of line: the float-float solve and stage preparation
// inline ff_log1pmx at every call site, and an inlined FP64 fallback at each of them
// costs instruction-cache space in the hot loops
static __device__ __noinline__ ff ff_log1pmx_wide(ff z) { return ff(log1pmx(double(z))); }
__device__ __forceinline__ ff ff_log1pmx(ff z) {
  if (fabsf(z.hi) <= 1e-3f) {
    const float t = z.hi;
    float tail = __fmaf_rn(t, 1.0f / 7.0f, -1.0f / 6.0f);
    tail = __fmaf_rn(tail, t, 0.2f);
    tail = __fmaf_rn(tail, t, -0.25f);
    tail = __fmul_rn(tail, __fmul_rn(t, t));
    constexpr float th = float(1.0 / 3.0);
    constexpr float tl = float(1.0 / 3.0 - double(th));
    const float pz = __fmul_rn(z.hi, th);
    float ez = __fmaf_rn(z.hi, th, -pz);
    ez = __fmaf_rn(z.hi, tl, ez);
    ez = __fmaf_rn(z.lo, th, ez);
    const ff s = fast_two_sum(-0.5f, pz);
    const ff poly = fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(ez, tail)));
    return (z * z) * poly;
  }
  return ff_log1pmx_wide(z);
}

// 1/sqrt(x): the FP32 approximation r (rsqrt.approx.ftz.f32, ~2^-23) refined with the
// residual t = 1 - x r^2 formed in float-float (r^2 exact by TwoProd) by the
// second-order step r (1 + t/2 + 3 t^2/8).
__device__ __forceinline__ ff ff_rsqrt(ff x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.hi));
  const float r2 = __fmul_rn(r, r);
  const float r2l = __fmaf_rn(r, r, -r2);
  const float pp = __fmul_rn(x.hi, r2);
  float e = __fmaf_rn(x.hi, r2, -pp);
  e = __fmaf_rn(x.hi, r2l, e);
  e = __fmaf_rn(x.lo, r2, e);
  const float t = __fsub_rn(__fsub_rn(1.0f, pp), e);
  const float c = __fmul_rn(__fmul_rn(r, t), __fmaf_rn(0.375f, t, 0.5f));
  return fast_two_sum(r, c);
}

// w(u + e) - w(u) in float-float (same formulas as entropy_var_increment)
__device__ __forceinline__ void entropy_var_increment_ff(const ff u[5], const ff e[5], const FluxConst<ff>& C,
                                                         ff dw[5]) {
  const ff one(1.0f, 0.0f);
  const ff rho = u[0];
  const ff rho1 = rho + e[0];
  const ff m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const ff Pr = C.gm1 * (rho * u[4] - ff_half(m2));
  const ff rr1 = rho * rho1;
  const ff inv = ff_rcp(rr1 * Pr);
  const ff pinv = Pr * inv;
  const ff ir = rho1 * pinv, ir1 = rho * pinv, ip = rho * rr1 * inv;
  const ff v0 = u[1] * ir, v1 = u[2] * ir, v2 = u[3] * ir;
  const ff v2s = m2 * ir * ir;
  const ff x = e[0] * ir;
  const ff d0 = (e[1] - v0 * e[0]) * ir1, d1 = (e[2] - v1 * e[0]) * ir1, d2 = (e[3] - v2 * e[0]) * ir1;
  const ff dv2 = d0 * d0 + d1 * d1 + d2 * d2;
  const ff y = C.gm1 * (e[4] - (v0 * e[1] + v1 * e[2] + v2 * e[3]) + ff_half(v2s * e[0]) - ff_half(rho1 * dv2)) * ip;
  const ff biy = (rho * ip) * ff_rcp(one + y);  // beta / (1 + y)
  const ff ds = (y + ff_log1pmx(y)) - C.gam * (x + ff_log1pmx(x));
  const ff xy = x - y;
  const ff opx = one + x;
  const ff dkin = ff_half(biy * (xy * v2s + opx * (ff_twice(v0 * d0 + v1 * d1 + v2 * d2) + dv2)));
  dw[0] = -(ds * C.inv_gm1) - dkin;
  dw[1] = biy * (xy * v0 + opx * d0);
  dw[2] = biy * (xy * v1 + opx * d1);
  dw[3] = biy * (xy * v2 + opx * d2);
  dw[4] = -(biy * xy);
}

// Lanes per element in the relaxation kernels: a group of SUB lanes solves one element,
// so for small Np two or four elements share a warp and the per-element scalar work
// (reductions, bracket and Newton logic, executed by every lane of the group) is paid
// once per 16 or 8 lanes instead of once per warp.  The FP64 solve keeps 16-lane groups
// up to p = 4 (8 nodes per lane there; 4 % faster than whole warps).  The float-float
// solve (FF) holds twice the registers per node value and is latency-bound: it takes
// whole warps from Np > 32 on (measured: 1 % faster for p = 3, where the FP64 solve is
// 1 % slower).
template <int P1, bool FF = false>
struct RelaxGroup {
  static constexpr int Np = P1 * P1 * P1;
  static constexpr int SUB = Np <= 32 ? 8 : ((Np <= 128 && !FF) ? 16 : 32);
  static constexpr int R = (Np + SUB - 1) / SUB;  // nodes per lane
  static constexpr int EPW = 32 / SUB;            // elements per warp
  static __device__ __forceinline__ unsigned mask(int lane) {
    return SUB == 32 ? 0xffffffffu : (((1u << SUB) - 1u) << (lane / SUB * SUB));
  }
};
template <int SUB>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = SUB / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}
template <int SUB>
__device__ __forceinline__ float group_sum_f(float v, unsigned mask) {
#pragma unroll
  for (int o = SUB / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Relaxation node data in float-float (mixed and ES_FP64X modes): the same quantities
// as RelaxNode, formed and evaluated on the FP32 pipe; the element sums, the bracket
// and the Newton/bisection steps stay in FP64.
struct RelaxNodeF {
  ff X0, Y0, V2, c;
};

__device__ __forceinline__ void relax_node_setup_ff(const ff u[5], const ff d[5], const FluxConst<ff>& C, ff c,
                                                    RelaxNodeF& nd) {
  const ff rho = u[0];
  const ff m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
  const ff Pr = C.gm1 * (rho * u[4] - ff_half(m2));
  const ff inv = ff_rcp(rho * Pr);
  const ff ir = Pr * inv, ip = rho * rho * inv;
  const ff v0 = u[1] * ir, v1 = u[2] * ir, v2 = u[3] * ir;
  const ff v2s = v0 * v0 + v1 * v1 + v2 * v2;
  const ff dv0 = (d[1] - v0 * d[0]) * ir, dv1 = (d[2] - v1 * d[0]) * ir, dv2 = (d[3] - v2 * d[0]) * ir;
  nd.X0 = d[0] * ir;
  nd.Y0 = C.gm1 * (d[4] - (v0 * d[1] + v1 * d[2] + v2 * d[3]) + ff_half(v2s * d[0])) * ip;
  nd.V2 = rho * (dv0 * dv0 + dv1 * dv1 + dv2 * dv2) * ip;
  nd.c = c;
}

// g^3 coefficient of D_n(g)/rho_n: with y2 = -(gam-1) V2/2 and L2 = y2 - Y0^2/2 (the g^2
// coefficient of log1p(y)),
//   D_3 = [-gam X0^3/6 + (2 Y0 L2 + y2 Y0)/3 - X0 L2]/(gam-1) - X0 V2/2;
// the g^2 coefficient is D_2 = [(gam-1) X0^2 + (X0 - Y0)^2]/(2 (gam-1)) + V2/2.
// Taken in FP32 by both relaxation solves: it only sets the starting point, whose last
// bits still decide where Newton's iterates stop, so every operation is an explicit
// round-to-nearest one (the compiler may then not fuse them differently from one build
// or register budget to the next)
__device__ __forceinline__ float relax_node_cubic_f(const RelaxNodeF& nd, float gam) {
  const float X = nd.X0.hi, Y = nd.Y0.hi, V = nd.V2.hi;
  const float gm1 = __fsub_rn(gam, 1.0f);
  const float y2 = __fmul_rn(__fmul_rn(-0.5f, gm1), V);
  const float L2 = __fmaf_rn(-0.5f * Y, Y, y2);
  const float s1 = __fmaf_rn(2.0f * Y, L2, __fmul_rn(y2, Y));
  const float x3 = __fmul_rn(__fmul_rn(X, X), X);
  float t = __fmul_rn(s1, 1.0f / 3.0f);
  t = __fmaf_rn(__fmul_rn(gam, -1.0f / 6.0f), x3, t);
  t = __fmaf_rn(-X, L2, t);
  return __fmaf_rn(-0.5f * X, V, __fdiv_rn(t, gm1));
}

// relax_node_eval in float-float (same formulas); false where the state at g is not physical
__device__ __forceinline__ bool relax_node_eval_ff(const RelaxNodeF& nd, ff g, const FluxConst<ff>& C, ff& D,
                                                   ff& dD) {
  const ff one(1.0f, 0.0f);
  const ff x = g * nd.X0;
  const ff opx = one + x;
  const ff K0 = ff_half(g * g * nd.V2);
  const ff Yb = g * nd.Y0 * opx - C.gm1 * K0;
  const ff opy_n = opx + Yb;  // (1+y)(1+x)
  if (!(opx.hi > 0.0f) || !(opy_n.hi > 0.0f)) return false;
  const ff inv = ff_rcp(opx * opy_n);
  const ff q = opy_n * inv;       // 1/(1+x)
  const ff iy = opx * opx * inv;  // 1/(1+y)
  const ff y = Yb * q;
  const ff K = K0 * q;
  const ff Lx = ff_log1pmx(x), Ly = ff_log1pmx(y);
  const ff l1px = x + Lx, l1py = y + Ly;
  const ff phi = opx * Lx + x * x;
  D = (C.gam * phi - Ly - x * l1py) * C.inv_gm1 + K;
  const ff dK = g * nd.V2 * q * (one - ff_half(x * q));
  const ff dy = nd.Y0 - C.gm1 * dK;
  dD = (nd.X0 * (C.gam * l1px - l1py) + dy * (y - x) * iy) * C.inv_gm1 + dK;
  return true;
}

// ---------------------------------------------------------------------------
// the parameter vector z = (z1, z1 v, z5, 1/z1) of a float-float state y, with
// z1 = sqrt(rho/p) = rho / sqrt(rho p), z5 = sqrt(rho p); false if rho or p <= 0
__device__ __forceinline__ bool param_vector_ff(const ff y[5], const FluxConst<ff>& C, ff z[6]) {
  const ff rho = y[0];
  const ff ir = ff_rcp(rho);
  const ff v0 = y[1] * ir, v1 = y[2] * ir, v2 = y[3] * ir;
  const ff p = C.gm1 * (y[4] - ff_half(y[1] * v0 + y[2] * v1 + y[3] * v2));
  const bool ok = rho.hi > 0.0f && p.hi > 0.0f;
  const ff rs = ff_rsqrt(rho * p);
  const ff z1 = rho * rs;
  z[0] = z1;
  z[1] = z1 * v0;
  z[2] = z1 * v1;
  z[3] = z1 * v2;
  z[4] = rho * p * rs;
  z[5] = p * rs;
  return ok;
}

// FP64 value of a flux-precision value (float: the bits placed on the integer pipe)
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64_bits(x); }
__device__ __forceinline__ double to_f64(ff x) { return double(x); }

// ---------------------------------------------------------------------------
// The stage state at one node in the flux precision TF (k_prep's per-node work).
//
// FP64 estimates with FP32 fluxes (ES_MIXED): the stage increment e = dt sum_j a_ij k_j
// in FP64 (the FP32 k_j placed into FP64 on the integer pipe), y = u + e, and the
// parameter vector formed from y in float-float and rounded once.
template <typename TF, int NPREV>
__device__ __forceinline__ void stage_increment_f64(const Params& P, const StagePrep& sp, long long N, long long g,
                                                    int inst, double e[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) e[v] = 0.0;
  if constexpr (NPREV != 0) {
    const double dt = geom_of(P, inst).dt;
#pragma unroll
    for (int j = 0; j < (NPREV >= 0 ? NPREV : sp.nprev); ++j) {
      const double c = sp.coef[j] * dt;
      const TF* kj = static_cast<const TF*>(sp.k[j]);
#pragma unroll
      for (int v = 0; v < 5; ++v) e[v] = fma(c, to_f64(kj[v * N + g]), e[v]);
    }
  }
}
template <typename TF>
__device__ __forceinline__ bool stage_z_f64(const Params& P, const double u[5], const double e[5], TF z[6]) {
  // y = u + e formed in float-float on the FP32 pipe (the FP64 pipe bounds this kernel):
  // the parameter vector is rounded to FP32 in the end either way
  ff yf[5], zf[6];
#pragma unroll
  for (int v = 0; v < 5; ++v) yf[v] = ff_from_double(u[v]) + ff_from_double(e[v]);
  const bool ok = param_vector_ff(yf, P.Cff, zf);
#pragma unroll
  for (int c = 0; c < 6; ++c) z[c] = tf_from_ff<TF>(zf[c]);
  return ok;
}

// Float-float estimates (ES_MIXED_FF, ES_FP64X): u split into float-float (integer
// pipe), e and y = u + e and the parameter vector in float-float.
template <typename TF, int NPREV>
__device__ __forceinline__ void stage_increment_ff(const Params& P, const StagePrep& sp, long long N, long long g,
                                                   int inst, const double u[5], ff uf[5], ff ef[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    uf[v] = ff_from_double(u[v]);
    ef[v] = ff(0.0f, 0.0f);
  }
  if constexpr (NPREV != 0) {
    const double dt = geom_of(P, inst).dt;
#pragma unroll
    for (int j = 0; j < (NPREV >= 0 ? NPREV : sp.nprev); ++j) {
      const ff c = ff_from_double(sp.coef[j] * dt);
      const TF* kj = static_cast<const TF*>(sp.k[j]);
#pragma unroll
      for (int v = 0; v < 5; ++v) ff_fma_acc(ef[v], c, to_ff(kj[v * N + g]));
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) ef[v] = ff_norm(ef[v]);
  }
}
template <typename TF, int NPREV>
__device__ __forceinline__ bool stage_z_ff(const Params& P, const ff uf[5], const ff ef[5], TF z[6]) {
  ff yf[5], zf[6];
#pragma unroll
  for (int v = 0; v < 5; ++v) yf[v] = NPREV != 0 ? uf[v] + ef[v] : uf[v];
  const bool ok = param_vector_ff(yf, P.Cff, zf);
#pragma unroll
  for (int c = 0; c < 6; ++c) z[c] = tf_from_ff<TF>(zf[c]);
  return ok;
}

// ---------------------------------------------------------------------------
// y = u (+ gamma d when the instance has a pending relaxed update and this is the
// step's first stage) + dt sum_j a_ij k_j over the stages with a_ij != 0.
// FP64 mode: everything in FP64.  Mixed mode with FP64 estimates (P.ff_est = 0):
// stage_increment_f64 / stage_z_f64 and w(y) - w(u) in FP64.  ES_FP64X and the mixed
// float-float mode: stage_increment_ff / stage_z_ff and w(y) - w(u) in float-float.
// FP64 selects the FP64-increment paths at compile time (they differ widely in
// register use).  NPREV >= 0 fixes the number of earlier stages at compile time;
// NPREV < 0 reads it from sp.nprev (tableaux with more than three nonzero a_ij in a row).
template <typename TF, int NPREV, bool FP64>
__global__ void k_prep(Params P, StagePrep sp, TF* __restrict__ aux, int* __restrict__ status) {
  const long long N = (long long)P.K * sp.Np;
  const double gam = P.gam;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int inst = inst_of(P, int(g / sp.Np));
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = sp.q[v * N + g];
    if (sp.pending && sp.pending[inst]) {
      const double gmm = sp.gamma_cur[inst];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        u[v] = u[v] + gmm * sp.d[v * N + g];
        sp.q[v * N + g] = u[v];
      }
    }
    if constexpr (FP64 && !std::is_same<TF, double>::value) {
      double e[5];
      stage_increment_f64<TF, NPREV>(P, sp, N, g, inst, e);
      TF z[6];
      if (!stage_z_f64<TF>(P, u, e, z)) atomicOr(status, kStatusNonphysical);
#pragma unroll
      for (int c = 0; c < 6; ++c) aux[c * N + g] = z[c];
      if (sp.dw) {
        double dw[5];
        entropy_var_increment(u, e, gam, P.Cd.inv_gm1, dw);
#pragma unroll
        for (int v = 0; v < 5; ++v) sp.dw[v * N + g] = dw[v];
      }
    } else if constexpr (FP64) {
      double y[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) y[v] = u[v];
      if constexpr (NPREV != 0) {
        const double dt = geom_of(P, inst).dt;
#pragma unroll
        for (int j = 0; j < (NPREV >= 0 ? NPREV : sp.nprev); ++j) {
          const double c = sp.coef[j] * dt;
          const double* kj = static_cast<const double*>(sp.k[j]);
#pragma unroll
          for (int v = 0; v < 5; ++v) y[v] = fma(c, kj[v * N + g], y[v]);
        }
      }
      const double rho = y[0];
      const double ir = fast_rcp(rho);
      const double v0 = y[1] * ir, v1 = y[2] * ir, v2 = y[3] * ir;
      const double p = (gam - 1.0) * (y[4] - 0.5 * rho * (v0 * v0 + v1 * v1 + v2 * v2));
      if (!(rho > 0.0) || !(p > 0.0)) atomicOr(status, kStatusNonphysical);
      // z1 = sqrt(rho/p) = rho / sqrt(rho p), z5 = sqrt(rho p)
      const double rs = rsqrt(rho * p);
      const double z1 = rho * rs;
      aux[0 * N + g] = z1;
      aux[1 * N + g] = z1 * v0;
      aux[2 * N + g] = z1 * v1;
      aux[3 * N + g] = z1 * v2;
      aux[4 * N + g] = rho * p * rs;
      aux[5 * N + g] = p * rs;  // 1/z1 = sqrt(p/rho)
      if (sp.dw) {
        double e[5], dw[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) e[v] = y[v] - u[v];
        entropy_var_increment(u, e, gam, P.Cd.inv_gm1, dw);
#pragma unroll
        for (int v = 0; v < 5; ++v) sp.dw[v * N + g] = dw[v];
      }
    } else {
      ff uf[5], ef[5];
      stage_increment_ff<TF, NPREV>(P, sp, N, g, inst, u, uf, ef);
      TF z[6];
      if (!stage_z_ff<TF, NPREV>(P, uf, ef, z)) atomicOr(status, kStatusNonphysical);
#pragma unroll
      for (int c = 0; c < 6; ++c) aux[c * N + g] = z[c];
      if (sp.dw) {
        ff dw[5];
        entropy_var_increment_ff(uf, ef, P.Cff, dw);
#pragma unroll
        for (int v = 0; v < 5; ++v) reinterpret_cast<ff*>(sp.dw)[v * N + g] = dw[v];
      }
    }
  }
}

// ---------------------------------------------------------------------------
template <int P1, typename TF>
__device__ __forceinline__ Zstate<TF> load_z(const TF* __restrict__ aux, long long N, long long g) {
  Zstate<TF> s;
#pragma unroll
  for (int c = 0; c < kAux; ++c) s.z[c] = aux[c * N + g];
  return s;
}

// Matrix interface dissipation in entropy variables (interface_diss = 2):
// f -= (1/2) R |Lambda| T R^T [[w]] along x_m with the eigenvectors
//   r1 = (1, u - a e_m, h - u_m a), r2 = (1, u, |u|^2/2), r3, r4 = (0, e_t, u_t) for
//   the two tangential directions t, r5 = (1, u + a e_m, h + u_m a),
// eigenvalues u_m - a, u_m (three times), u_m + a, and Barth's scaling
// T = diag(rho/(2 gam), rho (gam-1)/gam, p, p, rho/(2 gam)) (R T R^T = dq/dw), all at
// the mean state rho = zb1 zb5, u = zb_v/zb1, p = zb5/zb1 (a = sqrt(gam)/zb1,
// h = a^2/(gam-1) + |u|^2/2) of the parameter-vector averages zb.  The entropy-variable
// jump from the parameter vectors: [[w_v]] = [[z1 z_v]], [[w5]] = -[[z1^2]],
// [[w1]] = -[[s]]/(gam-1) - [[|z_v|^2]]/2, [[s]] = -(gam+1) ln(z1R/z1L) - (gam-1) ln(z5R/z5L).
template <typename TF>
__device__ __forceinline__ TF tf_log(TF x) { return log(x); }
template <>
__device__ __forceinline__ float tf_log<float>(float x) { return logf(x); }

template <typename TF>
__device__ __forceinline__ void matrix_dissipation(const Zstate<TF>& L, const Zstate<TF>& R, int m,
                                                   const FluxConst<TF>& C, TF f[5]) {
  TF zb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) zb[c] = TF(0.5) * (L.z[c] + R.z[c]);
  const TF iz1 = fast_rcp(zb[0]);
  const TF rho = zb[0] * zb[4];
  const TF p = zb[4] * iz1;
  const TF u[3] = {zb[1] * iz1, zb[2] * iz1, zb[3] * iz1};
  const TF a = C.sqrt_gam * iz1;
  const TF u2h = TF(0.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const TF h = a * a * C.inv_gm1 + u2h;
  const TF un = m == 0 ? u[0] : (m == 1 ? u[1] : u[2]);  // constant indices: u stays in registers
  const int t1 = m == 0 ? 1 : 0, t2 = m == 2 ? 1 : 2;
  // entropy-variable jump
  const TF ds = -(C.gam + TF(1)) * tf_log(R.z[0] * fast_rcp(L.z[0])) - C.gm1 * tf_log(R.z[4] * fast_rcp(L.z[4]));
  TF jw[5];
  jw[0] = -(ds * C.inv_gm1) -
          TF(0.5) * ((R.z[1] * R.z[1] + R.z[2] * R.z[2] + R.z[3] * R.z[3]) -
                     (L.z[1] * L.z[1] + L.z[2] * L.z[2] + L.z[3] * L.z[3]));
#pragma unroll
  for (int k = 0; k < 3; ++k) jw[1 + k] = R.z[0] * R.z[1 + k] - L.z[0] * L.z[1 + k];
  jw[4] = -(R.z[0] * R.z[0] - L.z[0] * L.z[0]);
  // characteristic amplitudes R^T [[w]], scaled by |lambda| T
  const TF jwm = m == 0 ? jw[1] : (m == 1 ? jw[2] : jw[3]);
  const TF jwt1 = t1 == 0 ? jw[1] : (t1 == 1 ? jw[2] : jw[3]);
  const TF jwt2 = t2 == 1 ? jw[2] : jw[3];
  const TF ut1 = t1 == 0 ? u[0] : (t1 == 1 ? u[1] : u[2]);
  const TF ut2 = t2 == 1 ? u[1] : u[2];
  const TF base = jw[0] + (u[0] * jw[1] + u[1] * jw[2] + u[2] * jw[3]);
  const TF s_ac = rho * TF(0.5) * fast_rcp(C.gam);
  TF a1 = (base - a * jwm + (h - un * a) * jw[4]) * (fabs(un - a) * s_ac);
  TF a2 = (base + u2h * jw[4]) * (fabs(un) * rho * C.gm1 * fast_rcp(C.gam));
  TF a3 = (jwt1 + ut1 * jw[4]) * (fabs(un) * p);
  TF a4 = (jwt2 + ut2 * jw[4]) * (fabs(un) * p);
  TF a5 = (base + a * jwm + (h + un * a) * jw[4]) * (fabs(un + a) * s_ac);
  // D = sum_k a_k r_k
  TF D[5];
  D[0] = a1 + a2 + a5;
#pragma unroll
  for (int k = 0; k < 3; ++k) D[1 + k] = (a1 + a2 + a5) * u[k];
  // the +-a e_m parts and the tangential vectors
  if (m == 0) D[1] += a * (a5 - a1);
  else if (m == 1) D[2] += a * (a5 - a1);
  else D[3] += a * (a5 - a1);
  if (t1 == 0) D[1] += a3;
  else D[2] += a3;
  if (t2 == 1) D[2] += a4;
  else D[3] += a4;
  D[4] = (a1 + a5) * h + un * a * (a5 - a1) + a2 * u2h + a3 * ut1 + a4 * ut2;
#pragma unroll
  for (int v = 0; v < 5; ++v) f[v] -= TF(0.5) * D[v];
}

// interface flux f_num(L, R) of the EC flux with optional Rusanov dissipation
template <typename TF>
__device__ __forceinline__ void face_flux(const Zstate<TF>& L, TF izL, const Zstate<TF>& R, TF izR, int m,
                                          const FluxConst<TF>& C, int diss, TF f[5]) {
  ec_flux(L, R, m, C, f);
  if (diss == 2) {
    matrix_dissipation(L, R, m, C, f);
  } else if (diss) {
    TF qL[5], qR[5], lL, lR;
    z_to_q(L, izL, C, qL, lL, m);
    z_to_q(R, izR, C, qR, lR, m);
    const TF lam = TF(0.5) * fmax(lL, lR);
#pragma unroll
    for (int v = 0; v < 5; ++v) f[v] -= lam * (qR[v] - qL[v]);
  }
}

// diss^V (interior penalty on the entropy-variable jump): C_mm(s) g for one side's
// state, accumulated into c.  C_mm is the block of the viscous flux F^V_m that
// multiplies dw/dx_m; with RT = p/rho = 1/z1^2, v = z_{2..4}/z1 and the velocity part
// b = g_{2..4} + v g_5 of the jump g (w_1 does not enter):
// C_mm g = (0, mu RT (b + e_m b_m/3), v . [mu RT (b + e_m b_m/3)] + kappa (RT)^2/R g_5).
template <typename TF>
__device__ __forceinline__ void visc_jump_flux(const Zstate<TF>& s, TF iz, const TF g[4], int m, TF mu, TF kap,
                                               TF iR, TF c[5]) {
  const TF v0 = s.z[1] * iz, v1 = s.z[2] * iz, v2 = s.z[3] * iz;
  const TF RT = iz * iz;
  const TF mrt = mu * RT;
  TF t0 = mrt * (g[0] + v0 * g[3]);
  TF t1 = mrt * (g[1] + v1 * g[3]);
  TF t2 = mrt * (g[2] + v2 * g[3]);
  if (m == 0) t0 += TF(1.0 / 3.0) * t0;
  else if (m == 1) t1 += TF(1.0 / 3.0) * t1;
  else t2 += TF(1.0 / 3.0) * t2;
  c[1] += t0;
  c[2] += t1;
  c[3] += t2;
  c[4] += t0 * v0 + t1 * v1 + t2 * v2 + kap * RT * RT * iR * g[3];
}

// adds sig (C_mm(L) + C_mm(R))/2 (w_L - w_R) to the interface flux f (w_{2..5} = z1 z_{2..4}, -z1^2)
template <typename TF>
__device__ __forceinline__ void visc_penalty(const Zstate<TF>& L, TF izL, const Zstate<TF>& R, TF izR, int m,
                                             TF sig, const Params& P, TF f[5]) {
  TF g[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) g[k] = L.z[0] * L.z[1 + k] - R.z[0] * R.z[1 + k];
  g[3] = R.z[0] * R.z[0] - L.z[0] * L.z[0];
  const TF mu = TF(P.mu), kap = TF(P.kappa_heat), iR = TF(P.inv_R);
  TF c[5] = {TF(0), TF(0), TF(0), TF(0), TF(0)};
  visc_jump_flux(L, izL, g, m, mu, kap, iR, c);
  visc_jump_flux(R, izR, g, m, mu, kap, iR, c);
  const TF hs = TF(0.5) * sig;
#pragma unroll
  for (int v = 1; v < 5; ++v) f[v] += hs * c[v];
}

// a prescribed boundary state's parameter vector and 1/z1 in the flux precision
template <typename TF>
__device__ __forceinline__ Zstate<TF> bc_z(const double* v, TF& iz) {
  Zstate<TF> z;
#pragma unroll
  for (int c = 0; c < 5; ++c) z.z[c] = tf_from_double<TF>(v[c]);
  iz = tf_from_double<TF>(v[5]);
  return z;
}

// VPEN: with the diss^V penalty (a separate instantiation keeps the common path's
// register count)
template <int P1, typename TF, bool VPEN>
__global__ void k_face(Params P, const TF* __restrict__ aux, TF* __restrict__ F, TF* __restrict__ FL) {
  constexpr int P2 = P1 * P1, Np = P1 * P2;
  const long long N = (long long)P.K * Np;
  const long long total = 3LL * P.K * P2;
  const FluxConst<TF> C = flux_const<TF>(P);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = int(idx / ((long long)P.K * P2));
    const long long rem = idx - (long long)m * P.K * P2;
    const int e = int(rem / P2), ab = int(rem % P2);
    const int a = ab % P1, b = ab / P1;
    const long long gL = (long long)e * Np + line_node<P1>(m, a, b, P1 - 1);
    const Zstate<TF> L = load_z<P1, TF>(aux, N, gL);
    const TF izL = aux[5 * N + gL];
    Zstate<TF> R;
    TF izR;
    if (at_boundary(P, e, m, 1)) {  // +x_m boundary: prescribed exterior state
      R = bc_z<TF>(bc_values(P, m, 1), izR);
    } else {
      const long long gR = (long long)neighbour(P, e, m, +1) * Np + line_node<P1>(m, a, b, 0);
      R = load_z<P1, TF>(aux, N, gR);
      izR = aux[5 * N + gR];
    }
    TF f[5];
    face_flux(L, izL, R, izR, m, C, P.diss, f);
    // diss^V penalty scale alpha (2/h_m)(1/omega_0)
    TF sig = TF(0);
    if constexpr (VPEN) {
      sig = TF(P.visc_pen * geom_of(P, inst_of(P, e)).metric[m] * P.inv_omega_end);
      visc_penalty(L, izL, R, izR, m, sig, P, f);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) F[((long long)(m * 5 + v) * P.K + e) * P2 + ab] = f[v];
    if (at_boundary(P, e, m, 0)) {  // -x_m boundary face of this element, into FL
      TF izB;
      const Zstate<TF> B = bc_z<TF>(bc_values(P, m, 0), izB);
      const long long g0 = (long long)e * Np + line_node<P1>(m, a, b, 0);
      const Zstate<TF> I = load_z<P1, TF>(aux, N, g0);
      const TF izI = aux[5 * N + g0];
      face_flux(B, izB, I, izI, m, C, P.diss, f);
      if constexpr (VPEN) visc_penalty(B, izB, I, izI, m, sig, P, f);
#pragma unroll
      for (int v = 0; v < 5; ++v) FL[((long long)(m * 5 + v) * P.K + e) * P2 + ab] = f[v];
    }
  }
}

// ---------------------------------------------------------------------------
// BR1 gradients and viscous flux per node.  fV[(m*4 + c) N + g], c = momentum
// x, y, z, energy.  theta_m = (2/h_m) [D w + (1/omega) (w_face_avg - w) n_m] for
// w_2..w_5 (the viscous flux needs no other component).  A CTA stages the
// entropy variables of its EPB elements in shared memory once; neighbours'
// face values come from global memory.
template <int P1, typename TF, int EPB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_grad(Params P, const TF* __restrict__ aux, TF* __restrict__ fV) {
  constexpr int P2 = P1 * P1, Np = P1 * P2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TF* ws = reinterpret_cast<TF*>(smem_raw);  // [4][EPB*Np]
  const long long N = (long long)P.K * Np;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, P.K - e0);
  const int nn = nel * Np;
  const TF mu = TF(P.mu), kap = TF(P.kappa_heat), iR = TF(P.inv_R);
  const TF iw = TF(P.inv_omega_end);
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const long long g = (long long)e0 * Np + t;
    const TF z1 = aux[g];
    ws[0 * EPB * Np + t] = z1 * aux[N + g];
    ws[1 * EPB * Np + t] = z1 * aux[2 * N + g];
    ws[2 * EPB * Np + t] = z1 * aux[3 * N + g];
    ws[3 * EPB * Np + t] = -z1 * z1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const int el = t / Np, n = t % Np;
    const int e = e0 + el;
    const long long g = (long long)e0 * Np + t;
    const InstGeom& G = geom_of(P, inst_of(P, e));
    const int ii[3] = {n % P1, (n / P1) % P1, n / P2};
    TF th[3][4];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int im = ii[m];
      const int a = m == 0 ? ii[1] : ii[0];
      const int b = m == 2 ? ii[1] : ii[2];
      TF acc[4] = {TF(0), TF(0), TF(0), TF(0)};
#pragma unroll
      for (int j = 0; j < P1; ++j) {
        const int nj = el * Np + line_node<P1>(m, a, b, j);
        const TF Dij = Tab<TF>::D(P, im * P1 + j);
#pragma unroll
        for (int c = 0; c < 4; ++c) fma_acc(acc[c], Dij, ws[c * EPB * Np + nj]);
      }
      if (im == P1 - 1 || im == 0) {
        const bool right = (im == P1 - 1);
        TF wn[4];
        if (at_boundary(P, e, m, right ? 1 : 0)) {  // prescribed exterior w2..w5
          const double* bv = bc_values(P, m, right ? 1 : 0);
#pragma unroll
          for (int c = 0; c < 4; ++c) wn[c] = tf_from_double<TF>(bv[6 + c]);
        } else {
          const int en = neighbour(P, e, m, right ? +1 : -1);
          const long long gn = (long long)en * Np + line_node<P1>(m, a, b, right ? 0 : P1 - 1);
          const TF zn1 = aux[gn];
          wn[0] = zn1 * aux[N + gn];
          wn[1] = zn1 * aux[2 * N + gn];
          wn[2] = zn1 * aux[3 * N + gn];
          wn[3] = -zn1 * zn1;
        }
        const TF sg = right ? TF(0.5) * iw : TF(-0.5) * iw;
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += sg * (wn[c] - ws[c * EPB * Np + t]);
      }
      const TF met = TF(G.metric[m]);
#pragma unroll
      for (int c = 0; c < 4; ++c) th[m][c] = met * acc[c];
    }
    // chain rule: v = -w_{2..4}/w_5 = z_{2..4}/z1, T = -1/(R w_5).  With a = -1/w_5 = 1/z1^2
    // and b_mk = theta_m,k + v_k theta_m,5: dv_k/dx_m = a b_mk, dT/dx_m = a^2/R theta_m,5;
    // tau is symmetric: off-diagonal mu a (b_mk + b_km), diagonal 2 mu a b_mm - (2/3) mu a sum b_jj
    const TF iz1 = aux[5 * N + g];
    const TF v[3] = {aux[N + g] * iz1, aux[2 * N + g] * iz1, aux[3 * N + g] * iz1};
    const TF a = iz1 * iz1;
    TF b[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int k = 0; k < 3; ++k) b[m][k] = th[m][k] + v[k] * th[m][3];
    const TF ma = mu * a;
    const TF dsum = (ma * TF(-2.0 / 3.0)) * (b[0][0] + b[1][1] + b[2][2]);
    const TF c1 = ma + ma;
    TF tau[3][3];
    tau[0][1] = tau[1][0] = ma * (b[0][1] + b[1][0]);
    tau[0][2] = tau[2][0] = ma * (b[0][2] + b[2][0]);
    tau[1][2] = tau[2][1] = ma * (b[1][2] + b[2][1]);
#pragma unroll
    for (int m = 0; m < 3; ++m) tau[m][m] = c1 * b[m][m] + dsum;
    const TF kt = kap * a * a * iR;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      TF fe = kt * th[m][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        fV[(long long)(m * 4 + k) * N + g] = tau[m][k];
        fe += tau[m][k] * v[k];
      }
      fV[(long long)(m * 4 + 3) * N + g] = fe;
    }
  }
}

// ---------------------------------------------------------------------------
// Shared memory of k_volume: the FP64 reduction rows of the node phase (first, so they
// stay 8-byte aligned), with FACES the neighbours' face-node parameter vectors in the
// same space (they are dead once the flux phase ends), then the element tile's
// parameter vector (kAux planes; with FACES also 1/z1) and the accumulator.
template <int P1, int EPB, bool FACES>
struct VolSmem {
  static constexpr int P2 = P1 * P1, Np = P1 * P2;
  static constexpr int ZP = FACES ? kAuxPlanes : kAux;
  static constexpr size_t red = size_t(2) * EPB * Np * sizeof(double);
  static constexpr size_t halo_floats = FACES ? size_t(6) * kAuxPlanes * EPB * P2 : 0;
  template <typename TF>
  static constexpr size_t head() {
    return red > halo_floats * sizeof(TF) ? red : ((halo_floats * sizeof(TF) + 15) / 16) * 16;
  }
  template <typename TF>
  static constexpr size_t bytes() {
    return head<TF>() + size_t(EPB) * Np * (ZP + 5) * sizeof(TF);
  }
};

// Flux differencing, interface terms and viscous divergence of EPB elements per CTA,
// one LGL line per thread and direction, then the node phase (k_i or d, element sums).
// FACES (FP32 fluxes on periodic Euler groups): the interface flux at both ends of each
// line is evaluated here from the neighbours' face-node parameter vectors, with
// k_face's arguments (the same bits on both elements of a face), instead of being read
// from F: one launch less per stage and no face-flux round trip through global memory.
// Register budget of the FP32 flux-differencing kernel, which waits on latency, not on its
// FP32 pipe (measured on GB300, volume time per step, best tile): the Navier--Stokes form at
// p = 4 runs 11-13 % faster at 85 registers than at its unbounded 106-121 (more warps per
// SM), the Euler form at p = 5 7 % faster at 64; at p = 2, 3 a bound gives nothing or less.
template <int P1, typename TF, bool NS>
struct VolRegs {
  static constexpr int cap = std::is_same<TF, float>::value ? (NS ? 80 : (P1 == 6 ? 64 : 0)) : 0;
};
template <int P1, typename TF, bool NS, int THREADS>
constexpr int vol_min_blocks() {
  return VolRegs<P1, TF, NS>::cap ? 65536 / (THREADS * VolRegs<P1, TF, NS>::cap) : 1;
}

template <int P1, typename TF, bool NS, int EPB, int THREADS, bool FACES>
__device__ __forceinline__ void volume_body(const Params& P, const StageVol& sv, const TF* __restrict__ aux,
                                            const TF* __restrict__ F, const TF* __restrict__ FL,
                                            const TF* __restrict__ fV) {
  using S = VolSmem<P1, EPB, FACES>;
  constexpr int P2 = P1 * P1, Np = P1 * P2;
  constexpr int ZP = S::ZP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* red = reinterpret_cast<double*>(smem_raw);               // [2][EPB*Np]
  TF* halo = reinterpret_cast<TF*>(smem_raw);                      // FACES: [dir, side][plane][EPB*P2]
  TF* za = reinterpret_cast<TF*>(smem_raw + S::template head<TF>());  // [ZP][EPB*Np]
  TF* acc = za + ZP * EPB * Np;                                    // [5][EPB*Np]
  const long long N = (long long)P.K * Np;
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, P.K - e0);
  const int nn = nel * Np;
  const FluxConst<TF> C = flux_const<TF>(P);
  const TF iw = tf_from_double<TF>(P.inv_omega_end);

  {
    // all of this thread's loads issued before the first shared-memory store (compile-time
    // trip count; the launch has THREADS threads)
    constexpr int NT = (EPB * Np + THREADS - 1) / THREADS;
    TF ld[NT][ZP];
    const TF* __restrict__ src = aux + (long long)e0 * Np;
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const int t = threadIdx.x + i * THREADS;
#pragma unroll
      for (int c = 0; c < ZP; ++c)
        if (t < nn) ld[i][c] = src[c * N + t];
    }
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const int t = threadIdx.x + i * THREADS;
#pragma unroll
      for (int c = 0; c < ZP; ++c)
        if (t < nn) za[c * EPB * Np + t] = ld[i][c];
    }
  }
  if constexpr (FACES) {
    // h = ((m * 2 + side) * EPB + el) * P2 + ab: side 0 is the -x_m neighbour's last node
    // on line (a, b), side 1 the +x_m neighbour's first (compile-time strides: no division
    // by the ragged tile's element count)
    constexpr int nh = 6 * EPB * P2;
    for (int h = threadIdx.x; h < nh; h += blockDim.x) {
      const int ab = h % P2;
      const int r = h / P2;
      const int el = r % EPB, ms = r / EPB;
      if (el >= nel) continue;
      const int m = ms >> 1, side = ms & 1;
      const int en = neighbour(P, e0 + el, m, side ? 1 : -1);
      const long long g = (long long)en * Np + line_node<P1>(m, ab % P1, ab / P1, side ? 0 : P1 - 1);
#pragma unroll
      for (int c = 0; c < kAuxPlanes; ++c) halo[(ms * kAuxPlanes + c) * EPB * P2 + el * P2 + ab] = aux[c * N + g];
    }
  }
  __syncthreads();

#pragma unroll 1
  for (int m = 0; m < 3; ++m) {
    for (int l = threadIdx.x; l < nel * P2; l += blockDim.x) {
      const int el = l / P2, ab = l % P2;
      const int a = ab % P1, b = ab / P1;
      const int e = e0 + el;
      const TF met = tf_from_double<TF>(geom_of(P, inst_of(P, e)).metric[m]);
      Zstate<TF> z[P1];
#pragma unroll
      for (int i = 0; i < P1; ++i) {
        const int n = el * Np + line_node<P1>(m, a, b, i);
#pragma unroll
        for (int c = 0; c < kAux; ++c) z[i].z[c] = za[c * EPB * Np + n];
      }
      TF r[P1][5];
#pragma unroll
      for (int i = 0; i < P1; ++i)
#pragma unroll
        for (int v = 0; v < 5; ++v) r[i][v] = TF(0);
#pragma unroll
      for (int i = 0; i < P1; ++i) {
#pragma unroll
        for (int j = i + 1; j < P1; ++j) {
          TF f[5];
          ec_flux(z[i], z[j], m, C, f);
          const TF dij = Tab<TF>::D2(P, i * P1 + j), dji = Tab<TF>::D2(P, j * P1 + i);
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            fma_acc(r[i][v], dij, f[v]);
            fma_acc(r[j][v], dji, f[v]);
          }
        }
      }
      // interface terms: + (1/omega_p) f_num(+face) at i = p, - (1/omega_0) f_num(-face) at i = 0
      // the -x_m face flux: the -x_m neighbour's +x_m flux, or the boundary flux in FL
      const bool lo_b = at_boundary(P, e, m, 0);
      const int em = lo_b ? e : neighbour(P, e, m, -1);
      if constexpr (FACES) {
        // f_num(this element, +x_m neighbour) and f_num(-x_m neighbour, this element)
        const int nl = el * Np + line_node<P1>(m, a, b, P1 - 1), nf = el * Np + line_node<P1>(m, a, b, 0);
        const TF* hm = halo + (m * 2) * kAuxPlanes * EPB * P2 + el * P2 + ab;
        const TF* hp = hm + kAuxPlanes * EPB * P2;
        Zstate<TF> Lm, Rp;
#pragma unroll
        for (int c = 0; c < kAux; ++c) {
          Lm.z[c] = hm[c * EPB * P2];
          Rp.z[c] = hp[c * EPB * P2];
        }
        TF fp[5], fm[5];
        face_flux(z[P1 - 1], za[5 * EPB * Np + nl], Rp, hp[5 * EPB * P2], m, C, P.diss, fp);
        face_flux(Lm, hm[5 * EPB * P2], z[0], za[5 * EPB * Np + nf], m, C, P.diss, fm);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          r[P1 - 1][v] += iw * fp[v];
          r[0][v] -= iw * fm[v];
        }
      } else {
        const TF* Fm = lo_b ? FL : F;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          r[P1 - 1][v] += iw * F[((long long)(m * 5 + v) * P.K + e) * P2 + ab];
          r[0][v] -= iw * Fm[((long long)(m * 5 + v) * P.K + em) * P2 + ab];
        }
      }
      if constexpr (NS) {
        // viscous divergence (2/h_m)[D F^V_m + lifting]; enters with the opposite sign of r
        const int ep = neighbour(P, e, m, +1);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const TF* fc = fV + (long long)(m * 4 + c) * N;
          TF fl[P1];
#pragma unroll
          for (int j = 0; j < P1; ++j) fl[j] = fc[(long long)e * Np + line_node<P1>(m, a, b, j)];
          // boundary faces take the interior viscous flux (no viscous penalty)
          const TF f_next = at_boundary(P, e, m, 1) ? fl[P1 - 1] : fc[(long long)ep * Np + line_node<P1>(m, a, b, 0)];
          const TF f_prev = lo_b ? fl[0] : fc[(long long)em * Np + line_node<P1>(m, a, b, P1 - 1)];
#pragma unroll
          for (int i = 0; i < P1; ++i) {
            TF s = TF(0);
#pragma unroll
            for (int j = 0; j < P1; ++j) fma_acc(s, Tab<TF>::D(P, i * P1 + j), fl[j]);
            if (i == P1 - 1) s += TF(0.5) * iw * (f_next - fl[P1 - 1]);
            if (i == 0) s -= TF(0.5) * iw * (f_prev - fl[0]);
            r[i][1 + c] -= s;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < P1; ++i) {
        const int n = el * Np + line_node<P1>(m, a, b, i);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const TF val = -met * r[i][v];
          acc[v * EPB * Np + n] = (m == 0) ? val : acc[v * EPB * Np + n] + val;
        }
      }
    }
    __syncthreads();
  }

  // node phase: write k_i (or, in the last stage, d = sum_j c_j k_j + c_self k_i), element sums
  const bool wantE = sv.E != nullptr;
  const bool wantA = sv.dw != nullptr;
  // d and the element sums in FP64 (FP64 mode; mixed mode with FP64 estimates), else
  // in float-float joined to FP64 once
  const bool fp64_sums = std::is_same<TF, double>::value || (std::is_same<TF, float>::value && !P.ff_est);
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const long long g = (long long)e0 * Np + t;
    const int n = t % Np;
    const InstGeom& G = geom_of(P, inst_of(P, e0 + t / Np));
    if (fp64_sums) {
      const double Pn = mass_weight<P1>(P, G.J, n);
      double k[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) k[v] = to_f64(acc[v * EPB * Np + t]);
      if (sv.d_out) {
        const double dt = G.dt;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          double dv = (sv.dcoef_self * dt) * k[v];
          for (int j = 0; j < sv.nd; ++j)
            dv = fma(sv.dcoef[j] * dt, to_f64(static_cast<const TF*>(sv.dk[j])[v * N + g]), dv);
          sv.d_out[v * N + g] = dv;
        }
      } else if (sv.kout64) {
#pragma unroll
        for (int v = 0; v < 5; ++v) sv.kout64[v * N + g] = k[v];
      } else {
        TF* ko = static_cast<TF*>(sv.kout);
#pragma unroll
        for (int v = 0; v < 5; ++v) ko[v * N + g] = acc[v * EPB * Np + t];
      }
      if (wantE) {
        Zstate<TF> s;
#pragma unroll
        for (int c = 0; c < kAux; ++c) s.z[c] = za[c * EPB * Np + t];
        TF w[5];
        z_to_w(s, C, w);
        double sum = 0.0;
#pragma unroll
        for (int v = 0; v < 5; ++v) sum += to_f64(w[v]) * k[v];
        red[t] = Pn * sum;
      }
      if (wantA) {
        double sum = 0.0;
#pragma unroll
        for (int v = 0; v < 5; ++v) sum += sv.dw[v * N + g] * k[v];
        red[EPB * Np + t] = Pn * G.dt * sum;
      }
    } else {
      // float-float estimates: k stays in the flux precision; d and the element sums
      // are formed in float-float and joined to FP64 once
      TF kt[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) kt[v] = acc[v * EPB * Np + t];
      if (sv.d_out) {
        // d = dt (b_i k_i + sum_j b_j k_j): the coefficients split on the host, dt on the
        // integer pipe; the earlier stages in order
        const ff dtf = ff_from_double(G.dt);
        const ff cs(sv.dcoef_self_ff[0], sv.dcoef_self_ff[1]);
        ff dv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) dv[v] = cs * to_ff(kt[v]);
        for (int j = 0; j < sv.nd; ++j) {
          const ff cj(sv.dcoef_ff[j][0], sv.dcoef_ff[j][1]);
          const TF* dk = static_cast<const TF*>(sv.dk[j]);
#pragma unroll
          for (int v = 0; v < 5; ++v) ff_fma_acc(dv[v], cj, to_ff(dk[v * N + g]));
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) sv.d_out[v * N + g] = double(ff_norm(dv[v]) * dtf);
      } else if (sv.kout64) {
#pragma unroll
        for (int v = 0; v < 5; ++v) sv.kout64[v * N + g] = double(kt[v]);
      } else {
        TF* ko = static_cast<TF*>(sv.kout);
#pragma unroll
        for (int v = 0; v < 5; ++v) ko[v * N + g] = kt[v];
      }
      if (wantE) {
        Zstate<TF> s;
#pragma unroll
        for (int c = 0; c < kAux; ++c) s.z[c] = za[c * EPB * Np + t];
        TF w[5];
        z_to_w(s, C, w);
        double sum = 0.0;
#pragma unroll
        for (int v = 0; v < 5; ++v) sum += double(w[v]) * double(kt[v]);
        red[t] = mass_weight<P1>(P, G.J, n) * sum;
      }
      if (wantA) {
        // omega_i omega_j omega_k w-increment . k in float-float; J dt enter per element
        ff sum(0.0f, 0.0f);
#pragma unroll
        for (int v = 0; v < 5; ++v) ff_fma_acc(sum, reinterpret_cast<const ff*>(sv.dw)[v * N + g], to_ff(kt[v]));
        reinterpret_cast<ff*>(red)[EPB * Np + t] = mass_weight_ff<P1>(P, n) * ff_norm(sum);
      }
    }
  }
  const bool doA = sv.A != nullptr && (wantA || sv.A_init);
  if (!wantE && !doA) return;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int el = warp; el < nel; el += blockDim.x >> 5) {
    double sE = 0.0, sA = 0.0;
    for (int n = lane; n < Np; n += 32) {
      if (wantE) sE += red[el * Np + n];
      if (fp64_sums && wantA) sA += red[EPB * Np + el * Np + n];
    }
    if (wantE) sE = warp_sum(sE);
    if (fp64_sums) {
      sA = warp_sum(sA);
    } else if (wantA) {
      ff s(0.0f, 0.0f);
      for (int n = lane; n < Np; n += 32) s = s + reinterpret_cast<const ff*>(red)[EPB * Np + el * Np + n];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        s = s + ff(__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o));
      const InstGeom& G = geom_of(P, inst_of(P, e0 + el));
      sA = double(s) * (G.J * G.dt);
    }
    if (lane == 0) {
      const int e = e0 + el;
      if (wantE) sv.E[e] = sE;
      if (doA) sv.A[e] = (sv.A_init ? 0.0 : sv.A[e]) + (wantA ? sv.A_scale * sA : 0.0);
    }
  }
}

// The kernel: the plain launch bound (the compiler's own register choice), or, where
// VolRegs sets a cap, the minimum blocks per SM that enforce it (a minimum of one block
// would change the compiler's choice for the uncapped kernels too).
template <int P1, typename TF, bool NS, int EPB, int THREADS, bool FACES = false>
__global__ void __launch_bounds__(THREADS) k_volume(Params P, StageVol sv, const TF* __restrict__ aux,
                                                   const TF* __restrict__ F, const TF* __restrict__ FL,
                                                   const TF* __restrict__ fV) {
  volume_body<P1, TF, NS, EPB, THREADS, FACES>(P, sv, aux, F, FL, fV);
}
template <int P1, typename TF, bool NS, int EPB, int THREADS, bool FACES = false>
__global__ void __launch_bounds__(THREADS, (vol_min_blocks<P1, TF, NS, THREADS>()))
    k_volume_capped(Params P, StageVol sv, const TF* __restrict__ aux, const TF* __restrict__ F,
                    const TF* __restrict__ FL, const TF* __restrict__ fV) {
  volume_body<P1, TF, NS, EPB, THREADS, FACES>(P, sv, aux, F, FL, fV);
}
template <int P1, typename TF, bool NS, int EPB, int THREADS, bool FACES = false>
constexpr auto vol_kernel() {
  if constexpr (VolRegs<P1, TF, NS>::cap != 0) return k_volume_capped<P1, TF, NS, EPB, THREADS, FACES>;
  else return k_volume<P1, TF, NS, EPB, THREADS, FACES>;
}

// ---------------------------------------------------------------------------
// Relaxation (one lane group per element, RelaxGroup).  Per node: X0 = d_rho/rho,
// dv = (d_m - v d_rho)/rho, Y0 = (gam-1)(d_E - v.d_m + |v|^2 d_rho/2)/p,
// V2 = rho |dv|^2/p, c = P_n rho.  r(g) = sum_n c D_n(g)/rho_n + g A,
// r'(g) = sum_n c dD_n/dg + A; a = r''(0)/2 = sum c (X0^2 + (X0-Y0)^2/(gam-1) + V2)/2.
// Newton from the root of the cubic model a g^2 + b g^3 + A g (b from
// relax_node_cubic_f, FP32), safeguarded by the bracket [lo, hi] (r(lo) <= 0 < r(hi)); r is
// convex, so Newton converges from above.
// Near the root the error after a step s is ~ s^2 r''/(2 r') ~ s^2/g, so a step
// |s| <= root_rtol g (default 1e-8) leaves an error ~1e-16 g: the updated iterate is
// returned without another evaluation.
template <int P1>
__global__ void k_relax(Params P, StageRelax sr) {
  using RG = RelaxGroup<P1>;
  constexpr int Np = RG::Np, R = RG::R, SUB = RG::SUB;
  const long long N = (long long)P.K * Np;
  const double gam = P.gam;
  const double inv_gm1 = P.Cd.inv_gm1;
  const float gamf = tf_from_double<float>(gam);
  const int lane = threadIdx.x & 31;
  const int sl = lane % SUB;                  // lane within the element's group
  const unsigned gmask = RG::mask(lane);
  const int warps_per_block = blockDim.x >> 5;
  for (int e = (blockIdx.x * warps_per_block + (threadIdx.x >> 5)) * RG::EPW + lane / SUB; e < P.K;
       e += gridDim.x * warps_per_block * RG::EPW) {
    const int inst = inst_of(P, e);
    const double J = geom_of(P, inst).J;
    RelaxNode nd[R];
    double a_part = 0.0, s_part = 0.0, A_part = 0.0;
    float b_part = 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = sl + SUB * r;
      nd[r].X0 = nd[r].Y0 = nd[r].V2 = nd[r].c = 0.0;
      if (n < Np) {
        const long long g = (long long)e * Np + n;
        double u[5], d[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = sr.u[v * N + g];
        if (sr.u_new) {
#pragma unroll
          for (int v = 0; v < 5; ++v) d[v] = sr.u_new[v * N + g] - u[v];
          if (sr.d_out) {
#pragma unroll
            for (int v = 0; v < 5; ++v) sr.d_out[v * N + g] = d[v];
          }
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) d[v] = sr.d_in[v * N + g];
        }
        // one division: 1/(rho Pr), Pr = rho p
        const double rho = u[0];
        const double m2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
        const double Pr = (gam - 1.0) * (rho * u[4] - 0.5 * m2);
        const double inv = fast_rcp(rho * Pr);
        const double ir = Pr * inv, ip = rho * rho * inv;
        const double v0 = u[1] * ir, v1 = u[2] * ir, v2 = u[3] * ir;
        const double v2s = m2 * ir * ir;
        const double dv0 = (d[1] - v0 * d[0]) * ir, dv1 = (d[2] - v1 * d[0]) * ir, dv2 = (d[3] - v2 * d[0]) * ir;
        const double Pn = mass_weight<P1>(P, J, n);
        nd[r].X0 = d[0] * ir;
        nd[r].Y0 = (gam - 1.0) * (d[4] - (v0 * d[1] + v1 * d[2] + v2 * d[3]) + 0.5 * v2s * d[0]) * ip;
        nd[r].V2 = rho * (dv0 * dv0 + dv1 * dv1 + dv2 * dv2) * ip;
        nd[r].c = Pn * rho;
        const double XY = nd[r].X0 - nd[r].Y0;
        a_part += 0.5 * nd[r].c * (nd[r].X0 * nd[r].X0 + XY * XY * inv_gm1 + nd[r].V2);
        s_part += nd[r].c;
        // the starting point's cubic term in FP32, from the node values rounded on the
        // integer pipe (the FP64 pipe bounds this kernel)
        const RelaxNodeF nf{ff(tf_from_double<float>(nd[r].X0), 0.0f), ff(tf_from_double<float>(nd[r].Y0), 0.0f),
                            ff(tf_from_double<float>(nd[r].V2), 0.0f), ff(0.0f, 0.0f)};
        b_part = __fmaf_rn(tf_from_double<float>(nd[r].c), relax_node_cubic_f(nf, gamf), b_part);
        if (sr.u_new) {
          // A = sum P w(u).d - d_eta with w = ((gam - s)/(gam-1) - beta|v|^2/2, beta v, -beta)
          const double beta = rho * ip;
          const double p = Pr * ir;
          const double sp = log(p) - gam * log(rho);
          const double w0 = (gam - sp) * inv_gm1 - 0.5 * beta * v2s;
          A_part += Pn * (w0 * d[0] + beta * (v0 * d[1] + v1 * d[2] + v2 * d[3]) - beta * d[4]);
        }
      }
    }
    const double a = group_sum<SUB>(a_part, gmask);
    const double ssum = group_sum<SUB>(s_part, gmask);
    // the cubic coefficient only moves the starting point: an FP32 sum
    const double bcub = group_sum_f<SUB>(b_part, gmask);
    double A;
    if (sr.u_new) A = group_sum<SUB>(A_part, gmask) - sr.deta[e];
    else A = sr.A[e];
    double gk = __longlong_as_double(0x7ff0000000000000LL);  // +inf: unconstrained
    // delta_kappa = sqrt(2 a / sum c) > delta_floor, compared without the root and the division
    if (2.0 * a > sr.delta_floor * sr.delta_floor * ssum) {
      if (!(A < 0.0)) {
        if (sl == 0) atomicOr(sr.status, kStatusNoRoot);
      } else {
        double lo = 0.0, hi = sr.gamma_max;
        bool hi_known = false;
        // start: root of the cubic model a g^2 + b g^3 + A g (one Newton step on
        // a + b g + A/g from the quadratic model's root -A/a), off by O(delta^2)
        double gcur = -A * fast_rcp(a);
        const double den = a + 2.0 * bcub * gcur;
        if (den > 0.0) gcur -= bcub * gcur * gcur * fast_rcp(den);
        gcur = fmin(fmax(gcur, 1e-3), sr.gamma_max);
        for (int it = 0; it < 100; ++it) {
          double sr_ = 0.0, sd_ = 0.0;
          bool ok = true;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            double D, dD;
            if (nd[r].c != 0.0) {
              if (relax_node_eval(nd[r], gcur, gam, inv_gm1, D, dD)) {
                sr_ += nd[r].c * D;
                sd_ += nd[r].c * dD;
              } else {
                ok = false;
              }
            }
          }
          const bool phys = __all_sync(gmask, ok);
          const double rv = group_sum<SUB>(sr_, gmask) + gcur * A;
          const double dv = group_sum<SUB>(sd_, gmask) + A;
          if (!phys || rv > 0.0) {
            hi = gcur;
            hi_known = true;
          } else {
            lo = gcur;
          }
          if (phys && rv == 0.0) {
            gk = gcur;
            break;
          }
          const double step = rv * fast_rcp(dv);
          const double newton = gcur - step;
          // converged: a step this small cannot leave the bracket by more than rounding
          if (phys && dv > 0.0 && fabs(step) <= sr.root_rtol * gcur) {
            gk = fmin(fmax(newton, lo), hi);
            break;
          }
          const bool nok = phys && dv > 0.0 && isfinite(newton) && newton > lo && newton < hi;
          if (hi - lo <= 8.881784197001252e-16 * fmax(1.0, gcur)) {  // 4 * 2^-52
            gk = lo;
            break;
          }
          if (nok) gcur = newton;
          else if (!hi_known) gcur = (gcur >= sr.gamma_max) ? sr.gamma_max : fmin(2.0 * gcur, sr.gamma_max);
          else gcur = 0.5 * (lo + hi);
          if (!hi_known && lo >= sr.gamma_max) {  // r(gamma_max) <= 0: capped
            gk = sr.gamma_max;
            break;
          }
        }
      }
    }
    if (sl == 0) {
      sr.gamma_elem[e] = gk;
      atomic_min_positive(sr.gmin_bits + inst, gk);
    }
  }
}

// ---------------------------------------------------------------------------
// k_relax in float-float for the mixed and ES_FP64X modes: node data, element sums,
// bracket and Newton steps on the FP32 pipe (es_ff.cuh; ~2^-47 relative), the root
// joined to FP64 once per element.  Same rules as k_relax; the bracket-width stop is
// 2^-44 max(1, gamma) (the float-float resolution) instead of 4 * 2^-52, and the
// Newton-step tolerance is at least 2^-40.
// float-float / FP32 sums over a lane group (butterfly within the group's lanes)
template <int SUB>
__device__ __forceinline__ ff group_sum_ff(ff v, unsigned mask) {
#pragma unroll
  for (int o = SUB / 2; o > 0; o >>= 1) v = v + ff(__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o));
  return v;
}
__device__ __forceinline__ ff ff_min(ff x, ff y) { return y < x ? y : x; }
__device__ __forceinline__ ff ff_max(ff x, ff y) { return x < y ? y : x; }

// 128 threads, at least 8 blocks per SM: 64 registers (measured, GB300: 21 % faster than
// the unbounded 121 registers for p = 3, 31 % for p = 4 -- the kernel waits on latency,
// and the extra warps hide it better than the registers would)
template <int P1>
__global__ void __launch_bounds__(128, 8) k_relax_ff(Params P, StageRelax sr) {
  using RG = RelaxGroup<P1, true>;
  constexpr int Np = RG::Np, R = RG::R, SUB = RG::SUB;
  const long long N = (long long)P.K * Np;
  const FluxConst<ff>& C = P.Cff;
  const int lane = threadIdx.x & 31;
  const int sl = lane % SUB;
  const unsigned gmask = RG::mask(lane);
  const int warps_per_block = blockDim.x >> 5;
  const float floor2 = float(sr.delta_floor * sr.delta_floor);
  // Newton-step stop: the caller's tolerance, not below 2^-40 (float-float steps carry
  // rounding noise of ~2^-47 gamma; the bracket-width stop 2^-44 ends finer requests)
  const float rtol = float(fmax(sr.root_rtol, 9.094947017729282e-13));
  const ff gmax = ff_from_double(sr.gamma_max);
  const ff zero(0.0f, 0.0f);
  for (int e = (blockIdx.x * warps_per_block + (threadIdx.x >> 5)) * RG::EPW + lane / SUB; e < P.K;
       e += gridDim.x * warps_per_block * RG::EPW) {
    const int inst = inst_of(P, e);
    const ff J = ff_from_double(geom_of(P, inst).J);
    RelaxNodeF nd[R];
    ff a_p = zero, s_p = zero;
    float b_p = 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = sl + SUB * r;
      nd[r] = RelaxNodeF{zero, zero, zero, zero};
      if (n < Np) {
        const long long g = (long long)e * Np + n;
        ff u[5], d[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          u[v] = ff_from_double(sr.u[v * N + g]);
          d[v] = ff_from_double(sr.d_in[v * N + g]);
        }
        relax_node_setup_ff(u, d, C, mass_weight_ff<P1>(P, n) * J * u[0], nd[r]);
        s_p = s_p + nd[r].c;
        const ff XY = nd[r].X0 - nd[r].Y0;
        ff_fma_acc(a_p, ff_half(nd[r].c), nd[r].X0 * nd[r].X0 + XY * XY * C.inv_gm1 + nd[r].V2);
        b_p = __fmaf_rn(nd[r].c.hi, relax_node_cubic_f(nd[r], C.gam.hi), b_p);
      }
    }
    const ff a = group_sum_ff<SUB>(ff_norm(a_p), gmask);
    const float ssum = group_sum_f<SUB>(s_p.hi, gmask);
    const float bcub = group_sum_f<SUB>(b_p, gmask);
    const ff A = ff_from_double(sr.A[e]);
    double gk = __longlong_as_double(0x7ff0000000000000LL);  // +inf: unconstrained
    if (2.0f * a.hi > floor2 * ssum) {                         // delta_kappa > delta_floor
      if (!(A.hi < 0.0f)) {
        if (sl == 0) atomicOr(sr.status, kStatusNoRoot);
      } else {
        ff lo = zero, hi = gmax;
        bool hi_known = false;
        ff gcur = -(A * ff_rcp(a));
        const ff bf(bcub, 0.0f);
        const ff den = a + ff_twice(bf * gcur);
        if (den.hi > 0.0f) gcur = gcur - bf * gcur * gcur * ff_rcp(den);
        gcur = ff_min(ff_max(gcur, ff(1e-3f, 0.0f)), gmax);
        for (int it = 0; it < 100; ++it) {
          ff sr_f = zero, sd_f = zero;
          bool ok = true;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            ff D, dD;
            if (nd[r].c.hi != 0.0f) {
              if (relax_node_eval_ff(nd[r], gcur, C, D, dD)) {
                ff_fma_acc(sr_f, nd[r].c, D);
                ff_fma_acc(sd_f, nd[r].c, dD);
              } else {
                ok = false;
              }
            }
          }
          const bool phys = __all_sync(gmask, ok);
          const ff rv = group_sum_ff<SUB>(ff_norm(sr_f), gmask) + gcur * A;
          const ff dv = group_sum_ff<SUB>(ff_norm(sd_f), gmask) + A;
          if (!phys || rv.hi > 0.0f) {
            hi = gcur;
            hi_known = true;
          } else {
            lo = gcur;
          }
          if (phys && rv.hi == 0.0f) {
            gk = double(gcur);
            break;
          }
          const ff step = rv * ff_rcp(dv);
          const ff newton = gcur - step;
          if (phys && dv.hi > 0.0f && fabsf(step.hi) <= rtol * gcur.hi) {
            gk = double(ff_min(ff_max(newton, lo), hi));
            break;
          }
          const bool nok = phys && dv.hi > 0.0f && isfinite(newton.hi) && lo < newton && newton < hi;
          if ((hi - lo).hi <= 5.684341886080802e-14f * fmaxf(1.0f, gcur.hi)) {  // 2^-44
            gk = double(lo);
            break;
          }
          if (nok) gcur = newton;
          else if (!hi_known) gcur = (gmax < gcur || !(gcur < gmax)) ? gmax : ff_min(ff_twice(gcur), gmax);
          else gcur = ff_half(lo + hi);
          if (!hi_known && !(lo < gmax)) {  // r(gamma_max) <= 0: capped
            gk = sr.gamma_max;
            break;
          }
        }
      }
    }
    if (sl == 0) {
      sr.gamma_elem[e] = gk;
      atomic_min_positive(sr.gmin_bits + inst, gk);
    }
  }
}

// ---------------------------------------------------------------------------
// Global relaxation (Eqs. (u-n-gamma), (t-n-gamma); the comparison mode of the
// paper): one root per instance of r(g) = sum_kappa r_kappa(g).  Node data are
// stored once; every Newton iteration evaluates per-element sums at the
// instance's current gamma and one block per instance reduces them in a fixed
// order (deterministic) and takes the Newton/bisection step.

// per node (X0, Y0, V2, c) into nodes[4][N]; per element a_kappa and sum c
template <int P1>
__global__ void k_gsetup(Params P, const double* __restrict__ u, const double* __restrict__ d,
                         double* __restrict__ nodes, double* __restrict__ elem_a, double* __restrict__ elem_s) {
  constexpr int Np = P1 * P1 * P1;
  const long long N = (long long)P.K * Np;
  const double gam = P.gam, inv_gm1 = 1.0 / (gam - 1.0);
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < P.K; e += gridDim.x * wpb) {
    const double J = geom_of(P, inst_of(P, e)).J;
    double a_part = 0.0, s_part = 0.0;
    for (int n = lane; n < Np; n += 32) {
      const long long g = (long long)e * Np + n;
      const double rho = u[g], m0 = u[N + g], m1 = u[2 * N + g], m2 = u[3 * N + g], E = u[4 * N + g];
      const double Pr = (gam - 1.0) * (rho * E - 0.5 * (m0 * m0 + m1 * m1 + m2 * m2));
      const double inv = 1.0 / (rho * Pr);
      const double ir = Pr * inv, ip = rho * rho * inv;
      const double v0 = m0 * ir, v1 = m1 * ir, v2 = m2 * ir;
      const double v2s = v0 * v0 + v1 * v1 + v2 * v2;
      const double d0 = d[g], d1 = d[N + g], d2 = d[2 * N + g], d3 = d[3 * N + g], d4 = d[4 * N + g];
      const double dv0 = (d1 - v0 * d0) * ir, dv1 = (d2 - v1 * d0) * ir, dv2 = (d3 - v2 * d0) * ir;
      const double X0 = d0 * ir;
      const double Y0 = (gam - 1.0) * (d4 - (v0 * d1 + v1 * d2 + v2 * d3) + 0.5 * v2s * d0) * ip;
      const double V2 = rho * (dv0 * dv0 + dv1 * dv1 + dv2 * dv2) * ip;
      const double c = mass_weight<P1>(P, J, n) * rho;
      nodes[g] = X0;
      nodes[N + g] = Y0;
      nodes[2 * N + g] = V2;
      nodes[3 * N + g] = c;
      const double XY = X0 - Y0;
      a_part += 0.5 * c * (X0 * X0 + XY * XY * inv_gm1 + V2);
      s_part += c;
    }
    a_part = warp_sum(a_part);
    s_part = warp_sum(s_part);
    if (lane == 0) {
      elem_a[e] = a_part;
      elem_s[e] = s_part;
    }
  }
}

// per element sum_n c D_n(g)/rho_n and its g-derivative at the instance's gamma (NaN if not physical)
template <int P1>
__global__ void k_geval(Params P, const double* __restrict__ nodes, const GlobalRelaxState* __restrict__ gs,
                        double* __restrict__ elem_r, double* __restrict__ elem_dr) {
  constexpr int Np = P1 * P1 * P1;
  const long long N = (long long)P.K * Np;
  const double gam = P.gam, inv_gm1 = 1.0 / (gam - 1.0);
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < P.K; e += gridDim.x * wpb) {
    const GlobalRelaxState& S = gs[inst_of(P, e)];
    if (S.done) continue;
    const double gcur = S.g;
    double r = 0.0, dr = 0.0;
    bool ok = true;
    for (int n = lane; n < Np; n += 32) {
      const long long g = (long long)e * Np + n;
      RelaxNode nd;
      nd.X0 = nodes[g];
      nd.Y0 = nodes[N + g];
      nd.V2 = nodes[2 * N + g];
      nd.c = nodes[3 * N + g];
      double D, dD;
      if (relax_node_eval(nd, gcur, gam, inv_gm1, D, dD)) {
        r += nd.c * D;
        dr += nd.c * dD;
      } else {
        ok = false;
      }
    }
    const bool phys = __all_sync(0xffffffffu, ok);
    r = warp_sum(r);
    dr = warp_sum(dr);
    if (lane == 0) {
      elem_r[e] = phys ? r : __longlong_as_double(0x7ff8000000000000LL);
      elem_dr[e] = dr;
    }
  }
}

// fixed-order block reduction of x[off .. off+n) (all threads get the sum)
__device__ inline double block_sum(const double* x, int off, int n, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[off + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double out = sh[0];
  __syncthreads();
  return out;
}

// one block per instance.  phase 0: totals, degenerate / no-root checks, initial
// gamma; phase 1: one safeguarded Newton step from the evaluated sums.
static __global__ void k_gnewton(Params P, GlobalRelaxState* gs, const double* __restrict__ elem_a,
                          const double* __restrict__ elem_s, const double* __restrict__ A,
                          const double* __restrict__ elem_r, const double* __restrict__ elem_dr,
                          unsigned long long* gmin_bits, int* status, double delta_floor, double gamma_max,
                          double root_rtol, int phase) {
  __shared__ double sh[256];
  const int inst = blockIdx.x;
  const InstGeom& G = geom_of(P, inst);
  const int off = G.off, n = G.nx * G.ny * G.nz;
  GlobalRelaxState& S = gs[inst];
  if (phase == 0) {
    const double a = block_sum(elem_a, off, n, sh);
    const double ssum = block_sum(elem_s, off, n, sh);
    const double At = block_sum(A, off, n, sh);
    if (threadIdx.x == 0) {
      S.a = a;
      S.A = At;
      S.lo = 0.0;
      S.hi = gamma_max;
      S.hi_known = 0;
      S.done = 0;
      S.result = __longlong_as_double(0x7ff0000000000000LL);
      if (!(sqrt(2.0 * a / ssum) > delta_floor)) {
        S.done = 1;
      } else if (!(At < 0.0)) {
        atomicOr(status, kStatusNoRoot);
        S.done = 1;
      } else {
        S.g = fmin(fmax(-At / a, 1e-3), gamma_max);
      }
    }
    return;
  }
  if (S.done) return;
  const double R = block_sum(elem_r, off, n, sh);
  const double DR = block_sum(elem_dr, off, n, sh);
  if (threadIdx.x != 0) return;
  const double gcur = S.g;
  const bool phys = !isnan(R);
  const double rv = R + gcur * S.A;
  const double dv = DR + S.A;
  if (!phys || rv > 0.0) {
    S.hi = gcur;
    S.hi_known = 1;
  } else {
    S.lo = gcur;
  }
  if (phys && rv == 0.0) {
    S.result = gcur;
    S.done = 1;
  } else {
    const double step = rv / dv;
    const double newton = gcur - step;
    const bool nok = phys && dv > 0.0 && isfinite(newton) && newton > S.lo && newton < S.hi;
    if (phys && dv > 0.0 && fabs(step) <= root_rtol * gcur) {
      S.result = fmin(fmax(newton, S.lo), S.hi);
      S.done = 1;
    } else if (S.hi - S.lo <= 8.881784197001252e-16 * fmax(1.0, gcur)) {
      S.result = S.lo;
      S.done = 1;
    } else {
      S.g = nok ? newton : (S.hi_known ? 0.5 * (S.lo + S.hi) : fmin(2.0 * gcur, gamma_max));
      if (!S.hi_known && S.lo >= gamma_max) {
        S.result = gamma_max;
        S.done = 1;
      }
    }
  }
  if (S.done) gmin_bits[inst] = (unsigned long long)__double_as_longlong(S.result);
}

// after the iterations: instances that did not converge take their last iterate;
// every element reports its instance's gamma
static __global__ void k_gfinish(Params P, GlobalRelaxState* gs, unsigned long long* gmin_bits, double* gamma_elem) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P.K; e += gridDim.x * blockDim.x) {
    const int inst = inst_of(P, e);
    const GlobalRelaxState& S = gs[inst];
    const double g = S.done ? S.result : S.g;
    gamma_elem[e] = g;
    if (e == geom_of(P, inst).off) gmin_bits[inst] = (unsigned long long)__double_as_longlong(g);
  }
}

// eta_kappa = sum_n P_n S(q_n), S = -rho (ln p - gam ln rho)/(gam-1); one warp per element
template <int P1>
__global__ void k_entropy(Params P, const double* __restrict__ q, double* __restrict__ eta) {
  constexpr int Np = P1 * P1 * P1;
  const long long N = (long long)P.K * Np;
  const double gam = P.gam;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < P.K; e += gridDim.x * wpb) {
    const double J = geom_of(P, inst_of(P, e)).J;
    double s = 0.0;
    for (int n = lane; n < Np; n += 32) {
      const long long g = (long long)e * Np + n;
      const double rho = q[g];
      const double ir = 1.0 / rho;
      const double m0 = q[N + g], m1 = q[2 * N + g], m2 = q[3 * N + g];
      const double p = (gam - 1.0) * (q[4 * N + g] - 0.5 * (m0 * m0 + m1 * m1 + m2 * m2) * ir);
      s += mass_weight<P1>(P, J, n) * (-rho * (log(p) - gam * log(rho)) / (gam - 1.0));
    }
    s = warp_sum(s);
    if (lane == 0) eta[e] = s;
  }
}

// The two sides of Theorem 2.3's local inequality for the step just taken (state u
// before its relaxed update, d = u_new - u, A from the stages): eta_old = eta_kappa(u)
// in the arithmetic of k_entropy, and the estimate
// deta = eta_kappa^new - eta_kappa(u) = sum_n P_n w(u_n).d_n - A, which equals
// dt sum_i b_i (eta_kappa' f)(y^i) of Eq. (eta-est-1-RK) because the stages accumulate
// A = -dt sum_i b_i sum_n P_n (w(y^i) - w(u)).k_i.  One warp per element.
template <int P1>
__global__ void k_estimate(Params P, const double* __restrict__ q, const double* __restrict__ d,
                           const double* __restrict__ A, double* __restrict__ eta_old, double* __restrict__ deta) {
  constexpr int Np = P1 * P1 * P1;
  const long long N = (long long)P.K * Np;
  const double gam = P.gam;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < P.K; e += gridDim.x * wpb) {
    const double J = geom_of(P, inst_of(P, e)).J;
    double s_eta = 0.0, s_wd = 0.0;
    for (int n = lane; n < Np; n += 32) {
      const long long g = (long long)e * Np + n;
      const double rho = q[g];
      const double ir = 1.0 / rho;
      const double m0 = q[N + g], m1 = q[2 * N + g], m2 = q[3 * N + g];
      const double p = (gam - 1.0) * (q[4 * N + g] - 0.5 * (m0 * m0 + m1 * m1 + m2 * m2) * ir);
      const double s = log(p) - gam * log(rho);
      const double Pn = mass_weight<P1>(P, J, n);
      s_eta += Pn * (-rho * s / (gam - 1.0));
      // w = ((gam - s)/(gam-1) - beta |v|^2/2, beta v, -beta), beta = rho/p
      const double beta = rho / p;
      const double v0 = m0 * ir, v1 = m1 * ir, v2 = m2 * ir;
      const double w0 = (gam - s) / (gam - 1.0) - 0.5 * beta * (v0 * v0 + v1 * v1 + v2 * v2);
      s_wd += Pn * (w0 * d[g] + beta * (v0 * d[N + g] + v1 * d[2 * N + g] + v2 * d[3 * N + g]) -
                    beta * d[4 * N + g]);
    }
    s_eta = warp_sum(s_eta);
    s_wd = warp_sum(s_wd);
    if (lane == 0) {
      if (eta_old) eta_old[e] = s_eta;
      if (deta) deta[e] = s_wd - A[e];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
template <typename TF, bool FP64>
void prep_launch(const Params& P, const StagePrep& sp, TF* a, int* status, cudaStream_t st, int grid) {
  switch (sp.nprev) {
    case 0: k_prep<TF, 0, FP64><<<grid, 256, 0, st>>>(P, sp, a, status); break;
    case 1: k_prep<TF, 1, FP64><<<grid, 256, 0, st>>>(P, sp, a, status); break;
    case 2: k_prep<TF, 2, FP64><<<grid, 256, 0, st>>>(P, sp, a, status); break;
    case 3: k_prep<TF, 3, FP64><<<grid, 256, 0, st>>>(P, sp, a, status); break;
    default: k_prep<TF, -1, FP64><<<grid, 256, 0, st>>>(P, sp, a, status); break;
  }
}

template <int P1, typename TF>
void Launcher<P1, TF>::prep(const Params& P, const StagePrep& sp, void* aux, int* status, cudaStream_t st,
                            int grid) {
  TF* a = static_cast<TF*>(aux);
  if constexpr (std::is_same<TF, double>::value) {
    prep_launch<TF, true>(P, sp, a, status, st, grid);
  } else if constexpr (std::is_same<TF, float>::value) {
    if (P.ff_est) prep_launch<TF, false>(P, sp, a, status, st, grid);
    else prep_launch<TF, true>(P, sp, a, status, st, grid);
  } else {
    prep_launch<TF, false>(P, sp, a, status, st, grid);
  }
}

template <int P1, typename TF>
void Launcher<P1, TF>::face(const Params& P, const void* aux, void* F, void* FL, cudaStream_t st, int grid) {
  if (P.visc_pen > 0.0)
    k_face<P1, TF, true><<<grid, 256, 0, st>>>(P, static_cast<const TF*>(aux), static_cast<TF*>(F), static_cast<TF*>(FL));
  else
    k_face<P1, TF, false><<<grid, 256, 0, st>>>(P, static_cast<const TF*>(aux), static_cast<TF*>(F), static_cast<TF*>(FL));
}

template <int P1, typename TF>
void Launcher<P1, TF>::grad(const Params& P, const void* aux, void* fV, cudaStream_t st, int) {
  using C = VolCfg<P1, 0>;
  const int grid = (P.K + C::EPB - 1) / C::EPB;
  const size_t smem = size_t(4) * C::EPB * P1 * P1 * P1 * sizeof(TF);
  k_grad<P1, TF, C::EPB, C::THREADS><<<grid, C::THREADS, smem, st>>>(P, static_cast<const TF*>(aux),
                                                                      static_cast<TF*>(fV));
}


template <int P1, typename TF, int V>
cudaError_t volume_setup_v() {
  using C = VolCfg<P1, V>;
  const int smem = (int)VolSmem<P1, C::EPB, false>::template bytes<TF>();
  cudaError_t e1 = cudaFuncSetAttribute(vol_kernel<P1, TF, false, C::EPB, C::THREADS>(),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaError_t e2 = cudaFuncSetAttribute(vol_kernel<P1, TF, true, C::EPB, C::THREADS>(),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e1 != cudaSuccess ? e1 : e2;
}

template <int P1, typename TF>
cudaError_t Launcher<P1, TF>::volume_setup() {
  cudaError_t e = volume_setup_v<P1, TF, 0>();
  if (e == cudaSuccess) e = volume_setup_v<P1, TF, 1>();
  if (e == cudaSuccess) e = volume_setup_v<P1, TF, 2>();
  return e;
}

template <int P1, typename TF, int V>
void volume_v(const Params& P, const StageVol& sv, const TF* aux, const TF* F, const TF* FL, const TF* fV, bool ns,
              cudaStream_t st) {
  using C = VolCfg<P1, V>;
  const int grid = (P.K + C::EPB - 1) / C::EPB;
  const size_t smem = VolSmem<P1, C::EPB, false>::template bytes<TF>();
  if (ns)
    vol_kernel<P1, TF, true, C::EPB, C::THREADS>()<<<grid, C::THREADS, smem, st>>>(P, sv, aux, F, FL, fV);
  else
    vol_kernel<P1, TF, false, C::EPB, C::THREADS>()<<<grid, C::THREADS, smem, st>>>(P, sv, aux, F, FL, fV);
}

template <int P1, typename TF>
void Launcher<P1, TF>::volume(const Params& P, const StageVol& sv, const void* aux, const void* F, const void* FL, const void* fV,
                              bool ns, cudaStream_t st, int variant) {
  const TF* a = static_cast<const TF*>(aux);
  const TF* f = static_cast<const TF*>(F);
  const TF* fl = static_cast<const TF*>(FL);
  const TF* v = static_cast<const TF*>(fV);
  if (variant == 1) volume_v<P1, TF, 1>(P, sv, a, f, fl, v, ns, st);
  else if (variant == 2) volume_v<P1, TF, 2>(P, sv, a, f, fl, v, ns, st);
  else volume_v<P1, TF, 0>(P, sv, a, f, fl, v, ns, st);
}

template <int P1, int V>
cudaError_t volface_setup_v() {
  using C = VolCfg<P1, V>;
  return cudaFuncSetAttribute(vol_kernel<P1, float, false, C::EPB, C::THREADS, true>(),
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)VolSmem<P1, C::EPB, true>::template bytes<float>());
}

template <int P1, typename TF>
cudaError_t Launcher<P1, TF>::volface_setup() {
  if constexpr (std::is_same<TF, float>::value) {
    cudaError_t e = volface_setup_v<P1, 0>();
    if (e == cudaSuccess) e = volface_setup_v<P1, 1>();
    if (e == cudaSuccess) e = volface_setup_v<P1, 2>();
    return e;
  }
  return cudaSuccess;
}

template <int P1, int V>
void volface_v(const Params& P, const StageVol& sv, const float* aux, cudaStream_t st) {
  using C = VolCfg<P1, V>;
  const int grid = (P.K + C::EPB - 1) / C::EPB;
  vol_kernel<P1, float, false, C::EPB, C::THREADS, true>()
      <<<grid, C::THREADS, VolSmem<P1, C::EPB, true>::template bytes<float>(), st>>>(P, sv, aux, nullptr, nullptr,
                                                                                     nullptr);
}

template <int P1, typename TF>
void Launcher<P1, TF>::volface(const Params& P, const StageVol& sv, const void* aux, cudaStream_t st, int variant) {
  if constexpr (std::is_same<TF, float>::value) {
    const float* a = static_cast<const float*>(aux);
    if (variant == 1) volface_v<P1, 1>(P, sv, a, st);
    else if (variant == 2) volface_v<P1, 2>(P, sv, a, st);
    else volface_v<P1, 0>(P, sv, a, st);
  }
}

template <int P1, typename TF>
void Launcher<P1, TF>::relax(const Params& P, const StageRelax& sr, cudaStream_t st, int grid) {
  // the u_new entry point (es_relax_step), the FP64 mode and the mixed mode with FP64
  // estimates solve in FP64; 4 warps per block, RelaxGroup::EPW elements per warp
  const bool fp64 = sr.u_new || std::is_same<TF, double>::value || (std::is_same<TF, float>::value && !P.ff_est);
  const int epb = 4 * (fp64 ? RelaxGroup<P1>::EPW : RelaxGroup<P1, true>::EPW);
  const int need = (P.K + epb - 1) / epb;
  const int g = grid < need ? grid : need;
  if (fp64) k_relax<P1><<<g, 128, 0, st>>>(P, sr);
  else k_relax_ff<P1><<<g, 128, 0, st>>>(P, sr);
}

template <int P1, typename TF>
void Launcher<P1, TF>::global_relax(const Params& P, const GlobalRelaxArgs& ga, cudaStream_t st, int grid,
                                    int iterations) {
  k_gsetup<P1><<<grid, 128, 0, st>>>(P, ga.u, ga.d, ga.nodes, ga.elem_a, ga.elem_s);
  k_gnewton<<<P.ninst, 256, 0, st>>>(P, ga.gs, ga.elem_a, ga.elem_s, ga.A, ga.elem_r, ga.elem_dr, ga.gmin_bits,
                                      ga.status, ga.delta_floor, ga.gamma_max, ga.root_rtol, 0);
  for (int it = 0; it < iterations; ++it) {
    k_geval<P1><<<grid, 128, 0, st>>>(P, ga.nodes, ga.gs, ga.elem_r, ga.elem_dr);
    k_gnewton<<<P.ninst, 256, 0, st>>>(P, ga.gs, ga.elem_a, ga.elem_s, ga.A, ga.elem_r, ga.elem_dr, ga.gmin_bits,
                                        ga.status, ga.delta_floor, ga.gamma_max, ga.root_rtol, 1);
  }
  k_gfinish<<<(P.K + 255) / 256, 256, 0, st>>>(P, ga.gs, ga.gmin_bits, ga.gamma_elem);
}

template <int P1, typename TF>
void Launcher<P1, TF>::entropy(const Params& P, const double* q, double* eta, cudaStream_t st, int grid) {
  k_entropy<P1><<<grid, 128, 0, st>>>(P, q, eta);
}

template <int P1, typename TF>
void Launcher<P1, TF>::estimate(const Params& P, const double* q, const double* d, const double* A, double* eta_old,
                                double* deta, cudaStream_t st, int grid) {
  k_estimate<P1><<<grid, 128, 0, st>>>(P, q, d, A, eta_old, deta);
}

}  // namespace es

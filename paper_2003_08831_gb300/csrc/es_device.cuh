// Device-side building blocks of the locally relaxed entropy-stable RK step.
//
// Pointwise thermodynamics of Section 3.1 (conserved q = (rho, rho U, rho E),
// P = rho R T, entropy S = -rho s with s = ln p - gamma ln rho, scaled by
// 1/(gamma - 1)), the Ismail--Roe entropy-conservative two-point flux with the
// series logarithmic mean, Rusanov interface dissipation, and the
// cancellation-free pieces of the relaxation function of
// Eq. (relaxation-local-gamma).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "es_ff.cuh"

namespace es {

constexpr int kMaxP1 = 6;
constexpr int kStatusNonphysical = 1;
constexpr int kStatusNoRoot = 2;

// Exterior values of a Dirichlet-penalty boundary, per direction and side, at the
// current stage time: the parameter vector z1..z5, 1/z1 and the entropy variables
// w2..w5 of the prescribed state (layout [3 directions][2 sides][kBcVals]).
constexpr int kBcVals = 10;

// Geometry of one periodic Cartesian instance (mesh) inside a group of
// instances sharing the LGL degree; a single-instance context is a group of one.
struct InstGeom {
  int nx, ny, nz, off;  // element grid; first element of the instance in the group
  double metric[3];     // 2/h_m
  double J;             // h1 h2 h3 / 8
  double dt;            // the instance's time step
};

// Constants of the gas law used by the flux, in the flux's precision.
template <typename T>
struct FluxConst {
  T gam, gm1, inv_gm1, sqrt_gam;
  T C1x, C2x;  // 4 c1 gam/(gam-1), c2 gam/(gam-1) with c1 = (gam+1)/(2 gam), c2 = (gam-1)/(2 gam)
  __host__ __device__ static FluxConst make(double g) {
    FluxConst c;
    c.gam = T(g);
    c.gm1 = T(g - 1.0);
    c.inv_gm1 = T(1.0 / (g - 1.0));
    c.sqrt_gam = T(sqrt(g));
    c.C1x = T(4.0 * (g + 1.0) / (2.0 * g) * g / (g - 1.0));
    c.C2x = T((g - 1.0) / (2.0 * g) * g / (g - 1.0));
    return c;
  }
};

// Operator tables and physics constants, passed by value to every kernel.
struct Params {
  double D[kMaxP1 * kMaxP1];   // SBP derivative on [-1, 1], row-major
  double D2[kMaxP1 * kMaxP1];  // 2 D_ij (i != j), 0 on the diagonal
  float Dff[2][kMaxP1 * kMaxP1];   // D and 2 D split into float-float (hi, lo); hi is
  float D2ff[2][kMaxP1 * kMaxP1];  // the FP32 table (round to nearest) of the mixed mode
  double omega[kMaxP1];        // LGL weights
  float omega_ff[2][kMaxP1];   // LGL weights split into float-float (hi, lo)
  double inv_omega_end;        // 1/omega_0 = 1/omega_p
  double gam;                  // ratio of specific heats
  double mu, kappa_heat, R;    // viscosity, heat conductivity mu c_p / Pr, gas constant
  double inv_R;                // 1/R
  double visc_pen;             // diss^V coefficient alpha (0: off; only with mu > 0)
  FluxConst<double> Cd;        // flux constants per precision (host-computed: no
  FluxConst<float> Cf;         // divisions or square roots in the kernels)
  FluxConst<ff> Cff;
  int K;                       // elements in the group
  int diss;                    // Rusanov interface dissipation on/off
  int p1;                      // p + 1
  int ninst;                   // instances in the group
  int ff_est;                  // FP32 fluxes: entropy increments, the relaxation sums and
                               // the gamma solve in float-float (1) or in FP64 (0)
  InstGeom g0;                 // the instance when geom is null (single-instance context)
  const InstGeom* geom;        // device table [ninst] (batches), or null
  const int* elem_inst;        // device [K]: instance of each element (batches), or null
  int bc[3];                   // per direction: 0 periodic, 1 Dirichlet penalty (single instance)
  const double* bcz;           // device [3][2][kBcVals] exterior values (see kBcVals), or null
  const int* nbr;              // device [K][6]: periodic neighbour of each element along -x_m, +x_m
                               // (index 2 m + side), or null (then computed from the geometry)
};

template <typename T> __device__ __forceinline__ const FluxConst<T>& flux_const(const Params& P);
template <> __device__ __forceinline__ const FluxConst<double>& flux_const<double>(const Params& P) { return P.Cd; }
template <> __device__ __forceinline__ const FluxConst<float>& flux_const<float>(const Params& P) { return P.Cf; }
template <> __device__ __forceinline__ const FluxConst<ff>& flux_const<ff>(const Params& P) { return P.Cff; }

// ---------------------------------------------------------------------------
// element / node index helpers
__device__ __forceinline__ int inst_of(const Params& P, int e) { return P.elem_inst ? P.elem_inst[e] : 0; }

__device__ __forceinline__ const InstGeom& geom_of(const Params& P, int inst) { return P.geom ? P.geom[inst] : P.g0; }

// Periodic neighbour of element e along direction m (dir = -1 or +1): from the context's
// table when there is one (one cached load), else from the element's grid position (five
// integer divisions).
__device__ __forceinline__ int neighbour(const Params& P, int e, int m, int dir) {
  if (P.nbr) return P.nbr[(long long)e * 6 + m * 2 + (dir > 0 ? 1 : 0)];
  const InstGeom& G = geom_of(P, inst_of(P, e));
  const int le = e - G.off;
  int ex = le % G.nx;
  int ey = (le / G.nx) % G.ny;
  int ez = le / (G.nx * G.ny);
  if (m == 0) ex = (ex + dir + G.nx) % G.nx;
  else if (m == 1) ey = (ey + dir + G.ny) % G.ny;
  else ez = (ez + dir + G.nz) % G.nz;
  return G.off + ex + G.nx * (ey + G.ny * ez);
}

// Dirichlet-penalty boundary faces: element e is first (side 0) or last (side 1)
// along a non-periodic direction m
__device__ __forceinline__ bool at_boundary(const Params& P, int e, int m, int side) {
  if (!P.bc[m]) return false;
  const InstGeom& G = geom_of(P, inst_of(P, e));
  const int le = e - G.off;
  const int idx = m == 0 ? le % G.nx : (m == 1 ? (le / G.nx) % G.ny : le / (G.nx * G.ny));
  const int n = m == 0 ? G.nx : (m == 1 ? G.ny : G.nz);
  return side == 0 ? idx == 0 : idx == n - 1;
}
__device__ __forceinline__ const double* bc_values(const Params& P, int m, int side) {
  return P.bcz + (m * 2 + side) * kBcVals;
}

// node index of position i on the line (a, b) in direction m
template <int P1>
__device__ __forceinline__ int line_node(int m, int a, int b, int i) {
  return m == 0 ? i + P1 * (a + P1 * b) : (m == 1 ? a + P1 * (i + P1 * b) : a + P1 * (b + P1 * i));
}

// mass weight P_n = J omega_i omega_j omega_k
template <int P1>
__device__ __forceinline__ double mass_weight(const Params& P, double J, int n) {
  int i = n % P1, j = (n / P1) % P1, k = n / (P1 * P1);
  return J * P.omega[i] * P.omega[j] * P.omega[k];
}

// operator entries in the flux precision T (float-float: the split tables)
template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ double D(const Params& P, int i) { return P.D[i]; }
  static __device__ __forceinline__ double D2(const Params& P, int i) { return P.D2[i]; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ float D(const Params& P, int i) { return P.Dff[0][i]; }
  static __device__ __forceinline__ float D2(const Params& P, int i) { return P.D2ff[0][i]; }
};
template <> struct Tab<ff> {
  static __device__ __forceinline__ ff D(const Params& P, int i) { return ff(P.Dff[0][i], P.Dff[1][i]); }
  static __device__ __forceinline__ ff D2(const Params& P, int i) { return ff(P.D2ff[0][i], P.D2ff[1][i]); }
};

// acc += a b in the flux precision (the float-float form keeps the product and
// sum errors, see es_ff.cuh; FP64/FP32 use one fma, as contraction would)
__device__ __forceinline__ void fma_acc(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void fma_acc(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void fma_acc(ff& acc, ff a, ff b) { ff_fma_acc(acc, a, b); }

// a double in the flux precision without FP64 instructions (float: the split rounded once)
template <typename T> __device__ __forceinline__ T tf_from_double(double x);
template <> __device__ __forceinline__ double tf_from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ ff tf_from_double<ff>(double x) { return ff_from_double(x); }
template <> __device__ __forceinline__ float tf_from_double<float>(double x) {
  const ff s = ff_from_double(x);
  return __fadd_rn(s.hi, s.lo);
}

// omega_i omega_j omega_k of node n in float-float
template <int P1>
__device__ __forceinline__ ff mass_weight_ff(const Params& P, int n) {
  const int i = n % P1, j = (n / P1) % P1, k = n / (P1 * P1);
  return ff(P.omega_ff[0][i], P.omega_ff[1][i]) * ff(P.omega_ff[0][j], P.omega_ff[1][j]) *
         ff(P.omega_ff[0][k], P.omega_ff[1][k]);
}

// ---------------------------------------------------------------------------
// Parameter-vector state used by the two-point flux: z = sqrt(rho/p) (1, v, p).
constexpr int kAux = 5;       // planes read by the volume kernel
constexpr int kAuxPlanes = 6; // + iz1 = 1/z1, read by the face kernel
template <typename T>
struct Zstate {
  T z[5];
};

// Series logarithmic-mean pieces.  For aL, aR > 0 with s = aL + aR,
// d = aL - aR and u = (d/s)^2:  ln-mean = (s/2) / F(u) with
// F(u) = atanh(sqrt u)/sqrt u = 1 + u/3 + u^2/5 + u^3/7 + ...  Below the
// threshold both F and 1/F are taken from their Taylor series (truncation
// below the type's rounding); above it the mean is d / ln(aL/aR).
template <typename T> struct LogMeanConst;
template <> struct LogMeanConst<double> { static constexpr double eps = 1.0e-4; };
template <> struct LogMeanConst<float> { static constexpr float eps = 1.0e-2f; };

// 1/x for FP64 without the IEEE division sequence: the hardware approximation r
// (PTX rcp.approx.ftz.f64) refined by one third-order step of the series
// 1/x = r/(1 - e) = r (1 + e + e^2 + ...), e = 1 - x r (three fmas; the truncation
// r e^3 is below 2^-60 for an approximation good to 2^-20).  x must be a normal
// positive or negative number (subnormals flush to zero); the result is within one
// unit in the last place of 1/x, not correctly rounded.
__device__ __forceinline__ double fast_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
// FP32 (the mixed modes' fluxes): the hardware approximation refined by one Newton step
// r + r (1 - x r), within about an ulp of 1/x, without the IEEE division's special-case
// path (x is a normal nonzero product of parameter-vector sums)
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return __fmaf_rn(r, __fmaf_rn(-x, r, 1.0f), r);
}
__device__ __forceinline__ ff fast_rcp(ff x) { return ff_rcp(x); }

// |z| <= t for a positive threshold t, on the integer pipe (sign bit cleared)
__device__ __forceinline__ bool abs_le(double z, double t) {
  return (__double_as_longlong(z) & 0x7fffffffffffffffLL) <= __double_as_longlong(t);
}

// u >= 0 (a square) compared with a positive threshold on the integer pipe:
// non-negative IEEE values order like their bit patterns (NaN compares false).
__device__ __forceinline__ bool below(double u, double eps) {
  return __double_as_longlong(u) < __double_as_longlong(eps);
}
__device__ __forceinline__ bool below(float u, float eps) { return __float_as_int(u) < __float_as_int(eps); }

// Ismail--Roe two-point flux in direction m between states a and b.
// With S = a + b, D = a - b for z1 and z5, the two logarithmic means enter only
// through f1 = S1/(2 ln-mean(z1)) and g5 = ln-mean(z5)/(2 S5):
//   rho_hat = z1_avg ln-mean(z5) = S1 S5 g5,   u_hat = (z_{2..4} sums)/S1,
//   p1_hat = S5/S1,   p2_hat = p1_hat (4 c1 g5 f1 + c2),
//   flux_m = (rho_hat u_m, rho_hat u_m u_hat + p1_hat e_m,
//             u_m gam/(gam-1) p2_hat + rho_hat u_m |u_hat|^2/2).
// Series branch (u = (D/S)^2 below the threshold): f1 = F(u1), g5 = (1/F)(u5)/4 with
// F(u) = 1 + u/3 + u^2/5 + u^3/7 and 1/F = 1 - u/3 - 4u^2/45 - 44u^3/945;
// otherwise f1 = S1 ln(a/b)/(2 D1), g5 = D5/(2 S5 ln(a/b)).
template <typename T>
__device__ __forceinline__ void ec_flux(const Zstate<T>& a, const Zstate<T>& b, int m, const FluxConst<T>& C,
                                        T f[5]) {
  const T S1 = a.z[0] + b.z[0], D1 = a.z[0] - b.z[0];
  const T S5 = a.z[4] + b.z[4], D5 = a.z[4] - b.z[4];
  const T P15 = S1 * S5;
  const T inv = fast_rcp(P15);
  const T inv1 = S5 * inv;          // 1/S1
  const T r1 = D1 * inv1;
  const T r5 = D5 * (S1 * inv);     // D5/S5
  const T u1 = r1 * r1, u5 = r5 * r5;
  const T eps = LogMeanConst<T>::eps;
  T f1, g5;
  if (below(u1, eps)) f1 = T(1) + u1 * (T(1.0 / 3.0) + u1 * (T(1.0 / 5.0) + u1 * T(1.0 / 7.0)));
  else f1 = T(0.5) * S1 * log(a.z[0] / b.z[0]) / D1;
  if (below(u5, eps)) g5 = T(0.25) - u5 * (T(1.0 / 12.0) + u5 * (T(1.0 / 45.0) + u5 * T(11.0 / 945.0)));
  else g5 = T(0.5) * D5 / (S5 * log(a.z[4] / b.z[4]));
  const T rho_hat = P15 * g5;
  const T u0 = (a.z[1] + b.z[1]) * inv1;
  const T uy = (a.z[2] + b.z[2]) * inv1;
  const T uz = (a.z[3] + b.z[3]) * inv1;
  const T p1 = S5 * inv1;
  const T p2g = p1 * (C.C1x * (g5 * f1) + C.C2x);  // gam/(gam-1) p2_hat
  const T um = m == 0 ? u0 : (m == 1 ? uy : uz);
  const T mass = rho_hat * um;
  const T q2 = u0 * u0 + uy * uy + uz * uz;
  f[0] = mass;
  // p1 joins the momentum flux of direction m inside one fma; constant indices keep f in
  // registers (m is a run-time value)
  f[1] = fma(mass, u0, m == 0 ? p1 : T(0));
  f[2] = fma(mass, uy, m == 1 ? p1 : T(0));
  f[3] = fma(mass, uz, m == 2 ? p1 : T(0));
  f[4] = um * p2g + (T(0.5) * mass) * q2;
}

// The same flux in float-float arithmetic (precision mode ES_FP64X).  The
// series branch keeps the leading u/3 (u/12) terms in float-float and the
// higher-order terms, below 2.1e-5 relative to them for u < 1e-4, in FP32; the
// sums and differences of the z's whose high parts agree within a factor two
// are exact in their high part (Sterbenz), so D = (a.hi - b.hi) + (a.lo - b.lo)
// carries a single rounding.  The rare logarithmic branch (u >= 1e-4) is taken
// in FP64.
__device__ __forceinline__ ff ff_series_f(ff u) {
  // F(u) = 1 + u/3 + u^2/5 + u^3/7
  constexpr float th = float(1.0 / 3.0);
  constexpr float tl = float(1.0 / 3.0 - double(th));
  const float p = __fmul_rn(u.hi, th);
  float e = __fmaf_rn(u.hi, th, -p);
  e = __fmaf_rn(u.hi, tl, e);
  e = __fmaf_rn(u.lo, th, e);
  const float q = __fmul_rn(u.hi, __fmaf_rn(u.hi, 1.0f / 7.0f, 0.2f));  // u/5 + u^2/7
  e = __fmaf_rn(u.hi, q, e);
  const ff s = fast_two_sum(1.0f, p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, e));
}
__device__ __forceinline__ ff ff_series_g(ff u) {
  // (1/F(u))/4 = 1/4 - u/12 - u^2/45 - 11 u^3/945
  constexpr float th = float(1.0 / 12.0);
  constexpr float tl = float(1.0 / 12.0 - double(th));
  const float p = __fmul_rn(u.hi, th);
  float e = __fmaf_rn(u.hi, th, -p);
  e = __fmaf_rn(u.hi, tl, e);
  e = __fmaf_rn(u.lo, th, e);
  const float q = __fmul_rn(u.hi, __fmaf_rn(u.hi, 11.0f / 945.0f, 1.0f / 45.0f));
  e = __fmaf_rn(u.hi, q, e);
  const ff s = fast_two_sum(0.25f, -p);
  return fast_two_sum(s.hi, __fsub_rn(s.lo, e));
}
__device__ __forceinline__ ff ff_exact_diff(ff a, ff b) {
  return ff_norm(ff(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ void ec_flux(const Zstate<ff>& a, const Zstate<ff>& b, int m, const FluxConst<ff>& C,
                                        ff f[5]) {
  const ff S1 = a.z[0] + b.z[0];
  const ff S5 = a.z[4] + b.z[4];
  const ff P15 = S1 * S5;
  const ff inv = ff_rcp(P15);
  const ff inv1 = S5 * inv;  // 1/S1
  const ff is5 = S1 * inv;   // 1/S5
  // high parts within a factor two: D exact up to the lo difference (else the
  // FP64 branch below recomputes the mean and u is only used for the test)
  const ff r1 = ff_exact_diff(a.z[0], b.z[0]) * inv1;
  const ff r5 = ff_exact_diff(a.z[4], b.z[4]) * is5;
  const ff u1 = r1 * r1, u5 = r5 * r5;
  ff f1, g5;
  if (u1.hi < 1e-4f) {
    f1 = ff_series_f(u1);
  } else {
    const double A = double(a.z[0]), B = double(b.z[0]);
    f1 = ff(0.5 * (A + B) * ::log(A / B) / (A - B));
  }
  if (u5.hi < 1e-4f) {
    g5 = ff_series_g(u5);
  } else {
    const double A = double(a.z[4]), B = double(b.z[4]);
    g5 = ff(0.5 * (A - B) / ((A + B) * ::log(A / B)));
  }
  const ff rho_hat = P15 * g5;
  const ff u0 = (a.z[1] + b.z[1]) * inv1;
  const ff uy = (a.z[2] + b.z[2]) * inv1;
  const ff uz = (a.z[3] + b.z[3]) * inv1;
  const ff p1 = S5 * inv1;
  const ff p2g = p1 * (C.C1x * (g5 * f1) + C.C2x);
  const ff um = m == 0 ? u0 : (m == 1 ? uy : uz);
  const ff mass = rho_hat * um;
  const ff q2 = u0 * u0 + uy * uy + uz * uz;
  f[0] = mass;
  f[1] = mass * u0;
  f[2] = mass * uy;
  f[3] = mass * uz;
  // constant indices keep f in registers (m is a run-time value)
  if (m == 0) f[1] += p1;
  else if (m == 1) f[2] += p1;
  else f[3] += p1;
  f[4] = um * p2g + ff(0.5f * mass.hi, 0.5f * mass.lo) * q2;
}

// Conserved state from the parameter vector and iz1 = 1/z1 = sqrt(p/rho):
// rho = z1 z5, v = z_{2..4}/z1, p = z5/z1, c = sqrt(gam)/z1.
template <typename T>
__device__ __forceinline__ void z_to_q(const Zstate<T>& s, T iz1, const FluxConst<T>& C, T q[5], T& vn_abs_plus_c,
                                       int m) {
  const T rho = s.z[0] * s.z[4];
  const T v0 = s.z[1] * iz1, v1 = s.z[2] * iz1, v2 = s.z[3] * iz1;
  const T p = s.z[4] * iz1;
  q[0] = rho;
  q[1] = rho * v0;
  q[2] = rho * v1;
  q[3] = rho * v2;
  q[4] = p * C.inv_gm1 + T(0.5) * rho * (v0 * v0 + v1 * v1 + v2 * v2);
  const T vm = m == 0 ? v0 : (m == 1 ? v1 : v2);
  vn_abs_plus_c = fabs(vm) + C.sqrt_gam * iz1;
}

// Entropy variables from the parameter vector:
// w = ((gam - s)/(gam-1) - |zv|^2/2, z1 zv, -z1^2), s = -(gam+1) ln z1 - (gam-1) ln z5.
// w_2..w_5 need no logarithm (the viscous terms use only those).
template <typename T>
__device__ __forceinline__ void z_to_wv(const Zstate<T>& s, T w[4]) {
  w[0] = s.z[0] * s.z[1];
  w[1] = s.z[0] * s.z[2];
  w[2] = s.z[0] * s.z[3];
  w[3] = -s.z[0] * s.z[0];
}
template <typename T>
__device__ __forceinline__ void z_to_w(const Zstate<T>& s, const FluxConst<T>& C, T w[5]) {
  const T sp = -(C.gam + T(1)) * log(s.z[0]) - (C.gam - T(1)) * log(s.z[4]);
  w[0] = (C.gam - sp) * C.inv_gm1 - T(0.5) * (s.z[1] * s.z[1] + s.z[2] * s.z[2] + s.z[3] * s.z[3]);
  z_to_wv(s, w + 1);
}

// ---------------------------------------------------------------------------
// log(1 + z) - z without cancellation.
// |z| <= 1e-3: Taylor series -z^2/2 + z^3/3 - ... + z^7/7 (the first omitted
//   term is below 2.5e-19 of the result).
// |z| <= 0.1: with t = z/(2+z), log1p(z) = 2 atanh(t) = 2 (t + t^3/3 + ...) and
//   z = 2t/(1-t), so log1p(z) - z = -t z + 2 t^3 (1/3 + t^2/5 + t^4/7 + ...);
//   |t| < 0.053 and eight terms of the even series reach 1e-17 relative.
// otherwise the direct difference (cancellation costs at most a factor 20).
__device__ __forceinline__ double log1pmx(double z) {
  if (abs_le(z, 1e-3)) {
    double s = 1.0 / 7.0;
    s = fma(s, z, -1.0 / 6.0);
    s = fma(s, z, 1.0 / 5.0);
    s = fma(s, z, -1.0 / 4.0);
    s = fma(s, z, 1.0 / 3.0);
    s = fma(s, z, -0.5);
    return z * z * s;
  }
  if (abs_le(z, 0.1)) {
    const double t = z * fast_rcp(2.0 + z);
    const double t2 = t * t;
    double s = 1.0 / 17.0;
    s = s * t2 + 1.0 / 15.0;
    s = s * t2 + 1.0 / 13.0;
    s = s * t2 + 1.0 / 11.0;
    s = s * t2 + 1.0 / 9.0;
    s = s * t2 + 1.0 / 7.0;
    s = s * t2 + 1.0 / 5.0;
    s = s * t2 + 1.0 / 3.0;
    return -t * z + 2.0 * t * t2 * s;
  }
  return log1p(z) - z;
}

// Per-node inputs of the relaxation function (see the relaxation kernel):
// X0 = d_rho/rho, Y0 = linearised d_p/p, V2 = rho |d_v|^2/p, c = P_n rho.
struct RelaxNode {
  double X0, Y0, V2, c;
};

// D_breg/rho at gamma and its gamma-derivative for one node:
//   x = g X0, K = g^2 V2/(2(1+x)), y = g Y0 - (gam-1) K,
//   D/rho = [gam phi(x) + psi(y) - x log1p(y)]/(gam-1) + K,
//   phi(x) = (1+x) log1p(x) - x, psi(y) = y - log1p(y);
//   d/dg (D/rho) = [X0 (gam log1p(x) - log1p(y)) + y' (y - x)/(1+y)]/(gam-1) + K',
//   K' = g V2/(1+x) (1 - x/(2(1+x))), y' = Y0 - (gam-1) K'.
// One division serves 1/(1+x) and 1/(1+y): with Yb = g Y0 (1+x) - (gam-1) g^2 V2/2,
// y = Yb/(1+x) and 1+y = (1+x+Yb)/(1+x).
// Returns false if the state at gamma is not physical (1+x <= 0 or 1+y <= 0).
__device__ __forceinline__ bool relax_node_eval(const RelaxNode& nd, double g, double gam, double inv_gm1,
                                                double& D, double& dD) {
  const double x = g * nd.X0;
  const double opx = 1.0 + x;
  const double K0 = 0.5 * g * g * nd.V2;
  const double Yb = g * nd.Y0 * opx - (gam - 1.0) * K0;
  const double opy_n = opx + Yb;  // (1+y)(1+x)
  if (!(opx > 0.0) || !(opy_n > 0.0)) return false;
  const double inv = fast_rcp(opx * opy_n);
  const double q = opy_n * inv;        // 1/(1+x)
  const double iy = opx * opx * inv;   // 1/(1+y)
  const double y = Yb * q;
  const double K = K0 * q;
  const double Lx = log1pmx(x), Ly = log1pmx(y);
  const double l1px = x + Lx, l1py = y + Ly;
  const double phi = opx * Lx + x * x;
  D = (gam * phi - Ly - x * l1py) * inv_gm1 + K;
  const double dK = g * nd.V2 * q * (1.0 - 0.5 * x * q);
  const double dy = nd.Y0 - (gam - 1.0) * dK;
  dD = (nd.X0 * (gam * l1px - l1py) + dy * (y - x) * iy) * inv_gm1 + dK;
  return true;
}

// ---------------------------------------------------------------------------
// warp reductions (butterfly: every lane ends with the same sum/min)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// positive doubles (and +inf) order like their bit patterns as unsigned integers
__device__ __forceinline__ void atomic_min_positive(unsigned long long* addr, double v) {
  atomicMin(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace es

// C ABI of the locally relaxed entropy-stable RK step (declared in include/es.h).
//
// Host side: LGL/SBP tables (Section 3.1), the Butcher tableaux named in
// Section 4, the context's device workspace, and the launch sequence of one
// relaxed step: for each stage i, k_prep -> k_face -> [k_grad] -> k_volume
// (Eq. (RK-step), Eq. (compressible_ns_diss)); then k_relax (gamma_kappa,
// Eq. (relaxation-local-gamma)), k_scalar (gamma = min_kappa gamma_kappa,
// Theorem 2.3; t += gamma dt, Eq. (t-n-gamma)); the relaxed update
// u += gamma d is fused into the next step's first k_prep.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/es.h"
#include "es_launch.h"

using namespace es;

// ---------------------------------------------------------------------------
// LGL nodes/weights and the SBP derivative (textbook definitions):
// nodes = +-1 and the roots of P_p', omega_i = 2/(p(p+1) P_p(x_i)^2),
// D_ij = P_p(x_i)/(P_p(x_j)(x_i - x_j)) (i != j), D_00 = -p(p+1)/4, D_pp = p(p+1)/4.
namespace {

void legendre_eval(int p, double x, double* Pp, double* Pm) {
  double a = 1.0, b = x;
  if (p == 0) { *Pp = 1.0; *Pm = 0.0; return; }
  for (int n = 1; n < p; ++n) {
    const double c = ((2 * n + 1) * x * b - n * a) / (n + 1);
    a = b;
    b = c;
  }
  *Pp = b;  // P_p
  *Pm = a;  // P_{p-1}
}

void lgl_tables(int p, double* x, double* w, double* D) {
  const int n = p + 1;
  for (int i = 0; i < n; ++i) x[i] = -std::cos(M_PI * i / p);
  // Newton on g(x) = p (P_{p-1}(x) - x P_p(x)) = (1 - x^2) P_p'(x), g'(x) = -p (p+1) P_p(x)
  for (int i = 1; i < p; ++i) {
    double xi = x[i];
    for (int it = 0; it < 100; ++it) {
      double Pp, Pm;
      legendre_eval(p, xi, &Pp, &Pm);
      const double g = p * (Pm - xi * Pp);
      const double dg = -p * (p + 1) * Pp;
      const double step = g / dg;
      xi -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    x[i] = xi;
  }
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 0; i <= p / 2; ++i) {  // exact symmetry of the node set
    const double s = 0.5 * (x[p - i] - x[i]);
    x[i] = -s;
    x[p - i] = s;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
  double Pv[kMaxP1];
  for (int i = 0; i < n; ++i) {
    double Pm;
    legendre_eval(p, x[i], &Pv[i], &Pm);
    w[i] = 2.0 / (p * (p + 1) * Pv[i] * Pv[i]);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) D[i * n + j] = (i == j) ? 0.0 : Pv[i] / (Pv[j] * (x[i] - x[j]));
  D[0] = -p * (p + 1) / 4.0;
  D[p * n + p] = p * (p + 1) / 4.0;
}

// Butcher tableaux (Section 4 names BSRK(4,3), RK(4,4) and, for p = 4, 5, BSRK(8,5)
// and VRK(9,6), whose coefficients it does not print).
struct Tableau {
  int s;          // stages entering u_new (trailing stages with b_i = 0 dropped)
  double a[kMaxStages][kMaxStages];
  double b[kMaxStages];
  double c[kMaxStages];  // stage times (boundary states are evaluated at t + c_i dt)
};

Tableau tableau(int rk) {
  Tableau t;
  std::memset(&t, 0, sizeof(t));
  if (rk == ES_RK_BS3) {  // Bogacki & Shampine 3(2); b_4 = 0 so stage 4 is not needed
    t.s = 3;
    t.a[1][0] = 0.5;
    t.a[2][1] = 0.75;
    t.c[1] = 0.5;
    t.c[2] = 0.75;
    t.b[0] = 2.0 / 9.0;
    t.b[1] = 1.0 / 3.0;
    t.b[2] = 4.0 / 9.0;
  } else if (rk == ES_RK_RK65) {  // Butcher's six-stage fifth-order method, b_i >= 0
    t.s = 6;
    t.a[1][0] = 0.25;
    t.a[2][0] = 0.125;
    t.a[2][1] = 0.125;
    t.a[3][1] = -0.5;
    t.a[3][2] = 1.0;
    t.a[4][0] = 3.0 / 16.0;
    t.a[4][3] = 9.0 / 16.0;
    t.a[5][0] = -3.0 / 7.0;
    t.a[5][1] = 2.0 / 7.0;
    t.a[5][2] = 12.0 / 7.0;
    t.a[5][3] = -12.0 / 7.0;
    t.a[5][4] = 8.0 / 7.0;
    t.c[1] = 0.25;
    t.c[2] = 0.25;
    t.c[3] = 0.5;
    t.c[4] = 0.75;
    t.c[5] = 1.0;
    t.b[0] = 7.0 / 90.0;
    t.b[2] = 32.0 / 90.0;
    t.b[3] = 12.0 / 90.0;
    t.b[4] = 32.0 / 90.0;
    t.b[5] = 7.0 / 90.0;
  } else {  // classical RK(4,4)
    t.s = 4;
    t.a[1][0] = 0.5;
    t.a[2][1] = 0.5;
    t.a[3][2] = 1.0;
    t.c[1] = 0.5;
    t.c[2] = 0.5;
    t.c[3] = 1.0;
    t.b[0] = 1.0 / 6.0;
    t.b[1] = 1.0 / 3.0;
    t.b[2] = 1.0 / 3.0;
    t.b[3] = 1.0 / 6.0;
  }
  return t;
}

}  // namespace


namespace es {

// Argument checks shared by every entry point that takes an es_config.
int validate_config(const es_config& C) {
  if (C.p < 2 || C.p > 5 || C.nx < 1 || C.ny < 1 || C.nz < 1) return ES_ERR_INVALID;
  if (!(C.gamma_gas > 1.0) || !(C.R > 0.0) || C.mu < 0.0 || (C.mu > 0.0 && !(C.Pr > 0.0))) return ES_ERR_INVALID;
  if (C.rk != ES_RK_BS3 && C.rk != ES_RK_RK4 && C.rk != ES_RK_RK65) return ES_ERR_INVALID;
  if (C.precision < ES_FP64 || C.precision > ES_MIXED_FF) return ES_ERR_INVALID;
  if (!(C.visc_diss >= 0.0) || !std::isfinite(C.visc_diss)) return ES_ERR_INVALID;
  if (C.relax != ES_RELAX_NONE && C.relax != ES_RELAX_LOCAL && C.relax != ES_RELAX_GLOBAL) return ES_ERR_INVALID;
  if (C.interface_diss < 0 || C.interface_diss > 2) return ES_ERR_INVALID;
  if (!(C.root_rtol >= 0.0) || !(C.root_rtol < 1.0)) return ES_ERR_INVALID;
  for (int m = 0; m < 3; ++m)
    if (!(C.hi[m] > C.lo[m])) return ES_ERR_INVALID;
  const long long K = (long long)C.nx * C.ny * C.nz;
  if (K > (1LL << 30)) return ES_ERR_INVALID;
  return ES_OK;
}

// Geometry of the instance described by C, its first element at off.
InstGeom instance_geom(const es_config& C, int off) {
  InstGeom g;
  g.nx = C.nx;
  g.ny = C.ny;
  g.nz = C.nz;
  g.off = off;
  double h[3];
  for (int m = 0; m < 3; ++m) {
    const int nm = m == 0 ? C.nx : (m == 1 ? C.ny : C.nz);
    h[m] = (C.hi[m] - C.lo[m]) / nm;
    g.metric[m] = 2.0 / h[m];
  }
  g.J = h[0] * h[1] * h[2] / 8.0;
  g.dt = 0.0;
  return g;
}

// Kernel parameters (LGL/SBP tables, metric, gas constants) of a configuration; host only,
// no allocation.
void build_params(const es_config& C, Params* out) {
  Params& P = *out;
  std::memset(&P, 0, sizeof(P));
  const int P1 = C.p + 1;
  double x[kMaxP1], w[kMaxP1], D[kMaxP1 * kMaxP1];
  lgl_tables(C.p, x, w, D);
  for (int i = 0; i < P1; ++i) {
    P.omega[i] = w[i];
    const ff wf(w[i]);
    P.omega_ff[0][i] = wf.hi;
    P.omega_ff[1][i] = wf.lo;
    for (int j = 0; j < P1; ++j) {
      P.D[i * P1 + j] = D[i * P1 + j];
      P.D2[i * P1 + j] = (i == j) ? 0.0 : 2.0 * D[i * P1 + j];
      const ff d1(P.D[i * P1 + j]), d2(P.D2[i * P1 + j]);
      P.Dff[0][i * P1 + j] = d1.hi;
      P.Dff[1][i * P1 + j] = d1.lo;
      P.D2ff[0][i * P1 + j] = d2.hi;
      P.D2ff[1][i * P1 + j] = d2.lo;
    }
  }
  P.inv_omega_end = 1.0 / w[0];
  P.gam = C.gamma_gas;
  P.mu = C.mu;
  P.R = C.R;
  P.inv_R = 1.0 / C.R;
  P.Cd = FluxConst<double>::make(C.gamma_gas);
  P.Cf = FluxConst<float>::make(C.gamma_gas);
  P.Cff = FluxConst<ff>::make(C.gamma_gas);
  P.kappa_heat = C.mu > 0.0 ? C.mu * C.gamma_gas * C.R / ((C.gamma_gas - 1.0) * C.Pr) : 0.0;
  P.K = C.nx * C.ny * C.nz;
  P.diss = C.interface_diss;
  P.p1 = P1;
  P.ninst = 1;
  P.ff_est = (C.precision == ES_MIXED_FF || C.precision == ES_FP64X) ? 1 : 0;
  P.visc_pen = C.mu > 0.0 ? C.visc_diss : 0.0;
  P.g0 = instance_geom(C, 0);
  P.geom = nullptr;
  P.elem_inst = nullptr;
}

int grid_for_sms(int sm_count, long long n, int block) {
  long long g = (n + block - 1) / block;
  const long long cap = (long long)sm_count * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// double -> float-float with the device split's result (ff_from_double): in its fast
// range (2^-74 <= |d| < 2^127, and zero) hi = d truncated to 24 significand bits and lo
// the remainder rounded once; elsewhere hi = fl32(d), lo = fl32(d - hi)
void ff_split_host(double d, float out[2]) {
  uint64_t b;
  std::memcpy(&b, &d, sizeof(b));
  const unsigned e = unsigned(b >> 52) & 0x7FFu;
  if (e - 949u < 202u || (b << 1) == 0) {
    const uint64_t bt = b & ~((uint64_t(1) << 29) - 1);
    double h;
    std::memcpy(&h, &bt, sizeof(h));
    out[0] = float(h);         // exact: 24 significand bits in range
    out[1] = float(d - h);     // d - h exact; one rounding
  } else {
    out[0] = float(d);
    out[1] = float(d - double(out[0]));
  }
}

}  // namespace es

// ---------------------------------------------------------------------------
// A group: instances sharing the LGL degree and the physics, stored as one SoA
// over the group's elements.  The single-instance context is a group of one;
// a batch is one group per degree.
// Dirichlet-penalty boundary data of a context (host copy; passed to k_bc_eval by value)
struct BcSpec {
  int kind[3];           // ES_BC_* per direction
  double q[3][2][5];     // ES_BC_STATE: exterior states (left, right)
  double vs[3][6];       // ES_BC_VISCOUS_SHOCK: V_f, alpha, H, speed, x_lo, x_hi
  double gam;
};

struct Group {
  es_config cfg;  // physics (and, for a context, the mesh)
  int P1 = 0, Np = 0, K = 0, ninst = 0;
  long long N = 0;
  size_t tf = 8;  // bytes per flux value (8 FP64 and float-float, 4 mixed)
  bool ffx = false;  // float-float flux arithmetic (ES_FP64X)
  Params P;
  int vol_variant = 0;
  std::vector<InstGeom> geom;      // host copy of the instance table
  std::vector<int> inst_ids;       // batch instance index of each local instance
  void* k[kMaxStages] = {};  // stage values, tf bytes each
  int nk = 0;                // allocated stage buffers
  void* aux = nullptr;
  void* F = nullptr;
  void* fV = nullptr;
  double* dw = nullptr;
  double* d = nullptr;
  double* A = nullptr;
  double* gamma_elem = nullptr;
  double* gamma_cur = nullptr;           // [ninst]
  unsigned long long* gmin = nullptr;    // [ninst]
  int* pending = nullptr;                // [ninst]
  double* t = nullptr;                   // [ninst] (batch)
  double* q = nullptr;                   // group-owned state (batch)
  double* gwork = nullptr;               // global relaxation: [4][K] element sums
  GlobalRelaxState* gstate = nullptr;    // global relaxation: [ninst]
  InstGeom* geom_dev = nullptr;
  int* elem_inst_dev = nullptr;
  BcSpec bc;                             // boundary kinds and data (contexts only)
  bool any_bc = false;
  void* FL = nullptr;                    // -x_m boundary-face fluxes (tf bytes each)
  double* bcz = nullptr;                 // [3][2][kBcVals] exterior values at the stage time
  double* est = nullptr;                 // batch estimate step: eta_old, deta, eta_new [3][K]
  int* nbr = nullptr;                    // [K][6] periodic neighbours (Params::nbr)
};

// The volume kernel with on-chip interface fluxes serves FP32 fluxes (ES_MIXED, ES_MIXED_FF)
// on periodic Euler groups.
bool stage_fusable(const Group& g) { return g.tf == 4 && g.cfg.mu == 0.0 && !g.any_bc; }
bool stage_fused(const Group& g) { return g.vol_variant >= kVolumeVariants && stage_fusable(g); }

// Launch bookkeeping shared by a context or a batch.
struct Engine {
  int device = 0, sm_count = 0;
  int* status = nullptr;
  Tableau tab;
  int relax = 1;
  long long launches = 0;
  bool capturing = false;
  bool profiling = false;
  struct Mark { int kind; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  double prof_ms[ES_KERNEL_COUNT] = {0};
  long long prof_n[ES_KERNEL_COUNT] = {0};
};

struct es_ctx {
  Engine eng;
  Group g;
  double* q_host_dev = nullptr;
  double* t_host_dev = nullptr;
  double* hist_host_dev = nullptr;
  int hist_cap = 0;
};

struct es_batch {
  Engine eng;
  std::vector<Group> groups;
  std::vector<std::pair<int, int>> where;  // instance -> (group, local instance)
  std::vector<es_config> cfgs;
  std::vector<cudaStream_t> side;          // one stream per group for graph capture
  std::vector<cudaEvent_t> fork, join;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t exec_stream = nullptr;
  long long kernels_per_step = 0;
};

namespace {

int cuda_check(cudaError_t e) {
  if (e != cudaSuccess) {
    std::fprintf(stderr, "es: CUDA error %s\n", cudaGetErrorString(e));
    return ES_ERR_CUDA;
  }
  return ES_OK;
}

int last_launch_error() { return cuda_check(cudaGetLastError()); }

template <typename T>
int dev_alloc(T** p, size_t count) {
  if (count == 0) { *p = nullptr; return ES_OK; }
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); return ES_ERR_NOMEM; }
  return ES_OK;
}

int dev_alloc_bytes(void** p, size_t bytes) {
  if (bytes == 0) { *p = nullptr; return ES_OK; }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); return ES_ERR_NOMEM; }
  return ES_OK;
}

template <typename F>
int dispatch(const Group& g, F&& f) {
  switch (g.P1) {
    case 3: return g.tf == 4 ? f(Launcher<3, float>()) : g.ffx ? f(Launcher<3, ff>()) : f(Launcher<3, double>());
    case 4: return g.tf == 4 ? f(Launcher<4, float>()) : g.ffx ? f(Launcher<4, ff>()) : f(Launcher<4, double>());
    case 5: return g.tf == 4 ? f(Launcher<5, float>()) : g.ffx ? f(Launcher<5, ff>()) : f(Launcher<5, double>());
    case 6: return g.tf == 4 ? f(Launcher<6, float>()) : g.ffx ? f(Launcher<6, ff>()) : f(Launcher<6, double>());
  }
  return ES_ERR_INVALID;
}

int engine_init(Engine& e, const es_config& C) {
  if (cudaGetDevice(&e.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&e.sm_count, cudaDevAttrMultiProcessorCount, e.device) != cudaSuccess) {
    cudaGetLastError();
    return ES_ERR_CUDA;
  }
  e.tab = tableau(C.rk);
  e.relax = C.relax;
  int rc = dev_alloc(&e.status, 1);
  if (rc == ES_OK) rc = cuda_check(cudaMemset(e.status, 0, sizeof(int)));
  return rc;
}

void engine_free(Engine& e) {
  for (auto& m : e.marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto ev : e.pool) cudaEventDestroy(ev);
  e.marks.clear();
  e.pool.clear();
  cudaFree(e.status);
  e.status = nullptr;
}

cudaEvent_t take_event(Engine& e) {
  if (!e.pool.empty()) {
    cudaEvent_t ev = e.pool.back();
    e.pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  if (cudaEventCreate(&ev) != cudaSuccess) {  // no event: that launch goes untimed
    cudaGetLastError();
    return nullptr;
  }
  return ev;
}

// Folds recorded event pairs into the per-kind totals (synchronises the device).
void flush_marks(Engine& e) {
  if (e.marks.empty()) return;
  cudaDeviceSynchronize();
  for (auto& m : e.marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      e.prof_ms[m.kind] += ms;
      e.prof_n[m.kind] += 1;
    }
    e.pool.push_back(m.a);
    e.pool.push_back(m.b);
  }
  e.marks.clear();
  cudaGetLastError();
}

// Brackets one launch with events when profiling is on (not while capturing a graph).
template <typename Fn>
void timed(Engine& e, int kind, cudaStream_t st, Fn&& fn) {
  e.launches += 1;
  if (!e.profiling || e.capturing) {
    fn();
    return;
  }
  if (e.marks.size() >= 4096) flush_marks(e);
  Engine::Mark m{kind, take_event(e), take_event(e)};
  if (!m.a || !m.b) {
    if (m.a) e.pool.push_back(m.a);
    if (m.b) e.pool.push_back(m.b);
    fn();
    return;
  }
  cudaEventRecord(m.a, st);
  fn();
  cudaEventRecord(m.b, st);
  e.marks.push_back(m);
}

void group_free(Group& g) {
  for (auto& p : g.k) cudaFree(p);
  cudaFree(g.aux);
  cudaFree(g.F);
  cudaFree(g.fV);
  cudaFree(g.dw);
  cudaFree(g.d);
  cudaFree(g.A);
  cudaFree(g.gamma_elem);
  cudaFree(g.gamma_cur);
  cudaFree(g.gmin);
  cudaFree(g.pending);
  cudaFree(g.t);
  cudaFree(g.q);
  cudaFree(g.gwork);
  cudaFree(g.gstate);
  cudaFree(g.geom_dev);
  cudaFree(g.elem_inst_dev);
  cudaFree(g.FL);
  cudaFree(g.bcz);
  cudaFree(g.est);
  cudaFree(g.nbr);
  g = Group();
}

// A caller's explicit tableau (es_set_tableau, es_batch_set_tableau): a[i*s + j] strictly
// lower triangular, sum_j a_ij = c_i, sum_i b_i = 1, b_i >= 0 when relaxing (Eq.
// (eta-est-1-RK)); trailing stages with b_i = 0 dropped.
int parse_tableau(int relax, int s, const double* a, const double* b, const double* cs, Tableau* out) {
  if (!a || !b || !cs || !out || s < 1 || s > kMaxStages) return ES_ERR_INVALID;
  Tableau t;
  std::memset(&t, 0, sizeof(t));
  double bsum = 0.0;
  for (int i = 0; i < s; ++i) {
    double row = 0.0;
    for (int j = 0; j < s; ++j) {
      const double v = a[i * s + j];
      if (!std::isfinite(v) || (j >= i && v != 0.0)) return ES_ERR_INVALID;
      if (j < i) t.a[i][j] = v;
      row += v;
    }
    if (!std::isfinite(b[i]) || !std::isfinite(cs[i])) return ES_ERR_INVALID;
    if (relax != ES_RELAX_NONE && b[i] < 0.0) return ES_ERR_INVALID;
    if (std::fabs(row - cs[i]) > 1e-13 * (1.0 + std::fabs(cs[i]))) return ES_ERR_INVALID;
    t.b[i] = b[i];
    t.c[i] = cs[i];
    bsum += b[i];
  }
  if (std::fabs(bsum - 1.0) > 1e-13) return ES_ERR_INVALID;
  int se = s;
  while (se > 0 && t.b[se - 1] == 0.0) --se;
  t.s = se;
  *out = t;
  return ES_OK;
}

// Stage buffers for an s-stage tableau (allocated on first need, kept).
int ensure_stage_buffers(Group& g, int s) {
  for (int i = g.nk; i < s; ++i) {
    const int rc = dev_alloc_bytes(&g.k[i], 5 * g.N * g.tf);
    if (rc != ES_OK) return rc;
    g.nk = i + 1;
  }
  return ES_OK;
}

// Allocates a group for the instances `insts` (same degree and physics).
int group_init(Group& g, const es_config* insts, int n, int stages, bool own_state) {
  const es_config& C = insts[0];
  g.cfg = C;
  g.P1 = C.p + 1;
  g.Np = g.P1 * g.P1 * g.P1;
  g.ninst = n;
  g.tf = (C.precision == ES_MIXED || C.precision == ES_MIXED_FF) ? 4 : 8;  // bytes per flux value (float-float: 8)
  g.ffx = C.precision == ES_FP64X;
  build_params(C, &g.P);
  long long K = 0;
  g.geom.resize(n);
  for (int i = 0; i < n; ++i) {
    g.geom[i] = instance_geom(insts[i], (int)K);
    K += (long long)insts[i].nx * insts[i].ny * insts[i].nz;
  }
  if (K > (1LL << 30)) return ES_ERR_INVALID;
  g.K = (int)K;
  g.N = K * g.Np;
  g.P.K = g.K;
  g.P.ninst = n;
  g.P.g0 = g.geom[0];
  const long long N = g.N;
  const long long P2 = (long long)g.P1 * g.P1;
  int rc = ES_OK;
  for (int i = 0; i < stages && rc == ES_OK; ++i) rc = dev_alloc_bytes(&g.k[i], 5 * N * g.tf);
  if (rc == ES_OK) g.nk = stages;
  if (rc == ES_OK) rc = dev_alloc_bytes(&g.aux, kAuxPlanes * N * g.tf);
  if (rc == ES_OK) rc = dev_alloc_bytes(&g.F, 15 * K * P2 * g.tf);
  if (rc == ES_OK && C.mu > 0.0) rc = dev_alloc_bytes(&g.fV, 12 * N * g.tf);
  if (rc == ES_OK) rc = dev_alloc(&g.dw, 5 * N);
  if (rc == ES_OK) rc = dev_alloc(&g.d, 5 * N);
  if (rc == ES_OK) rc = dev_alloc(&g.A, K);
  if (rc == ES_OK) rc = dev_alloc(&g.gamma_elem, K);
  if (rc == ES_OK) rc = dev_alloc(&g.gamma_cur, n);
  if (rc == ES_OK) rc = dev_alloc(&g.gmin, n);
  if (rc == ES_OK) rc = dev_alloc(&g.pending, n);
  if (rc == ES_OK) rc = dev_alloc(&g.t, n);
  if (rc == ES_OK && own_state) rc = dev_alloc(&g.q, 5 * N);
  if (rc == ES_OK && C.relax == ES_RELAX_GLOBAL) rc = dev_alloc(&g.gwork, 4 * K);
  if (rc == ES_OK && C.relax == ES_RELAX_GLOBAL) rc = dev_alloc(&g.gstate, n);
  if (rc == ES_OK && C.relax == ES_RELAX_GLOBAL) rc = cuda_check(cudaMemset(g.gstate, 0, n * sizeof(GlobalRelaxState)));
  if (rc == ES_OK) rc = cuda_check(cudaMemset(g.pending, 0, n * sizeof(int)));
  if (rc == ES_OK) rc = cuda_check(cudaMemset(g.gamma_cur, 0, n * sizeof(double)));
  if (rc == ES_OK) rc = cuda_check(cudaMemset(g.t, 0, n * sizeof(double)));
  if (rc == ES_OK && own_state) rc = cuda_check(cudaMemset(g.q, 0, 5 * N * sizeof(double)));
  if (rc == ES_OK && own_state) {  // batches: device instance tables (dt can change without re-capture)
    std::vector<int> ei(K);
    for (int i = 0; i < n; ++i) {
      const long long Ki = (long long)insts[i].nx * insts[i].ny * insts[i].nz;
      for (long long e = 0; e < Ki; ++e) ei[g.geom[i].off + e] = i;
    }
    rc = dev_alloc(&g.geom_dev, n);
    if (rc == ES_OK) rc = dev_alloc(&g.elem_inst_dev, K);
    if (rc == ES_OK) rc = cuda_check(cudaMemcpy(g.geom_dev, g.geom.data(), n * sizeof(InstGeom), cudaMemcpyHostToDevice));
    if (rc == ES_OK) rc = cuda_check(cudaMemcpy(g.elem_inst_dev, ei.data(), K * sizeof(int), cudaMemcpyHostToDevice));
    g.P.geom = g.geom_dev;
    g.P.elem_inst = g.elem_inst_dev;
  }
  if (rc == ES_OK) {  // periodic neighbour table: the kernels look neighbours up instead of dividing
    std::vector<int> nb(size_t(K) * 6);
    for (int i = 0; i < n; ++i) {
      const InstGeom& G = g.geom[i];
      const int dims[3] = {G.nx, G.ny, G.nz};
      for (int ez = 0; ez < G.nz; ++ez)
        for (int ey = 0; ey < G.ny; ++ey)
          for (int ex = 0; ex < G.nx; ++ex) {
            const int c[3] = {ex, ey, ez};
            const long long e = G.off + ex + (long long)G.nx * (ey + (long long)G.ny * ez);
            for (int m = 0; m < 3; ++m)
              for (int side = 0; side < 2; ++side) {
                int d[3] = {c[0], c[1], c[2]};
                d[m] = (d[m] + (side ? 1 : -1) + dims[m]) % dims[m];
                nb[e * 6 + m * 2 + side] = G.off + d[0] + G.nx * (d[1] + G.ny * d[2]);
              }
          }
    }
    rc = dev_alloc(&g.nbr, size_t(K) * 6);
    if (rc == ES_OK) rc = cuda_check(cudaMemcpy(g.nbr, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice));
    g.P.nbr = g.nbr;
  }
  if (rc == ES_OK) {  // gamma accumulators start at +inf, no update pending
    launch_reset(g.gmin, g.pending, n, nullptr);
    rc = cuda_check(cudaDeviceSynchronize());
  }
  if (rc == ES_OK) rc = dispatch(g, [&](auto L) { return cuda_check(decltype(L)::volume_setup()); });
  if (rc == ES_OK) rc = dispatch(g, [&](auto L) { return cuda_check(decltype(L)::volface_setup()); });
  return rc;
}

// Exterior values of the Dirichlet-penalty boundaries at time *t + t_off: one thread per
// (direction, side).  ES_BC_VISCOUS_SHOCK evaluates the Section 4.1.2 profile: V in
// (V_f, 1) solves x - speed t = (alpha/2) [log((1-V)(V-V_f)) + (1+V_f)/(1-V_f)
// log((1-V)/(V-V_f))] (bisection to the last bit), u = V, rho = 1/V, p from the constant
// total enthalpy H, lab velocity u + speed along the direction.
__global__ void k_bc_eval(BcSpec spec, const double* t, double t_off, double* out) {
  const int i = threadIdx.x;
  if (i >= 6) return;
  const int m = i / 2, side = i % 2;
  if (spec.kind[m] == ES_BC_PERIODIC) return;
  const double g = spec.gam;
  double q[5];
  if (spec.kind[m] == ES_BC_STATE) {
    for (int v = 0; v < 5; ++v) q[v] = spec.q[m][side][v];
  } else {
    const double vf = spec.vs[m][0], alpha = spec.vs[m][1], H = spec.vs[m][2], speed = spec.vs[m][3];
    const double time = (t ? t[0] : 0.0) + t_off;
    const double xi = spec.vs[m][4 + side] - speed * time;
    const double c = (1.0 + vf) / (1.0 - vf);
    double lo = vf, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      const double x = 0.5 * alpha * (log((1.0 - mid) * (mid - vf)) + c * log((1.0 - mid) / (mid - vf)));
      if (x > xi) lo = mid;
      else hi = mid;
    }
    const double u = 0.5 * (lo + hi);
    const double rho = 1.0 / u;
    const double p = (g - 1.0) / g * rho * (H - 0.5 * u * u);
    const double ul = u + speed;
    for (int v = 0; v < 5; ++v) q[v] = 0.0;
    q[0] = rho;
    q[1 + m] = rho * ul;
    q[4] = p / (g - 1.0) + 0.5 * rho * ul * ul;
  }
  const double rho = q[0];
  const double v0 = q[1] / rho, v1 = q[2] / rho, v2 = q[3] / rho;
  const double p = (g - 1.0) * (q[4] - 0.5 * rho * (v0 * v0 + v1 * v1 + v2 * v2));
  const double z1 = sqrt(rho / p);
  double* o = out + i * kBcVals;
  o[0] = z1;
  o[1] = z1 * v0;
  o[2] = z1 * v1;
  o[3] = z1 * v2;
  o[4] = sqrt(rho * p);
  o[5] = sqrt(p / rho);
  o[6] = rho * v0 / p;
  o[7] = rho * v1 / p;
  o[8] = rho * v2 / p;
  o[9] = -rho / p;
}

void launch_bc_eval(const BcSpec& spec, const double* t, double t_off, double* out, cudaStream_t st) {
  k_bc_eval<<<1, 32, 0, st>>>(spec, t, t_off, out);
}

int grid_for(const Engine& e, long long n, int block) { return grid_for_sms(e.sm_count, n, block); }

// One stage's right-hand side into kout or d (+ element sums), on state u (+ pending
// update) + dt sum_j coef[j] k[j].  With a fused variant (stage_fused) the volume kernel
// forms the interface fluxes itself and k_face is not launched.
int run_stage(Engine& E, Group& g, const StagePrep& sp, const StageVol& sv, cudaStream_t st,
              const double* t_dev = nullptr, double t_off = 0.0) {
  const bool ns = g.cfg.mu != 0.0;
  if (stage_fused(g)) {
    return dispatch(g, [&](auto L) {
      using Lc = decltype(L);
      timed(E, ES_KERNEL_PREP, st, [&] { Lc::prep(g.P, sp, g.aux, E.status, st, grid_for(E, g.N, 256)); });
      timed(E, ES_KERNEL_VOLUME, st,
            [&] { Lc::volface(g.P, sv, g.aux, st, g.vol_variant - kVolumeVariants); });
      return last_launch_error();
    });
  }
  if (g.any_bc) {  // exterior states at this stage's time t + c_i dt
    timed(E, ES_KERNEL_OTHER, st, [&] { launch_bc_eval(g.bc, t_dev ? t_dev : g.t, t_off, g.bcz, st); });
  }
  return dispatch(g, [&](auto L) {
    using Lc = decltype(L);
    timed(E, ES_KERNEL_PREP, st, [&] { Lc::prep(g.P, sp, g.aux, E.status, st, grid_for(E, g.N, 256)); });
    timed(E, ES_KERNEL_FACE, st,
          [&] { Lc::face(g.P, g.aux, g.F, g.FL, st, grid_for(E, 3LL * g.K * g.P1 * g.P1, 256)); });
    if (ns) timed(E, ES_KERNEL_GRAD, st, [&] { Lc::grad(g.P, g.aux, g.fV, st, grid_for(E, g.N, 256)); });
    timed(E, ES_KERNEL_VOLUME, st, [&] { Lc::volume(g.P, sv, g.aux, g.F, g.FL, g.fV, ns, st, g.vol_variant % kVolumeVariants); });
    return last_launch_error();
  });
}

int run_relax(Engine& E, Group& g, const StageRelax& sr, cudaStream_t st) {
  const int grid = (int)std::min<long long>((g.K + 3) / 4, (long long)E.sm_count * 16);
  return dispatch(g, [&](auto L) {
    timed(E, ES_KERNEL_RELAX, st, [&] { decltype(L)::relax(g.P, sr, st, grid); });
    return last_launch_error();
  });
}

StageRelax relax_base(Engine& E, Group& g) {
  StageRelax sr;
  std::memset(&sr, 0, sizeof(sr));
  sr.gamma_elem = g.gamma_elem;
  sr.gmin_bits = g.gmin;
  sr.status = E.status;
  // default floor: FP64 right-hand sides are exact to ~1e-15 of the state per step, so
  // 1e-8 leaves a wide margin; FP32 right-hand sides carry rounding noise of relative size
  // ~eps_32 times the flux-to-state cancellation, and below 64 eps_32 ~ 4e-6 an element's
  // relaxation would be fitted to that noise.
  const double floor_default = (g.cfg.precision == ES_MIXED || g.cfg.precision == ES_MIXED_FF) ? 4e-6 : 1e-8;
  sr.delta_floor = g.cfg.delta_floor > 0.0 ? g.cfg.delta_floor : floor_default;
  sr.gamma_max = 8.0;
  // Newton stop: a step |s| <= 1e-8 gamma leaves an error ~s^2/gamma ~ 1e-16 gamma
  sr.root_rtol = g.cfg.root_rtol > 0.0 ? g.cfg.root_rtol : 1e-8;
  return sr;
}

// One relaxed step of every instance of the group on state q: all stages, the
// gamma_kappa solve, gamma = min, t += gamma dt, pending update flag set.  The
// update u += gamma d itself runs in the next step's first k_prep (or group_finish).
// hist (device, per instance) receives gamma if not null.  With `estimate` the stages
// also accumulate A (and the entropy-variable increments it needs) when the method
// relaxes nothing, so that the step's entropy estimate can be formed afterwards.
int group_step(Engine& E, Group& g, double* q, double* t, double* hist, cudaStream_t st, bool estimate = false) {
  const Tableau& T = E.tab;
  const bool relax = E.relax != ES_RELAX_NONE;
  const bool acc_A = relax || estimate;
  int rc = ES_OK;
  for (int i = 0; i < T.s && rc == ES_OK; ++i) {
    StagePrep sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.q = q;
    sp.d = g.d;
    sp.gamma_cur = g.gamma_cur;
    sp.pending = (i == 0) ? g.pending : nullptr;
    sp.Np = g.Np;
    for (int j = 0; j < i; ++j) {
      if (T.a[i][j] != 0.0) {
        sp.coef[sp.nprev] = T.a[i][j];
        sp.k[sp.nprev] = g.k[j];
        sp.nprev++;
      }
    }
    const bool want_dw = acc_A && i > 0 && T.b[i] != 0.0;
    sp.dw = want_dw ? g.dw : nullptr;
    StageVol sv;
    std::memset(&sv, 0, sizeof(sv));
    sv.kout = g.k[i];
    if (i == T.s - 1) {  // last stage: write d = dt sum_j b_j k_j instead of k_s
      sv.d_out = g.d;
      sv.dcoef_self = T.b[i];
      ff_split_host(T.b[i], sv.dcoef_self_ff);
      for (int j = 0; j < i; ++j) {
        if (T.b[j] != 0.0) {
          sv.dcoef[sv.nd] = T.b[j];
          ff_split_host(T.b[j], sv.dcoef_ff[sv.nd]);
          sv.dk[sv.nd] = g.k[j];
          sv.nd++;
        }
      }
    }
    sv.dw = want_dw ? g.dw : nullptr;
    sv.A = acc_A ? g.A : nullptr;
    sv.A_scale = -T.b[i];
    sv.A_init = (i == 0);
    rc = run_stage(E, g, sp, sv, st, t, T.c[i] * g.P.g0.dt);
  }
  if (rc != ES_OK) return rc;
  StageRelax sr = relax_base(E, g);
  if (E.relax == ES_RELAX_GLOBAL) {
    GlobalRelaxArgs ga;
    std::memset(&ga, 0, sizeof(ga));
    ga.u = q;
    ga.d = g.d;
    ga.A = g.A;
    ga.nodes = g.dw;  // free after the last stage
    ga.elem_a = g.gwork;
    ga.elem_s = g.gwork + g.K;
    ga.elem_r = g.gwork + 2 * (long long)g.K;
    ga.elem_dr = g.gwork + 3 * (long long)g.K;
    ga.gs = g.gstate;
    ga.gmin_bits = g.gmin;
    ga.gamma_elem = g.gamma_elem;
    ga.status = E.status;
    ga.delta_floor = sr.delta_floor;
    ga.gamma_max = sr.gamma_max;
    ga.root_rtol = sr.root_rtol;
    const int grid = (int)std::min<long long>((g.K + 3) / 4, (long long)E.sm_count * 16);
    rc = dispatch(g, [&](auto L) {
      timed(E, ES_KERNEL_RELAX, st,
            [&] { decltype(L)::global_relax(g.P, ga, st, grid, kGlobalRelaxIterations); });
      return last_launch_error();
    });
  } else {
    sr.u = q;
    sr.d_in = g.d;
    sr.A = g.A;
    if (!relax) sr.delta_floor = INFINITY;  // every element unconstrained: gamma = 1
    rc = run_relax(E, g, sr, st);
  }
  if (rc != ES_OK) return rc;
  timed(E, ES_KERNEL_OTHER, st, [&] { launch_scalar(g.P, g.gmin, g.gamma_cur, t, hist, g.pending, relax ? 1 : 0, st); });
  return last_launch_error();
}

// Applies the pending relaxed update of every instance and clears the flags.
int group_finish(Engine& E, Group& g, double* q, cudaStream_t st) {
  timed(E, ES_KERNEL_OTHER, st,
        [&] { launch_update(g.P, q, q, g.d, g.gamma_cur, g.pending, g.Np, st, grid_for(E, 5 * g.N, 256)); });
  timed(E, ES_KERNEL_OTHER, st, [&] { launch_reset(g.gmin, g.pending, g.ninst, st); });
  return last_launch_error();
}

// nsteps relaxed steps of a single-instance context on device state q (in place).
int advance_device(es_ctx* c, double* q, int nsteps, double dt, double* t, double* hist, double* gamma_elem_out,
                   cudaStream_t st) {
  Group& g = c->g;
  g.P.g0.dt = dt;
  int rc = ES_OK;
  timed(c->eng, ES_KERNEL_OTHER, st, [&] { launch_reset(g.gmin, g.pending, g.ninst, st); });
  for (int n = 0; n < nsteps && rc == ES_OK; ++n) {
    rc = group_step(c->eng, g, q, t ? t : g.t, hist ? hist + n : nullptr, st);
    if (rc == ES_OK && gamma_elem_out && n == nsteps - 1)
      rc = cuda_check(cudaMemcpyAsync(gamma_elem_out, g.gamma_elem, sizeof(double) * g.K,
                                      cudaMemcpyDeviceToDevice, st));
  }
  if (rc == ES_OK && nsteps > 0) rc = group_finish(c->eng, g, q, st);
  return rc;
}

// The estimate of the step just taken (before its pending update): eta_kappa(u) and
// deta_kappa (k_estimate) into eta_old / deta (device, K each; either may be null).
int group_estimate(Engine& E, Group& g, const double* q, double* eta_old, double* deta, cudaStream_t st) {
  const int grid = (int)std::min<long long>((g.K + 3) / 4, (long long)E.sm_count * 16);
  return dispatch(g, [&](auto L) {
    timed(E, ES_KERNEL_OTHER, st, [&] { decltype(L)::estimate(g.P, q, g.d, g.A, eta_old, deta, st, grid); });
    return last_launch_error();
  });
}

// eta_kappa(q) of every element of the group into eta (device, K)
int group_entropy(Engine& E, Group& g, const double* q, double* eta, cudaStream_t st) {
  const int grid = (int)std::min<long long>((g.K + 3) / 4, (long long)E.sm_count * 16);
  return dispatch(g, [&](auto L) {
    timed(E, ES_KERNEL_OTHER, st, [&] { decltype(L)::entropy(g.P, q, eta, st, grid); });
    return last_launch_error();
  });
}

// Node coordinates [3][K][Np] of the mesh of C (host).
void node_coords(const es_config& C, double* xyz) {
  double x[kMaxP1], w[kMaxP1], D[kMaxP1 * kMaxP1];
  lgl_tables(C.p, x, w, D);
  const int P1 = C.p + 1;
  const int Np = P1 * P1 * P1;
  const int K = C.nx * C.ny * C.nz;
  const long long N = (long long)K * Np;
  const int nxyz[3] = {C.nx, C.ny, C.nz};
  for (int e = 0; e < K; ++e) {
    const int ei[3] = {e % nxyz[0], (e / nxyz[0]) % nxyz[1], e / (nxyz[0] * nxyz[1])};
    for (int n = 0; n < Np; ++n) {
      const int ni[3] = {n % P1, (n / P1) % P1, n / (P1 * P1)};
      for (int m = 0; m < 3; ++m) {
        const double h = (C.hi[m] - C.lo[m]) / nxyz[m];
        xyz[m * N + (long long)e * Np + n] = C.lo[m] + h * (ei[m] + 0.5 * (1.0 + x[ni[m]]));
      }
    }
  }
}

int status_read(Engine& E, cudaStream_t st) {
  int h = 0;
  int rc = cuda_check(cudaMemcpyAsync(&h, E.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (rc == ES_OK) rc = cuda_check(cudaStreamSynchronize(st));
  if (rc != ES_OK) return rc;
  if (h) {
    rc = cuda_check(cudaMemsetAsync(E.status, 0, sizeof(int), st));
    if (rc == ES_OK) rc = cuda_check(cudaStreamSynchronize(st));
    if (rc != ES_OK) return rc;
  }
  if (h & kStatusNonphysical) return ES_ERR_NONPHYSICAL;
  if (h & kStatusNoRoot) return ES_ERR_NO_ROOT;
  return ES_OK;
}

// Times each volume tile on the group's current state (one stage's RHS) and keeps the fastest.
int autotune_group(Engine& E, Group& g, const double* q, cudaStream_t st) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return ES_ERR_CUDA;
  float best = 1e30f;
  int best_v = 0;
  const int keep = g.vol_variant;
  const bool prof = E.profiling;
  E.profiling = false;
  int rc = ES_OK;
  const int nv = stage_fusable(g) ? kStageVariants : kVolumeVariants;
  for (int v = 0; v < nv && rc == ES_OK; ++v) {
    g.vol_variant = v;
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && rc == ES_OK; ++rep) {
      // a first stage into k[0], then a stage on y = u + dt/2 k[0] that accumulates A
      StagePrep sp;
      std::memset(&sp, 0, sizeof(sp));
      sp.q = const_cast<double*>(q);
      sp.Np = g.Np;
      StageVol sv;
      std::memset(&sv, 0, sizeof(sv));
      sv.kout = g.k[0];
      cudaEventRecord(a, st);
      rc = run_stage(E, g, sp, sv, st);
      if (rc == ES_OK && g.nk > 1) {
        sp.nprev = 1;
        sp.coef[0] = 0.5;
        sp.k[0] = g.k[0];
        sp.dw = g.dw;
        sv.kout = g.k[1];
        sv.dw = g.dw;
        sv.A = g.A;
        sv.A_scale = -0.5;
        sv.A_init = 1;
        rc = run_stage(E, g, sp, sv, st);
      }
      cudaEventRecord(b, st);
      if (rc == ES_OK) rc = cuda_check(cudaEventSynchronize(b));
      float ms = 0.f;
      if (rc == ES_OK) rc = cuda_check(cudaEventElapsedTime(&ms, a, b));
      if (ms < tmin) tmin = ms;
    }
    if (rc == ES_OK && tmin < best) {
      best = tmin;
      best_v = v;
    }
  }
  E.profiling = prof;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  g.vol_variant = rc == ES_OK ? best_v : keep;
  return rc;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int es_create(const es_config* cfg, es_ctx** out) {
  if (!out) return ES_ERR_INVALID;
  *out = nullptr;
  if (!cfg) return ES_ERR_INVALID;
  const es_config& C = *cfg;
  if (validate_config(C) != ES_OK) return ES_ERR_INVALID;
  es_ctx* c = new (std::nothrow) es_ctx();
  if (!c) return ES_ERR_NOMEM;
  int rc = engine_init(c->eng, C);
  if (rc == ES_OK) rc = group_init(c->g, &C, 1, c->eng.tab.s, false);
  if (rc != ES_OK) {
    group_free(c->g);
    engine_free(c->eng);
    delete c;
    return rc;
  }
  *out = c;
  return ES_OK;
}

void es_destroy(es_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  group_free(c->g);
  engine_free(c->eng);
  cudaFree(c->q_host_dev);
  cudaFree(c->t_host_dev);
  cudaFree(c->hist_host_dev);
  delete c;
}

int es_rhs(es_ctx* c, const double* q, double* dqdt, double* E_elem, void* stream) {
  if (!c || !q || !dqdt || q == dqdt) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  StagePrep sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.q = const_cast<double*>(q);  // read only: no pending update
  sp.Np = c->g.Np;
  StageVol sv;
  std::memset(&sv, 0, sizeof(sv));
  sv.kout64 = dqdt;
  sv.E = E_elem;
  return run_stage(c->eng, c->g, sp, sv, st);
}

int es_set_boundary(es_ctx* c, int dir, int kind, const double* params, int nparams) {
  if (!c || dir < 0 || dir > 2) return ES_ERR_INVALID;
  Group& g = c->g;
  BcSpec& b = g.bc;
  if (kind == ES_BC_PERIODIC) {
    b.kind[dir] = ES_BC_PERIODIC;
  } else if (kind == ES_BC_STATE) {
    if (!params || nparams != 10) return ES_ERR_INVALID;
    for (int s = 0; s < 2; ++s) {
      const double* q = params + 5 * s;
      const double p = (g.cfg.gamma_gas - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
      if (!(q[0] > 0.0) || !(p > 0.0)) return ES_ERR_INVALID;
      for (int v = 0; v < 5; ++v) b.q[dir][s][v] = q[v];
    }
    b.kind[dir] = ES_BC_STATE;
  } else if (kind == ES_BC_VISCOUS_SHOCK) {
    // params: Mach number, Reynolds number, Prandtl number, translation speed
    if (!params || nparams != 4) return ES_ERR_INVALID;
    const double M = params[0], Re = params[1], Pr = params[2], speed = params[3];
    const double gm = g.cfg.gamma_gas;
    if (!(M > 1.0) || !(Re > 0.0) || !(Pr > 0.0) || !std::isfinite(speed)) return ES_ERR_INVALID;
    b.vs[dir][0] = (2.0 + (gm - 1.0) * M * M) / ((gm + 1.0) * M * M);  // V_f
    b.vs[dir][1] = 2.0 * gm / (gm + 1.0) * (1.0 / Re) / Pr;          // alpha (mass flux 1)
    b.vs[dir][2] = gm / (gm - 1.0) / (gm * M * M) + 0.5;              // total enthalpy
    b.vs[dir][3] = speed;
    b.vs[dir][4] = g.cfg.lo[dir];
    b.vs[dir][5] = g.cfg.hi[dir];
    b.kind[dir] = ES_BC_VISCOUS_SHOCK;
  } else {
    return ES_ERR_INVALID;
  }
  b.gam = g.cfg.gamma_gas;
  g.any_bc = b.kind[0] != ES_BC_PERIODIC || b.kind[1] != ES_BC_PERIODIC || b.kind[2] != ES_BC_PERIODIC;
  int rc = ES_OK;
  if (g.any_bc && !g.FL) rc = dev_alloc_bytes(&g.FL, 15 * size_t(g.K) * g.P1 * g.P1 * g.tf);
  if (rc == ES_OK && g.any_bc && !g.bcz) {
    rc = dev_alloc(&g.bcz, 6 * kBcVals);
    if (rc == ES_OK) rc = cuda_check(cudaMemset(g.bcz, 0, sizeof(double) * 6 * kBcVals));
  }
  if (rc != ES_OK) return rc;
  for (int m = 0; m < 3; ++m) g.P.bc[m] = b.kind[m] != ES_BC_PERIODIC ? 1 : 0;
  g.P.bcz = g.bcz;
  if (g.vol_variant >= kVolumeVariants && !stage_fusable(g)) g.vol_variant -= kVolumeVariants;
  return ES_OK;
}

int es_set_time(es_ctx* c, double t) {
  if (!c || !std::isfinite(t)) return ES_ERR_INVALID;
  return cuda_check(cudaMemcpy(c->g.t, &t, sizeof(double), cudaMemcpyHostToDevice));
}

int es_set_tableau(es_ctx* c, int s, const double* a, const double* b, const double* cs) {
  if (!c) return ES_ERR_INVALID;
  Tableau t;
  int rc = parse_tableau(c->eng.relax, s, a, b, cs, &t);
  if (rc == ES_OK) rc = ensure_stage_buffers(c->g, t.s);
  if (rc == ES_OK) c->eng.tab = t;
  return rc;
}

int es_entropy(es_ctx* c, const double* q, double* eta, void* stream) {
  if (!c || !q || !eta) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Group& g = c->g;
  const int grid = (int)std::min<long long>((g.K + 3) / 4, (long long)c->eng.sm_count * 16);
  return dispatch(g, [&](auto L) {
    timed(c->eng, ES_KERNEL_OTHER, st, [&] { decltype(L)::entropy(g.P, q, eta, st, grid); });
    return last_launch_error();
  });
}

int es_relax_step(es_ctx* c, const double* u_old, const double* u_new, const double* d_eta, double* gamma_elem,
                  double* gamma, double* u_out, void* stream) {
  if (!c || !u_old || !u_new || !d_eta || !u_out || u_out == u_old) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Engine& E = c->eng;
  Group& g = c->g;
  Params P = g.P;
  P.g0.dt = 0.0;
  timed(E, ES_KERNEL_OTHER, st, [&] { launch_reset(g.gmin, g.pending, g.ninst, st); });
  StageRelax sr = relax_base(E, g);
  sr.u = u_old;
  sr.u_new = u_new;
  sr.deta = d_eta;
  sr.d_out = g.d;
  int rc = dispatch(g, [&](auto L) {
    const int grid = (int)std::min<long long>((g.K + 3) / 4, (long long)E.sm_count * 16);
    timed(E, ES_KERNEL_RELAX, st, [&] { decltype(L)::relax(P, sr, st, grid); });
    return last_launch_error();
  });
  if (rc != ES_OK) return rc;
  timed(E, ES_KERNEL_OTHER, st, [&] { launch_scalar(P, g.gmin, g.gamma_cur, g.t, nullptr, g.pending, 1, st); });
  timed(E, ES_KERNEL_OTHER, st,
        [&] { launch_update(P, u_out, u_old, g.d, g.gamma_cur, g.pending, g.Np, st, grid_for(E, 5 * g.N, 256)); });
  timed(E, ES_KERNEL_OTHER, st, [&] { launch_reset(g.gmin, g.pending, g.ninst, st); });
  rc = last_launch_error();
  if (rc != ES_OK) return rc;
  if (gamma_elem) {
    rc = cuda_check(cudaMemcpyAsync(gamma_elem, g.gamma_elem, sizeof(double) * g.K, cudaMemcpyDeviceToDevice, st));
    if (rc != ES_OK) return rc;
  }
  if (gamma) rc = cuda_check(cudaMemcpyAsync(gamma, g.gamma_cur, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return rc;
}

int es_advance(es_ctx* c, double* q, int nsteps, double dt, double* t, double* gamma_hist, double* gamma_elem,
               void* stream) {
  if (!c || !q || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return ES_ERR_INVALID;
  return advance_device(c, q, nsteps, dt, t, gamma_hist, gamma_elem, static_cast<cudaStream_t>(stream));
}

int es_step_estimate(es_ctx* c, double* q, double dt, double* t, double* gamma, double* gamma_elem, double* eta_old,
                     double* deta, double* eta_new, void* stream) {
  if (!c || !q || !(dt > 0.0) || !std::isfinite(dt)) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Engine& E = c->eng;
  Group& g = c->g;
  g.P.g0.dt = dt;
  timed(E, ES_KERNEL_OTHER, st, [&] { launch_reset(g.gmin, g.pending, g.ninst, st); });
  int rc = group_step(E, g, q, t ? t : g.t, gamma, st, true);
  if (rc == ES_OK && (eta_old || deta)) rc = group_estimate(E, g, q, eta_old, deta, st);
  if (rc == ES_OK && gamma_elem)
    rc = cuda_check(cudaMemcpyAsync(gamma_elem, g.gamma_elem, sizeof(double) * g.K, cudaMemcpyDeviceToDevice, st));
  if (rc == ES_OK) rc = group_finish(E, g, q, st);
  if (rc == ES_OK && eta_new) rc = group_entropy(E, g, q, eta_new, st);
  return rc;
}

int es_advance_host(es_ctx* c, double* q_host, int nsteps, double dt, double* t_host, double* gamma_hist_host,
                    void* stream) {
  if (!c || !q_host || !t_host || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ES_OK;
  if (!c->q_host_dev) rc = dev_alloc(&c->q_host_dev, 5 * c->g.N);
  if (rc == ES_OK && !c->t_host_dev) rc = dev_alloc(&c->t_host_dev, 1);
  if (rc == ES_OK && gamma_hist_host && c->hist_cap < nsteps) {
    cudaFree(c->hist_host_dev);
    c->hist_host_dev = nullptr;
    c->hist_cap = 0;
    rc = dev_alloc(&c->hist_host_dev, nsteps);
    if (rc == ES_OK) c->hist_cap = nsteps;
  }
  if (rc != ES_OK) return rc;
  const size_t qb = sizeof(double) * 5 * c->g.N;
  rc = cuda_check(cudaMemcpyAsync(c->q_host_dev, q_host, qb, cudaMemcpyHostToDevice, st));
  if (rc == ES_OK) rc = cuda_check(cudaMemcpyAsync(c->t_host_dev, t_host, sizeof(double), cudaMemcpyHostToDevice, st));
  if (rc == ES_OK)
    rc = advance_device(c, c->q_host_dev, nsteps, dt, c->t_host_dev, gamma_hist_host ? c->hist_host_dev : nullptr,
                        nullptr, st);
  if (rc == ES_OK) rc = cuda_check(cudaMemcpyAsync(q_host, c->q_host_dev, qb, cudaMemcpyDeviceToHost, st));
  if (rc == ES_OK) rc = cuda_check(cudaMemcpyAsync(t_host, c->t_host_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (rc == ES_OK && gamma_hist_host)
    rc = cuda_check(cudaMemcpyAsync(gamma_hist_host, c->hist_host_dev, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, st));
  if (rc == ES_OK) rc = cuda_check(cudaStreamSynchronize(st));
  return rc;
}

int es_autotune(es_ctx* c, const double* q, void* stream) {
  if (!c || !q) return ES_ERR_INVALID;
  return autotune_group(c->eng, c->g, q, static_cast<cudaStream_t>(stream));
}

int es_volume_variant(const es_ctx* c) { return c ? c->g.vol_variant : ES_ERR_INVALID; }

int es_set_volume_variant(es_ctx* c, int variant) {
  if (!c || variant < 0 || variant >= kStageVariants) return ES_ERR_INVALID;
  if (variant >= kVolumeVariants && !stage_fusable(c->g)) return ES_ERR_INVALID;
  c->g.vol_variant = variant;
  return ES_OK;
}

int es_node_coords(const es_ctx* c, double* xyz) {
  if (!c || !xyz) return ES_ERR_INVALID;
  node_coords(c->g.cfg, xyz);
  return ES_OK;
}

int es_status(es_ctx* c, void* stream) {
  if (!c) return ES_ERR_INVALID;
  return status_read(c->eng, static_cast<cudaStream_t>(stream));
}

long long es_launch_count(const es_ctx* c) { return c ? c->eng.launches : 0; }

int es_profile_enable(es_ctx* c, int enable) {
  if (!c) return ES_ERR_INVALID;
  if (!enable) flush_marks(c->eng);
  c->eng.profiling = enable != 0;
  return ES_OK;
}

int es_profile_read(es_ctx* c, double* ms, long long* launches) {
  if (!c || !ms || !launches) return ES_ERR_INVALID;
  flush_marks(c->eng);
  for (int k = 0; k < ES_KERNEL_COUNT; ++k) {
    ms[k] = c->eng.prof_ms[k];
    launches[k] = c->eng.prof_n[k];
    c->eng.prof_ms[k] = 0.0;
    c->eng.prof_n[k] = 0;
  }
  return ES_OK;
}

const char* es_strerror(int code) {
  switch (code) {
    case ES_OK: return "ok";
    case ES_ERR_INVALID: return "invalid argument or unsupported configuration";
    case ES_ERR_CUDA: return "CUDA runtime error";
    case ES_ERR_NONPHYSICAL: return "non-physical state (rho <= 0 or p <= 0)";
    case ES_ERR_NO_ROOT: return "no positive relaxation root (r'(0) >= 0)";
    case ES_ERR_NOMEM: return "out of memory";
    case ES_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of es_rhs_noalloc";
  }
  return "unknown error";
}

}  // extern "C"


// ---------------------------------------------------------------------------
// Batches: independent instances grouped by degree, one captured graph per step.
namespace {

bool same_physics(const es_config& a, const es_config& b) {
  return a.gamma_gas == b.gamma_gas && a.mu == b.mu && (a.mu == 0.0 || a.Pr == b.Pr) && a.R == b.R &&
         a.interface_diss == b.interface_diss && a.relax == b.relax && a.rk == b.rk && a.precision == b.precision &&
         a.delta_floor == b.delta_floor && a.visc_diss == b.visc_diss && a.root_rtol == b.root_rtol;
}

void batch_free(es_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->side) cudaStreamDestroy(s);
  for (auto e : b->fork) cudaEventDestroy(e);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->exec_stream) cudaStreamDestroy(b->exec_stream);
  for (auto& g : b->groups) group_free(g);
  engine_free(b->eng);
  delete b;
}

int batch_capture(es_batch* b) {
  Engine& E = b->eng;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  const long long before = E.launches;
  E.capturing = true;
  int rc = cuda_check(cudaStreamBeginCapture(b->exec_stream, cudaStreamCaptureModeThreadLocal));
  for (size_t gi = 0; gi < b->groups.size() && rc == ES_OK; ++gi) {
    Group& g = b->groups[gi];
    rc = cuda_check(cudaEventRecord(b->fork[gi], b->exec_stream));
    if (rc == ES_OK) rc = cuda_check(cudaStreamWaitEvent(b->side[gi], b->fork[gi], 0));
    if (rc == ES_OK) rc = group_step(E, g, g.q, g.t, nullptr, b->side[gi]);
    if (rc == ES_OK) rc = cuda_check(cudaEventRecord(b->join[gi], b->side[gi]));
    if (rc == ES_OK) rc = cuda_check(cudaStreamWaitEvent(b->exec_stream, b->join[gi], 0));
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->exec_stream, &graph);
  E.capturing = false;
  if (rc == ES_OK) rc = cuda_check(ec);
  if (rc == ES_OK) rc = cuda_check(cudaGraphInstantiate(&b->exec, graph, 0));
  if (graph) cudaGraphDestroy(graph);
  b->kernels_per_step = E.launches - before;
  E.launches = before;
  return rc;
}

}  // namespace

extern "C" {

int es_batch_create(const es_config* cfgs, int count, es_batch** out) {
  if (!out) return ES_ERR_INVALID;
  *out = nullptr;
  if (!cfgs || count < 1) return ES_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (validate_config(cfgs[i]) != ES_OK || !same_physics(cfgs[0], cfgs[i])) return ES_ERR_INVALID;
  es_batch* b = new (std::nothrow) es_batch();
  if (!b) return ES_ERR_NOMEM;
  b->cfgs.assign(cfgs, cfgs + count);
  b->where.resize(count);
  int rc = engine_init(b->eng, cfgs[0]);
  for (int p = 2; p <= 5 && rc == ES_OK; ++p) {
    std::vector<es_config> insts;
    std::vector<int> ids;
    for (int i = 0; i < count; ++i)
      if (cfgs[i].p == p) {
        insts.push_back(cfgs[i]);
        ids.push_back(i);
      }
    if (insts.empty()) continue;
    b->groups.emplace_back();
    Group& g = b->groups.back();
    rc = group_init(g, insts.data(), (int)insts.size(), b->eng.tab.s, true);
    g.inst_ids = ids;
    for (size_t j = 0; j < ids.size(); ++j) b->where[ids[j]] = {(int)b->groups.size() - 1, (int)j};
  }
  if (rc == ES_OK) rc = cuda_check(cudaStreamCreateWithFlags(&b->exec_stream, cudaStreamNonBlocking));
  for (size_t gi = 0; gi < b->groups.size() && rc == ES_OK; ++gi) {
    cudaStream_t s = nullptr;
    cudaEvent_t f = nullptr, j = nullptr;
    rc = cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (rc == ES_OK) rc = cuda_check(cudaEventCreateWithFlags(&f, cudaEventDisableTiming));
    if (rc == ES_OK) rc = cuda_check(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
    b->side.push_back(s);
    b->fork.push_back(f);
    b->join.push_back(j);
  }
  if (rc != ES_OK) {
    batch_free(b);
    return rc;
  }
  *out = b;
  return ES_OK;
}

void es_batch_destroy(es_batch* b) { batch_free(b); }

long long es_batch_nodes(const es_batch* b, int inst) {
  if (!b || inst < -1 || inst >= (int)b->cfgs.size()) return -1;
  long long total = 0;
  for (int i = 0; i < (int)b->cfgs.size(); ++i) {
    if (inst >= 0 && i != inst) continue;
    const es_config& C = b->cfgs[i];
    total += (long long)C.nx * C.ny * C.nz * (C.p + 1) * (C.p + 1) * (C.p + 1);
  }
  return total;
}

int es_batch_node_coords(const es_batch* b, int inst, double* xyz_host) {
  if (!b || !xyz_host || inst < 0 || inst >= (int)b->cfgs.size()) return ES_ERR_INVALID;
  node_coords(b->cfgs[inst], xyz_host);
  return ES_OK;
}

static int batch_copy(es_batch* b, int inst, double* host, bool to_device) {
  if (!b || !host || inst < 0 || inst >= (int)b->cfgs.size()) return ES_ERR_INVALID;
  const Group& g = b->groups[b->where[inst].first];
  const InstGeom& G = g.geom[b->where[inst].second];
  const long long Ki = (long long)G.nx * G.ny * G.nz;
  const size_t bytes = sizeof(double) * Ki * g.Np;
  int rc = cuda_check(cudaDeviceSynchronize());
  for (int v = 0; v < 5 && rc == ES_OK; ++v) {
    double* dev = g.q + v * g.N + (long long)G.off * g.Np;
    double* hp = host + v * Ki * g.Np;
    rc = cuda_check(to_device ? cudaMemcpy(dev, hp, bytes, cudaMemcpyHostToDevice)
                              : cudaMemcpy(hp, dev, bytes, cudaMemcpyDeviceToHost));
  }
  return rc;
}

int es_batch_set_state(es_batch* b, int inst, const double* q_host) {
  return batch_copy(b, inst, const_cast<double*>(q_host), true);
}

int es_batch_get_state(es_batch* b, int inst, double* q_host) { return batch_copy(b, inst, q_host, false); }

int es_batch_set_dt(es_batch* b, const double* dt_host) {
  if (!b || !dt_host) return ES_ERR_INVALID;
  int rc = cuda_check(cudaDeviceSynchronize());
  for (auto& g : b->groups) {
    for (int j = 0; j < g.ninst && rc == ES_OK; ++j) {
      const double dt = dt_host[g.inst_ids[j]];
      if (!(dt > 0.0) || !std::isfinite(dt)) return ES_ERR_INVALID;
      g.geom[j].dt = dt;
    }
    if (rc == ES_OK)
      rc = cuda_check(cudaMemcpy(g.geom_dev, g.geom.data(), g.ninst * sizeof(InstGeom), cudaMemcpyHostToDevice));
  }
  return rc;
}

int es_batch_set_tableau(es_batch* b, int s, const double* a, const double* bw, const double* cs) {
  if (!b) return ES_ERR_INVALID;
  Tableau t;
  int rc = parse_tableau(b->eng.relax, s, a, bw, cs, &t);
  if (rc != ES_OK) return rc;
  rc = cuda_check(cudaDeviceSynchronize());  // no captured step in flight
  for (auto& g : b->groups)
    if (rc == ES_OK) rc = ensure_stage_buffers(g, t.s);
  if (rc != ES_OK) return rc;
  if (b->exec) {  // the next es_batch_advance captures the new stages
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->eng.tab = t;
  return ES_OK;
}

int es_batch_autotune(es_batch* b, void* stream) {
  if (!b) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ES_OK;
  for (auto& g : b->groups) {
    if (rc == ES_OK) rc = autotune_group(b->eng, g, g.q, st);
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return rc;
}

int es_batch_volume_variant(const es_batch* b, int inst) {
  if (!b || inst < 0 || inst >= (int)b->cfgs.size()) return ES_ERR_INVALID;
  return b->groups[b->where[inst].first].vol_variant;
}

int es_batch_advance(es_batch* b, int nsteps, void* stream) {
  if (!b || nsteps < 0) return ES_ERR_INVALID;
  for (auto& g : b->groups)
    for (auto& G : g.geom)
      if (!(G.dt > 0.0)) return ES_ERR_INVALID;  // es_batch_set_dt first
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Engine& E = b->eng;
  int rc = ES_OK;
  if (!b->exec) rc = batch_capture(b);
  if (rc != ES_OK) return rc;
  cudaEvent_t ev = nullptr;
  rc = cuda_check(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  if (rc == ES_OK) rc = cuda_check(cudaEventRecord(ev, st));
  if (rc == ES_OK) rc = cuda_check(cudaStreamWaitEvent(b->exec_stream, ev, 0));
  for (int n = 0; n < nsteps && rc == ES_OK; ++n) {
    rc = cuda_check(cudaGraphLaunch(b->exec, b->exec_stream));
    E.launches += b->kernels_per_step;
  }
  for (auto& g : b->groups)
    if (rc == ES_OK && nsteps > 0) rc = group_finish(E, g, g.q, b->exec_stream);
  if (rc == ES_OK) rc = cuda_check(cudaEventRecord(ev, b->exec_stream));
  if (rc == ES_OK) rc = cuda_check(cudaStreamWaitEvent(st, ev, 0));
  if (ev) cudaEventDestroy(ev);
  return rc;
}

int es_batch_step_estimate(es_batch* b, void* stream) {
  if (!b) return ES_ERR_INVALID;
  for (auto& g : b->groups)
    for (auto& G : g.geom)
      if (!(G.dt > 0.0)) return ES_ERR_INVALID;  // es_batch_set_dt first
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Engine& E = b->eng;
  int rc = ES_OK;
  for (auto& g : b->groups) {
    if (rc == ES_OK && !g.est) rc = dev_alloc(&g.est, 3 * (size_t)g.K);
    if (rc == ES_OK) timed(E, ES_KERNEL_OTHER, st, [&] { launch_reset(g.gmin, g.pending, g.ninst, st); });
    if (rc == ES_OK) rc = group_step(E, g, g.q, g.t, nullptr, st, true);
    if (rc == ES_OK) rc = group_estimate(E, g, g.q, g.est, g.est + g.K, st);
    if (rc == ES_OK) rc = group_finish(E, g, g.q, st);
    if (rc == ES_OK) rc = group_entropy(E, g, g.q, g.est + 2 * (long long)g.K, st);
  }
  return rc;
}

int es_batch_get_estimate(es_batch* b, int inst, double* eta_old_host, double* deta_host, double* eta_new_host,
                          double* gamma_elem_host) {
  if (!b || inst < 0 || inst >= (int)b->cfgs.size()) return ES_ERR_INVALID;
  const Group& g = b->groups[b->where[inst].first];
  if (!g.est) return ES_ERR_INVALID;  // es_batch_step_estimate first
  const InstGeom& G = g.geom[b->where[inst].second];
  const size_t bytes = sizeof(double) * G.nx * G.ny * G.nz;
  int rc = cuda_check(cudaDeviceSynchronize());
  const double* src[4] = {g.est, g.est + g.K, g.est + 2 * (long long)g.K, g.gamma_elem};
  double* dst[4] = {eta_old_host, deta_host, eta_new_host, gamma_elem_host};
  for (int k = 0; k < 4 && rc == ES_OK; ++k)
    if (dst[k]) rc = cuda_check(cudaMemcpy(dst[k], src[k] + G.off, bytes, cudaMemcpyDeviceToHost));
  return rc;
}

int es_batch_times(es_batch* b, double* t_host, double* gamma_host) {
  if (!b) return ES_ERR_INVALID;
  int rc = cuda_check(cudaDeviceSynchronize());
  for (auto& g : b->groups) {
    std::vector<double> t(g.ninst), gm(g.ninst);
    if (rc == ES_OK) rc = cuda_check(cudaMemcpy(t.data(), g.t, g.ninst * sizeof(double), cudaMemcpyDeviceToHost));
    if (rc == ES_OK)
      rc = cuda_check(cudaMemcpy(gm.data(), g.gamma_cur, g.ninst * sizeof(double), cudaMemcpyDeviceToHost));
    for (int j = 0; j < g.ninst && rc == ES_OK; ++j) {
      if (t_host) t_host[g.inst_ids[j]] = t[j];
      if (gamma_host) gamma_host[g.inst_ids[j]] = gm[j];
    }
  }
  return rc;
}

int es_batch_status(es_batch* b, void* stream) {
  if (!b) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = cuda_check(cudaStreamSynchronize(b->exec_stream));
  if (rc != ES_OK) return rc;
  return status_read(b->eng, st);
}

long long es_batch_launch_count(const es_batch* b) { return b ? b->eng.launches : 0; }

int es_reciprocal(const double* x, double* out, long long n, void* stream);

}  // extern "C"

// ---------------------------------------------------------------------------
// small kernels
namespace {

__global__ void k_reciprocal(const double* __restrict__ x, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = fast_rcp(x[i]);
}

__global__ void k_scalar(int ninst, unsigned long long* gmin_bits, double* gamma_cur, double* t, double* hist,
                         int* pending, const InstGeom* geom, double dt0, int relax) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) {
    double g = __longlong_as_double((long long)gmin_bits[i]);
    if (!relax || !(g < INFINITY)) g = 1.0;
    const double dt = geom ? geom[i].dt : dt0;
    gamma_cur[i] = g;
    t[i] += g * dt;
    if (hist) hist[i] = g;
    pending[i] = 1;
    gmin_bits[i] = 0x7ff0000000000000ULL;
  }
}

__global__ void k_reset(unsigned long long* gmin_bits, int* pending, int ninst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x) {
    gmin_bits[i] = 0x7ff0000000000000ULL;
    pending[i] = 0;
  }
}

// out = base + gamma[inst] d where the instance has a pending update (out may alias base)
__global__ void k_update(Params P, double* out, const double* base, const double* __restrict__ d,
                         const double* __restrict__ gamma_cur, const int* __restrict__ pending, int Np) {
  const long long N = (long long)P.K * Np;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 5 * N;
       i += (long long)gridDim.x * blockDim.x) {
    const int inst = inst_of(P, int((i % N) / Np));
    if (pending[inst]) out[i] = base[i] + gamma_cur[inst] * d[i];
    else if (out != base) out[i] = base[i];
  }
}

}  // namespace

extern "C" int es_reciprocal(const double* x, double* out, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return ES_ERR_INVALID;
  if (n == 0) return ES_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ES_ERR_CUDA;
  k_reciprocal<<<grid_for_sms(sms, n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n);
  return cudaGetLastError() == cudaSuccess ? ES_OK : ES_ERR_CUDA;
}

namespace es {
void launch_scalar(const Params& P, unsigned long long* gmin_bits, double* gamma_cur, double* t, double* hist,
                   int* pending, int relax, cudaStream_t st) {
  const int blocks = (P.ninst + 127) / 128;
  k_scalar<<<blocks, 128, 0, st>>>(P.ninst, gmin_bits, gamma_cur, t, hist, pending, P.geom, P.g0.dt, relax);
}
void launch_reset(unsigned long long* gmin_bits, int* pending, int ninst, cudaStream_t st) {
  k_reset<<<(ninst + 127) / 128, 128, 0, st>>>(gmin_bits, pending, ninst);
}
void launch_update(const Params& P, double* out, const double* base, const double* d, const double* gamma_cur,
                   const int* pending, int Np, cudaStream_t st, int grid) {
  k_update<<<grid, 256, 0, st>>>(P, out, base, d, gamma_cur, pending, Np);
}
}  // namespace es

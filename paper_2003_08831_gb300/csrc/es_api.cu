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

// Butcher tableaux (Section 4 names BSRK(4,3) and RK(4,4)).
struct Tableau {
  int s;          // stages entering u_new
  double a[4][4];
  double b[4];
};

Tableau tableau(int rk) {
  Tableau t;
  std::memset(&t, 0, sizeof(t));
  if (rk == ES_RK_BS3) {  // Bogacki & Shampine 3(2); b_4 = 0 so stage 4 is not needed
    t.s = 3;
    t.a[1][0] = 0.5;
    t.a[2][1] = 0.75;
    t.b[0] = 2.0 / 9.0;
    t.b[1] = 1.0 / 3.0;
    t.b[2] = 4.0 / 9.0;
  } else {  // classical RK(4,4)
    t.s = 4;
    t.a[1][0] = 0.5;
    t.a[2][1] = 0.5;
    t.a[3][2] = 1.0;
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
  if (C.rk != ES_RK_BS3 && C.rk != ES_RK_RK4) return ES_ERR_INVALID;
  if (C.precision != ES_FP64 && C.precision != ES_MIXED) return ES_ERR_INVALID;
  if (C.relax != ES_RELAX_NONE && C.relax != ES_RELAX_LOCAL) return ES_ERR_INVALID;
  if (C.interface_diss != 0 && C.interface_diss != 1) return ES_ERR_INVALID;
  for (int m = 0; m < 3; ++m)
    if (!(C.hi[m] > C.lo[m])) return ES_ERR_INVALID;
  const long long K = (long long)C.nx * C.ny * C.nz;
  if (K > (1LL << 30)) return ES_ERR_INVALID;
  return ES_OK;
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
    for (int j = 0; j < P1; ++j) {
      P.D[i * P1 + j] = D[i * P1 + j];
      P.D2[i * P1 + j] = (i == j) ? 0.0 : 2.0 * D[i * P1 + j];
    }
  }
  P.inv_omega_end = 1.0 / w[0];
  double h[3];
  for (int m = 0; m < 3; ++m) {
    const int nm = m == 0 ? C.nx : (m == 1 ? C.ny : C.nz);
    h[m] = (C.hi[m] - C.lo[m]) / nm;
    P.metric[m] = 2.0 / h[m];
  }
  P.J = h[0] * h[1] * h[2] / 8.0;
  P.gam = C.gamma_gas;
  P.mu = C.mu;
  P.R = C.R;
  P.kappa_heat = C.mu > 0.0 ? C.mu * C.gamma_gas * C.R / ((C.gamma_gas - 1.0) * C.Pr) : 0.0;
  P.nx = C.nx;
  P.ny = C.ny;
  P.nz = C.nz;
  P.K = C.nx * C.ny * C.nz;
  P.diss = C.interface_diss;
  P.p1 = P1;
}

int grid_for_sms(int sm_count, long long n, int block) {
  long long g = (n + block - 1) / block;
  const long long cap = (long long)sm_count * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace es

// ---------------------------------------------------------------------------
struct es_ctx {
  es_config cfg;
  int P1, Np, K;
  long long N;  // K * Np
  Params P;
  Tableau tab;
  int sm_count;
  int device;
  size_t tf;  // bytes per flux value (8 FP64, 4 mixed)
  // workspace
  double* k[4] = {nullptr, nullptr, nullptr, nullptr};
  void* aux = nullptr;
  void* F = nullptr;
  void* fV = nullptr;
  double* dw = nullptr;
  double* d = nullptr;
  double* A = nullptr;
  double* gamma_elem = nullptr;
  double* scal = nullptr;  // [0] gamma_cur, [1] t scratch
  unsigned long long* gmin = nullptr;
  int* status = nullptr;
  // host-buffer path
  double* q_host_dev = nullptr;
  double* t_host_dev = nullptr;
  double* hist_host_dev = nullptr;
  int hist_cap = 0;
  long long launches = 0;
  // per-kernel event timing (es_profile_enable)
  bool profiling = false;
  struct Mark { int kind; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  double prof_ms[ES_KERNEL_COUNT] = {0};
  long long prof_n[ES_KERNEL_COUNT] = {0};
};

namespace {

int grid_for(const es_ctx* c, long long n, int block) { return grid_for_sms(c->sm_count, n, block); }

template <typename F>
int dispatch(const es_ctx* c, F&& f) {
  switch (c->P1) {
    case 3: return c->tf == 8 ? f(Launcher<3, double>()) : f(Launcher<3, float>());
    case 4: return c->tf == 8 ? f(Launcher<4, double>()) : f(Launcher<4, float>());
    case 5: return c->tf == 8 ? f(Launcher<5, double>()) : f(Launcher<5, float>());
    case 6: return c->tf == 8 ? f(Launcher<6, double>()) : f(Launcher<6, float>());
  }
  return ES_ERR_INVALID;
}

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

void free_ctx(es_ctx* c) {
  if (!c) return;
  for (auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  for (auto& p : c->k) cudaFree(p);
  cudaFree(c->aux);
  cudaFree(c->F);
  cudaFree(c->fV);
  cudaFree(c->dw);
  cudaFree(c->d);
  cudaFree(c->A);
  cudaFree(c->gamma_elem);
  cudaFree(c->scal);
  cudaFree(c->gmin);
  cudaFree(c->status);
  cudaFree(c->q_host_dev);
  cudaFree(c->t_host_dev);
  cudaFree(c->hist_host_dev);
  delete c;
}

cudaEvent_t take_event(es_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Folds recorded event pairs into the per-kind totals (synchronises the device).
void flush_marks(es_ctx* c) {
  if (c->marks.empty()) return;
  cudaDeviceSynchronize();
  for (auto& m : c->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      c->prof_ms[m.kind] += ms;
      c->prof_n[m.kind] += 1;
    }
    c->pool.push_back(m.a);
    c->pool.push_back(m.b);
  }
  c->marks.clear();
  cudaGetLastError();
}

// Brackets one launch with events when profiling is on.
template <typename Fn>
void timed(es_ctx* c, int kind, cudaStream_t st, Fn&& fn) {
  c->launches += 1;
  if (!c->profiling) {
    fn();
    return;
  }
  if (c->marks.size() >= 4096) flush_marks(c);
  es_ctx::Mark m{kind, take_event(c), take_event(c)};
  cudaEventRecord(m.a, st);
  fn();
  cudaEventRecord(m.b, st);
  c->marks.push_back(m);
}

// One stage's right-hand side into kout (+ element sums), on state
// u (+ update) + sum_j coef[j] k[j].
int run_stage(es_ctx* c, const StagePrep& sp, const StageVol& sv, cudaStream_t st) {
  const bool ns = c->cfg.mu != 0.0;
  return dispatch(c, [&](auto L) {
    using Lc = decltype(L);
    timed(c, ES_KERNEL_PREP, st, [&] { Lc::prep(c->P, sp, c->aux, c->status, st, grid_for(c, c->N, 256)); });
    timed(c, ES_KERNEL_FACE, st,
          [&] { Lc::face(c->P, c->aux, c->F, st, grid_for(c, 3LL * c->K * c->P1 * c->P1, 256)); });
    if (ns) timed(c, ES_KERNEL_GRAD, st, [&] { Lc::grad(c->P, c->aux, c->fV, st, grid_for(c, c->N, 256)); });
    timed(c, ES_KERNEL_VOLUME, st, [&] { Lc::volume(c->P, sv, c->aux, c->F, c->fV, ns, st); });
    return last_launch_error();
  });
}

int run_relax(es_ctx* c, const StageRelax& sr, cudaStream_t st) {
  const int grid = (int)std::min<long long>((c->K + 3) / 4, (long long)c->sm_count * 16);
  return dispatch(c, [&](auto L) {
    timed(c, ES_KERNEL_RELAX, st, [&] { decltype(L)::relax(c->P, sr, st, grid); });
    return last_launch_error();
  });
}

StageRelax relax_base(es_ctx* c) {
  StageRelax sr;
  std::memset(&sr, 0, sizeof(sr));
  sr.gamma_elem = c->gamma_elem;
  sr.gmin_bits = c->gmin;
  sr.status = c->status;
  sr.delta_floor = c->cfg.delta_floor > 0.0 ? c->cfg.delta_floor : 1e-8;
  sr.gamma_max = 8.0;
  return sr;
}

// nsteps relaxed steps on device state q (in place).
int advance_device(es_ctx* c, double* q, int nsteps, double dt, double* t, double* hist, double* gamma_elem_out,
                   cudaStream_t st) {
  const Tableau& T = c->tab;
  const bool relax = c->cfg.relax == ES_RELAX_LOCAL;
  int rc = ES_OK;
  timed(c, ES_KERNEL_OTHER, st, [&] { launch_reset_min(c->gmin, st); });
  for (int n = 0; n < nsteps && rc == ES_OK; ++n) {
    for (int i = 0; i < T.s && rc == ES_OK; ++i) {
      StagePrep sp;
      std::memset(&sp, 0, sizeof(sp));
      sp.q = q;
      sp.d = c->d;
      sp.gamma_cur = c->scal;
      sp.apply_update = (i == 0 && n > 0);
      sp.Np = c->Np;
      for (int j = 0; j < i; ++j) {
        if (T.a[i][j] != 0.0) {
          sp.coef[sp.nprev] = dt * T.a[i][j];
          sp.k[sp.nprev] = c->k[j];
          sp.nprev++;
        }
      }
      const bool want_dw = relax && i > 0 && T.b[i] != 0.0;
      sp.dw = want_dw ? c->dw : nullptr;
      StageVol sv;
      std::memset(&sv, 0, sizeof(sv));
      sv.kout = c->k[i];
      if (i == T.s - 1) {  // last stage: write d = dt sum_j b_j k_j instead of k_s
        sv.d_out = c->d;
        sv.dcoef_self = dt * T.b[i];
        for (int j = 0; j < i; ++j) {
          if (T.b[j] != 0.0) {
            sv.dcoef[sv.nd] = dt * T.b[j];
            sv.dk[sv.nd] = c->k[j];
            sv.nd++;
          }
        }
      }
      sv.dw = want_dw ? c->dw : nullptr;
      sv.A = relax ? c->A : nullptr;
      sv.A_scale = -dt * T.b[i];
      sv.A_init = (i == 0);
      rc = run_stage(c, sp, sv, st);
    }
    if (rc != ES_OK) break;
    StageRelax sr = relax_base(c);
    sr.u = q;
    sr.d_in = c->d;
    sr.A = c->A;
    if (!relax) sr.delta_floor = INFINITY;  // combine only: every element unconstrained
    rc = run_relax(c, sr, st);
    if (rc != ES_OK) break;
    timed(c, ES_KERNEL_OTHER, st,
          [&] { launch_scalar(c->gmin, c->scal, t ? t : c->scal + 1, hist, n, dt, relax ? 1 : 0, st); });
    if (gamma_elem_out && n == nsteps - 1)
      rc = cuda_check(cudaMemcpyAsync(gamma_elem_out, c->gamma_elem, sizeof(double) * c->K,
                                      cudaMemcpyDeviceToDevice, st));
  }
  if (rc == ES_OK && nsteps > 0) {
    timed(c, ES_KERNEL_OTHER, st,
          [&] { launch_update(q, q, c->d, c->scal, 5 * c->N, st, grid_for(c, 5 * c->N, 256)); });
    rc = last_launch_error();
  }
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
  const long long K = (long long)C.nx * C.ny * C.nz;

  es_ctx* c = new (std::nothrow) es_ctx();
  if (!c) return ES_ERR_NOMEM;
  c->cfg = C;
  c->P1 = C.p + 1;
  c->Np = c->P1 * c->P1 * c->P1;
  c->K = (int)K;
  c->N = K * c->Np;
  c->tf = C.precision == ES_MIXED ? 4 : 8;
  c->tab = tableau(C.rk);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return ES_ERR_CUDA;
  }

  build_params(C, &c->P);

  const long long N = c->N;
  const long long P2 = (long long)c->P1 * c->P1;
  int rc = ES_OK;
  for (int i = 0; i < c->tab.s && rc == ES_OK; ++i) rc = dev_alloc(&c->k[i], 5 * N);
  if (rc == ES_OK) rc = cuda_check(cudaMalloc(&c->aux, kAux * N * c->tf)) == ES_OK ? ES_OK : ES_ERR_NOMEM;
  if (rc == ES_OK) rc = cuda_check(cudaMalloc(&c->F, 15 * K * P2 * c->tf)) == ES_OK ? ES_OK : ES_ERR_NOMEM;
  if (rc == ES_OK && C.mu > 0.0) rc = cuda_check(cudaMalloc(&c->fV, 12 * N * c->tf)) == ES_OK ? ES_OK : ES_ERR_NOMEM;
  if (rc == ES_OK) rc = dev_alloc(&c->dw, 5 * N);
  if (rc == ES_OK) rc = dev_alloc(&c->d, 5 * N);
  if (rc == ES_OK) rc = dev_alloc(&c->A, K);
  if (rc == ES_OK) rc = dev_alloc(&c->gamma_elem, K);
  if (rc == ES_OK) rc = dev_alloc(&c->scal, 2);
  if (rc == ES_OK) rc = dev_alloc(&c->gmin, 1);
  if (rc == ES_OK) rc = dev_alloc(&c->status, 1);
  if (rc == ES_OK) rc = cuda_check(cudaMemset(c->status, 0, sizeof(int)));
  if (rc == ES_OK) rc = cuda_check(cudaMemset(c->scal, 0, 2 * sizeof(double)));
  if (rc == ES_OK) rc = dispatch(c, [&](auto L) { return cuda_check(decltype(L)::volume_setup()); });
  if (rc != ES_OK) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  return ES_OK;
}

void es_destroy(es_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  free_ctx(ctx);
}

int es_rhs(es_ctx* c, const double* q, double* dqdt, double* E_elem, void* stream) {
  if (!c || !q || !dqdt || q == dqdt) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  StagePrep sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.q = const_cast<double*>(q);  // read only: apply_update = 0
  sp.Np = c->Np;
  StageVol sv;
  std::memset(&sv, 0, sizeof(sv));
  sv.kout = dqdt;
  sv.E = E_elem;
  return run_stage(c, sp, sv, st);
}

int es_entropy(es_ctx* c, const double* q, double* eta, void* stream) {
  if (!c || !q || !eta) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = (int)std::min<long long>((c->K + 3) / 4, (long long)c->sm_count * 16);
  return dispatch(c, [&](auto L) {
    timed(c, ES_KERNEL_OTHER, st, [&] { decltype(L)::entropy(c->P, q, eta, st, grid); });
    return last_launch_error();
  });
}

int es_relax_step(es_ctx* c, const double* u_old, const double* u_new, const double* d_eta, double* gamma_elem,
                  double* gamma, double* u_out, void* stream) {
  if (!c || !u_old || !u_new || !d_eta || !u_out || u_out == u_old) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  timed(c, ES_KERNEL_OTHER, st, [&] { launch_reset_min(c->gmin, st); });
  StageRelax sr = relax_base(c);
  sr.u = u_old;
  sr.u_new = u_new;
  sr.deta = d_eta;
  sr.d_out = c->d;
  int rc = run_relax(c, sr, st);
  if (rc != ES_OK) return rc;
  timed(c, ES_KERNEL_OTHER, st, [&] { launch_scalar(c->gmin, c->scal, c->scal + 1, nullptr, 0, 0.0, 1, st); });
  timed(c, ES_KERNEL_OTHER, st,
        [&] { launch_update(u_out, u_old, c->d, c->scal, 5 * c->N, st, grid_for(c, 5 * c->N, 256)); });
  rc = last_launch_error();
  if (rc != ES_OK) return rc;
  if (gamma_elem) {
    rc = cuda_check(cudaMemcpyAsync(gamma_elem, c->gamma_elem, sizeof(double) * c->K, cudaMemcpyDeviceToDevice, st));
    if (rc != ES_OK) return rc;
  }
  if (gamma) rc = cuda_check(cudaMemcpyAsync(gamma, c->scal, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return rc;
}

int es_advance(es_ctx* c, double* q, int nsteps, double dt, double* t, double* gamma_hist, double* gamma_elem,
               void* stream) {
  if (!c || !q || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return ES_ERR_INVALID;
  return advance_device(c, q, nsteps, dt, t, gamma_hist, gamma_elem, static_cast<cudaStream_t>(stream));
}

int es_advance_host(es_ctx* c, double* q_host, int nsteps, double dt, double* t_host, double* gamma_hist_host,
                    void* stream) {
  if (!c || !q_host || !t_host || nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ES_OK;
  if (!c->q_host_dev) rc = dev_alloc(&c->q_host_dev, 5 * c->N);
  if (rc == ES_OK && !c->t_host_dev) rc = dev_alloc(&c->t_host_dev, 1);
  if (rc == ES_OK && gamma_hist_host && c->hist_cap < nsteps) {
    cudaFree(c->hist_host_dev);
    c->hist_host_dev = nullptr;
    c->hist_cap = 0;
    rc = dev_alloc(&c->hist_host_dev, nsteps);
    if (rc == ES_OK) c->hist_cap = nsteps;
  }
  if (rc != ES_OK) return rc;
  const size_t qb = sizeof(double) * 5 * c->N;
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

int es_node_coords(const es_ctx* c, double* xyz) {
  if (!c || !xyz) return ES_ERR_INVALID;
  double x[kMaxP1], w[kMaxP1], D[kMaxP1 * kMaxP1];
  lgl_tables(c->cfg.p, x, w, D);
  const int P1 = c->P1;
  const long long N = c->N;
  const int nxyz[3] = {c->cfg.nx, c->cfg.ny, c->cfg.nz};
  for (int e = 0; e < c->K; ++e) {
    const int ei[3] = {e % nxyz[0], (e / nxyz[0]) % nxyz[1], e / (nxyz[0] * nxyz[1])};
    for (int n = 0; n < c->Np; ++n) {
      const int ni[3] = {n % P1, (n / P1) % P1, n / (P1 * P1)};
      for (int m = 0; m < 3; ++m) {
        const double h = (c->cfg.hi[m] - c->cfg.lo[m]) / nxyz[m];
        xyz[m * N + (long long)e * c->Np + n] = c->cfg.lo[m] + h * (ei[m] + 0.5 * (1.0 + x[ni[m]]));
      }
    }
  }
  return ES_OK;
}

int es_status(es_ctx* c, void* stream) {
  if (!c) return ES_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  int rc = cuda_check(cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (rc == ES_OK) rc = cuda_check(cudaStreamSynchronize(st));
  if (rc != ES_OK) return rc;
  if (h) {
    rc = cuda_check(cudaMemsetAsync(c->status, 0, sizeof(int), st));
    if (rc == ES_OK) rc = cuda_check(cudaStreamSynchronize(st));
    if (rc != ES_OK) return rc;
  }
  if (h & kStatusNonphysical) return ES_ERR_NONPHYSICAL;
  if (h & kStatusNoRoot) return ES_ERR_NO_ROOT;
  return ES_OK;
}

long long es_launch_count(const es_ctx* c) { return c ? c->launches : 0; }

int es_profile_enable(es_ctx* c, int enable) {
  if (!c) return ES_ERR_INVALID;
  if (!enable) flush_marks(c);
  c->profiling = enable != 0;
  return ES_OK;
}

int es_profile_read(es_ctx* c, double* ms, long long* launches) {
  if (!c || !ms || !launches) return ES_ERR_INVALID;
  flush_marks(c);
  for (int k = 0; k < ES_KERNEL_COUNT; ++k) {
    ms[k] = c->prof_ms[k];
    launches[k] = c->prof_n[k];
    c->prof_ms[k] = 0.0;
    c->prof_n[k] = 0;
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
// small kernels
namespace {

__global__ void k_scalar(unsigned long long* gmin_bits, double* gamma_cur, double* t, double* hist, int step,
                         double dt, int relax) {
  double g = __longlong_as_double((long long)*gmin_bits);
  if (!relax || !(g < INFINITY)) g = 1.0;
  *gamma_cur = g;
  *t += g * dt;
  if (hist) hist[step] = g;
  *gmin_bits = 0x7ff0000000000000ULL;
}

__global__ void k_reset_min(unsigned long long* gmin_bits) { *gmin_bits = 0x7ff0000000000000ULL; }

// out = base + gamma d (out may alias base)
__global__ void k_update(double* out, const double* base, const double* __restrict__ d,
                         const double* __restrict__ gamma_cur, long long n) {
  const double g = *gamma_cur;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = base[i] + g * d[i];
}

}  // namespace

namespace es {
void launch_scalar(unsigned long long* gmin_bits, double* gamma_cur, double* t, double* hist, int step, double dt,
                   int relax, cudaStream_t st) {
  k_scalar<<<1, 1, 0, st>>>(gmin_bits, gamma_cur, t, hist, step, dt, relax);
}
void launch_reset_min(unsigned long long* gmin_bits, cudaStream_t st) { k_reset_min<<<1, 1, 0, st>>>(gmin_bits); }
void launch_update(double* out, const double* base, const double* d, const double* gamma_cur, long long n,
                   cudaStream_t st, int grid) {
  k_update<<<grid, 256, 0, st>>>(out, base, d, gamma_cur, n);
}
}  // namespace es

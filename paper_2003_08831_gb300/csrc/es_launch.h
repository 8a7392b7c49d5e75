// Host-visible launch interface between the C ABI (es_api.cu) and the
// per-degree kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "../../include/es.h"
#include "es_device.cuh"

namespace es {

// host helpers shared by the entry points (es_api.cu)
int validate_config(const es_config& C);
void build_params(const es_config& C, Params* out);
int grid_for_sms(int sm_count, long long n, int block);

// k_prep: stage state y = u (+ gamma d first) + sum_j coef[j] k[j]
struct StagePrep {
  double* q;                // u, updated in place when apply_update
  const double* d;          // previous step's increment (apply_update)
  const double* gamma_cur;  // device scalar (apply_update)
  int apply_update;
  int nprev;
  double coef[4];           // dt a_ij
  const double* k[4];
  double* dw;               // w(y) - w(u) output, or nullptr
  int Np;
};

// k_volume outputs
struct StageVol {
  double* kout;        // k_i = f(y^i) (unless d_out is set)
  double* d_out;       // last stage: d = dcoef_self k_i + sum_j dcoef[j] dk[j] instead of k_i
  int nd;
  double dcoef[4];
  const double* dk[4];
  double dcoef_self;
  double* E;           // (eta' f)(y^i) per element, or nullptr
  const double* dw;    // w(y^i) - w(u), or nullptr
  double* A;           // relaxation term accumulator, or nullptr
  double A_scale;      // -dt b_i
  int A_init;          // first stage of the step: A starts at zero
};

// k_relax inputs/outputs
struct StageRelax {
  const double* u;         // u_old
  const double* u_new;     // if set: d = u_new - u_old, A = sum P w(u).d - deta
  const double* deta;      // eta_new - eta_old per element (u_new mode)
  const double* d_in;      // d = u_new - u_old (RK mode: written by the last stage)
  const double* A;         // accumulated A (RK mode)
  double* d_out;           // u_new mode: d written here
  double* gamma_elem;
  unsigned long long* gmin_bits;
  int* status;
  double delta_floor;
  double gamma_max;
};

template <int P1, typename TF>
struct Launcher {
  static void prep(const Params& P, const StagePrep& sp, void* aux, int* status, cudaStream_t st, int grid);
  static void face(const Params& P, const void* aux, void* F, cudaStream_t st, int grid);
  static void grad(const Params& P, const void* aux, void* fV, cudaStream_t st, int grid);
  static size_t volume_smem();
  static cudaError_t volume_setup();
  static void volume(const Params& P, const StageVol& sv, const void* aux, const void* F, const void* fV, bool ns,
                     cudaStream_t st);
  static void relax(const Params& P, const StageRelax& sr, cudaStream_t st, int grid);
  static void entropy(const Params& P, const double* q, double* eta, cudaStream_t st, int grid);
};

// scalar step bookkeeping: gamma = min gamma_kappa (or 1), t += gamma dt,
// hist[step] = gamma, reset of the min accumulator
void launch_scalar(unsigned long long* gmin_bits, double* gamma_cur, double* t, double* hist, int step, double dt,
                   int relax, cudaStream_t st);
// out = base + gamma d over n values (out may alias base)
void launch_update(double* out, const double* base, const double* d, const double* gamma_cur, long long n,
                   cudaStream_t st, int grid);
void launch_reset_min(unsigned long long* gmin_bits, cudaStream_t st);

}  // namespace es

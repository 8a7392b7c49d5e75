// Host-visible launch interface between the C ABI (es_api.cu) and the
// per-degree kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "../../include/es.h"
#include "es_device.cuh"

namespace es {

// host helpers shared by the entry points (es_api.cu)
int validate_config(const es_config& C);
InstGeom instance_geom(const es_config& C, int off);
void build_params(const es_config& C, Params* out);
int grid_for_sms(int sm_count, long long n, int block);
void ff_split_host(double d, float out[2]);

// explicit Runge--Kutta tableaux of up to kMaxStages stages
constexpr int kMaxStages = 10;

// k_prep: stage state y = u (+ gamma d first) + dt sum_j coef[j] k[j]
struct StagePrep {
  double* q;                // u, updated in place when an update is pending
  const double* d;          // previous step's increment
  const double* gamma_cur;  // per instance: gamma of the previous step
  const int* pending;       // per instance: relaxed update u += gamma d not yet applied (nullptr: none)
  int nprev;
  double coef[kMaxStages];  // a_ij (multiplied by the instance's dt in the kernel)
  const void* k[kMaxStages];  // stage values in the flux precision (double, float or float-float)
  double* dw;               // w(y) - w(u) output, or nullptr (FP64; float-float estimate
                            // modes store (hi, lo) float pairs in the same 8 bytes)
  int Np;
};

// k_volume outputs
struct StageVol {
  void* kout;          // k_i = f(y^i) in the flux precision (unless d_out or kout64 is set)
  double* kout64;      // k_i = f(y^i) in FP64 (the right-hand-side entry points)
  double* d_out;       // last stage: d = dt (dcoef_self k_i + sum_j dcoef[j] dk[j]) instead of k_i
  int nd;
  double dcoef[kMaxStages];    // b_j
  const void* dk[kMaxStages];  // earlier stages' k in the flux precision
  double dcoef_self;   // b_i
  // the same coefficients as float-float pairs (hi, lo), split on the host exactly as
  // ff_from_double splits on the device (float-float estimate modes read these)
  float dcoef_ff[kMaxStages][2];
  float dcoef_self_ff[2];
  double* E;           // (eta' f)(y^i) per element, or nullptr
  const double* dw;    // w(y^i) - w(u), or nullptr (float-float estimate modes: (hi, lo)
                       // float pairs in the same 8 bytes per value)
  double* A;           // relaxation term accumulator, or nullptr
  double A_scale;      // -b_i (times the instance's dt in the kernel)
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
  unsigned long long* gmin_bits;  // per instance
  int* status;
  double delta_floor;
  double gamma_max;
  double root_rtol;        // Newton-step stop |step| <= root_rtol gamma
};

// global relaxation: per-instance Newton state
struct GlobalRelaxState {
  double g, lo, hi, a, A, result;
  int hi_known, done;
};

struct GlobalRelaxArgs {
  const double* u;
  const double* d;
  const double* A;       // per element
  double* nodes;         // [4][N] scratch
  double* elem_a;        // [K]
  double* elem_s;        // [K]
  double* elem_r;        // [K]
  double* elem_dr;       // [K]
  GlobalRelaxState* gs;  // [ninst]
  unsigned long long* gmin_bits;
  double* gamma_elem;
  int* status;
  double delta_floor, gamma_max, root_rtol;
};

constexpr int kGlobalRelaxIterations = 8;
// volume tiles 0..2: k_prep + k_face + k_volume; 3..5: k_prep + k_volume with the
// interface fluxes formed in the volume kernel (FP32 fluxes on periodic Euler groups)
constexpr int kVolumeVariants = 3;
constexpr int kStageVariants = 2 * kVolumeVariants;

template <int P1, typename TF>
struct Launcher {
  static void prep(const Params& P, const StagePrep& sp, void* aux, int* status, cudaStream_t st, int grid);
  // FL: -x_m boundary-face fluxes of the first elements along non-periodic directions (or null)
  static void face(const Params& P, const void* aux, void* F, void* FL, cudaStream_t st, int grid);
  static void grad(const Params& P, const void* aux, void* fV, cudaStream_t st, int grid);
  static cudaError_t volume_setup();
  // variant: volume tile (elements per CTA, threads), 0..kVolumeVariants-1
  static void volume(const Params& P, const StageVol& sv, const void* aux, const void* F, const void* FL,
                     const void* fV, bool ns, cudaStream_t st, int variant);
  // k_volume with the interface fluxes evaluated in the kernel (TF = float, Euler, periodic)
  static cudaError_t volface_setup();
  static void volface(const Params& P, const StageVol& sv, const void* aux, cudaStream_t st, int variant);
  static void relax(const Params& P, const StageRelax& sr, cudaStream_t st, int grid);
  static void entropy(const Params& P, const double* q, double* eta, cudaStream_t st, int grid);
  // Theorem 2.3's eta_kappa(u) and estimate deta_kappa = sum P w(u).d - A (either output may be null)
  static void estimate(const Params& P, const double* q, const double* d, const double* A, double* eta_old,
                       double* deta, cudaStream_t st, int grid);
  static void global_relax(const Params& P, const GlobalRelaxArgs& ga, cudaStream_t st, int grid, int iterations);
};

// per-instance step bookkeeping: gamma = min gamma_kappa (or 1), t += gamma dt,
// hist[i] = gamma (if hist), pending[i] = 1, reset of the min accumulator
void launch_scalar(const Params& P, unsigned long long* gmin_bits, double* gamma_cur, double* t, double* hist,
                   int* pending, int relax, cudaStream_t st);
// out = base + gamma[inst] d over the group's 5 K Np values where pending[inst] (out may alias base)
void launch_update(const Params& P, double* out, const double* base, const double* d, const double* gamma_cur,
                   const int* pending, int Np, cudaStream_t st, int grid);
void launch_reset(unsigned long long* gmin_bits, int* pending, int ninst, cudaStream_t st);

}  // namespace es

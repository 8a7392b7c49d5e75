// es_rhs_noalloc: the right-hand side without a context and without any
// allocation, for callers that cannot allocate device memory (see es.h).
//
// The kernels' scratch (parameter-vector state, interface fluxes, viscous
// fluxes, the status word) lives in one file-scope __device__ array of fixed
// size.  Host code never dereferences that symbol: on the first call on each
// device (with that device current) cudaGetSymbolAddress gives its device
// address, which is cached per device ordinal and passed to the kernels.
#include <cuda_runtime.h>

#include <cstdio>

#include "../../include/es.h"
#include "es_launch.h"

using namespace es;

namespace {

constexpr size_t kNoallocScratchBytes = size_t(ES_NOALLOC_SCRATCH_BYTES);
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// per device: scratch address and whether the one-time set-up has run
void* g_scratch_ptr[kMaxDevices];
int g_sm_count[kMaxDevices];
bool g_ready[kMaxDevices];

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename F>
int dispatch_p1(int P1, bool fp64, F&& f) {
  switch (P1) {
    case 3: return fp64 ? f(Launcher<3, double>()) : f(Launcher<3, float>());
    case 4: return fp64 ? f(Launcher<4, double>()) : f(Launcher<4, float>());
    case 5: return fp64 ? f(Launcher<5, double>()) : f(Launcher<5, float>());
    case 6: return fp64 ? f(Launcher<6, double>()) : f(Launcher<6, float>());
  }
  return ES_ERR_INVALID;
}

// A runtime call that failed also left its error as the thread's last error; it is
// taken back here so that the next call (ours or the caller's) does not report it.
int failed(cudaError_t e, const char* what) {
  std::fprintf(stderr, "es_rhs_noalloc: %s failed: %s\n", what, cudaGetErrorString(e));
  cudaGetLastError();
  return ES_ERR_CUDA;
}

int setup_device(int dev) {
  if (g_ready[dev]) return ES_OK;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return failed(e, "cudaGetSymbolAddress");
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return failed(e, "cudaDeviceGetAttribute");
  // opt the volume kernels into their dynamic shared memory (no allocation)
  for (int P1 = 3; P1 <= 6; ++P1) {
    for (int fp64 = 0; fp64 < 2; ++fp64) {
      const cudaError_t es = [&] {
        cudaError_t r = cudaSuccess;
        dispatch_p1(P1, fp64 != 0, [&](auto L) {
          r = decltype(L)::volume_setup();
          return ES_OK;
        });
        return r;
      }();
      if (es != cudaSuccess) return failed(es, "cudaFuncSetAttribute");
    }
  }
  g_scratch_ptr[dev] = ptr;
  g_sm_count[dev] = sms;
  g_ready[dev] = true;
  return ES_OK;
}

}  // namespace

extern "C" size_t es_rhs_noalloc_scratch_bytes(const es_config* cfg) {
  if (!cfg || validate_config(*cfg) != ES_OK) return 0;
  const size_t tf = (cfg->precision == ES_MIXED || cfg->precision == ES_MIXED_FF) ? 4 : 8;
  const size_t P1 = size_t(cfg->p) + 1;
  const size_t K = size_t(cfg->nx) * cfg->ny * cfg->nz;
  const size_t N = K * P1 * P1 * P1;
  size_t b = align256(sizeof(int));
  b += align256(kAuxPlanes * N * tf);
  b += align256(15 * K * P1 * P1 * tf);
  if (cfg->mu > 0.0) b += align256(12 * N * tf);
  return b;
}

extern "C" int es_rhs_noalloc(const es_config* cfg, const double* q, double* dqdt, double* E_elem, void* stream) {
  if (!cfg || !q || !dqdt || q == dqdt) return ES_ERR_INVALID;
  if (validate_config(*cfg) != ES_OK) return ES_ERR_INVALID;
  const size_t need = es_rhs_noalloc_scratch_bytes(cfg);
  if (need > kNoallocScratchBytes) return ES_ERR_TOO_LARGE;
  // an error left pending by earlier work stays the caller's: it is reported here
  // (before anything is enqueued) and not cleared, so that the launch check at the
  // end sees only this call's launches
  if (cudaPeekAtLastError() != cudaSuccess) return ES_ERR_CUDA;
  int dev = 0;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return failed(de, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return ES_ERR_CUDA;
  int rc = setup_device(dev);
  if (rc != ES_OK) return rc;

  Params P;
  build_params(*cfg, &P);
  const bool fp64 = cfg->precision != ES_MIXED && cfg->precision != ES_MIXED_FF;
  const size_t tf = fp64 ? 8 : 4;
  const int P1 = cfg->p + 1;
  const long long K = (long long)cfg->nx * cfg->ny * cfg->nz;
  const long long Np = (long long)P1 * P1 * P1;
  const long long N = K * Np;
  unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  int* status = reinterpret_cast<int*>(base);
  size_t off = align256(sizeof(int));
  void* aux = base + off;
  off += align256(kAuxPlanes * size_t(N) * tf);
  void* F = base + off;
  off += align256(15 * size_t(K) * P1 * P1 * tf);
  void* fV = cfg->mu > 0.0 ? static_cast<void*>(base + off) : nullptr;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the status word accumulates bits with atomicOr: it must start at zero
  const cudaError_t me = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (me != cudaSuccess) return failed(me, "cudaMemsetAsync");
  StagePrep sp = {};
  sp.q = const_cast<double*>(q);  // read only: apply_update = 0
  sp.Np = int(Np);
  StageVol sv = {};
  sv.kout64 = dqdt;
  sv.E = E_elem;
  const int sms = g_sm_count[dev];
  const bool ns = cfg->mu > 0.0;
  rc = dispatch_p1(P1, fp64, [&](auto L) {
    using Lc = decltype(L);
    Lc::prep(P, sp, aux, status, st, grid_for_sms(sms, N, 256));
    Lc::face(P, aux, F, nullptr, st, grid_for_sms(sms, 3LL * K * P1 * P1, 256));
    if (ns) Lc::grad(P, aux, fV, st, grid_for_sms(sms, N, 256));
    Lc::volume(P, sv, aux, F, nullptr, fV, ns, st, 0);
    return ES_OK;
  });
  if (rc != ES_OK) return rc;
  // the launches' own errors (no earlier error was pending at entry)
  const cudaError_t le = cudaGetLastError();
  return le == cudaSuccess ? ES_OK : failed(le, "kernel launch");
}

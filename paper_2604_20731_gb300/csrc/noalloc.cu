// Saturation step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a serving process whose own allocator
// owns the whole device memory budget, or a latency-critical loop that must
// not risk the implicit device synchronisation cudaMalloc/cudaFree can cause.
// ads_saturation_step_noalloc gives them one explicit saturation step that
// allocates nothing: the caller passes its device inputs and output, and all
// the working memory the step needs (basis and mass-matrix tables, per-axis
// source factors, the rows shared between strips, per-block partial sums)
// lives in one file-scope device array of fixed size, reserved on every GPU
// that loads the library for as long as the library stays loaded.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <mutex>
#include <thread>

#include "../../include/adsgb.h"
#include "kernels.cuh"

namespace adsgb {
ads_status validate_params(const ads_params* p, const crvpinn_params* cp);  // api.cu
}

using namespace adsgb;

namespace {

constexpr size_t kScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr int kMaxN = 512;
constexpr int kStripRows = 4;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host-side address of the array on each device.  In host code the name
// g_noalloc_scratch is only a stand-in, never a device address.
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

struct SrcVals {
  double cen[3 * kMaxSrc];
  double sig[kMaxSrc];
  double dt;
};

// writes the sources' centres/widths and the step size into the scratch; the
// status word is left alone, so a problem seen by any step stays visible until
// ads_saturation_step_noalloc_status reads and clears it
__global__ void k_noalloc_put(SrcVals v, double* cen, double* sig, double* dt) {
  int t = threadIdx.x;
  if (t < 3 * kMaxSrc) cen[t] = v.cen[t];
  if (t < kMaxSrc) sig[t] = v.sig[t];
  if (t == 0) *dt = v.dt;
}

// polls the stream until its work is done: cudaSuccess, or cudaErrorNotReady
// once kWaitSeconds have passed, or the stream's error
constexpr double kWaitSeconds = 10.0;
cudaError_t wait_stream(cudaStream_t st) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e != cudaErrorNotReady) return e;
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > kWaitSeconds)
      return cudaErrorNotReady;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Carve {
  unsigned char* base;
  size_t off = 0;
  double* take(size_t count) {
    double* p = reinterpret_cast<double*>(base + off);
    off += align256(count * sizeof(double));
    return p;
  }
};

}  // namespace

extern "C" ads_status ads_saturation_step_noalloc(const ads_params* p, const double* d_K,
                                                  const double* d_phi, const double* d_S,
                                                  const double* d_P, double dt, double* d_S_out,
                                                  void* stream) {
  if (!p || !d_K || !d_S || !d_P || !d_S_out) return ADS_ERR_INVALID_ARG;
  if (d_S == d_S_out) return ADS_ERR_INVALID_ARG;
  // the same parameter check as ads_init (no CUDA call), then this step's limits
  const ads_status v0 = validate_params(p, nullptr);
  if (v0 != ADS_OK) return v0;
  if (p->dim != 2 || p->ads_dtype != ADS_F64) return ADS_ERR_UNSUPPORTED;
  if (p->n > kMaxN) return ADS_ERR_INVALID_ARG;
  if (!(dt > 0) || !std::isfinite(dt)) return ADS_ERR_INVALID_ARG;
  const int n = p->n, nb = n + 2;
  const int nquad = quad_blocks(2, n, kStripRows);
  const int nys = ysolve_blocks(2, n);
  const int ldx = sweep_ld(n);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADS_ERR_CUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return ADS_ERR_CUDA;

  Carve cv{static_cast<unsigned char*>(base)};
  // the status word first, at a fixed place, so that the status call finds it
  int* flags = reinterpret_cast<int*>(cv.take(1));
  double* stats = cv.take(3);
  double* B = cv.take(9 * (size_t)n);
  double* dB = cv.take(9 * (size_t)n);
  double* l1 = cv.take((size_t)n + 4);
  double* l2 = cv.take((size_t)n + 4);
  double* dinv = cv.take((size_t)nb);
  double* Iw = cv.take((size_t)nb);
  double* gsrc = cv.take(3 * (size_t)kMaxSrc * n * 3);
  double* gnode = cv.take(3 * (size_t)kMaxSrc * (n + 1));
  double* tmp = cv.take(3 * ((size_t)n + 4));
  double* cen = cv.take(3 * kMaxSrc);
  double* sig = cv.take(kMaxSrc);
  double* dtp = cv.take(1);
  double* Xs = cv.take(2 * (size_t)nquad * ldx);
  double* Xm = cv.take((size_t)nb * ldx);
  double* src_part = cv.take((size_t)nquad);
  double* mass_part = cv.take((size_t)nys);
  if (cv.off > kScratchBytes) return ADS_ERR_INVALID_ARG;  // cannot happen for n <= kMaxN

  cudaStream_t st = (cudaStream_t)stream;
  SrcVals v{};
  for (int s = 0; s < kMaxSrc; ++s) v.sig[s] = 1.0;
  for (int s = 0; s < p->n_src; ++s) {
    for (int d = 0; d < 3; ++d) v.cen[s * 3 + d] = p->src[s].center[d];
    v.sig[s] = p->src[s].sigma;
  }
  v.dt = dt;
  k_noalloc_put<<<1, 32, 0, st>>>(v, cen, sig, dtp);
  // every table, spill row and partial below is fully rewritten before it is
  // read, so nothing in the shared array has to start at zero
  if (launch_axis_init(n, cen, sig, p->n_src, B, dB, l1, l2, dinv, Iw, gsrc, gnode, tmp, st) !=
      cudaSuccess)
    return ADS_ERR_CUDA;

  QuadArgs<double> a{};
  a.dim = 2;
  a.n = n;
  a.nb = nb;
  a.h = 1.0 / n;
  a.S = d_S;
  a.P = d_P;
  a.K = d_K;
  a.phi = d_phi;
  a.phi_c = p->phi;
  a.nodal = nullptr;
  a.ax.B = B;
  a.ax.dB = dB;
  a.ax.l1 = l1;
  a.ax.l2 = l2;
  a.ax.dinv = dinv;
  a.ax.Iw = Iw;
  a.ax.gsrc = gsrc;
  a.ax.gnode = gnode;
  a.n_src = p->n_src;
  for (int s = 0; s < kMaxSrc; ++s) {
    a.rate[s] = s < p->n_src ? p->src[s].rate : 0.0;
    a.kind[s] = s < p->n_src ? p->src[s].kind : 0;
  }
  a.inv_mu_g = 1.0 / p->mu_g;
  a.inv_mu_w = 1.0 / p->mu_w;
  a.grav_term = p->grav_sign * p->rho_g * p->grav;
  a.kz = p->kz_ratio;
  a.dt = dtp;
  if (launch_quad_xsweep<double>(a, 0, kStripRows, Xm, Xs, ldx, src_part, st) != cudaSuccess)
    return ADS_ERR_CUDA;
  if (launch_ysweep<double>(a, kStripRows, Xm, Xs, ldx, d_S_out, mass_part, flags, st) !=
      cudaSuccess)
    return ADS_ERR_CUDA;
  // int S_out from the y sweep's partials: sets bit 0 of the status word when
  // it is not finite (the context path runs the same check)
  if (launch_mass_finalize(mass_part, ysweep_blocks(n, sizeof(double)), nullptr, 0, 0, stats, flags,
                           st) != cudaSuccess)
    return ADS_ERR_CUDA;
  return ADS_OK;
}

extern "C" ads_status ads_saturation_step_noalloc_status(void* stream, int* flags_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADS_ERR_CUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return ADS_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // wait for the stream's queued steps, with a deadline, before the read
  // (a plain synchronise could block for ever behind a stuck kernel)
  if (wait_stream(st) != cudaSuccess) return ADS_ERR_TIMEOUT;
  int word = 0;
  if (cudaMemcpyAsync(&word, base, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return ADS_ERR_CUDA;
  if (cudaMemsetAsync(base, 0, sizeof(int), st) != cudaSuccess) return ADS_ERR_CUDA;
  if (wait_stream(st) != cudaSuccess) return ADS_ERR_TIMEOUT;
  if (flags_out) *flags_out = word;
  if (word & 8) return ADS_ERR_TIMEOUT;
  if (word & 1) return ADS_ERR_NONFINITE;
  return ADS_OK;
}

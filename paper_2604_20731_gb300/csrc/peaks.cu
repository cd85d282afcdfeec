// Measured issue rates of the arithmetic units the kernels lean on: the
// special-function unit (ex2.approx, rcp.approx: tanh costs one of each) and
// the FP32 FMA pipe (scalar fma and the packed fma.rn.f32x2 of sm_100+).
//
// The rooflines of the network forward (special-function bound) and of the
// saturation quadrature (FP32 issue bound) need these peaks; no vendor table
// of per-clock unit rates for sm_103 is at hand, so they are measured here:
// one wave of CTAs (the occupancy limit times the SM count), each thread
// running 8 independent dependency chains of one operation, timed with CUDA
// events and with the SM cycle counter.
#include <cuda_runtime.h>

#include "../../include/adsgb.h"
#include "kernels.cuh"

namespace adsgb {
namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

enum Op { kEx2 = 0, kRcp = 1, kTanh = 2, kFfma = 3, kFfma2 = 4, kNumOps = 5 };

template <int OP>
__global__ void __launch_bounds__(kThreads) k_unit_rate(float* sink, int iters, unsigned long long* cyc) {
  float x[kChains], y[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = 0.25f + 0.01f * (float)((threadIdx.x + c) & 15);
    y[c] = 0.5f + 0.01f * (float)c;
  }
  const float a = 0.9990234375f, b = 0.0009765625f;
  __syncthreads();
  const unsigned long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (OP == kEx2) {
        float t;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(-x[c]));  // stays in (0, 1]
        x[c] = t;
      } else if (OP == kRcp) {
        float t;
        // x <- 1/x + 1/2 (converges to about 1.21); the add keeps the two
        // reciprocals of a pair from folding into the identity
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(x[c]));
        x[c] = t + 0.5f;
      } else if (OP == kTanh) {
        float t, r;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(-x[c]));
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + t));  // in [1/2, 1)
        x[c] = r;
      } else if (OP == kFfma) {
        x[c] = fmaf(x[c], a, b);
        y[c] = fmaf(y[c], a, b);
      } else {
        float2 v = make_float2(x[c], y[c]);
        v = __ffma2_rn(v, make_float2(a, a), make_float2(b, b));
        x[c] = v.x;
        y[c] = v.y;
      }
    }
  }
  const unsigned long long t1 = clock64();
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c] + y[c];
  sink[blockIdx.x * kThreads + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// results one thread produces per iteration
constexpr int results_per_iter(int op) { return op >= kFfma ? 2 * kChains : kChains; }

template <int OP>
cudaError_t run_one(int iters, float* sink, unsigned long long* cyc, int blocks, cudaStream_t st) {
  k_unit_rate<OP><<<blocks, kThreads, 0, st>>>(sink, iters, cyc);
  return cudaGetLastError();
}

cudaError_t run_op(int op, int iters, float* sink, unsigned long long* cyc, int blocks, cudaStream_t st) {
  switch (op) {
    case kEx2: return run_one<kEx2>(iters, sink, cyc, blocks, st);
    case kRcp: return run_one<kRcp>(iters, sink, cyc, blocks, st);
    case kTanh: return run_one<kTanh>(iters, sink, cyc, blocks, st);
    case kFfma: return run_one<kFfma>(iters, sink, cyc, blocks, st);
    default: return run_one<kFfma2>(iters, sink, cyc, blocks, st);
  }
}

int occupancy(int op) {
  int nb = 0;
  cudaError_t e;
  switch (op) {
    case kEx2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_unit_rate<kEx2>, kThreads, 0); break;
    case kRcp: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_unit_rate<kRcp>, kThreads, 0); break;
    case kTanh: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_unit_rate<kTanh>, kThreads, 0); break;
    case kFfma: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_unit_rate<kFfma>, kThreads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_unit_rate<kFfma2>, kThreads, 0); break;
  }
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

}  // namespace
}  // namespace adsgb

using namespace adsgb;

extern "C" ads_status ads_measure_unit_rates(double* out, int nout) {
  if (!out || nout < 2 * kNumOps + 1) return ADS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ADS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ADS_ERR_CUDA;
  int maxb = 1;
  for (int op = 0; op < kNumOps; ++op) maxb = occupancy(op) > maxb ? occupancy(op) : maxb;
  const size_t nblk_max = (size_t)sms * maxb;
  float* sink = nullptr;
  unsigned long long* cyc = nullptr;
  unsigned long long* hcyc = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ads_status rc = ADS_OK;
  if (cudaMalloc(&sink, nblk_max * kThreads * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&cyc, nblk_max * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&hcyc, nblk_max * sizeof(unsigned long long)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = ADS_ERR_CUDA;
  }
  double clk_sum = 0.0;
  for (int op = 0; op < kNumOps && rc == ADS_OK; ++op) {
    const int blocks = sms * occupancy(op);
    const int iters = op >= kFfma ? 16384 : 4096;
    float best_ms = 1e30f;
    unsigned long long best_cyc = 0;
    for (int rep = 0; rep < 4 && rc == ADS_OK; ++rep) {  // first run is a warm-up
      if (cudaEventRecord(e0, st) != cudaSuccess || run_op(op, iters, sink, cyc, blocks, st) != cudaSuccess ||
          cudaEventRecord(e1, st) != cudaSuccess ||
          cudaMemcpyAsync(hcyc, cyc, blocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = ADS_ERR_CUDA;
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      unsigned long long cmax = 0;
      for (int b = 0; b < blocks; ++b) cmax = hcyc[b] > cmax ? hcyc[b] : cmax;
      if (rep > 0 && ms < best_ms) {
        best_ms = ms;
        best_cyc = cmax;
      }
    }
    if (rc != ADS_OK) break;
    const double results = (double)blocks * kThreads * iters * results_per_iter(op);
    out[op] = results / (best_ms * 1e-3);                      // results per second, whole GPU
    out[kNumOps + op] = results / sms / (double)best_cyc;      // results per clock per SM
    clk_sum += (double)best_cyc / (best_ms * 1e-3) / 1e6;      // SM MHz seen by the chains
  }
  if (rc == ADS_OK) out[2 * kNumOps] = clk_sum / kNumOps;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (hcyc) cudaFreeHost(hcyc);
  if (cyc) cudaFree(cyc);
  if (sink) cudaFree(sink);
  return rc;
}

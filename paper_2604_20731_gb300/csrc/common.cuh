// Shared device helpers for the adsgb kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define ADS_HD __host__ __device__ __forceinline__
#define ADS_D __device__ __forceinline__

namespace adsgb {

constexpr int kMaxSrc = 8;
constexpr int kLossRing = 4096;

// Gauss-Legendre rule with 3 points on [0,1]: 0.5 -+ sqrt(15)/10, 0.5;
// weights 5/18, 8/18, 5/18.
ADS_HD double gauss_x(int q) {
  return q == 0 ? 0.5 - 0.3872983346207416885 : (q == 1 ? 0.5 : 0.5 + 0.3872983346207416885);
}
ADS_HD double gauss_w(int q) { return q == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }

// Scalar parameters needed by the saturation and collocation kernels.
struct PhysParams {
  int dim, n;
  double h;
  double phi;
  double inv_mu_w, inv_mu_g, rho_w, rho_g;
  double grav, grav_sign, kz_ratio;
  int n_src;
  double src_rate[kMaxSrc];
  int src_kind[kMaxSrc];
};

template <typename T>
ADS_D T clamp01(T s) { return s < T(0) ? T(0) : (s > T(1) ? T(1) : s); }

// tanh from the exponential identity tanh x = 2 / (1 + e^{-2x}) - 1 with the
// hardware base-2 exponential and reciprocal (absolute error a few 1e-7; the
// limits come out exactly: e^{-2x} -> inf gives -1, -> 0 gives 1).
ADS_D float tanh_f32(float x) {
  float t, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(-2.8853900817779268f * x));  // -2 log2(e) x
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + t));
  return fmaf(2.0f, r, -1.0f);
}
ADS_D double tanh_any(double x) { return tanh(x); }
ADS_D float tanh_any(float x) { return tanh_f32(x); }

// Deterministic block sum of doubles (blockDim.x multiple of 32, <= 1024).
ADS_D double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r += sh[i];
  }
  return r;  // valid in thread 0
}

ADS_D double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    r = sh[0];
    for (int i = 1; i < nw; ++i) r = fmax(r, sh[i]);
  }
  return r;
}

// Asynchronous global -> shared copies (cp.async): the copy does not pass
// through registers, so a thread can keep many in flight and wait once.
ADS_D unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
ADS_D void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem)), "l"(gmem));
}
ADS_D void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(smem)), "l"(gmem));
}
ADS_D void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(smem)), "l"(gmem));
}
template <typename T>
ADS_D void cp_async_elem(T* smem, const T* gmem) {
  if (sizeof(T) == 8) cp_async8(smem, gmem);
  else cp_async4(smem, gmem);
}
ADS_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
ADS_D void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
ADS_D void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Allow a kernel the device's full opt-in dynamic shared memory (less its
// static shared memory).  Setting the limit to one launch's need would lower it
// for other launches of the same kernel (graphs captured for other sizes).
template <typename K>
inline void smem_optin(K k) {
  static int optin = 0;
  if (!optin) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (optin <= 0) optin = 48 * 1024;
  }
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// ---- bulk tensor copies (TMA) with bounded mbarrier waits ----
ADS_D unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
ADS_D void mbar_init_cta(uint64_t* mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive once and announce `bytes` of bulk-copy traffic on the barrier
ADS_D void mbar_arrive_tx(uint64_t* mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)),
               "r"(bytes)
               : "memory");
}
// wait for phase `parity`; false after `limit_ns` nanoseconds without it
ADS_D bool mbar_wait_for(uint64_t* mbar, unsigned parity, unsigned long long limit_ns) {
  const unsigned a = smem_addr(mbar);
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    unsigned done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = gtimer_ns();
    else if (gtimer_ns() - t0 > limit_ns) return false;
  }
}
// 2D tile load: box at element coordinates (x, y) of the tensor map into
// shared memory, completing on `mbar`.  x must be a multiple of 16 bytes'
// worth of elements; y may be negative (rows outside the tensor read as 0).
// one-dimensional bulk copy global -> shared, completing on `mbar` (both
// addresses 16-byte aligned, bytes a multiple of 16)
ADS_D void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(mbar))
      : "memory");
}
// order this thread's generic-proxy accesses to shared memory before later
// bulk-copy (async-proxy) accesses
ADS_D void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
ADS_D void tma_load_2d(void* smem_dst, const void* tmap, int x, int y, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(smem_dst)),
      "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x), "r"(y), "r"(smem_addr(mbar))
      : "memory");
}

// Compensated (Kahan) running sum.  FP32 sums whose small terms matter (the
// mass and source integrals) use it instead of an FP64 accumulator: FP64
// arithmetic on this GPU runs at a small fraction of the FP32 rate.
template <typename T>
struct CompSum {
  T s = T(0), c = T(0);
  ADS_D void add(T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  ADS_D double value() const { return (double)s - (double)c; }
};
template <>
struct CompSum<double> {
  double s = 0.0;
  ADS_D void add(double v) { s += v; }
  ADS_D double value() const { return s; }
};

}  // namespace adsgb

// Porosity and permeability given as images (Sec. 8.1).
//
// Sec. 8.1 gives each reservoir's porosity (values 0 to 1) and permeability
// (mDarcy) as a picture of the domain.  The method takes K and phi as nodal
// values on the (n+1)^d vertex grid: bi/trilinear at the Gauss points of the
// saturation step, the nodal value itself in the collocation coefficient of
// Eq. 23b.  This file brings a picture onto that grid.
//
// Reading: a pixel holds one value over its square (cube) of the unit domain,
// and a node takes that field's average over its dual cell, [x_i - h/2,
// x_i + h/2] per axis clipped to [0, 1] -- the arithmetic mean, which keeps
// the map's integral because the dual cells tile the domain, or the geometric
// mean exp(avg log), the usual way to upscale a log-normal permeability.  The
// same rule serves a picture finer or coarser than the mesh, in any ratio.
//
// Exact overlaps: in units of 1 / (2 n m) (n elements, m pixels along an axis)
// the dual cell of node i is [(2i - 1) m, (2i + 1) m] and pixel c is
// [2 n c, 2 n (c + 1)], so every overlap is an integer; only the pixels with a
// positive overlap are visited.
//
// One thread per node visits the pixels of its dual cell (a few per axis when
// the picture is close to the mesh's resolution): the sums run in FP64 in a
// fixed order, rows of x-sums, then slices.  A node's neighbours read the
// neighbouring pixels, so a warp's reads fall in a few contiguous runs of
// each row, and the pixels shared by two dual cells come from L2.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdint>
#include <thread>

#include "adsgb.h"

namespace {

constexpr int kMaxMapN = 1 << 16;        // elements per axis
constexpr int kMaxMapPixels = 1 << 24;   // pixels per axis
constexpr long long kMaxMapNodes = (1LL << 31) - 1;

struct MapAxis {
  long long m;      // pixels along the axis
  long long n;      // elements along the axis
};

struct MapArgs {
  MapAxis ax[3];    // x, y, z (z: one slice and one node in 2D)
  int flip_y;
  double scale, offset;
  long long nodes;  // prod(n_a + 1)
};

// The pixel range [c0, c1] of node i's dual cell along one axis and the cell's
// length, all in units of 1 / (2 n m).
__device__ __forceinline__ void dual_range(const MapAxis& a, long long i, long long& lo, long long& hi,
                                           long long& c0, long long& c1) {
  const long long two_n = 2 * a.n;
  lo = (2 * i - 1) * a.m;
  hi = (2 * i + 1) * a.m;
  if (lo < 0) lo = 0;
  if (hi > two_n * a.m) hi = two_n * a.m;
  c0 = lo / two_n;               // the pixel holding the cell's left end
  c1 = (hi - 1) / two_n;         // the last pixel starting before its right end
}

__device__ __forceinline__ double overlap(long long lo, long long hi, long long two_n, long long c) {
  const long long a = two_n * c, b = a + two_n;
  return (double)((hi < b ? hi : b) - (lo > a ? lo : a));
}

template <typename Tp>
__device__ __forceinline__ double pixel_value(const Tp* img, long long idx, double scale, double offset) {
  return fma(scale, (double)img[idx], offset);
}

template <typename Tp, bool GEO>
__global__ void __launch_bounds__(256) k_map_nodal(const Tp* __restrict__ img, MapArgs a,
                                                   double* __restrict__ out, int* __restrict__ nonfinite) {
  const long long nx1 = a.ax[0].n + 1, ny1 = a.ax[1].n + 1;
  const long long W = a.ax[0].m, H = a.ax[1].m;
  int bad = 0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < a.nodes;
       node += (long long)gridDim.x * blockDim.x) {
    const long long i = node % nx1, j = (node / nx1) % ny1, k = node / (nx1 * ny1);
    long long xl, xh, x0, x1, yl, yh, y0, y1, zl, zh, z0, z1;
    dual_range(a.ax[0], i, xl, xh, x0, x1);
    dual_range(a.ax[1], j, yl, yh, y0, y1);
    dual_range(a.ax[2], k, zl, zh, z0, z1);
    const long long tx = 2 * a.ax[0].n, ty = 2 * a.ax[1].n, tz = 2 * a.ax[2].n;
    double acc = 0.0;
    for (long long s = z0; s <= z1; ++s) {
      const double wz = overlap(zl, zh, tz, s);
      double acc_z = 0.0;
      for (long long r = y0; r <= y1; ++r) {
        const double wy = overlap(yl, yh, ty, r);
        const long long row = (s * H + (a.flip_y ? H - 1 - r : r)) * W;
        double acc_y = 0.0;
        for (long long c = x0; c <= x1; ++c) {
          const double v = pixel_value(img, row + c, a.scale, a.offset);
          acc_y = fma(overlap(xl, xh, tx, c), GEO ? log(v) : v, acc_y);
        }
        acc_z = fma(wy, acc_y, acc_z);
      }
      acc = fma(wz, acc_z, acc);
    }
    double res = acc / ((double)(xh - xl) * (double)(yh - yl) * (double)(zh - zl));
    if (GEO) res = exp(res);
    out[node] = res;
    bad |= !isfinite(res);
  }
  if (bad) atomicAdd(nonfinite, 1);
}

cudaError_t wait_bounded(cudaStream_t st, double seconds) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery(st);
    if (e != cudaErrorNotReady) return e;
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > seconds)
      return cudaErrorNotReady;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" ads_status ads_map_from_image(const void* d_img, int pixel_type, int dim, const int* img_shape,
                                         int flip_y, const int* n, int mean, double scale, double offset,
                                         double* d_nodal, void* stream) {
  if (!d_img || !img_shape || !n || !d_nodal) return ADS_ERR_INVALID_ARG;
  if (dim != 2 && dim != 3) return ADS_ERR_INVALID_ARG;
  if (pixel_type != ADS_PIXEL_F32 && pixel_type != ADS_PIXEL_U8) return ADS_ERR_INVALID_ARG;
  if (mean != ADS_MAP_ARITHMETIC && mean != ADS_MAP_GEOMETRIC) return ADS_ERR_INVALID_ARG;
  if (!std::isfinite(scale) || !std::isfinite(offset)) return ADS_ERR_INVALID_ARG;
  MapArgs a{};
  a.nodes = 1;
  long long pixels = 1;
  for (int ax = 0; ax < 3; ++ax) {
    if (ax < dim) {
      if (img_shape[ax] < 1 || img_shape[ax] > kMaxMapPixels || n[ax] < 1 || n[ax] > kMaxMapN)
        return ADS_ERR_INVALID_ARG;
      a.ax[ax] = MapAxis{img_shape[ax], n[ax]};
      a.nodes *= (long long)n[ax] + 1;
      pixels *= img_shape[ax];
      if (a.nodes > kMaxMapNodes) return ADS_ERR_INVALID_ARG;
    } else {
      a.ax[ax] = MapAxis{1, 1};  // one slice, whose single node weighs it by 1
    }
  }
  if (pixels > (1LL << 40)) return ADS_ERR_INVALID_ARG;
  const size_t psize = pixel_type == ADS_PIXEL_F32 ? sizeof(float) : 1;
  const uintptr_t i0 = reinterpret_cast<uintptr_t>(d_img), i1 = i0 + (uintptr_t)pixels * psize;
  const uintptr_t o0 = reinterpret_cast<uintptr_t>(d_nodal), o1 = o0 + (uintptr_t)a.nodes * sizeof(double);
  if (i0 < o1 && o0 < i1) return ADS_ERR_INVALID_ARG;       // the output would overwrite the picture
  if (pixel_type == ADS_PIXEL_F32 && (i0 & 3)) return ADS_ERR_INVALID_ARG;
  if (o0 & 7) return ADS_ERR_INVALID_ARG;
  a.flip_y = flip_y != 0;
  a.scale = scale;
  a.offset = offset;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* cnt = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&cnt), sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return ADS_ERR_OOM;
  }
  const long long want = (a.nodes + 255) / 256;
  const unsigned blocks = (unsigned)(want < (1LL << 20) ? want : (1LL << 20));
  cudaMemsetAsync(cnt, 0, sizeof(int), st);
  const bool geo = mean == ADS_MAP_GEOMETRIC;
  if (pixel_type == ADS_PIXEL_F32) {
    const float* p = static_cast<const float*>(d_img);
    if (geo) k_map_nodal<float, true><<<blocks, 256, 0, st>>>(p, a, d_nodal, cnt);
    else k_map_nodal<float, false><<<blocks, 256, 0, st>>>(p, a, d_nodal, cnt);
  } else {
    const unsigned char* p = static_cast<const unsigned char*>(d_img);
    if (geo) k_map_nodal<unsigned char, true><<<blocks, 256, 0, st>>>(p, a, d_nodal, cnt);
    else k_map_nodal<unsigned char, false><<<blocks, 256, 0, st>>>(p, a, d_nodal, cnt);
  }
  int h_cnt = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_cnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(cnt, st);
  if (e == cudaSuccess) e = wait_bounded(st, 10.0);
  if (e == cudaErrorNotReady) return ADS_ERR_TIMEOUT;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ADS_ERR_CUDA;
  }
  return h_cnt ? ADS_ERR_NONFINITE : ADS_OK;
}

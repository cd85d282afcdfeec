// IGA-ADS explicit saturation step on the GPU (Secs. 2-4 of the paper).
//
//  * one-off tables: B-spline values/derivatives at the Gauss points of every
//    element (Cox-de Boor, degree 2, open uniform knots), the 1D mass matrix
//    int B_i B_k (Eq. 14) and its LDL^T factors, per-axis Gaussian source
//    factors -- all in FP64;
//  * the fused strip kernel: Gauss quadrature of the right-hand side of the
//    L2 projection (Eq. 10b, weak form Eq. 10a) for a strip of element rows,
//    accumulated in shared memory, then the x-direction banded solve of the
//    strip's rows in shared memory (M^-1 = Mx^-1 (x) My^-1, Eq. 14);
//  * the y-direction sweep: one thread per column, coalesced row access,
//    adding the rows the strip above spilled, and accumulating int S.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kernels.cuh"

namespace adsgb {

// ---------------------------------------------------------------------------
// one-off tables (FP64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double knot(int i, int n) {
  // open uniform knot vector of degree 2: 0,0,0,1/n,...,(n-1)/n,1,1,1
  if (i <= 2) return 0.0;
  if (i >= n + 2) return 1.0;
  return double(i - 2) / double(n);
}

// Nonzero basis functions of degree p (<= 2) at x in knot span s (the
// triangular Cox-de Boor scheme); N[0..p] = B_{s-p..s}.
__device__ void nonzero_basis(int n, int s, double x, int p, double* N) {
  double left[3], right[3];
  N[0] = 1.0;
  for (int j = 1; j <= p; ++j) {
    left[j] = x - knot(s + 1 - j, n);
    right[j] = knot(s + j, n) - x;
    double saved = 0.0;
    for (int r = 0; r < j; ++r) {
      double tmp = N[r] / (right[r + 1] + left[j - r]);
      N[r] = saved + right[r + 1] * tmp;
      saved = left[j - r] * tmp;
    }
    N[j] = saved;
  }
}

__global__ void k_axis_tables(int n, double* B, double* dB) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * 3) return;
  int e = t / 3, q = t % 3;
  double h = 1.0 / n;
  double x = (e + gauss_x(q)) * h;
  int s = e + 2;
  double N2[3], N1[3];
  nonzero_basis(n, s, x, 2, N2);
  nonzero_basis(n, s, x, 1, N1);
  double c0 = 2.0 / (knot(s + 1, n) - knot(s - 1, n));
  double c1 = 2.0 / (knot(s + 2, n) - knot(s, n));
  double d[3] = {-c0 * N1[0], c0 * N1[0] - c1 * N1[1], c1 * N1[1]};
  for (int a = 0; a < 3; ++a) {
    B[(e * 3 + a) * 3 + q] = N2[a];
    dB[(e * 3 + a) * 3 + q] = d[a];
  }
}

__global__ void k_source_tables(int n, int n_src, const double* centers, const double* sigmas,
                                double* gsrc, double* gnode) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double h = 1.0 / n;
  const double two_pi = 6.283185307179586477;
  int total_g = 3 * kMaxSrc * n * 3;
  if (t < total_g) {
    int q = t % 3, e = (t / 3) % n, s = (t / (3 * n)) % kMaxSrc, c = t / (3 * n * kMaxSrc);
    double v = 0.0;
    if (s < n_src) {
      double x = (e + gauss_x(q)) * h, cen = centers[s * 3 + c], sg = sigmas[s];
      v = exp(-(x - cen) * (x - cen) / (2.0 * sg * sg)) / sqrt(two_pi * sg * sg);
    }
    gsrc[t] = v;
  }
  int total_n = 3 * kMaxSrc * (n + 1);
  if (t < total_n) {
    int i = t % (n + 1), s = (t / (n + 1)) % kMaxSrc, c = t / ((n + 1) * kMaxSrc);
    double v = 0.0;
    if (s < n_src) {
      double x = i * h, cen = centers[s * 3 + c], sg = sigmas[s];
      v = exp(-(x - cen) * (x - cen) / (2.0 * sg * sg)) / sqrt(two_pi * sg * sg);
    }
    gnode[t] = v;
  }
}

// 1D mass matrix by the same quadrature, then LDL^T of the symmetric
// pentadiagonal matrix (no pivoting: the matrix is SPD).  One thread: O(n).
__global__ void k_mass_ldlt(int n, const double* B, double* m0, double* m1, double* m2,
                            double* l1, double* l2, double* dinv, double* Iw) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int nb = n + 2;
  double h = 1.0 / n;
  for (int i = 0; i < nb; ++i) { m0[i] = m1[i] = m2[i] = 0.0; Iw[i] = 0.0; }
  for (int e = 0; e < n; ++e)
    for (int q = 0; q < 3; ++q) {
      double w = gauss_w(q) * h;
      for (int a = 0; a < 3; ++a) {
        double ba = B[(e * 3 + a) * 3 + q];
        Iw[e + a] += w * ba;
        for (int b = 0; b <= a; ++b) {
          double v = w * ba * B[(e * 3 + b) * 3 + q];
          int d = a - b;
          if (d == 0) m0[e + a] += v;
          else if (d == 1) m1[e + a] += v;
          else m2[e + a] += v;
        }
      }
    }
  double D1 = 0.0, D2 = 0.0, a1 = 0.0;  // D_{l-1}, D_{l-2}, a_{l-1}
  for (int l = 0; l < nb + 2; ++l) { l1[l] = 0.0; l2[l] = 0.0; }
  for (int l = 0; l < nb; ++l) {
    double bl = (l >= 2) ? m2[l] / D2 : 0.0;
    double al = (l >= 1) ? (m1[l] - bl * a1 * D2) / D1 : 0.0;
    double Dl = m0[l] - al * al * D1 - bl * bl * D2;
    l1[l] = al;
    l2[l] = bl;
    dinv[l] = 1.0 / Dl;
    D2 = D1;
    D1 = Dl;
    a1 = al;
  }
}

cudaError_t launch_axis_init(int n, const double* centers, const double* sigmas, int n_src,
                             double* B, double* dB, double* l1, double* l2, double* dinv,
                             double* Iw, double* gsrc, double* gnode, double* tmp, cudaStream_t st) {
  k_axis_tables<<<(n * 3 + 127) / 128, 128, 0, st>>>(n, B, dB);
  int tot = 3 * kMaxSrc * n * 3;
  if (3 * kMaxSrc * (n + 1) > tot) tot = 3 * kMaxSrc * (n + 1);
  k_source_tables<<<(tot + 255) / 256, 256, 0, st>>>(n, n_src, centers, sigmas, gsrc, gnode);
  // tmp: 3 x (n+4) doubles for the three diagonals of the mass matrix
  k_mass_ldlt<<<1, 1, 0, st>>>(n, B, tmp, tmp + (n + 4), tmp + 2 * (n + 4), l1, l2, dinv, Iw);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_convert(const double* s, T* d, size_t c) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < c) d[i] = (T)s[i];
}
template <typename T>
__global__ void k_to_double(const T* s, double* d, size_t c) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < c) d[i] = (double)s[i];
}
template <typename T>
cudaError_t launch_convert(const double* src, T* dst, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  k_convert<T><<<(unsigned)((count + 255) / 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  k_to_double<T><<<(unsigned)((count + 255) / 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double>(const double*, double*, size_t, cudaStream_t);
template cudaError_t launch_convert<float>(const double*, float*, size_t, cudaStream_t);
template cudaError_t launch_to_double<double>(const double*, double*, size_t, cudaStream_t);
template cudaError_t launch_to_double<float>(const float*, double*, size_t, cudaStream_t);

// ---------------------------------------------------------------------------
// 2D saturation step (Eq. 10b, Eqs. 14-15): element quadrature fused with the
// x-direction mass solve, then the y-direction mass solve
// ---------------------------------------------------------------------------
// Chunked LDL^T sweeps.  The banded factors are those of the whole line; a
// line is cut into chunks so that many threads sweep it at once.  A chunk
// runs the forward substitution from a zero state H rows before its first
// row, and the backward substitution from a zero state H rows after its last
// row (a start at or beyond the end of the line is exact).  The error of a
// zero start obeys the homogeneous recurrence of the unit lower factor, whose
// solutions shrink by rho = 0.43058 per row: rho is the root inside the unit
// circle of z^4 + 26 z^3 + 66 z^2 + 26 z + 1, the symbol of the interior row
// h [1, 26, 66, 26, 1] / 120 of the quadratic B-spline mass matrix.  With
// H = 24 (FP32) the truncation is 1.6e-9 of the solution's size and with
// H = 48 (FP64) 2.4e-18, both below the unit roundoff.
template <typename T>
struct SweepHalo;
template <>
struct SweepHalo<float> {
  static constexpr int H = 24;
};
template <>
struct SweepHalo<double> {
  static constexpr int H = 48;
};

constexpr int kQuadThreads = 256;
constexpr int kQuadCols = 30;  // DOF columns a warp completes per pass (32 element columns)

// In-place chunked LDL^T solve of `nrows` lines of length nb in shared memory
// (row stride ld).  Thread t sweeps chunk t % nch of line t / nch; the host
// picks the chunk length so that every task has a thread.  The halo values
// of a chunk are copied to registers before its neighbours overwrite them.
template <typename T>
ADS_D void sweep_lines_smem(T* buf, int nrows, int nb, int ld, int chunk,
                            const T* __restrict__ l1, const T* __restrict__ l2,
                            const T* __restrict__ dinv) {
  constexpr int H = SweepHalo<T>::H;
  const int nch = (nb + chunk - 1) / chunk;
  const int t = threadIdx.x;
  const bool act = t < nrows * nch;
  const int row = act ? t / nch : 0, ch = act ? t % nch : 0;
  T* line = buf + (size_t)row * ld;
  const int s = ch * chunk, e = min(nb, s + chunk);
  T hv[H];
  if (act) {
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int l = s - H + k;
      hv[k] = l >= 0 ? line[l] : T(0);
    }
  }
  __syncthreads();
  if (act) {
    T y1 = T(0), y2 = T(0);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int l = s - H + k;
      if (l >= 0) {
        const T y = hv[k] - __ldg(l1 + l) * y1 - __ldg(l2 + l) * y2;
        y2 = y1;
        y1 = y;
      }
    }
    constexpr int U = 8;  // batches: loads, recurrence in registers, stores
    int l = s;
    for (; l + U <= e; l += U) {
      T v[U], a1[U], a2[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        v[k] = line[l + k];
        a1[k] = __ldg(l1 + l + k);
        a2[k] = __ldg(l2 + l + k);
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        v[k] = v[k] - a1[k] * y1 - a2[k] * y2;
        y2 = y1;
        y1 = v[k];
      }
#pragma unroll
      for (int k = 0; k < U; ++k) line[l + k] = v[k];
    }
    for (; l < e; ++l) {
      const T y = line[l] - __ldg(l1 + l) * y1 - __ldg(l2 + l) * y2;
      line[l] = y;
      y2 = y1;
      y1 = y;
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int l = e + k;
      hv[k] = l < nb ? line[l] : T(0);
    }
  }
  __syncthreads();
  if (act) {
    T x1 = T(0), x2 = T(0);
#pragma unroll
    for (int k = H - 1; k >= 0; --k) {
      const int l = e + k;
      if (l < nb) {
        const T x = hv[k] * __ldg(dinv + l) - __ldg(l1 + l + 1) * x1 - __ldg(l2 + l + 2) * x2;
        x2 = x1;
        x1 = x;
      }
    }
    constexpr int U = 8;
    int l = e - 1;
    for (; l - U + 1 >= s; l -= U) {
      T v[U], dd[U], a1[U], a2[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        v[k] = line[l - k];
        dd[k] = __ldg(dinv + l - k);
        a1[k] = __ldg(l1 + l - k + 1);
        a2[k] = __ldg(l2 + l - k + 2);
      }
#pragma unroll
      for (int k = 0; k < U; ++k) {
        v[k] = v[k] * dd[k] - a1[k] * x1 - a2[k] * x2;
        x2 = x1;
        x1 = v[k];
      }
#pragma unroll
      for (int k = 0; k < U; ++k) line[l - k] = v[k];
    }
    for (; l >= s; --l) {
      const T x = line[l] * __ldg(dinv + l) - __ldg(l1 + l + 1) * x1 - __ldg(l2 + l + 2) * x2;
      line[l] = x;
      x2 = x1;
      x1 = x;
    }
  }
  __syncthreads();
}

// Pairs for the packed FP32 instructions of this GPU (fma.rn.f32x2: two
// correctly rounded FMAs in one issue slot); FP64 takes two scalar FMAs.
// The 1D basis tables pair up naturally: (B, dB) of an element column along
// x and (dB, B) of an element row along y, so that one packed FMA advances
// two of the sum-factorised contractions at once.
template <typename T>
struct PairOf;
template <>
struct PairOf<float> {
  using type = float2;
};
template <>
struct PairOf<double> {
  using type = double2;
};
template <typename T>
using P2 = typename PairOf<T>::type;
ADS_D float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
ADS_D double2 pfma(double2 a, double2 b, double2 c) { return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)); }
ADS_D float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
ADS_D double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }

// x-contractions of the coefficients of one DOF row over the three basis
// functions of element column ex, at the three Gauss abscissae: S, and the
// pair (P, dP/dx)
template <typename T>
struct XRow {
  T s[3];
  P2<T> ppd[3];
};
template <typename T>
ADS_D void xrow_load(const QuadArgs<T>& a, int r, int ex, const P2<T> (&xb)[3][3], XRow<T>& w) {
  const T* srow = a.S + (size_t)r * a.nb + ex;
  const T* prow = a.P + (size_t)r * a.nb + ex;
  const T s0 = __ldg(srow), s1 = __ldg(srow + 1), s2 = __ldg(srow + 2);
  const T p0 = __ldg(prow), p1 = __ldg(prow + 1), p2 = __ldg(prow + 2);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    w.s[q] = s0 * xb[0][q].x + s1 * xb[1][q].x + s2 * xb[2][q].x;
    w.ppd[q] = pfma(P2<T>{p2, p2}, xb[2][q], pfma(P2<T>{p1, p1}, xb[1][q], pmul(P2<T>{p0, p0}, xb[0][q])));
  }
}

template <typename T>
ADS_D T frac_div(T a, T b) { return a / b; }
template <>
ADS_D float frac_div<float>(float a, float b) { return __fdividef(a, b); }

// Strip b of `re` element rows.  Phase 1: warp w takes DOF columns
// [30 g, 30 g + 30) for g = w, w + 8, ...; lane j evaluates element column
// 30 g - 2 + j down the strip.  An element adds to the DOF columns ex, ex+1,
// ex+2, so lane j's column sums its own first-column term and the shuffled
// second- and third-column terms of lanes j-1 and j-2 (lanes 0 and 1 only
// feed their neighbours).  DOF-row sums roll down the strip in registers; a
// row is stored once no later element row touches it.  Phase 2: the x sweeps
// of the strip's rows in shared memory.  Phase 3: rows owned by the strip go
// to Xm, the two rows it shares with the next strip to Xs.
template <typename T, int MODE, int NS>
__global__ void __launch_bounds__(kQuadThreads, sizeof(T) == 4 ? 2 : 1)
    k_quad_xsweep_2d(QuadArgs<T> a, int re, int xchunk, T* __restrict__ Xm, T* __restrict__ Xs,
                     int ldx, double* src_part, int nstrip, int csz) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  T* acc = reinterpret_cast<T*>(smraw);  // [re + 2][nb]
  const int nb = a.nb, n = a.n, n1 = n + 1, tid = threadIdx.x, lane = tid & 31;
  const int nwarp = blockDim.x >> 5;
  const int b = blockIdx.x;
  const bool real = b < nstrip;  // the grid is padded to whole clusters
  const int e0 = b * re, e1 = real ? min(e0 + re, n) : e0;
  const int nrows = real ? e1 - e0 + 2 : 0;
  const T h2 = a.h * a.h;
  const T dt = MODE == 0 ? (T)(*a.dt) : T(0);
  const T dtphi_c = MODE == 0 ? dt / a.phi_c : T(0);
  CompSum<T> src;
  const int ngroups = real ? (nb + kQuadCols - 1) / kQuadCols : 0;
  for (int g = tid >> 5; g < ngroups; g += nwarp) {
    const int ex = g * kQuadCols - 2 + lane;  // element column of this lane = its DOF column
    const bool live = ex >= 0 && ex < n;
    const int xc = live ? ex : 0;
    // (B, dB) of the lane's element column at the three abscissae
    P2<T> xb[3][3];
#pragma unroll
    for (int i = 0; i < 9; ++i) xb[i / 3][i % 3] = P2<T>{__ldg(a.ax.B + xc * 9 + i), __ldg(a.ax.dB + xc * 9 + i)};
    // the sources' x profiles times their rates
    T gxr[NS][3];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int q = 0; q < 3; ++q)
        gxr[s][q] = s < a.n_src ? a.rate[s] * __ldg(a.ax.gsrc + ((size_t)(0 * kMaxSrc + s) * n + xc) * 3 + q) : T(0);
    XRow<T> w0, w1, w2;
    // K (or the nodal values) interpolated along x to the three abscissae on
    // the element's lower (0) and upper (1) node rows; phi at the nodes
    T kx0[3], kx1[3], f0[2] = {T(0), T(0)}, f1[2] = {T(0), T(0)};
    auto xinterp = [&](const T* row, T (&out)[3]) {
      const T v0 = __ldg(row), v1 = __ldg(row + 1);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const T xi = (T)gauss_x(q);
        out[q] = (T(1) - xi) * v0 + xi * v1;
      }
    };
    if (MODE == 0) {
      xrow_load(a, e0, xc, xb, w0);
      xrow_load(a, e0 + 1, xc, xb, w1);
      xinterp(a.K + (size_t)e0 * n1 + xc, kx0);
      if (a.phi) {
        f0[0] = __ldg(a.phi + (size_t)e0 * n1 + xc);
        f0[1] = __ldg(a.phi + (size_t)e0 * n1 + xc + 1);
      }
    } else {
      xinterp(a.nodal + (size_t)e0 * n1 + xc, kx0);
    }
    T A0 = T(0), A1 = T(0), A2 = T(0);
    for (int er = e0; er < e1; ++er) {
      // (dB, B) of the element row at the three abscissae
      P2<T> yb[3][3];
#pragma unroll
      for (int i = 0; i < 9; ++i) yb[i / 3][i % 3] = P2<T>{__ldg(a.ax.dB + er * 9 + i), __ldg(a.ax.B + er * 9 + i)};
      T loc[3][3];
      if (MODE == 0) {
        xrow_load(a, er + 2, xc, xb, w2);
        xinterp(a.K + (size_t)(er + 1) * n1 + xc, kx1);
        if (a.phi) {
          f1[0] = __ldg(a.phi + (size_t)(er + 1) * n1 + xc);
          f1[1] = __ldg(a.phi + (size_t)(er + 1) * n1 + xc + 1);
        }
        T gy[NS][3];
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int q = 0; q < 3; ++q)
            gy[s][q] = s < a.n_src ? __ldg(a.ax.gsrc + ((size_t)(1 * kMaxSrc + s) * n + er) * 3 + q) : T(0);
        P2<T> tt[3][3];  // [qy][aa]: (T1, T0), the test functions along x applied
        T esrc = T(0);   // tau/phi int q_g over the element (9 terms)
#pragma unroll
        for (int qy = 0; qy < 3; ++qy) {
          const T eta = (T)gauss_x(qy);
          P2<T> cc[3];  // (c0, cx) at the row's three points
          T cy[3];
#pragma unroll
          for (int qx = 0; qx < 3; ++qx) {
            // (dP/dy, dP/dx) and S at the point
            const P2<T> dp =
                pfma(yb[2][qy], w2.ppd[qx], pfma(yb[1][qy], w1.ppd[qx], pmul(yb[0][qy], w0.ppd[qx])));
            const T Sv = yb[0][qy].y * w0.s[qx] + yb[1][qy].y * w1.s[qx] + yb[2][qy].y * w2.s[qx];
            const T Kq = (T(1) - eta) * kx0[qx] + eta * kx1[qx];
            T dtphi = dtphi_c;
            if (a.phi) {
              const T xi = (T)gauss_x(qx);
              dtphi = dt / ((T(1) - eta) * ((T(1) - xi) * f0[0] + xi * f0[1]) + eta * ((T(1) - xi) * f1[0] + xi * f1[1]));
            }
            const T St = clamp01(Sv);
            const T lg = St * a.inv_mu_g, lw = (T(1) - St) * a.inv_mu_w;
            T qi = T(0), qp = T(0);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              const T gv = gxr[s][qx] * gy[s][qy];
              if (a.kind[s] == 0) qi += gv;
              else qp += gv;
            }
            // the producer draws the mobile fraction f_g of the total rate
            T qg = qi;
            if (qp != T(0)) qg -= frac_div(lg, lg + lw) * qp;
            const T w = (T)(gauss_w(qx) * gauss_w(qy)) * h2;
            const T cf = -w * dtphi * lg * Kq;
            cc[qx] = P2<T>{w * (Sv + dtphi * qg), cf * dp.y};
            cy[qx] = cf * (dp.x + a.grav_term);
            esrc += w * dtphi * qg;
          }
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            const P2<T> t0 = pfma(cc[2], xb[aa][2], pfma(cc[1], xb[aa][1], pmul(cc[0], xb[aa][0])));
            const T t1 = cy[0] * xb[aa][0].x + cy[1] * xb[aa][1].x + cy[2] * xb[aa][2].x;
            tt[qy][aa] = P2<T>{t1, t0.x + t0.y};
          }
        }
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            const P2<T> v = pfma(yb[bb][2], tt[2][aa], pfma(yb[bb][1], tt[1][aa], pmul(yb[bb][0], tt[0][aa])));
            loc[bb][aa] = live ? v.x + v.y : T(0);
          }
        // lanes 0 and 1 recompute elements the previous group owns
        if (live && lane >= 2) src.add(esrc);
        w0 = w1;
        w1 = w2;
#pragma unroll
        for (int q = 0; q < 3; ++q) kx0[q] = kx1[q];
        f0[0] = f1[0];
        f0[1] = f1[1];
      } else {
        xinterp(a.nodal + (size_t)(er + 1) * n1 + xc, kx1);
        T T0[3][3];
#pragma unroll
        for (int qy = 0; qy < 3; ++qy) {
          const T eta = (T)gauss_x(qy);
          T c0[3];
#pragma unroll
          for (int qx = 0; qx < 3; ++qx)
            c0[qx] = (T)(gauss_w(qx) * gauss_w(qy)) * h2 * ((T(1) - eta) * kx0[qx] + eta * kx1[qx]);
#pragma unroll
          for (int aa = 0; aa < 3; ++aa)
            T0[qy][aa] = c0[0] * xb[aa][0].x + c0[1] * xb[aa][1].x + c0[2] * xb[aa][2].x;
        }
#pragma unroll
        for (int bb = 0; bb < 3; ++bb)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            const T v = yb[bb][0].y * T0[0][aa] + yb[bb][1].y * T0[1][aa] + yb[bb][2].y * T0[2][aa];
            loc[bb][aa] = live ? v : T(0);
          }
#pragma unroll
        for (int q = 0; q < 3; ++q) kx0[q] = kx1[q];
      }
      // column sums across the warp: own first-column term + neighbours' terms
      T col[3];
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        const T from1 = __shfl_up_sync(0xffffffffu, loc[bb][1], 1);
        const T from2 = __shfl_up_sync(0xffffffffu, loc[bb][2], 2);
        col[bb] = loc[bb][0] + from1 + from2;
      }
      A0 += col[0];
      A1 += col[1];
      A2 += col[2];
      if (lane >= 2 && ex < nb) acc[(size_t)(er - e0) * nb + ex] = A0;
      A0 = A1;
      A1 = A2;
      A2 = T(0);
    }
    if (lane >= 2 && ex < nb) {
      acc[(size_t)(e1 - e0) * nb + ex] = A0;
      acc[(size_t)(e1 - e0 + 1) * nb + ex] = A1;
    }
  }
  __syncthreads();
  if (real) sweep_lines_smem<T>(acc, nrows, nb, nb, xchunk, a.ax.l1, a.ax.l2, a.ax.dinv);
  // The two rows after the strip's own (DOF rows e1, e1 + 1) are the first
  // two rows of strip b + 1.  Within a cluster they are added into the next
  // CTA's rows through distributed shared memory (after both x sweeps; the
  // sweep is linear, and own + shared is the one addition the y sweep would
  // do), so only the last strip of a cluster spills them to Xs, pair m of Xs
  // for cluster m.
  const int own = e1 - e0;
  const bool shared_rows = real && e1 < n;
  const int q = b % csz;
  const bool to_next = shared_rows && q + 1 < csz;
  const bool from_prev = real && q > 0;  // rows 0, 1 receive the previous strip's part
  auto put = [&](int r) {
    const bool spill = r >= own && shared_rows;
    if (spill && to_next) return;
    T* dst = spill ? Xs + ((size_t)(b / csz) * 2 + (r - own)) * ldx : Xm + (size_t)(e0 + r) * ldx;
    for (int k = tid; k < nb; k += blockDim.x) dst[k] = acc[(size_t)r * nb + k];
  };
  // rows no other CTA touches go out first, under the wait for the cluster
  for (int r = from_prev ? 2 : 0; r < nrows; ++r)
    if (!(r >= own && shared_rows && to_next)) put(r);
  if (csz > 1) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    if (to_next) {
      T* nxt = cl.map_shared_rank(acc, (int)cl.block_rank() + 1);
      for (int j = 0; j < 2; ++j)
        for (int k = tid; k < nb; k += blockDim.x) nxt[(size_t)j * nb + k] += acc[(size_t)(own + j) * nb + k];
    }
    cl.sync();
  }
  if (from_prev)
    for (int r = 0; r < 2 && r < nrows; ++r) put(r);
  if (MODE == 0) {
    const double tot = block_sum(src.value(), red);
    if (tid == 0 && real) src_part[b] = tot;
  }
}

int quad_rows(int n, size_t esize) {
  // strips of 4 element rows (two spill rows per 4) while two strips fit in
  // one SM's shared memory, else 2
  return (size_t)6 * (n + 2) * esize <= 110 * 1024 ? 4 : 2;
}

int quad_cluster(int re) { return re == 4 ? 2 : (re == 2 ? 4 : 1); }

int quad_blocks(int dim, int n, int re) {
  if (dim == 2) return (n + re - 1) / re;
  return n * ((n + re - 1) / re);
}

int sweep_ld(int n) { return ((n + 2 + 31) / 32) * 32; }

static int xsweep_chunk(int nrows, int nb) {
  int ch = 127;  // odd: the chunks of a row start in distinct shared-memory banks
  while ((long)nrows * ((nb + ch - 1) / ch) > kQuadThreads) ch += 2;
  return ch;
}

template <typename K, typename T>
static cudaError_t quad_launch_one(K k, const QuadArgs<T>& a, int re, int xch, T* Xm, T* Xs, int ldx,
                                   double* src_part, size_t smem, cudaStream_t st) {
  const int nblk = quad_blocks(2, a.n, re), csz = quad_cluster(re);
  smem_optin(k);
  if (csz == 1) {
    k<<<nblk, kQuadThreads, smem, st>>>(a, re, xch, Xm, Xs, ldx, src_part, nblk, 1);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((nblk + csz - 1) / csz * csz));
  cfg.blockDim = dim3(kQuadThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)csz;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a, re, xch, Xm, Xs, ldx, src_part, nblk, csz);
}

template <typename T, int MODE>
static cudaError_t quad_launch(const QuadArgs<T>& a, int re, int xch, T* Xm, T* Xs, int ldx,
                               double* src_part, size_t smem, cudaStream_t st) {
  if (a.n_src <= 2)
    return quad_launch_one(k_quad_xsweep_2d<T, MODE, 2>, a, re, xch, Xm, Xs, ldx, src_part, smem, st);
  return quad_launch_one(k_quad_xsweep_2d<T, MODE, kMaxSrc>, a, re, xch, Xm, Xs, ldx, src_part, smem, st);
}

template <typename T>
cudaError_t launch_quad_xsweep(const QuadArgs<T>& a, int mode, int re, T* Xm, T* Xs, int ldx,
                               double* src_part, cudaStream_t st) {
  if (a.dim != 2 || re < 2) return cudaErrorNotSupported;
  if (ldx < a.nb || (ldx * sizeof(T)) % 16 != 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)(re + 2) * a.nb * sizeof(T);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const int xch = xsweep_chunk(re + 2, a.nb);
  return mode == 0 ? quad_launch<T, 0>(a, re, xch, Xm, Xs, ldx, src_part, smem, st)
                   : quad_launch<T, 1>(a, re, xch, Xm, Xs, ldx, src_part, smem, st);
}

// y sweep.  CTA (i, j) owns rows [M i, M i + M) of the CW columns from CW j.
// Bulk tensor copies bring rows [M i - H, M i + M + H) of those columns of Xm
// (zero outside the mesh) and the spill rows of Xs that fall among them into
// shared memory; the spill rows are added, and thread c sweeps column c down
// and up the tile (the halo rows start the chunked sweeps, see above).  The
// owned rows go to `out` and their share of int S (basis integrals,
// compensated sum) to mass_part.
template <typename T>
struct YTile;
template <>
struct YTile<float> {
  static constexpr int CW = 128, M = 64;
};
template <>
struct YTile<double> {
  static constexpr int CW = 64, M = 64;
};
template <typename T>
__host__ __device__ constexpr int ytile_rows() { return YTile<T>::M + 2 * SweepHalo<T>::H; }
// spill rows a tile can meet: pairs at rows q re + {0, 1}
static int yspill_rows(int rb, int re) { return 2 * ((rb + re - 1) / re + 2); }

constexpr unsigned long long kCopyWaitNs = 1000000000ull;  // 1 s

template <typename T>
__global__ void __launch_bounds__(YTile<T>::CW)
    k_ysweep_2d(const __grid_constant__ CUtensorMap xm_map, const __grid_constant__ CUtensorMap xs_map,
                int n, int re, int nsp, int sb, T* __restrict__ out, const T* __restrict__ l1,
                const T* __restrict__ l2, const T* __restrict__ dinv, const T* __restrict__ Iw,
                double* mass_part, int* flags) {
  constexpr int CW = YTile<T>::CW, M = YTile<T>::M, H = SweepHalo<T>::H, RB = ytile_rows<T>();
  extern __shared__ __align__(1024) unsigned char ysm[];
  T* tile = reinterpret_cast<T*>(ysm);  // [RB][CW]
  T* stile = tile + RB * CW;              // [sb][CW] spill rows
  T* fl1 = stile + (size_t)sb * CW;       // factor rows of the tile: l1, l2 [RB + 2], dinv, Iw [RB]
  T* fl2 = fl1 + RB + 2;
  T* fdi = fl2 + RB + 2;
  T* fiw = fdi + RB;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(fiw + RB + ((8 / sizeof(T)) - 1)) ;
  mbar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(mbar) + 7) & ~uintptr_t(7));
  double* red = reinterpret_cast<double*>(mbar + 1);
  const int nb = n + 2, tid = threadIdx.x;
  const int s = blockIdx.x * M, e = min(nb, s + M), r0 = s - H;
  const int L0 = max(r0, 0), L1 = min(r0 + RB, nb);
  const int col = blockIdx.y * CW + tid;
  // first spill pair touching [L0, L1): q re + 1 >= L0, q >= 1
  const int qlo = max(1, (L0 - 1 + re - 1) / re);
  const int y0 = 2 * (qlo - 1);
  if (tid == 0) mbar_init_cta(mbar, 1);
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_tx(mbar, (unsigned)((RB + (nsp > 0 ? sb : 0)) * CW * sizeof(T)));
    tma_load_2d(tile, &xm_map, blockIdx.y * CW, r0, mbar);
    if (nsp > 0) tma_load_2d(stile, &xs_map, blockIdx.y * CW, y0, mbar);
  }
  for (int i = tid; i < RB + 2; i += CW) {
    const int l = r0 + i;
    const bool in = l >= 0 && l < nb + 2;
    fl1[i] = in ? __ldg(l1 + l) : T(0);
    fl2[i] = in ? __ldg(l2 + l) : T(0);
    if (i < RB) {
      fdi[i] = (l >= 0 && l < nb) ? __ldg(dinv + l) : T(0);
      fiw[i] = (l >= 0 && l < nb) ? __ldg(Iw + l) : T(0);
    }
  }
  const bool ok = mbar_wait_for(mbar, 0, kCopyWaitNs);
  if (__syncthreads_or(!ok)) {
    // a copy did not land in time: record it, give it one more bounded wait
    // so that it no longer writes into this CTA's shared memory, stop
    if (tid == 0) atomicOr(flags, 8);
    mbar_wait_for(mbar, 0, kCopyWaitNs);
    return;
  }
  T* cp = tile + tid;  // column `col` of the tile, row stride CW
  if (nsp > 0) {
    // DOF row l = q re + j (j = 0, 1; q >= 1) also holds the part of the strip
    // above it, Xs row 2 (q - 1) + j
    for (int q = qlo; q * re < L1; ++q)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int l = q * re + j, r = 2 * (q - 1) + j;
        if (l >= L0 && l < L1 && r < nsp) cp[(l - r0) * CW] += stile[(r - y0) * CW + tid];
      }
  }
  const int ilo = L0 - r0, ihi = L1 - r0;
  const int iown = e - r0;  // rows [H, iown) are owned
  // sweeps in batches of 8 rows: loads first, then the recurrence in
  // registers, then the stores (the tile and the factor rows share one
  // shared array, so the compiler would not move loads above stores)
  constexpr int U = 8;
  T y1 = T(0), y2 = T(0);
  int i = ilo;
  for (; i + U <= ihi; i += U) {
    T v[U], a1[U], a2[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      v[k] = cp[(i + k) * CW];
      a1[k] = fl1[i + k];
      a2[k] = fl2[i + k];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      v[k] = v[k] - a1[k] * y1 - a2[k] * y2;
      y2 = y1;
      y1 = v[k];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) cp[(i + k) * CW] = v[k];
  }
  for (; i < ihi; ++i) {
    const T y = cp[i * CW] - fl1[i] * y1 - fl2[i] * y2;
    cp[i * CW] = y;
    y2 = y1;
    y1 = y;
  }
  T x1 = T(0), x2 = T(0);
  CompSum<T> mass;
  i = ihi - 1;
  for (; i - U + 1 >= H; i -= U) {
    T v[U], dd[U], a1[U], a2[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      v[k] = cp[(i - k) * CW];
      dd[k] = fdi[i - k];
      a1[k] = fl1[i - k + 1];
      a2[k] = fl2[i - k + 2];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      v[k] = v[k] * dd[k] - a1[k] * x1 - a2[k] * x2;
      x2 = x1;
      x1 = v[k];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      cp[(i - k) * CW] = v[k];
      if (i - k < iown) mass.add(v[k] * fiw[i - k]);
    }
  }
  for (; i >= H; --i) {
    const T x = cp[i * CW] * fdi[i] - fl1[i + 1] * x1 - fl2[i + 2] * x2;
    cp[i * CW] = x;
    if (i < iown) mass.add(x * fiw[i]);
    x2 = x1;
    x1 = x;
  }
  double mcol = 0.0;
  if (col < nb) {
    for (int i = H; i < iown; ++i) out[(size_t)(r0 + i) * nb + col] = cp[i * CW];
    mcol = mass.value() * (double)__ldg(Iw + col);
  }
  const double tot = block_sum(mcol, red);
  if (tid == 0) mass_part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// Packed FP32 y-sweep factor rows: mesh row l at table row l + kYTabPad holds
// (l1[l], l2[l]) in the forward table and (1/D[l], l1[l+1], l2[l+2], int B_l)
// in the backward table, zeros for rows outside [0, n + 2), so a tile's
// factors arrive with one bulk copy per table and rows outside the mesh stay
// zero through both sweeps.
constexpr int kYTabPad = 32;
static size_t ysweep_table_rows(int n) {
  const size_t r = (size_t)n + 2 + 2 * kYTabPad + ytile_rows<float>() + YTile<float>::M;
  return (r + 1) & ~size_t(1);  // even: the backward table starts 16-byte aligned
}
size_t ysweep_table_bytes(int n) { return ysweep_table_rows(n) * (sizeof(float2) + sizeof(float4)); }

__global__ void k_ysweep_table(int n, int rows, const float* __restrict__ l1, const float* __restrict__ l2,
                               const float* __restrict__ dinv, const float* __restrict__ Iw, float2* fw,
                               float4* bw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= rows) return;
  const int l = k - kYTabPad, nb = n + 2;
  const bool in = l >= 0 && l < nb;
  fw[k] = in ? make_float2(l1[l], l2[l]) : make_float2(0.f, 0.f);
  bw[k] = in ? make_float4(dinv[l], l1[l + 1], l2[l + 2], Iw[l]) : make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t launch_ysweep_table(int n, const float* l1, const float* l2, const float* dinv, const float* Iw,
                                void* tab, cudaStream_t st) {
  const int rows = (int)ysweep_table_rows(n);
  float2* fw = reinterpret_cast<float2*>(tab);
  float4* bw = reinterpret_cast<float4*>(fw + rows);
  k_ysweep_table<<<(rows + 255) / 256, 256, 0, st>>>(n, rows, l1, l2, dinv, Iw, fw, bw);
  return cudaGetLastError();
}

// Forward and backward substitution of one tile column held in registers
// (rows [0, RB), owned rows [H, H + M)), and the int N-weighted sum of the
// owned rows.  UNI: every row of the tile has the factors (cf, cb), so they
// come from registers; the arithmetic is the same either way.
template <bool UNI, int RB, int H, int M>
__device__ __forceinline__ float ysweep_column(float (&v)[RB], const float2* fw, const float4* bw, float2 cf,
                                               float4 cb) {
  float y1 = 0.f, y2 = 0.f;
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const float2 f = UNI ? cf : fw[i];
    const float y = fmaf(-f.x, y1, fmaf(-f.y, y2, v[i]));
    v[i] = y;
    y2 = y1;
    y1 = y;
  }
  float x1 = 0.f, x2 = 0.f, ms[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = RB - 1; i >= H; --i) {
    const float4 f = UNI ? cb : bw[i];
    const float x = fmaf(-f.y, x1, fmaf(-f.z, x2, v[i] * f.x));
    v[i] = x;
    x2 = x1;
    x1 = x;
    if (i < H + M) ms[i & 7] = fmaf(x, f.w, ms[i & 7]);
  }
  return ((ms[0] + ms[1]) + (ms[2] + ms[3])) + ((ms[4] + ms[5]) + (ms[6] + ms[7]));
}

// FP32 y sweep, persistent, pipelined and register-resident.  One CTA per SM
// takes the tiles t = blockIdx.x + k gridDim.x (row chunk fastest, so that
// neighbouring CTAs share halo rows in L2) through NST shared-memory stages;
// the factor rows of a tile come by bulk copy from the packed table into one
// of NST + 1 slots.  Each thread lifts its column of the tile into registers,
// then the stage goes back to the bulk copies (tile k + NST) while the
// forward and backward substitutions, the int S partials and the stores run
// from registers.  Away from the ends of the mesh the factors of the
// uniform-knot mass matrix settle to one value; tiles whose factors all equal
// it take them from registers.  RE is the period of the spill rows (the
// quadrature's strip height times its cluster size); M and H are multiples of
// RE, so the spill rows of a tile are fixed by the row index alone, and the
// spill box starts at the spill pair of the tile's first period (rows before
// the first or after the last spill row read as zero).
template <int RE, int NST>
__global__ void __launch_bounds__(YTile<float>::CW, 3 - NST)
    k_ysweep_reg_2d(const __grid_constant__ CUtensorMap xm_map, const __grid_constant__ CUtensorMap xs_map,
                    int n, int nsp, int sb, int gx, int ntile, float* __restrict__ out,
                    const float2* __restrict__ tfw, const float4* __restrict__ tbw,
                    const float* __restrict__ Iw, double* mass_part, int* flags) {
  constexpr int CW = YTile<float>::CW, M = YTile<float>::M, H = SweepHalo<float>::H;
  constexpr int RB = ytile_rows<float>(), NF = NST + 1;
  static_assert(M % RE == 0 && H % RE == 0 && RB <= CW && H <= kYTabPad, "tile geometry");
  extern __shared__ __align__(1024) unsigned char yrg[];
  const size_t stage = (size_t)(RB + sb) * CW;  // floats per stage: tile, then spill rows
  float* st = reinterpret_cast<float*>(yrg);
  float4* fbw = reinterpret_cast<float4*>(st + NST * stage);  // [NF][RB]
  float2* ffw = reinterpret_cast<float2*>(fbw + NF * RB);     // [NF][RB]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(ffw + NF * RB);  // [NST]
  double* red = reinterpret_cast<double*>(mbar + 2);
  const int nb = n + 2, tid = threadIdx.x, G = gridDim.x;
  const unsigned tx = (unsigned)((RB + (nsp > 0 ? sb : 0)) * CW * sizeof(float) +
                                 RB * (sizeof(float2) + sizeof(float4)));
  // tile k of this CTA (t = blockIdx.x + k G) into stage k % NST, slot k % NF
  auto issue = [&](int t, int k) {
    const int r0 = (t % gx) * M - H, c0 = (t / gx) * CW, sg = k % NST, fs = k % NF;
    float* dst = st + sg * stage;
    mbar_arrive_tx(mbar + sg, tx);
    tma_load_2d(dst, &xm_map, c0, r0, mbar + sg);
    if (nsp > 0) tma_load_2d(dst + (size_t)RB * CW, &xs_map, c0, 2 * (r0 / RE - 1), mbar + sg);
    bulk_load(ffw + fs * RB, tfw + r0 + kYTabPad, RB * sizeof(float2), mbar + sg);
    bulk_load(fbw + fs * RB, tbw + r0 + kYTabPad, RB * sizeof(float4), mbar + sg);
  };
  if (tid < NST) mbar_init_cta(mbar + tid, 1);
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < NST; ++k)
      if ((int)blockIdx.x + k * G < ntile) issue(blockIdx.x + k * G, k);
  const int lm = nb / 2 + kYTabPad;
  const float2 cf = tfw[lm];
  const float4 cb = tbw[lm];
  double macc = 0.0;
  int it = 0;
  for (int t = blockIdx.x; t < ntile; t += G, ++it) {
    const int sg = it % NST, fs = it % NF;
    const int r0 = (t % gx) * M - H, col = (t / gx) * CW + tid;
    const float iwc = col < nb ? __ldg(Iw + col) : 0.f;
    const bool ok = mbar_wait_for(mbar + sg, (it / NST) & 1, kCopyWaitNs);
    if (__syncthreads_or(!ok)) {
      // a copy did not land in time: record it and let the copies in flight
      // land (bounded) before the CTA's shared memory is released
      if (tid == 0) {
        atomicOr(flags, 8);
        for (int d = 0; d < NST; ++d)
          if (t + d * G < ntile) mbar_wait_for(mbar + (it + d) % NST, ((it + d) / NST) & 1, kCopyWaitNs);
      }
      __syncthreads();
      return;
    }
    bool uni = true;
    if (tid < RB) {
      const float2 f2 = ffw[fs * RB + tid];
      const float4 f4 = fbw[fs * RB + tid];
      uni = f2.x == cf.x && f2.y == cf.y && f4.x == cb.x && f4.y == cb.y && f4.z == cb.z && f4.w == cb.w;
    }
    const float* cp = st + sg * stage + tid;
    float v[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) v[i] = cp[i * CW];
    if (nsp > 0) {
      // DOF row r0 + i with i mod RE = j < 2 also holds the part of the strip
      // above it: box row 2 floor(i / RE) + j
      const float* sp = cp + (size_t)RB * CW;
#pragma unroll
      for (int i = 0; i < RB; ++i)
        if (i % RE < 2) v[i] += sp[(2 * (i / RE) + i % RE) * CW];
    }
    // the tile is in registers: hand the stage back to the copies (the
    // block reduction is also the barrier that releases it)
    fence_async_smem();
    const bool generic = __syncthreads_or(!uni);
    if (tid == 0 && t + NST * G < ntile) issue(t + NST * G, it + NST);
    if (!generic) {
      const float m = ysweep_column<true, RB, H, M>(v, nullptr, nullptr, cf, cb);
      if (col < nb) {
        float* o = out + (size_t)(r0 + H) * nb + col;
#pragma unroll
        for (int i = H; i < H + M; ++i, o += nb) *o = v[i];
        macc += (double)m * (double)iwc;
      }
    } else {
      const float m = ysweep_column<false, RB, H, M>(v, ffw + fs * RB, fbw + fs * RB, cf, cb);
      if (col < nb) {
        float* o = out + (size_t)(r0 + H) * nb + col;
#pragma unroll
        for (int i = H; i < H + M; ++i, o += nb)
          if (r0 + i < nb) *o = v[i];
        macc += (double)m * (double)iwc;
      }
    }
  }
  const double tot = block_sum(macc, red);
  if (tid == 0) mass_part[blockIdx.x] = tot;
}

static size_t ysweep_reg_smem(int sb, int nst) {
  constexpr int RB = ytile_rows<float>();
  return (size_t)nst * (RB + sb) * YTile<float>::CW * sizeof(float) +
         (size_t)(nst + 1) * RB * (sizeof(float4) + sizeof(float2)) + 16 + 32 * sizeof(double);
}

static int device_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename T>
static size_t ysweep_smem(int sb) {
  constexpr int RB = ytile_rows<T>();
  return sizeof(T) * ((size_t)(RB + sb) * YTile<T>::CW + 4 * (size_t)RB + 4) + 16 + 32 * sizeof(double);
}

template <typename T>
static void ysweep_grid(int n, int* gx, int* gy) {
  const int nb = n + 2;
  *gx = (nb + YTile<T>::M - 1) / YTile<T>::M;
  *gy = (nb + YTile<T>::CW - 1) / YTile<T>::CW;
}

// launch shape of the register-resident FP32 y sweep for strips of `re` rows:
// the kernel, its stages and CTAs per SM.  Taken: the shape with the most
// tiles in flight per SM, then the most CTAs (one stage each in two CTAs
// beats two stages in one: a second CTA also hides the sweep's latency).
// kernel = nullptr: not taken (strips of other heights).
struct YRegCfg {
  void (*kernel)(CUtensorMap, CUtensorMap, int, int, int, int, int, float*, const float2*, const float4*,
                 const float*, double*, int*) = nullptr;
  int nst = 0, cps = 0;
  size_t smem = 0;
};
// per: the period of the spill rows (strip height times the quadrature's
// cluster size), 8 for the strips the quadrature uses
static YRegCfg ysweep_reg_cfg(int per) {
  static YRegCfg memo;
  static bool done = false;
  YRegCfg c;
  if (per != 8) return c;
  if (done) return memo;
  const int sb = yspill_rows(ytile_rows<float>(), per);
  for (int nst = 1; nst <= 2; ++nst) {
    auto k = nst == 2 ? k_ysweep_reg_2d<8, 2> : k_ysweep_reg_2d<8, 1>;
    smem_optin(k);
    const size_t smem = ysweep_reg_smem(sb, nst);
    int cps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cps, k, YTile<float>::CW, smem) != cudaSuccess) {
      cudaGetLastError();
      cps = 0;
    }
    if (cps > 2) cps = 2;
    if (cps > 0 && (nst * cps > c.nst * c.cps || (nst * cps == c.nst * c.cps && cps > c.cps))) {
      c.kernel = k;
      c.nst = nst;
      c.cps = cps;
      c.smem = smem;
    }
  }
  memo = c;
  done = true;
  return c;
}

int ysweep_blocks(int n, size_t esize) {
  int gx, gy;
  if (esize == sizeof(float)) {
    ysweep_grid<float>(n, &gx, &gy);
    const int re = quad_rows(n, esize);
    const YRegCfg c = ysweep_reg_cfg(re * quad_cluster(re));
    if (c.kernel) return gx * gy < c.cps * device_sms() ? gx * gy : c.cps * device_sms();  // persistent
    return gx * gy;
  }
  ysweep_grid<double>(n, &gx, &gy);
  return gx * gy;
}

int ysolve_blocks(int dim, int n) {
  if (dim != 2) return ((n + 2) * (n + 2) + 127) / 128;
  const int a = ysweep_blocks(n, sizeof(float)), b = ysweep_blocks(n, sizeof(double));
  return a > b ? a : b;
}

// cuTensorMapEncodeTiled, taken from the driver at run time
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// row-major [rows][cols] array with row stride ld (elements), boxes of
// box_rows x box_cols, zero fill outside
template <typename T>
static cudaError_t tile_map(const T* base, int rows, int cols, int ld, int box_rows, int box_cols,
                            CUtensorMap* map) {
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(T)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  if (enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
          2, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_ysweep(const QuadArgs<T>& a, int re, const T* Xm, const T* Xs, int ldx, T* out,
                          double* mass_part, int* flags, cudaStream_t st) {
  if (a.dim != 2 || re < 2) return cudaErrorNotSupported;
  if (ldx < a.nb || (ldx * sizeof(T)) % 16 != 0 || (reinterpret_cast<uintptr_t>(Xm) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(Xs) & 15) != 0)
    return cudaErrorInvalidValue;
  constexpr int RB = ytile_rows<T>(), CW = YTile<T>::CW;
  const int nb = a.nb;
  // the quadrature's clusters of csz strips leave one spill pair per cluster:
  // DOF rows q per + {0, 1} (q >= 1) take Xs rows 2 (q - 1) + {0, 1}
  const int csz = quad_cluster(re), per = re * csz;
  const int nstrip = (a.n + re - 1) / re, ncl = (nstrip + csz - 1) / csz, nsp = 2 * (ncl - 1);
  const int sb = yspill_rows(RB, per);
  if (sb > 256) return cudaErrorInvalidValue;
  CUtensorMap xm_map, xs_map;
  cudaError_t err = tile_map<T>(Xm, nb, nb, ldx, RB, CW, &xm_map);
  if (err != cudaSuccess) return err;
  if (nsp > 0) err = tile_map<T>(Xs, nsp, nb, ldx, sb, CW, &xs_map);
  else xs_map = xm_map;  // not read
  if (err != cudaSuccess) return err;
  int gx, gy;
  ysweep_grid<T>(a.n, &gx, &gy);
  if constexpr (sizeof(T) == sizeof(float)) {
    const YRegCfg c = ysweep_reg_cfg(per);
    if (re == quad_rows(a.n, sizeof(T)) && c.kernel) {
      if (!a.ax.ytab) return cudaErrorInvalidValue;
      const int ntile = gx * gy, grid = ysweep_blocks(a.n, sizeof(T));
      const float2* tfw = reinterpret_cast<const float2*>(a.ax.ytab);
      const float4* tbw = reinterpret_cast<const float4*>(tfw + ysweep_table_rows(a.n));
      c.kernel<<<grid, CW, c.smem, st>>>(xm_map, xs_map, a.n, nsp, sb, gx, ntile, out, tfw, tbw, a.ax.Iw,
                                         mass_part, flags);
      return cudaGetLastError();
    }
  }
  const size_t smem = ysweep_smem<T>(sb);
  auto k = k_ysweep_2d<T>;
  smem_optin(k);
  k<<<dim3(gx, gy), CW, smem, st>>>(xm_map, xs_map, a.n, per, nsp, sb, out, a.ax.l1, a.ax.l2,
                                    a.ax.dinv, a.ax.Iw, mass_part, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zsolve(const QuadArgs<T>&, T*, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}

// int S = sum_kl S_kl (int B_k)(int B_l): thread per column
template <typename T>
__global__ void __launch_bounds__(128) k_mass_2d(int n, const T* S, const T* Iw, double* part) {
  __shared__ double red[32];
  const int nb = n + 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (k < nb) {
    for (int l = 0; l < nb; ++l) m += (double)S[(size_t)l * nb + k] * (double)Iw[l];
    m *= (double)Iw[k];
  }
  double tot = block_sum(m, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename T>
cudaError_t launch_mass(const QuadArgs<T>& a, const T* S, double* mass_part, cudaStream_t st) {
  if (a.dim != 2) return cudaErrorNotSupported;
  int nblk = (a.nb + 127) / 128;
  k_mass_2d<T><<<nblk, 128, 0, st>>>(a.n, S, a.ax.Iw, mass_part);
  int nmax = ysolve_blocks(2, a.n);
  if (nblk < nmax) cudaMemsetAsync(mass_part + nblk, 0, sizeof(double) * (nmax - nblk), st);
  return cudaGetLastError();
}

// stats[0] = int S, stats[1] += step mass error, stats[2] += source integral
__global__ void __launch_bounds__(256) k_mass_finalize(const double* mp, int nm, const double* sp,
                                                       int ns, int mode, double* stats, int* flags) {
  __shared__ double red[32];
  double m = 0.0, s = 0.0;
  for (int i = threadIdx.x; i < nm; i += blockDim.x) m += mp[i];
  for (int i = threadIdx.x; i < ns; i += blockDim.x) s += sp[i];
  m = block_sum(m, red);
  s = block_sum(s, red);
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    stats[0] = m;
  } else {
    stats[1] += m - stats[0] - s;
    stats[2] += s;
    stats[0] = m;
  }
  if (!isfinite(m)) flags[0] |= 1;
}

cudaError_t launch_mass_finalize(const double* mass_part, int nmass, const double* src_part,
                                 int nsrc, int mode, double* stats, int* flags, cudaStream_t st) {
  k_mass_finalize<<<1, 256, 0, st>>>(mass_part, nmass, src_part, nsrc, mode, stats, flags);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CFL step size: max over Gauss points of |K (grad p + s rho_g g e)|/(mu_g phi)
// and of q_inj/phi
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_cfl_2d(QuadArgs<T> a, double* part) {
  __shared__ double red[32];
  const int n = a.n, nb = a.nb, n1 = n + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double vmax = 0.0, smax = 0.0;
  if (e < n * n) {
    const int ex = e % n, ey = e / n;
    const T* Bx = a.ax.B + ex * 9; const T* dBx = a.ax.dB + ex * 9;
    const T* By = a.ax.B + ey * 9; const T* dBy = a.ax.dB + ey * 9;
    T Px[3][3], Pdx[3][3];
    for (int b = 0; b < 3; ++b) {
      const T* prow = a.P + (size_t)(ey + b) * nb + ex;
      for (int q = 0; q < 3; ++q) {
        Px[b][q] = prow[0] * Bx[q] + prow[1] * Bx[3 + q] + prow[2] * Bx[6 + q];
        Pdx[b][q] = prow[0] * dBx[q] + prow[1] * dBx[3 + q] + prow[2] * dBx[6 + q];
      }
    }
    const T* Kr = a.K + (size_t)ey * n1 + ex;
    T k00 = Kr[0], k01 = Kr[1], k10 = Kr[n1], k11 = Kr[n1 + 1];
    T f00 = a.phi_c, f01 = a.phi_c, f10 = a.phi_c, f11 = a.phi_c;
    if (a.phi) {
      const T* Fr = a.phi + (size_t)ey * n1 + ex;
      f00 = Fr[0]; f01 = Fr[1]; f10 = Fr[n1]; f11 = Fr[n1 + 1];
    }
    for (int qy = 0; qy < 3; ++qy)
      for (int qx = 0; qx < 3; ++qx) {
        T xi = (T)gauss_x(qx), eta = (T)gauss_x(qy);
        T dpx = By[qy] * Pdx[0][qx] + By[3 + qy] * Pdx[1][qx] + By[6 + qy] * Pdx[2][qx];
        T dpy = dBy[qy] * Px[0][qx] + dBy[3 + qy] * Px[1][qx] + dBy[6 + qy] * Px[2][qx];
        T Kq = (T(1) - eta) * ((T(1) - xi) * k00 + xi * k01) + eta * ((T(1) - xi) * k10 + xi * k11);
        T phq = (T(1) - eta) * ((T(1) - xi) * f00 + xi * f01) + eta * ((T(1) - xi) * f10 + xi * f11);
        T fx = Kq * dpx, fy = Kq * (dpy + a.grav_term);
        double v = sqrt((double)(fx * fx + fy * fy)) * (double)a.inv_mu_g / (double)phq;
        vmax = fmax(vmax, v);
        T qi = T(0);
        for (int s = 0; s < a.n_src; ++s)
          if (a.kind[s] == 0)
            qi += a.rate[s] * a.ax.gsrc[((size_t)(0 * kMaxSrc + s) * n + ex) * 3 + qx] *
                  a.ax.gsrc[((size_t)(1 * kMaxSrc + s) * n + ey) * 3 + qy];
        smax = fmax(smax, (double)(qi / phq));
      }
  }
  double r1 = block_max(vmax, red);
  __syncthreads();
  double r2 = block_max(smax, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r1;
    part[2 * blockIdx.x + 1] = r2;
  }
}

int cfl_blocks(int dim, int n) {
  long long ne = 1;
  for (int i = 0; i < dim; ++i) ne *= n;
  return (int)((ne + 255) / 256);
}

template <typename T>
cudaError_t launch_cfl(const QuadArgs<T>& a, double* part, cudaStream_t st) {
  if (a.dim != 2) return cudaErrorNotSupported;
  k_cfl_2d<T><<<cfl_blocks(2, a.n), 256, 0, st>>>(a, part);
  return cudaGetLastError();
}

__global__ void k_cfl_finalize(const double* part, int nblk, double cfl, double frac, double cap,
                               double h, double* dt, int* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double vmax = 0.0, smax = 0.0;
  for (int i = 0; i < nblk; ++i) {
    vmax = fmax(vmax, part[2 * i]);
    smax = fmax(smax, part[2 * i + 1]);
  }
  double d = cap;
  if (vmax > 0.0) d = fmin(d, cfl * h / vmax);
  if (smax > 0.0) d = fmin(d, frac / smax);
  if (!isfinite(d) || d <= 0.0) flags[0] |= 2;
  *dt = d;
}

cudaError_t launch_cfl_finalize(const double* part, int nblk, double cfl, double src_frac,
                                double dt_cap, double h, double* dt, int* flags, cudaStream_t st) {
  k_cfl_finalize<<<1, 32, 0, st>>>(part, nblk, cfl, src_frac, dt_cap, h, dt, flags);
  return cudaGetLastError();
}

#define ADS_INST(T)                                                                              \
  template cudaError_t launch_quad_xsweep<T>(const QuadArgs<T>&, int, int, T*, T*, int, double*, \
                                             cudaStream_t);                                      \
  template cudaError_t launch_ysweep<T>(const QuadArgs<T>&, int, const T*, const T*, int, T*,    \
                                        double*, int*, cudaStream_t);                            \
  template cudaError_t launch_zsolve<T>(const QuadArgs<T>&, T*, double*, cudaStream_t);          \
  template cudaError_t launch_mass<T>(const QuadArgs<T>&, const T*, double*, cudaStream_t);      \
  template cudaError_t launch_cfl<T>(const QuadArgs<T>&, double*, cudaStream_t);
ADS_INST(double)
ADS_INST(float)

}  // namespace adsgb

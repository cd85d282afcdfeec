// Gram solve z = G^{-1} RES and the robust loss RES^T z (Eqs. 26-28) for 2D
// collocation grids whose interval count N is a power of two.
//
// G = h^-2 (T (x) I + I (x) T) with T = tridiag(-1, 2, -1) of size m = N - 1
// (the 5-point stencil of Eq. 26 with zero Dirichlet values).  The unnormalised
// sine transform D, (D x)_k = sum_j x_j sin(pi j k / N), diagonalises T with
// eigenvalues lambda_k = 2 - 2 cos(pi k / N) and satisfies D D = (N / 2) I, so
//
//   G^-1 = h^2 (2 / N)^2 (D (x) D) diag(1 / (lambda_i + lambda_j)) (D (x) D).
//
// The paper factorises G once and applies the factors by substitution; this
// route reaches the same z (up to rounding) with O(N^2 log N) work per
// application.  D is computed with a complex FFT of length L = 2N of the odd
// extension y = (0, x_1..x_{N-1}, 0, -x_{N-1}..-x_1): its transform is
// Y_k = -2i (D x)_k, so (D x)_k = -Im(Y_k) / 2.  Two lines a, b share one
// FFT: the transform of y_a + i y_b is -2i (D a)_k + 2 (D b)_k, so
// (D a)_k = -Im / 2 and (D b)_k = Re / 2.  The FFT is the Stockham
// self-sorting form with radix-4 passes (and one radix-2 pass when log2 L is
// odd) between two shared-memory buffers.
//
// Three passes over the m x m grid (row-major, x fastest):
//   rows:    D along x of every row                           (k_dst_rows)
//   columns: D along y, times s / (lambda_i + lambda_j), D along y again,
//            for a block of x-modes i                         (k_gram_cols)
//   rows:    D along x, and per-CTA partials of RES^T z        (k_dst_rows)
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.cuh"

namespace adsgb {

namespace {

template <typename T>
struct __align__(2 * sizeof(T)) Cx {
  T re, im;
};

constexpr int kFftThreads = 256;
constexpr int KB = 4;  // values a thread loads together before it stores any

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> w) {
  return Cx<T>{a.re * w.re - a.im * w.im, a.re * w.im + a.im * w.re};
}

// Stockham FFT of P lines of length L = 2^lg stored one after another in a
// (b is scratch of the same size); twiddles tw[q] = exp(-2 pi i q / L),
// q < L.  A pass of radix R over sub-transforms of length Ns: butterfly j
// reads x[j + r L/R], multiplies by exp(-2 pi i r k / (Ns R)) with
// k = j mod Ns, takes the R-point DFT and writes y[(j - k) R + k + r Ns].
// Returns the buffer that holds the result.
template <typename T>
__device__ __forceinline__ Cx<T>* fft_stockham(Cx<T>* a, Cx<T>* b, int P, int lg, const Cx<T>* tw) {
  const int L = 1 << lg;
  int Ns = 1, rem = lg;
  while (rem > 0) {
    const int lr = rem >= 2 ? 2 : 1, R = 1 << lr;
    const int nbl = L >> lr;  // butterflies per line
    for (int t = threadIdx.x; t < P * nbl; t += blockDim.x) {
      const int line = t >> (lg - lr), j = t & (nbl - 1);
      const Cx<T>* x = a + (line << lg);
      Cx<T>* y = b + (line << lg);
      const int k = j & (Ns - 1);
      const int step = k * (L / (Ns * R));
      const int base = (j - k) * R + k;
      if (R == 4) {
        Cx<T> v0 = x[j], v1 = x[j + nbl], v2 = x[j + 2 * nbl], v3 = x[j + 3 * nbl];
        if (k) {
          v1 = cmul(v1, tw[step]);
          v2 = cmul(v2, tw[2 * step]);
          v3 = cmul(v3, tw[3 * step]);
        }
        const Cx<T> a0{v0.re + v2.re, v0.im + v2.im}, a1{v0.re - v2.re, v0.im - v2.im};
        const Cx<T> a2{v1.re + v3.re, v1.im + v3.im};
        const Cx<T> a3{v1.im - v3.im, v3.re - v1.re};  // (v1 - v3) (-i)
        y[base] = Cx<T>{a0.re + a2.re, a0.im + a2.im};
        y[base + Ns] = Cx<T>{a1.re + a3.re, a1.im + a3.im};
        y[base + 2 * Ns] = Cx<T>{a0.re - a2.re, a0.im - a2.im};
        y[base + 3 * Ns] = Cx<T>{a1.re - a3.re, a1.im - a3.im};
      } else {
        Cx<T> v0 = x[j], v1 = x[j + nbl];
        if (k) v1 = cmul(v1, tw[step]);
        y[base] = Cx<T>{v0.re + v1.re, v0.im + v1.im};
        y[base + Ns] = Cx<T>{v0.re - v1.re, v0.im - v1.im};
      }
    }
    __syncthreads();
    Cx<T>* tmp = a;
    a = b;
    b = tmp;
    Ns <<= lr;
    rem -= lr;
  }
  return a;
}

// value j of the odd extension (length 2N) of x_1..x_{N-1} = v[0..N-2]
template <typename T>
__device__ __forceinline__ T odd_ext(const T* v, int j, int N, int stride) {
  if (j > 0 && j < N) return v[(size_t)(j - 1) * stride];
  if (j > N) return -v[(size_t)(2 * N - j - 1) * stride];
  return T(0);
}

// RES = A u + h^2 f on the interior nodes (Eqs. 24-25, 5-point form): the
// residual the first row pass computes itself when given the network values
template <typename T>
struct ResidualIn {
  const T* u;      // network values on the interior nodes, [m][m]; nullptr: read `in`
  const T* alpha;  // coefficients on all nodes, [N+1][N+1]
  const T* f;      // right-hand side on the interior nodes, [m][m]
  T h2;
  T* res;          // written: RES, [m][m]
};
template <typename T>
__device__ __forceinline__ T residual_at(const ResidualIn<T>& q, int N, int jj, int ii) {
  const int m = N - 1, n1 = N + 1;
  const size_t t = (size_t)jj * m + ii;
  const int j = jj + 1, i = ii + 1;  // node index
  const T c = q.u[t];
  const T w = ii > 0 ? q.u[t - 1] : T(0);
  const T e = ii < m - 1 ? q.u[t + 1] : T(0);
  const T s = jj > 0 ? q.u[t - m] : T(0);
  const T nn = jj < m - 1 ? q.u[t + m] : T(0);
  const T ac = q.alpha[(size_t)j * n1 + i];
  const T aw = q.alpha[(size_t)j * n1 + i - 1];
  const T as = q.alpha[(size_t)(j - 1) * n1 + i];
  T r = aw * (c - w) - ac * (e - c) + as * (c - s) - ac * (nn - c);
  return r + q.h2 * q.f[t];
}

// D along x for rows [r0, r0 + 2P) of the nrows rows of `in` into `out`,
// times `scale` (rows 2p and 2p + 1 of the CTA share line p).  With rin.u
// set (2D), the rows are first computed as RES = A u + h^2 f and written to
// rin.res.  With dotw != nullptr, also a partial of sum dotw * out over the
// CTA's rows.
template <typename T>
__device__ __forceinline__ void dst_rows_body(const T* __restrict__ in, T* __restrict__ out, int N, int lg, int P,
                                              const Cx<T>* __restrict__ tw, const T* __restrict__ dotw,
                                              double* dot_part, const ResidualIn<T>& rin, int nrows, T scale,
                                              int bid) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1;
  Cx<T>* tws = reinterpret_cast<Cx<T>*>(fsm);  // [L]
  Cx<T>* buf0 = tws + L;                       // [P][L]
  Cx<T>* buf1 = buf0 + (size_t)P * L;          // [P][L]
  __shared__ double red[32];
  const int r0 = bid * 2 * P;
  for (int q = threadIdx.x; q < L; q += blockDim.x) tws[q] = tw[q];
  const T* src = in;
  int sstride = m;  // row stride of the source rows
  size_t soff = (size_t)r0 * m;
  if (rin.u) {
    // the CTA's residual rows, staged in the second buffer ([2P][m] reals);
    // each thread computes a batch of KB values (loads issued together)
    // before it stores any
    T* stage = reinterpret_cast<T*>(buf1);
    const int tot = 2 * P * m;
    for (int b0 = 0; b0 < tot; b0 += KB * (int)blockDim.x) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        const int rr = idx / m, ii = idx - rr * m, row = r0 + rr;
        v[q] = (idx < tot && row < nrows) ? residual_at(rin, N, row, ii) : T(0);
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        const int rr = idx / m, ii = idx - rr * m, row = r0 + rr;
        if (idx < tot) {
          if (row < nrows) rin.res[(size_t)row * m + ii] = v[q];
          stage[idx] = v[q];
        }
      }
    }
    __syncthreads();
    src = stage;
    soff = 0;
  }
  // odd extensions: value i of row r goes to positions i + 1 and 2N - 1 - i
  // of its line (the real part for the even row of a pair, the imaginary
  // part for the odd row); positions 0 and N are zero
  {
    T* b0r = reinterpret_cast<T*>(buf0);
    for (int idx = threadIdx.x; idx < P * 2; idx += blockDim.x) {
      const int line = idx >> 1, part = idx & 1;
      b0r[2 * ((line << lg) + 0) + part] = T(0);
      b0r[2 * ((line << lg) + N) + part] = T(0);
    }
    const int tot = 2 * P * m;
    for (int b0 = 0; b0 < tot; b0 += KB * (int)blockDim.x) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        const int rr = idx / m, ii = idx - rr * m;
        v[q] = (idx < tot && r0 + rr < nrows) ? src[soff + (size_t)rr * sstride + ii] : T(0);
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        if (idx < tot) {
          const int rr = idx / m, ii = idx - rr * m, line = rr >> 1, part = rr & 1;
          b0r[2 * ((line << lg) + ii + 1) + part] = v[q];
          b0r[2 * ((line << lg) + 2 * N - 1 - ii) + part] = -v[q];
        }
      }
    }
  }
  __syncthreads();
  const Cx<T>* z = fft_stockham(buf0, buf1, P, lg, tws);
  CompSum<T> dot;
  const int tot = 2 * P * m;
  for (int b0 = 0; b0 < tot; b0 += KB * (int)blockDim.x) {
    T w[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int idx = b0 + q * blockDim.x + threadIdx.x;
      const int rr = idx / m, ii = idx - rr * m, row = r0 + rr;
      w[q] = (dotw && idx < tot && row < nrows) ? dotw[(size_t)row * m + ii] : T(0);
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int idx = b0 + q * blockDim.x + threadIdx.x;
      const int rr = idx / m, k = idx - rr * m + 1, row = r0 + rr;
      if (idx < tot && row < nrows) {
        const Cx<T> zk = z[((rr >> 1) << lg) + k];
        const T v = scale * ((rr & 1) ? T(0.5) * zk.re : T(-0.5) * zk.im);
        out[(size_t)row * m + k - 1] = v;
        if (dotw) dot.add(v * w[q]);
      }
    }
  }
  if (dotw) {
    const double tot = block_sum(dot.value(), red);
    if (threadIdx.x == 0) dot_part[bid] = tot;
  }
}
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    k_dst_rows(const T* __restrict__ in, T* __restrict__ out, int N, int lg, int P,
               const Cx<T>* __restrict__ tw, const T* __restrict__ dotw, double* dot_part,
               ResidualIn<T> rin, int nrows, T scale) {
  dst_rows_body<T>(in, out, N, lg, P, tw, dotw, dot_part, rin, nrows, scale, blockIdx.x);
}

// For x-modes i in [c0, c0 + 2P): D along y, times scale / (lam_i + lam_j),
// D along y again; in place.  Columns 2p and 2p + 1 of the CTA share line p.
template <typename T>
__device__ __forceinline__ void gram_cols_body(T* __restrict__ data, int N, int lg, int P,
                                               const Cx<T>* __restrict__ tw, const T* __restrict__ lam, T scale,
                                               int bid) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1, C = 2 * P;
  Cx<T>* tws = reinterpret_cast<Cx<T>*>(fsm);  // [L]
  Cx<T>* buf0 = tws + L;                       // [P][L]
  Cx<T>* buf1 = buf0 + (size_t)P * L;          // [P][L]
  const int c0 = bid * C;
  T* lams = reinterpret_cast<T*>(buf1);  // [m] eigenvalues until the first transform is done
  for (int q = threadIdx.x; q < L; q += blockDim.x) tws[q] = tw[q];
  for (int q = threadIdx.x; q < m; q += blockDim.x) lams[q] = lam[q];
  // odd extensions of the CTA's columns (column c of the CTA fastest: a warp
  // reads C neighbouring values of rows): value j of column c goes to
  // positions j + 1 and 2N - 1 - j of line c / 2 (part c % 2)
  {
    T* b0r = reinterpret_cast<T*>(buf0);
    for (int idx = threadIdx.x; idx < C; idx += blockDim.x) {
      const int line = idx >> 1, part = idx & 1;
      b0r[2 * ((line << lg) + 0) + part] = T(0);
      b0r[2 * ((line << lg) + N) + part] = T(0);
    }
    const int tot = C * m;
    for (int b0 = 0; b0 < tot; b0 += KB * (int)blockDim.x) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        const int c = idx % C, j = idx / C, col = c0 + c;
        v[q] = (idx < tot && col < m) ? data[(size_t)j * m + col] : T(0);
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        if (idx < tot) {
          const int c = idx % C, j = idx / C, line = c >> 1, part = c & 1;
          b0r[2 * ((line << lg) + j + 1) + part] = v[q];
          b0r[2 * ((line << lg) + 2 * N - 1 - j) + part] = -v[q];
        }
      }
    }
  }
  __syncthreads();
  // the eigenvalues to registers before the transform overwrites buf1
  T lc[KB], lk[KB];
  {
    const int tot = C * m;
    // (this thread's first KB scaled values; C m <= KB blockDim.x whenever
    // P L <= 1024, else the rest reread lams after the copy below)
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      const int idx = q * blockDim.x + threadIdx.x;
      const int c = idx / m, k = idx - c * m + 1, col = c0 + c;
      lc[q] = (idx < tot && col < m) ? lams[col] : T(1);
      lk[q] = idx < tot ? lams[k - 1] : T(1);
    }
  }
  __syncthreads();
  Cx<T>* z = fft_stockham(buf0, buf1, P, lg, tws);
  T* vt = reinterpret_cast<T*>(z == buf0 ? buf1 : buf0);  // [C][N] scaled transforms
  for (int q = 0; q < KB; ++q) {
    const int idx = q * blockDim.x + threadIdx.x;
    if (idx < C * m) {
      const int c = idx / m, k = idx - c * m + 1;
      const Cx<T> zk = z[((c >> 1) << lg) + k];
      const T d = (c & 1) ? T(0.5) * zk.re : T(-0.5) * zk.im;
      vt[c * N + k - 1] = d * (scale / (lc[q] + lk[q]));
    }
  }
  for (int idx = KB * blockDim.x + threadIdx.x; idx < C * m; idx += blockDim.x) {
    const int c = idx / m, k = idx - c * m + 1, col = c0 + c;
    const Cx<T> zk = z[((c >> 1) << lg) + k];
    const T d = (c & 1) ? T(0.5) * zk.re : T(-0.5) * zk.im;
    const T li = col < m ? lam[col] : T(1);
    vt[c * N + k - 1] = d * (scale / (li + lam[k - 1]));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < P * L; idx += blockDim.x) {
    const int line = idx >> lg, j = idx & (L - 1);
    z[idx] = Cx<T>{odd_ext(vt + (2 * line) * N, j, N, 1), odd_ext(vt + (2 * line + 1) * N, j, N, 1)};
  }
  __syncthreads();
  Cx<T>* w = fft_stockham(z, reinterpret_cast<Cx<T>*>(vt), P, lg, tws);
  for (int idx = threadIdx.x; idx < C * m; idx += blockDim.x) {
    const int c = idx % C, k = idx / C + 1;
    const int col = c0 + c;
    const Cx<T> wk = w[((c >> 1) << lg) + k];
    if (col < m) data[(size_t)(k - 1) * m + col] = (c & 1) ? T(0.5) * wk.re : T(-0.5) * wk.im;
  }
}
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    k_gram_cols(T* __restrict__ data, int N, int lg, int P, const Cx<T>* __restrict__ tw,
                const T* __restrict__ lam, T scale) {
  gram_cols_body<T>(data, N, lg, P, tw, lam, scale, blockIdx.x);
}

// ---- grouped passes (2D, FP32): one launch per pass over several contexts ----
struct RowsArgs {
  const float* in;
  float* out;
  int N, lg, P, nrows;
  const Cx<float>* tw;
  const float* dotw;
  double* dot_part;
  ResidualIn<float> rin;
  float scale;
};
struct ColsArgs {
  float* data;
  int N, lg, P;
  const Cx<float>* tw;
  const float* lam;
  float scale;
};
__global__ void __launch_bounds__(kFftThreads) k_dst_rows_grp(const RowsArgs* __restrict__ tab, GroupMap g) {
  const int2 c = g.cta[blockIdx.x];
  const RowsArgs& a = tab[c.x];
  dst_rows_body<float>(a.in, a.out, a.N, a.lg, a.P, a.tw, a.dotw, a.dot_part, a.rin, a.nrows, a.scale, c.y);
}
__global__ void __launch_bounds__(kFftThreads) k_gram_cols_grp(const ColsArgs* __restrict__ tab, GroupMap g) {
  const int2 c = g.cta[blockIdx.x];
  const ColsArgs& a = tab[c.x];
  gram_cols_body<float>(a.data, a.N, a.lg, a.P, a.tw, a.lam, a.scale, c.y);
}

// 3D: D along y of columns [c0, c0 + 2P) of plane blockIdx.y of the m x m x m
// grid ([z][y][x]), in place (columns 2p and 2p + 1 of the CTA share line p)
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    k_dst_cols(T* __restrict__ data, int N, int lg, int P, const Cx<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1, C = 2 * P;
  Cx<T>* tws = reinterpret_cast<Cx<T>*>(fsm);  // [L]
  Cx<T>* buf0 = tws + L;                       // [P][L]
  Cx<T>* buf1 = buf0 + (size_t)P * L;          // [P][L]
  const int c0 = blockIdx.x * C;
  T* plane = data + (size_t)blockIdx.y * m * m;
  for (int q = threadIdx.x; q < L; q += blockDim.x) tws[q] = tw[q];
  {
    T* b0r = reinterpret_cast<T*>(buf0);
    for (int idx = threadIdx.x; idx < C; idx += blockDim.x) {
      const int line = idx >> 1, part = idx & 1;
      b0r[2 * ((line << lg) + 0) + part] = T(0);
      b0r[2 * ((line << lg) + N) + part] = T(0);
    }
    const int tot = C * m;
    for (int b0 = 0; b0 < tot; b0 += KB * (int)blockDim.x) {
      T v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        const int c = idx % C, j = idx / C, col = c0 + c;
        v[q] = (idx < tot && col < m) ? plane[(size_t)j * m + col] : T(0);
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * blockDim.x + threadIdx.x;
        if (idx < tot) {
          const int c = idx % C, j = idx / C, line = c >> 1, part = c & 1;
          b0r[2 * ((line << lg) + j + 1) + part] = v[q];
          b0r[2 * ((line << lg) + 2 * N - 1 - j) + part] = -v[q];
        }
      }
    }
  }
  __syncthreads();
  const Cx<T>* z = fft_stockham(buf0, buf1, P, lg, tws);
  for (int idx = threadIdx.x; idx < C * m; idx += blockDim.x) {
    const int c = idx % C, k = idx / C + 1, col = c0 + c;
    const Cx<T> zk = z[((c >> 1) << lg) + k];
    if (col < m) plane[(size_t)(k - 1) * m + col] = (c & 1) ? T(0.5) * zk.re : T(-0.5) * zk.im;
  }
}

int log2_exact(int N) {
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  return (1 << lg) == N ? lg : -1;
}

// twiddles and two buffers of P lines of L complex values
template <typename T>
size_t fft_smem(int L, int P) {
  return ((size_t)L + 2 * (size_t)P * L) * sizeof(Cx<T>);
}

// line pairs per CTA: enough butterflies for the threads, within the shared memory
template <typename T>
int lines_per_cta(int L, int minP) {
  int P = 1024 / L;
  if (P < minP) P = minP;
  if (P < 1) P = 1;
  while (P > 1 && fft_smem<T>(L, P) > 200 * 1024) P /= 2;
  return P;
}

// ---------------------------------------------------------------------------
// The whole Gram solve (residual, rows, columns, rows, RES^T z) in one
// thread-block cluster, for FP32 and N <= 128: CTA r of the cluster owns rows
// [r R, r R + R) of the m x m grid and, for the column pass, the same range of
// columns.  The row transforms of its rows stay in its shared memory (slab);
// the column pass reads and writes the slabs of the other CTAs of the cluster
// through distributed shared memory, so the intermediate grid never leaves the
// chip and the solve is one launch instead of three.
// ---------------------------------------------------------------------------
namespace cgx = cooperative_groups;

// zero positions 0 and N of each of the P lines of buf (the odd extension's
// fixed zeros)
__device__ __forceinline__ void clear_ext_zeros(Cx<float>* buf, int P, int lg, int N) {
  for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
    buf[(idx << lg) + 0] = Cx<float>{0.f, 0.f};
    buf[(idx << lg) + N] = Cx<float>{0.f, 0.f};
  }
}
// value v of row (or column) q of the batch at index i of its line: positions
// i + 1 and 2N - 1 - i of line q / 2, part q % 2 (real, imaginary)
__device__ __forceinline__ void put_ext(Cx<float>* buf, int lg, int N, int q, int i, float v) {
  float* b = reinterpret_cast<float*>(buf);
  const int line = q >> 1, part = q & 1;
  b[2 * ((line << lg) + i + 1) + part] = v;
  b[2 * ((line << lg) + 2 * N - 1 - i) + part] = -v;
}
// (D x)_k of row (or column) q of the batch from the transform z
__device__ __forceinline__ float take_dst(const Cx<float>* z, int lg, int q, int k) {
  const Cx<float> zk = z[((q >> 1) << lg) + k];
  return (q & 1) ? 0.5f * zk.re : -0.5f * zk.im;
}

__global__ void __launch_bounds__(1024) k_gram_cluster(ResidualIn<float> rin, float* __restrict__ zout,
                                                       const Cx<float>* __restrict__ tw,
                                                       const float* __restrict__ lam, float scale,
                                                       double* dot_part, int N, int lg, int R, int P) {
  cgx::cluster_group cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1, tid = threadIdx.x, T = blockDim.x;
  Cx<float>* tws = reinterpret_cast<Cx<float>*>(fsm);  // [L]
  Cx<float>* buf0 = tws + L;                           // [P][L]
  Cx<float>* buf1 = buf0 + (size_t)P * L;              // [P][L]
  float* lams = reinterpret_cast<float*>(buf1 + (size_t)P * L);  // [m], padded to 4
  float* slab = lams + ((m + 3) & ~3);                           // [R][m]: this CTA's rows
  __shared__ double red[32];
  for (int q = tid; q < L; q += T) tws[q] = tw[q];
  for (int q = tid; q < m; q += T) lams[q] = lam[q];
  const int r0 = rank * R, nr = max(0, min(R, m - r0));
  const int bt = 2 * P * m;  // values per batch of 2P rows or columns
  // ---- rows: RES = A u + h^2 f, then D along x, into the slab ----
  for (int p0 = 0; p0 < nr; p0 += 2 * P) {
    __syncthreads();  // the buffers are free
    clear_ext_zeros(buf0, P, lg, N);
    for (int b0 = 0; b0 < bt; b0 += KB * T) {
      float v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * T + tid, rr = idx / m, ii = idx - rr * m;
        v[q] = (idx < bt && p0 + rr < nr) ? residual_at(rin, N, r0 + p0 + rr, ii) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * T + tid, rr = idx / m, ii = idx - rr * m;
        if (idx < bt) {
          if (p0 + rr < nr) rin.res[(size_t)(r0 + p0 + rr) * m + ii] = v[q];
          put_ext(buf0, lg, N, rr, ii, v[q]);
        }
      }
    }
    __syncthreads();
    const Cx<float>* z = fft_stockham(buf0, buf1, P, lg, tws);
    for (int idx = tid; idx < bt; idx += T) {
      const int rr = idx / m, k = idx - rr * m + 1;
      if (p0 + rr < nr) slab[(p0 + rr) * m + k - 1] = take_dst(z, lg, rr, k);
    }
  }
  cl.sync();  // every slab holds its rows' transforms
  // ---- columns: D along y, times scale / (lam_i + lam_j), D along y ----
  for (int p0 = 0; p0 < nr; p0 += 2 * P) {
    __syncthreads();
    clear_ext_zeros(buf0, P, lg, N);
    // column c of the batch fastest: a warp reads 2P neighbouring values of a
    // row of one slab
    for (int b0 = 0; b0 < bt; b0 += KB * T) {
      float v[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * T + tid, c = idx % (2 * P), j = idx / (2 * P);
        float x = 0.f;
        if (idx < bt && p0 + c < nr) {
          const float* rs = cl.map_shared_rank(slab, j / R);
          x = rs[(j % R) * m + r0 + p0 + c];
        }
        v[q] = x;
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * T + tid, c = idx % (2 * P), j = idx / (2 * P);
        if (idx < bt) put_ext(buf0, lg, N, c, j, v[q]);
      }
    }
    __syncthreads();
    Cx<float>* z = fft_stockham(buf0, buf1, P, lg, tws);
    Cx<float>* other = z == buf0 ? buf1 : buf0;
    float* vt = reinterpret_cast<float*>(other);  // [2P][N] scaled transforms
    for (int idx = tid; idx < bt; idx += T) {
      const int c = idx / m, k = idx - c * m + 1, col = r0 + p0 + c;
      const float li = p0 + c < nr ? lams[col] : 1.f;
      vt[c * N + k - 1] = take_dst(z, lg, c, k) * (scale / (li + lams[k - 1]));
    }
    __syncthreads();
    clear_ext_zeros(z, P, lg, N);
    for (int idx = tid; idx < bt; idx += T) {
      const int c = idx / m, i = idx - c * m;
      put_ext(z, lg, N, c, i, vt[c * N + i]);
    }
    __syncthreads();
    const Cx<float>* w = fft_stockham(z, other, P, lg, tws);
    // back into the slabs, column c of the batch fastest
    for (int idx = tid; idx < bt; idx += T) {
      const int c = idx % (2 * P), k = idx / (2 * P) + 1;
      if (p0 + c < nr) {
        float* rs = cl.map_shared_rank(slab, (k - 1) / R);
        rs[((k - 1) % R) * m + r0 + p0 + c] = take_dst(w, lg, c, k);
      }
    }
  }
  cl.sync();  // every slab holds its rows of the column pass
  // ---- rows: D along x gives z; partial of RES^T z ----
  CompSum<float> dot;
  for (int p0 = 0; p0 < nr; p0 += 2 * P) {
    __syncthreads();
    clear_ext_zeros(buf0, P, lg, N);
    for (int idx = tid; idx < bt; idx += T) {
      const int rr = idx / m, ii = idx - rr * m;
      put_ext(buf0, lg, N, rr, ii, p0 + rr < nr ? slab[(p0 + rr) * m + ii] : 0.f);
    }
    __syncthreads();
    const Cx<float>* z = fft_stockham(buf0, buf1, P, lg, tws);
    for (int b0 = 0; b0 < bt; b0 += KB * T) {
      float rv[KB];
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * T + tid, rr = idx / m, ii = idx - rr * m;
        rv[q] = (idx < bt && p0 + rr < nr) ? rin.res[(size_t)(r0 + p0 + rr) * m + ii] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < KB; ++q) {
        const int idx = b0 + q * T + tid, rr = idx / m, k = idx - rr * m + 1;
        if (idx < bt && p0 + rr < nr) {
          const float v = take_dst(z, lg, rr, k);
          zout[(size_t)(r0 + p0 + rr) * m + k - 1] = v;
          dot.add(v * rv[q]);
        }
      }
    }
  }
  const double tot = block_sum(dot.value(), red);
  if (tid == 0) dot_part[rank] = tot;
}

}  // namespace

// cluster size, rows per CTA, line pairs per batch, threads and shared memory
// of the one-cluster solve for N; CL = 0 when it does not apply (or the
// device cannot co-schedule the cluster)
GramClusterShape gram_cluster_shape(int N) {
  GramClusterShape s;
  const int lg = log2_exact(N);
  // 8 <= N <= 128: at N = 256 and 512 the cluster's 8-16 SMs take longer
  // (75 and 157 us) than the three passes over the whole GPU (39 and 51 us)
  if (lg < 3 || lg > 7) return s;
  const int L = 2 * N, m = N - 1, T = 1024;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int CL : {8}) {
    int R = (m + CL - 1) / CL;
    R += R & 1;
    int P = 4 * T / L;
    if (P > R / 2) P = R / 2;
    if (P < 1) P = 1;
    const size_t smem = ((size_t)L + 2 * (size_t)P * L) * sizeof(Cx<float>) +
                        (((size_t)m + 3) & ~size_t(3)) * sizeof(float) + (size_t)R * m * sizeof(float);
    if (smem + 1024 > (size_t)optin) continue;
    auto k = k_gram_cluster;
    // raise-only limit: contexts of other N launch this kernel with their own size
    smem_optin(k);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) != cudaSuccess || nc < 1) {
      cudaGetLastError();
      continue;
    }
    s.CL = CL;
    s.R = R;
    s.P = P;
    s.threads = T;
    s.smem = smem;
    return s;
  }
  return s;
}

cudaError_t launch_gram_cluster(const GramClusterShape& sh, int N, const float* u, const float* alpha,
                                const float* f, float h2, float* res_out, float* z, const float* tw,
                                const float* lam, double* dot_part, cudaStream_t st) {
  if (sh.CL <= 0) return cudaErrorNotSupported;
  const int lg = log2_exact(N) + 1;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = sh.CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(sh.CL);
  cfg.blockDim = dim3(sh.threads);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const ResidualIn<float> rin{u, alpha, f, h2, res_out};
  const float scale = h2 * (float)(4.0 / ((double)N * N));  // h^2 (2 / N)^2
  return cudaLaunchKernelEx(&cfg, k_gram_cluster, rin, z, reinterpret_cast<const Cx<float>*>(tw), lam, scale,
                            dot_part, N, lg, sh.R, sh.P);
}

bool gram_fft_supported(int dim, int N) {
  const int lg = log2_exact(N);
  if (dim == 3) return lg >= 3 && lg <= 9;  // N <= 512 (the 3D mesh limit)
  return dim == 2 && lg >= 3 && lg <= 11;  // L = 2N <= 4096
}

int gram_fft_dot_parts(int N, int dim) {
  const int m = N - 1, rows = dim == 3 ? m * m : m;
  const int P = lines_per_cta<double>(2 * N, 1);  // the row kernel's grid (FP64 bound)
  const int Pf = lines_per_cta<float>(2 * N, 1);
  const int g = (rows + 2 * P - 1) / (2 * P), gf = (rows + 2 * Pf - 1) / (2 * Pf);
  return g > gf ? g : gf;
}

template <typename T>
cudaError_t gram_fft_tables(int N, T* tw, T* lam) {
  const int L = 2 * N, m = N - 1;
  std::vector<T> h(2 * (size_t)L + m);
  const double pi = 3.14159265358979323846;
  for (int q = 0; q < L; ++q) {
    h[2 * q] = (T)std::cos(2.0 * pi * q / L);
    h[2 * q + 1] = (T)(-std::sin(2.0 * pi * q / L));
  }
  for (int k = 1; k <= m; ++k) {
    const double s = std::sin(pi * k / (2.0 * N));
    h[2 * L + k - 1] = (T)(4.0 * s * s);  // 2 - 2 cos(pi k / N)
  }
  cudaError_t e = cudaMemcpy(tw, h.data(), sizeof(T) * 2 * L, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(lam, h.data() + 2 * L, sizeof(T) * m, cudaMemcpyHostToDevice);
}

// pass 0: work = D_x res; pass 1: work <- h^2 (2/N)^2 D_y Lambda^-1 D_y work;
// pass 2: z = D_x work and the partials of res^T z
template <typename T>
cudaError_t launch_gram_fft(int pass, int N, const T* res, T* work, T* z, const T* tw, const T* lam,
                            T h2, double* dot_part, cudaStream_t st, const T* u, const T* alpha,
                            const T* f, T* res_out) {
  const int lg = log2_exact(N) + 1, L = 2 * N, m = N - 1;
  if (lg < 4 || lg > 12) return cudaErrorInvalidValue;
  const Cx<T>* twc = reinterpret_cast<const Cx<T>*>(tw);
  if (pass == 1) {
    const int P = lines_per_cta<T>(L, 2);
    const size_t smem = fft_smem<T>(L, P);
    auto k = k_gram_cols<T>;
    smem_optin(k);
    const T s = h2 * T(4.0 / ((double)N * N));  // h^2 (2 / N)^2
    k<<<(m + 2 * P - 1) / (2 * P), kFftThreads, smem, st>>>(work, N, lg, P, twc, lam, s);
  } else {
    const int P = lines_per_cta<T>(L, 1);
    const size_t smem = fft_smem<T>(L, P);
    auto k = k_dst_rows<T>;
    smem_optin(k);
    const int g = (m + 2 * P - 1) / (2 * P);
    ResidualIn<T> rin{nullptr, nullptr, nullptr, T(0), nullptr};
    if (pass == 0) {
      if (u) rin = ResidualIn<T>{u, alpha, f, h2, res_out};
      k<<<g, kFftThreads, smem, st>>>(res, work, N, lg, P, twc, nullptr, nullptr, rin, m, T(1));
    } else {
      k<<<g, kFftThreads, smem, st>>>(work, z, N, lg, P, twc, res, dot_part, rin, m, T(1));
    }
  }
  return cudaGetLastError();
}

// 3D (G = h^-2 (T (+) T (+) T)): pass 0: work = D_y D_x res (rows, then the
// columns of every plane); pass 2: z = h^2 (2/N)^2 D_x D_y work and the
// partials of res^T z.  Between them the caller solves the shifted
// tridiagonal systems along z for every (ky, kx) mode in place.
template <typename T>
cudaError_t launch_gram_fft3d(int pass, int N, const T* res, T* work, T* z, const T* tw, T h2,
                              double* dot_part, cudaStream_t st) {
  const int lg = log2_exact(N) + 1, L = 2 * N, m = N - 1;
  if (lg < 4 || lg > 10) return cudaErrorInvalidValue;
  const Cx<T>* twc = reinterpret_cast<const Cx<T>*>(tw);
  const int Pr = lines_per_cta<T>(L, 1), Pc = lines_per_cta<T>(L, 2);
  auto kr = k_dst_rows<T>;
  auto kc = k_dst_cols<T>;
  smem_optin(kr);
  smem_optin(kc);
  const int gr = (m * m + 2 * Pr - 1) / (2 * Pr);
  const dim3 gc((m + 2 * Pc - 1) / (2 * Pc), m);
  const ResidualIn<T> rin{nullptr, nullptr, nullptr, T(0), nullptr};
  if (pass == 0) {
    kr<<<gr, kFftThreads, fft_smem<T>(L, Pr), st>>>(res, work, N, lg, Pr, twc, nullptr, nullptr, rin, m * m, T(1));
    kc<<<gc, kFftThreads, fft_smem<T>(L, Pc), st>>>(work, N, lg, Pc, twc);
  } else {
    kc<<<gc, kFftThreads, fft_smem<T>(L, Pc), st>>>(work, N, lg, Pc, twc);
    const T s = h2 * T(4.0 / ((double)N * N));  // h^2 (2 / N)^2
    kr<<<gr, kFftThreads, fft_smem<T>(L, Pr), st>>>(work, z, N, lg, Pr, twc, res, dot_part, rin, m * m, s);
  }
  return cudaGetLastError();
}

struct GramGroup {
  DevGroup<RowsArgs> rows0, rows2;
  DevGroup<ColsArgs> cols;
  size_t smem_rows = 0, smem_cols = 0;
};

void gram_group_destroy(GramGroup* g) {
  if (!g) return;
  dev_group_free(g->rows0);
  dev_group_free(g->rows2);
  dev_group_free(g->cols);
  delete g;
}

cudaError_t gram_group_create(const GramGroupEntry* e, int n, GramGroup** out) {
  *out = nullptr;
  std::vector<RowsArgs> r0(n), r2(n);
  std::vector<ColsArgs> cc(n);
  std::vector<int> gr(n), gc(n);
  size_t sr = 0, sc = 0;
  for (int k = 0; k < n; ++k) {
    const int N = e[k].N, lg = log2_exact(N) + 1, L = 2 * N, m = N - 1;
    if (lg < 4 || lg > 12) return cudaErrorInvalidValue;
    const Cx<float>* twc = reinterpret_cast<const Cx<float>*>(e[k].tw);
    const int Pr = lines_per_cta<float>(L, 1), Pc = lines_per_cta<float>(L, 2);
    gr[k] = (m + 2 * Pr - 1) / (2 * Pr);
    gc[k] = (m + 2 * Pc - 1) / (2 * Pc);
    // the arguments launch_gram_fft gives its three passes
    r0[k] = RowsArgs{e[k].res, e[k].rhat, N, lg, Pr, m, twc, nullptr, nullptr,
                     ResidualIn<float>{e[k].u, e[k].alpha, e[k].f, e[k].h2, e[k].res}, 1.0f};
    r2[k] = RowsArgs{e[k].rhat, e[k].z, N, lg, Pr, m, twc, e[k].res, e[k].dot_part,
                     ResidualIn<float>{nullptr, nullptr, nullptr, 0.0f, nullptr}, 1.0f};
    cc[k] = ColsArgs{e[k].rhat, N, lg, Pc, twc, e[k].lam, e[k].h2 * float(4.0 / ((double)N * N))};
    sr = std::max(sr, fft_smem<float>(L, Pr));
    sc = std::max(sc, fft_smem<float>(L, Pc));
  }
  GramGroup* g = new GramGroup();
  cudaError_t err = dev_group_create(g->rows0, r0.data(), gr.data(), n);
  if (err == cudaSuccess) err = dev_group_create(g->rows2, r2.data(), gr.data(), n);
  if (err == cudaSuccess) err = dev_group_create(g->cols, cc.data(), gc.data(), n);
  if (err != cudaSuccess) {
    gram_group_destroy(g);
    return err;
  }
  g->smem_rows = sr;
  g->smem_cols = sc;
  *out = g;
  return cudaSuccess;
}

cudaError_t launch_gram_group(const GramGroup* g, int pass, cudaStream_t st) {
  if (pass == 1) {
    auto k = k_gram_cols_grp;
    smem_optin(k);
    if (g->cols.nctas > 0) k<<<g->cols.nctas, kFftThreads, g->smem_cols, st>>>(g->cols.tab, g->cols.map);
  } else {
    auto k = k_dst_rows_grp;
    smem_optin(k);
    const DevGroup<RowsArgs>& d = pass == 0 ? g->rows0 : g->rows2;
    if (d.nctas > 0) k<<<d.nctas, kFftThreads, g->smem_rows, st>>>(d.tab, d.map);
  }
  return cudaGetLastError();
}

template cudaError_t gram_fft_tables<float>(int, float*, float*);
template cudaError_t launch_gram_fft3d<float>(int, int, const float*, float*, float*, const float*, float,
                                              double*, cudaStream_t);
template cudaError_t launch_gram_fft3d<double>(int, int, const double*, double*, double*, const double*,
                                               double, double*, cudaStream_t);
template cudaError_t gram_fft_tables<double>(int, double*, double*);
template cudaError_t launch_gram_fft<float>(int, int, const float*, float*, float*, const float*,
                                            const float*, float, double*, cudaStream_t, const float*,
                                            const float*, const float*, float*);
template cudaError_t launch_gram_fft<double>(int, int, const double*, double*, double*,
                                             const double*, const double*, double, double*,
                                             cudaStream_t, const double*, const double*,
                                             const double*, double*);

}  // namespace adsgb

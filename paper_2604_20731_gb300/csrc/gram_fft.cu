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
#include <cuda_runtime.h>

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

// D along x for rows [r0, r0 + 2P) of `in` into `out` (rows 2p and 2p + 1 of
// the CTA share line p).  With rin.u set, the rows are first computed as
// RES = A u + h^2 f and written to rin.res.  With dotw != nullptr, also a
// partial of sum dotw * out over the CTA's rows.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    k_dst_rows(const T* __restrict__ in, T* __restrict__ out, int N, int lg, int P,
               const Cx<T>* __restrict__ tw, const T* __restrict__ dotw, double* dot_part,
               ResidualIn<T> rin) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1;
  Cx<T>* tws = reinterpret_cast<Cx<T>*>(fsm);  // [L]
  Cx<T>* buf0 = tws + L;                       // [P][L]
  Cx<T>* buf1 = buf0 + (size_t)P * L;          // [P][L]
  __shared__ double red[32];
  const int r0 = blockIdx.x * 2 * P;
  for (int q = threadIdx.x; q < L; q += blockDim.x) tws[q] = tw[q];
  const T* src = in;
  int sstride = m;  // row stride of the source rows
  size_t soff = (size_t)r0 * m;
  if (rin.u) {
    // the CTA's residual rows, staged in the second buffer ([2P][m] reals)
    T* stage = reinterpret_cast<T*>(buf1);
    for (int idx = threadIdx.x; idx < 2 * P * m; idx += blockDim.x) {
      const int rr = idx / m, ii = idx - rr * m;
      const int row = r0 + rr;
      T v = T(0);
      if (row < m) {
        v = residual_at(rin, N, row, ii);
        rin.res[(size_t)row * m + ii] = v;
      }
      stage[idx] = v;
    }
    __syncthreads();
    src = stage;
    soff = 0;
  }
  for (int idx = threadIdx.x; idx < P * L; idx += blockDim.x) {
    const int line = idx >> lg, j = idx & (L - 1);
    const int ra = r0 + 2 * line, rb = ra + 1;
    const T va = ra < m ? odd_ext(src + soff + (size_t)(2 * line) * sstride, j, N, 1) : T(0);
    const T vb = rb < m ? odd_ext(src + soff + (size_t)(2 * line + 1) * sstride, j, N, 1) : T(0);
    buf0[idx] = Cx<T>{va, vb};
  }
  __syncthreads();
  const Cx<T>* z = fft_stockham(buf0, buf1, P, lg, tws);
  CompSum<T> dot;
  for (int idx = threadIdx.x; idx < 2 * P * m; idx += blockDim.x) {
    const int rr = idx / m, k = idx - rr * m + 1;
    const int row = r0 + rr;
    if (row < m) {
      const Cx<T> zk = z[((rr >> 1) << lg) + k];
      const T v = (rr & 1) ? T(0.5) * zk.re : T(-0.5) * zk.im;
      out[(size_t)row * m + k - 1] = v;
      if (dotw) dot.add(v * dotw[(size_t)row * m + k - 1]);
    }
  }
  if (dotw) {
    const double tot = block_sum(dot.value(), red);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = tot;
  }
}

// For x-modes i in [c0, c0 + 2P): D along y, times scale / (lam_i + lam_j),
// D along y again; in place.  Columns 2p and 2p + 1 of the CTA share line p.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    k_gram_cols(T* __restrict__ data, int N, int lg, int P, const Cx<T>* __restrict__ tw,
                const T* __restrict__ lam, T scale) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1, C = 2 * P;
  Cx<T>* tws = reinterpret_cast<Cx<T>*>(fsm);  // [L]
  Cx<T>* buf0 = tws + L;                       // [P][L]
  Cx<T>* buf1 = buf0 + (size_t)P * L;          // [P][L]
  const int c0 = blockIdx.x * C;
  for (int q = threadIdx.x; q < L; q += blockDim.x) tws[q] = tw[q];
  // column c of the CTA fastest: a warp reads C neighbouring values of rows
  for (int idx = threadIdx.x; idx < C * L; idx += blockDim.x) {
    const int c = idx % C, j = idx / C;
    const int col = c0 + c;
    const T v = col < m ? odd_ext(data + col, j, N, m) : T(0);
    T* slot = reinterpret_cast<T*>(buf0 + ((c >> 1) << lg) + j);
    slot[c & 1] = v;
  }
  __syncthreads();
  Cx<T>* z = fft_stockham(buf0, buf1, P, lg, tws);
  T* vt = reinterpret_cast<T*>(z == buf0 ? buf1 : buf0);  // [C][N] scaled transforms
  for (int idx = threadIdx.x; idx < C * m; idx += blockDim.x) {
    const int c = idx / m, k = idx - c * m + 1;
    const int col = c0 + c;
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

}  // namespace

bool gram_fft_supported(int dim, int N) {
  const int lg = log2_exact(N);
  return dim == 2 && lg >= 3 && lg <= 11;  // L = 2N <= 4096
}

int gram_fft_dot_parts(int N) {
  const int m = N - 1, P = lines_per_cta<double>(2 * N, 1);  // the row kernel's grid (FP64 bound)
  const int Pf = lines_per_cta<float>(2 * N, 1);
  const int g = (m + 2 * P - 1) / (2 * P), gf = (m + 2 * Pf - 1) / (2 * Pf);
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
      k<<<g, kFftThreads, smem, st>>>(res, work, N, lg, P, twc, nullptr, nullptr, rin);
    } else {
      k<<<g, kFftThreads, smem, st>>>(work, z, N, lg, P, twc, res, dot_part, rin);
    }
  }
  return cudaGetLastError();
}

template cudaError_t gram_fft_tables<float>(int, float*, float*);
template cudaError_t gram_fft_tables<double>(int, double*, double*);
template cudaError_t launch_gram_fft<float>(int, int, const float*, float*, float*, const float*,
                                            const float*, float, double*, cudaStream_t, const float*,
                                            const float*, const float*, float*);
template cudaError_t launch_gram_fft<double>(int, int, const double*, double*, double*,
                                             const double*, const double*, double, double*,
                                             cudaStream_t, const double*, const double*,
                                             const double*, double*);

}  // namespace adsgb

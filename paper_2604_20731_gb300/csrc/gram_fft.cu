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
// Y_k = -2i (D x)_k, so (D x)_k = -Im(Y_k) / 2.
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

// Radix-2 decimation-in-time FFT, in place, of nl lines of length L = 2^lg
// held one after another in shared memory, input in bit-reversed order.
// Twiddles tw[k] = exp(-2 pi i k / L), k < L / 2.
template <typename T>
__device__ __forceinline__ void fft_lines(Cx<T>* buf, int nl, int lg, const Cx<T>* tw) {
  const int hl = 1 << (lg - 1);  // butterflies per line and stage
  const int nbf = nl * hl;
  for (int s = 0; s < lg; ++s) {
    const int half = 1 << s;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
      const int line = b >> (lg - 1), bl = b & (hl - 1);
      const int pos = bl & (half - 1), grp = bl >> s;
      const int i0 = (line << lg) + (grp << (s + 1)) + pos, i1 = i0 + half;
      const Cx<T> w = tw[pos << (lg - 1 - s)];
      const Cx<T> a = buf[i0], c = buf[i1];
      const T cr = c.re * w.re - c.im * w.im, ci = c.re * w.im + c.im * w.re;
      buf[i0] = Cx<T>{a.re + cr, a.im + ci};
      buf[i1] = Cx<T>{a.re - cr, a.im - ci};
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int j, int lg) { return (int)(__brev((unsigned)j) >> (32 - lg)); }

// value j of the odd extension (length 2N) of x_1..x_{N-1} = v[0..N-2]
template <typename T>
__device__ __forceinline__ T odd_ext(const T* v, int j, int N, int stride) {
  if (j > 0 && j < N) return v[(size_t)(j - 1) * stride];
  if (j > N) return -v[(size_t)(2 * N - j - 1) * stride];
  return T(0);
}

// D along x for rows [r0, r0 + rpc) of `in` into `out`, times `scale`.  With
// dotw != nullptr, also a partial of sum dotw * out over the CTA's rows.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    k_dst_rows(const T* __restrict__ in, T* __restrict__ out, int N, int lg, int rpc,
               const Cx<T>* __restrict__ tw, T scale, const T* __restrict__ dotw, double* dot_part) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1;
  Cx<T>* buf = reinterpret_cast<Cx<T>*>(fsm);  // [rpc][L]
  Cx<T>* tws = buf + (size_t)rpc * L;         // [L / 2]
  __shared__ double red[32];
  const int r0 = blockIdx.x * rpc;
  for (int k = threadIdx.x; k < L / 2; k += blockDim.x) tws[k] = tw[k];
  for (int idx = threadIdx.x; idx < rpc * L; idx += blockDim.x) {
    const int line = idx >> lg, j = idx & (L - 1);
    const int row = r0 + line;
    const T v = row < m ? odd_ext(in + (size_t)row * m, j, N, 1) : T(0);
    buf[(line << lg) + bitrev(j, lg)] = Cx<T>{v, T(0)};
  }
  __syncthreads();
  fft_lines(buf, rpc, lg, tws);
  CompSum<T> dot;
  for (int idx = threadIdx.x; idx < rpc * m; idx += blockDim.x) {
    const int line = idx / m, k = idx - line * m + 1;
    const int row = r0 + line;
    if (row < m) {
      const T v = T(-0.5) * buf[(line << lg) + k].im * scale;
      out[(size_t)row * m + k - 1] = v;
      if (dotw) dot.add(v * dotw[(size_t)row * m + k - 1]);
    }
  }
  if (dotw) {
    const double tot = block_sum(dot.value(), red);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = tot;
  }
}

// For x-modes i in [c0, c0 + cb): D along y, times scale / (lam_i + lam_j),
// D along y again; in place.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
    k_gram_cols(T* __restrict__ data, int N, int lg, int cb, const Cx<T>* __restrict__ tw,
                const T* __restrict__ lam, T scale) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int L = 1 << lg, m = N - 1;
  Cx<T>* buf = reinterpret_cast<Cx<T>*>(fsm);  // [cb][L]
  Cx<T>* tws = buf + (size_t)cb * L;          // [L / 2]
  T* vt = reinterpret_cast<T*>(tws + L / 2);  // [cb][N]: transformed, scaled columns
  const int c0 = blockIdx.x * cb;
  for (int k = threadIdx.x; k < L / 2; k += blockDim.x) tws[k] = tw[k];
  // column c fastest: a warp reads cb neighbouring values of several rows
  for (int idx = threadIdx.x; idx < cb * L; idx += blockDim.x) {
    const int c = idx % cb, j = idx / cb;
    const int col = c0 + c;
    const T v = col < m ? odd_ext(data + col, j, N, m) : T(0);
    buf[c * L + bitrev(j, lg)] = Cx<T>{v, T(0)};
  }
  __syncthreads();
  fft_lines(buf, cb, lg, tws);
  for (int idx = threadIdx.x; idx < cb * m; idx += blockDim.x) {
    const int c = idx / m, k = idx - c * m + 1;
    const int col = c0 + c;
    const T li = col < m ? lam[col] : T(1);
    vt[c * N + k - 1] = T(-0.5) * buf[c * L + k].im * (scale / (li + lam[k - 1]));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < cb * L; idx += blockDim.x) {
    const int c = idx >> lg, j = idx & (L - 1);
    buf[c * L + bitrev(j, lg)] = Cx<T>{odd_ext(vt + c * N, j, N, 1), T(0)};
  }
  __syncthreads();
  fft_lines(buf, cb, lg, tws);
  for (int idx = threadIdx.x; idx < cb * m; idx += blockDim.x) {
    const int c = idx % cb, k = idx / cb + 1;
    const int col = c0 + c;
    if (col < m) data[(size_t)(k - 1) * m + col] = T(-0.5) * buf[c * L + k].im;
  }
}

int log2_exact(int N) {
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  return (1 << lg) == N ? lg : -1;
}

int rows_per_cta(int L) { return L >= 2 * kFftThreads ? 1 : (2 * kFftThreads) / L; }

template <typename T>
size_t rows_smem(int L) {
  return ((size_t)rows_per_cta(L) * L + L / 2) * sizeof(Cx<T>);
}

// cb lines of L complex values, the twiddles and cb lines of N = L / 2 reals
template <typename T>
size_t cols_smem(int L, int cb) {
  return ((size_t)cb * L + L / 2) * sizeof(Cx<T>) + (size_t)cb * (L / 2) * sizeof(T);
}

// x-modes per CTA: enough CTAs to cover the SMs where the grid allows, 2..8
template <typename T>
int cols_per_cta(int L) {
  const int m = L / 2 - 1;
  int cb = 2;
  while (cb < 8 && m / (2 * cb) >= 152) cb *= 2;
  while (cb > 1 && cols_smem<T>(L, cb) > 200 * 1024) cb /= 2;
  return cb;
}

}  // namespace

bool gram_fft_supported(int dim, int N) {
  const int lg = log2_exact(N);
  return dim == 2 && lg >= 3 && lg <= 11;  // L = 2N <= 4096
}

int gram_fft_dot_parts(int N) {
  const int m = N - 1, rpc = rows_per_cta(2 * N);
  return (m + rpc - 1) / rpc;
}

template <typename T>
cudaError_t gram_fft_tables(int N, T* tw, T* lam) {
  const int L = 2 * N, m = N - 1;
  std::vector<T> h((size_t)L + m);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < L / 2; ++k) {
    h[2 * k] = (T)std::cos(2.0 * pi * k / L);
    h[2 * k + 1] = (T)(-std::sin(2.0 * pi * k / L));
  }
  for (int k = 1; k <= m; ++k) {
    const double s = std::sin(pi * k / (2.0 * N));
    h[L + k - 1] = (T)(4.0 * s * s);  // 2 - 2 cos(pi k / N)
  }
  cudaError_t e = cudaMemcpy(tw, h.data(), sizeof(T) * L, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(lam, h.data() + L, sizeof(T) * m, cudaMemcpyHostToDevice);
}

// pass 0: work = D_x res; pass 1: work <- h^2 (2/N)^2 D_y Lambda^-1 D_y work;
// pass 2: z = D_x work and the partials of res^T z
template <typename T>
cudaError_t launch_gram_fft(int pass, int N, const T* res, T* work, T* z, const T* tw, const T* lam,
                            T h2, double* dot_part, cudaStream_t st) {
  const int lg = log2_exact(N) + 1, L = 2 * N, m = N - 1;
  if (lg < 4 || lg > 12) return cudaErrorInvalidValue;
  const Cx<T>* twc = reinterpret_cast<const Cx<T>*>(tw);
  const int rpc = rows_per_cta(L), cb = cols_per_cta<T>(L);
  if (pass == 1) {
    const size_t smem = cols_smem<T>(L, cb);
    auto k = k_gram_cols<T>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const T s = h2 * T(4.0 / ((double)N * N));  // h^2 (2 / N)^2
    k<<<(m + cb - 1) / cb, kFftThreads, smem, st>>>(work, N, lg, cb, twc, lam, s);
  } else {
    const size_t smem = rows_smem<T>(L);
    auto k = k_dst_rows<T>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int g = (m + rpc - 1) / rpc;
    if (pass == 0) k<<<g, kFftThreads, smem, st>>>(res, work, N, lg, rpc, twc, T(1), nullptr, nullptr);
    else k<<<g, kFftThreads, smem, st>>>(work, z, N, lg, rpc, twc, T(1), res, dot_part);
  }
  return cudaGetLastError();
}

template cudaError_t gram_fft_tables<float>(int, float*, float*);
template cudaError_t gram_fft_tables<double>(int, double*, double*);
template cudaError_t launch_gram_fft<float>(int, int, const float*, float*, float*, const float*,
                                            const float*, float, double*, cudaStream_t);
template cudaError_t launch_gram_fft<double>(int, int, const double*, double*, double*,
                                             const double*, const double*, double, double*,
                                             cudaStream_t);

}  // namespace adsgb

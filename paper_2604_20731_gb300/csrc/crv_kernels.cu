// CRVPINN pressure kernels (Sec. 5 of the paper): nodal coefficients
// (Eq. 23b), the residual stencil (Eqs. 24-25) and its adjoint, the Gram
// matrix inverse (Eqs. 26-28) applied by fast diagonalisation, and the loss.
//
// G = h^-2 (I (x) T + T (x) I), T = tridiag(-1, 2, -1) = S Lambda S with the
// orthonormal sine matrix S_ik = sqrt(2/N) sin(pi i k / N).  Hence
//   G^-1 r = h^2 (I (x) S) (T (x) I + I (x) Lambda)^-1 (I (x) S) r:
// a sine transform along x (a dense (N-1)^2 GEMM), one shifted tridiagonal
// solve (Lambda_k + T) along y per mode k, and the inverse transform.  The
// paper's "LU once, substitutions per iteration" (Eq. 28) becomes: the
// shifted tridiagonal LU factors are computed once (FP64), the substitutions
// run every iteration.
#include <cuda_runtime.h>
#include <math.h>

#include "kernels.cuh"

namespace adsgb {

// ---------------------------------------------------------------------------
// nodal coefficients alpha = lambda(S) K, f = D+ . (g K rho lambda) - q  (2D)
// ---------------------------------------------------------------------------
// Value of a quadratic C1 spline at knot i of an open uniform knot vector:
// c_0 at the left end, c_{n+1} at the right end, (c_i + c_{i+1})/2 inside.
__device__ __forceinline__ void knot_weights(int i, int n, int& i0, double& w0, double& w1) {
  if (i == 0) { i0 = 0; w0 = 1.0; w1 = 0.0; }
  else if (i == n) { i0 = n; w0 = 0.0; w1 = 1.0; }
  else { i0 = i; w0 = 0.5; w1 = 0.5; }
}

template <typename T, typename TA>
__device__ __forceinline__ double nodal_sat_2d(const CrvArgs<T, TA>& a, int j, int i) {
  const int n = a.N, nb = n + 2;
  int i0, j0;
  double wx0, wx1, wy0, wy1;
  knot_weights(i, n, i0, wx0, wx1);
  knot_weights(j, n, j0, wy0, wy1);
  const TA* r0 = a.S + (size_t)j0 * nb + i0;
  const TA* r1 = r0 + nb;
  double v = wy0 * (wx0 * (double)r0[0] + wx1 * (double)r0[1]) +
             wy1 * (wx0 * (double)r1[0] + wx1 * (double)r1[1]);
  return v;
}

template <typename T, typename TA>
__global__ void k_crv_coeffs_2d(CrvArgs<T, TA> a) {
  const int N = a.N, n1 = N + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n1 * n1) return;
  const int j = t / n1, i = t % n1;
  double s = nodal_sat_2d(a, j, i);
  s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
  double lw = (1.0 - s) * a.inv_mu_w, lg = s * a.inv_mu_g;
  double K = (double)a.K[(size_t)j * n1 + i];
  a.alpha[t] = (T)((lw + lg) * K);
  if (i >= 1 && i <= N - 1 && j >= 1 && j <= N - 1) {
    // forward difference along the vertical (y) of F = -g K (rho_w lw + rho_g lg)
    double s1 = nodal_sat_2d(a, j + 1, i);
    s1 = s1 < 0.0 ? 0.0 : (s1 > 1.0 ? 1.0 : s1);
    double K1 = (double)a.K[(size_t)(j + 1) * n1 + i];
    double F0 = -a.grav * K * (a.rho_w * lw + a.rho_g * lg);
    double F1 = -a.grav * K1 * (a.rho_w * (1.0 - s1) * a.inv_mu_w + a.rho_g * s1 * a.inv_mu_g);
    double q = 0.0;
    for (int k = 0; k < a.n_src; ++k) {
      double g = a.rate[k] * (double)a.ax.gnode[(size_t)(0 * kMaxSrc + k) * n1 + i] *
                 (double)a.ax.gnode[(size_t)(1 * kMaxSrc + k) * n1 + j];
      q += (a.kind[k] == 0) ? g : -g;
    }
    a.f[(size_t)(j - 1) * (N - 1) + (i - 1)] = (T)((F1 - F0) * (double)N - q);
  }
}

// 3D: nodal saturation from the three per-axis knot weights; the vertical
// axis is z and carries kz_ratio in the gravity flux
template <typename T, typename TA>
__device__ __forceinline__ double nodal_sat_3d(const CrvArgs<T, TA>& a, int k, int j, int i) {
  const int n = a.N, nb = n + 2;
  int i0, j0, k0;
  double wx[2], wy[2], wz[2];
  knot_weights(i, n, i0, wx[0], wx[1]);
  knot_weights(j, n, j0, wy[0], wy[1]);
  knot_weights(k, n, k0, wz[0], wz[1]);
  double v = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b) {
      const TA* r = a.S + ((size_t)(k0 + c) * nb + (j0 + b)) * nb + i0;
      v += wz[c] * wy[b] * (wx[0] * (double)r[0] + wx[1] * (double)r[1]);
    }
  return v;
}

template <typename T, typename TA>
__global__ void k_crv_coeffs_3d(CrvArgs<T, TA> a) {
  const int N = a.N, n1 = N + 1, m = N - 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n1 * n1 * n1) return;
  const int i = (int)(t % n1), j = (int)((t / n1) % n1), k = (int)(t / ((long long)n1 * n1));
  double s = nodal_sat_3d(a, k, j, i);
  s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
  double lw = (1.0 - s) * a.inv_mu_w, lg = s * a.inv_mu_g;
  double K = (double)a.K[t];
  a.alpha[t] = (T)((lw + lg) * K);
  if (i >= 1 && i <= N - 1 && j >= 1 && j <= N - 1 && k >= 1 && k <= N - 1) {
    double s1 = nodal_sat_3d(a, k + 1, j, i);
    s1 = s1 < 0.0 ? 0.0 : (s1 > 1.0 ? 1.0 : s1);
    double K1 = (double)a.K[t + (long long)n1 * n1];
    double F0 = -a.grav * a.kz * K * (a.rho_w * lw + a.rho_g * lg);
    double F1 = -a.grav * a.kz * K1 * (a.rho_w * (1.0 - s1) * a.inv_mu_w + a.rho_g * s1 * a.inv_mu_g);
    double q = 0.0;
    for (int c = 0; c < a.n_src; ++c) {
      double g = a.rate[c] * (double)a.ax.gnode[(size_t)(0 * kMaxSrc + c) * n1 + i] *
                 (double)a.ax.gnode[(size_t)(1 * kMaxSrc + c) * n1 + j] *
                 (double)a.ax.gnode[(size_t)(2 * kMaxSrc + c) * n1 + k];
      q += (a.kind[c] == 0) ? g : -g;
    }
    a.f[((size_t)(k - 1) * m + (j - 1)) * m + (i - 1)] = (T)((F1 - F0) * (double)N - q);
  }
}

template <typename T, typename TA>
cudaError_t launch_crv_coeffs(const CrvArgs<T, TA>& a, cudaStream_t st) {
  if (a.dim == 3) {
    long long tot = (long long)(a.N + 1) * (a.N + 1) * (a.N + 1);
    k_crv_coeffs_3d<T, TA><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
  }
  int tot = (a.N + 1) * (a.N + 1);
  k_crv_coeffs_2d<T, TA><<<(tot + 255) / 256, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// stencil: out_k = scale * sum_dir [alpha_{k-e}(v_k - v_{k-e}) - alpha_k(v_{k+e} - v_k)]
//                  + h2 * f_k  (f nullable), v = 0 on the boundary.
// RES = A u + h^2 f uses scale 1; the adjoint dL/du = 2 A z uses scale 2.
// ---------------------------------------------------------------------------
// Loss finalisation (sum of the per-CTA partials of RES . z in a fixed
// order), fused into the adjoint stencil's first thread: it also advances the
// Adam step counter, logs the loss and stores the bias corrections.
// warp 0 of block 0: lane sums of parts lane, lane + 32, ..., then a fixed
// shuffle tree (deterministic), lane 0 finishes
__device__ __forceinline__ void loss_finalize_dev(const LossFin& lf) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < lf.nparts; i += 32) s += lf.part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  *lf.loss = s;
  if (!isfinite(s)) lf.flags[0] |= 4;
  if (lf.bump) {
    int tt = *lf.t + 1;
    *lf.t = tt;
    lf.log[(tt - 1) % kLossRing] = s;
    // beta^t as running products (bc[2], bc[3]) instead of pow: FP64
    // transcendentals are slow on this GPU and this warp holds the grid open
    const double b1t = lf.bc[2] * 0.9, b2t = lf.bc[3] * 0.999;
    lf.bc[2] = b1t;
    lf.bc[3] = b2t;
    lf.bc[0] = 1.0 / (1.0 - b1t);
    lf.bc[1] = 1.0 / (1.0 - b2t);
  }
}

template <typename T>
__device__ __forceinline__ void stencil_2d_body(int N, const T* __restrict__ alpha, const T* __restrict__ v,
                                                const T* __restrict__ f, T h2, T scale, T* __restrict__ out,
                                                const LossFin& lf, int bid) {
  const int m = N - 1, n1 = N + 1;
  const int t = bid * blockDim.x + threadIdx.x;
  if (lf.part && t < 32) loss_finalize_dev(lf);
  if (t >= m * m) return;
  const int jj = t / m, ii = t % m;  // interior index
  const int j = jj + 1, i = ii + 1;  // node index
  T c = v[t];
  T w = ii > 0 ? v[t - 1] : T(0);
  T e = ii < m - 1 ? v[t + 1] : T(0);
  T s = jj > 0 ? v[t - m] : T(0);
  T nn = jj < m - 1 ? v[t + m] : T(0);
  T ac = alpha[(size_t)j * n1 + i];
  T aw = alpha[(size_t)j * n1 + i - 1];
  T as = alpha[(size_t)(j - 1) * n1 + i];
  T r = aw * (c - w) - ac * (e - c) + as * (c - s) - ac * (nn - c);
  r *= scale;
  if (f) r += h2 * f[t];
  out[t] = r;
}
template <typename T>
__global__ void __launch_bounds__(256) k_stencil_2d(int N, const T* __restrict__ alpha,
                                                    const T* __restrict__ v, const T* __restrict__ f,
                                                    T h2, T scale, T* __restrict__ out, LossFin lf) {
  stencil_2d_body<T>(N, alpha, v, f, h2, scale, out, lf, blockIdx.x);
}
// grouped (FP32): CTA g.cta[b].y of context g.cta[b].x's launch
__global__ void __launch_bounds__(256) k_stencil_2d_grp(const StencilArgs* __restrict__ tab, GroupMap g) {
  const int2 c = g.cta[blockIdx.x];
  const StencilArgs& a = tab[c.x];
  stencil_2d_body<float>(a.N, a.alpha, a.v, a.f, a.h2, a.scale, a.out, a.lf, c.y);
}

// 7-point form: the z differences are weighted by kz
template <typename T>
__global__ void __launch_bounds__(256) k_stencil_3d(int N, T kz, const T* __restrict__ alpha,
                                                    const T* __restrict__ v, const T* __restrict__ f,
                                                    T h2, T scale, T* __restrict__ out, LossFin lf) {
  const int m = N - 1, n1 = N + 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (lf.part && t < 32) loss_finalize_dev(lf);
  if (t >= (long long)m * m * m) return;
  const int ii = (int)(t % m), jj = (int)((t / m) % m), kk = (int)(t / ((long long)m * m));
  const int i = ii + 1, j = jj + 1, k = kk + 1;
  const long long mm = (long long)m * m;
  T c = v[t];
  T w = ii > 0 ? v[t - 1] : T(0);
  T e = ii < m - 1 ? v[t + 1] : T(0);
  T s = jj > 0 ? v[t - m] : T(0);
  T nn = jj < m - 1 ? v[t + m] : T(0);
  T d = kk > 0 ? v[t - mm] : T(0);
  T up = kk < m - 1 ? v[t + mm] : T(0);
  const size_t nd = ((size_t)k * n1 + j) * n1 + i;
  T ac = alpha[nd];
  T aw = alpha[nd - 1];
  T as = alpha[nd - n1];
  T ad = alpha[nd - (size_t)n1 * n1];
  T r = aw * (c - w) - ac * (e - c) + as * (c - s) - ac * (nn - c) + kz * (ad * (c - d) - ac * (up - c));
  r *= scale;
  if (f) r += h2 * f[t];
  out[t] = r;
}

template <typename T>
cudaError_t launch_stencil(int dim, int N, T kz, const T* alpha, const T* u, const T* f, T h2,
                           T scale, T* out, const LossFin* lf, cudaStream_t st) {
  LossFin none{};
  if (dim == 3) {
    long long m = (long long)(N - 1) * (N - 1) * (N - 1);
    if (m <= 0) return cudaSuccess;
    k_stencil_3d<T><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(N, kz, alpha, u, f, h2, scale, out,
                                                                  lf ? *lf : none);
    return cudaGetLastError();
  }
  int m = (N - 1) * (N - 1);
  if (m <= 0) return cudaSuccess;
  k_stencil_2d<T><<<(m + 255) / 256, 256, 0, st>>>(N, alpha, u, f, h2, scale, out, lf ? *lf : none);
  return cudaGetLastError();
}

int stencil_blocks(int N) { return ((N - 1) * (N - 1) + 255) / 256; }

cudaError_t launch_stencil_grouped(const StencilArgs* tab, GroupMap g, int nctas, cudaStream_t st) {
  if (nctas > 0) k_stencil_2d_grp<<<nctas, 256, 0, st>>>(tab, g);
  return cudaGetLastError();
}

template <typename T, typename TA>
__global__ void k_embed_2d(int N, const T* u, TA* nodal) {
  const int n1 = N + 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n1 * n1) return;
  const int j = t / n1, i = t % n1;
  TA v = TA(0);
  if (i >= 1 && i <= N - 1 && j >= 1 && j <= N - 1) v = (TA)u[(size_t)(j - 1) * (N - 1) + (i - 1)];
  nodal[t] = v;
}

template <typename T, typename TA>
__global__ void k_embed_3d(int N, const T* u, TA* nodal) {
  const int n1 = N + 1, m = N - 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n1 * n1 * n1) return;
  const int i = (int)(t % n1), j = (int)((t / n1) % n1), k = (int)(t / ((long long)n1 * n1));
  TA v = TA(0);
  if (i >= 1 && i <= N - 1 && j >= 1 && j <= N - 1 && k >= 1 && k <= N - 1)
    v = (TA)u[((size_t)(k - 1) * m + (j - 1)) * m + (i - 1)];
  nodal[t] = v;
}

template <typename T, typename TA>
cudaError_t launch_embed(int dim, int N, const T* u, TA* nodal, cudaStream_t st) {
  if (dim == 3) {
    long long tot = (long long)(N + 1) * (N + 1) * (N + 1);
    k_embed_3d<T, TA><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(N, u, nodal);
    return cudaGetLastError();
  }
  int tot = (N + 1) * (N + 1);
  k_embed_2d<T, TA><<<(tot + 255) / 256, 256, 0, st>>>(N, u, nodal);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gram tables (FP64, once): S (m x m), inverse pivots of (Lambda_k + T)
// stored [j][k] so that a thread per mode k reads coalesced rows.
// ---------------------------------------------------------------------------
__global__ void k_gram_sine(int N, double* S) {
  const int m = N - 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  const int i = t / m + 1, k = t % m + 1;
  long long ik = (long long)i * k % (2LL * N);  // sin(pi ik/N) is 2N-periodic in ik
  S[t] = sqrt(2.0 / N) * sinpi((double)ik / (double)N);
}

__global__ void k_gram_pivots(int N, double* invd) {
  const int m = N - 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  double sk = sinpi((double)(k + 1) / (2.0 * N));
  double b = 2.0 + 4.0 * sk * sk;
  double d = b;
  for (int j = 0; j < m; ++j) {
    invd[(size_t)j * m + k] = 1.0 / d;
    d = b - 1.0 / d;
  }
}

// 3D: for the z sweep of mode (ky, kx) the shift is Lambda_ky + Lambda_kx;
// pivots stored [z][ky*m + kx]
__global__ void k_gram_pivots3d(int N, double* invd) {
  const int m = N - 1;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m * m) return;
  const int ky = c / m + 1, kx = c % m + 1;
  double sy = sinpi((double)ky / (2.0 * N)), sx = sinpi((double)kx / (2.0 * N));
  double b = 2.0 + 4.0 * sy * sy + 4.0 * sx * sx;
  double d = b;
  for (int j = 0; j < m; ++j) {
    invd[(size_t)j * m * m + c] = 1.0 / d;
    d = b - 1.0 / d;
  }
}

cudaError_t launch_gram_init(int dim, int N, double* Sdst, double* invd, cudaStream_t st) {
  int m = N - 1;
  k_gram_sine<<<(m * m + 255) / 256, 256, 0, st>>>(N, Sdst);
  if (dim == 3) k_gram_pivots3d<<<(m * m + 127) / 128, 128, 0, st>>>(N, invd);
  else k_gram_pivots<<<(m + 127) / 128, 128, 0, st>>>(N, invd);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// C = alpha * A * B (row-major, M x K times K x Nn), BM x BN tiles, 4x4 outputs
// per thread, register-blocked SIMT (the sine transforms of the Gram inverse).
// With dotB != nullptr the epilogue also forms this tile's part of
// sum_ij C_ij dotB_ij (the loss RES^T z) in FP64.
// ---------------------------------------------------------------------------
template <typename T, int BM, int BN>
__global__ void __launch_bounds__((BM / 4) * (BN / 4)) k_gemm(int M, int Nn, int K,
    const T* __restrict__ A, int lda, const T* __restrict__ B, int ldb, T* __restrict__ C, int ldc,
    T alpha, const T* __restrict__ dotB, double* dot_part, long long sA, long long sB, long long sC) {
  constexpr int BK = 16, NT = (BM / 4) * (BN / 4), TX = BN / 4;
  A += sA * blockIdx.z;
  B += sB * blockIdx.z;
  C += sC * blockIdx.z;
  constexpr int LA = BM * BK / NT, LB = BK * BN / NT;  // loads per thread per k-tile
  __shared__ T As[2][BK][BM + 4];
  __shared__ T Bs[2][BK][BN + 4];
  __shared__ double red[32];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  T ra[LA], rb[LB];
  // the next k-tile is loaded into registers while the current one is used
  auto gload = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      int e = tid + r * NT, mm = e / BK, kk = e % BK;
      int gm = m0 + mm, gk = k0 + kk;
      ra[r] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : T(0);
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      int e = tid + r * NT, kk = e / BN, nn = e % BN;
      int gk = k0 + kk, gn = n0 + nn;
      rb[r] = (gk < K && gn < Nn) ? B[(size_t)gk * ldb + gn] : T(0);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      int e = tid + r * NT, mm = e / BK, kk = e % BK;
      As[buf][kk][mm] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      int e = tid + r * NT, kk = e / BN, nn = e % BN;
      Bs[buf][kk][nn] = rb[r];
    }
  };
  T acc[4][4] = {};
  const int nk = (K + BK - 1) / BK;
  gload(0);
  sstore(0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) gload((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a4[4], b4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a4[i] = As[buf][kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b4[j] = Bs[buf][kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a4[i] * b4[j];
    }
    if (t + 1 < nk) sstore(buf ^ 1);
    __syncthreads();
  }
  double dsum = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx * 4 + j;
      if (gn < Nn) {
        T v = alpha * acc[i][j];
        C[(size_t)gm * ldc + gn] = v;
        if (dotB) dsum += (double)v * (double)dotB[(size_t)gm * ldc + gn];
      }
    }
  }
  if (dotB) {
    double tot = block_sum(dsum, red);
    if (tid == 0) dot_part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

static bool small_tiles(int M, int Nn) {
  return ((M + 63) / 64) * ((Nn + 63) / 64) < 304;
}

int gemm_blocks(int M, int Nn) {
  if (small_tiles(M, Nn)) return ((M + 31) / 32) * ((Nn + 31) / 32);
  return ((M + 63) / 64) * ((Nn + 63) / 64);
}

template <typename T>
cudaError_t launch_gemm(int M, int Nn, int K, const T* A, int lda, const T* B, int ldb, T* C,
                        int ldc, T alpha, const T* dotB, double* dot_part, cudaStream_t st,
                        int batch, long long sA, long long sB, long long sC) {
  if (batch > 1 && dotB) return cudaErrorInvalidValue;
  if (small_tiles(M, Nn) && batch == 1) {
    dim3 grid((Nn + 31) / 32, (M + 31) / 32, 1);
    k_gemm<T, 32, 32><<<grid, 64, 0, st>>>(M, Nn, K, A, lda, B, ldb, C, ldc, alpha, dotB, dot_part,
                                           sA, sB, sC);
  } else {
    dim3 grid((Nn + 63) / 64, (M + 63) / 64, batch);
    k_gemm<T, 64, 64><<<grid, 256, 0, st>>>(M, Nn, K, A, lda, B, ldb, C, ldc, alpha, dotB, dot_part,
                                            sA, sB, sC);
  }
  return cudaGetLastError();
}

// (Lambda_k + T) x = r along rows j for every column k, forward elimination
// then back substitution with the precomputed inverse pivots.  A CTA stages
// a block of CW columns (all rows, and their pivots) in shared memory with
// coalesced loads; one thread per column then runs the two sweeps there.
template <typename T>
__global__ void __launch_bounds__(256) k_tridiag_smem(int m, int ncols, int cw,
                                                      const T* __restrict__ invd, T* X) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);  // [m][cw]
  T* cs = xs + (size_t)m * cw;          // [m][cw]
  const int k0 = blockIdx.x * cw;
  const int ncw = min(cw, ncols - k0);
  for (int e = threadIdx.x; e < m * cw; e += blockDim.x) {
    int j = e / cw, kk = e % cw;
    if (kk < ncw) {
      cp_async_elem(&xs[e], &X[(size_t)j * ncols + k0 + kk]);
      cp_async_elem(&cs[e], &invd[(size_t)j * ncols + k0 + kk]);
    }
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  const int kk = threadIdx.x;
  if (kk < ncw) {
    T y = xs[kk];
    int j = 1;
    for (; j + 4 <= m; j += 4) {
      T x0 = xs[(j + 0) * cw + kk], x1 = xs[(j + 1) * cw + kk];
      T x2 = xs[(j + 2) * cw + kk], x3 = xs[(j + 3) * cw + kk];
      T c0 = cs[(j - 1) * cw + kk], c1 = cs[(j + 0) * cw + kk];
      T c2 = cs[(j + 1) * cw + kk], c3 = cs[(j + 2) * cw + kk];
      y = x0 + y * c0; xs[(j + 0) * cw + kk] = y;
      y = x1 + y * c1; xs[(j + 1) * cw + kk] = y;
      y = x2 + y * c2; xs[(j + 2) * cw + kk] = y;
      y = x3 + y * c3; xs[(j + 3) * cw + kk] = y;
    }
    for (; j < m; ++j) {
      y = xs[j * cw + kk] + y * cs[(j - 1) * cw + kk];
      xs[j * cw + kk] = y;
    }
    T x = xs[(m - 1) * cw + kk] * cs[(m - 1) * cw + kk];
    xs[(m - 1) * cw + kk] = x;
    j = m - 2;
    for (; j - 3 >= 0; j -= 4) {
      T y0 = xs[(j - 0) * cw + kk], y1 = xs[(j - 1) * cw + kk];
      T y2 = xs[(j - 2) * cw + kk], y3 = xs[(j - 3) * cw + kk];
      T c0 = cs[(j - 0) * cw + kk], c1 = cs[(j - 1) * cw + kk];
      T c2 = cs[(j - 2) * cw + kk], c3 = cs[(j - 3) * cw + kk];
      x = (y0 + x) * c0; xs[(j - 0) * cw + kk] = x;
      x = (y1 + x) * c1; xs[(j - 1) * cw + kk] = x;
      x = (y2 + x) * c2; xs[(j - 2) * cw + kk] = x;
      x = (y3 + x) * c3; xs[(j - 3) * cw + kk] = x;
    }
    for (; j >= 0; --j) {
      x = (xs[j * cw + kk] + x) * cs[j * cw + kk];
      xs[j * cw + kk] = x;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * cw; e += blockDim.x) {
    int j = e / cw, c = e % cw;
    if (c < ncw) X[(size_t)j * ncols + k0 + c] = xs[e];
  }
}

template <typename T>
cudaError_t launch_tridiag_cols(int nrows, int ncols, const T* invd, T* X, cudaStream_t st) {
  // columns per CTA: as many as fit 200 KB of shared memory, at most 32
  int cw = 32;
  while (cw > 1 && (size_t)2 * nrows * cw * sizeof(T) > 200 * 1024) cw /= 2;
  size_t smem = (size_t)2 * nrows * cw * sizeof(T);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  auto k = k_tridiag_smem<T>;
  smem_optin(k);
  k<<<(ncols + cw - 1) / cw, 256, smem, st>>>(nrows, ncols, cw, invd, X);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// loss = r . z (FP64 accumulation, fixed-order two-stage reduction)
// ---------------------------------------------------------------------------
int dot_blocks(int n) {
  int b = (n + 2047) / 2048;
  return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

template <typename T>
__global__ void __launch_bounds__(256) k_dot_partial(const T* a, const T* b, int n, double* part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  double tot = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename T>
cudaError_t launch_dot_partial(const T* a, const T* b, int n, double* part, int nblk,
                               cudaStream_t st) {
  k_dot_partial<T><<<nblk, 256, 0, st>>>(a, b, n, part);
  return cudaGetLastError();
}

__global__ void k_loss_finalize(const double* part, int nblk, double* loss, double* log, int* t,
                                double* bc, int* flags, int bump) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[i];
  *loss = s;
  if (!isfinite(s)) flags[0] |= 4;
  if (bump) {
    int tt = *t + 1;
    *t = tt;
    log[(tt - 1) % kLossRing] = s;
    const double b1t = bc[2] * 0.9, b2t = bc[3] * 0.999;
    bc[2] = b1t;
    bc[3] = b2t;
    bc[0] = 1.0 / (1.0 - b1t);
    bc[1] = 1.0 / (1.0 - b2t);
  }
}

// Adam's step counter and bias-correction state: t = 0, beta_1^t = beta_2^t = 1
__global__ void k_adam_reset(int* t, double* bc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *t = 0;
    bc[0] = bc[1] = 0.0;
    bc[2] = bc[3] = 1.0;
  }
}

cudaError_t launch_adam_reset(int* t, double* bc, cudaStream_t st) {
  k_adam_reset<<<1, 32, 0, st>>>(t, bc);
  return cudaGetLastError();
}

cudaError_t launch_loss_finalize(const double* part, int nblk, double* loss, double* loss_log,
                                 int* t, double* bc, int* flags, int bump_t, cudaStream_t st) {
  k_loss_finalize<<<1, 32, 0, st>>>(part, nblk, loss, loss_log, t, bc, flags, bump_t);
  return cudaGetLastError();
}

#define CRV_INST(T, TA)                                                                          \
  template cudaError_t launch_crv_coeffs<T, TA>(const CrvArgs<T, TA>&, cudaStream_t);            \
  template cudaError_t launch_embed<T, TA>(int, int, const T*, TA*, cudaStream_t);
CRV_INST(double, double)
CRV_INST(float, double)
CRV_INST(float, float)
CRV_INST(double, float)

#define CRV_INST1(T)                                                                              \
  template cudaError_t launch_stencil<T>(int, int, T, const T*, const T*, const T*, T, T, T*,    \
                                         const LossFin*, cudaStream_t);                           \
  template cudaError_t launch_gemm<T>(int, int, int, const T*, int, const T*, int, T*, int, T,   \
                                      const T*, double*, cudaStream_t, int, long long, long long, \
                                      long long);                                                 \
  template cudaError_t launch_tridiag_cols<T>(int, int, const T*, T*, cudaStream_t);             \
  template cudaError_t launch_dot_partial<T>(const T*, const T*, int, double*, int, cudaStream_t);
CRV_INST1(double)
CRV_INST1(float)

}  // namespace adsgb

// Galerkin B-spline pressure: the plain method of Sec. 7 (IGA-ADS with a
// direct solver for the pressure), 2D, FP64.
//
// The system is the weak form Eq. 12a in the B-spline space of Sec. 4
// (Eqs. 15-20, with the divergence of the scalar basis functions read as
// their gradient and the source taken with the sign of Eq. 12a):
//
//   sum_kl p_kl (lambda K grad B_kl, grad B_ij)
//       = (q_w + q_g, B_ij) - (g K (rho_w lambda_w + rho_g lambda_g), d B_ij / d y)
//
// for every interior B_ij, with p = 0 on the boundary (Sec. 8.1: the first and
// last basis function of each axis removed).  lambda = lambda_w + lambda_g of
// the clamped saturation, K the bilinear nodal map, both at the 3 x 3 Gauss
// points of each element; g points down the vertical (array axis 0) axis.
//
// Four kernels:
//   k_gal_gauss_2d     one thread per element: lambda K, source and gravity
//                      weights at its 9 Gauss points;
//   k_gal_assemble_2d  one thread per entry of the lower band of the
//                      stiffness matrix (unknowns in row-major (y, x) order,
//                      half bandwidth 2n + 2) and of the load vector, each
//                      summed over the elements both functions share -- no
//                      atomics, the order of the sums is fixed;
//   k_band_chol        one CTA: right-looking banded Cholesky L L^T in place;
//                      for n <= 78 the (2n+3)-row window of active rows lives
//                      in shared memory and each finished row is written out;
//   k_band_solve       one CTA: L y = F and L^T x = y by column sweeps, then x
//                      scattered into the (n+2)^2 coefficients (boundary 0).
// A pivot that is not positive and finite (non-finite or unphysical input)
// sets bit 0 of the context flags and the coefficients to NaN.
#include "kernels.cuh"

#include <math.h>

namespace adsgb {
namespace {

constexpr int kCholThreads = 1024;
constexpr int kSolveThreads = 1024;
constexpr size_t kSmemBudget = 200 * 1024;

template <typename TA>
__global__ void __launch_bounds__(128) k_gal_gauss_2d(GalArgs<TA> a, double* coef, double* r0,
                                                      double* r1) {
  const int n = a.n, nb = n + 2, n1 = n + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int ex = e % n, ey = e / n;
  const double* Bx = a.B + ex * 9;
  const double* By = a.B + ey * 9;
  const double h2 = 1.0 / ((double)n * (double)n);
  // S along x at the Gauss abscissae, for the element's three rows of coefficients
  double sx[3][3];
  for (int b = 0; b < 3; ++b) {
    const TA* row = a.S + (size_t)(ey + b) * nb + ex;
    for (int q = 0; q < 3; ++q)
      sx[b][q] = (double)row[0] * Bx[q] + (double)row[1] * Bx[3 + q] + (double)row[2] * Bx[6 + q];
  }
  const TA* Kr = a.K + (size_t)ey * n1 + ex;
  const double k00 = (double)Kr[0], k01 = (double)Kr[1], k10 = (double)Kr[n1], k11 = (double)Kr[n1 + 1];
  for (int qy = 0; qy < 3; ++qy) {
    const double eta = gauss_x(qy);
    for (int qx = 0; qx < 3; ++qx) {
      const double xi = gauss_x(qx);
      const double sv = By[qy] * sx[0][qx] + By[3 + qy] * sx[1][qx] + By[6 + qy] * sx[2][qx];
      const double st = sv < 0.0 ? 0.0 : (sv > 1.0 ? 1.0 : sv);
      const double lg = st * a.inv_mu_g, lw = (1.0 - st) * a.inv_mu_w;
      const double kq = (1.0 - eta) * ((1.0 - xi) * k00 + xi * k01) + eta * ((1.0 - xi) * k10 + xi * k11);
      double qt = 0.0;
      for (int s = 0; s < a.n_src; ++s) {
        const double g = a.rate[s] * a.gsrc[((size_t)(0 * kMaxSrc + s) * n + ex) * 3 + qx] *
                         a.gsrc[((size_t)(1 * kMaxSrc + s) * n + ey) * 3 + qy];
        qt += a.kind[s] == 0 ? g : -g;
      }
      const double w = gauss_w(qx) * gauss_w(qy) * h2;
      const size_t i = (size_t)e * 9 + qy * 3 + qx;
      coef[i] = w * (lg + lw) * kq;
      r0[i] = w * qt;
      r1[i] = -w * a.grav * kq * (lw * a.rho_w + lg * a.rho_g);
    }
  }
}

// A[u][u-j] (j = 0..2n+2) and F[u] for the interior unknown u = (iy-1) n + (ix-1)
__global__ void __launch_bounds__(256) k_gal_assemble_2d(int n, const double* B, const double* dB,
                                                         const double* coef, const double* r0,
                                                         const double* r1, double* L, double* F) {
  const int ld = 2 * n + 3;
  const long long total = (long long)n * n * ld;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int u = (int)(t / ld), j = (int)(t % ld);
    const int iy = u / n + 1, ix = u % n + 1;
    double val = 0.0;
    const int v = u - j;
    if (v >= 0) {
      const int ky = v / n + 1, kx = v % n + 1;
      if (abs(ix - kx) <= 2 && abs(iy - ky) <= 2) {
        // elements in both supports: ex in [max(ix, kx) - 2, min(ix, kx)] within [0, n)
        const int ex0 = max(max(ix, kx) - 2, 0), ex1 = min(min(ix, kx), n - 1);
        const int ey0 = max(max(iy, ky) - 2, 0), ey1 = min(min(iy, ky), n - 1);
        for (int ey = ey0; ey <= ey1; ++ey) {
          const double* By = B + ey * 9;
          const double* dBy = dB + ey * 9;
          const int bi = iy - ey, bk = ky - ey;
          for (int ex = ex0; ex <= ex1; ++ex) {
            const double* Bx = B + ex * 9;
            const double* dBx = dB + ex * 9;
            const int ai = ix - ex, ak = kx - ex;
            const double* c = coef + (size_t)(ey * n + ex) * 9;
            for (int qy = 0; qy < 3; ++qy) {
              const double yy = By[bi * 3 + qy] * By[bk * 3 + qy];
              const double dyy = dBy[bi * 3 + qy] * dBy[bk * 3 + qy];
              for (int qx = 0; qx < 3; ++qx)
                val += c[qy * 3 + qx] * (dBx[ai * 3 + qx] * dBx[ak * 3 + qx] * yy +
                                         Bx[ai * 3 + qx] * Bx[ak * 3 + qx] * dyy);
            }
          }
        }
      }
    }
    L[t] = val;
    if (j == 0) {
      double f = 0.0;
      for (int ey = max(iy - 2, 0); ey <= min(iy, n - 1); ++ey) {
        const double* By = B + ey * 9;
        const double* dBy = dB + ey * 9;
        const int bi = iy - ey;
        for (int ex = max(ix - 2, 0); ex <= min(ix, n - 1); ++ex) {
          const double* Bx = B + ex * 9;
          const int ai = ix - ex;
          const size_t e9 = (size_t)(ey * n + ex) * 9;
          for (int qy = 0; qy < 3; ++qy)
            for (int qx = 0; qx < 3; ++qx) {
              const size_t i = e9 + qy * 3 + qx;
              f += Bx[ai * 3 + qx] * (r0[i] * By[bi * 3 + qy] + r1[i] * dBy[bi * 3 + qy]);
            }
        }
      }
      F[u] = f;
    }
  }
}

// 1 / sqrt(d) of a pivot; a pivot that is not positive and finite sets *fail
// and is replaced by 1 so that the sweep still ends
__device__ __forceinline__ double pivot_rsqrt(double d, int* fail) {
  const double s = sqrt(d);
  if (!(d > 0.0) || !isfinite(s)) {
    *fail = 1;
    return 1.0;
  }
  return 1.0 / s;
}

// In-place banded Cholesky A = L L^T of the N x N matrix whose lower band row
// r is L[r * ld + j] = A[r][r - j], j = 0..ld-1; on return the diagonal slot
// L[r * ld] holds 1 / L_rr, the other slots the factor.  win: shared-memory
// window of ld rows (row r in slot r % ld) or not used.  FP64 runs at a small
// fraction of the FP32 rate on this GPU, so each pivot's square root and
// reciprocal are computed once, by the lane that finishes the pivot in the
// step before, and handed to the block through shared memory.
__global__ void __launch_bounds__(kCholThreads, 1) k_band_chol(int N, int ld, int use_win, double* L,
                                                               int* bad) {
  extern __shared__ double sm[];
  double* col = sm;         // [ld]: the scaled column of the current step
  double* win = sm + ld;    // [ld][ld] when use_win
  __shared__ int fail;
  __shared__ double pinv;   // 1 / L_kk of the current step
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int bw = ld - 1;
  // window: thread i < ld (ld <= 159 here) keeps element i of the next row to
  // enter the window in a register, loaded one step before it is needed
  double pre = 0.0;
  if (use_win) {
    const int rows = min(ld, N);
    for (int i = tid; i < rows * ld; i += blockDim.x) win[i] = L[i];
    if (tid < ld && ld < N) pre = L[(size_t)ld * ld + tid];
  }
  if (tid == 0) {
    fail = 0;
    pinv = pivot_rsqrt(L[0], &fail);
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double* rk = use_win ? win + (size_t)(k % ld) * ld : L + (size_t)k * ld;
    const int m = min(bw, N - 1 - k);
    const double inv = pinv;
    for (int i = 1 + tid; i <= m; i += blockDim.x) {
      double* ri = use_win ? win + (size_t)((k + i) % ld) * ld : L + (size_t)(k + i) * ld;
      const double v = ri[i] * inv;
      ri[i] = v;
      col[i] = v;
    }
    __syncthreads();
    // trailing update of rows k+1..k+m: A[k+ii][k+jj] -= L[k+ii][k] L[k+jj][k]
    for (int ii = 1 + warp; ii <= m; ii += nwarps) {
      double* ri = use_win ? win + (size_t)((k + ii) % ld) * ld : L + (size_t)(k + ii) * ld;
      const double ci = col[ii];
      for (int jj = 1 + lane; jj <= ii; jj += 32) ri[ii - jj] -= ci * col[jj];
    }
    // lane 0 of warp 0 made the last update of the next pivot (ii = jj = 1)
    if (tid == 0 && m >= 1) {
      const double* r1 = use_win ? win + (size_t)((k + 1) % ld) * ld : L + (size_t)(k + 1) * ld;
      pinv = pivot_rsqrt(r1[0], &fail);
    }
    if (use_win) {
      // row k is final: write it out, move row k + ld into its slot and start
      // loading row k + ld + 1 (untouched until it enters the window)
      if (tid < ld) {
        L[(size_t)k * ld + tid] = tid == 0 ? inv : rk[tid];
        if (k + ld < N) rk[tid] = pre;
        if (k + 1 + ld < N) pre = L[(size_t)(k + 1 + ld) * ld + tid];
      }
    } else if (tid == 0) {
      rk[0] = inv;
    }
    __syncthreads();
  }
  if (tid == 0) *bad = fail;
}

// L y = F, L^T x = y with the factor of k_band_chol (diagonal slots hold
// 1 / L_kk); x scattered into P ((n+2)^2, boundary ring 0).  Thread t handles
// the band offsets 1 + t + r * blockDim.x (r < kSolveR); the block has just
// enough warps for the band.  The pivot and the band entries of the next step
// are loaded one step ahead, so the sequential sweeps wait on shared memory
// and barriers, not on L2.
constexpr int kSolveR = 2;
static_assert(2 * kGalMaxN + 2 <= kSolveR * kSolveThreads, "band offsets per solve thread");
template <typename TA>
__global__ void __launch_bounds__(kSolveThreads) k_band_solve(int n, const double* __restrict__ L,
                                                              double* F, double* Y, int use_smem,
                                                              const int* bad, TA* P, int* flags) {
  extern __shared__ double sm[];
  const int N = n * n, ld = 2 * n + 3, bw = ld - 1, nb = n + 2, tid = threadIdx.x;
  double* f = use_smem ? sm : F;
  double* y = use_smem ? sm + N : Y;
  if (use_smem)
    for (int i = tid; i < N; i += blockDim.x) f[i] = F[i];
  // forward: step k uses L[k][0] and the column L[k+i][i], i = 1..min(bw, N-1-k)
  double lc[kSolveR], ln[kSolveR];
  double dn = L[0];
  for (int r = 0; r < kSolveR; ++r) {
    const int i = 1 + tid + r * blockDim.x;
    ln[r] = i <= min(bw, N - 1) ? L[(size_t)i * ld + i] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    const double dc = dn;
    for (int r = 0; r < kSolveR; ++r) lc[r] = ln[r];
    if (k + 1 < N) {
      dn = L[(size_t)(k + 1) * ld];
      const int m1 = min(bw, N - 2 - k);
      for (int r = 0; r < kSolveR; ++r) {
        const int i = 1 + tid + r * blockDim.x;
        ln[r] = i <= m1 ? L[(size_t)(k + 1 + i) * ld + i] : 0.0;
      }
    }
    const double yk = f[k] * dc;
    if (tid == 0) y[k] = yk;
    const int m = min(bw, N - 1 - k);
    for (int r = 0; r < kSolveR; ++r) {
      const int i = 1 + tid + r * blockDim.x;
      if (i <= m) f[k + i] -= lc[r] * yk;
    }
    __syncthreads();
  }
  // backward: step k uses L[k][0] and the row L[k][j], j = 1..min(bw, k); x overwrites f
  dn = L[(size_t)(N - 1) * ld];
  for (int r = 0; r < kSolveR; ++r) {
    const int j = 1 + tid + r * blockDim.x;
    ln[r] = j <= min(bw, N - 1) ? L[(size_t)(N - 1) * ld + j] : 0.0;
  }
  for (int k = N - 1; k >= 0; --k) {
    const double dc = dn;
    for (int r = 0; r < kSolveR; ++r) lc[r] = ln[r];
    if (k > 0) {
      dn = L[(size_t)(k - 1) * ld];
      const int m1 = min(bw, k - 1);
      for (int r = 0; r < kSolveR; ++r) {
        const int j = 1 + tid + r * blockDim.x;
        ln[r] = j <= m1 ? L[(size_t)(k - 1) * ld + j] : 0.0;
      }
    }
    const double xk = y[k] * dc;
    if (tid == 0) f[k] = xk;
    const int m = min(bw, k);
    for (int r = 0; r < kSolveR; ++r) {
      const int j = 1 + tid + r * blockDim.x;
      if (j <= m) y[k - j] -= lc[r] * xk;
    }
    __syncthreads();
  }
  const bool ok = *bad == 0;
  if (!ok && tid == 0) atomicOr(flags, 1);
  for (int i = tid; i < nb * nb; i += blockDim.x) {
    const int iy = i / nb, ix = i % nb;
    double v = 0.0;
    if (iy >= 1 && iy <= n && ix >= 1 && ix <= n) v = f[(iy - 1) * n + (ix - 1)];
    P[i] = (TA)(ok ? v : __longlong_as_double(0x7ff8000000000000LL));
  }
}

}  // namespace

bool galerkin_supported(int dim, int n) { return dim == 2 && n >= 2 && n <= kGalMaxN; }

size_t galerkin_work_bytes(int n) {
  const size_t N = (size_t)n * n, ld = 2 * (size_t)n + 3;
  // coef, r0, r1 (9 per element each), F, Y, the band, one int slot
  return sizeof(double) * (27 * N + 2 * N + N * ld + 1);
}

template <typename TA>
cudaError_t launch_galerkin_pressure(const GalArgs<TA>& a, cudaStream_t st) {
  const int n = a.n, N = n * n, ld = 2 * n + 3;
  double* coef = a.work;
  double* r0 = coef + 9 * (size_t)N;
  double* r1 = r0 + 9 * (size_t)N;
  double* F = r1 + 9 * (size_t)N;
  double* Y = F + N;
  double* L = Y + N;
  int* bad = reinterpret_cast<int*>(L + (size_t)N * ld);
  k_gal_gauss_2d<TA><<<(N + 127) / 128, 128, 0, st>>>(a, coef, r0, r1);
  const long long total = (long long)N * ld;
  long long nblk = (total + 255) / 256;
  if (nblk > 152LL * 64) nblk = 152LL * 64;
  k_gal_assemble_2d<<<(int)nblk, 256, 0, st>>>(n, a.B, a.dB, coef, r0, r1, L, F);
  const size_t win_bytes = sizeof(double) * ((size_t)ld * ld + ld);
  const int use_win = win_bytes <= kSmemBudget ? 1 : 0;
  const size_t chol_smem = use_win ? win_bytes : sizeof(double) * ld;
  smem_optin(k_band_chol);
  k_band_chol<<<1, kCholThreads, chol_smem, st>>>(N, ld, use_win, L, bad);
  const size_t vec_bytes = sizeof(double) * 2 * (size_t)N;
  const int use_smem = vec_bytes <= kSmemBudget ? 1 : 0;
  smem_optin(k_band_solve<TA>);
  int solve_threads = ((ld - 1 + 31) / 32) * 32;
  if (solve_threads > kSolveThreads) solve_threads = kSolveThreads;
  k_band_solve<TA><<<1, solve_threads, use_smem ? vec_bytes : 0, st>>>(n, L, F, Y, use_smem, bad,
                                                                      a.P, a.flags);
  return cudaGetLastError();
}

template cudaError_t launch_galerkin_pressure<double>(const GalArgs<double>&, cudaStream_t);
template cudaError_t launch_galerkin_pressure<float>(const GalArgs<float>&, cudaStream_t);

}  // namespace adsgb

// IGA-ADS explicit saturation step in 3D (tensor quadratic B-splines on the
// unit cube; Secs. 3-4 of the paper, written there for 2D, extended with the
// third Kronecker factor: M = Mx (x) My (x) Mz).
//
//   k_elem3d:   one thread per element; the Gauss points are taken plane by
//               plane along z, the fields sum-factorised (z, then y, then x)
//               and the test functions applied back (x, then y, then z into
//               the element's 27 right-hand-side entries, which are written
//               component-major: entry i of all elements contiguous).  MODE
//               0: saturation step; MODE 1: L2 projection of nodal values.
//   k_gather3d: one thread per DOF sums the contributions of its (up to) 27
//               elements in a fixed order (deterministic, no atomics).
//   k_xsolve3d: LDL^T sweeps along x (contiguous rows staged in shared memory).
//   k_line_slow: LDL^T sweeps along the slowest axis of a [batch][rows][cols]
//               view (y: batch = z-planes; z: one batch of nb^2 columns), one
//               thread per column, the column block staged in shared memory;
//               optionally accumulates int S (z sweep).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace adsgb {

// the fractional flow's quotient (the fast single-precision divide in FP32)
template <typename T>
ADS_D T frac3(T a, T b) { return a / b; }
template <>
ADS_D float frac3<float>(float a, float b) { return __fdividef(a, b); }

template <typename T, int MODE>
__global__ void __launch_bounds__(128) k_elem3d(QuadArgs<T> a, T* C, double* src_part) {
  __shared__ double red[32];
  const int n = a.n, nb = a.nb, n1 = n + 1;
  const long long ne = (long long)n * n * n;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double src = 0.0;
  if (e < ne) {
    const int ex = (int)(e % n), ey = (int)((e / n) % n), ez = (int)(e / ((long long)n * n));
    const T* Bx = a.ax.B + ex * 9;
    const T* dBx = a.ax.dB + ex * 9;
    const T* By = a.ax.B + ey * 9;
    const T* dBy = a.ax.dB + ey * 9;
    const T* Bz = a.ax.B + ez * 9;
    const T* dBz = a.ax.dB + ez * 9;
    T bx[3][3], dbx[3][3];  // [function][point], used at every point
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      bx[i / 3][i % 3] = __ldg(Bx + i);
      dbx[i / 3][i % 3] = __ldg(dBx + i);
    }
    const T h3 = a.h * a.h * a.h;
    // element right-hand side, accumulated plane by plane of Gauss points
    T R[3][3][3];  // [z fn][y fn][x fn]
#pragma unroll
    for (int i = 0; i < 27; ++i) R[i / 9][(i / 3) % 3][i % 3] = T(0);
    // coefficients (MODE 0: S and P) held for all planes in FP32; in FP64
    // (twice the registers) reread for each plane from the L1 cache
    constexpr bool kHold = sizeof(T) == sizeof(float);
    T s[3][3][3], p[3][3][3];
    T kc[2][2][2], fc[2][2][2];
    auto load_sp = [&]() {
#pragma unroll
      for (int b2 = 0; b2 < 3; ++b2)
#pragma unroll
        for (int b1 = 0; b1 < 3; ++b1) {
          const size_t row = ((size_t)(ez + b2) * nb + (ey + b1)) * nb + ex;
#pragma unroll
          for (int b0 = 0; b0 < 3; ++b0) {
            s[b2][b1][b0] = __ldg(a.S + row + b0);
            p[b2][b1][b0] = __ldg(a.P + row + b0);
          }
        }
    };
    if (MODE == 0 && kHold) load_sp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int dz = i >> 2, dy = (i >> 1) & 1, dx = i & 1;
      const size_t nd = ((size_t)(ez + dz) * n1 + (ey + dy)) * n1 + (ex + dx);
      kc[dz][dy][dx] = MODE == 0 ? __ldg(a.K + nd) : __ldg(a.nodal + nd);
      fc[dz][dy][dx] = (MODE == 0 && a.phi) ? __ldg(a.phi + nd) : a.phi_c;
    }
    const T dt = MODE == 0 ? (T)(*a.dt) : T(0);
    const T dtphi_c = MODE == 0 ? dt / a.phi_c : T(0);  // porosity without a map
    T src_e = T(0);  // this element's source integral (27 terms), then one FP64 add
    // (one plane's code, run three times: the unrolled body is large)
#pragma unroll 1
    for (int qz = 0; qz < 3; ++qz) {
      const T zeta = (T)gauss_x(qz), wzh3 = (T)gauss_w(qz) * h3;
      T bzq[3], dbzq[3];  // the z factors at this plane
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        bzq[c] = __ldg(Bz + c * 3 + qz);
        dbzq[c] = __ldg(dBz + c * 3 + qz);
      }
      // z contraction: S, P and dP/dz on this plane, per (y, x) function
      T Sz[3][3], Pz[3][3], Pzd[3][3];
      if (MODE == 0) {
        if (!kHold) load_sp();
#pragma unroll
        for (int b1 = 0; b1 < 3; ++b1)
#pragma unroll
          for (int b0 = 0; b0 < 3; ++b0) {
            Sz[b1][b0] = bzq[0] * s[0][b1][b0] + bzq[1] * s[1][b1][b0] + bzq[2] * s[2][b1][b0];
            Pz[b1][b0] = bzq[0] * p[0][b1][b0] + bzq[1] * p[1][b1][b0] + bzq[2] * p[2][b1][b0];
            Pzd[b1][b0] = dbzq[0] * p[0][b1][b0] + dbzq[1] * p[1][b1][b0] + dbzq[2] * p[2][b1][b0];
          }
      }
      // trilinear K, phi: the z interpolation on this plane
      T kz[2][2], fz[2][2];
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          kz[dy][dx] = (T(1) - zeta) * kc[0][dy][dx] + zeta * kc[1][dy][dx];
          fz[dy][dx] = (T(1) - zeta) * fc[0][dy][dx] + zeta * fc[1][dy][dx];
        }
      T Ty0[3][3], Tyz[3][3];  // [y fn][x fn]: y contraction of this plane
#pragma unroll
      for (int i = 0; i < 9; ++i) Ty0[i / 3][i % 3] = Tyz[i / 3][i % 3] = T(0);
#pragma unroll
      for (int qy = 0; qy < 3; ++qy) {
        const T eta = (T)gauss_x(qy);
        T byq[3], dbyq[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          byq[c] = __ldg(By + c * 3 + qy);
          dbyq[c] = __ldg(dBy + c * 3 + qy);
        }
        T Syz[3], Pyz[3], Pydy[3], Pzy[3];  // per x function
        if (MODE == 0) {
#pragma unroll
          for (int b0 = 0; b0 < 3; ++b0) {
            Syz[b0] = byq[0] * Sz[0][b0] + byq[1] * Sz[1][b0] + byq[2] * Sz[2][b0];
            Pyz[b0] = byq[0] * Pz[0][b0] + byq[1] * Pz[1][b0] + byq[2] * Pz[2][b0];
            Pydy[b0] = dbyq[0] * Pz[0][b0] + dbyq[1] * Pz[1][b0] + dbyq[2] * Pz[2][b0];
            Pzy[b0] = byq[0] * Pzd[0][b0] + byq[1] * Pzd[1][b0] + byq[2] * Pzd[2][b0];
          }
        }
        const T ky[2] = {(T(1) - eta) * kz[0][0] + eta * kz[1][0], (T(1) - eta) * kz[0][1] + eta * kz[1][1]};
        const T fy[2] = {(T(1) - eta) * fz[0][0] + eta * fz[1][0], (T(1) - eta) * fz[0][1] + eta * fz[1][1]};
        T Tx0[3] = {T(0), T(0), T(0)}, Txy[3] = {T(0), T(0), T(0)}, Txz[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int qx = 0; qx < 3; ++qx) {
          const T xi = (T)gauss_x(qx);
          const T w = (T)(gauss_w(qx) * gauss_w(qy)) * wzh3;
          const T Kq = (T(1) - xi) * ky[0] + xi * ky[1];
          T c0, cx = T(0), cy = T(0), cz = T(0);
          if (MODE == 0) {
            const T Sv = bx[0][qx] * Syz[0] + bx[1][qx] * Syz[1] + bx[2][qx] * Syz[2];
            const T dpx = dbx[0][qx] * Pyz[0] + dbx[1][qx] * Pyz[1] + dbx[2][qx] * Pyz[2];
            const T dpy = bx[0][qx] * Pydy[0] + bx[1][qx] * Pydy[1] + bx[2][qx] * Pydy[2];
            const T dpz = bx[0][qx] * Pzy[0] + bx[1][qx] * Pzy[1] + bx[2][qx] * Pzy[2];
            const T phq = (T(1) - xi) * fy[0] + xi * fy[1];
            const T St = clamp01(Sv);
            const T lg = St * a.inv_mu_g, lw = (T(1) - St) * a.inv_mu_w;
            T qi = T(0), qp = T(0);
            for (int sidx = 0; sidx < a.n_src; ++sidx) {
              const T gv = a.rate[sidx] * __ldg(a.ax.gsrc + ((size_t)(0 * kMaxSrc + sidx) * n + ex) * 3 + qx) *
                           __ldg(a.ax.gsrc + ((size_t)(1 * kMaxSrc + sidx) * n + ey) * 3 + qy) *
                           __ldg(a.ax.gsrc + ((size_t)(2 * kMaxSrc + sidx) * n + ez) * 3 + qz);
              if (a.kind[sidx] == 0) qi += gv;
              else qp += gv;
            }
            T qg = qi;
            if (qp != T(0)) qg -= frac3(lg, lg + lw) * qp;
            const T dtphi = a.phi ? dt / phq : dtphi_c;
            const T wq = w * dtphi * qg;
            c0 = w * Sv + wq;
            const T cf = -w * dtphi * lg * Kq;
            cx = cf * dpx;
            cy = cf * dpy;
            cz = cf * a.kz * (dpz + a.grav_term);
            src_e += wq;
          } else {
            c0 = w * Kq;  // (MODE 1: kc holds the nodal values)
          }
          // test functions along x
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            Tx0[aa] += c0 * bx[aa][qx] + cx * dbx[aa][qx];
            Txy[aa] += cy * bx[aa][qx];
            Txz[aa] += cz * bx[aa][qx];
          }
        }
        // along y
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            Ty0[b][aa] += byq[b] * Tx0[aa] + dbyq[b] * Txy[aa];
            Tyz[b][aa] += byq[b] * Txz[aa];
          }
      }
      // along z, into the element's right-hand side
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) R[c2][b][aa] += bzq[c2] * Ty0[b][aa] + dbzq[c2] * Tyz[b][aa];
    }
    src = (double)src_e;
    // component-major: component i of all elements is contiguous (coalesced)
#pragma unroll
    for (int i = 0; i < 27; ++i) C[(size_t)i * ne + e] = R[i / 9][(i / 3) % 3][i % 3];
  }
  if (MODE == 0) {
    double tot = block_sum(src, red);
    if (threadIdx.x == 0) src_part[blockIdx.x] = tot;
  }
}

// R[kz][ky][kx] = sum over elements e with e_d in [k_d - 2, k_d] of
// C[(kz-ez)*9 + (ky-ey)*3 + (kx-ex)][e], in a fixed order
template <typename T>
__global__ void __launch_bounds__(256) k_gather3d(int n, const T* __restrict__ C, T* __restrict__ R) {
  const int nb = n + 2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nb * nb * nb) return;
  const int kx = (int)(t % nb), ky = (int)((t / nb) % nb), kz = (int)(t / ((long long)nb * nb));
  const size_t ne = (size_t)n * n * n;
  T v = T(0);
  for (int dz = 0; dz < 3; ++dz) {
    const int ez = kz - dz;
    if (ez < 0 || ez >= n) continue;
    for (int dy = 0; dy < 3; ++dy) {
      const int ey = ky - dy;
      if (ey < 0 || ey >= n) continue;
      for (int dx = 0; dx < 3; ++dx) {
        const int ex = kx - dx;
        if (ex < 0 || ex >= n) continue;
        const size_t e = ((size_t)ez * n + ey) * n + ex;
        v += C[(size_t)((dz * 3 + dy) * 3 + dx) * ne + e];
      }
    }
  }
  R[t] = v;
}

// x sweeps: a CTA stages 32 contiguous rows (padded stride) and 32 threads
// run the LDL^T recurrences in shared memory
template <typename T>
__global__ void __launch_bounds__(256) k_xsolve3d(int nrows, int nb, T* X, const T* l1,
                                                  const T* l2, const T* dinv) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);
  const int ps = nb + 1;
  const int r0 = blockIdx.x * 32;
  const int nr = min(32, nrows - r0);
  for (int e = threadIdx.x; e < nr * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    cp_async_elem(&xs[r * ps + c], &X[(size_t)(r0 + r) * nb + c]);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  const int r = threadIdx.x;
  if (r < nr) {
    T* x = xs + r * ps;
    T ym1 = T(0), ym2 = T(0);
    for (int l = 0; l < nb; ++l) {
      T y = x[l] - l1[l] * ym1 - l2[l] * ym2;
      x[l] = y;
      ym2 = ym1;
      ym1 = y;
    }
    T xp1 = T(0), xp2 = T(0);
    for (int l = nb - 1; l >= 0; --l) {
      T v = x[l] * dinv[l] - l1[l + 1] * xp1 - l2[l + 2] * xp2;
      x[l] = v;
      xp2 = xp1;
      xp1 = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * nb; e += blockDim.x) {
    const int rr = e / nb, c = e % nb;
    X[(size_t)(r0 + rr) * nb + c] = xs[rr * ps + c];
  }
}

// sweeps along the slowest axis of X viewed as [batch][nb rows][ncols]; CTA =
// (column block of cw, batch); with Iw != nullptr each column also sums
// x_l Iw[l] and, if its column index decomposes as (y, x) over nb x nb,
// multiplies by Iw[y] Iw[x] (the z sweep of int S)
template <typename T>
__global__ void __launch_bounds__(256) k_line_slow(int nb, int ncols, int cw, T* X, const T* l1,
                                                   const T* l2, const T* dinv, const T* Iw,
                                                   double* mass_part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  T* xs = reinterpret_cast<T*>(smraw);  // [nb][cw]
  const int c0 = blockIdx.x * cw;
  const int ncw = min(cw, ncols - c0);
  T* base = X + (size_t)blockIdx.y * nb * ncols;
  for (int e = threadIdx.x; e < nb * cw; e += blockDim.x) {
    const int l = e / cw, c = e % cw;
    if (c < ncw) cp_async_elem(&xs[e], &base[(size_t)l * ncols + c0 + c]);
  }
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  double mass = 0.0;
  const int c = threadIdx.x;
  if (c < ncw) {
    T ym1 = T(0), ym2 = T(0);
    for (int l = 0; l < nb; ++l) {
      T y = xs[l * cw + c] - l1[l] * ym1 - l2[l] * ym2;
      xs[l * cw + c] = y;
      ym2 = ym1;
      ym1 = y;
    }
    T xp1 = T(0), xp2 = T(0);
    for (int l = nb - 1; l >= 0; --l) {
      T v = xs[l * cw + c] * dinv[l] - l1[l + 1] * xp1 - l2[l + 2] * xp2;
      xs[l * cw + c] = v;
      if (Iw) mass += (double)v * (double)Iw[l];
      xp2 = xp1;
      xp1 = v;
    }
    if (Iw) {
      const int col = c0 + c;
      mass *= (double)Iw[col / nb] * (double)Iw[col % nb];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nb * cw; e += blockDim.x) {
    const int l = e / cw, cc = e % cw;
    if (cc < ncw) base[(size_t)l * ncols + c0 + cc] = xs[e];
  }
  if (mass_part) {
    double tot = block_sum(mass, red);
    if (threadIdx.x == 0) mass_part[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

static int slow_cw(int nb, size_t es) {
  int cw = 32;
  while (cw > 1 && es * (size_t)nb * cw > 160 * 1024) cw /= 2;
  return cw;
}

size_t elem3d_scratch(int n, size_t es) { return (size_t)n * n * n * 27 * es; }
int quad3d_blocks(int n) { return (int)(((long long)n * n * n + 127) / 128); }
int zsolve3d_blocks(int n) {
  const int nb = n + 2;
  const int cw = slow_cw(nb, 8);
  return (nb * nb + cw - 1) / cw;
}

// RHS (element contributions + gather) into R
template <typename T>
cudaError_t launch_quad3d(const QuadArgs<T>& a, int mode, T* Cbuf, T* R, double* src_part,
                          cudaStream_t st) {
  const int nblk = quad3d_blocks(a.n);
  if (mode == 0) k_elem3d<T, 0><<<nblk, 128, 0, st>>>(a, Cbuf, src_part);
  else k_elem3d<T, 1><<<nblk, 128, 0, st>>>(a, Cbuf, src_part);
  const long long nd = (long long)a.nb * a.nb * a.nb;
  k_gather3d<T><<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(a.n, Cbuf, R);
  return cudaGetLastError();
}

// the three sweeps of M^-1 = Mx^-1 (x) My^-1 (x) Mz^-1, int S from the z sweep
template <typename T>
cudaError_t launch_solve3d(const QuadArgs<T>& a, T* X, double* mass_part, cudaStream_t st) {
  const int nb = a.nb;
  const int nrows = nb * nb;
  size_t smx = sizeof(T) * 32 * (size_t)(nb + 1);
  smem_optin(k_xsolve3d<T>);
  k_xsolve3d<T><<<(nrows + 31) / 32, 256, smx, st>>>(nrows, nb, X, a.ax.l1, a.ax.l2, a.ax.dinv);
  const int cw = slow_cw(nb, sizeof(T));
  const size_t sms = sizeof(T) * (size_t)nb * cw;
  smem_optin(k_line_slow<T>);
  // y: batch = z planes, rows = y, columns = x
  dim3 gy((nb + cw - 1) / cw, nb);
  k_line_slow<T><<<gy, 256, sms, st>>>(nb, nb, cw, X, a.ax.l1, a.ax.l2, a.ax.dinv, nullptr, nullptr);
  // z: one batch, rows = z, columns = (y, x)
  dim3 gz((nb * nb + cw - 1) / cw, 1);
  k_line_slow<T><<<gz, 256, sms, st>>>(nb, nb * nb, cw, X, a.ax.l1, a.ax.l2, a.ax.dinv,
                                       mass_part ? a.ax.Iw : nullptr, mass_part);
  const int nmax = zsolve3d_blocks(a.n);
  if (mass_part && (int)gz.x < nmax)
    cudaMemsetAsync(mass_part + gz.x, 0, sizeof(double) * (nmax - gz.x), st);
  return cudaGetLastError();
}

// int S = sum S_ijk Iw_i Iw_j Iw_k: thread per (y, x) column
template <typename T>
__global__ void __launch_bounds__(128) k_mass3d(int n, const T* S, const T* Iw, double* part) {
  __shared__ double red[32];
  const int nb = n + 2;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (c < nb * nb) {
    for (int l = 0; l < nb; ++l) m += (double)S[(size_t)l * nb * nb + c] * (double)Iw[l];
    m *= (double)Iw[c / nb] * (double)Iw[c % nb];
  }
  double tot = block_sum(m, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename T>
cudaError_t launch_mass3d(const QuadArgs<T>& a, const T* S, double* mass_part, cudaStream_t st) {
  const int nb = a.nb;
  const int nblk = (nb * nb + 127) / 128;
  k_mass3d<T><<<nblk, 128, 0, st>>>(a.n, S, a.ax.Iw, mass_part);
  const int nmax = zsolve3d_blocks(a.n);
  if (nblk < nmax) cudaMemsetAsync(mass_part + nblk, 0, sizeof(double) * (nmax - nblk), st);
  return cudaGetLastError();
}

// CFL in 3D: max over Gauss points of |K (grad p + s rho_g g e_z)|/(mu_g phi)
// and of q_inj/phi
template <typename T>
__global__ void __launch_bounds__(256) k_cfl3d(QuadArgs<T> a, double* part) {
  __shared__ double red[32];
  const int n = a.n, nb = a.nb, n1 = n + 1;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double vmax = 0.0, smax = 0.0;
  if (e < (long long)n * n * n) {
    const int ex = (int)(e % n), ey = (int)((e / n) % n), ez = (int)(e / ((long long)n * n));
    const T* Bx = a.ax.B + ex * 9; const T* dBx = a.ax.dB + ex * 9;
    const T* By = a.ax.B + ey * 9; const T* dBy = a.ax.dB + ey * 9;
    const T* Bz = a.ax.B + ez * 9; const T* dBz = a.ax.dB + ez * 9;
    for (int qz = 0; qz < 3; ++qz)
      for (int qy = 0; qy < 3; ++qy)
        for (int qx = 0; qx < 3; ++qx) {
          T dpx = T(0), dpy = T(0), dpz = T(0);
          for (int c2 = 0; c2 < 3; ++c2)
            for (int b = 0; b < 3; ++b)
              for (int aa = 0; aa < 3; ++aa) {
                const T pv = a.P[((size_t)(ez + c2) * nb + (ey + b)) * nb + ex + aa];
                dpx += pv * dBx[aa * 3 + qx] * By[b * 3 + qy] * Bz[c2 * 3 + qz];
                dpy += pv * Bx[aa * 3 + qx] * dBy[b * 3 + qy] * Bz[c2 * 3 + qz];
                dpz += pv * Bx[aa * 3 + qx] * By[b * 3 + qy] * dBz[c2 * 3 + qz];
              }
          const T zeta = (T)gauss_x(qz), eta = (T)gauss_x(qy), xi = (T)gauss_x(qx);
          T wz[2] = {T(1) - zeta, zeta}, wy[2] = {T(1) - eta, eta}, wx[2] = {T(1) - xi, xi};
          T Kq = T(0), phq = T(0);
          for (int i = 0; i < 8; ++i) {
            const int dz = i >> 2, dy = (i >> 1) & 1, dx = i & 1;
            const size_t nd = ((size_t)(ez + dz) * n1 + (ey + dy)) * n1 + (ex + dx);
            const T w = wz[dz] * wy[dy] * wx[dx];
            Kq += w * a.K[nd];
            phq += w * (a.phi ? a.phi[nd] : a.phi_c);
          }
          T fx = Kq * dpx, fy = Kq * dpy, fz = a.kz * Kq * (dpz + a.grav_term);
          double v = sqrt((double)(fx * fx + fy * fy + fz * fz)) * (double)a.inv_mu_g / (double)phq;
          vmax = fmax(vmax, v);
          T qi = T(0);
          for (int s = 0; s < a.n_src; ++s)
            if (a.kind[s] == 0)
              qi += a.rate[s] * a.ax.gsrc[((size_t)(0 * kMaxSrc + s) * n + ex) * 3 + qx] *
                    a.ax.gsrc[((size_t)(1 * kMaxSrc + s) * n + ey) * 3 + qy] *
                    a.ax.gsrc[((size_t)(2 * kMaxSrc + s) * n + ez) * 3 + qz];
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

template <typename T>
cudaError_t launch_cfl3d(const QuadArgs<T>& a, double* part, cudaStream_t st) {
  k_cfl3d<T><<<cfl_blocks(3, a.n), 256, 0, st>>>(a, part);
  return cudaGetLastError();
}

#define ADS3_INST(T)                                                                              \
  template cudaError_t launch_quad3d<T>(const QuadArgs<T>&, int, T*, T*, double*, cudaStream_t); \
  template cudaError_t launch_solve3d<T>(const QuadArgs<T>&, T*, double*, cudaStream_t);         \
  template cudaError_t launch_mass3d<T>(const QuadArgs<T>&, const T*, double*, cudaStream_t);    \
  template cudaError_t launch_cfl3d<T>(const QuadArgs<T>&, double*, cudaStream_t);
ADS3_INST(double)
ADS3_INST(float)

}  // namespace adsgb

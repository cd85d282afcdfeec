// Explicit saturation step for tensor B-splines of degree p = 2, 3 or 4 (Sec. 4:
// the basis of order r with continuity C^{r-1}, Eq. 11; the step of Eqs.
// 10b-13 and the Kronecker mass solve of Eq. 14), 2D, FP64.
//
// The quadratic path of ads_kernels.cu is shaped around p = 2 (three Gauss
// points, three functions per element, warp-shuffle assembly).  This path is
// written for any p up to 4 and for correctness first:
//   * the tables -- Gauss-Legendre points (p + 1 per element), the values and
//     derivatives of the p + 1 functions alive on each element, the banded
//     1D mass matrix M (bandwidth p), its LDL^T factors, the basis integrals
//     and the sources' per-axis Gaussian factors -- are computed on the host
//     once per plan (Cox-de Boor recursion on the open uniform knot vector)
//     and copied to the device;
//   * one thread per element evaluates the (p + 1)^2 Gauss points and writes
//     its (p + 1)^2 local right-hand-side terms;
//   * one thread per degree of freedom adds the terms of the (p + 1)^2
//     elements around it in a fixed order (no atomics: the sums do not depend
//     on scheduling);
//   * one thread per line solves M x = r along x, then along y, with the
//     banded factors (forward, diagonal, backward substitution).
// The step's vector-Jacobian product (gradients of J = lambda . S_out with
// respect to S, P and the sources' rates and centres) serves the inverse
// problem the conclusions name as future work -- where to put the injection
// well: it reuses the same tables, line solves and gathers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>
#include <thread>
#include <vector>

#include "adsgb.h"
#include "kernels.cuh"

namespace adsgb {
ads_status validate_params(const ads_params* p, const crvpinn_params* cp);  // api.cu

namespace {

constexpr int kMaxDeg = 4;
constexpr int kMaxDegN = 4096;  // largest mesh a plan takes

// arguments of the element kernel
struct DegArgs {
  int n, nb, n_src;
  double h2;                      // h^2 (the Jacobian of an element)
  double wq[kMaxDeg + 1];         // Gauss weights on [0, 1]
  double xi[kMaxDeg + 1];         // Gauss points on [0, 1] (the hat functions of the nodal maps)
  const double* B;                // [n][p+1 functions][p+1 points]
  const double* dB;               // d/dx, same layout
  const double* g;                // [2 axes][n_src][n][p+1]: per-axis Gaussian factors
  double rate[kMaxSrc];
  int kind[kMaxSrc];
  double inv_mu_g, inv_mu_w, grav_term, phi_c, dt;
  const double *K, *phi, *S, *P;  // K, phi nodal (n+1)^2 (phi nullable); S, P (n+p)^2
  double* part;                   // [n][n][p+1][p+1] local terms
  // vector-Jacobian product only
  double cen[kMaxSrc][2], sig[kMaxSrc];
  const double* mu;               // M^-1 lambda, (n+p)^2
  double* part2;                  // [n][n][p+1][p+1] local terms of dJ/dP
  double* psrc;                   // [n][n][3 n_src] per-element d/d(rate, cx, cy) terms
};

// One element: the weak form's integrand at the (p+1)^2 Gauss points (the
// same terms as the quadratic path) and its local terms against the (p+1)^2
// test functions alive on the element.
template <int P>
__global__ void __launch_bounds__(128) k_deg_elem(DegArgs a) {
  constexpr int Q = P + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n * a.n) return;
  const int ex = e % a.n, ey = e / a.n, n1 = a.n + 1;
  double s[Q][Q], pp[Q][Q];  // coefficients [row b][column c] of S and P on the element
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      s[b][c] = a.S[(size_t)(ey + b) * a.nb + ex + c];
      pp[b][c] = a.P[(size_t)(ey + b) * a.nb + ex + c];
    }
  const double* Bx = a.B + (size_t)ex * Q * Q;
  const double* dBx = a.dB + (size_t)ex * Q * Q;
  const double* By = a.B + (size_t)ey * Q * Q;
  const double* dBy = a.dB + (size_t)ey * Q * Q;
  const double k00 = a.K[(size_t)ey * n1 + ex], k01 = a.K[(size_t)ey * n1 + ex + 1];
  const double k10 = a.K[(size_t)(ey + 1) * n1 + ex], k11 = a.K[(size_t)(ey + 1) * n1 + ex + 1];
  double f00 = a.phi_c, f01 = a.phi_c, f10 = a.phi_c, f11 = a.phi_c;
  if (a.phi) {
    f00 = a.phi[(size_t)ey * n1 + ex];
    f01 = a.phi[(size_t)ey * n1 + ex + 1];
    f10 = a.phi[(size_t)(ey + 1) * n1 + ex];
    f11 = a.phi[(size_t)(ey + 1) * n1 + ex + 1];
  }
  double r[Q][Q];
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) r[b][c] = 0.0;
  for (int qy = 0; qy < Q; ++qy) {
    const double eta = a.xi[qy];
    for (int qx = 0; qx < Q; ++qx) {
      const double xi = a.xi[qx];
      // S, dP/dx, dP/dy at the point
      double Sv = 0.0, px = 0.0, py = 0.0;
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        double sb = 0.0, pb = 0.0, pdb = 0.0;
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          sb += s[b][c] * Bx[c * Q + qx];
          pb += pp[b][c] * Bx[c * Q + qx];
          pdb += pp[b][c] * dBx[c * Q + qx];
        }
        Sv += By[b * Q + qy] * sb;
        px += By[b * Q + qy] * pdb;
        py += dBy[b * Q + qy] * pb;
      }
      const double Kq = (1.0 - eta) * ((1.0 - xi) * k00 + xi * k01) + eta * ((1.0 - xi) * k10 + xi * k11);
      const double phq = (1.0 - eta) * ((1.0 - xi) * f00 + xi * f01) + eta * ((1.0 - xi) * f10 + xi * f11);
      const double St = Sv < 0.0 ? 0.0 : (Sv > 1.0 ? 1.0 : Sv);
      const double lg = St * a.inv_mu_g, lw = (1.0 - St) * a.inv_mu_w;
      double qi = 0.0, qp = 0.0;
      for (int k = 0; k < a.n_src; ++k) {
        const double gv = a.rate[k] * a.g[((size_t)(0 * a.n_src + k) * a.n + ex) * Q + qx] *
                          a.g[((size_t)(1 * a.n_src + k) * a.n + ey) * Q + qy];
        if (a.kind[k] == 0) qi += gv;
        else qp += gv;
      }
      const double qg = qi - lg / (lg + lw) * qp;
      const double W = a.wq[qx] * a.wq[qy] * a.h2;
      const double c0 = W * (Sv + a.dt / phq * qg);
      const double cf = -W * a.dt / phq * lg * Kq;
      const double cx = cf * px, cy = cf * (py + a.grav_term);
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const double vb = By[b * Q + qy], dvb = dBy[b * Q + qy];
#pragma unroll
        for (int c = 0; c < Q; ++c)
          r[b][c] += (c0 * vb + cy * dvb) * Bx[c * Q + qx] + cx * vb * dBx[c * Q + qx];
      }
    }
  }
  double* o = a.part + (size_t)e * Q * Q;
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) o[b * Q + c] = r[b][c];
}

// Vector-Jacobian product of the step on one element.  With mu = M^-1 lambda
// (M symmetric), J = lambda . S_out = mu . R(S, P, sources), and
//   mu . R = sum_q W [ (S + tau/phi q_g(S)) mu_h - tau/phi lambda_g(S) K
//                      (grad p + s rho_g g e_y) . grad mu_h ]
// at the Gauss points, mu_h the spline with coefficients mu.  Its partial
// derivatives at a point, times the basis, give the element's terms of
// dJ/dS (through S at the point), of dJ/dP (through grad p) and of the
// sources' rates and centres (through q_g).  The clamp of the mobility is
// differentiated inside (0, 1) and taken as flat outside.
template <int P>
__global__ void __launch_bounds__(128) k_deg_vjp(DegArgs a) {
  constexpr int Q = P + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n * a.n) return;
  const int ex = e % a.n, ey = e / a.n, n1 = a.n + 1;
  const double h = sqrt(a.h2);
  double s[Q][Q], pp[Q][Q], mu[Q][Q];
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      const size_t o = (size_t)(ey + b) * a.nb + ex + c;
      s[b][c] = a.S[o];
      pp[b][c] = a.P[o];
      mu[b][c] = a.mu[o];
    }
  const double* Bx = a.B + (size_t)ex * Q * Q;
  const double* dBx = a.dB + (size_t)ex * Q * Q;
  const double* By = a.B + (size_t)ey * Q * Q;
  const double* dBy = a.dB + (size_t)ey * Q * Q;
  const double k00 = a.K[(size_t)ey * n1 + ex], k01 = a.K[(size_t)ey * n1 + ex + 1];
  const double k10 = a.K[(size_t)(ey + 1) * n1 + ex], k11 = a.K[(size_t)(ey + 1) * n1 + ex + 1];
  double f00 = a.phi_c, f01 = a.phi_c, f10 = a.phi_c, f11 = a.phi_c;
  if (a.phi) {
    f00 = a.phi[(size_t)ey * n1 + ex];
    f01 = a.phi[(size_t)ey * n1 + ex + 1];
    f10 = a.phi[(size_t)(ey + 1) * n1 + ex];
    f11 = a.phi[(size_t)(ey + 1) * n1 + ex + 1];
  }
  double gs[Q][Q], gp[Q][Q], ps[3 * kMaxSrc];
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) gs[b][c] = gp[b][c] = 0.0;
  for (int k = 0; k < 3 * kMaxSrc; ++k) ps[k] = 0.0;
  for (int qy = 0; qy < Q; ++qy) {
    const double eta = a.xi[qy], y = (ey + eta) * h;
    for (int qx = 0; qx < Q; ++qx) {
      const double xi = a.xi[qx], x = (ex + xi) * h;
      double Sv = 0.0, px = 0.0, py = 0.0, mq = 0.0, mqx = 0.0, mqy = 0.0;
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        double sb = 0.0, pb = 0.0, pdb = 0.0, mb = 0.0, mdb = 0.0;
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          sb += s[b][c] * Bx[c * Q + qx];
          pb += pp[b][c] * Bx[c * Q + qx];
          pdb += pp[b][c] * dBx[c * Q + qx];
          mb += mu[b][c] * Bx[c * Q + qx];
          mdb += mu[b][c] * dBx[c * Q + qx];
        }
        Sv += By[b * Q + qy] * sb;
        px += By[b * Q + qy] * pdb;
        py += dBy[b * Q + qy] * pb;
        mq += By[b * Q + qy] * mb;
        mqx += By[b * Q + qy] * mdb;
        mqy += dBy[b * Q + qy] * mb;
      }
      const double Kq = (1.0 - eta) * ((1.0 - xi) * k00 + xi * k01) + eta * ((1.0 - xi) * k10 + xi * k11);
      const double phq = (1.0 - eta) * ((1.0 - xi) * f00 + xi * f01) + eta * ((1.0 - xi) * f10 + xi * f11);
      const bool inside = Sv > 0.0 && Sv < 1.0;
      const double St = Sv < 0.0 ? 0.0 : (Sv > 1.0 ? 1.0 : Sv);
      const double lg = St * a.inv_mu_g, lw = (1.0 - St) * a.inv_mu_w;
      const double dlg = inside ? a.inv_mu_g : 0.0, dlw = inside ? -a.inv_mu_w : 0.0;
      const double lt = lg + lw, fg = lg / lt, dfg = (dlg * lw - lg * dlw) / (lt * lt);
      double qp = 0.0;
      for (int k = 0; k < a.n_src; ++k)
        if (a.kind[k] != 0)
          qp += a.rate[k] * a.g[((size_t)(0 * a.n_src + k) * a.n + ex) * Q + qx] *
                a.g[((size_t)(1 * a.n_src + k) * a.n + ey) * Q + qy];
      const double W = a.wq[qx] * a.wq[qy] * a.h2, tp = a.dt / phq;
      const double flux = Kq * (px * mqx + (py + a.grav_term) * mqy);
      const double dFdS = W * ((1.0 - tp * dfg * qp) * mq - tp * dlg * flux);
      const double dFdpx = -W * tp * lg * Kq * mqx, dFdpy = -W * tp * lg * Kq * mqy;
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        const double vb = By[b * Q + qy], dvb = dBy[b * Q + qy];
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          gs[b][c] += dFdS * vb * Bx[c * Q + qx];
          gp[b][c] += dFdpx * vb * dBx[c * Q + qx] + dFdpy * dvb * Bx[c * Q + qx];
        }
      }
      // sources: q_g = sum_inj rate G - f_g sum_prod rate G, G the normalised
      // Gaussian; dG/dc = G (x - c) / sigma^2 per coordinate
      const double wm = W * tp * mq;
      for (int k = 0; k < a.n_src; ++k) {
        const double G = a.g[((size_t)(0 * a.n_src + k) * a.n + ex) * Q + qx] *
                         a.g[((size_t)(1 * a.n_src + k) * a.n + ey) * Q + qy];
        const double sgn = a.kind[k] == 0 ? 1.0 : -fg, is2 = 1.0 / (a.sig[k] * a.sig[k]);
        ps[3 * k] += wm * sgn * G;
        ps[3 * k + 1] += wm * sgn * a.rate[k] * G * (x - a.cen[k][0]) * is2;
        ps[3 * k + 2] += wm * sgn * a.rate[k] * G * (y - a.cen[k][1]) * is2;
      }
    }
  }
  double* o = a.part + (size_t)e * Q * Q;
  double* o2 = a.part2 + (size_t)e * Q * Q;
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      o[b * Q + c] = gs[b][c];
      o2[b * Q + c] = gp[b][c];
    }
  for (int k = 0; k < 3 * a.n_src; ++k) a.psrc[(size_t)e * 3 * a.n_src + k] = ps[k];
}

// L2 projection of a nodal field into the splines (Sec. 6, step 4: the
// network pressure, known at the nodes, enters the saturation step through
// its coefficients): local terms of int I_h u v for the element's test
// functions, I_h u the bilinear interpolant of the nodal values
template <int P>
__global__ void __launch_bounds__(128) k_deg_proj(DegArgs a, const double* __restrict__ nodal) {
  constexpr int Q = P + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n * a.n) return;
  const int ex = e % a.n, ey = e / a.n, n1 = a.n + 1;
  const double* Bx = a.B + (size_t)ex * Q * Q;
  const double* By = a.B + (size_t)ey * Q * Q;
  const double u00 = nodal[(size_t)ey * n1 + ex], u01 = nodal[(size_t)ey * n1 + ex + 1];
  const double u10 = nodal[(size_t)(ey + 1) * n1 + ex], u11 = nodal[(size_t)(ey + 1) * n1 + ex + 1];
  double r[Q][Q];
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) r[b][c] = 0.0;
  for (int qy = 0; qy < Q; ++qy) {
    const double eta = a.xi[qy];
    for (int qx = 0; qx < Q; ++qx) {
      const double xi = a.xi[qx];
      const double uq = (1.0 - eta) * ((1.0 - xi) * u00 + xi * u01) + eta * ((1.0 - xi) * u10 + xi * u11);
      const double c0 = a.wq[qx] * a.wq[qy] * a.h2 * uq;
#pragma unroll
      for (int b = 0; b < Q; ++b)
#pragma unroll
        for (int c = 0; c < Q; ++c) r[b][c] += c0 * By[b * Q + qy] * Bx[c * Q + qx];
    }
  }
  double* o = a.part + (size_t)e * Q * Q;
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) o[b * Q + c] = r[b][c];
}

// Adjoint of the projection: with mu = M^-1 g (M symmetric), element e's part
// of dJ/d(nodal) for J = g . M^-1 F(nodal): at each Gauss point the test sum
// sum_bc mu_bc B_b(y) B_c(x), weighted and spread to the element's four
// nodes by the bilinear hats (the transpose of the interpolation above);
// part[e][0..3] = the terms of nodes (ex, ey), (ex + 1, ey), (ex, ey + 1),
// (ex + 1, ey + 1)
template <int P>
__global__ void __launch_bounds__(128) k_deg_proj_vjp(DegArgs a, const double* __restrict__ mu,
                                                     double* __restrict__ part) {
  constexpr int Q = P + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n * a.n) return;
  const int ex = e % a.n, ey = e / a.n, nb = a.nb;
  const double* Bx = a.B + (size_t)ex * Q * Q;
  const double* By = a.B + (size_t)ey * Q * Q;
  double m[Q][Q];
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) m[b][c] = mu[(size_t)(ey + b) * nb + ex + c];
  double g00 = 0.0, g01 = 0.0, g10 = 0.0, g11 = 0.0;
  for (int qy = 0; qy < Q; ++qy) {
    const double eta = a.xi[qy];
    for (int qx = 0; qx < Q; ++qx) {
      const double xi = a.xi[qx];
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < Q; ++b)
#pragma unroll
        for (int c = 0; c < Q; ++c) t += m[b][c] * By[b * Q + qy] * Bx[c * Q + qx];
      const double c0 = a.wq[qx] * a.wq[qy] * a.h2 * t;
      g00 += c0 * (1.0 - eta) * (1.0 - xi);
      g01 += c0 * (1.0 - eta) * xi;
      g10 += c0 * eta * (1.0 - xi);
      g11 += c0 * eta * xi;
    }
  }
  double* o = part + (size_t)e * 4;
  o[0] = g00;
  o[1] = g01;
  o[2] = g10;
  o[3] = g11;
}

// node (i, j) adds the terms of its (up to four) elements in a fixed order
__global__ void __launch_bounds__(256) k_deg_node_gather(const double* __restrict__ part, int n,
                                                         double* __restrict__ out) {
  const int n1 = n + 1;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n1 * n1) return;
  const int i = d % n1, j = d / n1;
  double v = 0.0;
  if (i < n && j < n) v += part[((size_t)j * n + i) * 4 + 0];
  if (i > 0 && j < n) v += part[((size_t)j * n + i - 1) * 4 + 1];
  if (i < n && j > 0) v += part[((size_t)(j - 1) * n + i) * 4 + 2];
  if (i > 0 && j > 0) v += part[((size_t)(j - 1) * n + i - 1) * 4 + 3];
  out[d] = v;
}

// per element, the largest Darcy speed |K (grad p + s rho_g g e_y)| /
// (mu_g phi) and the largest injection rate q_inj / phi over its Gauss points
// (the step-size rule's two maxima), to out[e] and out[n^2 + e]
template <int P>
__global__ void __launch_bounds__(128) k_deg_cfl(DegArgs a, double inv_mu_g, double* __restrict__ out) {
  constexpr int Q = P + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = a.n * a.n;
  if (e >= ne) return;
  const int ex = e % a.n, ey = e / a.n, n1 = a.n + 1;
  double pp[Q][Q];
#pragma unroll
  for (int b = 0; b < Q; ++b)
#pragma unroll
    for (int c = 0; c < Q; ++c) pp[b][c] = a.P[(size_t)(ey + b) * a.nb + ex + c];
  const double* Bx = a.B + (size_t)ex * Q * Q;
  const double* dBx = a.dB + (size_t)ex * Q * Q;
  const double* By = a.B + (size_t)ey * Q * Q;
  const double* dBy = a.dB + (size_t)ey * Q * Q;
  const double k00 = a.K[(size_t)ey * n1 + ex], k01 = a.K[(size_t)ey * n1 + ex + 1];
  const double k10 = a.K[(size_t)(ey + 1) * n1 + ex], k11 = a.K[(size_t)(ey + 1) * n1 + ex + 1];
  double f00 = a.phi_c, f01 = a.phi_c, f10 = a.phi_c, f11 = a.phi_c;
  if (a.phi) {
    f00 = a.phi[(size_t)ey * n1 + ex];
    f01 = a.phi[(size_t)ey * n1 + ex + 1];
    f10 = a.phi[(size_t)(ey + 1) * n1 + ex];
    f11 = a.phi[(size_t)(ey + 1) * n1 + ex + 1];
  }
  double vmax = 0.0, smax = 0.0;
  for (int qy = 0; qy < Q; ++qy) {
    const double eta = a.xi[qy];
    for (int qx = 0; qx < Q; ++qx) {
      const double xi = a.xi[qx];
      double px = 0.0, py = 0.0;
#pragma unroll
      for (int b = 0; b < Q; ++b) {
        double pb = 0.0, pdb = 0.0;
#pragma unroll
        for (int c = 0; c < Q; ++c) {
          pb += pp[b][c] * Bx[c * Q + qx];
          pdb += pp[b][c] * dBx[c * Q + qx];
        }
        px += By[b * Q + qy] * pdb;
        py += dBy[b * Q + qy] * pb;
      }
      const double Kq = (1.0 - eta) * ((1.0 - xi) * k00 + xi * k01) + eta * ((1.0 - xi) * k10 + xi * k11);
      const double phq = (1.0 - eta) * ((1.0 - xi) * f00 + xi * f01) + eta * ((1.0 - xi) * f10 + xi * f11);
      const double fx = Kq * px, fy = Kq * (py + a.grav_term);
      vmax = fmax(vmax, sqrt(fx * fx + fy * fy) * inv_mu_g / phq);
      double qi = 0.0;
      for (int k = 0; k < a.n_src; ++k)
        if (a.kind[k] == 0)
          qi += a.rate[k] * a.g[((size_t)(0 * a.n_src + k) * a.n + ex) * Q + qx] *
                a.g[((size_t)(1 * a.n_src + k) * a.n + ey) * Q + qy];
      smax = fmax(smax, qi / phq);
    }
  }
  out[e] = vmax;
  out[ne + e] = smax;
}

// the largest of each of the two per-element columns (one block)
__global__ void __launch_bounds__(1024) k_deg_max2(const double* __restrict__ v, int ne, double* out) {
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    a = fmax(a, v[e]);
    b = fmax(b, v[ne + e]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = a;
    red[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x + 31) / 32; ++i) {
      a = fmax(a, red[0][i]);
      b = fmax(b, red[1][i]);
    }
    out[0] = a;
    out[1] = b;
  }
}

// the per-element source terms summed over the elements in a fixed order:
// block j sums column j of psrc [ne][ncol]
__global__ void __launch_bounds__(256) k_deg_colsum(const double* __restrict__ psrc, int ne, int ncol, double* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) v += psrc[(size_t)e * ncol + blockIdx.x];
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// One degree of freedom (j, i): the local terms of the elements (ey, ex) with
// ey in [j - p, j], ex in [i - p, i], added in a fixed order
template <int P>
__global__ void __launch_bounds__(256) k_deg_gather(const double* __restrict__ part, int n, double* __restrict__ R) {
  constexpr int Q = P + 1;
  const int nb = n + P;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nb * nb) return;
  const int i = d % nb, j = d / nb;
  double v = 0.0;
  for (int ey = j - P; ey <= j; ++ey) {
    if (ey < 0 || ey >= n) continue;
    for (int ex = i - P; ex <= i; ++ex) {
      if (ex < 0 || ex >= n) continue;
      v += part[((size_t)ey * n + ex) * Q * Q + (j - ey) * Q + (i - ex)];
    }
  }
  R[d] = v;
}

// M x = r along lines of nb values, in place: line t starts at R + t * lstride
// and steps by estride.  L[k][l] = L_{l, l-k} (k = 1..p) of the unit lower
// factor, dinv[l] = 1 / D_l.
template <int P>
__global__ void __launch_bounds__(128) k_deg_lines(double* R, int nb, int nlines, size_t lstride, size_t estride,
                                                   const double* __restrict__ L, const double* __restrict__ dinv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlines) return;
  double* x = R + (size_t)t * lstride;
  double y[P];  // the last p values of the forward (or backward) recurrence
#pragma unroll
  for (int k = 0; k < P; ++k) y[k] = 0.0;
  for (int l = 0; l < nb; ++l) {
    double v = x[(size_t)l * estride];
#pragma unroll
    for (int k = 1; k <= P; ++k) v -= L[(size_t)(k - 1) * nb + l] * y[k - 1];
#pragma unroll
    for (int k = P - 1; k > 0; --k) y[k] = y[k - 1];
    y[0] = v;
    x[(size_t)l * estride] = v * dinv[l];
  }
#pragma unroll
  for (int k = 0; k < P; ++k) y[k] = 0.0;
  for (int l = nb - 1; l >= 0; --l) {
    double v = x[(size_t)l * estride];
#pragma unroll
    for (int k = 1; k <= P; ++k)
      if (l + k < nb) v -= L[(size_t)(k - 1) * nb + l + k] * y[k - 1];
#pragma unroll
    for (int k = P - 1; k > 0; --k) y[k] = y[k - 1];
    y[0] = v;
    x[(size_t)l * estride] = v;
  }
}

// int S = sum_j sum_i Iw_j Iw_i S_ji, one block, a fixed order
__global__ void __launch_bounds__(1024) k_deg_mass(const double* __restrict__ S, int nb, const double* __restrict__ Iw,
                                                   double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (size_t d = threadIdx.x; d < (size_t)nb * nb; d += blockDim.x) m += Iw[d / nb] * Iw[d % nb] * S[d];
  const double tot = block_sum(m, red);
  if (threadIdx.x == 0) *out = tot;
}

// ---------------------------------------------------------------- host tables

// Gauss-Legendre rule with q points on [0, 1]: the roots of the Legendre
// polynomial P_q by Newton's method (three-term recurrence for P_q and its
// derivative), weights 1 / ((1 - t^2) P_q'(t)^2) on [0, 1].
void gauss_legendre01(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (t * p1 - p0) / (t * t - 1.0);
      const double step = p1 / dp;
      t -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= q; ++k) {
      const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = q * (t * p1 - p0) / (t * t - 1.0);
    x[q - 1 - i] = 0.5 * (t + 1.0);  // ascending
    w[q - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Cox-de Boor: the B-spline i of degree k on the knots t, at x (0/0 read as 0)
double bspline(const std::vector<double>& t, int i, int k, double x) {
  if (k == 0) return (t[i] <= x && x < t[i + 1]) ? 1.0 : 0.0;
  double v = 0.0;
  const double d1 = t[i + k] - t[i], d2 = t[i + k + 1] - t[i + 1];
  if (d1 > 0) v += (x - t[i]) / d1 * bspline(t, i, k - 1, x);
  if (d2 > 0) v += (t[i + k + 1] - x) / d2 * bspline(t, i + 1, k - 1, x);
  return v;
}
// its derivative: k (N_{i,k-1} / (t_{i+k} - t_i) - N_{i+1,k-1} / (t_{i+k+1} - t_{i+1}))
double bspline_d(const std::vector<double>& t, int i, int k, double x) {
  double v = 0.0;
  const double d1 = t[i + k] - t[i], d2 = t[i + k + 1] - t[i + 1];
  if (d1 > 0) v += k / d1 * bspline(t, i, k - 1, x);
  if (d2 > 0) v -= k / d2 * bspline(t, i + 1, k - 1, x);
  return v;
}

cudaError_t wait_stream_for(cudaStream_t st, double seconds) {
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
}  // namespace adsgb

struct ads_degree_plan {
  int p = 0, n = 0, nb = 0;
  adsgb::DegArgs args{};              // everything but the per-call fields
  double* dev = nullptr;              // one allocation: tables, local terms, mass
  double *B = nullptr, *dB = nullptr, *g = nullptr, *L = nullptr, *dinv = nullptr, *Iw = nullptr;
  double *part = nullptr, *mass = nullptr;
  double *part2 = nullptr, *psrc = nullptr, *work = nullptr, *dsrc = nullptr;  // the vector-Jacobian product
};

using adsgb::DegArgs;

namespace {
// the fixed-order gather of an element-term array into (n+p)^2 coefficients
void deg_gather(const ads_degree_plan* pl, const double* part, double* out, cudaStream_t st) {
  using namespace adsgb;
  const int nd = pl->nb * pl->nb, g = (nd + 255) / 256;
  switch (pl->p) {
    case 2: k_deg_gather<2><<<g, 256, 0, st>>>(part, pl->n, out); break;
    case 3: k_deg_gather<3><<<g, 256, 0, st>>>(part, pl->n, out); break;
    default: k_deg_gather<4><<<g, 256, 0, st>>>(part, pl->n, out); break;
  }
}
// x <- M^-1 x in place: the banded solves along x (rows nb apart, entries
// adjacent), then along y
void deg_mass_solve(const ads_degree_plan* pl, double* x, cudaStream_t st) {
  using namespace adsgb;
  const int nb = pl->nb, g = (nb + 127) / 128;
  auto k = pl->p == 2 ? k_deg_lines<2> : (pl->p == 3 ? k_deg_lines<3> : k_deg_lines<4>);
  k<<<g, 128, 0, st>>>(x, nb, nb, (size_t)nb, 1, pl->L, pl->dinv);
  k<<<g, 128, 0, st>>>(x, nb, nb, 1, (size_t)nb, pl->L, pl->dinv);
}
}  // namespace

extern "C" ads_status ads_degree_plan_create(const ads_params* params, int degree, ads_degree_plan** out) {
  using namespace adsgb;
  if (!out) return ADS_ERR_INVALID_ARG;
  *out = nullptr;
  const ads_status v = validate_params(params, nullptr);
  if (v != ADS_OK) return v;
  if (params->dim != 2 || params->ads_dtype != ADS_F64) return ADS_ERR_UNSUPPORTED;
  if (degree < 2 || degree > kMaxDeg) return ADS_ERR_INVALID_ARG;
  if (params->n > kMaxDegN) return ADS_ERR_INVALID_ARG;
  const int p = degree, q = p + 1, n = params->n, nb = n + p;
  const double h = 1.0 / n;
  // knots: p + 1 zeros, the interior nodes, p + 1 ones
  std::vector<double> t(n + 2 * p + 1);
  for (int k = 0; k < (int)t.size(); ++k) t[k] = k <= p ? 0.0 : (k >= n + p ? 1.0 : (double)(k - p) / n);
  double xq[kMaxDeg + 1], wq[kMaxDeg + 1];
  gauss_legendre01(q, xq, wq);
  // values and derivatives of functions e .. e + p on element e at its points
  std::vector<double> B((size_t)n * q * q), dB((size_t)n * q * q);
  for (int e = 0; e < n; ++e)
    for (int a = 0; a < q; ++a)
      for (int k = 0; k < q; ++k) {
        const double x = (e + xq[k]) * h;
        B[((size_t)e * q + a) * q + k] = bspline(t, e + a, p, x);
        dB[((size_t)e * q + a) * q + k] = bspline_d(t, e + a, p, x);
      }
  // banded mass matrix Mb[k][i] = M_{i, i+k} (k = 0..p) and the basis integrals
  std::vector<double> Mb((size_t)q * nb, 0.0), Iw(nb, 0.0);
  for (int e = 0; e < n; ++e)
    for (int k = 0; k < q; ++k) {
      const double wk = wq[k] * h;
      for (int a = 0; a < q; ++a) {
        const double ba = B[((size_t)e * q + a) * q + k];
        Iw[e + a] += wk * ba;
        for (int c = a; c < q; ++c) Mb[(size_t)(c - a) * nb + e + a] += wk * ba * B[((size_t)e * q + c) * q + k];
      }
    }
  // M = L D L^T, L unit lower with bandwidth p: Lf[k][l] = L_{l, l-k}
  std::vector<double> Lf((size_t)p * nb, 0.0), D(nb, 0.0), dinv(nb, 0.0);
  auto Lget = [&](int l, int k) { return k == 0 ? 1.0 : Lf[(size_t)(k - 1) * nb + l]; };
  for (int l = 0; l < nb; ++l) {
    for (int k = std::min(p, l); k >= 1; --k) {
      double v = Mb[(size_t)k * nb + (l - k)];  // M_{l-k, l}
      for (int j = k + 1; j <= std::min(p, l); ++j) v -= Lget(l, j) * D[l - j] * Lget(l - k, j - k);
      Lf[(size_t)(k - 1) * nb + l] = v / D[l - k];
    }
    double d = Mb[l];
    for (int j = 1; j <= std::min(p, l); ++j) d -= Lget(l, j) * Lget(l, j) * D[l - j];
    if (!(d > 0)) return ADS_ERR_INVALID_ARG;  // M is SPD; a zero pivot means a broken table
    D[l] = d;
    dinv[l] = 1.0 / d;
  }
  // per-axis Gaussian factors: exp(-(x - c)^2 / (2 s^2)) / sqrt(2 pi s^2); their
  // product over the two axes is the normalised 2D Gaussian of each source
  const int ns = params->n_src;
  std::vector<double> g((size_t)2 * (ns > 0 ? ns : 1) * n * q, 0.0);
  for (int ax = 0; ax < 2; ++ax)
    for (int k = 0; k < ns; ++k) {
      const double c = params->src[k].center[ax], s = params->src[k].sigma;
      for (int e = 0; e < n; ++e)
        for (int j = 0; j < q; ++j) {
          const double x = (e + xq[j]) * h;
          g[((size_t)(ax * ns + k) * n + e) * q + j] =
              std::exp(-(x - c) * (x - c) / (2.0 * s * s)) / std::sqrt(2.0 * M_PI * s * s);
        }
    }
  auto* pl = new (std::nothrow) ads_degree_plan();
  if (!pl) return ADS_ERR_OOM;
  pl->p = p;
  pl->n = n;
  pl->nb = nb;
  const size_t nB = B.size(), ng = g.size(), nL = Lf.size(), npart = (size_t)n * n * q * q;
  const size_t nps = (size_t)n * n * 3 * (ns > 0 ? ns : 1);
  const size_t total = 2 * nB + ng + nL + 2 * (size_t)nb + 2 * npart + 1 + nps + (size_t)nb * nb + 3 * kMaxSrc;
  if (cudaMalloc(&pl->dev, total * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete pl;
    return ADS_ERR_OOM;
  }
  double* c = pl->dev;
  pl->B = c; c += nB;
  pl->dB = c; c += nB;
  pl->g = c; c += ng;
  pl->L = c; c += nL;
  pl->dinv = c; c += nb;
  pl->Iw = c; c += nb;
  pl->part = c; c += npart;
  pl->part2 = c; c += npart;
  pl->psrc = c; c += nps;
  pl->work = c; c += (size_t)nb * nb;
  pl->dsrc = c; c += 3 * kMaxSrc;
  pl->mass = c;
  bool ok = cudaMemcpy(pl->B, B.data(), nB * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->dB, dB.data(), nB * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->g, g.data(), ng * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->L, Lf.data(), nL * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->dinv, dinv.data(), (size_t)nb * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(pl->Iw, Iw.data(), (size_t)nb * 8, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(pl->dev);
    delete pl;
    return ADS_ERR_CUDA;
  }
  DegArgs& a = pl->args;
  a.n = n;
  a.nb = nb;
  a.n_src = ns;
  a.h2 = h * h;
  for (int k = 0; k < q; ++k) {
    a.wq[k] = wq[k];
    a.xi[k] = xq[k];
  }
  a.B = pl->B;
  a.dB = pl->dB;
  a.g = pl->g;
  for (int k = 0; k < ns; ++k) {
    a.rate[k] = params->src[k].rate;
    a.kind[k] = params->src[k].kind;
    a.cen[k][0] = params->src[k].center[0];
    a.cen[k][1] = params->src[k].center[1];
    a.sig[k] = params->src[k].sigma;
  }
  a.inv_mu_g = 1.0 / params->mu_g;
  a.inv_mu_w = 1.0 / params->mu_w;
  a.grav_term = params->grav_sign * params->rho_g * params->grav;
  a.phi_c = params->phi;
  a.part = pl->part;
  a.part2 = pl->part2;
  a.psrc = pl->psrc;
  *out = pl;
  return ADS_OK;
}

extern "C" ads_status ads_degree_step(ads_degree_plan* pl, const double* d_K, const double* d_phi,
                                      const double* d_S, const double* d_P, double dt, double* d_S_out,
                                      void* stream) {
  using namespace adsgb;
  if (!pl || !d_K || !d_S || !d_P || !d_S_out) return ADS_ERR_INVALID_ARG;
  if (!(dt > 0) || !std::isfinite(dt)) return ADS_ERR_INVALID_ARG;
  if (d_S_out == d_S || d_S_out == d_P) return ADS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DegArgs a = pl->args;
  a.K = d_K;
  a.phi = d_phi;
  a.S = d_S;
  a.P = d_P;
  a.dt = dt;
  const int n = pl->n, ne = n * n;
  switch (pl->p) {
    case 2: k_deg_elem<2><<<(ne + 127) / 128, 128, 0, st>>>(a); break;
    case 3: k_deg_elem<3><<<(ne + 127) / 128, 128, 0, st>>>(a); break;
    default: k_deg_elem<4><<<(ne + 127) / 128, 128, 0, st>>>(a); break;
  }
  deg_gather(pl, pl->part, d_S_out, st);
  deg_mass_solve(pl, d_S_out, st);
  return cudaGetLastError() == cudaSuccess ? ADS_OK : ADS_ERR_CUDA;
}

extern "C" ads_status ads_degree_step_vjp(ads_degree_plan* pl, const double* d_K, const double* d_phi,
                                          const double* d_S, const double* d_P, double dt, const double* d_lambda,
                                          double* d_gS, double* d_gP, double* h_gsrc, void* stream) {
  using namespace adsgb;
  if (!pl || !d_K || !d_S || !d_P || !d_lambda || !d_gS || !d_gP) return ADS_ERR_INVALID_ARG;
  if (!(dt > 0) || !std::isfinite(dt)) return ADS_ERR_INVALID_ARG;
  if (d_gS == d_gP || d_gS == d_S || d_gS == d_P || d_gS == d_lambda || d_gP == d_S || d_gP == d_P ||
      d_gP == d_lambda)
    return ADS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = pl->n, nb = pl->nb, ne = n * n, ns = pl->args.n_src;
  // mu = M^-1 lambda
  if (cudaMemcpyAsync(pl->work, d_lambda, (size_t)nb * nb * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return ADS_ERR_CUDA;
  }
  deg_mass_solve(pl, pl->work, st);
  DegArgs a = pl->args;
  a.K = d_K;
  a.phi = d_phi;
  a.S = d_S;
  a.P = d_P;
  a.dt = dt;
  a.mu = pl->work;
  const int g = (ne + 127) / 128;
  switch (pl->p) {
    case 2: k_deg_vjp<2><<<g, 128, 0, st>>>(a); break;
    case 3: k_deg_vjp<3><<<g, 128, 0, st>>>(a); break;
    default: k_deg_vjp<4><<<g, 128, 0, st>>>(a); break;
  }
  deg_gather(pl, pl->part, d_gS, st);
  deg_gather(pl, pl->part2, d_gP, st);
  if (ns > 0) k_deg_colsum<<<3 * ns, 256, 0, st>>>(pl->psrc, ne, 3 * ns, pl->dsrc);
  if (cudaGetLastError() != cudaSuccess) return ADS_ERR_CUDA;
  if (h_gsrc && ns > 0) {
    if (cudaMemcpyAsync(h_gsrc, pl->dsrc, 3 * ns * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      cudaGetLastError();
      return ADS_ERR_CUDA;
    }
    const cudaError_t e = wait_stream_for(st, 10.0);
    if (e == cudaErrorNotReady) return ADS_ERR_TIMEOUT;
    if (e != cudaSuccess) return ADS_ERR_CUDA;
  }
  return ADS_OK;
}

extern "C" ads_status ads_degree_project(ads_degree_plan* pl, const double* d_nodal, double* d_out, void* stream) {
  using namespace adsgb;
  if (!pl || !d_nodal || !d_out) return ADS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int ne = pl->n * pl->n, g = (ne + 127) / 128;
  switch (pl->p) {
    case 2: k_deg_proj<2><<<g, 128, 0, st>>>(pl->args, d_nodal); break;
    case 3: k_deg_proj<3><<<g, 128, 0, st>>>(pl->args, d_nodal); break;
    default: k_deg_proj<4><<<g, 128, 0, st>>>(pl->args, d_nodal); break;
  }
  deg_gather(pl, pl->part, d_out, st);
  deg_mass_solve(pl, d_out, st);
  return cudaGetLastError() == cudaSuccess ? ADS_OK : ADS_ERR_CUDA;
}

extern "C" ads_status ads_degree_project_vjp(ads_degree_plan* pl, const double* d_g, double* d_gnodal,
                                             void* stream) {
  using namespace adsgb;
  if (!pl || !d_g || !d_gnodal || d_g == d_gnodal) return ADS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = pl->nb, n = pl->n, ne = n * n;
  if (cudaMemcpyAsync(pl->work, d_g, (size_t)nb * nb * sizeof(double), cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return ADS_ERR_CUDA;
  }
  deg_mass_solve(pl, pl->work, st);
  const int g = (ne + 127) / 128;
  switch (pl->p) {
    case 2: k_deg_proj_vjp<2><<<g, 128, 0, st>>>(pl->args, pl->work, pl->part); break;
    case 3: k_deg_proj_vjp<3><<<g, 128, 0, st>>>(pl->args, pl->work, pl->part); break;
    default: k_deg_proj_vjp<4><<<g, 128, 0, st>>>(pl->args, pl->work, pl->part); break;
  }
  const int n1 = n + 1;
  k_deg_node_gather<<<(n1 * n1 + 255) / 256, 256, 0, st>>>(pl->part, n, d_gnodal);
  return cudaGetLastError() == cudaSuccess ? ADS_OK : ADS_ERR_CUDA;
}

extern "C" ads_status ads_degree_cfl_dt(ads_degree_plan* pl, const double* d_K, const double* d_phi,
                                        const double* d_P, double cfl, double src_frac, double dt_cap, double* dt,
                                        void* stream) {
  using namespace adsgb;
  if (!pl || !d_K || !d_P || !dt) return ADS_ERR_INVALID_ARG;
  if (!(cfl > 0) || !std::isfinite(cfl) || !(src_frac > 0) || !std::isfinite(src_frac) || !(dt_cap > 0))
    return ADS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DegArgs a = pl->args;
  a.K = d_K;
  a.phi = d_phi;
  a.P = d_P;
  const int ne = pl->n * pl->n, g = (ne + 127) / 128;
  switch (pl->p) {
    case 2: k_deg_cfl<2><<<g, 128, 0, st>>>(a, a.inv_mu_g, pl->part); break;
    case 3: k_deg_cfl<3><<<g, 128, 0, st>>>(a, a.inv_mu_g, pl->part); break;
    default: k_deg_cfl<4><<<g, 128, 0, st>>>(a, a.inv_mu_g, pl->part); break;
  }
  k_deg_max2<<<1, 1024, 0, st>>>(pl->part, ne, pl->dsrc);
  if (cudaGetLastError() != cudaSuccess) return ADS_ERR_CUDA;
  double mx[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(mx, pl->dsrc, sizeof(mx), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    cudaGetLastError();
    return ADS_ERR_CUDA;
  }
  const cudaError_t e = wait_stream_for(st, 10.0);
  if (e == cudaErrorNotReady) return ADS_ERR_TIMEOUT;
  if (e != cudaSuccess) return ADS_ERR_CUDA;
  if (!std::isfinite(mx[0]) || !std::isfinite(mx[1])) return ADS_ERR_NONFINITE;
  // dt = min(dt_cap, cfl h / v_max, src_frac / s_max), the maxima over the Gauss points
  double d = dt_cap;
  if (mx[0] > 0) d = std::min(d, cfl / pl->n / mx[0]);
  if (mx[1] > 0) d = std::min(d, src_frac / mx[1]);
  *dt = d;
  return ADS_OK;
}

extern "C" ads_status ads_degree_mass(ads_degree_plan* pl, const double* d_S, double* mass, void* stream) {
  using namespace adsgb;
  if (!pl || !d_S || !mass) return ADS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_deg_mass<<<1, 1024, 0, st>>>(d_S, pl->nb, pl->Iw, pl->mass);
  if (cudaGetLastError() != cudaSuccess) return ADS_ERR_CUDA;
  if (cudaMemcpyAsync(mass, pl->mass, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    cudaGetLastError();
    return ADS_ERR_CUDA;
  }
  const cudaError_t e = wait_stream_for(st, 10.0);
  if (e == cudaErrorNotReady) return ADS_ERR_TIMEOUT;
  return e == cudaSuccess ? ADS_OK : ADS_ERR_CUDA;
}

extern "C" int ads_degree_coeffs(const ads_degree_plan* pl) { return pl ? pl->nb : 0; }

extern "C" void ads_degree_plan_destroy(ads_degree_plan* pl) {
  if (!pl) return;
  cudaFree(pl->dev);
  delete pl;
}

// Kernel argument structs and launcher declarations shared by the adsgb
// translation units.  Every launcher enqueues on the given stream and
// returns the launch status.
#pragma once
#include <cstring>
#include <vector>

#include "common.cuh"

namespace adsgb {

// ---------------------------------------------------------------------------
// Grouped launches (the batched form of a training iteration over several
// contexts of the same shape): one launch runs the CTAs of every context's
// own launch of a kernel.  CTA b of the grouped grid plays CTA cta[b].y of
// context cta[b].x's launch, whose grid is grid[cta[b].x]; the contexts'
// arguments come from a device table.  A context's results are those of its
// own launch: the same CTAs do the same work.
// ---------------------------------------------------------------------------
struct GroupMap {
  const int2* cta;  // [grouped CTAs] (context, CTA of that context's launch)
  const int* grid;  // [contexts] CTAs of the context's launch
};

// a device table of per-context arguments and its CTA map, in one allocation
template <typename A>
struct DevGroup {
  A* tab = nullptr;
  GroupMap map{nullptr, nullptr};
  int nctx = 0, nctas = 0;
  void* mem = nullptr;
};
template <typename A>
cudaError_t dev_group_create(DevGroup<A>& g, const A* args, const int* grids, int n) {
  int total = 0;
  for (int k = 0; k < n; ++k) total += grids[k] > 0 ? grids[k] : 0;
  const size_t tab_b = ((sizeof(A) * (size_t)n + 255) / 256) * 256;
  const size_t grid_b = ((sizeof(int) * (size_t)n + 255) / 256) * 256;
  const size_t map_b = sizeof(int2) * (size_t)(total > 0 ? total : 1);
  std::vector<unsigned char> h(tab_b + grid_b + map_b, 0);
  std::memcpy(h.data(), args, sizeof(A) * (size_t)n);
  int* gh = reinterpret_cast<int*>(h.data() + tab_b);
  int2* mh = reinterpret_cast<int2*>(h.data() + tab_b + grid_b);
  int b = 0;
  for (int k = 0; k < n; ++k) {
    gh[k] = grids[k] > 0 ? grids[k] : 0;
    for (int c = 0; c < gh[k]; ++c) mh[b++] = make_int2(k, c);
  }
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, h.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(mem, h.data(), h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(mem);
    return e;
  }
  unsigned char* d = static_cast<unsigned char*>(mem);
  g.mem = mem;
  g.tab = reinterpret_cast<A*>(d);
  g.map = GroupMap{reinterpret_cast<const int2*>(d + tab_b + grid_b), reinterpret_cast<const int*>(d + tab_b)};
  g.nctx = n;
  g.nctas = total;
  return cudaSuccess;
}
template <typename A>
void dev_group_free(DevGroup<A>& g) {
  if (g.mem) cudaFree(g.mem);
  g = DevGroup<A>{};
}

// ---------------------------------------------------------------------------
// per-axis tables (identical axes: uniform open knot vector, degree 2)
// ---------------------------------------------------------------------------
template <typename T>
struct AxisTabs {
  const T* B;      // [n][3 local fn][3 gauss pt]  basis values
  const T* dB;     // [n][3][3]                    d/dx (physical)
  const T* l1;     // [n+4] LDL^T of the 1D mass matrix: L[l][l-1] (0-padded)
  const T* l2;     // [n+4] L[l][l-2]
  const T* dinv;   // [n+2] 1/D[l]
  const T* Iw;     // [n+2] int B_l
  const T* gsrc;   // [3 axes][kMaxSrc][n][3] per-axis Gaussian factor at Gauss points
  const T* gnode;  // [3 axes][kMaxSrc][n+1] per-axis Gaussian factor at nodes
  const void* ytab = nullptr;  // FP32 2D: packed y-sweep factor rows (launch_ysweep_table)
};

template <typename T>
struct QuadArgs {
  int dim, n, nb;        // nb = n + 2
  T h;
  const T* S;            // coefficients (n+2)^d
  const T* P;            // coefficients (n+2)^d
  const T* K;            // nodal (n+1)^d
  const T* phi;          // nodal (n+1)^d or nullptr
  T phi_c;
  const T* nodal;        // projection: nodal values (n+1)^d
  AxisTabs<T> ax;
  int n_src;
  T rate[kMaxSrc];
  int kind[kMaxSrc];
  T inv_mu_g, inv_mu_w;
  T grav_term;           // grav_sign * rho_g * grav
  T kz;                  // vertical permeability ratio (3D)
  const double* dt;      // device step size
};

// ---- init (FP64, one-off) ----
cudaError_t launch_axis_init(int n, const double* centers /*[kMaxSrc][3]*/, const double* sigmas,
                             int n_src, double* B, double* dB, double* l1, double* l2, double* dinv,
                             double* Iw, double* gsrc, double* gnode, double* tmp /*3(n+4)*/,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_convert(const double* src, T* dst, size_t count, cudaStream_t st);
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, size_t count, cudaStream_t st);

// ---- saturation step ----
// Fused quadrature (MODE 0: saturation RHS of Eq. 10b; MODE 1: L2
// projection RHS of nodal values) + x-direction mass solve for a strip of
// `re` (>= 2) element rows.  Rows owned by the strip go to Xm, the two rows
// it shares with the next strip to Xs (both with row stride ldx, a multiple
// of 16 bytes; ldx >= n + 2).
template <typename T>
cudaError_t launch_quad_xsweep(const QuadArgs<T>& a, int mode, int re, T* Xm, T* Xs, int ldx,
                               double* src_part, cudaStream_t st);
// y-direction sweep of Xm plus the spill rows Xs into `out` (row stride n+2),
// with per-block partials of int S; sets bit 8 of flags if a bulk copy wait
// timed out.  FP32 with strips of quad_rows rows needs a.ax.ytab.
template <typename T>
cudaError_t launch_ysweep(const QuadArgs<T>& a, int re, const T* Xm, const T* Xs, int ldx, T* out,
                          double* mass_part, int* flags, cudaStream_t st);
template <typename T>
cudaError_t launch_zsolve(const QuadArgs<T>& a, T* X, double* mass_part, cudaStream_t st);
int quad_rows(int n, size_t esize);  // element rows per strip of the 2D quadrature
int quad_blocks(int dim, int n, int re);
// strips per thread-block cluster of the 2D quadrature: a cluster adds the
// rows its strips share through distributed shared memory, so only one pair of
// spill rows per cluster (every re * quad_cluster(re) = 8 rows for re = 2, 4)
// goes through Xs
int quad_cluster(int re);
int ysolve_blocks(int dim, int n);       // partial-sum slots (largest layout of either precision)
// packed FP32 factor rows for the 2D y sweep, built once per mesh from the
// FP32 LDL^T factors
size_t ysweep_table_bytes(int n);
cudaError_t launch_ysweep_table(int n, const float* l1, const float* l2, const float* dinv, const float* Iw,
                                void* tab, cudaStream_t st);
int ysweep_blocks(int n, size_t esize);  // slots one 2D y sweep writes
int sweep_ld(int n);  // row stride of the 2D sweep intermediates
// mass bookkeeping: mode 0 = set int S from partials; mode 1 = step update
// Adam state reset: t = 0 and the running powers of the betas to 1
cudaError_t launch_adam_reset(int* t, double* bc, cudaStream_t st);
cudaError_t launch_mass_finalize(const double* mass_part, int nmass, const double* src_part,
                                 int nsrc, int mode, double* stats, int* flags, cudaStream_t st);
template <typename T>
cudaError_t launch_mass(const QuadArgs<T>& a, const T* S, double* mass_part, cudaStream_t st);
template <typename T>
cudaError_t launch_cfl(const QuadArgs<T>& a, double* part /*2 per block*/, cudaStream_t st);
int cfl_blocks(int dim, int n);
cudaError_t launch_cfl_finalize(const double* part, int nblk, double cfl, double src_frac,
                                double dt_cap, double h, double* dt, int* flags, cudaStream_t st);

// ---- 3D saturation step ----
template <typename T>
cudaError_t launch_quad3d(const QuadArgs<T>& a, int mode, T* Cbuf, T* R, double* src_part,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_solve3d(const QuadArgs<T>& a, T* X, double* mass_part, cudaStream_t st);
template <typename T>
cudaError_t launch_mass3d(const QuadArgs<T>& a, const T* S, double* mass_part, cudaStream_t st);
template <typename T>
cudaError_t launch_cfl3d(const QuadArgs<T>& a, double* part, cudaStream_t st);
size_t elem3d_scratch(int n, size_t es);
int quad3d_blocks(int n);
int zsolve3d_blocks(int n);

// ---- CRVPINN ----
template <typename T, typename TA>
struct CrvArgs {
  int dim, N, M;         // N intervals, M = (N-1)^dim interior nodes
  T h;
  const TA* S;           // saturation coefficients (ADS precision)
  const TA* K;           // nodal permeability (ADS precision)
  AxisTabs<TA> ax;       // for the nodal source factors
  int n_src;
  double rate[kMaxSrc];
  int kind[kMaxSrc];
  double inv_mu_g, inv_mu_w, rho_w, rho_g, grav, kz;
  T* alpha;              // (N+1)^dim
  T* f;                  // M
};
template <typename T, typename TA>
cudaError_t launch_crv_coeffs(const CrvArgs<T, TA>& a, cudaStream_t st);
// loss finalisation fused into the adjoint stencil (part == nullptr: none)
struct LossFin {
  const double* part;
  int nparts;
  double* loss;
  double* log;
  int* t;
  double* bc;  // [1/(1 - beta_1^t), 1/(1 - beta_2^t), beta_1^t, beta_2^t]
  int* flags;
  int bump;
};
// grouped 2D stencil (FP32): a context's arguments as launch_stencil gives
// its kernel; stencil_blocks(N) CTAs per context
struct StencilArgs {
  int N;
  const float *alpha, *v, *f;
  float h2, scale;
  float* out;
  LossFin lf;
};
int stencil_blocks(int N);
cudaError_t launch_stencil_grouped(const StencilArgs* tab, GroupMap g, int nctas, cudaStream_t st);
// RES = A u + h^2 f (scale 1) or g = 2 A z (scale 2, f = nullptr)
template <typename T>
cudaError_t launch_stencil(int dim, int N, T kz, const T* alpha, const T* u, const T* f, T h2,
                           T scale, T* out, const LossFin* lf, cudaStream_t st);
// nodal array (N+1)^dim (ADS precision) from interior values (boundary 0)
template <typename T, typename TA>
cudaError_t launch_embed(int dim, int N, const T* u, TA* nodal, cudaStream_t st);

// Gram: sine transform matrix, per-mode tridiagonal inverse pivots
cudaError_t launch_gram_init(int dim, int N, double* Sdst, double* invd, cudaStream_t st);
template <typename T>
cudaError_t launch_gemm(int M, int Nn, int K, const T* A, int lda, const T* B, int ldb, T* C,
                        int ldc, T alpha, const T* dotB, double* dot_part, cudaStream_t st,
                        int batch = 1, long long sA = 0, long long sB = 0, long long sC = 0);
int gemm_blocks(int M, int Nn);
template <typename T>
cudaError_t launch_tridiag_cols(int nrows, int ncols, const T* invd, T* X, cudaStream_t st);
template <typename T>
cudaError_t launch_dot_partial(const T* a, const T* b, int n, double* part, int nblk, cudaStream_t st);
int dot_blocks(int n);
// loss finalize: loss = sum(part); writes loss, log ring, t += 1 and the
// Adam bias corrections
cudaError_t launch_loss_finalize(const double* part, int nblk, double* loss, double* loss_log,
                                 int* t, double* bc, int* flags, int bump_t, cudaStream_t st);

// ---- MLP ----
template <typename T>
struct MlpArgs {
  int din, width, npts, N, ld;  // ld: leading dimension of stored activations
  const T* theta;
  T* u;                         // [npts]
  T* acts;                      // [4][width][ld]
  const T* gu;                  // [npts] dL/du (backward)
  T* gpart;                     // [nblk][nparams]
  int nparams;
};
template <typename T>
cudaError_t launch_mlp_fwd(const MlpArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_mlp_bwd(const MlpArgs<T>& a, int nblk, cudaStream_t st);
int mlp_bwd_blocks(int npts, int width, int elem_bytes, int din);
template <typename T>
cudaError_t launch_grad_reduce_adam(const T* gpart, int nblk, int nparams, T* grad, T* theta,
                                    T* m, T* v, const double* bc, const double* lr, int do_update,
                                    cudaStream_t st);
// grouped (FP32): a context's arguments as launch_grad_reduce_adam gives its
// kernel; grad_adam_blocks(nparams) CTAs per context
struct AdamArgs {
  const float* gpart;
  int nblk, nparams;
  float *grad, *theta, *m, *v;
  const double *bc, *lr;
  int upd;
};
int grad_adam_blocks(int nparams);
cudaError_t launch_grad_adam_grouped(const AdamArgs* tab, GroupMap g, int nctas, cudaStream_t st);

// ---- MLP on tcgen05 tensor cores (BF16 operands, FP32 accumulation, width 64) ----
struct MlpTcArgs {
  int din, width, npts, N;
  const float* theta;     // FP32 master parameters
  float* u;               // [npts]
  unsigned char* acts;    // BF16 activations, [tile][4][128 x width] core-matrix tiles (nullable)
  unsigned char* wimage;  // forward: weight image, mlp_tc_fwd_image_bytes(width), 16-byte aligned;
                          // rewritten from theta by every forward launch
  int* wimage_ctr = nullptr;  // forward: tile-group counter at the end of the image (set by the launcher)
  const float* gu;        // [npts] dL/du
  float* gpart;           // [nblk][nparams]
  int nparams;
  int* flags;             // bit 8: a tensor-core wait timed out
  int min_tiles = 1;      // forward: fewest 128-point tiles per CTA (a smaller grid)
  // 128-point tiles of this launch: [tile0, tile0 + tile_count) (tile_count <= 0:
  // to the last tile).  acts holds the launch's tiles from its start, tile0 first.
  int tile0 = 0, tile_count = 0;
};
// Gram solve by sine transforms computed with FFTs (2D, N a power of two,
// 8 <= N <= 2048): tables, partial count of the loss, and the three passes
bool gram_fft_supported(int dim, int N);
int gram_fft_dot_parts(int N, int dim = 2);
template <typename T>
cudaError_t gram_fft_tables(int N, T* tw /*4N: 2N complex twiddles*/, T* lam /*N-1*/);
// pass 0 with u != nullptr first computes RES = A u + h^2 f (written to
// res_out) and transforms it (res is then unused)
template <typename T>
cudaError_t launch_gram_fft(int pass, int N, const T* res, T* work, T* z, const T* tw, const T* lam,
                            T h2, double* dot_part, cudaStream_t st, const T* u = nullptr,
                            const T* alpha = nullptr, const T* f = nullptr, T* res_out = nullptr);

// grouped (2D, FP32): each of the three passes over several contexts in one
// launch, with the arguments launch_gram_fft gives the context's own pass
// (pass 0 forms the residual from u)
struct GramGroupEntry {
  int N;
  const float *u, *alpha, *f;
  float h2;
  float *res, *rhat, *z;
  const float *tw, *lam;
  double* dot_part;
};
struct GramGroup;
cudaError_t gram_group_create(const GramGroupEntry* e, int n, GramGroup** out);
cudaError_t launch_gram_group(const GramGroup* g, int pass, cudaStream_t st);
void gram_group_destroy(GramGroup* g);

// 3D: pass 0 = the x and y transforms of res into work, pass 2 = the inverse
// transforms of work into z (times h^2 (2/N)^2) with the loss partials; the
// z tridiagonal solves in between are the caller's (launch_tridiag_cols)
template <typename T>
cudaError_t launch_gram_fft3d(int pass, int N, const T* res, T* work, T* z, const T* tw, T h2,
                              double* dot_part, cudaStream_t st);

// the whole FP32 Gram solve (residual, the three transform passes, the
// partials of RES^T z, one per CTA) in one thread-block cluster, 8 <= N <= 128
struct GramClusterShape {
  int CL = 0, R = 0, P = 0, threads = 0;  // CL = 0: not available
  size_t smem = 0;
};
GramClusterShape gram_cluster_shape(int N);
cudaError_t launch_gram_cluster(const GramClusterShape& sh, int N, const float* u, const float* alpha,
                                const float* f, float h2, float* res_out, float* z, const float* tw,
                                const float* lam, double* dot_part, cudaStream_t st);

// the forward is two launches: the weight image from theta, then the network
cudaError_t launch_mlp_fwd_tc(const MlpTcArgs& a, cudaStream_t st);
constexpr int kMlpTcFwdLaunches = 2;
size_t mlp_tc_fwd_image_bytes(int width);
cudaError_t launch_mlp_bwd_tc(const MlpTcArgs& a, int nblk, cudaStream_t st);
size_t mlp_tc_acts_bytes(int npts, int width);
// backward CTAs (= gradient partial rows): one per SM at most, and at least
// `min_tiles` 128-point tiles per CTA
int mlp_tc_bwd_blocks(int npts, int width, int din, int min_tiles = 1);
// grouped (width 64): a context's table entry (its launch arguments, with
// the tile range and counter set) and its forward CTA count; which = 0: the
// weight images (grid: stage blocks x contexts), 1: the forwards, 2: the
// backwards (g maps each grouped CTA to its context's CTA / partial row)
MlpTcArgs mlp_tc_group_args(const MlpTcArgs& a, int* fwd_ctas);
cudaError_t launch_mlp_tc_grouped(int which, int din, const MlpTcArgs* tab, int nctx, GroupMap g, int nctas,
                                  cudaStream_t st);

// ---- diagnostics: one bounded mbarrier wait run to its limit (or completed,
// with arrive != 0); bit 8 goes to *word on expiry.  src16: 16 readable,
// 16-byte aligned device bytes (the probe's own bulk copy)
cudaError_t launch_wait_probe(const void* src16, unsigned long long limit_ns, int arrive, int* word,
                              cudaStream_t st);

// ---- Galerkin B-spline pressure (the plain method; 2D, FP64 arithmetic) ----
constexpr int kGalMaxN = 512;
template <typename TA>
struct GalArgs {
  int n;
  const TA* S;            // saturation coefficients (n+2)^2
  const TA* K;            // nodal permeability (n+1)^2
  const double* B;        // FP64 axis tables [n][3][3]
  const double* dB;
  const double* gsrc;     // FP64 per-axis source factors
  int n_src;
  double rate[kMaxSrc];
  int kind[kMaxSrc];
  double inv_mu_g, inv_mu_w, rho_w, rho_g, grav;
  double* work;           // galerkin_work_bytes(n)
  TA* P;                  // out: pressure coefficients (n+2)^2, boundary ring 0
  int* flags;             // bit 0 set when a pivot is not positive and finite
};
bool galerkin_supported(int dim, int n);
size_t galerkin_work_bytes(int n);
template <typename TA>
cudaError_t launch_galerkin_pressure(const GalArgs<TA>& a, cudaStream_t st);

}  // namespace adsgb

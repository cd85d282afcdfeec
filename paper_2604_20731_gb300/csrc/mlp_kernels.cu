// CRVPINN network on the collocation grid (Sec. 5: PINN(x_ij) replaces p),
// SIMT path for FP32 and FP64 parameters.
//
//   a_1 = tanh(W_1 x' + b_1), a_l = tanh(W_l a_{l-1} + b_l) (l = 2..4),
//   u = W_5 a_4 + b_5,  x' = 2 x - 1 on the interior nodes x = (ih, jh).
//
// Forward: a CTA holds a tile of P points; activations stay in shared memory
// as [feature][point] tiles, each hidden layer is a register-blocked
// (W x W) x (W x P) product; the activations are also written to HBM for the
// backward pass.  Backward (hand-written, same layout): delta_4 = W_5^T g
// (1 - a_4^2), dW_l = sum_p delta_l a_{l-1}^T, delta_{l-1} = (W_l^T delta_l)
// (1 - a_{l-1}^2); each persistent CTA accumulates the gradient of its tiles
// in its own row of a partial-gradient buffer (no atomics: the final sum over
// CTAs runs in a fixed order, fused with Adam).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace adsgb {

template <typename T>
ADS_D void ld4(const T* p, T v[4]);
template <>
ADS_D void ld4<float>(const float* p, float v[4]) {
  float4 f = *reinterpret_cast<const float4*>(p);
  v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
template <>
ADS_D void ld4<double>(const double* p, double v[4]) {
  double2 a = *reinterpret_cast<const double2*>(p);
  double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <typename T>
ADS_D void st4(T* p, const T v[4]);
template <>
ADS_D void st4<float>(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
ADS_D void st4<double>(double* p, const double v[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

constexpr int kMlpThreads = 256;

// interior point index -> coordinates mapped to [-1,1]
template <typename T, int DIN>
ADS_D void point_coords(int idx, int N, T c[3]) {
  const int m = N - 1;
  int i = idx % m + 1;
  int j = (idx / m) % m + 1;
  int k = idx / (m * m) + 1;
  const T invN = T(1) / T(N);
  c[0] = T(2) * T(i) * invN - T(1);
  c[1] = T(2) * T(j) * invN - T(1);
  c[2] = DIN == 3 ? T(2) * T(k) * invN - T(1) : T(0);
}

template <typename T, int W, int DIN, int P>
__global__ void __launch_bounds__(kMlpThreads) k_mlp_fwd(MlpArgs<T> a) {
  constexpr int PS = P + 4;  // padded row stride of the activation tiles
  constexpr bool ALLW = (3 * W * W * sizeof(T) <= 64 * 1024);  // all hidden weights resident
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ws = reinterpret_cast<T*>(smraw);   // ALLW ? [3][W][W] : [W][W]
  T* bufA = Ws + (ALLW ? 3 : 1) * W * W; // [W][PS]
  T* bufB = bufA + W * PS;               // [W][PS]
  T* xin = bufB + W * PS;                // [DIN][P]
  const int tid = threadIdx.x;
  const int ntiles = (a.npts + P - 1) / P;
  const T* th = a.theta;
  const int ob1 = W * DIN, o2 = ob1 + W;
  const int o5 = o2 + 3 * (W * W + W);
  constexpr int TP = 4, NPG = P / TP, NOG = kMlpThreads / NPG, TO = W / NOG;
  static_assert(TO * NOG == W, "tile mapping");
  const int pg = tid % NPG, og = tid / NPG;
  if (ALLW)
    for (int e = tid; e < 3 * W * W; e += kMlpThreads) {
      int l = e / (W * W), r = e % (W * W);
      Ws[e] = th[o2 + l * (W * W + W) + r];
    }
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int p0 = tile * P;
    for (int p = tid; p < P; p += kMlpThreads) {
      T c[3];
      point_coords<T, DIN>(min(p0 + p, a.npts - 1), a.N, c);
      for (int d = 0; d < DIN; ++d) xin[d * P + p] = c[d];
    }
    __syncthreads();
    for (int e = tid; e < W * P; e += kMlpThreads) {
      const int o = e / P, p = e % P;
      T z = th[ob1 + o];
#pragma unroll
      for (int d = 0; d < DIN; ++d) z += th[o * DIN + d] * xin[d * P + p];
      T v = tanh_any(z);
      bufA[o * PS + p] = v;
      if (a.acts) a.acts[(size_t)o * a.ld + p0 + p] = v;
    }
    for (int l = 0; l < 3; ++l) {
      const T* bl = th + o2 + l * (W * W + W) + W * W;
      __syncthreads();
      if (!ALLW) {
        for (int e = tid; e < W * W; e += kMlpThreads) Ws[e] = th[o2 + l * (W * W + W) + e];
        __syncthreads();
      }
      const T* Wl = ALLW ? Ws + l * W * W : Ws;
      T acc[TO][TP];
#pragma unroll
      for (int i = 0; i < TO; ++i)
#pragma unroll
        for (int j = 0; j < TP; ++j) acc[i][j] = T(0);
#pragma unroll 4
      for (int k = 0; k < W; k += 4) {
        T wv[TO][4], av[4][TP];
#pragma unroll
        for (int i = 0; i < TO; ++i) ld4<T>(&Wl[(og * TO + i) * W + k], wv[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) ld4<T>(&bufA[(k + j) * PS + pg * TP], av[j]);
#pragma unroll
        for (int i = 0; i < TO; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < TP; ++q) acc[i][q] += wv[i][j] * av[j][q];
      }
#pragma unroll
      for (int i = 0; i < TO; ++i) {
        const int o = og * TO + i;
        const T b = bl[o];
        T v[TP];
#pragma unroll
        for (int q = 0; q < TP; ++q) v[q] = tanh_any(acc[i][q] + b);
        st4<T>(&bufB[o * PS + pg * TP], v);
        if (a.acts) st4<T>(&a.acts[((size_t)(l + 1) * W + o) * a.ld + p0 + pg * TP], v);
      }
      T* tmp = bufA; bufA = bufB; bufB = tmp;
    }
    __syncthreads();
    for (int p = tid; p < P; p += kMlpThreads) {
      T z = th[o5 + W];
#pragma unroll 8
      for (int k = 0; k < W; ++k) z += th[o5 + k] * bufA[k * PS + p];
      if (p0 + p < a.npts) a.u[p0 + p] = z;
    }
    __syncthreads();
  }
}

// shared memory of the backward kernel with nbuf activation buffers
template <typename T, int W, int DIN, int P>
constexpr size_t bwd_bytes(int nbuf) {
  return sizeof(T) * (((3 * W * W * sizeof(T) <= 64 * 1024) ? 3 : 1) * W * W +
                      (2 + nbuf) * W * (P + 4) + P + DIN * P + (W + 1 + 3 * W + W * DIN + W));
}
// two activation buffers only if two CTAs still fit on an SM (or if even one
// buffer does not allow two)
template <typename T, int W, int DIN, int P>
constexpr int bwd_nbuf() {
  return (bwd_bytes<T, W, DIN, P>(2) <= 112 * 1024 || bwd_bytes<T, W, DIN, P>(1) > 112 * 1024) ? 2 : 1;
}

template <typename T>
ADS_D T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Backward pass.  Thread mappings are chosen so that shared-memory reads are
// conflict-free: in the dW product a thread owns rows o = og*TOd + i of
// delta (broadcast within a half-warp) and rows k = kg + NKG*j of the
// activations (consecutive rows across lanes); the delta product reads
// weight rows by broadcast and activation columns contiguously.  For W <= 64
// the hidden-layer dW of all the CTA's tiles accumulate in registers and are
// written once; the small gradients (output layer, biases, first layer) are
// warp reductions accumulated in shared memory by a fixed owner.
template <typename T, int W, int DIN, int P>
__global__ void __launch_bounds__(kMlpThreads) k_mlp_bwd(MlpArgs<T> a) {
  constexpr int PS = P + 4;
  constexpr bool ALLW = (3 * W * W * sizeof(T) <= 64 * 1024);
  constexpr bool REGACC = (W <= 64);
  constexpr int NBUF = bwd_nbuf<T, W, DIN, P>();
  constexpr int NWARP = kMlpThreads / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Ws = reinterpret_cast<T*>(smraw);   // ALLW ? [3][W][W] : [W][W]
  T* dA = Ws + (ALLW ? 3 : 1) * W * W;   // delta_l      [W][PS]
  T* dB = dA + W * PS;                   // delta_{l-1}  [W][PS]
  T* aBuf = dB + W * PS;                 // activations [NBUF][W][PS]
  T* gP = aBuf + NBUF * W * PS;          // [P]
  T* xin = gP + P;                       // [DIN][P]
  T* gsm = xin + DIN * P;                // small gradients
  T* g5 = gsm;                           // dW_5 [W]
  T* gb5 = g5 + W;                       // db_5 [1]
  T* gbh = gb5 + 1;                      // db of hidden layers [3][W]
  T* g1 = gbh + 3 * W;                   // dW_1 [W][DIN]
  T* gb1 = g1 + W * DIN;                 // db_1 [W]
  constexpr int NSMALL = W + 1 + 3 * W + W * DIN + W;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ntiles = (a.npts + P - 1) / P;
  const T* th = a.theta;
  const int ob1 = W * DIN, o2 = ob1 + W;
  const int o5 = o2 + 3 * (W * W + W);
  T* gacc = a.gpart + (size_t)blockIdx.x * a.nparams;
  constexpr int TK = W / 16, NKG = W / TK, NOGd = kMlpThreads / NKG, TOd = W / NOGd;
  static_assert(TOd * NOGd == W, "dW tile mapping");
  constexpr int TP = 4, NPG = P / TP, NKGp = kMlpThreads / NPG, TKp = W / NKGp;
  static_assert(TKp * NKGp == W, "delta tile mapping");
  const int kg = tid % NKG, og = tid / NKG;
  // stage activations of `layer` for the tile at p0 with 16-byte async copies
  auto stage = [&](T* dst, int layer, int p0) {
    constexpr int CH = 16 / sizeof(T), PCH = P / CH;
    for (int c = tid; c < W * PCH; c += kMlpThreads) {
      const int k = c / PCH, pc = (c % PCH) * CH;
      cp_async16(&dst[k * PS + pc], &a.acts[((size_t)layer * W + k) * a.ld + p0 + pc]);
    }
    cp_async_commit();
  };
  T accW[REGACC ? 3 : 1][TOd][TK];
#pragma unroll
  for (int l = 0; l < (REGACC ? 3 : 1); ++l)
#pragma unroll
    for (int i = 0; i < TOd; ++i)
#pragma unroll
      for (int j = 0; j < TK; ++j) accW[l][i][j] = T(0);
  for (int i = tid; i < NSMALL; i += kMlpThreads) gsm[i] = T(0);
  if (!REGACC)
    for (int i = tid; i < a.nparams; i += kMlpThreads) gacc[i] = T(0);
  if (ALLW)
    for (int e = tid; e < 3 * W * W; e += kMlpThreads) {
      int l = e / (W * W), r = e % (W * W);
      Ws[e] = th[o2 + l * (W * W + W) + r];
    }
  // With two activation buffers the next stage's copy overlaps this stage's
  // math; with one (when two would not leave room for 2 CTAs per SM) each
  // stage issues its own copy and waits for it.
  auto buf_of = [&](int stg) { return aBuf + (NBUF == 2 ? (stg & 1) : 0) * W * PS; };
  int st = 0;
  if (NBUF == 2 && (int)blockIdx.x < ntiles) stage(aBuf, 3, blockIdx.x * P);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int p0 = tile * P;
    if (NBUF == 1) {
      __syncthreads();
      stage(aBuf, 3, p0);
    }
    cp_async_wait_all();
    __syncthreads();
    if (NBUF == 2) stage(buf_of(st + 1), 2, p0);
    for (int p = tid; p < P; p += kMlpThreads) {
      const int idx = p0 + p;
      gP[p] = idx < a.npts ? a.gu[idx] : T(0);
      T c[3];
      point_coords<T, DIN>(min(idx, a.npts - 1), a.N, c);
      for (int d = 0; d < DIN; ++d) xin[d * P + p] = c[d];
    }
    __syncthreads();
    {
      const T* aS = buf_of(st);
      // output layer: dW_5[k] = sum_p g_p a_4[k][p], db_5 = sum_p g_p
      for (int k = warp; k < W; k += NWARP) {
        T sum = T(0);
        for (int p = lane; p < P; p += 32) sum += gP[p] * aS[k * PS + p];
        sum = warp_sum(sum);
        if (lane == 0) g5[k] += sum;
      }
      if (warp == 0) {
        T sum = T(0);
        for (int p = lane; p < P; p += 32) sum += gP[p];
        sum = warp_sum(sum);
        if (lane == 0) gb5[0] += sum;
      }
      for (int e = tid; e < W * P; e += kMlpThreads) {
        const int k = e / P, p = e % P;
        const T av = aS[k * PS + p];
        dA[k * PS + p] = th[o5 + k] * gP[p] * (T(1) - av * av);
      }
      ++st;
    }
#pragma unroll
    for (int hl = 2; hl >= 0; --hl) {
      const int ow = o2 + hl * (W * W + W);
      if (NBUF == 1) {
        __syncthreads();
        stage(aBuf, hl, p0);
      }
      cp_async_wait_all();
      __syncthreads();
      if (NBUF == 2) {
        if (hl > 0) stage(buf_of(st + 1), hl - 1, p0);
        else if (tile + (int)gridDim.x < ntiles) stage(buf_of(st + 1), 3, (tile + gridDim.x) * P);
      }
      if (!ALLW) {
        for (int e = tid; e < W * W; e += kMlpThreads) Ws[e] = th[ow + e];
        __syncthreads();
      }
      const T* Wl = ALLW ? Ws + hl * W * W : Ws;
      const T* aS = buf_of(st);
      // dW[o][k] += sum_p dA[o][p] aS[k][p]
      {
        T acc[TOd][TK];
#pragma unroll
        for (int i = 0; i < TOd; ++i)
#pragma unroll
          for (int j = 0; j < TK; ++j) acc[i][j] = T(0);
#pragma unroll 2
        for (int p = 0; p < P; p += 4) {
          T dv[TOd][4], av[TK][4];
#pragma unroll
          for (int i = 0; i < TOd; ++i) ld4<T>(&dA[(og * TOd + i) * PS + p], dv[i]);
#pragma unroll
          for (int j = 0; j < TK; ++j) ld4<T>(&aS[(kg + NKG * j) * PS + p], av[j]);
#pragma unroll
          for (int i = 0; i < TOd; ++i)
#pragma unroll
            for (int j = 0; j < TK; ++j)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[i][j] += dv[i][q] * av[j][q];
        }
        if (REGACC) {
#pragma unroll
          for (int i = 0; i < TOd; ++i)
#pragma unroll
            for (int j = 0; j < TK; ++j) accW[REGACC ? hl : 0][i][j] += acc[i][j];
        } else {
#pragma unroll
          for (int i = 0; i < TOd; ++i)
#pragma unroll
            for (int j = 0; j < TK; ++j)
              gacc[ow + (og * TOd + i) * W + kg + NKG * j] += acc[i][j];
        }
      }
      // db[o] += sum_p dA[o][p]
      for (int o = warp; o < W; o += NWARP) {
        T sum = T(0);
        for (int p = lane; p < P; p += 32) sum += dA[o * PS + p];
        sum = warp_sum(sum);
        if (lane == 0) gbh[hl * W + o] += sum;
      }
      // delta_{l-1}[k][p] = (sum_o W[o][k] dA[o][p]) (1 - aS[k][p]^2)
      {
        const int pg = tid % NPG, kgp = tid / NPG;
        T acc[TKp][TP];
#pragma unroll
        for (int i = 0; i < TKp; ++i)
#pragma unroll
          for (int j = 0; j < TP; ++j) acc[i][j] = T(0);
#pragma unroll 4
        for (int o = 0; o < W; ++o) {
          T wv[TKp], dv[TP];
#pragma unroll
          for (int i = 0; i < TKp; i += 4) ld4<T>(&Wl[o * W + kgp * TKp + i], &wv[i]);
          ld4<T>(&dA[o * PS + pg * TP], dv);
#pragma unroll
          for (int i = 0; i < TKp; ++i)
#pragma unroll
            for (int q = 0; q < TP; ++q) acc[i][q] += wv[i] * dv[q];
        }
#pragma unroll
        for (int i = 0; i < TKp; ++i) {
          const int k = kgp * TKp + i;
          T av[TP], v[TP];
          ld4<T>(&aS[k * PS + pg * TP], av);
#pragma unroll
          for (int q = 0; q < TP; ++q) v[q] = acc[i][q] * (T(1) - av[q] * av[q]);
          st4<T>(&dB[k * PS + pg * TP], v);
        }
      }
      ++st;
      if (!ALLW) __syncthreads();  // Ws is reloaded by the next layer
      T* tmp = dA; dA = dB; dB = tmp;
    }
    __syncthreads();
    // first layer: dW_1[o][d] += sum_p delta_1[o][p] x'_d[p], db_1[o] += sum_p delta_1[o][p]
    for (int o = warp; o < W; o += NWARP) {
      T s[DIN + 1];
#pragma unroll
      for (int d = 0; d <= DIN; ++d) s[d] = T(0);
      for (int p = lane; p < P; p += 32) {
        const T dv = dA[o * PS + p];
#pragma unroll
        for (int d = 0; d < DIN; ++d) s[d] += dv * xin[d * P + p];
        s[DIN] += dv;
      }
#pragma unroll
      for (int d = 0; d <= DIN; ++d) s[d] = warp_sum(s[d]);
      if (lane == 0) {
#pragma unroll
        for (int d = 0; d < DIN; ++d) g1[o * DIN + d] += s[d];
        gb1[o] += s[DIN];
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // write this CTA's gradient row
  if (REGACC) {
#pragma unroll
    for (int hl = 0; hl < 3; ++hl) {
      const int ow = o2 + hl * (W * W + W);
#pragma unroll
      for (int i = 0; i < TOd; ++i)
#pragma unroll
        for (int j = 0; j < TK; ++j)
          gacc[ow + (og * TOd + i) * W + kg + NKG * j] = accW[REGACC ? hl : 0][i][j];
    }
  }
  for (int i = tid; i < W; i += kMlpThreads) {
    gacc[o5 + i] = g5[i];
    gacc[ob1 + i] = gb1[i];
    for (int hl = 0; hl < 3; ++hl) gacc[o2 + hl * (W * W + W) + W * W + i] = gbh[hl * W + i];
    for (int d = 0; d < DIN; ++d) gacc[i * DIN + d] = g1[i * DIN + d];
  }
  if (tid == 0) gacc[o5 + W] = gb5[0];
}

template <typename T, int W, int DIN>
static size_t fwd_smem() {
  constexpr int P = 64, PS = P + 4;
  constexpr bool ALLW = (3 * W * W * sizeof(T) <= 64 * 1024);
  return sizeof(T) * ((ALLW ? 3 : 1) * W * W + 2 * W * PS + DIN * P);
}
template <typename T, int W, int DIN>
static size_t bwd_smem() {
  return bwd_bytes<T, W, DIN, 64>(bwd_nbuf<T, W, DIN, 64>());
}

static int g_num_sms = 0;
static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

template <typename T, int W, int DIN>
static cudaError_t fwd_dispatch(const MlpArgs<T>& a, cudaStream_t st) {
  if constexpr (sizeof(T) == 8 && W > 64) {
    return cudaErrorNotSupported;  // shared-memory tiles exceed 227 KB
  }
  auto k = k_mlp_fwd<T, W, DIN, 64>;
  size_t smem = fwd_smem<T, W, DIN>();
  smem_optin(k);
  int ntiles = (a.npts + 63) / 64;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kMlpThreads, smem);
  if (occ < 1) occ = 1;
  int grid = ntiles < occ * num_sms() ? ntiles : occ * num_sms();
  k<<<grid, kMlpThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int W, int DIN>
static cudaError_t bwd_dispatch(const MlpArgs<T>& a, int nblk, cudaStream_t st) {
  if constexpr (sizeof(T) == 8 && W > 64) {
    return cudaErrorNotSupported;
  }
  auto k = k_mlp_bwd<T, W, DIN, 64>;
  size_t smem = bwd_smem<T, W, DIN>();
  smem_optin(k);
  k<<<nblk, kMlpThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int W, int DIN>
static int bwd_grid(int npts) {
  auto k = k_mlp_bwd<T, W, DIN, 64>;
  size_t smem = bwd_smem<T, W, DIN>();
  smem_optin(k);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kMlpThreads, smem);
  if (occ < 1) occ = 1;
  int ntiles = (npts + 63) / 64;
  return ntiles < occ * num_sms() ? ntiles : occ * num_sms();
}

int mlp_bwd_blocks(int npts, int width, int elem_bytes, int din) {
  if (elem_bytes == 4) {
    if (din == 2) return width == 64 ? bwd_grid<float, 64, 2>(npts) : bwd_grid<float, 128, 2>(npts);
    return width == 64 ? bwd_grid<float, 64, 3>(npts) : bwd_grid<float, 128, 3>(npts);
  }
  if (din == 2) return bwd_grid<double, 64, 2>(npts);
  return bwd_grid<double, 64, 3>(npts);
}

template <typename T>
cudaError_t launch_mlp_fwd(const MlpArgs<T>& a, cudaStream_t st) {
  if (a.npts <= 0) return cudaSuccess;
  if (a.din == 2 && a.width == 64) return fwd_dispatch<T, 64, 2>(a, st);
  if (a.din == 2 && a.width == 128) return fwd_dispatch<T, 128, 2>(a, st);
  if (a.din == 3 && a.width == 64) return fwd_dispatch<T, 64, 3>(a, st);
  if (a.din == 3 && a.width == 128) return fwd_dispatch<T, 128, 3>(a, st);
  return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_mlp_bwd(const MlpArgs<T>& a, int nblk, cudaStream_t st) {
  if (a.npts <= 0) return cudaSuccess;
  if (a.din == 2 && a.width == 64) return bwd_dispatch<T, 64, 2>(a, nblk, st);
  if (a.din == 2 && a.width == 128) return bwd_dispatch<T, 128, 2>(a, nblk, st);
  if (a.din == 3 && a.width == 64) return bwd_dispatch<T, 64, 3>(a, nblk, st);
  if (a.din == 3 && a.width == 128) return bwd_dispatch<T, 128, 3>(a, nblk, st);
  return cudaErrorNotSupported;
}

// grad = sum over CTA partial rows (fixed order); Adam (Kingma & Ba) with
// beta1 = 0.9, beta2 = 0.999, eps = 1e-8; bc = bias corrections 1/(1-beta^t).
// Sum of the per-block gradient partials and the Adam step.  A block covers
// 32 parameters; its 8 warps take every 8th partial (two accumulation chains
// each, for memory-level parallelism) and warp 0 adds the 8 warp sums in a
// fixed order (deterministic).
template <typename T>
__device__ __forceinline__ void grad_adam_body(const T* __restrict__ gpart, int nblk, int nparams, T* grad,
                                               T* theta, T* m, T* v, const double* bc, const double* lr, int upd,
                                               int bid) {
  __shared__ T part[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int i = bid * 32 + tx;
  T s0 = T(0), s1 = T(0);
  if (i < nparams) {
    int b = ty;
    for (; b + 8 < nblk; b += 16) {
      s0 += gpart[(size_t)b * nparams + i];
      s1 += gpart[(size_t)(b + 8) * nparams + i];
    }
    if (b < nblk) s0 += gpart[(size_t)b * nparams + i];
  }
  part[ty][tx] = s0 + s1;
  __syncthreads();
  if (ty != 0 || i >= nparams) return;
  T g = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) g += part[k][tx];
  grad[i] = g;
  if (!upd) return;
  const T b1 = T(0.9), b2 = T(0.999), eps = T(1e-8);
  T mi = b1 * m[i] + (T(1) - b1) * g;
  T vi = b2 * v[i] + (T(1) - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const T mh = mi * (T)bc[0];
  const T vh = vi * (T)bc[1];
  theta[i] -= (T)(*lr) * mh / (sqrt(vh) + eps);
}
template <typename T>
__global__ void __launch_bounds__(256) k_grad_adam(const T* __restrict__ gpart, int nblk,
                                                   int nparams, T* grad, T* theta, T* m, T* v,
                                                   const double* bc, const double* lr, int upd) {
  grad_adam_body<T>(gpart, nblk, nparams, grad, theta, m, v, bc, lr, upd, blockIdx.x);
}
// grouped (FP32): CTA g.cta[b].y of context g.cta[b].x's launch
__global__ void __launch_bounds__(256) k_grad_adam_grp(const AdamArgs* __restrict__ tab, GroupMap g) {
  const int2 c = g.cta[blockIdx.x];
  const AdamArgs& a = tab[c.x];
  grad_adam_body<float>(a.gpart, a.nblk, a.nparams, a.grad, a.theta, a.m, a.v, a.bc, a.lr, a.upd, c.y);
}

int grad_adam_blocks(int nparams) { return (nparams + 31) / 32; }

cudaError_t launch_grad_adam_grouped(const AdamArgs* tab, GroupMap g, int nctas, cudaStream_t st) {
  if (nctas > 0) k_grad_adam_grp<<<nctas, 256, 0, st>>>(tab, g);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad_reduce_adam(const T* gpart, int nblk, int nparams, T* grad, T* theta, T* m,
                                    T* v, const double* bc, const double* lr, int do_update,
                                    cudaStream_t st) {
  k_grad_adam<T><<<(nparams + 31) / 32, 256, 0, st>>>(gpart, nblk, nparams, grad, theta, m, v, bc,
                                                       lr, do_update);
  return cudaGetLastError();
}

#define MLP_INST(T)                                                                               \
  template cudaError_t launch_mlp_fwd<T>(const MlpArgs<T>&, cudaStream_t);                       \
  template cudaError_t launch_mlp_bwd<T>(const MlpArgs<T>&, int, cudaStream_t);                  \
  template cudaError_t launch_grad_reduce_adam<T>(const T*, int, int, T*, T*, T*, T*,            \
                                                  const double*, const double*, int, cudaStream_t);
MLP_INST(float)
MLP_INST(double)

}  // namespace adsgb

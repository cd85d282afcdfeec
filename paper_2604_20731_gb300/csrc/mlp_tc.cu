// CRVPINN network on the 5th-generation tensor cores (tcgen05, sm_103a):
// BF16 operands, FP32 accumulation in tensor memory (TMEM).  Widths 64, 128.
//
// Operand tiles live in shared memory in the no-swizzle canonical layout:
// 8-row x 16-byte core matrices; within a tile of R rows and C columns the
// byte offset of element (r, c) is (r/8)*RG + (c/8)*128 + (r%8)*16 + (c%8)*2
// with RG = (C/8)*128.  The same tile serves as a K-major operand (rows = M or
// N, columns = K; descriptor LBO = 128, SBO = RG) or as an MN-major operand
// (rows = K, columns = M or N; LBO = RG, SBO = 128).
//
// Forward, per tile of 128 collocation points (TMEM lane t = point t; two
// epilogue threads per point, one issuing thread):
//   a_1 = tanh(W_1 x' + b_1) on the CUDA cores (K = 2 or 3);
//   for the three hidden layers: D[t][o] = s (sum_k a[t][k] W[o][k] + b[o])
//   with s = -2 log2 e folded into the staged weights and the bias carried by
//   an extra K block (see TcSmemF), the activations held as a BF16 pair
//   a = a_hi + a_lo (two MMA chains into one FP32 accumulator) -- the
//   residual differences neighbouring network values, so per-point rounding
//   of the activations to BF16 alone would swamp it on fine grids; the
//   epilogue reads its row of D from TMEM, applies tanh = 2 / (1 + 2^D) - 1
//   and writes the next pair (and, for the backward pass, the BF16 row to
//   HBM);
//   u = W_5 a_4 + b_5 in FP32 from registers.
// Backward, per tile (persistent CTAs; gradients accumulate in TMEM over all
// of a CTA's tiles):
//   D_l (for dW_l, db_l) += Delta_l^T [a_{l-1} | 1] -- M = 64 output rows
//   (width 64; the ring form for width 128 uses M = 128), N = 80 (64 inputs +
//   a ones column, appended in shared memory, giving db), K = 128 points,
//   both operands MN-major views of the [point][feature] tiles;
//   Delta_{l-1} = (Delta_l W_l) (1 - a_{l-1}^2) -- M = 128 points, N = 64,
//   K = 64, W_l read MN-major from the backward's own weight tiles.
//   The output layer is the same product with Delta_5 = [g, 0, ...] and the
//   first layer with [x' | 1] as the second operand.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace adsgb {
namespace {

constexpr int kW = 64;           // hidden width of this path
constexpr int kTP = 128;         // points per tile = MMA M = TMEM lanes
constexpr int kWP = kW + 16;     // activation tile width incl. ones column
constexpr int kDP = 128;         // M of the ring form's weight-gradient products (rows past W unused)
constexpr int kXP = 16;          // input tile width: x', 1, zeros
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

ADS_D uint32_t core_off(int r, int c, int rg) {
  return (uint32_t)((r >> 3) * rg + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Stored activations of a 128-point tile (written by the forward, read by the
// backward): a_1 .. a_4 one after another, [128][W] BF16 each, nothing else.
// Width 128 keeps the core-matrix layout of the shared tiles (row groups
// outermost).  Width 64 keeps each 8-column chunk's 128 rows together (2 KB
// per chunk, 16 B per row), so that a warp's 32 rows of one chunk are 512
// contiguous bytes, and so that the backward's shared copy of a_1 .. a_3 can
// place two constant chunks, [1, 0, ..., 0] and zeros, behind the 64 columns
// and read [a | 1] as one N = 80 operand whose product gives the bias
// gradient with the weight gradient: the constant columns never travel
// through HBM.
ADS_HD constexpr int st_layer_bytes(int W) { return kTP * W * 2; }
ADS_HD constexpr int st_tile_bytes(int W) { return 4 * st_layer_bytes(W); }
constexpr int kChunk = kTP * 16;  // one 8-column chunk of a width-64 stored layer
ADS_HD constexpr uint32_t st_off(int W, int r, int c) {
  return W == 64 ? (uint32_t)((c >> 3) * kChunk + r * 16 + (c & 7) * 2)
                 : (uint32_t)((r >> 3) * (W / 8) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Shared-memory matrix descriptor (no swizzle): bits 0-13 start address >> 4,
// 16-29 leading-dimension byte offset >> 4, 32-45 stride-dimension byte offset
// >> 4, bit 46 the descriptor version of tcgen05, base offset and swizzle 0.
// The two views below give the same bits as sdesc, written so that a k-step
// costs one 32-bit add: shared addresses are below 256 KB, so the start
// address field (bits 0-13, address >> 4) never carries into the fields above.
// K-major view of a tile (rows = M/N, columns = K), k-step of 16 columns:
// LBO 128 B, SBO = rg
ADS_D uint64_t desc_k(uint32_t base, int rg, int kstep) {
  const uint32_t lo = (base >> 4) + (uint32_t)kstep * 16u + (8u << 16);
  const uint32_t hi = ((uint32_t)rg >> 4) | (1u << 14);  // SBO, descriptor version
  return ((uint64_t)hi << 32) | lo;
}
// MN-major view of a tile (rows = K, columns = M/N), k-step of 16 rows:
// LBO = rg, SBO 128 B
ADS_D uint64_t desc_mn(uint32_t base, int rg, int kstep) {
  const uint32_t lo = (base >> 4) + (uint32_t)kstep * ((2u * (uint32_t)rg) >> 4) + (((uint32_t)rg >> 4) << 16);
  const uint32_t hi = 8u | (1u << 14);
  return ((uint64_t)hi << 32) | lo;
}
// instruction descriptor: BF16 x BF16 -> FP32, M x N, operand majors
ADS_HD uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

ADS_D void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
ADS_D void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_addr(mbar)));
}
ADS_D void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
ADS_D void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

ADS_D unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the mbarrier phase `parity`, giving up after about a second
// (returns false then; the caller records an error and stops)
ADS_D bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = now_ns();
    else if (now_ns() - t0 > kWaitNs) return false;
  }
}



// CTA barrier that also orders tcgen05 operations and generic-proxy shared
// stores before the tensor cores read them; returns the CTA-uniform abort flag
ADS_D bool sync_abort(volatile int* abort_flag) {
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *abort_flag != 0;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
ADS_D void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}


// 32 consecutive TMEM columns of this warp's lanes, without waiting; the
// values are valid after tmem_wait32 on the same registers
ADS_D void tmem_ld32_async(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// pin 32 registers after the preceding wait (no instruction is emitted)
ADS_D void reg_pin32(uint32_t r[32]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}
// 32 consecutive TMEM columns
ADS_D void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  tmem_ld32_async(taddr, r);
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  reg_pin32(r);
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

ADS_D uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// write 8 values (one 16-byte atom) of row r starting at column c (c % 8 == 0)
ADS_D void st_atom(unsigned char* tile, int rg, int r, int c, const float v[8]) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(tile + core_off(r, c, rg)) = q;
}
// the same 8 values at a given address (16-byte aligned)
ADS_D void st_atom_at(unsigned char* p, const float v[8]) {
  *reinterpret_cast<uint4*>(p) =
      make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}

// 8 BF16 values (one 16-byte atom) at a given address, as FP32
ADS_D void ld_atom_at(const unsigned char* p, float v[8]) {
  uint4 q = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 f = __bfloat1622float2(h[j]);
    v[2 * j] = f.x;
    v[2 * j + 1] = f.y;
  }
}

ADS_D void ld_atom(const unsigned char* tile, int rg, int r, int c, float v[8]) {
  uint4 q = *reinterpret_cast<const uint4*>(tile + core_off(r, c, rg));
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 f = __bfloat1622float2(h[j]);
    v[2 * j] = f.x;
    v[2 * j + 1] = f.y;
  }
}

template <int DIN>
ADS_D void coords(int idx, int N, float c[3]) {
  const int m = N - 1;
  const float invN = 1.0f / (float)N;
  c[0] = 2.0f * (float)(idx % m + 1) * invN - 1.0f;
  c[1] = 2.0f * (float)((idx / m) % m + 1) * invN - 1.0f;
  c[2] = DIN == 3 ? 2.0f * (float)(idx / (m * m) + 1) * invN - 1.0f : 0.0f;
}

// load the three hidden weight matrices W_l[o][k] (FP32 master, 16-byte
// aligned rows) as BF16 tiles.  Each thread takes atoms e = tid + i NTHR and
// issues the loads of a batch of them before any store, so the CTA waits
// for about one memory latency per batch instead of one per atom.
template <int W, int NTHR>
ADS_D void load_hidden_weights(const float* __restrict__ th, int o2, unsigned char* wt, int tid) {
  constexpr int RG = (W / 8) * 128, NA = 3 * W * (W / 8), PER = (NA + NTHR - 1) / NTHR, B = 6;
#pragma unroll
  for (int i0 = 0; i0 < PER; i0 += B) {
    float4 q[B][2];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int e = tid + (i0 + i) * NTHR;
      if (i0 + i < PER && e < NA) {
        const int l = e / (W * (W / 8)), rem = e % (W * (W / 8));
        const int o = rem / (W / 8), c = (rem % (W / 8)) * 8;
        const float4* src = reinterpret_cast<const float4*>(th + o2 + l * (W * W + W) + o * W + c);
        q[i][0] = __ldg(src);
        q[i][1] = __ldg(src + 1);
      }
    }
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int e = tid + (i0 + i) * NTHR;
      if (i0 + i < PER && e < NA) {
        const int l = e / (W * (W / 8)), rem = e % (W * (W / 8));
        const int o = rem / (W / 8), c = (rem % (W / 8)) * 8;
        const float v[8] = {q[i][0].x, q[i][0].y, q[i][0].z, q[i][0].w, q[i][1].x, q[i][1].y, q[i][1].z, q[i][1].w};
        st_atom(wt + l * W * W * 2, RG, o, c, v);
      }
    }
  }
}

// TMEM lane of row o of an M = 64 accumulator: 16 rows in the first 16 lanes
// of each 32-lane quadrant (measured with a probe MMA on this GPU); the row a
// thread of warps 0-3 reads, or -1
ADS_HD constexpr int m64_row(int tid) { return (tid & 31) < 16 ? 16 * (tid >> 5) + (tid & 31) : -1; }

// One hidden layer's gradient into the CTA's partial row: dW[o][k] (o, k < W)
// sits in TMEM row o (lane o, or the M = 64 lane of row o with M64), columns
// k of `lane_col` (tmem address with the warp's lane offset and the layer's
// first column); its bias gradient is TMEM column W (TB) or `bias_o`.
// Threads of warps 0-3 read their lanes (warp-collective loads), the rows meet
// in shared memory S (W x (W + 1) floats), and the CTA writes g[o W + k] and
// g[W W + o] with consecutive threads on consecutive addresses.  Called by
// every thread of the CTA (two barriers inside).
template <int W, int NTHR, bool TB, bool M64 = false>
ADS_D void dw_layer_out(uint32_t lane_col, bool live, float bias_o, float* S, float* g, int tid) {
  constexpr int SW = W + 1;
  const int o = M64 ? m64_row(tid) : tid;
  if (live && tid < kTP) {
#pragma unroll 1
    for (int c = 0; c < (TB ? W + 16 : W); c += 16) {
      float v[16];
      tmem_ld16(lane_col + c, v);  // warp-collective
      if (o >= 0 && o < W) {
        if (c < W) {
#pragma unroll
          for (int j = 0; j < 16; ++j) S[o * SW + c + j] = v[j];
        } else {
          S[o * SW + W] = v[0];
        }
      }
    }
    if (!TB && o >= 0 && o < W) S[o * SW + W] = bias_o;
  }
  __syncthreads();
  if (live)
    for (int e = tid; e < W * W + W; e += NTHR)
      g[e] = e < W * W ? S[(e / W) * SW + (e % W)] : S[(e - W * W) * SW + W];
  __syncthreads();
}

// Forward operands.  The hidden weights are staged as BF16 tiles of
// s W_l and the bias s b_l (s = -2 log2 e) in one more K block of 16 columns
// (column W: bf16(s b), column W + 1: bf16(s b - bf16(s b)), the rest 0),
// and the activation hi tile carries the matching columns [1, 1, 0, ...].  A
// layer's products then leave z' = s (W_l a + b_l) in TMEM, and tanh z =
// 2 / (1 + 2^z') - 1 needs neither a bias add nor a multiply.
constexpr float kTanhScale = -2.8853900817779268f;  // -2 log2(e)

template <int W>
struct TcSmemF {
  static constexpr int NS = W == 64 ? 2 : 1;           // tiles in flight per CTA
  static constexpr int KC = W + 16;                    // K of the hi operands
  static constexpr int ACT_SZ = kTP * KC * 2;          // [128][KC] bf16 hi | 1 1 0 ...
  static constexpr int ACTLO_SZ = kTP * W * 2;         // [128][W] bf16 lo
  static constexpr int NVEC = W + 3 * W + W + 4;       // fp32: s b_1 [W], s W_1 [3][W], W_5 [W], b_5
  // byte offsets.  [VEC | WT] is the weight image, staged in global memory by
  // k_stage_fwd and brought in by two bulk copies.
  static constexpr int VEC = 0;
  static constexpr int VEC_SZ = (NVEC * 4 + 127) / 128 * 128;
  static constexpr int WT = VEC + VEC_SZ;              // 3 x [W][KC] bf16: s W_l | s b_l
  static constexpr int WT_SZ = 3 * W * KC * 2;
  static constexpr int IMG = WT + WT_SZ;               // bytes of the image
  static constexpr int ACT = IMG;                      // NS hi tiles
  static constexpr int ACTLO = ACT + NS * ACT_SZ;      // NS lo tiles
  static constexpr int BAR = ACTLO + NS * ACTLO_SZ;    // mbarriers: vec, wt, ready[NS], prod[NS]; tmem base; abort
  static constexpr int TPR = 2;                        // epilogue threads per point row (W / 2 columns each)
  static constexpr int UPART = BAR + 64;               // fp32 [2][NS][TPR - 1][128]: output-layer partial sums
  static constexpr int TOTAL = UPART + 2 * NS * (TPR - 1) * kTP * 4;
};

// The weight image of the forward, from the FP32 master parameters: the
// constant vectors (FP32) and the three hidden layers as BF16 K-major tiles
// (one 16-byte atom of 8 values per thread)
template <int W, int DIN>
__device__ __forceinline__ void stage_fwd_body(const float* __restrict__ th, unsigned char* __restrict__ img,
                                               int bid) {
  using L = TcSmemF<W>;
  constexpr int KC = L::KC, RG = (KC / 8) * 128, APR = KC / 8, NA = 3 * W * APR, NV = L::VEC_SZ / 4;
  const int ob1 = W * DIN, o2 = ob1 + W, o5 = o2 + 3 * (W * W + W);
  const int e = bid * 256 + threadIdx.x;
  if (e == 0) *reinterpret_cast<int*>(img + L::IMG) = 0;  // the forward's tile-group counter
  if (e < NA) {
    const int l = e / (W * APR), rem = e % (W * APR), o = rem / APR, c = (rem % APR) * 8;
    const float* Wl = th + o2 + l * (W * W + W);
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (c < W) {
      const float4* src = reinterpret_cast<const float4*>(Wl + o * W + c);
      const float4 q0 = __ldg(src), q1 = __ldg(src + 1);
      const float q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = kTanhScale * q[j];
    } else if (c == W) {
      const float sb = kTanhScale * __ldg(Wl + W * W + o);
      v[0] = sb;                                              // rounds to bf16(s b) in st_atom
      v[1] = sb - __bfloat162float(__float2bfloat16_rn(sb));  // the remainder, rounded there too
    }
    st_atom(img + L::WT + l * W * KC * 2, RG, o, c, v);
  } else if (e < NA + NV) {
    const int i = e - NA;
    float val = 0.0f;
    if (i < W) {
      val = kTanhScale * th[ob1 + i];
    } else if (i < 4 * W) {
      const int d = (i - W) / W, o = (i - W) % W;
      val = d < DIN ? kTanhScale * th[o * DIN + d] : 0.0f;
    } else if (i < 5 * W) {
      val = th[o5 + i - 4 * W];
    } else if (i == 5 * W) {
      val = th[o5 + W];
    }
    reinterpret_cast<float*>(img + L::VEC)[i] = val;
  }
}
template <int W, int DIN>
__global__ void __launch_bounds__(256) k_stage_fwd(const float* __restrict__ th, unsigned char* __restrict__ img) {
  stage_fwd_body<W, DIN>(th, img, blockIdx.x);
}
// grouped: context blockIdx.y of the table
template <int W, int DIN>
__global__ void __launch_bounds__(256) k_stage_fwd_grp(const MlpTcArgs* __restrict__ tab) {
  const MlpTcArgs& a = tab[blockIdx.y];
  stage_fwd_body<W, DIN>(a.theta, a.wimage, blockIdx.x);
}

ADS_D void mbar_expect(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
               : "memory");
}
ADS_D void mbar_arrive1(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}
// barrier 1 over the NTHR epilogue threads of the forward; returns whether
// any of them passed `v` true (the same answer in every thread)
template <int NTHR>
ADS_D bool epi_barrier_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\nbar.red.or.pred po, 1, %2, pi;\nselp.u32 %0, 1, 0, po;\n}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NTHR)
      : "memory");
  return r != 0;
}

ADS_D float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
ADS_D float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// tanh of two pre-activations given as z' = -2 log2(e) z: 2 / (1 + 2^z') - 1,
// the FP32 steps on packed pairs (one instruction per pair)
ADS_D float2 tanh2_scaled(float2 zs) {
  const float2 t = make_float2(ex2_approx(zs.x), ex2_approx(zs.y));
  const float2 d = __fadd2_rn(t, make_float2(1.0f, 1.0f));
  const float2 r = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  return __ffma2_rn(r, make_float2(2.0f, 2.0f), make_float2(-1.0f, -1.0f));
}
// The same with the reciprocal on the FP32 pipe instead of the special-
// function unit, for a share of the activations (the unit then carries one
// ex2 per activation and only some of the reciprocals).  Newton-Raphson for
// 1/d: the initial guess is the integer difference R - bits(d), whose value
// read as a float is within 5.1 % of 1/d for every normal d (R = 0x7EF311C0
// minimises the largest relative error over the mantissa; found by direct
// search), then three steps y <- y + y (1 - d y), each squaring the relative
// error: 5.1e-2, 2.6e-3, 6.5e-6, 4e-11 -- below FP32 rounding.  z' is capped
// at 64 so that d stays finite; 2 / (1 + 2^64) - 1 is -1 in FP32, as the
// uncapped form gives.
constexpr int kRcpSeed = 0x7EF311C0;
ADS_D float2 tanh2_scaled_nr(float2 zs) {
  const float2 t = make_float2(ex2_approx(fminf(zs.x, 64.0f)), ex2_approx(fminf(zs.y, 64.0f)));
  const float2 d = __fadd2_rn(t, make_float2(1.0f, 1.0f));
  const float2 nd = make_float2(-d.x, -d.y);
  float2 y = make_float2(__int_as_float(kRcpSeed - __float_as_int(d.x)), __int_as_float(kRcpSeed - __float_as_int(d.y)));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float2 e = __ffma2_rn(nd, y, make_float2(1.0f, 1.0f));
    y = __ffma2_rn(y, e, y);
  }
  return __ffma2_rn(y, make_float2(2.0f, 2.0f), make_float2(-1.0f, -1.0f));
}
// 8 values (one atom) as a BF16 pair hi + lo, to tiles of row-group strides
// rgh and rgl, and the hi half also to the address `g` (nullable); the
// remainder v - hi is formed on packed pairs
ADS_D void st_atom_split2(unsigned char* hi, int rgh, unsigned char* lo, int rgl, unsigned char* g, int r, int c,
                          const float v[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    const uint32_t hb = *reinterpret_cast<uint32_t*>(&b);
    const float2 bf = make_float2(__uint_as_float(hb << 16), __uint_as_float(hb & 0xFFFF0000u));
    const float2 rem = __ffma2_rn(bf, make_float2(-1.0f, -1.0f), make_float2(v[2 * j], v[2 * j + 1]));
    __nv_bfloat162 lb = __floats2bfloat162_rn(rem.x, rem.y);
    h[j] = hb;
    l[j] = *reinterpret_cast<uint32_t*>(&lb);
  }
  const uint4 qh = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(hi + core_off(r, c, rgh)) = qh;
  *reinterpret_cast<uint4*>(lo + core_off(r, c, rgl)) = make_uint4(l[0], l[1], l[2], l[3]);
  if (g) *reinterpret_cast<uint4*>(g) = qh;
}

// forward: TPR = 2 epilogue threads per point row, W / 2 feature columns each
// (eight warps; warps w and w + 4 read the same TMEM lanes; sixteen warps of
// 32 columns each were measured slower at W = 128), and one issuing warp.  For W = 64 a CTA carries two tiles
// at once (slots 0 and 1, each with its own operand tiles, TMEM accumulator,
// "written" and "products done" mbarriers): the tensor cores work on one slot
// while the epilogue warps work on the other.  The issuing warp only waits for
// a slot's operand tiles and issues its products, so the epilogue warps never
// wait for an issue; they meet only at the end of each tile group, to add the
// parts of the output layer (in a fixed order).
// epilogue threads (TPR per point row) and the issuing warp
template <int W>
ADS_HD constexpr int fwd_epi() { return TcSmemF<W>::TPR * kTP; }
template <int W>
ADS_HD constexpr int fwd_threads() { return fwd_epi<W>() + 32; }

template <int W, int DIN>
__device__ __forceinline__ void fwd_tc_body(const MlpTcArgs& a) {
  using L = TcSmemF<W>;
  constexpr int NS = L::NS;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* act = sm + L::ACT;
  unsigned char* actlo = sm + L::ACTLO;
  const float* fb1 = reinterpret_cast<const float*>(sm + L::VEC);  // s b_1
  const float* fW1 = fb1 + W;                                       // s W_1, [3][W]
  const float* fW5 = fW1 + 3 * W;
  uint64_t* mb_vec = reinterpret_cast<uint64_t*>(sm + L::BAR);
  uint64_t* mb_wt = mb_vec + 1;
  uint64_t* mb_ready = mb_vec + 2;    // [NS] a slot's operand tiles written (one arrive per epilogue warp)
  uint64_t* mb_prod = mb_ready + NS;  // [NS] a slot's products complete (issuer commit)
  uint32_t* tbase = reinterpret_cast<uint32_t*>(sm + L::BAR + 48);
  volatile int* abort_flag = reinterpret_cast<int*>(sm + L::BAR + 52);
  volatile int* group = reinterpret_cast<int*>(sm + L::BAR + 56);  // the current tile group
  float* upart = reinterpret_cast<float*>(sm + L::UPART);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kFwdEpi = fwd_epi<W>(), TPR = L::TPR, NEW = kFwdEpi / 32;  // NEW: epilogue warps
  const bool epi = tid < kFwdEpi;
  const int row = tid & (kTP - 1), part = tid >> 7;
  constexpr int KC = L::KC, RGH = (KC / 8) * 128, RGL = (W / 8) * 128, WH = W / TPR;
  const int cb = part * WH;  // an epilogue thread's first feature column
  if (tid == kFwdEpi) {
    *abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_vec)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_wt)));
    for (int s = 0; s < NS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mb_ready + s)), "r"(NEW));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_prod + s)));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the constant vectors first: layer 1 needs only them
    mbar_expect(mb_vec, L::VEC_SZ);
    bulk_load(sm + L::VEC, a.wimage + L::VEC, L::VEC_SZ, mb_vec);
    mbar_expect(mb_wt, L::WT_SZ);
    bulk_load(sm + L::WT, a.wimage + L::WT, L::WT_SZ, mb_wt);
  }
  if (tid < kTP) {
    // the constant columns of the hi operands: [1, 1, 0, ..., 0] (bias hi, lo)
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      unsigned char* ah = act + s * L::ACT_SZ;
      *reinterpret_cast<uint4*>(ah + core_off(tid, W, RGH)) = make_uint4(0x3F803F80u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(ah + core_off(tid, W + 8, RGH)) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tbase)), "r"(NS * W));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  const int ntiles = a.tile_count;  // local tile t is global tile a.tile0 + t
  if (!epi) {
    // ---------------- issuing thread ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(kTP, W, 0, 0);
      const uint32_t act_s = smem_addr(act), actlo_s = smem_addr(actlo), wt_s = smem_addr(sm + L::WT);
      uint32_t ph_ready[NS];
      int issued[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        ph_ready[s] = 0;
        issued[s] = 0;
      }
      bool ok = mbar_wait(mb_wt, 0);
      while (ok) {
        // slot 0's first operands announce the tile group (or the end)
        if (*abort_flag || !mbar_wait(mb_ready, ph_ready[0])) {
          ok = false;
          break;
        }
        ph_ready[0] ^= 1;
        const int t0 = NS * *group;
        if (t0 >= ntiles) break;
        for (int l = 0; ok && l < 3; ++l) {
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            if (!ok || t0 + s >= ntiles) continue;
            if (l > 0 || s > 0) {
              if (*abort_flag || !mbar_wait(mb_ready + s, ph_ready[s])) {
                ok = false;
                continue;
              }
              ph_ready[s] ^= 1;
            }
            tc_fence_after();
            // [a_hi | 1 1] [s W | s b_hi s b_lo]^T + a_lo (s W)^T: two BF16
            // chains into the slot's FP32 accumulator
            const uint32_t wl = wt_s + l * W * KC * 2, d = tmem + s * W;
            const uint32_t ah = act_s + s * L::ACT_SZ, al = actlo_s + s * L::ACTLO_SZ;
#pragma unroll
            for (int ks = 0; ks < KC / 16; ++ks)
              mma_bf16(d, desc_k(ah, RGH, ks), desc_k(wl, RGH, ks), idesc, ks > 0);
#pragma unroll
            for (int ks = 0; ks < W / 16; ++ks) mma_bf16(d, desc_k(al, RGL, ks), desc_k(wl, RGH, ks), idesc, 1u);
            mma_commit(mb_prod + s);
            ++issued[s];
          }
        }
      }
      if (!ok) *abort_flag = 1;
      // every product has completed before the accumulators are freed (a
      // no-op wait unless the epilogue warps stopped early)
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (issued[s] > 0) mbar_wait(mb_prod + s, (uint32_t)(issued[s] - 1) & 1u);
    }
  } else {
    // ---------------- epilogue warps ----------------
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    if (!mbar_wait(mb_vec, 0)) *abort_flag = 1;
    const float b5 = fW5[W];
    uint32_t ph_prod[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) ph_prod[s] = 0;
    auto ready = [&](int s) {
      fence_async_smem();  // generic stores before the tensor cores read them
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(mb_ready + s);
    };
    // tile groups (NS adjacent tiles) come from a counter shared by the
    // launch, so that the CTAs on an SM finish together however the warps
    // are scheduled; thread 0 takes the next group while the current one runs
    if (tid == 0) *group = atomicAdd(a.wimage_ctr, 1);
    epi_barrier_any<kFwdEpi>(false);
    int pass = 0;
    for (;; ++pass) {
      const int tb = NS * *group;
      if (tb >= ntiles) {
        ready(0);  // tells the issuer that there is no further group
        break;
      }
      int p0[NS];
      bool valid[NS];
      unsigned char* gt[NS];
      float2 u2[NS];
      // layer 1 of each slot on the CUDA cores, z' = s (W_1 x' + b_1) on
      // pairs of units
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int tile = tb + s;
        valid[s] = tile < ntiles;  // CTA-uniform
        p0[s] = (a.tile0 + tile) * kTP;
        gt[s] = nullptr;
        u2[s] = make_float2(part == 0 ? b5 : 0.0f, 0.0f);
        if (!valid[s]) continue;
        float x[3];
        coords<DIN>(min(p0[s] + row, a.npts - 1), a.N, x);
        gt[s] = a.acts ? a.acts + (size_t)tile * st_tile_bytes(W) : nullptr;
        unsigned char* ah = act + s * L::ACT_SZ;
        unsigned char* al = actlo + s * L::ACTLO_SZ;
#pragma unroll
        for (int c = 0; c < WH; c += 8) {
          float v[8];
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const int o = cb + c + j;
            float2 z = *reinterpret_cast<const float2*>(fb1 + o);
#pragma unroll
            for (int d = 0; d < DIN; ++d)
              z = __ffma2_rn(*reinterpret_cast<const float2*>(fW1 + d * W + o), make_float2(x[d], x[d]), z);
            // one pair in two with its reciprocal on the FP32 pipe
            const float2 t = (j & 2) ? tanh2_scaled_nr(z) : tanh2_scaled(z);
            v[j] = t.x;
            v[j + 1] = t.y;
          }
          st_atom_split2(ah, RGH, al, RGL, gt[s] ? gt[s] + st_off(W, row, cb + c) : nullptr, row, cb + c, v);
        }
        ready(s);
      }
      // hidden layers 2..4: per slot, wait for its products, then the
      // epilogue, whose tiles (layers 2, 3) feed the slot's next products
      for (int l = 0; l < 3; ++l) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          if (!valid[s]) continue;
          if (!*abort_flag && !mbar_wait(mb_prod + s, ph_prod[s])) *abort_flag = 1;
          ph_prod[s] ^= 1;
          tc_fence_after();
          unsigned char* ah = act + s * L::ACT_SZ;
          unsigned char* al = actlo + s * L::ACTLO_SZ;
          unsigned char* g = gt[s] ? gt[s] + (l + 1) * st_layer_bytes(W) : nullptr;
#pragma unroll
          for (int c0 = 0; c0 < WH; c0 += 32) {
            float d[32];
            tmem_ld32(lane_base + s * W + cb + c0, d);
#pragma unroll
            for (int c = 0; c < 32; c += 8) {
              float v[8];
#pragma unroll
              for (int j = 0; j < 8; j += 2) {
                const float2 zz = make_float2(d[c + j], d[c + j + 1]);
                const float2 t = (j & 2) ? tanh2_scaled_nr(zz) : tanh2_scaled(zz);
                v[j] = t.x;
                v[j + 1] = t.y;
              }
              unsigned char* gp = g ? g + st_off(W, row, cb + c0 + c) : nullptr;
              if (l < 2) {
                st_atom_split2(ah, RGH, al, RGL, gp, row, cb + c0 + c, v);
              } else {
                if (gp) st_atom_at(gp, v);
                // the output layer in FP32 from the unrounded activations
#pragma unroll
                for (int j = 0; j < 8; j += 2)
                  u2[s] = __ffma2_rn(make_float2(v[j], v[j + 1]),
                                     *reinterpret_cast<const float2*>(fW5 + cb + c0 + c + j), u2[s]);
              }
            }
          }
          if (l < 2) ready(s);
        }
      }
      // the two halves of each slot's output-layer sums (double-buffered by
      // pass); the barrier also publishes the next group and makes the stop
      // decision the same everywhere.  (The issuer read this pass's group
      // before it issued the products these epilogues waited for.)
      float* up = upart + (pass & 1) * NS * (TPR - 1) * kTP;
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (part) up[(s * (TPR - 1) + part - 1) * kTP + row] = u2[s].x + u2[s].y;
      if (tid == 0) *group = atomicAdd(a.wimage_ctr, 1);
      const bool stop = epi_barrier_any<kFwdEpi>(*abort_flag != 0);
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (!part && valid[s] && !stop && p0[s] + row < a.npts) {
          float u = u2[s].x + u2[s].y;
#pragma unroll
          for (int q = 0; q < TPR - 1; ++q) u += up[(s * (TPR - 1) + q) * kTP + row];
          a.u[p0[s] + row] = u;
        }
      if (stop) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && tid == 0) atomicOr(a.flags, 8);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NS * W));
}
template <int W, int DIN>
__global__ void __launch_bounds__(fwd_threads<W>(), W == 64 ? 2 : 1) k_mlp_fwd_tc(MlpTcArgs a) {
  fwd_tc_body<W, DIN>(a);
}
// grouped: the CTAs of several contexts' forwards in one launch (each
// context's tile groups come from its own counter)
template <int W, int DIN>
__global__ void __launch_bounds__(fwd_threads<W>(), W == 64 ? 2 : 1)
    k_mlp_fwd_tc_grp(const MlpTcArgs* __restrict__ tab, GroupMap g) {
  fwd_tc_body<W, DIN>(tab[g.cta[blockIdx.x].x]);
}

// ---------------------------------------------------------------------------
// backward, width 64: the products on the tensor cores, one CTA per SM (the
// accumulators fill the 512 TMEM columns).  Warp-specialised: warps 0-7 run
// the delta epilogues (point row tid % 128, feature columns 32 (tid / 128) ..
// + 32), warp 8 issues every product.  A product is a single-thread
// instruction that takes tens of cycles to issue while these shapes (N = 16..64)
// take fewer cycles to run, so only each layer's delta product Delta_L W_L
// sits on the epilogues' path; the weight and bias gradient products run under
// the epilogues.  One thread issues all products of an accumulator, in a fixed
// order (deterministic sums); products complete in issue order.  The output
// layer's gradient (a_4^T g, sum g) is a per-thread running sum over the CTA's
// tiles, reduced over the rows once at the end in a fixed order.  The four
// stored activation layers of a point tile (64 KB) arrive by four bulk
// copies on one barrier into a double buffer, the next tile's copies running
// under the current tile.  Bias gradients come with the weight gradients from
// the [a | 1] copies (the constant chunks are written once per launch).  The delta tiles are 64 columns wide; the weight-
// gradient products read them as M = 128 operands whose rows 64 .. 127 (the
// next rows' values) land in accumulator rows that are never read.
constexpr int kBwdEpi = 2 * kTP;          // epilogue threads: two per point row
constexpr int kBwdThreads = kBwdEpi + 32;  // eight epilogue warps, one issuing warp
struct TcSmemB {
  static constexpr int W = 0;                              // 3 x [64][64] bf16       24 KB
  static constexpr int LAYER = (kWP / 8) * kChunk;         // [a | 1]: 10 chunks of 2 KB  20 KB
  static constexpr int ACT_TILE = 3 * LAYER + st_layer_bytes(kW);  // a_1..a_3 as [a | 1], a_4  76 KB
  static constexpr int ACT = W + 3 * kW * kW * 2;          // 2 buffers             152 KB
  static constexpr int DEL_SZ = kTP * kW * 2;              // [128][64] bf16          16 KB
  static constexpr int DEL = ACT + 2 * ACT_TILE;           // 2 delta tiles           32 KB
  static constexpr int XIN_SZ = kTP * kXP * 2;
  static constexpr int XIN = DEL + 2 * DEL_SZ;             // 2 x [128][16] bf16: x', 1, 0  8 KB
  static constexpr int VEC = XIN + 2 * XIN_SZ;             // fp32: W5 [64]
  static constexpr int BAR = VEC + kW * 4;                 // 7 mbarriers, tmem base, abort flag
  static constexpr int TOTAL = BAR + 64;
};
// the backward's copy of stored layer l (a_1 .. a_4 for l = 0 .. 3) in a buffer
ADS_HD constexpr int bwd_layer(int l) { return l * TcSmemB::LAYER; }
// MN-major view of a width-64 [a | 1] copy (rows = K = points, columns = N):
// 8-point groups 128 B apart (LBO), 8-column chunks 2 KB apart (SBO); a
// k-step of 16 points is 256 B
ADS_D uint64_t desc_mn_chunk(uint32_t base, int kstep) {
  const uint32_t lo = (base >> 4) + (uint32_t)kstep * 16u + (8u << 16);
  const uint32_t hi = ((uint32_t)kChunk >> 4) | (1u << 14);
  return ((uint64_t)hi << 32) | lo;
}
// TMEM columns: delta product [0,64), dW5 [64,144), dW4 [144,224),
// dW3 [224,304), dW2 [304,384), dW1 [384,400); in each dW block the weight
// part is columns [0,64) and the bias part column 64 (of [64,80))
constexpr int kColDel = 0, kColW5 = 64, kColW4 = 144, kColW1 = 384;
ADS_D int col_dw(int L) { return L == 5 ? kColW5 : (L == 1 ? kColW1 : kColW4 + (4 - L) * kWP); }


template <int DIN>
__device__ __forceinline__ void bwd_tc_body(const MlpTcArgs& a, int bid, int nblk) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* wt = sm + TcSmemB::W;
  unsigned char* act = sm + TcSmemB::ACT;  // [buffer][a_1..a_4]
  unsigned char* del = sm + TcSmemB::DEL;  // two delta tiles
  unsigned char* xin = sm + TcSmemB::XIN;
  float* fW5 = reinterpret_cast<float*>(sm + TcSmemB::VEC);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + TcSmemB::BAR);
  uint64_t* mb_prod = mbar;       // delta product of a layer complete (issuer commit)
  uint64_t* mb_load = mbar + 1;   // [2] activation buffers loaded (bulk copy)
  uint64_t* mb_ready = mbar + 3;  // a delta tile written (one arrive per epilogue warp)
  uint64_t* mb_done = mbar + 4;   // every product of a tile complete (issuer commit)
  uint64_t* mb_free = mbar + 5;   // a tile's products up to dW_2 complete: its activation
                                  // buffer and delta tiles are free (issuer commit)
  // x' and Delta_4 of a tile written (one arrive per epilogue warp).  Apart
  // from mb_ready: a warp may write the next tile's Delta_4 once mb_free has
  // completed, before a slower warp has arrived for the previous Delta_1
  uint64_t* mb_ready4 = mbar + 6;
  uint32_t* tbase = reinterpret_cast<uint32_t*>(sm + TcSmemB::BAR + 56);
  volatile int* abort_flag = reinterpret_cast<int*>(sm + TcSmemB::BAR + 60);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool epi = tid < kBwdEpi;
  const int row = tid & (kTP - 1), c0 = 32 * (tid >> 7);  // epilogue: point row, first column
  constexpr int RGW = (kW / 8) * 128, RGD = RGW, RGX = (kXP / 8) * 128;
  // a tile's activations: 64 KB in HBM (four layers of 16 KB), 76 KB in a
  // shared buffer (a_1 .. a_3 followed by their constant chunks)
  constexpr uint32_t kSmTile = TcSmemB::ACT_TILE, kGlTile = st_tile_bytes(kW), kGlLayer = st_layer_bytes(kW);
  const float* th = a.theta;
  const int ob1 = kW * DIN, o2 = ob1 + kW, o5 = o2 + 3 * (kW * kW + kW);
  const int ntiles = a.tile_count;  // local tile t is global tile a.tile0 + t
  if (epi) {
    load_hidden_weights<kW, kBwdEpi>(th, o2, wt, tid);
    for (int i = tid; i < kW; i += kBwdEpi) fW5[i] = th[o5 + i];
    // the constant chunks of [a_l | 1] in both buffers: [1, 0, ..., 0] and
    // zeros in every row (the copies of a tile never write them)
    for (int i = tid; i < 2 * 3 * 2 * kTP; i += kBwdEpi) {
      const int r = i % kTP, ch = (i / kTP) % 2, l = (i / (2 * kTP)) % 3, b = i / (6 * kTP);
      *reinterpret_cast<uint4*>(act + b * kSmTile + bwd_layer(l) + (8 + ch) * kChunk + r * 16) =
          ch == 0 ? make_uint4(0x3F80u, 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    }
  }
  if (tid == 0) {
    *abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_prod)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_load)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_load + 1)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_addr(mb_ready)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_done)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_free)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_addr(mb_ready4)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tbase)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  bool first = true;  // this CTA has not finished a tile

  float acc5[32];  // epilogue: running sums of g a_4 over the CTA's tiles (this row, 32 columns)
  float acc5b = 0.0f;  // and of g
#pragma unroll
  for (int j = 0; j < 32; ++j) acc5[j] = 0.0f;
  if (tid == kBwdEpi) {
    // ---------------- issuing thread ----------------
    const uint32_t wt_s = smem_addr(wt), act_s = smem_addr(act), del_s = smem_addr(del),
                   xin_s = smem_addr(xin);
    // dW_l | db_l: M = 128 (o; rows 64 .. 127 unused), N = 80 ([a | 1]), K = points
    // M = 64: exactly the 64 output rows (the M = 64 accumulator layout, m64_row)
    const uint32_t id_dw = idesc_bf16(kW, kWP, 1, 1);
    const uint32_t id_db = idesc_bf16(kW, kXP, 1, 1);  // dW_1 | db_1: N = 16 ([x' | 1])
    const uint32_t id_dp = idesc_bf16(kTP, kW, 0, 1);   // delta product: M = points, N = 64, K = 64
    uint32_t ph_ready = 0, ph_ready4 = 0, ph_free = 0, lph = 0;
    int pend = -1;  // buffer whose bulk copy is in flight (at most one), or -1
    auto fail = [&]() { *abort_flag = 1; };
    // the four stored layers of a tile into buffer b (one barrier)
    auto load_tile = [&](int b, int t) {
      mbar_expect(mb_load + b, kGlTile);
      const unsigned char* src = a.acts + (size_t)t * kGlTile;
#pragma unroll
      for (int l = 0; l < 4; ++l) bulk_load(act + b * kSmTile + bwd_layer(l), src + l * kGlLayer, kGlLayer, mb_load + b);
      pend = b;
    };
    if (bid < ntiles) load_tile(0, bid);
    int it = 0;
    for (int tile = bid; tile < ntiles && !*abort_flag; tile += nblk, ++it) {
      const int buf = it & 1;
      const uint32_t actb_s = act_s + buf * kSmTile;
      if (!mbar_wait(mb_load + buf, (lph >> buf) & 1u)) { fail(); break; }
      lph ^= 1u << buf;
      pend = -1;
      // the previous tile's products have read the other buffer: wait for
      // them, then fetch the next tile into it
      if (it > 0) {
        if (!mbar_wait(mb_free, ph_free)) { fail(); break; }
        ph_free ^= 1;
      }
      if (tile + nblk < ntiles) load_tile(1 - buf, tile + nblk);
      // x' and Delta_4 written
      if (!mbar_wait(mb_ready4, ph_ready4)) { fail(); break; }
      ph_ready4 ^= 1;
      tc_fence_after();
      int cur = 1;  // delta tile holding Delta_L
      bool bad = false;
      for (int L = 4; L >= 2; --L) {
        if (L < 4) {
          if (!mbar_wait(mb_ready, ph_ready)) { bad = true; break; }
          ph_ready ^= 1;
          tc_fence_after();
        }
        const uint32_t dcur = del_s + cur * TcSmemB::DEL_SZ;
        const uint32_t ain = actb_s + bwd_layer(L - 2);  // [a_{L-1} | 1]
        const uint32_t wl = wt_s + (L - 2) * kW * kW * 2;
        // Delta_L W_L, then its commit: the epilogues wait for this alone
#pragma unroll
        for (int ks = 0; ks < kW / 16; ++ks)
          mma_bf16(tmem + kColDel, desc_k(dcur, RGD, ks), desc_mn(wl, RGW, ks), id_dp, ks > 0);
        mma_commit(mb_prod);
        // dW_L | db_L += Delta_L^T [a_{L-1} | 1]
#pragma unroll
        for (int ks = 0; ks < kTP / 16; ++ks) {
          const uint64_t da = desc_mn(dcur, RGD, ks);
          const uint32_t acc = (ks > 0 || !first) ? 1u : 0u;
          mma_bf16(tmem + col_dw(L), da, desc_mn_chunk(ain, ks), id_dw, acc);
        }
        cur = 1 - cur;
      }
      if (bad) { fail(); break; }
      // the activation buffer and delta tile 1 are free once these complete
      // (products complete in issue order); dW_1 reads only Delta_1 and x'
      mma_commit(mb_free);
      // Delta_1 written: dW_1, db_1 += Delta_1^T [x' | 1]
      if (!mbar_wait(mb_ready, ph_ready)) { fail(); break; }
      ph_ready ^= 1;
      tc_fence_after();
      {
        const uint32_t dcur = del_s + cur * TcSmemB::DEL_SZ;
#pragma unroll
        for (int ks = 0; ks < kTP / 16; ++ks)
          mma_bf16(tmem + col_dw(1), desc_mn(dcur, RGD, ks), desc_mn(xin_s + buf * TcSmemB::XIN_SZ, RGX, ks), id_db,
                   (ks > 0 || !first) ? 1u : 0u);
      }
      mma_commit(mb_done);
      first = false;
    }
    // a prefetch still in flight after an abort must land before the CTA's
    // shared memory is released
    if (*abort_flag && pend >= 0) mbar_wait(mb_load + pend, (lph >> pend) & 1u);
  } else if (epi) {
    // ---------------- epilogue warps: point row `row`, columns c0 .. c0 + 32 ----------------
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t ph_prod = 0, ph_free = 0, lph = 0;
    auto arrive_ready = [&](uint64_t* mb) {
      fence_async_smem();  // generic stores before the tensor cores read them
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(mb);
    };
    int it = 0;
    // dL/du of this row: loaded one tile ahead
    float g_next = 0.0f;
    if (bid < ntiles) {
      const int i0 = (a.tile0 + bid) * kTP + row;
      g_next = i0 < a.npts ? a.gu[i0] : 0.0f;
    }
    for (int tile = bid; tile < ntiles && !*abort_flag; tile += nblk, ++it) {
      const int buf = it & 1;
      const unsigned char* actb = act + buf * kSmTile;
      const int idx = (a.tile0 + tile) * kTP + row;
      const float g = g_next;
      if (tile + nblk < ntiles) {
        const int i1 = idx + nblk * kTP;
        g_next = i1 < a.npts ? a.gu[i1] : 0.0f;
      }
      float x[3];
      coords<DIN>(min(idx, a.npts - 1), a.N, x);
      // this tile's activations; Delta_4 = W_5 g (1 - a_4^2) and the
      // output-layer sums in registers before the previous tile's products
      // have released x' and the delta tiles
      if (!mbar_wait(mb_load + buf, (lph >> buf) & 1u)) { *abort_flag = 1; break; }
      lph ^= 1u << buf;
      float v4[32];
#pragma unroll
      for (int c = 0; c < 32; c += 8) {
        float av[8];
        ld_atom_at(actb + bwd_layer(3) + st_off(kW, row, c0 + c), av);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          v4[c + j] = fW5[c0 + c + j] * g * (1.0f - av[j] * av[j]);
          acc5[c + j] += g * av[j];
        }
      }
      acc5b += g;
      // the previous tile's products up to dW_2 have released delta tile 1;
      // x' goes to this tile's buffer (the tile before the previous one
      // read it, and its dW_1 completed before the previous tile's dW_2)
      if (it > 0) {
        if (!mbar_wait(mb_free, ph_free)) { *abort_flag = 1; break; }
        ph_free ^= 1;
        tc_fence_after();
      }
      if (c0 == 0) {
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int d = 0; d < DIN; ++d) v[d] = x[d];
        v[DIN] = 1.0f;
        st_atom(xin + buf * TcSmemB::XIN_SZ, RGX, row, 0, v);
        st_atom(xin + buf * TcSmemB::XIN_SZ, RGX, row, 8, z);
      }
#pragma unroll
      for (int c = 0; c < 32; c += 8) st_atom(del + TcSmemB::DEL_SZ, RGD, row, c0 + c, v4 + c);
      arrive_ready(mb_ready4);
      int cur = 1;
      bool bad = false;
      for (int L = 4; L >= 2; --L) {
        // Delta_{L-1} = (Delta_L W_L)(1 - a_{L-1}^2) into the other delta
        // tile; the second factor before the product is ready
        const unsigned char* aprev = actb + bwd_layer(L - 2);
        float sq[32];
#pragma unroll
        for (int c = 0; c < 32; c += 8) {
          float av[8];
          ld_atom_at(aprev + st_off(kW, row, c0 + c), av);
#pragma unroll
          for (int j = 0; j < 8; ++j) sq[c + j] = 1.0f - av[j] * av[j];
        }
        if (!mbar_wait(mb_prod, ph_prod)) { bad = true; break; }
        ph_prod ^= 1;
        tc_fence_after();
        unsigned char* dn = del + (1 - cur) * TcSmemB::DEL_SZ;
        uint32_t dr[32];
        tmem_ld32_async(lane_base + kColDel + c0, dr);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        reg_pin32(dr);
#pragma unroll
        for (int c = 0; c < 32; c += 8) {
          float v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(dr[c + j]) * sq[c + j];
          st_atom(dn, RGD, row, c0 + c, v);
        }
        arrive_ready(mb_ready);
        cur = 1 - cur;
      }
      if (bad) { *abort_flag = 1; break; }
      first = false;
    }
    // the last tile's products, before the accumulators are read (mb_done
    // completes once per tile; the last tile's phase has parity (it - 1) & 1)
    if (!first && !*abort_flag) {
      if (!mbar_wait(mb_done, (uint32_t)(it - 1) & 1u)) *abort_flag = 1;
      tc_fence_after();
    }
  }
  __syncthreads();
  const bool aborted = *abort_flag != 0;
  const bool had_tiles = bid < ntiles;
  const bool live = !aborted && had_tiles;
  float* gacc = a.gpart + (size_t)bid * a.nparams;
  // output layer: the rows' running sums through shared memory (the
  // activation buffers are idle now), added over the rows in a fixed order
  constexpr int kRedBytes = (kTP * (kW + 1) * 4 + 1023) / 1024 * 1024;
  if (live) {
    float* red = reinterpret_cast<float*>(act);  // [128 rows][65]
    if (epi) {
#pragma unroll
      for (int j = 0; j < 32; ++j) red[row * 65 + c0 + j] = acc5[j];
      if (c0 == 0) red[row * 65 + kW] = acc5b;
    }
    __syncthreads();
    if (tid <= kW) {
      float sum = 0.0f;
      for (int r = 0; r < kTP; ++r) sum += red[r * 65 + tid];
      gacc[o5 + tid] = sum;
    }
  }
  // hidden layers: row o of the M = 64 accumulators in lane m64_row of warps
  // 0-3, through shared memory past the output-layer sums
  const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  float* S = reinterpret_cast<float*>(act + kRedBytes);
  for (int L = 4; L >= 2; --L)
    dw_layer_out<kW, kBwdThreads, true, true>(lane_base + col_dw(L), live, 0.0f, S,
                                              gacc + o2 + (L - 2) * (kW * kW + kW), tid);
  if (tid < kTP) {
    const int o = m64_row(tid);
    if (live) {
      float v[16];
      tmem_ld16(lane_base + col_dw(1), v);  // warp-collective
      if (o >= 0 && o < kW) {
        for (int d = 0; d < DIN; ++d) gacc[o * DIN + d] = v[d];
        gacc[ob1 + o] = v[DIN];
      }
    } else if (!had_tiles) {
      for (int i = tid; i < a.nparams; i += kTP) gacc[i] = 0.0f;  // CTA without tiles
    }
  }
  if (aborted && tid == 0) atomicOr(a.flags, 8);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}
template <int DIN>
__global__ void __launch_bounds__(kBwdThreads) k_mlp_bwd_tc(MlpTcArgs a) {
  bwd_tc_body<DIN>(a, blockIdx.x, gridDim.x);
}
// grouped: CTA g.cta[b].y of context g.cta[b].x's backward (its gradient
// partial row), as in that context's own launch
template <int DIN>
__global__ void __launch_bounds__(kBwdThreads) k_mlp_bwd_tc_grp(const MlpTcArgs* __restrict__ tab, GroupMap g) {
  const int2 m = g.cta[blockIdx.x];
  bwd_tc_body<DIN>(tab[m.x], m.y, g.grid[m.x]);
}


// backward, ring form (W = 128; it also compiles for W = 64).  TMEM holds
// the delta product (W columns) and the three hidden dW accumulators (3 x W):
// all 512 columns for W = 128.  The small gradients (biases,
// output layer, first layer) are per-thread FP32 sums over the points
// (thread o owns output o; fixed order).  Activation tiles stream through a
// two-slot ring, each prefetched while the previous stage computes; the delta
// tile (zero-padded to 128 columns so that dW is an M = 128 product) is
// rewritten in place once the products that read it have completed.
// ---------------------------------------------------------------------------

// Weighted column sums of a BF16 [128][C] core-matrix tile over its 128 rows:
// out[k][o] += sum_t w_k[t] T[t][o] for o < W, k < NW.  Thread layout: ri =
// tid % 8 (row within a core matrix), cg = (tid / 8) % (W / 8) (column group),
// and the row groups are split over the remaining thread index, so that a
// quarter-warp reads 8 consecutive rows of one core-matrix column (128
// contiguous bytes, conflict-free).  Partial sums meet in `red` and are added
// in a fixed order by thread o.
template <int W, int NW>
ADS_D void tile_colsums(const unsigned char* tile, int rg, const float* const* w, float* red,
                        float* out) {
  constexpr int CG = W / 8, NSETS = kTP / (8 * CG), NPART = 8 * NSETS;
  static_assert(kTP % (8 * CG) == 0 && NW <= 4, "one block of kTP threads covers whole row sets");
  const int tid = threadIdx.x;
  const int ri = tid % 8, cg = (tid / 8) % CG, set = tid / (8 * CG);
  float acc[NW][8];
#pragma unroll
  for (int k = 0; k < NW; ++k)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[k][j] = 0.f;
  for (int g = set; g < kTP / 8; g += NSETS) {
    const int t = g * 8 + ri;
    float v[8];
    ld_atom(tile, rg, t, cg * 8, v);
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const float wk = w[k] ? w[k][t] : 1.0f;
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[k][j] += wk * v[j];
    }
  }
  const int part = ri + 8 * set;
#pragma unroll
  for (int k = 0; k < NW; ++k)
#pragma unroll
    for (int j = 0; j < 8; ++j) red[(k * NPART + part) * W + cg * 8 + j] = acc[k][j];
  __syncthreads();
  if (tid < W) {
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      float sum = 0.f;
      for (int q = 0; q < NPART; ++q) sum += red[(k * NPART + q) * W + tid];
      out[k] += sum;
    }
  }
  __syncthreads();
}

template <int W>
struct TcSmemB2 {
  static constexpr int WT = 0;                             // 3 x [W][W] bf16
  static constexpr int ACT = WT + 3 * W * W * 2;           // 2 x [128][W] bf16
  static constexpr int ACT_SZ = kTP * W * 2;
  static constexpr int DEL = ACT + 2 * ACT_SZ;             // [128][128] bf16
  static constexpr int VEC = DEL + kTP * kDP * 2;          // fp32: W5 [W], g [128], x' [3][128]
  static constexpr int RED = VEC + (W + kTP + 3 * kTP) * 4;  // column-sum partials [4][1024/W][W] fp32
  static constexpr int BAR = RED + 4 * (8 * kTP / W) * W * 4;
  static constexpr int TOTAL = BAR + 32;
};

template <int W, int DIN>
__global__ void __launch_bounds__(kTP) k_mlp_bwd_tcr(MlpTcArgs a) {
  static_assert(W == 128, "ring form: the core-matrix layout of stored width-128 tiles");
  constexpr int NCOL = 4 * W;  // TMEM columns: delta product + three dW
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* wt = sm + TcSmemB2<W>::WT;
  unsigned char* act = sm + TcSmemB2<W>::ACT;  // two slots
  unsigned char* del = sm + TcSmemB2<W>::DEL;
  float* fW5 = reinterpret_cast<float*>(sm + TcSmemB2<W>::VEC);
  float* gs = fW5 + W;
  float* xs = gs + kTP;  // [3][128]
  float* red = reinterpret_cast<float*>(sm + TcSmemB2<W>::RED);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + TcSmemB2<W>::BAR);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(sm + TcSmemB2<W>::BAR + 8);
  volatile int* abort_flag = reinterpret_cast<int*>(sm + TcSmemB2<W>::BAR + 12);
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int RG = (W / 8) * 128, RGD = (kDP / 8) * 128;
  const float* th = a.theta;
  const int ob1 = W * DIN, o2 = ob1 + W, o5 = o2 + 3 * (W * W + W);
  load_hidden_weights<W, kTP>(th, o2, wt, tid);
  if (tid < W) fW5[tid] = th[o5 + tid];
  if (W < kDP) {  // zero padding columns of the delta tile (never rewritten)
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int c = W; c < kDP; c += 8) st_atom(del, RGD, tid, c, z);
  }
  if (tid == 0) {
    *abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tbase)), "r"(NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
  const uint32_t wt_s = smem_addr(wt), act_s = smem_addr(act), del_s = smem_addr(del);
  const uint32_t id_dw = idesc_bf16(kDP, W, 1, 1);  // dW_l: M = 128 (o, padded), N = W (k), K = points
  const uint32_t id_dp = idesc_bf16(kTP, W, 0, 1);  // delta product: M = points, N = W, K = W
  auto col_dw2 = [](int L) { return W + (4 - L) * W; };  // dW4, dW3, dW2 after the delta product
  // per-thread small gradients (thread o)
  float g_w5 = 0.f, g_b5 = 0.f, g_b1 = 0.f, g_w1[3] = {0.f, 0.f, 0.f}, g_bh[3] = {0.f, 0.f, 0.f};
  uint32_t phase = 0;
  bool aborted = false, first = true;
  const int ntiles = a.tile_count;  // local tile t is global tile a.tile0 + t
  auto stage = [&](int slot, int L, int tile) {  // activations a_{L+1} (L = 0..3) of `tile`
    const unsigned char* src = a.acts + (size_t)tile * st_tile_bytes(W) + L * st_layer_bytes(W);
    unsigned char* dst = act + slot * TcSmemB2<W>::ACT_SZ;
    for (int ch = tid; ch < kTP * W * 2 / 16; ch += kTP) cp_async16(dst + ch * 16, src + ch * 16);
    cp_async_commit();
  };
  if ((int)blockIdx.x < ntiles) stage(0, 3, blockIdx.x);
  for (int tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x) {
    const int p0 = (a.tile0 + tile) * kTP;
    const int idx = p0 + tid;
    const float g = idx < a.npts ? a.gu[idx] : 0.0f;
    {
      float x[3];
      coords<DIN>(min(idx, a.npts - 1), a.N, x);
      gs[tid] = g;
      for (int d = 0; d < 3; ++d) xs[d * kTP + tid] = x[d];
    }
    cp_async_wait_all();
    if (sync_abort(abort_flag)) {
      aborted = true;
      break;
    }
    stage(1, 2, tile);  // a_3 into the other slot
    const unsigned char* a4 = act;  // slot 0
    // output layer: dW_5[o] += sum_t g_t a_4[t][o], db_5 += sum_t g_t
    {
      const float* wts[1] = {gs};
      tile_colsums<W, 1>(a4, RG, wts, red, &g_w5);
      if (tid == 0) {
        float sb = 0.f;
        for (int t = 0; t < kTP; ++t) sb += gs[t];
        g_b5 += sb;
      }
    }
    // Delta_4 = W_5 g (1 - a_4^2), row tid
#pragma unroll
    for (int c = 0; c < W; c += 8) {
      float av[8], v[8];
      ld_atom(a4, RG, tid, c, av);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = fW5[c + j] * g * (1.0f - av[j] * av[j]);
      st_atom(del, RGD, tid, c, v);
    }
    int slot = 1;  // slot of a_{L-1}
    for (int L = 4; L >= 2; --L) {
      cp_async_wait_all();
      if (sync_abort(abort_flag)) {
        aborted = true;
        break;
      }
      // the slot not holding a_{L-1} is free: prefetch the next activations
      if (L > 2) stage(1 - slot, L - 3, tile);                     // a_{L-2}
      else if (tile + (int)gridDim.x < ntiles) stage(1 - slot, 3, tile + gridDim.x);  // next a_4
      const uint32_t ain = act_s + slot * TcSmemB2<W>::ACT_SZ;
      if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < kTP / 16; ++ks)
          mma_bf16(tmem + col_dw2(L), desc_mn(del_s, RGD, ks), desc_mn(ain, RG, ks), id_dw,
                   (ks > 0 || !first) ? 1u : 0u);
        const uint32_t wl = wt_s + (L - 2) * W * W * 2;
#pragma unroll
        for (int ks = 0; ks < W / 16; ++ks)
          mma_bf16(tmem, desc_k(del_s, RGD, ks), desc_mn(wl, RG, ks), id_dp, ks > 0);
        mma_commit(mbar);
      }
      // db_L[o] += sum_t Delta_L[t][o] while the products run (ends with a CTA barrier,
      // so every column sum has read Delta_L before it is rewritten below)
      {
        const float* wts[1] = {nullptr};
        tile_colsums<W, 1>(del, RGD, wts, red, &g_bh[L - 2]);
      }
      if (!mbar_wait(mbar, phase)) *abort_flag = 1;
      phase ^= 1;
      tc_fence_after();
      // Delta_{L-1} = (Delta_L W_L)(1 - a_{L-1}^2), rewritten in place
      const unsigned char* aprev = act + slot * TcSmemB2<W>::ACT_SZ;
#pragma unroll 2
      for (int c = 0; c < W; c += 16) {
        float dv[16];
        tmem_ld16(lane_base + c, dv);
        float av[8], v[8];
        ld_atom(aprev, RG, tid, c, av);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = dv[j] * (1.0f - av[j] * av[j]);
        st_atom(del, RGD, tid, c, v);
        ld_atom(aprev, RG, tid, c + 8, av);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = dv[8 + j] * (1.0f - av[j] * av[j]);
        st_atom(del, RGD, tid, c + 8, v);
      }
      slot = 1 - slot;
    }
    if (aborted) break;
    __syncthreads();
    // first layer: dW_1[o][d] += sum_t Delta_1[t][o] x'_d[t], db_1[o] += sum_t Delta_1[t][o]
    {
      float sums[DIN + 1];
#pragma unroll
      for (int d = 0; d <= DIN; ++d) sums[d] = 0.f;
      const float* wts[DIN + 1];
#pragma unroll
      for (int d = 0; d < DIN; ++d) wts[d] = xs + d * kTP;
      wts[DIN] = nullptr;
      tile_colsums<W, DIN + 1>(del, RGD, wts, red, sums);  // ends with a CTA barrier
#pragma unroll
      for (int d = 0; d < DIN; ++d) g_w1[d] += sums[d];
      g_b1 += sums[DIN];
    }
    first = false;
  }
  cp_async_wait_all();
  float* gacc = a.gpart + (size_t)blockIdx.x * a.nparams;
  const int o = tid;
  aborted = sync_abort(abort_flag);
  // hidden layers through shared memory (the weight tiles are idle now:
  // every product that read them has completed)
  float* S = reinterpret_cast<float*>(wt);
  static_assert(W * (W + 1) * 4 <= 3 * W * W * 2, "one layer's rows fit the weight tiles");
  for (int L = 4; L >= 2; --L)
    dw_layer_out<W, kTP, false>(lane_base + col_dw2(L), !aborted && !first, g_bh[L - 2], S,
                                gacc + o2 + (L - 2) * (W * W + W), tid);
  if (!aborted && !first) {
    if (o < W) {
      gacc[o5 + o] = g_w5;
      for (int d = 0; d < DIN; ++d) gacc[o * DIN + d] = g_w1[d];
      gacc[ob1 + o] = g_b1;
    }
    if (o == 0) gacc[o5 + W] = g_b5;
  } else if (first) {
    for (int i = tid; i < a.nparams; i += kTP) gacc[i] = 0.0f;
  }
  if (aborted && tid == 0) atomicOr(a.flags, 8);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL));
}

int g_sms = 0;
int sms() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

}  // namespace

size_t mlp_tc_acts_bytes(int npts, int width) {
  int ntiles = (npts + kTP - 1) / kTP;
  return (size_t)ntiles * st_tile_bytes(width);
}



// CTAs of a tensor-memory kernel that fit on one SM: shared memory (with the
// per-block reservation), registers, threads and TMEM columns.  (The runtime's
// occupancy query reports one block per SM for kernels that allocate TMEM.)
template <typename K>
static int tc_residency(K k, size_t smem, int tmem_cols, int threads = kTP) {
  static int per_sm = 0, reserved = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (per_sm <= 0) per_sm = 1;
  }
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, k);
  int occ = per_sm / (int)(smem + reserved);
  const int regs_per_warp = ((fa.numRegs > 0 ? fa.numRegs : 255) * 32 + 255) / 256 * 256;
  const int by_regs = 65536 / (regs_per_warp * (threads / 32));
  if (by_regs < occ) occ = by_regs;
  if (2048 / threads < occ) occ = 2048 / threads;
  if (512 / tmem_cols < occ) occ = 512 / tmem_cols;
  return occ < 1 ? 1 : occ;
}

template <int W, int DIN>
static int bwd_tc_occ() {
  auto k = k_mlp_bwd_tcr<W, DIN>;
  const size_t smem = TcSmemB2<W>::TOTAL;
  smem_optin(k);
  return tc_residency(k, smem, 4 * W);
}

int mlp_tc_bwd_blocks(int npts, int width, int din, int min_tiles) {
  const int ntiles = (npts + kTP - 1) / kTP;
  int occ = 1;
  if (width != 64) occ = din == 2 ? bwd_tc_occ<128, 2>() : bwd_tc_occ<128, 3>();
  // width 64: the all-tensor-core kernel holds 512 TMEM columns, one CTA per SM
  int nb = occ * sms();
  const int want = (ntiles + min_tiles - 1) / (min_tiles > 0 ? min_tiles : 1);
  if (want < nb) nb = want;
  if (nb < 1) nb = 1;
  return ntiles < nb ? ntiles : nb;
}

// the launch's tile range made explicit
static MlpTcArgs tile_range(MlpTcArgs a) {
  const int tot = (a.npts + kTP - 1) / kTP;
  if (a.tile0 < 0) a.tile0 = 0;
  if (a.tile0 > tot) a.tile0 = tot;
  if (a.tile_count <= 0 || a.tile0 + a.tile_count > tot) a.tile_count = tot - a.tile0;
  return a;
}

template <int W, int DIN>
static constexpr int stage_blocks() {
  using L = TcSmemF<W>;
  return (3 * W * (L::KC / 8) + L::VEC_SZ / 4 + 255) / 256;
}

// the forward kernel's grid: at most its residency, at least min_tiles tiles per CTA
template <int W, int DIN>
static int fwd_grid(const MlpTcArgs& a) {
  using L = TcSmemF<W>;
  const int ntiles = a.tile_count;
  if (ntiles <= 0) return 0;
  auto k = k_mlp_fwd_tc<W, DIN>;
  smem_optin(k);
  const int occ = tc_residency(k, L::TOTAL, L::NS * W, fwd_threads<W>());
  int grid = ntiles < occ * sms() ? ntiles : occ * sms();
  const int want = (ntiles + a.min_tiles - 1) / (a.min_tiles > 0 ? a.min_tiles : 1);
  if (want < grid) grid = want > 0 ? want : 1;
  return grid;
}

template <int W, int DIN>
static cudaError_t fwd_tc(const MlpTcArgs& a, cudaStream_t st) {
  using L = TcSmemF<W>;
  const int grid = fwd_grid<W, DIN>(a);
  if (grid <= 0) return cudaSuccess;
  // the weight image from the current parameters, then the forward
  k_stage_fwd<W, DIN><<<stage_blocks<W, DIN>(), 256, 0, st>>>(a.theta, a.wimage);
  MlpTcArgs b = a;
  b.wimage_ctr = reinterpret_cast<int*>(a.wimage + L::IMG);
  k_mlp_fwd_tc<W, DIN><<<grid, fwd_threads<W>(), L::TOTAL, st>>>(b);
  return cudaGetLastError();
}

size_t mlp_tc_fwd_image_bytes(int width) {
  return (width == 64 ? TcSmemF<64>::IMG : TcSmemF<128>::IMG) + 16;  // + the tile-group counter
}

cudaError_t launch_mlp_fwd_tc(const MlpTcArgs& a0, cudaStream_t st) {
  if (a0.npts <= 0) return cudaSuccess;
  if (reinterpret_cast<uintptr_t>(a0.theta) & 15) return cudaErrorInvalidValue;  // 16-byte weight rows
  if (!a0.wimage || (reinterpret_cast<uintptr_t>(a0.wimage) & 15)) return cudaErrorInvalidValue;
  const MlpTcArgs a = tile_range(a0);
  if (a.width == 64) return a.din == 2 ? fwd_tc<64, 2>(a, st) : fwd_tc<64, 3>(a, st);
  if (a.width == 128) return a.din == 2 ? fwd_tc<128, 2>(a, st) : fwd_tc<128, 3>(a, st);
  return cudaErrorNotSupported;
}

// ---- grouped launches (width 64): the tables hold each context's launch
// arguments as mlp_tc_group_args makes them ----
MlpTcArgs mlp_tc_group_args(const MlpTcArgs& a0, int* fwd_ctas) {
  MlpTcArgs a = tile_range(a0);
  a.wimage_ctr = reinterpret_cast<int*>(a.wimage + TcSmemF<64>::IMG);
  *fwd_ctas = a.width != 64 ? 0 : (a.din == 2 ? fwd_grid<64, 2>(a) : fwd_grid<64, 3>(a));
  return a;
}

cudaError_t launch_mlp_tc_grouped(int which, int din, const MlpTcArgs* tab, int nctx, GroupMap g, int nctas,
                                  cudaStream_t st) {
  if (nctx <= 0 || nctas <= 0) return cudaSuccess;
  if (din != 2 && din != 3) return cudaErrorInvalidValue;
  if (which == 0) {  // the weight images
    const dim3 grid(stage_blocks<64, 2>(), nctx);
    if (din == 2) k_stage_fwd_grp<64, 2><<<grid, 256, 0, st>>>(tab);
    else k_stage_fwd_grp<64, 3><<<grid, 256, 0, st>>>(tab);
  } else if (which == 1) {  // the forwards
    auto k = din == 2 ? k_mlp_fwd_tc_grp<64, 2> : k_mlp_fwd_tc_grp<64, 3>;
    smem_optin(k);
    k<<<nctas, fwd_threads<64>(), TcSmemF<64>::TOTAL, st>>>(tab, g);
  } else if (which == 2) {  // the backwards
    auto k = din == 2 ? k_mlp_bwd_tc_grp<2> : k_mlp_bwd_tc_grp<3>;
    smem_optin(k);
    k<<<nctas, kBwdThreads, TcSmemB::TOTAL, st>>>(tab, g);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int W, int DIN>
static cudaError_t bwd_tc(const MlpTcArgs& a, int nblk, cudaStream_t st) {
  auto k = k_mlp_bwd_tcr<W, DIN>;
  const size_t smem = TcSmemB2<W>::TOTAL;
  smem_optin(k);
  k<<<nblk, kTP, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mlp_bwd_tc(const MlpTcArgs& a0, int nblk, cudaStream_t st) {
  if (reinterpret_cast<uintptr_t>(a0.theta) & 15) return cudaErrorInvalidValue;  // 16-byte weight rows
  const MlpTcArgs a = tile_range(a0);
  if (a.width == 64) {
    const size_t smem = TcSmemB::TOTAL;
    auto k = a.din == 2 ? k_mlp_bwd_tc<2> : k_mlp_bwd_tc<3>;
    smem_optin(k);
    k<<<nblk, kBwdThreads, smem, st>>>(a);
    return cudaGetLastError();
  }
  if (a.width == 128) return a.din == 2 ? bwd_tc<128, 2>(a, nblk, st) : bwd_tc<128, 3>(a, nblk, st);
  return cudaErrorNotSupported;
}

}  // namespace adsgb

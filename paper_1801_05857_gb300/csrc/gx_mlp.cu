// The scoring network of the guided deadlock search (no counterpart in the
// paper): a small MLP that predicts a state's distance to the nearest deadlock
// from the histogram of its processes' local states.
//
//   x  = bf16(hist / n)                 (hist[i] = processes in local state i, i < 16;
//                                        n = sum of hist = the network's processes)
//   h1 = bf16(relu(W1 x + b1))          W1: 128 x 16
//   h2 = relu(W2 h1 + b2)               W2: 128 x 128
//   y  = w3 . h2 + b3
//
// The one-hot local state of each process, averaged over processes, is the
// input: the first layer's weights are shared by all processes, and the
// input has the same scale at every network size, which is what lets a
// network trained on small instances score states of larger ones.
// Weights are used in BF16 (rounded to nearest even from FP32 master copies
// that the optimiser updates), and so is each layer's input (x and h1 are
// rounded from FP32), so that both layers are BF16 x BF16 products with
// FP32 accumulation -- the operand types of the tensor cores.  Inference
// (gx_mlp_forward, and the guided search's scoring) and the gradient
// (gx_mlp_grad, gx_mlp_train: grad_tc_kernel below) run on the tensor cores
// (gx_tc.cuh).
//
// Parameter vector (FP32, GX_MLP_PARAMS floats): W1 | b1 | W2 | b2 | w3 | b3.
// Loss: mean over the batch of (y - label)^2.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "gx_kernels.h"
#include "gx_tc.cuh"

namespace gxm {

constexpr int IN = GX_MLP_IN;
constexpr int H = GX_MLP_HIDDEN;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + H * IN;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H;
constexpr int NPARAM = OFF_B3 + 1;
static_assert(NPARAM == GX_MLP_PARAMS, "parameter count");
constexpr int kGradCtas = GX_MLP_GRAD_CTAS;  // at most this many CTAs, one partial gradient each

// g[i] = sum over the CTAs c, in order, of partial[c][i]; *loss likewise.
__global__ void reduce_kernel(const float* __restrict__ partial, const float* __restrict__ partial_loss, int ctas,
                              float* __restrict__ g, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < NPARAM) {
    float acc = 0.f;
    for (int c = 0; c < ctas; ++c) acc += partial[(uint64_t)c * NPARAM + i];
    g[i] = acc;
  }
  if (i == 0) {
    float l = 0.f;
    for (int c = 0; c < ctas; ++c) l += partial_loss[c];
    *loss = l;
  }
}

// Inference on the tensor cores: persistent over tiles of 128 examples.
__device__ unsigned int g_tc_error;
// The weights gx_mlp_forward scores with, packed for the tensor cores (one
// copy per device; calls hold g_forward_mutex from packing to completion).
__device__ gxt::TcWeights g_tc_packed;

__global__ void __launch_bounds__(gxt::kRows) mlp_tc_forward_kernel(const gxt::TcWeights* __restrict__ packed,
                                                                     const uint8_t* __restrict__ hist, uint64_t n,
                                                                     float* __restrict__ out) {
  extern __shared__ __align__(16) uint8_t tsm[];
  const uint64_t tiles = (n + gxt::kRows - 1) / gxt::kRows;
  if (blockIdx.x >= tiles) return;
  gxt::TcScorer sc = gxt::tc_setup(tsm, packed);
  if (!sc.ok) {
    gxt::tc_teardown(sc);
    if (threadIdx.x == 0) atomicOr(&g_tc_error, 1u);
    return;
  }
  for (uint64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const uint64_t row = tile * gxt::kRows + threadIdx.x;
    uint32_t hw[4] = {0, 0, 0, 0};
    if (row < n) {
      const uint8_t* h = hist + row * IN;
#pragma unroll
      for (int i = 0; i < IN; ++i) hw[i >> 2] |= (uint32_t)h[i] << ((i & 3) * 8);
    }
    float y = 0.f;
    if (!gxt::tc_score_tile(sc, hw, y)) {
      if (threadIdx.x == 0) atomicOr(&g_tc_error, 1u);
      break;
    }
    if (row < n) out[row] = y;
  }
  gxt::tc_teardown(sc);
}

// ---- Gradient on the tensor cores.  One CTA of 128 threads per tile of 128
// examples (thread t: example t of the tile, TMEM lane t), all of TMEM (512
// columns) per CTA.  Every product is a tcgen05 BF16 x BF16 -> FP32 MMA with
// K-major operands in shared memory (transposed operands are written
// transposed, so every descriptor has the same form as the scorer's):
//   A1  = X W1^T,  H = bf16(relu(A1 + b1))              (forward, as the scorer)
//   A2  = H W2^T,  y = b3 + w3 . relu(A2 + b2)
//   dy  = 2 (y - label) / n,  D2 = dy w3^T o (A2 + b2 > 0)        (thread-local)
//   DH  = D2 W2                                          [128 x 128]
//   [gW2 | gb2] += D2^T [H | 1]                          N = 128 + 16 (ones rows)
//   DA1 = DH o (A1 + b1 > 0)
//   [gW1 | gb1] += DA1^T [X | 1]                         N = 16 + 16
// The gradients accumulate in TMEM over the CTA's tiles, in tile order; gw3 and
// gb3 are summed on the CUDA cores (a fixed butterfly over each warp's lanes,
// then the warps in order), so a CTA's partial gradient does not depend on
// scheduling.  D2 and DA1 enter their products rounded to BF16.
constexpr uint32_t kTrainCols = 512;
constexpr uint32_t kColAcc = 0, kColDH = 128, kColGW2 = 256, kColGW1 = 400;
// instruction descriptors: M = 128 with N = 128, 144 (H^T and 16 ones rows), 32 (X^T and 16 ones rows)
constexpr uint32_t kI128 = gxt::idesc_bf16_f32(128, 128), kI144 = gxt::idesc_bf16_f32(128, 144),
                   kI32 = gxt::idesc_bf16_f32(128, 32);

// The parameters as a training CTA holds them: the scorer's image plus W2
// transposed (the B operand of DH = D2 W2: rows j, K = k).
struct __align__(16) TcTrainWeights {
  gxt::TcWeights fw;
  uint8_t w2t[H * H * 2];
};
static_assert(sizeof(TcTrainWeights) % 16 == 0, "bulk copies move multiples of 16 bytes");

struct __align__(1024) TrainSmem {
  uint8_t x[gxt::kRows * IN * 2];      // A of layer 1: [r][i], K groups 2
  uint8_t xto[32 * gxt::kRows * 2];    // B of gW1|gb1: rows 0-15 X^T [i][r], rows 16-31 ones; K groups 16
  uint8_t h[gxt::kRows * H * 2];       // A of layer 2: H [r][j]; then DA1^T [j][r], A of gW1
  uint8_t hto[(H + 16) * gxt::kRows * 2];  // B of gW2|gb2: rows 0-127 H^T [j][r], rows 128-143 ones
  uint8_t d[gxt::kRows * H * 2];       // A of DH: D2 [r][k]
  uint8_t dt[H * gxt::kRows * 2];      // A of gW2: D2^T [k][r]
  TcTrainWeights wt;
  float red[4][H];                     // per-warp sums of the gw3 terms
  float redl[4][2];                    // per-warp loss and gb3
  uint32_t tmem_slot;
  unsigned long long mbar, mbar_load;
};
constexpr size_t kTrainSmemBytes = sizeof(TrainSmem) + 1024;  // + alignment slack
static_assert(kTrainSmemBytes <= 232448, "a training CTA must fit the SM's shared memory");

// W2^T in the core-matrix layout: item (row j, K group g) packs W2[8g .. 8g+7][j].
constexpr int kTrainPackItems = gxt::kTcPackItems + H * 16;
__global__ void train_pack_kernel(const float* __restrict__ p, TcTrainWeights* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kTrainPackItems; i += gridDim.x * blockDim.x) {
    if (i < gxt::kTcPackItems) {
      gxt::tc_pack_item(p, &out->fw, i);
      continue;
    }
    const int item = i - gxt::kTcPackItems, j = item >> 4, g = item & 15;
    const float* c = p + OFF_W2 + (g * 8) * H + j;  // W2[8g][j], stride H down the column
    uint4 q;
    q.x = gxt::pack_bf16x2(c[0 * H], c[1 * H]);
    q.y = gxt::pack_bf16x2(c[2 * H], c[3 * H]);
    q.z = gxt::pack_bf16x2(c[4 * H], c[5 * H]);
    q.w = gxt::pack_bf16x2(c[6 * H], c[7 * H]);
    *reinterpret_cast<uint4*>(out->w2t + gxt::core_offset(j, g * 8, 16)) = q;
  }
}
constexpr int kTrainPackBlocks = (kTrainPackItems + 255) / 256;

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// Sum of v over the warp's 32 lanes for 32 columns at once, in a fixed order
// (recursive halving: at step h the lanes with bit h set keep the upper half of
// their columns), so lane l ends with the sum of column l.
__device__ __forceinline__ float warp_column_sums(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int half = 16; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float send = up ? v[i] : v[i + half];
      const float keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, half);
    }
  }
  return v[0];
}

__device__ unsigned int g_train_error;  // a bounded wait gave up (GX_ERR_SPIN_LIMIT)
// The weights a gradient is taken at, packed for the tensor cores (one copy per
// device; calls hold g_train_mutex from packing to completion).
__device__ TcTrainWeights g_train_packed;

// CTA c takes tiles c, c + gridDim.x, ... of the n examples (example index[s]
// for slot s when index is given) and writes its partial gradient of the mean
// loss (inv_n = 1 / n) to partial[c], its loss to partial_loss[c].
__global__ void __launch_bounds__(gxt::kRows, 1) grad_tc_kernel(const TcTrainWeights* __restrict__ packed,
                                                                const uint8_t* __restrict__ hist,
                                                                const float* __restrict__ label, uint64_t n,
                                                                const uint64_t* __restrict__ index, float inv_n,
                                                                float* __restrict__ partial,
                                                                float* __restrict__ partial_loss) {
  extern __shared__ __align__(16) uint8_t gsm[];
  TrainSmem* s = reinterpret_cast<TrainSmem*>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~uintptr_t(1023));
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const uint64_t tiles = (n + gxt::kRows - 1) / gxt::kRows;
  if (blockIdx.x >= tiles) return;
  using namespace gxt;
  if (t == 0) {
    mbar_init(saddr(&s->mbar), 1);
    mbar_init(saddr(&s->mbar_load), 1);
    mbar_expect_tx(saddr(&s->mbar_load), (uint32_t)sizeof(TcTrainWeights));
    bulk_g2s(saddr(&s->wt), packed, (uint32_t)sizeof(TcTrainWeights), saddr(&s->mbar_load));
  }
  if (t < 32) {
    __syncwarp();
    tmem_alloc(saddr(&s->tmem_slot), kTrainCols);
    tmem_relinquish();
  }
  // the ones rows of the two stacked B operands (their products give the bias gradients)
  for (int i = t; i < 16 * gxt::kRows; i += gxt::kRows) {
    st_bf16(s->xto, core_offset(16 + i / gxt::kRows, i % gxt::kRows, 16), 1.f);
    st_bf16(s->hto, core_offset(H + i / gxt::kRows, i % gxt::kRows, 16), 1.f);
  }
  tc_fence_before();
  tc_sync();
  tc_fence_after();
  bool ok = mbar_wait_bounded(saddr(&s->mbar_load), 0);
  if (!ok) ok = mbar_wait_bounded(saddr(&s->mbar_load), 0);  // the copy must land before the CTA leaves
  ok = tc_sync_or(!ok) == 0;
  const uint32_t tm = s->tmem_slot, lb = (uint32_t)(t & ~31) << 16;
  constexpr uint32_t i128 = kI128, i144 = kI144, i32 = kI32;
  uint32_t phase = 0;
  // one commit, then every thread waits; false when any thread gave up
  auto commit_wait = [&]() -> bool {
    if (t == 0) mma_commit(saddr(&s->mbar));
    const bool w = mbar_wait_bounded(saddr(&s->mbar), phase);
    phase ^= 1u;
    const int bad = tc_sync_or(!w);
    tc_fence_after();
    return bad == 0;
  };
  float gw3acc[4] = {0.f, 0.f, 0.f, 0.f}, gb3acc = 0.f, lossacc = 0.f;
  uint32_t first = 1;
  const TcWeights& W = s->wt.fw;
  for (uint64_t tile = blockIdx.x; ok && tile < tiles; tile += gridDim.x) {
    const uint64_t row = tile * gxt::kRows + t;
    const bool valid = row < n;
    const uint64_t ex = valid ? (index ? index[row] : row) : 0;
    // X = bf16(hist / processes), and X^T
    uint32_t cnt[IN], tot = 0;
#pragma unroll
    for (int i = 0; i < IN; ++i) {
      cnt[i] = valid ? hist[ex * IN + i] : 0u;
      tot += cnt[i];
    }
    const float inv = tot ? 1.f / (float)tot : 0.f;
    {
      uint32_t q[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) q[i] = pack_bf16x2((float)cnt[2 * i] * inv, (float)cnt[2 * i + 1] * inv);
      *reinterpret_cast<uint4*>(s->x + core_offset(t, 0, 2)) = make_uint4(q[0], q[1], q[2], q[3]);
      *reinterpret_cast<uint4*>(s->x + core_offset(t, 8, 2)) = make_uint4(q[4], q[5], q[6], q[7]);
#pragma unroll
      for (int i = 0; i < IN; ++i) st_bf16(s->xto, core_offset(i, t, 16), (float)cnt[i] * inv);
    }
    const float lab = valid ? label[ex] : 0.f;
    fence_async_smem();
    tc_sync();
    if (t == 0) {
      tc_fence_after();
      mma_bf16_i(tm + kColAcc, smem_desc(saddr(s->x), 128, 256), smem_desc(saddr(W.w1), 128, 256), i128, 0u);
    }
    if (!(ok = commit_wait())) break;
    // H = bf16(relu(A1 + b1)) and H^T; the ReLU's mask of A1 kept for the backward pass
    uint32_t mask1[4];
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float a[32];
      tmem_ld32(tm + lb + kColAcc + 32 * c, a);
      uint32_t m = 0, q[16];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        a[e] += W.b1[32 * c + e];
        if (a[e] > 0.f) m |= 1u << e;
        a[e] = fmaxf(a[e], 0.f);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) q[e] = pack_bf16x2(a[2 * e], a[2 * e + 1]);
#pragma unroll
      for (int g = 0; g < 4; ++g)
        *reinterpret_cast<uint4*>(s->h + core_offset(t, 32 * c + 8 * g, 16)) =
            make_uint4(q[4 * g], q[4 * g + 1], q[4 * g + 2], q[4 * g + 3]);
#pragma unroll
      for (int e = 0; e < 32; ++e) st_bf16(s->hto, core_offset(32 * c + e, t, 16), a[e]);
      mask1[c] = m;
    }
    tc_fence_before();
    fence_async_smem();
    tc_sync();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (uint32_t kk = 0; kk < H / 16; ++kk)
        mma_bf16_i(tm + kColAcc, smem_desc(saddr(s->h) + 256u * kk, 128, 2048),
                   smem_desc(saddr(W.w2) + 256u * kk, 128, 2048), i128, kk > 0 ? 1u : 0u);
    }
    if (!(ok = commit_wait())) break;
    // y, then dy, D2 = dy w3 o (A2 + b2 > 0) and the gw3 terms dy relu(A2 + b2)
    float y = W.b3;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float a[32];
      tmem_ld32(tm + lb + kColAcc + 32 * c, a);
#pragma unroll
      for (int e = 0; e < 32; ++e) y += W.w3[32 * c + e] * fmaxf(a[e] + W.b2[32 * c + e], 0.f);
    }
    const float dy = valid ? 2.f * (y - lab) * inv_n : 0.f;
    if (valid) lossacc += (y - lab) * (y - lab) * inv_n;
    gb3acc += dy;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float a[32], v[32];
      tmem_ld32(tm + lb + kColAcc + 32 * c, a);
      uint32_t q[16];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const float z = a[e] + W.b2[32 * c + e];
        v[e] = dy * fmaxf(z, 0.f);
        a[e] = z > 0.f ? dy * W.w3[32 * c + e] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) q[e] = pack_bf16x2(a[2 * e], a[2 * e + 1]);
#pragma unroll
      for (int g = 0; g < 4; ++g)
        *reinterpret_cast<uint4*>(s->d + core_offset(t, 32 * c + 8 * g, 16)) =
            make_uint4(q[4 * g], q[4 * g + 1], q[4 * g + 2], q[4 * g + 3]);
#pragma unroll
      for (int e = 0; e < 32; ++e) st_bf16(s->dt, core_offset(32 * c + e, t, 16), a[e]);
      gw3acc[c] += warp_column_sums(v);
    }
    tc_fence_before();
    fence_async_smem();
    tc_sync();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (uint32_t kk = 0; kk < H / 16; ++kk)
        mma_bf16_i(tm + kColDH, smem_desc(saddr(s->d) + 256u * kk, 128, 2048),
                   smem_desc(saddr(s->wt.w2t) + 256u * kk, 128, 2048), i128, kk > 0 ? 1u : 0u);
#pragma unroll
      for (uint32_t kk = 0; kk < gxt::kRows / 16; ++kk)
        mma_bf16_i(tm + kColGW2, smem_desc(saddr(s->dt) + 256u * kk, 128, 2048),
                   smem_desc(saddr(s->hto) + 256u * kk, 128, 2048), i144, (first && kk == 0) ? 0u : 1u);
    }
    if (!(ok = commit_wait())) break;
    // DA1 = DH o (A1 + b1 > 0), written transposed over H (free since layer 2 ran)
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float a[32];
      tmem_ld32(tm + lb + kColDH + 32 * c, a);
#pragma unroll
      for (int e = 0; e < 32; ++e)
        st_bf16(s->h, core_offset(32 * c + e, t, 16), ((mask1[c] >> e) & 1u) ? a[e] : 0.f);
    }
    tc_fence_before();
    fence_async_smem();
    tc_sync();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (uint32_t kk = 0; kk < gxt::kRows / 16; ++kk)
        mma_bf16_i(tm + kColGW1, smem_desc(saddr(s->h) + 256u * kk, 128, 2048),
                   smem_desc(saddr(s->xto) + 256u * kk, 128, 2048), i32, (first && kk == 0) ? 0u : 1u);
    }
    if (!(ok = commit_wait())) break;
    first = 0;
  }
  if (ok) {
    // thread t: row t of gW2 and gW1 (hidden unit t), gb2[t], gb1[t]
    float* g = partial + (uint64_t)blockIdx.x * NPARAM;
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float a[32];
      tmem_ld32(tm + lb + kColGW2 + 32 * c, a);
#pragma unroll
      for (int e = 0; e < 32; ++e) g[OFF_W2 + t * H + 32 * c + e] = a[e];
    }
    {
      float a[32];
      tmem_ld32(tm + lb + kColGW2 + H, a);  // columns 384-415: gb2 (ones rows), then gW1
      g[OFF_B2 + t] = a[0];
      tmem_ld32(tm + lb + kColGW1, a);      // columns 400-431: gW1, then gb1 (ones rows)
#pragma unroll
      for (int i = 0; i < IN; ++i) g[OFF_W1 + t * IN + i] = a[i];
      g[OFF_B1 + t] = a[IN];
    }
    // gw3 and gb3, loss: the warps' sums in warp order
#pragma unroll
    for (int c = 0; c < 4; ++c) s->red[wid][32 * c + lane] = gw3acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lossacc += __shfl_xor_sync(0xFFFFFFFFu, lossacc, o);
      gb3acc += __shfl_xor_sync(0xFFFFFFFFu, gb3acc, o);
    }
    if (lane == 0) {
      s->redl[wid][0] = lossacc;
      s->redl[wid][1] = gb3acc;
    }
    tc_sync();
    g[OFF_W3 + t] = ((s->red[0][t] + s->red[1][t]) + s->red[2][t]) + s->red[3][t];
    if (t == 0) {
      g[OFF_B3] = ((s->redl[0][1] + s->redl[1][1]) + s->redl[2][1]) + s->redl[3][1];
      partial_loss[blockIdx.x] = ((s->redl[0][0] + s->redl[1][0]) + s->redl[2][0]) + s->redl[3][0];
    }
  } else if (t == 0) {
    atomicOr(&g_train_error, 1u);
  }
  tc_fence_before();
  tc_sync();
  if (t < 32) {
    tc_fence_after();
    tmem_dealloc(tm, kTrainCols);
  }
}

// Self-test of the bounded wait every tensor-core product is awaited with: one
// warp waits on an mbarrier that nothing arrives on, for `limit` polls, and
// records that it gave up.
__device__ unsigned int g_wait_gave_up;

__global__ void wait_selftest_kernel(uint32_t limit) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) gxt::mbar_init(gxt::saddr(&bar), 1);
  __syncthreads();
  const bool done = gxt::mbar_wait_bounded(gxt::saddr(&bar), 0, limit);
  if (threadIdx.x == 0) g_wait_gave_up = done ? 0u : 1u;
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters; clears the gradient.
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            float* __restrict__ g, float lr, float b1t, float b2t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / (1.f - b1t)) / (sqrtf(vi / (1.f - b2t)) + 1e-8f);
  g[i] = 0.f;
}

// Mini-batch indices: batch element j of step s is example mix64(seed + s * B + j) mod n.
__global__ void sample_kernel(uint64_t* __restrict__ idx, uint32_t batch, uint64_t n, uint64_t seed,
                              uint64_t step) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= batch) return;
  uint64_t z = seed + step * batch + j + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  idx[j] = (z ^ (z >> 31)) % n;
}

}  // namespace gxm

namespace {
#define GM_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return gx::fail(GX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

// Kernel attributes belong to the current device, so they are set on every
// call (a few microseconds) rather than once per process.
gx_status set_smem() {
  GM_CUDA(cudaFuncSetAttribute(gxm::mlp_tc_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)gxt::kTcSmemBytes));
  // all of the SM's unified L1/shared memory as shared memory, so that 3 tiles fit per SM
  GM_CUDA(cudaFuncSetAttribute(gxm::mlp_tc_forward_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  GM_CUDA(cudaFuncSetAttribute(gxm::grad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)gxm::kTrainSmemBytes));
  GM_CUDA(cudaFuncSetAttribute(gxm::grad_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  return GX_OK;
}
}  // namespace

extern "C" {

gx_status gx_mlp_init(float* params, uint64_t seed, void* stream) {
  gx::clear_error();
  if (!params) return gx::fail(GX_ERR_INVALID, "params is NULL");
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a splitmix64 stream, biases 0
  std::vector<float> h(gxm::NPARAM, 0.f);
  uint64_t s = seed;
  auto next = [&]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
  };
  auto fill = [&](int off, int count, int fan_in) {
    const double r = 1.0 / std::sqrt((double)fan_in);
    for (int i = 0; i < count; ++i) h[off + i] = (float)((2.0 * next() - 1.0) * r);
  };
  fill(gxm::OFF_W1, gxm::H * gxm::IN, gxm::IN);
  fill(gxm::OFF_W2, gxm::H * gxm::H, gxm::H);
  fill(gxm::OFF_W3, gxm::H, gxm::H);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  GM_CUDA(cudaMemcpyAsync(params, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, st));
  GM_CUDA(cudaStreamSynchronize(st));
  return GX_OK;
}

static std::mutex g_forward_mutex;
static std::mutex g_train_mutex;

// The gradient at params over n examples (slot j takes example index[j] when
// index is given) on the tensor cores: pack the weights, then one CTA per tile
// of 128 examples, at most GX_MLP_GRAD_CTAS CTAs, each writing its partial
// gradient; the caller sums them (reduce_kernel).  Returns the CTA count.
int launch_grad_tc(const float* params, const uint8_t* hist, const float* label, uint64_t n, const uint64_t* index,
                   float* partial, float* partial_loss, gxm::TcTrainWeights* packed, cudaStream_t st) {
  const uint64_t tiles = (n + gxt::kRows - 1) / gxt::kRows;
  const int grid = (int)std::min<uint64_t>(tiles, gxm::kGradCtas);
  gxm::train_pack_kernel<<<gxm::kTrainPackBlocks, 256, 0, st>>>(params, packed);
  gxm::grad_tc_kernel<<<grid, gxt::kRows, gxm::kTrainSmemBytes, st>>>(packed, hist, label, n, index,
                                                                       1.0f / (float)n, partial, partial_loss);
  return grid;
}

gx_status gx_mlp_forward(const float* params, const uint8_t* hist, uint64_t n, float* out, void* stream) {
  gx::clear_error();
  if (!params || (n && (!hist || !out))) return gx::fail(GX_ERR_INVALID, "NULL device pointer");
  if (n == 0) return GX_OK;
  gx_status s = set_smem();
  if (s != GX_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  GM_CUDA(cudaGetDevice(&dev));
  GM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint64_t tiles = (n + gxt::kRows - 1) / gxt::kRows;
  const uint64_t grid = std::min<uint64_t>(tiles, (uint64_t)sms * gxt::tc_ctas_per_sm(dev));
  const unsigned int zero = 0;
  GM_CUDA(cudaMemcpyToSymbolAsync(gxm::g_tc_error, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st));
  std::lock_guard<std::mutex> lock(g_forward_mutex);
  gxt::TcWeights* packed = nullptr;
  GM_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&packed), gxm::g_tc_packed));
  gxt::tc_pack_kernel<<<gxt::kTcPackBlocks, 256, 0, st>>>(params, packed);
  gxm::mlp_tc_forward_kernel<<<(unsigned)grid, gxt::kRows, gxt::kTcSmemBytes, st>>>(packed, hist, n, out);
  GM_CUDA(cudaGetLastError());
  unsigned int err = 0;
  GM_CUDA(cudaMemcpyFromSymbolAsync(&err, gxm::g_tc_error, sizeof(err), 0, cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  if (err) return gx::fail(GX_ERR_SPIN_LIMIT, "tensor-core scoring timed out waiting for an MMA");
  return GX_OK;
}

gx_status gx_wait_selftest(uint32_t spin_limit, void* stream) {
  gx::clear_error();
  if (spin_limit == 0 || spin_limit > gxt::kSpinLimit)
    return gx::fail(GX_ERR_INVALID, "spin_limit must be 1.." + std::to_string(gxt::kSpinLimit));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned int unset = 2u;
  GM_CUDA(cudaMemcpyToSymbolAsync(gxm::g_wait_gave_up, &unset, sizeof(unset), 0, cudaMemcpyHostToDevice, st));
  gxm::wait_selftest_kernel<<<1, 32, 0, st>>>(spin_limit);
  GM_CUDA(cudaGetLastError());
  unsigned int gave_up = 2u;
  GM_CUDA(cudaMemcpyFromSymbolAsync(&gave_up, gxm::g_wait_gave_up, sizeof(gave_up), 0, cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  if (gave_up == 1u)
    return gx::fail(GX_ERR_SPIN_LIMIT, "the wait gave up after " + std::to_string(spin_limit) + " polls");
  if (gave_up != 0u) return gx::fail(GX_ERR_CUDA, "the self-test kernel did not report");
  return GX_OK;
}

gx_status gx_mlp_grad(const float* params, const uint8_t* hist, const float* label, uint64_t n,
                      float* grad, float* loss, void* stream) {
  gx::clear_error();
  if (!params || !grad || !loss || (n && (!hist || !label))) return gx::fail(GX_ERR_INVALID, "NULL device pointer");
  if (n == 0) return GX_OK;
  gx_status s = set_smem();
  if (s != GX_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = (int)std::min<uint64_t>((n + gxt::kRows - 1) / gxt::kRows, gxm::kGradCtas);
  float* scratch = nullptr;  // one partial gradient and loss per CTA
  GM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(float) * (uint64_t)grid * (gxm::NPARAM + 1), st));
  const unsigned int zero = 0;
  GM_CUDA(cudaMemcpyToSymbolAsync(gxm::g_train_error, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st));
  std::lock_guard<std::mutex> lock(g_train_mutex);
  gxm::TcTrainWeights* packed = nullptr;
  GM_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&packed), gxm::g_train_packed));
  launch_grad_tc(params, hist, label, n, nullptr, scratch, scratch + (uint64_t)grid * gxm::NPARAM, packed, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    gxm::reduce_kernel<<<(gxm::NPARAM + 255) / 256, 256, 0, st>>>(scratch, scratch + (uint64_t)grid * gxm::NPARAM,
                                                                  grid, grad, loss);
    e = cudaGetLastError();
  }
  cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, std::string("gradient kernels: ") + cudaGetErrorString(e));
  unsigned int err = 0;
  GM_CUDA(cudaMemcpyFromSymbolAsync(&err, gxm::g_train_error, sizeof(err), 0, cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  if (err) return gx::fail(GX_ERR_SPIN_LIMIT, "tensor-core gradient timed out waiting for an MMA");
  return GX_OK;
}

gx_status gx_mlp_train(float* params, float* state, const uint8_t* hist, const float* label, uint64_t n,
                       uint32_t batch, uint32_t steps, float lr, uint64_t seed, float* loss, void* stream) {
  gx::clear_error();
  if (!params || !state || !hist || !label || !loss) return gx::fail(GX_ERR_INVALID, "NULL device pointer");
  if (n == 0 || batch == 0) return gx::fail(GX_ERR_INVALID, "empty training set or batch");
  gx_status s = set_smem();
  if (s != GX_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // state: m | v | g | partial gradients (GX_MLP_GRAD_CTAS x NPARAM) | partial
  // losses (GX_MLP_GRAD_CTAS) | indices (batch, 8-byte aligned)
  float* m = state;
  float* v = state + gxm::NPARAM;
  float* g = state + 2 * gxm::NPARAM;
  float* partial = state + 3 * gxm::NPARAM;
  float* partial_loss = partial + (uint64_t)gxm::kGradCtas * gxm::NPARAM;
  uint64_t* idx = reinterpret_cast<uint64_t*>(partial_loss + gxm::kGradCtas + 1);
  idx = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(idx) + 7) & ~uintptr_t(7));
  GM_CUDA(cudaMemsetAsync(state, 0, sizeof(float) * 3 * gxm::NPARAM, st));
  GM_CUDA(cudaMemsetAsync(loss, 0, sizeof(float) * steps, st));
  const unsigned int zero = 0;
  GM_CUDA(cudaMemcpyToSymbolAsync(gxm::g_train_error, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st));
  std::lock_guard<std::mutex> lock(g_train_mutex);
  gxm::TcTrainWeights* packed = nullptr;
  GM_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&packed), gxm::g_train_packed));
  double b1t = 1.0, b2t = 1.0;
  for (uint32_t t = 0; t < steps; ++t) {
    b1t *= 0.9;
    b2t *= 0.999;
    gxm::sample_kernel<<<(batch + 255) / 256, 256, 0, st>>>(idx, batch, n, seed, t);
    const int grid = launch_grad_tc(params, hist, label, batch, idx, partial, partial_loss, packed, st);
    gxm::reduce_kernel<<<(gxm::NPARAM + 255) / 256, 256, 0, st>>>(partial, partial_loss, grid, g, loss + t);
    gxm::adam_kernel<<<(gxm::NPARAM + 255) / 256, 256, 0, st>>>(params, m, v, g, lr, (float)b1t, (float)b2t);
  }
  GM_CUDA(cudaGetLastError());
  unsigned int err = 0;
  GM_CUDA(cudaMemcpyFromSymbolAsync(&err, gxm::g_train_error, sizeof(err), 0, cudaMemcpyDeviceToHost, st));
  GM_CUDA(cudaStreamSynchronize(st));
  if (err) return gx::fail(GX_ERR_SPIN_LIMIT, "tensor-core gradient timed out waiting for an MMA");
  return GX_OK;
}

}  // extern "C"

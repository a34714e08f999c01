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
// (gx_mlp_forward, and the guided search's scoring) runs on the tensor cores
// (gx_tc.cuh); the gradient kernel below computes the same network on the
// CUDA cores.
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
constexpr int LD2 = H + 1;  // padded row of W2 in shared memory (no bank conflicts)
constexpr int EPB = 16;     // examples per chunk of the gradient kernel
constexpr int kGradCtas = GX_MLP_GRAD_CTAS;  // at most this many CTAs, one partial gradient each

__device__ __forceinline__ float bf(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

__device__ __forceinline__ float block_sum128(float v, float* red) {
  // blockDim.x == 128
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  const float t = red[0] + red[1] + red[2] + red[3];
  __syncthreads();
  return t;
}

// Forward and backward on the CUDA cores; thread k owns hidden unit k.  CTA
// c takes the chunks of EPB examples c, c + gridDim.x, ... and writes its
// part of the gradient of the mean loss over n examples to partial[c] (and
// its part of the loss to partial_loss[c]); reduce_kernel sums the parts in a
// fixed order, so a gradient does not depend on the order CTAs finish in.
__global__ void __launch_bounds__(H) grad_kernel(const float* __restrict__ p, const uint8_t* __restrict__ hist,
                                                 const float* __restrict__ label, uint64_t n,
                                                 const uint64_t* __restrict__ index, float inv_n,
                                                 float* __restrict__ partial, float* __restrict__ partial_loss) {
  extern __shared__ float sm[];
  float* W2 = sm;                 // [H][LD2]
  float* gW2 = W2 + H * LD2;      // [H][LD2]
  float* h1 = gW2 + H * LD2;      // [H]
  float* dh2 = h1 + H;            // [H]
  float* x = dh2 + H;             // [IN]
  float* red = x + IN;            // [4]
  const int k = threadIdx.x;
  for (int i = k; i < H * H; i += H) {
    W2[(i / H) * LD2 + (i % H)] = bf(p[OFF_W2 + i]);
    gW2[(i / H) * LD2 + (i % H)] = 0.f;
  }
  float w1[IN];
#pragma unroll
  for (int i = 0; i < IN; ++i) w1[i] = bf(p[OFF_W1 + k * IN + i]);
  const float b1 = p[OFF_B1 + k], b2 = p[OFF_B2 + k], w3 = bf(p[OFF_W3 + k]), b3 = p[OFF_B3];
  float gw1[IN];
#pragma unroll
  for (int i = 0; i < IN; ++i) gw1[i] = 0.f;
  float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, lsum = 0.f;
  __syncthreads();
  const uint64_t chunks = (n + EPB - 1) / EPB;
  for (uint64_t chunk = blockIdx.x; chunk < chunks; chunk += gridDim.x)
  for (int e = 0; e < EPB; ++e) {
    const uint64_t slot = chunk * EPB + e;
    if (slot >= n) break;  // uniform in the block
    const uint64_t ex = index ? index[slot] : slot;
    if (k < 32) {  // warp 0: x = bf16(hist * (1 / number of processes))
      const uint32_t h = k < IN ? hist[ex * IN + k] : 0u;
      uint32_t n = h;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
      if (k < IN) x[k] = n ? bf((float)h * (1.0f / (float)n)) : 0.f;
    }
    __syncthreads();
    float a1 = b1;
#pragma unroll
    for (int i = 0; i < IN; ++i) a1 += w1[i] * x[i];
    const float z1 = bf(fmaxf(a1, 0.f));
    h1[k] = z1;
    __syncthreads();
    float a2 = b2;
    for (int j = 0; j < H; ++j) a2 += W2[k * LD2 + j] * h1[j];
    const float z2 = fmaxf(a2, 0.f);
    const float y = block_sum128(w3 * z2, red) + b3;
    const float dy = 2.f * (y - label[ex]) * inv_n;
    if (k == 0) lsum += (y - label[ex]) * (y - label[ex]) * inv_n;
    gb3 += dy;
    gw3 += dy * z2;
    const float d2 = a2 > 0.f ? dy * w3 : 0.f;
    dh2[k] = d2;
    gb2 += d2;
    for (int j = 0; j < H; ++j) gW2[k * LD2 + j] += d2 * h1[j];
    __syncthreads();
    float s = 0.f;
    for (int q = 0; q < H; ++q) s += W2[q * LD2 + k] * dh2[q];
    const float d1 = a1 > 0.f ? s : 0.f;
    gb1 += d1;
#pragma unroll
    for (int i = 0; i < IN; ++i) gw1[i] += d1 * x[i];
    __syncthreads();
  }
  __syncthreads();
  float* g = partial + (uint64_t)blockIdx.x * NPARAM;
  for (int i = k; i < H * H; i += H) g[OFF_W2 + i] = gW2[(i / H) * LD2 + (i % H)];
#pragma unroll
  for (int i = 0; i < IN; ++i) g[OFF_W1 + k * IN + i] = gw1[i];
  g[OFF_B1 + k] = gb1;
  g[OFF_B2 + k] = gb2;
  g[OFF_W3 + k] = gw3;
  if (k == 0) {
    g[OFF_B3] = gb3;
    partial_loss[blockIdx.x] = lsum;
  }
}

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

constexpr size_t kGradSmemBytes = sizeof(float) * (2 * H * LD2 + 2 * H + IN + 4);

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
  GM_CUDA(cudaFuncSetAttribute(gxm::grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)gxm::kGradSmemBytes));
  GM_CUDA(cudaFuncSetAttribute(gxm::mlp_tc_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)gxt::kTcSmemBytes));
  // all of the SM's unified L1/shared memory as shared memory, so that 3 tiles fit per SM
  GM_CUDA(cudaFuncSetAttribute(gxm::mlp_tc_forward_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
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
  const int grid = (int)std::min<uint64_t>((n + gxm::EPB - 1) / gxm::EPB, gxm::kGradCtas);
  float* scratch = nullptr;  // one partial gradient and loss per CTA
  GM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&scratch), sizeof(float) * (uint64_t)grid * (gxm::NPARAM + 1), st));
  gxm::grad_kernel<<<grid, gxm::H, gxm::kGradSmemBytes, st>>>(params, hist, label, n, nullptr, 1.0f / (float)n,
                                                              scratch, scratch + (uint64_t)grid * gxm::NPARAM);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    gxm::reduce_kernel<<<(gxm::NPARAM + 255) / 256, 256, 0, st>>>(scratch, scratch + (uint64_t)grid * gxm::NPARAM,
                                                                  grid, grad, loss);
    e = cudaGetLastError();
  }
  cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, std::string("gradient kernels: ") + cudaGetErrorString(e));
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
  const int grid = (int)std::min<uint64_t>((batch + gxm::EPB - 1) / gxm::EPB, gxm::kGradCtas);
  double b1t = 1.0, b2t = 1.0;
  for (uint32_t t = 0; t < steps; ++t) {
    b1t *= 0.9;
    b2t *= 0.999;
    gxm::sample_kernel<<<(batch + 255) / 256, 256, 0, st>>>(idx, batch, n, seed, t);
    gxm::grad_kernel<<<grid, gxm::H, gxm::kGradSmemBytes, st>>>(params, hist, label, batch, idx,
                                                                1.0f / (float)batch, partial, partial_loss);
    gxm::reduce_kernel<<<(gxm::NPARAM + 255) / 256, 256, 0, st>>>(partial, partial_loss, grid, g, loss + t);
    gxm::adam_kernel<<<(gxm::NPARAM + 255) / 256, 256, 0, st>>>(params, m, v, g, lr, (float)b1t, (float)b2t);
  }
  GM_CUDA(cudaGetLastError());
  GM_CUDA(cudaStreamSynchronize(st));
  return GX_OK;
}

}  // extern "C"

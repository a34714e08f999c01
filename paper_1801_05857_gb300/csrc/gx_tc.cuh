// Tensor-core scoring of the guide network on sm_103a (5th-generation tensor
// cores): both layers of the MLP as tcgen05.mma BF16 x BF16 -> FP32 products
// with the accumulator in tensor memory (TMEM), 128 states per tile.
//
// The scoring threads are warps 0-3 of their CTA (128 threads, which
// synchronise among themselves on a named barrier, so a larger CTA may score
// too); thread t owns row t of a tile (one state), which is also TMEM lane t
// of the M = 128 accumulator, so every epilogue is thread-local:
//
//   X  (128 x 16 BF16)  = bf16(hist / sum(hist))      (fraction of processes per local state)
//   A1 = X W1^T         -> TMEM columns [0, 128)      one MMA, K = 16
//   H  (128 x 128 BF16) = bf16(relu(A1 + b1))          written to shared memory
//   A2 = H W2^T         -> TMEM columns [0, 128)      eight MMAs, K = 16 each
//   y  = b3 + sum_k w3[k] relu(A2[k] + b2[k])          FP32, in registers
//
// Operands live in shared memory in the no-swizzle K-major layout: 8 x 8
// core matrices of 128 contiguous bytes (row r of a core at byte 16 r), core
// (i, j) for row group i and K group j at byte 128 (i * KG + j), KG = K / 8.
// Hence the descriptor's leading-dimension offset (next core along K) is 128
// bytes and its stride-dimension offset (next core along M or N) is 128 KG.
// MMA step kk covers K groups 2kk and 2kk + 1 and starts 256 kk bytes in.
//
// Waits on the MMA-completion barrier are bounded; on a timeout the CTA
// reports it, releases its TMEM and stops.

#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gx.h"

namespace gxt {

constexpr int kRows = 128;             // states per tile = MMA M = TMEM lanes
constexpr int kIn = GX_MLP_IN;         // 16
constexpr int kHid = GX_MLP_HIDDEN;    // 128
constexpr uint32_t kTmemCols = 128;    // one FP32 accumulator, reused by both layers
constexpr uint32_t kSpinLimit = 1u << 22;

static_assert(kIn == 16 && kHid == 128, "tile shapes assume a 16-128-128-1 network");

// Instruction descriptor of tcgen05.mma .kind::f16: FP32 accumulator (bits
// 4-5 = 1), BF16 A and B (bits 7-9 = 1, bits 10-12 = 1), both K-major
// (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t idesc_bf16_f32(uint32_t m, uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_bf16_f32(128, 128);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (bits 16-29), stride byte offset >> 4 (bits 32-45),
// descriptor version 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The scoring threads (warps 0-3 of the CTA, TMEM lanes 0-127) synchronise on
// named barrier 1 among themselves, so a larger CTA whose other warps do
// something else can score tiles too.
constexpr int kTcBarrier = 1;
__device__ __forceinline__ void tc_sync() {
  asm volatile("bar.sync %0, %1;" ::"n"(kTcBarrier), "n"(kRows) : "memory");
}
// OR of pred over the scoring threads, in every one of them.
__device__ __forceinline__ int tc_sync_or(int pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.b32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.b32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "n"(kTcBarrier), "n"(kRows)
      : "memory");
  return r;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_slot), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Poll the barrier's phase at most `limit` times; false when it never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, uint32_t limit = kSpinLimit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// D[tmem] (+)= A * B^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
// The same with an explicit instruction descriptor (other N), issued by one thread.
__device__ __forceinline__ void mma_bf16_i(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on mbar once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32 w .. 32 w + 31); waits for the load before returning.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&b);
}

// 1 / (number of processes) for a histogram packed 4 counts per word; 0 when empty.
__device__ __forceinline__ float feature_scale(const uint32_t (&hw)[4]) {
  uint32_t n = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) n += (hw[i] & 0xFFu) + ((hw[i] >> 8) & 0xFFu) + ((hw[i] >> 16) & 0xFFu) + (hw[i] >> 24);
  return n ? 1.0f / (float)n : 0.f;
}

// Byte offset of element (row, k) in a no-swizzle K-major operand with KG
// K groups of 8 elements.
__host__ __device__ constexpr uint32_t core_offset(uint32_t row, uint32_t k, uint32_t KG) {
  return ((row >> 3) * KG + (k >> 3)) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

// The weights of the guide network as a scoring CTA holds them in shared
// memory: W1 and W2 as BF16 B operands in the core-matrix layout, the FP32
// biases, w3 rounded to BF16 (kept as FP32) and b3.  One copy per search is
// packed in global memory by tc_pack_kernel; every CTA then fetches it with a
// single bulk copy.
struct __align__(16) TcWeights {
  uint8_t w1[kHid * kIn * 2];     // B of layer 1 (W1 as N x K), K groups: 2
  uint8_t w2[kHid * kHid * 2];    // B of layer 2 (W2 as N x K), K groups: 16
  float b1[kHid], b2[kHid], w3[kHid];
  float b3, pad[3];
};
static_assert(sizeof(TcWeights) % 16 == 0, "bulk copies move multiples of 16 bytes");

// Shared memory of the scorer (dynamic, 1024-byte aligned by the caller).
struct __align__(1024) TcSmem {
  uint8_t x[kRows * kIn * 2];     // A of layer 1, K groups: 2
  uint8_t h[kRows * kHid * 2];    // A of layer 2, K groups: 16
  TcWeights wt;                   // starts 1024-byte aligned (36864)
  uint32_t tmem_slot;
  unsigned long long mbar;        // MMA completion
  unsigned long long mbar_load;   // the weights' bulk copy
};
static_assert(sizeof(TcSmem) == 75776, "three scoring CTAs per SM need at most 74 KB each");
constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 1024;  // + alignment slack

// Scoring CTAs per SM, from the device's shared memory (the occupancy query
// reports 1 for these kernels): as many tiles as fit, at most 4 so that their
// TMEM columns (128 each) never exceed the SM's 512.
inline int tc_ctas_per_sm(int dev) {
  int smem_sm = 0, reserved = 0;
  if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
    return 1;
  const int n = smem_sm / (int)(kTcSmemBytes + (size_t)reserved);
  return n < 1 ? 1 : (n > 4 ? 4 : n);
}

__device__ __forceinline__ TcSmem* tc_smem(void* dyn) {
  const uintptr_t p = (reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023);
  return reinterpret_cast<TcSmem*>(p);
}

// Scorer state of one CTA.
struct TcScorer {
  TcSmem* s;
  uint32_t tmem;
  uint32_t phase;
  bool ok;  // the weights arrived
};

// Packing the weights: BF16 (round to nearest even) for W1, W2 and w3, from
// the FP32 parameter layout W1 (128 x 16) | b1 | W2 (128 x 128) | b2 | w3 | b3.
// Thread `item` of a grid of at least kTcPackItems threads writes its part of
// the packed weights: W1 (256 groups of 8), W2 (2048 groups of 8), one row of
// b1, b2 and w3 (128), and b3.
constexpr int kTcPackItems = kHid * 2 + kHid * 16 + kHid + 1;
__device__ __forceinline__ void tc_pack_item(const float* __restrict__ p, TcWeights* __restrict__ out, int item) {
  const float* pW1 = p;
  const float* pb1 = pW1 + kHid * kIn;
  const float* pW2 = pb1 + kHid;
  const float* pb2 = pW2 + kHid * kHid;
  const float* pw3 = pb2 + kHid;
  auto group8 = [](const float* src) {
    uint4 q;
    q.x = pack_bf16x2(src[0], src[1]);
    q.y = pack_bf16x2(src[2], src[3]);
    q.z = pack_bf16x2(src[4], src[5]);
    q.w = pack_bf16x2(src[6], src[7]);
    return q;
  };
  if (item < kHid * 2) {
    const int row = item >> 1, g = item & 1;
    *reinterpret_cast<uint4*>(out->w1 + core_offset(row, g * 8, 2)) = group8(pW1 + row * kIn + g * 8);
  } else if ((item -= kHid * 2) < kHid * 16) {
    const int row = item >> 4, g = item & 15;
    *reinterpret_cast<uint4*>(out->w2 + core_offset(row, g * 8, 16)) = group8(pW2 + row * kHid + g * 8);
  } else if ((item -= kHid * 16) < kHid) {
    out->b1[item] = pb1[item];
    out->b2[item] = pb2[item];
    out->w3[item] = __bfloat162float(__float2bfloat16_rn(pw3[item]));
  } else if (item == kHid) {
    out->b3 = pw3[kHid];
    out->pad[0] = out->pad[1] = out->pad[2] = 0.f;
  }
}

namespace {
// Packs the FP32 parameters p into the scorer's weight image (any grid; one
// item per thread with kTcPackBlocks blocks of 256 threads).
__global__ void tc_pack_kernel(const float* __restrict__ p, TcWeights* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kTcPackItems; i += gridDim.x * blockDim.x)
    tc_pack_item(p, out, i);
}
}  // namespace
constexpr int kTcPackBlocks = (kTcPackItems + 255) / 256;

// Arrive once on mbar and expect `bytes` more from asynchronous copies.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Bulk copy (TMA, no tensor map) of `bytes` from global memory into this
// CTA's shared memory; both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// Set up a scoring CTA: fetch the packed weights with one bulk copy while
// warp 0 allocates the TMEM accumulator.  sc.ok is false (in every thread)
// when the copy did not complete within the bounded wait.
__device__ __forceinline__ TcScorer tc_setup(void* dyn, const TcWeights* __restrict__ packed) {
  TcSmem* s = tc_smem(dyn);
  const int t = threadIdx.x;
  if (t == 0) {
    mbar_init(saddr(&s->mbar), 1);
    mbar_init(saddr(&s->mbar_load), 1);
    mbar_expect_tx(saddr(&s->mbar_load), (uint32_t)sizeof(TcWeights));
    bulk_g2s(saddr(&s->wt), packed, (uint32_t)sizeof(TcWeights), saddr(&s->mbar_load));
  }
  if (t < 32) {
    __syncwarp();  // the allocation is warp-aligned
    tmem_alloc(saddr(&s->tmem_slot), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  tc_sync();
  tc_fence_after();
  bool ok = mbar_wait_bounded(saddr(&s->mbar_load), 0);
  if (!ok) ok = mbar_wait_bounded(saddr(&s->mbar_load), 0);  // the copy must land before the CTA leaves
  const int bad = tc_sync_or(!ok);
  return TcScorer{s, s->tmem_slot, 0u, bad == 0};
}

__device__ __forceinline__ void tc_teardown(const TcScorer& sc) {
  tc_fence_before();
  tc_sync();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(sc.tmem, kTmemCols);
  }
}

// Wait for the last commit; false (in every thread) when any thread gave up.
__device__ __forceinline__ bool tc_wait(TcScorer& sc) {
  const bool ok = mbar_wait_bounded(saddr(&sc.s->mbar), sc.phase);
  sc.phase ^= 1u;
  const int bad = tc_sync_or(!ok);
  tc_fence_after();
  return bad == 0;
}

// Score one tile.  Thread t passes the 16 histogram bytes of its state (4
// per word, entry i = processes in local state i) and gets the score in y.
// Rows of states that do not exist pass zeros.  Returns false after a
// timed-out wait (uniform across the CTA).
__device__ __forceinline__ bool tc_score_tile(TcScorer& sc, const uint32_t (&hw)[4], float& y) {
  TcSmem* s = sc.s;
  const uint32_t t = threadIdx.x;
  const uint32_t lane_base = (t & ~31u) << 16;  // TMEM lane field of this warp
  // X: the fraction of the state's processes in each local state, hist * (1 / sum hist)
  // in FP32, rounded to BF16 (0 for an empty row)
  {
    const float inv = feature_scale(hw);
    uint32_t q[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t w = hw[i >> 1];
      const uint32_t sh = (i & 1) * 16;
      q[i] = pack_bf16x2((float)((w >> sh) & 0xFFu) * inv, (float)((w >> (sh + 8)) & 0xFFu) * inv);
    }
    *reinterpret_cast<uint4*>(s->x + core_offset(t, 0, 2)) = make_uint4(q[0], q[1], q[2], q[3]);
    *reinterpret_cast<uint4*>(s->x + core_offset(t, 8, 2)) = make_uint4(q[4], q[5], q[6], q[7]);
  }
  fence_async_smem();
  tc_sync();
  if (t == 0) {
    tc_fence_after();
    mma_bf16(sc.tmem, smem_desc(saddr(s->x), 128, 256), smem_desc(saddr(s->wt.w1), 128, 256), 0u);
    mma_commit(saddr(&s->mbar));
  }
  if (!tc_wait(sc)) return false;
  // layer-1 epilogue: H row t = bf16(relu(A1 + b1))
#pragma unroll 1
  for (int c0 = 0; c0 < kHid; c0 += 32) {
    float acc[32];
    tmem_ld32(sc.tmem + lane_base + (uint32_t)c0, acc);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t q[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = c0 + g * 8 + 2 * e;
        q[e] = pack_bf16x2(fmaxf(acc[g * 8 + 2 * e] + s->wt.b1[c], 0.f), fmaxf(acc[g * 8 + 2 * e + 1] + s->wt.b1[c + 1], 0.f));
      }
      *reinterpret_cast<uint4*>(s->h + core_offset(t, (uint32_t)(c0 + g * 8), 16)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
  }
  tc_fence_before();
  fence_async_smem();
  tc_sync();
  if (t == 0) {
    tc_fence_after();
    const uint32_t ha = saddr(s->h), wa = saddr(s->wt.w2);
#pragma unroll
    for (uint32_t kk = 0; kk < kHid / 16; ++kk)
      mma_bf16(sc.tmem, smem_desc(ha + 256u * kk, 128, 2048), smem_desc(wa + 256u * kk, 128, 2048), kk > 0 ? 1u : 0u);
    mma_commit(saddr(&s->mbar));
  }
  if (!tc_wait(sc)) return false;
  // layer-2 epilogue: y = b3 + w3 . relu(A2 + b2)
  float acc_y = s->wt.b3;
#pragma unroll 1
  for (int c0 = 0; c0 < kHid; c0 += 32) {
    float acc[32];
    tmem_ld32(sc.tmem + lane_base + (uint32_t)c0, acc);
#pragma unroll
    for (int e = 0; e < 32; ++e) acc_y += s->wt.w3[c0 + e] * fmaxf(acc[e] + s->wt.b2[c0 + e], 0.f);
  }
  y = acc_y;
  // our TMEM reads and the tile's shared-memory use end before the next tile starts
  tc_fence_before();
  tc_sync();
  return true;
}

}  // namespace gxt

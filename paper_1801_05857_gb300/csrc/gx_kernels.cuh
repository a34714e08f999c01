// Templated kernels of the exploration path, instantiated per slot width W in
// gx_kernels_w{1,2,4}.cu.
//
//   expand_kernel  one BFS level (Sec. 3): claim open vectors, count and
//                  generate successors from the staged network tables,
//                  find-or-put each successor (Sec. 4.1), append the new ones
//                  to the next level, count transitions, record deadlocks.
//   init_kernel    inserts the initial vector (level 0).
//   fop_kernel     the isolated hash-table experiment of Sec. 5.1.
#pragma once

#include "gx_device.cuh"
#include "gx_kernels.h"

namespace gxd {

using gx::Ctl;
using gx::NetBlobLayout;

// ---- network tables (a uint32 blob; see gx_net.cpp for its layout)

template <int W>
__device__ __forceinline__ uint32_t local_state(const uint32_t* t, const NetBlobLayout& L,
                                                const uint32_t (&v)[W], uint32_t p) {
  return (word_at<W>(v, t[L.proc_word + p]) >> t[L.proc_shift + p]) & t[L.proc_mask + p];
}

// Offsets [o[0], o[1]) of class c's deltas for local state s.
__device__ __forceinline__ const uint32_t* class_range(const uint32_t* t, const NetBlobLayout& L,
                                                       uint32_t c, uint32_t s) {
  return t + L.coff + t[L.cls_base + c] + s;
}

// Number of successors of v, with multiplicity: every local edge of every
// process, plus for every rule the product of its participants' edge counts.
template <int W>
__device__ __forceinline__ uint32_t count_succ(const uint32_t* t, const NetBlobLayout& L,
                                               const uint32_t (&v)[W]) {
  uint32_t n = 0;
  for (uint32_t p = 0; p < L.n_procs; ++p) {
    const uint32_t* o = class_range(t, L, p, local_state<W>(t, L, v, p));
    n += o[1] - o[0];
  }
  for (uint32_t r = 0; r < L.n_rules; ++r) {
    uint32_t prod = 1;
    const uint32_t j1 = t[L.rule_off + r + 1];
    for (uint32_t j = t[L.rule_off + r]; j < j1 && prod; ++j) {
      const uint32_t c = t[L.rule_cls + j];
      const uint32_t* o = class_range(t, L, c, local_state<W>(t, L, v, t[L.cls_proc + c]));
      prod *= o[1] - o[0];
    }
    n += prod;
  }
  return n;
}

// Resumable enumeration of the successors of one vector: first the local
// edges process by process, then each enabled rule's combinations in
// mixed-radix order.  next() must be called at most count_succ() times.
struct SuccIter {
  uint32_t p, e, e_end, wd;  // local phase
  uint32_t r, cur, k, k_end; // rule phase
  __device__ __forceinline__ void init() { p = e = e_end = wd = r = cur = k = k_end = 0; }
};

template <int W>
__device__ __forceinline__ void next_succ(SuccIter& it, const uint32_t* t, const NetBlobLayout& L,
                                          const uint32_t (&v)[W], uint32_t (&out)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) out[w] = v[w];
  while (it.e == it.e_end && it.p < L.n_procs) {
    const uint32_t p = it.p++;
    const uint32_t* o = class_range(t, L, p, local_state<W>(t, L, v, p));
    it.e = o[0];
    it.e_end = o[1];
    it.wd = t[L.proc_word + p];
  }
  if (it.e < it.e_end) {
    xor_at<W>(out, it.wd, t[L.cdelta + it.e]);
    ++it.e;
    return;
  }
  while (it.k == it.k_end && it.r < L.n_rules) {
    const uint32_t r = it.r++;
    uint32_t prod = 1;
    const uint32_t j1 = t[L.rule_off + r + 1];
    for (uint32_t j = t[L.rule_off + r]; j < j1 && prod; ++j) {
      const uint32_t c = t[L.rule_cls + j];
      const uint32_t* o = class_range(t, L, c, local_state<W>(t, L, v, t[L.cls_proc + c]));
      prod *= o[1] - o[0];
    }
    it.cur = r;
    it.k = 0;
    it.k_end = prod;
  }
  uint32_t x = it.k++;
  const uint32_t j1 = t[L.rule_off + it.cur + 1];
  for (uint32_t j = t[L.rule_off + it.cur]; j < j1; ++j) {
    const uint32_t c = t[L.rule_cls + j];
    const uint32_t p = t[L.cls_proc + c];
    const uint32_t* o = class_range(t, L, c, local_state<W>(t, L, v, p));
    const uint32_t cnt = o[1] - o[0];
    const uint32_t i = x % cnt;
    x /= cnt;
    xor_at<W>(out, t[L.proc_word + p], t[L.cdelta + o[0] + i]);
  }
}

// Order-free digest of one state: h = fold_p mix64(h ^ (p << 32 | s_p)).
template <int W>
__device__ __forceinline__ uint64_t state_digest(const uint32_t* t, const NetBlobLayout& L,
                                                 const uint32_t (&v)[W]) {
  uint64_t h = 0;
  for (uint32_t p = 0; p < L.n_procs; ++p)
    h = mix64(h ^ (((uint64_t)p << 32) | local_state<W>(t, L, v, p)));
  return h;
}

template <int W>
__device__ __forceinline__ void load_vec(const uint32_t* p, uint32_t (&v)[W]) {
  if constexpr (W == 1) {
    v[0] = p[0];
  } else if constexpr (W == 2) {
    uint2 x = *reinterpret_cast<const uint2*>(p);
    v[0] = x.x;
    v[1] = x.y;
  } else {
    uint4 x = *reinterpret_cast<const uint4*>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
}

template <int W>
__device__ __forceinline__ void store_vec(uint32_t* p, const uint32_t (&v)[W]) {
  if constexpr (W == 1) {
    p[0] = v[0];
  } else if constexpr (W == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
  } else {
    *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULLMASK, x, o);
  return x;
}

// Shared-memory prologue shared by the kernels: hash multipliers, then
// (optionally) the network blob.
__device__ __forceinline__ const uint32_t* stage_tables(uint32_t* sm, const gx::Muls& muls,
                                                        int rounds, const uint32_t* blob,
                                                        uint32_t blob_words, int stage,
                                                        const uint64_t*& s_muls) {
  uint64_t* m = reinterpret_cast<uint64_t*>(sm);
  for (int i = threadIdx.x; i < rounds; i += blockDim.x) m[i] = muls.m[i];
  s_muls = m;
  if (!stage) return blob;
  uint32_t* s_tab = sm + 2 * kMaxRounds;
  const uint4* src = reinterpret_cast<const uint4*>(blob);
  uint4* dst = reinterpret_cast<uint4*>(s_tab);
  for (uint32_t i = threadIdx.x; i < blob_words / 4; i += blockDim.x) dst[i] = src[i];
  return s_tab;
}

template <int W, int B, int G>
__global__ void __launch_bounds__(gx::kBlock) expand_kernel(const gx::ExpandArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint64_t* muls;
  const uint32_t* t = stage_tables(sm, a.muls, a.rounds, a.blob, a.blob_words, a.stage, muls);
  __syncthreads();
  const NetBlobLayout& L = a.lay;
  const int lane = threadIdx.x & 31;
  const Group<G> g;
  unsigned long long trans = 0;
  uint32_t probes = 0, err = 0;

  while (true) {
    unsigned long long chunk = 0;
    if (lane == 0) chunk = atomicAdd(&a.ctl->claim, 32ull);
    chunk = __shfl_sync(FULLMASK, chunk, 0);
    const uint64_t start = a.cur_begin + chunk;
    if (start >= a.cur_end) break;
    const uint64_t idx = start + lane;
    const bool valid = idx < a.cur_end;
    uint32_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = 0;
    if (valid) load_vec<W>(a.frontier + (idx & a.fmask) * W, v);
    uint32_t remaining = valid ? count_succ<W>(t, L, v) : 0u;
    trans += remaining;
    if (valid && remaining == 0) {
      const uint64_t h = state_digest<W>(t, L, v);
      const unsigned long long di = atomicAdd(&a.ctl->dl_count, 1ull);
      atomicAdd(&a.ctl->dl_sum, (unsigned long long)h);
      atomicXor(&a.ctl->dl_xor, (unsigned long long)h);
      if (di < a.dl_cap) store_vec<W>(a.dl_buf + di * W, v);
    }
    SuccIter it;
    it.init();
    while (__any_sync(FULLMASK, remaining != 0)) {
      uint32_t s[W];
      const bool has = remaining != 0;
      if (has) {
        next_succ<W>(it, t, L, v, s);
        --remaining;
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) s[w] = 0;
      }
      bool inserted = false;
#pragma unroll 1
      for (int l = 0; l < G; ++l) {
        const int src = g.base + l;
        if (!g.template bcast<int>(has ? 1 : 0, src)) continue;  // uniform in the group
        uint32_t x[W];
#pragma unroll
        for (int w = 0; w < W; ++w) x[w] = g.template bcast<uint32_t>(s[w], src);
        const int r = find_or_put<W, B, G>(a.table, a.log2nb, a.rounds, muls, x, g, probes);
        if (r == FOP_FULL) err |= gx::ERR_TABLE_FULL;
        if (g.glane == l && r == FOP_INSERTED) inserted = true;
      }
      const uint32_t im = __ballot_sync(FULLMASK, inserted);
      if (im) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&a.ctl->next_end, (unsigned long long)__popc(im));
        base = __shfl_sync(FULLMASK, base, 0);
        if (inserted) {
          const uint64_t pos = base + __popc(im & ((1u << lane) - 1u));
          if (pos - a.cur_begin <= a.fmask) store_vec<W>(a.frontier + (pos & a.fmask) * W, s);
          else err |= gx::ERR_FRONTIER;
        }
      }
    }
  }
  trans = warp_sum(trans);
  const unsigned long long pr = warp_sum((unsigned long long)probes);
  err = __reduce_or_sync(FULLMASK, err);
  if (lane == 0) {
    if (trans) atomicAdd(&a.ctl->transitions, trans);
    if (pr) atomicAdd(&a.ctl->probes, pr);
    if (err) atomicOr(&a.ctl->error, err);
  }
}

template <int W, int B, int G>
__global__ void init_kernel(const gx::InitArgs a) {
  __shared__ uint64_t muls[kMaxRounds];
  for (int i = threadIdx.x; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  __syncthreads();
  if ((int)threadIdx.x >= G) return;
  const Group<G> g;
  uint32_t v[W];
#pragma unroll
  for (int w = 0; w < W; ++w) v[w] = a.vec[w];
  uint32_t probes = 0;
  const int r = find_or_put<W, B, G>(a.table, a.log2nb, a.rounds, muls, v, g, probes);
  if (g.glane == 0) {
    if (r == FOP_INSERTED) {
      store_vec<W>(a.frontier, v);
      a.ctl->next_end = 1ull;
    } else {
      a.ctl->error |= gx::ERR_TABLE_FULL;
    }
  }
}

// Sec. 5.1: every group of G lanes takes one key at a time.
template <int W, int B, int G>
__global__ void __launch_bounds__(gx::kBlock) fop_kernel(const gx::FopArgs a) {
  __shared__ uint64_t muls[kMaxRounds];
  for (int i = threadIdx.x; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const Group<G> g;
  const uint64_t groups = (uint64_t)gridDim.x * blockDim.x / G;
  uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  uint32_t probes = 0;
  unsigned long long ins = 0, fnd = 0, fail = 0;
  // the loop bound is uniform per warp: all groups of a warp leave together
  const uint64_t warp_first = ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) / G;
  for (uint64_t wi = warp_first; wi < a.n; wi += groups, i += groups) {
    if (i < a.n) {
      uint32_t v[W];
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = a.keys[i * W + w] | kTag;
      const int r = find_or_put<W, B, G>(a.table, a.log2nb, a.rounds, muls, v, g, probes);
      if (g.glane == 0) {
        if (a.result) a.result[i] = (uint8_t)(r == FOP_INSERTED ? 1 : (r == FOP_FOUND ? 0 : 2));
        ins += r == FOP_INSERTED;
        fnd += r == FOP_FOUND;
        fail += r == FOP_FULL;
      }
    }
  }
  ins = warp_sum(ins);
  fnd = warp_sum(fnd);
  fail = warp_sum(fail);
  if (lane == 0) {
    if (ins) atomicAdd(&a.counters[0], ins);
    if (fnd) atomicAdd(&a.counters[1], fnd);
    if (fail) atomicAdd(&a.counters[2], fail);
  }
}

}  // namespace gxd

namespace gx {

template <int W, int B, int G>
cudaError_t launch_expand(const ExpandArgs& a, int grid, size_t smem, cudaStream_t st) {
  gxd::expand_kernel<W, B, G><<<grid, kBlock, smem, st>>>(a);
  return cudaGetLastError();
}
template <int W, int B, int G>
cudaError_t launch_init(const InitArgs& a, cudaStream_t st) {
  gxd::init_kernel<W, B, G><<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}
template <int W, int B, int G>
cudaError_t launch_fop(const FopArgs& a, int grid, cudaStream_t st) {
  gxd::fop_kernel<W, B, G><<<grid, kBlock, 0, st>>>(a);
  return cudaGetLastError();
}

template <int W, int B, int G>
const KernelSet* kernel_set() {
  static const KernelSet ks{&launch_expand<W, B, G>, &launch_init<W, B, G>, &launch_fop<W, B, G>,
                            reinterpret_cast<const void*>(&gxd::expand_kernel<W, B, G>),
                            reinterpret_cast<const void*>(&gxd::fop_kernel<W, B, G>)};
  return &ks;
}

}  // namespace gx

// Dispatch helper: G must be a power of two dividing B / W.
#define GX_CASE(W, B, G) \
  if (b == B && g == G) return gx::kernel_set<W, B, G>();

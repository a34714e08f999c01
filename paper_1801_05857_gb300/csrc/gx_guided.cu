// Learned guidance for deadlock search (no counterpart in the paper; the
// search it reorders is the exploration of Sec. 3 with on-the-fly deadlock
// detection, and every state still goes through the find-or-put of Sec. 4.1).
//
// Training examples (gx_training_set): after a gx_explore, every state in the
// table gets its distance to the nearest deadlock by level-by-level
// relaxation -- distance 0 for states without successors, distance r for a
// state with a successor at distance r - 1 -- looking successors up in the
// same table.  Then each state becomes one example: the histogram of its
// processes' local states and the capped, normalised distance, and the
// examples are sorted by content so that the set comes out the same way on
// every run.
//
// Guided search (gx_find_deadlocks, GX_DL_GUIDED): open states live in
// priority bins (stacks) by score.  Each iteration:
//   * one CTA pops up to guided_batch states from the best non-empty bin;
//   * a persistent kernel expands them: it logs each (state, parent log
//     index), detects deadlocks, find-or-puts every successor and appends
//     each new one, with its local-state histogram, to a pending buffer;
//   * the scoring kernel runs the MLP on the pending states, 128 per tile, on
//     the tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM;
//     gx_tc.cuh) and pushes each state to the bin of its score.
// Every state is pushed once and popped once, so the search ends either at a
// deadlock or after the whole state space.

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "gx_kernels.cuh"
#include "gx_tc.cuh"

namespace gx {

struct GuidedCtl {
  unsigned long long found;      // smallest log index of a deadlock found, ~0 if none
  unsigned long long batch_n;    // states popped for the current iteration
  unsigned long long log_base;   // log index of the first popped state
  unsigned long long log_count;  // states logged (expanded) so far
  unsigned long long inserted;   // states inserted into the table
  unsigned long long transitions;
  unsigned long long probes;
  unsigned int error, done;
  unsigned long long dl_count;
  unsigned long long pending;    // new states appended by the current iteration's expansion
  unsigned long long iters;      // iterations run
  unsigned long long path_len;   // states on the deadlock's path (gx_guided_trace), 0 if none
};

struct GuidedArgs {
  const uint32_t* blob;
  NetBlobLayout lay;
  uint32_t blob_words;
  int stage;
  Muls muls;
  int rounds, log2nb;
  uint32_t* table;
  GuidedCtl* ctl;
  unsigned long long* bin_count;  // [nbins]
  uint32_t* bins;                 // [nbins][bin_cap] entries of E words
  uint64_t bin_cap;
  int nbins;
  float scale;
  uint32_t* batch;                // [batch_cap] entries
  uint32_t batch_cap;
  uint32_t* log;                  // [log_cap] entries
  uint64_t log_cap;
  const float* params;            // MLP, FP32
  gxt::TcWeights* tcw;            // params packed for the scorer, once per search
  uint4* pend_hist;               // [pend_cap] local-state histograms of new states
  uint32_t* pend;                 // [pend_cap] entries of E words (vector, parent)
  uint64_t pend_cap;
  uint32_t init_vec[4];
  cudaGraphConditionalHandle cond;  // device-driven iteration loop
  unsigned long long max_iters;
};

constexpr unsigned int ERR_BINS = 16u, ERR_LOG = 32u, ERR_WIDE = 64u, ERR_PENDING = 128u;

}  // namespace gx

namespace gxd {

using gx::GuidedArgs;
using gx::GuidedCtl;


// Slot index of v in the table, or -1 when v is not stored.  Slots of a
// bucket fill in order and are never freed, so an empty slot ends the search.
template <int W, int B>
__device__ __forceinline__ int64_t find_slot(const uint32_t* __restrict__ table, int log2nb, int rounds,
                                             const uint64_t* __restrict__ muls, const uint32_t (&v)[W]) {
  constexpr int S = B / W;
  const uint64_t h = vec_hash<W>(v);
  const uint64_t b0 = bucket_of(h, muls[0], log2nb);
  for (int k = 0; k < rounds; ++k) {
    const uint64_t b = k == 0 ? b0 : bucket_in_span<B>(h, muls[k], log2nb, b0);
    uint32_t s[B];
    load_words<B>(table + b * (uint64_t)B, s);
#pragma unroll
    for (int j = 0; j < S; ++j) {
      bool eq = true, empty = true;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        eq &= s[j * W + w] == v[w];
        empty &= s[j * W + w] == 0u;
      }
      if (eq) return (int64_t)(b * S + j);
      if (empty) return -1;
    }
  }
  return -1;
}

template <int W>
__device__ __forceinline__ bool slot_vec(const uint32_t* table, uint64_t i, uint32_t (&v)[W]) {
  load_vec<W>(table + i * W, v);
  bool tagged = true;
#pragma unroll
  for (int w = 0; w < W; ++w) tagged &= (v[w] & kTag) != 0;
  return tagged;
}

// Histogram of local-state indices (each < 16, else *bad is set), 4 per word.
template <int W>
__device__ __forceinline__ void local_hist(const uint32_t* t, const NetBlobLayout& L, const uint32_t (&v)[W],
                                           uint32_t (&hw)[4], uint32_t& bad) {
  hw[0] = hw[1] = hw[2] = hw[3] = 0;
  for (uint32_t p = 0; p < L.n_procs; ++p) {
    const uint32_t s = local_state<W>(t, L, v, p);
    if (s >= 16) {
      bad = 1;
      continue;
    }
    const uint32_t inc = 1u << ((s & 3) * 8);
    if ((s >> 2) == 0) hw[0] += inc;
    else if ((s >> 2) == 1) hw[1] += inc;
    else if ((s >> 2) == 2) hw[2] += inc;
    else hw[3] += inc;
  }
}

constexpr uint32_t INF = 0xFFFFFFFFu;

template <int W>
__global__ void __launch_bounds__(gx::kBlock) label_init_kernel(const uint32_t* table, uint64_t slots, const uint32_t* t,
                                                                NetBlobLayout L, uint32_t* dist) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
    uint32_t v[W];
    if (!slot_vec<W>(table, i, v)) {
      dist[i] = INF;
      continue;
    }
    dist[i] = count_succ<W>(t, L, v) == 0 ? 0u : INF;
  }
}

template <int W, int B>
__global__ void __launch_bounds__(gx::kBlock) label_sweep_kernel(const uint32_t* table, uint64_t slots,
                                                                 const uint32_t* t, NetBlobLayout L, gx::Muls mm,
                                                                 int rounds, int log2nb, uint32_t* dist, uint32_t r,
                                                                 unsigned long long* changed) {
  __shared__ uint64_t muls[kMaxRounds];
  for (int i = threadIdx.x; i < rounds; i += blockDim.x) muls[i] = mm.m[i];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t any = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
    if (dist[i] != INF) continue;
    uint32_t v[W];
    if (!slot_vec<W>(table, i, v)) continue;
    const uint32_t cnt = count_succ<W>(t, L, v);
    SuccIter it;
    it.init();
    for (uint32_t k = 0; k < cnt; ++k) {
      uint32_t s[W];
      next_succ<W>(it, t, L, v, s);
      const int64_t j = find_slot<W, B>(table, log2nb, rounds, muls, s);
      if (j >= 0 && dist[j] == r - 1) {
        dist[i] = r;
        any = 1;
        break;
      }
    }
  }
  if (__any_sync(FULLMASK, any != 0) && (threadIdx.x & 31) == 0) atomicAdd(changed, 1ull);
}

// Content order of the training examples: the gather appends at atomic
// positions, so the examples are sorted by their own content (the 16
// histogram bytes, then the label's bits, compared as unsigned words) to make
// the training set -- and everything trained from it -- the same on every run.
// Equal keys are identical examples, so an unstable sort is enough: a bitonic
// sort over a power-of-two buffer padded with all-ones keys (no histogram byte
// reaches 0xFF).
__device__ __forceinline__ bool ex_greater(const uint4& a, uint32_t la, const uint4& b, uint32_t lb) {
  if (a.x != b.x) return a.x > b.x;
  if (a.y != b.y) return a.y > b.y;
  if (a.z != b.z) return a.z > b.z;
  if (a.w != b.w) return a.w > b.w;
  return la > lb;
}

__global__ void ex_load_kernel(const uint8_t* hist, const float* label, uint64_t n, uint64_t n2, uint4* h,
                               uint32_t* l) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (uint64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      h[i] = reinterpret_cast<const uint4*>(hist)[i];
      l[i] = __float_as_uint(label[i]);
    } else {
      h[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
      l[i] = ~0u;
    }
  }
}

// One compare-exchange pass of the bitonic network: stage k, distance j.
__global__ void ex_bitonic_kernel(uint4* h, uint32_t* l, uint64_t n2, uint64_t k, uint64_t j) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t p = i ^ j;
    if (p <= i) continue;
    const uint4 a = h[i], b = h[p];
    const uint32_t la = l[i], lb = l[p];
    const bool up = (i & k) == 0;
    if (up == ex_greater(a, la, b, lb)) {
      h[i] = b;
      h[p] = a;
      l[i] = lb;
      l[p] = la;
    }
  }
}

__global__ void ex_store_kernel(const uint4* h, const uint32_t* l, uint64_t n, uint8_t* hist, float* label) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    reinterpret_cast<uint4*>(hist)[i] = h[i];
    label[i] = __uint_as_float(l[i]);
  }
}

template <int W>
__global__ void __launch_bounds__(gx::kBlock) label_gather_kernel(const uint32_t* table, uint64_t slots,
                                                                  const uint32_t* t, NetBlobLayout L,
                                                                  const uint32_t* dist, uint32_t max_dist,
                                                                  uint8_t* hist_out, float* label_out, uint64_t cap,
                                                                  unsigned long long* count,
                                                                  unsigned long long* bad_flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
    uint32_t v[W];
    if (!slot_vec<W>(table, i, v)) continue;
    uint32_t hw[4], bad = 0;
    local_hist<W>(t, L, v, hw, bad);
    if (bad) atomicOr(bad_flag, 1ull);
    const unsigned long long pos = atomicAdd(count, 1ull);
    if (pos >= cap) continue;
    uint32_t* dst = reinterpret_cast<uint32_t*>(hist_out + pos * 16);
    dst[0] = hw[0];
    dst[1] = hw[1];
    dst[2] = hw[2];
    dst[3] = hw[3];
    const uint32_t d = dist[i] == INF ? max_dist : min(dist[i], max_dist);
    label_out[pos] = (float)d / (float)max_dist;
  }
}

// ---- guided search

template <int W>
__device__ __forceinline__ void push_bin(const GuidedArgs& a, float score, const uint32_t (&v)[W], uint32_t parent,
                                         uint32_t& err) {
  constexpr int E = W + 1;
  int b0 = (int)(score / a.scale * (float)a.nbins);
  b0 = b0 < 0 ? 0 : (b0 >= a.nbins ? a.nbins - 1 : b0);
  // The calling lanes that share a bin reserve their slots with one atomic
  // (scores cluster, and same-address atomics serialise in L2).
  {
    const uint32_t peers = __match_any_sync(__activemask(), b0);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&a.bin_count[b0], (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const unsigned long long pos = base + __popc(peers & ((1u << lane) - 1u));
    if (pos < a.bin_cap) {
      uint32_t* e = a.bins + ((uint64_t)b0 * a.bin_cap + pos) * E;
#pragma unroll
      for (int w = 0; w < W; ++w) e[w] = v[w];
      e[W] = parent;
      return;
    }
  }
  // a full bin spills into the next one (cyclically): the bins together hold
  // as many entries as the table has slots, so some bin always has room
  for (int i = 1; i < a.nbins; ++i) {
    const int b = (b0 + i) % a.nbins;
    const unsigned long long pos = atomicAdd(&a.bin_count[b], 1ull);
    if (pos < a.bin_cap) {
      uint32_t* e = a.bins + ((uint64_t)b * a.bin_cap + pos) * E;
#pragma unroll
      for (int w = 0; w < W; ++w) e[w] = v[w];
      e[W] = parent;
      return;
    }
  }
  err |= gx::ERR_BINS;
}

// The initial state: into the table and the first bin (as the only open
// state its score does not matter).
template <int W, int B>
__global__ void __launch_bounds__(32) guided_init_kernel(const GuidedArgs a) {
  __shared__ uint64_t muls[kMaxRounds];
  for (int i = threadIdx.x; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  __syncwarp();
  if (threadIdx.x != 0) return;
  uint32_t v[W];
#pragma unroll
  for (int w = 0; w < W; ++w) v[w] = a.init_vec[w];
  uint32_t hw[4], bad = 0;
  local_hist<W>(a.blob, a.lay, v, hw, bad);
  const Group<1> g;
  uint32_t probes = 0, err = bad ? gx::ERR_WIDE : 0u;
  const int r = find_or_put<W, B, 1>(a.table, a.log2nb, a.rounds, muls, v, g, probes);
  if (r != FOP_INSERTED) err |= gx::ERR_TABLE_FULL;
  else {
    a.ctl->inserted = 1;
    push_bin<W>(a, 0.f, v, 0xFFFFFFFFu, err);
  }
  if (err) atomicOr(&a.ctl->error, err);
}

// Pop the next batch from the best non-empty bin (one CTA of up to 1024
// threads, all calling).  The bins are scanned in parallel, one counter per
// thread.  Returns (in every thread) whether a batch was taken; sets done
// when every bin is empty.
template <int W>
__device__ __forceinline__ bool select_batch(const GuidedArgs& a) {
  constexpr int E = W + 1;
  __shared__ int best;
  __shared__ unsigned long long take, top;
  GuidedCtl& c = *a.ctl;
  const bool go = c.found == ~0ull && !c.error;  // uniform: read before anyone writes
  __syncthreads();
  if (threadIdx.x == 0) {
    best = 0x7FFFFFFF;
    c.batch_n = 0;
    c.pending = 0;
  }
  __syncthreads();
  if (!go) return false;
  for (int b = threadIdx.x; b < a.nbins; b += blockDim.x) {
    unsigned long long cnt = a.bin_count[b];
    if (cnt > a.bin_cap) {  // failed pushes left the counter past the end
      cnt = a.bin_cap;
      a.bin_count[b] = cnt;
    }
    if (cnt > 0) atomicMin(&best, b);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (best == 0x7FFFFFFF) {
      c.done = 1;
      best = -1;
    } else {
      const unsigned long long cnt = a.bin_count[best];
      take = cnt < a.batch_cap ? cnt : a.batch_cap;
      top = cnt - take;
      if (c.log_count + take > a.log_cap) {
        c.error |= gx::ERR_LOG;
        best = -1;
      } else {
        a.bin_count[best] = top;
        c.batch_n = take;
        c.log_base = c.log_count;
        c.log_count += take;
      }
    }
  }
  __syncthreads();
  if (best < 0) return false;
  const uint32_t* src = a.bins + ((uint64_t)best * a.bin_cap + top) * E;
  for (uint64_t i = threadIdx.x; i < take * E; i += blockDim.x) a.batch[i] = src[i];
  return true;
}

// One CTA: pop the next batch (the host-driven loop).
template <int W>
__global__ void __launch_bounds__(1024) guided_select_kernel(const GuidedArgs a) {
  select_batch<W>(a);
}

template <int W, int B>
__global__ void __launch_bounds__(gx::kBlock) guided_expand_kernel(const GuidedArgs a) {
  constexpr int E = W + 1;
  constexpr int kWarps = gx::kBlock / 32;
  const unsigned long long n = a.ctl->batch_n;
  if ((unsigned long long)blockIdx.x * kWarps >= n) return;  // no state for this CTA
  extern __shared__ __align__(16) uint32_t gsm[];
  __shared__ uint64_t muls[kMaxRounds];
  __shared__ unsigned long long s_sum[3][kWarps];
  __shared__ uint32_t s_err[kWarps];
  for (int i = threadIdx.x; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  const uint32_t* t = a.blob;
  if (a.stage) {
    uint32_t* s_tab = gsm;
    for (uint32_t i = threadIdx.x; i < a.blob_words; i += blockDim.x) s_tab[i] = a.blob[i];
    t = s_tab;
  }
  __syncthreads();
  const NetBlobLayout& L = a.lay;
  const int lane = threadIdx.x & 31;
  const Group<1> g;
  const unsigned long long log_base = a.ctl->log_base;
  unsigned long long trans = 0, ins = 0;
  uint32_t probes = 0, err = 0;
  // One warp per state: a batch holds a few thousand states, so the time of an
  // iteration is the latency of one state's successors; lane l takes
  // successors l, l + 32, ... and their find-or-puts overlap.  Warp w of the
  // grid takes states w, w + (warps of the grid), ...
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kWarps;
  for (unsigned long long idx = (unsigned long long)blockIdx.x * kWarps + (threadIdx.x >> 5); idx < n;
       idx += nwarps) {
    uint32_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = a.batch[idx * E + w];
    const unsigned long long li = log_base + idx;
    if (lane == 0) {
      uint32_t* le = a.log + li * E;
#pragma unroll
      for (int w = 0; w < W; ++w) le[w] = v[w];
      le[W] = a.batch[idx * E + W];
    }
    const uint32_t total = count_succ<W>(t, L, v);  // the same in every lane
    if (lane == 0) {
      trans += total;
      if (total == 0) {
        atomicMin(&a.ctl->found, li);
        atomicAdd(&a.ctl->dl_count, 1ull);
      }
    }
    for (uint32_t k0 = 0; k0 < total; k0 += 32) {
      const uint32_t k = k0 + lane;
      uint32_t s[W];
      bool inserted = false;
      if (k < total) {
        seek_succ<W>(t, L, v, k, s);
        const int r = find_or_put<W, B, 1>(a.table, a.log2nb, a.rounds, muls, s, g, probes);
        if (r == FOP_FULL) err |= gx::ERR_TABLE_FULL;
        inserted = r == FOP_INSERTED;
      }
      uint32_t hw[4] = {0, 0, 0, 0}, bad = 0;
      if (inserted) local_hist<W>(t, L, s, hw, bad);
      if (bad) err |= gx::ERR_WIDE;
      const uint32_t im = __ballot_sync(FULLMASK, inserted);
      ins += inserted ? 1u : 0u;
      if (im) {  // append the new states to the pending buffer, one atomic per warp
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&a.ctl->pending, (unsigned long long)__popc(im));
        base = __shfl_sync(FULLMASK, base, 0);
        if (inserted) {
          const unsigned long long pos = base + __popc(im & ((1u << lane) - 1u));
          if (pos < a.pend_cap) {
            a.pend_hist[pos] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            uint32_t* e = a.pend + pos * E;
#pragma unroll
            for (int w = 0; w < W; ++w) e[w] = s[w];
            e[W] = (uint32_t)li;
          } else {
            err |= gx::ERR_PENDING;
          }
        }
      }
    }
  }
  // the CTA's totals, one atomic per counter (every warp's at once would queue
  // on the same addresses)
  trans = warp_sum(trans);
  ins = warp_sum(ins);
  const unsigned long long pr = warp_sum((unsigned long long)probes);
  err = __reduce_or_sync(FULLMASK, err);
  const int wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_sum[0][wid] = trans;
    s_sum[1][wid] = ins;
    s_sum[2][wid] = pr;
    s_err[wid] = err;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long x = 0;
    for (int w = 0; w < kWarps; ++w) x += threadIdx.x < 3 ? s_sum[threadIdx.x][w] : (unsigned long long)s_err[w];
    if (x) {
      if (threadIdx.x == 0) atomicAdd(&a.ctl->transitions, x);
      else if (threadIdx.x == 1) atomicAdd(&a.ctl->inserted, x);
      else if (threadIdx.x == 2) atomicAdd(&a.ctl->probes, x);
      else {
        uint32_t e = 0;
        for (int w = 0; w < kWarps; ++w) e |= s_err[w];
        atomicOr(&a.ctl->error, e);
      }
    }
  }
}

// Score the pending states on the tensor cores and push each to its bin.
// 128 threads; persistent over tiles of 128 states.
template <int W>
__global__ void __launch_bounds__(gxt::kRows) guided_score_kernel(const GuidedArgs a) {
  constexpr int E = W + 1;
  extern __shared__ __align__(16) uint8_t tsm[];
  unsigned long long n = a.ctl->pending;
  if (n > a.pend_cap) n = a.pend_cap;  // the expansion reported the overflow
  const unsigned long long tiles = (n + gxt::kRows - 1) / gxt::kRows;
  if (blockIdx.x >= tiles) return;
  gxt::TcScorer sc = gxt::tc_setup(tsm, a.tcw);
  uint32_t err = 0;
  if (!sc.ok) {
    gxt::tc_teardown(sc);
    if (threadIdx.x == 0) atomicOr(&a.ctl->error, gx::ERR_SPIN);
    return;
  }
  for (unsigned long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const unsigned long long row = tile * gxt::kRows + threadIdx.x;
    const bool valid = row < n;
    uint32_t hw[4] = {0, 0, 0, 0};
    if (valid) {
      const uint4 q = a.pend_hist[row];
      hw[0] = q.x;
      hw[1] = q.y;
      hw[2] = q.z;
      hw[3] = q.w;
    }
    float y = 0.f;
    if (!gxt::tc_score_tile(sc, hw, y)) {
      err |= gx::ERR_SPIN;
      break;
    }
    if (valid) {
      uint32_t v[W];
      const uint32_t* e = a.pend + row * E;
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = e[w];
      push_bin<W>(a, y, v, e[W], err);
    }
  }
  gxt::tc_teardown(sc);
  if (err) atomicOr(&a.ctl->error, err);
}

// Expansion and scoring in one kernel (gx_explore_opts.guided_fused): the
// same one-warp-per-state expansion as guided_expand_kernel, but a CTA keeps
// the states its warps insert, with their histograms, in shared memory, and
// its warps 0-3 score them 128 at a time on the tensor cores (gx_tc.cuh,
// synchronising among themselves on a named barrier) and push them to their
// bins -- no pending buffer and no scoring kernel.  The warps of a CTA walk
// their states' successors in lock-step chunks of 32 (a CTA barrier after each
// chunk), so at most 127 + 16 x 32 states wait for a tile.
constexpr int kFusedWarps = 16;
constexpr int kFusedThreads = kFusedWarps * 32;
constexpr int kFusedRows = gxt::kRows - 1 + kFusedThreads;

template <int W>
__host__ __device__ constexpr size_t fused_smem_bytes(size_t blob_bytes) {
  return gxt::kTcSmemBytes + 16ull * kFusedRows + 4ull * (W + 1) * kFusedRows + blob_bytes;
}

template <int W, int B>
__global__ void __launch_bounds__(kFusedThreads, 2) guided_fused_kernel(const GuidedArgs a) {
  constexpr int E = W + 1;
  const unsigned long long n = a.ctl->batch_n;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * kFusedWarps;
  if ((unsigned long long)blockIdx.x * kFusedWarps >= n) return;  // no state for this CTA
  extern __shared__ __align__(16) uint8_t fsm[];
  uint8_t* tc_area = fsm;  // the scorer's 1024-aligned part lies within its first kTcSmemBytes
  uint4* rows_h = reinterpret_cast<uint4*>(fsm + gxt::kTcSmemBytes);
  uint32_t* rows_e = reinterpret_cast<uint32_t*>(rows_h + kFusedRows);
  uint32_t* s_tab = rows_e + E * kFusedRows;
  __shared__ uint64_t muls[kMaxRounds];
  __shared__ unsigned int s_rows, s_steps, s_ok;
  __shared__ unsigned long long s_sum[3][kFusedWarps];
  __shared__ uint32_t s_err[kFusedWarps];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  const uint32_t* t = a.blob;
  if (a.stage) {
    for (uint32_t i = tid; i < a.blob_words; i += blockDim.x) s_tab[i] = a.blob[i];
    t = s_tab;
  }
  uint32_t err = 0;
  gxt::TcScorer sc{};
  if (tid < gxt::kRows) {
    sc = gxt::tc_setup(tc_area, a.tcw);
    if (tid == 0) s_ok = sc.ok ? 1u : 0u;
  }
  if (tid == 0) s_rows = 0;
  __syncthreads();
  if (!s_ok) err |= gx::ERR_SPIN;
  const NetBlobLayout& L = a.lay;
  const Group<1> g;
  const unsigned long long log_base = a.ctl->log_base;
  unsigned long long trans = 0, ins = 0;
  uint32_t probes = 0;

  // Score rows [0, m) (m <= 128) with the scoring threads and push them to their bins.
  auto score_rows = [&](unsigned int m) {
    if (tid < gxt::kRows && s_ok) {
      uint32_t hw[4] = {0, 0, 0, 0};
      const bool valid = (unsigned int)tid < m;
      if (valid) {
        const uint4 q = rows_h[tid];
        hw[0] = q.x;
        hw[1] = q.y;
        hw[2] = q.z;
        hw[3] = q.w;
      }
      float y = 0.f;
      if (!gxt::tc_score_tile(sc, hw, y)) {
        err |= gx::ERR_SPIN;
        if (tid == 0) s_ok = 0;
      } else if (valid) {
        uint32_t v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = rows_e[tid * E + w];
        push_bin<W>(a, y, v, rows_e[tid * E + W], err);
      }
    }
  };

  const unsigned long long first = (unsigned long long)blockIdx.x * kFusedWarps;
  const unsigned long long rounds = (n - first + nwarps - 1) / nwarps;  // the same for the whole CTA
  for (unsigned long long r = 0; r < rounds; ++r) {
    const unsigned long long idx = first + wid + r * nwarps;
    const bool has = idx < n;
    uint32_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = has ? a.batch[idx * E + w] : 0u;
    const unsigned long long li = log_base + idx;
    uint32_t total = 0;
    if (has) {
      if (lane == 0) {
        uint32_t* le = a.log + li * E;
#pragma unroll
        for (int w = 0; w < W; ++w) le[w] = v[w];
        le[W] = a.batch[idx * E + W];
      }
      total = count_succ<W>(t, L, v);
      if (lane == 0) {
        trans += total;
        if (total == 0) {
          atomicMin(&a.ctl->found, li);
          atomicAdd(&a.ctl->dl_count, 1ull);
        }
      }
    }
    if (tid == 0) s_steps = 0;
    __syncthreads();
    if (lane == 0 && total) atomicMax(&s_steps, (total + 31u) / 32u);
    __syncthreads();
    const uint32_t steps = s_steps;
    for (uint32_t c = 0; c < steps; ++c) {
      const uint32_t k = c * 32 + lane;
      uint32_t s[W];
      bool inserted = false;
      if (k < total) {
        seek_succ<W>(t, L, v, k, s);
        const int res = find_or_put<W, B, 1>(a.table, a.log2nb, a.rounds, muls, s, g, probes);
        if (res == FOP_FULL) err |= gx::ERR_TABLE_FULL;
        inserted = res == FOP_INSERTED;
      }
      uint32_t hw[4] = {0, 0, 0, 0}, bad = 0;
      if (inserted) local_hist<W>(t, L, s, hw, bad);
      if (bad) err |= gx::ERR_WIDE;
      const uint32_t im = __ballot_sync(FULLMASK, inserted);
      ins += inserted ? 1u : 0u;
      if (im) {  // rows for the warp's new states, one shared-memory atomic per warp
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(&s_rows, (unsigned int)__popc(im));
        base = __shfl_sync(FULLMASK, base, 0);
        if (inserted) {
          const unsigned int row = base + __popc(im & ((1u << lane) - 1u));
          rows_h[row] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
#pragma unroll
          for (int w = 0; w < W; ++w) rows_e[row * E + w] = s[w];
          rows_e[row * E + W] = (uint32_t)li;
        }
      }
      __syncthreads();
      // full tiles: score rows [0, 128), move the rest to the front
      while (s_rows >= (unsigned int)gxt::kRows) {
        const unsigned int m = s_rows;
        score_rows(gxt::kRows);
        __syncthreads();
        const unsigned int left = m - gxt::kRows;  // < 16 x 32
        uint4 hq = make_uint4(0, 0, 0, 0);
        uint32_t eq[E];
        if ((unsigned int)tid < left) {
          hq = rows_h[gxt::kRows + tid];
#pragma unroll
          for (int w = 0; w < E; ++w) eq[w] = rows_e[(gxt::kRows + tid) * E + w];
        }
        __syncthreads();
        if ((unsigned int)tid < left) {
          rows_h[tid] = hq;
#pragma unroll
          for (int w = 0; w < E; ++w) rows_e[tid * E + w] = eq[w];
        }
        if (tid == 0) s_rows = left;
        __syncthreads();
      }
    }
  }
  if (s_rows > 0) score_rows(s_rows);  // the last, partial tile
  if (tid < gxt::kRows) gxt::tc_teardown(sc);
  // the CTA's totals, one atomic per counter
  trans = warp_sum(trans);
  ins = warp_sum(ins);
  const unsigned long long pr = warp_sum((unsigned long long)probes);
  err = __reduce_or_sync(FULLMASK, err);
  if (lane == 0) {
    s_sum[0][wid] = trans;
    s_sum[1][wid] = ins;
    s_sum[2][wid] = pr;
    s_err[wid] = err;
  }
  __syncthreads();
  if (tid < 4) {
    unsigned long long x = 0;
    for (int w = 0; w < kFusedWarps; ++w) x += tid < 3 ? s_sum[tid][w] : (unsigned long long)s_err[w];
    if (x) {
      if (tid == 0) atomicAdd(&a.ctl->transitions, x);
      else if (tid == 1) atomicAdd(&a.ctl->inserted, x);
      else if (tid == 2) atomicAdd(&a.ctl->probes, x);
      else {
        uint32_t e = 0;
        for (int w = 0; w < kFusedWarps; ++w) e |= s_err[w];
        atomicOr(&a.ctl->error, e);
      }
    }
  }
}

// ---- the device-driven iteration loop and the deadlock's path

// Control block at the start of a search (the rest was cleared).
__global__ void guided_reset_kernel(const GuidedArgs a) { a.ctl->found = ~0ull; }

// Start of the device-driven loop (one CTA of 1024 threads): pop the first
// batch; the loop runs if there is one.
template <int W>
__global__ void __launch_bounds__(1024) guided_loop_start_kernel(const GuidedArgs a) {
  const bool more = select_batch<W>(a);
  if (threadIdx.x == 0) cudaGraphSetConditional(a.cond, more ? 1u : 0u);
}

// After {expand, score}: go on unless a deadlock was found, the open set is
// empty, an error occurred or the iteration bound (every iteration expands at
// least one state, so the log size bounds it) was reached -- and if going on,
// pop the next batch here, so that an iteration takes three kernels.
template <int W>
__global__ void __launch_bounds__(1024) guided_advance_kernel(const GuidedArgs a) {
  GuidedCtl& c = *a.ctl;
  __shared__ int s_more;
  if (threadIdx.x == 0) {
    c.iters += 1;
    s_more = c.found == ~0ull && !c.done && !c.error && c.iters < a.max_iters;
  }
  __syncthreads();
  bool more = s_more != 0;
  if (more) more = select_batch<W>(a);
  if (threadIdx.x == 0) cudaGraphSetConditional(a.cond, more ? 1u : 0u);
}

// One thread: follow the parent log indices from the deadlock back to the
// initial state, writing the path (deadlock first, E words per state) to out;
// c.path_len = its length, or 0 when it does not fit in cap states.
template <int W>
__global__ void guided_path_kernel(const GuidedArgs a, uint32_t* out, uint64_t cap) {
  constexpr int E = W + 1;
  GuidedCtl& c = *a.ctl;
  c.path_len = 0;
  if (c.found == ~0ull) return;
  uint64_t li = c.found, n = 0;
  while (n < cap) {
    const uint32_t* e = a.log + li * E;
#pragma unroll
    for (int w = 0; w < E; ++w) out[n * E + w] = e[w];
    ++n;
    if (e[W] == 0xFFFFFFFFu) {
      c.path_len = n;
      return;
    }
    li = e[W];
  }
}

}  // namespace gxd

namespace gx {
namespace {

#define GG_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return gx::fail(GX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

struct GKernels {
  void (*sweep)(const uint32_t*, uint64_t, const uint32_t*, NetBlobLayout, Muls, int, int, uint32_t*, uint32_t,
                unsigned long long*);
  const void* init;
  const void* select;
  const void* expand;
  const void* score;
  const void* path;
  const void* start;    // pop the first batch and start the device loop
  const void* advance;  // end an iteration and pop the next batch
  const void* fused;    // expansion with the scoring in the same kernel
};

template <int W, int B>
GKernels gk() {
  return GKernels{&gxd::label_sweep_kernel<W, B>, reinterpret_cast<const void*>(&gxd::guided_init_kernel<W, B>),
                  reinterpret_cast<const void*>(&gxd::guided_select_kernel<W>),
                  reinterpret_cast<const void*>(&gxd::guided_expand_kernel<W, B>),
                  reinterpret_cast<const void*>(&gxd::guided_score_kernel<W>),
                  reinterpret_cast<const void*>(&gxd::guided_path_kernel<W>),
                  reinterpret_cast<const void*>(&gxd::guided_loop_start_kernel<W>),
                  reinterpret_cast<const void*>(&gxd::guided_advance_kernel<W>),
                  reinterpret_cast<const void*>(&gxd::guided_fused_kernel<W, B>)};
}

bool gk_lookup(int W, int B, GKernels& k) {
#define GX_GK(w, b) \
  if (W == w && B == b) { k = gk<w, b>(); return true; }
  GX_GK(1, 4) GX_GK(1, 8) GX_GK(1, 16) GX_GK(1, 32)
  GX_GK(2, 4) GX_GK(2, 8) GX_GK(2, 16) GX_GK(2, 32)
  GX_GK(4, 4) GX_GK(4, 8) GX_GK(4, 16) GX_GK(4, 32)
#undef GX_GK
  return false;
}

int log2_of(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

struct GPlan {
  int W, B, rounds, nbins;
  float scale;
  uint32_t batch_cap;
  uint64_t nb, slots, bin_cap, log_cap, pend_cap;
  uint64_t off_ctl, off_blob, off_tcw, off_bincnt, off_table, off_bins, off_batch, off_log, off_pend_hist, off_pend,
      total;
  GKernels k;
};

gx_status guided_plan(const Net& net, const gx_explore_opts* o, GPlan& P) {
  gx_explore_opts d;
  gx_default_opts(&d);
  if (!o) o = &d;
  P.W = (int)net.slot_words;
  P.B = o->bucket_words ? (int)o->bucket_words : 8;
  if (P.B < P.W || !gk_lookup(P.W, P.B, P.k)) return fail(GX_ERR_INVALID, "unsupported bucket_words for guided search");
  P.rounds = o->hash_rounds ? (int)o->hash_rounds : 8;
  if (P.rounds < 1 || P.rounds > kMaxRounds) return fail(GX_ERR_INVALID, "hash_rounds must be 1..64");
  P.nbins = o->guided_bins ? (int)o->guided_bins : 32;
  if (P.nbins < 1 || P.nbins > 1024) return fail(GX_ERR_INVALID, "guided_bins must be 1..1024");
  P.scale = o->guided_scale > 0.f ? o->guided_scale : 1.0f;
  P.batch_cap = o->guided_batch ? o->guided_batch : 8192;
  const uint64_t table_bytes = o->table_bytes ? o->table_bytes : (1ull << 30);
  uint64_t nb = 1;
  while (nb * 2 * 4ull * P.B <= table_bytes) nb *= 2;
  if (nb < 2) return fail(GX_ERR_INVALID, "table_bytes is smaller than two buckets");
  P.nb = nb;
  P.slots = nb * (uint64_t)(P.B / P.W);
  P.log_cap = P.slots;                                   // every state is expanded at most once
  P.bin_cap = std::max<uint64_t>(P.batch_cap, (P.slots + P.nbins - 1) / P.nbins + 1);
  // one iteration inserts at most batch x (successors of a state) states, and
  // never more than the table holds
  P.pend_cap = std::min<uint64_t>(P.slots, (uint64_t)P.batch_cap * std::max<uint64_t>(net.max_succ, 1));
  const uint64_t E = (uint64_t)P.W + 1;
  uint64_t off = 0;
  P.off_ctl = off;
  off = a256(off + sizeof(GuidedCtl));
  P.off_blob = off;
  off = a256(off + 4ull * net.blob.size());
  P.off_tcw = off;
  off = a256(off + sizeof(gxt::TcWeights));
  P.off_bincnt = off;
  off = a256(off + 8ull * P.nbins);
  P.off_table = off;
  off = a256(off + 4ull * P.B * P.nb);
  P.off_bins = off;
  off = a256(off + 4ull * E * P.bin_cap * P.nbins);
  P.off_batch = off;
  off = a256(off + 4ull * E * P.batch_cap);
  P.off_log = off;
  off = a256(off + 4ull * E * P.log_cap);
  P.off_pend_hist = off;
  off = a256(off + 16ull * P.pend_cap);
  P.off_pend = off;
  off = a256(off + 4ull * E * P.pend_cap);
  P.total = off;
  return GX_OK;
}

}  // namespace

void release_guided(gx_net* h) {
  if (h->guided_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(h->guided_exec));
  if (h->guided_graph) cudaGraphDestroy(static_cast<cudaGraph_t>(h->guided_graph));
  h->guided_exec = nullptr;
  h->guided_graph = nullptr;
  h->guided_key.clear();
}

namespace {

// One guided search as a graph: clear the control block, bins and table,
// insert the initial state, pop the first batch, then WHILE(cond) {expand,
// score, advance (which pops the next batch)}.
gx_status build_guided_graph(gx_net* h, const GPlan& P, GuidedArgs a, int grid, size_t smem, int score_grid,
                             bool fused, int fused_grid, size_t fused_smem) {
  release_guided(h);
  h->release_guided = &release_guided;
  cudaGraph_t g;
  GG_CUDA(cudaGraphCreate(&g, 0));
  h->guided_graph = g;
  cudaGraphConditionalHandle cond;
  GG_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  a.cond = cond;
  std::vector<cudaGraphNode_t> clears;
  auto add_memset = [&](void* dst, uint64_t words) -> cudaError_t {
    cudaMemsetParams mp{};
    mp.dst = dst;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = words;
    mp.height = 1;
    cudaGraphNode_t nd;
    cudaError_t e = cudaGraphAddMemsetNode(&nd, g, nullptr, 0, &mp);
    clears.push_back(nd);
    return e;
  };
  GG_CUDA(add_memset(a.ctl, sizeof(GuidedCtl) / 4));
  {  // the scorer's weight image, packed once per search
    const float* pp = a.params;
    gxt::TcWeights* pw = a.tcw;
    void* pargs[] = {&pp, &pw};
    cudaKernelNodeParams kp{};
    kp.func = reinterpret_cast<void*>(&gxt::tc_pack_kernel);
    kp.gridDim = dim3(gxt::kTcPackBlocks);
    kp.blockDim = dim3(256);
    kp.kernelParams = pargs;
    cudaGraphNode_t nd;
    GG_CUDA(cudaGraphAddKernelNode(&nd, g, nullptr, 0, &kp));
    clears.push_back(nd);
  }
  GG_CUDA(add_memset(a.bin_count, 2ull * P.nbins));
  const uint64_t words = (uint64_t)P.B * P.nb;
  constexpr uint64_t kPiece = 1ull << 30;
  for (uint64_t w0 = 0; w0 < words; w0 += kPiece) GG_CUDA(add_memset(a.table + w0, std::min(kPiece, words - w0)));
  auto add_kernel = [&](cudaGraph_t gr, const cudaGraphNode_t* deps, size_t nd, const void* fn, dim3 gd, dim3 bd,
                        size_t sh, cudaGraphNode_t* out) -> cudaError_t {
    void* args[] = {&a};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = gd;
    kp.blockDim = bd;
    kp.sharedMemBytes = (unsigned)sh;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, gr, deps, nd, &kp);
  };
  cudaGraphNode_t reset, init, start, ex, sc, adv, cnode;
  GG_CUDA(add_kernel(g, clears.data(), clears.size(), reinterpret_cast<const void*>(&gxd::guided_reset_kernel),
                     dim3(1), dim3(1), 0, &reset));
  GG_CUDA(add_kernel(g, &reset, 1, P.k.init, dim3(1), dim3(32), 0, &init));
  GG_CUDA(add_kernel(g, &init, 1, P.k.start, dim3(1), dim3(1024), 0, &start));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  GG_CUDA(cudaGraphAddNode(&cnode, g, &start, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (fused) {
    GG_CUDA(add_kernel(body, nullptr, 0, P.k.fused, dim3(fused_grid), dim3(gxd::kFusedThreads), fused_smem, &ex));
    GG_CUDA(add_kernel(body, &ex, 1, P.k.advance, dim3(1), dim3(1024), 0, &adv));
  } else {
    GG_CUDA(add_kernel(body, nullptr, 0, P.k.expand, dim3(grid), dim3(kBlock), smem, &ex));
    GG_CUDA(add_kernel(body, &ex, 1, P.k.score, dim3(score_grid), dim3(gxt::kRows), gxt::kTcSmemBytes, &sc));
    GG_CUDA(add_kernel(body, &sc, 1, P.k.advance, dim3(1), dim3(1024), 0, &adv));
  }
  cudaGraphExec_t exec;
  GG_CUDA(cudaGraphInstantiate(&exec, g, 0));
  h->guided_exec = exec;
  return GX_OK;
}

}  // namespace

gx_status run_guided(gx_net* h, const gx_explore_opts* opts, void* ws, uint64_t ws_bytes, cudaStream_t st) {
  const Net& net = h->net;
  if (!h->guided_params) return fail(GX_ERR_INVALID, "guided mode needs scoring weights (gx_guided_set_weights)");
  for (uint32_t p = 0; p < net.n_procs; ++p)
    if (net.n_states[p] > 16) return fail(GX_ERR_INVALID, "guided mode needs at most 16 local states per process");
  GPlan P;
  gx_status s = guided_plan(net, opts, P);
  if (s != GX_OK) return s;
  if (!ws) return fail(GX_ERR_INVALID, "guided search needs a workspace (gx_guided_workspace_bytes)");
  if (ws_bytes < P.total)
    return fail(GX_ERR_OOM, "workspace holds " + std::to_string(ws_bytes) + " bytes, need " + std::to_string(P.total));
  int dev = 0, sms = 0, optin = 0;
  GG_CUDA(cudaGetDevice(&dev));
  GG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  char* base = static_cast<char*>(ws);
  GuidedCtl* ctl = reinterpret_cast<GuidedCtl*>(base + P.off_ctl);
  GuidedArgs a{};
  a.blob = reinterpret_cast<const uint32_t*>(base + P.off_blob);
  a.lay = net.lay;
  a.blob_words = (uint32_t)net.blob.size();
  hash_multipliers(a.muls.m, kMaxRounds);
  a.rounds = P.rounds;
  a.log2nb = log2_of(P.nb);
  a.table = reinterpret_cast<uint32_t*>(base + P.off_table);
  a.ctl = ctl;
  a.bin_count = reinterpret_cast<unsigned long long*>(base + P.off_bincnt);
  a.bins = reinterpret_cast<uint32_t*>(base + P.off_bins);
  a.bin_cap = P.bin_cap;
  a.nbins = P.nbins;
  a.scale = P.scale;
  a.batch = reinterpret_cast<uint32_t*>(base + P.off_batch);
  a.batch_cap = P.batch_cap;
  a.log = reinterpret_cast<uint32_t*>(base + P.off_log);
  a.log_cap = P.log_cap;
  a.params = h->guided_params;
  a.tcw = reinterpret_cast<gxt::TcWeights*>(base + P.off_tcw);
  a.pend_hist = reinterpret_cast<uint4*>(base + P.off_pend_hist);
  a.pend = reinterpret_cast<uint32_t*>(base + P.off_pend);
  a.pend_cap = P.pend_cap;
  for (int w = 0; w < 4; ++w) a.init_vec[w] = net.init_vec[w];
  const size_t blob_bytes = 4ull * net.blob.size();
  a.stage = (blob_bytes <= (size_t)optin - 32 * 1024) ? 1 : 0;
  const size_t smem = a.stage ? blob_bytes : 0;
  GG_CUDA(cudaFuncSetAttribute(P.k.expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GG_CUDA(cudaFuncSetAttribute(P.k.score, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gxt::kTcSmemBytes));
  GG_CUDA(cudaFuncSetAttribute(P.k.score, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  int per_sm = 0;
  GG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.k.expand, kBlock, smem));
  const int grid = sms * std::max(per_sm, 1);
  const int score_grid = sms * gxt::tc_ctas_per_sm(dev);
  // the fused kernel: its shared memory holds the scorer, the staged rows and the blob
  const bool fused = opts && opts->guided_fused;
  auto fused_bytes = [&](size_t b) {
    return P.W == 1 ? gxd::fused_smem_bytes<1>(b) : P.W == 2 ? gxd::fused_smem_bytes<2>(b) : gxd::fused_smem_bytes<4>(b);
  };
  size_t fused_smem = 0;
  int fused_grid = 0;
  if (fused) {
    a.stage = fused_bytes(blob_bytes) <= (size_t)optin ? 1 : 0;  // else the tables are read from global memory
    fused_smem = fused_bytes(a.stage ? blob_bytes : 0);
    GG_CUDA(cudaFuncSetAttribute(P.k.fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem));
    int fp = 0;
    GG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fp, P.k.fused, gxd::kFusedThreads, fused_smem));
    fp = std::min(std::max(fp, 1), 4);  // TMEM: 128 columns per CTA, 512 per SM
    fused_grid = sms * fp;
  }

  cudaEvent_t e0, e1;
  GG_CUDA(cudaEventCreate(&e0));
  GG_CUDA(cudaEventCreate(&e1));
  GG_CUDA(cudaEventRecord(e0, st));
  GG_CUDA(cudaMemcpyAsync(base + P.off_blob, net.blob.data(), blob_bytes, cudaMemcpyHostToDevice, st));
  a.max_iters = P.log_cap + 2;  // each iteration expands a state or ends the search
  GuidedCtl hc{};
  uint64_t iters = 0;
  const bool device_loop = !(opts && opts->host_loop);
  if (device_loop) {
    // the graph holds the arguments by value: rebuild it when anything changes
    std::vector<unsigned char> key(sizeof(gx_explore_opts) + 4 * sizeof(uint64_t));
    const uint64_t extra[4] = {reinterpret_cast<uint64_t>(ws), P.total, reinterpret_cast<uint64_t>(a.params),
                               (uint64_t)smem};
    if (opts) std::memcpy(key.data(), opts, sizeof(gx_explore_opts));
    std::memcpy(key.data() + sizeof(gx_explore_opts), extra, sizeof(extra));
    if (!h->guided_exec || h->guided_key != key) {
      s = build_guided_graph(h, P, a, grid, smem, score_grid, fused, fused_grid, fused_smem);
      if (s != GX_OK) return s;
      h->guided_key = key;
    }
    GG_CUDA(cudaGraphLaunch(static_cast<cudaGraphExec_t>(h->guided_exec), st));
  } else {
    GuidedCtl init{};
    init.found = ~0ull;
    GG_CUDA(cudaMemcpyAsync(ctl, &init, sizeof(init), cudaMemcpyHostToDevice, st));
    GG_CUDA(cudaMemsetAsync(a.bin_count, 0, 8ull * P.nbins, st));
    GG_CUDA(cudaMemsetAsync(a.table, 0, 4ull * P.B * P.nb, st));
    gxt::tc_pack_kernel<<<gxt::kTcPackBlocks, 256, 0, st>>>(a.params, a.tcw);
    GG_CUDA(cudaGetLastError());
    void* args[] = {&a};
    GG_CUDA(cudaLaunchKernel(P.k.init, dim3(1), dim3(32), args, 0, st));
    while (true) {
      GG_CUDA(cudaLaunchKernel(P.k.select, dim3(1), dim3(1024), args, 0, st));
      if (fused) {
        GG_CUDA(cudaLaunchKernel(P.k.fused, dim3(fused_grid), dim3(gxd::kFusedThreads), args, fused_smem, st));
      } else {
        GG_CUDA(cudaLaunchKernel(P.k.expand, dim3(grid), dim3(kBlock), args, smem, st));
        GG_CUDA(cudaLaunchKernel(P.k.score, dim3(score_grid), dim3(gxt::kRows), args, gxt::kTcSmemBytes, st));
      }
      GG_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
      ++iters;
      if (hc.found != ~0ull || hc.done || hc.error) break;
    }
  }
  // the deadlock's path, walked on the device into the batch buffer (free now)
  {
    uint32_t* out = a.batch;
    uint64_t cap = a.batch_cap;
    void* pargs[] = {&a, &out, &cap};
    GG_CUDA(cudaLaunchKernel(P.k.path, dim3(1), dim3(1), pargs, 0, st));
  }
  GG_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaEventRecord(e1, st));
  GG_CUDA(cudaStreamSynchronize(st));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);

  // the path of the deadlock: follow parent log indices back to the initial state
  h->guided_trace.clear();
  h->deadlocks.clear();
  h->violations.clear();
  const int E = P.W + 1;
  if (device_loop) iters = hc.iters;
  if (hc.found != ~0ull && hc.path_len > 0) {
    // deadlock first in the buffer: reverse while unpacking
    std::vector<uint32_t> raw(hc.path_len * (uint64_t)E);
    GG_CUDA(cudaMemcpy(raw.data(), a.batch, 4ull * raw.size(), cudaMemcpyDeviceToHost));
    std::vector<uint32_t> local(net.n_procs);
    for (uint64_t i = hc.path_len; i-- > 0;) {
      uint32_t w4[4] = {0, 0, 0, 0};
      for (int w = 0; w < P.W; ++w) w4[w] = raw[i * E + w];
      unpack_host(net, w4, local.data());
      h->guided_trace.insert(h->guided_trace.end(), local.begin(), local.end());
    }
    h->deadlocks = local;
  } else if (hc.found != ~0ull) {  // a path longer than the batch buffer: one entry at a time
    std::vector<std::vector<uint32_t>> path;
    uint64_t li = hc.found;
    while (true) {
      uint32_t e[5] = {0, 0, 0, 0, 0};
      GG_CUDA(cudaMemcpy(e, a.log + li * E, 4ull * E, cudaMemcpyDeviceToHost));
      uint32_t w4[4] = {0, 0, 0, 0};
      for (int w = 0; w < P.W; ++w) w4[w] = e[w];
      std::vector<uint32_t> local(net.n_procs);
      unpack_host(net, w4, local.data());
      path.push_back(local);
      if (e[P.W] == 0xFFFFFFFFu || path.size() > P.log_cap) break;
      li = e[P.W];
    }
    std::reverse(path.begin(), path.end());
    for (const auto& st2 : path) h->guided_trace.insert(h->guided_trace.end(), st2.begin(), st2.end());
    h->deadlocks = path.back();
  }
  gx_stats_t& S = h->stats;
  std::memset(&S, 0, sizeof(S));
  S.states = hc.inserted;
  S.explored = hc.log_count;
  S.transitions = hc.transitions;
  S.deadlock_count = hc.found != ~0ull ? 1 : 0;
  S.first_deadlock_level = hc.found != ~0ull ? (int64_t)(h->guided_trace.size() / net.n_procs) - 1 : -1;
  S.table_slots = P.slots;
  S.vector_words = net.vector_words;
  S.slot_words = (uint32_t)P.W;
  S.bucket_words = (uint32_t)P.B;
  S.group_lanes = 1;
  S.hash_rounds = (uint32_t)P.rounds;
  S.complete = hc.done ? 1u : 0u;
  S.fill = (double)hc.inserted / (double)P.slots;
  S.gpu_ms = ms;
  S.expand_launches = iters;
  S.probes = hc.probes;
  h->levels.clear();
  h->have_result = true;
  gx_status rs = GX_OK;
  if (hc.error & ERR_TABLE_FULL) rs = fail(GX_ERR_TABLE_FULL, "hash table full during guided search");
  else if (hc.error & ERR_BINS) rs = fail(GX_ERR_FRONTIER_OVERFLOW, "priority bins full");
  else if (hc.error & ERR_LOG) rs = fail(GX_ERR_OOM, "log of expanded states full");
  else if (hc.error & ERR_WIDE) rs = fail(GX_ERR_INVALID, "a local state index is 16 or more");
  else if (hc.error & ERR_PENDING) rs = fail(GX_ERR_FRONTIER_OVERFLOW, "pending buffer of new states full");
  else if (hc.error & ERR_SPIN) rs = fail(GX_ERR_SPIN_LIMIT, "tensor-core scoring timed out waiting for an MMA");
  S.status = (uint32_t)rs;
  return rs;
}

}  // namespace gx

extern "C" {

gx_status gx_guided_set_weights(gx_net* h, const float* params) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  h->guided_params = params;
  return GX_OK;
}

gx_status gx_guided_workspace_bytes(const gx_net* h, const gx_explore_opts* opts, uint64_t* bytes) {
  gx::clear_error();
  if (!h || !bytes) return gx::fail(GX_ERR_INVALID, "net or bytes is NULL");
  gx::GPlan P;
  gx_status s = gx::guided_plan(h->net, opts, P);
  if (s != GX_OK) return s;
  *bytes = P.total;
  return GX_OK;
}

gx_status gx_guided_trace(const gx_net* h, uint32_t* out, uint32_t cap, uint32_t* len) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  const uint32_t n = h->net.n_procs;
  const uint32_t states = (uint32_t)(h->guided_trace.size() / n);
  if (cap && !out) return gx::fail(GX_ERR_INVALID, "out is NULL");
  const uint32_t k = std::min(states, cap);
  if (k) std::memcpy(out, h->guided_trace.data(), 4ull * n * k);
  if (len) *len = states;
  return GX_OK;
}

gx_status gx_training_set(gx_net* h, void* ws, uint64_t ws_bytes, void* stream, uint32_t* dist,
                          uint32_t max_dist, uint8_t* hist_out, float* label_out, uint64_t cap, uint64_t* n_out) {
  gx::clear_error();
  if (!h || !ws || !dist) return gx::fail(GX_ERR_INVALID, "net, workspace or dist_scratch is NULL");
  if (!h->have_result || h->levels.empty()) return gx::fail(GX_ERR_STATE, "run gx_explore on this network first");
  if (ws_bytes && ws_bytes < h->ws_total) return gx::fail(GX_ERR_INVALID, "workspace smaller than the last search's");
  if (max_dist == 0) return gx::fail(GX_ERR_INVALID, "max_dist must be positive");
  if (cap && (!hist_out || !label_out)) return gx::fail(GX_ERR_INVALID, "output arrays are NULL");
  const gx_stats_t& S = h->stats;
  gx::GKernels k;
  if (!gx::gk_lookup((int)S.slot_words, (int)S.bucket_words, k))
    return gx::fail(GX_ERR_INVALID, "no labelling kernel for this table layout");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  const uint32_t* table = reinterpret_cast<const uint32_t*>(base + h->ws_off_table);
  const uint32_t* blob = reinterpret_cast<const uint32_t*>(base + h->ws_off_blob);
  gx::Ctl* ctl = reinterpret_cast<gx::Ctl*>(base + h->ws_off_ctl);
  unsigned long long* flags = ctl->digest;  // [0] changed, [1] count, [2] bad
  const uint64_t slots = S.table_slots;
  const int W = (int)S.slot_words;
  gx::Muls mm;
  gx::hash_multipliers(mm.m, gx::kMaxRounds);
  const int log2nb = gx::log2_of(slots * W / S.bucket_words);
  int dev = 0, sms = 0;
  GG_CUDA(cudaGetDevice(&dev));
  GG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * 8;
  if (W == 1) gxd::label_init_kernel<1><<<grid, gx::kBlock, 0, st>>>(table, slots, blob, h->net.lay, dist);
  else if (W == 2) gxd::label_init_kernel<2><<<grid, gx::kBlock, 0, st>>>(table, slots, blob, h->net.lay, dist);
  else gxd::label_init_kernel<4><<<grid, gx::kBlock, 0, st>>>(table, slots, blob, h->net.lay, dist);
  GG_CUDA(cudaGetLastError());
  for (uint32_t r = 1; r <= max_dist; ++r) {
    GG_CUDA(cudaMemsetAsync(flags, 0, 8, st));
    k.sweep<<<grid, gx::kBlock, 0, st>>>(table, slots, blob, h->net.lay, mm, (int)S.hash_rounds, log2nb, dist, r,
                                         flags);
    GG_CUDA(cudaGetLastError());
    unsigned long long changed = 0;
    GG_CUDA(cudaMemcpyAsync(&changed, flags, 8, cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    if (!changed) break;
  }
  GG_CUDA(cudaMemsetAsync(flags + 1, 0, 16, st));
  if (W == 1)
    gxd::label_gather_kernel<1><<<grid, gx::kBlock, 0, st>>>(table, slots, blob, h->net.lay, dist, max_dist, hist_out,
                                                              label_out, cap, flags + 1, flags + 2);
  else if (W == 2)
    gxd::label_gather_kernel<2><<<grid, gx::kBlock, 0, st>>>(table, slots, blob, h->net.lay, dist, max_dist, hist_out,
                                                              label_out, cap, flags + 1, flags + 2);
  else
    gxd::label_gather_kernel<4><<<grid, gx::kBlock, 0, st>>>(table, slots, blob, h->net.lay, dist, max_dist, hist_out,
                                                              label_out, cap, flags + 1, flags + 2);
  GG_CUDA(cudaGetLastError());
  unsigned long long res[2] = {0, 0};
  GG_CUDA(cudaMemcpyAsync(res, flags + 1, 16, cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  if (n_out) *n_out = res[0];
  if (res[1]) return gx::fail(GX_ERR_INVALID, "a process has a local state index of 16 or more");
  // content order (see ex_bitonic_kernel)
  const uint64_t m = std::min<uint64_t>(res[0], cap);
  if (m > 1) {
    uint64_t n2 = 1;
    while (n2 < m) n2 <<= 1;
    uint4* sh = nullptr;
    uint32_t* sl = nullptr;
    GG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&sh), 16 * n2, st));
    GG_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&sl), 4 * n2, st));
    const int sgrid = sms * 8;
    gxd::ex_load_kernel<<<sgrid, 256, 0, st>>>(hist_out, label_out, m, n2, sh, sl);
    for (uint64_t k2 = 2; k2 <= n2; k2 <<= 1)
      for (uint64_t j = k2 >> 1; j > 0; j >>= 1) gxd::ex_bitonic_kernel<<<sgrid, 256, 0, st>>>(sh, sl, n2, k2, j);
    gxd::ex_store_kernel<<<sgrid, 256, 0, st>>>(sh, sl, m, hist_out, label_out);
    const cudaError_t le = cudaGetLastError();
    GG_CUDA(cudaFreeAsync(sh, st));
    GG_CUDA(cudaFreeAsync(sl, st));
    GG_CUDA(le);
    GG_CUDA(cudaStreamSynchronize(st));
  }
  return GX_OK;
}

}  // extern "C"

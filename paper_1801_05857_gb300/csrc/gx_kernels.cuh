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
// The two phases share the iterator's four words (it keeps register use low
// in the level kernel): idx counts processes 0..n_procs-1 and then rules
// (n_procs + r); [e, e_end) is the current process's delta range, or the
// current rule's combination counter and count; wd is the current process's
// word, or the current rule.
struct SuccIter {
  uint32_t idx, e, e_end, wd;
  __device__ __forceinline__ void init() { idx = e = e_end = wd = 0; }
};

template <int W>
__device__ __forceinline__ void next_succ(SuccIter& it, const uint32_t* t, const NetBlobLayout& L,
                                          const uint32_t (&v)[W], uint32_t (&out)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) out[w] = v[w];
  if (it.idx <= L.n_procs) {  // local phase (or its end)
    while (it.e == it.e_end && it.idx < L.n_procs) {
      const uint32_t p = it.idx++;
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
  }
  while (it.e == it.e_end && it.idx < L.n_procs + L.n_rules) {
    const uint32_t r = it.idx++ - L.n_procs;
    uint32_t prod = 1;
    const uint32_t j1 = t[L.rule_off + r + 1];
    for (uint32_t j = t[L.rule_off + r]; j < j1 && prod; ++j) {
      const uint32_t c = t[L.rule_cls + j];
      const uint32_t* o = class_range(t, L, c, local_state<W>(t, L, v, t[L.cls_proc + c]));
      prod *= o[1] - o[0];
    }
    it.wd = r;
    it.e = 0;
    it.e_end = prod;
  }
  uint32_t x = it.e++;
  const uint32_t j1 = t[L.rule_off + it.wd + 1];
  for (uint32_t j = t[L.rule_off + it.wd]; j < j1; ++j) {
    const uint32_t c = t[L.rule_cls + j];
    const uint32_t p = t[L.cls_proc + c];
    const uint32_t* o = class_range(t, L, c, local_state<W>(t, L, v, p));
    const uint32_t cnt = o[1] - o[0];
    uint32_t i = 0;
    if (cnt > 1) {  // one matching edge is the common case: no division
      i = x % cnt;
      x /= cnt;
    }
    xor_at<W>(out, t[L.proc_word + p], t[L.cdelta + o[0] + i]);
  }
}

// Successor k (k < count_succ) of v, in next_succ's order, without walking
// the ones before it: O(processes + rules) table reads.  Lets the lanes of a
// warp take different successors of one state at once.
template <int W>
__device__ __forceinline__ void seek_succ(const uint32_t* t, const NetBlobLayout& L, const uint32_t (&v)[W],
                                          uint32_t k, uint32_t (&out)[W]) {
#pragma unroll
  for (int w = 0; w < W; ++w) out[w] = v[w];
  for (uint32_t p = 0; p < L.n_procs; ++p) {
    const uint32_t* o = class_range(t, L, p, local_state<W>(t, L, v, p));
    const uint32_t c = o[1] - o[0];
    if (k < c) {
      xor_at<W>(out, t[L.proc_word + p], t[L.cdelta + o[0] + k]);
      return;
    }
    k -= c;
  }
  for (uint32_t r = 0; r < L.n_rules; ++r) {
    const uint32_t j0 = t[L.rule_off + r], j1 = t[L.rule_off + r + 1];
    uint32_t prod = 1;
    for (uint32_t j = j0; j < j1 && prod; ++j) {
      const uint32_t c = t[L.rule_cls + j];
      const uint32_t* o = class_range(t, L, c, local_state<W>(t, L, v, t[L.cls_proc + c]));
      prod *= o[1] - o[0];
    }
    if (k < prod) {
      uint32_t x = k;
      for (uint32_t j = j0; j < j1; ++j) {
        const uint32_t c = t[L.rule_cls + j];
        const uint32_t p = t[L.cls_proc + c];
        const uint32_t* o = class_range(t, L, c, local_state<W>(t, L, v, p));
        const uint32_t cnt = o[1] - o[0];
        uint32_t i = 0;
        if (cnt > 1) {
          i = x % cnt;
          x /= cnt;
        }
        xor_at<W>(out, t[L.proc_word + p], t[L.cdelta + o[0] + i]);
      }
      return;
    }
    k -= prod;
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

// Safety check (Sec. 3: the negated property is one more automaton of the
// network): v violates when its watched field holds the automaton's error
// state.  A violation is counted, folded into the violation digest and kept
// while there is room.
template <int W>
__device__ __forceinline__ void check_watch(const gx::ExpandArgs& a, const uint32_t* t, const NetBlobLayout& L,
                                            const uint32_t (&v)[W]) {
  uint32_t w = v[0];
#pragma unroll
  for (int i = 1; i < W; ++i)
    if (a.watch_word == (uint32_t)i) w = v[i];
  if (((w >> a.watch_shift) & a.watch_mask) != a.watch_value) return;
  const uint64_t h = state_digest<W>(t, L, v);
  const unsigned long long vi = atomicAdd(&a.ctl->viol_count, 1ull);
  atomicAdd(&a.ctl->viol_sum, (unsigned long long)h);
  atomicXor(&a.ctl->viol_xor, (unsigned long long)h);
  if (vi < a.viol_cap) store_vec<W>(a.viol_buf + vi * W, v);
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

// Offsets in a 64-bit key of the payload of words 1..3 (ExpandArgs.gkey_shift).
struct GKey {
  uint32_t s[3];
};

// Where find-or-put inserts and where new vectors go: one network's table and
// frontier ring (the level being expanded starts at begin()).  Target holds
// the values (the batched kernel loads them per network); ParamTarget reads
// them from the single-network kernel's parameters, which live in the
// constant bank and so take no registers in the inner loop.
struct Target {
  uint32_t* tab;
  int l2nb, nrounds;
  unsigned long long* nend;
  uint32_t* front;
  uint64_t fm;
  uint64_t cur_begin;
  __device__ __forceinline__ uint32_t* table() const { return tab; }
  __device__ __forceinline__ int log2nb() const { return l2nb; }
  __device__ __forceinline__ int rounds() const { return nrounds; }
  __device__ __forceinline__ unsigned long long* next_end() const { return nend; }
  __device__ __forceinline__ uint32_t* frontier() const { return front; }
  __device__ __forceinline__ uint64_t fmask() const { return fm; }
  __device__ __forceinline__ uint64_t begin() const { return cur_begin; }
  __device__ __forceinline__ uint64_t region_mask() const { return 0; }
  __device__ __forceinline__ uint64_t region_bits() const { return 0; }
  __device__ __forceinline__ unsigned long long* gcache() const { return nullptr; }
  __device__ __forceinline__ uint64_t gcache_mask() const { return 0; }
  __device__ __forceinline__ GKey gkey() const { return GKey{{64u, 64u, 64u}}; }
};

struct ParamTarget {
  const gx::ExpandArgs& a;
  const unsigned long long* range;  // [begin, end) of the level, in shared memory
  __device__ __forceinline__ uint32_t* table() const { return a.table; }
  __device__ __forceinline__ int log2nb() const { return a.log2nb; }
  __device__ __forceinline__ int rounds() const { return a.rounds; }
  __device__ __forceinline__ unsigned long long* next_end() const { return &a.ctl->next_end; }
  __device__ __forceinline__ uint32_t* frontier() const { return a.frontier; }
  __device__ __forceinline__ uint64_t fmask() const { return a.fmask; }
  __device__ __forceinline__ uint64_t begin() const { return range[0]; }
  __device__ __forceinline__ uint64_t region_mask() const { return a.region_mask; }
  __device__ __forceinline__ uint64_t region_bits() const { return a.region_bits; }
  __device__ __forceinline__ unsigned long long* gcache() const { return a.gcache; }
  __device__ __forceinline__ uint64_t gcache_mask() const { return a.gcache_mask; }
  __device__ __forceinline__ GKey gkey() const { return GKey{{a.gkey_shift[0], a.gkey_shift[1], a.gkey_shift[2]}}; }
};

// Per-warp staging of new vectors in shared memory: lanes that inserted a
// vector append it here (ballot + popc, no atomic); every 32 staged vectors
// are written to the next level with one global atomicAdd and one coalesced
// store.  flush() writes what is left.  All 32 lanes call push/flush together.
constexpr int kStage = 64;  // vectors per warp (at most 31 + 32 are ever staged)

struct WarpStage {
  uint32_t* buf;  // kStage * W words of this warp
  int n;          // staged vectors (uniform in the warp)

  template <int W, class T>
  __device__ __forceinline__ void write_out(const T& a, int m, uint32_t& err) {
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.next_end(), (unsigned long long)m);
    base = __shfl_sync(FULLMASK, base, 0);
    if (lane < m) {
      const uint64_t pos = base + lane;
      uint32_t v[W];
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = buf[lane * W + w];
      if (pos - a.begin() <= a.fmask()) store_vec<W>(a.frontier() + (pos & a.fmask()) * W, v);
      else err |= gx::ERR_FRONTIER;
    }
  }

  template <int W, class T>
  __device__ __forceinline__ void push(const T& a, bool ins, const uint32_t (&v)[W],
                                       uint32_t& err) {
    const int lane = threadIdx.x & 31;
    const uint32_t im = __ballot_sync(FULLMASK, ins);
    if (ins) {
      const int at = n + __popc(im & ((1u << lane) - 1u));
#pragma unroll
      for (int w = 0; w < W; ++w) buf[at * W + w] = v[w];
    }
    n += __popc(im);
    if (n >= 32) {
      __syncwarp();
      write_out<W>(a, 32, err);
      __syncwarp();
      // move the remainder (fewer than 32) to the front
      if (lane < n - 32) {
#pragma unroll
        for (int w = 0; w < W; ++w) buf[lane * W + w] = buf[(32 + lane) * W + w];
      }
      n -= 32;
      __syncwarp();
    }
  }

  template <int W, class T>
  __device__ __forceinline__ void flush(const T& a, uint32_t& err) {
    __syncwarp();
    if (n > 0) write_out<W>(a, n, err);
    n = 0;
    __syncwarp();
  }
};

// Per-warp cache of recently seen vectors (the block-local state cache of
// Fig. 2, in shared memory, per warp): direct-mapped, overwritten on a miss,
// never cleared.  Every vector written into it is passed to find-or-put by the
// lane that wrote it, so a hit means the vector is in the table or being put
// there by this warp, and its find-or-put can be skipped.  Only for 1- and
// 2-word vectors, whose entries are read and written by single aligned
// shared-memory accesses (a torn entry could otherwise fake a hit).
struct WarpCache {
  uint32_t* base;  // 2^log2 entries of W words, or nullptr
  uint32_t mask;
  template <int W>
  __device__ __forceinline__ bool seen(uint64_t h, const uint32_t (&v)[W]) const {
    if constexpr (W == 1) {
      uint32_t* e = base + ((uint32_t)h & mask);
      if (*e == v[0]) return true;
      *e = v[0];
      return false;
    } else if constexpr (W == 2) {
      unsigned long long* e = reinterpret_cast<unsigned long long*>(base) + ((uint32_t)h & mask);
      const unsigned long long x = (unsigned long long)v[0] | ((unsigned long long)v[1] << 32);
      if (*e == x) return true;
      *e = x;
      return false;
    } else {
      static_assert(W == 4, "slot width");
      uint4* e = reinterpret_cast<uint4*>(base) + ((uint32_t)h & mask);
      const uint4 c = *e;
      if (c.x == v[0] && c.y == v[1] && c.z == v[2] && c.w == v[3]) return true;
      *e = make_uint4(v[0], v[1], v[2], v[3]);
      return false;
    }
  }
};

// GPU-wide cache of recently seen vectors: direct-mapped, 2^k 64-bit entries in
// global memory (a few MB, so it stays in L2), cleared at the start of a search.
// A vector is written into it after its find-or-put found or inserted it, so
// every entry is a vector of the table and a hit can skip the table probe.
// Only 1- and 2-word vectors: an aligned 64-bit load or store is one access, so
// an entry is never seen half-written.  Successors of a level mostly lead into
// the levels just before and after it, which were inserted or looked up
// moments earlier by some warp of the GPU.
template <int W>
__device__ __forceinline__ unsigned long long gcache_key(const uint32_t (&v)[W], const GKey& k) {
  if constexpr (W == 1) {
    return (unsigned long long)v[0];
  } else if constexpr (W == 2) {
    return (unsigned long long)v[0] | ((unsigned long long)v[1] << 32);
  } else {
    // the payload bits of the words side by side (fields sit at the low bits of
    // each word, so the words' payloads do not overlap): one key per vector
    unsigned long long key = v[0] & ~kTag;
#pragma unroll
    for (int w = 1; w < W; ++w)
      if (k.s[w - 1] < 64) key |= (unsigned long long)(v[w] & ~kTag) << k.s[w - 1];
    return key;
  }
}
// Keys of 1- and 2-word vectors carry the tag bits and are never 0 (an empty
// entry); the one 4-word vector whose key is 0 is never cached.
template <int W>
__device__ __forceinline__ bool gcache_hit(const unsigned long long* c, uint64_t mask, uint64_t h,
                                           const uint32_t (&v)[W], const GKey& k) {
  const unsigned long long key = gcache_key<W>(v, k);
  return (W <= 2 || key != 0ull) && __ldcg(c + ((h >> 32) & mask)) == key;
}
template <int W>
__device__ __forceinline__ void gcache_put(unsigned long long* c, uint64_t mask, uint64_t h, const uint32_t (&v)[W],
                                           const GKey& k) {
  const unsigned long long key = gcache_key<W>(v, k);
  if (W <= 2 || key != 0ull) __stcg(c + ((h >> 32) & mask), key);
}

// Successors each lane generates per round.  insert_lanes takes K per lane
// (the group issues the first-bucket loads of up to four items before it
// resolves any of them); measured on the mid network, K = 2 or 4 costs more in
// registers and occupancy than it gains in loads in flight, so K = 1.
template <int G>
struct PerLane {
  static constexpr int K = 1;
};

// Find-or-put of the K vectors each lane holds (has[k]: lane holds vector k),
// G lanes per bucket.  Phase 1 issues the first-bucket loads of all G*K items
// of the group; phase 2 resolves them in order (found in the first bucket, or
// the full find-or-put with the CAS and further rounds).  Vectors this call
// inserted go to the warp's staging buffer.
// Must be called by all 32 lanes of the warp together.
template <int W, int B, int G, int K, class T>
__device__ __forceinline__ void insert_lanes(const T& a, const uint64_t* muls,
                                             const Group<G>& g, const bool (&has)[K],
                                             const uint32_t (&s)[K][W], uint32_t& probes,
                                             uint32_t& err, WarpStage& st,
                                             const WarpCache& cache = WarpCache{nullptr, 0}) {
  constexpr int LW = (B / W / G) * W;
  constexpr int NI = G * K;            // items of the group this round
  constexpr int CH = NI < 4 ? NI : 4;  // items in flight at a time
  bool inserted[K];
#pragma unroll
  for (int k = 0; k < K; ++k) inserted[k] = false;
#pragma unroll 1
  for (int c = 0; c < NI; c += CH) {
    uint32_t x[CH][W];
    uint32_t pre[CH][LW];
    bool hv[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int i = c + j;
      const int src = g.base + i / K;
      hv[j] = g.template bcast<int>(has[i % K] ? 1 : 0, src) != 0;  // uniform in the group
#pragma unroll
      for (int w = 0; w < W; ++w) x[j][w] = g.template bcast<uint32_t>(s[i % K][w], src);
      if (hv[j]) {
        const uint64_t hh = vec_hash<W>(x[j]);
        const uint64_t b = bucket_of(hh, muls[0], a.log2nb());
        // region passes: a vector whose first bucket lies outside this pass's region is
        // left to the pass of that region (tested before the cache, which may only hold
        // vectors that went to find-or-put)
        if ((b & a.region_mask()) != a.region_bits()) {
          hv[j] = false;
        } else if (cache.base || a.gcache()) {
          // A vector this warp has already sent to find-or-put needs no second lookup,
          // nor does one that any warp found or inserted moments ago.  One lane of the
          // group reads (and writes) the caches and the group takes its answer: other
          // warps write the GPU-wide cache at any moment, and lanes of a group are not
          // guaranteed to read it in one instruction, so their own reads could disagree
          // and split the group before find-or-put's group-wide votes.
          int known = 0;
          if (g.glane == 0)
            known = (cache.base && cache.template seen<W>(hh, x[j])) ||
                    (a.gcache() && gcache_hit<W>(a.gcache(), a.gcache_mask(), hh, x[j], a.gkey()));
          if (g.template bcast<int>(known, g.base)) hv[j] = false;
        }
        if (hv[j]) {
          load_words<LW>(a.table() + b * (uint64_t)B + (uint64_t)g.glane * LW, pre[j]);
          probes += g.glane == 0;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      if (!hv[j]) continue;
      const int i = c + j;
      const int r = find_or_put_from<W, B, G, true>(a.table(), a.log2nb(), a.rounds(), muls, x[j], g, probes,
                                                    pre[j]);
      if (r == FOP_FULL) err |= gx::ERR_TABLE_FULL;
      else if (a.gcache() && g.glane == 0)
        gcache_put<W>(a.gcache(), a.gcache_mask(), vec_hash<W>(x[j]), x[j], a.gkey());
      if (g.glane == i / K && r == FOP_INSERTED) inserted[i % K] = true;
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) st.push<W>(a, inserted[k], s[k], err);
}

// One lane per bucket (G = 1): find-or-put of the vector x of every lane with
// has set (the filters of insert_lanes already passed), its new vectors staged
// for the next level.  All 32 lanes call it together.
template <int W, int B, class T>
__device__ __forceinline__ void resolve_lanes(const T& a, const uint64_t* muls, bool has, const uint32_t (&x)[W],
                                              const uint64_t hh, uint32_t& probes, uint32_t& err, WarpStage& st) {
  constexpr int LW = (B / W) * W;
  const Group<1> g;
  bool inserted = false;
  uint32_t pre[LW];
  if (has) {
    const uint64_t b = bucket_of(hh, muls[0], a.log2nb());
    load_words<LW>(a.table() + b * (uint64_t)B, pre);
    ++probes;
    const int r = find_or_put_hashed<W, B, 1, true>(a.table(), a.log2nb(), a.rounds(), muls, x, hh, g, probes, pre);
    if (r == FOP_FULL) err |= gx::ERR_TABLE_FULL;
    else if (a.gcache()) gcache_put<W>(a.gcache(), a.gcache_mask(), hh, x, a.gkey());
    inserted = r == FOP_INSERTED;
  }
  st.push<W>(a, inserted, x, err);
}

// Per-warp queue of successors waiting for their find-or-put (G = 1).  The lanes
// of a warp expand different states, whose successor counts differ: one
// successor per lane and round leaves the lanes of the states with fewer
// successors idle in the rounds that follow.  So each round only generates one
// successor per lane and queues the ones the filters keep (region, per-warp
// cache, GPU-wide cache); whenever 32 are queued, every lane resolves one, so
// the bucket reads and compare-and-swaps run with all 32 lanes busy.
constexpr int kQueue = 64;  // at most 31 left + 32 new

template <int W>
struct WarpQueue {
  uint32_t* buf;             // kQueue * W words of this warp
  unsigned long long* hash;  // kQueue hashes (vec_hash) of the queued vectors
  int n;                     // queued vectors (uniform in the warp)
};

// Resident CTAs per SM the level kernel is compiled for (register budget).
// A lane holds min(G, 4) first buckets in flight of B / G words each; up to
// 8 such words fit 48 registers (5 CTAs), up to 16 fit 64 (4 CTAs), more get
// 85 (3 CTAs); 4-word slots with 4 or more lanes per bucket also get 3.
// (Checked with -Xptxas -v: at most a few bytes spill; the queued kernel for
// 4-word slots in 8-word buckets spills 48 bytes and is still the fastest
// there: 3.50 s on the memory-scaled network against 3.76 s at 4 CTAs and 64
// registers.  4-word slots in 16-word buckets spill 48 bytes at 48 registers
// and ran slower.)  The level kernel is latency-bound, so the extra CTA pays: 4-word
// slots in 8-word buckets explore the memory-scaled network in 4.49 s at 5
// CTAs, 4.94 s at 4 (plain kernel).
template <int W, int B, int G>
struct ExpandOcc {
  static constexpr int inflight = (G < 4 ? G : 4) * (B / G);
  static constexpr int min_ctas =
      (inflight <= 8 && (W <= 2 || G == 1)) ? 5 : ((inflight <= 16 && !(W == 4 && G >= 4)) ? 4 : 3);
};

// Q: the per-warp successor queue.  Generation rounds append the successors that
// pass the filters (region, caches) to a queue in shared memory, and find-or-put
// runs 32 queued successors at a time with every lane busy.  Built by default
// for 1- and 2-word vectors with one lane per bucket; for 4-word vectors in 4-
// and 8-word buckets it is a second kernel, chosen when region passes discard
// most successors (memory-scaled network, 2 passes: 3.52 s queued against 4.48 s;
// the 1.08e8-state irregular network in 4 GiB, 1 pass: 57.8 ms queued against
// 49.4 ms).
template <int W, int B, int G, bool Q = (G == 1 && W <= 2)>
__global__ void __launch_bounds__(gx::kBlock, ExpandOcc<W, B, G>::min_ctas) expand_kernel(const gx::ExpandArgs a) {
  static_assert(!Q || G == 1, "the successor queue needs one lane per bucket");
  extern __shared__ __align__(16) uint32_t sm[];
  // the level being expanded: from the parameters, or (device-driven level
  // loop) from the control block the previous level's advance step wrote.
  // Kept in shared memory, not registers, for the inner loop's sake.
  __shared__ unsigned long long s_range[2];
  if (a.dev_range) {
    const uint64_t b0 = a.ctl->cur_begin, e0 = a.ctl->cur_end;
    // a fixed full-size grid: CTAs beyond the level's first chunks leave at once
    const uint64_t per_cta = 32ull * (gx::kBlock / 32);
    if ((uint64_t)blockIdx.x * per_cta >= e0 - b0) return;
    if (threadIdx.x == 0) {
      s_range[0] = b0;
      s_range[1] = e0;
    }
  } else if (threadIdx.x == 0) {
    s_range[0] = a.cur_begin;
    s_range[1] = a.cur_end;
  }
  const uint64_t* muls;
  const uint32_t* t = stage_tables(sm, a.muls, a.rounds, a.blob, a.blob_words, a.stage, muls);
  __syncthreads();
  const NetBlobLayout& L = a.lay;
  const int lane = threadIdx.x & 31;
  const Group<G> g;
  uint32_t trans = 0;  // per thread and launch: far below 2^32
  uint32_t probes = 0, err = 0;
  __shared__ uint32_t stage_mem[gx::kBlock / 32][kStage * W];
  WarpStage st{stage_mem[threadIdx.x >> 5], 0};
  constexpr bool kQueued = Q;
  __shared__ uint32_t queue_mem[kQueued ? gx::kBlock / 32 : 1][kQueued ? kQueue * W : 1];
  __shared__ unsigned long long queue_hash[kQueued ? gx::kBlock / 32 : 1][kQueued ? kQueue : 1];
  WarpQueue<W> wq{queue_mem[kQueued ? threadIdx.x >> 5 : 0], queue_hash[kQueued ? threadIdx.x >> 5 : 0], 0};
  const ParamTarget tg{a, s_range};
  WarpCache cache{nullptr, 0};
  if (a.cache_log2 > 0) {
    uint32_t* cbase = sm + 2 * kMaxRounds + (a.stage ? a.blob_words : 0);  // 16-byte aligned
    const uint32_t per_warp = (1u << a.cache_log2) * W;
    cache.base = cbase + (threadIdx.x >> 5) * per_warp;
    cache.mask = (1u << a.cache_log2) - 1u;
    for (uint32_t i = lane; i < per_warp; i += 32) cache.base[i] = 0u;  // 0 is never a stored vector
    __syncwarp();
  }

  while (true) {
    unsigned long long chunk = 0;
    if (lane == 0) chunk = atomicAdd(&a.ctl->claim, 32ull);
    chunk = __shfl_sync(FULLMASK, chunk, 0);
    const uint64_t start = s_range[0] + chunk;
    if (start >= s_range[1]) break;
    const uint64_t idx = start + lane;
    const bool valid = idx < s_range[1];
    uint32_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = 0;
    if (valid) load_vec<W>(a.frontier + (idx & a.fmask) * W, v);
    uint32_t remaining = valid ? count_succ<W>(t, L, v) : 0u;
    // with region passes, the level's states are accounted for in the first pass only
    const bool acct = valid && a.count_states;
    if (acct) trans += remaining;
    if (acct && remaining == 0) {
      const uint64_t h = state_digest<W>(t, L, v);
      const unsigned long long di = atomicAdd(&a.ctl->dl_count, 1ull);
      atomicAdd(&a.ctl->dl_sum, (unsigned long long)h);
      atomicXor(&a.ctl->dl_xor, (unsigned long long)h);
      if (di < a.dl_cap) store_vec<W>(a.dl_buf + di * W, v);
    }
    if (a.watch && acct) check_watch<W>(a, t, L, v);
    SuccIter it;
    it.init();
    if constexpr (kQueued) {
      while (__any_sync(FULLMASK, remaining != 0)) {
        uint32_t x[W];
        uint64_t hh = 0;
        bool keep = remaining != 0;
        if (keep) {
          next_succ<W>(it, t, L, v, x);
          --remaining;
          hh = vec_hash<W>(x);
          const uint64_t b = bucket_of(hh, muls[0], a.log2nb);
          // the filters of insert_lanes: region, per-warp cache, GPU-wide cache
          if ((b & a.region_mask) != a.region_bits) keep = false;
          else if (cache.base && cache.template seen<W>(hh, x)) keep = false;
          else if (a.gcache && gcache_hit<W>(a.gcache, a.gcache_mask, hh, x, tg.gkey())) keep = false;
        }
        const uint32_t km = __ballot_sync(FULLMASK, keep);
        if (keep) {
          const int at = wq.n + __popc(km & ((1u << lane) - 1u));
#pragma unroll
          for (int w = 0; w < W; ++w) wq.buf[at * W + w] = x[w];
          wq.hash[at] = hh;
        }
        wq.n += __popc(km);
        if (wq.n >= 32) {
          __syncwarp();
          uint32_t y[W];
#pragma unroll
          for (int w = 0; w < W; ++w) y[w] = wq.buf[lane * W + w];
          resolve_lanes<W, B>(tg, muls, true, y, wq.hash[lane], probes, err, st);
          __syncwarp();
          if (lane < wq.n - 32) {
#pragma unroll
            for (int w = 0; w < W; ++w) wq.buf[lane * W + w] = wq.buf[(32 + lane) * W + w];
            wq.hash[lane] = wq.hash[32 + lane];
          }
          wq.n -= 32;
          __syncwarp();
        }
      }
    } else {
      constexpr int K = PerLane<G>::K;
      while (__any_sync(FULLMASK, remaining != 0)) {
        uint32_t s[K][W];
        bool has[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          has[k] = remaining != 0;
          if (has[k]) {
            next_succ<W>(it, t, L, v, s[k]);
            --remaining;
          } else {
#pragma unroll
            for (int w = 0; w < W; ++w) s[k][w] = 0;
          }
        }
        insert_lanes<W, B, G, K>(tg, muls, g, has, s, probes, err, st, cache);
      }
    }
  }
  if constexpr (kQueued) {  // what is left in the queue
    __syncwarp();
    const bool has = lane < wq.n;
    uint32_t y[W];
#pragma unroll
    for (int w = 0; w < W; ++w) y[w] = has ? wq.buf[lane * W + w] : 0u;
    resolve_lanes<W, B>(tg, muls, has, y, has ? wq.hash[lane] : 0ull, probes, err, st);
    wq.n = 0;
  }
  st.flush<W>(tg, err);
  // the CTA's totals, one atomic per counter: at the end of a level every warp
  // finishes at once, and per-warp atomics would queue on two addresses
  __shared__ unsigned long long s_tot[2][gx::kBlock / 32];
  __shared__ uint32_t s_err[gx::kBlock / 32];
  const unsigned long long trans_w = warp_sum((unsigned long long)trans);
  const unsigned long long pr = warp_sum((unsigned long long)probes);
  err = __reduce_or_sync(FULLMASK, err);
  if (lane == 0) {
    s_tot[0][threadIdx.x >> 5] = trans_w;
    s_tot[1][threadIdx.x >> 5] = pr;
    s_err[threadIdx.x >> 5] = err;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    unsigned long long x = 0;
    if (threadIdx.x < 2)
      for (int w = 0; w < gx::kBlock / 32; ++w) x += s_tot[threadIdx.x][w];
    if (threadIdx.x == 0 && x) atomicAdd(&a.ctl->transitions, x);
    if (threadIdx.x == 1 && x) atomicAdd(&a.ctl->probes, x);
    if (threadIdx.x == 2) {
      uint32_t e = 0;
      for (int w = 0; w < gx::kBlock / 32; ++w) e |= s_err[w];
      if (e) atomicOr(&a.ctl->error, e);
    }
  }
}


// ---- partitioned expansion (see PartArgs)

// Exclusive scan of one value per thread over the block (blockDim.x == kBlock).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t& total, uint32_t* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULLMASK, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) scratch[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < (gx::kBlock / 32) ? scratch[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULLMASK, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < (gx::kBlock / 32)) scratch[lane] = wi - w;  // exclusive warp offsets
    if (lane == (gx::kBlock / 32) - 1) scratch[gx::kBlock / 32] = wi;
  }
  __syncthreads();
  const uint32_t r = scratch[wid] + inc - x;
  total = scratch[gx::kBlock / 32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void part_range(const gx::ExpandArgs& a, const gx::PartArgs& pa, int b,
                                           uint64_t& lo, uint64_t& hi) {
  lo = a.cur_begin + (uint64_t)b * pa.range;
  hi = lo + pa.range;
  if (hi > a.cur_end) hi = a.cur_end;
  if (lo > hi) lo = hi;
}

// Pass 1: successors per (CTA, slice).  No other side effect, so a level may still
// fall back to the direct kernel after it.
template <int W>
__global__ void __launch_bounds__(gx::kBlock) part_count_kernel(const gx::ExpandArgs a, const gx::PartArgs pa) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint64_t* muls;
  const uint32_t* t = stage_tables(sm, a.muls, 1, a.blob, a.blob_words, a.stage, muls);
  uint32_t* hist = sm + 2 * kMaxRounds + (a.stage ? a.blob_words : 0);
  __shared__ uint32_t scan_scratch[gx::kBlock / 32 + 1];
  const int P = 1 << pa.logp;
  for (int q = threadIdx.x; q < P; q += blockDim.x) hist[q] = 0;
  __syncthreads();
  const NetBlobLayout& L = a.lay;
  const uint64_t mul0 = muls[0];
  const int shift = 64 - pa.logp;
  uint64_t lo, hi;
  part_range(a, pa, blockIdx.x, lo, hi);
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    uint32_t v[W];
    load_vec<W>(a.frontier + (i & a.fmask) * W, v);
    const uint32_t cnt = count_succ<W>(t, L, v);
    SuccIter it;
    it.init();
    for (uint32_t k = 0; k < cnt; ++k) {
      uint32_t s[W];
      next_succ<W>(it, t, L, v, s);
      atomicAdd(&hist[(uint32_t)((vec_hash<W>(s) * mul0) >> shift)], 1u);
    }
  }
  __syncthreads();
  uint32_t mine = 0;
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    pa.hist[(uint64_t)blockIdx.x * P + q] = hist[q];
    mine += hist[q];
  }
  uint32_t total;
  block_exclusive_scan(mine, total, scan_scratch);
  if (threadIdx.x == 0) pa.tot[blockIdx.x] = total;
}

// Pass 2: per slice q (one CTA each), exclusive scan over the batch's CTAs.
// (A template only so that every translation unit may include this header.)
template <int Unused>
__global__ void __launch_bounds__(gx::kBlock) part_scan_kernel(const gx::PartArgs pa) {
  __shared__ uint32_t scan_scratch[gx::kBlock / 32 + 1];
  const int q = blockIdx.x;
  const int P = 1 << pa.logp;
  uint32_t running = 0;
  for (int base = pa.b0; base < pa.b1; base += blockDim.x) {
    const int b = base + threadIdx.x;
    const uint32_t x = b < pa.b1 ? pa.hist[(uint64_t)b * P + q] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(x, total, scan_scratch);
    if (b < pa.b1) pa.off[(uint64_t)b * P + q] = running + ex;
    running += total;
  }
  if (threadIdx.x == 0) pa.ptot[q] = running;
}

// Pass 3: regenerate the successors and write them slice-major; transitions and
// deadlocks of the batch's frontier states are accounted here.
template <int W>
__global__ void __launch_bounds__(gx::kBlock) part_scatter_kernel(const gx::ExpandArgs a, const gx::PartArgs pa) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint64_t* muls;
  const uint32_t* t = stage_tables(sm, a.muls, 1, a.blob, a.blob_words, a.stage, muls);
  uint32_t* cur = sm + 2 * kMaxRounds + (a.stage ? a.blob_words : 0);
  __shared__ uint32_t scan_scratch[gx::kBlock / 32 + 1];
  const int P = 1 << pa.logp;
  const int b = pa.b0 + blockIdx.x;
  // cursor of slice q = (successors of the batch in slices < q) + (of CTAs before b in slice q)
  uint32_t running = 0;
  __syncthreads();
  for (int base = 0; base < P; base += blockDim.x) {
    const int q = base + threadIdx.x;
    const uint32_t x = q < P ? pa.ptot[q] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(x, total, scan_scratch);
    if (q < P) cur[q] = running + ex + pa.off[(uint64_t)b * P + q];
    running += total;
  }
  __syncthreads();
  const NetBlobLayout& L = a.lay;
  const uint64_t mul0 = muls[0];
  const int shift = 64 - pa.logp;
  uint64_t lo, hi;
  part_range(a, pa, b, lo, hi);
  unsigned long long trans = 0;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    uint32_t v[W];
    load_vec<W>(a.frontier + (i & a.fmask) * W, v);
    const uint32_t cnt = count_succ<W>(t, L, v);
    trans += cnt;
    if (cnt == 0) {
      const uint64_t h = state_digest<W>(t, L, v);
      const unsigned long long di = atomicAdd(&a.ctl->dl_count, 1ull);
      atomicAdd(&a.ctl->dl_sum, (unsigned long long)h);
      atomicXor(&a.ctl->dl_xor, (unsigned long long)h);
      if (di < a.dl_cap) store_vec<W>(a.dl_buf + di * W, v);
    }
    if (a.watch) check_watch<W>(a, t, L, v);
    SuccIter it;
    it.init();
    for (uint32_t k = 0; k < cnt; ++k) {
      uint32_t s[W];
      next_succ<W>(it, t, L, v, s);
      const uint32_t q = (uint32_t)((vec_hash<W>(s) * mul0) >> shift);
      const uint32_t pos = atomicAdd(&cur[q], 1u);
      store_vec<W>(pa.succ + (uint64_t)pos * W, s);
    }
  }
  trans = warp_sum(trans);
  if ((threadIdx.x & 31) == 0 && trans) atomicAdd(&a.ctl->transitions, trans);
}

// Pass 4: find-or-put of the buffered successors in buffer order (slice by slice).
template <int W, int B, int G>
__global__ void __launch_bounds__(gx::kBlock) part_probe_kernel(const gx::ExpandArgs a, const uint32_t* succ,
                                                                uint64_t n) {
  __shared__ uint64_t muls[kMaxRounds];
  for (int i = threadIdx.x; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const Group<G> g;
  uint32_t probes = 0, err = 0;
  __shared__ uint32_t stage_mem[gx::kBlock / 32][kStage * W];
  WarpStage st{stage_mem[threadIdx.x >> 5], 0};
  __shared__ unsigned long long s_range[2];
  if (threadIdx.x == 0) {
    s_range[0] = a.cur_begin;
    s_range[1] = a.cur_end;
  }
  __syncthreads();
  const ParamTarget tg{a, s_range};
  while (true) {
    unsigned long long chunk = 0;
    if (lane == 0) chunk = atomicAdd(&a.ctl->claim, 32ull);
    chunk = __shfl_sync(FULLMASK, chunk, 0);
    if (chunk >= n) break;
    const uint64_t idx = chunk + lane;
    bool has[1] = {idx < n};
    uint32_t s[1][W];
#pragma unroll
    for (int w = 0; w < W; ++w) s[0][w] = 0;
    if (has[0]) load_vec<W>(succ + idx * W, s[0]);
    insert_lanes<W, B, G, 1>(tg, muls, g, has, s, probes, err, st);
  }
  st.flush<W>(tg, err);
  const unsigned long long pr = warp_sum((unsigned long long)probes);
  err = __reduce_or_sync(FULLMASK, err);
  if (lane == 0) {
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

template <int W, int B, int G, bool Q = (G == 1 && W <= 2)>
cudaError_t launch_expand(const ExpandArgs& a, int grid, size_t smem, cudaStream_t st) {
  gxd::expand_kernel<W, B, G, Q><<<grid, kBlock, smem, st>>>(a);
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

template <int W>
cudaError_t launch_part_count(const ExpandArgs& a, const PartArgs& p, size_t smem, cudaStream_t st) {
  gxd::part_count_kernel<W><<<p.nb, kBlock, smem, st>>>(a, p);
  return cudaGetLastError();
}
inline cudaError_t launch_part_scan(const PartArgs& p, cudaStream_t st) {
  gxd::part_scan_kernel<0><<<1 << p.logp, kBlock, 0, st>>>(p);
  return cudaGetLastError();
}
template <int W>
cudaError_t launch_part_scatter(const ExpandArgs& a, const PartArgs& p, size_t smem, cudaStream_t st) {
  gxd::part_scatter_kernel<W><<<p.b1 - p.b0, kBlock, smem, st>>>(a, p);
  return cudaGetLastError();
}
template <int W, int B, int G>
cudaError_t launch_part_probe(const ExpandArgs& a, const uint32_t* succ, uint64_t n, int grid, cudaStream_t st) {
  gxd::part_probe_kernel<W, B, G><<<grid, kBlock, 0, st>>>(a, succ, n);
  return cudaGetLastError();
}

// The queued level kernel as a second choice: 4-word vectors, one lane per bucket
// of at most 8 words (with larger buckets it measured slower than the plain one).
template <int W, int B, int G>
constexpr bool kSecondQueued = W == 4 && G == 1 && B <= 8;

using ExpandLauncher = cudaError_t (*)(const ExpandArgs&, int, size_t, cudaStream_t);
template <int W, int B, int G>
ExpandLauncher queued_launcher() {
  if constexpr (kSecondQueued<W, B, G>) return &launch_expand<W, B, G, true>;
  else return nullptr;
}
template <int W, int B, int G>
const void* queued_fn() {
  if constexpr (kSecondQueued<W, B, G>) return reinterpret_cast<const void*>(&gxd::expand_kernel<W, B, G, true>);
  else return nullptr;
}

template <int W, int B, int G>
const KernelSet* kernel_set() {
  static const KernelSet ks{&launch_expand<W, B, G>,
                            &launch_part_count<W>,
                            &launch_part_scan,
                            &launch_part_scatter<W>,
                            &launch_part_probe<W, B, G>,
                            &launch_init<W, B, G>,
                            &launch_fop<W, B, G>,
                            reinterpret_cast<const void*>(&gxd::expand_kernel<W, B, G>),
                            reinterpret_cast<const void*>(&gxd::fop_kernel<W, B, G>),
                            reinterpret_cast<const void*>(&gxd::part_count_kernel<W>),
                            reinterpret_cast<const void*>(&gxd::part_scatter_kernel<W>),
                            reinterpret_cast<const void*>(&gxd::part_probe_kernel<W, B, G>),
                            reinterpret_cast<const void*>(&gxd::init_kernel<W, B, G>),
                            queued_launcher<W, B, G>(),
                            queued_fn<W, B, G>()};
  return &ks;
}

}  // namespace gx

// Dispatch helper: G must be a power of two dividing B / W.
#define GX_CASE(W, B, G) \
  if (b == B && g == G) return gx::kernel_set<W, B, G>();

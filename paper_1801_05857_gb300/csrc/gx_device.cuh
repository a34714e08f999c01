// Device primitives of the exploration path: vector hashing, tagged slots,
// compare-and-swap of a whole slot, and the group-cooperative find-or-put of
// Sec. 4.1 (Figs. 3-4) with the configurable bucket size of Sec. 4.2 (Fig. 5).
//
// Table layout.  The table is an array of 2^log2nb buckets of B uint32 words.
// A bucket holds S = B / W slots of W words (W = vector words, 3 padded to
// 4).  Every word of a stored vector has bit 31 set, so a slot whose words are
// all zero is empty and a slot is a consistent stored vector exactly when all
// its words carry the tag.
//
// Cooperation.  A group of G consecutive lanes of a warp serves one bucket
// (the paper's "thread group per bucket"; G = B / W gives one lane per slot,
// the GB300 counterpart of the paper's one thread per word -- each lane loads
// its slot with one vector load).  Each lane reads SPL = S / G slots.
//
// Differences from the paper's table, on purpose:
//   * insertion claims a whole slot with one 32/64/128-bit atomic CAS instead
//     of relying on half-warp writes being scheduled without interruption
//     (that assumption does not hold under independent thread scheduling);
//   * a slot that is read half-written (not all words tagged) is treated as a
//     candidate for the CAS, whose return value is the slot's true content,
//     so no read ever has to wait for another writer;
//   * the hash-constant sets of Sec. 4.1 are multiply-shift multipliers
//     (Dietzfelbinger et al. 1997) over a splitmix64-mixed vector.
#pragma once

#include <cstdint>

namespace gxd {

constexpr uint32_t kTag = 0x80000000u;
constexpr uint32_t FULLMASK = 0xFFFFFFFFu;
constexpr int kMaxRounds = 64;

enum : int { FOP_FOUND = 0, FOP_INSERTED = 1, FOP_FULL = 2 };

// splitmix64 output function (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <int W>
__device__ __forceinline__ uint64_t vec_hash(const uint32_t (&v)[W]) {
  uint64_t x;
  if constexpr (W == 1) {
    x = v[0];
  } else if constexpr (W == 2) {
    x = (uint64_t)v[0] | ((uint64_t)v[1] << 32);
  } else {
    // the upper half multiplied by an odd constant (a bijection), added to the lower
    // half, then one finaliser: one mix64 per vector instead of two
    x = ((uint64_t)v[0] | ((uint64_t)v[1] << 32)) +
        ((uint64_t)v[2] | ((uint64_t)v[3] << 32)) * 0xD6E8FEB86659FD93ull;
  }
  return mix64(x);
}

// Bucket of hash-constant set `round`: multiply-shift with an odd multiplier.
__device__ __forceinline__ uint64_t bucket_of(uint64_t h, uint64_t mul, int log2nb) {
  return (h * mul) >> (64 - log2nb);
}

// Span of the later hash rounds: 2^kSpanLog2Bytes bytes of table (64 GiB).
// Random reads run at the full rate inside any 64 GiB of device memory and
// about 4x slower across 128 GiB (the reach of the GPU's address translation),
// so in a larger table every round after the first stays inside the 64 GiB
// span that round 0 picked: the top bits of the bucket come from round 0, the
// rest from the round's own multiplier.  Tables of at most 64 GiB are not
// affected.  A region pass that takes the successors of one span (or part of
// one) then reads nothing outside it, in any round.
constexpr int kSpanLog2Bytes = 36;

// Bucket of round k >= 1 for a table of 2^log2nb buckets of B words, given
// round 0's bucket b0.
template <int B>
__device__ __forceinline__ uint64_t bucket_in_span(uint64_t h, uint64_t mul, int log2nb, uint64_t b0) {
  static_assert(B >= 1 && B <= 64 && (B & (B - 1)) == 0, "bucket words: a power of two up to 64");
  constexpr int kSpanLog2 = kSpanLog2Bytes - 2 - (B >= 2) - (B >= 4) - (B >= 8) - (B >= 16) - (B >= 32) - (B >= 64);
  if (log2nb <= kSpanLog2) return bucket_of(h, mul, log2nb);
  return ((b0 >> kSpanLog2) << kSpanLog2) | bucket_of(h, mul, kSpanLog2);
}

// ---- loads that bypass L1 (the table is shared by all SMs; slots only ever
// go from empty to one final value, so a stale copy is never wrong, but L1
// allocation is pure overhead for random probes).
template <int LW>
__device__ __forceinline__ void load_words(const uint32_t* p, uint32_t (&s)[LW]) {
  if constexpr (LW == 1) {
    s[0] = __ldcg(p);
  } else if constexpr (LW == 2) {
    uint2 x = __ldcg(reinterpret_cast<const uint2*>(p));
    s[0] = x.x;
    s[1] = x.y;
  } else if constexpr (LW == 4) {
    uint4 x = __ldcg(reinterpret_cast<const uint4*>(p));
    s[0] = x.x;
    s[1] = x.y;
    s[2] = x.z;
    s[3] = x.w;
  } else {
    // 256-bit loads (sm_100 and later): one instruction per 32-byte sector
    static_assert(LW % 8 == 0, "lane load width");
#pragma unroll
    for (int i = 0; i < LW / 8; ++i) {
      asm volatile("ld.global.cg.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(s[8 * i + 0]), "=r"(s[8 * i + 1]), "=r"(s[8 * i + 2]), "=r"(s[8 * i + 3]),
                     "=r"(s[8 * i + 4]), "=r"(s[8 * i + 5]), "=r"(s[8 * i + 6]), "=r"(s[8 * i + 7])
                   : "l"(p + 8 * i));
    }
  }
}

// Compare-and-swap of a whole empty slot (all zero) to v.  Returns true if
// this call stored v; otherwise `old` holds the slot's content.
template <int W>
__device__ __forceinline__ bool cas_slot(uint32_t* p, const uint32_t (&v)[W], uint32_t (&old)[W]) {
  if constexpr (W == 1) {
    old[0] = atomicCAS(p, 0u, v[0]);
    return old[0] == 0u;
  } else if constexpr (W == 2) {
    unsigned long long nv = (unsigned long long)v[0] | ((unsigned long long)v[1] << 32);
    unsigned long long o = atomicCAS(reinterpret_cast<unsigned long long*>(p), 0ull, nv);
    old[0] = (uint32_t)o;
    old[1] = (uint32_t)(o >> 32);
    return o == 0ull;
  } else {
    static_assert(W == 4, "slot width");
    unsigned long long nlo = (unsigned long long)v[0] | ((unsigned long long)v[1] << 32);
    unsigned long long nhi = (unsigned long long)v[2] | ((unsigned long long)v[3] << 32);
    unsigned long long olo, ohi;
    asm volatile(
        "{\n\t.reg .b128 d, c, n;\n\t"
        "mov.b128 c, {%2, %2};\n\t"
        "mov.b128 n, {%3, %4};\n\t"
        "atom.global.cas.b128 d, [%5], c, n;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(olo), "=l"(ohi)
        : "l"(0ull), "l"(nlo), "l"(nhi), "l"(p)
        : "memory");
    old[0] = (uint32_t)olo;
    old[1] = (uint32_t)(olo >> 32);
    old[2] = (uint32_t)ohi;
    old[3] = (uint32_t)(ohi >> 32);
    return (olo | ohi) == 0ull;
  }
}

template <int G>
struct Group {
  uint32_t mask;  // lanes of this group within the warp
  int base;       // first lane of the group
  int glane;      // lane index within the group
  __device__ __forceinline__ Group() {
    const int lane = threadIdx.x & 31;
    base = lane & ~(G - 1);
    glane = lane - base;
    mask = (G == 32) ? FULLMASK : (((1u << G) - 1u) << base);
  }
  __device__ __forceinline__ bool any(bool p) const {
    if constexpr (G == 1) return p;
    else return __any_sync(mask, p);
  }
  __device__ __forceinline__ uint32_t ballot(bool p) const {
    if constexpr (G == 1) return p ? (1u << (threadIdx.x & 31)) : 0u;
    else return __ballot_sync(mask, p);
  }
  template <typename T>
  __device__ __forceinline__ T bcast(T x, int src_lane) const {
    if constexpr (G == 1) return x;
    else return __shfl_sync(mask, x, src_lane);
  }
};

// Find-or-put of vector v (identical in every lane of the group).  All G lanes
// of the group must call it together.  Returns FOP_FOUND, FOP_INSERTED or
// FOP_FULL (no free slot under any of the `rounds` hash-constant sets), the
// same value in every lane of the group.  `probes` of the group's first lane
// is increased by the number of buckets read (once per bucket, not per lane).
// With PRE, `pre` already holds this lane's part of the first bucket (read by
// the caller, and counted there), so round 0 starts without a load.
// find_or_put_hashed takes h = vec_hash(v) from the caller.
template <int W, int B, int G, bool PRE>
__device__ __forceinline__ int find_or_put_hashed(uint32_t* __restrict__ table, int log2nb, int rounds,
                                                  const uint64_t* __restrict__ muls,
                                                  const uint32_t (&v)[W], const uint64_t h, const Group<G>& g,
                                                  uint32_t& probes, const uint32_t (&pre)[(B / W / G) * W]) {
  constexpr int S = B / W;
  static_assert(S >= 1 && S % G == 0, "group size must divide the slots per bucket");
  constexpr int SPL = S / G;
  constexpr int LW = SPL * W;
  const uint64_t b0 = bucket_of(h, muls[0], log2nb);
  for (int k = 0; k < rounds; ++k) {
    const uint64_t b = k == 0 ? b0 : bucket_in_span<B>(h, muls[k], log2nb, b0);
    uint32_t* lane_slots = table + b * (uint64_t)B + (uint64_t)g.glane * LW;
    uint32_t s[LW];
    if (PRE && k == 0) {
#pragma unroll
      for (int i = 0; i < LW; ++i) s[i] = pre[i];
    } else {
      load_words<LW>(lane_slots, s);
      probes += g.glane == 0;
    }
    bool match = false;
    uint32_t cand = 0;  // slots that are empty or half-written
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
      bool eq = true, tagged = true;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        eq &= (s[j * W + w] == v[w]);
        tagged &= (s[j * W + w] & kTag) != 0;
      }
      match |= eq;
      if (!tagged) cand |= 1u << j;
    }
    if (g.any(match)) return FOP_FOUND;
    // Claim the first candidate slot of the group; on failure the CAS tells
    // what the slot holds: our vector (found) or another one (try the next).
    while (true) {
      const uint32_t want = g.ballot(cand != 0);
      if (want == 0) break;
      const int leader = __ffs(want) - 1;
      int res = -1;
      if ((int)(threadIdx.x & 31) == leader) {
        const int j = __ffs(cand) - 1;
        uint32_t old[W];
        if (cas_slot<W>(lane_slots + j * W, v, old)) {
          res = FOP_INSERTED;
        } else {
          bool eq = true;
#pragma unroll
          for (int w = 0; w < W; ++w) eq &= (old[w] == v[w]);
          if (eq) res = FOP_FOUND;
          cand &= ~(1u << j);
        }
      }
      res = g.bcast(res, leader);
      if (res >= 0) return res;
    }
  }
  return FOP_FULL;
}

template <int W, int B, int G, bool PRE>
__device__ __forceinline__ int find_or_put_from(uint32_t* __restrict__ table, int log2nb, int rounds,
                                                const uint64_t* __restrict__ muls,
                                                const uint32_t (&v)[W], const Group<G>& g,
                                                uint32_t& probes, const uint32_t (&pre)[(B / W / G) * W]) {
  return find_or_put_hashed<W, B, G, PRE>(table, log2nb, rounds, muls, v, vec_hash<W>(v), g, probes, pre);
}

template <int W, int B, int G>
__device__ __forceinline__ int find_or_put(uint32_t* __restrict__ table, int log2nb, int rounds,
                                           const uint64_t* __restrict__ muls,
                                           const uint32_t (&v)[W], const Group<G>& g,
                                           uint32_t& probes) {
  const uint32_t none[(B / W / G) * W] = {};
  return find_or_put_from<W, B, G, false>(table, log2nb, rounds, muls, v, g, probes, none);
}

// ---- vector fields

template <int W>
__device__ __forceinline__ uint32_t word_at(const uint32_t (&v)[W], uint32_t i) {
  uint32_t r = v[0];
#pragma unroll
  for (int k = 1; k < W; ++k)
    if (i == (uint32_t)k) r = v[k];
  return r;
}

template <int W>
__device__ __forceinline__ void xor_at(uint32_t (&v)[W], uint32_t i, uint32_t d) {
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (i == (uint32_t)k) v[k] ^= d;
}

}  // namespace gxd

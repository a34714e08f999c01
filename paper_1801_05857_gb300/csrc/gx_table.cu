// C ABI of the isolated hash-table experiment (Sec. 5.1), of the cuckoo table
// Sec. 4.1 compares against, and of the random-access probes that give the
// table its roofline.

#include <string>

#include "gx_kernels.cuh"

namespace gxd {

// Counter-based position stream: access i of a probe run goes to unit
// mix64(seed + i) & (n_units - 1) (n_units a power of two), so every access is
// independent.  Each thread keeps K accesses in flight; a unit is read with
// 256-bit loads (one load for a 32-byte unit).
template <int K, int UW>
__global__ void __launch_bounds__(gx::kBlock)
probe_gather_kernel(const uint32_t* __restrict__ buf, uint64_t unit_mask, uint64_t n, uint64_t seed,
                    unsigned long long* sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * K;
  uint32_t acc = 0;
  for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * K; i0 < n; i0 += stride) {
    uint32_t x[K][UW];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const uint64_t u = mix64(seed + i0 + j) & unit_mask;
      if (i0 + j < n) load_words<UW>(buf + u * UW, x[j]);
      else
#pragma unroll
        for (int w = 0; w < UW; ++w) x[j][w] = 0;
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
      for (int w = 0; w < UW; ++w) acc ^= x[j][w];
  }
  acc = __reduce_xor_sync(FULLMASK, acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicXor(sink, (unsigned long long)acc);
}

// Gathers with a chosen launch shape and access locality, for measuring the
// random-access ceiling itself.  Access i reads LW words at the start of unit
// u(i) of UNIT_WORDS words (LW = 1 touches one word, which still moves the
// whole sector, with one register per access in flight).  Each thread issues
// K accesses before it uses any.  With group_bits = g > 0, the 32 x K accesses
// of one warp iteration fall in one randomly chosen aligned block of 2^g
// units (locality within a page), otherwise every access is independent.
template <int K, int LW>
__global__ void __launch_bounds__(gx::kBlock)
probe_sweep_kernel(const uint32_t* __restrict__ buf, int unit_words, uint64_t unit_mask, uint32_t group_bits,
                   uint64_t n, uint64_t seed, unsigned long long* sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * K;
  const uint64_t inner = (1ull << group_bits) - 1ull;
  uint32_t acc = 0;
  for (uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * K; i0 < n; i0 += stride) {
    // i0 / (32 K) is the same in every lane of the warp (the stride is a multiple of 32 K)
    const uint64_t block = group_bits ? (mix64(~seed ^ (i0 / (32ull * K))) & unit_mask & ~inner) : 0ull;
    // every position is inside the buffer, so all K loads are issued without a
    // branch; those past n are simply not used
    uint32_t x[K][LW];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const uint64_t r = mix64(seed + i0 + j);
      const uint64_t u = group_bits ? (block | (r & inner)) : (r & unit_mask);
      load_words<LW>(buf + u * (uint64_t)unit_words, x[j]);
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (i0 + j < n)
#pragma unroll
        for (int w = 0; w < LW; ++w) acc ^= x[j][w];
  }
  acc = __reduce_xor_sync(FULLMASK, acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicXor(sink, (unsigned long long)acc);
}

__global__ void __launch_bounds__(gx::kBlock)
probe_cas_kernel(uint32_t* __restrict__ buf, uint64_t unit_mask, int unit_words, uint64_t n,
                 uint64_t seed, unsigned long long* sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t acc = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t u = mix64(seed + i) & unit_mask;
    uint32_t* p = buf + u * unit_words;
    const uint32_t tag = (uint32_t)(i | 1u) | kTag;
    if (unit_words == 1) {
      uint32_t v[1] = {tag}, o[1];
      cas_slot<1>(p, v, o);
      acc ^= o[0];
    } else if (unit_words == 2) {
      uint32_t v[2] = {tag, tag}, o[2];
      cas_slot<2>(p, v, o);
      acc ^= o[0] ^ o[1];
    } else {
      uint32_t v[4] = {tag, tag, tag, tag}, o[4];
      cas_slot<4>(p, v, o);
      acc ^= o[0] ^ o[3];
    }
  }
  acc = __reduce_xor_sync(FULLMASK, acc);
  if ((threadIdx.x & 31) == 0 && acc) atomicXor(sink, (unsigned long long)acc);
}

// ---- Cuckoo hashing (Pagh & Rodler 2004) in the GPU form of Alcantara et al.,
// the alternative table Sec. 4.1 weighs against its own.  One thread per key.
// A slot is one tagged key: 32 bits for 1-word keys, 64 bits for 2-word keys,
// so a lookup or an exchange is one aligned access.  Position i of a key is
// (mix64(key) * m_i) >> (64 - log2 slots).
constexpr int kCuckooMaxHash = 8;

struct CuckooArgs {
  const uint32_t* keys;
  uint64_t n;
  void* table;
  int log2slots, n_hash, max_chain;
  uint64_t m[kCuckooMaxHash];
  uint8_t* result;
  unsigned long long* counters;  // inserted, found, failed, exchanges
};

template <int W>
struct CuckooSlot;
template <>
struct CuckooSlot<1> {
  using T = uint32_t;
  static __device__ __forceinline__ T pack(const uint32_t* k) { return k[0] | kTag; }
  static __device__ __forceinline__ uint64_t hash(T x) { return mix64(x); }
};
template <>
struct CuckooSlot<2> {
  using T = unsigned long long;
  static __device__ __forceinline__ T pack(const uint32_t* k) {
    return (T)(k[0] | kTag) | ((T)(k[1] | kTag) << 32);
  }
  static __device__ __forceinline__ uint64_t hash(T x) { return mix64(x); }
};

template <int W>
__global__ void __launch_bounds__(gx::kBlock) cuckoo_kernel(const CuckooArgs a) {
  using S = CuckooSlot<W>;
  using T = typename S::T;
  T* table = static_cast<T*>(a.table);
  const int sh = 64 - a.log2slots;
  const int k = a.n_hash;
  unsigned long long ins = 0, fnd = 0, fail = 0, exch = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const T key = S::pack(a.keys + i * W);
    const uint64_t h = S::hash(key);
    // lookup: the first position alone (where most keys sit), then the others at once
    bool found = __ldcg(&table[(h * a.m[0]) >> sh]) == key;
    if (!found) {
      T s[kCuckooMaxHash];
#pragma unroll
      for (int j = 1; j < kCuckooMaxHash; ++j) s[j] = j < k ? __ldcg(&table[(h * a.m[j]) >> sh]) : T(0);
#pragma unroll
      for (int j = 1; j < kCuckooMaxHash; ++j) found |= (j < k && s[j] == key);
    }
    int r = FOP_FOUND;
    if (!found) {
      // insertion: exchange into position 0; an evicted key moves on to the position
      // after the one it sat in, at most max_chain exchanges in all
      r = FOP_INSERTED;
      T x = key;
      uint64_t pos = (h * a.m[0]) >> sh;
      int step = 0;
      for (;; ++step) {
        if (step == a.max_chain) {  // the key carried now is dropped
          r = FOP_FULL;
          break;
        }
        const T old = atomicExch(&table[pos], x);
        if (old == T(0)) break;
        if (old == x) {  // the slot already held the carried key
          if (step == 0) r = FOP_FOUND;
          break;
        }
        x = old;
        const uint64_t ho = S::hash(old);
        int j = 0;
        while (j < k - 1 && ((ho * a.m[j]) >> sh) != pos) ++j;
        j = (j + 1 == k) ? 0 : j + 1;
        pos = (ho * a.m[j]) >> sh;
      }
      exch += (unsigned long long)(step + (r != FOP_FULL));
    }
    if (a.result) a.result[i] = (uint8_t)(r == FOP_INSERTED ? 1 : (r == FOP_FOUND ? 0 : 2));
    ins += r == FOP_INSERTED;
    fnd += r == FOP_FOUND;
    fail += r == FOP_FULL;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ins += __shfl_xor_sync(FULLMASK, ins, o);
    fnd += __shfl_xor_sync(FULLMASK, fnd, o);
    fail += __shfl_xor_sync(FULLMASK, fail, o);
    exch += __shfl_xor_sync(FULLMASK, exch, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ins) atomicAdd(&a.counters[0], ins);
    if (fnd) atomicAdd(&a.counters[1], fnd);
    if (fail) atomicAdd(&a.counters[2], fail);
    if (exch) atomicAdd(&a.counters[3], exch);
  }
}

}  // namespace gxd

namespace {

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

}  // namespace

extern "C" {

gx_status gx_find_or_put(const uint32_t* keys, uint64_t n_keys, uint32_t key_words,
                         uint32_t bucket_words, uint32_t group_lanes, uint32_t hash_rounds,
                         uint32_t* table, uint64_t table_words, uint8_t* result,
                         uint64_t* counters, void* stream) {
  gx::clear_error();
  if (key_words != 1 && key_words != 2 && key_words != 4)
    return gx::fail(GX_ERR_INVALID, "key_words must be 1, 2 or 4");
  const int W = (int)key_words;
  const int B = bucket_words ? (int)bucket_words : 8;
  if (B != 4 && B != 8 && B != 16 && B != 32) return gx::fail(GX_ERR_INVALID, "bucket_words must be 4, 8, 16 or 32");
  if (B < W) return gx::fail(GX_ERR_INVALID, "bucket smaller than one key");
  const int S = B / W;
  const int G = group_lanes ? (int)group_lanes : (S < 32 ? S : 32);
  const int rounds = hash_rounds ? (int)hash_rounds : 8;
  if (rounds < 1 || rounds > gx::kMaxRounds) return gx::fail(GX_ERR_INVALID, "hash_rounds must be 1..64");
  const gx::KernelSet* ks = gx::kernels_for(W, B, G);
  if (!ks) return gx::fail(GX_ERR_INVALID, "group_lanes must be a power of two dividing bucket_words / key_words");
  if (!table || !counters || (n_keys && !keys)) return gx::fail(GX_ERR_INVALID, "NULL device pointer");
  if (reinterpret_cast<uintptr_t>(table) % 256) return gx::fail(GX_ERR_INVALID, "table is not 256-byte aligned");
  if (table_words % B) return gx::fail(GX_ERR_INVALID, "table_words is not a multiple of bucket_words");
  const uint64_t nb = table_words / B;
  if (nb < 2 || (nb & (nb - 1))) return gx::fail(GX_ERR_INVALID, "bucket count must be a power of two >= 2");
  if (n_keys == 0) return GX_OK;
  int log2nb = 0;
  while ((1ull << log2nb) < nb) ++log2nb;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  gx::FopArgs a{};
  a.keys = keys;
  a.n = n_keys;
  a.table = table;
  a.log2nb = log2nb;
  a.rounds = rounds;
  gx::hash_multipliers(a.muls.m, gx::kMaxRounds);
  a.result = result;
  a.counters = reinterpret_cast<unsigned long long*>(counters);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ks->fop_fn, gx::kBlock, 0);
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, cudaGetErrorString(e));
  const uint64_t groups_needed = n_keys;
  const uint64_t blocks_needed = (groups_needed * G + gx::kBlock - 1) / gx::kBlock;
  // A grid of 16 times the CTAs that fit at once (the loop is grid-stride and a CTA's
  // setup is 64 multipliers): random reads from a grid whose CTAs finish and start during
  // the launch run faster than from a resident one (10^8 keys at d = 1, 8-word buckets,
  // one lane per bucket: 27.3 against 23.8 G keys/s; at d = 21: 56.2 against 50.3).
  const uint64_t cap = (uint64_t)sm_count() * (per_sm > 0 ? per_sm : 1) * 16;
  const int grid = (int)(blocks_needed < cap ? blocks_needed : cap);
  e = ks->fop(a, grid > 0 ? grid : 1, st);
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, cudaGetErrorString(e));
  return GX_OK;
}

gx_status gx_cuckoo_find_or_put(const uint32_t* keys, uint64_t n_keys, uint32_t key_words,
                                uint32_t n_hash, uint32_t max_chain, const uint64_t* muls,
                                uint32_t* table, uint64_t table_slots, uint8_t* result,
                                uint64_t* counters, void* stream) {
  gx::clear_error();
  if (key_words != 1 && key_words != 2) return gx::fail(GX_ERR_INVALID, "key_words must be 1 or 2");
  const int k = n_hash ? (int)n_hash : 4;
  if (k < 2 || k > gxd::kCuckooMaxHash) return gx::fail(GX_ERR_INVALID, "n_hash must be 2..8");
  const int chain = max_chain ? (int)max_chain : 128;
  if (chain < 1 || chain > 4096) return gx::fail(GX_ERR_INVALID, "max_chain must be 1..4096");
  if (!table || !counters || (n_keys && !keys)) return gx::fail(GX_ERR_INVALID, "NULL device pointer");
  if (reinterpret_cast<uintptr_t>(table) % 256) return gx::fail(GX_ERR_INVALID, "table is not 256-byte aligned");
  if (table_slots < 2 || (table_slots & (table_slots - 1)))
    return gx::fail(GX_ERR_INVALID, "table_slots must be a power of two >= 2");
  gxd::CuckooArgs a{};
  if (muls) {
    for (int j = 0; j < k; ++j) {
      if (!(muls[j] & 1)) return gx::fail(GX_ERR_INVALID, "hash multipliers must be odd");
      a.m[j] = muls[j];
    }
  } else {
    gx::hash_multipliers(a.m, k);
  }
  if (n_keys == 0) return GX_OK;
  int log2slots = 0;
  while ((1ull << log2slots) < table_slots) ++log2slots;
  a.keys = keys;
  a.n = n_keys;
  a.table = table;
  a.log2slots = log2slots;
  a.n_hash = k;
  a.max_chain = chain;
  a.result = result;
  a.counters = reinterpret_cast<unsigned long long*>(counters);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int per_sm = 0;
  cudaError_t e = key_words == 1
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gxd::cuckoo_kernel<1>, gx::kBlock, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gxd::cuckoo_kernel<2>, gx::kBlock, 0);
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, cudaGetErrorString(e));
  const uint64_t blocks_needed = (n_keys + gx::kBlock - 1) / gx::kBlock;
  // the same grid as gx_find_or_put's (16 times the CTAs that fit at once), so that the
  // comparison of the two tables is on equal terms
  const uint64_t cap = (uint64_t)sm_count() * (per_sm > 0 ? per_sm : 1) * 16;
  const int grid = (int)(blocks_needed < cap ? blocks_needed : cap);
  if (key_words == 1) gxd::cuckoo_kernel<1><<<grid > 0 ? grid : 1, gx::kBlock, 0, st>>>(a);
  else gxd::cuckoo_kernel<2><<<grid > 0 ? grid : 1, gx::kBlock, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, cudaGetErrorString(e));
  return GX_OK;
}

gx_status gx_probe_random(uint32_t kind, uint32_t* buffer, uint64_t words, uint64_t n,
                          uint32_t bytes, uint64_t seed, uint64_t* sink, void* stream) {
  gx::clear_error();
  if (!buffer || !sink) return gx::fail(GX_ERR_INVALID, "NULL device pointer");
  if (reinterpret_cast<uintptr_t>(buffer) % 256) return gx::fail(GX_ERR_INVALID, "buffer is not 256-byte aligned");
  int unit_words;
  if (kind == 0) {
    if (bytes != 16 && bytes != 32 && bytes != 64 && bytes != 128)
      return gx::fail(GX_ERR_INVALID, "gather bytes must be 16, 32, 64 or 128");
    unit_words = (int)bytes / 4;
  } else if (kind == 1) {
    if (bytes != 4 && bytes != 8 && bytes != 16) return gx::fail(GX_ERR_INVALID, "CAS bytes must be 4, 8 or 16");
    unit_words = (int)bytes / 4;
  } else {
    return gx::fail(GX_ERR_INVALID, "kind must be 0 (gather) or 1 (CAS)");
  }
  uint64_t n_units = 1;
  while (n_units * 2 * unit_words <= words) n_units *= 2;  // largest power of two that fits
  if ((uint64_t)unit_words > words) return gx::fail(GX_ERR_INVALID, "buffer smaller than one access");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = sm_count() * 8;
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(sink);
  if (kind == 0) {
    // 4 accesses in flight per thread for small units, 2 for 64/128-byte units
    if (unit_words == 4) gxd::probe_gather_kernel<4, 4><<<grid, gx::kBlock, 0, st>>>(buffer, n_units - 1, n, seed, sk);
    else if (unit_words == 8) gxd::probe_gather_kernel<4, 8><<<grid, gx::kBlock, 0, st>>>(buffer, n_units - 1, n, seed, sk);
    else if (unit_words == 16) gxd::probe_gather_kernel<2, 16><<<grid, gx::kBlock, 0, st>>>(buffer, n_units - 1, n, seed, sk);
    else gxd::probe_gather_kernel<2, 32><<<grid, gx::kBlock, 0, st>>>(buffer, n_units - 1, n, seed, sk);
  } else
    gxd::probe_cas_kernel<<<grid, gx::kBlock, 0, st>>>(buffer, n_units - 1, unit_words, n, seed,
                                                       reinterpret_cast<unsigned long long*>(sink));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, cudaGetErrorString(e));
  return GX_OK;
}

gx_status gx_probe_gather(uint32_t* buffer, uint64_t words, uint64_t n, uint32_t unit_bytes,
                          uint32_t load_bytes, uint32_t in_flight, uint32_t ctas_per_sm, uint32_t group_log2,
                          uint64_t seed, uint64_t* sink, void* stream, uint32_t* ctas_used) {
  gx::clear_error();
  if (!buffer || !sink) return gx::fail(GX_ERR_INVALID, "NULL device pointer");
  if (reinterpret_cast<uintptr_t>(buffer) % 256) return gx::fail(GX_ERR_INVALID, "buffer is not 256-byte aligned");
  if (unit_bytes != 32 && unit_bytes != 64 && unit_bytes != 128)
    return gx::fail(GX_ERR_INVALID, "unit_bytes must be 32, 64 or 128");
  if (load_bytes != 4 && load_bytes != unit_bytes)
    return gx::fail(GX_ERR_INVALID, "load_bytes must be 4 or unit_bytes");
  const int K = (int)in_flight;
  if (K != 1 && K != 2 && K != 4 && K != 8 && K != 16 && K != 32)
    return gx::fail(GX_ERR_INVALID, "in_flight must be 1, 2, 4, 8, 16 or 32");
  if (load_bytes > 4 && K > 16) return gx::fail(GX_ERR_INVALID, "in_flight above 16 only with 4-byte loads");
  if (load_bytes > 64 && K > 4) return gx::fail(GX_ERR_INVALID, "in_flight above 4 only with loads of at most 64 bytes");
  if (ctas_per_sm < 1 || ctas_per_sm > 32) return gx::fail(GX_ERR_INVALID, "ctas_per_sm must be 1..32");
  const int unit_words = (int)unit_bytes / 4;
  if ((uint64_t)unit_words > words) return gx::fail(GX_ERR_INVALID, "buffer smaller than one access");
  uint64_t n_units = 1;
  while (n_units * 2 * unit_words <= words) n_units *= 2;
  uint32_t gbits = 0;
  if (group_log2) {
    uint32_t ub = unit_bytes == 32 ? 5 : unit_bytes == 64 ? 6 : 7;
    if (group_log2 < ub) return gx::fail(GX_ERR_INVALID, "group_log2 smaller than one unit");
    gbits = group_log2 - ub;
    if ((1ull << gbits) > n_units) return gx::fail(GX_ERR_INVALID, "locality group larger than the buffer");
  }
  const void* fn = nullptr;
  using Fn = void (*)(const uint32_t*, int, uint64_t, uint32_t, uint64_t, uint64_t, unsigned long long*);
  Fn f = nullptr;
  const int lw = (int)load_bytes / 4;
#define GX_SWEEP(KK, LL) \
  if (K == KK && lw == LL) f = gxd::probe_sweep_kernel<KK, LL>;
  GX_SWEEP(1, 1) GX_SWEEP(2, 1) GX_SWEEP(4, 1) GX_SWEEP(8, 1) GX_SWEEP(16, 1) GX_SWEEP(32, 1)
  GX_SWEEP(1, 8) GX_SWEEP(2, 8) GX_SWEEP(4, 8) GX_SWEEP(8, 8) GX_SWEEP(16, 8)
  GX_SWEEP(1, 16) GX_SWEEP(2, 16) GX_SWEEP(4, 16) GX_SWEEP(8, 16) GX_SWEEP(16, 16)
  GX_SWEEP(1, 32) GX_SWEEP(2, 32) GX_SWEEP(4, 32)
#undef GX_SWEEP
  if (!f) return gx::fail(GX_ERR_INVALID, "no such probe shape");
  fn = reinterpret_cast<const void*>(f);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, gx::kBlock, 0);
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, cudaGetErrorString(e));
  // up to 8: lowered to what fits at once (a resident grid); above 8: as asked, so the
  // grid runs in more than one wave
  const int ctas = ctas_per_sm > 8 ? (int)ctas_per_sm
                                   : ((int)ctas_per_sm < per_sm ? (int)ctas_per_sm : (per_sm > 0 ? per_sm : 1));
  if (ctas_used) *ctas_used = (uint32_t)ctas;
  if (n == 0) return GX_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  f<<<sm_count() * ctas, gx::kBlock, 0, st>>>(buffer, unit_words, n_units - 1, gbits, n, seed,
                                               reinterpret_cast<unsigned long long*>(sink));
  e = cudaGetLastError();
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, cudaGetErrorString(e));
  return GX_OK;
}

}  // extern "C"

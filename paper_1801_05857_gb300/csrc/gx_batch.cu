// Batched exploration: many independent networks in one persistent launch
// per BFS iteration, the iterations driven on the device by a CUDA graph with
// a conditional WHILE node (no counterpart in the paper, which explores one
// network at a time; the per-network work is the level expansion of Sec. 3
// with the find-or-put of Sec. 4.1).
//
// Graph (built once per workspace / options, relaunched per call):
//   memset(all tables) -> init (initial vector of every network) -> advance(first)
//   -> WHILE(any network active) { expand_all ; advance }
// advance records each network's finished level, moves its level window,
// computes the prefix of 32-state chunks over the active networks and sets
// the loop condition.  expand_all is persistent: every warp claims chunks of
// any network's current level.
//
// Workspace: per-network descriptors | chunk prefix | claim counter |
//            network blobs | level arrays | frontier rings | tables (contiguous)

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "gx_kernels.cuh"

namespace gx {

struct BNet {
  const uint32_t* blob;
  NetBlobLayout lay;
  uint32_t* table;
  int log2nb;
  uint32_t levels_cap;
  uint32_t* frontier;
  uint64_t fmask;
  unsigned long long* levels;
  unsigned long long cur_begin, cur_end, next_end;
  unsigned long long transitions, dl_count, dl_sum, dl_xor, probes;
  unsigned int error, active, n_levels;
  int first_dl;
  uint32_t init_vec[4];
};

struct BatchArgs {
  BNet* nets;
  int n;
  int rounds;
  int chunk;  // states per claimed chunk
  Muls muls;
  unsigned long long* prefix;  // n + 1 entries
  unsigned long long* claim;
  unsigned long long* iters;   // iterations of the WHILE loop so far
  unsigned long long* unit;    // states per claim this iteration: chunk, or 1 (one warp per state)
  unsigned long long wide_states;  // iterations with at most this many states use unit 1
  unsigned long long max_iters;
  cudaGraphConditionalHandle cond;
};

constexpr unsigned int ERR_LEVELS = 8u;  // a network needed more levels than levels_cap

}  // namespace gx

namespace gxd {

using gx::BatchArgs;
using gx::BNet;

template <int W, int B, int G>
__global__ void __launch_bounds__(gx::kBlock) batch_init_kernel(const BatchArgs a) {
  __shared__ uint64_t muls[kMaxRounds];
  for (int i = threadIdx.x; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  __syncthreads();
  const int net = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (net >= a.n || (int)(threadIdx.x & 31) >= G) return;
  BNet& b = a.nets[net];
  const Group<G> g;
  uint32_t v[W];
#pragma unroll
  for (int w = 0; w < W; ++w) v[w] = b.init_vec[w];
  uint32_t probes = 0;
  const int r = find_or_put<W, B, G>(b.table, b.log2nb, a.rounds, muls, v, g, probes);
  if (g.glane == 0) {
    if (r == FOP_INSERTED) store_vec<W>(b.frontier, v);
    b.cur_begin = 0;
    b.cur_end = 1;
    b.next_end = 1;
    b.transitions = b.dl_count = b.dl_sum = b.dl_xor = 0;
    b.probes = probes;
    b.error = r == FOP_INSERTED ? 0u : gx::ERR_TABLE_FULL;
    b.active = r == FOP_INSERTED ? 1u : 0u;
    b.first_dl = -1;
    b.n_levels = 1;
    b.levels[0] = 1;
  }
}

// One CTA: finish the level just expanded for every network, then lay out the
// next iteration's chunks.
__global__ void __launch_bounds__(1024) batch_advance_kernel(const BatchArgs a, int first) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long carry, s_unit;
  if (threadIdx.x == 0) carry = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // 1. close the level just expanded and count the states of the next one
  unsigned long long states = 0;
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    BNet& b = a.nets[i];
    if (!first && b.active) {
      const unsigned long long fresh = b.next_end - b.cur_end;
      if (b.dl_count > 0 && b.first_dl < 0) b.first_dl = (int)b.n_levels - 1;
      if (fresh > 0) {
        if (b.n_levels < b.levels_cap) b.levels[b.n_levels] = fresh;
        else b.error |= gx::ERR_LEVELS;
        b.n_levels += 1;
      }
      if (b.error || fresh == 0) {
        b.active = 0;
      } else {
        b.cur_begin = b.cur_end;
        b.cur_end = b.next_end;
      }
    }
    if (b.active) states += b.cur_end - b.cur_begin;
  }
  states = warp_sum(states);
  if (lane == 0) warp_tot[wid] = states;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += warp_tot[w];
    // few states in all: give each one a warp, so that its successors' lookups overlap
    s_unit = tot <= a.wide_states ? 1ull : (unsigned long long)a.chunk;
  }
  __syncthreads();
  const unsigned long long unit = s_unit;
  // 2. claims per network and their exclusive prefix sums
  for (int base = 0; base < a.n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    unsigned long long chunks = 0;
    if (i < a.n) {
      const BNet& b = a.nets[i];
      if (b.active) chunks = (b.cur_end - b.cur_begin + unit - 1) / unit;
    }
    // block-wide inclusive scan of chunks
    unsigned long long inc = chunks;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULLMASK, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      const int nw = blockDim.x / 32;
      unsigned long long w = lane < nw ? warp_tot[lane] : 0ull;
      unsigned long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULLMASK, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < nw) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    const unsigned long long ex = carry + warp_tot[wid] + inc - chunks;
    if (i < a.n) a.prefix[i] = ex;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + chunks;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // iteration guard: every active network gains one level per iteration, so
    // more than max_iters iterations cannot happen; stop the loop regardless
    const unsigned long long it = first ? 0ull : *a.iters + 1;
    *a.iters = it;
    bool more = carry > 0;
    if (more && it >= a.max_iters) {
      for (int i = 0; i < a.n; ++i)
        if (a.nets[i].active) {
          a.nets[i].error |= gx::ERR_LEVELS;
          a.nets[i].active = 0;
        }
      more = false;
    }
    a.prefix[a.n] = carry;
    *a.claim = 0;
    *a.unit = unit;
    cudaGraphSetConditional(a.cond, more ? 1u : 0u);
  }
}

// Per-warp cache of seen vectors in the batched kernel (1- and 2-word slots).
// Networks have separate tables, so a hit is only valid for the network whose
// vectors filled the cache: a warp clears its cache whenever it moves to a
// chunk of another network.
constexpr int kBatchCacheLog2 = 9;

// The network a warp is working on, staged in shared memory when the warp
// moves to it, so that its layout and table pointers take no registers in the
// inner loop.
struct WarpNet {
  NetBlobLayout lay;
  const uint32_t* blob;
  uint32_t* table;
  unsigned long long* next_end;
  uint32_t* frontier;
  uint64_t fmask, cur_begin;
  int log2nb;
};

struct SmemTarget {
  const WarpNet* w;
  int nrounds;
  __device__ __forceinline__ uint32_t* table() const { return w->table; }
  __device__ __forceinline__ int log2nb() const { return w->log2nb; }
  __device__ __forceinline__ int rounds() const { return nrounds; }
  __device__ __forceinline__ unsigned long long* next_end() const { return w->next_end; }
  __device__ __forceinline__ uint32_t* frontier() const { return w->frontier; }
  __device__ __forceinline__ uint64_t fmask() const { return w->fmask; }
  __device__ __forceinline__ uint64_t begin() const { return w->cur_begin; }
  __device__ __forceinline__ uint64_t region_mask() const { return 0; }
  __device__ __forceinline__ uint64_t region_bits() const { return 0; }
  __device__ __forceinline__ unsigned long long* gcache() const { return nullptr; }
  __device__ __forceinline__ uint64_t gcache_mask() const { return 0; }
  __device__ __forceinline__ GKey gkey() const { return GKey{{64u, 64u, 64u}}; }
};

// The batched kernel keeps a network index and chunk bounds besides the
// single-network kernel's state: one CTA per SM fewer (at most 4) keeps its
// common instantiations free of spills; 4 and 5 measured the same time.
template <int W, int B, int G>
struct BatchOcc {
  static constexpr int min_ctas = ExpandOcc<W, B, G>::min_ctas < 4 ? ExpandOcc<W, B, G>::min_ctas : 4;
};

template <int W, int B, int G>
__global__ void __launch_bounds__(gx::kBlock, BatchOcc<W, B, G>::min_ctas) batch_expand_kernel(const BatchArgs a) {
  // a fixed full-size grid: CTAs beyond what this iteration's chunks need leave
  // before claiming (in the batch's long tail most iterations have few chunks)
  if ((unsigned long long)blockIdx.x * (gx::kBlock / 32) >= __ldcg(a.prefix + a.n)) return;
  __shared__ uint64_t muls[kMaxRounds];
  for (int i = threadIdx.x; i < a.rounds; i += blockDim.x) muls[i] = a.muls.m[i];
  __shared__ uint32_t stage_mem[gx::kBlock / 32][kStage * W];
  constexpr int CW = W <= 2 ? W : 1;
  __shared__ __align__(16) uint32_t cache_mem[gx::kBlock / 32][(1 << kBatchCacheLog2) * CW];
  __shared__ WarpNet s_net[gx::kBlock / 32];
  __syncthreads();
  WarpNet& wn = s_net[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const Group<G> g;
  WarpStage st{stage_mem[threadIdx.x >> 5], 0};
  WarpCache cache{W <= 2 ? cache_mem[threadIdx.x >> 5] : nullptr, (1u << kBatchCacheLog2) - 1u};
  int cached_net = -1;
  __shared__ unsigned long long s_chunk[gx::kBlock / 32][2];  // [first, end) of the warp's chunk
  unsigned long long* chunk_range = s_chunk[threadIdx.x >> 5];
  constexpr int K = PerLane<G>::K;
  const unsigned long long unit = __ldcg(a.unit);  // 1: one warp per state this iteration
  while (true) {
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(a.claim, 1ull);
    c = __shfl_sync(FULLMASK, c, 0);
    if (c >= __ldcg(a.prefix + a.n)) break;  // chunks of this iteration, all networks
    // the network whose chunks contain c: largest i with prefix[i] <= c
    int lo = 0, hi = a.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldcg(a.prefix + mid) <= c) lo = mid;
      else hi = mid - 1;
    }
    BNet& b = a.nets[lo];
    if (lo != cached_net) {  // stage the network; the cache holds one network's vectors at a time
      if (lane == 0) {
        wn.lay = b.lay;
        wn.blob = b.blob;
        wn.table = b.table;
        wn.next_end = &b.next_end;
        wn.frontier = b.frontier;
        wn.fmask = b.fmask;
        wn.cur_begin = b.cur_begin;
        wn.log2nb = b.log2nb;
      }
      if (W <= 2)
        for (uint32_t i = lane; i < (1u << kBatchCacheLog2) * CW; i += 32) cache_mem[threadIdx.x >> 5][i] = 0u;
      __syncwarp();
      cached_net = lo;
    }
    const uint32_t* t = wn.blob;
    const NetBlobLayout& L = wn.lay;
    const SmemTarget tg{&wn, a.rounds};
    if (lane == 0) {
      const uint64_t first = wn.cur_begin + (c - __ldcg(a.prefix + lo)) * unit;
      const uint64_t end = b.cur_end;
      chunk_range[0] = first;
      chunk_range[1] = first + unit < end ? first + unit : end;
    }
    __syncwarp();
    uint32_t trans = 0;  // per claim: below 2^32 (a state's successors are, and chunks stay far below)
    uint32_t probes = 0, err = 0;
    // Lane layout: one state per lane (unit > 1), or, in an iteration with few
    // states, one state per warp (unit == 1): every lane holds the state and
    // takes its successors l, l + 32, ... (found by index), so their
    // find-or-puts overlap instead of forming one lane's chain.
    static_assert(K == 1, "one successor per lane and round");
    const bool wide = unit == 1;
    for (uint64_t sub = chunk_range[0]; sub < chunk_range[1]; sub += 32) {
      const uint64_t idx = wide ? sub : sub + lane;
      const bool valid = idx < chunk_range[1];
      uint32_t v[W];
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = 0;
      if (valid) load_vec<W>(wn.frontier + (idx & wn.fmask) * W, v);
      const uint32_t cnt = valid ? count_succ<W>(t, L, v) : 0u;
      if (valid && (!wide || lane == 0)) {  // the lane that accounts for the state
        trans += cnt;
        if (cnt == 0) {
          const uint64_t h = state_digest<W>(t, L, v);
          atomicAdd(&b.dl_count, 1ull);
          atomicAdd(&b.dl_sum, (unsigned long long)h);
          atomicXor(&b.dl_xor, (unsigned long long)h);
        }
      }
      uint32_t remaining = !wide ? cnt : (cnt > (uint32_t)lane ? (cnt - lane + 31) / 32 : 0u);
      uint32_t kk = lane;  // wide: index of this lane's next successor
      SuccIter it;
      it.init();
      while (__any_sync(FULLMASK, remaining != 0)) {
        uint32_t s[K][W];
        bool has[K];
        has[0] = remaining != 0;
        if (has[0]) {
          if (wide) {
            seek_succ<W>(t, L, v, kk, s[0]);
            kk += 32;
          } else {
            next_succ<W>(it, t, L, v, s[0]);
          }
          --remaining;
        } else {
#pragma unroll
          for (int w = 0; w < W; ++w) s[0][w] = 0;
        }
        insert_lanes<W, B, G, K>(tg, muls, g, has, s, probes, err, st, cache);
      }
    }
    st.flush<W>(tg, err);
    const unsigned long long tr = warp_sum((unsigned long long)trans);
    const unsigned long long pr = warp_sum((unsigned long long)probes);
    err = __reduce_or_sync(FULLMASK, err);
    if (lane == 0) {
      if (tr) atomicAdd(&b.transitions, tr);
      if (pr) atomicAdd(&b.probes, pr);
      if (err) atomicOr(&b.error, err);
    }
  }
}

}  // namespace gxd

namespace gx {
namespace {

struct BatchKernels {
  const void* init;
  const void* expand;
};

template <int W, int B, int G>
BatchKernels batch_kernels() {
  return BatchKernels{reinterpret_cast<const void*>(&gxd::batch_init_kernel<W, B, G>),
                      reinterpret_cast<const void*>(&gxd::batch_expand_kernel<W, B, G>)};
}

// (B, G) pairs built for batches; the autotuner picks among them.
const int kCands[][2] = {{4, 1}, {8, 1}, {8, 2}, {16, 1}, {16, 2}, {32, 2}, {32, 4}};

bool lookup(int W, int B, int G, BatchKernels& out) {
#define GX_BK(w, b, g) \
  if (W == w && B == b && G == g) { out = batch_kernels<w, b, g>(); return true; }
  GX_BK(1, 4, 1) GX_BK(1, 8, 1) GX_BK(1, 8, 2) GX_BK(1, 16, 1) GX_BK(1, 16, 2) GX_BK(1, 32, 2) GX_BK(1, 32, 4)
  GX_BK(2, 4, 1) GX_BK(2, 8, 1) GX_BK(2, 8, 2) GX_BK(2, 16, 1) GX_BK(2, 16, 2) GX_BK(2, 32, 2) GX_BK(2, 32, 4)
  GX_BK(4, 4, 1) GX_BK(4, 8, 1) GX_BK(4, 8, 2) GX_BK(4, 16, 1) GX_BK(4, 16, 2) GX_BK(4, 32, 2) GX_BK(4, 32, 4)
#undef GX_BK
  return false;
}

#define GB_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return gx::fail(GX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }
inline uint64_t p2ceil(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p *= 2;
  return p;
}

struct BatchPlan {
  int W = 0, B = 0, G = 0, rounds = 0, chunk = 0;
  uint32_t levels_cap = 0, wide = 0;
  std::vector<uint64_t> slots, fcap;
  uint64_t off_nets = 0, off_prefix = 0, off_claim = 0, off_blobs = 0, off_levels = 0,
           off_fronts = 0, off_tables = 0, table_words = 0, total = 0;
  std::vector<uint64_t> blob_off, front_off, table_off;
  BatchKernels k{};
};

}  // namespace
}  // namespace gx

struct gx_batch {
  std::vector<gx::Net> nets;
  uint32_t W = 0;  // widest slot of the batch; narrower networks are padded to it
  // results of the last run
  bool have_result = false;
  std::vector<gx::BNet> res;
  std::vector<std::vector<uint64_t>> levels;
  double gpu_ms = 0;
  // cached graph
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  void* exec_ws = nullptr;
  std::vector<uint64_t> exec_key;
  std::vector<uint64_t> last_plan_slots;
  uint32_t last_W = 0, last_B = 0, last_G = 0, last_rounds = 0;
  ~gx_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

namespace gx {
namespace {

gx_status batch_plan(const gx_batch* h, const gx_batch_opts* o, BatchPlan& P) {
  gx_batch_opts d{};
  if (!o) o = &d;
  const uint32_t n = (uint32_t)h->nets.size();
  P.W = (int)h->W;
  P.B = o->bucket_words ? (int)o->bucket_words : 8;
  P.G = o->group_lanes ? (int)o->group_lanes : 1;
  P.rounds = o->hash_rounds ? (int)o->hash_rounds : 8;
  P.chunk = o->chunk_states ? (int)o->chunk_states : 32;
  if (P.rounds < 1 || P.rounds > kMaxRounds) return fail(GX_ERR_INVALID, "hash_rounds must be 1..64");
  if (P.chunk < 32 || P.chunk % 32 || P.chunk > 4096)
    return fail(GX_ERR_INVALID, "chunk_states must be a multiple of 32 in 32..4096");
  if (!lookup(P.W, P.B, P.G, P.k))
    return fail(GX_ERR_INVALID, "no batch kernel for bucket_words " + std::to_string(P.B) + ", group_lanes " +
                                    std::to_string(P.G) + " with " + std::to_string(P.W) + "-word slots");
  P.levels_cap = o->levels_cap ? o->levels_cap : 4096;
  P.wide = o->wide_factor ? o->wide_factor : 4u;
  P.slots.resize(n);
  P.fcap.resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    uint64_t s = o->expected_states ? p2ceil(std::max<uint64_t>(1024, (o->expected_states[i] * 4 + 2) / 3))
                                    : (o->table_slots ? p2ceil(o->table_slots) : (1ull << 20));
    const uint64_t min_slots = std::max<uint64_t>(1024, 2ull * P.B / P.W);
    P.slots[i] = std::max(s, min_slots);
    // with expected sizes the ring holds a whole network (slots >= 4/3 of its states), so two
    // consecutive levels always fit; otherwise half the table
    P.fcap[i] = std::max<uint64_t>(4096, o->expected_states ? P.slots[i] : P.slots[i] / 2);
  }
  uint64_t off = 0;
  P.off_nets = off;
  off = a256(off + sizeof(BNet) * n);
  P.off_prefix = off;
  off = a256(off + 8ull * (n + 1));
  P.off_claim = off;
  off = a256(off + 24);  // claim counter, iteration counter, states per claim
  P.off_blobs = off;
  P.blob_off.resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    P.blob_off[i] = off;
    off = a256(off + 4ull * h->nets[i].blob.size());
  }
  P.off_levels = off;
  off = a256(off + 8ull * P.levels_cap * n);
  P.off_fronts = off;
  P.front_off.resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    P.front_off[i] = off;
    off = a256(off + 4ull * P.W * P.fcap[i]);
  }
  P.off_tables = off;
  P.table_off.resize(n);
  for (uint32_t i = 0; i < n; ++i) {
    P.table_off[i] = off;
    off += 4ull * P.W * P.slots[i];  // power-of-two sizes of at least 4 KiB: stays aligned
  }
  P.table_words = (off - P.off_tables) / 4;
  P.total = a256(off);
  return GX_OK;
}

gx_status build_graph(gx_batch* h, const BatchPlan& P, void* ws, int sms) {
  if (h->exec) {
    cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
  }
  if (h->graph) {
    cudaGraphDestroy(h->graph);
    h->graph = nullptr;
  }
  char* base = static_cast<char*>(ws);
  const int n = (int)h->nets.size();
  cudaGraph_t g;
  GB_CUDA(cudaGraphCreate(&g, 0));
  h->graph = g;
  cudaGraphConditionalHandle cond;
  GB_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));

  int per_sm = 0;
  GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.k.expand, kBlock, 0));
  const int grid = sms * std::max(per_sm, 1);

  BatchArgs a{};
  a.nets = reinterpret_cast<BNet*>(base + P.off_nets);
  a.n = n;
  a.rounds = P.rounds;
  a.chunk = P.chunk;
  hash_multipliers(a.muls.m, kMaxRounds);
  a.prefix = reinterpret_cast<unsigned long long*>(base + P.off_prefix);
  a.claim = reinterpret_cast<unsigned long long*>(base + P.off_claim);
  a.iters = a.claim + 1;
  a.unit = a.claim + 2;
  a.wide_states = P.wide == GX_BATCH_WIDE_OFF ? 0ull : (unsigned long long)P.wide * grid * (kBlock / 32);
  a.max_iters = (unsigned long long)P.levels_cap + 1;
  a.cond = cond;

  // memset of every table
  cudaGraphNode_t mset;
  cudaMemsetParams mp{};
  mp.dst = base + P.off_tables;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = P.table_words;
  mp.height = 1;
  mp.pitch = 0;
  GB_CUDA(cudaGraphAddMemsetNode(&mset, g, nullptr, 0, &mp));

  auto add_kernel = [&](cudaGraph_t gr, const cudaGraphNode_t* deps, size_t nd, const void* fn,
                        dim3 grid, dim3 block, void** args, cudaGraphNode_t* out) -> cudaError_t {
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, gr, deps, nd, &kp);
  };
  void* args_a[] = {&a};
  int first1 = 1, first0 = 0;
  void* args_adv1[] = {&a, &first1};
  void* args_adv0[] = {&a, &first0};

  cudaGraphNode_t init, adv1;
  const int per_block = kBlock / 32;
  GB_CUDA(add_kernel(g, &mset, 1, P.k.init, dim3((n + per_block - 1) / per_block), dim3(kBlock), args_a, &init));
  GB_CUDA(add_kernel(g, &init, 1, reinterpret_cast<const void*>(&gxd::batch_advance_kernel), dim3(1),
                     dim3(1024), args_adv1, &adv1));

  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  GB_CUDA(cudaGraphAddNode(&cnode, g, &adv1, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];

  cudaGraphNode_t ex, adv0;
  GB_CUDA(add_kernel(body, nullptr, 0, P.k.expand, dim3(grid), dim3(kBlock), args_a, &ex));
  GB_CUDA(add_kernel(body, &ex, 1, reinterpret_cast<const void*>(&gxd::batch_advance_kernel), dim3(1),
                     dim3(1024), args_adv0, &adv0));
  cudaGraphExec_t exec;
  GB_CUDA(cudaGraphInstantiate(&exec, g, 0));
  h->exec = exec;
  h->exec_ws = ws;
  return GX_OK;
}

gx_status run_batch(gx_batch* h, const gx_batch_opts* o, void* ws, uint64_t ws_bytes, cudaStream_t st) {
  BatchPlan P;
  gx_status s = batch_plan(h, o, P);
  if (s != GX_OK) return s;
  if (!ws) return fail(GX_ERR_INVALID, "batched exploration needs a workspace (gx_batch_workspace_bytes)");
  if (ws_bytes < P.total)
    return fail(GX_ERR_OOM, "workspace holds " + std::to_string(ws_bytes) + " bytes, need " + std::to_string(P.total));
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(GX_ERR_INVALID, "workspace is not 256-byte aligned");
  const int n = (int)h->nets.size();
  int dev = 0, sms = 0;
  GB_CUDA(cudaGetDevice(&dev));
  GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  char* base = static_cast<char*>(ws);

  // descriptors and tables
  std::vector<BNet> bn(n);
  for (int i = 0; i < n; ++i) {
    const Net& net = h->nets[i];
    BNet& b = bn[i];
    std::memset(&b, 0, sizeof(b));
    b.blob = reinterpret_cast<const uint32_t*>(base + P.blob_off[i]);
    b.lay = net.lay;
    b.table = reinterpret_cast<uint32_t*>(base + P.table_off[i]);
    uint64_t nb = P.slots[i] * P.W / P.B;
    int l = 0;
    while ((1ull << l) < nb) ++l;
    b.log2nb = l;
    b.levels_cap = P.levels_cap;
    b.frontier = reinterpret_cast<uint32_t*>(base + P.front_off[i]);
    b.fmask = P.fcap[i] - 1;
    b.levels = reinterpret_cast<unsigned long long*>(base + P.off_levels) + (uint64_t)i * P.levels_cap;
    // the initial vector, padded to the batch's slot width (padding words carry only the tag)
    for (int w = 0; w < 4; ++w) b.init_vec[w] = w < P.W ? (net.init_vec[w] | kTag) : 0u;
    GB_CUDA(cudaMemcpyAsync(base + P.blob_off[i], net.blob.data(), 4 * net.blob.size(), cudaMemcpyHostToDevice, st));
  }
  GB_CUDA(cudaMemcpyAsync(base + P.off_nets, bn.data(), sizeof(BNet) * n, cudaMemcpyHostToDevice, st));

  // everything the graph holds by value: kernels, launch shapes, and where the
  // tables it clears start and end (they move when per-network sizes change)
  std::vector<uint64_t> key{(uint64_t)P.B, (uint64_t)P.G, (uint64_t)P.rounds, (uint64_t)P.chunk,
                            P.levels_cap, P.total, P.off_tables, P.table_words, P.wide};
  if (!h->exec || h->exec_ws != ws || h->exec_key != key) {
    s = build_graph(h, P, ws, sms);
    if (s != GX_OK) return s;
    h->exec_key = key;
  }
  cudaEvent_t e0, e1;
  GB_CUDA(cudaEventCreate(&e0));
  GB_CUDA(cudaEventCreate(&e1));
  GB_CUDA(cudaEventRecord(e0, st));
  GB_CUDA(cudaGraphLaunch(h->exec, st));
  GB_CUDA(cudaEventRecord(e1, st));
  h->res.resize(n);
  GB_CUDA(cudaMemcpyAsync(h->res.data(), base + P.off_nets, sizeof(BNet) * n, cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaStreamSynchronize(st));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->gpu_ms = ms;
  std::vector<unsigned long long> lv((uint64_t)n * P.levels_cap);
  GB_CUDA(cudaMemcpyAsync(lv.data(), base + P.off_levels, 8ull * lv.size(), cudaMemcpyDeviceToHost, st));
  GB_CUDA(cudaStreamSynchronize(st));
  h->levels.assign(n, {});
  gx_status rs = GX_OK;
  for (int i = 0; i < n; ++i) {
    const uint32_t k = std::min<uint32_t>(h->res[i].n_levels, P.levels_cap);
    h->levels[i].assign(lv.begin() + (uint64_t)i * P.levels_cap, lv.begin() + (uint64_t)i * P.levels_cap + k);
    if (h->res[i].error && rs == GX_OK) {
      const unsigned e = h->res[i].error;
      rs = (e & ERR_TABLE_FULL)  ? fail(GX_ERR_TABLE_FULL, "network " + std::to_string(i) + ": hash table full")
         : (e & ERR_FRONTIER)    ? fail(GX_ERR_FRONTIER_OVERFLOW, "network " + std::to_string(i) + ": frontier overflow")
         : (e & ERR_LEVELS)      ? fail(GX_ERR_OOM, "network " + std::to_string(i) + ": more levels than levels_cap")
                                 : fail(GX_ERR_SPIN_LIMIT, "network " + std::to_string(i) + ": device wait gave up");
    }
  }
  h->have_result = true;
  h->last_plan_slots = P.slots;
  h->last_W = (uint32_t)P.W;
  h->last_B = (uint32_t)P.B;
  h->last_G = (uint32_t)P.G;
  h->last_rounds = (uint32_t)P.rounds;
  return rs;
}

}  // namespace
}  // namespace gx

extern "C" {

gx_status gx_batch_create(const gx_net* const* nets, uint32_t n, gx_batch** out) {
  gx::clear_error();
  if (!nets || !out || n == 0) return gx::fail(GX_ERR_INVALID, "nets, n or out is invalid");
  gx_batch* h = new gx_batch();
  for (uint32_t i = 0; i < n; ++i) {
    if (!nets[i]) {
      delete h;
      return gx::fail(GX_ERR_INVALID, "nets[" + std::to_string(i) + "] is NULL");
    }
    h->nets.push_back(nets[i]->net);
    h->W = std::max(h->W, nets[i]->net.slot_words);
  }
  *out = h;
  return GX_OK;
}

void gx_batch_free(gx_batch* b) { delete b; }

gx_status gx_batch_workspace_bytes(const gx_batch* b, const gx_batch_opts* opts, uint64_t* bytes) {
  gx::clear_error();
  if (!b || !bytes) return gx::fail(GX_ERR_INVALID, "batch or bytes is NULL");
  gx::BatchPlan P;
  gx_status s = gx::batch_plan(b, opts, P);
  if (s != GX_OK) return s;
  *bytes = P.total;
  return GX_OK;
}

gx_status gx_batch_explore(gx_batch* b, const gx_batch_opts* opts, void* ws, uint64_t ws_bytes, void* stream) {
  gx::clear_error();
  if (!b) return gx::fail(GX_ERR_INVALID, "batch is NULL");
  return gx::run_batch(b, opts, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

gx_status gx_batch_stats(const gx_batch* b, uint32_t i, gx_stats_t* out) {
  gx::clear_error();
  if (!b || !out) return gx::fail(GX_ERR_INVALID, "batch or out is NULL");
  if (!b->have_result) return gx::fail(GX_ERR_STATE, "no batched exploration has run");
  if (i >= b->res.size()) return gx::fail(GX_ERR_INVALID, "network index out of range");
  const gx::BNet& r = b->res[i];
  std::memset(out, 0, sizeof(*out));
  out->states = r.next_end;
  out->explored = r.cur_end;  // end of the last level that was expanded
  out->transitions = r.transitions;
  out->n_levels = r.n_levels;
  out->deadlock_count = r.dl_count;
  out->deadlock_sum = r.dl_sum;
  out->deadlock_xor = r.dl_xor;
  out->first_deadlock_level = r.first_dl;
  out->table_slots = b->last_plan_slots[i];
  out->vector_words = b->nets[i].vector_words;
  out->slot_words = b->last_W;
  out->bucket_words = b->last_B;
  out->group_lanes = b->last_G;
  out->hash_rounds = b->last_rounds;
  out->complete = (!r.active && !r.error) ? 1u : 0u;
  out->status = r.error ? 1u : 0u;
  out->fill = (double)r.next_end / (double)out->table_slots;
  out->gpu_ms = b->gpu_ms;
  out->probes = r.probes;
  return GX_OK;
}

gx_status gx_batch_levels(const gx_batch* b, uint32_t i, uint64_t* out, uint32_t cap, uint32_t* n) {
  gx::clear_error();
  if (!b) return gx::fail(GX_ERR_INVALID, "batch is NULL");
  if (!b->have_result) return gx::fail(GX_ERR_STATE, "no batched exploration has run");
  if (i >= b->levels.size()) return gx::fail(GX_ERR_INVALID, "network index out of range");
  if (cap && !out) return gx::fail(GX_ERR_INVALID, "out is NULL");
  const auto& L = b->levels[i];
  for (size_t k = 0; k < L.size() && k < cap; ++k) out[k] = L[k];
  if (n) *n = (uint32_t)L.size();
  return GX_OK;
}

gx_status gx_batch_autotune(gx_batch* b, gx_batch_opts* io, void* ws, uint64_t ws_bytes, void* stream,
                            double* best_ms) {
  gx::clear_error();
  if (!b || !io) return gx::fail(GX_ERR_INVALID, "batch or opts is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t chunks[] = {32, 64, 128};
  gx_batch_opts best = *io;
  double best_t = 1e30;
  for (const auto& c : gx::kCands) {
    if (c[0] < (int)b->W) continue;
    for (uint32_t ch : chunks) {
      gx_batch_opts o = *io;
      o.bucket_words = (uint32_t)c[0];
      o.group_lanes = (uint32_t)c[1];
      o.chunk_states = ch;
      gx::BatchPlan P;
      if (gx::batch_plan(b, &o, P) != GX_OK || P.total > ws_bytes) continue;
      // one warm-up (graph build), then the median of three timed runs
      gx_status s = gx::run_batch(b, &o, ws, ws_bytes, st);
      if (s != GX_OK) continue;
      double t[3];
      for (double& x : t) {
        if (gx::run_batch(b, &o, ws, ws_bytes, st) != GX_OK) x = 1e30;
        else x = b->gpu_ms;
      }
      std::sort(t, t + 3);
      if (t[1] < best_t) {
        best_t = t[1];
        best = o;
      }
    }
  }
  gx::clear_error();
  if (best_t >= 1e30) return gx::fail(GX_ERR_INVALID, "no candidate configuration ran");
  *io = best;
  if (best_ms) *best_ms = best_t;
  return GX_OK;
}

}  // extern "C"

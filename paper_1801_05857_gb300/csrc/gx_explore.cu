// The level loop and the C ABI of the exploration path.
//
// One search (Sec. 3): clear the table, insert the initial vector (level 0),
// then per level launch one persistent expansion kernel over the open
// vectors of that level.  By default the levels run on the device: one CUDA
// graph whose conditional WHILE node repeats {expand, advance}, where the
// one-thread advance step records the level, moves the level range on and
// decides whether to go on, so the host waits once per search.  With
// host_loop (and on the partitioned path) the host reads the control block
// between levels instead ("only the general progress is checked on the host
// side", Sec. 3).
//
// Workspace (one device buffer, 256-byte aligned regions):
//   control block | network blob | deadlock buffer |
//   frontier ring | hash table
// The frontier is a ring of vectors indexed by absolute position: the level
// being expanded occupies [cur_begin, cur_end) and its successors are
// appended from cur_end on; the ring overflows when a level and its
// successor level together exceed its capacity.  This replaces the paper's
// scan of the hash table for open vectors (Sec. 4: the table keeps the open
// and closed sets) -- a per-level table scan would read the whole table once
// per level.

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "gx_kernels.cuh"

namespace gx {

void hash_multipliers(uint64_t* out, int n) {
  // splitmix64 stream from a fixed seed; forcing the low bit makes each odd
  uint64_t s = 0x243F6A8885A308D3ull;  // digits of pi
  for (int i = 0; i < n; ++i) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    out[i] = (z ^ (z >> 31)) | 1ull;
  }
}

}  // namespace gx

namespace gx {

// The device-driven level loop (see run_search).
struct LoopArgs {
  Ctl* ctl;
  unsigned long long* lv_size;    // [cap] level sizes (level 0 = 1)
  unsigned long long* lv_tns;     // [cap] per expanded level: device time in ns (%globaltimer)
  unsigned long long* lv_probes;  // [cap] cumulative bucket reads after the level
  unsigned long long* lv_trans;   // [cap] cumulative transitions after the level
  uint32_t cap;
  int stop_dl, stop_viol;
  uint64_t max_levels;            // 0 = no limit
  cudaGraphConditionalHandle cond;
};

constexpr uint32_t kLoopLevels = 4096;  // levels the device loop records before the host takes over

}  // namespace gx

namespace gxd {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Level 0 = {initial state}; start the loop unless the insertion failed.
__global__ void loop_start_kernel(const gx::LoopArgs L) {
  gx::Ctl& c = *L.ctl;
  c.cur_begin = 0;
  c.cur_end = 1;
  c.n_levels = 1;
  c.levels_done = 0;
  c.explored = 0;
  c.first_dl = -1;
  c.first_viol = -1;
  c.complete = 0;
  c.yielded = 0;
  c.claim = 0;
  L.lv_size[0] = 1;
  c.t_prev = global_ns();
  cudaGraphSetConditional(L.cond, c.error ? 0u : 1u);
}

// After the expansion of level [cur_begin, cur_end): the host loop's
// bookkeeping, done on the device.
__global__ void level_advance_kernel(const gx::LoopArgs L) {
  gx::Ctl& c = *L.ctl;
  const unsigned long long k = c.levels_done;
  const unsigned long long t = global_ns();
  if (k < L.cap) {
    L.lv_tns[k] = t - c.t_prev;
    L.lv_probes[k] = c.probes;
    L.lv_trans[k] = c.transitions;
  }
  c.t_prev = t;
  c.levels_done = k + 1;
  c.explored += c.cur_end - c.cur_begin;
  if (c.first_dl < 0 && c.dl_count > 0) c.first_dl = (long long)c.n_levels - 1;
  if (c.first_viol < 0 && c.viol_count > 0) c.first_viol = (long long)c.n_levels - 1;
  const unsigned long long next_end = c.next_end;
  if (next_end > c.cur_end) {
    if (c.n_levels < L.cap) L.lv_size[c.n_levels] = next_end - c.cur_end;
    c.n_levels += 1;
  }
  bool more = true;
  if (c.error) {
    more = false;
  } else if (next_end == c.cur_end) {
    c.complete = 1;
    more = false;
  } else {
    c.cur_begin = c.cur_end;
    c.cur_end = next_end;
    c.claim = 0;
    if ((L.stop_dl && c.dl_count > 0) || (L.stop_viol && c.viol_count > 0) ||
        (L.max_levels && c.levels_done >= L.max_levels)) {
      more = false;
    } else if (c.n_levels >= L.cap) {  // arrays full: the host loop continues from here
      c.yielded = 1;
      more = false;
    }
  }
  cudaGraphSetConditional(L.cond, more ? 1u : 0u);
}

template <int W>
__global__ void __launch_bounds__(gx::kBlock) digest_kernel(const gx::DigestArgs a) {
  unsigned long long cnt = 0, sum = 0, xr = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.slots; i += stride) {
    uint32_t v[W];
    load_vec<W>(a.table + i * W, v);
    bool tagged = true;
#pragma unroll
    for (int w = 0; w < W; ++w) tagged &= (v[w] & kTag) != 0;
    if (!tagged) continue;
    const uint64_t h = state_digest<W>(a.blob, a.lay, v);
    cnt += 1;
    sum += h;
    xr ^= h;
  }
  cnt = warp_sum(cnt);
  sum = warp_sum(sum);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) xr ^= __shfl_xor_sync(FULLMASK, xr, o);
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicAdd(&a.out[0], cnt);
    atomicAdd(&a.out[1], sum);
    atomicXor(&a.out[2], xr);
  }
}

}  // namespace gxd

namespace gx {

cudaError_t launch_digest(int W, const DigestArgs& a, int grid, cudaStream_t st) {
  if (W == 1) gxd::digest_kernel<1><<<grid, kBlock, 0, st>>>(a);
  else if (W == 2) gxd::digest_kernel<2><<<grid, kBlock, 0, st>>>(a);
  else gxd::digest_kernel<4><<<grid, kBlock, 0, st>>>(a);
  return cudaGetLastError();
}

namespace {

constexpr uint64_t kAlign = 256;
inline uint64_t align_up(uint64_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
inline uint64_t pow2_floor(uint64_t x) {
  uint64_t p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}
inline uint64_t pow2_ceil(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p *= 2;
  return p;
}
inline int ilog2(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

#define GX_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return gx::fail(GX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

constexpr int kPartCtas = 1024;  // CTAs of the partitioned count/scatter passes (at most)
// Largest table region one pass of the direct path probes by default: random
// 32-byte reads run at the full rate over any 64 GiB of a table and 4x slower
// over 128 GiB (the GPU's address-translation reach); the later hash rounds of
// a vector stay inside the same 64 GiB span as its first (bucket_in_span).
constexpr uint64_t kAutoRegionBytes = 1ull << gxd::kSpanLog2Bytes;
constexpr uint32_t kAutoCache = 0xFFFFFFFFu;  // warp_cache_log2 / global_cache_log2: automatic

// Arguments of pass q of `passes` region passes over a table of 2^log2nb buckets.
inline ExpandArgs region_pass(const ExpandArgs& a, uint32_t passes, uint32_t q) {
  ExpandArgs r = a;
  int lp = 0;
  while ((1u << lp) < passes) ++lp;
  const int shift = a.log2nb - lp;
  r.region_mask = passes > 1 ? (uint64_t)(passes - 1) << shift : 0ull;
  r.region_bits = (uint64_t)q << shift;
  r.count_states = q == 0 ? 1 : 0;
  return r;
}

struct Plan {
  int W = 0, B = 0, G = 0, rounds = 0;
  uint32_t dl_cap = 0;
  uint32_t viol_cap = 0;   // violating states kept (safety check)
  uint64_t nb = 0;         // buckets (power of two)
  uint64_t fcap = 0;       // frontier ring capacity (power of two)
  int logp = 0;            // table slices for the partitioned path (0 = path off)
  uint64_t cs = 0;         // successor buffer capacity (vectors)
  uint64_t part_min = 0;   // smallest level that may use the partitioned path
  uint32_t regions = 1;    // passes per level of the direct path (region passes)
  uint64_t gcache = 0;     // entries of the GPU-wide cache of seen vectors (0 = off)
  uint32_t gkey[3] = {64, 64, 64};  // key offsets of words 1..3 (4-word vectors)
  uint32_t warp_log2 = 0;  // per-warp cache of seen vectors: 2^warp_log2 entries (0 = off)
  uint64_t off_ctl = 0, off_blob = 0, off_dl = 0, off_viol = 0, off_loop = 0, off_front = 0, off_table = 0;
  uint64_t off_hist = 0, off_off = 0, off_ptot = 0, off_tot = 0, off_succ = 0, off_gcache = 0;
  uint64_t total = 0;
  const KernelSet* ks = nullptr;
  // the level kernel: ks->expand, or the queued second kernel with region passes
  cudaError_t (*expand)(const ExpandArgs&, int, size_t, cudaStream_t) = nullptr;
  const void* expand_fn = nullptr;
};

gx_status make_plan(const Net& net, const gx_explore_opts* o, Plan& P) {
  gx_explore_opts d;
  gx_default_opts(&d);
  if (!o) o = &d;
  P.W = (int)net.slot_words;
  P.B = o->bucket_words ? (int)o->bucket_words : 8;
  if (P.B != 4 && P.B != 8 && P.B != 16 && P.B != 32)
    return fail(GX_ERR_INVALID, "bucket_words must be 4, 8, 16 or 32");
  if (P.B < P.W)
    return fail(GX_ERR_INVALID, "bucket_words " + std::to_string(P.B) + " is smaller than the " +
                                    std::to_string(P.W) + "-word slots of this network");
  const int S = P.B / P.W;
  P.G = o->group_lanes ? (int)o->group_lanes : std::min(S, 32);
  if (P.G < 1 || (P.G & (P.G - 1)) || P.G > S || P.G > 32)
    return fail(GX_ERR_INVALID, "group_lanes must be a power of two between 1 and bucket_words / slot words (" +
                                    std::to_string(S) + ")");
  P.rounds = o->hash_rounds ? (int)o->hash_rounds : 8;
  if (P.rounds < 1 || P.rounds > kMaxRounds) return fail(GX_ERR_INVALID, "hash_rounds must be 1..64");
  P.ks = kernels_for(P.W, P.B, P.G);
  if (!P.ks) return fail(GX_ERR_INVALID, "no kernel built for this (slot, bucket, group) size");
  const uint64_t table_bytes = o->table_bytes ? o->table_bytes : (1ull << 30);
  const uint64_t bucket_bytes = 4ull * P.B;
  if (table_bytes < 2 * bucket_bytes) return fail(GX_ERR_INVALID, "table_bytes is smaller than two buckets");
  P.nb = pow2_floor(table_bytes / bucket_bytes);
  const uint64_t slots = P.nb * (uint64_t)S;
  P.fcap = pow2_ceil(o->frontier_states ? o->frontier_states : std::max<uint64_t>(4096, slots / 4));
  P.dl_cap = o->deadlock_cap ? o->deadlock_cap : 1024;
  if (o->watch) {
    if (o->watch_proc >= net.n_procs) return fail(GX_ERR_INVALID, "watch_proc is not a process of the network");
    if (o->watch_state >= net.n_states[o->watch_proc])
      return fail(GX_ERR_INVALID, "watch_state is not a local state of watch_proc");
    P.viol_cap = o->violation_cap ? o->violation_cap : 1024;
  }
  // partitioned path: slices of about 32 MiB, at most 4096 of them
  const uint64_t tbytes = 4ull * P.B * P.nb;
  if (o->slice_log2) {
    if (o->slice_log2 > 12) return fail(GX_ERR_INVALID, "slice_log2 must be at most 12");
    P.logp = (int)o->slice_log2;
  } else {
    P.logp = 0;
    while (P.logp < 12 && (tbytes >> (P.logp + 1)) >= (32ull << 20)) ++P.logp;
  }
  if ((1ull << P.logp) > P.nb) P.logp = ilog2(P.nb);
  P.part_min = o->partition_min_states;
  if (P.part_min == 0) P.logp = 0;  // path off
  // region passes: explicit, or the fewest passes whose table regions fit the
  // GPU's address-translation reach for random accesses (64 GiB measured)
  if (o->region_passes) {
    const uint32_t r = o->region_passes;
    if (r > 16 || (r & (r - 1))) return fail(GX_ERR_INVALID, "region_passes must be a power of two from 1 to 16");
    P.regions = r;
  } else {
    P.regions = 1;
    while (P.regions < 16 && tbytes / P.regions > kAutoRegionBytes) P.regions *= 2;
  }
  if (P.regions > P.nb) P.regions = (uint32_t)P.nb;
  // with region passes most generated successors fall outside the pass's region:
  // the queued kernel (where it is a second one) probes only those inside it, 32 at a time
  const bool queued = P.regions > 1 && P.ks->expand_queued;
  P.expand = queued ? P.ks->expand_queued : P.ks->expand;
  P.expand_fn = queued ? P.ks->expand_queued_fn : P.ks->expand_fn;
  // the caches of seen vectors: auto = the GPU-wide one (2^23 entries) for 1- and
  // 2-word vectors in tables of at least 2^26 slots with one lane per bucket (where it
  // was measured), else the per-warp one (2^9)
  // (4-word vectors use it only when their fields fit one 64-bit key)
  const bool key_fits = P.W <= 2 || gx::cache_key_shifts(net, P.gkey);
  if (o->global_cache_log2 == kAutoCache) {
    if (P.W <= 2 && P.G == 1 && slots >= (1ull << 26)) P.gcache = 1ull << 23;
  } else if (o->global_cache_log2) {
    if (o->global_cache_log2 > 26) return fail(GX_ERR_INVALID, "global_cache_log2 must be at most 26");
    if (key_fits) P.gcache = 1ull << o->global_cache_log2;
  }
  // (the queued 4-word kernel: 2^6, whose 4 KiB per CTA leave room for 5 CTAs per SM;
  // 2^9 took 4.55 s on the memory-scaled network, 2^6 3.52 s)
  P.warp_log2 = o->warp_cache_log2 == kAutoCache ? (P.gcache ? 0u : queued ? 6u : 9u) : o->warp_cache_log2;
  P.cs = o->successor_buffer ? o->successor_buffer : std::min<uint64_t>(slots / 2, (1ull << 32) - 1);
  if (P.logp == 0) P.cs = 0;  // partitioned path off: no buffer
  if (P.cs >= (1ull << 32)) return fail(GX_ERR_INVALID, "successor_buffer must be below 2^32 vectors");
  uint64_t off = 0;
  P.off_ctl = off;
  off = align_up(off + sizeof(Ctl));
  P.off_blob = off;
  off = align_up(off + 4ull * net.blob.size());
  P.off_dl = off;
  off = align_up(off + 4ull * P.W * P.dl_cap);
  P.off_viol = off;
  off = align_up(off + 4ull * P.W * P.viol_cap);
  P.off_loop = off;
  off = align_up(off + 4ull * 8ull * kLoopLevels);
  P.off_front = off;
  off = align_up(off + 4ull * P.W * P.fcap);
  P.off_table = off;
  off = align_up(off + 4ull * P.B * P.nb);
  const uint64_t np = P.logp ? (1ull << P.logp) : 0;
  P.off_hist = off;
  off = align_up(off + 4ull * kPartCtas * np);
  P.off_off = off;
  off = align_up(off + 4ull * kPartCtas * np);
  P.off_ptot = off;
  off = align_up(off + 4ull * np);
  P.off_tot = off;
  off = align_up(off + (np ? 4ull * kPartCtas : 0));
  P.off_succ = off;
  off = align_up(off + 4ull * P.W * P.cs);
  P.off_gcache = off;
  off = align_up(off + 8ull * P.gcache);
  P.total = off;
  return GX_OK;
}

struct Device {
  int sms = 0;
  size_t smem_optin = 0;
};

gx_status device_info(Device& d) {
  int dev = 0;
  GX_CUDA(cudaGetDevice(&dev));
  GX_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
  int so = 0;
  GX_CUDA(cudaDeviceGetAttribute(&so, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  d.smem_optin = (size_t)so;
  return GX_OK;
}

// Pinned host copies of the control block and of the per-CTA successor
// totals of the partitioned path, one set per thread.
struct HostCtl {
  Ctl* p = nullptr;
  uint32_t* tot = nullptr;
  ~HostCtl() {
    if (p) cudaFreeHost(p);
    if (tot) cudaFreeHost(tot);
  }
};
thread_local HostCtl g_hctl;

gx_status host_ctl(Ctl*& out, uint32_t*& tot) {
  if (!g_hctl.p) GX_CUDA(cudaMallocHost(reinterpret_cast<void**>(&g_hctl.p), sizeof(Ctl)));
  if (!g_hctl.tot) GX_CUDA(cudaMallocHost(reinterpret_cast<void**>(&g_hctl.tot), 4ull * kPartCtas));
  out = g_hctl.p;
  tot = g_hctl.tot;
  return GX_OK;
}

void release_loop(gx_net* h) {
  if (h->loop_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(h->loop_exec));
  if (h->loop_graph) cudaGraphDestroy(static_cast<cudaGraph_t>(h->loop_graph));
  h->loop_exec = nullptr;
  h->loop_graph = nullptr;
  h->loop_key.clear();
}

// The device-driven search as one graph: clear the control block and the
// table, insert the initial vector, start, then WHILE(cond) {expand; advance}.
gx_status build_loop_graph(gx_net* h, const Plan& P, Ctl* ctl, uint32_t* table, const InitArgs& ia,
                           const ExpandArgs& eg, LoopArgs la, size_t smem, uint64_t grid) {
  release_loop(h);
  h->release = &release_loop;
  cudaGraph_t g;
  GX_CUDA(cudaGraphCreate(&g, 0));
  h->loop_graph = g;
  cudaGraphConditionalHandle cond;
  GX_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
  la.cond = cond;
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
  GX_CUDA(add_memset(ctl, sizeof(Ctl) / 4));
  const uint64_t words = (uint64_t)P.B * P.nb;
  constexpr uint64_t kPiece = 1ull << 30;  // words per memset node
  for (uint64_t w0 = 0; w0 < words; w0 += kPiece) GX_CUDA(add_memset(table + w0, std::min(kPiece, words - w0)));
  if (eg.gcache) GX_CUDA(add_memset(eg.gcache, 2 * P.gcache));
  auto add_kernel = [&](cudaGraph_t gr, const cudaGraphNode_t* deps, size_t nd, const void* fn, dim3 gd, dim3 bd,
                        size_t sh, void** args, cudaGraphNode_t* out) -> cudaError_t {
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = gd;
    kp.blockDim = bd;
    kp.sharedMemBytes = (unsigned)sh;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, gr, deps, nd, &kp);
  };
  InitArgs ia_c = ia;
  ExpandArgs eg_c = region_pass(eg, P.regions, 0);
  void* args_i[] = {&ia_c};
  void* args_l[] = {&la};
  void* args_e[] = {&eg_c};
  cudaGraphNode_t init, start, ex, adv;
  GX_CUDA(add_kernel(g, clears.data(), clears.size(), P.ks->init_fn, dim3(1), dim3(32), 0, args_i, &init));
  GX_CUDA(add_kernel(g, &init, 1, reinterpret_cast<const void*>(&gxd::loop_start_kernel), dim3(1), dim3(1), 0,
                     args_l, &start));
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  GX_CUDA(cudaGraphAddNode(&cnode, g, &start, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  GX_CUDA(add_kernel(body, nullptr, 0, P.expand_fn, dim3((unsigned)grid), dim3(kBlock), smem, args_e, &ex));
  // region passes after the first: clear the claim counter, expand again
  for (uint32_t q = 1; q < P.regions; ++q) {
    ExpandArgs eq = region_pass(eg, P.regions, q);
    void* args_q[] = {&eq};
    cudaMemsetParams mp{};
    mp.dst = &ctl->claim;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = sizeof(ctl->claim) / 4;
    mp.height = 1;
    cudaGraphNode_t mz, exq;
    GX_CUDA(cudaGraphAddMemsetNode(&mz, body, &ex, 1, &mp));
    GX_CUDA(add_kernel(body, &mz, 1, P.expand_fn, dim3((unsigned)grid), dim3(kBlock), smem, args_q, &exq));
    ex = exq;
  }
  GX_CUDA(add_kernel(body, &ex, 1, reinterpret_cast<const void*>(&gxd::level_advance_kernel), dim3(1), dim3(1), 0,
                     args_l, &adv));
  cudaGraphExec_t exec;
  GX_CUDA(cudaGraphInstantiate(&exec, g, 0));
  h->loop_exec = exec;
  return GX_OK;
}

gx_status run_search(gx_net* h, const gx_explore_opts* opts, bool stop_first, void* ws,
                     uint64_t ws_bytes, cudaStream_t st) {
  const Net& net = h->net;
  gx_explore_opts d;
  gx_default_opts(&d);
  const gx_explore_opts* o = opts ? opts : &d;
  Plan P;
  gx_status s = make_plan(net, o, P);
  if (s != GX_OK) return s;
  Device dev;
  if ((s = device_info(dev)) != GX_OK) return s;
  Ctl* hc = nullptr;
  uint32_t* htot = nullptr;
  if ((s = host_ctl(hc, htot)) != GX_OK) return s;

  bool owned = false;
  if (!ws) {
    GX_CUDA(cudaMallocAsync(&ws, P.total, st));
    owned = true;
  } else {
    if (ws_bytes < P.total)
      return fail(GX_ERR_OOM, "workspace holds " + std::to_string(ws_bytes) + " bytes, need " +
                                  std::to_string(P.total));
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(GX_ERR_INVALID, "workspace is not 256-byte aligned");
  }
  struct Freer {
    void* p;
    bool own;
    cudaStream_t st;
    ~Freer() {
      if (own && p) cudaFreeAsync(p, st);
    }
  } freer{ws, owned, st};

  char* base = static_cast<char*>(ws);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + P.off_ctl);
  uint32_t* blob = reinterpret_cast<uint32_t*>(base + P.off_blob);
  uint32_t* dl = reinterpret_cast<uint32_t*>(base + P.off_dl);
  uint32_t* front = reinterpret_cast<uint32_t*>(base + P.off_front);
  uint32_t* table = reinterpret_cast<uint32_t*>(base + P.off_table);

  GX_CUDA(cudaMemcpyAsync(blob, net.blob.data(), 4 * net.blob.size(), cudaMemcpyHostToDevice, st));

  cudaEvent_t ev0, ev1, ek0, ek1;
  GX_CUDA(cudaEventCreate(&ev0));
  GX_CUDA(cudaEventCreate(&ev1));
  GX_CUDA(cudaEventCreate(&ek0));
  GX_CUDA(cudaEventCreate(&ek1));
  struct EvFree {
    cudaEvent_t a, b, c, d;
    ~EvFree() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaEventDestroy(c);
      cudaEventDestroy(d);
    }
  } evfree{ev0, ev1, ek0, ek1};

  // levels on the device unless asked otherwise; the partitioned path needs the host
  const bool device_loop = !o->host_loop && P.logp == 0;
  GX_CUDA(cudaEventRecord(ev0, st));
  unsigned long long* gcache = P.gcache ? reinterpret_cast<unsigned long long*>(base + P.off_gcache) : nullptr;
  if (!device_loop) {
    GX_CUDA(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
    GX_CUDA(cudaMemsetAsync(table, 0, 4ull * P.B * P.nb, st));
    if (gcache) GX_CUDA(cudaMemsetAsync(gcache, 0, 8ull * P.gcache, st));
  }

  InitArgs ia{};
  hash_multipliers(ia.muls.m, kMaxRounds);
  ia.rounds = P.rounds;
  ia.log2nb = ilog2(P.nb);
  ia.table = table;
  ia.frontier = front;
  ia.ctl = ctl;
  for (int w = 0; w < 4; ++w) ia.vec[w] = net.init_vec[w];
  if (!device_loop) GX_CUDA(P.ks->init(ia, st));

  ExpandArgs ea{};
  ea.blob = blob;
  ea.blob_words = (uint32_t)net.blob.size();
  ea.lay = net.lay;
  ea.muls = ia.muls;
  ea.rounds = P.rounds;
  ea.log2nb = ia.log2nb;
  ea.table = table;
  ea.frontier = front;
  ea.fmask = P.fcap - 1;
  ea.ctl = ctl;
  ea.dl_buf = dl;
  ea.dl_cap = P.dl_cap;
  ea.count_states = 1;  // region passes set their own (region_pass)
  ea.gcache = gcache;
  ea.gcache_mask = P.gcache ? P.gcache - 1 : 0;
  for (int w = 0; w < 3; ++w) ea.gkey_shift[w] = P.gkey[w];
  uint32_t* viol = reinterpret_cast<uint32_t*>(base + P.off_viol);
  if (o->watch) {
    const uint32_t wp = o->watch_proc;
    ea.watch = 1;
    ea.watch_word = net.field_word[wp];
    ea.watch_shift = net.field_shift[wp];
    ea.watch_mask = (1u << net.field_bits[wp]) - 1u;
    ea.watch_value = o->watch_state;
    ea.viol_buf = viol;
    ea.viol_cap = P.viol_cap;
  }
  size_t smem = 8ull * kMaxRounds;
  const size_t blob_bytes = 4ull * net.blob.size();
  ea.stage = (smem + blob_bytes <= std::min<size_t>(dev.smem_optin, 96 * 1024)) ? 1 : 0;
  if (ea.stage) smem += blob_bytes;
  ea.cache_log2 = 0;
  if (P.warp_log2) {
    ea.cache_log2 = (int)P.warp_log2;
    if (ea.cache_log2 > 12) return fail(GX_ERR_INVALID, "warp_cache_log2 must be at most 12");
    if (P.W == 4) ea.cache_log2 -= 1;  // 16-byte entries: the same bytes as 2^n 2-word ones
    smem += 4ull * P.W * (kBlock / 32) * (1ull << ea.cache_log2);
    if (smem > dev.smem_optin)
      return fail(GX_ERR_INVALID, "warp cache of 2^" + std::to_string(ea.cache_log2) + " entries per warp needs " +
                                      std::to_string(smem) + " bytes of shared memory per CTA, more than " +
                                      std::to_string(dev.smem_optin));
  }
  GX_CUDA(cudaFuncSetAttribute(P.expand_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.expand_fn, kBlock, smem));
  if (per_sm < 1) return fail(GX_ERR_INVALID, "expansion kernel does not fit on an SM");
  if (o->ctas_per_sm) per_sm = std::min<int>(per_sm, (int)o->ctas_per_sm);
  const uint64_t max_grid = (uint64_t)dev.sms * per_sm;

  std::vector<uint64_t> levels{1};
  uint64_t cur_begin = 0, cur_end = 1, explored = 0;
  int64_t first_dl = -1, first_viol = -1;
  const bool stop_viol = o->watch && o->stop_at_first_violation;
  double expand_ms = 0;
  uint64_t launches = 0, levels_done = 0;
  uint32_t err = 0;
  std::vector<double> lv_ms;
  std::vector<uint64_t> lv_probes, lv_trans;
  uint64_t prev_probes = 0, prev_trans = 0;
  bool complete = false, finished = false;
  uint64_t kernel_launches = device_loop ? 0 : 1, device_levels = 0, d2h_loop = 0, dev_expand = 0;
  if (device_loop) {
    LoopArgs la{};
    la.ctl = ctl;
    unsigned long long* lv = reinterpret_cast<unsigned long long*>(base + P.off_loop);
    la.lv_size = lv;
    la.lv_tns = lv + kLoopLevels;
    la.lv_probes = lv + 2 * kLoopLevels;
    la.lv_trans = lv + 3 * kLoopLevels;
    la.cap = kLoopLevels;
    la.stop_dl = stop_first ? 1 : 0;
    la.stop_viol = stop_viol ? 1 : 0;
    la.max_levels = o->max_levels;
    ExpandArgs eg = ea;
    eg.dev_range = 1;
    // the graph holds every argument by value: rebuild it when anything changes
    std::vector<unsigned char> key(sizeof(gx_explore_opts) + 5 * sizeof(uint64_t));
    const uint64_t extra[5] = {reinterpret_cast<uint64_t>(ws), P.total, stop_first ? 1ull : 0ull, smem, max_grid};
    std::memcpy(key.data(), o, sizeof(gx_explore_opts));
    std::memcpy(key.data() + sizeof(gx_explore_opts), extra, sizeof(extra));
    if (!h->loop_exec || h->loop_key != key) {
      s = build_loop_graph(h, P, ctl, table, ia, eg, la, smem, max_grid);
      if (s != GX_OK) return s;
      h->loop_key = key;
    }
    GX_CUDA(cudaGraphLaunch(static_cast<cudaGraphExec_t>(h->loop_exec), st));
    GX_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    std::vector<unsigned long long> hl(4ull * kLoopLevels);
    GX_CUDA(cudaMemcpyAsync(hl.data(), lv, 8ull * hl.size(), cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaStreamSynchronize(st));
    d2h_loop = sizeof(Ctl) + 8ull * hl.size();
    const uint64_t nd = hc->levels_done;
    const uint64_t nl = std::min<uint64_t>(hc->n_levels, kLoopLevels);
    levels.assign(hl.begin(), hl.begin() + nl);
    for (uint64_t k = 0; k < nd && k < kLoopLevels; ++k) {
      lv_ms.push_back(1e-6 * (double)hl[kLoopLevels + k]);
      lv_probes.push_back(hl[2 * kLoopLevels + k] - prev_probes);
      lv_trans.push_back(hl[3 * kLoopLevels + k] - prev_trans);
      prev_probes = hl[2 * kLoopLevels + k];
      prev_trans = hl[3 * kLoopLevels + k];
      expand_ms += lv_ms.back();
    }
    explored = hc->explored;
    levels_done = nd;
    launches = nd * P.regions;
    dev_expand = launches;
    device_levels = nd;
    kernel_launches = 2 + (P.regions + 1) * nd;  // init, start, then the passes + advance per level
    first_dl = hc->first_dl;
    first_viol = hc->first_viol;
    complete = hc->complete != 0;
    err = hc->error;
    cur_begin = hc->cur_begin;
    cur_end = hc->cur_end;
    finished = !hc->yielded;
  }
  // partitioned path set-up
  PartArgs pa{};
  size_t psmem = 0;
  int probe_grid = 0;
  if (P.logp) {
    pa.hist = reinterpret_cast<uint32_t*>(base + P.off_hist);
    pa.off = reinterpret_cast<uint32_t*>(base + P.off_off);
    pa.ptot = reinterpret_cast<uint32_t*>(base + P.off_ptot);
    pa.tot = reinterpret_cast<uint32_t*>(base + P.off_tot);
    pa.succ = reinterpret_cast<uint32_t*>(base + P.off_succ);
    pa.logp = P.logp;
    psmem = 8ull * kMaxRounds + (ea.stage ? blob_bytes : 0) + (4ull << P.logp);
    GX_CUDA(cudaFuncSetAttribute(P.ks->part_count_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
    GX_CUDA(cudaFuncSetAttribute(P.ks->part_scatter_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
    int pp = 0;
    GX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pp, P.ks->part_probe_fn, kBlock, 0));
    probe_grid = dev.sms * std::max(pp, 1);
  }
  uint64_t part_levels = 0, d2h_tot = 0;

  while (!finished) {
    const uint64_t F = cur_end - cur_begin;
    ea.cur_begin = cur_begin;
    ea.cur_end = cur_end;
    const bool part = P.logp && F >= P.part_min;
    GX_CUDA(cudaEventRecord(ek0, st));
    bool direct = !part;
    if (part) {
      pa.nb = (int)std::max<uint64_t>(1, std::min<uint64_t>(kPartCtas, F / kBlock));
      pa.range = (F + pa.nb - 1) / pa.nb;
      GX_CUDA(P.ks->part_count(ea, pa, psmem, st));
      ++launches;
      GX_CUDA(cudaMemcpyAsync(htot, pa.tot, 4ull * pa.nb, cudaMemcpyDeviceToHost, st));
      d2h_tot += 4ull * pa.nb;
      GX_CUDA(cudaStreamSynchronize(st));
      uint32_t biggest = 0;
      for (int b = 0; b < pa.nb; ++b) biggest = std::max(biggest, htot[b]);
      direct = biggest > P.cs;  // one CTA's successors do not fit: expand this level directly
      if (!direct) {
        ++part_levels;
        int b0 = 0;
        while (b0 < pa.nb) {
          uint64_t n = 0;
          int b1 = b0;
          while (b1 < pa.nb && n + htot[b1] <= P.cs) n += htot[b1++];
          pa.b0 = b0;
          pa.b1 = b1;
          GX_CUDA(P.ks->part_scan(pa, st));
          GX_CUDA(P.ks->part_scatter(ea, pa, psmem, st));
          GX_CUDA(cudaMemsetAsync(&ctl->claim, 0, sizeof(unsigned long long), st));
          GX_CUDA(P.ks->part_probe(ea, pa.succ, n, probe_grid, st));
          launches += 3;
          b0 = b1;
        }
      }
    }
    if (direct) {
      const uint64_t warps = (F + 31) / 32;
      const uint64_t want = (warps + kBlock / 32 - 1) / (kBlock / 32);
      const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, max_grid));
      for (uint32_t q = 0; q < P.regions; ++q) {
        GX_CUDA(cudaMemsetAsync(&ctl->claim, 0, sizeof(unsigned long long), st));
        GX_CUDA(P.expand(region_pass(ea, P.regions, q), grid, smem, st));
        ++launches;
      }
    }
    GX_CUDA(cudaEventRecord(ek1, st));
    GX_CUDA(cudaMemcpyAsync(hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaStreamSynchronize(st));
    float ms = 0;
    GX_CUDA(cudaEventElapsedTime(&ms, ek0, ek1));
    expand_ms += ms;
    ++levels_done;
    lv_ms.push_back(ms);
    lv_probes.push_back(hc->probes - prev_probes);
    lv_trans.push_back(hc->transitions - prev_trans);
    prev_probes = hc->probes;
    prev_trans = hc->transitions;
    explored += cur_end - cur_begin;
    if (first_dl < 0 && hc->dl_count > 0) first_dl = (int64_t)levels.size() - 1;
    if (first_viol < 0 && hc->viol_count > 0) first_viol = (int64_t)levels.size() - 1;
    err = hc->error;
    const uint64_t next_end = hc->next_end;
    if (next_end > cur_end) levels.push_back(next_end - cur_end);
    if (err) break;
    if (next_end == cur_end) {
      complete = true;
      break;
    }
    cur_begin = cur_end;
    cur_end = next_end;
    if (stop_first && hc->dl_count > 0) break;
    if (stop_viol && hc->viol_count > 0) break;
    if (o->max_levels && levels_done >= o->max_levels) break;
  }
  GX_CUDA(cudaEventRecord(ev1, st));
  GX_CUDA(cudaStreamSynchronize(st));
  float total_ms = 0;
  GX_CUDA(cudaEventElapsedTime(&total_ms, ev0, ev1));

  // deadlock states
  const uint64_t ndl = std::min<uint64_t>(hc->dl_count, P.dl_cap);
  std::vector<uint32_t> dlw(ndl * P.W);
  if (ndl) {
    GX_CUDA(cudaMemcpyAsync(dlw.data(), dl, 4 * dlw.size(), cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaStreamSynchronize(st));
  }
  h->deadlocks.assign(ndl * net.n_procs, 0);
  for (uint64_t i = 0; i < ndl; ++i) {
    uint32_t w4[4] = {0, 0, 0, 0};
    for (int w = 0; w < P.W; ++w) w4[w] = dlw[i * P.W + w];
    unpack_host(net, w4, h->deadlocks.data() + i * net.n_procs);
  }

  // violating states (safety check)
  const uint64_t nvi = std::min<uint64_t>(hc->viol_count, P.viol_cap);
  std::vector<uint32_t> viw(nvi * P.W);
  if (nvi) {
    GX_CUDA(cudaMemcpyAsync(viw.data(), viol, 4 * viw.size(), cudaMemcpyDeviceToHost, st));
    GX_CUDA(cudaStreamSynchronize(st));
  }
  h->violations.assign(nvi * net.n_procs, 0);
  for (uint64_t i = 0; i < nvi; ++i) {
    uint32_t w4[4] = {0, 0, 0, 0};
    for (int w = 0; w < P.W; ++w) w4[w] = viw[i * P.W + w];
    unpack_host(net, w4, h->violations.data() + i * net.n_procs);
  }

  gx_stats_t& S = h->stats;
  std::memset(&S, 0, sizeof(S));
  S.states = hc->next_end;
  S.explored = explored;
  S.transitions = hc->transitions;
  S.n_levels = levels.size();
  S.deadlock_count = hc->dl_count;
  S.deadlock_sum = hc->dl_sum;
  S.deadlock_xor = hc->dl_xor;
  S.first_deadlock_level = first_dl;
  S.violation_count = hc->viol_count;
  S.violation_sum = hc->viol_sum;
  S.violation_xor = hc->viol_xor;
  S.first_violation_level = first_viol;
  S.table_slots = P.nb * (uint64_t)(P.B / P.W);
  S.vector_words = net.vector_words;
  S.slot_words = (uint32_t)P.W;
  S.bucket_words = (uint32_t)P.B;
  S.group_lanes = (uint32_t)P.G;
  S.hash_rounds = (uint32_t)P.rounds;
  S.complete = complete ? 1 : 0;
  S.fill = (double)S.states / (double)S.table_slots;
  S.gpu_ms = total_ms;
  S.expand_ms = expand_ms;
  S.expand_launches = launches;
  S.kernel_launches = kernel_launches + (launches - dev_expand);
  S.region_passes = P.regions;
  S.global_cache_entries = P.gcache;
  S.device_levels = device_levels;
  S.probes = hc->probes;
  S.partitioned_levels = part_levels;
  S.h2d_bytes = 4ull * net.blob.size();
  S.d2h_bytes = sizeof(Ctl) * (levels_done - device_levels) + d2h_loop + 4ull * (dlw.size() + viw.size()) + d2h_tot;
  h->levels = levels;
  h->level_ms = lv_ms;
  h->level_probes = lv_probes;
  h->level_transitions = lv_trans;
  h->ws_off_ctl = P.off_ctl;
  h->ws_off_blob = P.off_blob;
  h->ws_off_table = P.off_table;
  h->ws_total = P.total;
  h->have_result = true;
  gx_status rs = GX_OK;
  if (err & ERR_TABLE_FULL) rs = fail(GX_ERR_TABLE_FULL, "hash table full: no free slot under any hash-constant set");
  else if (err & ERR_FRONTIER) rs = fail(GX_ERR_FRONTIER_OVERFLOW, "frontier ring overflow; raise frontier_states");
  else if (err & ERR_SPIN) rs = fail(GX_ERR_SPIN_LIMIT, "a device wait hit its iteration limit");
  S.status = (uint32_t)rs;
  return rs;
}

}  // namespace
}  // namespace gx

extern "C" {

gx_status gx_workspace_bytes(const gx_net* h, const gx_explore_opts* opts, uint64_t* bytes) {
  gx::clear_error();
  if (!h || !bytes) return gx::fail(GX_ERR_INVALID, "net or bytes is NULL");
  gx::Plan P;
  gx_status s = gx::make_plan(h->net, opts, P);
  if (s != GX_OK) return s;
  *bytes = P.total;
  return GX_OK;
}

gx_status gx_explore(gx_net* h, const gx_explore_opts* opts, void* ws, uint64_t ws_bytes, void* stream) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  return gx::run_search(h, opts, opts && opts->stop_at_first_deadlock, ws, ws_bytes,
                        static_cast<cudaStream_t>(stream));
}

gx_status gx_find_deadlocks(gx_net* h, const gx_explore_opts* opts, uint32_t mode, void* ws,
                            uint64_t ws_bytes, void* stream, uint32_t* out_states, uint32_t cap,
                            uint64_t* n_found) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  if (cap && !out_states) return gx::fail(GX_ERR_INVALID, "out_states is NULL");
  gx_status s;
  if (mode == GX_DL_BFS_FIRST || mode == GX_DL_BFS_ALL) {
    s = gx::run_search(h, opts, mode == GX_DL_BFS_FIRST, ws, ws_bytes, static_cast<cudaStream_t>(stream));
  } else if (mode == GX_DL_GUIDED) {
    if (opts && opts->watch) return gx::fail(GX_ERR_INVALID, "the safety check (watch) runs with BFS searches only");
    s = gx::run_guided(h, opts, ws, ws_bytes, static_cast<cudaStream_t>(stream));
  } else {
    return gx::fail(GX_ERR_INVALID, "unknown deadlock-search mode");
  }
  if (!h->have_result) return s;
  const uint32_t n = h->net.n_procs;
  const uint64_t have = h->deadlocks.size() / n;
  const uint64_t k = std::min<uint64_t>(have, cap);
  if (k) std::memcpy(out_states, h->deadlocks.data(), 4ull * n * k);
  if (n_found) *n_found = h->stats.deadlock_count;
  return s;
}

gx_status gx_stats(const gx_net* h, gx_stats_t* out) {
  gx::clear_error();
  if (!h || !out) return gx::fail(GX_ERR_INVALID, "net or out is NULL");
  if (!h->have_result) return gx::fail(GX_ERR_STATE, "no search has run on this network");
  *out = h->stats;
  return GX_OK;
}

gx_status gx_levels(const gx_net* h, uint64_t* out, uint32_t cap, uint32_t* n_levels) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  if (!h->have_result) return gx::fail(GX_ERR_STATE, "no search has run on this network");
  if (cap && !out) return gx::fail(GX_ERR_INVALID, "out is NULL");
  for (size_t i = 0; i < h->levels.size() && i < cap; ++i) out[i] = h->levels[i];
  if (n_levels) *n_levels = (uint32_t)h->levels.size();
  return GX_OK;
}

gx_status gx_level_profile(const gx_net* h, double* ms, uint64_t* probes, uint64_t* transitions, uint32_t cap,
                           uint32_t* n) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  if (!h->have_result) return gx::fail(GX_ERR_STATE, "no search has run on this network");
  const size_t k = h->level_ms.size();
  for (size_t i = 0; i < k && i < cap; ++i) {
    if (ms) ms[i] = h->level_ms[i];
    if (probes) probes[i] = h->level_probes[i];
    if (transitions) transitions[i] = h->level_transitions[i];
  }
  if (n) *n = (uint32_t)k;
  return GX_OK;
}

gx_status gx_violations(const gx_net* h, uint32_t* out, uint32_t cap, uint32_t* n) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  if (!h->have_result) return gx::fail(GX_ERR_STATE, "no search has run on this network");
  if (cap && !out) return gx::fail(GX_ERR_INVALID, "out is NULL");
  const uint32_t np = h->net.n_procs;
  const uint64_t have = h->violations.size() / np;
  const uint64_t k = std::min<uint64_t>(have, cap);
  if (k) std::memcpy(out, h->violations.data(), 4ull * np * k);
  if (n) *n = (uint32_t)k;
  return GX_OK;
}

gx_status gx_deadlocks(const gx_net* h, uint32_t* out, uint32_t cap, uint32_t* n) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  if (!h->have_result) return gx::fail(GX_ERR_STATE, "no search has run on this network");
  if (cap && !out) return gx::fail(GX_ERR_INVALID, "out is NULL");
  const uint32_t np = h->net.n_procs;
  const uint64_t have = h->deadlocks.size() / np;
  const uint64_t k = std::min<uint64_t>(have, cap);
  if (k) std::memcpy(out, h->deadlocks.data(), 4ull * np * k);
  if (n) *n = (uint32_t)k;
  return GX_OK;
}

gx_status gx_set_digest(gx_net* h, void* ws, uint64_t ws_bytes, void* stream, uint64_t* count,
                        uint64_t* sum, uint64_t* xr) {
  gx::clear_error();
  if (!h || !ws) return gx::fail(GX_ERR_INVALID, "net or workspace is NULL");
  if (!h->have_result) return gx::fail(GX_ERR_STATE, "no search has run on this network");
  if (ws_bytes && ws_bytes < h->ws_total) return gx::fail(GX_ERR_INVALID, "workspace smaller than the last search's");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gx::Device dev;
  gx_status s = gx::device_info(dev);
  if (s != GX_OK) return s;
  char* base = static_cast<char*>(ws);
  unsigned long long* out = reinterpret_cast<gx::Ctl*>(base + h->ws_off_ctl)->digest;
  GX_CUDA(cudaMemsetAsync(out, 0, 3 * sizeof(unsigned long long), st));
  gx::DigestArgs a{};
  a.table = reinterpret_cast<const uint32_t*>(base + h->ws_off_table);
  a.slots = h->stats.table_slots;
  a.blob = reinterpret_cast<const uint32_t*>(base + h->ws_off_blob);
  a.lay = h->net.lay;
  a.out = out;
  GX_CUDA(gx::launch_digest((int)h->stats.slot_words, a, dev.sms * 8, st));
  unsigned long long r[3];
  GX_CUDA(cudaMemcpyAsync(r, out, sizeof(r), cudaMemcpyDeviceToHost, st));
  GX_CUDA(cudaStreamSynchronize(st));
  if (count) *count = r[0];
  if (sum) *sum = r[1];
  if (xr) *xr = r[2];
  return GX_OK;
}

}  // extern "C"

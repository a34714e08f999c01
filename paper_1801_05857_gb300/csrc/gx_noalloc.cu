// gx_explore_noalloc: breadth-first exploration that allocates nothing.
//
// Some callers cannot allocate device memory at all: a host framework that has
// reserved the GPU's memory for its own pool at start-up (a cudaMalloc then
// fails, or bypasses the framework's accounting), or a latency-critical caller
// that must not pay cudaFree's implicit device-wide synchronisation.  This
// entry point runs the same level-expansion kernels as gx_explore on scratch
// memory that the library owns statically: one file-scope __device__ array
// of kScratchBytes.  Every GPU that loads the library holds that array until
// the process exits.
//
// The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (the host-side name of a __device__ array is only a
// stand-in, never a device address) and caches it; make that first call before
// any stream capture.  All calls share the array and it keeps the last call's
// contents, so each call clears the parts that must start at zero (control
// block, hash table and the GPU-wide cache of seen vectors).  Calls whose GPU work overlaps -- on two streams or
// from two threads -- race on the array and give wrong results.

#include <algorithm>
#include <cstring>
#include <string>

#include "gx_kernels.cuh"

namespace {

constexpr uint64_t kScratchBytes = GX_NOALLOC_SCRATCH_BYTES;
static_assert(kScratchBytes % 256 == 0, "scratch size");
constexpr uint64_t kDefaultTableBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, per device (set up on first use).
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

gx_status scratch_for_current_device(unsigned char*& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gx::fail(GX_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return gx::fail(GX_ERR_INVALID, "device ordinal beyond 63");
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess)
      return gx::fail(GX_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  out = g_scratch_ptr[dev];
  return GX_OK;
}

#define NA_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return gx::fail(GX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
  } while (0)

}  // namespace

extern "C" {

gx_status gx_explore_noalloc(const gx_net* h, const gx_explore_opts* opts, void* stream,
                             gx_stats_t* stats_out, uint64_t* levels_out, uint32_t levels_cap,
                             uint32_t* n_levels) {
  gx::clear_error();
  if (!h || !stats_out) return gx::fail(GX_ERR_INVALID, "net or stats_out is NULL");
  if (levels_cap && !levels_out) return gx::fail(GX_ERR_INVALID, "levels_out is NULL");
  const gx::Net& net = h->net;
  gx_explore_opts d;
  gx_default_opts(&d);
  const gx_explore_opts* o = opts ? opts : &d;
  // the slice-partitioned path needs a successor buffer this entry point does not have
  if (o->partition_min_states)
    return gx::fail(GX_ERR_INVALID, "gx_explore_noalloc has no partitioned path: set partition_min_states to 0");
  if (o->watch) {
    if (o->watch_proc >= net.n_procs) return gx::fail(GX_ERR_INVALID, "watch_proc is not a process of the network");
    if (o->watch_state >= net.n_states[o->watch_proc])
      return gx::fail(GX_ERR_INVALID, "watch_state is not a local state of watch_proc");
  }

  // --- sizes (same rules as gx_explore, with a smaller default table)
  const int W = (int)net.slot_words;
  const int B = o->bucket_words ? (int)o->bucket_words : 8;
  if (B != 4 && B != 8 && B != 16 && B != 32) return gx::fail(GX_ERR_INVALID, "bucket_words must be 4, 8, 16 or 32");
  if (B < W) return gx::fail(GX_ERR_INVALID, "bucket_words is smaller than one slot");
  const int S = B / W;
  const int G = o->group_lanes ? (int)o->group_lanes : std::min(S, 32);
  const int rounds = o->hash_rounds ? (int)o->hash_rounds : 8;
  if (rounds < 1 || rounds > gx::kMaxRounds) return gx::fail(GX_ERR_INVALID, "hash_rounds must be 1..64");
  const gx::KernelSet* ks = gx::kernels_for(W, B, G);
  if (!ks) return gx::fail(GX_ERR_INVALID, "group_lanes must be a power of two dividing bucket_words / slot words");
  uint32_t regions = o->region_passes ? o->region_passes : 1;  // tables here are far below 64 GiB
  if (regions > 16 || (regions & (regions - 1)))
    return gx::fail(GX_ERR_INVALID, "region_passes must be a power of two from 1 to 16");
  const uint64_t table_bytes = o->table_bytes ? o->table_bytes : kDefaultTableBytes;
  uint64_t nb = 1;
  while (nb * 2 * 4ull * B <= table_bytes) nb *= 2;
  if (nb < 2) return gx::fail(GX_ERR_INVALID, "table_bytes is smaller than two buckets");
  const uint64_t slots = nb * (uint64_t)S;
  const uint64_t fwant = o->frontier_states ? o->frontier_states : std::max<uint64_t>(4096, slots / 4);
  uint64_t fcap = 1;
  while (fcap < fwant) fcap *= 2;
  // caches of seen vectors, as gx_explore chooses them (gx_explore_opts)
  uint64_t gentries = 0;
  uint32_t gkey[3] = {64, 64, 64};
  const bool key_fits = W <= 2 || gx::cache_key_shifts(net, gkey);
  if (o->global_cache_log2 == 0xFFFFFFFFu) {
    if (W <= 2 && G == 1 && (table_bytes / (4ull * W)) >= (1ull << 26)) gentries = 1ull << 23;
  } else if (o->global_cache_log2) {
    if (o->global_cache_log2 > 26) return gx::fail(GX_ERR_INVALID, "global_cache_log2 must be at most 26");
    if (key_fits) gentries = 1ull << o->global_cache_log2;
  }
  if (regions > nb) regions = (uint32_t)nb;
  // the level kernel, as gx_explore chooses it: the queued second kernel with region passes
  const bool queued = regions > 1 && ks->expand_queued;
  const auto expand = queued ? ks->expand_queued : ks->expand;
  const void* expand_fn = queued ? ks->expand_queued_fn : ks->expand_fn;
  const uint32_t warp_log2 =
      o->warp_cache_log2 == 0xFFFFFFFFu ? (gentries ? 0u : queued ? 6u : 9u) : o->warp_cache_log2;
  const uint64_t off_ctl = 0;
  const uint64_t off_blob = align256(sizeof(gx::Ctl));
  const uint64_t off_front = align256(off_blob + 4ull * net.blob.size());
  const uint64_t off_table = align256(off_front + 4ull * W * fcap);
  const uint64_t off_gcache = align256(off_table + 4ull * B * nb);
  const uint64_t total = align256(off_gcache + 8ull * gentries);
  if (total > kScratchBytes)
    return gx::fail(GX_ERR_INVALID, "gx_explore_noalloc needs " + std::to_string(total) +
                                        " bytes of scratch but its static array holds " +
                                        std::to_string(kScratchBytes) +
                                        "; lower table_bytes / frontier_states or use gx_explore");

  unsigned char* base = nullptr;
  gx_status s = scratch_for_current_device(base);
  if (s != GX_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, smem_optin = 0;
  NA_CUDA(cudaGetDevice(&dev));
  NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  NA_CUDA(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

  gx::Ctl* ctl = reinterpret_cast<gx::Ctl*>(base + off_ctl);
  uint32_t* blob = reinterpret_cast<uint32_t*>(base + off_blob);
  uint32_t* front = reinterpret_cast<uint32_t*>(base + off_front);
  uint32_t* table = reinterpret_cast<uint32_t*>(base + off_table);

  // the array keeps the previous call's contents: clear control block, table and cache
  NA_CUDA(cudaMemcpyAsync(blob, net.blob.data(), 4 * net.blob.size(), cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemsetAsync(ctl, 0, sizeof(gx::Ctl), st));
  NA_CUDA(cudaMemsetAsync(table, 0, 4ull * B * nb, st));
  unsigned long long* gcache = gentries ? reinterpret_cast<unsigned long long*>(base + off_gcache) : nullptr;
  if (gcache) NA_CUDA(cudaMemsetAsync(gcache, 0, 8ull * gentries, st));

  int log2nb = 0;
  while ((1ull << log2nb) < nb) ++log2nb;
  int log2r = 0;
  while ((1u << log2r) < regions) ++log2r;
  gx::InitArgs ia{};
  gx::hash_multipliers(ia.muls.m, gx::kMaxRounds);
  ia.rounds = rounds;
  ia.log2nb = log2nb;
  ia.table = table;
  ia.frontier = front;
  ia.ctl = ctl;
  for (int w = 0; w < 4; ++w) ia.vec[w] = net.init_vec[w];
  NA_CUDA(ks->init(ia, st));

  gx::ExpandArgs ea{};
  ea.blob = blob;
  ea.blob_words = (uint32_t)net.blob.size();
  ea.lay = net.lay;
  ea.muls = ia.muls;
  ea.rounds = rounds;
  ea.log2nb = log2nb;
  ea.table = table;
  ea.frontier = front;
  ea.fmask = fcap - 1;
  ea.ctl = ctl;
  ea.dl_buf = nullptr;
  ea.dl_cap = 0;  // deadlocks are counted and digested, not stored
  ea.count_states = 1;
  ea.gcache = gcache;
  ea.gcache_mask = gentries ? gentries - 1 : 0;
  for (int w = 0; w < 3; ++w) ea.gkey_shift[w] = gkey[w];
  if (o->watch) {  // the safety check: violations counted and digested, not stored
    const uint32_t wp = o->watch_proc;
    ea.watch = 1;
    ea.watch_word = net.field_word[wp];
    ea.watch_shift = net.field_shift[wp];
    ea.watch_mask = (1u << net.field_bits[wp]) - 1u;
    ea.watch_value = o->watch_state;
    ea.viol_buf = nullptr;
    ea.viol_cap = 0;
  }
  size_t smem = 8ull * gx::kMaxRounds;
  const size_t blob_bytes = 4ull * net.blob.size();
  ea.stage = (smem + blob_bytes <= std::min<size_t>((size_t)smem_optin, 96 * 1024)) ? 1 : 0;
  if (ea.stage) smem += blob_bytes;
  // the per-warp cache of seen vectors lives in shared memory: same rule as gx_explore
  ea.cache_log2 = 0;
  if (warp_log2) {
    ea.cache_log2 = (int)warp_log2;
    if (ea.cache_log2 > 12) return gx::fail(GX_ERR_INVALID, "warp_cache_log2 must be at most 12");
    if (W == 4) ea.cache_log2 -= 1;  // 16-byte entries: the same bytes as 2^n 2-word ones
    smem += 4ull * W * (gx::kBlock / 32) * (1ull << ea.cache_log2);
    if (smem > (size_t)smem_optin)
      return gx::fail(GX_ERR_INVALID, "warp cache of 2^" + std::to_string(ea.cache_log2) +
                                          " entries per warp needs " + std::to_string(smem) +
                                          " bytes of shared memory per CTA, more than " +
                                          std::to_string(smem_optin));
  }
  NA_CUDA(cudaFuncSetAttribute(expand_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  NA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_fn, gx::kBlock, smem));
  if (per_sm < 1) return gx::fail(GX_ERR_INVALID, "expansion kernel does not fit on an SM");
  if (o->ctas_per_sm) per_sm = std::min<int>(per_sm, (int)o->ctas_per_sm);
  const uint64_t max_grid = (uint64_t)sms * per_sm;

  gx::Ctl hc;  // pageable copy of the control block
  uint64_t cur_begin = 0, cur_end = 1, explored = 0, launches = 0;
  uint32_t nlv = 1;
  if (levels_cap) levels_out[0] = 1;
  int64_t first_dl = -1, first_viol = -1;
  const bool stop_viol = o->watch && o->stop_at_first_violation;
  bool complete = false;
  while (true) {
    ea.cur_begin = cur_begin;
    ea.cur_end = cur_end;
    const uint64_t warps = (cur_end - cur_begin + 31) / 32;
    const uint64_t want = (warps + gx::kBlock / 32 - 1) / (gx::kBlock / 32);
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, max_grid));
    // region passes (gx_explore_opts.region_passes): pass q probes region q of the table
    for (uint32_t q = 0; q < regions; ++q) {
      gx::ExpandArgs eq = ea;
      eq.region_mask = regions > 1 ? (uint64_t)(regions - 1) << (log2nb - log2r) : 0ull;
      eq.region_bits = (uint64_t)q << (log2nb - log2r);
      eq.count_states = q == 0 ? 1 : 0;
      NA_CUDA(cudaMemsetAsync(&ctl->claim, 0, sizeof(unsigned long long), st));
      NA_CUDA(expand(eq, grid, smem, st));
    }
    NA_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(gx::Ctl), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    ++launches;
    explored += cur_end - cur_begin;
    if (first_dl < 0 && hc.dl_count > 0) first_dl = (int64_t)nlv - 1;
    if (first_viol < 0 && hc.viol_count > 0) first_viol = (int64_t)nlv - 1;
    if (hc.next_end > cur_end) {
      if (nlv < levels_cap) levels_out[nlv] = hc.next_end - cur_end;
      ++nlv;
    }
    if (hc.error) break;
    if (hc.next_end == cur_end) {
      complete = true;
      break;
    }
    cur_begin = cur_end;
    cur_end = hc.next_end;
    if (o->stop_at_first_deadlock && hc.dl_count > 0) break;
    if (stop_viol && hc.viol_count > 0) break;
    if (o->max_levels && launches >= o->max_levels) break;
  }

  gx_stats_t& S2 = *stats_out;
  std::memset(&S2, 0, sizeof(S2));
  S2.states = hc.next_end;
  S2.explored = explored;
  S2.transitions = hc.transitions;
  S2.n_levels = nlv;
  S2.deadlock_count = hc.dl_count;
  S2.deadlock_sum = hc.dl_sum;
  S2.deadlock_xor = hc.dl_xor;
  S2.first_deadlock_level = first_dl;
  S2.violation_count = hc.viol_count;
  S2.violation_sum = hc.viol_sum;
  S2.violation_xor = hc.viol_xor;
  S2.first_violation_level = first_viol;
  S2.table_slots = slots;
  S2.vector_words = net.vector_words;
  S2.slot_words = (uint32_t)W;
  S2.bucket_words = (uint32_t)B;
  S2.group_lanes = (uint32_t)G;
  S2.hash_rounds = (uint32_t)rounds;
  S2.complete = complete ? 1 : 0;
  S2.fill = (double)S2.states / (double)slots;
  S2.expand_launches = launches * regions;
  S2.region_passes = regions;
  S2.global_cache_entries = gentries;
  S2.probes = hc.probes;
  S2.h2d_bytes = 4ull * net.blob.size();
  S2.d2h_bytes = sizeof(gx::Ctl) * launches;
  if (n_levels) *n_levels = nlv;
  gx_status rs = GX_OK;
  if (hc.error & gx::ERR_TABLE_FULL) rs = gx::fail(GX_ERR_TABLE_FULL, "hash table full: no free slot under any hash-constant set");
  else if (hc.error & gx::ERR_FRONTIER) rs = gx::fail(GX_ERR_FRONTIER_OVERFLOW, "frontier ring overflow; raise frontier_states");
  else if (hc.error & gx::ERR_SPIN) rs = gx::fail(GX_ERR_SPIN_LIMIT, "a device wait hit its iteration limit");
  S2.status = (uint32_t)rs;
  return rs;
}

}  // extern "C"

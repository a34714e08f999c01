// Host-visible interface between the level loop and the templated kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "gx_internal.h"

namespace gx {

constexpr int kMaxRounds = 64;
constexpr int kBlock = 256;  // threads per CTA for every exploration kernel

enum : uint32_t { ERR_TABLE_FULL = 1u, ERR_FRONTIER = 2u, ERR_SPIN = 4u };

// Device control block of one search (lives at the start of the workspace).
struct Ctl {
  unsigned long long claim;        // frontier chunks handed out in the current level
  unsigned long long next_end;     // absolute end of the frontier ring's filled part
  unsigned long long transitions;  // successors generated, with multiplicity
  unsigned long long dl_count, dl_sum, dl_xor;
  unsigned long long probes;       // buckets read by find-or-put
  unsigned int error;              // ERR_* bits
  unsigned int pad;
  unsigned long long digest[3];    // gx_set_digest: count, sum, xor
  unsigned long long viol_count, viol_sum, viol_xor;  // safety check
  // device-driven level loop: the level to expand next and the loop's bookkeeping
  unsigned long long cur_begin, cur_end;
  unsigned long long n_levels;      // entries of the level-size list (level 0 included)
  unsigned long long levels_done;   // levels expanded
  unsigned long long explored;
  unsigned long long t_prev;        // %globaltimer (ns) at the end of the previous level
  long long first_dl, first_viol;   // level of the first deadlock / violation, -1 if none
  unsigned int complete, yielded;   // the frontier ran empty / the level arrays filled up
};
static_assert(sizeof(Ctl) <= 256, "control block");

// Hash-constant multipliers travel by value in the kernel parameters.
struct Muls {
  uint64_t m[kMaxRounds];
};

struct ExpandArgs {
  const uint32_t* blob;      // encoded network (global memory)
  uint32_t blob_words;
  int stage;                 // 1: copy the blob into shared memory first
  NetBlobLayout lay;
  Muls muls;                 // hash-constant multipliers
  int rounds;
  int log2nb;                // table has 2^log2nb buckets
  uint32_t* table;
  uint32_t* frontier;        // ring of vectors, W words each
  uint64_t fmask;            // ring capacity - 1 (capacity is a power of two)
  uint64_t cur_begin, cur_end;  // absolute indices of the level being expanded
  Ctl* ctl;
  uint32_t* dl_buf;          // deadlock vectors, W words each
  uint32_t dl_cap;
  int cache_log2;            // per-warp cache of recently seen vectors: 2^cache_log2 entries (0 = off)
  // safety check: a state whose field (word, shift, mask) equals watch_value violates
  int watch;
  uint32_t watch_word, watch_shift, watch_mask, watch_value;
  uint32_t* viol_buf;        // violating vectors, W words each
  uint32_t viol_cap;
  int dev_range;             // 1: read cur_begin / cur_end from the control block
  // Region passes: a level is expanded in several passes, and a pass probes only
  // the successors whose first bucket b has (b & region_mask) == region_bits, so
  // the table accesses of one pass stay inside one region of the table (see
  // gx_explore_opts.region_passes).  region_mask = 0: one pass, no filter.
  uint64_t region_mask, region_bits;
  int count_states;          // 1: this pass counts transitions, deadlocks and violations
  // GPU-wide cache of recently seen vectors: 2^k entries of 64 bits in global
  // memory, small enough to stay in L2; nullptr = off.  An entry holds a vector's
  // 64-bit key: the vector itself for 1- and 2-word vectors, its payload bits
  // packed for 4-word vectors whose fields take at most 64 bits (gkey_shift).
  unsigned long long* gcache;
  uint64_t gcache_mask;
  // 4-word vectors: bit offset in the key of the payload of words 1, 2, 3
  // (word 0 at offset 0; 64 = the word carries no field)
  uint32_t gkey_shift[3];
};

// Partitioned expansion of one level (or one batch of it): successors are
// counted per table slice, scattered slice-major into a buffer, then probed
// slice by slice so the probed part of the table stays in L2.
struct PartArgs {
  uint32_t* hist;   // [nb * P]: successors of CTA b that fall in slice q, at b * P + q
  uint32_t* off;    // [nb * P]: exclusive scan over the batch's CTAs, per slice
  uint32_t* ptot;   // [P]: successors of the batch per slice
  uint32_t* tot;    // [nb]: successors per CTA
  uint32_t* succ;   // successor buffer, W words per vector, slice-major
  int nb;           // CTAs of the count and scatter passes (static frontier ranges)
  int logp;         // P = 2^logp slices
  uint64_t range;   // frontier states per CTA
  int b0, b1;       // CTAs of the current batch
};

struct InitArgs {
  Muls muls;
  int rounds, log2nb;
  uint32_t* table;
  uint32_t* frontier;
  Ctl* ctl;
  uint32_t vec[4];
};

struct DigestArgs {
  const uint32_t* table;
  uint64_t slots;
  const uint32_t* blob;
  NetBlobLayout lay;
  unsigned long long* out;   // count, sum, xor
};

struct FopArgs {
  const uint32_t* keys;
  uint64_t n;
  uint32_t* table;
  int log2nb, rounds;
  Muls muls;
  uint8_t* result;
  unsigned long long* counters;  // inserted, found, failed
};

struct KernelSet {
  cudaError_t (*expand)(const ExpandArgs&, int grid, size_t smem, cudaStream_t);
  cudaError_t (*part_count)(const ExpandArgs&, const PartArgs&, size_t smem, cudaStream_t);
  cudaError_t (*part_scan)(const PartArgs&, cudaStream_t);
  cudaError_t (*part_scatter)(const ExpandArgs&, const PartArgs&, size_t smem, cudaStream_t);
  cudaError_t (*part_probe)(const ExpandArgs&, const uint32_t* succ, uint64_t n, int grid, cudaStream_t);
  cudaError_t (*init)(const InitArgs&, cudaStream_t);
  cudaError_t (*fop)(const FopArgs&, int grid, cudaStream_t);
  const void* expand_fn;  // for occupancy queries and attributes
  const void* fop_fn;
  const void* part_count_fn;
  const void* part_scatter_fn;
  const void* part_probe_fn;
  const void* init_fn;    // for graph kernel nodes
  // the level kernel with the per-warp successor queue, where it is a second
  // kernel (4-word vectors, one lane per bucket of at most 8 words); else nullptr
  cudaError_t (*expand_queued)(const ExpandArgs&, int grid, size_t smem, cudaStream_t);
  const void* expand_queued_fn;
};

// Kernels for slot width W, bucket words B and group lanes G; nullptr if the
// combination is not built.
const KernelSet* kernels_w1(int B, int G);
const KernelSet* kernels_w2(int B, int G);
const KernelSet* kernels_w4(int B, int G);
inline const KernelSet* kernels_for(int W, int B, int G) {
  if (W == 1) return kernels_w1(B, G);
  if (W == 2) return kernels_w2(B, G);
  if (W == 4) return kernels_w4(B, G);
  return nullptr;
}

cudaError_t launch_digest(int W, const DigestArgs& a, int grid, cudaStream_t st);

// Hash-constant multipliers: odd 64-bit values drawn from splitmix64.
void hash_multipliers(uint64_t* out, int n);

// GX_DL_GUIDED search (gx_guided.cu).
gx_status run_guided(gx_net* h, const gx_explore_opts* opts, void* ws, uint64_t ws_bytes, cudaStream_t st);

}  // namespace gx

// Internal host-side definitions shared by the gx translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "gx.h"

namespace gx {

// Error reporting: every entry point records a message and returns a status.
gx_status fail(gx_status st, const std::string& msg);
void clear_error();

// Words of one packed vector are tagged in bit 31 (always set in a stored
// vector) so that an all-zero slot means "empty"; payload uses bits 0..30.
constexpr uint32_t kTag = 0x80000000u;
constexpr uint32_t kPayloadBits = 31;
constexpr uint32_t kMaxWords = 4;

// Encoded network tables, one uint32 blob uploaded to the device and staged
// into shared memory by the kernels.  Offsets (in words) of each array:
struct NetBlobLayout {
  uint32_t n_procs, n_classes, n_rules;
  uint32_t proc_word;   // [n_procs]  word index of each process field
  uint32_t proc_shift;  // [n_procs]  bit offset
  uint32_t proc_mask;   // [n_procs]  (1 << bits) - 1
  uint32_t cls_proc;    // [n_classes] process of each edge class
  uint32_t cls_base;    // [n_classes] start of the class's offset array in `coff`
  uint32_t coff;        // per class: n_states(proc) + 1 offsets into `cdelta`
  uint32_t cdelta;      // xor deltas (s ^ t) << shift, one per edge of the class
  uint32_t rule_off;    // [n_rules + 1] into rule_cls
  uint32_t rule_cls;    // class id of each rule participant
  uint32_t total;       // blob length in words
};

struct Net {
  uint32_t n_procs = 0, n_labels = 0;
  uint32_t vector_words = 0;  // L after packing (1..4)
  uint32_t slot_words = 0;    // W: L, with 3 padded to 4
  std::vector<uint32_t> n_states, initial;
  std::vector<uint32_t> field_word, field_shift, field_bits;
  uint32_t max_rule_parts = 0;
  // upper bound on the successors of any state: per process the most local
  // edges from one state, plus per rule the product over its participants of
  // the most matching edges from one state (capped at 2^40)
  uint64_t max_succ = 0;
  uint64_t n_edges = 0;  // transitions over all process LTSs
  std::vector<uint32_t> blob;
  NetBlobLayout lay{};
  uint32_t init_vec[kMaxWords] = {0, 0, 0, 0};
};

// Bit offsets of words 1..3 in the 64-bit key that the GPU-wide cache of seen
// vectors stores for a vector: each word's payload (its fields sit at the low
// bits of the word) follows the previous word's, and a word without fields gets
// 64 (left out).  Returns false when the fields take more than 64 bits in all,
// so that no such key exists.
inline bool cache_key_shifts(const Net& n, uint32_t (&s)[3]) {
  uint32_t used[kMaxWords] = {0, 0, 0, 0};
  for (uint32_t p = 0; p < n.n_procs; ++p) {
    const uint32_t end = n.field_shift[p] + n.field_bits[p];
    if (end > used[n.field_word[p]]) used[n.field_word[p]] = end;
  }
  uint32_t off = used[0];
  for (int w = 1; w < 4; ++w) {
    s[w - 1] = used[w] ? off : 64u;
    off += used[w];
  }
  return off <= 64;
}

}  // namespace gx

// The opaque handle: the encoded network plus the results of the last search.
struct gx_net {
  gx::Net net;
  bool have_result = false;
  gx_stats_t stats{};
  std::vector<uint64_t> levels;
  // per expanded level: device time, buckets read, transitions
  std::vector<double> level_ms;
  std::vector<uint64_t> level_probes, level_transitions;
  std::vector<uint32_t> deadlocks;  // unpacked, n_procs per state
  std::vector<uint32_t> violations; // unpacked, n_procs per state (safety check)
  // workspace regions of the last search (for gx_set_digest, gx_training_set)
  uint64_t ws_off_ctl = 0, ws_off_blob = 0, ws_off_table = 0, ws_total = 0;
  // guided search: scoring weights (device, caller-owned) and the last deadlock's path
  const float* guided_params = nullptr;
  std::vector<uint32_t> guided_trace;
  // label names of a network read from text (gx_load_exp); empty otherwise
  std::vector<std::string> label_names;
  // cached executable graph of the device-driven level loop (CUDA objects kept
  // opaque here), the key it was built for, and the function that frees it
  void* loop_graph = nullptr;
  void* loop_exec = nullptr;
  std::vector<unsigned char> loop_key;
  void (*release)(gx_net*) = nullptr;
  // the same for the guided search's iteration loop
  void* guided_graph = nullptr;
  void* guided_exec = nullptr;
  std::vector<unsigned char> guided_key;
  void (*release_guided)(gx_net*) = nullptr;
  gx_net() = default;
  gx_net(const gx_net&) = delete;
  gx_net& operator=(const gx_net&) = delete;
  ~gx_net() {
    if (release) release(this);
    if (release_guided) release_guided(this);
  }
};

namespace gx {
// Host-side codec (used for the initial vector and to unpack reported states).
void pack_host(const Net& net, const uint32_t* local, uint32_t* words);
void unpack_host(const Net& net, const uint32_t* words, uint32_t* local);
}  // namespace gx

// Network validation and encoding (host side of the C ABI).
//
// A network of LTSs (Sec. 3, Fig. 1) is turned into:
//   * a bit-packed vector layout: ceil(log2 n_states) bits per process,
//     fields packed LSB-first into 32-bit words with bit 31 reserved as the
//     occupied tag, no field straddling two words, at most four words
//     (Sec. 4.2 notes vectors generally fit in four integers; Sec. 5.2 shows
//     the step from one word to two for the token ring at 11 nodes);
//   * edge classes: per process the edges whose label is not one of its rule
//     labels ("local" class), and per (process, label) pair used by a rule the
//     edges with that label.  Each class stores, per local state, the xor
//     deltas (s ^ t) << shift of its edges, so a successor is the source
//     vector with one word xor-ed per moving process;
//   * the rule table: per rule, the classes of its participants.
// The whole encoding is one uint32 blob (a few KB for the networks of
// interest) that the kernels stage into shared memory -- the role the paper
// gives to texture memory (Sec. 3).

#include <algorithm>
#include <cstring>
#include <set>
#include <string>

#include "gx_internal.h"

namespace gx {

static thread_local std::string g_last_error;

gx_status fail(gx_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}
void clear_error() { g_last_error.clear(); }

void pack_host(const Net& net, const uint32_t* local, uint32_t* words) {
  for (uint32_t w = 0; w < kMaxWords; ++w) words[w] = w < net.slot_words ? kTag : 0;
  for (uint32_t p = 0; p < net.n_procs; ++p)
    words[net.field_word[p]] |= local[p] << net.field_shift[p];
}

void unpack_host(const Net& net, const uint32_t* words, uint32_t* local) {
  for (uint32_t p = 0; p < net.n_procs; ++p)
    local[p] = (words[net.field_word[p]] >> net.field_shift[p]) & ((1u << net.field_bits[p]) - 1);
}

static uint32_t bits_for(uint32_t n_states) {
  uint32_t b = 1;
  while ((1ull << b) < n_states) ++b;
  return b;
}

static gx_status encode(const gx_net_desc* d, Net& net) {
  if (!d) return fail(GX_ERR_INVALID, "desc is NULL");
  if (d->n_procs == 0) return fail(GX_ERR_INVALID, "network has no process");
  if (d->n_procs > 124) return fail(GX_ERR_INVALID, "more than 124 processes cannot fit 4 words");
  if (!d->procs) return fail(GX_ERR_INVALID, "procs is NULL");
  if (d->n_rules && !d->rules) return fail(GX_ERR_INVALID, "rules is NULL");
  const uint32_t n = d->n_procs;
  net.n_procs = n;
  net.n_labels = d->n_labels;
  net.n_states.resize(n);
  net.initial.resize(n);
  net.field_word.resize(n);
  net.field_shift.resize(n);
  net.field_bits.resize(n);

  // --- vector layout
  uint32_t word = 0, shift = 0;
  for (uint32_t p = 0; p < n; ++p) {
    const gx_lts& P = d->procs[p];
    if (P.n_states == 0) return fail(GX_ERR_INVALID, "process " + std::to_string(p) + " has no state");
    if (P.n_states > (1u << 30)) return fail(GX_ERR_INVALID, "process " + std::to_string(p) + " has too many states");
    if (P.initial >= P.n_states) return fail(GX_ERR_INVALID, "process " + std::to_string(p) + ": initial state out of range");
    if (P.n_edges && (!P.src || !P.label || !P.dst))
      return fail(GX_ERR_INVALID, "process " + std::to_string(p) + ": edge arrays are NULL");
    for (uint32_t e = 0; e < P.n_edges; ++e) {
      if (P.src[e] >= P.n_states || P.dst[e] >= P.n_states)
        return fail(GX_ERR_INVALID, "process " + std::to_string(p) + ": edge " + std::to_string(e) + " state out of range");
      if (P.label[e] >= d->n_labels)
        return fail(GX_ERR_INVALID, "process " + std::to_string(p) + ": edge " + std::to_string(e) + " label out of range");
    }
    net.n_states[p] = P.n_states;
    net.initial[p] = P.initial;
    net.n_edges += P.n_edges;
    uint32_t b = bits_for(P.n_states);
    if (shift + b > kPayloadBits) {
      ++word;
      shift = 0;
    }
    net.field_word[p] = word;
    net.field_shift[p] = shift;
    net.field_bits[p] = b;
    shift += b;
  }
  net.vector_words = word + 1;
  if (net.vector_words > kMaxWords)
    return fail(GX_ERR_INVALID, "state vector needs " + std::to_string(net.vector_words) +
                                    " words; at most 4 are supported (31 payload bits each)");
  net.slot_words = net.vector_words == 3 ? 4 : net.vector_words;

  // --- rules and the (process, label) pairs they use
  std::vector<std::set<uint32_t>> rule_labels(n);
  net.max_rule_parts = 0;
  for (uint32_t r = 0; r < d->n_rules; ++r) {
    const gx_rule& R = d->rules[r];
    if (R.n_parts == 0) return fail(GX_ERR_INVALID, "rule " + std::to_string(r) + " is empty");
    if (!R.proc || !R.label) return fail(GX_ERR_INVALID, "rule " + std::to_string(r) + ": arrays are NULL");
    std::set<uint32_t> seen;
    for (uint32_t j = 0; j < R.n_parts; ++j) {
      if (R.proc[j] >= n) return fail(GX_ERR_INVALID, "rule " + std::to_string(r) + ": process out of range");
      if (R.label[j] >= d->n_labels) return fail(GX_ERR_INVALID, "rule " + std::to_string(r) + ": label out of range");
      if (!seen.insert(R.proc[j]).second)
        return fail(GX_ERR_INVALID, "rule " + std::to_string(r) + ": a process takes part twice");
      rule_labels[R.proc[j]].insert(R.label[j]);
    }
    if (R.n_parts > net.max_rule_parts) net.max_rule_parts = R.n_parts;
  }
  if (net.max_rule_parts > 16) return fail(GX_ERR_INVALID, "rules with more than 16 participants are not supported");

  // --- edge classes: [0, n) local, then one per (process, rule label) pair
  struct Cls { uint32_t proc; int64_t label; };  // label -1 = local class
  std::vector<Cls> classes;
  for (uint32_t p = 0; p < n; ++p) classes.push_back({p, -1});
  std::vector<std::vector<std::pair<uint32_t, uint32_t>>> class_of(n);  // (label, class)
  for (uint32_t p = 0; p < n; ++p)
    for (uint32_t a : rule_labels[p]) {
      class_of[p].push_back({a, (uint32_t)classes.size()});
      classes.push_back({p, (int64_t)a});
    }
  auto find_class = [&](uint32_t p, uint32_t a) -> uint32_t {
    for (auto& pr : class_of[p])
      if (pr.first == a) return pr.second;
    return 0xFFFFFFFFu;
  };

  // --- blob
  NetBlobLayout& L = net.lay;
  L.n_procs = n;
  L.n_classes = (uint32_t)classes.size();
  L.n_rules = d->n_rules;
  std::vector<uint32_t> proc_word(n), proc_shift(n), proc_mask(n), cls_proc, cls_base, coff, cdelta,
      rule_off{0}, rule_cls;
  for (uint32_t p = 0; p < n; ++p) {
    proc_word[p] = net.field_word[p];
    proc_shift[p] = net.field_shift[p];
    proc_mask[p] = (net.field_bits[p] >= 32) ? 0xFFFFFFFFu : ((1u << net.field_bits[p]) - 1);
  }
  for (const Cls& c : classes) {
    const gx_lts& P = d->procs[c.proc];
    cls_proc.push_back(c.proc);
    cls_base.push_back((uint32_t)coff.size());
    // bucket edges by source state, keeping input order within a state
    std::vector<std::vector<uint32_t>> by_src(P.n_states);
    for (uint32_t e = 0; e < P.n_edges; ++e) {
      bool in_rule = rule_labels[c.proc].count(P.label[e]) != 0;
      bool take = c.label < 0 ? !in_rule : (P.label[e] == (uint32_t)c.label);
      if (take) by_src[P.src[e]].push_back((P.src[e] ^ P.dst[e]) << net.field_shift[c.proc]);
    }
    for (uint32_t s = 0; s < P.n_states; ++s) {
      coff.push_back((uint32_t)cdelta.size());
      for (uint32_t x : by_src[s]) cdelta.push_back(x);
    }
    coff.push_back((uint32_t)cdelta.size());
  }
  for (uint32_t r = 0; r < d->n_rules; ++r) {
    const gx_rule& R = d->rules[r];
    for (uint32_t j = 0; j < R.n_parts; ++j) rule_cls.push_back(find_class(R.proc[j], R.label[j]));
    rule_off.push_back((uint32_t)rule_cls.size());
  }
  // --- successor bound (sizes buffers that hold one batch's new states)
  std::vector<uint64_t> cls_maxdeg(classes.size(), 0);
  for (size_t c = 0; c < classes.size(); ++c) {
    const uint32_t ns = d->procs[classes[c].proc].n_states;
    for (uint32_t s = 0; s < ns; ++s)
      cls_maxdeg[c] = std::max<uint64_t>(cls_maxdeg[c], coff[cls_base[c] + s + 1] - coff[cls_base[c] + s]);
  }
  constexpr uint64_t kSuccCap = 1ull << 40;
  uint64_t bound = 0;
  for (uint32_t p = 0; p < n; ++p) bound += cls_maxdeg[p];
  for (uint32_t r = 0; r < d->n_rules; ++r) {
    uint64_t prod = 1;
    for (uint32_t j = rule_off[r]; j < rule_off[r + 1]; ++j) {
      const uint64_t m = cls_maxdeg[rule_cls[j]];
      prod = (m && prod > kSuccCap / m) ? kSuccCap : prod * m;
    }
    bound = std::min(kSuccCap, bound + prod);
  }
  // The kernels count one state's successors, and a rule's combinations, in 32 bits.
  if (bound > 0xFFFFFFFFull) return fail(GX_ERR_INVALID, "a state can have 2^32 or more successors");
  net.max_succ = bound;
  std::vector<uint32_t>& B = net.blob;
  B.clear();
  auto put = [&](const std::vector<uint32_t>& v) {
    uint32_t at = (uint32_t)B.size();
    B.insert(B.end(), v.begin(), v.end());
    return at;
  };
  L.proc_word = put(proc_word);
  L.proc_shift = put(proc_shift);
  L.proc_mask = put(proc_mask);
  L.cls_proc = put(cls_proc);
  L.cls_base = put(cls_base);
  L.coff = put(coff);
  L.cdelta = put(cdelta);
  L.rule_off = put(rule_off);
  L.rule_cls = put(rule_cls);
  while (B.size() % 4) B.push_back(0);  // 16-byte multiple for vectorised staging
  L.total = (uint32_t)B.size();

  pack_host(net, net.initial.data(), net.init_vec);
  return GX_OK;
}

}  // namespace gx

extern "C" {

const char* gx_last_error(void) { return gx::g_last_error.c_str(); }

gx_status gx_load_network(const gx_net_desc* desc, gx_net** out) {
  gx::clear_error();
  if (!out) return gx::fail(GX_ERR_INVALID, "out is NULL");
  gx_net* h = new gx_net();
  gx_status st = gx::encode(desc, h->net);
  if (st != GX_OK) {
    delete h;
    return st;
  }
  *out = h;
  return GX_OK;
}

void gx_free(gx_net* net) { delete net; }

gx_status gx_layout(const gx_net* h, uint32_t* vector_words, uint32_t* field_word,
                    uint32_t* field_offset, uint32_t* field_bits) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  const gx::Net& n = h->net;
  if (vector_words) *vector_words = n.slot_words;
  for (uint32_t p = 0; p < n.n_procs; ++p) {
    if (field_word) field_word[p] = n.field_word[p];
    if (field_offset) field_offset[p] = n.field_shift[p];
    if (field_bits) field_bits[p] = n.field_bits[p];
  }
  return GX_OK;
}

gx_status gx_default_opts(gx_explore_opts* o) {
  gx::clear_error();
  if (!o) return gx::fail(GX_ERR_INVALID, "opts is NULL");
  std::memset(o, 0, sizeof(*o));
  o->bucket_words = 8;
  o->hash_rounds = 8;
  o->deadlock_cap = 1024;
  o->warp_cache_log2 = 0xFFFFFFFFu;    // automatic: see gx_explore_opts
  o->global_cache_log2 = 0xFFFFFFFFu;
  return GX_OK;
}

}  // extern "C"

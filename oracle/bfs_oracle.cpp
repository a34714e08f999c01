// TEST INFRASTRUCTURE ONLY -- the CPU oracle for the exploration path.
//
// Only the tests, the smoke check and the bench's CPU-baseline leg may load
// this library.  It shares no code, header or table with the CUDA path: it
// has its own state representation (one byte or one uint16 per process, in a
// std::string), its own successor enumeration and a std::unordered_set as the
// visited set.  It is deliberately plain and single-threaded.
//
// What it computes (Sec. 3, "GPUs and GPUexplore"):
//   * the synchronous product of a network of LTSs (Fig. 1): a global state
//     is one local state per process;
//   * a (process, label) pair that occurs in some synchronisation rule only
//     moves inside that rule; every other edge moves its process alone
//     (the reading under which Fig. 1 has 8 states and 24 transitions);
//   * a rule fires when every participant has an edge with its label from
//     its current local state; each combination of such edges is one
//     transition (the Cartesian product);
//   * breadth-first exploration from the initial state, level by level
//     (Sec. 4: the hash table keeps the open and closed sets of a BFS);
//   * transitions are counted with multiplicity over explored states, and a
//     state with no outgoing transition is a deadlock (Sec. 1/3, on-the-fly
//     deadlock checking);
//   * safety checking (Sec. 3: the negation of a safety property is added to
//     the network as one more automaton): an explored state whose watched
//     process is in the watched local state -- the automaton's error state --
//     is a violation.
//
// Digest of a state set (a definition shared by specification with the GPU
// path, implemented here on its own): for a global state with local states
// s_0..s_{n-1},
//     h = 0;  for p in 0..n-1:  h = sm64(h ^ ((uint64)p << 32 | s_p))
// where sm64 is the splitmix64 output function (Steele, Lea & Flood 2014):
//     z = x + 0x9E3779B97F4A7C15; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
//     z = (z ^ z>>27) * 0x94D049BB133111EB; return z ^ z>>31.
// A set's digest is (count, sum of h mod 2^64, xor of h); it does not depend
// on the order in which the states are found.

#include <chrono>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

struct Edge {
  uint32_t src, label, dst;
};

struct Net {
  uint32_t n_procs = 0, n_labels = 0;
  std::vector<uint32_t> n_states, initial;
  std::vector<std::vector<Edge>> edges;                                  // per process
  std::vector<std::vector<std::pair<uint32_t, uint32_t>>> rules;         // (proc, label)
  std::vector<std::vector<char>> label_in_rule;                          // [proc][label]
  int width = 1;                                                         // bytes per process
};

uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint32_t get_local(const Net& net, const std::string& key, uint32_t p) {
  if (net.width == 1) return (uint8_t)key[p];
  return (uint32_t)(uint8_t)key[2 * p] | ((uint32_t)(uint8_t)key[2 * p + 1] << 8);
}

void set_local(const Net& net, std::string& key, uint32_t p, uint32_t s) {
  if (net.width == 1) {
    key[p] = (char)(uint8_t)s;
  } else {
    key[2 * p] = (char)(uint8_t)(s & 0xFF);
    key[2 * p + 1] = (char)(uint8_t)(s >> 8);
  }
}

uint64_t state_digest(const Net& net, const std::string& key) {
  uint64_t h = 0;
  for (uint32_t p = 0; p < net.n_procs; ++p)
    h = sm64(h ^ (((uint64_t)p << 32) | get_local(net, key, p)));
  return h;
}

// All successors of `key`, with multiplicity, in a fixed order:
// first every process's edges whose label is not one of its rule labels,
// then every rule's combinations.
void successors(const Net& net, const std::string& key, std::vector<std::string>& out) {
  out.clear();
  // (i) independent moves of one process
  for (uint32_t p = 0; p < net.n_procs; ++p) {
    uint32_t s = get_local(net, key, p);
    for (const Edge& e : net.edges[p]) {
      if (e.src != s || net.label_in_rule[p][e.label]) continue;
      std::string t = key;
      set_local(net, t, p, e.dst);
      out.push_back(t);
    }
  }
  // (ii) synchronised moves: the product of the participants' matching edges
  for (const auto& rule : net.rules) {
    std::vector<std::vector<uint32_t>> choices;  // per participant: destinations
    bool enabled = true;
    for (const auto& part : rule) {
      uint32_t p = part.first, a = part.second;
      uint32_t s = get_local(net, key, p);
      std::vector<uint32_t> dsts;
      for (const Edge& e : net.edges[p])
        if (e.src == s && e.label == a) dsts.push_back(e.dst);
      if (dsts.empty()) { enabled = false; break; }
      choices.push_back(dsts);
    }
    if (!enabled) continue;
    std::vector<size_t> pick(choices.size(), 0);
    while (true) {
      std::string t = key;
      for (size_t j = 0; j < rule.size(); ++j) set_local(net, t, rule[j].first, choices[j][pick[j]]);
      out.push_back(t);
      size_t j = 0;
      while (j < pick.size() && ++pick[j] == choices[j].size()) { pick[j] = 0; ++j; }
      if (j == pick.size()) break;
    }
  }
}

int decode(Net& net, uint32_t n_procs, uint32_t n_labels, const uint32_t* n_states,
           const uint32_t* initial, const uint32_t* edge_off, const uint32_t* edges,
           uint32_t n_rules, const uint32_t* rule_off, const uint32_t* rule_parts) {
  net.n_procs = n_procs;
  net.n_labels = n_labels;
  net.n_states.assign(n_states, n_states + n_procs);
  net.initial.assign(initial, initial + n_procs);
  net.edges.assign(n_procs, {});
  uint32_t max_states = 0;
  for (uint32_t p = 0; p < n_procs; ++p) {
    if (n_states[p] == 0 || initial[p] >= n_states[p]) return 1;
    if (n_states[p] > max_states) max_states = n_states[p];
    for (uint32_t e = edge_off[p]; e < edge_off[p + 1]; ++e) {
      Edge ed{edges[3 * e], edges[3 * e + 1], edges[3 * e + 2]};
      if (ed.src >= n_states[p] || ed.dst >= n_states[p] || ed.label >= n_labels) return 1;
      net.edges[p].push_back(ed);
    }
  }
  if (max_states > 65536) return 1;
  net.width = max_states <= 256 ? 1 : 2;
  net.label_in_rule.assign(n_procs, std::vector<char>(n_labels, 0));
  net.rules.assign(n_rules, {});
  for (uint32_t r = 0; r < n_rules; ++r) {
    for (uint32_t j = rule_off[r]; j < rule_off[r + 1]; ++j) {
      uint32_t p = rule_parts[2 * j], a = rule_parts[2 * j + 1];
      if (p >= n_procs || a >= n_labels) return 1;
      for (const auto& q : net.rules[r])
        if (q.first == p) return 1;  // a process takes part at most once per rule
      net.rules[r].push_back({p, a});
      net.label_in_rule[p][a] = 1;
    }
    if (net.rules[r].empty()) return 1;
  }
  return 0;
}

std::string initial_key(const Net& net) {
  std::string key(net.n_procs * net.width, '\0');
  for (uint32_t p = 0; p < net.n_procs; ++p) set_local(net, key, p, net.initial[p]);
  return key;
}

void unpack(const Net& net, const std::string& key, uint32_t* out) {
  for (uint32_t p = 0; p < net.n_procs; ++p) out[p] = get_local(net, key, p);
}

}  // namespace

extern "C" {

typedef struct oracle_result {
  uint64_t states;              // distinct states found (all levels, incl. the last one built)
  uint64_t explored;            // states whose successors were generated
  uint64_t transitions;         // sum over explored states of |succ| (with multiplicity)
  uint64_t n_levels;            // number of BFS levels found (level 0 = {initial})
  uint64_t deadlock_count;      // explored states with no successor
  uint64_t deadlock_sum, deadlock_xor;
  uint64_t set_sum, set_xor;    // digest of every state found
  int64_t first_deadlock_level; // -1 if none
  uint64_t complete;            // 1 if the search ran to the end (no early stop)
  double seconds;               // wall time of the search itself
  uint64_t violation_count;     // explored states with local state watch_state in watch_proc
  uint64_t violation_sum, violation_xor;
  int64_t first_violation_level; // -1 if none
} oracle_result;

// Breadth-first exploration.  stop_at_first_deadlock: finish the level in
// which the first deadlock was met, then stop.  max_explored: stop after the
// level during which this many states had been explored (0 = no limit);
// used only to time a bounded sample.  levels_out[k] = size of level k;
// deadlocks_out receives up to deadlocks_cap deadlock states (n_procs local
// states each), in discovery order.  watch_proc < n_procs turns on the
// safety check (violations_out as deadlocks_out); stop_at_first_violation
// finishes the level of the first violation, then stops.
int oracle_explore(uint32_t n_procs, uint32_t n_labels, const uint32_t* n_states,
                   const uint32_t* initial, const uint32_t* edge_off, const uint32_t* edges,
                   uint32_t n_rules, const uint32_t* rule_off, const uint32_t* rule_parts,
                   uint32_t stop_at_first_deadlock, uint64_t max_explored,
                   oracle_result* res, uint64_t* levels_out, uint32_t levels_cap,
                   uint32_t* deadlocks_out, uint32_t deadlocks_cap,
                   uint32_t watch_proc, uint32_t watch_state, uint32_t stop_at_first_violation,
                   uint32_t* violations_out, uint32_t violations_cap) {
  Net net;
  if (decode(net, n_procs, n_labels, n_states, initial, edge_off, edges, n_rules, rule_off,
             rule_parts))
    return 1;
  std::memset(res, 0, sizeof(*res));
  res->first_deadlock_level = -1;
  res->first_violation_level = -1;
  auto t0 = std::chrono::steady_clock::now();

  std::unordered_set<std::string> visited;
  std::vector<std::string> level{initial_key(net)}, next, succ;
  visited.insert(level[0]);
  uint64_t set_sum = 0, set_xor = 0;
  {
    uint64_t h = state_digest(net, level[0]);
    set_sum += h;
    set_xor ^= h;
  }
  std::vector<uint64_t> sizes;
  bool stop = false;
  while (!level.empty()) {
    sizes.push_back(level.size());
    if (stop) break;
    next.clear();
    for (const std::string& s : level) {
      successors(net, s, succ);
      res->explored++;
      res->transitions += succ.size();
      if (succ.empty()) {
        uint64_t h = state_digest(net, s);
        if (res->deadlock_count < deadlocks_cap) unpack(net, s, deadlocks_out + res->deadlock_count * n_procs);
        res->deadlock_count++;
        res->deadlock_sum += h;
        res->deadlock_xor ^= h;
        if (res->first_deadlock_level < 0) res->first_deadlock_level = (int64_t)sizes.size() - 1;
      }
      if (watch_proc < n_procs && get_local(net, s, watch_proc) == watch_state) {
        uint64_t h = state_digest(net, s);
        if (res->violation_count < violations_cap)
          unpack(net, s, violations_out + res->violation_count * n_procs);
        res->violation_count++;
        res->violation_sum += h;
        res->violation_xor ^= h;
        if (res->first_violation_level < 0) res->first_violation_level = (int64_t)sizes.size() - 1;
      }
      for (const std::string& t : succ) {
        if (visited.insert(t).second) {
          uint64_t h = state_digest(net, t);
          set_sum += h;
          set_xor ^= h;
          next.push_back(t);
        }
      }
    }
    if (stop_at_first_deadlock && res->deadlock_count > 0) stop = true;
    if (stop_at_first_violation && res->violation_count > 0) stop = true;
    if (max_explored && res->explored >= max_explored) stop = true;
    level.swap(next);
  }
  res->complete = level.empty() ? 1 : 0;
  auto t1 = std::chrono::steady_clock::now();
  res->seconds = std::chrono::duration<double>(t1 - t0).count();
  res->states = visited.size();
  res->n_levels = sizes.size();
  res->set_sum = set_sum;
  res->set_xor = set_xor;
  for (size_t k = 0; k < sizes.size() && k < levels_cap; ++k) levels_out[k] = sizes[k];
  return 0;
}

// Digest of one global state given as n local states (for replaying reported states).
uint64_t oracle_state_digest(uint32_t n_procs, const uint32_t* local) {
  uint64_t h = 0;
  for (uint32_t p = 0; p < n_procs; ++p) h = sm64(h ^ (((uint64_t)p << 32) | local[p]));
  return h;
}

// Successors of one global state (local states in `state`), with multiplicity.
// Writes up to cap successors (n_procs local states each) and returns the
// full count, or -1 on an invalid network.
int64_t oracle_successors(uint32_t n_procs, uint32_t n_labels, const uint32_t* n_states,
                          const uint32_t* initial, const uint32_t* edge_off, const uint32_t* edges,
                          uint32_t n_rules, const uint32_t* rule_off, const uint32_t* rule_parts,
                          const uint32_t* state, uint32_t* out, uint64_t cap) {
  Net net;
  if (decode(net, n_procs, n_labels, n_states, initial, edge_off, edges, n_rules, rule_off,
             rule_parts))
    return -1;
  std::string key(net.n_procs * net.width, '\0');
  for (uint32_t p = 0; p < n_procs; ++p) {
    if (state[p] >= n_states[p]) return -1;
    set_local(net, key, p, state[p]);
  }
  std::vector<std::string> succ;
  successors(net, key, succ);
  for (size_t i = 0; i < succ.size() && i < cap; ++i) unpack(net, succ[i], out + i * n_procs);
  return (int64_t)succ.size();
}

// Full reachable graph and, for every reachable state, its BFS distance
// backwards to the nearest deadlock (UINT32_MAX when no deadlock is
// reachable from it).  states_out: n_procs local states per state in BFS
// discovery order; dist_out: one entry per state.  Returns the state count,
// or -1 (invalid network) / -2 (more than cap states).
int64_t oracle_deadlock_distances(uint32_t n_procs, uint32_t n_labels, const uint32_t* n_states,
                                  const uint32_t* initial, const uint32_t* edge_off,
                                  const uint32_t* edges, uint32_t n_rules, const uint32_t* rule_off,
                                  const uint32_t* rule_parts, uint32_t* states_out,
                                  uint32_t* dist_out, uint64_t cap) {
  Net net;
  if (decode(net, n_procs, n_labels, n_states, initial, edge_off, edges, n_rules, rule_off,
             rule_parts))
    return -1;
  std::unordered_map<std::string, uint64_t> index;
  std::vector<std::string> order{initial_key(net)};
  index.emplace(order[0], 0);
  std::vector<std::vector<uint64_t>> preds(1);
  std::vector<uint64_t> deadlocks, succ_idx;
  std::vector<std::string> succ;
  for (uint64_t i = 0; i < order.size(); ++i) {
    if (order.size() > cap) return -2;
    std::string s = order[i];
    successors(net, s, succ);
    if (succ.empty()) deadlocks.push_back(i);
    for (const std::string& t : succ) {
      auto it = index.find(t);
      uint64_t j;
      if (it == index.end()) {
        j = order.size();
        index.emplace(t, j);
        order.push_back(t);
        preds.emplace_back();
      } else {
        j = it->second;
      }
      preds[j].push_back(i);
    }
  }
  if (order.size() > cap) return -2;
  std::vector<uint32_t> dist(order.size(), UINT32_MAX);
  std::vector<uint64_t> queue;
  for (uint64_t d : deadlocks) {
    dist[d] = 0;
    queue.push_back(d);
  }
  for (size_t q = 0; q < queue.size(); ++q) {
    uint64_t v = queue[q];
    for (uint64_t u : preds[v])
      if (dist[u] == UINT32_MAX) {
        dist[u] = dist[v] + 1;
        queue.push_back(u);
      }
  }
  for (uint64_t i = 0; i < order.size(); ++i) {
    unpack(net, order[i], states_out + i * n_procs);
    dist_out[i] = dist[i];
  }
  return (int64_t)order.size();
}

}  // extern "C"

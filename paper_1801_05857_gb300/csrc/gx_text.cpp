// Text front end: networks in the paper's input format (Sec. 3, Fig. 1).
//
// A network is an EXP.OPEN composition of LTS files:
//
//     par using
//         send * rec * _   -> trans,
//         send * _   * rec -> trans
//     in
//         "producer.aut" || "consumer.aut" || "consumer.aut"
//     end par
//
// Each synchronisation vector has one entry per process: a label, or '_'
// when the process does not take part; the label after '->' names the
// result.  Each file is an LTS in Aldebaran format:
//
//     des (initial, n_transitions, n_states)
//     (src, "label", dst)
//     ...
//
// Labels are global strings (the same text in two files is the same label);
// quotes are optional around labels without commas, quotes or parentheses.
// A (process, label) pair that occurs in some vector moves only through
// vectors; every other transition of a process interleaves (the reading under
// which Fig. 1 has 8 states and 24 transitions).  Comments (* ... *) may
// appear anywhere in the composition.  The result is encoded by the same path
// as gx_load_network.

#include <algorithm>
#include <cctype>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "gx_internal.h"

namespace gx {
namespace {

struct Cursor {
  const char* s;
  size_t i = 0, n = 0;
  int line = 1;
  std::string what;  // file name for messages

  explicit Cursor(const char* text, std::string name) : s(text), n(std::strlen(text)), what(std::move(name)) {}

  std::string where() const { return what + " line " + std::to_string(line); }
  bool eof() const { return i >= n; }
  char peek() const { return i < n ? s[i] : '\0'; }
  void bump() {
    if (s[i] == '\n') ++line;
    ++i;
  }
  // whitespace and (* ... *) comments; false on an unterminated comment
  bool skip(bool comments) {
    while (i < n) {
      if (std::isspace((unsigned char)s[i])) {
        bump();
      } else if (comments && s[i] == '(' && i + 1 < n && s[i + 1] == '*') {
        i += 2;
        while (i + 1 < n && !(s[i] == '*' && s[i + 1] == ')')) bump();
        if (i + 1 >= n) return false;
        i += 2;
      } else {
        break;
      }
    }
    return true;
  }
  bool eat(char c) {
    if (peek() != c) return false;
    bump();
    return true;
  }
  bool eat(const char* w) {
    const size_t k = std::strlen(w);
    if (i + k > n || std::strncmp(s + i, w, k) != 0) return false;
    i += k;
    return true;
  }
  bool keyword(const char* w) {  // w followed by a non-identifier character
    const size_t k = std::strlen(w);
    if (i + k > n || std::strncmp(s + i, w, k) != 0) return false;
    if (i + k < n && (std::isalnum((unsigned char)s[i + k]) || s[i + k] == '_')) return false;
    i += k;
    return true;
  }
  bool number(uint64_t& v) {
    if (!std::isdigit((unsigned char)peek())) return false;
    v = 0;
    while (std::isdigit((unsigned char)peek())) {
      v = v * 10 + (uint64_t)(s[i] - '0');
      if (v > 0xFFFFFFFFull) return false;
      ++i;
    }
    return true;
  }
  bool quoted(std::string& out) {
    if (!eat('"')) return false;
    out.clear();
    while (i < n && s[i] != '"' && s[i] != '\n') out.push_back(s[i++]);
    return eat('"');
  }
};

gx_status bad(const Cursor& c, const std::string& msg) { return fail(GX_ERR_INVALID, c.where() + ": " + msg); }

struct ParsedLts {
  uint32_t n_states = 0, initial = 0;
  std::vector<uint32_t> src, label, dst;
};

struct Labels {
  std::map<std::string, uint32_t> id;
  std::vector<std::string> name;
  uint32_t get(const std::string& s) {
    auto it = id.find(s);
    if (it != id.end()) return it->second;
    const uint32_t k = (uint32_t)name.size();
    id.emplace(s, k);
    name.push_back(s);
    return k;
  }
};

// An unquoted .aut label: up to the next ',' on the line, trimmed.
bool aut_label(Cursor& c, std::string& out) {
  if (c.peek() == '"') return c.quoted(out);
  out.clear();
  while (!c.eof() && c.peek() != ',' && c.peek() != '\n' && c.peek() != ')' && c.peek() != '(') out.push_back(c.s[c.i++]);
  while (!out.empty() && std::isspace((unsigned char)out.back())) out.pop_back();
  return !out.empty();
}

gx_status parse_aut(Cursor& c, Labels& labels, ParsedLts& L) {
  c.skip(false);
  if (!c.keyword("des")) return bad(c, "expected 'des (initial, transitions, states)'");
  uint64_t init = 0, nt = 0, ns = 0;
  c.skip(false);
  if (!c.eat('(')) return bad(c, "expected '(' after des");
  c.skip(false);
  if (!c.number(init)) return bad(c, "expected the initial state");
  c.skip(false);
  if (!c.eat(',')) return bad(c, "expected ','");
  c.skip(false);
  if (!c.number(nt)) return bad(c, "expected the number of transitions");
  c.skip(false);
  if (!c.eat(',')) return bad(c, "expected ','");
  c.skip(false);
  if (!c.number(ns)) return bad(c, "expected the number of states");
  c.skip(false);
  if (!c.eat(')')) return bad(c, "expected ')'");
  if (ns == 0) return bad(c, "an LTS needs at least one state");
  if (init >= ns) return bad(c, "initial state " + std::to_string(init) + " is not below " + std::to_string(ns));
  L.n_states = (uint32_t)ns;
  L.initial = (uint32_t)init;
  for (uint64_t k = 0; k < nt; ++k) {
    c.skip(false);
    uint64_t a = 0, b = 0;
    std::string lab;
    if (!c.eat('(')) return bad(c, "expected transition " + std::to_string(k) + " of " + std::to_string(nt));
    c.skip(false);
    if (!c.number(a)) return bad(c, "expected a source state");
    c.skip(false);
    if (!c.eat(',')) return bad(c, "expected ','");
    c.skip(false);
    if (!aut_label(c, lab)) return bad(c, "expected a label");
    c.skip(false);
    if (!c.eat(',')) return bad(c, "expected ','");
    c.skip(false);
    if (!c.number(b)) return bad(c, "expected a target state");
    c.skip(false);
    if (!c.eat(')')) return bad(c, "expected ')'");
    if (a >= ns || b >= ns) return bad(c, "state out of range 0.." + std::to_string(ns - 1));
    L.src.push_back((uint32_t)a);
    L.label.push_back(labels.get(lab));
    L.dst.push_back((uint32_t)b);
  }
  c.skip(false);
  if (!c.eof()) return bad(c, "text after the last of the " + std::to_string(nt) + " transitions");
  return GX_OK;
}

// A label in a synchronisation vector: "quoted", an identifier, or '_'.
bool exp_label(Cursor& c, std::string& out) {
  if (c.peek() == '"') return c.quoted(out);
  out.clear();
  while (!c.eof() && (std::isalnum((unsigned char)c.peek()) || c.peek() == '_' || c.peek() == '!' ||
                      c.peek() == '?' || c.peek() == '.'))
    out.push_back(c.s[c.i++]);
  return !out.empty();
}

struct Vector {
  std::vector<std::string> entry;  // one per process, "_" = not taking part
  std::string result;
  int line;
};

gx_status parse_exp(Cursor& c, std::vector<Vector>& vecs, std::vector<std::string>& files) {
  if (!c.skip(true)) return bad(c, "unterminated comment");
  if (!c.keyword("par")) return bad(c, "expected 'par'");
  if (!c.skip(true)) return bad(c, "unterminated comment");
  if (c.keyword("using")) {
    while (true) {
      Vector v;
      while (true) {
        if (!c.skip(true)) return bad(c, "unterminated comment");
        if (v.entry.empty()) v.line = c.line;
        std::string lab;
        if (!exp_label(c, lab)) return bad(c, "expected a label or '_' in a synchronisation vector");
        v.entry.push_back(lab);
        if (!c.skip(true)) return bad(c, "unterminated comment");
        if (c.eat('*')) continue;
        if (c.eat("->")) break;
        return bad(c, "expected '*' or '->' in a synchronisation vector");
      }
      if (!c.skip(true)) return bad(c, "unterminated comment");
      if (!exp_label(c, v.result) || v.result == "_") return bad(c, "expected the result label after '->'");
      vecs.push_back(v);
      if (!c.skip(true)) return bad(c, "unterminated comment");
      if (c.eat(',')) continue;
      break;
    }
  }
  if (!c.skip(true)) return bad(c, "unterminated comment");
  if (!c.keyword("in")) return bad(c, "expected 'in'");
  while (true) {
    if (!c.skip(true)) return bad(c, "unterminated comment");
    std::string f;
    if (!c.quoted(f)) return bad(c, "expected a quoted LTS file name");
    files.push_back(f);
    if (!c.skip(true)) return bad(c, "unterminated comment");
    if (c.eat("||")) continue;
    break;
  }
  if (!c.keyword("end")) return bad(c, "expected '||' or 'end par'");
  if (!c.skip(true)) return bad(c, "unterminated comment");
  if (!c.keyword("par")) return bad(c, "expected 'par' after 'end'");
  if (!c.skip(true)) return bad(c, "unterminated comment");
  if (!c.eof()) return bad(c, "text after 'end par'");
  return GX_OK;
}

}  // namespace
}  // namespace gx

extern "C" {

gx_status gx_load_exp(const char* exp_text, uint32_t n_files, const char* const* file_names,
                      const char* const* file_texts, gx_net** out) {
  using namespace gx;
  clear_error();
  if (!exp_text || !out) return fail(GX_ERR_INVALID, "exp_text or out is NULL");
  if (n_files && (!file_names || !file_texts)) return fail(GX_ERR_INVALID, "file arrays are NULL");
  Cursor c(exp_text, "composition");
  std::vector<Vector> vecs;
  std::vector<std::string> files;
  gx_status st = parse_exp(c, vecs, files);
  if (st != GX_OK) return st;
  const uint32_t n = (uint32_t)files.size();
  for (const Vector& v : vecs)
    if (v.entry.size() != n)
      return fail(GX_ERR_INVALID, "composition line " + std::to_string(v.line) + ": synchronisation vector has " +
                                      std::to_string(v.entry.size()) + " entries for " + std::to_string(n) +
                                      " processes");
  // each referenced file is parsed once; processes that name the same file share it
  Labels labels;
  std::map<std::string, ParsedLts> parsed;
  for (const std::string& f : files) {
    if (parsed.count(f)) continue;
    const char* text = nullptr;
    for (uint32_t k = 0; k < n_files; ++k)
      if (file_names[k] && f == file_names[k]) text = file_texts[k];
    if (!text) return fail(GX_ERR_INVALID, "composition names \"" + f + "\", which was not given");
    Cursor fc(text, f);
    ParsedLts L;
    if ((st = parse_aut(fc, labels, L)) != GX_OK) return st;
    parsed.emplace(f, std::move(L));
  }
  std::vector<uint32_t> rproc, rlab;
  std::vector<std::pair<size_t, size_t>> rspan;
  std::vector<uint32_t> rresult;
  for (const Vector& v : vecs) {
    const size_t b = rproc.size();
    for (uint32_t p = 0; p < n; ++p)
      if (v.entry[p] != "_") {
        rproc.push_back(p);
        rlab.push_back(labels.get(v.entry[p]));
      }
    if (rproc.size() == b)
      return fail(GX_ERR_INVALID, "composition line " + std::to_string(v.line) + ": vector without participants");
    rspan.push_back({b, rproc.size() - b});
    rresult.push_back(labels.get(v.result));
  }
  std::vector<gx_lts> procs(n);
  for (uint32_t p = 0; p < n; ++p) {
    const ParsedLts& L = parsed.at(files[p]);
    procs[p] = gx_lts{L.n_states, (uint32_t)L.src.size(), L.initial, L.src.data(), L.label.data(), L.dst.data()};
  }
  std::vector<gx_rule> rules(vecs.size());
  for (size_t r = 0; r < vecs.size(); ++r)
    rules[r] = gx_rule{(uint32_t)rspan[r].second, rproc.data() + rspan[r].first, rlab.data() + rspan[r].first,
                       rresult[r]};
  gx_net_desc d{n, (uint32_t)labels.name.size(), procs.data(), (uint32_t)rules.size(), rules.data()};
  gx_net* h = nullptr;
  if ((st = gx_load_network(&d, &h)) != GX_OK) return st;
  h->label_names = labels.name;
  *out = h;
  return GX_OK;
}

gx_status gx_label_name(const gx_net* h, uint32_t label, char* buf, uint32_t cap, uint32_t* len) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  if (label >= h->net.n_labels) return gx::fail(GX_ERR_INVALID, "label out of range");
  const std::string name = label < h->label_names.size() ? h->label_names[label] : std::to_string(label);
  if (len) *len = (uint32_t)name.size();
  if (cap) {
    if (!buf) return gx::fail(GX_ERR_INVALID, "buf is NULL");
    const size_t k = std::min<size_t>(name.size(), cap - 1);
    std::memcpy(buf, name.data(), k);
    buf[k] = '\0';
  }
  return GX_OK;
}

gx_status gx_network_counts(const gx_net* h, uint32_t* n_procs, uint32_t* n_labels, uint32_t* n_rules,
                            uint64_t* n_edges) {
  gx::clear_error();
  if (!h) return gx::fail(GX_ERR_INVALID, "net is NULL");
  if (n_procs) *n_procs = h->net.n_procs;
  if (n_labels) *n_labels = h->net.n_labels;
  if (n_rules) *n_rules = h->net.lay.n_rules;
  if (n_edges) *n_edges = h->net.n_edges;
  return GX_OK;
}

}  // extern "C"

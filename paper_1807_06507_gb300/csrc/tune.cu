// tune.cu -- the tune cache: launch parameters chosen by the autotuner
// (paper_1807_06507_gb300/autotune.py) per (device, plan kind, ndim, dtype,
// window), stored as JSON and read by the plans.
//
// File format ("format": "swcorr-tune-1"):
//   {"format": "swcorr-tune-1",
//    "entries": [{"device": "NVIDIA GB300", "kind": "plain", "ndim": 2,
//                 "dtype": "u16", "k": [7, 7], "prefetch": 4,
//                 "tile_rows": 28, "ctas_per_sm": 16, ...}, ...]}
// Unknown keys are ignored.  A file that does not parse, or an entry with a
// value out of range, is rejected as a whole: plans then use the built-in
// defaults.  Host code only.
#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "hostapi.h"

namespace swc {
namespace {

// ---------------------------------------------------------------- JSON
struct JVal {
  enum Kind { NUL, BOOL, NUM, STR, ARR, OBJ } kind = NUL;
  double num = 0.0;
  bool b = false;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
  const JVal* get(const char* key) const {
    for (const auto& kv : obj)
      if (kv.first == key) return &kv.second;
    return nullptr;
  }
};

class JParser {
 public:
  explicit JParser(const std::string& s) : s_(s) {}
  bool parse(JVal* out) {
    if (!value(out, 0)) return false;
    ws();
    return i_ == s_.size();
  }

 private:
  const std::string& s_;
  size_t i_ = 0;
  void ws() {
    while (i_ < s_.size() && std::isspace((unsigned char)s_[i_])) i_++;
  }
  bool lit(const char* w) {
    const size_t n = std::strlen(w);
    if (s_.compare(i_, n, w) != 0) return false;
    i_ += n;
    return true;
  }
  bool string(std::string* out) {
    if (i_ >= s_.size() || s_[i_] != '"') return false;
    i_++;
    out->clear();
    while (i_ < s_.size() && s_[i_] != '"') {
      char c = s_[i_++];
      if (c == '\\') {
        if (i_ >= s_.size()) return false;
        const char e = s_[i_++];
        switch (e) {
          case '"': c = '"'; break;
          case '\\': c = '\\'; break;
          case '/': c = '/'; break;
          case 'n': c = '\n'; break;
          case 't': c = '\t'; break;
          case 'r': c = '\r'; break;
          case 'b': c = '\b'; break;
          case 'f': c = '\f'; break;
          case 'u':  // keep the escape verbatim (names here are ASCII)
            if (i_ + 4 > s_.size()) return false;
            out->append("\\u");
            out->append(s_, i_, 4);
            i_ += 4;
            continue;
          default: return false;
        }
      } else if ((unsigned char)c < 0x20) {
        return false;
      }
      out->push_back(c);
    }
    if (i_ >= s_.size()) return false;
    i_++;
    return true;
  }
  bool number(double* out) {
    const char* b = s_.c_str() + i_;
    char* e = nullptr;
    *out = std::strtod(b, &e);
    if (e == b) return false;
    i_ += (size_t)(e - b);
    return true;
  }
  bool value(JVal* v, int depth) {
    if (depth > 32) return false;
    ws();
    if (i_ >= s_.size()) return false;
    const char c = s_[i_];
    if (c == '{') {
      v->kind = JVal::OBJ;
      i_++;
      ws();
      if (i_ < s_.size() && s_[i_] == '}') {
        i_++;
        return true;
      }
      while (true) {
        ws();
        std::string key;
        if (!string(&key)) return false;
        ws();
        if (i_ >= s_.size() || s_[i_] != ':') return false;
        i_++;
        JVal child;
        if (!value(&child, depth + 1)) return false;
        v->obj.emplace_back(std::move(key), std::move(child));
        ws();
        if (i_ < s_.size() && s_[i_] == ',') {
          i_++;
          continue;
        }
        if (i_ < s_.size() && s_[i_] == '}') {
          i_++;
          return true;
        }
        return false;
      }
    }
    if (c == '[') {
      v->kind = JVal::ARR;
      i_++;
      ws();
      if (i_ < s_.size() && s_[i_] == ']') {
        i_++;
        return true;
      }
      while (true) {
        JVal child;
        if (!value(&child, depth + 1)) return false;
        v->arr.push_back(std::move(child));
        ws();
        if (i_ < s_.size() && s_[i_] == ',') {
          i_++;
          continue;
        }
        if (i_ < s_.size() && s_[i_] == ']') {
          i_++;
          return true;
        }
        return false;
      }
    }
    if (c == '"') {
      v->kind = JVal::STR;
      return string(&v->str);
    }
    if (lit("true")) {
      v->kind = JVal::BOOL;
      v->b = true;
      return true;
    }
    if (lit("false")) {
      v->kind = JVal::BOOL;
      return true;
    }
    if (lit("null")) {
      v->kind = JVal::NUL;
      return true;
    }
    v->kind = JVal::NUM;
    return number(&v->num);
  }
};

// ---------------------------------------------------------------- cache
struct Entry {
  std::string device;
  std::string kind;  // "plain" or "batched"
  int ndim = 0;
  int dtype = 0;
  std::vector<int> k;
  swcorr_tune tune{};
};

std::mutex g_mu;
bool g_loaded = false;            // a load was attempted (file or env)
std::vector<Entry> g_entries;

bool int_field(const JVal& o, const char* key, int lo, int hi, int* out, bool required) {
  const JVal* v = o.get(key);
  if (!v) {
    if (required) return false;
    *out = 0;
    return true;
  }
  if (v->kind != JVal::NUM || v->num != (double)(long long)v->num || v->num < lo || v->num > hi) return false;
  *out = (int)v->num;
  return true;
}

// Parses the whole file; on any error returns false and leaves *out empty.
bool parse_file(const std::string& text, std::vector<Entry>* out, std::string* why) {
  JVal root;
  if (!JParser(text).parse(&root) || root.kind != JVal::OBJ) {
    *why = "not a JSON object";
    return false;
  }
  const JVal* fmt = root.get("format");
  if (!fmt || fmt->kind != JVal::STR || fmt->str != "swcorr-tune-1") {
    *why = "missing \"format\": \"swcorr-tune-1\"";
    return false;
  }
  const JVal* ents = root.get("entries");
  if (!ents || ents->kind != JVal::ARR) {
    *why = "missing \"entries\" array";
    return false;
  }
  std::vector<Entry> res;
  for (size_t i = 0; i < ents->arr.size(); i++) {
    const JVal& o = ents->arr[i];
    Entry e;
    const JVal* dev = o.get("device");
    const JVal* kind = o.get("kind");
    const JVal* dt = o.get("dtype");
    const JVal* k = o.get("k");
    if (o.kind != JVal::OBJ || !dev || dev->kind != JVal::STR || !dt || dt->kind != JVal::STR || !k ||
        k->kind != JVal::ARR) {
      *why = "entry " + std::to_string(i) + ": needs device, dtype and k";
      return false;
    }
    e.device = dev->str;
    e.kind = (kind && kind->kind == JVal::STR) ? kind->str : "plain";
    if (e.kind != "plain" && e.kind != "batched") {
      *why = "entry " + std::to_string(i) + ": kind must be plain or batched";
      return false;
    }
    if (dt->str == "u16") {
      e.dtype = SWCORR_U16;
    } else if (dt->str == "f32") {
      e.dtype = SWCORR_F32;
    } else {
      *why = "entry " + std::to_string(i) + ": dtype must be u16 or f32";
      return false;
    }
    if (!int_field(o, "ndim", 1, 3, &e.ndim, true) || (int)k->arr.size() != e.ndim) {
      *why = "entry " + std::to_string(i) + ": ndim must be 1..3 with one k per dimension";
      return false;
    }
    for (const JVal& kv : k->arr) {
      if (kv.kind != JVal::NUM || kv.num != (double)(long long)kv.num || kv.num < 0 || kv.num > 1e9) {
        *why = "entry " + std::to_string(i) + ": bad k";
        return false;
      }
      e.k.push_back((int)kv.num);
    }
    if (!int_field(o, "prefetch", 0, SWCORR_TUNE_MAX_PREFETCH, &e.tune.prefetch, false) ||
        !int_field(o, "tile_rows", 0, SWCORR_TUNE_MAX_TILE_ROWS, &e.tune.tile_rows, false) ||
        !int_field(o, "ctas_per_sm", 0, SWCORR_TUNE_MAX_CTAS_PER_SM, &e.tune.ctas_per_sm, false)) {
      *why = "entry " + std::to_string(i) + ": prefetch, tile_rows or ctas_per_sm out of range";
      return false;
    }
    res.push_back(std::move(e));
  }
  *out = std::move(res);
  return true;
}

swcorr_status load_locked(const char* path) {
  g_loaded = true;
  g_entries.clear();
  if (!path || !*path) return SWCORR_OK;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(SWCORR_ERR_INVALID_ARG, "tune file %s cannot be opened", path);
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) {
    text.append(buf, n);
    if (text.size() > (16u << 20)) {
      std::fclose(f);
      return fail(SWCORR_ERR_INVALID_ARG, "tune file %s is larger than 16 MiB", path);
    }
  }
  std::fclose(f);
  std::string why;
  std::vector<Entry> ents;
  if (!parse_file(text, &ents, &why)) return fail(SWCORR_ERR_INVALID_ARG, "tune file %s ignored: %s", path, why.c_str());
  g_entries = std::move(ents);
  return SWCORR_OK;
}

void ensure_loaded_locked() {
  if (g_loaded) return;
  // a file that cannot be read or parsed leaves the defaults in force (its
  // reason stays readable through swcorr_last_error)
  load_locked(std::getenv("SWCORR_TUNE_FILE"));
}

}  // namespace

bool tune_lookup(const char* device, const char* kind, int ndim, const int32_t* k, swcorr_dtype dtype,
                 swcorr_tune* out) {
  std::lock_guard<std::mutex> lk(g_mu);
  ensure_loaded_locked();
  for (const Entry& e : g_entries) {
    if (e.kind != kind || e.ndim != ndim || e.dtype != (int)dtype) continue;
    if (device && e.device != device) continue;
    bool same = true;
    if (e.kind == "plain")  // the batched entry serves every window
      for (int d = 0; d < ndim; d++) same = same && k && e.k[d] == k[d];
    if (!same) continue;
    *out = e.tune;
    return true;
  }
  return false;
}

swcorr_status tune_check(const swcorr_tune* t) {
  if (!t) return SWCORR_OK;
  for (int i = 0; i < 5; i++)
    if (t->reserved[i] != 0) return fail(SWCORR_ERR_INVALID_ARG, "tune.reserved must be 0");
  if (t->prefetch < 0 || t->prefetch > SWCORR_TUNE_MAX_PREFETCH)
    return fail(SWCORR_ERR_INVALID_ARG, "tune.prefetch = %d outside 0..%d", t->prefetch, SWCORR_TUNE_MAX_PREFETCH);
  if (t->tile_rows < 0 || t->tile_rows > SWCORR_TUNE_MAX_TILE_ROWS)
    return fail(SWCORR_ERR_INVALID_ARG, "tune.tile_rows = %d outside 0..%d", t->tile_rows, SWCORR_TUNE_MAX_TILE_ROWS);
  if (t->ctas_per_sm < 0 || t->ctas_per_sm > SWCORR_TUNE_MAX_CTAS_PER_SM)
    return fail(SWCORR_ERR_INVALID_ARG, "tune.ctas_per_sm = %d outside 0..%d", t->ctas_per_sm,
                SWCORR_TUNE_MAX_CTAS_PER_SM);
  return SWCORR_OK;
}

}  // namespace swc

extern "C" {

swcorr_status swcorr_set_tune_file(const char* path) {
  std::lock_guard<std::mutex> lk(swc::g_mu);
  return swc::load_locked(path);
}

int swcorr_tune_lookup(const char* device, int batched, int ndim, const int32_t* k, swcorr_dtype dtype,
                       swcorr_tune* out) {
  if (!out || ndim < 1 || ndim > 3 || (!k && !batched)) return 0;
  return swc::tune_lookup(device, batched ? "batched" : "plain", ndim, k, dtype, out) ? 1 : 0;
}

}  // extern "C"

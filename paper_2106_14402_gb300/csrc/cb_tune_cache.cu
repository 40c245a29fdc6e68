// On-disk cache of autotuned tier bounds: a JSON file mapping a key
// (device name, semiring, sizing mode, size class of the operands) to the
// bounds cb_autotune found and their time, so that a later run on the same
// kind of device and workload skips the timing grid.  Host code only.
//
// File layout (written by this file; read back by the small JSON reader
// below, which accepts any well-formed JSON and then looks for this shape):
//   {"format": "cb-tune-cache-1",
//    "entries": {"<key>": {"sym_hash_max": 1024, "num_hash_max": 2048,
//                          "learn_max": 512, "cf_esc": 1.25,
//                          "cf_prereduce": 4, "ms": 12.5}, ...}}
// Updates rewrite the whole file through a temporary file and a rename, so
// a reader never sees a half-written cache.
#include <cerrno>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include <unistd.h>

#include "cb.h"

namespace {

constexpr const char* kFormat = "cb-tune-cache-1";

// ---- a minimal JSON value and reader --------------------------------------

struct JValue {
  enum Kind { kNull, kBool, kNum, kStr, kArr, kObj } kind = kNull;
  double num = 0.0;
  bool b = false;
  std::string str;
  std::vector<JValue> arr;
  std::vector<std::pair<std::string, JValue>> obj;  // in file order
  const JValue* get(const char* k) const {
    for (const auto& kv : obj)
      if (kv.first == k) return &kv.second;
    return nullptr;
  }
};

struct Reader {
  const char* p;
  const char* end;
  int depth = 0;
  void ws() {
    while (p < end && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) ++p;
  }
  bool lit(const char* s) {
    const size_t n = std::strlen(s);
    if ((size_t)(end - p) < n || std::strncmp(p, s, n) != 0) return false;
    p += n;
    return true;
  }
  bool string(std::string& out) {
    if (p >= end || *p != '"') return false;
    ++p;
    out.clear();
    while (p < end && *p != '"') {
      char c = *p++;
      if ((unsigned char)c < 0x20) return false;
      if (c == '\\') {
        if (p >= end) return false;
        const char e = *p++;
        switch (e) {
          case '"': c = '"'; break;
          case '\\': c = '\\'; break;
          case '/': c = '/'; break;
          case 'b': c = '\b'; break;
          case 'f': c = '\f'; break;
          case 'n': c = '\n'; break;
          case 'r': c = '\r'; break;
          case 't': c = '\t'; break;
          case 'u': {  // kept only for ASCII code points
            if (end - p < 4) return false;
            unsigned v = 0;
            for (int i = 0; i < 4; ++i) {
              const char h = *p++;
              v <<= 4;
              if (h >= '0' && h <= '9') v |= (unsigned)(h - '0');
              else if (h >= 'a' && h <= 'f') v |= (unsigned)(h - 'a' + 10);
              else if (h >= 'A' && h <= 'F') v |= (unsigned)(h - 'A' + 10);
              else return false;
            }
            if (v >= 0x80) return false;
            c = (char)v;
            break;
          }
          default: return false;
        }
      }
      out.push_back(c);
    }
    if (p >= end) return false;
    ++p;
    return true;
  }
  bool value(JValue& v) {
    if (++depth > 32) return false;
    ws();
    if (p >= end) return false;
    bool ok = true;
    if (*p == '{') {
      v.kind = JValue::kObj;
      ++p;
      ws();
      if (p < end && *p == '}') {
        ++p;
      } else {
        for (;;) {
          ws();
          std::string k;
          if (!string(k)) { ok = false; break; }
          ws();
          if (p >= end || *p != ':') { ok = false; break; }
          ++p;
          JValue x;
          if (!value(x)) { ok = false; break; }
          v.obj.emplace_back(std::move(k), std::move(x));
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == '}') { ++p; break; }
          ok = false;
          break;
        }
      }
    } else if (*p == '[') {
      v.kind = JValue::kArr;
      ++p;
      ws();
      if (p < end && *p == ']') {
        ++p;
      } else {
        for (;;) {
          JValue x;
          if (!value(x)) { ok = false; break; }
          v.arr.push_back(std::move(x));
          ws();
          if (p < end && *p == ',') { ++p; continue; }
          if (p < end && *p == ']') { ++p; break; }
          ok = false;
          break;
        }
      }
    } else if (*p == '"') {
      v.kind = JValue::kStr;
      ok = string(v.str);
    } else if (lit("true")) {
      v.kind = JValue::kBool;
      v.b = true;
    } else if (lit("false")) {
      v.kind = JValue::kBool;
    } else if (lit("null")) {
      v.kind = JValue::kNull;
    } else {
      // a number: JSON's grammar checked by hand, the value by strtod
      const char* s = p;
      if (p < end && *p == '-') ++p;
      const char* d0 = p;
      while (p < end && *p >= '0' && *p <= '9') ++p;
      if (p == d0) return false;
      if (p < end && *p == '.') {
        ++p;
        const char* f0 = p;
        while (p < end && *p >= '0' && *p <= '9') ++p;
        if (p == f0) return false;
      }
      if (p < end && (*p == 'e' || *p == 'E')) {
        ++p;
        if (p < end && (*p == '+' || *p == '-')) ++p;
        const char* e0 = p;
        while (p < end && *p >= '0' && *p <= '9') ++p;
        if (p == e0) return false;
      }
      v.kind = JValue::kNum;
      v.num = std::strtod(std::string(s, p).c_str(), nullptr);
    }
    --depth;
    return ok;
  }
};

bool parse(const std::string& text, JValue& out) {
  Reader r{text.data(), text.data() + text.size()};
  if (!r.value(out)) return false;
  r.ws();
  return r.p == r.end;
}

// ---- the cache -----------------------------------------------------------

struct Entry {
  cb_tune t;
  float ms;
};

// 0: read (or absent: empty), CB_ERR_ARG: not a cache of this format
int read_cache(const char* path, std::map<std::string, Entry>& out) {
  out.clear();
  FILE* f = std::fopen(path, "rb");
  if (!f) return errno == ENOENT ? CB_OK : CB_ERR_ARG;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  const bool err = std::ferror(f) != 0;
  std::fclose(f);
  if (err) return CB_ERR_ARG;
  JValue root;
  if (!parse(text, root) || root.kind != JValue::kObj) return CB_ERR_ARG;
  const JValue* fmt = root.get("format");
  const JValue* ents = root.get("entries");
  if (!fmt || fmt->kind != JValue::kStr || fmt->str != kFormat || !ents || ents->kind != JValue::kObj)
    return CB_ERR_ARG;
  for (const auto& kv : ents->obj) {
    const JValue& e = kv.second;
    if (e.kind != JValue::kObj) return CB_ERR_ARG;
    const char* names[] = {"sym_hash_max", "num_hash_max", "learn_max", "cf_esc", "cf_prereduce", "ms"};
    double v[6];
    for (int i = 0; i < 6; ++i) {
      const JValue* x = e.get(names[i]);
      if (!x || x->kind != JValue::kNum || !std::isfinite(x->num)) return CB_ERR_ARG;
      v[i] = x->num;
    }
    for (int i = 0; i < 3; ++i)
      if (v[i] != std::floor(v[i]) || std::fabs(v[i]) > 1e9) return CB_ERR_ARG;
    Entry en;
    en.t.sym_hash_max = (int32_t)v[0];
    en.t.num_hash_max = (int32_t)v[1];
    en.t.learn_max = (int32_t)v[2];
    en.t.cf_esc = (float)v[3];
    en.t.cf_prereduce = (float)v[4];
    en.ms = (float)v[5];
    out[kv.first] = en;
  }
  return CB_OK;
}

void put_string(std::string& o, const std::string& s) {
  o.push_back('"');
  for (const char c : s) {
    if (c == '"' || c == '\\') {
      o.push_back('\\');
      o.push_back(c);
    } else if ((unsigned char)c < 0x20) {
      char u[8];
      std::snprintf(u, sizeof u, "\\u%04x", (unsigned)(unsigned char)c);
      o += u;
    } else {
      o.push_back(c);
    }
  }
  o.push_back('"');
}

int write_cache(const char* path, const std::map<std::string, Entry>& m) {
  std::string o = "{\"format\": ";
  put_string(o, kFormat);
  o += ",\n \"entries\": {";
  bool first = true;
  for (const auto& kv : m) {
    o += first ? "\n  " : ",\n  ";
    first = false;
    put_string(o, kv.first);
    // cf_prereduce may hold 1e30 ("never"): %.9g keeps every float exactly
    char b[256];
    std::snprintf(b, sizeof b,
                  ": {\"sym_hash_max\": %d, \"num_hash_max\": %d, \"learn_max\": %d, "
                  "\"cf_esc\": %.9g, \"cf_prereduce\": %.9g, \"ms\": %.9g}",
                  kv.second.t.sym_hash_max, kv.second.t.num_hash_max, kv.second.t.learn_max,
                  (double)kv.second.t.cf_esc, (double)kv.second.t.cf_prereduce, (double)kv.second.ms);
    o += b;
  }
  o += "\n }}\n";
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return CB_ERR_ARG;
  const bool ok = std::fwrite(o.data(), 1, o.size(), f) == o.size();
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return CB_ERR_ARG;
  }
  return CB_OK;
}

// nearest power of two's exponent of x (x >= 1), 0 for x <= 1
int size_class(int64_t x) {
  return x <= 1 ? 0 : (int)std::lround(std::log2((double)x));
}

}  // namespace

extern "C" {

int cb_tune_key(const char* device_name, cb_semiring sr, int32_t sizing, int64_t nrows, int64_t nnz_a,
                int64_t nnz_b, char* buf, int64_t buf_len) {
  if (!device_name || !buf || buf_len <= 0 || nrows < 0 || nnz_a < 0 || nnz_b < 0) return CB_ERR_ARG;
  const int n = std::snprintf(buf, (size_t)buf_len, "%s|sr%d|sizing%d|m2^%d|a2^%d|b2^%d", device_name,
                              (int)sr, (int)sizing, size_class(nrows), size_class(nnz_a),
                              size_class(nnz_b));
  if (n < 0 || n >= buf_len) {
    buf[0] = '\0';
    return CB_ERR_ARG;
  }
  return CB_OK;
}

int cb_tune_cache_get(const char* path, const char* key, cb_tune* tune, float* ms, int* found) {
  if (!path || !key || !tune || !found) return CB_ERR_ARG;
  *found = 0;
  std::map<std::string, Entry> m;
  const int rc = read_cache(path, m);
  if (rc != CB_OK) return rc;
  const auto it = m.find(key);
  if (it == m.end()) return CB_OK;
  *tune = it->second.t;
  if (ms) *ms = it->second.ms;
  *found = 1;
  return CB_OK;
}

int cb_tune_cache_put(const char* path, const char* key, const cb_tune* tune, float ms) {
  if (!path || !key || !tune) return CB_ERR_ARG;
  std::map<std::string, Entry> m;
  const int rc = read_cache(path, m);
  if (rc != CB_OK) return rc;  // an unreadable or foreign file is left alone
  m[key] = Entry{*tune, ms};
  return write_cache(path, m);
}

}  // extern "C"

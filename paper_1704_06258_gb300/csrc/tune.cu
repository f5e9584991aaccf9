// Tile-shape cache of the autotuner (host code only).
//
// The tensor-core evaluator's tile shape (MMA width, pipeline stages, raster
// order; see TcTile) is chosen per problem bucket by timing the candidates
// (usaphmp_autotune in capi.cu).  The choice is kept in a small JSON file so
// that later processes skip the timing:
//
//   {"format": "usaphmp-tile-cache-1",
//    "entries": [
//      {"device": "NVIDIA GB300", "n_blocks": 8, "p": 20, "B_pow2": 4096,
//       "ntile": 256, "stages": 3, "raster": 0, "pair": 0, "ms": 0.2091}, ...]}
//
// A bucket is (device name, ceil(n/128) row blocks, p, B rounded up to a
// power of two): the tile count and the per-tile work of the kernel depend on
// these only.  The reader accepts any JSON text (objects, arrays, strings,
// numbers, literals) and ignores unknown keys; the writer rewrites the whole
// file through a temporary file and a rename.
#include "usaphmp.h"

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <utility>
#include <vector>

#include "kernels.cuh"

namespace usaphmp {
namespace {

struct JVal {
  enum Kind { Null, Bool, Num, Str, Arr, Obj } kind = Null;
  double num = 0;
  std::string str;
  std::vector<JVal> arr;
  std::vector<std::pair<std::string, JVal>> obj;
  const JVal* get(const char* key) const {
    for (const auto& kv : obj)
      if (kv.first == key) return &kv.second;
    return nullptr;
  }
};

struct Parser {
  const std::string& s;
  size_t i = 0;
  bool bad = false;
  explicit Parser(const std::string& text) : s(text) {}

  void ws() {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) ++i;
  }
  bool eat(char c) {
    ws();
    if (i < s.size() && s[i] == c) { ++i; return true; }
    return false;
  }
  std::string string_lit() {
    std::string out;
    if (!eat('"')) { bad = true; return out; }
    while (i < s.size() && s[i] != '"') {
      char c = s[i++];
      if (c == '\\') {
        if (i >= s.size()) { bad = true; return out; }
        const char e = s[i++];
        switch (e) {
          case 'n': c = '\n'; break;
          case 't': c = '\t'; break;
          case 'r': c = '\r'; break;
          case 'b': c = '\b'; break;
          case 'f': c = '\f'; break;
          case 'u':  // keep \uXXXX as written: device names are ASCII
            out += "\\u";
            continue;
          default: c = e;  // \" \\ \/
        }
      }
      out += c;
    }
    if (i >= s.size()) { bad = true; return out; }
    ++i;
    return out;
  }
  JVal value(int depth = 0) {
    JVal v;
    ws();
    if (depth > 64 || i >= s.size()) { bad = true; return v; }
    const char c = s[i];
    if (c == '{') {
      ++i;
      v.kind = JVal::Obj;
      if (eat('}')) return v;
      do {
        std::string k = string_lit();
        if (bad || !eat(':')) { bad = true; return v; }
        JVal x = value(depth + 1);
        if (bad) return v;
        v.obj.emplace_back(std::move(k), std::move(x));
      } while (eat(','));
      if (!eat('}')) bad = true;
    } else if (c == '[') {
      ++i;
      v.kind = JVal::Arr;
      if (eat(']')) return v;
      do {
        JVal x = value(depth + 1);
        if (bad) return v;
        v.arr.push_back(std::move(x));
      } while (eat(','));
      if (!eat(']')) bad = true;
    } else if (c == '"') {
      v.kind = JVal::Str;
      v.str = string_lit();
    } else if (s.compare(i, 4, "true") == 0) {
      v.kind = JVal::Bool; v.num = 1; i += 4;
    } else if (s.compare(i, 5, "false") == 0) {
      v.kind = JVal::Bool; i += 5;
    } else if (s.compare(i, 4, "null") == 0) {
      i += 4;
    } else {
      const char* b = s.c_str() + i;
      char* e = nullptr;
      v.num = std::strtod(b, &e);
      if (e == b) { bad = true; return v; }
      v.kind = JVal::Num;
      i += (size_t)(e - b);
    }
    return v;
  }
};

struct Entry {
  std::string device;
  int n_blocks = 0, p = 0, b_pow2 = 0;
  usaphmp_tile tile{};
  double ms = 0;
};

int pow2_at_least(int x) {
  int v = 1;
  while (v < x && v < (1 << 30)) v <<= 1;
  return v;
}

std::string quote(const std::string& s) {
  std::string out = "\"";
  for (char c : s) {
    if (c == '"' || c == '\\') out += '\\';
    if ((unsigned char)c < 0x20) continue;
    out += c;
  }
  return out + "\"";
}

// Reads the entries of `path`.  A missing file is an empty cache (0); an
// unreadable or malformed one is an error (-1, message in *why).
int read_cache(const char* path, std::vector<Entry>& out, std::string* why) {
  out.clear();
  std::ifstream f(path, std::ios::binary);
  if (!f) return 0;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string text = ss.str();
  Parser ps(text);
  const JVal root = ps.value();
  ps.ws();
  if (ps.bad || ps.i != text.size() || root.kind != JVal::Obj) {
    *why = std::string("tile cache ") + path + ": not a JSON object";
    return -1;
  }
  const JVal* fmt = root.get("format");
  if (!fmt || fmt->kind != JVal::Str || fmt->str != "usaphmp-tile-cache-1") {
    *why = std::string("tile cache ") + path + ": unknown format";
    return -1;
  }
  const JVal* ents = root.get("entries");
  if (!ents || ents->kind != JVal::Arr) {
    *why = std::string("tile cache ") + path + ": no entries array";
    return -1;
  }
  for (const JVal& e : ents->arr) {
    if (e.kind != JVal::Obj) continue;
    auto num = [&](const char* k, double* v) {
      const JVal* x = e.get(k);
      if (!x || x->kind != JVal::Num) return false;
      *v = x->num;
      return true;
    };
    const JVal* dev = e.get("device");
    double nb, p, b, nt, st, ra, ms = 0;
    if (!dev || dev->kind != JVal::Str || !num("n_blocks", &nb) || !num("p", &p) || !num("B_pow2", &b) ||
        !num("ntile", &nt) || !num("stages", &st) || !num("raster", &ra))
      continue;  // an entry of another shape: skipped
    num("ms", &ms);
    double pr = 0;
    num("pair", &pr);   // absent in caches written before pair mode: 0
    Entry x;
    x.device = dev->str;
    x.n_blocks = (int)nb; x.p = (int)p; x.b_pow2 = (int)b;
    x.tile.ntile = (int32_t)nt; x.tile.stages = (int32_t)st; x.tile.raster = (int32_t)ra;
    x.tile.pair = (int32_t)pr;
    x.ms = ms;
    out.push_back(x);
  }
  return 0;
}

int write_cache(const char* path, const std::vector<Entry>& ents, std::string* why) {
  std::string text = "{\"format\": \"usaphmp-tile-cache-1\",\n \"entries\": [";
  for (size_t k = 0; k < ents.size(); ++k) {
    const Entry& e = ents[k];
    char buf[512];
    std::snprintf(buf, sizeof(buf),
                  "%s\n  {\"device\": %s, \"n_blocks\": %d, \"p\": %d, \"B_pow2\": %d, \"ntile\": %d, "
                  "\"stages\": %d, \"raster\": %d, \"pair\": %d, \"ms\": %.6f}",
                  k ? "," : "", quote(e.device).c_str(), e.n_blocks, e.p, e.b_pow2, e.tile.ntile, e.tile.stages,
                  e.tile.raster, e.tile.pair, e.ms);
    text += buf;
  }
  text += "\n ]}\n";
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
    if (!f) {
      *why = "tile cache: cannot write " + tmp;
      return -1;
    }
    f << text;
    if (!f) {
      *why = "tile cache: write failed on " + tmp;
      return -1;
    }
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    *why = std::string("tile cache: cannot replace ") + path;
    return -1;
  }
  return 0;
}

}  // namespace
}  // namespace usaphmp

using namespace usaphmp;

extern "C" {

int usaphmp_tile_cache_lookup(const char* path, const char* device, int32_t n, int32_t p, int32_t B,
                              usaphmp_tile* out, double* ms) {
  if (!path || !device || !out) return report_error(USAPHMP_EINVAL, "NULL argument");
  std::vector<Entry> ents;
  std::string why;
  if (read_cache(path, ents, &why) != 0) return report_error(USAPHMP_EINVAL, why);
  const int nb = (n + 127) / 128, bp = pow2_at_least(B);
  for (const Entry& e : ents)
    if (e.device == device && e.n_blocks == nb && e.p == p && e.b_pow2 == bp) {
      *out = e.tile;
      if (ms) *ms = e.ms;
      return 1;
    }
  return 0;
}

int usaphmp_tile_cache_store(const char* path, const char* device, int32_t n, int32_t p, int32_t B,
                             const usaphmp_tile* tile, double ms) {
  if (!path || !device || !tile) return report_error(USAPHMP_EINVAL, "NULL argument");
  std::vector<Entry> ents;
  std::string why;
  if (read_cache(path, ents, &why) != 0) return report_error(USAPHMP_EINVAL, why);
  Entry x;
  x.device = device;
  x.n_blocks = (n + 127) / 128;
  x.p = p;
  x.b_pow2 = pow2_at_least(B);
  x.tile = *tile;
  x.ms = ms;
  bool replaced = false;
  for (Entry& e : ents)
    if (e.device == x.device && e.n_blocks == x.n_blocks && e.p == x.p && e.b_pow2 == x.b_pow2) {
      e = x;
      replaced = true;
    }
  if (!replaced) ents.push_back(x);
  if (write_cache(path, ents, &why) != 0) return report_error(USAPHMP_EIO, why);
  return USAPHMP_OK;
}

}  // extern "C"

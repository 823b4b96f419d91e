// Autotuner support (host only): the size class of a batched call and the
// JSON cache file of chosen (kernel, tile shape) per device, library size and
// class.  The paper has no counterpart; batching and autotuning are this
// library's own.
//
// Cache file format (written by fps_tune_cache_put, read back by any version):
//   {"fps_tune_cache": 1, "entries": [
//     {"device": "<name>", "n": <records>, "class": "q12-k10-l0", "path": 6, "param": 96, "ms": 31.2},
//     ...]}
// Writers merge by (device, n, class), write a temporary file and rename it
// over the old one, so a reader never sees a half-written file.
#include <cctype>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <unistd.h>
#include <vector>

#include "fps_internal.h"

namespace fps {
namespace {

struct Entry {
  std::string device;
  int64_t n = 0;
  std::string cls;
  int path = 0;
  int param = 0;
  double ms = 0.0;
};

std::mutex g_cache_mu;   // one writer at a time inside this process

// Recursive-descent reader for the subset of JSON the cache uses (objects,
// arrays, strings with simple escapes, numbers, true/false/null).  Values that
// are not entries are skipped; any syntax error makes the whole file unreadable.
class Reader {
 public:
  explicit Reader(const std::string& t) : s_(t) {}

  bool entries(std::vector<Entry>* out) {
    ws();
    if (!eat('{')) return false;
    ws();
    if (eat('}')) return true;
    for (;;) {
      std::string key;
      if (!str(&key)) return false;
      ws();
      if (!eat(':')) return false;
      ws();
      if (key == "entries") {
        if (!entry_array(out)) return false;
      } else if (!skip()) {
        return false;
      }
      ws();
      if (eat('}')) return true;
      if (!eat(',')) return false;
      ws();
    }
  }

 private:
  const std::string& s_;
  size_t i_ = 0;

  void ws() {
    while (i_ < s_.size() && std::isspace(static_cast<unsigned char>(s_[i_]))) ++i_;
  }
  bool eat(char c) {
    if (i_ < s_.size() && s_[i_] == c) {
      ++i_;
      return true;
    }
    return false;
  }
  bool str(std::string* out) {
    if (!eat('"')) return false;
    out->clear();
    while (i_ < s_.size()) {
      char c = s_[i_++];
      if (c == '"') return true;
      if (c == '\\') {
        if (i_ >= s_.size()) return false;
        char e = s_[i_++];
        if (e == 'n')
          c = '\n';
        else if (e == 't')
          c = '\t';
        else if (e == '"' || e == '\\' || e == '/')
          c = e;
        else
          return false;   // \uXXXX never appears in files this library writes
      }
      out->push_back(c);
    }
    return false;
  }
  bool num(double* out) {
    const char* b = s_.c_str() + i_;
    char* e = nullptr;
    errno = 0;
    const double v = std::strtod(b, &e);
    if (e == b || errno != 0 || !std::isfinite(v)) return false;
    i_ += static_cast<size_t>(e - b);
    *out = v;
    return true;
  }
  bool word(const char* w) {
    const size_t n = std::strlen(w);
    if (s_.compare(i_, n, w) != 0) return false;
    i_ += n;
    return true;
  }
  bool skip() {   // any value
    ws();
    if (i_ >= s_.size()) return false;
    const char c = s_[i_];
    if (c == '"') {
      std::string t;
      return str(&t);
    }
    if (c == '{' || c == '[') {
      const char close = c == '{' ? '}' : ']';
      ++i_;
      ws();
      if (eat(close)) return true;
      for (;;) {
        if (c == '{') {
          std::string k;
          if (!str(&k)) return false;
          ws();
          if (!eat(':')) return false;
        }
        if (!skip()) return false;
        ws();
        if (eat(close)) return true;
        if (!eat(',')) return false;
        ws();
      }
    }
    if (word("true") || word("false") || word("null")) return true;
    double d;
    return num(&d);
  }
  bool entry_array(std::vector<Entry>* out) {
    if (!eat('[')) return false;
    ws();
    if (eat(']')) return true;
    for (;;) {
      Entry e;
      bool has_dev = false, has_n = false, has_cls = false, has_path = false;
      if (!eat('{')) return false;
      ws();
      if (!eat('}')) {
        for (;;) {
          std::string key;
          if (!str(&key)) return false;
          ws();
          if (!eat(':')) return false;
          ws();
          double d = 0.0;
          if (key == "device") {
            if (!str(&e.device)) return false;
            has_dev = true;
          } else if (key == "class") {
            if (!str(&e.cls)) return false;
            has_cls = true;
          } else if (key == "n" || key == "path" || key == "param" || key == "ms") {
            if (!num(&d)) return false;
            if (key == "n") {
              e.n = static_cast<int64_t>(d);
              has_n = true;
            } else if (key == "path") {
              e.path = static_cast<int>(d);
              has_path = true;
            } else if (key == "param") {
              e.param = static_cast<int>(d);
            } else {
              e.ms = d;
            }
          } else if (!skip()) {
            return false;
          }
          ws();
          if (eat('}')) break;
          if (!eat(',')) return false;
          ws();
        }
      }
      if (has_dev && has_n && has_cls && has_path) out->push_back(e);
      ws();
      if (eat(']')) return true;
      if (!eat(',')) return false;
      ws();
    }
  }
};

// false: the file cannot be read or is not a cache file
bool read_entries(const char* path, std::vector<Entry>* out) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  std::fclose(f);
  Reader r(text);
  std::vector<Entry> es;
  if (!r.entries(&es)) return false;
  *out = std::move(es);
  return true;
}

void put_json_string(std::string* o, const std::string& v) {
  o->push_back('"');
  for (char c : v) {
    if (c == '"' || c == '\\') {
      o->push_back('\\');
      o->push_back(c);
    } else if (c == '\n') {
      *o += "\\n";
    } else if (c == '\t') {
      *o += "\\t";
    } else if (static_cast<unsigned char>(c) >= 0x20) {
      o->push_back(c);
    }
  }
  o->push_back('"');
}

bool write_entries(const char* path, const std::vector<Entry>& es) {
  std::string o = "{\"fps_tune_cache\": 1, \"entries\": [\n";
  for (size_t i = 0; i < es.size(); ++i) {
    const Entry& e = es[i];
    char num[160];
    o += " {\"device\": ";
    put_json_string(&o, e.device);
    std::snprintf(num, sizeof(num), ", \"n\": %lld, \"class\": ", static_cast<long long>(e.n));
    o += num;
    put_json_string(&o, e.cls);
    std::snprintf(num, sizeof(num), ", \"path\": %d, \"param\": %d, \"ms\": %.4f}", e.path, e.param, e.ms);
    o += num;
    o += i + 1 < es.size() ? ",\n" : "\n";
  }
  o += "]}\n";
  const std::string tmp = std::string(path) + ".tmp" + std::to_string(static_cast<long long>(getpid()));
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  const bool ok = std::fwrite(o.data(), 1, o.size(), f) == o.size();
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return false;
  }
  return true;
}

int ceil_log2(int64_t v) {
  int c = 0;
  while ((int64_t{1} << c) < v) ++c;
  return c;
}

}  // namespace

std::string tune_class_name(int Q, int k_max, bool learned) {
  char buf[FPS_TUNE_CLASS_LEN];
  std::snprintf(buf, sizeof(buf), "q%d-k%d-l%d", ceil_log2(Q < 1 ? 1 : Q), ceil_log2(int64_t{k_max} + 1),
                learned ? 1 : 0);
  return buf;
}

bool tune_cache_get(const char* path, const char* device, int64_t n, const std::string& cls, int* p, int* param,
                    double* ms) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  std::vector<Entry> es;
  if (!read_entries(path, &es)) return false;
  for (const Entry& e : es) {
    if (e.device == device && e.n == n && e.cls == cls) {
      *p = e.path;
      *param = e.param;
      *ms = e.ms;
      return true;
    }
  }
  return false;
}

bool tune_cache_put(const char* path, const char* device, int64_t n, const std::string& cls, int p, int param,
                    double ms) {
  std::lock_guard<std::mutex> lock(g_cache_mu);
  std::vector<Entry> es;
  read_entries(path, &es);   // a missing or unreadable file starts a new one
  bool found = false;
  for (Entry& e : es) {
    if (e.device == device && e.n == n && e.cls == cls) {
      e.path = p;
      e.param = param;
      e.ms = ms;
      found = true;
    }
  }
  if (!found) {
    Entry e;
    e.device = device;
    e.n = n;
    e.cls = cls;
    e.path = p;
    e.param = param;
    e.ms = ms;
    es.push_back(e);
  }
  return write_entries(path, es);
}

}  // namespace fps

extern "C" fps_status fps_tune_class(int Q, int k_max, int learned, char* out) {
  if (!out || Q < 0 || k_max < 0) return FPS_ERR_INVALID_ARG;
  const std::string c = fps::tune_class_name(Q, k_max, learned != 0);
  std::snprintf(out, FPS_TUNE_CLASS_LEN, "%s", c.c_str());
  return FPS_OK;
}

extern "C" fps_status fps_tune_cache_get(const char* path, const char* device, int64_t n, const char* cls,
                                         int* fps_path_out, int* tile_param, double* ms) {
  if (!path || !device || !cls || !fps_path_out || !tile_param || !ms) return FPS_ERR_INVALID_ARG;
  return fps::tune_cache_get(path, device, n, cls, fps_path_out, tile_param, ms) ? FPS_OK : FPS_ERR_IO;
}

extern "C" fps_status fps_tune_cache_put(const char* path, const char* device, int64_t n, const char* cls,
                                         int fps_path_in, int tile_param, double ms) {
  if (!path || !device || !cls || !std::isfinite(ms)) return FPS_ERR_INVALID_ARG;
  return fps::tune_cache_put(path, device, n, cls, fps_path_in, tile_param, ms) ? FPS_OK : FPS_ERR_IO;
}

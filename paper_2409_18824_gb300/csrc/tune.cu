// Autotuner and tuning cache of the star sweeps.  The paper's loop tiling and
// unrolling are compile-time passes (arXiv 2409.18824 Sec. 6, 6.1); here the
// tile shape (kernel variant), the k-chunk count of the launch grid and the
// temporal depth are picked by timing candidates on the device, per grid
// extents, and kept in a process-wide cache that the planners consult and
// that can be saved to and loaded from a JSON file.
#include <ctype.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"
#include "work_sched.h"

namespace stn {

namespace {

struct Key {
  std::string dev;
  int esize, r;
  i64 nx, ny, nz;
  bool operator<(const Key& o) const {
    return std::tie(dev, esize, r, nx, ny, nz) < std::tie(o.dev, o.esize, o.r, o.nx, o.ny, o.nz);
  }
};

struct Val {
  int variant, chunks, depth;
  double glups, default_glups;
};

std::mutex g_mu;
std::map<Key, Val> g_cache;
std::atomic<long long> g_count{0};  // entries (lets lookups skip the lock when empty)
std::once_flag g_env_once;

int tune_einval(const std::string& msg) {
  set_error("invalid argument: " + msg);
  return STN_EINVAL;
}

// Name of the current device, cached per ordinal ("" when there is none).
std::string current_device_name() {
  static std::mutex mu;
  static std::map<int, std::string> names;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return "";
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = names.find(dev);
  if (it != names.end()) return it->second;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return "";
  }
  prop.name[sizeof(prop.name) - 1] = 0;
  return names[dev] = prop.name;
}

int check_key(i64 nx, i64 ny, i64 nz, int esize, int radius) {
  if (esize != 4 && esize != 8) return tune_einval("esize must be 4 or 8");
  if (radius != 1 && radius != 2) return tune_einval("radius must be 1 or 2");
  const i64 lim = (i64)1 << 28;
  if (nx < 1 || ny < 1 || nz < 1 || nx > lim || ny > lim || nz > lim)
    return tune_einval("interior extents must be in [1, 2^28]");
  return STN_OK;
}

int check_val(int variant, int chunks, int depth) {
  if (variant < 0 || variant > 3) return tune_einval("variant must be 0, 1, 2 or 3");
  if (chunks < 1 || chunks > 65535) return tune_einval("chunks must be in [1, 65535]");
  if (depth < 1 || depth > 4) return tune_einval("depth must be in [1, 4]");
  return STN_OK;
}

void put_locked(const Key& k, const Val& v) {
  g_cache[k] = v;
  g_count.store((long long)g_cache.size());
}

// ---- JSON (the cache's own flat format) ---------------------------------------
// Entries are flat objects: string or number values, no nesting.  Objects are
// read key by key in order (never by searching the text, so a key's name
// inside a string value cannot be mistaken for the key).

// Reads the string starting at t[*i] == '"' (escapes decoded; \uXXXX only for
// code points below 256, which is all the writer emits) and moves *i past it.
bool json_read_string(const std::string& t, size_t* i, std::string* out) {
  std::string v;
  for (size_t k = *i + 1; k < t.size(); k++) {
    const char c = t[k];
    if (c == '"') {
      *out = v;
      *i = k + 1;
      return true;
    }
    if ((unsigned char)c < 0x20) return false;  // raw control characters are not JSON
    if (c != '\\') {
      v += c;
      continue;
    }
    if (++k >= t.size()) return false;
    switch (t[k]) {
      case '"': v += '"'; break;
      case '\\': v += '\\'; break;
      case '/': v += '/'; break;
      case 'b': v += '\b'; break;
      case 'f': v += '\f'; break;
      case 'n': v += '\n'; break;
      case 'r': v += '\r'; break;
      case 't': v += '\t'; break;
      case 'u': {
        if (k + 4 >= t.size()) return false;
        unsigned cp = 0;
        for (int h = 1; h <= 4; h++) {
          const char x = t[k + h];
          cp <<= 4;
          if (x >= '0' && x <= '9') cp |= (unsigned)(x - '0');
          else if (x >= 'a' && x <= 'f') cp |= (unsigned)(x - 'a' + 10);
          else if (x >= 'A' && x <= 'F') cp |= (unsigned)(x - 'A' + 10);
          else return false;
        }
        if (cp > 0xff) return false;
        v += (char)cp;
        k += 4;
        break;
      }
      default: return false;
    }
  }
  return false;
}

struct JsonValue {
  bool is_str = false;
  std::string text;  // the decoded string, or the number's characters
};

void json_skip_ws(const std::string& t, size_t* i) {
  while (*i < t.size() && (t[*i] == ' ' || t[*i] == '\t' || t[*i] == '\n' || t[*i] == '\r')) ++*i;
}

// Reads the flat object starting at t[*i] == '{' into `f` (a repeated key
// keeps its last value) and moves *i past its '}'; false on any syntax error.
bool json_read_object(const std::string& t, size_t* i, std::map<std::string, JsonValue>* f) {
  size_t k = *i + 1;
  json_skip_ws(t, &k);
  if (k < t.size() && t[k] == '}') {
    *i = k + 1;
    return true;
  }
  for (;;) {
    json_skip_ws(t, &k);
    if (k >= t.size() || t[k] != '"') return false;
    std::string key;
    if (!json_read_string(t, &k, &key)) return false;
    json_skip_ws(t, &k);
    if (k >= t.size() || t[k] != ':') return false;
    ++k;
    json_skip_ws(t, &k);
    if (k >= t.size()) return false;
    JsonValue v;
    if (t[k] == '"') {
      v.is_str = true;
      if (!json_read_string(t, &k, &v.text)) return false;
    } else {
      const size_t s0 = k;
      while (k < t.size() && (isdigit((unsigned char)t[k]) || t[k] == '-' || t[k] == '+' || t[k] == '.' ||
                              t[k] == 'e' || t[k] == 'E'))
        k++;
      if (k == s0) return false;
      v.text = t.substr(s0, k - s0);
    }
    (*f)[key] = v;
    json_skip_ws(t, &k);
    if (k >= t.size()) return false;
    if (t[k] == ',') {
      k++;
      continue;
    }
    if (t[k] != '}') return false;
    *i = k + 1;
    return true;
  }
}

bool json_field_number(const std::map<std::string, JsonValue>& f, const char* key, double* out) {
  const auto it = f.find(key);
  if (it == f.end() || it->second.is_str) return false;
  const char* s = it->second.text.c_str();
  char* end = nullptr;
  const double v = strtod(s, &end);
  if (end != s + it->second.text.size() || !isfinite(v)) return false;
  *out = v;
  return true;
}

bool json_field_int(const std::map<std::string, JsonValue>& f, const char* key, i64* out) {
  double v;
  if (!json_field_number(f, key, &v) || v != floor(v) || fabs(v) > 9.0e15) return false;
  *out = (i64)v;
  return true;
}

bool json_field_string(const std::map<std::string, JsonValue>& f, const char* key, std::string* out) {
  const auto it = f.find(key);
  if (it == f.end() || !it->second.is_str) return false;
  *out = it->second.text;
  return true;
}

// JSON string body of s: quotes and backslashes escaped, control bytes as
// \u00XX, every other byte as it is.
std::string json_escape(const std::string& s) {
  std::string o;
  for (char c : s) {
    if (c == '"' || c == '\\') {
      o += '\\';
      o += c;
    } else if ((unsigned char)c < 0x20) {
      char u[8];
      snprintf(u, sizeof u, "\\u%04x", (unsigned)(unsigned char)c);
      o += u;
    } else {
      o += c;
    }
  }
  return o;
}

void load_env_once() {
  std::call_once(g_env_once, [] {
    const char* p = getenv("STN_TUNE_CACHE");
    if (p && *p) {
      FILE* f = fopen(p, "rb");
      if (f) {
        fclose(f);
        (void)stencil_tune_cache_load(p);
        clear_error();
      }
    }
  });
}

// ---- timing ----------------------------------------------------------------------
constexpr int kTrialSweeps = 12;  // divisible by every temporal depth 1..4

template <typename T>
int run_sweeps(T* a, T* b, const Grid& g, const double* c, int depth, int sweeps, cudaStream_t s) {
  T* cur = a;
  T* nxt = b;
  const int step = depth > 1 ? depth : 1;
  for (int i = 0; i + step <= sweeps; i += step) {
    const int rc = depth > 1 ? launch_temporal<T>(cur, nxt, g, c, depth, s)
                             : launch_star<T>(cur, nullptr, nxt, g, c, kSweep, nullptr, s);
    if (rc) return rc;
    std::swap(cur, nxt);
  }
  return STN_OK;
}

int ck(cudaError_t e, const char* what) { return e == cudaSuccess ? STN_OK : cuda_fail(e, what); }

// Seconds per sweep of one configuration (forced on this thread).
template <typename T>
int time_choice(T* a, T* b, const Grid& g, const double* c, const StarChoice& ch, int sweeps,
                cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* sec) {
  star_force() = ch;
  int rc = run_sweeps<T>(a, b, g, c, ch.depth, 2 * (ch.depth > 1 ? ch.depth : 1), s);
  if (!rc) rc = ck(cudaEventRecord(e0, s), "cudaEventRecord");
  if (!rc) rc = run_sweeps<T>(a, b, g, c, ch.depth, sweeps, s);
  star_force() = StarChoice();
  if (rc) return rc;
  STN_CUDA_TRY(cudaEventRecord(e1, s));
  STN_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.f;
  STN_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  *sec = (double)ms * 1e-3 / sweeps;
  return STN_OK;
}

// k-chunk counts to try for one variant: the built-in plan's own, half, twice
// and four times it, and the counts that give 2, 4, 6, 8 and 16 blocks per SM.
std::vector<int> chunk_candidates(const Grid& g, int variant, size_t esize) {
  const ZPlan p = plan_star(g, variant, esize);  // the caller bypasses the cache
  const i64 tiles = (i64)p.tiles_x * p.tiles_y;
  const i64 max_chunks = (g.nz + 3) / 4;
  std::vector<i64> c = {p.chunks, p.chunks / 2, p.chunks * 2, p.chunks * 4};
  const i64 sms = device_sms();
  for (int per_sm : {2, 4, 6, 8, 16}) c.push_back((sms * per_sm + tiles - 1) / (tiles > 0 ? tiles : 1));
  std::vector<int> out;
  for (i64 v : c) {
    if (v < 1) v = 1;
    if (v > max_chunks) v = max_chunks;
    if (v > 65535) v = 65535;
    // the count the plan would actually launch for this request
    const i64 kchunk = (g.nz + v - 1) / v;
    const int eff = (int)((g.nz + kchunk - 1) / kchunk);
    if (tiles * eff > (i64)1 << 30) continue;
    if (std::find(out.begin(), out.end(), eff) == out.end()) out.push_back(eff);
  }
  return out;
}

template <typename T>
int autotune_t(const Grid& g, const double* coeffs, int sweeps, cudaStream_t s, stn_tune_entry* best) {
  const size_t bytes = (size_t)g.count() * sizeof(T);
  T* a = nullptr;
  T* b = nullptr;
  cudaError_t e = cudaMalloc((void**)&a, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (a) cudaFree(a);
    set_error("device allocation of the autotuner's scratch grids failed");
    return STN_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ck(cudaEventCreate(&e0), "cudaEventCreate");
  if (!rc) rc = ck(cudaEventCreate(&e1), "cudaEventCreate");
  if (!rc) rc = ck(cudaMemsetAsync(a, 0, bytes, s), "cudaMemsetAsync");
  if (!rc) rc = ck(cudaMemsetAsync(b, 0, bytes, s), "cudaMemsetAsync");

  // candidates: the built-in plan first, then every variant x chunk count,
  // then the temporal depths the kernels support for this type and radius
  std::vector<StarChoice> cand;
  star_force() = StarChoice();
  star_force().no_cache = true;  // plan as if nothing were tuned yet
  StarChoice def;
  def.variant = star_variant(g, sizeof(T), nullptr, nullptr, nullptr);
  def.chunks = plan_star(g, def.variant, sizeof(T)).chunks;
  def.depth = 1;
  cand.push_back(def);
  // the column kernel is offered only where it can address the grid
  star_force().variant = kStarColumn;
  const bool col_ok = star_variant(g, sizeof(T), nullptr, nullptr, nullptr) == kStarColumn;
  star_force().variant = -1;
  for (int v = 0; v <= 3; v++) {
    if (v == kStarColumn && !col_ok) continue;
    if (v == kStarStaged && !staged_applicable(g, sizeof(T))) continue;
    for (int c : chunk_candidates(g, v, sizeof(T))) {
      StarChoice ch;
      ch.variant = v;
      ch.chunks = c;
      ch.depth = 1;
      if (ch.variant == def.variant && ch.chunks == def.chunks) continue;
      cand.push_back(ch);
    }
  }
  for (int d = 2; d <= 4; d++) {
    if (temporal_depth_supported(d, sizeof(T), g.r) != d) continue;
    StarChoice ch = def;
    ch.depth = d;
    cand.push_back(ch);
  }
  star_force() = StarChoice();
  std::vector<double> t(cand.size(), INFINITY);
  for (int round = 0; round < 2 && !rc; round++) {
    for (size_t i = 0; i < cand.size() && !rc; i++) {
      double sec = 0;
      rc = time_choice<T>(a, b, g, coeffs, cand[i], sweeps, s, e0, e1, &sec);
      if (!rc) t[i] = std::min(t[i], sec);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const cudaError_t se = cudaStreamSynchronize(s);
  cudaFree(a);
  cudaFree(b);
  if (rc) return rc;
  STN_CUDA_TRY(se);

  size_t bi = 0;
  for (size_t i = 1; i < cand.size(); i++)
    if (t[i] < t[bi]) bi = i;
  // keep the built-in plan unless another is clearly faster (timing noise)
  if (bi != 0 && !(t[bi] < 0.98 * t[0])) bi = 0;
  const double lups = (double)g.interior();
  memset(best, 0, sizeof *best);
  const std::string dev = current_device_name();
  snprintf(best->device, sizeof best->device, "%s", dev.c_str());
  best->nx = g.nx;
  best->ny = g.ny;
  best->nz = g.nz;
  best->esize = (int)sizeof(T);
  best->radius = g.r;
  best->variant = cand[bi].variant;
  best->chunks = cand[bi].chunks;
  best->depth = cand[bi].depth;
  best->glups = lups / t[bi] * 1e-9;
  best->default_glups = lups / t[0] * 1e-9;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    put_locked(Key{dev, best->esize, best->radius, g.nx, g.ny, g.nz},
               Val{best->variant, best->chunks, best->depth, best->glups, best->default_glups});
  }
  const char* path = getenv("STN_TUNE_CACHE");
  if (path && *path) {
    const int src = stencil_tune_cache_save(path);
    if (src) return src;
  }
  return STN_OK;
}

}  // namespace

bool tune_cache_lookup(const Grid& g, size_t esize, StarChoice* out) {
  if (star_force().no_cache) return false;
  load_env_once();
  if (g_count.load(std::memory_order_relaxed) == 0) return false;
  const std::string dev = current_device_name();
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(Key{dev, (int)esize, g.r, g.nx, g.ny, g.nz});
  if (it == g_cache.end()) return false;
  out->variant = it->second.variant;
  out->chunks = it->second.chunks;
  out->depth = it->second.depth;
  return true;
}

}  // namespace stn

using namespace stn;

extern "C" {

int stencil_autotune_sweep(int64_t nx, int64_t ny, int64_t nz, int esize, int radius, const double* coeffs,
                           int trial_sweeps, stn_tune_entry* best, void* stream) {
  clear_error();
  if (!best) return tune_einval("NULL best");
  if (int rc = check_key(nx, ny, nz, esize, radius)) return rc;
  const double cells = (double)(nx + 2 * radius) * (double)(ny + 2 * radius) * (double)(nz + 2 * radius);
  if (cells > 9.0e15) return tune_einval("grid too large");
  if (trial_sweeps < 0) return tune_einval("trial_sweeps < 0");
  double c[3] = {0.0, 1.0 / 6.0, 0.0};
  if (coeffs)
    for (int d = 0; d <= radius; d++) c[d] = coeffs[d];
  // whole multiples of 12 sweeps, so every temporal depth times the same count
  int sweeps = trial_sweeps > 0 ? trial_sweeps : kTrialSweeps;
  sweeps = (sweeps + kTrialSweeps - 1) / kTrialSweeps * kTrialSweeps;
  load_env_once();
  const Grid g{nx, ny, nz, radius};
  cudaStream_t s = (cudaStream_t)stream;
  return esize == 8 ? autotune_t<double>(g, c, sweeps, s, best) : autotune_t<float>(g, c, sweeps, s, best);
}

int stencil_tune_cache_put(const stn_tune_entry* e) {
  clear_error();
  if (!e) return tune_einval("NULL entry");
  if (int rc = check_key(e->nx, e->ny, e->nz, e->esize, e->radius)) return rc;
  if (int rc = check_val(e->variant, e->chunks, e->depth)) return rc;
  load_env_once();
  char name[sizeof e->device + 1];
  memcpy(name, e->device, sizeof e->device);
  name[sizeof e->device] = 0;
  const std::string dev = name[0] ? std::string(name) : current_device_name();
  std::lock_guard<std::mutex> lk(g_mu);
  put_locked(Key{dev, e->esize, e->radius, e->nx, e->ny, e->nz},
             Val{e->variant, e->chunks, e->depth, e->glups, e->default_glups});
  return STN_OK;
}

int stencil_tune_cache_get(const char* device, int64_t nx, int64_t ny, int64_t nz, int esize, int radius,
                           stn_tune_entry* out) {
  clear_error();
  if (!out) return tune_einval("NULL out");
  if (int rc = check_key(nx, ny, nz, esize, radius)) return rc;
  load_env_once();
  const std::string dev = device && *device ? std::string(device) : current_device_name();
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_cache.find(Key{dev, esize, radius, nx, ny, nz});
  if (it == g_cache.end()) return 0;
  memset(out, 0, sizeof *out);
  snprintf(out->device, sizeof out->device, "%s", dev.c_str());
  out->nx = nx;
  out->ny = ny;
  out->nz = nz;
  out->esize = esize;
  out->radius = radius;
  out->variant = it->second.variant;
  out->chunks = it->second.chunks;
  out->depth = it->second.depth;
  out->glups = it->second.glups;
  out->default_glups = it->second.default_glups;
  return 1;
}

int64_t stencil_tune_cache_size(void) {
  load_env_once();
  std::lock_guard<std::mutex> lk(g_mu);
  return (int64_t)g_cache.size();
}

int stencil_tune_cache_clear(void) {
  clear_error();
  load_env_once();
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache.clear();
  g_count.store(0);
  return STN_OK;
}

int stencil_tune_cache_save(const char* path) {
  clear_error();
  if (!path) return tune_einval("NULL path");
  std::string text = "{\"stencil_tune_cache\": 1, \"entries\": [\n";
  {
    std::lock_guard<std::mutex> lk(g_mu);
    size_t i = 0;
    for (const auto& kv : g_cache) {
      char buf[1024];
      snprintf(buf, sizeof buf,
               "  {\"device\": \"%s\", \"esize\": %d, \"radius\": %d, \"nx\": %lld, \"ny\": %lld, \"nz\": %lld, "
               "\"variant\": %d, \"chunks\": %d, \"depth\": %d, \"glups\": %.17g, \"default_glups\": %.17g}%s\n",
               json_escape(kv.first.dev).c_str(), kv.first.esize, kv.first.r, (long long)kv.first.nx,
               (long long)kv.first.ny, (long long)kv.first.nz, kv.second.variant, kv.second.chunks,
               kv.second.depth, kv.second.glups, kv.second.default_glups, ++i < g_cache.size() ? "," : "");
      text += buf;
    }
  }
  text += "]}\n";
  FILE* f = fopen(path, "wb");
  if (!f) return tune_einval(std::string("cannot write ") + path);
  const bool ok = fwrite(text.data(), 1, text.size(), f) == text.size();
  const bool closed = fclose(f) == 0;
  if (!ok || !closed) return tune_einval(std::string("cannot write ") + path);
  return STN_OK;
}

int stencil_tune_cache_load(const char* path) {
  clear_error();
  if (!path) return tune_einval("NULL path");
  FILE* f = fopen(path, "rb");
  if (!f) return tune_einval(std::string("cannot read ") + path);
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) {
    text.append(buf, n);
    if (text.size() > ((size_t)64 << 20)) break;
  }
  fclose(f);
  if (text.find("\"stencil_tune_cache\"") == std::string::npos) return tune_einval("not a tuning cache file");
  size_t p = text.find("\"entries\"");
  if (p == std::string::npos) return tune_einval("tuning cache without entries");
  p = text.find('[', p);
  if (p == std::string::npos) return tune_einval("tuning cache without an entry list");
  std::vector<std::pair<Key, Val>> got;
  size_t i = p + 1;
  json_skip_ws(text, &i);
  bool first = true;
  for (;;) {
    if (i >= text.size()) return tune_einval("unterminated entry list");
    if (text[i] == ']') break;
    if (!first) {
      if (text[i] != ',') return tune_einval("malformed entry list");
      i++;
      json_skip_ws(text, &i);
    }
    first = false;
    if (i >= text.size() || text[i] != '{') return tune_einval("malformed entry list");
    const size_t o = i;
    std::map<std::string, JsonValue> fields;
    if (!json_read_object(text, &i, &fields)) return tune_einval("malformed tuning cache entry");
    const std::string obj = text.substr(o, std::min<size_t>(i - o, 200));
    std::string dev;
    i64 esize, r, nx, ny, nz, variant, chunks, depth;
    double glups = 0, dglups = 0;
    if (!json_field_string(fields, "device", &dev) || !json_field_int(fields, "esize", &esize) ||
        !json_field_int(fields, "radius", &r) || !json_field_int(fields, "nx", &nx) ||
        !json_field_int(fields, "ny", &ny) || !json_field_int(fields, "nz", &nz) ||
        !json_field_int(fields, "variant", &variant) || !json_field_int(fields, "chunks", &chunks) ||
        !json_field_int(fields, "depth", &depth))
      return tune_einval("malformed tuning cache entry: " + obj);
    if (fields.count("glups") && !json_field_number(fields, "glups", &glups))
      return tune_einval("malformed tuning cache entry: " + obj);
    if (fields.count("default_glups") && !json_field_number(fields, "default_glups", &dglups))
      return tune_einval("malformed tuning cache entry: " + obj);
    if (dev.size() >= sizeof(((stn_tune_entry*)nullptr)->device))
      return tune_einval("tuning cache entry with a device name of 64 bytes or more");
    if (esize > 8 || r > 2 || variant > 3 || chunks > 65535 || depth > 4)
      return tune_einval("tuning cache entry out of range: " + obj);
    if (int rc = check_key(nx, ny, nz, (int)esize, (int)r)) return rc;
    if (int rc = check_val((int)variant, (int)chunks, (int)depth)) return rc;
    got.push_back({Key{dev, (int)esize, (int)r, nx, ny, nz}, Val{(int)variant, (int)chunks, (int)depth, glups, dglups}});
    json_skip_ws(text, &i);
  }
  std::lock_guard<std::mutex> lk(g_mu);
  for (const auto& kv : got) put_locked(kv.first, kv.second);
  return (int)got.size();
}

int stencil_plan_query(const char* op, int64_t nx, int64_t ny, int64_t nz, int esize, int radius,
                       stn_launch_plan* out) {
  clear_error();
  if (!op || !out) return tune_einval("NULL op or out");
  if (int rc = check_key(nx, ny, nz, esize, radius)) return rc;
  const double cells = (double)(nx + 2 * radius) * (double)(ny + 2 * radius) * (double)(nz + 2 * radius);
  if (cells > 9.0e15) return tune_einval("grid too large");
  const Grid g{nx, ny, nz, radius};
  LaunchPlan q;
  if (strcmp(op, "sweep") == 0) {
    q = sweep_launch_plan(g, (size_t)esize);
  } else if (strcmp(op, "varcoef_sweep") == 0) {
    q = var_launch_plan(g, (size_t)esize);
  } else if (strcmp(op, "batch_unit") == 0) {
    if (nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return tune_einval("batched problem extent too large");
    q = batch_unit_plan(nx, ny, nz);
    if ((i64)q.grid_x * q.grid_y * q.grid_z > kMaxPassUnits)
      return tune_einval("batched problem needs more than 2^22 work units per pass");
  } else if (strcmp(op, "sweep2d") == 0) {
    if (nz != 1) return tune_einval("sweep2d plans take nz = 1");
    q = sweep2d_launch_plan(Grid2{nx, ny, radius}, (size_t)esize);
  } else {
    return tune_einval(std::string("unknown op ") + op);
  }
  if (strcmp(op, "batch_unit") != 0)
    if (int rc = check_launch_grid(q.grid_x, q.grid_y, q.grid_z)) return rc;
  out->variant = q.variant;
  out->grid_x = q.grid_x;
  out->grid_y = q.grid_y;
  out->grid_z = q.grid_z;
  out->block_threads = q.block_threads;
  out->tile_w = q.tile_w;
  out->tile_h = q.tile_h;
  out->kchunk = q.kchunk;
  out->stage_elems = q.stage_elems;
  out->smem_bytes = q.smem;
  out->row_stride = q.row_stride;
  out->row_pad = q.row_pad;
  out->bulk_copy = q.bulk_copy;
  out->reserved = 0;
  out->scratch_bytes = q.scratch;
  out->xchg_offset = q.xchg_off;
  return STN_OK;
}

}  // extern "C"

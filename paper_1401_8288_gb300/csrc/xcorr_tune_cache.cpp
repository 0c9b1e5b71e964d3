// xcorr_tune_cache.cpp -- the autotuners' results, kept per process and in
// JSON-lines files.
//
// An entry maps a problem (the tuner's scope -- a plan or a batch subarray --,
// the device's name and SM count, the input format, N_i, the channel count and
// the samples per execute) to the launch shape that won and its time.  The
// file format is one JSON object per line with exactly the fields save()
// writes; load() reads those fields back and skips (and counts) any line it
// cannot read, so a file edited by hand or written by another version does not
// stop a run.  Shapes are stored by number, so each line also carries the
// revision of the library's shape table (kShapeTable): a line from another
// revision names other shapes and is skipped.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "xcorr_internal.h"

namespace xc {
namespace {

// Revision of the launch-shape table the stored stage_variant numbers refer to; raised whenever
// a shape number comes to mean another launch.
constexpr int kShapeTable = 2;

using Key = std::tuple<std::string, std::string, int, int, int, int, int>;  // scope, device, sms, fmt, N_i, C, T
struct Entry {
  xcorr_tuning t;
  float ms;
};

std::mutex g_mu;
std::map<Key, Entry> g_cache;

Key to_key(const TuneKey& k) { return Key(k.scope, k.device, k.sms, k.fmt, k.n_inputs, k.n_channels, k.n_time); }

// The text of "name": in line, or nullptr.
const char* field(const char* line, const char* name) {
  char pat[64];
  std::snprintf(pat, sizeof(pat), "\"%s\":", name);
  const char* p = std::strstr(line, pat);
  if (!p) return nullptr;
  p += std::strlen(pat);
  while (*p == ' ') ++p;
  return p;
}

bool int_field(const char* line, const char* name, int* out) {
  const char* p = field(line, name);
  if (!p) return false;
  char* end = nullptr;
  const long v = std::strtol(p, &end, 10);
  if (end == p || v < -(1L << 30) || v > (1L << 30)) return false;
  *out = static_cast<int>(v);
  return true;
}

bool str_field(const char* line, const char* name, std::string* out) {
  const char* p = field(line, name);
  if (!p || *p != '"') return false;
  const char* q = std::strchr(p + 1, '"');
  if (!q) return false;
  out->assign(p + 1, q);
  return out->find('\\') == std::string::npos;
}

}  // namespace

TuneKey tune_key(const char* scope, int fmt, int n_inputs, int n_channels, int n_time) {
  static std::mutex mu;
  static std::map<int, std::pair<std::string, int>> devices;  // ordinal -> (name, SMs)
  TuneKey k;
  k.scope = scope;
  k.fmt = fmt;
  k.n_inputs = n_inputs;
  k.n_channels = n_channels;
  k.n_time = n_time;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return k;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = devices.find(dev);
  if (it == devices.end()) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
      cudaGetLastError();
      return k;
    }
    std::string name(prop.name);
    for (char& ch : name)
      if (ch == '"' || ch == '\\') ch = '_';
    it = devices.emplace(dev, std::make_pair(name, prop.multiProcessorCount)).first;
  }
  k.device = it->second.first;
  k.sms = it->second.second;
  return k;
}

bool tune_cache_get(const TuneKey& k, xcorr_tuning* t, float* ms) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(to_key(k));
  if (it == g_cache.end()) return false;
  if (t) *t = it->second.t;
  if (ms) *ms = it->second.ms;
  return true;
}

void tune_cache_put(const TuneKey& k, const xcorr_tuning& t, float ms) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache[to_key(k)] = Entry{t, ms};
}

}  // namespace xc

extern "C" {

xcorr_status xcorr_tuning_cache_load(const char* path, int* n_loaded, int* n_skipped) {
  if (!path) return xc::set_error(XCORR_ERR_INVALID_ARG, "path is NULL");
  FILE* f = std::fopen(path, "r");
  if (!f) return xc::set_error(XCORR_ERR_INVALID_ARG, std::string("cannot open ") + path);
  int loaded = 0, skipped = 0;
  char line[1024];
  while (std::fgets(line, sizeof(line), f)) {
    if (line[0] == '\n' || line[0] == '\0') continue;
    xc::TuneKey k;
    xcorr_tuning t{};
    int ms_milli = 0;
    bool ok = xc::str_field(line, "scope", &k.scope) && xc::str_field(line, "device", &k.device) &&
              xc::int_field(line, "sms", &k.sms) && xc::int_field(line, "fmt", &k.fmt) &&
              xc::int_field(line, "n_inputs", &k.n_inputs) && xc::int_field(line, "n_channels", &k.n_channels) &&
              xc::int_field(line, "n_time", &k.n_time) && xc::int_field(line, "stage_variant", &t.stage_variant) &&
              xc::int_field(line, "groups", &t.groups) && xc::int_field(line, "x_streams", &t.x_streams) &&
              xc::int_field(line, "unfused", &t.unfused) && xc::int_field(line, "us", &ms_milli);
    int table = -1;
    ok = ok && xc::int_field(line, "shape_table", &table) && table == xc::kShapeTable;
    ok = ok && t.stage_variant >= 0 && t.stage_variant < xc::kFusedVariants && t.groups >= 0 &&
         t.groups <= xc::kMaxGroups && (t.x_streams == 1 || t.x_streams == 2) && (t.unfused == 0 || t.unfused == 1);
    if (!ok) {
      ++skipped;
      continue;
    }
    xc::tune_cache_put(k, t, 1e-3f * static_cast<float>(ms_milli));
    ++loaded;
  }
  std::fclose(f);
  if (n_loaded) *n_loaded = loaded;
  if (n_skipped) *n_skipped = skipped;
  return XCORR_OK;
}

xcorr_status xcorr_tuning_cache_save(const char* path, int* n_saved) {
  if (!path) return xc::set_error(XCORR_ERR_INVALID_ARG, "path is NULL");
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return xc::set_error(XCORR_ERR_INVALID_ARG, std::string("cannot write ") + tmp);
  int n = 0;
  {
    std::lock_guard<std::mutex> lock(xc::g_mu);
    for (const auto& kv : xc::g_cache) {
      const xc::Key& k = kv.first;
      const xc::Entry& e = kv.second;
      std::fprintf(f,
                   "{\"scope\": \"%s\", \"device\": \"%s\", \"sms\": %d, \"fmt\": %d, \"n_inputs\": %d, "
                   "\"n_channels\": %d, \"n_time\": %d, \"stage_variant\": %d, \"groups\": %d, \"x_streams\": %d, "
                   "\"unfused\": %d, \"us\": %d, \"shape_table\": %d}\n",
                   std::get<0>(k).c_str(), std::get<1>(k).c_str(), std::get<2>(k), std::get<3>(k), std::get<4>(k),
                   std::get<5>(k), std::get<6>(k), e.t.stage_variant, e.t.groups, e.t.x_streams, e.t.unfused,
                   static_cast<int>(e.ms * 1000.f + 0.5f), xc::kShapeTable);
      ++n;
    }
  }
  const bool ok = std::fflush(f) == 0;
  std::fclose(f);
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return xc::set_error(XCORR_ERR_INVALID_ARG, std::string("cannot write ") + path);
  }
  if (n_saved) *n_saved = n;
  return XCORR_OK;
}

xcorr_status xcorr_tuning_cache_clear(void) {
  std::lock_guard<std::mutex> lock(xc::g_mu);
  xc::g_cache.clear();
  return XCORR_OK;
}

}  // extern "C"

// Launch-shape autotuner with a JSON cache.
//
// Some launch parameters do not change what a kernel computes, only how fast:
// the persistent CG's CTA width (256 threads, two CTAs per SM, or 512
// threads, one CTA per SM).  For every problem shape (precision, grid, sphere,
// projector rows, columns, packing) the first launches try each candidate in
// turn and time them (CUDA events on the work stream, per CG iteration since
// launches differ in iteration count); once every candidate has two samples
// the fastest is kept for the rest of the process and written to the cache
// file, which later processes read instead of measuring again.
//
// Cache file: $LIBGW_TUNE_CACHE if set, else $XDG_CACHE_HOME/libgw/tune.json,
// else $HOME/.cache/libgw/tune.json; one "key": value pair per line.  A file
// that cannot be read or written only means measuring again.
#include <sys/stat.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tune.h"

namespace gw {

namespace {

struct Entry {
  std::vector<int> cand;
  std::vector<std::vector<double>> samples;   // per candidate
  int best = 0;                               // 0: undecided
};

std::mutex g_mu;
std::map<std::string, int> g_file;            // decisions read from or written to the cache
std::map<std::string, Entry> g_live;
bool g_loaded = false;

std::string cache_path() {
  if (const char* p = std::getenv("LIBGW_TUNE_CACHE")) return p;
  std::string base;
  if (const char* x = std::getenv("XDG_CACHE_HOME")) base = x;
  else if (const char* h = std::getenv("HOME")) base = std::string(h) + "/.cache";
  else return "";
  return base + "/libgw/tune.json";
}

void load_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const std::string path = cache_path();
  if (path.empty()) return;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return;
  char line[512];
  while (std::fgets(line, sizeof(line), f)) {
    // "key": value
    const char* q1 = std::strchr(line, '"');
    if (!q1) continue;
    const char* q2 = std::strchr(q1 + 1, '"');
    if (!q2) continue;
    const char* colon = std::strchr(q2, ':');
    if (!colon) continue;
    const int v = std::atoi(colon + 1);
    if (v > 0) g_file[std::string(q1 + 1, q2)] = v;
  }
  std::fclose(f);
}

void save_locked() {
  const std::string path = cache_path();
  if (path.empty()) return;
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    // create the directory chain (errors ignored: the open below decides)
    std::string dir = path.substr(0, slash);
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{\n");
  size_t k = 0;
  for (const auto& kv : g_file)
    std::fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++k < g_file.size() ? "," : "");
  std::fprintf(f, "}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

}  // namespace

int tune_pick(const std::string& key, const std::vector<int>& cand, bool enabled) {
  if (!enabled || cand.empty()) return cand.empty() ? 0 : cand[0];
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  auto fit = g_file.find(key);
  if (fit != g_file.end()) return fit->second;
  Entry& e = g_live[key];
  if (e.cand.empty()) {
    e.cand = cand;
    e.samples.assign(cand.size(), {});
  }
  if (e.best) return e.best;
  size_t pick = 0;
  for (size_t i = 1; i < e.cand.size(); ++i)
    if (e.samples[i].size() < e.samples[pick].size()) pick = i;
  return e.cand[pick];
}

void tune_report(const std::string& key, int choice, double cost) {
  if (!(cost > 0.0)) return;
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_live.find(key);
  if (it == g_live.end() || it->second.best) return;
  Entry& e = it->second;
  for (size_t i = 0; i < e.cand.size(); ++i)
    if (e.cand[i] == choice) e.samples[i].push_back(cost);
  for (const auto& s : e.samples)
    if (s.size() < 2) return;
  size_t b = 0;
  double bc = 1e300;
  for (size_t i = 0; i < e.cand.size(); ++i) {
    double m = 1e300;
    for (double c : e.samples[i]) m = std::min(m, c);
    if (m < bc) { bc = m; b = i; }
  }
  e.best = e.cand[b];
  g_file[key] = e.best;
  save_locked();
}

int tune_known(const std::string& key) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_locked();
  auto fit = g_file.find(key);
  if (fit != g_file.end()) return fit->second;
  auto lit = g_live.find(key);
  return lit != g_live.end() ? lit->second.best : 0;
}

}  // namespace gw

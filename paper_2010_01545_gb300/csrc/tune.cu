// tune.cu -- the tuning cache file (see tune.h).
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <fcntl.h>
#include <sys/file.h>
#include <sys/stat.h>
#include <unistd.h>

#include "tune.h"

namespace advect {
namespace {

std::mutex g_mu;
std::map<std::string, std::string> g_cache;
bool g_loaded = false;

void mkdirs(const std::string& path) {
  for (size_t p = 1; p < path.size(); ++p)
    if (path[p] == '/') mkdir(path.substr(0, p).c_str(), 0755);
}

// Parse "key": "value" pairs of a flat JSON object written by save_locked()
// into `into` (entries already there are kept when keep_existing).
void read_file(std::map<std::string, std::string>& into, bool keep_existing) {
  FILE* f = fopen(tune_cache_path().c_str(), "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  fclose(f);
  size_t i = 0;
  auto read_str = [&](std::string& out) -> bool {
    i = text.find('"', i);
    if (i == std::string::npos) return false;
    size_t j = text.find('"', i + 1);
    if (j == std::string::npos) return false;
    out = text.substr(i + 1, j - i - 1);
    i = j + 1;
    return true;
  };
  std::string k, v;
  while (read_str(k) && read_str(v))
    if (!keep_existing || !into.count(k)) into[k] = v;
}

void load_locked() {
  g_loaded = true;
  read_file(g_cache, false);
}

// Write the cache.  Several processes (one per rank) may tune at once: an
// exclusive lock on a side file serialises them, the file is re-read under
// the lock so entries other processes wrote are kept, and each process
// writes its own temporary file before the atomic rename.
void save_locked() {
  const std::string path = tune_cache_path();
  mkdirs(path);
  const int lock = open((path + ".lock").c_str(), O_CREAT | O_RDWR, 0644);
  if (lock >= 0) flock(lock, LOCK_EX);
  read_file(g_cache, true);
  const std::string tmp = path + ".tmp." + std::to_string((long)getpid());
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) {
    if (lock >= 0) close(lock);
    return;
  }
  fprintf(f, "{\n");
  size_t q = 0;
  for (const auto& kv : g_cache)
    fprintf(f, "  \"%s\": \"%s\"%s\n", kv.first.c_str(), kv.second.c_str(), ++q < g_cache.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path.c_str());
  if (lock >= 0) close(lock);  // releases the lock
}

}  // namespace

std::string tune_cache_path() {
  const char* p = getenv("ADVECT_TUNE_CACHE");
  if (p && *p) return p;
  const char* home = getenv("HOME");
  return std::string(home && *home ? home : "/tmp") + "/.cache/advect_gb300/tune.json";
}

bool tune_env_enabled() {
  const char* p = getenv("ADVECT_TUNE");
  return p && p[0] == '1';
}

bool tune_cache_get(const std::string& key, std::string& value) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load_locked();
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  value = it->second;
  return true;
}

void tune_cache_put(const std::string& key, const std::string& value) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_loaded) load_locked();
  g_cache[key] = value;
  save_locked();
}

}  // namespace advect

// The library's autotune cache: a flat JSON object of "key": [int, ...]
// entries in $BM_AUTOTUNE_CACHE, else ~/.cache/branch_mpc_gb300_autotune.json
// (the batched form's launch shape per batch signature, and the FP64
// factor's launch schedule per system shape and GPU). Reads and writes are
// serialized within the process; a lost or unreadable file only costs a
// new tuning run.
#include <stdio.h>
#include <stdlib.h>
#include <sys/stat.h>

#include <mutex>
#include <string>
#include <vector>

namespace bm {
namespace {

std::mutex g_tune_mutex;

std::string cache_path() {
  const char *p = getenv("BM_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char *home = getenv("HOME");
  return std::string(home && *home ? home : "/tmp") + "/.cache/branch_mpc_gb300_autotune.json";
}

std::string read_all(const std::string &path) {
  std::string s;
  if (FILE *f = fopen(path.c_str(), "r")) {
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
    fclose(f);
  }
  return s;
}

}  // namespace

bool tune_cache_lookup(const std::string &key, std::vector<int> &vals) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  const std::string s = read_all(cache_path());
  const std::string needle = "\"" + key + "\": [";
  const size_t p = s.find(needle);
  if (p == std::string::npos) return false;
  const size_t e = s.find(']', p + needle.size());
  if (e == std::string::npos) return false;
  vals.clear();
  const char *c = s.c_str() + p + needle.size();
  const char *end = s.c_str() + e;
  while (c < end) {
    char *next = nullptr;
    const long v = strtol(c, &next, 10);
    if (next == c) break;
    vals.push_back((int)v);
    c = next;
    while (c < end && (*c == ',' || *c == ' ')) ++c;
  }
  return !vals.empty();
}

void tune_cache_store(const std::string &key, const std::vector<int> &vals) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  const std::string path = cache_path();
  const std::string s = read_all(path);
  std::vector<std::string> entries;
  size_t p = 0;
  while ((p = s.find('"', p)) != std::string::npos) {
    const size_t q = s.find('"', p + 1);
    const size_t e = q == std::string::npos ? q : s.find(']', q);
    if (q == std::string::npos || e == std::string::npos) break;
    if (s.substr(p + 1, q - p - 1) != key) entries.push_back(s.substr(p, e - p + 1));
    p = e + 1;
  }
  std::string mine = "\"" + key + "\": [";
  for (size_t i = 0; i < vals.size(); ++i) mine += (i ? ", " : "") + std::to_string(vals[i]);
  mine += "]";
  entries.push_back(mine);
  const std::string dir = path.substr(0, path.find_last_of('/'));
  for (size_t i = 1; i <= dir.size(); ++i)   // create missing directories (best effort)
    if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  FILE *f = fopen(path.c_str(), "w");
  if (!f) return;
  fputs("{\n", f);
  for (size_t i = 0; i < entries.size(); ++i)
    fprintf(f, "  %s%s\n", entries[i].c_str(), i + 1 < entries.size() ? "," : "");
  fputs("}\n", f);
  fclose(f);
}

}  // namespace bm

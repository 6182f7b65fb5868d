// tune.cu -- the autotuner's cache.  A tuned choice (the solve column block,
// the split count of the tall Gram products) is measured once per problem
// shape on the running GPU and remembered in-process; with a cache file the
// choices also survive the process (one "key value" pair per line).
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"

namespace pdeshep {

namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
std::map<std::string, bool> g_loaded;  // cache files already read

void load_file_locked(const char* path) {
  if (!path || !*path || g_loaded[path]) return;
  g_loaded[path] = true;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[512];
  int v = 0;
  while (fscanf(f, "%511s %d", key, &v) == 2) g_tune[key] = v;
  fclose(f);
}
}  // namespace

std::string tune_key(const char* what, int64_t n, int b, int cplx, int precision, int nsys, int max_cols) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string gpu = "gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) gpu = prop.name;
  for (char& c : gpu)
    if (c == ' ') c = '_';
  char buf[512];
  snprintf(buf, sizeof(buf), "%s/%s/n%lld/b%d/c%d/p%d/s%d/m%d", what, gpu.c_str(), (long long)n, b, cplx,
           precision, nsys, max_cols);
  return buf;
}

// 1 and *value set if the key is known (in-process or in the cache file)
int tune_lookup(const char* path, const std::string& key, int* value) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  load_file_locked(path);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return 0;
  *value = it->second;
  return 1;
}

void tune_store(const char* path, const std::string& key, int value) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = value;
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d\n", key.c_str(), value);
  fclose(f);
}

void tune_forget_all() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_loaded.clear();
}

}  // namespace pdeshep

extern "C" void pdeshep_tune_reset(void) { pdeshep::tune_forget_all(); }

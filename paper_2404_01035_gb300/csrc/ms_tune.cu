// Autotuner: times every compiled tile shape and a set of z-chunk sizes for a
// context on its current state and keeps the fastest; results are cached in a
// small JSON file keyed by device, dim, N, K, dtype and grid.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "ms_rt.h"
#include "ms_trace.h"

using namespace msgb;

namespace {

std::string cache_key(const ms_ctx* c) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (auto& ch : name)
    if (ch == '"' || ch == ' ') ch = '_';
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s|d%d|N%d|K%d|%s|%dx%dx%d", name.c_str(), c->m.dim, c->m.N, c->m.NM + 1,
                c->m.dtype ? "f64" : "f32", c->m.nx, c->m.ny, c->m.nz);
  return buf;
}

// Entries are lines of the form
//   "key": {"tx": 32, "ty": 8, "split": 1, "zchunk": 16, "ms": 0.1},
std::map<std::string, std::string> read_cache(const char* path) {
  std::map<std::string, std::string> m;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    size_t a = line.find('"');
    size_t b = a == std::string::npos ? a : line.find('"', a + 1);
    size_t l = b == std::string::npos ? b : line.find('{', b);
    size_t r = l == std::string::npos ? l : line.find('}', l);
    if (r == std::string::npos) continue;
    m[line.substr(a + 1, b - a - 1)] = line.substr(l, r - l + 1);
  }
  return m;
}

void write_cache(const char* path, const std::map<std::string, std::string>& m) {
  std::ofstream out(path);
  out << "{\n";
  size_t i = 0;
  for (auto& kv : m) out << "  \"" << kv.first << "\": " << kv.second << (++i < m.size() ? ",\n" : "\n");
  out << "}\n";
}

bool parse_int(const std::string& s, const char* field, int* v) {
  size_t p = s.find(std::string("\"") + field + "\"");
  if (p == std::string::npos) return false;
  p = s.find(':', p);
  return p != std::string::npos && std::sscanf(s.c_str() + p + 1, "%d", v) == 1;
}

}  // namespace

extern "C" ms_status ms_tune(ms_ctx* c, const char* cache_path, int steps, double* best_ms) {
  TraceRange trace("ms_tune");
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  if (steps < 1) steps = 10;
  const std::string key = cache_key(c);
  auto variants = step_variants(c->m.dim, c->m.N, c->m.NM, c->m.dtype);
  std::map<std::string, std::string> cache;
  if (cache_path) {
    cache = read_cache(cache_path);
    auto it = cache.find(key);
    int tx, ty, zc, split = 0;
    if (it != cache.end() && parse_int(it->second, "tx", &tx) && parse_int(it->second, "ty", &ty) &&
        parse_int(it->second, "zchunk", &zc)) {
      parse_int(it->second, "split", &split);
      for (auto* v : variants)
        if (v->tx == tx && v->ty == ty && v->split == split) {
          if (best_ms) {
            size_t p = it->second.find("\"ms\"");
            double ms = 0;
            if (p != std::string::npos) std::sscanf(it->second.c_str() + it->second.find(':', p) + 1, "%lf", &ms);
            *best_ms = ms;
          }
          return apply_launch(c, v, zc);
        }
    }
  }
  // save the state, time every candidate from the same state, restore
  void* saved = dev_alloc(c->hook, c->state_bytes);
  if (!saved) return fail(c, MS_ERR_OOM, "tuner scratch allocation failed");
  const int cur0 = c->cur;
  const int64_t step0 = c->step;
  const double t0 = c->t;
  cudaError_t e = cudaMemcpyAsync(saved, c->buf[c->cur], c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  std::vector<int> zcs;
  if (c->m.dim == 3) {
    for (int z : {8, 12, 16, 24, 32, 64})
      if (z <= c->m.nz) zcs.push_back(z);
    if (zcs.empty()) zcs.push_back(c->m.nz);
  } else {
    zcs.push_back(1);
  }
  const StepKernel* best = nullptr;
  int best_zc = 1;
  double best_t = 1e300;
  ms_status st = MS_OK;
  for (auto* v : variants) {
    for (int zc : zcs) {
      if ((st = apply_launch(c, v, zc)) != MS_OK) break;
      c->cur = cur0;
      e = cudaMemcpyAsync(c->buf[c->cur], saved, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
      if ((st = refresh_codes(c)) != MS_OK) break;
      c->step = step0;
      c->t = t0;
      for (int i = 0; i < 2 && st == MS_OK; ++i) st = launch_one_step(c);
      cudaEventRecord(ev0, c->stream);
      for (int i = 0; i < steps && st == MS_OK; ++i) st = launch_one_step(c);
      cudaEventRecord(ev1, c->stream);
      if (st != MS_OK) break;
      if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, ev0, ev1);
      const double per = ms / steps;
      if (per < best_t) {
        best_t = per;
        best = v;
        best_zc = zc;
      }
    }
    if (st != MS_OK || e != cudaSuccess) break;
  }
  c->cur = cur0;
  cudaMemcpyAsync(c->buf[c->cur], saved, c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
  refresh_codes(c);
  cudaStreamSynchronize(c->stream);
  c->step = step0;
  c->t = t0;
  dev_free(c->hook, saved);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (st != MS_OK) return st;
  if (e != cudaSuccess) return cuda_fail(c, e, "tuning");
  if (!best) return fail(c, MS_ERR_STATE, "no tile variant ran");
  st = apply_launch(c, best, best_zc);
  if (st != MS_OK) return st;
  if (best_ms) *best_ms = best_t;
  if (cache_path) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "{\"tx\": %d, \"ty\": %d, \"split\": %d, \"zchunk\": %d, \"ms\": %.9g}",
                  best->tx, best->ty, best->split, c->lg.zchunk, best_t);
    cache[key] = buf;
    write_cache(cache_path, cache);
  }
  return MS_OK;
}

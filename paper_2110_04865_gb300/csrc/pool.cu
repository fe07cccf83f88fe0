// Caching device allocator, error messages, options and device queries.
//
// Graph construction and computation allocate large, short-lived buffers;
// cudaMalloc/cudaFree on every call would serialize the device and cost far
// more than the kernels for small graphs.  Freed blocks are kept per device
// in a size-ordered free list and reused for any request of at most the
// block's size and at least half of it.  On an allocation failure every
// cached block of the device is released and the request retried once.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace msf {

namespace {

struct Block {
  size_t bytes;
  int device;
};

std::mutex g_pool_mu;
std::multimap<std::pair<int, size_t>, void *> g_free;   // (device, bytes) -> ptr
std::unordered_map<void *, Block> g_live;                 // allocated or cached
// blocks freed behind work still queued on a stream: reusable once the event
// recorded after that work has completed
std::vector<std::pair<void *, cudaEvent_t>> g_pending;

void reclaim_pending_locked() {
  for (size_t i = 0; i < g_pending.size();) {
    if (cudaEventQuery(g_pending[i].second) == cudaSuccess) {
      auto it = g_live.find(g_pending[i].first);
      if (it != g_live.end()) g_free.emplace(std::make_pair(it->second.device, it->second.bytes), it->first);
      cudaEventDestroy(g_pending[i].second);
      g_pending[i] = g_pending.back();
      g_pending.pop_back();
    } else {
      ++i;
    }
  }
  cudaGetLastError();  // a not-ready query is not an error
}
thread_local std::string g_last_error;

size_t round_size(size_t b) {
  if (b == 0) b = 1;
  if (b <= (1u << 20)) {
    size_t r = 512;
    while (r < b) r <<= 1;
    return r;
  }
  const size_t q = 2u << 20;
  return (b + q - 1) / q * q;
}

void release_device_locked(int dev) {
  for (auto it = g_free.begin(); it != g_free.end();) {
    if (it->first.first == dev) {
      cudaFree(it->second);
      g_live.erase(it->second);
      it = g_free.erase(it);
    } else {
      ++it;
    }
  }
}

}  // namespace

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MSF_ERR_OOM : MSF_ERR_CUDA;
}

// MSF_TRACE=1 reports every cudaMalloc of the pool and every release of its
// cache to stderr (allocation churn shows up there).
bool pool_tracing() {
  static int t = -1;
  if (t < 0) {
    const char *e = std::getenv("MSF_TRACE");
    t = (e && e[0] == '1') ? 1 : 0;
  }
  return t == 1;
}

void *pool_alloc(size_t bytes, int *err) {
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t want = round_size(bytes);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pending.empty()) reclaim_pending_locked();
  auto it = g_free.lower_bound({dev, want});
  if (it != g_free.end() && it->first.first == dev && it->first.second <= 2 * want) {
    void *p = it->second;
    g_free.erase(it);
    *err = MSF_OK;
    return p;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (pool_tracing()) std::fprintf(stderr, "[msf] pool: cudaMalloc %zu bytes on device %d: %s\n", want, dev,
                                   e == cudaSuccess ? "ok" : "failed, releasing the cache");
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_device_locked(dev);
    e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *err = MSF_ERR_OOM;
      set_error("device allocation of " + std::to_string(want) + " bytes failed");
      return nullptr;
    }
  }
  g_live[p] = Block{want, dev};
  *err = MSF_OK;
  return p;
}

void pool_free(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_live.find(p);
  if (it == g_live.end()) return;
  g_free.emplace(std::make_pair(it->second.device, it->second.bytes), p);
}

void pool_free_after(void *p, cudaStream_t s) {
  if (!p) return;
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ev, s) != cudaSuccess) {
    // no event: wait for the stream instead
    cudaGetLastError();
    if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(s);
    pool_free(p);
    return;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  g_pending.emplace_back(p, ev);
}

void pool_release_all() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (auto &kv : g_free) {
    cudaFree(kv.second);
    g_live.erase(kv.second);
  }
  g_free.clear();
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

Options &options() {
  static Options o;
  return o;
}

const char *last_error_cstr() { return g_last_error.c_str(); }

}  // namespace msf

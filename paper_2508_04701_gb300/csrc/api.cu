// Library-wide state of libsirius: error messages, launch counter, scratch acquisition.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace sirius {

static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }
static thread_local bool g_count_off = false;
void count_launch(int k) {
  if (!g_count_off) g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed);
}
void set_launch_counting(bool on) { g_count_off = !on; }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

// Injected allocation failures (sirius_inject_alloc_failures): how many of the next
// library-owned scratch allocations fail as if the device were out of memory.
static std::atomic<int32_t> g_inject_oom{0};

static bool take_injected_failure() {
  int32_t k = g_inject_oom.load(std::memory_order_relaxed);
  while (k > 0) {
    if (g_inject_oom.compare_exchange_weak(k, k - 1, std::memory_order_relaxed)) return true;
  }
  return false;
}

sirius_status Scratch::acquire(void* d_scratch, size_t have, size_t need, cudaStream_t s) {
  stream = s;
  if (d_scratch) {
    if (have < need) {
      set_error("scratch buffer has %zu bytes, the call needs %zu", have, need);
      return SIRIUS_ERR_SCRATCH;
    }
    if (((uintptr_t)d_scratch & 255) != 0) {
      set_error("scratch buffer must be 256-byte aligned");
      return SIRIUS_ERR_INVALID;
    }
    base = (char*)d_scratch;
    bytes = have;
    return SIRIUS_OK;
  }
  if (need == 0) return SIRIUS_OK;
  if (take_injected_failure()) {
    set_error("scratch allocation of %zu bytes failed (injected failure)", need);
    return SIRIUS_ERR_OOM;
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, need, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMallocAsync(%zu) failed: %s", need, cudaGetErrorString(e));
    return SIRIUS_ERR_OOM;
  }
  base = (char*)p;
  bytes = need;
  owned = true;
  return SIRIUS_OK;
}

// ------------------------------------------------------------------ phase timing
namespace {
struct ProfRec {
  int phase;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_ev_pool;

cudaEvent_t pool_event() {
  if (!g_ev_pool.empty()) {
    cudaEvent_t e = g_ev_pool.back();
    g_ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

PhaseTimer::PhaseTimer(cudaStream_t s, int p) : phase(p), stream(s) {
  if (p < 0 || !g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaEvent_t e = pool_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) a = e;
}

PhaseTimer::~PhaseTimer() {
  if (!a) return;
  std::lock_guard<std::mutex> g(g_prof_mu);
  cudaEvent_t b = pool_event();
  if (b && cudaEventRecord(b, stream) == cudaSuccess) {
    g_prof.push_back(ProfRec{phase, (cudaEvent_t)a, b});
  } else {
    g_ev_pool.push_back((cudaEvent_t)a);
    if (b) g_ev_pool.push_back(b);
  }
}

Scratch::~Scratch() {
  if (owned && base) cudaFreeAsync(base, stream);
}

}  // namespace sirius

extern "C" {

int32_t sirius_version(void) { return 100; }
const char* sirius_last_error(void) { return sirius::g_err; }
uint64_t sirius_launch_count(void) { return sirius::g_launches.load(); }
int32_t sirius_device_sm_count(void) { return sirius::sm_count(); }

void sirius_profile_start(void) {
  std::lock_guard<std::mutex> g(sirius::g_prof_mu);
  for (auto& r : sirius::g_prof) {
    sirius::g_ev_pool.push_back(r.a);
    sirius::g_ev_pool.push_back(r.b);
  }
  sirius::g_prof.clear();
  sirius::g_prof_on = true;
}

sirius_status sirius_profile_stop(double* ms, int64_t* launches, int32_t nphases) {
  sirius::g_prof_on = false;
  std::lock_guard<std::mutex> g(sirius::g_prof_mu);
  for (int32_t p = 0; p < nphases; ++p) {
    if (ms) ms[p] = 0;
    if (launches) launches[p] = 0;
  }
  sirius_status st = SIRIUS_OK;
  for (auto& r : sirius::g_prof) {
    float t = 0;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      st = SIRIUS_ERR_CUDA;
    } else if (r.phase >= 0 && r.phase < nphases) {
      if (ms) ms[r.phase] += t;
      if (launches) launches[r.phase] += 1;
    }
    sirius::g_ev_pool.push_back(r.a);
    sirius::g_ev_pool.push_back(r.b);
  }
  sirius::g_prof.clear();
  return st;
}

}  // extern "C"

extern "C" int32_t sirius_inject_alloc_failures(int32_t count) {
  return sirius::g_inject_oom.exchange(count < 0 ? 0 : count, std::memory_order_relaxed);
}

// Status, last-error and counter entry points.
#include <stdarg.h>
#include <stdio.h>

#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "host.hpp"

namespace mpc {

// One status word per device that loads the library (see record_status()).
__device__ int g_device_status = 0;

int* device_status_ptr() {
  static int* cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (cached[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    cached[dev] = static_cast<int*>(p);
  }
  return cached[dev];
}

namespace {
thread_local char t_last_error[512] = "";

std::atomic<uint64_t> s_calls{0}, s_rounds{0}, s_bytes{0}, s_and{0}, s_triples{0}, s_macs{0},
    s_launches{0};

// Profiling state: per kernel name, the event pairs recorded since the last reset.
struct ProfSlot {
  std::string name;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs;
  size_t used = 0;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfSlot> g_prof;
}  // namespace

KernelTimer::KernelTimer(const char* name, cudaStream_t s) : slot_(-1), s_(s) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  int i = 0;
  for (; i < (int)g_prof.size(); ++i)
    if (g_prof[i].name == name) break;
  if (i == (int)g_prof.size()) {
    g_prof.emplace_back();
    g_prof.back().name = name;
  }
  ProfSlot& ps = g_prof[i];
  if (ps.used == ps.pairs.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    ps.pairs.emplace_back(a, b);
  }
  if (cudaEventRecord(ps.pairs[ps.used].first, s) != cudaSuccess) return;
  slot_ = i;
}

KernelTimer::~KernelTimer() {
  if (slot_ < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfSlot& ps = g_prof[slot_];
  if (cudaEventRecord(ps.pairs[ps.used].second, s_) == cudaSuccess) ps.used++;
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  s_launches.fetch_add(1, std::memory_order_relaxed);
  return MPC_OK;
}

void stats_add(uint64_t rounds, uint64_t bytes_opened, uint64_t and_gates, uint64_t triple_words,
               uint64_t ring_macs) {
  s_calls.fetch_add(1, std::memory_order_relaxed);
  s_rounds.fetch_add(rounds, std::memory_order_relaxed);
  s_bytes.fetch_add(bytes_opened, std::memory_order_relaxed);
  s_and.fetch_add(and_gates, std::memory_order_relaxed);
  s_triples.fetch_add(triple_words, std::memory_order_relaxed);
  s_macs.fetch_add(ring_macs, std::memory_order_relaxed);
}

}  // namespace mpc

extern "C" {

const char* mpc_last_error(void) { return mpc::t_last_error; }

int mpc_sync_status(void* stream) {
  cudaError_t e = cudaStreamSynchronize(mpc::as_stream(stream));
  if (e != cudaSuccess) return mpc::fail(MPC_ECUDA, "stream: %s", cudaGetErrorString(e));
  int status = 0;
  e = cudaMemcpyFromSymbol(&status, mpc::g_device_status, sizeof(int));
  if (e != cudaSuccess) return mpc::fail(MPC_ECUDA, "status read: %s", cudaGetErrorString(e));
  if (status != 0) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(mpc::g_device_status, &zero, sizeof(int));
    if (e != cudaSuccess) return mpc::fail(MPC_ECUDA, "status clear: %s", cudaGetErrorString(e));
    return mpc::fail(status, "device reported status %d", status);
  }
  return MPC_OK;
}

int mpc_get_stats(mpc_stats_t* out) {
  MPC_REQUIRE(out != nullptr, "null stats pointer");
  out->calls = mpc::s_calls.load();
  out->rounds = mpc::s_rounds.load();
  out->bytes_opened = mpc::s_bytes.load();
  out->and_gates = mpc::s_and.load();
  out->triple_words = mpc::s_triples.load();
  out->ring_macs = mpc::s_macs.load();
  out->launches = mpc::s_launches.load();
  return MPC_OK;
}

int mpc_reset_stats(void) {
  mpc::s_calls = 0;
  mpc::s_rounds = 0;
  mpc::s_bytes = 0;
  mpc::s_and = 0;
  mpc::s_triples = 0;
  mpc::s_macs = 0;
  mpc::s_launches = 0;
  return MPC_OK;
}

int mpc_profile_enable(int on) {
  mpc::g_prof_on.store(on != 0);
  return MPC_OK;
}

int mpc_profile_reset(void) {
  std::lock_guard<std::mutex> lk(mpc::g_prof_mu);
  for (auto& ps : mpc::g_prof) ps.used = 0;
  return MPC_OK;
}

int mpc_profile_read(const char* kernel, uint64_t* launches, double* total_ms) {
  MPC_REQUIRE(kernel && launches && total_ms, "null pointer");
  std::lock_guard<std::mutex> lk(mpc::g_prof_mu);
  *launches = 0;
  *total_ms = 0.0;
  for (auto& ps : mpc::g_prof) {
    if (ps.name != kernel) continue;
    for (size_t i = 0; i < ps.used; ++i) {
      cudaError_t e = cudaEventSynchronize(ps.pairs[i].second);
      if (e != cudaSuccess) return mpc::fail(MPC_ECUDA, "profile sync: %s", cudaGetErrorString(e));
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ps.pairs[i].first, ps.pairs[i].second);
      if (e != cudaSuccess) return mpc::fail(MPC_ECUDA, "profile read: %s", cudaGetErrorString(e));
      *total_ms += ms;
    }
    *launches = ps.used;
  }
  return MPC_OK;
}

int mpc_profile_busy(const char* kernel, double* busy_ms) {
  MPC_REQUIRE(kernel && busy_ms, "null pointer");
  std::lock_guard<std::mutex> lk(mpc::g_prof_mu);
  *busy_ms = 0.0;
  std::vector<std::pair<double, double>> iv;
  cudaEvent_t ref = nullptr;
  for (auto& ps : mpc::g_prof) {
    if (ps.name != kernel) continue;
    for (size_t i = 0; i < ps.used; ++i) {
      cudaError_t e = cudaEventSynchronize(ps.pairs[i].second);
      if (e != cudaSuccess) return mpc::fail(MPC_ECUDA, "profile sync: %s", cudaGetErrorString(e));
      if (!ref) ref = ps.pairs[i].first;
      float a = 0.f, b = 0.f;
      e = cudaEventElapsedTime(&a, ref, ps.pairs[i].first);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ref, ps.pairs[i].second);
      if (e != cudaSuccess) return mpc::fail(MPC_ECUDA, "profile read: %s", cudaGetErrorString(e));
      iv.emplace_back((double)a, (double)b);
    }
  }
  std::sort(iv.begin(), iv.end());
  double cur_a = 0.0, cur_b = 0.0;
  bool open = false;
  for (const auto& x : iv) {
    if (open && x.first <= cur_b) {
      cur_b = std::max(cur_b, x.second);
    } else {
      if (open) *busy_ms += cur_b - cur_a;
      cur_a = x.first;
      cur_b = x.second;
      open = true;
    }
  }
  if (open) *busy_ms += cur_b - cur_a;
  return MPC_OK;
}

}  // extern "C"

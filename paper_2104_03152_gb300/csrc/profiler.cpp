// Launch accounting and the optional kernel profiler.
//
// Every kernel launch of the library goes through a Launch scope, which counts it. While profiling
// is on, the scope also records a CUDA event before and after the launch on the launching stream
// and remembers the launch's algorithmic bytes (each operand read once, each result written once,
// each distinct key read once), so device time and bandwidth per kernel family can be read back.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/tcks.h"
#include "kernels.h"

namespace tcks {

namespace {

const char* const kNames[K_COUNT] = {"ntt_fwd",      "ntt_inv",    "elementwise", "tensor",    "drop_combine",
                                     "modup",        "ks_inner_p", "ks_moddown",  "vecmat_reduce", "keygen",
                                     "encrypt",      "encode",     "decode",      "vecmat_acc", "decrypt",
                                     "vecmat_dh_acc", "lincomb", "combine"};

struct Rec {
  u32 id;
  cudaEvent_t a, b;
  double bytes, ops;
  u32 tag;
};

struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

Prof& prof() {
  static Prof p;
  return p;
}

std::atomic<unsigned long long> g_launches{0};
std::atomic<bool> g_on{false};

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(u64 n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

Launch::Launch(KernelId id, cudaStream_t st, double algo_bytes, double algo_ops, u32 tag)
    : id_(id), st_(st), bytes_(algo_bytes), ops_(algo_ops), tag_(tag) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;  // no events in graphs
  Prof& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  a_ = p.get();
  cudaEventRecord((cudaEvent_t)a_, st);
  active_ = true;
}

Launch::~Launch() {
  if (!active_) return;
  Prof& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  cudaEvent_t b = p.get();
  cudaEventRecord(b, st_);
  p.recs.push_back(Rec{(u32)id_, (cudaEvent_t)a_, b, bytes_, ops_, tag_});
}

}  // namespace tcks

using namespace tcks;

extern "C" {

uint64_t tcks_launch_count(void) { return g_launches.load(); }

tcks_status tcks_profile_start(void) {
  Prof& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  for (Rec& r : p.recs) {
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.recs.clear();
  p.on = true;
  g_on.store(true);
  return TCKS_OK;
}

tcks_status tcks_profile_stop(void) {
  g_on.store(false);
  prof().on = false;
  return TCKS_OK;
}

uint32_t tcks_profile_count(void) { return K_COUNT; }

tcks_status tcks_profile_read(uint32_t idx, const char** name, uint64_t* launches, double* ms, double* algo_bytes) {
  if (idx >= K_COUNT) return TCKS_ERR_INVALID_ARG;
  Prof& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  uint64_t n = 0;
  double t = 0, by = 0;
  for (const Rec& r : p.recs) {
    if (r.id != idx) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return TCKS_ERR_CUDA;
    float e = 0;
    if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) return TCKS_ERR_CUDA;
    ++n;
    t += e;
    by += r.bytes;
  }
  if (name) *name = kNames[idx];
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (algo_bytes) *algo_bytes = by;
  return TCKS_OK;
}

tcks_status tcks_profile_read_ops(uint32_t idx, double* algo_ops) {
  if (idx >= K_COUNT || !algo_ops) return TCKS_ERR_INVALID_ARG;
  Prof& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  double ops = 0;
  for (const Rec& r : p.recs)
    if (r.id == idx) ops += r.ops;
  *algo_ops = ops;
  return TCKS_OK;
}

tcks_status tcks_profile_records(uint32_t idx, uint32_t capacity, uint32_t* tags, double* ms, double* algo_ops,
                                 uint32_t* count) {
  if (idx >= K_COUNT || !count) return TCKS_ERR_INVALID_ARG;
  Prof& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  uint32_t n = 0;
  for (const Rec& r : p.recs) {
    if (r.id != idx) continue;
    if (n < capacity) {
      if (cudaEventSynchronize(r.b) != cudaSuccess) return TCKS_ERR_CUDA;
      float e = 0;
      if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) return TCKS_ERR_CUDA;
      if (tags) tags[n] = r.tag;
      if (ms) ms[n] = e;
      if (algo_ops) algo_ops[n] = r.ops;
    }
    ++n;
  }
  *count = n;
  return TCKS_OK;
}

}  // extern "C"

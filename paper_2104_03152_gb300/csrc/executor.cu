// Persistent executor: one kernel, resident for as long as there is work, that takes NTT / INTT tasks
// from a queue instead of one launch per job -- the device-side counterpart of the batched launches
// for streams of small jobs (a serving loop's transforms) where a launch costs as much as the work.
//
// The queue is a ring of one-limb tasks in pinned, mapped host memory: the host writes tasks, then
// publishes them by a release store of `tail`; each CTA claims the next task index with an atomic on
// a device counter, waits until the index is published, transforms that limb in shared memory and,
// once its stores are visible to the system, marks the slot finished with the task's index. Tasks
// finish in any order, so the host reads completion per slot: it reuses a slot only once the task it
// held is marked, and a ticket is complete once every task up to it is. Every wait is bounded: a CTA that sees no
// published task within the idle limit (measured with the GPU's global timer, and capped at an
// iteration count as well) writes TCKS_ERR_TIMEOUT to the status word, and every CTA leaves when it
// sees a non-zero status or the close flag. Nothing ever waits on another kernel.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <cuda/atomic>
#include <thread>

#include "context.h"
#include "debug_checks.cuh"
#include "limb_launch.cuh"
#include "ntt.cuh"

using namespace tcks;

namespace tcks {
void count_launch();
}  // namespace tcks

namespace {

struct ExecTask {
  const u64* src;  // one limb of N words
  u64* dst;
  u32 mod;
  u32 inverse;
  unsigned long long finished;  // index + 1 of the last task of this slot whose results are stored (device)
};

// Host-mapped control block followed by the task ring.
struct ExecQueue {
  unsigned long long tail;    // tasks published (host, release)
  int status;                 // 0, or TCKS_ERR_TIMEOUT written by the kernel
  int closed;                 // set by the host to end the kernel
  unsigned long long pad[6];  // keeps the ring 64-byte aligned
  ExecTask tasks[1];
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename W>
__global__ void k_executor(DevTables T, ExecQueue* q, unsigned long long* head, u32 capacity,
                           unsigned long long idle_ns, unsigned long long max_spins) {
  TCKS_SMEM(W);
  __shared__ ExecTask task;
  __shared__ int stop;
  const u32 n = 1u << T.log_n;
  unsigned long long idx = 0;  // thread 0's current task
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> tail(q->tail);
  cuda::atomic_ref<int, cuda::thread_scope_system> status(q->status), closed(q->closed);
  for (;;) {
    if (threadIdx.x == 0) {
      idx = atomicAdd(head, 1ull);
      stop = 0;
      // idle = no task published at all: the limits restart whenever the tail moves
      unsigned long long t0 = global_ns(), seen = tail.load(cuda::memory_order_relaxed), spins = 0;
      for (;;) {
        const unsigned long long t = tail.load(cuda::memory_order_acquire);
        if (t > idx) break;
        if (closed.load(cuda::memory_order_relaxed) || status.load(cuda::memory_order_relaxed)) {
          stop = 1;
          break;
        }
        if (t != seen) {
          seen = t;
          t0 = global_ns();
          spins = 0;
        } else if (global_ns() - t0 > idle_ns || ++spins > max_spins) {  // nothing published in time
          status.store(TCKS_ERR_TIMEOUT, cuda::memory_order_relaxed);
          stop = 1;
          break;
        }
        __nanosleep(1000);
      }
      if (!stop) {  // ordered after the acquire of tail
        const volatile ExecTask* v = &q->tasks[idx % capacity];
        task.src = (const u64*)v->src;
        task.dst = (u64*)v->dst;
        task.mod = v->mod;
        task.inverse = v->inverse;
        if (dbg_fail(T.dbg, task.mod < T.n_mods, DBG_MOD_INDEX) | dbg_fail(T.dbg, task.src && task.dst, DBG_NULL)) {
          status.store(TCKS_ERR_DEBUG_CHECK, cuda::memory_order_relaxed);  // debug builds: stop on a bad task
          stop = 1;
        }
      }
    }
    __syncthreads();
    if (stop) return;
    const ModConst m = T.mods[task.mod];
    for (u32 k = 2 * threadIdx.x; k < n; k += 2 * blockDim.x) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(task.src + k);
      s[sw(k)] = (W)v.x;
      s[sw(k + 1)] = (W)v.y;
    }
    __syncthreads();
    if (task.inverse) {
      ntt_inv_slice<W, 0>(s, T, task.mod, 0);
      for (u32 k = 2 * threadIdx.x; k < n; k += 2 * blockDim.x)
        *reinterpret_cast<ulonglong2*>(task.dst + k) =
            make_ulonglong2(Ar<W>::inv_out(s[sw(k)], m), Ar<W>::inv_out(s[sw(k + 1)], m));
    } else {
      ntt_fwd_slice<W, 0>(s, T, task.mod, 0);
      for (u32 k = 2 * threadIdx.x; k < n; k += 2 * blockDim.x)
        *reinterpret_cast<ulonglong2*>(task.dst + k) =
            make_ulonglong2(Ar<W>::fwd_out(s[sw(k)], m), Ar<W>::fwd_out(s[sw(k + 1)], m));
    }
    __syncthreads();  // every thread's stores are issued before the task is marked
    if (threadIdx.x == 0) {
      __threadfence_system();
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_system>(q->tasks[idx % capacity].finished)
          .store(idx + 1, cuda::memory_order_release);
    }
  }
}

}  // namespace

struct tcks_executor {
  tcks_ctx* ctx = nullptr;     // retained
  cudaStream_t stream = nullptr;
  ExecQueue* hq = nullptr;     // host view
  ExecQueue* dq = nullptr;     // device view of the same mapped memory
  unsigned long long* head = nullptr;  // device claim counter
  unsigned long long prefix = 0;       // every task below this index has finished (host view)
  u32 capacity = 0;
  bool running = false;
};

#define EXEC_BEGIN                 \
  try {                            \
    tcks::NvtxRange tcks_nvtx_range_(__func__); \
    tcks::drop_stale_cuda_error();
#define EXEC_END                                                     \
  }                                                                  \
  catch (const tcks::Error& e) {                                     \
    return tcks::abi_record(e.code, e.msg);                          \
  }                                                                  \
  catch (const std::bad_alloc&) {                                    \
    return tcks::abi_record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed"); \
  }                                                                  \
  tcks::abi_clear();                                                 \
  return TCKS_OK;

namespace {

unsigned long long host_load(const unsigned long long* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }
int host_load_int(const int* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

void executor_release(tcks_executor* e) {
  if (!e) return;
  if (e->stream) {
    cudaStreamSynchronize(e->stream);
    cudaStreamDestroy(e->stream);
  }
  if (e->head) e->ctx->dev_free(e->head);
  if (e->hq) cudaFreeHost(e->hq);
  if (e->ctx) ctx_release(e->ctx);
  delete e;
  cudaGetLastError();  // clean-up statuses are not reported
}

}  // namespace

extern "C" {

tcks_status tcks_executor_start(tcks_ctx* c, uint32_t capacity, int64_t idle_timeout_ns, tcks_executor** out) {
  struct Guard {
    tcks_executor* e = nullptr;
    ~Guard() { executor_release(e); }
  } guard;
  EXEC_BEGIN
  if (!c || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (c->params.log_n > 13) fail(TCKS_ERR_UNSUPPORTED, "the executor transforms limbs of N <= 2^13 (one CTA each)");
  if (capacity < 1 || capacity > (1u << 24)) fail(TCKS_ERR_INVALID_ARG, "capacity must be in [1, 2^24] tasks");
  if (idle_timeout_ns <= 0) fail(TCKS_ERR_INVALID_ARG, "the idle limit must be positive");
  guard.e = new tcks_executor();
  tcks_executor* e = guard.e;
  e->ctx = c;
  ctx_retain(c);
  e->capacity = capacity;
  const size_t bytes = sizeof(ExecQueue) + sizeof(ExecTask) * ((size_t)capacity - 1);
  check_cuda(cudaHostAlloc((void**)&e->hq, bytes, cudaHostAllocMapped), "executor queue");
  std::memset((void*)e->hq, 0, bytes);
  check_cuda(cudaHostGetDevicePointer((void**)&e->dq, e->hq, 0), "executor queue");
  e->head = (unsigned long long*)c->dev_alloc(sizeof(unsigned long long));
  check_cuda(cudaMemsetAsync(e->head, 0, sizeof(unsigned long long), c->stream), "executor head");
  check_cuda(cudaStreamSynchronize(c->stream), "executor head");
  check_cuda(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking), "executor stream");
  int sms = 0;
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device), "SM count");
  const LimbShape sh = limb_shape(c->params.log_n);
  const size_t smem = c->T.narrow ? sh.smem / 2 : sh.smem;
  const unsigned long long idle = (unsigned long long)idle_timeout_ns;
  const unsigned long long max_spins = idle / 500 + 4096;  // each spin sleeps about a microsecond
  const void* k = c->T.narrow ? (const void*)k_executor<u32> : (const void*)k_executor<u64>;
  ensure_smem(k, smem);
  count_launch();
  if (c->T.narrow)
    k_executor<u32><<<(u32)sms, sh.threads, smem, e->stream>>>(c->T, e->dq, e->head, capacity, idle, max_spins);
  else
    k_executor<u64><<<(u32)sms, sh.threads, smem, e->stream>>>(c->T, e->dq, e->head, capacity, idle, max_spins);
  check_launch("executor");
  e->running = true;
  *out = e;
  guard.e = nullptr;
  EXEC_END
}

tcks_status tcks_executor_post(tcks_executor* e, uint32_t op, const uint64_t* d_in, uint64_t* d_out, uint32_t polys,
                               uint32_t level, uint64_t* ticket) {
  EXEC_BEGIN
  if (!e || !d_in || !d_out || !ticket) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (op != TCKS_EXEC_NTT && op != TCKS_EXEC_INTT) fail(TCKS_ERR_INVALID_ARG, "unknown op");
  tcks_ctx* c = e->ctx;
  if (level < 1 || level > c->L + c->K) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  const int st = host_load_int(&e->hq->status);
  if (st)
    fail((tcks_status)st, st == TCKS_ERR_TIMEOUT ? "the executor has stopped: no task was published within its idle limit"
                                                 : "the executor has stopped on a task that failed a debug range check");
  if (e->hq->closed) fail(TCKS_ERR_INVALID_ARG, "the executor is closed");
  const unsigned long long count = (unsigned long long)polys * level;
  if (count > e->capacity) fail(TCKS_ERR_INVALID_ARG, "more tasks than the queue holds");
  const unsigned long long t = e->hq->tail;
  const u64 n = c->N;
  const auto t0 = std::chrono::steady_clock::now();
  for (unsigned long long k = 0; k < count; ++k) {
    ExecTask& task = e->hq->tasks[(t + k) % e->capacity];
    // the slot is free once the task it held (index t + k - capacity) has finished (bounded wait)
    const unsigned long long prev = t + k >= e->capacity ? t + k - e->capacity + 1 : 0;
    while (host_load(&task.finished) < prev) {
      if (host_load_int(&e->hq->status)) fail(TCKS_ERR_TIMEOUT, "the executor stopped while the queue was full");
      if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(10))
        fail(TCKS_ERR_TIMEOUT, "no queue slot freed within 10 s");
      std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    task.src = d_in + k * n;
    task.dst = d_out + k * n;
    task.mod = (u32)(k % level);
    task.inverse = op == TCKS_EXEC_INTT ? 1u : 0u;
  }
  __atomic_store_n(&e->hq->tail, t + count, __ATOMIC_RELEASE);
  *ticket = t + count;
  EXEC_END
}

tcks_status tcks_executor_wait(tcks_executor* e, uint64_t ticket, int64_t timeout_ns) {
  EXEC_BEGIN
  if (!e) fail(TCKS_ERR_INVALID_ARG, "null executor");
  if (ticket > e->hq->tail) fail(TCKS_ERR_INVALID_ARG, "ticket beyond the last posted task");
  const auto t0 = std::chrono::steady_clock::now();
  auto pause = std::chrono::microseconds(1);
  for (;;) {
    // a slot is reused only after its task finished, so a mark >= index + 1 means that task finished
    while (e->prefix < ticket && host_load(&e->hq->tasks[e->prefix % e->capacity].finished) >= e->prefix + 1)
      ++e->prefix;
    if (e->prefix >= ticket) break;
    const int st = host_load_int(&e->hq->status);
    if (st) fail((tcks_status)st, "the executor stopped before the ticket's tasks completed");
    if (timeout_ns >= 0 && std::chrono::steady_clock::now() - t0 >= std::chrono::nanoseconds(timeout_ns))
      fail(TCKS_ERR_TIMEOUT, "the ticket's tasks have not completed within " + std::to_string(timeout_ns) + " ns");
    std::this_thread::sleep_for(pause);
    if (pause < std::chrono::microseconds(50)) pause *= 2;
  }
  EXEC_END
}

tcks_status tcks_executor_close(tcks_executor* e, int32_t* device_status) {
  EXEC_BEGIN
  if (!e) fail(TCKS_ERR_INVALID_ARG, "null executor");
  __atomic_store_n(&e->hq->closed, 1, __ATOMIC_RELEASE);
  // every wait in the kernel checks the flag; give it (bounded) time to leave
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t q;
  while ((q = cudaStreamQuery(e->stream)) == cudaErrorNotReady) {
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(30))
      fail(TCKS_ERR_TIMEOUT, "the executor kernel did not leave within 30 s of the close");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  if (q != cudaSuccess) fail(TCKS_ERR_CUDA, std::string("executor: ") + cudaGetErrorString(q));
  if (device_status) *device_status = host_load_int(&e->hq->status);
  e->running = false;
  EXEC_END
}

void tcks_executor_free(tcks_executor* e) {
  if (!e) return;
  if (e->running) tcks_executor_close(e, nullptr);
  executor_release(e);
}

}  // extern "C"

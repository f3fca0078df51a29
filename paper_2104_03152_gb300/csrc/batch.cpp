// Batched launches over a descriptor table of independent jobs (several contexts, N and levels):
// the device-side replacement for the CPU thread pool that runs TenSEAL's per-ciphertext work.
//   * NTT / INTT jobs: with several contexts of N in [2^13, 2^16] and one word type, one columns launch
//     and one slices launch per direction for all of them (mixed N, levels and buffers); otherwise per
//     context, one launch of k_ntt_desc over its jobs, split only past kNttDescMax batches;
//   * relinearize / rotate jobs: the batched key-switch sequence (ModUp, inner product, ModDown)
//     per job, in sub-batches whose scratch stays under a fixed bound;
//   * each context's work is queued on its own stream, forked from and joined back into the first
//     job's context stream, so that different N overlap on the device.
// The whole batch can be captured once as a CUDA graph and replayed.
#include <algorithm>
#include <chrono>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "context.h"
#include "debug_checks.cuh"

using namespace tcks;

namespace tcks {

namespace {

constexpr u64 kScratchBound = 4ull << 30;  // bytes of key-switch scratch per sub-batch

// Key-switch scratch words per ciphertext at level ell: coefficients, digits, P limbs.
u64 ks_scratch_words(const tcks_ctx* c, u32 ell) {
  return (u64)ell * c->N + ks_digit_words(c, ell) + ks_top_words(c);
}

// log2 of the CTAs per limb of the limb kernels (clusters above N = 2^14)
u32 cluster_log(const tcks_ctx* c) { return c->params.log_n > 14 ? c->params.log_n - 14 : 0; }

u32 sub_batch(const tcks_ctx* c, u32 ell, u32 count) {
  const u64 per = ks_scratch_words(c, ell) * 8;
  return (u32)std::max<u64>(1, std::min<u64>(count, kScratchBound / per));
}

// Rotation of `count` ciphertexts [count][2][ell][N] by one step: out = tau_g(c0) + ModDown(<digits, gk_0>),
// ModDown(<digits, gk_1>) with the automorphism folded into the reads.
void op_rotate_batch(tcks_ctx* c, const u64* in, u32 count, u32 ell, int32_t step, u64* out) {
  const size_t n = c->N;
  const u64 cw = ct_words(c, ell);
  const u32 k = step_mod(c, step);
  if (k == 0) {
    check_cuda(cudaMemcpyAsync(out, in, (size_t)count * cw * 8, cudaMemcpyDeviceToDevice, c->stream), "rotate by 0");
    return;
  }
  const KeyTable& kt = key_table(c, {k}, ell);
  const u32 sb = sub_batch(c, ell, count);
  const u64 dw = ks_digit_words(c, ell);
  DevBuf coef(c, (size_t)sb * ell * n), digits(c, (size_t)sb * dw), top(c, (size_t)sb * ks_top_words(c));
  for (u32 b0 = 0; b0 < count; b0 += sb) {
    const u32 bn = std::min(sb, count - b0);
    const u64* src = in + (size_t)b0 * cw;
    ks_modup(c, src + (size_t)ell * n, cw, bn, ell, coef.p, digits.p);
    KsPlan p{};
    p.keys = kt.d;
    p.digits = digits.p;
    p.digits_b = dw;
    p.top = top.p;
    p.out = out + (size_t)b0 * cw;
    p.out_b = cw;
    p.add0 = src;
    p.add0_b = cw;
    p.R = 1;
    p.B = bn;
    p.add_perm = 1;
    ks_switch(c, ell, p);
  }
  check_launch("rotate batch");
}

void op_relin_batch(tcks_ctx* c, const u64* in, u32 count, u32 ell, u64* out) {
  const u32 sb = sub_batch(c, ell, count);
  const u64 w3 = (u64)3 * ell * c->N, w2 = ct_words(c, ell);
  for (u32 b0 = 0; b0 < count; b0 += sb)
    op_relinearize(c, in + (size_t)b0 * w3, ell, out + (size_t)b0 * w2, std::min(sb, count - b0));
}

void validate(const tcks_batch_job* jobs, u32 n_jobs) {
  if (!jobs || !n_jobs) fail(TCKS_ERR_INVALID_ARG, "empty job list");
  for (u32 i = 0; i < n_jobs; ++i) {
    const tcks_batch_job& j = jobs[i];
    if (!j.ctx || (j.count && (!j.d_in || !j.d_out)))
      fail(TCKS_ERR_INVALID_ARG, "job " + std::to_string(i) + ": null pointer");
    tcks_ctx* c = j.ctx;
    switch (j.op) {
      case TCKS_JOB_NTT:
      case TCKS_JOB_INTT:
        if (j.level < 1 || j.level > c->L + 1) fail(TCKS_ERR_INVALID_ARG, "job " + std::to_string(i) + ": level out of range");
        if ((u64)j.count * j.level > 0x7fffffffull >> cluster_log(c))
          fail(TCKS_ERR_INVALID_ARG, "job " + std::to_string(i) + ": too many limbs for one launch");
        break;
      case TCKS_JOB_RELIN:
        if (j.level < 1 || j.level > c->L) fail(TCKS_ERR_INVALID_ARG, "job " + std::to_string(i) + ": level out of range");
        key_table(c, {0u}, j.level);
        break;
      case TCKS_JOB_ROTATE:
        if (j.level < 1 || j.level > c->L) fail(TCKS_ERR_INVALID_ARG, "job " + std::to_string(i) + ": level out of range");
        if (step_mod(c, j.step)) galois_key_for(c, j.step, j.level);
        if (j.count && j.d_in == j.d_out) fail(TCKS_ERR_INVALID_ARG, "job " + std::to_string(i) + ": rotation output overlaps input");
        break;
      default:
        fail(TCKS_ERR_INVALID_ARG, "job " + std::to_string(i) + ": unknown op");
    }
  }
  if (kDebugChecks) {  // jobs of one batch may run concurrently: no job writes what another touches
    auto extent = [](const tcks_batch_job& j, bool out) -> u64 {
      const u64 limb = (u64)j.ctx->N * 8;
      const u32 polys = j.op == TCKS_JOB_NTT || j.op == TCKS_JOB_INTT ? 1 : (j.op == TCKS_JOB_RELIN && !out ? 3 : 2);
      return (u64)j.count * polys * j.level * limb;
    };
    auto overlap = [](const void* a, u64 na, const void* b, u64 nb) {
      const char *x = (const char*)a, *y = (const char*)b;
      return na && nb && x < y + nb && y < x + na;
    };
    for (u32 i = 0; i < n_jobs; ++i)
      for (u32 k = 0; k < n_jobs; ++k) {
        if (i == k) continue;
        const tcks_batch_job &a = jobs[i], &b = jobs[k];
        if (overlap(a.d_out, extent(a, true), b.d_out, extent(b, true)) ||
            overlap(a.d_out, extent(a, true), b.d_in, extent(b, false)))
          fail(TCKS_ERR_DEBUG_CHECK, "job " + std::to_string(i) + " writes memory that job " + std::to_string(k) + " uses");
      }
  }
}

void run_ctx_ntt(tcks_ctx* c, const std::vector<const tcks_batch_job*>& js, bool inverse) {
  NttDescTable tab{};
  u32 total = 0;
  auto flush = [&]() {
    if (kDebugChecks) {  // offsets from 0, monotone, adding up to the launch
      u32 at = 0;
      for (u32 i = 0; i < tab.n; ++i) {
        if (tab.d[i].first != at || !tab.d[i].level || tab.d[i].limbs % tab.d[i].level)
          fail(TCKS_ERR_DEBUG_CHECK, "NTT descriptor " + std::to_string(i) + " out of order or range");
        at += tab.d[i].limbs;
      }
      if (at != total) fail(TCKS_ERR_DEBUG_CHECK, "NTT descriptors do not add up to the launch");
    }
    launch_ntt_desc(c->T, inverse, tab, total, c->stream);
    tab.n = 0;
    total = 0;
  };
  for (const tcks_batch_job* j : js) {
    if (!j->count) continue;
    const u64 limbs = (u64)j->count * j->level;
    if (tab.n == kNttDescMax || total + limbs > (0x7fffffffull >> cluster_log(c))) flush();
    tab.d[tab.n++] = NttDesc{j->d_in, j->d_out, total, j->level, (u32)limbs, 0};
    total += (u32)limbs;
  }
  flush();
  check_launch("batched NTT");
}

// Queue every job; contexts other than the first run on their own streams between a fork and a join.
void run_jobs(const tcks_batch_job* jobs, u32 n_jobs) {
  std::vector<tcks_ctx*> order;
  std::map<tcks_ctx*, std::vector<const tcks_batch_job*>> by_ctx;
  for (u32 i = 0; i < n_jobs; ++i) {
    if (!by_ctx.count(jobs[i].ctx)) order.push_back(jobs[i].ctx);
    by_ctx[jobs[i].ctx].push_back(&jobs[i]);
  }
  cudaStream_t origin = order[0]->stream;
  std::vector<cudaEvent_t> events;
  struct Events {
    std::vector<cudaEvent_t>& v;
    ~Events() {
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
  } guard{events};
  auto new_event = [&]() {
    cudaEvent_t e;
    check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    events.push_back(e);
    return e;
  };
  // The NTT / INTT jobs of every context (N >= 2^13, one word type) as one columns launch and one
  // slices launch per direction on the first job's stream; otherwise per context, below.
  bool multi_done = false;
  if (order.size() > 1) {
    std::vector<MultiNttBatch> fwd_b, inv_b;
    for (u32 i = 0; i < n_jobs; ++i) {
      const tcks_batch_job& j = jobs[i];
      if (!j.count || (j.op != TCKS_JOB_NTT && j.op != TCKS_JOB_INTT)) continue;
      (j.op == TCKS_JOB_NTT ? fwd_b : inv_b).push_back(MultiNttBatch{&j.ctx->T, j.d_in, j.d_out, j.count, j.level});
    }
    auto fits = [](const std::vector<MultiNttBatch>& b) {
      if (b.empty()) return true;
      if (b.size() > kMultiDescMax) return false;
      std::vector<const void*> ctxs;
      for (const MultiNttBatch& x : b) {
        if (x.T->log_n < 13 || x.T->log_n > 16 || x.T->narrow != b[0].T->narrow) return false;
        if (std::find(ctxs.begin(), ctxs.end(), (const void*)x.T->mods) == ctxs.end()) ctxs.push_back(x.T->mods);
      }
      return ctxs.size() <= kMultiCtxMax;
    };
    if (fits(fwd_b) && fits(inv_b) && (!fwd_b.empty() || !inv_b.empty())) {
      if (!fwd_b.empty()) launch_ntt_multi(false, fwd_b.data(), (u32)fwd_b.size(), origin);
      if (!inv_b.empty()) launch_ntt_multi(true, inv_b.data(), (u32)inv_b.size(), origin);
      check_launch("batched NTT over contexts");
      multi_done = true;
    }
  }
  cudaEvent_t fork = new_event();
  check_cuda(cudaEventRecord(fork, origin), "fork");
  for (tcks_ctx* c : order) {
    if (c->stream != origin) check_cuda(cudaStreamWaitEvent(c->stream, fork, 0), "fork wait");
    const auto& js = by_ctx[c];
    std::vector<const tcks_batch_job*> fwd, inv;
    for (const tcks_batch_job* j : js) {
      if (j->op == TCKS_JOB_NTT) fwd.push_back(j);
      if (j->op == TCKS_JOB_INTT) inv.push_back(j);
    }
    if (!multi_done && !fwd.empty()) run_ctx_ntt(c, fwd, false);
    if (!multi_done && !inv.empty()) run_ctx_ntt(c, inv, true);
    for (const tcks_batch_job* j : js) {
      if (!j->count) continue;
      if (j->op == TCKS_JOB_RELIN) op_relin_batch(c, j->d_in, j->count, j->level, j->d_out);
      if (j->op == TCKS_JOB_ROTATE) op_rotate_batch(c, j->d_in, j->count, j->level, j->step, j->d_out);
    }
    if (c->stream != origin) {
      cudaEvent_t join = new_event();
      check_cuda(cudaEventRecord(join, c->stream), "join");
      check_cuda(cudaStreamWaitEvent(origin, join, 0), "join wait");
    }
  }
}

}  // namespace

}  // namespace tcks

struct tcks_batch {
  std::vector<tcks_ctx*> ctxs;  // retained until the handle is freed
  cudaEvent_t done = nullptr;   // recorded on the origin stream after every job (and join)
};

struct tcks_batch_graph {
  std::vector<tcks_ctx*> ctxs;  // retained
  cudaStream_t origin = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  u64 launches = 0;
  std::vector<std::pair<tcks_ctx*, char*>> blocks;  // capture arenas of contexts with a caller allocator
};

#define BATCH_BEGIN \
  try {                 \
    tcks::NvtxRange tcks_nvtx_range_(__func__); \
    tcks::drop_stale_cuda_error();
#define BATCH_END                                                    \
  }                                                                  \
  catch (const tcks::Error& e) {                                     \
    return tcks::abi_record(e.code, e.msg);                          \
  }                                                                  \
  catch (const std::bad_alloc&) {                                    \
    return tcks::abi_record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed"); \
  }                                                                  \
  tcks::abi_clear();                                                 \
  return TCKS_OK;

extern "C" {

namespace {
std::vector<tcks_ctx*> contexts_of(const tcks_batch_job* jobs, u32 n_jobs) {
  std::vector<tcks_ctx*> v;
  for (u32 i = 0; i < n_jobs; ++i)
    if (std::find(v.begin(), v.end(), jobs[i].ctx) == v.end()) v.push_back(jobs[i].ctx);
  return v;
}
}  // namespace

tcks_status tcks_batch_run(const tcks_batch_job* jobs, uint32_t n_jobs) {
  BATCH_BEGIN
  validate(jobs, n_jobs);
  run_jobs(jobs, n_jobs);
  if (kDebugChecks) debug_word_check(contexts_of(jobs, n_jobs), "batch run");
  BATCH_END
}

void tcks_batch_free(tcks_batch* b) {
  if (!b) return;
  if (b->done) {
    cudaEventSynchronize(b->done);
    cudaEventDestroy(b->done);
  }
  for (tcks_ctx* c : b->ctxs) ctx_release(c);
  delete b;
  cudaGetLastError();  // clean-up statuses are not reported
}

tcks_status tcks_batch_submit(const tcks_batch_job* jobs, uint32_t n_jobs, tcks_batch** out) {
  struct Guard {
    tcks_batch* b = nullptr;
    ~Guard() { tcks_batch_free(b); }
  } guard;
  BATCH_BEGIN
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  validate(jobs, n_jobs);
  guard.b = new tcks_batch();
  for (u32 i = 0; i < n_jobs; ++i) {
    tcks_ctx* c = jobs[i].ctx;
    if (std::find(guard.b->ctxs.begin(), guard.b->ctxs.end(), c) == guard.b->ctxs.end()) {
      ctx_retain(c);
      guard.b->ctxs.push_back(c);
    }
  }
  check_cuda(cudaEventCreateWithFlags(&guard.b->done, cudaEventDisableTiming), "batch event");
  run_jobs(jobs, n_jobs);
  check_cuda(cudaEventRecord(guard.b->done, jobs[0].ctx->stream), "batch event");
  *out = guard.b;
  guard.b = nullptr;
  BATCH_END
}

tcks_status tcks_batch_wait(tcks_batch* b, int64_t timeout_ns) {
  BATCH_BEGIN
  if (!b || !b->done) fail(TCKS_ERR_INVALID_ARG, "null batch");
  // A host-side wait: the event is polled, with sleeps that grow to 100 us, until it completes or the
  // deadline passes. Nothing on the device waits.
  const auto start = std::chrono::steady_clock::now();
  auto pause = std::chrono::microseconds(2);
  for (;;) {
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) fail(TCKS_ERR_CUDA, std::string("batch: ") + cudaGetErrorString(e));
    if (timeout_ns >= 0 && std::chrono::steady_clock::now() - start >= std::chrono::nanoseconds(timeout_ns))
      fail(TCKS_ERR_TIMEOUT, "the batch has not completed within " + std::to_string(timeout_ns) + " ns");
    std::this_thread::sleep_for(pause);
    if (pause < std::chrono::microseconds(100)) pause *= 2;
  }
  if (kDebugChecks) debug_word_check(b->ctxs, "batch wait");
  BATCH_END
}

void tcks_batch_graph_free(tcks_batch_graph* g) {
  if (!g) return;
  if (g->origin) cudaStreamSynchronize(g->origin);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (const auto& b : g->blocks) arena_release(b.first, b.second);
  for (tcks_ctx* c : g->ctxs) ctx_release(c);
  delete g;
  cudaGetLastError();  // clean-up statuses are not reported
}

tcks_status tcks_batch_graph_create(const tcks_batch_job* jobs, uint32_t n_jobs, tcks_batch_graph** out) {
  struct Guard {
    tcks_batch_graph* g = nullptr;
    ~Guard() { tcks_batch_graph_free(g); }
  } guard;
  BATCH_BEGIN
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  validate(jobs, n_jobs);
  guard.g = new tcks_batch_graph();
  tcks_batch_graph* g = guard.g;
  for (u32 i = 0; i < n_jobs; ++i) {
    tcks_ctx* c = jobs[i].ctx;
    if (std::find(g->ctxs.begin(), g->ctxs.end(), c) == g->ctxs.end()) {
      ctx_retain(c);
      g->ctxs.push_back(c);
    }
  }
  g->origin = jobs[0].ctx->stream;
  // one eager pass builds every cached key table (their host copies cannot run inside a capture)
  run_jobs(jobs, n_jobs);
  for (tcks_ctx* c : g->ctxs) check_cuda(cudaStreamSynchronize(c->stream), "graph warm-up");
  // contexts with a caller allocator: a second uncaptured pass measures the scratch the capture takes
  struct ArenaGuard {
    const std::vector<tcks_ctx*>& ctxs;
    ~ArenaGuard() { arena_off(ctxs); }
  } arena_guard{g->ctxs};
  bool any_caller_alloc = false;
  for (tcks_ctx* c : g->ctxs) any_caller_alloc |= c->has_alloc;
  if (any_caller_alloc) {
    arena_record(g->ctxs);
    run_jobs(jobs, n_jobs);
    for (tcks_ctx* c : g->ctxs) check_cuda(cudaStreamSynchronize(c->stream), "graph scratch pass");
    arena_serve(g->ctxs, g->blocks);
  }
  const u64 n0 = tcks_launch_count();
  check_cuda(cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeThreadLocal), "begin capture");
  try {
    run_jobs(jobs, n_jobs);
  } catch (...) {
    cudaGraph_t dead = nullptr;
    cudaStreamEndCapture(g->origin, &dead);
    if (dead) cudaGraphDestroy(dead);
    throw;
  }
  check_cuda(cudaStreamEndCapture(g->origin, &g->graph), "end capture");
  arena_off(g->ctxs);
  g->launches = tcks_launch_count() - n0;
  check_cuda(cudaGraphInstantiate(&g->exec, g->graph, 0), "graph instantiate");
  *out = g;
  guard.g = nullptr;
  BATCH_END
}

tcks_status tcks_batch_graph_run(tcks_batch_graph* g) {
  BATCH_BEGIN
  if (!g) fail(TCKS_ERR_INVALID_ARG, "null graph");
  check_cuda(cudaGraphLaunch(g->exec, g->origin), "graph launch");
  count_launches(g->launches);
  if (kDebugChecks) debug_word_check(g->ctxs, "graph replay");
  BATCH_END
}

int32_t tcks_debug_checks(void) { return kDebugChecks ? 1 : 0; }

tcks_status tcks_debug_selftest(tcks_ctx* c, uint64_t* d_buf, uint32_t polys, uint32_t level, uint32_t understate,
                                uint32_t* word) {
  BATCH_BEGIN
  if (!c || !d_buf || !word) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *word = 0;
  if (!kDebugChecks) fail(TCKS_ERR_UNSUPPORTED, "the device range checks are compiled into debug builds only");
  if (c->params.log_n < 13 || c->params.log_n > 16) fail(TCKS_ERR_UNSUPPORTED, "the self-test takes N in [2^13, 2^16]");
  if (!polys || level < 1 || level > c->L + c->K) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  if (understate > (u64)polys * level) fail(TCKS_ERR_INVALID_ARG, "understate exceeds the limbs");
  const MultiNttBatch b{&c->T, d_buf, d_buf, polys, level};
  if (!launch_ntt_multi(false, &b, 1, c->stream, understate)) fail(TCKS_ERR_UNSUPPORTED, "the launch does not fit");
  check_launch("debug self-test");
  check_cuda(cudaStreamSynchronize(c->stream), "debug self-test");
  u32 w = 0;
  check_cuda(cudaMemcpy(&w, c->T.dbg, sizeof(u32), cudaMemcpyDeviceToHost), "debug word");
  check_cuda(cudaMemset(c->T.dbg, 0, sizeof(u32)), "debug word");
  *word = w;
  BATCH_END
}

tcks_status tcks_batch_graph_launches(const tcks_batch_graph* g, uint64_t* launches) {
  BATCH_BEGIN
  if (!g || !launches) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *launches = g->launches;
  BATCH_END
}

}  // extern "C"

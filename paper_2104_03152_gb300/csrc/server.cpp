// Serving loop for encrypted inference requests: continuous batching at stage granularity with
// admission by an HBM budget.
//
// A server holds lanes. A lane is a model on one context: the MNIST-shaped CNN (five stages, see
// cnn.cpp) or a vector x plain-matrix product (one stage). Requests are queued on submit and
// admitted in arrival order while the device budget (resident keys and model plaintexts of every
// lane, plus a per-request allowance for its live ciphertext and the stage scratch) and the in-flight
// cap allow. Lanes run asynchronously on their contexts' streams: a step first collects the lanes
// whose previous launch has completed (a CUDA event per lane), then, on every idle lane, groups its
// admitted requests by stage and runs each group's stage as one batched pass (up to max_batch
// requests per group). Under load each request advances one stage per lane launch (stage-level
// pipelining); at light load (no more waiting requests than max_batch) the launch carries them
// through all remaining stages. When no lane could start new work the step waits (bounded) for the
// first lane to finish. So a slow lane (a 4095-rotation vector x matrix
// batch) does not hold back a fast one (a CNN stage), and a request that arrives while others are
// running joins stage 0 at its lane's next launch. Results are bit-identical to the single-request
// path (every stage is exact modular arithmetic and no kernel depends on the batch composition).
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "context.h"

using namespace tcks;

namespace tcks {
void cnn_stage(const tcks_cnn* m, u32 stage, const u64* x, u32 count, u64* out);
u32 cnn_stage_level(const tcks_cnn* m, u32 stage);
u64 cnn_resident_bytes(const tcks_cnn* m);
tcks_ctx* cnn_context(const tcks_cnn* m);
double cnn_out_scale(const tcks_cnn* m, u32 stage, double in_scale);
}  // namespace tcks

namespace {

struct Lane {
  bool is_cnn;
  const tcks_cnn* cnn;
  const tcks_matrix* M;
  tcks_ctx* ctx;
  u32 stages;
  u64 req_bytes;  // allowance per in-flight request
  cudaEvent_t ev;  // recorded after the lane's last launch
  bool busy;       // a launch is in flight
};

struct Req {
  u64 id;
  u32 lane;
  u32 stage;
  tcks_ct* ct;  // current state, owned
  u64 cost;
  bool running;  // part of its lane's launch in flight
};

}  // namespace

struct tcks_server {
  u64 budget;
  u32 max_in_flight, max_batch;
  std::vector<Lane> lanes;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::map<u64, Req*> done;
  std::vector<u64> completed_ids;  // since the last poll
  u64 next_id = 1;
  u64 in_use = 0;
  u64 resident = 0;
  std::vector<tcks_ctx*> ctxs;  // distinct contexts, counted once in `resident`
};

#define SRV_BEGIN \
  try {                 \
    tcks::NvtxRange tcks_nvtx_range_(__func__); \
    tcks::drop_stale_cuda_error();
#define SRV_END                                                        \
  }                                                                    \
  catch (const tcks::Error& e) {                                       \
    return tcks::abi_record(e.code, e.msg);                            \
  }                                                                    \
  catch (const std::bad_alloc&) {                                      \
    return tcks::abi_record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed"); \
  }                                                                    \
  tcks::abi_clear();                                                   \
  return TCKS_OK;

static void add_context(tcks_server* s, tcks_ctx* c) {
  if (std::find(s->ctxs.begin(), s->ctxs.end(), c) != s->ctxs.end()) return;
  s->ctxs.push_back(c);
  s->resident += c->key_bytes() + c->table_bytes;
}

extern "C" {

tcks_status tcks_server_create(uint64_t hbm_budget_bytes, uint32_t max_in_flight, uint32_t max_batch,
                               tcks_server** out) {
  SRV_BEGIN
  if (!out || !max_in_flight || !max_batch) fail(TCKS_ERR_INVALID_ARG, "null output or zero caps");
  *out = new tcks_server();
  (*out)->budget = hbm_budget_bytes;
  (*out)->max_in_flight = max_in_flight;
  (*out)->max_batch = max_batch;
  SRV_END
}

void tcks_server_free(tcks_server* s) {
  if (!s) return;
  for (tcks_ctx* c : s->ctxs) cudaStreamSynchronize(c->stream);
  for (Lane& L : s->lanes)
    if (L.ev) cudaEventDestroy(L.ev);
  for (Req* r : s->queue) {
    free_ct(r->ct);
    delete r;
  }
  for (Req* r : s->active) {
    free_ct(r->ct);
    delete r;
  }
  for (auto& kv : s->done) {
    free_ct(kv.second->ct);
    delete kv.second;
  }
  delete s;
  cudaGetLastError();  // clean-up statuses are not reported
}

tcks_status tcks_server_add_cnn(tcks_server* s, const tcks_cnn* m, uint32_t* lane) {
  SRV_BEGIN
  if (!s || !m || !lane) fail(TCKS_ERR_INVALID_ARG, "null argument");
  tcks_ctx* c = cnn_context(m);
  add_context(s, c);
  s->resident += cnn_resident_bytes(m);
  // live ciphertext plus a conservative share of the stage scratch (ModUp digits, rotated
  // partials, tensor products): 64 top-level ciphertexts
  const u64 req = (u64)65 * ct_words(c, cnn_stage_level(m, 0)) * 8;
  s->lanes.push_back(Lane{true, m, nullptr, c, 5, req, nullptr, false});
  *lane = (u32)s->lanes.size() - 1;
  SRV_END
}

tcks_status tcks_server_add_vecmat(tcks_server* s, const tcks_matrix* M, uint32_t* lane) {
  SRV_BEGIN
  if (!s || !M || !lane) fail(TCKS_ERR_INVALID_ARG, "null argument");
  tcks_ctx* c = M->ctx;
  add_context(s, c);
  s->resident += (u64)M->diags * M->limbs() * c->N * 8;
  const u64 req = (u64)65 * ct_words(c, M->level) * 8;
  s->lanes.push_back(Lane{false, nullptr, M, c, 1, req, nullptr, false});
  *lane = (u32)s->lanes.size() - 1;
  SRV_END
}

tcks_status tcks_server_submit(tcks_server* s, uint32_t lane, const tcks_ct* in, uint64_t* id) {
  SRV_BEGIN
  if (!s || !in || !id) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (lane >= s->lanes.size()) fail(TCKS_ERR_INVALID_ARG, "no such lane");
  const Lane& L = s->lanes[lane];
  if (in->ctx != L.ctx) fail(TCKS_ERR_INVALID_ARG, "ciphertext belongs to another context");
  need_relinearized(in);
  const u32 want = L.is_cnn ? cnn_stage_level(L.cnn, 0) : L.M->level;
  if (in->level != want) fail(TCKS_ERR_LEVEL_MISMATCH, "request ciphertext at the wrong level for this lane");
  if (s->resident + L.req_bytes > s->budget)
    fail(TCKS_ERR_BUDGET_EXCEEDED, "the request can never fit: resident " + std::to_string(s->resident) +
                                        " B + per-request " + std::to_string(L.req_bytes) + " B > budget " +
                                        std::to_string(s->budget) + " B");
  tcks_ct* copy = new_ct(L.ctx, in->level, in->scale);
  check_cuda(cudaMemcpyAsync(copy->d, in->d, ct_words(L.ctx, in->level) * 8, cudaMemcpyDeviceToDevice,
                             L.ctx->stream),
             "submit");
  Req* r = new Req{s->next_id++, lane, 0, copy, L.req_bytes, false};
  s->queue.push_back(r);
  *id = r->id;
  SRV_END
}

// Collect the lanes whose launch has completed; their requests that passed the last stage finish.
static u32 harvest(tcks_server* s) {
  u32 fin = 0;
  for (Lane& L : s->lanes) {
    if (!L.busy) continue;
    const cudaError_t q = cudaEventQuery(L.ev);
    if (q == cudaErrorNotReady) continue;
    check_cuda(q, "server lane");
    L.busy = false;
  }
  for (auto it = s->active.begin(); it != s->active.end();) {
    Req* r = *it;
    const Lane& L = s->lanes[r->lane];
    if (r->running && !L.busy) r->running = false;
    if (!r->running && r->stage == L.stages) {
      s->in_use -= r->cost;
      s->done[r->id] = r;
      s->completed_ids.push_back(r->id);
      it = s->active.erase(it);
      ++fin;
    } else {
      ++it;
    }
  }
  return fin;
}

// Run one stage for a group of requests of a lane (gather, batched stage, scatter); each request
// advances one stage.
static void run_group(tcks_server* s, Lane& L, u32 stage, std::vector<Req*>& g) {
  tcks_ctx* c = L.ctx;
  const u32 count = (u32)g.size();
  const std::string range = "lane " + std::to_string(&L - s->lanes.data()) + " stage " + std::to_string(stage) +
                            " requests " + std::to_string(g.front()->id) + ".." + std::to_string(g.back()->id) +
                            " (" + std::to_string(count) + ")";
  NvtxRange nvtx(range.c_str());
  const u32 lin = g[0]->ct->level;
  const u32 lout = L.is_cnn ? cnn_stage_level(L.cnn, stage + 1) : lin - 1;
  const u64 win = ct_words(c, lin), wout = ct_words(c, lout);
  DevBuf x(c, (size_t)count * win), y(c, (size_t)count * wout);
  for (u32 i = 0; i < count; ++i)
    check_cuda(cudaMemcpyAsync(x.p + i * win, g[i]->ct->d, win * 8, cudaMemcpyDeviceToDevice, c->stream), "gather");
  double sc;
  if (L.is_cnn) {
    cnn_stage(L.cnn, stage, x.p, count, y.p);
    sc = cnn_out_scale(L.cnn, stage, g[0]->ct->scale);
  } else {
    op_vecmat(c, x.p, win, count, lin, L.M, y.p);
    sc = g[0]->ct->scale * L.M->scale / (double)c->host.chain[lin - 1];
  }
  for (u32 i = 0; i < count; ++i) {
    tcks_ct* nx = new_ct(c, lout, sc);
    check_cuda(cudaMemcpyAsync(nx->d, y.p + i * wout, wout * 8, cudaMemcpyDeviceToDevice, c->stream), "scatter");
    free_ct(g[i]->ct);  // stream-ordered: released after the gather above has read it
    g[i]->ct = nx;
    g[i]->stage += 1;
    g[i]->running = true;
  }
  (void)s;
}

// Launch an idle lane's work; returns whether anything was launched. Under load (more waiting
// requests than max_batch) every stage runs once for up to max_batch requests at that stage, so the
// stages of different requests overlap (a pipeline); at light load the waiting requests are carried
// through all their remaining stages in this launch, merging into one group as they reach the same
// stage, so that a request does not wait one lane cycle per stage.
static bool launch_lane(tcks_server* s, u32 lane) {
  Lane& L = s->lanes[lane];
  std::vector<Req*> ready;
  for (Req* r : s->active)
    if (r->lane == lane && !r->running && r->stage < L.stages) ready.push_back(r);
  if (ready.empty()) return false;
  if (ready.size() <= s->max_batch) {
    u32 first = L.stages;
    for (Req* r : ready) first = std::min(first, r->stage);
    for (u32 stage = first; stage < L.stages; ++stage) {
      std::vector<Req*> g;
      for (Req* r : ready)
        if (r->stage == stage) g.push_back(r);  // includes requests advanced from earlier stages here
      if (!g.empty()) run_group(s, L, stage, g);
    }
  } else {
    std::map<u32, std::vector<Req*>> groups;  // by stage, oldest first
    for (Req* r : ready) {
      auto& g = groups[r->stage];
      if (g.size() < s->max_batch) g.push_back(r);
    }
    for (auto& kv : groups) run_group(s, L, kv.first, kv.second);
  }
  if (!L.ev) check_cuda(cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming), "lane event");
  check_cuda(cudaEventRecord(L.ev, L.ctx->stream), "lane event");
  L.busy = true;
  return true;
}

// One scheduling step; *completed = requests finished in this step.
tcks_status tcks_server_step(tcks_server* s, uint32_t* completed) {
  SRV_BEGIN
  if (!s) fail(TCKS_ERR_INVALID_ARG, "null server");
  u32 fin = harvest(s);
  // admission in arrival order
  while (!s->queue.empty() && s->active.size() < s->max_in_flight) {
    Req* r = s->queue.front();
    if (s->resident + s->in_use + r->cost > s->budget) break;
    s->queue.pop_front();
    s->in_use += r->cost;
    s->active.push_back(r);
  }
  bool launched = false;
  for (u32 l = 0; l < s->lanes.size(); ++l)
    if (!s->lanes[l].busy) launched |= launch_lane(s, l);
  if (!launched) {
    // nothing new could start: wait (bounded) until some lane finishes
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      bool any_busy = false, any_done = false;
      for (Lane& L : s->lanes) {
        if (!L.busy) continue;
        any_busy = true;
        const cudaError_t q = cudaEventQuery(L.ev);
        if (q != cudaErrorNotReady) any_done = true;
      }
      if (!any_busy || any_done) break;
      if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(300))
        fail(TCKS_ERR_TIMEOUT, "no server lane finished within 300 s");
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    fin += harvest(s);
  }
  if (completed) *completed = fin;
  SRV_END
}

tcks_status tcks_server_poll(tcks_server* s, uint64_t* ids, uint32_t cap, uint32_t* n) {
  SRV_BEGIN
  if (!s || !n || (cap && !ids)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  const u32 k = (u32)std::min<size_t>(cap, s->completed_ids.size());
  for (u32 i = 0; i < k; ++i) ids[i] = s->completed_ids[i];
  s->completed_ids.erase(s->completed_ids.begin(), s->completed_ids.begin() + k);
  *n = k;
  SRV_END
}

tcks_status tcks_server_take(tcks_server* s, uint64_t id, tcks_ct** out) {
  SRV_BEGIN
  if (!s || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  auto it = s->done.find(id);
  if (it == s->done.end()) fail(TCKS_ERR_NOT_READY, "request " + std::to_string(id) + " has not completed");
  *out = it->second->ct;
  delete it->second;
  s->done.erase(it);
  SRV_END
}

tcks_status tcks_server_stats(const tcks_server* s, uint64_t* queued, uint64_t* in_flight, uint64_t* finished,
                              uint64_t* bytes_in_use, uint64_t* bytes_resident) {
  SRV_BEGIN
  if (!s) fail(TCKS_ERR_INVALID_ARG, "null server");
  if (queued) *queued = s->queue.size();
  if (in_flight) *in_flight = s->active.size();
  if (finished) *finished = s->done.size();
  if (bytes_in_use) *bytes_in_use = s->in_use;
  if (bytes_resident) *bytes_resident = s->resident;
  SRV_END
}

}  // extern "C"

// C ABI of the library (include/tcks.h): handle management, argument checks, and the composition of
// kernels into the CKKSVector operations of TenSEAL (§2-§3).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "context.h"

using namespace tcks;

namespace {

thread_local std::string g_last_error;

tcks_status record(tcks_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

static void ctx_destroy(tcks_ctx* c);

#define TCKS_API_BEGIN \
  try {                 \
    tcks::NvtxRange tcks_nvtx_range_(__func__); \
    tcks::drop_stale_cuda_error();
#define TCKS_API_END                                                   \
  }                                                                    \
  catch (const tcks::Error& e) {                                       \
    return record(e.code, e.msg);                                      \
  }                                                                    \
  catch (const std::bad_alloc&) {                                      \
    return record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed");   \
  }                                                                    \
  catch (const std::exception& e) {                                    \
    return record(TCKS_ERR_INVALID_ARG, e.what());                     \
  }                                                                    \
  g_last_error.clear();                                                \
  return TCKS_OK;

namespace tcks {

[[noreturn]] void fail(tcks_status code, const std::string& msg) { throw Error{code, msg}; }

tcks_status abi_record(tcks_status code, const std::string& msg) { return record(code, msg); }
void abi_clear() { g_last_error.clear(); }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(TCKS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void check_launch(const char* what) { check_cuda(cudaGetLastError(), what); }
void drop_stale_cuda_error() { cudaGetLastError(); }

tcks_ct* new_ct(tcks_ctx* c, u32 level, double scale) {
  DevBuf b(c, ct_words(c, level));
  tcks_ct* ct = new tcks_ct{c, b.release(), level, scale};
  ctx_retain(c);
  return ct;
}

tcks_ct* new_ct_sized(tcks_ctx* c, u32 size, u32 level, double scale) {
  DevBuf b(c, (size_t)size * level * c->N);
  tcks_ct* ct = new tcks_ct{c, b.release(), level, scale, size};
  ctx_retain(c);
  return ct;
}

u64 ksk_words(const tcks_ctx* c, u32 Kt) {
  if (!c->hyb) return (u64)Kt * 2 * (Kt + 1) * c->N;
  return (u64)((Kt + c->alpha - 1) / c->alpha) * 2 * (Kt + c->K) * c->N;
}

u64 ks_digit_words(const tcks_ctx* c, u32 ell) {
  if (!c->hyb) return (u64)ell * (ell + 1) * c->N;
  return (u64)((ell + c->alpha - 1) / c->alpha) * (ell + c->K) * c->N;
}

u64 ks_top_words(const tcks_ctx* c) { return (u64)2 * c->K * c->N; }

void ks_modup(tcks_ctx* c, const u64* x, u64 x_stride, u32 count, u32 ell, u64* coef_tmp, u64* digits) {
  if (c->hyb)
    launch_modup_hyb(c->T, c->H, x, x_stride, count, ell, coef_tmp, digits, c->stream);
  else
    launch_modup(c->T, x, x_stride, count, ell, coef_tmp, digits, c->stream);
}

void ks_switch(tcks_ctx* c, u32 ell, const KsPlan& plan) {
  if (c->hyb)
    launch_keyswitch_hyb(c->T, c->H, ell, plan, c->stream);
  else
    launch_keyswitch(c->T, ell, plan, c->stream);
}

void need_one_prime_ks(const tcks_ctx* c, const char* what) {
  if (c && c->hyb)
    fail(TCKS_ERR_UNSUPPORTED, std::string(what) + " is written for the one-prime key switch (alpha = 1, one special "
                               "prime); this context uses hybrid key switching");
}

void need_relinearized(const tcks_ct* ct) {
  if (ct && ct->size != 2)
    fail(TCKS_ERR_INVALID_ARG, "a three-component ciphertext must be relinearized first (tcks_relinearize)");
}

tcks_pt* new_pt(tcks_ctx* c, u32 level, double scale) {
  DevBuf b(c, pt_words(c, level));
  tcks_pt* pt = new tcks_pt{c, b.release(), level, scale};
  ctx_retain(c);
  return pt;
}

void free_ct(tcks_ct* ct) {
  if (!ct) return;
  tcks_ctx* c = ct->ctx;
  if (ct->d) c->dev_free(ct->d);
  delete ct;
  ctx_release(c);
}

void ctx_retain(tcks_ctx* c) { c->refs.fetch_add(1); }

void ctx_release(tcks_ctx* c) {
  if (c->refs.fetch_sub(1) == 1) ::ctx_destroy(c);
}

u32 step_mod(const tcks_ctx* c, int64_t step) {
  const int64_t half = (int64_t)c->N / 2;
  int64_t k = step % half;
  if (k < 0) k += half;
  return (u32)k;
}

const GaloisKey& galois_key_for(tcks_ctx* c, int64_t step, u32 ell) {
  const u32 k = step_mod(c, step);
  auto it = c->galois.find(k);
  if (it == c->galois.end()) fail(TCKS_ERR_NO_GALOIS_KEY, "no Galois key for rotation step " + std::to_string(k));
  if (it->second.K < ell)
    fail(TCKS_ERR_LEVEL_EXHAUSTED, "Galois key for step " + std::to_string(k) + " is trimmed to level " +
                                       std::to_string(it->second.K) + " < " + std::to_string(ell));
  return it->second;
}

void op_rescale_polys(tcks_ctx* c, const u64* in, u32 ell, u32 polys, u64* out) {
  if (ell < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "rescale needs level >= 2");
  DevBuf top(c, (size_t)polys * c->N);
  launch_rescale(c->T, in, ell, polys, top.p, out, c->stream);
  check_launch("rescale");
}

void op_rescale(tcks_ctx* c, const u64* in, u32 ell, u64* out, u32 count) {
  if (ell < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "rescale needs level >= 2");
  DevBuf top(c, (size_t)2 * count * c->N);
  launch_rescale(c->T, in, ell, 2 * count, top.p, out, c->stream);
  check_launch("rescale");
}

const KeyTable& key_table(tcks_ctx* c, const std::vector<u32>& steps, u32 ell) {
  auto it = c->key_tables.find(steps);
  if (it == c->key_tables.end()) {
    std::vector<KsKey> h(steps.size());
    u32 min_K = ~0u;
    for (size_t i = 0; i < steps.size(); ++i) {
      if (steps[i] == 0) {
        h[i] = KsKey{c->rlk, c->L, 1u};
      } else {
        const GaloisKey& gk = galois_key_for(c, steps[i], 1);
        h[i] = KsKey{gk.d, gk.K, (u32)galois_element(c->params.log_n, steps[i]), nullptr};
        if (c->T.narrow) {  // the double-hoisted accumulation reads the key's 32-bit copy
          auto nk = c->narrow_keys.find(gk.d);
          if (nk == c->narrow_keys.end()) {
            const u64 words = ksk_words(c, gk.K);
            u32* d32 = (u32*)c->dev_alloc(words * 4);
            launch_narrow_copy(gk.d, d32, words, c->stream);
            check_launch("32-bit key copy");
            nk = c->narrow_keys.emplace(gk.d, std::make_pair(d32, words)).first;
          }
          h[i].key32 = nk->second.first;
        }
      }
      min_K = h[i].K < min_K ? h[i].K : min_K;
    }
    KeyTable t;
    t.n = (u32)h.size();
    t.min_K = min_K;
    for (const KsKey& k : h) t.max_K = k.K > t.max_K ? k.K : t.max_K;
    t.keys32 = true;
    for (const KsKey& k : h) t.keys32 = t.keys32 && k.key32 != nullptr;
    t.aligned16 = true;
    for (const KsKey& k : h) t.aligned16 = t.aligned16 && ((uintptr_t)k.key & 15) == 0;
    t.d = (KsKey*)c->dev_alloc(sizeof(KsKey) * h.size());
    check_cuda(cudaMemcpyAsync(t.d, h.data(), sizeof(KsKey) * h.size(), cudaMemcpyHostToDevice, c->stream),
               "key table");
    check_cuda(cudaStreamSynchronize(c->stream), "key table");
    it = c->key_tables.emplace(steps, t).first;
  }
  if (it->second.min_K < ell) {
    for (u32 st : steps) galois_key_for(c, st, ell);  // raises with the step that is too short
  }
  return it->second;
}

void op_relinearize(tcks_ctx* c, const u64* d3, u32 ell, u64* out, u32 count) {
  const size_t n = c->N;
  const KeyTable& kt = key_table(c, {0u}, ell);
  const u64 dw = ks_digit_words(c, ell);
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * dw), top(c, (size_t)count * ks_top_words(c));
  const u64 d3_stride = (u64)3 * ell * n;
  ks_modup(c, d3 + (size_t)2 * ell * n, d3_stride, count, ell, coef.p, digits.p);
  KsPlan p{};
  p.keys = kt.d;
  p.digits = digits.p;
  p.digits_b = dw;
  p.top = top.p;
  p.out = out;
  p.out_b = (u64)2 * ell * n;
  p.out_r = 0;
  p.add0 = d3;
  p.add0_b = d3_stride;
  p.add1 = d3 + (size_t)ell * n;
  p.add1_b = d3_stride;
  p.R = 1;
  p.B = count;
  p.add_perm = 0;
  ks_switch(c, ell, p);
  check_launch("relinearize");
}

void op_relin_rescale(tcks_ctx* c, const u64* d3, u32 ell, u64* out, u32 count) {
  if (ell < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "rescale needs level >= 2");
  const size_t n = c->N;
  if (c->hyb) {  // the merged rounding is written for one special prime: relinearize, then rescale
    DevBuf rel(c, (size_t)count * ct_words(c, ell));
    op_relinearize(c, d3, ell, rel.p, count);
    op_rescale(c, rel.p, ell, out, count);
    return;
  }
  const KeyTable& kt = key_table(c, {0u}, ell);
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * ell * (ell + 1) * n);
  DevBuf top(c, (size_t)count * 2 * n), top2(c, (size_t)count * 2 * n);
  const u64 d3_stride = (u64)3 * ell * n;
  launch_modup(c->T, d3 + (size_t)2 * ell * n, d3_stride, count, ell, coef.p, digits.p, c->stream);
  KsPlan p{};
  p.keys = kt.d;
  p.digits = digits.p;
  p.digits_b = (u64)ell * (ell + 1) * n;
  p.top = top.p;
  p.out = out;
  p.out_b = (u64)2 * (ell - 1) * n;
  p.add0 = d3;
  p.add0_b = d3_stride;
  p.add1 = d3 + (size_t)ell * n;
  p.add1_b = d3_stride;
  p.R = 1;
  p.B = count;
  launch_relin_rescale(c->T, c->host, ell, p, top2.p, c->stream);
  check_launch("relinearize + rescale");
}

void op_rotate_add(tcks_ctx* c, u64* base, u64 stride, u32 count, u32 ell, int32_t step) {
  const size_t n = c->N;
  const u32 k = step_mod(c, step);
  if (k == 0) {  // rot by 0 is the identity: ct <- 2 ct
    for (u32 i = 0; i < count; ++i)
      launch_elementwise(c->T, OP_ADD, base + i * stride, base + i * stride, base + i * stride, ell, 2, c->stream);
    return;
  }
  const KeyTable& kt = key_table(c, {k}, ell);
  const u64 dw = ks_digit_words(c, ell);
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * dw);
  DevBuf tmp(c, (size_t)count * ct_words(c, ell)), top(c, (size_t)count * ks_top_words(c));
  ks_modup(c, base + (size_t)ell * n, stride, count, ell, coef.p, digits.p);
  KsPlan p{};
  p.keys = kt.d;
  p.digits = digits.p;
  p.digits_b = dw;
  p.top = top.p;
  p.out = tmp.p;
  p.out_b = ct_words(c, ell);
  p.add0 = base;
  p.add0_b = stride;
  p.R = 1;
  p.B = count;
  p.add_perm = 1;
  ks_switch(c, ell, p);
  if (stride == ct_words(c, ell)) {
    launch_elementwise(c->T, OP_ADD, base, tmp.p, base, ell, 2 * count, c->stream);
  } else {
    for (u32 i = 0; i < count; ++i)
      launch_elementwise(c->T, OP_ADD, base + i * stride, tmp.p + i * ct_words(c, ell), base + i * stride, ell, 2,
                         c->stream);
  }
  check_launch("rotate-add");
}

void op_rotate_add_to(tcks_ctx* c, const u64* in, u64 in_stride, u32 count, u32 ell, int32_t step, u64* out,
                      u64 out_stride, const u64* bias) {
  need_one_prime_ks(c, "the fused rotate-and-add");
  const size_t n = c->N;
  const u64 w = ct_words(c, ell);
  if (count > 1 && (in_stride < w || out_stride < w)) fail(TCKS_ERR_INVALID_ARG, "rotate-add: overlapping batch entries");
  const u64 in_end = (count - 1) * in_stride + w, out_end = (count - 1) * out_stride + w;
  if (out < in + in_end && in < out + out_end) fail(TCKS_ERR_INVALID_ARG, "rotate-add: out overlaps in");
  const u32 k = step_mod(c, step);
  if (k == 0) {  // rot by 0 is the identity: out = 2 in (+ bias)
    for (u32 i = 0; i < count; ++i) {
      launch_elementwise(c->T, OP_ADD, in + i * in_stride, in + i * in_stride, out + i * out_stride, ell, 2, c->stream);
      if (bias) launch_elementwise(c->T, OP_ADD_PLAIN, out + i * out_stride, bias, out + i * out_stride, ell, 2, c->stream);
    }
    return;
  }
  const KeyTable& kt = key_table(c, {k}, ell);
  const u64 dw = ks_digit_words(c, ell);
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * dw);
  DevBuf top(c, (size_t)count * ks_top_words(c));
  ks_modup(c, in + (size_t)ell * n, in_stride, count, ell, coef.p, digits.p);
  KsPlan p{};
  p.keys = kt.d;
  p.digits = digits.p;
  p.digits_b = dw;
  p.top = top.p;
  p.out = out;
  p.out_b = out_stride;
  p.add0 = in;  // the automorphed c0 of in
  p.add0_b = in_stride;
  p.add_perm = 1;
  p.addx = in;  // in itself, both components
  p.addx_b = in_stride;
  p.addp = bias;
  p.R = 1;
  p.B = count;
  launch_keyswitch(c->T, ell, p, c->stream);
  check_launch("rotate-add");
}

void op_rotate_hoisted(tcks_ctx* c, const u64* ct, u32 ell, const int32_t* steps, u32 n_steps, u64* const* outs) {
  const size_t n = c->N;
  std::vector<u32> ks;
  std::vector<u32> where;  // output index of each non-trivial step
  for (u32 i = 0; i < n_steps; ++i) {
    const u32 k = step_mod(c, steps[i]);
    if (k == 0) {
      check_cuda(cudaMemcpyAsync(outs[i], ct, ct_words(c, ell) * 8, cudaMemcpyDeviceToDevice, c->stream),
                 "rotate by 0");
    } else {
      ks.push_back(k);
      where.push_back(i);
    }
  }
  if (ks.empty()) return;
  const KeyTable& kt = key_table(c, ks, ell);
  const u32 R = (u32)ks.size();
  DevBuf coef(c, (size_t)ell * n), digits(c, (size_t)ks_digit_words(c, ell));
  DevBuf tmp(c, (size_t)R * ct_words(c, ell)), top(c, (size_t)R * ks_top_words(c));
  ks_modup(c, ct + (size_t)ell * n, 0, 1, ell, coef.p, digits.p);
  KsPlan p{};
  p.keys = kt.d;
  p.digits = digits.p;
  p.top = top.p;
  p.out = tmp.p;
  p.out_r = ct_words(c, ell);
  p.add0 = ct;
  p.R = R;
  p.B = 1;
  p.add_perm = 1;
  ks_switch(c, ell, p);
  for (u32 r = 0; r < R; ++r)
    check_cuda(cudaMemcpyAsync(outs[where[r]], tmp.p + (size_t)r * ct_words(c, ell), ct_words(c, ell) * 8,
                               cudaMemcpyDeviceToDevice, c->stream),
               "rotate copy");
  check_launch("rotate");
}

void encode_into(tcks_ctx* c, const double* d_v, size_t n, double scale, u32 level, u64* pt_out, bool ext) {
  if (c->params.log_n > 14) fail(TCKS_ERR_UNSUPPORTED, "encoding is implemented for N <= 2^14");
  DevBuf coeffs(c, c->N);
  check_cuda(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "encode status");
  launch_encode_coeffs(c->T, c->F, d_v, (u32)n, scale, (i64*)coeffs.p, c->d_status, c->stream);
  launch_coeffs_to_ntt(c->T, (const i64*)coeffs.p, level, pt_out, c->stream, ext);
  check_launch("encode");
  int status = 0;
  check_cuda(cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "encode status");
  check_cuda(cudaStreamSynchronize(c->stream), "encode");
  if (status) fail(TCKS_ERR_VALUE_OVERFLOW, "encode: |scale * m_i| >= 2^62");
}

}  // namespace tcks

void* tcks_ctx::dev_alloc(size_t bytes) {
  if (bytes == 0) bytes = 8;
  void* p = nullptr;
  const size_t rounded = (bytes + 255) & ~(size_t)255;
  if (arena.mode == ARENA_SERVE) {
    if (arena.used + rounded > arena.size)
      fail(TCKS_ERR_OUT_OF_MEMORY, "the captured pass allocated more than the recorded pass (" +
                                       std::to_string(arena.used + rounded) + " > " + std::to_string(arena.size) + " bytes)");
    p = arena.base + arena.used;
    arena.used += rounded;
    return p;
  }
  if (arena.mode == ARENA_RECORD) arena.recorded += rounded;
  if (has_alloc) {
    p = alloc.alloc(bytes, (void*)stream, alloc.user);
    if (!p) fail(TCKS_ERR_OUT_OF_MEMORY, "allocator callback returned NULL for " + std::to_string(bytes) + " bytes");
    return p;
  }
  const cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(TCKS_ERR_OUT_OF_MEMORY, "device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  return p;
}

void tcks_ctx::dev_free(void* p) {
  if (!p) return;
  for (const auto& b : graph_blocks)
    if ((char*)p >= b.first && (char*)p < b.first + b.second) return;  // a graph's block: released with the graph
  if (arena.mode == ARENA_SERVE && (char*)p >= arena.base && (char*)p < arena.base + arena.size) return;
  if (has_alloc)
    alloc.free(p, (void*)stream, alloc.user);
  else if (cudaFreeAsync(p, stream) != cudaSuccess)
    cudaGetLastError();  // a release has no caller to report to; keep it out of the next launch check
}

namespace tcks {

void arena_record(const std::vector<tcks_ctx*>& ctxs) {
  for (tcks_ctx* c : ctxs)
    if (c->has_alloc) c->arena = tcks_ctx::CaptureArena{tcks_ctx::ARENA_RECORD, 0, nullptr, 0, 0};
}

void arena_serve(const std::vector<tcks_ctx*>& ctxs, std::vector<std::pair<tcks_ctx*, char*>>& held) {
  for (tcks_ctx* c : ctxs) {
    if (!c->has_alloc || c->arena.mode != tcks_ctx::ARENA_RECORD) continue;
    const size_t size = c->arena.recorded ? c->arena.recorded : 256;
    c->arena.mode = tcks_ctx::ARENA_OFF;
    char* base = (char*)c->dev_alloc(size);
    c->graph_blocks.push_back({base, size});
    held.push_back({c, base});
    c->arena = tcks_ctx::CaptureArena{tcks_ctx::ARENA_SERVE, 0, base, 0, size};
  }
}

void debug_word_check(const std::vector<tcks_ctx*>& ctxs, const char* where) {
  for (tcks_ctx* c : ctxs) {
    u32 w = 0;
    check_cuda(cudaMemcpyAsync(&w, c->T.dbg, sizeof(u32), cudaMemcpyDeviceToHost, c->stream), "debug word");
    check_cuda(cudaStreamSynchronize(c->stream), where);
    if (!w) continue;
    check_cuda(cudaMemsetAsync(c->T.dbg, 0, sizeof(u32), c->stream), "debug word");
    char bits[16];
    std::snprintf(bits, sizeof bits, "0x%x", w);
    fail(TCKS_ERR_DEBUG_CHECK, std::string(where) + ": a device range check failed (error bits " + bits +
                                   ": 1 context index, 2 limb range, 4 prime index, 8 null pointer)");
  }
}

void kernel_error_check(tcks_ctx* c) {
  u32 w = 0;
  check_cuda(cudaMemcpyAsync(&w, c->T.kerr, sizeof(u32), cudaMemcpyDeviceToHost, c->stream), "kernel error word");
  check_cuda(cudaStreamSynchronize(c->stream), "kernel error word");
  if (!w) return;
  check_cuda(cudaMemsetAsync(c->T.kerr, 0, sizeof(u32), c->stream), "kernel error word");
  if (w & 1u) fail(TCKS_ERR_TIMEOUT, "a kernel's bounded wait for its staged operands ran out; its results are invalid");
  fail(TCKS_ERR_CUDA, "a kernel refused a bulk copy from a source off its 16-byte alignment; its results are invalid");
}

void arena_off(const std::vector<tcks_ctx*>& ctxs) {
  for (tcks_ctx* c : ctxs) c->arena = tcks_ctx::CaptureArena{};
}

void arena_release(tcks_ctx* c, char* block) {
  cudaStreamSynchronize(c->stream);
  for (size_t i = 0; i < c->graph_blocks.size(); ++i)
    if (c->graph_blocks[i].first == block) {
      c->graph_blocks.erase(c->graph_blocks.begin() + (long)i);
      c->dev_free(block);
      return;
    }
}

}  // namespace tcks

void tcks_ctx::keys_changed() {
  for (auto& kv : key_tables) dev_free(kv.second.d);
  key_tables.clear();
  for (auto& kv : narrow_keys) dev_free(kv.second.first);
  narrow_keys.clear();
}

tcks::u64 tcks_ctx::key_bytes() const {
  u64 b = 0;
  const u64 n = N;
  b += (u64)(L + K) * n * 8 + (u64)2 * L * n * 8 + ksk_words(this, L) * 8;
  // with 32-bit chains each Galois key may also hold its 32-bit copy (made with the key tables)
  for (const auto& kv : galois) b += ksk_words(this, kv.second.K) * (T.narrow ? 12 : 8);
  return b;
}

// =============================================================================================
extern "C" {

const char* tcks_status_string(tcks_status s) {
  switch (s) {
    case TCKS_OK: return "OK";
    case TCKS_ERR_INVALID_ARG: return "INVALID_ARG";
    case TCKS_ERR_BAD_PARAMS: return "BAD_PARAMS";
    case TCKS_ERR_NO_GALOIS_KEY: return "NO_GALOIS_KEY";
    case TCKS_ERR_LEVEL_EXHAUSTED: return "LEVEL_EXHAUSTED";
    case TCKS_ERR_SCALE_MISMATCH: return "SCALE_MISMATCH";
    case TCKS_ERR_LEVEL_MISMATCH: return "LEVEL_MISMATCH";
    case TCKS_ERR_OUT_OF_MEMORY: return "OUT_OF_MEMORY";
    case TCKS_ERR_BUDGET_EXCEEDED: return "BUDGET_EXCEEDED";
    case TCKS_ERR_CUDA: return "CUDA_ERROR";
    case TCKS_ERR_TIMEOUT: return "TIMEOUT";
    case TCKS_ERR_VALUE_OVERFLOW: return "VALUE_OVERFLOW";
    case TCKS_ERR_UNSUPPORTED: return "UNSUPPORTED";
    case TCKS_ERR_NOT_READY: return "NOT_READY";
    case TCKS_ERR_DEBUG_CHECK: return "DEBUG_CHECK";
    default: return "UNKNOWN";
  }
}

const char* tcks_last_error_detail(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------------------ parameters ---
tcks_status tcks_params_create(uint32_t log_n, const uint32_t* bit_sizes, uint32_t n_primes, double scale,
                               tcks_params** out) {
  TCKS_API_BEGIN
  if (!out || !bit_sizes) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (log_n < 3 || log_n > 16) fail(TCKS_ERR_BAD_PARAMS, "log_n must be in [3, 16]");
  if (n_primes < 2 || n_primes > 64) fail(TCKS_ERR_BAD_PARAMS, "need 2..64 primes (data primes + special primes)");
  if (!(scale > 0) || !std::isfinite(scale)) fail(TCKS_ERR_BAD_PARAMS, "scale must be positive");
  std::vector<u64> chain;
  if (!find_chain(log_n, bit_sizes, n_primes, chain))
    fail(TCKS_ERR_BAD_PARAMS, "no NTT-friendly prime for some bit size (sizes must be in [20, 61])");
  tcks_params* p = new tcks_params{log_n, std::vector<u32>(bit_sizes, bit_sizes + n_primes), chain, scale};
  *out = p;
  TCKS_API_END
}

tcks_status tcks_params_create_primes(uint32_t log_n, const uint64_t* primes, uint32_t n_primes, double scale,
                                      tcks_params** out) {
  TCKS_API_BEGIN
  if (!out || !primes) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (log_n < 3 || log_n > 16) fail(TCKS_ERR_BAD_PARAMS, "log_n must be in [3, 16]");
  if (n_primes < 2 || n_primes > 64) fail(TCKS_ERR_BAD_PARAMS, "need 2..64 primes (data primes + special primes)");
  if (!(scale > 0) || !std::isfinite(scale)) fail(TCKS_ERR_BAD_PARAMS, "scale must be positive");
  std::vector<u64> chain(primes, primes + n_primes);
  std::vector<u32> bits;
  const u64 two_n = 2ull << log_n;
  for (u32 i = 0; i < n_primes; ++i) {
    const u64 q = chain[i];
    if (q >= (1ull << 61) || !is_prime_u64(q) || q % two_n != 1)
      fail(TCKS_ERR_BAD_PARAMS, "prime " + std::to_string(i) + " is not a prime below 2^61 with q == 1 mod 2N");
    for (u32 j = 0; j < i; ++j)
      if (chain[j] == q) fail(TCKS_ERR_BAD_PARAMS, "prime " + std::to_string(i) + " repeats an earlier one");
    u32 b = 0;
    while (b < 64 && (q >> b)) ++b;
    bits.push_back(b);
  }
  *out = new tcks_params{log_n, bits, chain, scale};
  TCKS_API_END
}

tcks_status tcks_params_create_hybrid(uint32_t log_n, const uint64_t* primes, uint32_t n_primes, uint32_t n_special,
                                      uint32_t alpha, double scale, tcks_params** out) {
  TCKS_API_BEGIN
  if (!out || !primes) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (n_special < 1 || n_special > 8 || alpha < 1 || alpha > 8)
    fail(TCKS_ERR_BAD_PARAMS, "n_special and alpha must be in [1, 8]");
  if (n_primes <= n_special || n_primes - n_special > CRT_MAXW - 2)
    fail(TCKS_ERR_BAD_PARAMS, "need 1..32 data primes before the special primes");
  tcks_params* p = nullptr;
  const tcks_status st = tcks_params_create_primes(log_n, primes, n_primes - n_special + 1, scale, &p);
  if (st != TCKS_OK) return st;
  std::unique_ptr<tcks_params> guard(p);
  // the whole chain (the special primes too) must be NTT-friendly primes
  p->chain.assign(primes, primes + n_primes);
  p->bits.clear();
  const u64 two_n = 2ull << log_n;
  for (u32 i = 0; i < n_primes; ++i) {
    const u64 q = p->chain[i];
    if (q >= (1ull << 61) || !is_prime_u64(q) || q % two_n != 1)
      fail(TCKS_ERR_BAD_PARAMS, "prime " + std::to_string(i) + " is not a prime below 2^61 with q == 1 mod 2N");
    for (u32 j = 0; j < i; ++j)
      if (p->chain[j] == q) fail(TCKS_ERR_BAD_PARAMS, "prime " + std::to_string(i) + " repeats an earlier one");
    u32 b = 0;
    while (b < 64 && (q >> b)) ++b;
    p->bits.push_back(b);
  }
  // P must exceed the product of every digit's primes, or the key-switch error (D_j e_j / P) grows
  // with the ratio; compared on bit lengths
  const u32 L = n_primes - n_special;
  double logP = 0;
  for (u32 k = 0; k < n_special; ++k) logP += std::log2((double)p->chain[L + k]);
  for (u32 j = 0; j * alpha < L; ++j) {
    double logQ = 0;
    for (u32 i = j * alpha; i < std::min(L, (j + 1) * alpha); ++i) logQ += std::log2((double)p->chain[i]);
    if (logQ > logP) fail(TCKS_ERR_BAD_PARAMS, "the special primes' product is below digit " + std::to_string(j));
  }
  p->n_special = n_special;
  p->alpha = alpha;
  *out = guard.release();
  TCKS_API_END
}

void tcks_params_free(tcks_params* p) { delete p; }

tcks_status tcks_params_primes(const tcks_params* p, uint64_t* primes, uint32_t capacity) {
  TCKS_API_BEGIN
  if (!p || !primes) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (capacity < p->chain.size()) fail(TCKS_ERR_INVALID_ARG, "capacity too small");
  for (size_t i = 0; i < p->chain.size(); ++i) primes[i] = p->chain[i];
  TCKS_API_END
}

// --------------------------------------------------------------------------------- context ---
tcks_status tcks_context_create(const tcks_params* params, uint64_t seed, uint32_t flags,
                                const tcks_allocator* allocator, void* cuda_stream, tcks_ctx** out) {
  tcks_ctx* c = nullptr;
  TCKS_API_BEGIN
  if (!params || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  c = new tcks_ctx();
  c->params = *params;
  c->N = 1u << params->log_n;
  c->K = params->n_special;
  c->alpha = params->alpha;
  c->hyb = c->K > 1 || c->alpha > 1;
  c->L = (u32)params->chain.size() - c->K;
  if (c->L < 1 || c->L > CRT_MAXW - 2)
    fail(TCKS_ERR_BAD_PARAMS, "a context takes 1.." + std::to_string(CRT_MAXW - 2) + " data primes");
  c->flags = flags;
  c->seed = seed;
  check_cuda(cudaGetDevice(&c->device), "cudaGetDevice");
  if (allocator && allocator->alloc && allocator->free) {
    c->alloc = *allocator;
    c->has_alloc = true;
  }
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    check_cuda(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    c->own_stream = true;
  }
  if (!c->has_alloc) {
    // keep freed blocks in the device pool instead of returning them to the driver
    cudaMemPool_t pool;
    check_cuda(cudaDeviceGetDefaultMemPool(&pool, c->device), "default mem pool");
    u64 threshold = ~0ull;
    check_cuda(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold), "mem pool threshold");
  }
  if (!build_tables(params->log_n, params->chain, c->host)) fail(TCKS_ERR_BAD_PARAMS, "a prime has no 2N-th root");
  const u32 nm = c->L + c->K, n = c->N;
  const HostTables& H = c->host;
  c->d_mods = c->dev_alloc(sizeof(ModConst) * nm);
  c->d_pairs = c->dev_alloc(sizeof(PairConst) * nm * nm);
  c->d_tw = (u64*)c->dev_alloc(sizeof(u64) * H.tw.size());
  if (H.narrow) c->d_tw32 = (u32*)c->dev_alloc(sizeof(u32) * H.tw32.size());
  c->d_slot = (u32*)c->dev_alloc(sizeof(u32) * H.slot_index.size());
  c->d_zeta = (double*)c->dev_alloc(sizeof(double) * H.zeta.size());
  c->d_status = (int*)c->dev_alloc(sizeof(int) * 4);  // [0] kernel status words, [2] debug error word
  check_cuda(cudaMemsetAsync(c->d_status, 0, sizeof(int) * 4, c->stream), "status words");
  // CRT words per level: Q_l and (Q_l - 1)/2
  std::vector<u64> qw((size_t)2 * c->L * CRT_MAXW, 0);
  for (u32 l = 1; l <= c->L; ++l) {
    std::vector<u64> Q(CRT_MAXW, 0);
    Q[0] = 1;
    for (u32 i = 0; i < l; ++i) {
      unsigned __int128 carry = 0;
      for (u32 w = 0; w < CRT_MAXW; ++w) {
        const unsigned __int128 t = (unsigned __int128)Q[w] * H.chain[i] + carry;
        Q[w] = (u64)t;
        carry = t >> 64;
      }
    }
    for (u32 w = 0; w < CRT_MAXW; ++w) {
      qw[(size_t)(l - 1) * CRT_MAXW + w] = Q[w];
      const u64 hi = (w + 1 < CRT_MAXW) ? Q[w + 1] : 0;
      qw[((size_t)c->L + l - 1) * CRT_MAXW + w] = (Q[w] >> 1) | (hi << 63);  // Q odd: (Q-1)/2 = Q >> 1
    }
  }
  c->d_qwords = (u64*)c->dev_alloc(sizeof(u64) * qw.size());
  cudaStream_t s = c->stream;
  check_cuda(cudaMemcpyAsync(c->d_mods, H.mods.data(), sizeof(ModConst) * nm, cudaMemcpyHostToDevice, s), "H2D");
  check_cuda(cudaMemcpyAsync(c->d_pairs, H.pairs.data(), sizeof(PairConst) * nm * nm, cudaMemcpyHostToDevice, s), "H2D");
  check_cuda(cudaMemcpyAsync(c->d_tw, H.tw.data(), sizeof(u64) * H.tw.size(), cudaMemcpyHostToDevice, s), "H2D");
  if (H.narrow)
    check_cuda(cudaMemcpyAsync(c->d_tw32, H.tw32.data(), sizeof(u32) * H.tw32.size(), cudaMemcpyHostToDevice, s),
               "H2D");
  check_cuda(cudaMemcpyAsync(c->d_slot, H.slot_index.data(), sizeof(u32) * H.slot_index.size(), cudaMemcpyHostToDevice, s), "H2D");
  check_cuda(cudaMemcpyAsync(c->d_zeta, H.zeta.data(), sizeof(double) * H.zeta.size(), cudaMemcpyHostToDevice, s), "H2D");
  check_cuda(cudaMemcpyAsync(c->d_qwords, qw.data(), sizeof(u64) * qw.size(), cudaMemcpyHostToDevice, s), "H2D");
  c->table_bytes = sizeof(ModConst) * nm + sizeof(PairConst) * nm * nm + 8 * H.tw.size() + 4 * H.tw32.size() +
                   4 * H.slot_index.size() + 8 * H.zeta.size() + 8 * qw.size();
  c->T.mods = (const ModConst*)c->d_mods;
  c->T.pairs = (const PairConst*)c->d_pairs;
  c->T.tw = c->d_tw;
  c->T.tw32 = c->d_tw32;
  c->T.narrow = H.narrow ? 1u : 0u;
  c->T.log_n = params->log_n;
  c->T.n_mods = nm;
  c->T.L = c->L;
  c->T.dbg = (u32*)(c->d_status + 2);
  c->T.kerr = (u32*)(c->d_status + 3);
  if (c->hyb) {  // hybrid key-switching constants
    const std::vector<u64> hv = hyb_constants(params->chain, c->L, c->K, c->alpha, &c->H);
    c->d_hyb = (u64*)c->dev_alloc(sizeof(u64) * hv.size());
    check_cuda(cudaMemcpyAsync(c->d_hyb, hv.data(), sizeof(u64) * hv.size(), cudaMemcpyHostToDevice, s), "H2D");
    hyb_bind(c->d_hyb, &c->H);
    c->table_bytes += 8 * hv.size();
  }
  c->F.slot_index = c->d_slot;
  c->F.zeta = c->d_zeta;
  // keys (§2.1): secret, public, relinearization
  c->sk = (u64*)c->dev_alloc(sizeof(u64) * (size_t)nm * n);
  c->pk = (u64*)c->dev_alloc(sizeof(u64) * (size_t)2 * c->L * n);
  c->rlk = (u64*)c->dev_alloc(sizeof(u64) * ksk_words(c, c->L));
  launch_keygen_secret(c->T, seed, c->sk, s);
  launch_keygen_public(c->T, seed, c->sk, c->pk, s);
  if (c->hyb)
    launch_keygen_switch_hyb(c->T, c->H, seed, 0, c->sk, c->L, c->rlk, s);
  else
    launch_keygen_switch(c->T, seed, 0, c->sk, c->L, c->rlk, s);
  check_launch("keygen");
  check_cuda(cudaStreamSynchronize(s), "context create");
  *out = c;
  c = nullptr;
  TCKS_API_END
}

void tcks_ctx_free(tcks_ctx* c) {
  if (!c) return;
  ctx_release(c);
}

}  // extern "C"

static void ctx_destroy(tcks_ctx* c) {
  cudaStreamSynchronize(c->stream);
  c->keys_changed();
  for (auto& kv : c->galois) c->dev_free(kv.second.d);
  void* bufs[] = {c->d_mods, c->d_pairs, c->d_tw,  c->d_tw32, c->d_slot, c->d_zeta,
                  c->d_qwords, c->d_status, c->sk, c->pk,   c->rlk, c->d_hyb};
  for (void* b : bufs) c->dev_free(b);
  cudaStreamSynchronize(c->stream);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  cudaGetLastError();  // clean-up statuses are not reported: leave no error behind for later calls
}

extern "C" {

tcks_status tcks_ctx_info(const tcks_ctx* c, uint32_t* log_n, uint32_t* n_data_primes, double* scale) {
  TCKS_API_BEGIN
  if (!c) fail(TCKS_ERR_INVALID_ARG, "null context");
  if (log_n) *log_n = c->params.log_n;
  if (n_data_primes) *n_data_primes = c->L;
  if (scale) *scale = c->params.scale;
  TCKS_API_END
}

tcks_status tcks_ctx_key_bytes(const tcks_ctx* c, uint64_t* bytes) {
  TCKS_API_BEGIN
  if (!c || !bytes) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *bytes = c->key_bytes() + c->table_bytes;
  TCKS_API_END
}

tcks_status tcks_ctx_synchronize(tcks_ctx* c) {
  TCKS_API_BEGIN
  if (!c) fail(TCKS_ERR_INVALID_ARG, "null context");
  check_cuda(cudaStreamSynchronize(c->stream), "synchronize");
  kernel_error_check(c);
  TCKS_API_END
}

tcks_status tcks_ctx_set_launch_shape(tcks_ctx* c, uint32_t limb_threads, uint32_t accum_rpt, uint32_t accum_form) {
  TCKS_API_BEGIN
  if (!c) fail(TCKS_ERR_INVALID_ARG, "null context");
  if (limb_threads && (limb_threads % 32 || limb_threads > 1024)) fail(TCKS_ERR_INVALID_ARG, "limb_threads: 0 or a multiple of 32 up to 1024");
  if (accum_rpt > 2 && accum_rpt != 4) fail(TCKS_ERR_INVALID_ARG, "accum_rpt: 0 (default), 1, 2 or 4");
  if (accum_form > 4) fail(TCKS_ERR_INVALID_ARG, "accum_form: 0 (per-thread loads) or 1..4 (staged where possible)");
  c->T.limb_threads = limb_threads;
  c->T.dh_rpt = accum_rpt;
  c->T.dh_form = accum_form;
  TCKS_API_END
}

tcks_status tcks_ctx_get_launch_shape(const tcks_ctx* c, uint32_t* limb_threads, uint32_t* accum_rpt, uint32_t* accum_form) {
  TCKS_API_BEGIN
  if (!c || !limb_threads || !accum_rpt || !accum_form) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *limb_threads = c->T.limb_threads;
  *accum_rpt = c->T.dh_rpt;
  *accum_form = c->T.dh_form;
  TCKS_API_END
}

tcks_status tcks_ctx_set_flags(tcks_ctx* c, uint32_t flags) {
  TCKS_API_BEGIN
  if (!c) fail(TCKS_ERR_INVALID_ARG, "null context");
  if (flags & ~(u32)(TCKS_AUTO_RELIN | TCKS_AUTO_RESCALE | TCKS_DOUBLE_HOIST | TCKS_RECT_DIAG | TCKS_CONV_HOIST |
                     TCKS_CONV_SHARED | TCKS_CONV_PACK | TCKS_MERGED_RESCALE | TCKS_CONV_FOLD))
    fail(TCKS_ERR_INVALID_ARG, "unknown flag");
  c->flags = flags;
  TCKS_API_END
}

tcks_status tcks_gen_galois_keys(tcks_ctx* c, const int32_t* steps, uint32_t n_steps, uint32_t max_level) {
  TCKS_API_BEGIN
  if (!c || (n_steps && !steps)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  const u32 K = max_level == 0 ? c->L : max_level;
  if (K > c->L) fail(TCKS_ERR_INVALID_ARG, "max_level exceeds the number of data primes");
  c->keys_changed();
  for (u32 i = 0; i < n_steps; ++i) {
    const u32 k = step_mod(c, steps[i]);
    if (k == 0) continue;
    auto it = c->galois.find(k);
    if (it != c->galois.end()) {
      // a trimmed key is a prefix of the longer one (same sampler counters): keep the longer key
      if (it->second.K >= K) continue;
      c->dev_free(it->second.d);
      c->galois.erase(it);
    }
    GaloisKey gk;
    gk.K = K;
    gk.d = (u64*)c->dev_alloc(sizeof(u64) * ksk_words(c, K));
    const u32 g = (u32)galois_element(c->params.log_n, k);
    if (c->hyb)
      launch_keygen_switch_hyb(c->T, c->H, c->seed, g, c->sk, K, gk.d, c->stream);
    else
      launch_keygen_switch(c->T, c->seed, g, c->sk, K, gk.d, c->stream);
    check_launch("galois keygen");
    c->galois[k] = gk;
  }
  TCKS_API_END
}

tcks_status tcks_has_galois_key(const tcks_ctx* c, int32_t step, uint32_t* key_level) {
  TCKS_API_BEGIN
  if (!c) fail(TCKS_ERR_INVALID_ARG, "null context");
  auto it = c->galois.find(step_mod(c, step));
  if (it == c->galois.end()) fail(TCKS_ERR_NO_GALOIS_KEY, "no key");
  if (key_level) *key_level = it->second.K;
  TCKS_API_END
}

static u64* key_slot(tcks_ctx* c, uint32_t kind, int32_t step, size_t* words, u32* K_out) {
  const size_t n = c->N;
  const u32 L = c->L;
  switch (kind) {
    case TCKS_KEY_SECRET: *words = (size_t)(L + c->K) * n; return c->sk;
    case TCKS_KEY_PUBLIC: *words = (size_t)2 * L * n; return c->pk;
    case TCKS_KEY_RELIN: *words = ksk_words(c, L); return c->rlk;
    case TCKS_KEY_GALOIS: {
      auto it = c->galois.find(step_mod(c, step));
      if (it == c->galois.end()) fail(TCKS_ERR_NO_GALOIS_KEY, "no Galois key for this step");
      const u32 K = it->second.K;
      *words = ksk_words(c, K);
      if (K_out) *K_out = K;
      return it->second.d;
    }
    default: fail(TCKS_ERR_INVALID_ARG, "unknown key kind");
  }
}

tcks_status tcks_export_key(tcks_ctx* c, uint32_t kind, int32_t step, uint64_t* host, size_t n_words) {
  TCKS_API_BEGIN
  if (!c || !host) fail(TCKS_ERR_INVALID_ARG, "null argument");
  size_t words = 0;
  u64* d = key_slot(c, kind, step, &words, nullptr);
  if (n_words != words) fail(TCKS_ERR_INVALID_ARG, "n_words does not match the key layout");
  check_cuda(cudaMemcpyAsync(host, d, words * 8, cudaMemcpyDeviceToHost, c->stream), "export key");
  check_cuda(cudaStreamSynchronize(c->stream), "export key");
  TCKS_API_END
}

tcks_status tcks_import_key(tcks_ctx* c, uint32_t kind, int32_t step, uint32_t key_level, const uint64_t* host,
                            size_t n_words) {
  TCKS_API_BEGIN
  if (!c || !host) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (kind == TCKS_KEY_GALOIS) {
    const u32 k = step_mod(c, step);
    if (k == 0) fail(TCKS_ERR_INVALID_ARG, "step 0 has no key");
    const u32 K = key_level == 0 ? c->L : key_level;
    if (K > c->L) fail(TCKS_ERR_INVALID_ARG, "key_level exceeds L");
    const size_t words = ksk_words(c, K);
    if (n_words != words) fail(TCKS_ERR_INVALID_ARG, "n_words does not match the key layout");
    c->keys_changed();
    auto it = c->galois.find(k);
    if (it != c->galois.end()) {
      c->dev_free(it->second.d);
      c->galois.erase(it);
    }
    GaloisKey gk;
    gk.K = K;
    gk.d = (u64*)c->dev_alloc(words * 8);
    check_cuda(cudaMemcpyAsync(gk.d, host, words * 8, cudaMemcpyHostToDevice, c->stream), "import key");
    c->galois[k] = gk;
  } else {
    size_t words = 0;
    u64* d = key_slot(c, kind, step, &words, nullptr);
    if (n_words != words) fail(TCKS_ERR_INVALID_ARG, "n_words does not match the key layout");
    check_cuda(cudaMemcpyAsync(d, host, words * 8, cudaMemcpyHostToDevice, c->stream), "import key");
  }
  check_cuda(cudaStreamSynchronize(c->stream), "import key");
  TCKS_API_END
}

// ----------------------------------------------------------------------- encode / encrypt ----
tcks_status tcks_encode_device(tcks_ctx* c, const double* d_v, size_t n, double scale, uint32_t level,
                               tcks_pt** out) {
  TCKS_API_BEGIN
  if (!c || !out || (n && !d_v)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "more values than slots");
  const u32 l = level == 0 ? c->L : level;
  if (l > c->L) fail(TCKS_ERR_INVALID_ARG, "level exceeds L");
  const double sc = scale > 0 ? scale : c->params.scale;
  tcks_pt* pt = new_pt(c, l, sc);
  try {
    encode_into(c, d_v, n, sc, l, pt->d);
  } catch (...) {
    c->dev_free(pt->d);
    delete pt;
    throw;
  }
  *out = pt;
  TCKS_API_END
}

tcks_status tcks_encode(tcks_ctx* c, const double* v, size_t n, double scale, uint32_t level, tcks_pt** out) {
  TCKS_API_BEGIN
  if (!c || !out || (n && !v)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "more values than slots");
  DevBuf dv(c, n ? n : 1);
  if (n) check_cuda(cudaMemcpyAsync(dv.p, v, n * 8, cudaMemcpyHostToDevice, c->stream), "encode H2D");
  const tcks_status s = tcks_encode_device(c, (const double*)dv.p, n, scale, level, out);
  if (s != TCKS_OK) return s;
  TCKS_API_END
}

tcks_status tcks_decode(tcks_ctx* c, const tcks_pt* pt, double* out, size_t n) {
  TCKS_API_BEGIN
  if (!c || !pt || (n && !out)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "more values than slots");
  if (c->params.log_n > 14) fail(TCKS_ERR_UNSUPPORTED, "decoding is implemented for N <= 2^14");
  const size_t N = c->N;
  DevBuf coef(c, (size_t)pt->level * N), p(c, N), z(c, n ? n : 1);
  launch_ntt(c->T, true, pt->d, 0, coef.p, 0, pt->level, 0, pt->level, c->stream);
  launch_crt_compose(c->T, coef.p, pt->level, c->d_qwords, (double*)p.p, c->stream);
  launch_decode_slots(c->T, c->F, (const double*)p.p, pt->scale, (u32)n, (double*)z.p, c->stream);
  check_launch("decode");
  if (n) check_cuda(cudaMemcpyAsync(out, z.p, n * 8, cudaMemcpyDeviceToHost, c->stream), "decode D2H");
  check_cuda(cudaStreamSynchronize(c->stream), "decode");
  TCKS_API_END
}

tcks_status tcks_encrypt(tcks_ctx* c, const tcks_pt* pt, uint64_t seed, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!c || !pt || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tcks_ct* ct = new_ct(c, pt->level, pt->scale);
  launch_encrypt(c->T, seed, c->pk, pt->d, pt->level, ct->d, c->stream);
  check_launch("encrypt");
  *out = ct;
  TCKS_API_END
}

tcks_status tcks_encrypt_symmetric(tcks_ctx* c, const tcks_pt* pt, uint64_t seed_a, uint64_t seed_e, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!c || !pt || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (pt->ctx != c) fail(TCKS_ERR_INVALID_ARG, "plaintext of another context");
  tcks_ct* ct = new_ct(c, pt->level, pt->scale);
  launch_encrypt_sym(c->T, seed_a, seed_e, c->sk, pt->d, pt->level, ct->d, c->stream);
  check_launch("secret-key encrypt");
  *out = ct;
  TCKS_API_END
}

tcks_status tcks_decrypt(tcks_ctx* c, const tcks_ct* ct, tcks_pt** out) {
  TCKS_API_BEGIN
  if (!c || !ct || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tcks_pt* pt = new_pt(c, ct->level, ct->scale);
  launch_decrypt(c->T, ct->d, c->sk, pt->d, ct->level, c->stream, ct->size);
  check_launch("decrypt");
  *out = pt;
  TCKS_API_END
}

tcks_status tcks_ct_import(tcks_ctx* c, const uint64_t* limbs, uint32_t level, double scale, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!c || !limbs || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (level < 1 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  tcks_ct* ct = new_ct(c, level, scale);
  check_cuda(cudaMemcpyAsync(ct->d, limbs, ct_words(c, level) * 8, cudaMemcpyHostToDevice, c->stream), "ct import");
  check_cuda(cudaStreamSynchronize(c->stream), "ct import");
  *out = ct;
  TCKS_API_END
}

tcks_status tcks_ct_import_sized(tcks_ctx* c, const uint64_t* limbs, uint32_t size, uint32_t level, double scale,
                                 tcks_ct** out) {
  TCKS_API_BEGIN
  if (!c || !limbs || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (size != 2 && size != 3) fail(TCKS_ERR_INVALID_ARG, "a ciphertext has 2 or 3 components");
  if (level < 1 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  tcks_ct* ct = new_ct_sized(c, size, level, scale);
  const size_t words = (size_t)size * level * c->N;
  try {
    check_cuda(cudaMemcpyAsync(ct->d, limbs, words * 8, cudaMemcpyHostToDevice, c->stream), "ct import");
    check_cuda(cudaStreamSynchronize(c->stream), "ct import");
  } catch (...) {
    free_ct(ct);
    throw;
  }
  *out = ct;
  TCKS_API_END
}

tcks_status tcks_ct_size(const tcks_ct* ct, uint32_t* size) {
  TCKS_API_BEGIN
  if (!ct || !size) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *size = ct->size;
  TCKS_API_END
}

tcks_status tcks_ct_import_batch(tcks_ctx* c, const uint64_t* limbs, uint32_t count, uint32_t level, double scale,
                                 tcks_ct** outs) {
  std::vector<tcks_ct*> made;
  TCKS_API_BEGIN
  if (!c || !outs || (count && !limbs)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  for (u32 i = 0; i < count; ++i) outs[i] = nullptr;
  if (level < 1 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  const u64 w = ct_words(c, level);
  try {
    for (u32 i = 0; i < count; ++i) {
      made.push_back(new_ct(c, level, scale));
      check_cuda(cudaMemcpyAsync(made.back()->d, limbs + (size_t)i * w, w * 8, cudaMemcpyHostToDevice, c->stream),
                 "ct import");
    }
    check_cuda(cudaStreamSynchronize(c->stream), "ct import");
  } catch (...) {
    for (tcks_ct* t : made) free_ct(t);
    throw;
  }
  for (u32 i = 0; i < count; ++i) outs[i] = made[i];
  TCKS_API_END
}

tcks_status tcks_ct_export_batch(const tcks_ct* const* cts, uint32_t count, uint64_t* limbs, size_t n_words) {
  TCKS_API_BEGIN
  if (!cts || (count && !limbs)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (!count) return TCKS_OK;
  if (!cts[0]) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
  tcks_ctx* c = cts[0]->ctx;
  const u32 level = cts[0]->level;
  const u64 w = ct_words(c, level);
  if (n_words != (size_t)count * w) fail(TCKS_ERR_INVALID_ARG, "n_words does not match [count][2][level][N]");
  for (u32 i = 0; i < count; ++i) {
    if (!cts[i] || cts[i]->ctx != c || cts[i]->level != level)
      fail(TCKS_ERR_INVALID_ARG, "the batch must share one context and level");
    need_relinearized(cts[i]);
  }
  for (u32 i = 0; i < count; ++i)
    check_cuda(cudaMemcpyAsync(limbs + (size_t)i * w, cts[i]->d, w * 8, cudaMemcpyDeviceToHost, c->stream), "ct export");
  check_cuda(cudaStreamSynchronize(c->stream), "ct export");
  TCKS_API_END
}

tcks_status tcks_ct_export(const tcks_ct* ct, uint64_t* limbs, size_t n_words) {
  TCKS_API_BEGIN
  if (!ct || !limbs) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (n_words != (size_t)ct->size * ct->level * ct->ctx->N)
    fail(TCKS_ERR_INVALID_ARG, "n_words does not match [size][level][N]");
  check_cuda(cudaMemcpyAsync(limbs, ct->d, n_words * 8, cudaMemcpyDeviceToHost, ct->ctx->stream), "ct export");
  check_cuda(cudaStreamSynchronize(ct->ctx->stream), "ct export");
  kernel_error_check(ct->ctx);
  TCKS_API_END
}

// ------------------------------------------------------------------------- wire format ----

tcks_status tcks_ct_serialized_size(const tcks_ct* ct, uint64_t* bytes) {
  TCKS_API_BEGIN
  if (!ct || !bytes) fail(TCKS_ERR_INVALID_ARG, "null argument");
  need_relinearized(ct);
  *bytes = kWireHeader + wire_payload_bytes(ct->ctx->T, ct->ctx->host.chain.data(), ct->level);
  TCKS_API_END
}

tcks_status tcks_ct_serialize(const tcks_ct* ct, uint8_t* out, uint64_t cap, uint64_t* written) {
  TCKS_API_BEGIN
  if (!ct || !out || !written) fail(TCKS_ERR_INVALID_ARG, "null argument");
  tcks_ctx* c = ct->ctx;
  need_relinearized(ct);
  const u64 payload = wire_payload_bytes(c->T, c->host.chain.data(), ct->level);
  if (cap < kWireHeader + payload) fail(TCKS_ERR_INVALID_ARG, "capacity below the serialized size");
  DevBuf buf(c, (payload + 7) / 8);
  launch_pack(c->T, ct->d, ct->level, (unsigned char*)buf.p, c->stream);
  check_launch("serialize");
  check_cuda(cudaMemcpyAsync(out + kWireHeader, buf.p, payload, cudaMemcpyDeviceToHost, c->stream), "serialize");
  std::memcpy(out, kWireMagic, 4);
  out[4] = 1;  // version
  out[5] = 0;  // kind: ciphertext
  out[6] = (uint8_t)c->params.log_n;
  out[7] = (uint8_t)ct->level;
  std::memcpy(out + 8, &ct->scale, 8);
  check_cuda(cudaStreamSynchronize(c->stream), "serialize");
  *written = kWireHeader + payload;
  TCKS_API_END
}

tcks_status tcks_ct_serialized_size_seeded(const tcks_ct* ct, uint64_t* bytes) {
  TCKS_API_BEGIN
  if (!ct || !bytes) fail(TCKS_ERR_INVALID_ARG, "null argument");
  need_relinearized(ct);
  *bytes = kWireHeader + 8 + wire_payload_bytes(ct->ctx->T, ct->ctx->host.chain.data(), ct->level) / 2;
  TCKS_API_END
}

tcks_status tcks_ct_serialize_seeded(const tcks_ct* ct, uint64_t seed_a, uint8_t* out, uint64_t cap,
                                     uint64_t* written) {
  TCKS_API_BEGIN
  if (!ct || !out || !written) fail(TCKS_ERR_INVALID_ARG, "null argument");
  tcks_ctx* c = ct->ctx;
  need_relinearized(ct);
  const u64 payload = wire_payload_bytes(c->T, c->host.chain.data(), ct->level) / 2;
  if (cap < kWireHeader + 8 + payload) fail(TCKS_ERR_INVALID_ARG, "capacity below the serialized size");
  // the receiver regenerates c1 from the seed: refuse a ciphertext whose c1 is not that polynomial
  check_cuda(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "seeded status");
  launch_sym_a(c->T, seed_a, ct->level, ct->d + (size_t)ct->level * c->N, true, c->d_status, c->stream);
  DevBuf buf(c, (payload + 7) / 8);
  launch_pack(c->T, ct->d, ct->level, (unsigned char*)buf.p, c->stream, 1);
  check_launch("serialize (seeded)");
  int status = 0;
  check_cuda(cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "seeded status");
  check_cuda(cudaMemcpyAsync(out + kWireHeader + 8, buf.p, payload, cudaMemcpyDeviceToHost, c->stream), "serialize");
  check_cuda(cudaStreamSynchronize(c->stream), "serialize");
  if (status) fail(TCKS_ERR_INVALID_ARG, "c1 is not the uniform polynomial of this seed");
  std::memcpy(out, kWireMagic, 4);
  out[4] = 1;  // version
  out[5] = 1;  // kind: seeded secret-key ciphertext
  out[6] = (uint8_t)c->params.log_n;
  out[7] = (uint8_t)ct->level;
  std::memcpy(out + 8, &ct->scale, 8);
  for (int b = 0; b < 8; ++b) out[kWireHeader + b] = (uint8_t)(seed_a >> (8 * b));
  *written = kWireHeader + 8 + payload;
  TCKS_API_END
}

tcks_status tcks_ct_deserialize(tcks_ctx* c, const uint8_t* in, uint64_t size, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!c || !in || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (size < kWireHeader || std::memcmp(in, kWireMagic, 4) != 0) fail(TCKS_ERR_INVALID_ARG, "not a serialized ciphertext");
  if (in[4] != 1 || in[5] > 1) fail(TCKS_ERR_INVALID_ARG, "unsupported version or kind");
  const bool seeded = in[5] == 1;
  if (in[6] != c->params.log_n) fail(TCKS_ERR_INVALID_ARG, "ring degree differs from the context's");
  const u32 level = in[7];
  if (level < 1 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  double scale;
  std::memcpy(&scale, in + 8, 8);
  const u64 full = wire_payload_bytes(c->T, c->host.chain.data(), level);
  const u64 payload = seeded ? full / 2 : full;
  const u64 head = kWireHeader + (seeded ? 8 : 0);
  if (size != head + payload) fail(TCKS_ERR_INVALID_ARG, "size does not match the header");
  u64 seed_a = 0;
  if (seeded)
    for (int b = 0; b < 8; ++b) seed_a |= (u64)in[kWireHeader + b] << (8 * b);
  tcks_ct* r = new_ct(c, level, scale);
  try {
    DevBuf buf(c, (payload + 7) / 8);
    check_cuda(cudaMemcpyAsync(buf.p, in + head, payload, cudaMemcpyHostToDevice, c->stream), "deserialize");
    check_cuda(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "deserialize status");
    launch_unpack(c->T, (const unsigned char*)buf.p, level, r->d, c->d_status, c->stream, seeded ? 1 : 2);
    if (seeded) launch_sym_a(c->T, seed_a, level, r->d + (size_t)level * c->N, false, nullptr, c->stream);
    check_launch("deserialize");
    int status = 0;
    check_cuda(cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "deserialize");
    check_cuda(cudaStreamSynchronize(c->stream), "deserialize");
    if (status) fail(TCKS_ERR_INVALID_ARG, "a residue is not below its prime");
  } catch (...) {
    free_ct(r);
    throw;
  }
  *out = r;
  TCKS_API_END
}

tcks_status tcks_pt_import(tcks_ctx* c, const uint64_t* limbs, uint32_t level, double scale, tcks_pt** out) {
  TCKS_API_BEGIN
  if (!c || !limbs || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (level < 1 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  tcks_pt* pt = new_pt(c, level, scale);
  check_cuda(cudaMemcpyAsync(pt->d, limbs, pt_words(c, level) * 8, cudaMemcpyHostToDevice, c->stream), "pt import");
  check_cuda(cudaStreamSynchronize(c->stream), "pt import");
  *out = pt;
  TCKS_API_END
}

tcks_status tcks_pt_export(const tcks_pt* pt, uint64_t* limbs, size_t n_words) {
  TCKS_API_BEGIN
  if (!pt || !limbs) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (n_words != pt_words(pt->ctx, pt->level)) fail(TCKS_ERR_INVALID_ARG, "n_words does not match [level][N]");
  check_cuda(cudaMemcpyAsync(limbs, pt->d, n_words * 8, cudaMemcpyDeviceToHost, pt->ctx->stream), "pt export");
  check_cuda(cudaStreamSynchronize(pt->ctx->stream), "pt export");
  TCKS_API_END
}

tcks_status tcks_ct_info(const tcks_ct* ct, uint32_t* level, double* scale) {
  TCKS_API_BEGIN
  if (!ct) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
  if (level) *level = ct->level;
  if (scale) *scale = ct->scale;
  TCKS_API_END
}

tcks_status tcks_pt_info(const tcks_pt* pt, uint32_t* level, double* scale) {
  TCKS_API_BEGIN
  if (!pt) fail(TCKS_ERR_INVALID_ARG, "null plaintext");
  if (level) *level = pt->level;
  if (scale) *scale = pt->scale;
  TCKS_API_END
}

tcks_status tcks_ct_device_ptr(const tcks_ct* ct, uint64_t** d_limbs) {
  TCKS_API_BEGIN
  if (!ct || !d_limbs) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *d_limbs = ct->d;
  TCKS_API_END
}

void tcks_ct_free(tcks_ct* ct) { free_ct(ct); }

void tcks_pt_free(tcks_pt* pt) {
  if (!pt) return;
  tcks_ctx* c = pt->ctx;
  if (pt->d) c->dev_free(pt->d);
  delete pt;
  ctx_release(c);
}

// ------------------------------------------------------------------------ element-wise ops ----
static void check_pair(const tcks_ct* a, const tcks_ct* b, bool need_scale) {
  if (!a || !b) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
  if (a->ctx != b->ctx) fail(TCKS_ERR_INVALID_ARG, "operands belong to different contexts");
  if (a->level != b->level) fail(TCKS_ERR_LEVEL_MISMATCH, "operands at different levels");
  if (need_scale && a->scale != b->scale) fail(TCKS_ERR_SCALE_MISMATCH, "operands at different scales");
}

// Sum or difference; with a three-component operand the result has three components, a missing
// third component being the zero polynomial.
static tcks_status binary_ct(const tcks_ct* a, const tcks_ct* b, u32 op, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null output");
  *out = nullptr;
  check_pair(a, b, true);
  tcks_ctx* c = a->ctx;
  const u32 size = std::max(a->size, b->size), common = std::min(a->size, b->size);
  tcks_ct* r = new_ct_sized(c, size, a->level, a->scale);
  const size_t pw = (size_t)a->level * c->N;  // words of one component
  launch_elementwise(c->T, op, a->d, b->d, r->d, a->level, common, c->stream);
  if (size > common) {
    const tcks_ct* big = a->size > b->size ? a : b;
    if (big == b && op == OP_SUB)
      launch_elementwise(c->T, OP_NEG, b->d + 2 * pw, nullptr, r->d + 2 * pw, a->level, 1, c->stream);
    else
      check_cuda(cudaMemcpyAsync(r->d + 2 * pw, big->d + 2 * pw, pw * 8, cudaMemcpyDeviceToDevice, c->stream),
                 "third component");
  }
  check_launch("elementwise");
  *out = r;
  TCKS_API_END
}

tcks_status tcks_add(const tcks_ct* a, const tcks_ct* b, tcks_ct** out) { return binary_ct(a, b, OP_ADD, out); }
tcks_status tcks_sub(const tcks_ct* a, const tcks_ct* b, tcks_ct** out) { return binary_ct(a, b, OP_SUB, out); }

tcks_status tcks_negate(const tcks_ct* a, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tcks_ct* r = new_ct_sized(a->ctx, a->size, a->level, a->scale);
  launch_elementwise(a->ctx->T, OP_NEG, a->d, nullptr, r->d, a->level, a->size, a->ctx->stream);
  check_launch("negate");
  *out = r;
  TCKS_API_END
}

static tcks_status plain_op(const tcks_ct* a, const tcks_pt* p, u32 op, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !p || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (a->ctx != p->ctx) fail(TCKS_ERR_INVALID_ARG, "operands belong to different contexts");
  if (p->level < a->level) fail(TCKS_ERR_LEVEL_MISMATCH, "plaintext level below the ciphertext level");
  if (op != OP_MUL_PLAIN && p->scale != a->scale) fail(TCKS_ERR_SCALE_MISMATCH, "plaintext scale differs");
  tcks_ct* r = new_ct_sized(a->ctx, a->size, a->level, op == OP_MUL_PLAIN ? a->scale * p->scale : a->scale);
  // add/sub change c0 only: a third component is copied as it is; a product multiplies every component
  launch_elementwise(a->ctx->T, op, a->d, p->d, r->d, a->level, op == OP_MUL_PLAIN ? a->size : 2, a->ctx->stream);
  if (op != OP_MUL_PLAIN && a->size == 3) {
    const size_t pw = (size_t)a->level * a->ctx->N;
    check_cuda(cudaMemcpyAsync(r->d + 2 * pw, a->d + 2 * pw, pw * 8, cudaMemcpyDeviceToDevice, a->ctx->stream),
               "third component");
  }
  check_launch("plain op");
  *out = r;
  TCKS_API_END
}

tcks_status tcks_add_plain(const tcks_ct* a, const tcks_pt* p, tcks_ct** out) { return plain_op(a, p, OP_ADD_PLAIN, out); }
tcks_status tcks_sub_plain(const tcks_ct* a, const tcks_pt* p, tcks_ct** out) { return plain_op(a, p, OP_SUB_PLAIN, out); }
tcks_status tcks_mul_plain(const tcks_ct* a, const tcks_pt* p, tcks_ct** out) { return plain_op(a, p, OP_MUL_PLAIN, out); }

tcks_status tcks_mul(const tcks_ct* a, const tcks_ct* b, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null output");
  *out = nullptr;
  check_pair(a, b, false);
  need_relinearized(a);
  need_relinearized(b);
  tcks_ctx* c = a->ctx;
  const u32 ell = a->level;
  const bool rescale = (c->flags & TCKS_AUTO_RESCALE) != 0;
  if (rescale && ell < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "multiply with auto-rescale needs level >= 2");
  const double sc = a->scale * b->scale;
  if (!(c->flags & TCKS_AUTO_RELIN)) {  // the three-component product, rescaled component by component
    if (!rescale) {
      tcks_ct* r = new_ct_sized(c, 3, ell, sc);
      launch_tensor(c->T, a->d, b->d, r->d, ell, 1, c->stream);
      check_launch("tensor");
      *out = r;
      return TCKS_OK;
    }
    DevBuf d3(c, (size_t)3 * ell * c->N);
    launch_tensor(c->T, a->d, b->d, d3.p, ell, 1, c->stream);
    tcks_ct* r = new_ct_sized(c, 3, ell - 1, sc / (double)c->host.chain[ell - 1]);
    try {
      op_rescale_polys(c, d3.p, ell, 3, r->d);
    } catch (...) {
      free_ct(r);
      throw;
    }
    *out = r;
    return TCKS_OK;
  }
  DevBuf d3(c, (size_t)3 * ell * c->N);
  launch_tensor(c->T, a->d, b->d, d3.p, ell, 1, c->stream);
  check_launch("tensor");
  if (!rescale) {
    tcks_ct* r = new_ct(c, ell, sc);
    op_relinearize(c, d3.p, ell, r->d);
    *out = r;
  } else if (c->flags & TCKS_MERGED_RESCALE) {
    tcks_ct* r = new_ct(c, ell - 1, sc / (double)c->host.chain[ell - 1]);
    op_relin_rescale(c, d3.p, ell, r->d);
    *out = r;
  } else {
    DevBuf rel(c, ct_words(c, ell));
    op_relinearize(c, d3.p, ell, rel.p);
    tcks_ct* r = new_ct(c, ell - 1, sc / (double)c->host.chain[ell - 1]);
    op_rescale(c, rel.p, ell, r->d);
    *out = r;
  }
  TCKS_API_END
}

tcks_status tcks_square(const tcks_ct* a, tcks_ct** out) { return tcks_mul(a, a, out); }

tcks_status tcks_relinearize(tcks_ct* ct) {
  TCKS_API_BEGIN
  if (!ct) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
  if (ct->size == 2) return TCKS_OK;
  tcks_ctx* c = ct->ctx;
  DevBuf nb(c, ct_words(c, ct->level));
  op_relinearize(c, ct->d, ct->level, nb.p);
  c->dev_free(ct->d);
  ct->d = nb.release();
  ct->size = 2;
  TCKS_API_END
}

tcks_status tcks_rescale(tcks_ct* ct) {
  TCKS_API_BEGIN
  if (!ct) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
  tcks_ctx* c = ct->ctx;
  if (ct->level < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "rescale needs level >= 2");
  DevBuf nb(c, (size_t)ct->size * (ct->level - 1) * c->N);
  op_rescale_polys(c, ct->d, ct->level, ct->size, nb.p);
  c->dev_free(ct->d);
  ct->d = nb.release();
  ct->scale = ct->scale / (double)c->host.chain[ct->level - 1];
  ct->level -= 1;
  TCKS_API_END
}

tcks_status tcks_mod_switch(tcks_ct* ct, uint32_t level) {
  TCKS_API_BEGIN
  if (!ct) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
  if (level < 1 || level > ct->level) fail(TCKS_ERR_INVALID_ARG, "target level out of range");
  if (level == ct->level) return TCKS_OK;
  tcks_ctx* c = ct->ctx;
  DevBuf nb(c, (size_t)ct->size * level * c->N);
  const size_t n = c->N;
  check_cuda(cudaMemcpy2DAsync(nb.p, (size_t)level * n * 8, ct->d, (size_t)ct->level * n * 8, (size_t)level * n * 8,
                               ct->size, cudaMemcpyDeviceToDevice, c->stream),
             "mod switch");
  c->dev_free(ct->d);
  ct->d = nb.release();
  ct->level = level;
  TCKS_API_END
}

tcks_status tcks_ntt_inplace(tcks_ctx* c, uint64_t* d_limbs, uint32_t polys, uint32_t level, int32_t inverse) {
  TCKS_API_BEGIN
  if (!c || !d_limbs) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (level < 1 || level > c->L + 1) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  const u64 n = c->N;
  launch_ntt(c->T, inverse != 0, d_limbs, (u64)level * n, d_limbs, (u64)level * n, polys * level, 0, level,
             c->stream);
  check_launch("ntt");
  TCKS_API_END
}

// ------------------------------------------------------------------------------- rotations ----
tcks_status tcks_rotate(const tcks_ct* a, int32_t step, tcks_ct** out) { return tcks_rotate_hoisted(a, &step, 1, out); }

tcks_status tcks_rotate_hoisted(const tcks_ct* a, const int32_t* steps, uint32_t n_steps, tcks_ct** outs) {
  std::vector<tcks_ct*> made;
  TCKS_API_BEGIN
  if (!a || !outs || (n_steps && !steps)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  for (u32 i = 0; i < n_steps; ++i) outs[i] = nullptr;
  need_relinearized(a);
  tcks_ctx* c = a->ctx;
  for (u32 i = 0; i < n_steps; ++i)
    if (step_mod(c, steps[i])) galois_key_for(c, steps[i], a->level);  // validate first
  std::vector<u64*> ptrs(n_steps);
  for (u32 i = 0; i < n_steps; ++i) {
    made.push_back(new_ct(c, a->level, a->scale));
    ptrs[i] = made.back()->d;
  }
  op_rotate_hoisted(c, a->d, a->level, steps, n_steps, ptrs.data());
  for (u32 i = 0; i < n_steps; ++i) outs[i] = made[i];
  made.clear();
  return TCKS_OK;
  }
  catch (const tcks::Error& e) {
    for (tcks_ct* m : made) free_ct(m);
    return record(e.code, e.msg);
  }
  catch (const std::bad_alloc&) {
    for (tcks_ct* m : made) free_ct(m);
    return record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed");
  }
}

// --------------------------------------------------------------------------- composites ----
tcks_status tcks_rotate_sum_hoisted(const tcks_ct* a, const int32_t* steps, uint32_t n_steps, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !out || (n_steps && !steps)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  need_relinearized(a);
  tcks_ctx* c = a->ctx;
  std::vector<int32_t> st(steps, steps + n_steps);
  for (int32_t s : st) {  // validate before launching anything
    if (!step_mod(c, s)) fail(TCKS_ERR_INVALID_ARG, "a rotation sum step of 0 (the identity is always included)");
    galois_key_for(c, s, a->level);
  }
  tcks_ct* r = new_ct(c, a->level, a->scale);
  try {
    op_rotsum_hoisted(c, a->d, ct_words(c, a->level), 1, a->level, st, r->d);
  } catch (...) {
    free_ct(r);
    throw;
  }
  *out = r;
  TCKS_API_END
}

tcks_status tcks_sum(const tcks_ct* a, uint32_t n, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tcks_ctx* c = a->ctx;
  if (n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "n exceeds the slot count");
  need_relinearized(a);
  for (u32 m = 0; m + 1 < c->params.log_n; ++m) galois_key_for(c, (int32_t)(1u << m), a->level);
  tcks_ct* r = new_ct(c, a->level, a->scale);
  check_cuda(cudaMemcpyAsync(r->d, a->d, ct_words(c, a->level) * 8, cudaMemcpyDeviceToDevice, c->stream), "sum copy");
  try {
    op_sum(c, r->d, r->level);
  } catch (...) {
    free_ct(r);
    throw;
  }
  *out = r;
  TCKS_API_END
}

tcks_status tcks_dot(const tcks_ct* a, const tcks_ct* b, uint32_t n, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null output");
  *out = nullptr;
  tcks_ct* prod = nullptr;
  tcks_status s = tcks_mul(a, b, &prod);
  if (s != TCKS_OK) return s;
  s = tcks_sum(prod, n, out);
  free_ct(prod);
  if (s != TCKS_OK) return s;
  TCKS_API_END
}

tcks_status tcks_dot_plain(const tcks_ct* a, const double* w, uint32_t n, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !w || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  need_relinearized(a);
  tcks_pt* p = nullptr;
  tcks_status s = tcks_encode(a->ctx, w, n, 0.0, a->level, &p);
  if (s != TCKS_OK) return s;
  tcks_ct* prod = nullptr;
  s = tcks_mul_plain(a, p, &prod);
  tcks_pt_free(p);
  if (s != TCKS_OK) return s;
  s = tcks_rescale(prod);
  if (s == TCKS_OK) s = tcks_sum(prod, n, out);
  free_ct(prod);
  if (s != TCKS_OK) return s;
  TCKS_API_END
}

tcks_status tcks_matrix_encode(tcks_ctx* c, const double* M, uint32_t rows, uint32_t cols, uint32_t level,
                               tcks_matrix** out) {
  TCKS_API_BEGIN
  if (!c || !M || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const u32 slots = c->N / 2;
  if (rows == 0 || cols == 0 || cols > rows || rows > slots || (rows & (rows - 1)) || slots % rows)
    fail(TCKS_ERR_INVALID_ARG, "need cols <= rows, rows a power of two dividing N/2");
  const u32 l = level == 0 ? c->L : level;
  if (l < 2 || l > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range (needs >= 2 for the rescale)");
  // each diagonal over the extended basis (level limbs, then P): the single-hoisted product reads
  // the first `level` limbs, the double-hoisted one all of them
  DevBuf d(c, (size_t)rows * (l + 1) * c->N);
  DevBuf dv(c, slots);
  std::vector<double> diag(slots);
  for (u32 k = 0; k < rows; ++k) {
    std::fill(diag.begin(), diag.end(), 0.0);
    for (u32 s2 = 0; s2 < cols; ++s2) diag[s2] = M[(size_t)((s2 + k) % rows) * cols + s2];
    check_cuda(cudaMemcpyAsync(dv.p, diag.data(), (size_t)slots * 8, cudaMemcpyHostToDevice, c->stream), "diag H2D");
    encode_into(c, (const double*)dv.p, slots, c->params.scale, l, d.p + (size_t)k * (l + 1) * c->N, true);
  }
  *out = new tcks_matrix{c, rows, cols, l, 1, c->params.scale, d.release(), rows, 0};
  ctx_retain(c);
  TCKS_API_END
}

tcks_status tcks_matrix_encode_rect(tcks_ctx* c, const double* M, uint32_t rows, uint32_t cols, uint32_t level,
                                   tcks_matrix** out) {
  TCKS_API_BEGIN
  if (!c || !M || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const u32 slots = c->N / 2;
  if (rows == 0 || cols == 0 || cols > rows || rows > slots || (rows & (rows - 1)) || slots % rows)
    fail(TCKS_ERR_INVALID_ARG, "need cols <= rows, rows a power of two dividing N/2");
  const u32 l = level == 0 ? c->L : level;
  if (l < 2 || l > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range (needs >= 2 for the rescale)");
  u32 mw = 1;
  while (mw < cols) mw <<= 1;
  // d_k[t] = M[(t' + k) mod n][t' mod m'] with t' = t mod n, zero where t' mod m' >= cols; period n
  DevBuf d(c, (size_t)mw * (l + 1) * c->N);
  DevBuf dv(c, slots);
  std::vector<double> diag(slots);
  for (u32 k = 0; k < mw; ++k) {
    for (u32 t = 0; t < slots; ++t) {
      const u32 tp = t % rows, col = tp % mw;
      diag[t] = col < cols ? M[(size_t)((tp + k) % rows) * cols + col] : 0.0;
    }
    check_cuda(cudaMemcpyAsync(dv.p, diag.data(), (size_t)slots * 8, cudaMemcpyHostToDevice, c->stream), "diag H2D");
    encode_into(c, (const double*)dv.p, slots, c->params.scale, l, d.p + (size_t)k * (l + 1) * c->N, true);
  }
  *out = new tcks_matrix{c, rows, cols, l, 1, c->params.scale, d.release(), mw, 1};
  ctx_retain(c);
  TCKS_API_END
}

tcks_status tcks_matrix_import(tcks_ctx* c, const uint64_t* diag_limbs, uint32_t rows, uint32_t cols, uint32_t level,
                               double scale, tcks_matrix** out) {
  TCKS_API_BEGIN
  if (!c || !diag_limbs || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const u32 slots = c->N / 2;
  if (rows == 0 || cols == 0 || cols > rows || rows > slots || (rows & (rows - 1)) || slots % rows)
    fail(TCKS_ERR_INVALID_ARG, "need cols <= rows, rows a power of two dividing N/2");
  if (level < 2 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  const size_t words = (size_t)rows * level * c->N;
  DevBuf d(c, words);
  check_cuda(cudaMemcpyAsync(d.p, diag_limbs, words * 8, cudaMemcpyHostToDevice, c->stream), "matrix import");
  check_cuda(cudaStreamSynchronize(c->stream), "matrix import");
  *out = new tcks_matrix{c, rows, cols, level, 0, scale, d.release(), rows, 0};
  ctx_retain(c);
  TCKS_API_END
}

tcks_status tcks_matrix_import_ext(tcks_ctx* c, const uint64_t* diag_limbs, uint32_t rows, uint32_t cols,
                                   uint32_t level, double scale, tcks_matrix** out) {
  TCKS_API_BEGIN
  if (!c || !diag_limbs || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const u32 slots = c->N / 2;
  if (rows == 0 || cols == 0 || cols > rows || rows > slots || (rows & (rows - 1)) || slots % rows)
    fail(TCKS_ERR_INVALID_ARG, "need cols <= rows, rows a power of two dividing N/2");
  if (level < 2 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  const size_t words = (size_t)rows * (level + 1) * c->N;
  DevBuf d(c, words);
  check_cuda(cudaMemcpyAsync(d.p, diag_limbs, words * 8, cudaMemcpyHostToDevice, c->stream), "matrix import");
  check_cuda(cudaStreamSynchronize(c->stream), "matrix import");
  *out = new tcks_matrix{c, rows, cols, level, 1, scale, d.release(), rows, 0};
  ctx_retain(c);
  TCKS_API_END
}

tcks_status tcks_matrix_import_rect(tcks_ctx* c, const uint64_t* diag_limbs, uint32_t rows, uint32_t cols,
                                    uint32_t level, double scale, tcks_matrix** out) {
  TCKS_API_BEGIN
  if (!c || !diag_limbs || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const u32 slots = c->N / 2;
  if (rows == 0 || cols == 0 || cols > rows || rows > slots || (rows & (rows - 1)) || slots % rows)
    fail(TCKS_ERR_INVALID_ARG, "need cols <= rows, rows a power of two dividing N/2");
  if (level < 2 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  u32 mw = 1;
  while (mw < cols) mw <<= 1;
  const size_t words = (size_t)mw * (level + 1) * c->N;
  DevBuf d(c, words);
  check_cuda(cudaMemcpyAsync(d.p, diag_limbs, words * 8, cudaMemcpyHostToDevice, c->stream), "matrix import");
  check_cuda(cudaStreamSynchronize(c->stream), "matrix import");
  *out = new tcks_matrix{c, rows, cols, level, 1, scale, d.release(), mw, 1};
  ctx_retain(c);
  TCKS_API_END
}

void tcks_matrix_free(tcks_matrix* m) {
  if (!m) return;
  tcks_ctx* c = m->ctx;
  c->dev_free(m->d);
  delete m;
  ctx_release(c);
}

tcks_status tcks_vecmat_plain(const tcks_ct* a, const tcks_matrix* M, tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !M || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  need_relinearized(a);
  tcks_ctx* c = a->ctx;
  if (M->ctx != c) fail(TCKS_ERR_INVALID_ARG, "matrix belongs to another context");
  if (M->level < a->level) fail(TCKS_ERR_LEVEL_MISMATCH, "matrix encoded below the ciphertext level");
  if (a->level < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "vecmat needs level >= 2");
  tcks_ct* r = new_ct(c, a->level - 1, a->scale * M->scale / (double)c->host.chain[a->level - 1]);
  try {
    op_vecmat(c, a->d, 0, 1, a->level, M, r->d);
  } catch (...) {
    free_ct(r);
    throw;
  }
  *out = r;
  TCKS_API_END
}

tcks_status tcks_vecmat_plain_batch(const tcks_ct* const* in, uint32_t count, const tcks_matrix* M, tcks_ct** outs) {
  std::vector<tcks_ct*> made;
  TCKS_API_BEGIN
  if (!M || !outs || (count && !in)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  for (u32 i = 0; i < count; ++i) outs[i] = nullptr;
  if (!count) return TCKS_OK;
  tcks_ctx* c = M->ctx;
  const u32 ell = in[0] ? in[0]->level : 0;
  for (u32 i = 0; i < count; ++i) {
    if (!in[i] || in[i]->ctx != c) fail(TCKS_ERR_INVALID_ARG, "ciphertext missing or of another context");
    need_relinearized(in[i]);
    if (in[i]->level != ell) fail(TCKS_ERR_LEVEL_MISMATCH, "the batch must share one level");
    if (in[i]->scale != in[0]->scale) fail(TCKS_ERR_SCALE_MISMATCH, "the batch must share one scale");
  }
  if (M->level < ell) fail(TCKS_ERR_LEVEL_MISMATCH, "matrix encoded below the ciphertext level");
  if (ell < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "vecmat needs level >= 2");
  const u64 wi = ct_words(c, ell), wo = ct_words(c, ell - 1);
  DevBuf x(c, (size_t)count * wi), y(c, (size_t)count * wo);
  for (u32 i = 0; i < count; ++i)
    check_cuda(cudaMemcpyAsync(x.p + i * wi, in[i]->d, wi * 8, cudaMemcpyDeviceToDevice, c->stream), "gather");
  op_vecmat(c, x.p, wi, count, ell, M, y.p);
  const double scale = in[0]->scale * M->scale / (double)c->host.chain[ell - 1];
  try {
    for (u32 i = 0; i < count; ++i) {
      made.push_back(new_ct(c, ell - 1, scale));
      check_cuda(cudaMemcpyAsync(made.back()->d, y.p + i * wo, wo * 8, cudaMemcpyDeviceToDevice, c->stream), "scatter");
    }
  } catch (...) {
    for (tcks_ct* t : made) free_ct(t);
    throw;
  }
  for (u32 i = 0; i < count; ++i) outs[i] = made[i];
  TCKS_API_END
}

tcks_status tcks_im2col_encode(const double* img, uint32_t H, uint32_t W, uint32_t kh, uint32_t kw, uint32_t stride,
                               double* out_slots, size_t cap, uint32_t* n_windows) {
  TCKS_API_BEGIN
  if (!img || !out_slots || !n_windows) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (kh == 0 || kw == 0 || stride == 0 || kh > H || kw > W) fail(TCKS_ERR_INVALID_ARG, "bad kernel geometry");
  const u32 oh = (H - kh) / stride + 1, ow = (W - kw) / stride + 1;
  const u64 windows = (u64)oh * ow, taps = (u64)kh * kw;
  if (windows * taps > cap) fail(TCKS_ERR_INVALID_ARG, "output capacity too small for windows * taps");
  for (size_t i = 0; i < cap; ++i) out_slots[i] = 0.0;
  for (u32 r = 0; r < oh; ++r)
    for (u32 cc = 0; cc < ow; ++cc) {
      const u64 w = (u64)r * ow + cc;
      for (u64 t = 0; t < taps; ++t)
        out_slots[t * windows + w] = img[(size_t)(stride * r + t / kw) * W + (stride * cc + t % kw)];
    }
  *n_windows = (uint32_t)windows;
  TCKS_API_END
}

tcks_status tcks_conv2d_im2col_pt(const tcks_ct* a, const tcks_pt* kernel, uint32_t taps, uint32_t windows,
                                  tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !kernel || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  need_relinearized(a);
  tcks_ctx* c = a->ctx;
  if (kernel->ctx != c) fail(TCKS_ERR_INVALID_ARG, "kernel belongs to another context");
  if (kernel->level < a->level) fail(TCKS_ERR_LEVEL_MISMATCH, "kernel encoded below the ciphertext level");
  if (a->level < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "conv needs level >= 2");
  if (taps == 0 || windows == 0 || (u64)windows * taps > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "bad conv geometry");
  tcks_ct* r = new_ct(c, a->level - 1, a->scale * kernel->scale / (double)c->host.chain[a->level - 1]);
  try {
    op_conv(c, a->d, a->level, kernel->d, taps, windows, r->d);
  } catch (...) {
    free_ct(r);
    throw;
  }
  *out = r;
  TCKS_API_END
}

tcks_status tcks_conv2d_im2col(const tcks_ct* a, const double* kernel, uint32_t taps, uint32_t windows,
                               tcks_ct** out) {
  TCKS_API_BEGIN
  if (!a || !kernel || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  need_relinearized(a);
  tcks_ctx* c = a->ctx;
  const u32 slots = c->N / 2;
  if (taps == 0 || windows == 0 || (u64)windows * taps > slots) fail(TCKS_ERR_INVALID_ARG, "bad conv geometry");
  std::vector<double> lay(slots, 0.0);
  for (u32 t = 0; t < taps; ++t)
    for (u32 w = 0; w < windows; ++w) lay[(size_t)t * windows + w] = kernel[t];
  tcks_pt* p = nullptr;
  tcks_status s = tcks_encode(c, lay.data(), slots, 0.0, a->level, &p);
  if (s != TCKS_OK) return s;
  s = tcks_conv2d_im2col_pt(a, p, taps, windows, out);
  tcks_pt_free(p);
  if (s != TCKS_OK) return s;
  TCKS_API_END
}

}  // extern "C"

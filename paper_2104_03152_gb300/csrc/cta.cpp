// Ciphertext arrays: the storage of TenSEAL's CKKSTensor (§2.3: an N-dimensional tensor of real values
// encrypted as a tensor of ciphertexts, optionally with one axis batched into the slots). All of a
// tensor's ciphertexts live in one device allocation, so that its element-wise operations, its
// products and its reductions are single batched launches; the tensor's shape, broadcasting and axis
// bookkeeping are host logic above this layer.
#include <cmath>
#include <cstring>
#include <vector>

#include "context.h"

using namespace tcks;

namespace {

#define CTA_BEGIN \
  try {           \
    tcks::NvtxRange tcks_nvtx_range_(__func__); \
    tcks::drop_stale_cuda_error();
#define CTA_END                                                                  \
  }                                                                              \
  catch (const tcks::Error& e) {                                                 \
    return tcks::abi_record(e.code, e.msg);                                      \
  }                                                                              \
  catch (const std::bad_alloc&) {                                                \
    return tcks::abi_record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed");   \
  }                                                                              \
  tcks::abi_clear();                                                             \
  return TCKS_OK;

u64 cta_words(const tcks_ctx* c, u32 count, u32 level) { return (u64)count * ct_words(c, level); }

tcks_cta* new_cta(tcks_ctx* c, u32 count, u32 level, double scale) {
  DevBuf b(c, cta_words(c, count, level));
  tcks_cta* a = new tcks_cta{c, b.release(), count, level, scale};
  ctx_retain(c);
  return a;
}

struct CtaOut {  // an array under construction, freed unless handed to the caller
  tcks_cta* a = nullptr;
  ~CtaOut() {
    if (a) tcks_cta_free(a);
  }
  tcks_cta* release() {
    tcks_cta* r = a;
    a = nullptr;
    return r;
  }
};

void check_cta(const tcks_cta* a) {
  if (!a) fail(TCKS_ERR_INVALID_ARG, "null ciphertext array");
}

u64 residue(int64_t v, u64 q) {
  if (v >= 0) return (u64)v % q;
  const u64 r = (u64)(-v) % q;
  return r ? q - r : 0;
}

// In-place rescale of an array (level - 1, scale / q_last).
void cta_rescale(tcks_cta* a) {
  tcks_ctx* c = a->ctx;
  if (a->level < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "rescale needs level >= 2");
  DevBuf nb(c, cta_words(c, a->count, a->level - 1));
  op_rescale(c, a->d, a->level, nb.p, a->count);
  check_launch("array rescale");
  c->dev_free(a->d);
  a->d = nb.release();
  a->scale = a->scale / (double)c->host.chain[a->level - 1];
  a->level -= 1;
}

}  // namespace

extern "C" {

void tcks_cta_free(tcks_cta* a) {
  if (!a) return;
  tcks_ctx* c = a->ctx;
  c->dev_free(a->d);
  delete a;
  ctx_release(c);
}

tcks_status tcks_cta_info(const tcks_cta* a, uint32_t* count, uint32_t* level, double* scale) {
  CTA_BEGIN
  check_cta(a);
  if (count) *count = a->count;
  if (level) *level = a->level;
  if (scale) *scale = a->scale;
  CTA_END
}

tcks_status tcks_cta_import(tcks_ctx* c, const uint64_t* limbs, uint32_t count, uint32_t level, double scale,
                            tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  if (!c || !out || (count && !limbs)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!count) fail(TCKS_ERR_INVALID_ARG, "empty array");
  if (level < 1 || level > c->L) fail(TCKS_ERR_INVALID_ARG, "level out of range");
  r.a = new_cta(c, count, level, scale);
  check_cuda(cudaMemcpyAsync(r.a->d, limbs, cta_words(c, count, level) * 8, cudaMemcpyHostToDevice, c->stream),
             "array import");
  check_cuda(cudaStreamSynchronize(c->stream), "array import");
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_export(const tcks_cta* a, uint64_t* limbs, size_t n_words) {
  CTA_BEGIN
  check_cta(a);
  if (!limbs) fail(TCKS_ERR_INVALID_ARG, "null argument");
  tcks_ctx* c = a->ctx;
  if (n_words != cta_words(c, a->count, a->level)) fail(TCKS_ERR_INVALID_ARG, "n_words != count * 2 * level * N");
  check_cuda(cudaMemcpyAsync(limbs, a->d, n_words * 8, cudaMemcpyDeviceToHost, c->stream), "array export");
  check_cuda(cudaStreamSynchronize(c->stream), "array export");
  CTA_END
}

tcks_status tcks_cta_from_cts(const tcks_ct* const* cts, uint32_t count, tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  if (!out || !cts || !count) fail(TCKS_ERR_INVALID_ARG, "null argument or empty array");
  *out = nullptr;
  if (!cts[0]) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
  tcks_ctx* c = cts[0]->ctx;
  for (u32 i = 0; i < count; ++i) {
    if (!cts[i] || cts[i]->ctx != c) fail(TCKS_ERR_INVALID_ARG, "ciphertext missing or of another context");
    need_relinearized(cts[i]);
    if (cts[i]->level != cts[0]->level) fail(TCKS_ERR_LEVEL_MISMATCH, "ciphertexts at different levels");
    if (cts[i]->scale != cts[0]->scale) fail(TCKS_ERR_SCALE_MISMATCH, "ciphertexts at different scales");
  }
  r.a = new_cta(c, count, cts[0]->level, cts[0]->scale);
  const u64 w = ct_words(c, r.a->level);
  for (u32 i = 0; i < count; ++i)
    check_cuda(cudaMemcpyAsync(r.a->d + i * w, cts[i]->d, w * 8, cudaMemcpyDeviceToDevice, c->stream), "gather");
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_get(const tcks_cta* a, uint32_t i, tcks_ct** out) {
  CTA_BEGIN
  check_cta(a);
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (i >= a->count) fail(TCKS_ERR_INVALID_ARG, "index out of range");
  tcks_ctx* c = a->ctx;
  tcks_ct* ct = new_ct(c, a->level, a->scale);
  const u64 w = ct_words(c, a->level);
  const cudaError_t e = cudaMemcpyAsync(ct->d, a->d + i * w, w * 8, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) {
    free_ct(ct);
    check_cuda(e, "array get");
  }
  *out = ct;
  CTA_END
}

tcks_status tcks_cta_encrypt(tcks_ctx* c, const double* values, uint32_t count, uint32_t n, uint32_t level,
                             uint64_t seed, tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  if (!c || !out || (count && n && !values)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!count) fail(TCKS_ERR_INVALID_ARG, "empty array");
  if (n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "more values than slots");
  const u32 l = level == 0 ? c->L : level;
  if (l > c->L) fail(TCKS_ERR_INVALID_ARG, "level exceeds L");
  const double sc = c->params.scale;
  r.a = new_cta(c, count, l, sc);
  DevBuf dv(c, (size_t)count * n + 1), pt(c, pt_words(c, l));
  if (n)
    check_cuda(cudaMemcpyAsync(dv.p, values, (size_t)count * n * 8, cudaMemcpyHostToDevice, c->stream), "values");
  const u64 w = ct_words(c, l);
  for (u32 i = 0; i < count; ++i) {
    encode_into(c, (const double*)dv.p + (size_t)i * n, n, sc, l, pt.p);
    launch_encrypt(c->T, seed + i, c->pk, pt.p, l, r.a->d + i * w, c->stream);
    check_launch("array encrypt");
  }
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_decrypt(const tcks_cta* a, double* values, uint32_t n) {
  CTA_BEGIN
  check_cta(a);
  tcks_ctx* c = a->ctx;
  if (n && !values) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "more values than slots");
  if (c->params.log_n > 14) fail(TCKS_ERR_UNSUPPORTED, "decoding is implemented for N <= 2^14");
  const size_t N = c->N;
  const u32 l = a->level;
  DevBuf pt(c, (size_t)l * N), coef(c, (size_t)l * N), p(c, N), z(c, (size_t)a->count * n + 1);
  for (u32 i = 0; i < a->count; ++i) {
    launch_decrypt(c->T, a->d + i * ct_words(c, l), c->sk, pt.p, l, c->stream);
    launch_ntt(c->T, true, pt.p, 0, coef.p, 0, l, 0, l, c->stream);
    launch_crt_compose(c->T, coef.p, l, c->d_qwords, (double*)p.p, c->stream);
    launch_decode_slots(c->T, c->F, (const double*)p.p, a->scale, n, (double*)z.p + (size_t)i * n, c->stream);
    check_launch("array decrypt");
  }
  if (n)
    check_cuda(cudaMemcpyAsync(values, z.p, (size_t)a->count * n * 8, cudaMemcpyDeviceToHost, c->stream),
               "decrypt D2H");
  check_cuda(cudaStreamSynchronize(c->stream), "array decrypt");
  CTA_END
}

tcks_status tcks_cta_binary(uint32_t op, const tcks_cta* a, const tcks_cta* b, tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  check_cta(a);
  check_cta(b);
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (op > TCKS_CTA_MUL) fail(TCKS_ERR_INVALID_ARG, "unknown operation");
  tcks_ctx* c = a->ctx;
  if (b->ctx != c) fail(TCKS_ERR_INVALID_ARG, "arrays of different contexts");
  if (a->count != b->count) fail(TCKS_ERR_INVALID_ARG, "arrays of different lengths");
  if (a->level != b->level) fail(TCKS_ERR_LEVEL_MISMATCH, "arrays at different levels");
  const u32 l = a->level;
  if (op != TCKS_CTA_MUL) {
    if (a->scale != b->scale) fail(TCKS_ERR_SCALE_MISMATCH, "arrays at different scales");
    r.a = new_cta(c, a->count, l, a->scale);
    launch_elementwise(c->T, op == TCKS_CTA_ADD ? OP_ADD : OP_SUB, a->d, b->d, r.a->d, l, 2 * a->count, c->stream);
    check_launch("array add / sub");
  } else {
    if (!(c->flags & TCKS_AUTO_RELIN))
      fail(TCKS_ERR_UNSUPPORTED, "enc x enc without automatic relinearization has no 2-component result");
    const bool rescale = (c->flags & TCKS_AUTO_RESCALE) != 0;
    if (rescale && l < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "multiply with auto-rescale needs level >= 2");
    DevBuf d3(c, (size_t)3 * l * c->N * a->count);
    launch_tensor(c->T, a->d, b->d, d3.p, l, a->count, c->stream);
    check_launch("array tensor");
    r.a = new_cta(c, a->count, l, a->scale * b->scale);
    op_relinearize(c, d3.p, l, r.a->d, a->count);
    if (rescale) cta_rescale(r.a);
  }
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_negate(const tcks_cta* a, tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  check_cta(a);
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tcks_ctx* c = a->ctx;
  r.a = new_cta(c, a->count, a->level, a->scale);
  launch_elementwise(c->T, OP_NEG, a->d, nullptr, r.a->d, a->level, 2 * a->count, c->stream);
  check_launch("array negate");
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_plain(uint32_t op, const tcks_cta* a, const double* values, uint32_t n, tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  check_cta(a);
  if (!out || (n && !values)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (op > TCKS_CTA_MUL) fail(TCKS_ERR_INVALID_ARG, "unknown operation");
  tcks_ctx* c = a->ctx;
  if (n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "more values than slots");
  const u32 l = a->level;
  const bool mul = op == TCKS_CTA_MUL;
  const bool rescale = mul && (c->flags & TCKS_AUTO_RESCALE) != 0;
  if (rescale && l < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "multiply with auto-rescale needs level >= 2");
  const double ps = mul ? c->params.scale : a->scale;
  DevBuf dv(c, (size_t)a->count * n + 1), pts(c, (size_t)a->count * pt_words(c, l));
  if (n)
    check_cuda(cudaMemcpyAsync(dv.p, values, (size_t)a->count * n * 8, cudaMemcpyHostToDevice, c->stream), "values");
  for (u32 i = 0; i < a->count; ++i)
    encode_into(c, (const double*)dv.p + (size_t)i * n, n, ps, l, pts.p + i * pt_words(c, l));
  r.a = new_cta(c, a->count, l, mul ? a->scale * ps : a->scale);
  const u32 ew = op == TCKS_CTA_ADD ? OP_ADD_PLAIN : op == TCKS_CTA_SUB ? OP_SUB_PLAIN : OP_MUL_PLAIN;
  launch_elementwise(c->T, ew, a->d, pts.p, r.a->d, l, 2 * a->count, c->stream, pt_words(c, l));
  check_launch("array plain op");
  if (rescale) cta_rescale(r.a);
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_combine(const tcks_cta* a, const uint32_t* idx, const double* w, uint32_t outputs,
                             uint32_t terms, int32_t mode, tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  check_cta(a);
  if (!out || !idx || !w) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (!outputs || !terms) fail(TCKS_ERR_INVALID_ARG, "empty combination");
  if (mode != 0 && mode != 1) fail(TCKS_ERR_INVALID_ARG, "mode must be 0 (integers) or 1 (reals at the scale)");
  tcks_ctx* c = a->ctx;
  const u32 l = a->level;
  const bool rescale = mode == 1 && (c->flags & TCKS_AUTO_RESCALE) != 0;
  if (rescale && l < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "multiply with auto-rescale needs level >= 2");
  const u64 nt = (u64)outputs * terms;
  std::vector<u64> coef(nt * l);
  const double S = c->params.scale;
  for (u64 t = 0; t < nt; ++t) {
    if (idx[t] >= a->count) fail(TCKS_ERR_INVALID_ARG, "index out of range");
    int64_t v;
    if (mode == 0) {
      if (!(std::fabs(w[t]) < 9007199254740992.0) || w[t] != std::floor(w[t]))
        fail(TCKS_ERR_INVALID_ARG, "mode 0 takes integer weights below 2^53");
      v = (int64_t)w[t];
    } else {
      const double x = w[t] * S;
      if (!(std::fabs(x) < 4611686018427387904.0)) fail(TCKS_ERR_VALUE_OVERFLOW, "|w * scale| >= 2^62");
      v = (int64_t)std::nearbyint(x);
    }
    for (u32 j = 0; j < l; ++j) coef[t * l + j] = residue(v, c->host.chain[j]);
  }
  DevBuf didx(c, (nt + 1) / 2), dcoef(c, coef.size());
  check_cuda(cudaMemcpyAsync(didx.p, idx, nt * 4, cudaMemcpyHostToDevice, c->stream), "indices");
  check_cuda(cudaMemcpyAsync(dcoef.p, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice, c->stream), "weights");
  r.a = new_cta(c, outputs, l, mode == 1 ? a->scale * S : a->scale);
  launch_combine(c->T, a->d, l, (const u32*)didx.p, dcoef.p, outputs, terms, r.a->d, c->stream);
  check_launch("array combine");
  if (rescale) cta_rescale(r.a);
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_sum_slots(const tcks_cta* a, uint32_t n, tcks_cta** out) {
  CtaOut r;
  CTA_BEGIN
  check_cta(a);
  if (!out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tcks_ctx* c = a->ctx;
  if (n < 1 || n > c->N / 2) fail(TCKS_ERR_INVALID_ARG, "n must be in [1, N/2]");
  std::vector<u32> steps;
  for (u32 s = 1; s < n; s <<= 1) steps.push_back(s);
  for (u32 s : steps) galois_key_for(c, s, a->level);  // fails with NO_GALOIS_KEY before any launch
  r.a = new_cta(c, a->count, a->level, a->scale);
  check_cuda(cudaMemcpyAsync(r.a->d, a->d, cta_words(c, a->count, a->level) * 8, cudaMemcpyDeviceToDevice, c->stream),
             "array copy");
  for (u32 s : steps) op_rotate_add(c, r.a->d, ct_words(c, a->level), a->count, a->level, (int32_t)s);
  *out = r.release();
  CTA_END
}

tcks_status tcks_cta_rescale(tcks_cta* a) {
  CTA_BEGIN
  check_cta(a);
  cta_rescale(a);
  CTA_END
}

tcks_status tcks_cta_mod_switch(tcks_cta* a, uint32_t level) {
  CTA_BEGIN
  check_cta(a);
  if (level < 1 || level > a->level) fail(TCKS_ERR_INVALID_ARG, "target level out of range");
  if (level == a->level) return TCKS_OK;
  tcks_ctx* c = a->ctx;
  DevBuf nb(c, cta_words(c, a->count, level));
  const size_t n = c->N;
  check_cuda(cudaMemcpy2DAsync(nb.p, (size_t)level * n * 8, a->d, (size_t)a->level * n * 8, (size_t)level * n * 8,
                               (size_t)2 * a->count, cudaMemcpyDeviceToDevice, c->stream),
             "array mod switch");
  c->dev_free(a->d);
  a->d = nb.release();
  a->level = level;
  CTA_END
}

}  // extern "C"

// Composite operations of TenSEAL's CKKSVector (§3.1 dot product / vector x plain matrix, §3.2
// im2col convolution) as schedules of the library's kernels.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

using namespace tcks;

namespace tcks {

static int ceil_log2(u64 x) {
  int r = 0;
  while ((1ull << r) < x) ++r;
  return r;
}

void op_sum(tcks_ctx* c, u64* ct, u32 ell) {
  for (u32 m = 0; m + 1 < c->params.log_n; ++m) op_rotate_add(c, ct, 0, 1, ell, (int32_t)(1u << m));
}

// y = v M by the diagonal method with a replicated input, for `count` ciphertexts at once:
//   replicate (rotate-and-add by N/2 - rows*2^i), ModUp of c1 once per ciphertext, then for every
//   rotation step k = 1..rows-1 the P-limb stage of the key switch (k_ks_inner_p) and the fused
//   ModDown + multiply-accumulate with the diagonal d_k (k_vecmat_acc), the k = 0 term and the
//   partial sums folded by k_vecmat_reduce, and the rescale. Rotations are processed in blocks so
//   that the P-limb scratch stays bounded (~512 MB).
// The same product with the ModDown taken once after the sum over rotations (double hoisting):
// replicate, ModUp once per ciphertext, one element-wise pass over all rotations accumulating the
// key-switch inner products times the extended-basis diagonals (k_vecmat_dh_acc), the fold of its
// chunk partials, INTT of the P limbs, one ModDown per (request, component, prime) with the k = 0
// term and tau(c0) part added (k_vecmat_dh_moddown), and the rescale. No transform runs per rotation.
static void op_vecmat_dh(tcks_ctx* c, const u64* ct, u64 cw, u32 count, u32 ell, const tcks_matrix* M, const KeyTable* kt,
                         u64* out) {
  const size_t n = c->N;
  const u32 R = M->diags - 1;
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * ell * (ell + 1) * n);
  launch_modup(c->T, ct + (size_t)ell * n, cw, count, ell, coef.p, digits.p, c->stream);
  VecmatDhPlan p{};
  p.keys = kt->d;
  p.keys_aligned = kt->aligned16;
  p.keys_K = kt->min_K == kt->max_K ? kt->min_K : 0;
  p.keys32 = kt->keys32;
  p.digits = digits.p;
  p.digits_b = (u64)ell * (ell + 1) * n;
  p.ct = ct;
  p.ct_b = cw;
  p.diag = M->d;
  p.diag_stride = (u64)M->limbs() * n;
  p.p_limb = M->level;
  p.R = R;
  p.B = count;
  // chunks of rotations: enough CTAs for a few waves of 256-thread CTAs on every SM
  const u64 base = vecmat_dh_base_ctas(c->T, ell, p), want = 152ull * 8 * 4;
  u32 chunks = (u32)std::min<u64>(R, std::max<u64>(1, (want + base - 1) / base));
  const u32 chunk = (R + chunks - 1) / chunks;
  chunks = (R + chunk - 1) / chunk;
  DevBuf partial(c, (size_t)count * chunks * 3 * (ell + 1) * n);
  p.partial = partial.p;
  p.chunk = chunk;
  p.chunks = chunks;
  launch_vecmat_dh_acc(c->T, ell, p, c->stream);
  launch_vecmat_dh_fold(c->T, ell, p, c->stream);
  DevBuf top(c, (size_t)2 * count * n);
  const u64 per_rq = (u64)chunks * 3 * (ell + 1) * n;
  // the P limb of both components, one launch
  launch_ntt(c->T, true, partial.p + (u64)ell * n, per_rq, top.p, n, count, c->L, 1, c->stream, 2, (u64)(ell + 1) * n,
             (u64)count * n);
  if (c->flags & TCKS_MERGED_RESCALE) {  // ModDown and rescale in one rounding
    DevBuf top2(c, (size_t)2 * count * n);
    launch_vecmat_dh_moddown_rs(c->T, c->host, ell, p, top.p, top2.p, out, ct_words(c, ell - 1), c->stream);
  } else {
    DevBuf acc(c, (size_t)count * cw);
    launch_vecmat_dh_moddown(c->T, ell, p, top.p, acc.p, cw, c->stream);
    op_rescale(c, acc.p, ell, out, count);
  }
  check_launch("vecmat (double hoisted)");
}

static void vecmat_single_hoisted(tcks_ctx* c, const u64* ct, u64 cw, u32 count, u32 ell, const tcks_matrix* M,
                                  const KeyTable* kt, u64* out);

// x + sum over `steps` of rot(x, s) for `count` ciphertexts [count][2][ell][N] (stride cw), with one
// ModUp and one ModDown per ciphertext: the double-hoisted accumulation with unit diagonals. out may
// alias x. The scale is unchanged.
void op_rotsum_hoisted(tcks_ctx* c, u64* x, u64 cw, u32 count, u32 ell, const std::vector<int32_t>& steps, u64* out,
                       const u64* bias) {
  need_one_prime_ks(c, "the hoisted rotation sum");
  const size_t n = c->N;
  std::vector<u32> ks;
  for (int32_t s : steps) {
    const u32 k = step_mod(c, s);
    if (!k) fail(TCKS_ERR_INVALID_ARG, "a rotation sum step of 0 (the identity is always included)");
    ks.push_back(k);
  }
  if (ks.empty()) {
    if (out != x)
      for (u32 i = 0; i < count; ++i)
        check_cuda(cudaMemcpyAsync(out + i * cw, x + i * cw, ct_words(c, ell) * 8, cudaMemcpyDeviceToDevice, c->stream),
                   "copy");
    if (bias)
      for (u32 i = 0; i < count; ++i)
        launch_elementwise(c->T, OP_ADD_PLAIN, out + i * cw, bias, out + i * cw, ell, 2, c->stream);
    return;
  }
  const KeyTable& kt = key_table(c, ks, ell);
  const u32 R = (u32)ks.size();
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * ell * (ell + 1) * n);
  launch_modup(c->T, x + (size_t)ell * n, cw, count, ell, coef.p, digits.p, c->stream);
  VecmatDhPlan p{};
  p.keys = kt.d;
  p.keys_aligned = kt.aligned16;
  p.keys_K = kt.min_K == kt.max_K ? kt.min_K : 0;
  p.keys32 = kt.keys32;
  p.digits = digits.p;
  p.digits_b = (u64)ell * (ell + 1) * n;
  p.ct = x;
  p.ct_b = cw;
  p.diag = nullptr;  // unit diagonals
  p.addp = bias;
  p.R = R;
  p.B = count;
  // chunks of rotations: enough CTAs for a few waves of 256-thread CTAs on every SM
  const u64 base = vecmat_dh_base_ctas(c->T, ell, p), want = 152ull * 8 * 4;
  u32 chunks = (u32)std::min<u64>(R, std::max<u64>(1, (want + base - 1) / base));
  const u32 chunk = (R + chunks - 1) / chunks;
  chunks = (R + chunk - 1) / chunk;
  DevBuf partial(c, (size_t)count * chunks * 3 * (ell + 1) * n);
  p.partial = partial.p;
  p.chunk = chunk;
  p.chunks = chunks;
  launch_vecmat_dh_acc(c->T, ell, p, c->stream);
  launch_vecmat_dh_fold(c->T, ell, p, c->stream);
  DevBuf top(c, (size_t)2 * count * n);
  const u64 per_rq = (u64)chunks * 3 * (ell + 1) * n;
  // the P limb of both components, one launch
  launch_ntt(c->T, true, partial.p + (u64)ell * n, per_rq, top.p, n, count, c->L, 1, c->stream, 2, (u64)(ell + 1) * n,
             (u64)count * n);
  launch_vecmat_dh_moddown(c->T, ell, p, top.p, out, cw, c->stream);
  check_launch("hoisted rotation sum");
}

void op_dh_sum_multi(tcks_ctx* c, const u64* x, u64 cw, u32 count, u32 ell, const std::vector<int32_t>& steps,
                     const u64* diags, u64 diag_stride, u64 set_stride, u32 p_limb, u32 outs, u64* out, u64 out_b,
                     u64 out_o, bool merged, u32 keep) {
  need_one_prime_ks(c, "the double-hoisted rotation sum");
  if (keep && (!merged || keep > ell - 1)) fail(TCKS_ERR_INVALID_ARG, "keep: a merged rescale to at most ell - 1 limbs");
  const size_t n = c->N;
  std::vector<u32> ks;
  for (int32_t st : steps) {
    const u32 k = step_mod(c, st);
    if (!k) fail(TCKS_ERR_INVALID_ARG, "a double-hoisted sum takes non-zero steps");
    ks.push_back(k);
  }
  const KeyTable& kt = key_table(c, ks, ell);
  const u32 R = (u32)ks.size();
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * ell * (ell + 1) * n);
  launch_modup(c->T, x + (size_t)ell * n, cw, count, ell, coef.p, digits.p, c->stream);
  VecmatDhPlan p{};
  p.keys = kt.d;
  p.keys_aligned = kt.aligned16;
  p.keys_K = kt.min_K == kt.max_K ? kt.min_K : 0;
  p.keys32 = kt.keys32;
  p.digits = digits.p;
  p.digits_b = (u64)ell * (ell + 1) * n;
  p.ct = x;
  p.ct_b = cw;
  p.diag = diags;
  p.diag_stride = diag_stride;
  p.diag_set = set_stride;
  p.p_limb = p_limb;
  p.outs = outs;
  p.keep = keep;
  p.R = R;
  p.B = count;
  // chunks of rotations: enough CTAs for a few waves of 256-thread CTAs on every SM
  const u64 base = vecmat_dh_base_ctas(c->T, ell, p), want = 152ull * 8 * 4;
  u32 chunks = (u32)std::min<u64>(R, std::max<u64>(1, (want + base - 1) / base));
  const u32 chunk = (R + chunks - 1) / chunks;
  chunks = (R + chunk - 1) / chunk;
  DevBuf partial(c, (size_t)count * outs * chunks * 3 * (ell + 1) * n);
  p.partial = partial.p;
  p.chunk = chunk;
  p.chunks = chunks;
  launch_vecmat_dh_acc(c->T, ell, p, c->stream);
  launch_vecmat_dh_fold(c->T, ell, p, c->stream);
  const u32 ro = count * outs;
  DevBuf top(c, (size_t)2 * ro * n);
  const u64 per_ro = (u64)chunks * 3 * (ell + 1) * n;
  launch_ntt(c->T, true, partial.p + (u64)ell * n, per_ro, top.p, n, ro, c->L, 1, c->stream, 2, (u64)(ell + 1) * n,
             (u64)ro * n);
  if (merged) {
    DevBuf top2(c, (size_t)2 * ro * n);
    launch_vecmat_dh_moddown_rs(c->T, c->host, ell, p, top.p, top2.p, out, out_b, c->stream, outs > 1 ? out_o : 0);
  } else {
    launch_vecmat_dh_moddown(c->T, ell, p, top.p, out, out_b, c->stream, outs > 1 ? out_o : 0);
  }
  check_launch("double-hoisted sum");
}

void op_vecmat(tcks_ctx* c, const u64* ct_in, u64 ct_stride, u32 count, u32 ell, const tcks_matrix* M, u64* out,
               u32 input_period, const u64* bias) {
  need_one_prime_ks(c, "the vector x matrix product");
  const bool dh = (c->flags & TCKS_DOUBLE_HOIST) != 0;
  if (dh && !M->ext)
    fail(TCKS_ERR_UNSUPPORTED, "double-hoisted vector x matrix needs the diagonals modulo P (tcks_matrix_encode or "
                               "tcks_matrix_import_ext)");
  const u32 rows = M->rows, diags = M->diags;
  const u32 slots = c->N / 2;
  const u64 cw = ct_words(c, ell);
  std::vector<int32_t> rep;
  const u64 period = input_period ? input_period : slots;
  for (u32 m = 0; ((u64)rows << m) < period; ++m) rep.push_back((int32_t)(slots - (rows << m)));
  std::vector<u32> steps;
  for (u32 k = 1; k < diags; ++k) steps.push_back(k);
  // rectangular form: the rotate-and-add chain by diags * 2^j after the rescale
  std::vector<int32_t> chain;
  if (M->rect)
    for (u32 w = diags; w < rows; w <<= 1) chain.push_back((int32_t)w);
  for (int32_t s : rep) galois_key_for(c, s, ell);  // validate before launching anything
  for (int32_t s : chain) galois_key_for(c, s, ell - 1);
  const KeyTable* kt = steps.empty() ? nullptr : &key_table(c, steps, ell);
  const u64 out_w = ct_words(c, ell - 1);
  const u64 in_s = count > 1 ? ct_stride : cw;
  // The sums read x: the input itself when nothing replicates it and it is laid out as the sums need
  // (the input is read-only there), else its replica. The first rotate-and-add of the replication
  // reads the input and writes the replica.
  DevBuf ct;
  const u64* x = ct_in;
  const bool overlap = out < ct_in + (count - 1) * in_s + cw && ct_in < out + (count - 1) * out_w + out_w;
  if (!rep.empty() && in_s >= cw) {
    ct = DevBuf(c, (size_t)count * cw);
    op_rotate_add_to(c, ct_in, in_s, count, ell, rep[0], ct.p, cw);
    for (size_t k = 1; k < rep.size(); ++k) op_rotate_add(c, ct.p, cw, count, ell, rep[k]);
    x = ct.p;
  } else if (!rep.empty() || steps.empty() || overlap || in_s != cw) {
    ct = DevBuf(c, (size_t)count * cw);
    if (in_s == cw) {
      check_cuda(cudaMemcpyAsync(ct.p, ct_in, (size_t)count * cw * 8, cudaMemcpyDeviceToDevice, c->stream), "copy");
    } else {
      for (u32 i = 0; i < count; ++i)
        check_cuda(cudaMemcpyAsync(ct.p + i * cw, ct_in + i * in_s, cw * 8, cudaMemcpyDeviceToDevice, c->stream),
                   "copy");
    }
    for (int32_t s : rep) op_rotate_add(c, ct.p, cw, count, ell, s);
    x = ct.p;
  }
  if (steps.empty()) {
    DevBuf acc(c, (size_t)count * cw);
    launch_elementwise(c->T, OP_MUL_PLAIN, x, M->d, acc.p, ell, 2 * count, c->stream);
    op_rescale(c, acc.p, ell, out, count);
  } else if (dh) {
    op_vecmat_dh(c, x, cw, count, ell, M, kt, out);
  } else {
    vecmat_single_hoisted(c, x, cw, count, ell, M, kt, out);
  }
  // The rotate-and-add chain alternates between out and a scratch so that its last step writes out
  // (adding the bias in the same epilogue); an odd chain takes its first step in place.
  size_t k = 0;
  if (chain.size() % 2) op_rotate_add(c, out, out_w, count, ell - 1, chain[k++]);
  if (k < chain.size()) {
    DevBuf tmp(c, (size_t)count * out_w);
    for (; k < chain.size(); k += 2) {
      op_rotate_add_to(c, out, out_w, count, ell - 1, chain[k], tmp.p, out_w);
      op_rotate_add_to(c, tmp.p, out_w, count, ell - 1, chain[k + 1], out, out_w,
                       k + 2 == chain.size() ? bias : nullptr);
    }
  } else if (bias) {
    launch_elementwise(c->T, OP_ADD_PLAIN, out, bias, out, ell - 1, 2 * count, c->stream);
  }
  check_launch("vecmat");
}

// The sum over rotations with one ModDown per rotation: ModUp once per ciphertext, then per block of
// rotations the P-limb stage (k_ks_inner_p) and the fused ModDown + multiply-accumulate
// (k_vecmat_acc), then the k = 0 term and the chunk partials (k_vecmat_reduce), then the rescale.
static void vecmat_single_hoisted(tcks_ctx* c, const u64* ct, u64 cw, u32 count, u32 ell, const tcks_matrix* M,
                                  const KeyTable* kt, u64* out) {
  const size_t n = c->N;
  DevBuf acc(c, (size_t)count * cw);
  DevBuf coef(c, (size_t)count * ell * n), digits(c, (size_t)count * ell * (ell + 1) * n);
  launch_modup(c->T, ct + (size_t)ell * n, cw, count, ell, coef.p, digits.p, c->stream);
  const u32 R = M->diags - 1;
  const u64 per_rot = (u64)count * 2 * n;  // P-limb scratch words per rotation
  u32 RB = (u32)std::max<u64>(1, ((u64)64 << 20) / per_rot);  // 512 MB of scratch per block
  if (RB > R) RB = R;
  // chunks per block: the fewest that give at least two waves of CTAs (count * 2 ell * chunks) with a
  // full-enough last wave (>= 90% of the slots busy on average), up to 64 chunks
  const u64 gpu_slots = vecmat_slots(c->T), per_chunk = (u64)count * 2 * ell;
  u32 chunks_pb = 1;
  for (u32 k = 1; k <= std::min<u32>(RB, 64); ++k) {
    chunks_pb = k;
    const u64 ctas = per_chunk * k, waves = (ctas + gpu_slots - 1) / gpu_slots;
    if (ctas >= 2 * gpu_slots && (double)ctas / (double)(waves * gpu_slots) >= 0.9) break;
  }
  const u32 chunk = (RB + chunks_pb - 1) / chunks_pb;
  chunks_pb = (RB + chunk - 1) / chunk;
  DevBuf top(c, (size_t)per_rot * RB);
  // chunk partials per request, reused (accumulated) across the rotation blocks
  DevBuf partial(c, (size_t)count * chunks_pb * cw);
  const u64 diag_stride = (u64)M->limbs() * n;
  for (u32 rb0 = 0; rb0 < R; rb0 += RB) {
    const u32 rbn = std::min(RB, R - rb0);
    KsPlan p{};
    p.keys = kt->d + rb0;
    p.digits = digits.p;
    p.digits_b = (u64)ell * (ell + 1) * n;
    p.top = top.p;
    p.out = nullptr;
    p.R = rbn;
    p.B = count;
    launch_ks_inner_p(c->T, ell, p, c->stream);
    VecmatPlan v{};
    v.keys = kt->d + rb0;
    v.digits = digits.p;
    v.digits_b = (u64)ell * (ell + 1) * n;
    v.top = top.p;
    v.ct = ct;
    v.ct_b = cw;
    v.diag = M->d + (size_t)rb0 * diag_stride;
    v.diag_stride = diag_stride;
    v.R = rbn;
    v.B = count;
    v.chunk = chunk;
    v.chunks = chunks_pb;  // a short last block leaves its upper chunks empty (zero rotations)
    v.partial = partial.p;
    v.partial_b = (u64)chunks_pb * cw;
    v.accumulate = rb0 > 0;
    launch_vecmat_acc(c->T, ell, v, c->stream);
    check_launch("vecmat block");
  }
  VecmatPlan red{};
  red.ct = ct;
  red.ct_b = cw;
  red.diag = M->d;
  red.partial = partial.p;
  red.partial_b = (u64)chunks_pb * cw;
  red.B = count;
  red.chunks = chunks_pb;
  launch_vecmat_reduce(c->T, ell, red, acc.p, c->stream);
  op_rescale(c, acc.p, ell, out, count);
}

// One im2col convolution kernel (§3.2): rescale(ct * kernel), then rotate-and-add by windows*2^i.
void op_conv(tcks_ctx* c, const u64* ct, u32 ell, const u64* kernel_pt, u32 taps, u32 windows, u64* out) {
  const int steps = ceil_log2(taps);
  for (int m = 0; m < steps; ++m) galois_key_for(c, (int32_t)(windows << m), ell - 1);
  DevBuf prod(c, ct_words(c, ell));
  launch_elementwise(c->T, OP_MUL_PLAIN, ct, kernel_pt, prod.p, ell, 2, c->stream);
  op_rescale(c, prod.p, ell, out);
  for (int m = 0; m < steps; ++m) op_rotate_add(c, out, 0, 1, ell - 1, (int32_t)(windows << m));
}

}  // namespace tcks

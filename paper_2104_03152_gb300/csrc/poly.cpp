// Element-wise power and polynomial evaluation of CKKSVectors (§3: "power" with a circuit of minimum
// multiplicative depth, "polyval" with a minimal circuit), batched over ciphertexts that share a level
// and a scale.
//
// Powers: x^(2m) = (x^m)^2, and for i not a power of two x^i = x^(2^m) x^(i - 2^m) with 2^m the
// largest power of two below i, so x^i has depth ceil(log2 i); every product takes its operands to the
// lower of their levels (limbs dropped), then tensor product, relinearization and rescale.
// Polynomial: with l the lowest level among the needed powers, S the context scale and q = q_{l-1}
// the prime of the final rescale, term i is multiplied by the integer constant rint(a_i S q / s_i)
// (s_i its scale), so every product has the scale S q; one fused pass (k_lincomb) drops the limbs,
// multiplies, sums and adds rint(a_0 S) q, and one rescale gives the result at level l - 1 and scale S.
// Adding rint(a_0 S) q before the rescale is the same as adding rint(a_0 S) after it: the rescale
// subtracts the residue modulo q, which the added multiple of q does not change, then divides by q.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "context.h"

using namespace tcks;

namespace {

struct Prod {
  u32 i, a, b;  // x^i = x^a x^b
};

u32 top_pow2(u32 i) { return 1u << (31 - __builtin_clz(i)); }

u32 ceil_log2(u32 k) {
  u32 r = 0;
  while ((1u << r) < k) ++r;
  return r;
}

// The products of the minimum-depth circuit that yields x^k for every k in ks, in increasing i.
std::vector<Prod> power_products(const std::vector<u32>& ks) {
  u32 top = 1;
  for (u32 k : ks) top = k > top ? k : top;
  std::vector<char> need(top + 1, 0);
  std::vector<u32> todo(ks);
  while (!todo.empty()) {
    const u32 i = todo.back();
    todo.pop_back();
    if (i <= 1 || need[i]) continue;
    need[i] = 1;
    const u32 m = top_pow2(i);
    if (m == i) {
      todo.push_back(i / 2);
    } else {
      todo.push_back(m);
      todo.push_back(i - m);
    }
  }
  std::vector<Prod> out;
  for (u32 i = 2; i <= top; ++i) {
    if (!need[i]) continue;
    const u32 m = top_pow2(i);
    out.push_back(m == i ? Prod{i, i / 2, i / 2} : Prod{i, m, i - m});
  }
  return out;
}

// `count` ciphertexts [count][2][level][N] at one scale.
struct Batch {
  u64* d = nullptr;
  u32 level = 0;
  double scale = 0.0;
  bool owned = false;
};

struct PowerTable {
  tcks_ctx* c;
  std::map<u32, Batch> p;
  ~PowerTable() {
    for (auto& kv : p)
      if (kv.second.owned) c->dev_free(kv.second.d);
  }
};

u64 residue(int64_t v, u64 q) {
  if (v >= 0) return (u64)v % q;
  const u64 r = (u64)(-v) % q;
  return r ? q - r : 0;
}

// x^a x^b for a batch: both operands at the lower level, tensor product, relinearize, rescale.
Batch batch_mul(tcks_ctx* c, const Batch& A, const Batch& B, u32 count) {
  const u32 lvl = A.level < B.level ? A.level : B.level;
  if (lvl < 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "a product of the power circuit needs level >= 2");
  const size_t n = c->N;
  auto at_level = [&](const Batch& X, DevBuf& tmp) -> const u64* {
    if (X.level == lvl) return X.d;
    tmp = DevBuf(c, (size_t)count * 2 * lvl * n);
    check_cuda(cudaMemcpy2DAsync(tmp.p, (size_t)lvl * n * 8, X.d, (size_t)X.level * n * 8, (size_t)lvl * n * 8,
                                 (size_t)2 * count, cudaMemcpyDeviceToDevice, c->stream),
               "limb drop");
    return tmp.p;
  };
  DevBuf ta, tb;
  const u64* a = at_level(A, ta);
  const u64* b = A.d == B.d ? a : at_level(B, tb);
  DevBuf d3(c, (size_t)count * 3 * lvl * n), rel(c, (size_t)count * 2 * lvl * n);
  launch_tensor(c->T, a, b, d3.p, lvl, count, c->stream);
  check_launch("power: tensor");
  op_relinearize(c, d3.p, lvl, rel.p, count);
  DevBuf out(c, (size_t)count * 2 * (lvl - 1) * n);
  op_rescale(c, rel.p, lvl, out.p, count);
  check_launch("power: rescale");
  Batch r;
  r.level = lvl - 1;
  r.scale = (A.scale * B.scale) / (double)c->host.chain[lvl - 1];
  r.owned = true;
  r.d = out.release();
  return r;
}

void powers(tcks_ctx* c, PowerTable& t, const std::vector<u32>& ks, u32 count) {
  for (const Prod& pr : power_products(ks)) t.p[pr.i] = batch_mul(c, t.p.at(pr.a), t.p.at(pr.b), count);
}

// x^k for a batch (k >= 1); the result is owned.
Batch op_power(tcks_ctx* c, const Batch& x, u32 count, u32 k) {
  if (k < 1) fail(TCKS_ERR_INVALID_ARG, "power: k must be >= 1");
  if (x.level < ceil_log2(k) + 1) fail(TCKS_ERR_LEVEL_EXHAUSTED, "power: not enough levels for x^k");
  if (k == 1) {
    Batch r = x;
    DevBuf cp(c, (size_t)count * ct_words(c, x.level));
    check_cuda(cudaMemcpyAsync(cp.p, x.d, (size_t)count * ct_words(c, x.level) * 8, cudaMemcpyDeviceToDevice,
                               c->stream),
               "power: copy");
    r.d = cp.release();
    r.owned = true;
    return r;
  }
  PowerTable t{c, {}};
  t.p[1] = x;
  t.p[1].owned = false;
  powers(c, t, {k}, count);
  Batch r = t.p.at(k);
  t.p.at(k).owned = false;  // handed to the caller
  return r;
}

// sum_i a_i x^i for a batch; the result (level l - 1, scale S) is owned.
Batch op_polyval(tcks_ctx* c, const Batch& x, u32 count, std::vector<double> a) {
  while (!a.empty() && a.back() == 0.0) a.pop_back();
  std::vector<u32> ks;
  for (u32 i = 1; i < a.size(); ++i)
    if (a[i] != 0.0) ks.push_back(i);
  if (ks.empty()) fail(TCKS_ERR_INVALID_ARG, "polyval needs a non-zero coefficient of degree >= 1");
  const u32 depth = ceil_log2(ks.back());
  if (x.level < depth + 2) fail(TCKS_ERR_LEVEL_EXHAUSTED, "polyval: not enough levels for this degree");
  PowerTable t{c, {}};
  t.p[1] = x;
  t.p[1].owned = false;
  powers(c, t, ks, count);
  u32 lt = x.level;
  for (u32 k : ks) lt = t.p.at(k).level < lt ? t.p.at(k).level : lt;
  const double S = c->params.scale;
  const u64 qd = c->host.chain[lt - 1];
  const double q = (double)qd;
  const double lim = 4611686018427387904.0;  // 2^62
  std::vector<u64> coef((size_t)ks.size() * lt), cst(lt, 0);
  for (size_t ti = 0; ti < ks.size(); ++ti) {
    const double tt = S * q / t.p.at(ks[ti]).scale;
    const double v = a[ks[ti]] * tt;
    if (!(std::fabs(v) < lim)) fail(TCKS_ERR_VALUE_OVERFLOW, "polyval: |a_i * scale| >= 2^62");
    const int64_t ci = (int64_t)std::nearbyint(v);
    for (u32 j = 0; j < lt; ++j) coef[ti * lt + j] = residue(ci, c->host.chain[j]);
  }
  const bool has_cst = a[0] != 0.0;
  if (has_cst) {
    const double v = a[0] * S;
    if (!(std::fabs(v) < lim)) fail(TCKS_ERR_VALUE_OVERFLOW, "polyval: |a_0 * scale| >= 2^62");
    const int64_t c0 = (int64_t)std::nearbyint(v);
    for (u32 j = 0; j + 1 < lt; ++j) {
      const u64 qj = c->host.chain[j];
      cst[j] = (u64)(((unsigned __int128)residue(c0, qj) * (qd % qj)) % qj);
    }
  }
  const size_t n = c->N;
  DevBuf acc(c, (size_t)count * 2 * lt * n);
  for (size_t t0 = 0; t0 < ks.size(); t0 += kLincombMax) {
    LincombArgs A{};
    A.terms = (u32)std::min<size_t>(kLincombMax, ks.size() - t0);
    for (u32 i = 0; i < A.terms; ++i) {
      const Batch& T = t.p.at(ks[t0 + i]);
      A.x[i] = T.d;
      A.level[i] = T.level;
      for (u32 j = 0; j < lt; ++j) A.coef[i][j] = coef[(t0 + i) * lt + j];
    }
    A.has_cst = t0 == 0 && has_cst;
    for (u32 j = 0; j < lt; ++j) A.cst[j] = cst[j];
    A.prev = t0 == 0 ? nullptr : acc.p;
    A.ell = lt;
    A.count = count;
    launch_lincomb(c->T, A, acc.p, c->stream);
    check_launch("polyval: combination");
  }
  DevBuf res(c, (size_t)count * 2 * (lt - 1) * n);
  op_rescale(c, acc.p, lt, res.p, count);
  check_launch("polyval: rescale");
  Batch r;
  r.level = lt - 1;
  r.scale = S;
  r.owned = true;
  r.d = res.release();
  return r;
}

template <typename F>
tcks_status run_batch(const tcks_ct* const* x, u32 count, tcks_ct** outs, F&& fn) {
  struct Made {
    std::vector<tcks_ct*> v;
    ~Made() {
      for (tcks_ct* p : v) free_ct(p);
    }
  } owned;
  try {
    drop_stale_cuda_error();
    if (!outs || (count && !x)) fail(TCKS_ERR_INVALID_ARG, "null argument");
    for (u32 i = 0; i < count; ++i) outs[i] = nullptr;
    if (!count) {
      abi_clear();
      return TCKS_OK;
    }
    if (!x[0]) fail(TCKS_ERR_INVALID_ARG, "null ciphertext");
    tcks_ctx* c = x[0]->ctx;
    for (u32 i = 0; i < count; ++i) {
      if (!x[i] || x[i]->ctx != c) fail(TCKS_ERR_INVALID_ARG, "ciphertext missing or of another context");
      need_relinearized(x[i]);
      if (x[i]->level != x[0]->level) fail(TCKS_ERR_LEVEL_MISMATCH, "the batch's ciphertexts differ in level");
      if (x[i]->scale != x[0]->scale) fail(TCKS_ERR_SCALE_MISMATCH, "the batch's ciphertexts differ in scale");
    }
    const u64 w_in = ct_words(c, x[0]->level);
    DevBuf gathered;
    Batch in;
    in.level = x[0]->level;
    in.scale = x[0]->scale;
    if (count == 1) {
      in.d = x[0]->d;
    } else {
      gathered = DevBuf(c, (size_t)count * w_in);
      for (u32 i = 0; i < count; ++i)
        check_cuda(cudaMemcpyAsync(gathered.p + i * w_in, x[i]->d, w_in * 8, cudaMemcpyDeviceToDevice, c->stream),
                   "gather");
      in.d = gathered.p;
    }
    Batch r = fn(c, in);
    DevBuf rb;
    rb.ctx = c;
    rb.p = r.d;
    const u64 w_out = ct_words(c, r.level);
    if (count == 1) {
      tcks_ct* ct = new tcks_ct{c, rb.release(), r.level, r.scale};
      ctx_retain(c);
      owned.v.push_back(ct);
    } else {
      for (u32 i = 0; i < count; ++i) {
        owned.v.push_back(new_ct(c, r.level, r.scale));
        check_cuda(cudaMemcpyAsync(owned.v.back()->d, rb.p + i * w_out, w_out * 8, cudaMemcpyDeviceToDevice,
                                   c->stream),
                   "scatter");
      }
    }
    for (u32 i = 0; i < count; ++i) outs[i] = owned.v[i];
    owned.v.clear();
  } catch (const Error& e) {
    return abi_record(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return abi_record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed");
  }
  abi_clear();
  return TCKS_OK;
}

// The same on a ciphertext array (already one contiguous batch): the result becomes a new array.
template <typename F>
tcks_status run_cta(const tcks_cta* a, tcks_cta** out, F&& fn) {
  try {
    drop_stale_cuda_error();
    if (!a || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    tcks_ctx* c = a->ctx;
    Batch in;
    in.d = a->d;
    in.level = a->level;
    in.scale = a->scale;
    Batch r = fn(c, in);
    *out = new tcks_cta{c, r.d, a->count, r.level, r.scale};
    ctx_retain(c);
  } catch (const Error& e) {
    return abi_record(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return abi_record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed");
  }
  abi_clear();
  return TCKS_OK;
}

}  // namespace

extern "C" {

tcks_status tcks_power_batch(const tcks_ct* const* x, uint32_t count, uint32_t k, tcks_ct** outs) {
  return run_batch(x, count, outs, [&](tcks_ctx* c, const Batch& in) { return op_power(c, in, count, k); });
}

tcks_status tcks_power(const tcks_ct* x, uint32_t k, tcks_ct** out) { return tcks_power_batch(&x, 1, k, out); }

tcks_status tcks_polyval_batch(const tcks_ct* const* x, uint32_t count, const double* coeffs, uint32_t n_coeffs,
                               tcks_ct** outs) {
  if (!coeffs && n_coeffs) return abi_record(TCKS_ERR_INVALID_ARG, "null coefficients");
  std::vector<double> a(coeffs, coeffs + n_coeffs);
  return run_batch(x, count, outs, [&](tcks_ctx* c, const Batch& in) { return op_polyval(c, in, count, a); });
}

tcks_status tcks_polyval(const tcks_ct* x, const double* coeffs, uint32_t n_coeffs, tcks_ct** out) {
  return tcks_polyval_batch(&x, 1, coeffs, n_coeffs, out);
}

tcks_status tcks_cta_power(const tcks_cta* a, uint32_t k, tcks_cta** out) {
  return run_cta(a, out, [&](tcks_ctx* c, const Batch& in) { return op_power(c, in, a->count, k); });
}

tcks_status tcks_cta_polyval(const tcks_cta* a, const double* coeffs, uint32_t n_coeffs, tcks_cta** out) {
  if (!coeffs && n_coeffs) return abi_record(TCKS_ERR_INVALID_ARG, "null coefficients");
  std::vector<double> v(coeffs, coeffs + n_coeffs);
  return run_cta(a, out, [&](tcks_ctx* c, const Batch& in) { return op_polyval(c, in, a->count, v); });
}

}  // extern "C"

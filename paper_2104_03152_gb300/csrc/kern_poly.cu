// Linear combinations of ciphertexts with integer constants: the combination step of polynomial
// evaluation (§3, polyval), out = sum_t c_t x^(i_t) (+ prev) with the constant added to component 0,
// for `count` ciphertexts at once; and the gathered combination of an encrypted tensor's ciphertexts
// (gather, sum along an axis, product with a plain matrix), out[o] = sum_t c[o][t] x[idx[o][t]].
//
// Each term is a batch of ciphertexts [count][2][level_t][N] at a level >= ell; only its first ell
// limbs are read, which is the limb drop that brings it to level ell. c_t is an integer constant given
// by its residues c_t mod q_j; the products are accumulated exactly (64-bit with a carry count for
// 31-bit primes, 128-bit otherwise) and reduced once. Memory-bound: one pass over the terms' first
// ell limbs and one write.
#include <cuda_runtime.h>

#include "context.h"
#include "kernels.h"
#include "ntt.cuh"

namespace tcks {

namespace {

template <typename W>
__global__ void __launch_bounds__(256) k_lincomb(DevTables T, LincombArgs A, u64* __restrict__ out) {
  const u32 log_n = T.log_n, ell = A.ell;
  const u64 n = 1ull << log_n;
  const u64 per_ct = 2ull * ell * n;
  const u64 total2 = (per_ct * A.count) >> 1;
  for (u64 e2 = (u64)blockIdx.x * blockDim.x + threadIdx.x; e2 < total2; e2 += (u64)gridDim.x * blockDim.x) {
    const u64 e = e2 << 1;
    const u64 r = e / per_ct, o = e - r * per_ct;  // ciphertext, offset inside it
    const u64 row = o >> log_n;                    // component * ell + limb
    const u32 j = (u32)(row % ell), b = (u32)(row / ell);
    const u64 k = o & (n - 1);
    const ModConst m = T.mods[j];
    typename Ew<W>::Acc a0, a1;
    for (u32 t = 0; t < A.terms; ++t) {
      const u64 lt = A.level[t];
      const ulonglong2 x =
          *reinterpret_cast<const ulonglong2*>(A.x[t] + r * 2 * lt * n + ((u64)b * lt + j) * n + k);
      const u64 c = A.coef[t][j];
      a0.mac(x.x, c);
      a1.mac(x.y, c);
    }
    u64 v0 = a0.get(m), v1 = a1.get(m);
    if (A.prev) {
      const ulonglong2 p = *reinterpret_cast<const ulonglong2*>(A.prev + e);
      v0 = add_mod(v0, p.x, m.q);
      v1 = add_mod(v1, p.y, m.q);
    }
    if (b == 0 && A.has_cst) {
      v0 = add_mod(v0, A.cst[j], m.q);
      v1 = add_mod(v1, A.cst[j], m.q);
    }
    *reinterpret_cast<ulonglong2*>(out + e) = make_ulonglong2(v0, v1);
  }
}

// One thread per pair of coefficients of an output row (o, b, j); the terms' rows are read in the
// same coalesced order, the coefficient of a term is one broadcast load.
template <typename W>
__global__ void __launch_bounds__(256) k_combine(DevTables T, const u64* __restrict__ x, u32 level,
                                                 const u32* __restrict__ idx, const u64* __restrict__ coef,
                                                 u32 outputs, u32 terms, u64* __restrict__ out) {
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u64 per_ct = 2ull * level * n;
  const u64 total2 = (per_ct * outputs) >> 1;
  for (u64 e2 = (u64)blockIdx.x * blockDim.x + threadIdx.x; e2 < total2; e2 += (u64)gridDim.x * blockDim.x) {
    const u64 e = e2 << 1;
    const u64 o = e / per_ct, off = e - o * per_ct;  // output ciphertext, offset inside it
    const u32 j = (u32)((off >> log_n) % level);
    const ModConst m = T.mods[j];
    typename Ew<W>::Acc a0, a1;
    const u32* it = idx + o * terms;
    const u64* ct = coef + o * terms * level + j;
    for (u32 t = 0; t < terms; ++t) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(x + (u64)it[t] * per_ct + off);
      const u64 c = ct[(u64)t * level];
      a0.mac(v.x, c);
      a1.mac(v.y, c);
    }
    *reinterpret_cast<ulonglong2*>(out + e) = make_ulonglong2(a0.get(m), a1.get(m));
  }
}

// out[r] = sum_t x_t[r] * m_t (slot-wise products with a plaintext each, summed before one rounding)
// for `count` ciphertexts at level ell: x_t at x + t * x_stride ([count][2][ell][N]), m_t [>= ell][N].
template <typename W>
__global__ void __launch_bounds__(256) k_mulsum(DevTables T, MulSumArgs A, u64* __restrict__ out) {
  const u32 log_n = T.log_n, ell = A.ell;
  const u64 n = 1ull << log_n;
  const u64 total2 = ((2ull * ell * A.count) << log_n) >> 1;
  for (u64 e2 = (u64)blockIdx.x * blockDim.x + threadIdx.x; e2 < total2; e2 += (u64)gridDim.x * blockDim.x) {
    const u64 e = e2 << 1;
    const u32 j = (u32)((e >> log_n) % ell);
    const u64 k = e & (n - 1);
    const ModConst m = T.mods[j];
    typename Ew<W>::Acc a0, a1;
    for (u32 t = 0; t < A.terms; ++t) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(A.x + (u64)t * A.x_stride + e);
      const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(A.m[t] + (u64)j * n + k);
      a0.mac(v.x, w.x);
      a1.mac(v.y, w.y);
    }
    *reinterpret_cast<ulonglong2*>(out + e) = make_ulonglong2(a0.get(m), a1.get(m));
  }
}

}  // namespace

void launch_mulsum(const DevTables& T, const MulSumArgs& A, u64* out, cudaStream_t st) {
  const u64 per = (2ull * A.ell * A.count) << T.log_n;
  u64 blocks = (per / 2 + 255) / 256;
  const u64 cap = 152ull * 8;
  if (blocks > cap) blocks = cap;
  if (!blocks) blocks = 1;
  Launch L(K_ELEMENTWISE, st, 8.0 * per * (A.terms + 1) + 8.0 * A.terms * ((u64)A.ell << T.log_n),
           (double)per * A.terms);
  if (T.narrow)
    k_mulsum<u32><<<(u32)blocks, 256, 0, st>>>(T, A, out);
  else
    k_mulsum<u64><<<(u32)blocks, 256, 0, st>>>(T, A, out);
}

void launch_combine(const DevTables& T, const u64* x, u32 level, const u32* idx, const u64* coef, u32 outputs,
                    u32 terms, u64* out, cudaStream_t st) {
  const u64 per_ct = (2ull * level) << T.log_n;
  const u64 e2 = (per_ct * outputs) >> 1;
  u64 blocks = (e2 + 255) / 256;
  const u64 cap = 152ull * 8;
  if (blocks > cap) blocks = cap;
  if (!blocks) blocks = 1;
  Launch L(K_COMBINE, st, 8.0 * per_ct * outputs * (terms + 1), (double)per_ct * outputs * terms);
  if (T.narrow)
    k_combine<u32><<<(u32)blocks, 256, 0, st>>>(T, x, level, idx, coef, outputs, terms, out);
  else
    k_combine<u64><<<(u32)blocks, 256, 0, st>>>(T, x, level, idx, coef, outputs, terms, out);
}

void launch_lincomb(const DevTables& T, const LincombArgs& A, u64* out, cudaStream_t st) {
  const u64 per_ct = (2ull * A.ell) << T.log_n;
  const u64 e2 = (per_ct * A.count) >> 1;
  const double by = 8.0 * per_ct * A.count * (A.terms + 1 + (A.prev ? 1 : 0));
  const double ops = (double)per_ct * A.count * A.terms;
  u64 blocks = (e2 + 255) / 256;
  const u64 cap = 152ull * 8;
  if (blocks > cap) blocks = cap;
  if (!blocks) blocks = 1;
  Launch L(K_LINCOMB, st, by, ops);
  if (T.narrow)
    k_lincomb<u32><<<(u32)blocks, 256, 0, st>>>(T, A, out);
  else
    k_lincomb<u64><<<(u32)blocks, 256, 0, st>>>(T, A, out);
}

}  // namespace tcks

// Device-side modular arithmetic on u64 RNS limbs (moduli q < 2^62).
//
// Multiplication by a precomputed constant uses Shoup's method (w' = floor(w * 2^64 / q)); products
// of two variables use an exact Barrett reduction of the 128-bit product with mu = floor(2^128 / q);
// NTT butterflies follow Harvey's lazy-reduction bounds ([0, 4q) forward, [0, 2q) inverse), so
// q < 2^62 keeps every intermediate inside 64 bits. Every value written to global memory is
// canonical in [0, q).
#pragma once
#include <cstdint>

#include "tcks_types.h"

namespace tcks {

__device__ __forceinline__ u64 csub(u64 a, u64 q) { return a >= q ? a - q : a; }
__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }
__device__ __forceinline__ u64 neg_mod(u64 a, u64 q) { return a ? q - a : 0; }

// a * w mod q in [0, 2q) for any a < 2^64 (Shoup).
__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 w_sh, u64 q) {
  return a * w - __umul64hi(a, w_sh) * q;
}
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 w_sh, u64 q) { return csub(mul_shoup_lazy(a, w, w_sh, q), q); }

// (hi:lo) mod q for any 128-bit value. qhat = floor((hi:lo) * mu / 2^128) is computed exactly
// (modulo 2^64), and floor(x/q) - 1 <= qhat <= floor(x/q), so one conditional subtraction ends it.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const ModConst& m) {
  const u64 h0 = __umul64hi(lo, m.mu_lo);
  const u64 b_lo = hi * m.mu_lo, b_hi = __umul64hi(hi, m.mu_lo);
  const u64 c_lo = lo * m.mu_hi, c_hi = __umul64hi(lo, m.mu_hi);
  u64 s = h0 + b_lo;
  u64 carry = s < h0;
  const u64 s2 = s + c_lo;
  carry += s2 < s;
  const u64 qhat = hi * m.mu_hi + b_hi + c_hi + carry;
  return csub(lo - qhat * m.q, m.q);
}

__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const ModConst& m) { return reduce128(__umul64hi(a, b), a * b, m); }

// x mod q for x < 2^64 with mu64 = floor(2^64 / q).
__device__ __forceinline__ u64 reduce64(u64 x, const ModConst& m) { return csub(x - __umul64hi(x, m.mu64) * m.q, m.q); }

// 128-bit accumulator helpers.
struct Acc128 {
  u64 lo, hi;
};
__device__ __forceinline__ void mac128(Acc128& acc, u64 a, u64 b) {
  const u64 plo = a * b, phi = __umul64hi(a, b);
  const u64 lo = acc.lo + plo;
  acc.hi += phi + (lo < plo);
  acc.lo = lo;
}

// x mod q for x < 2^32 and q < 2^31 with mu32 = floor(2^32 / q): the quotient estimate is at most
// one short, so one conditional subtraction finishes.
__device__ __forceinline__ u32 reduce32(u32 x, const ModConst& m) {
  const u32 q = (u32)m.q;
  const u32 r = x - __umulhi(x, (u32)m.mu32) * q;
  return r >= q ? r - q : r;
}

// Lift a residue x in [0, q_src) to the balanced integer bal(x) taken modulo the target prime:
// bal(x) = x if x <= (q_src - 1)/2, else x - q_src. qsrc_mod_t = q_src mod q_t.
__device__ __forceinline__ u64 lift_balanced(u64 x, u64 half_src, u64 qsrc_mod_t, const ModConst& t) {
  const u64 r = reduce64(x, t);
  return x > half_src ? sub_mod(r, qsrc_mod_t, t.q) : r;
}
// The same for the word type of a limb kernel: with 32-bit words every prime is below 2^31, so the
// residue fits one word and the reduction is a 32-bit one.
template <typename W>
__device__ __forceinline__ W lift_balanced_w(u64 x, u64 half_src, u64 qsrc_mod_t, const ModConst& t) {
  if constexpr (sizeof(W) == 4) {
    const u32 r = reduce32((u32)x, t), c = (u32)qsrc_mod_t;
    return x > half_src ? (r >= c ? r - c : r + (u32)t.q - c) : r;
  } else {
    return lift_balanced(x, half_src, qsrc_mod_t, t);
  }
}

// The balanced integer x, |x| < P q_l / 2, with x = rp (mod P) and x = rl (mod q_l), reduced modulo
// the target prime t: Garner's x = rp + P ((rl - rp) P^-1 mod q_l), then P q_l subtracted above the
// half. With every prime below 2^31 (NARROW) P q_l < 2^62 and x fits one 64-bit word (two 32-bit
// reductions and one 64-bit one); otherwise 128-bit words.
template <bool NARROW>
__device__ __forceinline__ u64 crt2_lift(u64 rp, u64 rl, const Crt2& k, const ModConst& ml, const ModConst& t) {
  if constexpr (NARROW) {
    const u32 a = reduce32((u32)rp, ml), q = (u32)k.ql;
    const u32 d = (u32)rl >= a ? (u32)rl - a : (u32)rl + q - a;
    u32 u = d * (u32)k.pinv_l - __umulhi(d, k.pinv_sh32) * q;  // Shoup: d P^-1 mod q_l in [0, 2 q_l)
    u = u >= q ? u - q : u;
    const u64 x = rp + k.P * u;
    const bool neg = x > k.half_lo;
    const u64 r = reduce64(neg ? k.pq_lo - x : x, t);
    return neg ? (r ? t.q - r : 0) : r;
  }
  const u64 a = reduce64(rp, ml);
  const u64 d = rl >= a ? rl - a : rl + k.ql - a;
  const u64 u = mul_mod(d, k.pinv_l, ml);
  u64 lo = k.P * u, hi = __umul64hi(k.P, u);
  lo += rp;
  hi += lo < rp;
  const bool neg = hi > k.half_hi || (hi == k.half_hi && lo > k.half_lo);
  if (neg) {  // magnitude P q_l - x
    const u64 nlo = k.pq_lo - lo;
    hi = k.pq_hi - hi - (k.pq_lo < lo);
    lo = nlo;
  }
  const u64 r = reduce128(hi, lo, t);
  return neg ? (r ? t.q - r : 0) : r;
}

// Bit reverse of the low `bits` bits.
__device__ __forceinline__ u32 brv(u32 x, u32 bits) { return __brev(x) >> (32 - bits); }

// Source index of the NTT-domain Galois automorphism tau_g: out[k] = in[src(k)] with
// 2*brv(src)+1 == (2*brv(k)+1)*g (mod 2N). The product is taken modulo 2^32, which 2N divides.
__device__ __forceinline__ u32 galois_src(u32 k, u32 g, u32 log_n) {
  const u32 e = ((2u * brv(k, log_n) + 1u) * g) & ((2u << log_n) - 1u);
  return brv((e - 1u) >> 1, log_n);
}

}  // namespace tcks

// Accumulators of the double-hoisted vector x matrix product, shared by its per-thread and staged
// kernels (kern_vecmat.cu, kern_dh_bulk.cu).
#pragma once
#include "dev_arith.cuh"
#include "tcks_types.h"

namespace tcks {

// Lazy sum of products over the whole rotation loop: products of two residues are added without
// reduction and the sum is reduced once at the end. 32-bit words: a 128-bit sum of four 32-bit words
// fed through the carry flag; it also takes a key-switch sum unreduced (below 2^66) times a diagonal
// value, so the rotation loop has no reduction at all. 64-bit words: products < 2^122 in a 128-bit
// sum with a count of 2^128 carries.
template <typename W>
struct DhAcc;
template <>
struct DhAcc<u32> {
  u32 w0 = 0, w1 = 0, w2 = 0, w3 = 0;
  // += x y, x, y < 2^32 (below 2^34 such products the sum stays below 2^96: no carry into w3)
  __device__ __forceinline__ void mac(u64 x, u64 y) {
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(w0), "+r"(w1), "+r"(w2)
        : "r"((u32)x), "r"((u32)y));
  }
  __device__ __forceinline__ void add(u64 x) {
    asm("add.cc.u32 %0, %0, %2;\n\t"
        "addc.u32 %1, %1, 0;"
        : "+r"(w0), "+r"(w1)
        : "r"((u32)x));
  }
  // += (s + c 2^64) d, d < 2^32; kCarry = false: c is known to be 0
  template <bool kCarry>
  __device__ __forceinline__ void mac_wide(u64 s, u32 c, u64 d) {
    const u32 sl = (u32)s, sh = (u32)(s >> 32), dv = (u32)d;
    asm("mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(w0), "+r"(w1), "+r"(w2), "+r"(w3)
        : "r"(sl), "r"(sh), "r"(dv));
    if (kCarry)
      asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\t"
          "madc.hi.u32 %1, %2, %3, %1;"
          : "+r"(w2), "+r"(w3)
          : "r"(c), "r"(dv));
  }
  // += s + c 2^64
  __device__ __forceinline__ void add_wide(u64 s, u32 c) {
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(w0), "+r"(w1), "+r"(w2), "+r"(w3)
        : "r"((u32)s), "r"((u32)(s >> 32)), "r"(c));
  }
  // Horner over the words: every step reduces a value below 2^64
  __device__ __forceinline__ u64 get(const ModConst& m) const {
    u64 r = reduce64(((u64)w3 << 32) | w2, m);
    r = reduce64((r << 32) | w1, m);
    return reduce64((r << 32) | w0, m);
  }
};
template <>
struct DhAcc<u64> {
  u64 lo = 0, hi = 0;
  u32 top = 0;
  __device__ __forceinline__ void add(u64 x) {
    const u64 l = lo + x;
    const u64 h = hi + (l < x);
    top += h < hi;
    lo = l;
    hi = h;
  }
  __device__ __forceinline__ void mac(u64 x, u64 y) {
    const u64 plo = x * y, phi = __umul64hi(x, y);
    const u64 l = lo + plo;
    const u64 h1 = hi + phi;
    top += h1 < phi;
    const u64 h2 = h1 + (l < plo);
    top += h2 < h1;
    lo = l;
    hi = h2;
  }
  __device__ __forceinline__ u64 get(const ModConst& m) const {
    u64 r = reduce128(hi, lo, m);
    if (top) r = add_mod(r, mul_mod(mul_mod(m.r64, m.r64, m), top, m), m.q);  // top * 2^128 mod q
    return r;
  }
};

// partial layout: [B][chunks][3][ell+1][N] with component 2 = A_0 (slot ell unused)
__device__ __forceinline__ u64 dh_off(u32 rq, u32 chunk, u32 chunks, u32 comp, u32 slot, u32 ell, u32 log_n) {
  return ((((u64)rq * chunks + chunk) * 3 + comp) * (ell + 1) + slot) << log_n;
}

}  // namespace tcks

// Negacyclic NTT / INTT of one limb held in shared memory, run by a whole CTA.
//
// Forward: natural-order input, bit-reversed output, out_j = sum_i a_i psi^((2 brv(j) + 1) i)
// (Cooley-Tukey butterflies with psi^brv(m + i) at stage m, block i; Longa-Naehrig 2016).
// Inverse: Gentleman-Sande butterflies with psi^-brv(m + i); the caller applies N^-1.
// Each thread owns groups of four elements spanning two consecutive stages (a radix-4 step in
// registers), so shared memory is read and written once per two stages; a single radix-2 stage
// finishes an odd stage count.
#pragma once
#include "dev_arith.cuh"

namespace tcks {

__device__ __forceinline__ const u64* tw_at(const DevTables& T, u32 mod, u32 which) {
  return T.tw + ((u64)mod * 4 + which) * (1ull << T.log_n);
}

// Harvey forward butterfly: X, Y in [0, 4q) -> X + WY, X - WY in [0, 4q).
__device__ __forceinline__ void ct_bfly(u64& X, u64& Y, u64 W, u64 Wsh, u64 q, u64 two_q) {
  const u64 x = csub(X, two_q);
  const u64 t = mul_shoup_lazy(Y, W, Wsh, q);
  X = x + t;
  Y = x - t + two_q;
}

// Harvey inverse butterfly: X, Y in [0, 2q) -> X + Y, (X - Y) W in [0, 2q).
__device__ __forceinline__ void gs_bfly(u64& X, u64& Y, u64 W, u64 Wsh, u64 q, u64 two_q) {
  const u64 u = csub(X + Y, two_q);
  Y = mul_shoup_lazy(X - Y + two_q, W, Wsh, q);
  X = u;
}

// In-place forward transform of s[0, N); input in [0, 4q), output in [0, 4q).
__device__ __forceinline__ void ntt_fwd_smem(u64* s, const DevTables& T, u32 mod) {
  const u32 log_n = T.log_n;
  const u32 n = 1u << log_n;
  const u64 q = T.mods[mod].q, two_q = 2 * q;
  const u64* tw = tw_at(T, mod, 0);
  const u64* tws = tw_at(T, mod, 1);
  u32 st = 0;
  // pairs of stages: stage st (t = N >> (st+1)) and st+1 (t/2)
  for (; st + 1 < log_n; st += 2) {
    const u32 log_t2 = log_n - 2 - st;  // t2 = N >> (st + 2): stride of the second stage
    const u32 t2 = 1u << log_t2;
    const u32 m = 1u << st;
    for (u32 g = threadIdx.x; g < (n >> 2); g += blockDim.x) {
      const u32 blk = g >> log_t2;        // block of the first stage (size 4*t2)
      const u32 j = g & (t2 - 1);
      const u32 base = (blk << (log_t2 + 2)) + j;
      u64 a0 = s[base], a1 = s[base + t2], a2 = s[base + 2 * t2], a3 = s[base + 3 * t2];
      const u64 w = tw[m + blk], wsh = tws[m + blk];
      ct_bfly(a0, a2, w, wsh, q, two_q);
      ct_bfly(a1, a3, w, wsh, q, two_q);
      const u32 m2 = 2 * m + 2 * blk;
      ct_bfly(a0, a1, tw[m2], tws[m2], q, two_q);
      ct_bfly(a2, a3, tw[m2 + 1], tws[m2 + 1], q, two_q);
      s[base] = a0;
      s[base + t2] = a1;
      s[base + 2 * t2] = a2;
      s[base + 3 * t2] = a3;
    }
    __syncthreads();
  }
  if (st < log_n) {  // last single stage, t = 1
    const u32 m = 1u << st;
    for (u32 b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
      u64 X = s[2 * b], Y = s[2 * b + 1];
      ct_bfly(X, Y, tw[m + b], tws[m + b], q, two_q);
      s[2 * b] = X;
      s[2 * b + 1] = Y;
    }
    __syncthreads();
  }
}

// In-place inverse transform (without the N^-1 factor); input in [0, 2q), output in [0, 2q).
__device__ __forceinline__ void ntt_inv_smem(u64* s, const DevTables& T, u32 mod) {
  const u32 log_n = T.log_n;
  const u32 n = 1u << log_n;
  const u64 q = T.mods[mod].q, two_q = 2 * q;
  const u64* tw = tw_at(T, mod, 2);
  const u64* tws = tw_at(T, mod, 3);
  u32 st = 0;
  if (log_n & 1u) {  // a single first stage (t = 1, m = N/2) makes the remaining count even
    const u32 m = n >> 1;
    for (u32 b = threadIdx.x; b < (n >> 1); b += blockDim.x) {
      u64 X = s[2 * b], Y = s[2 * b + 1];
      gs_bfly(X, Y, tw[m + b], tws[m + b], q, two_q);
      s[2 * b] = X;
      s[2 * b + 1] = Y;
    }
    __syncthreads();
    st = 1;
  }
  for (; st < log_n; st += 2) {
    // stages st (t = 2^st, m = N >> (st+1)) and st+1 (t' = 2t, m' = m/2)
    const u32 log_t = st;
    const u32 t = 1u << log_t;
    const u32 m = n >> (st + 1);
    for (u32 g = threadIdx.x; g < (n >> 2); g += blockDim.x) {
      const u32 blk = g >> log_t;  // block of the second stage (size 4t)
      const u32 j = g & (t - 1);
      const u32 base = (blk << (log_t + 2)) + j;
      u64 a0 = s[base], a1 = s[base + t], a2 = s[base + 2 * t], a3 = s[base + 3 * t];
      const u32 i0 = 2 * blk;  // first-stage block indices 2*blk and 2*blk+1
      gs_bfly(a0, a1, tw[m + i0], tws[m + i0], q, two_q);
      gs_bfly(a2, a3, tw[m + i0 + 1], tws[m + i0 + 1], q, two_q);
      const u32 m2 = (m >> 1) + blk;
      gs_bfly(a0, a2, tw[m2], tws[m2], q, two_q);
      gs_bfly(a1, a3, tw[m2], tws[m2], q, two_q);
      s[base] = a0;
      s[base + t] = a1;
      s[base + 2 * t] = a2;
      s[base + 3 * t] = a3;
    }
    __syncthreads();
  }
}

// Canonical value of a forward-transform output in [0, 4q).
__device__ __forceinline__ u64 fwd_final(u64 x, u64 q) { return csub(csub(x, 2 * q), q); }
// Canonical value of an inverse-transform output in [0, 2q) times N^-1.
__device__ __forceinline__ u64 inv_final(u64 x, const ModConst& m) { return mul_shoup(x, m.ninv, m.ninv_sh, m.q); }

}  // namespace tcks

// Negacyclic NTT / INTT of one limb held in shared memory, run by a CTA or a thread-block cluster.
//
// Forward: natural-order input, bit-reversed output, out_j = sum_i a_i psi^((2 brv(j) + 1) i)
// (Cooley-Tukey butterflies with psi^brv(m + i) at stage m, block i; Longa-Naehrig 2016).
// Inverse: Gentleman-Sande butterflies with psi^-brv(m + i); the caller applies N^-1.
//
// Limbs up to 2^14 words sit in one CTA's shared memory. Larger limbs (N = 2^15, 2^16) are split over
// a cluster of C = 2 or 4 CTAs, CTA `rank` holding elements [rank*N/C, (rank+1)*N/C): the stages whose
// butterflies cross that split (the first log2 C forward stages, the last log2 C inverse stages) read
// the partner elements from the other CTAs' shared memory (DSMEM) and keep their own result; every
// other stage is local. Local stages run as radix-8 rounds in registers (three stages per shared
// memory round trip), with a radix-4 or radix-2 round for the remainder.
#pragma once
#include <cooperative_groups.h>

#include "dev_arith.cuh"

namespace tcks {

// Shared-memory position of limb element i: the low four bits are XORed with the 16-word row index,
// so the strided accesses of the small-distance rounds spread over all bank pairs (8-byte words:
// 16 words span the 32 banks) while each row keeps its 16 words.
__device__ __forceinline__ u32 sw(u32 i) { return i ^ ((i >> 4) & 15u); }

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

// R = 2^LR elements x[q] = element base + q * stride (stride = the round's smallest butterfly distance)
// through forward stages st .. st+LR-1; gblk = global index of the block of stage st.
template <int LR>
__device__ __forceinline__ void fwd_group(u64 (&x)[1 << LR], u32 st, u32 gblk, const u64* tw, const u64* tws, u64 q,
                                          u64 two_q) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int u = 0; u < LR; ++u) {
    const int h = R >> (u + 1);  // distance (in elements of the group) at sub-stage u
#pragma unroll
    for (int b = 0; b < (1 << u); ++b) {
      const u32 idx = ((1u << st) << u) + (gblk << u) + b;
      const u64 w = tw[idx], wsh = tws[idx];
#pragma unroll
      for (int x0 = 0; x0 < h; ++x0) ct_bfly(x[b * 2 * h + x0], x[b * 2 * h + x0 + h], w, wsh, q, two_q);
    }
  }
}

// Inverse stages st .. st+LR-1 on R elements base + q * 2^st; m0 = N >> (st+1); gblk = global block
// index (at the round's last sub-stage) of the group.
template <int LR>
__device__ __forceinline__ void inv_group(u64 (&x)[1 << LR], u32 log_n, u32 st, u32 gblk, const u64* tw,
                                          const u64* tws, u64 q, u64 two_q) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int u = 0; u < LR; ++u) {
    const int h = 1 << u;
    const u32 m = (1u << log_n) >> (st + u + 1);
#pragma unroll
    for (int b = 0; b < (R >> (u + 1)); ++b) {
      const u32 idx = m + (gblk << (LR - u - 1)) + b;
      const u64 w = tw[idx], wsh = tws[idx];
#pragma unroll
      for (int x0 = 0; x0 < h; ++x0) gs_bfly(x[b * 2 * h + x0], x[b * 2 * h + x0 + h], w, wsh, q, two_q);
    }
  }
}

// One local forward round of LR stages starting at stage st over the CTA's slice s[0, ns).
template <int LR>
__device__ __forceinline__ void fwd_round(u64* s, u32 log_n, u32 log_ns, u32 rank, u32 st, const u64* tw,
                                          const u64* tws, u64 q, u64 two_q) {
  constexpr int R = 1 << LR;
  const u32 log_tr = log_n - st - LR;  // smallest distance of the round
  const u32 tr = 1u << log_tr;
  const u32 groups = (1u << log_ns) >> LR;
  const u32 gbase = (rank << log_ns) >> (log_tr + LR);  // global block offset of this slice at stage st
  for (u32 g = threadIdx.x; g < groups; g += blockDim.x) {
    const u32 blk = g >> log_tr, j = g & (tr - 1);
    const u32 base = (blk << (log_tr + LR)) + j;
    u64 x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = s[sw(base + k * tr)];
    fwd_group<LR>(x, st, gbase + blk, tw, tws, q, two_q);
#pragma unroll
    for (int k = 0; k < R; ++k) s[sw(base + k * tr)] = x[k];
  }
  __syncthreads();
}

template <int LR>
__device__ __forceinline__ void inv_round(u64* s, u32 log_n, u32 log_ns, u32 rank, u32 st, const u64* tw,
                                          const u64* tws, u64 q, u64 two_q) {
  constexpr int R = 1 << LR;
  const u32 log_t = st;
  const u32 t = 1u << log_t;
  const u32 groups = (1u << log_ns) >> LR;
  const u32 gbase = (rank << log_ns) >> (log_t + LR);  // global block offset at the round's last sub-stage
  for (u32 g = threadIdx.x; g < groups; g += blockDim.x) {
    const u32 blk = g >> log_t, j = g & (t - 1);
    const u32 base = (blk << (log_t + LR)) + j;
    u64 x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = s[sw(base + k * t)];
    inv_group<LR>(x, log_n, st, gbase + blk, tw, tws, q, two_q);
#pragma unroll
    for (int k = 0; k < R; ++k) s[sw(base + k * t)] = x[k];
  }
  __syncthreads();
}

// Cross-CTA forward stages 0 .. LC-1 (C = 2^LC CTAs): element j of every CTA's slice forms a group
// of C; each CTA computes the group and keeps its own element. The slice s must be complete in
// every CTA of the cluster (the caller's prologue), and s is overwritten only after all reads.
template <int LC>
__device__ __forceinline__ void fwd_cross(u64* s, u32 log_ns, u32 rank, const u64* tw, const u64* tws, u64 q,
                                          u64 two_q) {
  namespace cg = cooperative_groups;
  constexpr int C = 1 << LC;
  constexpr int PER = 8;  // elements a thread finishes before the write-back barrier
  cg::cluster_group cl = cg::this_cluster();
  const u32 ns = 1u << log_ns;
  const u64* rem[C];
#pragma unroll
  for (int r = 0; r < C; ++r) rem[r] = cl.map_shared_rank(s, r);
  cl.sync();
  for (u32 c0 = 0; c0 < ns; c0 += blockDim.x * PER) {
    u64 keep[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const u32 j = c0 + e * blockDim.x + threadIdx.x;
      if (j < ns) {
        u64 x[C];
#pragma unroll
        for (int r = 0; r < C; ++r) x[r] = rem[r][sw(j)];
        fwd_group<LC>(x, 0, 0, tw, tws, q, two_q);
        keep[e] = x[0];
#pragma unroll
        for (int r = 1; r < C; ++r)
          if ((u32)r == rank) keep[e] = x[r];
      }
    }
    cl.sync();
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const u32 j = c0 + e * blockDim.x + threadIdx.x;
      if (j < ns) s[sw(j)] = keep[e];
    }
    cl.sync();
  }
}

// Cross-CTA inverse stages (the last LC): after all local stages; results go to s in place.
template <int LC>
__device__ __forceinline__ void inv_cross(u64* s, u32 log_n, u32 log_ns, u32 rank, const u64* tw, const u64* tws,
                                          u64 q, u64 two_q) {
  namespace cg = cooperative_groups;
  constexpr int C = 1 << LC;
  constexpr int PER = 8;
  cg::cluster_group cl = cg::this_cluster();
  const u32 ns = 1u << log_ns;
  const u64* rem[C];
#pragma unroll
  for (int r = 0; r < C; ++r) rem[r] = cl.map_shared_rank(s, r);
  cl.sync();
  for (u32 c0 = 0; c0 < ns; c0 += blockDim.x * PER) {
    u64 keep[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const u32 j = c0 + e * blockDim.x + threadIdx.x;
      if (j < ns) {
        u64 x[C];
#pragma unroll
        for (int r = 0; r < C; ++r) x[r] = rem[r][sw(j)];
        inv_group<LC>(x, log_n, log_ns, 0, tw, tws, q, two_q);
        keep[e] = x[0];
#pragma unroll
        for (int r = 1; r < C; ++r)
          if ((u32)r == rank) keep[e] = x[r];
      }
    }
    cl.sync();
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const u32 j = c0 + e * blockDim.x + threadIdx.x;
      if (j < ns) s[sw(j)] = keep[e];
    }
    cl.sync();
  }
}

// Forward transform of the CTA's slice s[0, N/C) of a limb split over C = 2^LC CTAs (LC = 0: the
// whole limb). Input in [0, 4q), output in [0, 4q). Ends with a barrier.
template <int LC>
__device__ __forceinline__ void ntt_fwd_slice(u64* s, const DevTables& T, u32 mod, u32 rank) {
  const u32 log_n = T.log_n, log_ns = log_n - LC;
  const u64 q = T.mods[mod].q, two_q = 2 * q;
  const u64* tw = tw_at(T, mod, 0);
  const u64* tws = tw_at(T, mod, 1);
  if constexpr (LC > 0) fwd_cross<LC>(s, log_ns, rank, tw, tws, q, two_q);
  u32 st = LC;
  const u32 left = log_n - st;
  // remainder round first (radix-2 or radix-4), then radix-8 rounds
  if (left % 3 == 1) {
    fwd_round<1>(s, log_n, log_ns, rank, st, tw, tws, q, two_q);
    st += 1;
  } else if (left % 3 == 2) {
    fwd_round<2>(s, log_n, log_ns, rank, st, tw, tws, q, two_q);
    st += 2;
  }
  for (; st < log_n; st += 3) fwd_round<3>(s, log_n, log_ns, rank, st, tw, tws, q, two_q);
}

// Inverse transform (without N^-1) of the CTA's slice; input in [0, 2q), output in [0, 2q).
template <int LC>
__device__ __forceinline__ void ntt_inv_slice(u64* s, const DevTables& T, u32 mod, u32 rank) {
  const u32 log_n = T.log_n, log_ns = log_n - LC;
  const u64 q = T.mods[mod].q, two_q = 2 * q;
  const u64* tw = tw_at(T, mod, 2);
  const u64* tws = tw_at(T, mod, 3);
  u32 st = 0;
  for (; st + 3 <= log_ns; st += 3) inv_round<3>(s, log_n, log_ns, rank, st, tw, tws, q, two_q);
  if (log_ns - st == 2) inv_round<2>(s, log_n, log_ns, rank, st, tw, tws, q, two_q);
  if (log_ns - st == 1) inv_round<1>(s, log_n, log_ns, rank, st, tw, tws, q, two_q);
  if constexpr (LC > 0) inv_cross<LC>(s, log_n, log_ns, rank, tw, tws, q, two_q);
}

// Whole-limb wrappers (single CTA).
__device__ __forceinline__ void ntt_fwd_smem(u64* s, const DevTables& T, u32 mod) { ntt_fwd_slice<0>(s, T, mod, 0); }
__device__ __forceinline__ void ntt_inv_smem(u64* s, const DevTables& T, u32 mod) { ntt_inv_slice<0>(s, T, mod, 0); }

// Canonical value of a forward-transform output in [0, 4q).
__device__ __forceinline__ u64 fwd_final(u64 x, u64 q) { return csub(csub(x, 2 * q), q); }
// Canonical value of an inverse-transform output in [0, 2q) times N^-1.
__device__ __forceinline__ u64 inv_final(u64 x, const ModConst& m) { return mul_shoup(x, m.ninv, m.ninv_sh, m.q); }

// Launch geometry of a limb transform: cluster size 2^log_c, threads per CTA, shared memory bytes.
struct LimbShape {
  u32 log_c;
  u32 threads;
  size_t smem;
};
__host__ __device__ inline LimbShape limb_shape(u32 log_n) {
  LimbShape s;
  s.log_c = log_n > 14 ? log_n - 14 : 0;
  const u32 log_ns = log_n - s.log_c;
  u32 t = (1u << log_ns) / 32;  // 4 radix-8 groups per thread
  if (t < 32) t = 32;
  if (t > 512) t = 512;
  s.threads = t;
  s.smem = (size_t)8 << log_ns;
  return s;
}

}  // namespace tcks

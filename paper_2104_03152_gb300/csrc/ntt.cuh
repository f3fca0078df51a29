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
//
// Word types: W = u64 for any prime below 2^62 (Harvey's lazy butterflies: [0, 4q) forward,
// [0, 2q) inverse, 64-bit Shoup); W = u32 when every prime of the chain is below 2^31 (32-bit Shoup
// companions, half the shared memory): lazy butterflies for primes below 2^30, fully reduced ones for
// primes in [2^30, 2^31). Both give the canonical result.
#pragma once
#include <cooperative_groups.h>

#include "dev_arith.cuh"

namespace tcks {

// Shared-memory position of limb element i: the low four bits are XORed with the 16-word row index,
// so the strided accesses of the small-distance rounds spread over the banks while each row keeps
// its 16 words.
__device__ __forceinline__ u32 sw(u32 i) { return i ^ ((i >> 4) & 15u); }

__device__ __forceinline__ const u64* tw_at(const DevTables& T, u32 mod, u32 which) {
  return T.tw + ((u64)mod * 4 + which) * (1ull << T.log_n);
}

template <typename W>
struct Ar;

// 64-bit words, Harvey lazy reduction.
template <>
struct Ar<u64> {
  static __device__ __forceinline__ const u64* tw(const DevTables& T, u32 mod, u32 which) { return tw_at(T, mod, which); }
  // X, Y in [0, 4q) -> X + WY, X - WY in [0, 4q).
  static __device__ __forceinline__ void ct(u64& X, u64& Y, u64 W, u64 Wsh, u64 q) {
    const u64 two_q = 2 * q;
    const u64 x = csub(X, two_q);
    const u64 t = mul_shoup_lazy(Y, W, Wsh, q);
    X = x + t;
    Y = x - t + two_q;
  }
  // X, Y in [0, 2q) -> X + Y, (X - Y) W in [0, 2q).
  static __device__ __forceinline__ void gs(u64& X, u64& Y, u64 W, u64 Wsh, u64 q) {
    const u64 two_q = 2 * q;
    const u64 u = csub(X + Y, two_q);
    Y = mul_shoup_lazy(X - Y + two_q, W, Wsh, q);
    X = u;
  }
  static __device__ __forceinline__ u64 fwd_out(u64 x, const ModConst& m) { return csub(csub(x, 2 * m.q), m.q); }
  static __device__ __forceinline__ u64 inv_out(u64 x, const ModConst& m) { return mul_shoup(x, m.ninv, m.ninv_sh, m.q); }
};

// 32-bit words (q < 2^31), every value fully reduced.
__device__ __forceinline__ u32 csub32(u32 a, u32 q) { return a >= q ? a - q : a; }
__device__ __forceinline__ u32 shoup32(u32 a, u32 w, u32 wsh, u32 q) {
  return csub32(a * w - __umulhi(a, wsh) * q, q);
}
template <>
struct Ar<u32> {
  // which = 0, 1: the forward (twiddle, Shoup) pairs; 2, 3: the inverse ones (one table per
  // direction, read as pairs by the butterfly groups)
  static __device__ __forceinline__ const u32* tw(const DevTables& T, u32 mod, u32 which) {
    return T.tw32 + ((u64)mod * 2 + (which >> 1)) * (2ull << T.log_n);
  }
  static __device__ __forceinline__ void ct(u32& X, u32& Y, u32 W, u32 Wsh, u32 q) {
    const u32 t = shoup32(Y, W, Wsh, q);
    const u32 x = X;
    X = csub32(x + t, q);
    Y = x >= t ? x - t : x + q - t;
  }
  static __device__ __forceinline__ void gs(u32& X, u32& Y, u32 W, u32 Wsh, u32 q) {
    const u32 x = X, y = Y;
    X = csub32(x + y, q);
    Y = shoup32(x >= y ? x - y : x + q - y, W, Wsh, q);
  }
  static __device__ __forceinline__ u64 fwd_out(u32 x, const ModConst&) { return x; }
  static __device__ __forceinline__ u64 inv_out(u32 x, const ModConst& m) {
    return shoup32(x, (u32)m.ninv, (u32)m.ninv_sh32, (u32)m.q);
  }
};

// 32-bit words with Harvey's lazy bounds for primes below 2^30 ([0, 4q) forward, [0, 2q) inverse fit
// in 32 bits): about half the integer operations of the fully reduced butterfly. The slice transforms
// take this policy for such primes (one uniform branch per CTA) and finish in canonical form.
struct Ar32Lazy {
  // X, Y in [0, 4q) -> X + WY, X - WY in [0, 4q).
  static __device__ __forceinline__ void ct(u32& X, u32& Y, u32 W, u32 Wsh, u32 q) {
    const u32 two_q = 2 * q;
    const u32 x = csub32(X, two_q);
    const u32 t = Y * W - __umulhi(Y, Wsh) * q;  // in [0, 2q)
    X = x + t;
    Y = x - t + two_q;
  }
  // X, Y in [0, 2q) -> X + Y, (X - Y) W in [0, 2q).
  static __device__ __forceinline__ void gs(u32& X, u32& Y, u32 W, u32 Wsh, u32 q) {
    const u32 two_q = 2 * q;
    const u32 u = csub32(X + Y, two_q);
    const u32 d = X - Y + two_q;
    Y = d * W - __umulhi(d, Wsh) * q;
    X = u;
  }
};


// 32-bit words with primes so small that (2 log N + 4) q < 2^32: the forward butterfly without any
// conditional subtraction. The Shoup product is in [0, 2q) for any input word, so a value in [0, k q)
// leaves a stage in [0, (k + 2) q); an input below 4q ends the log N stages below (2 log N + 4) q,
// still one word, and one 32-bit Barrett reduction per element finishes the transform.
struct Ar32Grow {
  static __device__ __forceinline__ void ct(u32& X, u32& Y, u32 W, u32 Wsh, u32 q) {
    const u32 x = X;
    const u32 t = Y * W - __umulhi(Y, Wsh) * q;  // in [0, 2q)
    X = x + t;
    Y = x - t + 2 * q;
  }
  static __device__ __forceinline__ void gs(u32& X, u32& Y, u32 W, u32 Wsh, u32 q) { Ar32Lazy::gs(X, Y, W, Wsh, q); }
};

// Twiddle idx and its Shoup companion: 64-bit words from two tables, 32-bit words as one pair.
__device__ __forceinline__ void load_tw(const u64* tw, const u64* tws, u32 idx, u64& w, u64& wsh) {
  w = tw[idx];
  wsh = tws[idx];
}
__device__ __forceinline__ void load_tw(const u32* tw, const u32*, u32 idx, u32& w, u32& wsh) {
  const uint2 p = reinterpret_cast<const uint2*>(tw)[idx];
  w = p.x;
  wsh = p.y;
}

// R = 2^LR elements x[q] = element base + q * stride (stride = the round's smallest butterfly
// distance) through forward stages st .. st+LR-1; gblk = global index of the block of stage st.
template <typename W, int LR, typename A = Ar<W>>
__device__ __forceinline__ void fwd_group(W (&x)[1 << LR], u32 st, u32 gblk, const W* tw, const W* tws, W q) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int u = 0; u < LR; ++u) {
    const int h = R >> (u + 1);  // distance (in elements of the group) at sub-stage u
#pragma unroll
    for (int b = 0; b < (1 << u); ++b) {
      const u32 idx = ((1u << st) << u) + (gblk << u) + b;
      W w, wsh;
      load_tw(tw, tws, idx, w, wsh);
#pragma unroll
      for (int x0 = 0; x0 < h; ++x0) A::ct(x[b * 2 * h + x0], x[b * 2 * h + x0 + h], w, wsh, q);
    }
  }
}

// Inverse stages st .. st+LR-1 on R elements base + q * 2^st; gblk = global block index (at the
// round's last sub-stage) of the group.
template <typename W, int LR, typename A = Ar<W>>
__device__ __forceinline__ void inv_group(W (&x)[1 << LR], u32 log_n, u32 st, u32 gblk, const W* tw, const W* tws,
                                          W q) {
  constexpr int R = 1 << LR;
#pragma unroll
  for (int u = 0; u < LR; ++u) {
    const int h = 1 << u;
    const u32 m = (1u << log_n) >> (st + u + 1);
#pragma unroll
    for (int b = 0; b < (R >> (u + 1)); ++b) {
      const u32 idx = m + (gblk << (LR - u - 1)) + b;
      W w, wsh;
      load_tw(tw, tws, idx, w, wsh);
#pragma unroll
      for (int x0 = 0; x0 < h; ++x0) A::gs(x[b * 2 * h + x0], x[b * 2 * h + x0 + h], w, wsh, q);
    }
  }
}

// One local forward round of LR stages starting at stage st over the CTA's slice s[0, ns).
template <typename W, int LR, typename A = Ar<W>>
__device__ __forceinline__ void fwd_round(W* s, u32 log_n, u32 log_ns, u32 rank, u32 st, const W* tw, const W* tws,
                                          W q) {
  constexpr int R = 1 << LR;
  const u32 log_tr = log_n - st - LR;  // smallest distance of the round
  const u32 tr = 1u << log_tr;
  const u32 groups = (1u << log_ns) >> LR;
  const u32 gbase = (rank << log_ns) >> (log_tr + LR);  // global block offset of this slice at stage st
  for (u32 g = threadIdx.x; g < groups; g += blockDim.x) {
    const u32 blk = g >> log_tr, j = g & (tr - 1);
    const u32 base = (blk << (log_tr + LR)) + j;
    W x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = s[sw(base + k * tr)];
    fwd_group<W, LR, A>(x, st, gbase + blk, tw, tws, q);
#pragma unroll
    for (int k = 0; k < R; ++k) s[sw(base + k * tr)] = x[k];
  }
  __syncthreads();
}

template <typename W, int LR, typename A = Ar<W>>
__device__ __forceinline__ void inv_round(W* s, u32 log_n, u32 log_ns, u32 rank, u32 st, const W* tw, const W* tws,
                                          W q) {
  constexpr int R = 1 << LR;
  const u32 log_t = st;
  const u32 t = 1u << log_t;
  const u32 groups = (1u << log_ns) >> LR;
  const u32 gbase = (rank << log_ns) >> (log_t + LR);  // global block offset at the round's last sub-stage
  for (u32 g = threadIdx.x; g < groups; g += blockDim.x) {
    const u32 blk = g >> log_t, j = g & (t - 1);
    const u32 base = (blk << (log_t + LR)) + j;
    W x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = s[sw(base + k * t)];
    inv_group<W, LR, A>(x, log_n, st, gbase + blk, tw, tws, q);
#pragma unroll
    for (int k = 0; k < R; ++k) s[sw(base + k * t)] = x[k];
  }
  __syncthreads();
}

// Cross-CTA stages (C = 2^LC CTAs): element j of every CTA's slice forms a group of C; each CTA
// computes the group and keeps its own element. FWD: the first LC forward stages (the slice must be
// complete in every CTA); otherwise the last LC inverse stages. s is overwritten only after all reads.
template <typename W, int LC, bool FWD, typename A = Ar<W>>
__device__ __forceinline__ void cross_stages(W* s, u32 log_n, u32 log_ns, u32 rank, const W* tw, const W* tws, W q) {
  namespace cg = cooperative_groups;
  constexpr int C = 1 << LC;
  constexpr int PER = 8;  // elements a thread finishes before the write-back barrier
  cg::cluster_group cl = cg::this_cluster();
  const u32 ns = 1u << log_ns;
  const W* rem[C];
#pragma unroll
  for (int r = 0; r < C; ++r) rem[r] = cl.map_shared_rank(s, r);
  cl.sync();
  for (u32 c0 = 0; c0 < ns; c0 += blockDim.x * PER) {
    W keep[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      const u32 j = c0 + e * blockDim.x + threadIdx.x;
      if (j < ns) {
        W x[C];
#pragma unroll
        for (int r = 0; r < C; ++r) x[r] = rem[r][sw(j)];
        if (FWD)
          fwd_group<W, LC, A>(x, 0, 0, tw, tws, q);
        else
          inv_group<W, LC, A>(x, log_n, log_ns, 0, tw, tws, q);
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

// The stages a slice of 2^log_ns consecutive elements (slice `rank` of the limb) completes on its
// own: forward stages log_n - log_ns .. log_n - 1 (the earlier ones pair elements of different
// slices), or inverse stages 0 .. log_ns - 1. Each ends with a barrier.
// Stages per local round (radix-8). Radix-16 rounds for 32-bit words were measured: one shared-memory
// round trip fewer, but the register pressure they add slowed the fused key-switch kernels more than
// it sped up the plain transforms.
constexpr int kRadixBits32 = 3;
template <typename W>
struct RadixBits {
  static constexpr int value = sizeof(W) == 4 ? kRadixBits32 : 3;
};

template <typename W, typename A = Ar<W>>
__device__ __forceinline__ void ntt_fwd_local_rounds(W* s, u32 log_n, u32 log_ns, u32 rank, const W* tw, const W* tws,
                                                     W q) {
  constexpr int RB = RadixBits<W>::value;
  u32 st = log_n - log_ns;
  // remainder round first, then full rounds of RB stages
  const u32 rem = log_ns % RB;
  if (rem == 1) fwd_round<W, 1, A>(s, log_n, log_ns, rank, st, tw, tws, q);
  if (rem == 2) fwd_round<W, 2, A>(s, log_n, log_ns, rank, st, tw, tws, q);
  if constexpr (RB > 3)
    if (rem == 3) fwd_round<W, 3, A>(s, log_n, log_ns, rank, st, tw, tws, q);
  st += rem;
#pragma unroll
  for (; st < log_n; st += RB) fwd_round<W, RB, A>(s, log_n, log_ns, rank, st, tw, tws, q);
}
template <typename W, typename A = Ar<W>>
__device__ __forceinline__ void ntt_inv_local_rounds(W* s, u32 log_n, u32 log_ns, u32 rank, const W* tw, const W* tws,
                                                     W q) {
  constexpr int RB = RadixBits<W>::value;
  u32 st = 0;
#pragma unroll
  for (; st + RB <= log_ns; st += RB) inv_round<W, RB, A>(s, log_n, log_ns, rank, st, tw, tws, q);
  if constexpr (RB > 3)
    if (log_ns - st == 3) inv_round<W, 3, A>(s, log_n, log_ns, rank, st, tw, tws, q);
  if (log_ns - st == 2) inv_round<W, 2, A>(s, log_n, log_ns, rank, st, tw, tws, q);
  if (log_ns - st == 1) inv_round<W, 1, A>(s, log_n, log_ns, rank, st, tw, tws, q);
}

// Forward transform of the CTA's slice s[0, N/C) of a limb split over C = 2^LC CTAs (LC = 0: the
// whole limb). Input canonical (or in [0, 4q) for W = u64); output in [0, 4q) (u64) or canonical
// (u32); Ar<W>::fwd_out gives the canonical value. Ends with a barrier.
template <typename W, int LC, int LOGN>
__device__ __forceinline__ void ntt_fwd_slice_n(W* s, const DevTables& T, u32 mod, u32 rank) {
  const u32 log_n = LOGN > 0 ? (u32)LOGN : T.log_n, log_ns = log_n - LC;
  const W q = (W)T.mods[mod].q;
  const W* tw = Ar<W>::tw(T, mod, 0);
  const W* tws = Ar<W>::tw(T, mod, 1);
  if constexpr (sizeof(W) == 4) {
    if ((u64)q * (2 * log_n + 4) < (1ull << 32)) {  // no subtractions in the stages, one reduction after
      if constexpr (LC > 0) cross_stages<W, LC, true, Ar32Grow>(s, log_n, log_ns, rank, tw, tws, q);
      ntt_fwd_local_rounds<W, Ar32Grow>(s, log_n, log_ns, rank, tw, tws, q);
      const ModConst& m = T.mods[mod];
      for (u32 k = threadIdx.x; k < (1u << log_ns); k += blockDim.x) s[k] = reduce32(s[k], m);
      __syncthreads();
      return;
    }
    if (q < (1u << 30)) {  // lazy butterflies, then [0, 4q) -> [0, q)
      if constexpr (LC > 0) cross_stages<W, LC, true, Ar32Lazy>(s, log_n, log_ns, rank, tw, tws, q);
      ntt_fwd_local_rounds<W, Ar32Lazy>(s, log_n, log_ns, rank, tw, tws, q);
      for (u32 k = threadIdx.x; k < (1u << log_ns); k += blockDim.x) s[k] = csub32(csub32(s[k], 2 * q), q);
      __syncthreads();
      return;
    }
  }
  if constexpr (LC > 0) cross_stages<W, LC, true>(s, log_n, log_ns, rank, tw, tws, q);
  ntt_fwd_local_rounds<W>(s, log_n, log_ns, rank, tw, tws, q);
}
template <typename W, int LC>
__device__ __forceinline__ void ntt_fwd_slice(W* s, const DevTables& T, u32 mod, u32 rank) {
  if constexpr (LC == 0) {
    if (T.log_n == 13) {  // the encrypted network's ring: the size fixed at compile time
      ntt_fwd_slice_n<W, 0, 13>(s, T, mod, rank);
      return;
    }
  }
  ntt_fwd_slice_n<W, LC, 0>(s, T, mod, rank);
}

// Inverse transform (without N^-1) of the CTA's slice; input canonical, output in [0, 2q) (u64, and
// u32 primes below 2^30) or canonical (other u32 primes); Ar<W>::inv_out applies N^-1 and gives the
// canonical value.
template <typename W, int LC, int LOGN>
__device__ __forceinline__ void ntt_inv_slice_n(W* s, const DevTables& T, u32 mod, u32 rank) {
  const u32 log_n = LOGN > 0 ? (u32)LOGN : T.log_n, log_ns = log_n - LC;
  const W q = (W)T.mods[mod].q;
  const W* tw = Ar<W>::tw(T, mod, 2);
  const W* tws = Ar<W>::tw(T, mod, 3);
  if constexpr (sizeof(W) == 4) {
    if (q < (1u << 30)) {  // lazy butterflies: output in [0, 2q), which Ar<u32>::inv_out accepts
      ntt_inv_local_rounds<W, Ar32Lazy>(s, log_n, log_ns, rank, tw, tws, q);
      if constexpr (LC > 0) cross_stages<W, LC, false, Ar32Lazy>(s, log_n, log_ns, rank, tw, tws, q);
      return;
    }
  }
  ntt_inv_local_rounds<W>(s, log_n, log_ns, rank, tw, tws, q);
  if constexpr (LC > 0) cross_stages<W, LC, false>(s, log_n, log_ns, rank, tw, tws, q);
}
template <typename W, int LC>
__device__ __forceinline__ void ntt_inv_slice(W* s, const DevTables& T, u32 mod, u32 rank) {
  if constexpr (LC == 0) {
    if (T.log_n == 13) {
      ntt_inv_slice_n<W, 0, 13>(s, T, mod, rank);
      return;
    }
  }
  ntt_inv_slice_n<W, LC, 0>(s, T, mod, rank);
}

// ---------------------------------------- forward transform fed by its producer, relaxed output ----
// fwd_round at stage 0 of a whole limb with the groups' inputs taken from load(index) instead of the
// shared slice: the first round of a transform whose input is computed on the fly (a lift from
// another prime), which saves the staging pass through shared memory and its barrier.
template <typename W, int LR, typename A, typename F>
__device__ __forceinline__ void fwd_round_load(W* s, u32 log_n, const W* tw, const W* tws, W q, F&& load) {
  constexpr int R = 1 << LR;
  const u32 tr = 1u << (log_n - LR);  // the first stage's distance is N / 2; N / R groups
  for (u32 g = threadIdx.x; g < tr; g += blockDim.x) {
    W x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = (W)load(g + k * tr);
    fwd_group<W, LR, A>(x, 0, 0, tw, tws, q);
#pragma unroll
    for (int k = 0; k < R; ++k) s[sw(g + k * tr)] = x[k];
  }
  __syncthreads();
}

// Forward transform of a whole limb (one CTA) whose input element k is load(k) (canonical), the first
// round reading it directly. The butterflies and their order are ntt_fwd_slice's; the output is left
// as its rounds leave it (64-bit words: [0, 4q); 32-bit words: below 2^32, without the final
// canonicalisation pass), and fwd_fin gives the canonical value. Ends with a barrier.
// LOGN > 0 fixes the ring size at compile time: the rounds unroll and their strides, swizzled offsets
// and twiddle indices fold into constants.
template <typename W, int LOGN, typename F>
__device__ __forceinline__ void ntt_fwd_limb_load_n(W* s, const DevTables& T, u32 mod, F&& load) {
  constexpr int RB = RadixBits<W>::value;
  static_assert(RB == 3, "the first round below covers remainders of radix-8 rounds");
  const u32 log_n = LOGN > 0 ? (u32)LOGN : T.log_n;
  const W q = (W)T.mods[mod].q;
  const W* tw = Ar<W>::tw(T, mod, 0);
  const W* tws = Ar<W>::tw(T, mod, 1);
  auto run = [&](auto policy) {
    using A = decltype(policy);
    const u32 first = log_n % RB ? log_n % RB : RB;
    if (first == 1)
      fwd_round_load<W, 1, A>(s, log_n, tw, tws, q, load);
    else if (first == 2)
      fwd_round_load<W, 2, A>(s, log_n, tw, tws, q, load);
    else
      fwd_round_load<W, 3, A>(s, log_n, tw, tws, q, load);
#pragma unroll
    for (u32 st = first; st < log_n; st += RB) fwd_round<W, RB, A>(s, log_n, log_n, 0, st, tw, tws, q);
  };
  if constexpr (sizeof(W) == 4) {
    if ((u64)q * (2 * log_n + 4) < (1ull << 32)) {
      run(Ar32Grow{});
      return;
    }
    if (q < (1u << 30)) {
      run(Ar32Lazy{});
      return;
    }
  }
  run(Ar<W>{});
}

// The last forward round of a whole limb (its smallest distance is 1): group g holds the outputs
// 8g .. 8g + 7 in registers, which go to store(8g, x) instead of back to shared memory.
template <typename W, typename A, typename G>
__device__ __forceinline__ void fwd_round_store(u32 log_n, u32 st, const W* s, const W* tw, const W* tws, W q, G&& store) {
  constexpr int LR = 3, R = 1 << LR;
  const u32 groups = (1u << log_n) >> LR;
  for (u32 g = threadIdx.x; g < groups; g += blockDim.x) {
    const u32 base = g << LR;
    W x[R];
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = s[sw(base + k)];
    fwd_group<W, LR, A>(x, st, g, tw, tws, q);
    store(base, x);
  }
}

// ntt_fwd_limb_load whose last round hands each thread's 8 consecutive outputs (relaxed as
// ntt_fwd_limb_load leaves them; fwd_fin gives the canonical values) to store(first index, x[8])
// instead of writing them back: one shared-memory pass and a barrier fewer for a caller that only
// writes the transform out. Shared memory is left partly stale; no barrier at the end.
template <typename W, int LOGN, typename F, typename G>
__device__ __forceinline__ void ntt_fwd_limb_load_store_n(W* s, const DevTables& T, u32 mod, F&& load, G&& store) {
  constexpr int RB = RadixBits<W>::value;
  static_assert(RB == 3, "the rounds below are radix-8");
  const u32 log_n = LOGN > 0 ? (u32)LOGN : T.log_n;
  const W q = (W)T.mods[mod].q;
  const W* tw = Ar<W>::tw(T, mod, 0);
  const W* tws = Ar<W>::tw(T, mod, 1);
  auto run = [&](auto policy) {
    using A = decltype(policy);
    const u32 first = log_n % RB ? log_n % RB : RB;
    if (first == 1)
      fwd_round_load<W, 1, A>(s, log_n, tw, tws, q, load);
    else if (first == 2)
      fwd_round_load<W, 2, A>(s, log_n, tw, tws, q, load);
    else
      fwd_round_load<W, 3, A>(s, log_n, tw, tws, q, load);
#pragma unroll
    for (u32 st = first; st + RB < log_n; st += RB) fwd_round<W, RB, A>(s, log_n, log_n, 0, st, tw, tws, q);
    fwd_round_store<W, A>(log_n, log_n - RB, s, tw, tws, q, store);
  };
  if constexpr (sizeof(W) == 4) {
    if ((u64)q * (2 * log_n + 4) < (1ull << 32)) {
      run(Ar32Grow{});
      return;
    }
    if (q < (1u << 30)) {
      run(Ar32Lazy{});
      return;
    }
  }
  run(Ar<W>{});
}

template <typename W, typename F>
__device__ __forceinline__ void ntt_fwd_limb_load(W* s, const DevTables& T, u32 mod, F&& load);

template <typename W, typename F, typename G>
__device__ __forceinline__ void ntt_fwd_limb_load_store(W* s, const DevTables& T, u32 mod, F&& load, G&& store) {
  if (T.log_n == 13) {
    ntt_fwd_limb_load_store_n<W, 13>(s, T, mod, load, store);
  } else if (T.log_n > 3) {
    ntt_fwd_limb_load_store_n<W, 0>(s, T, mod, load, store);
  } else {  // N = 8: the first round is the last; transform in shared memory, then hand the words out
    ntt_fwd_limb_load<W>(s, T, mod, load);
    W x[8];
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = s[sw(k)];
      store(0u, x);
    }
  }
}

// The entry point: N = 2^13 (the encrypted network's ring) with the size fixed, any other size as is.
template <typename W, typename F>
__device__ __forceinline__ void ntt_fwd_limb_load(W* s, const DevTables& T, u32 mod, F&& load) {
  if (T.log_n == 13)
    ntt_fwd_limb_load_n<W, 13>(s, T, mod, load);
  else
    ntt_fwd_limb_load_n<W, 0>(s, T, mod, load);
}

// The canonical value of a forward output left relaxed by ntt_fwd_limb_load (or a canonical one): a
// 32-bit Barrett reduction is exact for any word below 2^32 when q < 2^31.
__device__ __forceinline__ u64 fwd_fin(u32 x, const ModConst& m) { return reduce32(x, m); }
__device__ __forceinline__ u64 fwd_fin(u64 x, const ModConst& m) { return Ar<u64>::fwd_out(x, m); }

// ------------------------------------------------------------ word-typed element arithmetic ----
// Helpers for the kernels' prologues and epilogues: a W-typed multiply, Shoup multiply by a pair
// constant, and the key-switch inner product.
template <typename W>
struct Ew;

template <>
struct Ew<u64> {
  static __device__ __forceinline__ u64 mul(u64 a, u64 b, const ModConst& m) { return mul_mod(a, b, m); }
  static __device__ __forceinline__ u64 shoup_inv(u64 a, const PairConst& p, const ModConst& m) {
    return mul_shoup(a, p.inv_qa, p.inv_qa_sh, m.q);
  }
  // a (q_a mod q_b)
  static __device__ __forceinline__ u64 mul_pc(u64 a, const PairConst& p, const ModConst& m) {
    return mul_mod(a, p.qa_mod_b, m);
  }
  // sum_j d_j * w_j mod q, 128-bit lazy accumulation
  struct Acc {
    Acc128 a{0, 0};
    __device__ __forceinline__ void mac(u64 d, u64 w) { mac128(a, d, w); }
    __device__ __forceinline__ u64 get(const ModConst& m) const { return reduce128(a.hi, a.lo, m); }
  };
};

template <>
struct Ew<u32> {
  static __device__ __forceinline__ u64 mul(u64 a, u64 b, const ModConst& m) {
    return reduce64((u64)(u32)a * (u32)b, m);
  }
  static __device__ __forceinline__ u64 shoup_inv(u64 a, const PairConst& p, const ModConst& m) {
    return shoup32((u32)a, (u32)p.inv_qa, (u32)p.inv_qa_sh32, (u32)m.q);
  }
  static __device__ __forceinline__ u64 mul_pc(u64 a, const PairConst& p, const ModConst& m) {
    return shoup32((u32)a, (u32)p.qa_mod_b, (u32)p.qa_mod_b_sh32, (u32)m.q);
  }
  // products of 31-bit residues are below 2^62; a 64-bit sum with a carry count holds any ell
  struct Acc {
    u64 lo = 0;
    u32 carry = 0;
    __device__ __forceinline__ void mac(u64 d, u64 w) {
      const u64 p = (u64)(u32)d * (u32)w;
      lo += p;
      carry += lo < p;
    }
    // fold a partial sum of products (below 2^64) into the sum
    __device__ __forceinline__ void add64(u64 p) {
      lo += p;
      carry += lo < p;
    }
    __device__ __forceinline__ u64 get(const ModConst& m) const {
      const u64 v = reduce64(lo, m);
      return carry ? reduce64(v + (u64)carry * m.r64, m) : v;
    }
  };
};

// Key-switch inner product sum_j d_j w_j over the digits j < E (E = 0: the level is known only at run
// time), one reduction at the end. 64-bit words: the 128-bit lazy sum. 32-bit words: the products
// (below 2^62) are summed in plain 64-bit registers in groups of four (4 (2^31 - 1)^2 < 2^64), each
// group folded into a carry-counted sum, so with E known a product costs one multiply-add.
template <typename W, int E>
struct KsSum {
  typename Ew<W>::Acc acc;
  __device__ __forceinline__ void mac(u64 d, u64 w, u32) { acc.mac(d, w); }
  __device__ __forceinline__ u64 get(const ModConst& m) const { return acc.get(m); }
};
template <int E>
struct KsSum<u32, E> {
  u64 part = 0;
  typename Ew<u32>::Acc acc;
  __device__ __forceinline__ void mac(u64 d, u64 w, u32 j) {
    part += (u64)(u32)d * (u32)w;
    if ((E == 0 || E > 4) && (j & 3u) == 3u) {
      acc.add64(part);
      part = 0;
    }
  }
  __device__ __forceinline__ u64 get(const ModConst& m) {
    if (E > 0 && E <= 4) return reduce64(part, m);
    acc.add64(part);
    return acc.get(m);
  }
  // The sum unreduced, as lo + c 2^64 (c = 0 when E <= 4); ends the sum like get().
  __device__ __forceinline__ u64 raw(u32& c) {
    if (E > 0 && E <= 4) {
      c = 0;
      return part;
    }
    acc.add64(part);
    c = acc.carry;
    return acc.lo;
  }
};

// Launch geometry of a limb transform: cluster size 2^log_c, threads per CTA, shared memory bytes
// for 8-byte words (u32 limbs use half).
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

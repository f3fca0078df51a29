// Vector x plain matrix with the ModDown taken once, after the sum over rotations (double
// hoisting), for a batch of B requests at level ell over the rotations k = 1..R of one matrix:
//
//   U_b[i] = sum_k (sum_j tau_k(D_j)[i] * gk^(k)_j[b][i]) * d_k[i]      slots i < ell and P
//   A_0[i] = sum_k tau_k(c0)[i] * d_k[i]                                  i < ell
//   out_b[i] = A_b[i] + c_b[i] d_0[i] + (U_b[i] - NTT_i(bal_P(INTT_P(U_b[P])))) * P^-1
//
// k_vecmat_dh_acc is element-wise (no transform inside the rotation loop): one thread owns a few
// elements of one (request, slot i) and walks a chunk of rotations, reading the digits through the
// Galois permutation and each key limb, diagonal and c0 limb once; the grid orders requests fastest
// so that the CTAs sharing a key limb run together, and the slots slowest so that one slot's digits
// stay in the L2 while its element blocks run. k_vecmat_dh_fold sums the chunk partials;
// k_vecmat_dh_moddown finishes (one limb job per request, component and prime).
#include <cuda_runtime.h>

#include "../../include/tcks.h"
#include "context.h"
#include "kernels.h"
#include "dh_acc.cuh"
#include "limb_launch.cuh"
#include "ntt.cuh"

namespace tcks {

namespace {

constexpr u32 kDhThreads = 256;

// CTAs per SM the accumulation is compiled for, and rotations whose loads it keeps in flight (32-bit
// words). The fixed-ring form holds two rotations' operands in registers: from level 6 on that needs
// more than the 80 registers of three CTAs per SM (it spilled), so those levels take two CTAs per SM;
// at level 5 one rotation at a time at three CTAs per SM measured faster than either. Four requests
// per thread take two CTAs per SM.
template <int ELL, int KO, int LOGN, int RPT>
__host__ __device__ constexpr int dh_min_ctas() {
  return KO > 1 ? 3 : LOGN > 0 ? (ELL >= 6 || RPT == 4 ? 2 : 3) : 1;
}
template <typename W, int ELL, int LOGN>
__host__ __device__ constexpr int dh_rot_unroll() {
  return sizeof(W) == 4 && !(LOGN > 0 && ELL == 5) ? 2 : 1;
}


// Thread = EPT elements (stride kDhThreads) x RPT requests of one slot i: the key limbs, the
// diagonal and the Galois index of a rotation are loaded once for the RPT requests.
// ELL > 0 fixes the level at compile time (the digit loop unrolls, its offsets become constants);
// ELL = 0 takes it from the argument.
// KO outputs per request (KO > 1 with RPT = 1): the key-switch sums of a rotation are formed once
// and multiplied by each output's diagonal.
// LOGN > 0 (with ELL > 0) fixes the ring size too, for plans whose keys all sit at level ELL: every key
// and digit stride is then a compile-time constant, so each load is a base plus an immediate offset.
// KEYS_AT = false: the keys share one level above ELL (p.keys_K), a run-time value uniform over the
// launch, so only the key strides are computed.
template <typename W, int EPT, int RPT, int ELL, int KO = 1, int LOGN = 0, bool KEYS_AT = true>
__global__ void __launch_bounds__(kDhThreads, dh_min_ctas<ELL, KO, LOGN, RPT>()) k_vecmat_dh_acc(DevTables T, u32 ell_arg,
                                                               const __grid_constant__ VecmatDhPlan p) {
  static_assert(LOGN == 0 || ELL > 0, "a fixed ring size needs a fixed level");
  const u32 ell = ELL > 0 ? (u32)ELL : ell_arg;
  const u32 log_n = LOGN > 0 ? (u32)LOGN : T.log_n;
  const u64 n = 1ull << log_n;
  const u32 slots = ell + 1;
  const u32 groups = (p.B + RPT - 1) / RPT;
  const u32 eblocks = (u32)((n + kDhThreads * EPT - 1) / (kDhThreads * EPT));
  // Requests fastest (the CTAs sharing a key block run together), then element blocks, then the slot:
  // while the CTAs of slot i run, the working set is that slot's digits of every request and its key
  // limbs, which fits the L2, so each digit limb is read from DRAM once although every element block
  // reads it through a different permutation at every rotation.
  const u32 rg = blockIdx.x % groups;
  const u32 rest = blockIdx.x / groups;
  const u32 eb = rest % eblocks, i = rest / eblocks;
  const u32 chunk = blockIdx.y;
  const u32 mod = i < ell ? i : T.L;
  const ModConst m = T.mods[mod];
  const W* digits[RPT];
  const u64* c0[RPT];
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr) {
    const u32 rq = min(rg * RPT + rr, p.B - 1);  // a short last group repeats a request, never stored
    digits[rr] = reinterpret_cast<const W*>(p.digits) + rq * p.digits_b + (u64)i * n;  // digit j at + j * slots * n
    c0[rr] = p.ct + rq * p.ct_b + (u64)i * n;
  }
  const u32 base = eb * kDhThreads * EPT + threadIdx.x;
  DhAcc<W> u0[EPT][RPT * KO], u1[EPT][RPT * KO], a0[EPT][RPT * KO];
  const u32 r0 = chunk * p.chunk, r1 = min(p.R, r0 + p.chunk);
  const bool unit = p.diag == nullptr;  // a hoisted rotation sum: every diagonal is 1
  constexpr int kRotUnroll = dh_rot_unroll<W, ELL, LOGN>();
#pragma unroll kRotUnroll
  for (u32 r = r0; r < r1; ++r) {
    const KsKey kk = p.keys[r];
    // LOGN > 0: every key at level ELL, or (KEYS_AT = false) at the plan's shared level (checked by the host)
    const u32 kK = LOGN > 0 ? (KEYS_AT ? (u32)ELL : p.keys_K) : kk.K;
    const u32 key_slot = i < ell ? i : kK;
    const u64* dk = unit ? nullptr : p.diag + (u64)(r + 1) * p.diag_stride + (u64)(i < ell ? i : p.p_limb) * n;
    const u64* k0 = kk.key + (u64)key_slot * n;     // digit j's component b at + (2j + b) (K+1) n
    // LOGN > 0 (32-bit words): the key's 32-bit copy, half the bytes (the host checked it exists)
    const u32* k32 = LOGN > 0 ? kk.key32 + (u64)key_slot * n : nullptr;
    const u64 kstep = (u64)(kK + 1) * n;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      const u32 g = base + e * kDhThreads;
      if (g < n) {
        const u32 src = galois_src(g, kk.g, log_n);
        KsSum<W, ELL> s0[RPT], s1[RPT];
#pragma unroll
        for (u32 j = 0; j < ell; ++j) {
          u64 w0, w1;
          if constexpr (LOGN > 0) {
            w0 = k32[2 * j * kstep + g];
            w1 = k32[(2 * j + 1) * kstep + g];
          } else {
            w0 = k0[2 * j * kstep + g];
            w1 = k0[(2 * j + 1) * kstep + g];
          }
#pragma unroll
          for (int rr = 0; rr < RPT; ++rr) {
            const u64 d = digits[rr][(u64)j * slots * n + src];
            s0[rr].mac(d, w0, j);
            s1[rr].mac(d, w1, j);
          }
        }
        constexpr bool kCarry = ELL == 0 || ELL > 4;
        if (unit) {
#pragma unroll
          for (int rr = 0; rr < RPT; ++rr) {
            if constexpr (sizeof(W) == 4) {
              u32 c;
              u64 v = s0[rr].raw(c);
              u0[e][rr].add_wide(v, c);
              v = s1[rr].raw(c);
              u1[e][rr].add_wide(v, c);
            } else {
              u0[e][rr].add(s0[rr].get(m));
              u1[e][rr].add(s1[rr].get(m));
            }
            if (i < ell) a0[e][rr].add(c0[rr][src]);
          }
        } else if (KO == 1) {
          const u64 dv = dk[g];
#pragma unroll
          for (int rr = 0; rr < RPT; ++rr) {
            if constexpr (sizeof(W) == 4) {
              u32 c;
              u64 v = s0[rr].raw(c);
              u0[e][rr].template mac_wide<kCarry>(v, c, dv);
              v = s1[rr].raw(c);
              u1[e][rr].template mac_wide<kCarry>(v, c, dv);
            } else {
              u0[e][rr].mac(s0[rr].get(m), dv);
              u1[e][rr].mac(s1[rr].get(m), dv);
            }
            if (i < ell) a0[e][rr].mac(c0[rr][src], dv);
          }
        } else {
          const u64 v0 = s0[0].get(m), v1 = s1[0].get(m), x0 = i < ell ? c0[0][src] : 0;
#pragma unroll
          for (int o = 0; o < KO; ++o) {
            const u64 dv = dk[(u64)o * p.diag_set + g];
            u0[e][o].mac(v0, dv);
            u1[e][o].mac(v1, dv);
            if (i < ell) a0[e][o].mac(x0, dv);
          }
        }
      }
    }
  }
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const u32 g = base + e * kDhThreads;
#pragma unroll
    for (int rr = 0; rr < RPT * KO; ++rr) {
      const u32 rq = KO == 1 ? rg * RPT + rr : rg;  // KO > 1: rr is the output
      const u32 ro = KO == 1 ? rq : rq * KO + rr;   // index of the partial
      if (g < n && rq < p.B) {
        p.partial[dh_off(ro, chunk, p.chunks, 0, i, ell, log_n) + g] = u0[e][rr].get(m);
        p.partial[dh_off(ro, chunk, p.chunks, 1, i, ell, log_n) + g] = u1[e][rr].get(m);
        if (i < ell) p.partial[dh_off(ro, chunk, p.chunks, 2, i, ell, log_n) + g] = a0[e][rr].get(m);
      }
    }
  }
}

// Launch shape per word type: elements and requests per thread.
constexpr int kEpt32 = 1, kRpt32 = 2, kEpt64 = 1, kRpt64 = 1;

// Calibration in the accumulation's own form (32-bit words, RPT = 2 requests per thread, level ELL,
// one output): per iteration, for both requests, the two key-switch sums over ELL digits (KsSum, no
// reduction), their unreduced products with the diagonal value into the 128-bit carry-chain sums
// (DhAcc::mac_wide) and the c0 product (DhAcc::mac), all from registers. Each of the kernel's loads (a
// digit, two key words, the diagonal, c0) becomes one XOR with the iteration count, so the operands
// change every iteration and the instruction mix matches the kernel's arithmetic plus one issue slot
// per load. One op = one product-accumulate, counted as in the kernel: 2 (2 ELL + 3) per iteration.
template <int ELL>
__global__ void __launch_bounds__(kDhThreads, 1) k_dh_peak(ModConst m, u32 iters, u64* __restrict__ sink) {
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u32 mask = 0x7FFFFFFFu;
  u32 d[2][ELL], w0[ELL], w1[ELL], x[2];
  u32 dv = (u32)(tid * 5 + 3) & mask;
#pragma unroll
  for (int j = 0; j < ELL; ++j) {
    w0[j] = (u32)(tid * 11 + j) & mask;
    w1[j] = (u32)(tid * 17 + j + 5) & mask;
#pragma unroll
    for (int r = 0; r < 2; ++r) d[r][j] = (u32)(tid * 7 + 3 * j + r) & mask;
  }
  x[0] = (u32)(tid * 13) & mask;
  x[1] = (u32)(tid * 19 + 1) & mask;
  DhAcc<u32> u0[2], u1[2], a0[2];
  constexpr bool kCarry = ELL > 4;
  for (u32 it = 0; it < iters; ++it) {
    dv ^= it;
    KsSum<u32, ELL> s0[2], s1[2];
#pragma unroll
    for (int j = 0; j < ELL; ++j) {
      w0[j] ^= it;
      w1[j] ^= it;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        d[r][j] ^= it;
        s0[r].mac(d[r][j], w0[j], (u32)j);
        s1[r].mac(d[r][j], w1[j], (u32)j);
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      u32 c;
      u64 v = s0[r].raw(c);
      u0[r].template mac_wide<kCarry>(v, c, dv);
      v = s1[r].raw(c);
      u1[r].template mac_wide<kCarry>(v, c, dv);
      x[r] ^= it;
      a0[r].mac(x[r], dv);
    }
  }
  u64 h = 0;
#pragma unroll
  for (int r = 0; r < 2; ++r) h ^= u0[r].get(m) ^ u1[r].get(m) ^ a0[r].get(m);
  sink[tid] = h;
}

// Sum of the chunk partials into chunk 0 (in place), every (request, component, slot).
__global__ void k_vecmat_dh_fold(DevTables T, u32 ell, const __grid_constant__ VecmatDhPlan p) {
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 slots = ell + 1;
  const u64 per_rq = 3ull * slots * n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < per_rq * p.B * dh_outs(p);
       e += (u64)gridDim.x * blockDim.x) {
    const u32 rq = (u32)(e / per_rq);
    const u64 o = e - (u64)rq * per_rq;
    const u32 slot = (u32)((o >> log_n) % slots);
    const u64 q = T.mods[slot < ell ? slot : T.L].q;
    u64* base = p.partial + (u64)rq * p.chunks * per_rq + o;
    u64 s = base[0];
    for (u32 c = 1; c < p.chunks; ++c) s = add_mod(s, base[(u64)c * per_rq], q);
    base[0] = s;
  }
}

// out_b[i] = A_b[i] + c_b[i] d_0[i] + (U_b[i] - NTT_i(bal_P(top_b) mod q_i)) * P^-1.
// Limb job = (b * ell + i) * B * outs + request * outs + output; top [2][B * outs][N] holds INTT_P(U_b[P]).
template <typename W, int LC>
__global__ void k_vecmat_dh_moddown(DevTables T, u32 ell, const __grid_constant__ VecmatDhPlan p, const u64* top,
                                    u64* out, u64 out_b, u64 out_o) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 outs = dh_outs(p), bo = p.B * outs;
  const u32 ro = sl.job % bo, bi = sl.job / bo, b = bi / ell, i = bi % ell;
  const u32 rq = ro / outs, o = ro % outs;
  const ModConst mi = T.mods[i];
  const ModConst mp = T.mods[T.L];
  const PairConst pc = T.pairs[(u64)T.L * T.n_mods + i];
  const u64* t = top + ((u64)b * bo + ro) * n + sl.off;
  if constexpr (LC == 0) {  // the lift feeds the first butterfly round directly
    ntt_fwd_limb_load<W>(s, T, i, [&](u32 k) { return lift_balanced_w<W>(t[k], mp.half, pc.qa_mod_b, mi); });
  } else {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) s[sw(k)] = lift_balanced_w<W>(t[k], mp.half, pc.qa_mod_b, mi);
    __syncthreads();
    ntt_fwd_slice<W, LC>(s, T, i, sl.rank);
  }
  const u64* U = p.partial + dh_off(ro, 0, p.chunks, b, i, ell, log_n);
  const u64* A = p.partial + dh_off(ro, 0, p.chunks, 2, i, ell, log_n);
  const u64* cb = p.ct + rq * p.ct_b + ((u64)b * ell + i) * n;
  const u64* d0 = p.diag ? p.diag + (u64)o * p.diag_set + (u64)i * n : nullptr;  // unit diagonals: c_b itself
  u64* dst = out + (out_o ? rq * out_b + o * out_o : ro * out_b) + ((u64)b * ell + i) * n;
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
    const u32 g = sl.off + k;
    u64 v = Ew<W>::shoup_inv(sub_mod(U[g], fwd_fin(s[sw(k)], mi), mi.q), pc, mi);
    v = add_mod(v, d0 ? Ew<W>::mul(cb[g], d0[g], mi) : cb[g], mi.q);
    if (b == 0) v = add_mod(v, A[g], mi.q);
    if (b == 0 && p.addp) v = add_mod(v, p.addp[(u64)i * n + g], mi.q);
    dst[g] = v;
  }
}

static decltype(&k_vecmat_dh_moddown<u64, 0>) const K6_k_vecmat_dh_moddown[6] = TCKS_K6(k_vecmat_dh_moddown);

// The ModDown and the following rescale by q_l (l = ell - 1) as one rounding. Z_b = P (A_b + c_b d_0) +
// U_b over the data limbs (A_b only for b = 0), Z_b[P] = U_b[P].
// Stage 1: the coefficient form of Z_b[l], limb job = b * B * outs + request * outs + output; top2
// [2][B * outs][N].
template <typename W, int LC>
__global__ void k_dh_top_l(DevTables T, u32 ell, const __grid_constant__ VecmatDhPlan p, u64* top2) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 outs = dh_outs(p), bo = p.B * outs;
  const u32 ro = sl.job % bo, b = sl.job / bo, rq = ro / outs, o = ro % outs;
  const u32 l = ell - 1;
  const ModConst m = T.mods[l];
  const PairConst pm = T.pairs[(u64)T.L * T.n_mods + l];  // P mod q_l
  const u64* U = p.partial + dh_off(ro, 0, p.chunks, b, l, ell, log_n);
  const u64* A = p.partial + dh_off(ro, 0, p.chunks, 2, l, ell, log_n);
  const u64* cb = p.ct + rq * p.ct_b + ((u64)b * ell + l) * n;
  const u64* d0 = p.diag ? p.diag + (u64)o * p.diag_set + (u64)l * n : nullptr;
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
    const u32 g = sl.off + k;
    u64 a = d0 ? Ew<W>::mul(cb[g], d0[g], m) : cb[g];
    if (b == 0) a = add_mod(a, A[g], m.q);
    s[sw(k)] = (W)add_mod(U[g], Ew<W>::mul_pc(a, pm, m), m.q);
  }
  __syncthreads();
  ntt_inv_slice<W, LC>(s, T, l, sl.rank);
  u64* dst = top2 + ((u64)b * bo + ro) * n + sl.off;
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) dst[k] = Ar<W>::inv_out(s[sw(k)], m);
}

constexpr u32 kMdBatch = 4;

// Stage 2: out_b[i] = (Z_b[i] - NTT_i([Z_b]_{P q_l} mod q_i)) (P q_l)^-1, i < kp (kp = p.keep, else ell - 1);
// limb job = (b kp + i) * B * outs + request * outs + output; top [2][B * outs][N] holds INTT_P(U_b[P]).
template <typename W, int LC>
__global__ void k_vecmat_dh_moddown_rs(DevTables T, u32 ell, const __grid_constant__ VecmatDhPlan p, const u64* top,
                                       const u64* top2, Crt2 k2, u64* out, u64 out_b, u64 out_o) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 outs = dh_outs(p), bo = p.B * outs, lo = ell - 1, kp = p.keep ? p.keep : lo;
  const u32 ro = sl.job % bo, bi = sl.job / bo, b = bi / kp, i = bi % kp;
  const u32 rq = ro / outs, o = ro % outs;
  const ModConst mi = T.mods[i], ml = T.mods[lo];
  const PairConst pp = T.pairs[(u64)T.L * T.n_mods + i];  // P mod q_i, P^-1 mod q_i
  const PairConst pl = T.pairs[(u64)lo * T.n_mods + i];   // q_l^-1 mod q_i
  const u64* tp = top + ((u64)b * bo + ro) * n + sl.off;
  const u64* tl = top2 + ((u64)b * bo + ro) * n + sl.off;
  if constexpr (LC == 0) {
    ntt_fwd_limb_load<W>(s, T, i, [&](u32 k) { return crt2_lift<sizeof(W) == 4>(tp[k], tl[k], k2, ml, mi); });
  } else {
#pragma unroll 4
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) s[sw(k)] = (W)crt2_lift<sizeof(W) == 4>(tp[k], tl[k], k2, ml, mi);
    __syncthreads();
    ntt_fwd_slice<W, LC>(s, T, i, sl.rank);
  }
  const u64* U = p.partial + dh_off(ro, 0, p.chunks, b, i, ell, log_n);
  const u64* A = p.partial + dh_off(ro, 0, p.chunks, 2, i, ell, log_n);
  const u64* cb = p.ct + rq * p.ct_b + ((u64)b * ell + i) * n;
  const u64* d0 = p.diag ? p.diag + (u64)o * p.diag_set + (u64)i * n : nullptr;
  u64* dst = out + (out_o ? rq * out_b + o * out_o : ro * out_b) + ((u64)b * kp + i) * n;
  // the operands of kMdBatch elements are loaded before any of them is finished (the stores could
  // alias the loads as far as the compiler knows, which would serialise them)
  for (u32 k0 = threadIdx.x; k0 < sl.ns; k0 += kMdBatch * blockDim.x) {
    u64 uv[kMdBatch], cv[kMdBatch], dv[kMdBatch], av[kMdBatch];
#pragma unroll
    for (u32 t = 0; t < kMdBatch; ++t) {
      const u32 k = k0 + t * blockDim.x;
      if (k < sl.ns) {
        const u32 g = sl.off + k;
        uv[t] = U[g];
        cv[t] = cb[g];
        dv[t] = d0 ? d0[g] : 0;
        av[t] = b == 0 ? A[g] : 0;
      }
    }
#pragma unroll
    for (u32 t = 0; t < kMdBatch; ++t) {
      const u32 k = k0 + t * blockDim.x;
      if (k < sl.ns) {
        u64 a = d0 ? Ew<W>::mul(cv[t], dv[t], mi) : cv[t];
        if (b == 0) a = add_mod(a, av[t], mi.q);
        const u64 z = add_mod(uv[t], Ew<W>::mul_pc(a, pp, mi), mi.q);
        const u64 v = sub_mod(z, fwd_fin(s[sw(k)], mi), mi.q);
        dst[sl.off + k] = Ew<W>::shoup_inv(Ew<W>::shoup_inv(v, pp, mi), pl, mi);
      }
    }
  }
}

static decltype(&k_dh_top_l<u64, 0>) const K6_k_dh_top_l[6] = TCKS_K6(k_dh_top_l);
static decltype(&k_vecmat_dh_moddown_rs<u64, 0>) const K6_k_vecmat_dh_moddown_rs[6] = TCKS_K6(k_vecmat_dh_moddown_rs);

}  // namespace

// The level as a template argument up to 8 limbs (every level of the CNN and the 4096x256 product).
// With 32-bit words at N = 2^13 and every key at the plan's level, the ring size is fixed as well; with
// the keys sharing a level above the plan's (two requests per thread, one output), the ring size alone.
static bool dh_fixed_ring(const DevTables& T, u32 ell, const VecmatDhPlan& p) {
  return T.narrow && T.log_n == 13 && p.keys_K == ell && p.keys32 && ell >= 1 && ell <= 8;
}
static bool dh_fixed_ring_keys_above(const DevTables& T, u32 ell, const VecmatDhPlan& p, u32 rpt, u32 outs) {
  return T.narrow && T.log_n == 13 && p.keys_K > ell && p.keys32 && ell >= 1 && ell <= 8 && rpt == 2 && outs == 1;
}

template <typename W, int EPT, int RPT, int KO>
static void dh_acc_launch(dim3 grid, cudaStream_t st, const DevTables& T, u32 ell, const VecmatDhPlan& p) {
  const bool fixed = sizeof(W) == 4 && dh_fixed_ring(T, ell, p);
  constexpr bool kAbove = sizeof(W) == 4 && RPT == 2 && KO == 1;  // the shape with a keys-above form
  const bool above = kAbove && dh_fixed_ring_keys_above(T, ell, p, RPT, KO);
  switch (ell) {
// RPT = 4 exists in the fixed-ring form only (dh_rpt never picks it elsewhere).
#define TCKS_DH_CASE(E)                                                                          \
  case E:                                                                                        \
    if (fixed)                                                                                   \
      k_vecmat_dh_acc<W, EPT, RPT, E, KO, sizeof(W) == 4 ? 13 : 0><<<grid, kDhThreads, 0, st>>>(T, ell, p); \
    else if constexpr (RPT != 4) {                                                               \
      if (above)                                                                                 \
        k_vecmat_dh_acc<W, EPT, RPT, E, KO, kAbove ? 13 : 0, !kAbove><<<grid, kDhThreads, 0, st>>>(T, ell, p); \
      else                                                                                       \
        k_vecmat_dh_acc<W, EPT, RPT, E, KO><<<grid, kDhThreads, 0, st>>>(T, ell, p);           \
    }                                                                                            \
    return;
    TCKS_DH_CASE(1) TCKS_DH_CASE(2) TCKS_DH_CASE(3) TCKS_DH_CASE(4)
    TCKS_DH_CASE(5) TCKS_DH_CASE(6) TCKS_DH_CASE(7) TCKS_DH_CASE(8)
#undef TCKS_DH_CASE
    default:
      if constexpr (RPT != 4) k_vecmat_dh_acc<W, EPT, RPT, 0, KO><<<grid, kDhThreads, 0, st>>>(T, ell, p);
  }
}

// Requests per thread of a plan's launch: 1 with several outputs; with 32-bit words the tuned value 1 or
// 2 everywhere, or else four in the fixed-ring form at the plan's own level (each key word and diagonal
// then serves four requests; two CTAs per SM) -- at levels 4 and 5 by default (tuned 0), at every level
// with tuned 4 -- and two elsewhere (and in the staged form).
static u32 dh_rpt(const DevTables& T, u32 ell, const VecmatDhPlan& p) {
  if (dh_outs(p) > 1) return 1;
  if (!T.narrow) return kRpt64;
  const u32 t = T.dh_rpt;
  if (t == 1 || t == 2) return t;
  if (!dh_bulk_applies(T, ell, p) && dh_fixed_ring(T, ell, p) && (t == 4 || ell == 4 || ell == 5)) return 4;
  return kRpt32;
}

u32 vecmat_dh_base_ctas(const DevTables& T, u32 ell, const VecmatDhPlan& p) {
  const u64 n = 1ull << T.log_n;
  const u32 ept = T.narrow ? kEpt32 : kEpt64, rpt = dh_rpt(T, ell, p);
  const u64 eblocks = (n + kDhThreads * ept - 1) / (kDhThreads * ept);
  return (u32)(eblocks * (ell + 1) * ((p.B + rpt - 1) / rpt));
}

void launch_vecmat_dh_acc(const DevTables& T, u32 ell, const VecmatDhPlan& p, cudaStream_t st) {
  const double n = (double)(1u << T.log_n);
  const double wd = T.narrow ? 0.5 : 1.0;  // digit words in 8-byte units
  const u32 outs = dh_outs(p);
  const bool bulk = dh_bulk_applies(T, ell, p);
  const u32 rpt = dh_rpt(T, ell, p);
  const bool fixed_ring = dh_fixed_ring(T, ell, p) || dh_fixed_ring_keys_above(T, ell, p, rpt, outs);
  const double kw = !bulk && fixed_ring ? 0.5 : 1.0;  // the fixed-ring forms read the keys' 32-bit copies
  const double by = 8.0 * n *
                    ((double)p.B * (wd * ell * (ell + 1.0) + ell) +
                     (double)p.R * (kw * 2.0 * ell * (ell + 1.0) + (p.diag ? ell + 1.0 : 0.0)) +
                     (double)p.B * p.chunks * (3.0 * ell + 2.0));
  if ((outs != 1 && outs != 4) || (outs > 1 && !p.diag))
    fail(TCKS_ERR_UNSUPPORTED, "double-hoisted sums take 1 or 4 outputs per request (4 with diagonals)");
  // product-accumulates per (request, rotation, element): the key-switch sums 2 ell (ell + 1), then per
  // output the two components' and the c0 term's diagonal products (additions for unit diagonals)
  const double ops = (double)p.B * p.R * n * (2.0 * ell * (ell + 1.0) + outs * (2.0 * (ell + 1.0) + ell));
  // profiler tag: level, outputs, unit diagonals (bit 16), staged operands (bit 17), fixed ring size (bit 18),
  // four requests per thread (bit 19)
  Launch L(K_VECMAT_DH, st, by + 8.0 * n * (outs - 1.0) * (p.R * (ell + 1.0) + p.B * p.chunks * (3.0 * ell + 2.0)), ops,
           ell | (outs << 8) | ((p.diag ? 0u : 1u) << 16) | ((bulk ? 1u : 0u) << 17) |
               ((!bulk && fixed_ring ? 1u : 0u) << 18) | ((rpt == 4 ? 1u : 0u) << 19));
  const dim3 grid(vecmat_dh_base_ctas(T, ell, p), p.chunks);
  if (bulk) {
    launch_vecmat_dh_acc_bulk(T, ell, p, rpt, st);
    return;
  }
  if (outs == 4) {
    if (T.narrow)
      dh_acc_launch<u32, 1, 1, 4>(grid, st, T, ell, p);
    else
      dh_acc_launch<u64, 1, 1, 4>(grid, st, T, ell, p);
  } else if (T.narrow) {
    if (rpt == 4)
      dh_acc_launch<u32, kEpt32, 4, 1>(grid, st, T, ell, p);
    else if (rpt == 1)
      dh_acc_launch<u32, kEpt32, 1, 1>(grid, st, T, ell, p);
    else
      dh_acc_launch<u32, kEpt32, kRpt32, 1>(grid, st, T, ell, p);
  } else {
    dh_acc_launch<u64, kEpt64, kRpt64, 1>(grid, st, T, ell, p);
  }
}

void launch_vecmat_dh_fold(const DevTables& T, u32 ell, const VecmatDhPlan& p, cudaStream_t st) {
  if (p.chunks < 2) return;
  const u64 e = (u64)p.B * dh_outs(p) * 3 * (ell + 1) << T.log_n;
  Launch L(K_MULACC, st, 8.0 * (double)e * (p.chunks + 1.0));
  const u32 blocks = (u32)std::min<u64>((e + 255) / 256, 152ull * 16);
  k_vecmat_dh_fold<<<blocks, 256, 0, st>>>(T, ell, p);
}

void launch_vecmat_dh_moddown_rs(const DevTables& T, const HostTables& H, u32 ell, const VecmatDhPlan& p,
                                 const u64* top, u64* top2, u64* out, u64 out_b, cudaStream_t st, u64 out_o) {
  const double n = (double)(1u << T.log_n);
  const double bo = (double)p.B * dh_outs(p);
  {
    Launch L(K_KS_MODDOWN, st, 8.0 * n * bo * 2.0 * 5.0, 2.0 * bo * (0.5 * n * T.log_n + 2.0 * n));
    launch_limb(K6_k_dh_top_l, T.narrow, (u32)(2 * bo), 1, T.log_n, st, T.limb_threads, T, ell, p, top2);
  }
  const Crt2 k2 = crt2_constants(H, T.L, ell - 1);
  const double jobs = 2.0 * (p.keep ? p.keep : ell - 1) * bo;
  Launch L(K_KS_MODDOWN, st, 8.0 * n * jobs * 7.0, jobs * (0.5 * n * T.log_n + 4.0 * n));
  launch_limb(K6_k_vecmat_dh_moddown_rs, T.narrow, (u32)jobs, 1, T.log_n, st, T.limb_threads, T, ell, p,
              (const u64*)top, (const u64*)top2, k2, out, out_b, out_o);
}

void launch_vecmat_dh_moddown(const DevTables& T, u32 ell, const VecmatDhPlan& p, const u64* top, u64* out, u64 out_b,
                              cudaStream_t st, u64 out_o) {
  const double n = (double)(1u << T.log_n);
  const double jobs = 2.0 * ell * p.B * dh_outs(p);
  Launch L(K_KS_MODDOWN, st, 8.0 * n * (jobs * 5.0 + ell * dh_outs(p)), jobs * (0.5 * n * T.log_n + 2.0 * n));
  launch_limb(K6_k_vecmat_dh_moddown, T.narrow, 2 * ell * p.B * dh_outs(p), 1, T.log_n, st, T.limb_threads, T, ell, p,
              top, out, out_b, out_o);
}

}  // namespace tcks

// The product-accumulate rate of the double-hoisted accumulation's own form (k_dh_peak) at level
// `ell` (1..8) on the current device, every SM busy: the ceiling its roofline is read against.
extern "C" tcks_status tcks_calibrate_dh_macs(uint32_t ell, double* per_second) {
  using namespace tcks;
  if (!per_second || ell < 1 || ell > 8) return TCKS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TCKS_ERR_CUDA;
  const u32 blocks = (u32)sms * 8, iters = 2048;
  const u64 total = (u64)kDhThreads * blocks;
  const u64 q = 1073479681ull;  // a 30-bit prime
  ModConst m{};
  m.q = q;
  m.mu64 = ~0ull / q;
  const unsigned __int128 mu = ~(unsigned __int128)0 / q;
  m.mu_hi = (u64)(mu >> 64);
  m.mu_lo = (u64)mu;
  m.r64 = (u64)(((unsigned __int128)1 << 64) % q);
  m.mu32 = (1ull << 32) / q;
  u64* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  double best = 0;
  tcks_status st = TCKS_OK;
  if (cudaMalloc(&sink, total * 8) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess) {
    st = TCKS_ERR_CUDA;
  } else {
    for (int rep = 0; rep < 4 && st == TCKS_OK; ++rep) {
      cudaEventRecord(a, 0);
      switch (ell) {
#define TCKS_DHP(E) \
  case E: k_dh_peak<E><<<blocks, kDhThreads>>>(m, iters, sink); break;
        TCKS_DHP(1) TCKS_DHP(2) TCKS_DHP(3) TCKS_DHP(4) TCKS_DHP(5) TCKS_DHP(6) TCKS_DHP(7) TCKS_DHP(8)
#undef TCKS_DHP
      }
      cudaEventRecord(b, 0);
      if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        st = TCKS_ERR_CUDA;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms > 0) best = std::max(best, (double)total * iters * 2.0 * (2.0 * ell + 3.0) / (ms * 1e-3));
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  *per_second = best;
  return st;
}


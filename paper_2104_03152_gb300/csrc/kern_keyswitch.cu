// Key-switching kernels: ModUp, the inner product with the key and INTT of the special limb, the
// ModDown (alone or merged with the following rescale) with the Galois automorphism folded into the
// inner product's reads, and the fused ModDown + multiply-accumulate of the per-rotation vector x
// plain-matrix product. Limb kernels as in kern_core.cu: one CTA per limb for N <= 2^14, a cluster of
// 2 or 4 CTAs above.
#include <cuda_runtime.h>

#include <string>
#include <type_traits>
#include <utility>

#include "context.h"
#include "kernels.h"
#include "limb_launch.cuh"
#include "ntt.cuh"

namespace tcks {

// Modular butterflies of one length-N transform: (N / 2) log2 N.
static double bfly_per_limb(u32 log_n) { return 0.5 * (double)(1u << log_n) * log_n; }

// Grid of a grid-stride element kernel over elems2 element pairs (at most 16 CTAs per SM).
static u32 ew_blocks(u64 elems2) {
  u64 b = (elems2 + 255) / 256;
  const u64 cap = 152ull * 16;
  return (u32)(b < cap ? (b ? b : 1) : cap);
}

// ------------------------------------------------------------------------ key switching ----
// ModUp (one digit per prime) for a batch (y) of inputs: digit j = bal_{q_j}(x_j) lifted to slot i
// (prime q_i for i < ell, P for i = ell) and NTT'd; digits [batch][ell][ell+1][N] of W-sized words
// (32-bit on chains below 2^31, which halves the bytes every key-switch consumer reads). Slot i == j
// is x_j itself. x_coef holds the inputs' INTT, [batch][ell][N].
template <typename W, int LC>
__global__ void k_modup(DevTables T, const u64* __restrict__ x_ntt, u64 x_stride, const u64* __restrict__ x_coef,
                        u32 ell, u64* __restrict__ digits) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 j = sl.job / (ell + 1), slot = sl.job % (ell + 1);
  W* out = reinterpret_cast<W*>(digits) + ((sl.y * ell + j) * (ell + 1) + slot) * n + sl.off;
  if (slot == j) {
    const u64* in = x_ntt + sl.y * x_stride + (u64)j * n + sl.off;
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) out[k] = (W)in[k];
    return;
  }
  const u32 tmod = slot < ell ? slot : T.L;
  const ModConst mt = T.mods[tmod];
  const u64 half_j = T.mods[j].half;
  const u64 qj_mod_t = T.pairs[(u64)j * T.n_mods + tmod].qa_mod_b;
  const u64* in = x_coef + (sl.y * ell + j) * n + sl.off;
  if constexpr (LC == 0) {
    // the lift feeds the first butterfly round and the last round writes the digit out directly
    ntt_fwd_limb_load_store<W>(
        s, T, tmod, [&](u32 k) { return lift_balanced_w<W>(in[k], half_j, qj_mod_t, mt); },
        [&](u32 base, const W(&x)[8]) {
          W v[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = (W)fwd_fin(x[k], mt);
          if constexpr (sizeof(W) == 4) {
            uint4* o = reinterpret_cast<uint4*>(out + base);
            o[0] = make_uint4(v[0], v[1], v[2], v[3]);
            o[1] = make_uint4(v[4], v[5], v[6], v[7]);
          } else {
            ulonglong2* o = reinterpret_cast<ulonglong2*>(out + base);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = make_ulonglong2(v[2 * k], v[2 * k + 1]);
          }
        });
  } else {
#pragma unroll 4
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) s[sw(k)] = lift_balanced_w<W>(in[k], half_j, qj_mod_t, mt);
    __syncthreads();
    ntt_fwd_slice<W, LC>(s, T, tmod, sl.rank);
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) out[k] = (W)fwd_fin(s[sw(k)], mt);
  }
}

static decltype(&k_modup<u64, 0>) const K6_k_modup[6] = TCKS_K6(k_modup);

void launch_modup(const DevTables& T, const u64* x_ntt, u64 x_stride, u32 count, u32 ell, u64* x_coef_tmp,
                  u64* digits, cudaStream_t st) {
  const u64 n = 1ull << T.log_n;
  launch_ntt(T, true, x_ntt, x_stride, x_coef_tmp, (u64)ell * n, count * ell, 0, ell, st);
  const double wd = T.narrow ? 4.0 : 8.0;  // bytes of a digit word
  Launch L(K_MODUP, st, n * count * (16.0 * ell + wd * ell * (ell + 1)),
           (double)count * ell * ell * bfly_per_limb(T.log_n));
  launch_limb(K6_k_modup, T.narrow, ell * (ell + 1), count, T.log_n, st, T.limb_threads, T, x_ntt, x_stride, (const u64*)x_coef_tmp, ell, digits);
}

// Calls f(std::integral_constant<int, E>) with E = ell for ell <= 8 (E = 0 above), so that a loop over
// the digits inside f unrolls with constant offsets; ell is uniform across the CTA.
template <typename F>
__device__ __forceinline__ void ell_dispatch(u32 ell, F&& f) {
  switch (ell) {
    case 1: f(std::integral_constant<int, 1>{}); return;
    case 2: f(std::integral_constant<int, 2>{}); return;
    case 3: f(std::integral_constant<int, 3>{}); return;
    case 4: f(std::integral_constant<int, 4>{}); return;
    case 5: f(std::integral_constant<int, 5>{}); return;
    case 6: f(std::integral_constant<int, 6>{}); return;
    case 7: f(std::integral_constant<int, 7>{}); return;
    case 8: f(std::integral_constant<int, 8>{}); return;
    default: f(std::integral_constant<int, 0>{});
  }
}

// Inner product of (automorphed) digits with one key component on slot `slot`:
//   sum_j D_j[slot][src] * key_j[b][key_slot][k], lazy accumulation, one reduction.
// E > 0: ell == E known at compile time.
template <typename W, int E = 0>
__device__ __forceinline__ u64 ks_inner(const W* __restrict__ digits, u32 ell_arg, u32 slot, const u64* __restrict__ key,
                                        u32 K, u32 key_slot, u32 b, u32 k, u32 src, u64 n, const ModConst& m) {
  const u32 ell = E > 0 ? (u32)E : ell_arg;
  KsSum<W, E> acc;
#pragma unroll
  for (u32 j = 0; j < ell; ++j) {
    const u64 d = digits[((u64)j * (ell + 1) + slot) * n + src];
    const u64 w = key[(((u64)j * 2 + b) * (K + 1) + key_slot) * n + k];
    acc.mac(d, w, j);
  }
  return acc.get(m);
}

// Stage 1: u_b[P] = sum_j tau_g(D_j)[P] * key_j[b][P], then INTT mod P -> top. Limb job = b * B +
// request (requests fastest, so that the CTAs reading one key limb run together and share it through
// L2), entry y = rotation.
template <typename W, int LC>
__global__ void k_ks_inner_p(DevTables T, u32 ell, const __grid_constant__ KsPlan plan) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  if (sl.y >= plan.R) return;
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 rq = sl.job % plan.B, r = (u32)sl.y;
  const u64 yy = (u64)r * plan.B + rq;  // entry of the P-limb scratch [R][B][2][N]
  const KsKey kk = plan.keys[r];
  const W* digits = reinterpret_cast<const W*>(plan.digits) + rq * plan.digits_b;
  const u32 b = sl.job / plan.B;
  const ModConst mp = T.mods[T.L];
  ell_dispatch(ell, [&](auto E) {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
      const u32 g = sl.off + k;
      const u32 src = kk.g == 1 ? g : galois_src(g, kk.g, log_n);
      s[sw(k)] = (W)ks_inner<W, decltype(E)::value>(digits, ell, ell, kk.key, kk.K, kk.K, b, g, src, n, mp);
    }
  });
  __syncthreads();
  ntt_inv_slice<W, LC>(s, T, T.L, sl.rank);
  u64* top = plan.top + (yy * 2 + b) * n + sl.off;
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) top[k] = Ar<W>::inv_out(s[sw(k)], mp);
}

// Stage 2 (ModDown): out_b[i] = (u_b[i] - NTT_i(bal_P(top_b) mod q_i)) * P^-1 + addend_b[i].
// Limb job = (b * ell + i) * B + request (requests fastest), entry y = rotation.
template <typename W, int LC>
__global__ void k_ks_moddown(DevTables T, u32 ell, const __grid_constant__ KsPlan plan) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  if (sl.y >= plan.R) return;
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 rq = sl.job % plan.B, r = (u32)sl.y;
  const u64 yy = (u64)r * plan.B + rq;
  const KsKey kk = plan.keys[r];
  const W* digits = reinterpret_cast<const W*>(plan.digits) + rq * plan.digits_b;
  const u32 bi = sl.job / plan.B, b = bi / ell, i = bi % ell;
  const ModConst mi = T.mods[i];
  const ModConst mp = T.mods[T.L];
  const PairConst pc = T.pairs[(u64)T.L * T.n_mods + i];
  const u64* top = plan.top + (yy * 2 + b) * n + sl.off;
  if constexpr (LC == 0) {
    ntt_fwd_limb_load<W>(s, T, i, [&](u32 k) { return lift_balanced_w<W>(top[k], mp.half, pc.qa_mod_b, mi); });
  } else {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) s[sw(k)] = lift_balanced_w<W>(top[k], mp.half, pc.qa_mod_b, mi);
    __syncthreads();
    ntt_fwd_slice<W, LC>(s, T, i, sl.rank);
  }
  const u64* add = b == 0 ? (plan.add0 ? plan.add0 + rq * plan.add0_b : nullptr)
                          : (plan.add1 ? plan.add1 + rq * plan.add1_b : nullptr);
  const u64* addx = plan.addx ? plan.addx + rq * plan.addx_b + ((u64)b * ell + i) * n : nullptr;
  const u64* addp = b == 0 && plan.addp ? plan.addp + (u64)i * n : nullptr;
  u64* dst = plan.out + rq * plan.out_b + r * plan.out_r + ((u64)b * ell + i) * n;
  ell_dispatch(ell, [&](auto E) {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
      const u32 g = sl.off + k;
      const u32 src = kk.g == 1 ? g : galois_src(g, kk.g, log_n);
      const u64 u = ks_inner<W, decltype(E)::value>(digits, ell, i, kk.key, kk.K, i, b, g, src, n, mi);
      u64 v = Ew<W>::shoup_inv(sub_mod(u, fwd_fin(s[sw(k)], mi), mi.q), pc, mi);
      if (add) v = add_mod(v, add[(u64)i * n + (plan.add_perm ? src : g)], mi.q);
      if (addx) v = add_mod(v, addx[g], mi.q);
      if (addp) v = add_mod(v, addp[g], mi.q);
      dst[g] = v;
    }
  });
}

// Relinearization with its ModDown and the following rescale as one rounding (R = 1, no automorphism).
// Stage 1: per (request, component b) the coefficient forms of the two limbs the rounding drops:
// which = 0: u_b[P]; which = 1: u_b[l] + P add_b[l], l = ell - 1. Limb job = ((b B + rq) 2 + which);
// top [B][2][N] and top2 [B][2][N].
template <typename W, int LC>
__global__ void k_ks_top_rs(DevTables T, u32 ell, const __grid_constant__ KsPlan plan, u64* top2) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 which = sl.job & 1u, br = sl.job >> 1, b = br / plan.B, rq = br % plan.B;
  const u32 l = ell - 1;
  const u32 slot = which ? l : ell, mod = which ? l : T.L;
  const KsKey kk = plan.keys[0];
  const W* digits = reinterpret_cast<const W*>(plan.digits) + rq * plan.digits_b;
  const ModConst m = T.mods[mod];
  const PairConst pm = T.pairs[(u64)T.L * T.n_mods + l];  // P mod q_l
  const u64* add = b == 0 ? plan.add0 + rq * plan.add0_b : plan.add1 + rq * plan.add1_b;
  ell_dispatch(ell, [&](auto E) {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
      const u32 g = sl.off + k;
      u64 v = ks_inner<W, decltype(E)::value>(digits, ell, slot, kk.key, kk.K, which ? l : kk.K, b, g, g, n, m);
      if (which) v = add_mod(v, Ew<W>::mul_pc(add[(u64)l * n + g], pm, m), m.q);
      s[sw(k)] = (W)v;
    }
  });
  __syncthreads();
  ntt_inv_slice<W, LC>(s, T, mod, sl.rank);
  u64* dst = (which ? top2 : plan.top) + ((u64)rq * 2 + b) * n + sl.off;
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) dst[k] = Ar<W>::inv_out(s[sw(k)], m);
}

// Stage 2: out_b[i] = (u_b[i] + P add_b[i] - NTT_i([Z]_{P q_l} mod q_i)) (P q_l)^-1, i < ell - 1.
// Limb job = (b (ell - 1) + i) B + rq; out + rq out_b receives [2][ell-1][N].
template <typename W, int LC>
__global__ void k_ks_moddown_rs(DevTables T, u32 ell, const __grid_constant__ KsPlan plan, const u64* top2, Crt2 k2) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 lo = ell - 1;
  const u32 rq = sl.job % plan.B, bi = sl.job / plan.B, b = bi / lo, i = bi % lo;
  const KsKey kk = plan.keys[0];
  const W* digits = reinterpret_cast<const W*>(plan.digits) + rq * plan.digits_b;
  const ModConst mi = T.mods[i], mp = T.mods[T.L], ml = T.mods[lo];
  const PairConst pp = T.pairs[(u64)T.L * T.n_mods + i];  // P mod q_i, P^-1 mod q_i
  const PairConst pl = T.pairs[(u64)lo * T.n_mods + i];   // q_l^-1 mod q_i
  (void)mp;
  const u64* tp = plan.top + ((u64)rq * 2 + b) * n + sl.off;
  const u64* tl = top2 + ((u64)rq * 2 + b) * n + sl.off;
  if constexpr (LC == 0) {
    ntt_fwd_limb_load<W>(s, T, i, [&](u32 k) { return crt2_lift<sizeof(W) == 4>(tp[k], tl[k], k2, ml, mi); });
  } else {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) s[sw(k)] = (W)crt2_lift<sizeof(W) == 4>(tp[k], tl[k], k2, ml, mi);
    __syncthreads();
    ntt_fwd_slice<W, LC>(s, T, i, sl.rank);
  }
  const u64* add = b == 0 ? plan.add0 + rq * plan.add0_b : plan.add1 + rq * plan.add1_b;
  u64* dst = plan.out + rq * plan.out_b + ((u64)b * lo + i) * n;
  ell_dispatch(ell, [&](auto E) {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
      const u32 g = sl.off + k;
      const u64 u = ks_inner<W, decltype(E)::value>(digits, ell, i, kk.key, kk.K, i, b, g, g, n, mi);
      const u64 z = add_mod(u, Ew<W>::mul_pc(add[(u64)i * n + g], pp, mi), mi.q);
      const u64 v = sub_mod(z, fwd_fin(s[sw(k)], mi), mi.q);
      dst[g] = Ew<W>::shoup_inv(Ew<W>::shoup_inv(v, pp, mi), pl, mi);
    }
  });
}

static decltype(&k_ks_top_rs<u64, 0>) const K6_k_ks_top_rs[6] = TCKS_K6(k_ks_top_rs);
static decltype(&k_ks_moddown_rs<u64, 0>) const K6_k_ks_moddown_rs[6] = TCKS_K6(k_ks_moddown_rs);

Crt2 crt2_constants(const HostTables& H, u32 L, u32 l) {
  using u128 = unsigned __int128;
  Crt2 k{};
  k.P = H.chain[L];
  k.ql = H.chain[l];
  k.l = l;
  // P^-1 mod q_l by Fermat
  u64 base = k.P % k.ql, e = k.ql - 2, r = 1;
  while (e) {
    if (e & 1) r = (u64)((u128)r * base % k.ql);
    base = (u64)((u128)base * base % k.ql);
    e >>= 1;
  }
  k.pinv_l = r;
  k.pinv_sh32 = k.ql < (1ull << 31) ? (u32)(((u128)r << 32) / k.ql) : 0;
  const u128 pq = (u128)k.P * k.ql, half = (pq - 1) / 2;
  k.pq_lo = (u64)pq;
  k.pq_hi = (u64)(pq >> 64);
  k.half_lo = (u64)half;
  k.half_hi = (u64)(half >> 64);
  return k;
}

void launch_relin_rescale(const DevTables& T, const HostTables& H, u32 ell, const KsPlan& plan, u64* top2,
                          cudaStream_t st) {
  const u64 n = 1ull << T.log_n;
  {
    Launch L(K_KS_P, st, 8.0 * n * (plan.B * 2.0 * (ell + 2.0)), 4.0 * plan.B * ((double)ell * n + bfly_per_limb(T.log_n)));
    launch_limb(K6_k_ks_top_rs, T.narrow, 4 * plan.B, 1, T.log_n, st, T.limb_threads, T, ell, plan, top2);
  }
  const Crt2 k2 = crt2_constants(H, T.L, ell - 1);
  Launch L(K_KS_MODDOWN, st, 8.0 * n * plan.B * (ell * ell + 2.0 * ell + 4.0 * (ell - 1.0)),
           2.0 * (ell - 1.0) * plan.B * ((ell + 2.0) * n + bfly_per_limb(T.log_n)));
  launch_limb(K6_k_ks_moddown_rs, T.narrow, 2 * (ell - 1) * plan.B, 1, T.log_n, st, T.limb_threads, T, ell, plan,
              (const u64*)top2, k2);
}

// Algorithmic bytes of a plan: distinct digit sets and keys once, scratch and outputs once.
static void ks_plan_bytes(const KsPlan& p, u32 ell, u32 log_n, bool narrow, double* inner, double* moddown) {
  const double n = (double)(1u << log_n);
  const double jobs = (double)p.B * p.R;
  const double digit_sets = (p.digits_b ? p.B : 1) * (narrow ? 0.5 : 1.0);  // in 8-byte units
  const double key_sets = p.R;  // each rotation index has its own key, shared by the batch
  const double adds = (p.add0 ? (p.add0_b ? p.B : 1) : 0) + (p.add1 ? (p.add1_b ? p.B : 1) : 0);
  *inner = 8.0 * n * (digit_sets * ell + key_sets * 2.0 * ell + 2.0 * jobs);
  *moddown =
      8.0 * n * (digit_sets * ell * ell + key_sets * 2.0 * ell * ell + 2.0 * jobs + adds * ell + 2.0 * ell * jobs);
}

static decltype(&k_ks_inner_p<u64, 0>) const K6_k_ks_inner_p[6] = TCKS_K6(k_ks_inner_p);

void launch_ks_inner_p(const DevTables& T, u32 ell, const KsPlan& plan, cudaStream_t st) {
  const u64 jobs = (u64)plan.B * plan.R;
  if (!jobs) return;
  double bi, bm;
  ks_plan_bytes(plan, ell, T.log_n, T.narrow != 0, &bi, &bm);
  Launch L(K_KS_P, st, bi, 2.0 * jobs * ((double)ell * (1u << T.log_n) + bfly_per_limb(T.log_n)));
  launch_limb(K6_k_ks_inner_p, T.narrow, 2 * plan.B, plan.R, T.log_n, st, T.limb_threads, T, ell, plan);
}

static decltype(&k_ks_moddown<u64, 0>) const K6_k_ks_moddown[6] = TCKS_K6(k_ks_moddown);

void launch_keyswitch(const DevTables& T, u32 ell, const KsPlan& plan, cudaStream_t st) {
  const u64 jobs = (u64)plan.B * plan.R;
  if (!jobs) return;
  launch_ks_inner_p(T, ell, plan, st);
  double bi, bm;
  ks_plan_bytes(plan, ell, T.log_n, T.narrow != 0, &bi, &bm);
  Launch L(K_KS_MODDOWN, st, bm,
           2.0 * ell * jobs * ((ell + 1.0) * (1u << T.log_n) + bfly_per_limb(T.log_n)));
  launch_limb(K6_k_ks_moddown, T.narrow, 2 * ell * plan.B, plan.R, T.log_n, st, T.limb_threads, T, ell, plan);
}

// -------------------------------------------------- vector x plain matrix: fused ModDown + MAC ----
// For request rq and the rotations r of this CTA's chunk (step k = r + 1): the rotated ciphertext
// rot_k = (tau(c0) + ModDown(u_0), ModDown(u_1)) is multiplied by the diagonal d_k and summed into
// a per-chunk partial [B][chunks][2][ell][N]. Limb job = chunk * 2 * ell + b * ell + i.
// Two accumulation modes: up to 8192-element slices thread t keeps the sums of elements
// t + e * blockDim.x (e < 16) in registers and stores them once; for 16384-element slices, whose
// register accumulators would not fit a CTA's register file with 64-bit words, every rotation adds
// into the partial in place (each thread owns the same elements throughout, the CTA's partial is
// L2-resident).
constexpr int kVmEpt = 16;
static bool vecmat_in_place(u32 log_n) { return (log_n > 14 ? 14 : log_n) >= 14; }
static u32 vecmat_threads(u32 log_n) {
  const u32 ns = 1u << (log_n > 14 ? 14 : log_n);
  if (vecmat_in_place(log_n)) return 512;
  return ns / kVmEpt < 32 ? 32 : ns / kVmEpt;
}

// The rotated-and-multiplied element g of rotation r: (tau(c0) + ModDown(u_b))[i][g] * d_k[i][g].
template <typename W>
__device__ __forceinline__ u64 vecmat_term(const W* s, u32 k, u32 g, const KsKey& kk, const W* digits, u32 ell, u32 i,
                                           u32 b, u64 n, u32 log_n, const u64* c0, const u64* dk, const ModConst& mi,
                                           const PairConst& pc) {
  const u32 src = galois_src(g, kk.g, log_n);
  const u64 u = ks_inner<W>(digits, ell, i, kk.key, kk.K, i, b, g, src, n, mi);
  u64 v = Ew<W>::shoup_inv(sub_mod(u, Ar<W>::fwd_out(s[sw(k)], mi), mi.q), pc, mi);
  if (b == 0) v = add_mod(v, c0[(u64)i * n + src], mi.q);
  return Ew<W>::mul(v, dk[g], mi);
}

template <typename W, int LC, bool IN_PLACE>
__device__ __forceinline__ void vecmat_acc_body(W* s, const DevTables& T, u32 ell, const VecmatPlan& plan) {
  const Slice sl = slice_of<LC>(T);
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 rq = sl.job % plan.B;  // requests fastest: CTAs reading the same keys run together
  const u32 job = sl.job / plan.B;
  const u32 chunk = job / (2 * ell), bi = job % (2 * ell);
  const u32 b = bi / ell, i = bi % ell;
  const ModConst mi = T.mods[i];
  const ModConst mp = T.mods[T.L];
  const PairConst pc = T.pairs[(u64)T.L * T.n_mods + i];
  const W* digits = reinterpret_cast<const W*>(plan.digits) + rq * plan.digits_b;
  const u64* c0 = plan.ct + rq * plan.ct_b;  // component 0, [ell][N]
  u64* dst = plan.partial + rq * plan.partial_b + (((u64)chunk * 2 + b) * ell + i) * n + sl.off;
  const u32 r0 = chunk * plan.chunk;
  const u32 r1 = min(plan.R, r0 + plan.chunk);
  W acc[IN_PLACE ? 1 : kVmEpt];
  if (!IN_PLACE) {
#pragma unroll
    for (int e = 0; e < kVmEpt; ++e) acc[e] = 0;
  } else if (!plan.accumulate && r0 >= r1) {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) dst[k] = 0;  // an empty chunk still defines its partial
  }
  for (u32 r = r0; r < r1; ++r) {
    const KsKey kk = plan.keys[r];
    const u64* top = plan.top + (((u64)r * plan.B + rq) * 2 + b) * n + sl.off;
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) s[sw(k)] = lift_balanced_w<W>(top[k], mp.half, pc.qa_mod_b, mi);
    __syncthreads();
    ntt_fwd_slice<W, LC>(s, T, i, sl.rank);
    const u64* dk = plan.diag + (u64)(r + 1) * plan.diag_stride + (u64)i * n;
    if (IN_PLACE) {
      const bool overwrite = r == r0 && !plan.accumulate;
      for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
        const u64 t = vecmat_term<W>(s, k, sl.off + k, kk, digits, ell, i, b, n, log_n, c0, dk, mi, pc);
        dst[k] = overwrite ? t : add_mod(dst[k], t, mi.q);
      }
    } else {
#pragma unroll
      for (int e = 0; e < kVmEpt; ++e) {
        const u32 k = threadIdx.x + e * blockDim.x;
        if (k < sl.ns)
          acc[e] = (W)add_mod(acc[e], vecmat_term<W>(s, k, sl.off + k, kk, digits, ell, i, b, n, log_n, c0, dk, mi, pc),
                              mi.q);
      }
    }
    __syncthreads();  // s is refilled for the next rotation
  }
  if (!IN_PLACE) {
#pragma unroll
    for (int e = 0; e < kVmEpt; ++e) {
      const u32 k = threadIdx.x + e * blockDim.x;
      if (k < sl.ns) dst[k] = plan.accumulate ? add_mod(dst[k], acc[e], mi.q) : acc[e];
    }
  }
}

// 32-bit words: two 512-thread CTAs per SM (registers capped at 64) to hide the L2 latency of the
// digit, key and diagonal reads behind the other CTA's transform.
template <typename W, int LC>
__global__ void __launch_bounds__(512, (sizeof(W) == 4 && LC == 0) ? 2 : 1)
    k_vecmat_acc(DevTables T, u32 ell, const __grid_constant__ VecmatPlan plan) {
  TCKS_SMEM(W);
  vecmat_acc_body<W, LC, false>(s, T, ell, plan);
}
template <typename W, int LC>
__global__ void __launch_bounds__(512, 1) k_vecmat_acc_ip(DevTables T, u32 ell, const __grid_constant__ VecmatPlan plan) {
  TCKS_SMEM(W);
  vecmat_acc_body<W, LC, true>(s, T, ell, plan);
}

// out[rq] = ct[rq] * d_0 + sum over chunks of partial[rq][chunk]; out [B][2][ell][N].
__global__ void k_vecmat_reduce(DevTables T, u32 ell, const __grid_constant__ VecmatPlan plan, u64* __restrict__ out) {
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u64 per_comp = (u64)ell * n, per_ct = 2 * per_comp;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < per_ct * plan.B; e += (u64)gridDim.x * blockDim.x) {
    const u64 rq = e / per_ct, o = e - rq * per_ct;
    const u64 lo_off = o % per_comp;  // offset inside the component
    const ModConst m = T.mods[lo_off >> log_n];
    Acc128 a{0, 0};
    mac128(a, plan.ct[rq * plan.ct_b + o], plan.diag[lo_off]);
    for (u32 c = 0; c < plan.chunks; ++c) {
      const u64 v = plan.partial[rq * plan.partial_b + c * per_ct + o];
      const u64 lo = a.lo + v;
      a.hi += lo < v;
      a.lo = lo;
    }
    out[rq * per_ct + o] = reduce128(a.hi, a.lo, m);
  }
}

static decltype(&k_vecmat_acc<u64, 0>) const K6_k_vecmat_acc[6] = TCKS_K6(k_vecmat_acc);
static decltype(&k_vecmat_acc_ip<u64, 0>) const K6_k_vecmat_acc_ip[6] = TCKS_K6(k_vecmat_acc_ip);

// CTAs of k_vecmat_acc the whole GPU holds at once (SMs x resident CTAs per SM) for this chain.
u32 vecmat_slots(const DevTables& T) {
  const LimbShape sh = limb_shape(T.log_n);
  const u32 idx = (T.narrow ? 3 : 0) + sh.log_c;
  const void* k = vecmat_in_place(T.log_n) ? (const void*)K6_k_vecmat_acc_ip[idx] : (const void*)K6_k_vecmat_acc[idx];
  const size_t smem = T.narrow ? sh.smem / 2 : sh.smem;
  ensure_smem(k, smem);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (int)vecmat_threads(T.log_n), smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return (u32)(sms * per_sm) >> sh.log_c;  // clusters of 2^log_c CTAs share the count
}

void launch_vecmat_acc(const DevTables& T, u32 ell, const VecmatPlan& plan, cudaStream_t st) {
  const double n = (double)(1u << T.log_n);
  // per (request, rotation): the P-limb scratch; per rotation: key limbs and diagonal; per request:
  // digits, c0 and the partial outputs
  const double wd = T.narrow ? 0.5 : 1.0;  // digit words in 8-byte units
  const double by = 8.0 * n *
                    ((double)plan.B * plan.R * 2.0 + plan.R * (2.0 * ell * ell + ell) + plan.B * (wd * ell * ell + ell) +
                     (double)plan.B * plan.chunks * 2.0 * ell * (plan.accumulate ? 2.0 : 1.0));
  Launch L(K_VECMAT, st, by,
           (double)plan.B * plan.R * 2.0 * ell * ((ell + 2.0) * n + bfly_per_limb(T.log_n)));
  if (vecmat_in_place(T.log_n))
    launch_limb(K6_k_vecmat_acc_ip, T.narrow, plan.chunks * 2 * ell * plan.B, 1, T.log_n, st, vecmat_threads(T.log_n),
                T, ell, plan);
  else
    launch_limb(K6_k_vecmat_acc, T.narrow, plan.chunks * 2 * ell * plan.B, 1, T.log_n, st, vecmat_threads(T.log_n), T,
                ell, plan);
}

void launch_vecmat_reduce(const DevTables& T, u32 ell, const VecmatPlan& plan, u64* out, cudaStream_t st) {
  const double n = (double)(1u << T.log_n);
  const u64 e = (u64)plan.B * 2 * ell << T.log_n;
  Launch L(K_MULACC, st, 8.0 * ((double)e * (2.0 + plan.chunks) + ell * n));
  k_vecmat_reduce<<<ew_blocks(e / 2 + 1), 256, 0, st>>>(T, ell, plan, out);
}



// Largest CTA size every limb kernel of this file accepts for the word type and cluster split.
u32 limb_threads_cap_keyswitch(bool narrow, u32 log_c) {
  const u32 i = (narrow ? 3 : 0) + log_c;
  auto cap_of = [](const void* k) -> u32 {
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, k) != cudaSuccess) return 0;
    return (u32)a.maxThreadsPerBlock;
  };
  u32 cap = 1024;
  for (u32 t : {cap_of((const void*)K6_k_modup[i]), cap_of((const void*)K6_k_ks_inner_p[i]),
                cap_of((const void*)K6_k_ks_moddown[i]), cap_of((const void*)K6_k_ks_top_rs[i]),
                cap_of((const void*)K6_k_ks_moddown_rs[i])})
    cap = t < cap ? t : cap;
  return cap;
}

}  // namespace tcks

// Hybrid key switching: digits of `alpha` data primes and K special primes P = p_0 ... p_{K-1}
// (Han and Ki, CT-RSA 2020, on the full-RNS CKKS of Cheon, Han, Kim, Kim and Song, SAC 2018).
//
// At level ell digit j covers the data primes G_j = {q_i : j alpha <= i < min((j+1) alpha, ell)}
// with product Q_j; dnum = ceil(ell / alpha) digits. Chain order: q_0..q_{L-1}, p_0..p_{K-1}.
//   ModUp:    y_i = x_i (Q_j/q_i)^-1 mod q_i (coefficient form, k_hyb_scale), then for every slot t
//             outside G_j  D_j[t] = sum_{i in G_j} bal(y_i) (Q_j/q_i) mod q_t  and its NTT
//             (k_modup_hyb, the exact balanced base conversion); slots inside G_j copy x_t.
//   inner:    u_b[t] = sum_j tau_g(D_j)[t] key_j[b][t] over the data slots and the special slots.
//   ModDown:  w_k = INTT(u_b[p_k]) (P/p_k)^-1 mod p_k (k_ks_hyb_p),
//             out_b[i] = (u_b[i] - NTT_i(sum_k bal(w_k) (P/p_k) mod q_i)) P^-1 + addend (k_ks_hyb_moddown).
// The balanced terms make the conversions commute with the Galois automorphism (an odd function of
// each coefficient), so a hoisted rotation equals a plain one bit for bit. With alpha = 1 and K = 1 the
// arithmetic is exactly that of the one-prime key switch in kern_core.cu.
//
// Layouts: digits [B][dnum][ell + K][N] (W words), key of level Kt [dnum(Kt)][2][Kt + K][N], P-limb
// scratch top [R][B][2][K][N] (u64, coefficient form, already times (P/p_k)^-1).
#include <cuda_runtime.h>

#include "kernels.h"
#include "limb_launch.cuh"
#include "ntt.cuh"

namespace tcks {

namespace {

__device__ __forceinline__ u32 hyb_chain(u32 t, u32 data, u32 L) { return t < data ? t : L + (t - data); }

// (hi:lo) - cnt * c mod q with c < q < 2^61 and cnt <= 8 (so cnt * c < 2^64): the lazily summed
// conversion minus its balancing correction (each negative balanced term subtracts q_i (Q/q_i) = Q).
__device__ __forceinline__ u64 conv_finish(const Acc128& a, u32 cnt, u64 c, const ModConst& m) {
  return sub_mod(reduce128(a.hi, a.lo, m), reduce64((u64)cnt * c, m), m.q);
}

}  // namespace

// y = x * (Q_j / q_i)^-1 mod q_i for every coefficient limb of `count` inputs [count][ell][N] (in place);
// limb i belongs to digit i / alpha, whose group at level ell has min(alpha, ell - j alpha) primes.
__global__ void k_hyb_scale(DevTables T, HybTables H, u64* __restrict__ coef, u32 ell, u32 count) {
  const u32 log_n = T.log_n;
  const u64 total = ((u64)count * ell) << log_n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
    const u32 i = (u32)((e >> log_n) % ell);
    const u32 j = i / H.alpha, r = min(H.alpha, ell - j * H.alpha), mbr = i - j * H.alpha;
    const u64* c = H.up_inv + (((u64)j * H.alpha + (r - 1)) * H.alpha + mbr) * 2;
    coef[e] = mul_shoup(coef[e], c[0], c[1], T.mods[i].q);
  }
}

void launch_hyb_scale(const DevTables& T, const HybTables& H, u64* coef, u32 ell, u32 count, cudaStream_t st) {
  const u64 e = ((u64)count * ell) << T.log_n;
  Launch L(K_MODUP, st, 16.0 * e, (double)e);
  u64 blocks = (e + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  k_hyb_scale<<<(u32)blocks, 256, 0, st>>>(T, H, coef, ell, count);
}

// Digit j, slot t of request y: limb job = j * (ell + K) + t.
template <typename W, int LC>
__global__ void k_modup_hyb(DevTables T, HybTables H, const u64* __restrict__ x_ntt, u64 x_stride,
                            const u64* __restrict__ y_coef, u32 ell, u64* __restrict__ digits) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 S = ell + H.K, dn = (ell + H.alpha - 1) / H.alpha;
  const u32 j = sl.job / S, t = sl.job % S;
  W* out = reinterpret_cast<W*>(digits) + ((sl.y * dn + j) * S + t) * n + sl.off;
  const u32 g0 = j * H.alpha, r = min(H.alpha, ell - g0);
  if (t >= g0 && t < g0 + r) {  // a prime of the digit itself: its own residues
    const u64* in = x_ntt + sl.y * x_stride + (u64)t * n + sl.off;
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) out[k] = (W)in[k];
    return;
  }
  const u32 l = hyb_chain(t, ell, T.L);
  const ModConst mt = T.mods[l];
  const u64 vidx = (u64)j * H.alpha + (r - 1);  // the group variant (digit, size)
  const u64* conv = H.up_conv + vidx * H.alpha * T.n_mods;
  const u64 qg = H.up_qg[vidx * T.n_mods + l];
  const u64* y = y_coef + (sl.y * ell + g0) * n + sl.off;
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
    Acc128 a{0, 0};
    u32 neg = 0;
    for (u32 m = 0; m < r; ++m) {
      const u64 v = y[(u64)m * n + k];
      mac128(a, v, conv[(u64)m * T.n_mods + l]);
      neg += v > T.mods[g0 + m].half;
    }
    s[sw(k)] = (W)conv_finish(a, neg, qg, mt);
  }
  __syncthreads();
  ntt_fwd_slice<W, LC>(s, T, l, sl.rank);
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) out[k] = (W)Ar<W>::fwd_out(s[sw(k)], mt);
}

static decltype(&k_modup_hyb<u64, 0>) const K6_k_modup_hyb[6] = TCKS_K6(k_modup_hyb);

void launch_modup_hyb(const DevTables& T, const HybTables& H, const u64* x_ntt, u64 x_stride, u32 count, u32 ell,
                      u64* y_coef_tmp, u64* digits, cudaStream_t st) {
  const u64 n = 1ull << T.log_n;
  launch_ntt(T, true, x_ntt, x_stride, y_coef_tmp, (u64)ell * n, count * ell, 0, ell, st);
  launch_hyb_scale(T, H, y_coef_tmp, ell, count, st);
  const u32 dn = (ell + H.alpha - 1) / H.alpha, S = ell + H.K;
  const double wd = T.narrow ? 4.0 : 8.0;
  const double converted = (double)dn * S - ell;  // limbs that are converted and transformed
  Launch L(K_MODUP, st, n * count * (16.0 * ell + wd * dn * S),
           (double)count * converted * (0.5 * n * T.log_n + (double)H.alpha * n));
  launch_limb(K6_k_modup_hyb, T.narrow, dn * S, count, T.log_n, st, T.limb_threads, T, H, x_ntt, x_stride,
              (const u64*)y_coef_tmp, ell, digits);
}

// Inner product on special slot k of request rq, rotation r, component b; then its INTT and the factor
// (P / p_k)^-1. Limb job = (b K + k) B + rq, entry y = rotation.
template <typename W, int LC>
__global__ void k_ks_hyb_p(DevTables T, HybTables H, u32 ell, const __grid_constant__ KsPlan plan) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  if (sl.y >= plan.R) return;
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 rq = sl.job % plan.B, bk = sl.job / plan.B, b = bk / H.K, k = bk % H.K, r = (u32)sl.y;
  const KsKey kk = plan.keys[r];
  const u32 S = ell + H.K, KS = kk.K + H.K, dn = (ell + H.alpha - 1) / H.alpha;
  const u32 l = T.L + k;
  const ModConst mp = T.mods[l];
  const W* dg = reinterpret_cast<const W*>(plan.digits) + rq * plan.digits_b + (u64)(ell + k) * n;
  const u64* key = kk.key + ((u64)b * KS + kk.K + k) * n;
  for (u32 e = threadIdx.x; e < sl.ns; e += blockDim.x) {
    const u32 g = sl.off + e;
    const u32 src = kk.g == 1 ? g : galois_src(g, kk.g, log_n);
    KsSum<W, 0> acc;
    for (u32 j = 0; j < dn; ++j) acc.mac(dg[(u64)j * S * n + src], key[(u64)j * 2 * KS * n + g], j);
    s[sw(e)] = (W)acc.get(mp);
  }
  __syncthreads();
  ntt_inv_slice<W, LC>(s, T, l, sl.rank);
  const u64 ci = H.down_inv[2 * k], ci_sh = H.down_inv[2 * k + 1];
  u64* top = plan.top + ((((u64)r * plan.B + rq) * 2 + b) * H.K + k) * n + sl.off;
  for (u32 e = threadIdx.x; e < sl.ns; e += blockDim.x)
    top[e] = mul_shoup(Ar<W>::inv_out(s[sw(e)], mp), ci, ci_sh, mp.q);
}

// ModDown of data slot i: limb job = (b ell + i) B + rq, entry y = rotation.
template <typename W, int LC>
__global__ void k_ks_hyb_moddown(DevTables T, HybTables H, u32 ell, const __grid_constant__ KsPlan plan) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  if (sl.y >= plan.R) return;
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 rq = sl.job % plan.B, bi = sl.job / plan.B, b = bi / ell, i = bi % ell, r = (u32)sl.y;
  const KsKey kk = plan.keys[r];
  const u32 S = ell + H.K, KS = kk.K + H.K, dn = (ell + H.alpha - 1) / H.alpha;
  const ModConst mi = T.mods[i];
  const u64* top = plan.top + (((u64)r * plan.B + rq) * 2 + b) * H.K * n + sl.off;
  const u64 pmod = H.down_P[i];
  for (u32 e = threadIdx.x; e < sl.ns; e += blockDim.x) {
    Acc128 a{0, 0};
    u32 neg = 0;
    for (u32 k = 0; k < H.K; ++k) {
      const u64 w = top[(u64)k * n + e];
      mac128(a, w, H.down_conv[(u64)k * T.n_mods + i]);
      neg += w > T.mods[T.L + k].half;
    }
    s[sw(e)] = (W)conv_finish(a, neg, pmod, mi);
  }
  __syncthreads();
  ntt_fwd_slice<W, LC>(s, T, i, sl.rank);
  const u64* add = b == 0 ? (plan.add0 ? plan.add0 + rq * plan.add0_b : nullptr)
                          : (plan.add1 ? plan.add1 + rq * plan.add1_b : nullptr);
  u64* dst = plan.out + rq * plan.out_b + r * plan.out_r + ((u64)b * ell + i) * n;
  const W* dg = reinterpret_cast<const W*>(plan.digits) + rq * plan.digits_b + (u64)i * n;
  const u64* key = kk.key + ((u64)b * KS + i) * n;
  const u64 pinv = H.pinv[2 * i], pinv_sh = H.pinv[2 * i + 1];
  for (u32 e = threadIdx.x; e < sl.ns; e += blockDim.x) {
    const u32 g = sl.off + e;
    const u32 src = kk.g == 1 ? g : galois_src(g, kk.g, log_n);
    KsSum<W, 0> acc;
    for (u32 j = 0; j < dn; ++j) acc.mac(dg[(u64)j * S * n + src], key[(u64)j * 2 * KS * n + g], j);
    const u64 u = acc.get(mi);
    u64 v = mul_shoup(sub_mod(u, Ar<W>::fwd_out(s[sw(e)], mi), mi.q), pinv, pinv_sh, mi.q);
    if (add) v = add_mod(v, add[(u64)i * n + (plan.add_perm ? src : g)], mi.q);
    dst[g] = v;
  }
}

static decltype(&k_ks_hyb_p<u64, 0>) const K6_k_ks_hyb_p[6] = TCKS_K6(k_ks_hyb_p);
static decltype(&k_ks_hyb_moddown<u64, 0>) const K6_k_ks_hyb_moddown[6] = TCKS_K6(k_ks_hyb_moddown);

void launch_keyswitch_hyb(const DevTables& T, const HybTables& H, u32 ell, const KsPlan& plan, cudaStream_t st) {
  const u64 jobs = (u64)plan.B * plan.R;
  if (!jobs) return;
  const double n = (double)(1u << T.log_n), bf = 0.5 * n * T.log_n;
  const u32 dn = (ell + H.alpha - 1) / H.alpha, K = H.K;
  const double wd = T.narrow ? 0.5 : 1.0;  // digit words in 8-byte units
  const double digit_sets = plan.digits_b ? plan.B : 1;
  const double adds = (plan.add0 ? (plan.add0_b ? plan.B : 1) : 0) + (plan.add1 ? (plan.add1_b ? plan.B : 1) : 0);
  {
    // reads: the digits' special slots, the keys' special limbs; writes: the P-limb scratch
    Launch L(K_KS_P, st, 8.0 * n * (digit_sets * wd * dn * K + plan.R * 2.0 * dn * K + 2.0 * K * jobs),
             2.0 * K * jobs * (dn * n + bf + n));
    launch_limb(K6_k_ks_hyb_p, T.narrow, 2 * K * plan.B, plan.R, T.log_n, st, T.limb_threads, T, H, ell, plan);
  }
  Launch L(K_KS_MODDOWN, st,
           8.0 * n * (digit_sets * wd * dn * ell + plan.R * 2.0 * dn * ell + 2.0 * K * jobs + adds * ell +
                      2.0 * ell * jobs),
           2.0 * ell * jobs * (dn * n + K * n + bf + n));
  launch_limb(K6_k_ks_hyb_moddown, T.narrow, 2 * ell * plan.B, plan.R, T.log_n, st, T.limb_threads, T, H, ell, plan);
}

}  // namespace tcks

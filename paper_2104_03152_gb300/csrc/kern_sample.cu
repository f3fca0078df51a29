// Key generation and public-key encryption on the device, driven by a counter-based generator so
// that every coefficient is drawn independently of launch shape: Philox4x64-10 (Salmon et al.,
// SC'11) with key = (seed, stream tag) and counter = (coefficient index, chain index of the limb,
// 0, 0). Draws: uniform residue = (w1:w0) mod q, ternary = (w0 mod 3) - 1, centred binomial
// error (eta = 21) = popcount(w0 & (2^21-1)) - popcount((w0 >> 21) & (2^21-1)).
// Stream tags: 1 s, 2 pk.a, 3 pk.e, 4 enc.u, 5 enc.e0, 6 enc.e1, 7 secret-key encryption a (public
// seed), 8 secret-key encryption e (private seed); switching key of kind `kind`
// (0 = relinearization, else the Galois element) digit j: a -> (kind<<32)|0x80000000|2j,
// e -> the same | 1.
#include <cuda_runtime.h>

#include "kernels.h"
#include "limb_launch.cuh"
#include "ntt.cuh"

namespace tcks {

namespace {

struct Philox4 {
  u64 w[4];
};

__device__ __forceinline__ Philox4 philox(u64 seed, u64 tag, u64 index, u64 limb) {
  u64 c0 = index, c1 = limb, c2 = 0, c3 = 0;
  u64 k0 = seed, k1 = tag;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const u64 lo0 = 0xD2E7470EE14C6C93ull * c0, hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c0);
    const u64 lo1 = 0xCA5A826395121157ull * c2, hi1 = __umul64hi(0xCA5A826395121157ull, c2);
    const u64 n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
  Philox4 o;
  o.w[0] = c0;
  o.w[1] = c1;
  o.w[2] = c2;
  o.w[3] = c3;
  return o;
}

__device__ __forceinline__ u64 draw_uniform(u64 seed, u64 tag, u64 index, u64 limb, const ModConst& m) {
  const Philox4 r = philox(seed, tag, index, limb);
  return reduce128(r.w[1], r.w[0], m);
}

__device__ __forceinline__ int draw_ternary(u64 seed, u64 tag, u64 index) {
  return (int)(philox(seed, tag, index, 0).w[0] % 3ull) - 1;
}

__device__ __forceinline__ int draw_cbd(u64 seed, u64 tag, u64 index) {
  const u64 w = philox(seed, tag, index, 0).w[0];
  return __popcll(w & 0x1FFFFFull) - __popcll((w >> 21) & 0x1FFFFFull);
}

__device__ __forceinline__ u64 small_to_residue(int v, u64 q) { return v >= 0 ? (u64)v : q - (u64)(-v); }

enum : u32 { SMALL_TERNARY = 0, SMALL_CBD = 1 };

// Fill the CTA's slice of s[] with a small polynomial (ternary / CBD, drawn at the global
// coefficient index) reduced mod the chain prime, and NTT it; on return s holds values in [0, 4q).
template <typename W, int LC>
__device__ __forceinline__ void small_ntt(W* s, const DevTables& T, u32 mod, u32 kind, u64 seed, u64 tag,
                                          u32 rank, u32 ns) {
  const u64 q = T.mods[mod].q;
  const u32 off = rank * ns;
  for (u32 k = threadIdx.x; k < ns; k += blockDim.x) {
    const int v = kind == SMALL_TERNARY ? draw_ternary(seed, tag, off + k) : draw_cbd(seed, tag, off + k);
    s[sw(k)] = (W)small_to_residue(v, q);
  }
  __syncthreads();
  ntt_fwd_slice<W, LC>(s, T, mod, rank);
}

__device__ __forceinline__ u64 mulq_s(u64 a, u64 b, const ModConst& m, u32 narrow) {
  return narrow ? reduce64(a * b, m) : mul_mod(a, b, m);
}

// Limb slot -> chain index when a layout holds `count` data limbs followed by P.
__device__ __forceinline__ u32 slot_chain(u32 slot, u32 count, u32 L) { return slot < count ? slot : L; }

}  // namespace

// s: [n_mods][N] (every prime of the chain), one limb job per prime.
template <typename W, int LC>
__global__ void k_keygen_secret(DevTables T, u64 seed, u64* __restrict__ s_out) {
  TCKS_SMEM(W);
  const Slice P = slice_of<LC>(T);
  const u32 mod = P.job;  // 0..n_mods-1 (the special primes last)
  small_ntt<W, LC>(s, T, mod, SMALL_TERNARY, seed, 1, P.rank, P.ns);
  const u64 q = T.mods[mod].q;
  u64* out = s_out + ((u64)mod << T.log_n) + P.off;
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) out[k] = Ar<W>::fwd_out(s[sw(k)], T.mods[mod]);
}

// pk: [2][L][N]; pk0 = -a*s + e, pk1 = a.
template <typename W, int LC>
__global__ void k_keygen_public(DevTables T, u64 seed, const u64* __restrict__ sk, u64* __restrict__ pk) {
  TCKS_SMEM(W);
  const Slice P = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 l = P.job;
  const ModConst m = T.mods[l];
  small_ntt<W, LC>(s, T, l, SMALL_CBD, seed, 3, P.rank, P.ns);
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) {
    const u32 g = P.off + k;
    const u64 a = draw_uniform(seed, 2, g, l, m);
    const u64 e = Ar<W>::fwd_out(s[sw(k)], m);
    pk[(u64)l * n + g] = add_mod(neg_mod(mulq_s(a, sk[(u64)l * n + g], m, T.narrow), m.q), e, m.q);
    pk[((u64)T.L + l) * n + g] = a;
  }
}

// Switching key of level K: [K][2][K+1][N]; limb job = digit j * (K+1) + slot.
//   b_j[slot] = -a*s + e + [chain(slot) == j] * (P mod q_j) * s'
template <typename W, int LC>
__global__ void k_keygen_switch(DevTables T, u64 seed, u32 kind, const u64* __restrict__ sk, u32 K,
                                u64* __restrict__ ksk) {
  TCKS_SMEM(W);
  const Slice P = slice_of<LC>(T);
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 j = P.job / (K + 1), slot = P.job % (K + 1);
  const u32 l = slot_chain(slot, K, T.L);
  const ModConst m = T.mods[l];
  const u64 tag_a = ((u64)kind << 32) | 0x80000000ull | (2ull * j);
  const u64 tag_e = tag_a | 1ull;
  small_ntt<W, LC>(s, T, l, SMALL_CBD, seed, tag_e, P.rank, P.ns);
  const u64 gadget = (l == j) ? T.pairs[(u64)T.L * T.n_mods + l].qa_mod_b : 0;  // P mod q_j
  const u64* s_l = sk + (u64)l * n;
  u64* b0 = ksk + (((u64)j * 2 + 0) * (K + 1) + slot) * n;
  u64* b1 = ksk + (((u64)j * 2 + 1) * (K + 1) + slot) * n;
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) {
    const u32 g = P.off + k;
    const u64 a = draw_uniform(seed, tag_a, g, l, m);
    u64 v = add_mod(neg_mod(mulq_s(a, s_l[g], m, T.narrow), m.q), Ar<W>::fwd_out(s[sw(k)], m), m.q);
    if (gadget) {
      const u64 sp = kind == 0 ? mulq_s(s_l[g], s_l[g], m, T.narrow) : s_l[galois_src(g, kind, log_n)];
      v = add_mod(v, mulq_s(gadget, sp, m, T.narrow), m.q);
    }
    b0[g] = v;
    b1[g] = a;
  }
}

// Switching key of level Kt for hybrid key switching (digits of alpha data primes, K special primes
// with product P): [dnum(Kt)][2][Kt + K][N], limb job = digit j * (Kt + K) + slot t;
//   b_j[t] = -a s + e + [t is a data prime of digit j] * (P mod q_t) * s'
// with the sampler counters of the one-prime key (tags from the digit index, limbs by chain index).
template <typename W, int LC>
__global__ void k_keygen_switch_hyb(DevTables T, HybTables H, u64 seed, u32 kind, const u64* __restrict__ sk,
                                    u32 Kt, u64* __restrict__ ksk) {
  TCKS_SMEM(W);
  const Slice P = slice_of<LC>(T);
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 S = Kt + H.K;
  const u32 j = P.job / S, slot = P.job % S;
  const u32 l = slot < Kt ? slot : T.L + (slot - Kt);
  const ModConst m = T.mods[l];
  const u64 tag_a = ((u64)kind << 32) | 0x80000000ull | (2ull * j);
  const u64 tag_e = tag_a | 1ull;
  small_ntt<W, LC>(s, T, l, SMALL_CBD, seed, tag_e, P.rank, P.ns);
  const u64 gadget = (l < T.L && l / H.alpha == j) ? H.down_P[l] : 0;  // P mod q_l
  const u64* s_l = sk + (u64)l * n;
  u64* b0 = ksk + (((u64)j * 2 + 0) * S + slot) * n;
  u64* b1 = ksk + (((u64)j * 2 + 1) * S + slot) * n;
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) {
    const u32 g = P.off + k;
    const u64 a = draw_uniform(seed, tag_a, g, l, m);
    u64 v = add_mod(neg_mod(mulq_s(a, s_l[g], m, T.narrow), m.q), Ar<W>::fwd_out(s[sw(k)], m), m.q);
    if (gadget) {
      const u64 sp = kind == 0 ? mulq_s(s_l[g], s_l[g], m, T.narrow) : s_l[galois_src(g, kind, log_n)];
      v = add_mod(v, mulq_s(gadget, sp, m, T.narrow), m.q);
    }
    b0[g] = v;
    b1[g] = a;
  }
}

// Encryption at level ell, limb job = limb: c0 = u*pk0 + e0 + m, c1 = u*pk1 + e1.
template <typename W, int LC>
__global__ void k_encrypt(DevTables T, u64 seed, const u64* __restrict__ pk, const u64* __restrict__ pt, u32 ell,
                          u64* __restrict__ out) {
  TCKS_SMEM(W);
  const Slice P = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 l = P.job;
  const ModConst m = T.mods[l];
  u64* c0 = out + (u64)l * n + P.off;
  u64* c1 = out + ((u64)ell + l) * n + P.off;
  const u64* p0 = pk + (u64)l * n + P.off;
  const u64* p1 = pk + ((u64)T.L + l) * n + P.off;
  const u64* ml = pt + (u64)l * n + P.off;
  small_ntt<W, LC>(s, T, l, SMALL_TERNARY, seed, 4, P.rank, P.ns);
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) {
    const u64 u = Ar<W>::fwd_out(s[sw(k)], m);
    c0[k] = add_mod(mulq_s(u, p0[k], m, T.narrow), ml[k], m.q);
    c1[k] = mulq_s(u, p1[k], m, T.narrow);
  }
  __syncthreads();
  small_ntt<W, LC>(s, T, l, SMALL_CBD, seed, 5, P.rank, P.ns);
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) c0[k] = add_mod(c0[k], Ar<W>::fwd_out(s[sw(k)], m), m.q);
  __syncthreads();
  small_ntt<W, LC>(s, T, l, SMALL_CBD, seed, 6, P.rank, P.ns);
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) c1[k] = add_mod(c1[k], Ar<W>::fwd_out(s[sw(k)], m), m.q);
}

// Secret-key encryption at level ell, limb job = limb: c1 = a, uniform from the public seed (stream 7)
// drawn directly in NTT form, c0 = -a*s + e + m with e from the private seed (stream 8).
template <typename W, int LC>
__global__ void k_encrypt_sym(DevTables T, u64 seed_a, u64 seed_e, const u64* __restrict__ sk,
                              const u64* __restrict__ pt, u32 ell, u64* __restrict__ out) {
  TCKS_SMEM(W);
  const Slice P = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 l = P.job;
  const ModConst m = T.mods[l];
  small_ntt<W, LC>(s, T, l, SMALL_CBD, seed_e, 8, P.rank, P.ns);
  for (u32 k = threadIdx.x; k < P.ns; k += blockDim.x) {
    const u32 g = P.off + k;
    const u64 a = draw_uniform(seed_a, 7, g, l, m);
    const u64 e = Ar<W>::fwd_out(s[sw(k)], m);
    out[(u64)l * n + g] =
        add_mod(add_mod(neg_mod(mulq_s(a, sk[(u64)l * n + g], m, T.narrow), m.q), e, m.q), pt[(u64)l * n + g], m.q);
    out[((u64)ell + l) * n + g] = a;
  }
}

// The uniform polynomial of a public seed over limbs 0..ell-1 ([ell][N], NTT form): with check == 0
// written to a, otherwise compared with a and any difference flagged in *status.
__global__ void k_sym_a(DevTables T, u64 seed_a, u32 ell, u64* __restrict__ a, int check, int* __restrict__ status) {
  const u64 n = 1ull << T.log_n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < (u64)ell * n; e += (u64)gridDim.x * blockDim.x) {
    const u32 l = (u32)(e >> T.log_n);
    const u64 v = draw_uniform(seed_a, 7, e & (n - 1), l, T.mods[l]);
    if (!check)
      a[e] = v;
    else if (a[e] != v)
      atomicExch(status, 1);
  }
}

// k_sym_a for count requests: request r's polynomial from seeds[r] at a + r a_stride.
__global__ void k_sym_a_batch(DevTables T, const u64* __restrict__ seeds, u32 ell, u64* __restrict__ a, u64 a_stride,
                              u32 count) {
  const u64 n = 1ull << T.log_n, per = (u64)ell * n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < per * count; e += (u64)gridDim.x * blockDim.x) {
    const u64 r = e / per, x = e - r * per;
    const u32 l = (u32)(x >> T.log_n);
    a[r * a_stride + x] = draw_uniform(seeds[r], 7, x & (n - 1), l, T.mods[l]);
  }
}

static decltype(&k_keygen_secret<u64, 0>) const K6_k_keygen_secret[6] = TCKS_K6(k_keygen_secret);
static decltype(&k_keygen_public<u64, 0>) const K6_k_keygen_public[6] = TCKS_K6(k_keygen_public);
static decltype(&k_keygen_switch<u64, 0>) const K6_k_keygen_switch[6] = TCKS_K6(k_keygen_switch);
static decltype(&k_keygen_switch_hyb<u64, 0>) const K6_k_keygen_switch_hyb[6] = TCKS_K6(k_keygen_switch_hyb);
static decltype(&k_encrypt<u64, 0>) const K6_k_encrypt[6] = TCKS_K6(k_encrypt);
static decltype(&k_encrypt_sym<u64, 0>) const K6_k_encrypt_sym[6] = TCKS_K6(k_encrypt_sym);

// Largest CTA size every limb kernel of this file accepts for the word type and cluster split.
u32 limb_threads_cap_sample(bool narrow, u32 log_c) {
  const u32 i = (narrow ? 3 : 0) + log_c;
  u32 cap = 1024;
  const void* ks[5] = {(const void*)K6_k_keygen_secret[i], (const void*)K6_k_keygen_public[i],
                       (const void*)K6_k_keygen_switch[i], (const void*)K6_k_encrypt[i],
                       (const void*)K6_k_encrypt_sym[i]};
  for (const void* k : ks) {
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, k) != cudaSuccess) return 0;
    cap = (u32)a.maxThreadsPerBlock < cap ? (u32)a.maxThreadsPerBlock : cap;
  }
  return cap;
}

void launch_keygen_secret(const DevTables& T, u64 seed, u64* s, cudaStream_t st) {
  Launch L(K_KEYGEN, st, 8.0 * T.n_mods * (1u << T.log_n));
  launch_limb(K6_k_keygen_secret, T.narrow, T.n_mods, 1, T.log_n, st, T.limb_threads, T, seed, s);
}

void launch_keygen_switch_hyb(const DevTables& T, const HybTables& H, u64 seed, u32 kind, const u64* s, u32 Kt,
                              u64* ksk, cudaStream_t st) {
  const u32 dn = (Kt + H.alpha - 1) / H.alpha, S = Kt + H.K;
  Launch L(K_KEYGEN, st, 8.0 * 2 * dn * S * (1u << T.log_n));
  launch_limb(K6_k_keygen_switch_hyb, T.narrow, dn * S, 1, T.log_n, st, T.limb_threads, T, H, seed, kind, s, Kt, ksk);
}

void launch_keygen_public(const DevTables& T, u64 seed, const u64* s, u64* pk, cudaStream_t st) {
  Launch L(K_KEYGEN, st, 8.0 * 3 * T.L * (1u << T.log_n));
  launch_limb(K6_k_keygen_public, T.narrow, T.L, 1, T.log_n, st, T.limb_threads, T, seed, s, pk);
}

void launch_keygen_switch(const DevTables& T, u64 seed, u32 kind, const u64* s, u32 K, u64* ksk, cudaStream_t st) {
  Launch L(K_KEYGEN, st, 8.0 * 2 * K * (K + 1) * (1u << T.log_n));
  launch_limb(K6_k_keygen_switch, T.narrow, K * (K + 1), 1, T.log_n, st, T.limb_threads, T, seed, kind, s, K, ksk);
}

void launch_encrypt(const DevTables& T, u64 seed, const u64* pk, const u64* pt, u32 ell, u64* out, cudaStream_t st) {
  Launch L(K_ENCRYPT, st, 8.0 * 5 * ell * (1u << T.log_n));
  launch_limb(K6_k_encrypt, T.narrow, ell, 1, T.log_n, st, T.limb_threads, T, seed, pk, pt, ell, out);
}

void launch_encrypt_sym(const DevTables& T, u64 seed_a, u64 seed_e, const u64* sk, const u64* pt, u32 ell, u64* out,
                        cudaStream_t st) {
  Launch L(K_ENCRYPT, st, 8.0 * 4 * ell * (1u << T.log_n));
  launch_limb(K6_k_encrypt_sym, T.narrow, ell, 1, T.log_n, st, T.limb_threads, T, seed_a, seed_e, sk, pt, ell, out);
}

void launch_sym_a(const DevTables& T, u64 seed_a, u32 ell, u64* a, bool check, int* status, cudaStream_t st) {
  const u64 e = (u64)ell << T.log_n;
  Launch L(K_ENCRYPT, st, 8.0 * e);
  u64 blocks = (e + 255) / 256;
  if (blocks > 152ull * 8) blocks = 152ull * 8;
  k_sym_a<<<(u32)blocks, 256, 0, st>>>(T, seed_a, ell, a, check ? 1 : 0, status);
}

void launch_sym_a_batch(const DevTables& T, const u64* seeds, u32 ell, u64* a, u64 a_stride, u32 count, cudaStream_t st) {
  const u64 e = ((u64)ell << T.log_n) * count;
  Launch L(K_ENCRYPT, st, 8.0 * e);
  u64 blocks = (e + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  k_sym_a_batch<<<(u32)blocks, 256, 0, st>>>(T, seeds, ell, a, a_stride, count);
}

}  // namespace tcks

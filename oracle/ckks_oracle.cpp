// Plain CPU oracle for the RNS-CKKS arithmetic behind TenSEAL's CKKSVector.
//
// TEST INFRASTRUCTURE ONLY. The tests, the package smoke check and the CPU-baseline leg of the
// benchmark load this library; the GPU library never links, includes or calls it, and it shares no
// source, header or table generator with the GPU library.
//
// The paper (TenSEAL, §2) builds on the CKKS scheme of Cheon et al. 2017 through SEAL and prints no
// CKKS mathematics itself, so every function below writes out the standard RNS-CKKS definition it
// names, in the plainest form: every modular product is an exact 128-bit product reduced with '%',
// residues are always canonical in [0, q), there is no lazy reduction and no precomputed
// Shoup/Barrett constant. Loops run in the order the definition states. OpenMP is used only on
// outer loops whose iterations write disjoint outputs, so results do not depend on thread count.
//
// Layouts (all u64 residues, row-major):
//   polynomial in RNS form, level ell:    [ell][N]        limb i is modulo q_i
//   ciphertext (CKKSVector, §2.3):        [2][ell][N]     (c0, c1), NTT form
//   secret key:                           [L+1][N]        limbs q_0..q_{L-1}, then P
//   public key:                           [2][L][N]
//   switching key (relin / Galois):       [K][2][K+1][N]  digit j, component b, limb (P last);
//                                         K = the key's level (L for a full key). A key of level K
//                                         holds exactly the digits j < K and limbs q_0..q_{K-1}, P
//                                         of the full key, and serves every ciphertext level <= K.
//   hoisted digits at level ell:          [ell][ell+1][N] digit j, slot i (slot ell is P)
// A parameter set holds L data primes followed by one special prime P.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef uint32_t u32;
typedef unsigned __int128 u128;

namespace {

// ----------------------------------------------------------------------------------------------
// Exact modular arithmetic on canonical residues (q < 2^62).
// ----------------------------------------------------------------------------------------------
inline u64 mulm(u64 a, u64 b, u64 q) { return (u64)(((u128)a * (u128)b) % q); }
inline u64 addm(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
inline u64 subm(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }
inline u64 negm(u64 a, u64 q) { return a == 0 ? 0 : q - a; }

u64 powm(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulm(r, b, q);
    b = mulm(b, b, q);
    e >>= 1;
  }
  return r;
}

// q prime: Fermat inverse.
u64 invm(u64 a, u64 q) { return powm(a, q - 2, q); }

// Signed integer to its canonical residue.
u64 from_signed(int64_t v, u64 q) {
  if (v >= 0) return (u64)v % q;
  u64 m = (u64)(-(v + 1)) + 1;  // |v| without overflow
  return negm(m % q, q);
}

// Balanced representative of x in [0, q): x if x <= (q-1)/2, else x - q.
inline int64_t balanced(u64 x, u64 q) { return x <= (q - 1) / 2 ? (int64_t)x : -(int64_t)(q - x); }

u32 bit_reverse(u32 x, u32 bits) {
  u32 r = 0;
  for (u32 i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

// ----------------------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its published definition.
// ----------------------------------------------------------------------------------------------
const u64 PHILOX_M0 = 0xD2E7470EE14C6C93ull;
const u64 PHILOX_M1 = 0xCA5A826395121157ull;
const u64 PHILOX_W0 = 0x9E3779B97F4A7C15ull;
const u64 PHILOX_W1 = 0xBB67AE8584CAA73Bull;

void philox4x64_10(const u64 ctr[4], const u64 key[2], u64 out[4]) {
  u64 x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  u64 k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    u128 p0 = (u128)PHILOX_M0 * x0;
    u128 p1 = (u128)PHILOX_M1 * x2;
    u64 hi0 = (u64)(p0 >> 64), lo0 = (u64)p0;
    u64 hi1 = (u64)(p1 >> 64), lo1 = (u64)p1;
    u64 y0 = hi1 ^ x1 ^ k0;
    u64 y1 = lo1;
    u64 y2 = hi0 ^ x3 ^ k1;
    u64 y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Sampler reading of the unspecified randomness: key = (seed, stream tag), counter = (coefficient
// index, limb index, 0, 0); one Philox call per coefficient (per limb for the uniform sampler).
void philox_words(u64 seed, u64 tag, u64 i, u64 limb, u64 w[4]) {
  u64 ctr[4] = {i, limb, 0, 0};
  u64 key[2] = {seed, tag};
  philox4x64_10(ctr, key, w);
}

// Uniform residue mod q for limb `limb`: the 128-bit word (w1:w0) reduced mod q.
u64 sample_uniform(u64 seed, u64 tag, u64 i, u64 limb, u64 q) {
  u64 w[4];
  philox_words(seed, tag, i, limb, w);
  u128 v = ((u128)w[1] << 64) | (u128)w[0];
  return (u64)(v % q);
}

// Ternary coefficient in {-1, 0, 1}: (w0 mod 3) - 1.
int64_t sample_ternary(u64 seed, u64 tag, u64 i) {
  u64 w[4];
  philox_words(seed, tag, i, 0, w);
  return (int64_t)(w[0] % 3) - 1;
}

int popcount64(u64 x) {
  int c = 0;
  while (x) {
    c += (int)(x & 1);
    x >>= 1;
  }
  return c;
}

// Centered binomial error, eta = 21: popcount of 21 bits minus popcount of the next 21 bits of w0.
int64_t sample_cbd(u64 seed, u64 tag, u64 i) {
  u64 w[4];
  philox_words(seed, tag, i, 0, w);
  const u64 mask = (1ull << 21) - 1;
  return (int64_t)popcount64(w[0] & mask) - (int64_t)popcount64((w[0] >> 21) & mask);
}

}  // namespace

// ==============================================================================================
// Exported functions.
// ==============================================================================================
extern "C" {

// ---------------------------------------------------------------- primes and roots (O1, O2) ---

// Deterministic Miller-Rabin; the first twelve prime bases decide every n < 2^64.
int orc_is_prime(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (u64 p : bases)
    if (n % p == 0) return n == p ? 1 : 0;
  u64 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (u64 a : bases) {
    u64 x = powm(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int r = 1; r < s; ++r) {
      x = mulm(x, x, n);
      if (x == n - 1) {
        witness = false;
        break;
      }
    }
    if (witness) return 0;
  }
  return 1;
}

// For each bit size b in order: the largest prime c < 2^b with c == 1 (mod 2N), c > 2^(b-1), not
// chosen before. Returns 0, or -1 when some size has no such prime.
int orc_gen_primes(u32 log_n, const u32* bits, u32 count, u64* out) {
  const u64 m = 2ull << log_n;
  for (u32 k = 0; k < count; ++k) {
    const u32 b = bits[k];
    if (b < 2 || b > 61) return -1;
    const u64 top = (1ull << b) - 1;
    const u64 low = 1ull << (b - 1);
    if (top < m + 1) return -1;
    u64 c = ((top - 1) / m) * m + 1;
    int found = 0;
    while (c > low) {
      int taken = 0;
      for (u32 t = 0; t < k; ++t)
        if (out[t] == c) taken = 1;
      if (!taken && orc_is_prime(c)) {
        out[k] = c;
        found = 1;
        break;
      }
      if (c < m) break;
      c -= m;
    }
    if (!found) return -1;
  }
  return 0;
}

// The numerically smallest primitive 2N-th root of unity mod q (psi^N == -1), or 0 if q != 1 mod 2N.
// Every primitive 2N-th root is psi0^k for odd k, so the minimum is found over those N powers.
u64 orc_min_psi(u64 q, u32 log_n) {
  const u64 n = 1ull << log_n, m = 2 * n;
  if ((q - 1) % m != 0) return 0;
  u64 psi0 = 0;
  for (u64 x = 2; x < q; ++x) {
    u64 c = powm(x, (q - 1) / m, q);
    if (powm(c, n, q) == q - 1) {
      psi0 = c;
      break;
    }
  }
  if (psi0 == 0) return 0;
  const u64 sq = mulm(psi0, psi0, q);
  u64 cur = psi0, best = psi0;
  for (u64 k = 3; k < m; k += 2) {
    cur = mulm(cur, sq, q);
    if (cur < best) best = cur;
  }
  return best;
}

u32 orc_bit_reverse(u32 x, u32 bits) { return bit_reverse(x, bits); }

// ------------------------------------------------------------------------------- Philox (O5) ---

void orc_philox4x64(const u64* ctr, const u64* key, u64* out) { philox4x64_10(ctr, key, out); }

// ------------------------------------------------------------------------------ the NTT (O3) ---

// Definition: out_j = sum_i a_i * psi^((2*brv(j)+1)*i) mod q. O(N^2).
void orc_ntt_naive(const u64* a, u64* out, u32 log_n, u64 q, u64 psi) {
  const u64 n = 1ull << log_n;
  for (u64 j = 0; j < n; ++j) {
    const u64 w = powm(psi, 2 * (u64)bit_reverse((u32)j, log_n) + 1, q);
    u64 acc = 0, x = 1;
    for (u64 i = 0; i < n; ++i) {
      acc = addm(acc, mulm(a[i], x, q), q);
      x = mulm(x, w, q);
    }
    out[j] = acc;
  }
}

}  // extern "C"

namespace {

// Twiddles psi^brv(k) and psi^-brv(k), k < N, for the iterative transforms.
void make_twiddles(u32 log_n, u64 q, u64 psi, std::vector<u64>& tw, std::vector<u64>& itw) {
  const u64 n = 1ull << log_n;
  tw.assign(n, 0);
  itw.assign(n, 0);
  const u64 ipsi = invm(psi, q);
  for (u64 k = 0; k < n; ++k) {
    const u64 e = bit_reverse((u32)k, log_n);
    tw[k] = powm(psi, e, q);
    itw[k] = powm(ipsi, e, q);
  }
}

// Iterative negacyclic Cooley-Tukey transform, natural order in, bit-reversed order out
// (Longa and Naehrig 2016): stage m (= 1, 2, 4, ...) pairs a[j] with a[j + t], t = N/(2m), in
// block i with twiddle psi^brv(m+i).
void ntt_ct(u64* a, u32 log_n, u64 q, const u64* tw) {
  const u64 n = 1ull << log_n;
  u64 t = n;
  for (u64 m = 1; m < n; m <<= 1) {
    t >>= 1;
    for (u64 i = 0; i < m; ++i) {
      const u64 w = tw[m + i];
      const u64 j1 = 2 * i * t;
      for (u64 j = j1; j < j1 + t; ++j) {
        const u64 u = a[j];
        const u64 v = mulm(a[j + t], w, q);
        a[j] = addm(u, v, q);
        a[j + t] = subm(u, v, q);
      }
    }
  }
}

// Its inverse, Gentleman-Sande butterflies with psi^-brv(m+i), then multiplication by N^-1.
void intt_gs(u64* a, u32 log_n, u64 q, const u64* itw) {
  const u64 n = 1ull << log_n;
  u64 t = 1;
  for (u64 m = n >> 1; m >= 1; m >>= 1) {
    for (u64 i = 0; i < m; ++i) {
      const u64 w = itw[m + i];
      const u64 j1 = 2 * i * t;
      for (u64 j = j1; j < j1 + t; ++j) {
        const u64 u = a[j];
        const u64 v = a[j + t];
        a[j] = addm(u, v, q);
        a[j + t] = mulm(subm(u, v, q), w, q);
      }
    }
    t <<= 1;
  }
  const u64 ninv = invm(n % q, q);
  for (u64 j = 0; j < n; ++j) a[j] = mulm(a[j], ninv, q);
}

}  // namespace

// Oracle context: the modulus chain (L data primes then P), each prime's root and twiddles.
struct OrcCtx {
  u32 log_n;
  u64 n;
  u32 L;                 // number of data primes
  u32 K = 1;             // number of special primes (hybrid key switching: K > 1 allowed)
  std::vector<u64> q;    // size L + K; q[L] = P when K = 1, else the special primes p_0..p_{K-1}
  std::vector<u64> psi;  // smallest primitive 2N-th root per prime
  std::vector<std::vector<u64>> tw, itw;
};

namespace {

inline u64* limb(u64* base, u64 n, u64 idx) { return base + idx * n; }
inline const u64* limb(const u64* base, u64 n, u64 idx) { return base + idx * n; }

void ntt_mod(const OrcCtx* c, u64* a, u32 mod_idx) { ntt_ct(a, c->log_n, c->q[mod_idx], c->tw[mod_idx].data()); }
void intt_mod(const OrcCtx* c, u64* a, u32 mod_idx) { intt_gs(a, c->log_n, c->q[mod_idx], c->itw[mod_idx].data()); }

// Small signed coefficients -> NTT-form limb modulo q[mod_idx].
void signed_to_ntt(const OrcCtx* c, const int64_t* v, u32 mod_idx, u64* out) {
  const u64 q = c->q[mod_idx];
  for (u64 i = 0; i < c->n; ++i) out[i] = from_signed(v[i], q);
  ntt_mod(c, out, mod_idx);
}

// NTT-domain automorphism index map (O15): out[j] = in[j'] with 2brv(j')+1 == (2brv(j)+1)*g mod 2N.
std::vector<u32> automorphism_index(const OrcCtx* c, u32 g) {
  const u64 m = 2 * c->n;
  std::vector<u32> src(c->n);
  for (u64 j = 0; j < c->n; ++j) {
    const u64 e = ((2 * (u64)bit_reverse((u32)j, c->log_n) + 1) * (u64)g) % m;
    src[j] = bit_reverse((u32)((e - 1) / 2), c->log_n);
  }
  return src;
}

}  // namespace

extern "C" {

// In-place transform with explicit root (used by the pins on arbitrary primes).
void orc_ntt(u64* a, u32 log_n, u64 q, u64 psi) {
  std::vector<u64> tw, itw;
  make_twiddles(log_n, q, psi, tw, itw);
  ntt_ct(a, log_n, q, tw.data());
}

void orc_intt(u64* a, u32 log_n, u64 q, u64 psi) {
  std::vector<u64> tw, itw;
  make_twiddles(log_n, q, psi, tw, itw);
  intt_gs(a, log_n, q, itw.data());
}

// ------------------------------------------------------------------------------ the context ---

// primes: L data primes followed by P (n_primes = L + 1). Returns NULL if a prime has no 2N-th root.
OrcCtx* orc_ctx_new(u32 log_n, const u64* primes, u32 n_primes) {
  if (n_primes < 2) return nullptr;
  OrcCtx* c = new OrcCtx();
  c->log_n = log_n;
  c->n = 1ull << log_n;
  c->L = n_primes - 1;
  c->q.assign(primes, primes + n_primes);
  c->psi.resize(n_primes);
  c->tw.resize(n_primes);
  c->itw.resize(n_primes);
  for (u32 k = 0; k < n_primes; ++k) {
    c->psi[k] = orc_min_psi(c->q[k], log_n);
    if (c->psi[k] == 0) {
      delete c;
      return nullptr;
    }
    make_twiddles(log_n, c->q[k], c->psi[k], c->tw[k], c->itw[k]);
  }
  return c;
}

// A chain for hybrid key switching: n_primes - n_special data primes, then the n_special special
// primes whose product is P.
OrcCtx* orc_ctx_new_hybrid(u32 log_n, const u64* primes, u32 n_primes, u32 n_special) {
  if (n_special < 1 || n_primes <= n_special) return nullptr;
  OrcCtx* c = orc_ctx_new(log_n, primes, n_primes);
  if (!c) return nullptr;
  c->L = n_primes - n_special;
  c->K = n_special;
  return c;
}

void orc_ctx_free(OrcCtx* c) { delete c; }

u64 orc_ctx_psi(const OrcCtx* c, u32 mod_idx) { return c->psi[mod_idx]; }

void orc_ntt_limb(const OrcCtx* c, u64* a, u32 mod_idx) { ntt_mod(c, a, mod_idx); }
void orc_intt_limb(const OrcCtx* c, u64* a, u32 mod_idx) { intt_mod(c, a, mod_idx); }

// Galois element of a left rotation by `step` slots (O15): 5^step mod 2N, step taken mod N/2.
u32 orc_galois_elt(const OrcCtx* c, int64_t step) {
  const int64_t half = (int64_t)(c->n / 2);
  int64_t k = step % half;
  if (k < 0) k += half;
  return (u32)powm(5, (u64)k, 2 * c->n);
}

// Automorphism a(X) -> a(X^g) on NTT-form limbs: n_limbs consecutive limbs of N.
void orc_automorphism_ntt(const OrcCtx* c, const u64* a, u32 n_limbs, u32 g, u64* out) {
  const std::vector<u32> src = automorphism_index(c, g);
  for (u32 l = 0; l < n_limbs; ++l)
    for (u64 j = 0; j < c->n; ++j) out[l * c->n + j] = a[l * c->n + src[j]];
}

// The same automorphism on a coefficient-domain limb: coefficient i goes to i*g mod 2N, negated
// when that index is >= N (X^N = -1).
void orc_automorphism_coeff(const OrcCtx* c, const u64* a, u64 q, u32 g, u64* out) {
  const u64 m = 2 * c->n;
  for (u64 i = 0; i < c->n; ++i) {
    const u64 e = (i * (u64)g) % m;
    if (e < c->n)
      out[e] = a[i];
    else
      out[e - c->n] = negm(a[i], q);
  }
}

// ------------------------------------------------------------------------------- keys (O6-O8) ---
// Stream tags of the sampler (one per sampled polynomial).
//   1 secret s; 2 public a; 3 public e; 4 encryption u; 5 encryption e0; 6 encryption e1;
//   7 secret-key encryption a (from the public seed); 8 secret-key encryption e (from the private seed);
//   switching key for `kind` (0 = relinearization, otherwise the Galois element g), digit j:
//   a_j: (kind << 32) | 0x80000000 | (2j), e_j: (kind << 32) | 0x80000000 | (2j + 1).

// s ternary; stored in NTT form over every prime of the chain (L + 1, or L + K for hybrid chains).
void orc_keygen_secret(const OrcCtx* c, u64 seed, u64* s) {
  std::vector<int64_t> v(c->n);
  for (u64 i = 0; i < c->n; ++i) v[i] = sample_ternary(seed, 1, i);
  for (u32 l = 0; l < (u32)c->q.size(); ++l) signed_to_ntt(c, v.data(), l, limb(s, c->n, l));
}

// pk = (-a*s + e, a) over the data primes; a sampled uniformly per limb directly in NTT form.
void orc_keygen_public(const OrcCtx* c, u64 seed, const u64* s, u64* pk) {
  std::vector<int64_t> e(c->n);
  for (u64 i = 0; i < c->n; ++i) e[i] = sample_cbd(seed, 3, i);
  std::vector<u64> et(c->n);
  for (u32 l = 0; l < c->L; ++l) {
    const u64 q = c->q[l];
    signed_to_ntt(c, e.data(), l, et.data());
    u64* p0 = limb(pk, c->n, l);
    u64* p1 = limb(pk, c->n, c->L + l);
    const u64* sl = limb(s, c->n, l);
    for (u64 i = 0; i < c->n; ++i) {
      const u64 a = sample_uniform(seed, 2, i, l, q);
      p1[i] = a;
      p0[i] = addm(negm(mulm(a, sl[i], q), q), et[i], q);
    }
  }
}

// Switching key from s' to s, one digit per data prime (O6):
//   b_j[i] = -a_j[i]*s[i] + e_j[i] + [i == j] * (P mod q_j) * s'[i],  a_j uniform, e_j CBD,
// over limbs i = q_0..q_{L-1}, P. s and s' are NTT form over L + 1 primes.
void orc_keygen_switch(const OrcCtx* c, u64 seed, u64 kind, const u64* s, const u64* s_prime, u32 key_level,
                       u64* ksk) {
  const u32 L = c->L, K = key_level;
  const u64 n = c->n;
  const u64 P = c->q[L];
#pragma omp parallel for schedule(dynamic)
  for (int jj = 0; jj < (int)K; ++jj) {
    const u32 j = (u32)jj;
    const u64 tag_a = (kind << 32) | 0x80000000ull | (2ull * j);
    const u64 tag_e = (kind << 32) | 0x80000000ull | (2ull * j + 1);
    std::vector<int64_t> e(n);
    for (u64 i = 0; i < n; ++i) e[i] = sample_cbd(seed, tag_e, i);
    std::vector<u64> et(n);
    for (u32 slot = 0; slot <= K; ++slot) {
      const u32 l = (slot < K) ? slot : L;  // chain index of this limb
      const u64 q = c->q[l];
      signed_to_ntt(c, e.data(), l, et.data());
      u64* b0 = ksk + (((u64)j * 2 + 0) * (K + 1) + slot) * n;
      u64* b1 = ksk + (((u64)j * 2 + 1) * (K + 1) + slot) * n;
      const u64* sl = limb(s, n, l);
      const u64* spl = limb(s_prime, n, l);
      const u64 gadget = (l == j) ? (P % q) : 0;
      for (u64 i = 0; i < n; ++i) {
        const u64 a = sample_uniform(seed, tag_a, i, l, q);
        b1[i] = a;
        u64 v = addm(negm(mulm(a, sl[i], q), q), et[i], q);
        if (l == j) v = addm(v, mulm(gadget, spl[i], q), q);
        b0[i] = v;
      }
    }
  }
}

// Relinearization key: s' = s^2 (O7).
void orc_keygen_relin(const OrcCtx* c, u64 seed, const u64* s, u32 key_level, u64* ksk) {
  std::vector<u64> s2((u64)(c->L + 1) * c->n);
  for (u32 l = 0; l <= c->L; ++l)
    for (u64 i = 0; i < c->n; ++i) s2[l * c->n + i] = mulm(s[l * c->n + i], s[l * c->n + i], c->q[l]);
  orc_keygen_switch(c, seed, 0, s, s2.data(), key_level, ksk);
}

// Galois key for element g: s' = tau_g(s) (O8).
void orc_keygen_galois(const OrcCtx* c, u64 seed, const u64* s, u32 g, u32 key_level, u64* ksk) {
  std::vector<u64> sg((u64)(c->L + 1) * c->n);
  orc_automorphism_ntt(c, s, c->L + 1, g, sg.data());
  orc_keygen_switch(c, seed, g, s, sg.data(), key_level, ksk);
}

// --------------------------------------------------------------------------- encoding (O9) ---

// Inverse canonical embedding of n_in real slot values (zero-padded to N/2):
//   m_i = (2/N) * sum_j z_j * cos(pi * (5^j * i mod 2N) / N),   the real part of z_j * zeta^(-5^j i)
// then p_i = round-half-away(scale * m_i). pre (optional, N doubles) receives scale * m_i before
// rounding. Returns 0, or -2 when some |scale * m_i| >= 2^62.
static int encode_coeffs(const OrcCtx* c, const double* z, u32 n_in, double scale, double* pre, int64_t* p) {
  const u64 n = c->n, m = 2 * n, slots = n / 2;
  std::vector<double> cosv(m);
  for (u64 k = 0; k < m; ++k) cosv[k] = std::cos(M_PI * (double)k / (double)n);
  std::vector<u64> e(slots);
  u64 g = 1;
  for (u64 j = 0; j < slots; ++j) {
    e[j] = g;
    g = (g * 5) % m;
  }
  int status = 0;
#pragma omp parallel for schedule(static)
  for (int64_t ii = 0; ii < (int64_t)n; ++ii) {
    const u64 i = (u64)ii;
    double s = 0.0;
    for (u64 j = 0; j < n_in; ++j) s += z[j] * cosv[(e[j] * i) % m];
    const double mi = (2.0 / (double)n) * s;
    const double x = scale * mi;
    if (pre) pre[i] = x;
    if (!(std::fabs(x) < 4611686018427387904.0)) {
#pragma omp atomic write
      status = -2;
      p[i] = 0;
    } else {
      p[i] = (int64_t)std::llround(x);
    }
  }
  return status;
}

// Encode (O9): the coefficients above reduced into limbs q_0..q_{level-1} and NTT'd. Returns 0, -1
// on bad size, -2 on overflow.
int orc_encode(const OrcCtx* c, const double* z, u32 n_in, double scale, u32 level, double* pre, u64* pt) {
  const u64 n = c->n;
  if (n_in > n / 2 || level < 1 || level > c->L) return -1;
  std::vector<int64_t> p(n);
  const int status = encode_coeffs(c, z, n_in, scale, pre, p.data());
  if (status) return status;
  for (u32 l = 0; l < level; ++l) signed_to_ntt(c, p.data(), l, limb(pt, n, l));
  return 0;
}

// The same plaintext over the extended basis: limbs q_0..q_{level-1}, then the special prime P
// (limb `level`) -- the same integer polynomial, as the double-hoisted product needs.
int orc_encode_ext(const OrcCtx* c, const double* z, u32 n_in, double scale, u32 level, double* pre, u64* pt) {
  const u64 n = c->n;
  if (n_in > n / 2 || level < 1 || level > c->L) return -1;
  std::vector<int64_t> p(n);
  const int status = encode_coeffs(c, z, n_in, scale, pre, p.data());
  if (status) return status;
  for (u32 l = 0; l < level; ++l) signed_to_ntt(c, p.data(), l, limb(pt, n, l));
  signed_to_ntt(c, p.data(), c->L, limb(pt, n, level));
  return 0;
}

// Decoding sum (O10) on centred integer coefficients p (already CRT-composed, as doubles):
//   z_j = sum_i (p_i / scale) * cos(pi * (5^j * i mod 2N) / N),  j < n_out.
void orc_decode_sum(const OrcCtx* c, const double* p, double scale, u32 n_out, double* z) {
  const u64 n = c->n, m = 2 * n;
  std::vector<double> cosv(m);
  for (u64 k = 0; k < m; ++k) cosv[k] = std::cos(M_PI * (double)k / (double)n);
  std::vector<u64> e(n_out);
  u64 g = 1;
  for (u64 j = 0; j < n_out; ++j) {
    e[j] = g;
    g = (g * 5) % m;
  }
#pragma omp parallel for schedule(static)
  for (int64_t jj = 0; jj < (int64_t)n_out; ++jj) {
    const u64 j = (u64)jj;
    double s = 0.0;
    for (u64 i = 0; i < n; ++i) s += (p[i] / scale) * cosv[(e[j] * i) % m];
    z[j] = s;
  }
}

// -------------------------------------------------------------- encrypt / decrypt (O11) -------

// Public-key encryption at level `level` (limbs q_0..q_{level-1}; identical to encrypting at L and
// dropping the upper limbs): c0 = u*pk0 + e0 + m, c1 = u*pk1 + e1.
void orc_encrypt(const OrcCtx* c, const u64* pk, const u64* pt, u32 level, u64 seed, u64* ct) {
  const u64 n = c->n;
  std::vector<int64_t> u(n), e0(n), e1(n);
  for (u64 i = 0; i < n; ++i) {
    u[i] = sample_ternary(seed, 4, i);
    e0[i] = sample_cbd(seed, 5, i);
    e1[i] = sample_cbd(seed, 6, i);
  }
  std::vector<u64> ut(n), e0t(n), e1t(n);
  for (u32 l = 0; l < level; ++l) {
    const u64 q = c->q[l];
    signed_to_ntt(c, u.data(), l, ut.data());
    signed_to_ntt(c, e0.data(), l, e0t.data());
    signed_to_ntt(c, e1.data(), l, e1t.data());
    const u64* p0 = limb(pk, n, l);
    const u64* p1 = limb(pk, n, c->L + l);
    const u64* ml = limb(pt, n, l);
    u64* c0 = limb(ct, n, l);
    u64* c1 = limb(ct, n, level + l);
    for (u64 i = 0; i < n; ++i) {
      c0[i] = addm(addm(mulm(ut[i], p0[i], q), e0t[i], q), ml[i], q);
      c1[i] = addm(mulm(ut[i], p1[i], q), e1t[i], q);
    }
  }
}

// The uniform polynomial a of a secret-key encryption, sampled per limb directly in NTT form from the
// public seed (stream 7): [level][N].
void orc_sample_sym_a(const OrcCtx* c, u32 level, u64 seed_a, u64* a) {
  for (u32 l = 0; l < level; ++l)
    for (u64 i = 0; i < c->n; ++i) limb(a, c->n, l)[i] = sample_uniform(seed_a, 7, i, l, c->q[l]);
}

// Secret-key encryption: ct = (-a*s + e + m, a), a from the public seed (stream 7), e CBD from the
// private seed (stream 8). Only c0 and seed_a need to travel: the receiver regenerates a.
void orc_encrypt_symmetric(const OrcCtx* c, const u64* s, const u64* pt, u32 level, u64 seed_a, u64 seed_e,
                           u64* ct) {
  const u64 n = c->n;
  std::vector<int64_t> e(n);
  for (u64 i = 0; i < n; ++i) e[i] = sample_cbd(seed_e, 8, i);
  std::vector<u64> et(n);
  orc_sample_sym_a(c, level, seed_a, limb(ct, n, level));
  for (u32 l = 0; l < level; ++l) {
    const u64 q = c->q[l];
    signed_to_ntt(c, e.data(), l, et.data());
    const u64* a = limb(ct, n, level + l);
    const u64* sl = limb(s, n, l);
    const u64* ml = limb(pt, n, l);
    u64* c0 = limb(ct, n, l);
    for (u64 i = 0; i < n; ++i) c0[i] = addm(addm(negm(mulm(a[i], sl[i], q), q), et[i], q), ml[i], q);
  }
}

// m = c0 + c1*s over limbs q_0..q_{level-1}.
void orc_decrypt(const OrcCtx* c, const u64* s, const u64* ct, u32 level, u64* pt) {
  const u64 n = c->n;
  for (u32 l = 0; l < level; ++l) {
    const u64 q = c->q[l];
    const u64* c0 = limb(ct, n, l);
    const u64* c1 = limb(ct, n, level + l);
    const u64* sl = limb(s, n, l);
    u64* m = limb(pt, n, l);
    for (u64 i = 0; i < n; ++i) m[i] = addm(c0[i], mulm(c1[i], sl[i], q), q);
  }
}

// Decryption of a ciphertext of `size` components (size 3 = an unrelinearized product, whose third
// component pairs with s^2): m = sum_k c_k s^k, limb by limb in NTT form.
void orc_decrypt_sized(const OrcCtx* c, const u64* s, const u64* ct, u32 level, u32 size, u64* pt) {
  const u64 n = c->n;
  for (u32 l = 0; l < level; ++l) {
    const u64 q = c->q[l];
    const u64* sl = limb(s, n, l);
    u64* m = limb(pt, n, l);
    for (u64 i = 0; i < n; ++i) {
      u64 acc = limb(ct, n, l)[i], sk = sl[i];
      for (u32 k = 1; k < size; ++k) {
        acc = addm(acc, mulm(limb(ct, n, (u64)k * level + l)[i], sk, q), q);
        sk = mulm(sk, sl[i], q);
      }
      m[i] = acc;
    }
  }
}

// ------------------------------------------------------------- element-wise ops (O12, O13) ---
// All take n_polys polynomials of `level` limbs laid out back to back.

void orc_add(const OrcCtx* c, const u64* a, const u64* b, u32 level, u32 n_polys, u64* out) {
  for (u32 p = 0; p < n_polys; ++p)
    for (u32 l = 0; l < level; ++l)
      for (u64 i = 0; i < c->n; ++i) {
        const u64 k = ((u64)p * level + l) * c->n + i;
        out[k] = addm(a[k], b[k], c->q[l]);
      }
}

void orc_sub(const OrcCtx* c, const u64* a, const u64* b, u32 level, u32 n_polys, u64* out) {
  for (u32 p = 0; p < n_polys; ++p)
    for (u32 l = 0; l < level; ++l)
      for (u64 i = 0; i < c->n; ++i) {
        const u64 k = ((u64)p * level + l) * c->n + i;
        out[k] = subm(a[k], b[k], c->q[l]);
      }
}

void orc_negate(const OrcCtx* c, const u64* a, u32 level, u32 n_polys, u64* out) {
  for (u32 p = 0; p < n_polys; ++p)
    for (u32 l = 0; l < level; ++l)
      for (u64 i = 0; i < c->n; ++i) {
        const u64 k = ((u64)p * level + l) * c->n + i;
        out[k] = negm(a[k], c->q[l]);
      }
}

// ct (+|-|*) plaintext. add/sub touch c0 only; mul multiplies both components.
void orc_add_plain(const OrcCtx* c, const u64* ct, const u64* pt, u32 level, u64* out) {
  const u64 n = c->n;
  std::memcpy(out, ct, sizeof(u64) * 2 * level * n);
  for (u32 l = 0; l < level; ++l)
    for (u64 i = 0; i < n; ++i) out[l * n + i] = addm(ct[l * n + i], pt[l * n + i], c->q[l]);
}

void orc_sub_plain(const OrcCtx* c, const u64* ct, const u64* pt, u32 level, u64* out) {
  const u64 n = c->n;
  std::memcpy(out, ct, sizeof(u64) * 2 * level * n);
  for (u32 l = 0; l < level; ++l)
    for (u64 i = 0; i < n; ++i) out[l * n + i] = subm(ct[l * n + i], pt[l * n + i], c->q[l]);
}

void orc_mul_plain_polys(const OrcCtx* c, const u64* ct, const u64* pt, u32 level, u32 polys, u64* out);
void orc_mul_plain(const OrcCtx* c, const u64* ct, const u64* pt, u32 level, u64* out) {
  orc_mul_plain_polys(c, ct, pt, level, 2, out);
}

// Every one of `polys` components times the plaintext.
void orc_mul_plain_polys(const OrcCtx* c, const u64* ct, const u64* pt, u32 level, u32 polys, u64* out) {
  const u64 n = c->n;
  for (u32 p = 0; p < polys; ++p)
    for (u32 l = 0; l < level; ++l)
      for (u64 i = 0; i < n; ++i) {
        const u64 k = ((u64)p * level + l) * n + i;
        out[k] = mulm(ct[k], pt[l * n + i], c->q[l]);
      }
}

// Tensor product (O13): (d0, d1, d2) = (a0*b0, a0*b1 + a1*b0, a1*b1), output [3][level][N].
void orc_tensor(const OrcCtx* c, const u64* a, const u64* b, u32 level, u64* out) {
  const u64 n = c->n;
  for (u32 l = 0; l < level; ++l) {
    const u64 q = c->q[l];
    const u64 *a0 = limb(a, n, l), *a1 = limb(a, n, level + l);
    const u64 *b0 = limb(b, n, l), *b1 = limb(b, n, level + l);
    u64* d0 = limb(out, n, l);
    u64* d1 = limb(out, n, level + l);
    u64* d2 = limb(out, n, 2 * level + l);
    for (u64 i = 0; i < n; ++i) {
      d0[i] = mulm(a0[i], b0[i], q);
      d1[i] = addm(mulm(a0[i], b1[i], q), mulm(a1[i], b0[i], q), q);
      d2[i] = mulm(a1[i], b1[i], q);
    }
  }
}

// ----------------------------------------------------------------- rescale (O14) ---------------
// c'_i = (c_i - (bal(c_{ell-1}) mod q_i)) * q_{ell-1}^-1 mod q_i, i < ell-1, for both components;
// the correction term is lifted in the coefficient domain and NTT'd per target prime.
void orc_rescale_polys(const OrcCtx* c, const u64* ct, u32 level, u32 polys, u64* out);
void orc_rescale(const OrcCtx* c, const u64* ct, u32 level, u64* out) { orc_rescale_polys(c, ct, level, 2, out); }

// Rescale (O14) of `polys` polynomials [polys][level][N] -> [polys][level-1][N], each on its own.
void orc_rescale_polys(const OrcCtx* c, const u64* ct, u32 level, u32 polys, u64* out) {
  const u64 n = c->n;
  const u32 last = level - 1;
  const u64 ql = c->q[last];
  for (u32 p = 0; p < polys; ++p) {
    std::vector<u64> top(limb(ct, n, (u64)p * level + last), limb(ct, n, (u64)p * level + last) + n);
    intt_mod(c, top.data(), last);
#pragma omp parallel for schedule(static)
    for (int ii = 0; ii < (int)last; ++ii) {
      const u32 i = (u32)ii;
      const u64 q = c->q[i];
      std::vector<u64> t(n);
      for (u64 k = 0; k < n; ++k) t[k] = from_signed(balanced(top[k], ql), q);
      ntt_mod(c, t.data(), i);
      const u64 inv = invm(ql % q, q);
      const u64* src = limb(ct, n, (u64)p * level + i);
      u64* dst = limb(out, n, (u64)p * last + i);
      for (u64 k = 0; k < n; ++k) dst[k] = mulm(subm(src[k], t[k], q), inv, q);
    }
  }
}

// ------------------------------------------------------------- key switching (O16-O18) ---------

// ModUp with one digit per prime (alpha = 1): digit j = bal_{q_j}([x]_{q_j}) as an integer
// polynomial, lifted to every slot i < level (prime q_i) and to slot `level` (prime P), NTT form.
void orc_modup(const OrcCtx* c, const u64* x, u32 level, u64* digits) {
  const u64 n = c->n;
  const u32 slots = level + 1;
#pragma omp parallel for schedule(dynamic)
  for (int jj = 0; jj < (int)level; ++jj) {
    const u32 j = (u32)jj;
    std::vector<u64> coef(limb(x, n, j), limb(x, n, j) + n);
    intt_mod(c, coef.data(), j);
    std::vector<int64_t> d(n);
    for (u64 k = 0; k < n; ++k) d[k] = balanced(coef[k], c->q[j]);
    for (u32 i = 0; i < slots; ++i) {
      const u32 mod_idx = (i < level) ? i : c->L;
      signed_to_ntt(c, d.data(), mod_idx, digits + ((u64)j * slots + i) * n);
    }
  }
}

// ModDown and rescale taken as one rounding (reading A25): for b = 0, 1, the extended-basis value
// Z = P * A_b + U_b over q_0..q_{level-1} (U_b's P limb alone at P), divided by P q_{level-1} with
// rounding: out_b[i] = (Z[i] - ([Z]_{P q} mod q_i)) * (P q)^-1 mod q_i, i < level - 1, with [Z]_{P q}
// the balanced representative of Z modulo P q_{level-1}, composed from its residues modulo P and
// q_{level-1} (Garner) in 128-bit integers. U [2][level+1][N], A [2][level][N] (NTT form), out
// [2][level-1][N].
static void moddown_rescale(const OrcCtx* c, const u64* U, const u64* A, u32 level, u64* out) {
  const u64 n = c->n;
  const u32 L = c->L, slots = level + 1, l = level - 1;
  const u64 P = c->q[L], ql = c->q[l];
  typedef unsigned __int128 u128;
  const u128 pq = (u128)P * ql;
  const u64 pinv_l = invm(P % ql, ql);
  for (u32 b = 0; b < 2; ++b) {
    std::vector<u64> z((u64)level * n);
    for (u32 i = 0; i < level; ++i) {
      const u64 q = c->q[i];
      const u64 pm = P % q;
      for (u64 e = 0; e < n; ++e)
        z[(u64)i * n + e] = addm(mulm(pm, A[((u64)b * level + i) * n + e], q), U[((u64)b * slots + i) * n + e], q);
    }
    std::vector<u64> rp(U + ((u64)b * slots + level) * n, U + ((u64)b * slots + level + 1) * n);
    std::vector<u64> rl(z.begin() + (u64)l * n, z.begin() + (u64)level * n);
    intt_mod(c, rp.data(), L);
    intt_mod(c, rl.data(), l);
    // v = rp + P * ((rl - rp) P^-1 mod q_l) in [0, P q_l), then balanced
    std::vector<u128> v(n);
    std::vector<bool> neg(n);
    for (u64 e = 0; e < n; ++e) {
      const u64 t = mulm(subm(rl[e], rp[e] % ql, ql), pinv_l, ql);
      const u128 x = (u128)rp[e] + (u128)P * t;
      neg[e] = x > (pq - 1) / 2;
      v[e] = neg[e] ? pq - x : x;  // magnitude
    }
    for (u32 i = 0; i < l; ++i) {
      const u64 q = c->q[i];
      std::vector<u64> t(n);
      for (u64 e = 0; e < n; ++e) {
        const u64 r = (u64)(v[e] % q);
        t[e] = neg[e] ? negm(r, q) : r;
      }
      ntt_mod(c, t.data(), i);
      const u64 inv = invm(mulm(P % q, ql % q, q), q);
      u64* dst = out + ((u64)b * l + i) * n;
      for (u64 e = 0; e < n; ++e) dst[e] = mulm(subm(z[(u64)i * n + e], t[e], q), inv, q);
    }
  }
}

// Inner products of (optionally automorphed) digits with a switching key over slots i < level and P:
//   u_b[i] = sum_j tau_g(D_j)[i] * ksk_j[b][i].  u [2][level+1][N].
static void ks_inner_all(const OrcCtx* c, const u64* digits, u32 level, const u64* ksk, u32 key_level, u32 g, u64* u) {
  const u64 n = c->n;
  const u32 L = c->L, slots = level + 1, K = key_level;
  const std::vector<u32> src = automorphism_index(c, g);
#pragma omp parallel for collapse(2) schedule(static)
  for (int b = 0; b < 2; ++b)
    for (int ii = 0; ii < (int)slots; ++ii) {
      const u32 i = (u32)ii;
      const u32 mod_idx = (i < level) ? i : L;
      const u32 key_slot = (i < level) ? i : K;
      const u64 q = c->q[mod_idx];
      u64* acc = u + ((u64)b * slots + i) * n;
      for (u64 k = 0; k < n; ++k) acc[k] = 0;
      for (u32 j = 0; j < level; ++j) {
        const u64* dj = digits + ((u64)j * slots + i) * n;
        const u64* kj = ksk + (((u64)j * 2 + (u64)b) * (K + 1) + key_slot) * n;
        for (u64 k = 0; k < n; ++k) acc[k] = addm(acc[k], mulm(dj[src[k]], kj[k], q), q);
      }
    }
}

// Inner product of (optionally automorphed) digits with a switching key, then ModDown:
//   u_b[i] = sum_j tau_g(D_j)[i] * ksk_j[b][i]  over slots i < level and P,
//   out_b[i] = (u_b[i] - (bal_P(u_b[P]) mod q_i)) * P^-1 mod q_i.
// g = 1 means no automorphism. The key has level key_level >= level. out is [2][level][N].
void orc_keyswitch_digits(const OrcCtx* c, const u64* digits, u32 level, const u64* ksk, u32 key_level, u32 g,
                          u64* out) {
  const u64 n = c->n;
  const u32 L = c->L, slots = level + 1, K = key_level;
  const u64 P = c->q[L];
  const std::vector<u32> src = automorphism_index(c, g);
  std::vector<u64> u((u64)2 * slots * n);
#pragma omp parallel for collapse(2) schedule(static)
  for (int b = 0; b < 2; ++b)
    for (int ii = 0; ii < (int)slots; ++ii) {
      const u32 i = (u32)ii;
      const u32 mod_idx = (i < level) ? i : L;   // chain index
      const u32 key_slot = (i < level) ? i : K;  // limb slot inside the key
      const u64 q = c->q[mod_idx];
      u64* acc = u.data() + ((u64)b * slots + i) * n;
      for (u64 k = 0; k < n; ++k) acc[k] = 0;
      for (u32 j = 0; j < level; ++j) {
        const u64* dj = digits + ((u64)j * slots + i) * n;
        const u64* kj = ksk + (((u64)j * 2 + (u64)b) * (K + 1) + key_slot) * n;
        for (u64 k = 0; k < n; ++k) acc[k] = addm(acc[k], mulm(dj[src[k]], kj[k], q), q);
      }
    }
  for (u32 b = 0; b < 2; ++b) {
    std::vector<u64> top(u.data() + ((u64)b * slots + level) * n, u.data() + ((u64)b * slots + level + 1) * n);
    intt_mod(c, top.data(), L);
#pragma omp parallel for schedule(static)
    for (int ii = 0; ii < (int)level; ++ii) {
      const u32 i = (u32)ii;
      const u64 q = c->q[i];
      std::vector<u64> t(n);
      for (u64 k = 0; k < n; ++k) t[k] = from_signed(balanced(top[k], P), q);
      ntt_mod(c, t.data(), i);
      const u64 pinv = invm(P % q, q);
      const u64* ui = u.data() + ((u64)b * slots + i) * n;
      u64* dst = out + ((u64)b * level + i) * n;
      for (u64 k = 0; k < n; ++k) dst[k] = mulm(subm(ui[k], t[k], q), pinv, q);
    }
  }
}

// Key switch of one NTT-form polynomial x at `level` (O16): out = ModDown(sum_j D_j * ksk_j).
void orc_keyswitch(const OrcCtx* c, const u64* x, u32 level, const u64* ksk, u32 key_level, u64* out) {
  std::vector<u64> digits((u64)level * (level + 1) * c->n);
  orc_modup(c, x, level, digits.data());
  orc_keyswitch_digits(c, digits.data(), level, ksk, key_level, 1, out);
}

// Relinearization (O17) of [3][level][N] -> [2][level][N]: (d0 + KS(d2)_0, d1 + KS(d2)_1).
void orc_relinearize(const OrcCtx* c, const u64* d, u32 level, const u64* rlk, u32 key_level, u64* out) {
  const u64 n = c->n;
  std::vector<u64> ks((u64)2 * level * n);
  orc_keyswitch(c, d + (u64)2 * level * n, level, rlk, key_level, ks.data());
  orc_add(c, d, ks.data(), level, 2, out);
}

// Relinearization and rescale as one rounding (reading A25): [3][level][N] -> [2][level-1][N],
// round((P (d0, d1) + sum_j D_j(d2) * rlk_j) / (P q_{level-1})).
void orc_relinearize_rescale(const OrcCtx* c, const u64* d, u32 level, const u64* rlk, u32 key_level, u64* out) {
  const u64 n = c->n;
  std::vector<u64> digits((u64)level * (level + 1) * n), u((u64)2 * (level + 1) * n);
  orc_modup(c, d + (u64)2 * level * n, level, digits.data());
  ks_inner_all(c, digits.data(), level, rlk, key_level, 1, u.data());
  moddown_rescale(c, u.data(), d, level, out);
}

// Rotation (O18), key switch after the automorphism:
//   (tau_g(c0) + KS(tau_g(c1))_0, KS(tau_g(c1))_1).
void orc_rotate(const OrcCtx* c, const u64* ct, u32 level, u32 g, const u64* gk, u32 key_level, u64* out) {
  const u64 n = c->n;
  std::vector<u64> t((u64)2 * level * n);
  orc_automorphism_ntt(c, ct, 2 * level, g, t.data());
  std::vector<u64> ks((u64)2 * level * n);
  orc_keyswitch(c, t.data() + (u64)level * n, level, gk, key_level, ks.data());
  orc_add(c, t.data(), ks.data(), level, 1, out);
  std::memcpy(out + (u64)level * n, ks.data() + (u64)level * n, sizeof(u64) * level * n);
}

// Hoisted rotation (O18): digits of c1 computed once (orc_modup) and the automorphism applied to
// the digits inside orc_keyswitch_digits: (tau_g(c0) + KS_0, KS_1).
void orc_rotate_from_digits(const OrcCtx* c, const u64* ct, const u64* digits, u32 level, u32 g, const u64* gk,
                            u32 key_level, u64* out) {
  const u64 n = c->n;
  std::vector<u64> ks((u64)2 * level * n);
  orc_keyswitch_digits(c, digits, level, gk, key_level, g, ks.data());
  std::vector<u64> c0g((u64)level * n);
  orc_automorphism_ntt(c, ct, level, g, c0g.data());
  orc_add(c, c0g.data(), ks.data(), level, 1, out);
  std::memcpy(out + (u64)level * n, ks.data() + (u64)level * n, sizeof(u64) * level * n);
}

// Vector x plain matrix by the diagonal method with the ModDown taken once, after the sum over
// rotations ("double hoisting"; the rotation count and the hoisted decomposition are those of the
// single-hoisted product, only the place of the division by P moves). Inputs: ct [2][level][N] (the
// replicated input vector), digits = ModUp(c1) [level][level+1][N], the diagonals over the extended
// basis diag_ext [rows][level+1][N] (the same integer polynomial d_k modulo q_0..q_{level-1} and P),
// and for k = 1..rows-1 the Galois key of rotation k (keys[k-1], level key_levels[k-1], element
// g_elts[k-1]). Steps:
//   1. U_b[i] = sum_{k>=1} (sum_j tau_k(D_j)[i] * gk^(k)_j[b][i]) * d_k[i]   for slots i < level and P;
//   2. A_0[i] = c0[i] d_0[i] + sum_{k>=1} tau_k(c0)[i] d_k[i],  A_1[i] = c1[i] d_0[i]   (i < level);
//   3. out_b[i] = A_b[i] + (U_b[i] - (bal_P(U_b[P]) mod q_i)) * P^-1 mod q_i.
// The caller rescales. out [2][level][N].
static void vecmat_dh_impl(const OrcCtx* c, const u64* ct, const u64* digits, u32 level, u32 rows,
                           const u64* diag_ext, const u64* const* keys, const u32* key_levels, const u32* g_elts,
                           bool merged, u64* out);

void orc_vecmat_dh(const OrcCtx* c, const u64* ct, const u64* digits, u32 level, u32 rows, const u64* diag_ext,
                   const u64* const* keys, const u32* key_levels, const u32* g_elts, u64* out) {
  vecmat_dh_impl(c, ct, digits, level, rows, diag_ext, keys, key_levels, g_elts, false, out);
}

// The same sum with its ModDown and the following rescale taken as one rounding (reading A25):
// out [2][level-1][N].
void orc_vecmat_dh_rs(const OrcCtx* c, const u64* ct, const u64* digits, u32 level, u32 rows, const u64* diag_ext,
                      const u64* const* keys, const u32* key_levels, const u32* g_elts, u64* out) {
  vecmat_dh_impl(c, ct, digits, level, rows, diag_ext, keys, key_levels, g_elts, true, out);
}

static void vecmat_dh_impl(const OrcCtx* c, const u64* ct, const u64* digits, u32 level, u32 rows,
                           const u64* diag_ext, const u64* const* keys, const u32* key_levels, const u32* g_elts,
                           bool merged, u64* out) {
  const u64 n = c->n;
  const u32 L = c->L, slots = level + 1;
  const u64 P = c->q[L];
  std::vector<u64> U((u64)2 * slots * n, 0), A((u64)2 * level * n);
  // step 2, the k = 0 term
  for (u32 b = 0; b < 2; ++b)
    for (u32 i = 0; i < level; ++i)
      for (u64 e = 0; e < n; ++e)
        A[((u64)b * level + i) * n + e] =
            mulm(ct[((u64)b * level + i) * n + e], diag_ext[(u64)i * n + e], c->q[i]);
  for (u32 k = 1; k < rows; ++k) {
    const std::vector<u32> src = automorphism_index(c, g_elts[k - 1]);
    const u64* gk = keys[k - 1];
    const u32 K = key_levels[k - 1];
    const u64* dk = diag_ext + (u64)k * slots * n;
    // step 1
#pragma omp parallel for collapse(2) schedule(static)
    for (int b = 0; b < 2; ++b)
      for (int ii = 0; ii < (int)slots; ++ii) {
        const u32 i = (u32)ii;
        const u32 mod_idx = i < level ? i : L;
        const u32 key_slot = i < level ? i : K;
        const u64 q = c->q[mod_idx];
        u64* acc = U.data() + ((u64)b * slots + i) * n;
        for (u64 e = 0; e < n; ++e) {
          u64 u = 0;
          for (u32 j = 0; j < level; ++j)
            u = addm(u, mulm(digits[((u64)j * slots + i) * n + src[e]],
                             gk[(((u64)j * 2 + (u64)b) * (K + 1) + key_slot) * n + e], q), q);
          acc[e] = addm(acc[e], mulm(u, dk[(u64)i * n + e], q), q);
        }
      }
    // step 2
    for (u32 i = 0; i < level; ++i)
      for (u64 e = 0; e < n; ++e)
        A[(u64)i * n + e] = addm(A[(u64)i * n + e], mulm(ct[(u64)i * n + src[e]], dk[(u64)i * n + e], c->q[i]), c->q[i]);
  }
  if (merged) {
    moddown_rescale(c, U.data(), A.data(), level, out);
    return;
  }
  // step 3
  for (u32 b = 0; b < 2; ++b) {
    std::vector<u64> top(U.data() + ((u64)b * slots + level) * n, U.data() + ((u64)b * slots + level + 1) * n);
    intt_mod(c, top.data(), L);
    for (u32 i = 0; i < level; ++i) {
      const u64 q = c->q[i];
      std::vector<u64> t(n);
      for (u64 e = 0; e < n; ++e) t[e] = from_signed(balanced(top[e], P), q);
      ntt_mod(c, t.data(), i);
      const u64 pinv = invm(P % q, q);
      const u64* ui = U.data() + ((u64)b * slots + i) * n;
      const u64* ai = A.data() + ((u64)b * level + i) * n;
      u64* dst = out + ((u64)b * level + i) * n;
      for (u64 e = 0; e < n; ++e) dst[e] = addm(ai[e], mulm(subm(ui[e], t[e], q), pinv, q), q);
    }
  }
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}


// ----------------------------------------------------- hybrid key switching (reading A26) ------
// The generalisation of O16-O18 to digits of alpha data primes and K special primes P = p_0 ...
// p_{K-1} (the hybrid key switching of Han and Ki, CT-RSA 2020, on the RNS variant of Cheon, Han,
// Kim, Kim and Song, SAC 2018). Digit j at level ell covers the data primes G_j = {q_i : j alpha <= i
// < min((j+1) alpha, ell)}, Q_j their product; dnum(ell) = ceil(ell / alpha) digits. Chain layout:
// q_0..q_{L-1}, then p_0..p_{K-1} (chain indices L..L+K-1). With alpha = 1 and K = 1 every function
// below computes exactly what its one-prime counterpart above computes.
//   switching key of level Kt:  [dnum(Kt)][2][Kt + K][N], limb slot t < Kt is q_t, slot Kt + k is p_k;
//   digits at level ell:        [dnum(ell)][ell + K][N], slot t < ell is q_t, slot ell + k is p_k.

namespace {

u32 hyb_digits(u32 level, u32 alpha) { return (level + alpha - 1) / alpha; }

// Chain index of limb slot t in a layout of `data` data limbs followed by the K special primes.
u32 hyb_chain(const OrcCtx* c, u32 t, u32 data) { return t < data ? t : c->L + (t - data); }

// The product of the special primes modulo q: P mod q.
u64 special_product_mod(const OrcCtx* c, u64 q) {
  u64 r = 1 % q;
  for (u32 k = 0; k < c->K; ++k) r = mulm(r, c->q[c->L + k] % q, q);
  return r;
}

}  // namespace

// Switching key from s' to s (O6 generalised): for digit j < dnum(Kt) and limb slot t,
//   b_j[t] = -a_j[t] s[t] + e_j[t] + [t is a data prime of G_j] * (P mod q_t) * s'[t],
// a_j uniform per limb, e_j CBD; the stream tags of O6 (digit index j). s and s' are NTT form over all
// L + K primes.
void orc_keygen_switch_hyb(const OrcCtx* c, u64 seed, u64 kind, const u64* s, const u64* s_prime, u32 alpha,
                           u32 key_level, u64* ksk) {
  const u32 Kt = key_level, slots = key_level + c->K, dn = hyb_digits(key_level, alpha);
  const u64 n = c->n;
#pragma omp parallel for schedule(dynamic)
  for (int jj = 0; jj < (int)dn; ++jj) {
    const u32 j = (u32)jj;
    const u64 tag_a = (kind << 32) | 0x80000000ull | (2ull * j);
    const u64 tag_e = (kind << 32) | 0x80000000ull | (2ull * j + 1);
    std::vector<int64_t> e(n);
    for (u64 i = 0; i < n; ++i) e[i] = sample_cbd(seed, tag_e, i);
    std::vector<u64> et(n);
    for (u32 t = 0; t < slots; ++t) {
      const u32 l = hyb_chain(c, t, Kt);
      const u64 q = c->q[l];
      signed_to_ntt(c, e.data(), l, et.data());
      u64* b0 = ksk + (((u64)j * 2 + 0) * slots + t) * n;
      u64* b1 = ksk + (((u64)j * 2 + 1) * slots + t) * n;
      const u64* sl = limb(s, n, l);
      const u64* spl = limb(s_prime, n, l);
      const bool in_group = l < c->L && l / alpha == j;
      const u64 gadget = in_group ? special_product_mod(c, q) : 0;
      for (u64 i = 0; i < n; ++i) {
        const u64 a = sample_uniform(seed, tag_a, i, l, q);
        b1[i] = a;
        u64 v = addm(negm(mulm(a, sl[i], q), q), et[i], q);
        if (in_group) v = addm(v, mulm(gadget, spl[i], q), q);
        b0[i] = v;
      }
    }
  }
}

void orc_keygen_relin_hyb(const OrcCtx* c, u64 seed, const u64* s, u32 alpha, u32 key_level, u64* ksk) {
  const u32 nm = (u32)c->q.size();
  std::vector<u64> s2((u64)nm * c->n);
  for (u32 l = 0; l < nm; ++l)
    for (u64 i = 0; i < c->n; ++i) s2[l * c->n + i] = mulm(s[l * c->n + i], s[l * c->n + i], c->q[l]);
  orc_keygen_switch_hyb(c, seed, 0, s, s2.data(), alpha, key_level, ksk);
}

void orc_keygen_galois_hyb(const OrcCtx* c, u64 seed, const u64* s, u32 g, u32 alpha, u32 key_level, u64* ksk) {
  const u32 nm = (u32)c->q.size();
  std::vector<u64> sg((u64)nm * c->n);
  orc_automorphism_ntt(c, s, nm, g, sg.data());
  orc_keygen_switch_hyb(c, seed, g, s, sg.data(), alpha, key_level, ksk);
}

// ModUp (O16 generalised) of x [level][N] (NTT form): for digit j, with x_i the coefficient form of
// limb i and i in G_j,
//   y_i = bal( x_i * [(Q_j / q_i)^-1]_{q_i} mod q_i ),
//   D_j = sum_{i in G_j} y_i * (Q_j / q_i)                (an integer polynomial, |D_j| <= |G_j| Q_j / 2),
// the fast base conversion with balanced terms; D_j mod q_t for every slot t outside G_j (the other
// data primes below `level` and the special primes), NTT form; slot t inside G_j is x_t itself.
void orc_modup_hyb(const OrcCtx* c, const u64* x, u32 level, u32 alpha, u64* digits) {
  const u64 n = c->n;
  const u32 slots = level + c->K, dn = hyb_digits(level, alpha);
  std::vector<std::vector<u64>> coef(level);
#pragma omp parallel for schedule(dynamic)
  for (int ii = 0; ii < (int)level; ++ii) {
    coef[ii].assign(limb(x, n, ii), limb(x, n, ii) + n);
    intt_mod(c, coef[ii].data(), (u32)ii);
  }
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int jj = 0; jj < (int)dn; ++jj)
    for (int tt = 0; tt < (int)slots; ++tt) {
      const u32 j = (u32)jj, t = (u32)tt;
      const u32 g0 = j * alpha, g1 = std::min((j + 1) * alpha, level);
      u64* out = digits + ((u64)j * slots + t) * n;
      if (t >= g0 && t < g1) {  // a prime of the digit itself: the input limb
        std::memcpy(out, limb(x, n, t), sizeof(u64) * n);
        continue;
      }
      const u32 l = hyb_chain(c, t, level);
      const u64 qt = c->q[l];
      for (u64 k = 0; k < n; ++k) out[k] = 0;
      for (u32 i = g0; i < g1; ++i) {
        const u64 qi = c->q[i];
        u64 hat_i = 1 % qi, hat_t = 1 % qt;  // Q_j / q_i modulo q_i and modulo q_t
        for (u32 m = g0; m < g1; ++m)
          if (m != i) {
            hat_i = mulm(hat_i, c->q[m] % qi, qi);
            hat_t = mulm(hat_t, c->q[m] % qt, qt);
          }
        const u64 inv_i = invm(hat_i, qi);
        for (u64 k = 0; k < n; ++k) {
          const int64_t y = balanced(mulm(coef[i][k], inv_i, qi), qi);
          out[k] = addm(out[k], mulm(from_signed(y, qt), hat_t, qt), qt);
        }
      }
      ntt_mod(c, out, l);
    }
}

// Inner product of (optionally automorphed) digits with a switching key of level key_level >= level,
// then ModDown by P (O16 generalised): for b = 0, 1 and every slot t < level + K,
//   u_b[t] = sum_{j < dnum(level)} tau_g(D_j)[t] * ksk_j[b][t'],  t' = t (data) or key_level + k (p_k);
// then with z_k the coefficient form of u_b[p_k] and
//   w_k = bal( z_k * [(P / p_k)^-1]_{p_k} mod p_k ),   C_b = sum_k w_k * (P / p_k)   (|C_b| <= K P / 2),
//   out_b[i] = (u_b[i] - (C_b mod q_i)) * P^-1 mod q_i,  i < level.
void orc_keyswitch_digits_hyb(const OrcCtx* c, const u64* digits, u32 level, u32 alpha, const u64* ksk,
                              u32 key_level, u32 g, u64* out) {
  const u64 n = c->n;
  const u32 K = c->K, slots = level + K, kslots = key_level + K, dn = hyb_digits(level, alpha);
  const std::vector<u32> src = automorphism_index(c, g);
  std::vector<u64> u((u64)2 * slots * n);
#pragma omp parallel for collapse(2) schedule(static)
  for (int b = 0; b < 2; ++b)
    for (int tt = 0; tt < (int)slots; ++tt) {
      const u32 t = (u32)tt;
      const u32 l = hyb_chain(c, t, level);
      const u32 key_slot = t < level ? t : key_level + (t - level);
      const u64 q = c->q[l];
      u64* acc = u.data() + ((u64)b * slots + t) * n;
      for (u64 k = 0; k < n; ++k) acc[k] = 0;
      for (u32 j = 0; j < dn; ++j) {
        const u64* dj = digits + ((u64)j * slots + t) * n;
        const u64* kj = ksk + (((u64)j * 2 + (u64)b) * kslots + key_slot) * n;
        for (u64 k = 0; k < n; ++k) acc[k] = addm(acc[k], mulm(dj[src[k]], kj[k], q), q);
      }
    }
  for (u32 b = 0; b < 2; ++b) {
    // w_k for every special prime, as signed coefficients
    std::vector<std::vector<int64_t>> w(K, std::vector<int64_t>(n));
    for (u32 k = 0; k < K; ++k) {
      const u64 pk = c->q[c->L + k];
      std::vector<u64> z(u.data() + ((u64)b * slots + level + k) * n, u.data() + ((u64)b * slots + level + k + 1) * n);
      intt_mod(c, z.data(), c->L + k);
      u64 hat = 1 % pk;  // P / p_k modulo p_k
      for (u32 m = 0; m < K; ++m)
        if (m != k) hat = mulm(hat, c->q[c->L + m] % pk, pk);
      const u64 inv = invm(hat, pk);
      for (u64 e = 0; e < n; ++e) w[k][e] = balanced(mulm(z[e], inv, pk), pk);
    }
#pragma omp parallel for schedule(static)
    for (int ii = 0; ii < (int)level; ++ii) {
      const u32 i = (u32)ii;
      const u64 q = c->q[i];
      std::vector<u64> t(n, 0);
      for (u32 k = 0; k < K; ++k) {
        u64 hat = 1 % q;  // P / p_k modulo q_i
        for (u32 m = 0; m < K; ++m)
          if (m != k) hat = mulm(hat, c->q[c->L + m] % q, q);
        for (u64 e = 0; e < n; ++e) t[e] = addm(t[e], mulm(from_signed(w[k][e], q), hat, q), q);
      }
      ntt_mod(c, t.data(), i);
      const u64 pinv = invm(special_product_mod(c, q), q);
      const u64* ui = u.data() + ((u64)b * slots + i) * n;
      u64* dst = out + ((u64)b * level + i) * n;
      for (u64 e = 0; e < n; ++e) dst[e] = mulm(subm(ui[e], t[e], q), pinv, q);
    }
  }
}

void orc_keyswitch_hyb(const OrcCtx* c, const u64* x, u32 level, u32 alpha, const u64* ksk, u32 key_level, u64* out) {
  std::vector<u64> digits((u64)hyb_digits(level, alpha) * (level + c->K) * c->n);
  orc_modup_hyb(c, x, level, alpha, digits.data());
  orc_keyswitch_digits_hyb(c, digits.data(), level, alpha, ksk, key_level, 1, out);
}

// Relinearization (O17) with the hybrid key switch: (d0 + KS(d2)_0, d1 + KS(d2)_1).
void orc_relinearize_hyb(const OrcCtx* c, const u64* d, u32 level, u32 alpha, const u64* rlk, u32 key_level,
                         u64* out) {
  const u64 n = c->n;
  std::vector<u64> ks((u64)2 * level * n);
  orc_keyswitch_hyb(c, d + (u64)2 * level * n, level, alpha, rlk, key_level, ks.data());
  orc_add(c, d, ks.data(), level, 2, out);
}

// Rotation (O18) with the hybrid key switch: (tau_g(c0) + KS(tau_g(c1))_0, KS(tau_g(c1))_1).
void orc_rotate_hyb(const OrcCtx* c, const u64* ct, u32 level, u32 alpha, u32 g, const u64* gk, u32 key_level,
                    u64* out) {
  const u64 n = c->n;
  std::vector<u64> t((u64)2 * level * n);
  orc_automorphism_ntt(c, ct, 2 * level, g, t.data());
  std::vector<u64> ks((u64)2 * level * n);
  orc_keyswitch_hyb(c, t.data() + (u64)level * n, level, alpha, gk, key_level, ks.data());
  orc_add(c, t.data(), ks.data(), level, 1, out);
  std::memcpy(out + (u64)level * n, ks.data() + (u64)level * n, sizeof(u64) * level * n);
}

// Hoisted rotation: the digits of c1 (orc_modup_hyb) computed once, the automorphism applied to them
// inside the inner product.
void orc_rotate_from_digits_hyb(const OrcCtx* c, const u64* ct, const u64* digits, u32 level, u32 alpha, u32 g,
                                const u64* gk, u32 key_level, u64* out) {
  const u64 n = c->n;
  std::vector<u64> ks((u64)2 * level * n);
  orc_keyswitch_digits_hyb(c, digits, level, alpha, gk, key_level, g, ks.data());
  std::vector<u64> c0g((u64)level * n);
  orc_automorphism_ntt(c, ct, level, g, c0g.data());
  orc_add(c, c0g.data(), ks.data(), level, 1, out);
  std::memcpy(out + (u64)level * n, ks.data() + (u64)level * n, sizeof(u64) * level * n);
}

}  // extern "C"

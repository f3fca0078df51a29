// Host parameter layer of the GPU library: the modulus chain, roots of unity and the constant
// tables the kernels read. Independent of the CPU oracle (no shared source).
//
// Prime chain: for each requested bit size b in order, the largest prime q < 2^b with
// q == 1 (mod 2N), q > 2^(b-1), not already in the chain (so that a 2N-th root of unity exists
// and the negacyclic NTT of size N is defined modulo q). Root: the smallest primitive 2N-th root.
#include "params.h"

#include <cmath>
#include <cstring>

namespace tcks {

namespace {

typedef unsigned __int128 u128;

inline u64 mulmod_h(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }

u64 powmod_h(u64 base, u64 exp, u64 m) {
  u64 result = 1 % m, x = base % m;
  for (; exp; exp >>= 1, x = mulmod_h(x, x, m))
    if (exp & 1) result = mulmod_h(result, x, m);
  return result;
}

// Strong-probable-prime test to base a (n odd, n > a).
bool sprp(u64 n, u64 a) {
  u64 d = n - 1;
  unsigned r = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++r;
  }
  u64 y = powmod_h(a, d, n);
  if (y == 1 || y == n - 1) return true;
  while (--r) {
    y = mulmod_h(y, y, n);
    if (y == n - 1) return true;
    if (y == 1) return false;
  }
  return false;
}

u32 reverse_bits(u32 v, u32 width) {
  u32 out = 0;
  for (u32 b = 0; b < width; ++b, v >>= 1) out = (out << 1) | (v & 1u);
  return out;
}

}  // namespace

bool is_prime_u64(u64 n) {
  const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : small) {
    if (n == p) return true;
    if (n % p == 0) return false;
  }
  for (u64 a : small)
    if (!sprp(n, a)) return false;
  return true;  // the twelve bases are deterministic below 3.3e24
}

bool find_chain(u32 log_n, const u32* bits, u32 count, std::vector<u64>& chain) {
  chain.clear();
  const u64 step = 2ull << log_n;
  for (u32 k = 0; k < count; ++k) {
    const u32 b = bits[k];
    if (b < 20 || b > 61) return false;
    const u64 hi = 1ull << b, lo = 1ull << (b - 1);
    // candidates are 1 + step * t below 2^b, scanned downward
    u64 t = (hi - 2) / step;
    bool ok = false;
    for (; t > 0; --t) {
      const u64 c = 1 + step * t;
      if (c <= lo) break;
      bool dup = false;
      for (u64 x : chain) dup |= (x == c);
      if (!dup && is_prime_u64(c)) {
        chain.push_back(c);
        ok = true;
        break;
      }
    }
    if (!ok) return false;
  }
  return true;
}

u64 smallest_psi(u64 q, u32 log_n) {
  const u64 n = 1ull << log_n, order = 2 * n;
  if ((q - 1) % order) return 0;
  // A primitive 2N-th root: g^((q-1)/2N) for a g whose power has order exactly 2N (its N-th power is -1).
  u64 root = 0;
  for (u64 g = 2; g < q && !root; ++g) {
    const u64 c = powmod_h(g, (q - 1) / order, q);
    if (powmod_h(c, n, q) == q - 1) root = c;
  }
  if (!root) return 0;
  // The primitive 2N-th roots are exactly root^k for odd k < 2N; take the least of them.
  const u64 r2 = mulmod_h(root, root, q);
  u64 best = root;
  u64 v = root;
  for (u64 k = 1; k < n; ++k) {
    v = mulmod_h(v, r2, q);
    best = v < best ? v : best;
  }
  return best;
}

u64 invmod_h(u64 a, u64 q) { return powmod_h(a, q - 2, q); }

u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

bool build_tables(u32 log_n, const std::vector<u64>& chain, HostTables& out) {
  const u32 nm = (u32)chain.size();
  const u64 n = 1ull << log_n;
  out.log_n = log_n;
  out.chain = chain;
  out.psi.resize(nm);
  out.mods.resize(nm);
  out.pairs.resize((size_t)nm * nm);
  out.tw.assign((size_t)nm * 4 * n, 0);
  out.narrow = true;
  for (u64 q : chain) out.narrow = out.narrow && q < (1ull << 31);
  if (out.narrow) out.tw32.assign((size_t)nm * 4 * n, 0);
  for (u32 i = 0; i < nm; ++i) {
    const u64 q = chain[i];
    const u64 psi = smallest_psi(q, log_n);
    if (!psi) return false;
    out.psi[i] = psi;
    ModConst& m = out.mods[i];
    std::memset(&m, 0, sizeof(m));
    m.q = q;
    m.mu64 = (u64)(~(u128)0 >> 64) / q;  // floor((2^64 - 1) / q) = floor(2^64 / q) for odd q > 1
    const u128 mu = (~(u128)0) / q;       // floor((2^128 - 1) / q) = floor(2^128 / q)
    m.mu_hi = (u64)(mu >> 64);
    m.mu_lo = (u64)mu;
    m.ninv = invmod_h(n % q, q);
    m.ninv_sh = shoup_of(m.ninv, q);
    m.half = (q - 1) / 2;
    m.r64 = (u64)(((u128)1 << 64) % q);
    m.ninv_sh32 = (u64)(((u128)m.ninv << 32) / q);
    m.mu32 = q < (1ull << 31) ? (1ull << 32) / q : 0;
    // twiddles: psi^brv(k) and psi^-brv(k) with Shoup companions
    u64* t0 = &out.tw[((size_t)i * 4 + 0) * n];
    u64* t1 = &out.tw[((size_t)i * 4 + 1) * n];
    u64* t2 = &out.tw[((size_t)i * 4 + 2) * n];
    u64* t3 = &out.tw[((size_t)i * 4 + 3) * n];
    const u64 ipsi = invmod_h(psi, q);
    std::vector<u64> pw(n), ipw(n);
    pw[0] = 1;
    ipw[0] = 1;
    for (u64 k = 1; k < n; ++k) {
      pw[k] = mulmod_h(pw[k - 1], psi, q);
      ipw[k] = mulmod_h(ipw[k - 1], ipsi, q);
    }
    for (u64 k = 0; k < n; ++k) {
      const u32 r = reverse_bits((u32)k, log_n);
      t0[k] = pw[r];
      t1[k] = shoup_of(pw[r], q);
      t2[k] = ipw[r];
      t3[k] = shoup_of(ipw[r], q);
      if (out.narrow) {
        u32* n32 = &out.tw32[(size_t)i * 4 * n];  // (twiddle, Shoup) pairs: forward [N][2], inverse [N][2]
        n32[2 * k] = (u32)pw[r];
        n32[2 * k + 1] = (u32)(((u128)pw[r] << 32) / q);
        n32[2 * n + 2 * k] = (u32)ipw[r];
        n32[2 * n + 2 * k + 1] = (u32)(((u128)ipw[r] << 32) / q);
      }
    }
  }
  for (u32 a = 0; a < nm; ++a)
    for (u32 b = 0; b < nm; ++b) {
      PairConst& p = out.pairs[(size_t)a * nm + b];
      std::memset(&p, 0, sizeof(p));
      p.qa_mod_b = chain[a] % chain[b];
      if (chain[b] < (1ull << 31)) p.qa_mod_b_sh32 = (u64)(((u128)p.qa_mod_b << 32) / chain[b]);
      if (a != b) {
        p.inv_qa = invmod_h(p.qa_mod_b, chain[b]);
        p.inv_qa_sh = shoup_of(p.inv_qa, chain[b]);
        p.inv_qa_sh32 = (u64)(((u128)p.inv_qa << 32) / chain[b]);
      }
    }
  // rotation group: slot j sits at DFT index (5^j mod 2N - 1) / 4 of the size-N/2 transform
  const u64 slots = n / 2;
  out.slot_index.resize(slots);
  u64 g = 1;
  for (u64 j = 0; j < slots; ++j) {
    out.slot_index[j] = (u32)((g - 1) / 4);
    g = (g * 5) & (2 * n - 1);
  }
  // zeta^k = exp(i pi k / N), k < 2N (FP64), as interleaved (re, im)
  out.zeta.resize(4 * n);
  for (u64 k = 0; k < 2 * n; ++k) {
    const double ang = M_PI * (double)k / (double)n;
    out.zeta[2 * k] = std::cos(ang);
    out.zeta[2 * k + 1] = std::sin(ang);
  }
  return true;
}

std::vector<u64> hyb_constants(const std::vector<u64>& chain, u32 L, u32 K, u32 alpha, HybTables* H) {
  const u32 nm = L + K, dn = (L + alpha - 1) / alpha, V = dn * alpha;
  std::vector<u64> v;
  auto section = [&](size_t words) {
    const size_t off = v.size();
    v.resize(off + words, 0);
    return off;
  };
  const size_t o_inv = section((size_t)V * alpha * 2), o_conv = section((size_t)V * alpha * nm),
               o_qg = section((size_t)V * nm), o_dinv = section((size_t)K * 2), o_dconv = section((size_t)K * nm),
               o_dP = section(nm), o_pinv = section((size_t)L * 2);
  // ModUp: digit j holding r primes q_{j alpha + m}, m < r
  for (u32 j = 0; j < dn; ++j)
    for (u32 r = 1; r <= alpha; ++r) {
      if (j * alpha + r > L) break;
      const u32 var = j * alpha + (r - 1);
      for (u32 m = 0; m < r; ++m) {
        const u64 qi = chain[j * alpha + m];
        u64 hat = 1;  // (Q_v / q_i) mod q_i
        for (u32 m2 = 0; m2 < r; ++m2)
          if (m2 != m) hat = mulmod_h(hat, chain[j * alpha + m2] % qi, qi);
        const u64 inv = invmod_h(hat, qi);
        v[o_inv + ((size_t)var * alpha + m) * 2] = inv;
        v[o_inv + ((size_t)var * alpha + m) * 2 + 1] = shoup_of(inv, qi);
        for (u32 t = 0; t < nm; ++t) {
          const u64 qt = chain[t];
          u64 c = 1 % qt;  // (Q_v / q_i) mod q_t
          for (u32 m2 = 0; m2 < r; ++m2)
            if (m2 != m) c = mulmod_h(c, chain[j * alpha + m2] % qt, qt);
          v[o_conv + ((size_t)var * alpha + m) * nm + t] = c;
        }
      }
      for (u32 t = 0; t < nm; ++t) {
        const u64 qt = chain[t];
        u64 c = 1 % qt;  // Q_v mod q_t
        for (u32 m = 0; m < r; ++m) c = mulmod_h(c, chain[j * alpha + m] % qt, qt);
        v[o_qg + (size_t)var * nm + t] = c;
      }
    }
  // ModDown: P = p_0 ... p_{K-1}
  for (u32 k = 0; k < K; ++k) {
    const u64 pk = chain[L + k];
    u64 hat = 1 % pk;
    for (u32 k2 = 0; k2 < K; ++k2)
      if (k2 != k) hat = mulmod_h(hat, chain[L + k2] % pk, pk);
    const u64 inv = invmod_h(hat, pk);
    v[o_dinv + 2 * k] = inv;
    v[o_dinv + 2 * k + 1] = shoup_of(inv, pk);
    for (u32 t = 0; t < nm; ++t) {
      const u64 qt = chain[t];
      u64 c = 1 % qt;
      for (u32 k2 = 0; k2 < K; ++k2)
        if (k2 != k) c = mulmod_h(c, chain[L + k2] % qt, qt);
      v[o_dconv + (size_t)k * nm + t] = c;
    }
  }
  for (u32 t = 0; t < nm; ++t) {
    const u64 qt = chain[t];
    u64 c = 1 % qt;
    for (u32 k = 0; k < K; ++k) c = mulmod_h(c, chain[L + k] % qt, qt);
    v[o_dP + t] = c;
    if (t < L) {
      const u64 inv = invmod_h(c, qt);
      v[o_pinv + 2 * t] = inv;
      v[o_pinv + 2 * t + 1] = shoup_of(inv, qt);
    }
  }
  H->alpha = alpha;
  H->K = K;
  const size_t offs[7] = {o_inv, o_conv, o_qg, o_dinv, o_dconv, o_dP, o_pinv};
  const u64** fields[7] = {&H->up_inv, &H->up_conv, &H->up_qg, &H->down_inv, &H->down_conv, &H->down_P, &H->pinv};
  for (int f = 0; f < 7; ++f) *fields[f] = reinterpret_cast<const u64*>(offs[f]);
  return v;
}

void hyb_bind(const u64* d_base, HybTables* H) {
  const u64** fields[7] = {&H->up_inv, &H->up_conv, &H->up_qg, &H->down_inv, &H->down_conv, &H->down_P, &H->pinv};
  for (int f = 0; f < 7; ++f) *fields[f] = d_base + reinterpret_cast<size_t>(*fields[f]);
}

u64 galois_element(u32 log_n, int64_t step) {
  const int64_t half = (int64_t)1 << (log_n - 1);
  int64_t k = step % half;
  if (k < 0) k += half;
  const u64 mask = (2ull << log_n) - 1;
  u64 g = 1, base = 5;
  for (u64 e = (u64)k; e; e >>= 1, base = (base * base) & mask)
    if (e & 1) g = (g * base) & mask;
  return g;
}

}  // namespace tcks

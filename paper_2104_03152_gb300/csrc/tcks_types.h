// Types shared by the library's host code and its kernels.
#pragma once
#include <cstddef>
#include <cstdint>

namespace tcks {

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;

// Per-prime constants (device copy indexed by chain position; P sits at index L).
struct ModConst {
  u64 q;
  u64 mu64;          // floor(2^64 / q)
  u64 mu_hi, mu_lo;  // floor(2^128 / q)
  u64 ninv, ninv_sh; // N^-1 mod q and its Shoup companion
  u64 half;          // (q - 1) / 2
  u64 r64;           // 2^64 mod q
  u64 ninv_sh32;     // floor(ninv * 2^32 / q) (narrow chains, q < 2^31)
  u64 mu32;          // floor(2^32 / q) (narrow chains, q < 2^31; 0 otherwise)
};

// Pairwise constants for prime a (source) and prime b (target): [a][b].
struct PairConst {
  u64 qa_mod_b;      // q_a mod q_b
  u64 inv_qa;        // q_a^-1 mod q_b (0 when a == b)
  u64 inv_qa_sh;     // Shoup companion of inv_qa
  u64 inv_qa_sh32;   // floor(inv_qa * 2^32 / q_b) (narrow chains)
  u64 qa_mod_b_sh32; // floor(qa_mod_b * 2^32 / q_b) (narrow chains)
};

// Constants of a two-prime CRT lift (P and q_l = the prime a rescale drops): residues modulo P and q_l
// -> the balanced integer modulo P q_l (Garner), used when a ModDown and the following rescale are
// taken as one rounding.
struct Crt2 {
  u64 P, ql;
  u64 pinv_l;          // P^-1 mod q_l
  u64 pq_lo, pq_hi;    // P q_l
  u64 half_lo, half_hi;  // (P q_l - 1) / 2
  u32 l;               // chain index of q_l
  u32 pinv_sh32;       // floor(pinv_l 2^32 / q_l) (narrow chains, q_l < 2^31; 0 otherwise)
};

// Constants of hybrid key switching (digits of alpha data primes, K special primes with product P),
// device pointers. A "group variant" v = j alpha + (r - 1) is digit j holding r primes (the last
// digit of a level holds fewer than alpha); its members are q_{j alpha + m}, m < r, and Q_v their
// product.
struct HybTables {
  const u64* up_inv;     // [variant][alpha][2]: (Q_v / q_i)^-1 mod q_i and its Shoup companion
  const u64* up_conv;    // [variant][alpha][n_mods]: (Q_v / q_i) mod t
  const u64* up_qg;      // [variant][n_mods]: Q_v mod t
  const u64* down_inv;   // [K][2]: (P / p_k)^-1 mod p_k and its Shoup companion
  const u64* down_conv;  // [K][n_mods]: (P / p_k) mod t
  const u64* down_P;     // [n_mods]: P mod t
  const u64* pinv;       // [L][2]: P^-1 mod q_i and its Shoup companion
  u32 alpha, K;
};

// Everything a kernel needs about the modulus chain, passed by value.
struct DevTables {
  const ModConst* mods;    // [n_mods]
  const PairConst* pairs;  // [n_mods][n_mods]
  const u64* tw;           // [n_mods][4][N]: psi^brv(k), Shoup, psi^-brv(k), Shoup
  const u32* tw32;         // [n_mods][2][N][2]: forward, inverse (twiddle, 32-bit Shoup) pairs (narrow chains only)
  u32 log_n;
  u32 n_mods;  // L + K (L + 1 with the one-prime key switch)
  u32 L;       // number of data primes; the special primes (P) follow at chain index L ...
  u32 narrow;  // every prime < 2^31: kernels use 32-bit arithmetic
  u32 limb_threads;  // threads per CTA of the limb kernels (0 = the default for N), set by the autotuner
  u32 dh_rpt;        // requests per thread of the double-hoisted accumulation, 32-bit words (0 = default 2)
  u32* dbg;          // error word of the debug build's device range checks (debug_checks.cuh)
  u32* kerr;         // error word of bounded device waits that gave up and of refused bulk copies
  u32 dh_form;       // double-hoisted accumulation: 0 = per-thread loads; 1, 2, 3, 4 = operands staged
                     // by bulk copies where possible, with 256 x 2, 256 x 3, 128 x 3, 128 x 4 elements
                     // per CTA x stages (set by the autotuner)
  u32 pad3;
};

}  // namespace tcks

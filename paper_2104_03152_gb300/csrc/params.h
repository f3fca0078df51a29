// Host parameter layer: modulus chain, roots, constant tables (see params.cpp).
#pragma once
#include <cstdint>
#include <vector>

#include "tcks_types.h"

namespace tcks {

struct HostTables {
  u32 log_n = 0;
  std::vector<u64> chain;        // data primes then P
  std::vector<u64> psi;          // smallest primitive 2N-th root per prime
  std::vector<ModConst> mods;    // per prime
  std::vector<PairConst> pairs;  // [a][b]
  std::vector<u64> tw;           // [prime][4][N]
  std::vector<u32> tw32;         // [prime][2][N][2]: forward then inverse (twiddle, 32-bit Shoup) pairs (narrow chains)
  bool narrow = false;           // every prime < 2^31
  std::vector<u32> slot_index;   // slot j -> (5^j mod 2N - 1)/4, j < N/2
  std::vector<double> zeta;      // exp(i pi k / N), k < 2N, interleaved (re, im)
};

bool is_prime_u64(u64 n);
bool find_chain(u32 log_n, const u32* bits, u32 count, std::vector<u64>& chain);
u64 smallest_psi(u64 q, u32 log_n);
u64 invmod_h(u64 a, u64 q);
u64 shoup_of(u64 w, u64 q);
bool build_tables(u32 log_n, const std::vector<u64>& chain, HostTables& out);
// Constants of hybrid key switching for the chain (L data primes, then K special primes): one flat
// array (layout of HybTables, sections in its field order); H receives alpha, K and every section's
// offset into the array, which hyb_bind turns into device pointers once the array is on the device.
std::vector<u64> hyb_constants(const std::vector<u64>& chain, u32 L, u32 K, u32 alpha, HybTables* H);
void hyb_bind(const u64* d_base, HybTables* H);
// 5^step mod 2N with step taken modulo N/2 (left rotation by `step` slots).
u64 galois_element(u32 log_n, int64_t step);

}  // namespace tcks

// Internal definitions of the ABI's opaque handles and shared host helpers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tcks.h"
#include "kernels.h"
#include "params.h"

struct tcks_params {
  tcks::u32 log_n;
  std::vector<tcks::u32> bits;
  std::vector<tcks::u64> chain;  // data primes, then the n_special special primes (P their product)
  double scale;
  tcks::u32 n_special = 1;  // hybrid key switching: K > 1 special primes and/or
  tcks::u32 alpha = 1;      // digits of alpha > 1 data primes
};

namespace tcks {

struct GaloisKey {
  u64* d = nullptr;
  u32 K = 0;
};

// Device array of KsKey entries for a list of rotation steps (step 0 = the relinearization key).
struct KeyTable {
  KsKey* d = nullptr;
  u32 n = 0;
  u32 min_K = 0;  // smallest key level in the table
  u32 max_K = 0;  // largest key level in the table
  bool aligned16 = false;  // every key starts on a 16-byte boundary
  bool keys32 = false;     // every key has a 32-bit copy (32-bit chains)
};

// A profiler range around one ABI call (or one stage of a served request group), visible in Nsight
// Systems / Compute timelines; the header-only NVTX calls cost a few nanoseconds when no tool listens.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Status with message, raised by internal helpers and turned into a return code at the ABI.
struct Error {
  tcks_status code;
  std::string msg;
};

}  // namespace tcks

struct tcks_ctx {
  tcks_params params;
  tcks::HostTables host;
  tcks::DevTables T{};
  tcks::FftTables F{};
  tcks::u32 N = 0, L = 0;
  tcks::u32 K = 1, alpha = 1;    // special primes, data primes per key-switching digit
  bool hyb = false;              // hybrid key switching (K > 1 or alpha > 1)
  tcks::HybTables H{};           // its constants (device pointers into d_hyb)
  tcks::u64* d_hyb = nullptr;
  // device tables
  void* d_mods = nullptr;
  void* d_pairs = nullptr;
  tcks::u64* d_tw = nullptr;
  tcks::u32* d_tw32 = nullptr;
  tcks::u32* d_slot = nullptr;
  double* d_zeta = nullptr;
  tcks::u64* d_qwords = nullptr;
  int* d_status = nullptr;
  // execution
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  tcks_allocator alloc{};
  bool has_alloc = false;
  tcks::u32 flags = 0;
  tcks::u64 seed = 0;
  int device = 0;
  // keys
  tcks::u64* sk = nullptr;   // [L+K][N]
  tcks::u64* pk = nullptr;   // [2][L][N]
  tcks::u64* rlk = nullptr;  // [L][2][L+1][N], or with hybrid key switching [dnum(L)][2][L+K][N]
  std::map<tcks::u32, tcks::GaloisKey> galois;  // step mod N/2 -> key
  std::map<std::vector<tcks::u32>, tcks::KeyTable> key_tables;  // cached device key tables
  // 32-bit copies of Galois keys (chains of primes below 2^31), made with the key tables that use them
  // and dropped with them: key -> (copy, words)
  std::map<const tcks::u64*, std::pair<tcks::u32*, tcks::u64>> narrow_keys;
  tcks::u64 table_bytes = 0;
  // References: the caller's handle plus every object made from the context (ciphertexts,
  // plaintexts, matrices, models, graphs). The context is destroyed when the last one goes.
  std::atomic<int> refs{1};

  // Graph capture with a caller allocator, whose callbacks cannot run inside a capture: an uncaptured
  // pass counts the bytes the work allocates (mode RECORD), one block of that size comes from the
  // allocator, and the captured pass takes its allocations from the block in order (mode SERVE; no
  // region is reused, since forked streams would race on it). Blocks that graphs hold are never passed
  // to the allocator's free by dev_free.
  enum ArenaMode { ARENA_OFF = 0, ARENA_RECORD = 1, ARENA_SERVE = 2 };
  struct CaptureArena {
    ArenaMode mode = ARENA_OFF;
    size_t recorded = 0;  // RECORD: bytes requested, each rounded up to 256
    char* base = nullptr;  // SERVE: the block and how much of it is handed out
    size_t used = 0, size = 0;
  } arena;
  std::vector<std::pair<char*, size_t>> graph_blocks;  // blocks held by live graphs

  // Galois keys changed: drop every cached key table.
  void keys_changed();

  void* dev_alloc(size_t bytes);
  void dev_free(void* p);
  tcks::u64 key_bytes() const;
};

struct tcks_ct {
  tcks_ctx* ctx;
  tcks::u64* d;  // [size][level][N]
  tcks::u32 level;
  double scale;
  tcks::u32 size = 2;  // 3: an unrelinearized enc x enc product (c0, c1, c2), decrypted as c0 + c1 s + c2 s^2
};

struct tcks_pt {
  tcks_ctx* ctx;
  tcks::u64* d;  // [level][N]
  tcks::u32 level;
  double scale;
};

struct tcks_matrix {
  tcks_ctx* ctx;
  tcks::u32 rows, cols, level;
  tcks::u32 ext;    // 1: every diagonal also carries its limb modulo the special prime P (last)
  double scale;
  tcks::u64* d;     // [diags][level + ext][N] encoded diagonals
  tcks::u32 diags;  // rows (square form) or the rectangular width m' (rectangular form)
  tcks::u32 rect;   // 1: rectangular (hybrid) diagonals, followed by log2(rows / diags) rotate-and-adds
  tcks::u32 limbs() const { return level + ext; }  // limbs per stored diagonal
};

// An array of `count` ciphertexts of one level and scale in one device allocation (an encrypted
// tensor's storage): ciphertext i at d + i * 2 * level * N.
struct tcks_cta {
  tcks_ctx* ctx;
  tcks::u64* d;
  tcks::u32 count, level;
  double scale;
};

namespace tcks {

void ctx_retain(tcks_ctx* c);
void ctx_release(tcks_ctx* c);

// Device buffer owned by a context, released (stream-ordered) when it goes out of scope.
struct DevBuf {
  tcks_ctx* ctx = nullptr;
  u64* p = nullptr;
  DevBuf() = default;
  DevBuf(tcks_ctx* c, size_t words) : ctx(c), p((u64*)c->dev_alloc(words * sizeof(u64))) {}
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : ctx(o.ctx), p(o.p) { o.p = nullptr; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      if (p) ctx->dev_free(p);
      ctx = o.ctx;
      p = o.p;
      o.p = nullptr;
    }
    return *this;
  }
  ~DevBuf() {
    if (p) ctx->dev_free(p);
  }
  u64* release() {
    u64* r = p;
    p = nullptr;
    return r;
  }
};

void check_cuda(cudaError_t e, const char* what);
void check_launch(const char* what);
[[noreturn]] void fail(tcks_status code, const std::string& msg);
// Record / clear the calling thread's last error for the ABI (api.cpp); count graph-replayed launches.
tcks_status abi_record(tcks_status code, const std::string& msg);
void abi_clear();
void count_launches(u64 n);
// Clear a non-sticky CUDA error left in this thread by a call outside the library's checks (another
// library, or a clean-up call whose status is ignored), so that the next launch check reports only
// its own launch. Sticky errors stay: the next CUDA call reports them again.
void drop_stale_cuda_error();

inline size_t ct_words(const tcks_ctx* c, u32 level) { return (size_t)2 * level * c->N; }
inline size_t pt_words(const tcks_ctx* c, u32 level) { return (size_t)level * c->N; }

tcks_ct* new_ct(tcks_ctx* c, u32 level, double scale);  // uninitialised limbs
tcks_ct* new_ct_sized(tcks_ctx* c, u32 size, u32 level, double scale);  // [size][level][N], uninitialised
// Capture arenas (see tcks_ctx::CaptureArena): arena_record before the uncaptured pass, arena_serve
// after it (one block per context with a caller allocator, recorded in `held`), arena_off after the
// capture; arena_release frees a graph's block when the graph goes.
void arena_record(const std::vector<tcks_ctx*>& ctxs);
void arena_serve(const std::vector<tcks_ctx*>& ctxs, std::vector<std::pair<tcks_ctx*, char*>>& held);
void arena_off(const std::vector<tcks_ctx*>& ctxs);
void arena_release(tcks_ctx* c, char* block);
// Debug builds: synchronize each context's stream, read its error word and fail with
// TCKS_ERR_DEBUG_CHECK (the word cleared) when a range check has set a bit.
void debug_word_check(const std::vector<tcks_ctx*>& ctxs, const char* where);
// After the caller synchronized the context's stream: fail when a kernel recorded a bounded wait that
// gave up (TCKS_ERR_TIMEOUT) or a refused bulk copy (TCKS_ERR_CUDA) in the kernel error word (cleared).
void kernel_error_check(tcks_ctx* c);
// Every operation but the element-wise ones, rescale, mod-switch, decrypt and export takes the
// two-component form: a three-component product has to be relinearized first.
void need_relinearized(const tcks_ct* ct);
// Key switching, one-prime or hybrid as the context says: words of a switching key of level Kt, of
// the digits of one input at level ell, of the P-limb scratch of one (request, rotation); ModUp of
// `count` inputs; the inner products and ModDown of a plan.
u64 ksk_words(const tcks_ctx* c, u32 Kt);
u64 ks_digit_words(const tcks_ctx* c, u32 ell);
u64 ks_top_words(const tcks_ctx* c);
void ks_modup(tcks_ctx* c, const u64* x, u64 x_stride, u32 count, u32 ell, u64* coef_tmp, u64* digits);
void ks_switch(tcks_ctx* c, u32 ell, const KsPlan& plan);
// The fused schedules (vector x matrix products, hoisted rotation sums, the CNN) are written for the
// one-prime key switch: UNSUPPORTED on a context with hybrid key switching.
void need_one_prime_ks(const tcks_ctx* c, const char* what);
tcks_pt* new_pt(tcks_ctx* c, u32 level, double scale);
void free_ct(tcks_ct* ct);

// Internal ops on device buffers (results written to caller-provided buffers).
// Rescale `count` ciphertexts [count][2][ell][N] -> [count][2][ell-1][N].
void op_rescale(tcks_ctx* c, const u64* in, u32 ell, u64* out, u32 count = 1);
// Rescale of `polys` polynomials [polys][ell][N] -> [polys][ell-1][N] (a three-component product: 3).
void op_rescale_polys(tcks_ctx* c, const u64* in, u32 ell, u32 polys, u64* out);
// Relinearize `count` tensor products [count][3][ell][N] -> [count][2][ell][N].
void op_relinearize(tcks_ctx* c, const u64* d3, u32 ell, u64* out, u32 count = 1);
// The same followed by the rescale, both in one rounding -> [count][2][ell-1][N].
void op_relin_rescale(tcks_ctx* c, const u64* d3, u32 ell, u64* out, u32 count = 1);
// Rotations of one ciphertext from shared digits: outs[i] = rot(ct, steps[i]) (each [2][ell][N]).
void op_rotate_hoisted(tcks_ctx* c, const u64* ct, u32 ell, const int32_t* steps, u32 n, u64* const* outs);
// ct_i <- ct_i + rot(ct_i, step) for count ciphertexts at base + i * stride (words).
void op_rotate_add(tcks_ctx* c, u64* base, u64 stride, u32 count, u32 ell, int32_t step);
// out_i = in_i + rot(in_i, step) (+ the plaintext bias [ell][N] on component 0, if given) for count
// ciphertexts in + i in_stride -> out + i out_stride; out must not overlap in. One-prime key switch:
// the additions ride in the ModDown's epilogue.
void op_rotate_add_to(tcks_ctx* c, const u64* in, u64 in_stride, u32 count, u32 ell, int32_t step, u64* out,
                      u64 out_stride, const u64* bias = nullptr);
const GaloisKey& galois_key_for(tcks_ctx* c, int64_t step, u32 ell);
// Device key table for `steps` (0 = relinearization key); every key must cover level ell.
const KeyTable& key_table(tcks_ctx* c, const std::vector<u32>& steps, u32 ell);
u32 step_mod(const tcks_ctx* c, int64_t step);
void encode_into(tcks_ctx* c, const double* d_v, size_t n, double scale, u32 level, u64* pt_out, bool ext = false);
// composite.cpp
void op_sum(tcks_ctx* c, u64* ct, u32 ell);  // in place
// count ciphertexts ct + i * ct_stride at level ell -> out [count][2][ell-1][N]
// input_period: 0, the input holds the vector in slots [0, rows) and zeros elsewhere (replicated over
// all slots first); P, it already repeats with period P (zeros in [rows, P)): replicated from P down
// to rows only (P = rows: no replication).
// bias: a plaintext [ell-1][N] added to component 0 of every output, or null.
void op_vecmat(tcks_ctx* c, const u64* ct, u64 ct_stride, u32 count, u32 ell, const tcks_matrix* M, u64* out,
               u32 input_period = 0, const u64* bias = nullptr);
void op_conv(tcks_ctx* c, const u64* ct, u32 ell, const u64* kernel_pt, u32 taps, u32 windows, u64* out);
// x + sum over steps of rot(x, s) (+ the plaintext bias [ell][N] on component 0, if given); out may alias x.
void op_rotsum_hoisted(tcks_ctx* c, u64* x, u64 cw, u32 count, u32 ell, const std::vector<int32_t>& steps, u64* out,
                       const u64* bias = nullptr);
// sum_k rot(x, s_k) * d_{o,k} (s_0 = 0, s_k = steps[k-1]) for `count` ciphertexts (stride cw) and `outs`
// (1 or 4) diagonal sets over the extended basis: set o at diags + o * set_stride, diagonal k at
// + k * diag_stride, its P limb at p_limb. One ModUp per ciphertext, one ModDown per output; output o
// of ciphertext r at out + r * out_b + o * out_o ([2][ell][N]); scale x's times the diagonals'.
// merged: the ModDown and a rescale by q_{ell-1} in one rounding, outputs [2][ell-1][N]; keep > 0
// (merged only): each output component keeps its first `keep` limbs, [2][keep][N] (a modulus switch).
void op_dh_sum_multi(tcks_ctx* c, const u64* x, u64 cw, u32 count, u32 ell, const std::vector<int32_t>& steps,
                     const u64* diags, u64 diag_stride, u64 set_stride, u32 p_limb, u32 outs, u64* out, u64 out_b,
                     u64 out_o, bool merged = false, u32 keep = 0);

}  // namespace tcks

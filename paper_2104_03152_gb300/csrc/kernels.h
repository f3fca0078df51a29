// Host-side launch wrappers of the library's kernels (one translation unit per kernel family).
#pragma once
#include <cuda_runtime.h>

#include "tcks_types.h"
#include "params.h"

namespace tcks {

// Kernel families for launch accounting and the profiler (profiler.cpp).
enum KernelId : u32 {
  K_NTT_FWD = 0, K_NTT_INV, K_ELEMENTWISE, K_TENSOR, K_DROP, K_MODUP, K_KS_P, K_KS_MODDOWN, K_MULACC, K_KEYGEN,
  K_ENCRYPT, K_ENCODE, K_DECODE, K_VECMAT, K_DECRYPT, K_VECMAT_DH, K_LINCOMB, K_COMBINE, K_COUNT
};
// Scope around one kernel launch: counts it and, while profiling is on, records CUDA events on the
// launching stream before and after it together with its algorithmic bytes.
class Launch {
 public:
  // algo_ops: modular butterflies plus modular multiplies / multiply-accumulates of the launch
  // tag: a launch-shape label the profiler keeps per record (0 = none)
  Launch(KernelId id, cudaStream_t st, double algo_bytes, double algo_ops = 0.0, u32 tag = 0);
  ~Launch();
  Launch(const Launch&) = delete;
  Launch& operator=(const Launch&) = delete;

 private:
  KernelId id_;
  cudaStream_t st_;
  double bytes_;
  double ops_;
  u32 tag_;
  void* a_ = nullptr;
  bool active_ = false;
};

// ---- kern_core.cu
u32 ntt_threads(u32 log_n);
// Raise a kernel's dynamic shared-memory limit to `bytes` and its carveout to the maximum.
void ensure_smem(const void* kernel, size_t bytes);
// count jobs: limb (j % per) of entry (j / per), src + (j/per)*src_outer + (j%per)*N -> dst likewise
// (may alias for in place), prime mod_base + j % per.
// A table of polynomial batches for one NTT launch (same N and chain, their own levels).
struct NttDesc {
  const u64* src;  // [polys][level][N]
  u64* dst;        // [polys][level][N] (may equal src)
  u32 first;       // index of the batch's first limb job in the launch
  u32 level;
  u32 limbs;       // limb jobs of the batch (polys x level)
  u32 pad;
};
constexpr u32 kNttDescMax = 96;
struct NttDescTable {
  NttDesc d[kNttDescMax];  // sorted by `first`, d[0].first == 0
  u32 n;
  u32 pad;
};
void launch_ntt_desc(const DevTables& T, bool inverse, const NttDescTable& tab, u32 total_jobs, cudaStream_t st);
// Polynomial batches of several contexts (N in [2^13, 2^16], one word type) transformed by one
// columns launch and one launch over 8192-element slices: batch i is [polys][level][N] of context
// ctx, from src to dst (equal pointers: in place).
constexpr u32 kMultiCtxMax = 8, kMultiDescMax = 48;
struct MultiNttDesc {
  const u64* src;
  u64* dst;
  u64 first;      // first slice job of the batch in the slices launch
  u64 col_first;  // first column item of the batch in the columns launch
  u32 level, limbs, ctx, pad;
};
struct MultiNttTable {
  DevTables T[kMultiCtxMax];
  MultiNttDesc d[kMultiDescMax];
  u32 n, n_ctx;
  u64 slice_jobs, col_items;
};
struct MultiNttBatch {
  const DevTables* T;
  const u64* src;
  u64* dst;
  u32 polys, level;
};
// True when the batches fit one launch pair (at most kMultiCtxMax contexts and kMultiDescMax batches,
// every N >= 2^13, one word type). Returns the number of launches made (0 when they do not fit).
// understate (debug builds' self-test only, 0 otherwise): declare the last batch `understate` limbs
// shorter than the grid covers, so that its range check has to skip them.
u32 launch_ntt_multi(bool inverse, const MultiNttBatch* batches, u32 n, cudaStream_t st, u32 understate = 0);
// Largest CTA size the limb kernels of each file accept (0 when the query fails).
u32 limb_threads_cap_core(bool narrow, u32 log_c);
u32 limb_threads_cap_keyswitch(bool narrow, u32 log_c);  // the key-switching file's kernels (in the core cap)
u32 limb_threads_cap_sample(bool narrow, u32 log_c);
u32 limb_threads_cap_fft(bool narrow, u32 log_c);
// Bit-packed wire format of a ciphertext [2][level][N] (kern_wire.cu): payload bytes, pack into
// `out` (device), unpack with a range check (status set to 1 on a residue >= q_i).
// Serialized ciphertext: a 16-byte header (magic "TCKS", version 1, kind 0 = both components or
// 1 = c0 and the 8-byte seed of c1 right after the header, log N, level, scale as f64), then the payload.
inline constexpr unsigned char kWireMagic[4] = {'T', 'C', 'K', 'S'};
inline constexpr u64 kWireHeader = 16;
u64 wire_payload_bytes(const DevTables& T, const u64* host_primes, u32 level);
// comps = 2: both components; comps = 1: component 0 only (the seeded format).
void launch_pack(const DevTables& T, const u64* ct, u32 level, unsigned char* out, cudaStream_t st, u32 comps = 2);
void launch_unpack(const DevTables& T, const unsigned char* in, u32 level, u64* ct, int* status, cudaStream_t st,
                   u32 comps = 2);
// count ciphertexts at once: request r's ciphertext at ct + r ct_stride (words), its payload at
// r out_stride / r in_stride (bytes); count * comps <= 65535
void launch_pack_batch(const DevTables& T, const u64* ct, u64 ct_stride, u32 level, unsigned char* out, u64 out_stride,
                       u32 count, cudaStream_t st, u32 comps = 2);
void launch_unpack_batch(const DevTables& T, const unsigned char* in, u64 in_stride, u32 level, u64* ct, u64 ct_stride,
                         u32 count, int* status, cudaStream_t st, u32 comps = 2);
// count limb jobs (job k: limb k % per of batch entry k / per, prime mod_base + k % per), repeated for
// ny entries of a second index y (src + y src_y, dst + y dst_y; one launch on one-CTA limbs).
void launch_ntt(const DevTables& T, bool inverse, const u64* src, u64 src_outer, u64* dst, u64 dst_outer,
                u32 count, u32 mod_base, u32 per, cudaStream_t st, u32 ny = 1, u64 src_y = 0, u64 dst_y = 0);
enum : u32 { OP_ADD = 0, OP_SUB = 1, OP_NEG = 2, OP_MUL_PLAIN = 3, OP_ADD_PLAIN = 4, OP_SUB_PLAIN = 5 };
// [polys][ell][N] operands; plain ops share one plaintext across all polynomials (b_stride = 0) or
// read one plaintext per ciphertext, b_stride words apart.
void launch_elementwise(const DevTables& T, u32 op, const u64* a, const u64* b, u64* out, u32 ell, u32 polys,
                        cudaStream_t st, u64 b_stride = 0);
// count pairs [count][2][ell][N] -> [count][3][ell][N].
void launch_tensor(const DevTables& T, const u64* a, const u64* b, u64* out, u32 ell, u32 count, cudaStream_t st);
void launch_decrypt(const DevTables& T, const u64* ct, const u64* s, u64* pt, u32 ell, cudaStream_t st, u32 size = 2);
// polys polynomials [polys][ell][N] -> [polys][ell-1][N]; top_tmp: [polys][N] scratch.
void launch_rescale(const DevTables& T, const u64* ct, u32 ell, u32 polys, u64* top_tmp, u64* out, cudaStream_t st);
// count inputs x_ntt + c * x_stride ([ell][N] each) -> digits [count][ell][ell+1][N];
// x_coef_tmp: [count][ell][N] scratch.
void launch_modup(const DevTables& T, const u64* x_ntt, u64 x_stride, u32 count, u32 ell, u64* x_coef_tmp,
                  u64* digits, cudaStream_t st);

// A key for rotation index r of a plan: switching key of level K, Galois element g (1 = none).
struct KsKey {
  const u64* key;
  u32 K;
  u32 g;
  const u32* key32;  // the same key's words as 32-bit words (32-bit chains, made with the key table), or null
};
// 32-bit copy of n 64-bit words whose values fit 32 bits (keys of a chain of primes below 2^31).
void launch_narrow_copy(const u64* src, u32* dst, u64 n, cudaStream_t st);
// B requests x R key switches of hoisted digits. Request rq, rotation r: digits + rq*digits_b,
// key keys[r] (device array), P-limb scratch top [R][B][2][N], output out + rq*out_b + r*out_r
// ([2][ell][N]), addends add0 + rq*add0_b / add1 + rq*add1_b ([ell][N], read through the
// automorphism when add_perm is set; null for none).
struct KsPlan {
  const KsKey* keys;
  const u64* digits;
  u64 digits_b;
  u64* top;
  u64* out;
  u64 out_b, out_r;
  const u64* add0;
  u64 add0_b;
  const u64* add1;
  u64 add1_b;
  u32 R, B, add_perm, pad;
  // one-prime ModDown only (k_ks_moddown): addx + rq addx_b ([2][ell][N], unpermuted) added to both
  // components, and the plaintext addp ([ell][N], shared by the requests) to component 0
  const u64* addx;
  u64 addx_b;
  const u64* addp;
};
void launch_keyswitch(const DevTables& T, u32 ell, const KsPlan& plan, cudaStream_t st);
// ---- kern_hybrid.cu: hybrid key switching (digits of H.alpha data primes, H.K special primes).
// ModUp of count inputs x_ntt + c x_stride ([ell][N]) -> digits [count][dnum][ell + K][N] (W words);
// y_coef_tmp: [count][ell][N] scratch.
void launch_modup_hyb(const DevTables& T, const HybTables& H, const u64* x_ntt, u64 x_stride, u32 count, u32 ell,
                      u64* y_coef_tmp, u64* digits, cudaStream_t st);
// The inner products and the ModDown of a plan over hybrid digits (digits_b = dnum (ell + K) N words
// per request); plan.top is [R][B][2][K][N] scratch.
void launch_keyswitch_hyb(const DevTables& T, const HybTables& H, u32 ell, const KsPlan& plan, cudaStream_t st);
// Switching key of level Kt: [dnum(Kt)][2][Kt + K][N] (kern_sample.cu).
void launch_keygen_switch_hyb(const DevTables& T, const HybTables& H, u64 seed, u32 kind, const u64* s, u32 Kt,
                              u64* ksk, cudaStream_t st);
// Relinearization of plan.B tensor products (R = 1, addends add0/add1 = d0, d1) with the rescale by
// q_{ell-1} in the same rounding: out + rq out_b receives [2][ell-1][N]; top2 scratch [B][2][N].
void launch_relin_rescale(const DevTables& T, const HostTables& H, u32 ell, const KsPlan& plan, u64* top2,
                          cudaStream_t st);
Crt2 crt2_constants(const HostTables& H, u32 L, u32 l);
// Vector x plain matrix after ModUp and the P-limb stage of R = n-1 rotations (steps 1..R):
// keys[r] = key of step r+1; top [R][B][2][N] from the KsPlan stage 1; ct + rq*ct_b the input
// ([2][ell][N]); diag + k*diag_stride the diagonal d_k (k = 0..R); partial [B][chunks][2][ell][N]
// scratch. Output out [B][2][ell][N] = sum_k rot(ct, k) * d_k, before the rescale.
struct VecmatPlan {
  const KsKey* keys;
  const u64* digits;
  u64 digits_b;
  const u64* top;
  const u64* ct;
  u64 ct_b;
  const u64* diag;
  u64 diag_stride;
  u64* partial;    // partial of request rq, chunk c: partial + rq * partial_b + c * [2][ell][N]
  u64 partial_b;
  u32 R, B, chunk, chunks;
  u32 accumulate;  // 0: write the chunk partials; 1: add into them (later rotation blocks)
  u32 pad;
};

// Double-hoisted vector x matrix over R = rows - 1 rotations for B requests at level ell (see
// kern_vecmat.cu): keys[r] = the key of rotation r + 1; digits + rq * digits_b the request's ModUp
// digits [ell][ell+1][N]; ct + rq * ct_b its (replicated) ciphertext [2][ell][N]; diag + k *
// diag_stride diagonal k over the extended basis (data limbs from 0, the P limb at p_limb, which is
// the matrix's level and may exceed ell). outs > 1: that many outputs per request from the same
// rotations, output o with the diagonal set at diag + o * diag_set (outs = 0 means 1). partial
// [B * outs][chunks][3][ell+1][N], output o of request rq at index rq * outs + o.
struct VecmatDhPlan {
  const KsKey* keys;
  const u64* digits;
  u64 digits_b;
  const u64* ct;
  u64 ct_b;
  const u64* diag;
  u64 diag_stride;
  u64 diag_set;
  u64* partial;
  u32 R, B, chunk, chunks;
  u32 p_limb, outs;
  u32 keys_aligned;  // every key of `keys` starts on a 16-byte boundary (bulk copies may read it)
  u32 keys_K;        // the level of every key of `keys` when they share one, else 0
  u32 keys32;        // every key of `keys` has its 32-bit copy (key32)
  u32 keep;          // k_vecmat_dh_moddown_rs: limbs kept per output component (0: all ell - 1; fewer: a
                     // modulus switch down to `keep` limbs in the same pass, the dropped limbs never formed)
  const u64* addp;   // k_vecmat_dh_moddown: a plaintext [ell][N] added to component 0 of every output, or null
};
// Outputs per request of a plan (1 or 4).
__host__ __device__ inline u32 dh_outs(const VecmatDhPlan& p) { return p.outs > 1 ? p.outs : 1; }
// CTAs of one chunk of k_vecmat_dh_acc (element blocks x slots x requests).
u32 vecmat_dh_base_ctas(const DevTables& T, u32 ell, const VecmatDhPlan& p);
void launch_vecmat_dh_acc(const DevTables& T, u32 ell, const VecmatDhPlan& p, cudaStream_t st);
// The same accumulation with each rotation's operands staged in shared memory by bulk copies
// (kern_dh_bulk.cu): whether it applies to a plan (T.dh_form 1..4, 32-bit words, level 1..8, 16-byte
// aligned operands), and its launch (rpt requests per thread; the elements per CTA and stages of
// T.dh_form: 1 = 256 x 2, 2 = 256 x 3, 3 = 128 x 3, 4 = 128 x 4).
bool dh_bulk_applies(const DevTables& T, u32 ell, const VecmatDhPlan& p);
void launch_vecmat_dh_acc_bulk(const DevTables& T, u32 ell, const VecmatDhPlan& p, u32 rpt, cudaStream_t st);
void launch_vecmat_dh_fold(const DevTables& T, u32 ell, const VecmatDhPlan& p, cudaStream_t st);
// top [2][B * outs][N] = INTT_P of the folded U_b[P]; out + (rq * outs + o) * out_b receives output o
// of request rq, [2][ell][N] (before the rescale), plus p.addp on component 0 when given.
// out_o: words between consecutive outputs of one request (0: outputs follow each other, out_b apart,
// request-major); with out_o != 0 output o of request rq goes to out + rq * out_b + o * out_o.
void launch_vecmat_dh_moddown(const DevTables& T, u32 ell, const VecmatDhPlan& p, const u64* top, u64* out, u64 out_b,
                              cudaStream_t st, u64 out_o = 0);
// The same ModDown and the following rescale as one rounding: outputs [2][ell-1][N] (same placement
// rules), or [2][p.keep][N] when p.keep > 0; top2 scratch [2][B * outs][N].
void launch_vecmat_dh_moddown_rs(const DevTables& T, const HostTables& H, u32 ell, const VecmatDhPlan& p,
                                 const u64* top, u64* top2, u64* out, u64 out_b, cudaStream_t st, u64 out_o = 0);
// Stage 1 of a KsPlan alone (the P-limb inner product and its INTT into plan.top).
void launch_ks_inner_p(const DevTables& T, u32 ell, const KsPlan& plan, cudaStream_t st);
// The fused ModDown + multiply-accumulate over the plan's R rotations, chunk rotations per CTA.
// CTAs (clusters above N = 2^14) of the fused vector x matrix kernel the GPU runs at once.
u32 vecmat_slots(const DevTables& T);
void launch_vecmat_acc(const DevTables& T, u32 ell, const VecmatPlan& plan, cudaStream_t st);
// out [B][2][ell][N] = ct * diag[0] + sum of plan.chunks partials per request.
void launch_vecmat_reduce(const DevTables& T, u32 ell, const VecmatPlan& plan, u64* out, cudaStream_t st);

// ---- kern_sample.cu (Philox4x64-10 sampler; key = (seed, tag), counter = (index, limb, 0, 0))
// Secret key: ternary, NTT form over the data primes and P: out [L+1][N].
void launch_keygen_secret(const DevTables& T, u64 seed, u64* s, cudaStream_t st);
// Public key (-a*s + e, a) over the L data primes: out [2][L][N].
void launch_keygen_public(const DevTables& T, u64 seed, const u64* s, u64* pk, cudaStream_t st);
// Switching key of level K from s' to s: kind 0 = relinearization (s' = s^2), otherwise the Galois
// element g (s' = tau_g(s)); out [K][2][K+1][N].
void launch_keygen_switch(const DevTables& T, u64 seed, u32 kind, const u64* s, u32 K, u64* ksk, cudaStream_t st);
// Public-key encryption at level ell: out [2][ell][N]; scratch none.
void launch_encrypt(const DevTables& T, u64 seed, const u64* pk, const u64* pt, u32 ell, u64* out, cudaStream_t st);
// Secret-key encryption (c1 = a from the public seed, c0 = -a s + e + m, e from the private seed).
void launch_encrypt_sym(const DevTables& T, u64 seed_a, u64 seed_e, const u64* sk, const u64* pt, u32 ell, u64* out,
                        cudaStream_t st);
// a [ell][N] = the uniform polynomial of seed_a; check: compare instead of writing (status = 1 on a mismatch).
void launch_sym_a(const DevTables& T, u64 seed_a, u32 ell, u64* a, bool check, int* status, cudaStream_t st);
// c1 of count seeded ciphertexts: a + r a_stride receives the uniform polynomial of seeds[r] (device)
void launch_sym_a_batch(const DevTables& T, const u64* seeds, u32 ell, u64* a, u64 a_stride, u32 count, cudaStream_t st);

// ---- kern_fft.cu (FP64 canonical embedding)
struct FftTables {
  const u32* slot_index;  // [N/2]
  const double* zeta;     // [2N][2]
};
// n_in device doubles -> integer coefficients (int64 [N]) at `scale`; *d_status = 1 on overflow.
void launch_encode_coeffs(const DevTables& T, const FftTables& F, const double* d_z, u32 n_in, double scale,
                          i64* d_coeffs, int* d_status, cudaStream_t st);
// int64 coefficients -> NTT-form plaintext [ell][N].
// ext: one more limb (index ell) modulo the special prime P, the extended-basis encoding.
void launch_coeffs_to_ntt(const DevTables& T, const i64* d_coeffs, u32 ell, u64* pt, cudaStream_t st,
                          bool ext = false);
// Coefficient-domain residues [ell][N] -> centred integers as doubles [N] (exact CRT, correctly
// rounded); q_words: [L][MAXW] products Q_l and [L][MAXW] (Q_l - 1)/2 per level.
constexpr u32 CRT_MAXW = 34;
void launch_crt_compose(const DevTables& T, const u64* coef, u32 ell, const u64* d_qwords, double* out,
                        cudaStream_t st);
// p [N] doubles -> slot values [n_out].
void launch_decode_slots(const DevTables& T, const FftTables& F, const double* p, double scale, u32 n_out,
                         double* out, cudaStream_t st);

// ---- kern_poly.cu
// out[count][2][ell][N] = sum_t coef[t][j] * x_t (first ell limbs of [count][2][level[t]][N]) + prev,
// plus cst[j] on component 0 when has_cst (prev may be null, and may equal out). The constants travel
// in the launch's parameters (no host-to-device copy, capturable in a graph).
constexpr u32 kLincombMax = 8, kLincombMaxEll = 32;
struct LincombArgs {
  const u64* x[kLincombMax];
  u32 level[kLincombMax];
  u64 coef[kLincombMax][kLincombMaxEll];  // residues c_t mod q_j
  u64 cst[kLincombMaxEll];
  const u64* prev;
  u32 terms, ell, count, has_cst;
};
void launch_lincomb(const DevTables& T, const LincombArgs& A, u64* out, cudaStream_t st);
// out [count][2][ell][N] = sum_t x_t * m_t slot-wise: x_t = x + t * x_stride ([count][2][ell][N]),
// m_t a plaintext [>= ell][N] (one per term, shared by the ciphertexts).
struct MulSumArgs {
  const u64* x;
  u64 x_stride;
  const u64* m[kLincombMax];
  u32 terms, ell, count, pad;
};
void launch_mulsum(const DevTables& T, const MulSumArgs& A, u64* out, cudaStream_t st);
// Gathered combination over an array of ciphertexts x [count][2][level][N] (ciphertext i at
// x + i * 2 * level * N): out[o] = sum_{t < terms} coef[o][t][j] * x[idx[o][t]] on limb j, for
// `outputs` ciphertexts [outputs][2][level][N]. idx [outputs][terms], coef [outputs][terms][level]
// residues, both on the device.
void launch_combine(const DevTables& T, const u64* x, u32 level, const u32* idx, const u64* coef, u32 outputs,
                    u32 terms, u64* out, cudaStream_t st);

}  // namespace tcks

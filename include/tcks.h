/*
 * tcks.h — C ABI of a GB300 (sm_103a) RNS-CKKS library for encrypted vectors.
 *
 * What it computes: the CKKSVector operations of TenSEAL (arXiv 2104.03152, §2-§3 and Table 3) —
 * a context holding secret, public, relinearization and Galois keys with automatic
 * relinearization / rescaling (§2.1), encode / encrypt / decrypt / decode of up to N/2 real slots
 * per ciphertext (§3), element-wise add / sub / negate / multiply with encrypted or plain operands,
 * rotation, sum, dot products and the vector x plain-matrix product (§3.1), and the im2col
 * convolution (§3.2) — down to the polynomial layer (negacyclic NTT, RNS key switching, Galois
 * automorphisms, rescaling). The CKKS scheme itself (Cheon et al. 2017, which the paper builds on)
 * is implemented in its RNS form with one special prime P and one key-switching digit per prime.
 *
 * Conventions
 *   Handles are opaque. Every `**out` argument receives a newly created object owned by the caller,
 *   released with the matching *_free call. Inputs are never modified unless the call says
 *   "in place". Every call returns a tcks_status (0 = OK, < 0 = error) and never throws; on error no
 *   output is produced and tcks_last_error_detail() (thread-local) explains it.
 *   Levels count data primes: a ciphertext at level l has limbs q_0..q_{l-1}.
 *   Device layouts: a ciphertext is u64 [2][level][N] (NTT form, canonical residues in [0, q_i)),
 *   a plaintext u64 [level][N]. Host buffers use the same row-major layouts.
 *   Concurrency: all work of a context runs asynchronously on the context's CUDA stream, in call
 *   order. Calls that return host data (decode, decrypt-to-host, *_export) synchronise that stream.
 *   A context must not be used from two host threads at once.
 *   Scales are doubles carried with each object: multiplication multiplies them, rescale divides by
 *   the dropped prime (as a double); add / sub require bitwise-equal scales and equal levels.
 */
#ifndef TCKS_H
#define TCKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tcks_status;
enum {
  TCKS_OK = 0,
  TCKS_ERR_INVALID_ARG = -1,     /* null pointer, size out of range, bad layout */
  TCKS_ERR_BAD_PARAMS = -2,      /* N not a power of two in [2^3, 2^16], or no NTT-friendly prime */
  TCKS_ERR_NO_GALOIS_KEY = -3,   /* rotation step without a generated Galois key */
  TCKS_ERR_LEVEL_EXHAUSTED = -4, /* rescale at level 1, or a key trimmed below the needed level */
  TCKS_ERR_SCALE_MISMATCH = -5,  /* add / sub of operands whose scales differ */
  TCKS_ERR_LEVEL_MISMATCH = -6,  /* binary op on operands at different levels */
  TCKS_ERR_OUT_OF_MEMORY = -7,   /* device allocation failed */
  TCKS_ERR_BUDGET_EXCEEDED = -8, /* serving admission: HBM budget would be exceeded */
  TCKS_ERR_CUDA = -9,            /* a CUDA runtime call failed (detail has the CUDA message) */
  TCKS_ERR_TIMEOUT = -10,        /* a bounded wait ran out (tcks_batch_wait, the serving loop) */
  TCKS_ERR_VALUE_OVERFLOW = -11, /* encode: |scale * m_i| >= 2^62 */
  TCKS_ERR_UNSUPPORTED = -12,    /* valid request this build does not implement (detail says what) */
  TCKS_ERR_NOT_READY = -13,      /* serving: the request has not completed yet */
  TCKS_ERR_DEBUG_CHECK = -14     /* debug build: a descriptor index or bound check failed (detail says which) */
};

const char* tcks_status_string(tcks_status s);
/* Thread-local text of the last error raised on this thread ("" if none). */
const char* tcks_last_error_detail(void);

typedef struct tcks_params tcks_params;
typedef struct tcks_ctx tcks_ctx;
typedef struct tcks_ct tcks_ct;
typedef struct tcks_pt tcks_pt;
typedef struct tcks_matrix tcks_matrix;

/* Optional device allocator (e.g. PyTorch's caching allocator bound by the Python layer). Both
 * callbacks are stream-ordered on `stream`. NULL selects the library's own stream-ordered pool. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, void* stream, void* user);
  void* user;
} tcks_allocator;

/* ---------------------------------------------------------------------------- parameters ---- */
/* Coefficient-modulus chain (the CKKS parameters of §5 and the appendix Tables 4-5: poly degree N = 2^log_n and
 * the bit sizes of the coefficient modulus, last entry = the special prime P). For each bit size
 * in order the prime is the largest c < 2^b, c > 2^(b-1), c == 1 (mod 2N), not chosen before.
 * n_primes >= 2 (at least one data prime plus P), every size in [20, 61]. `scale` is the default
 * encoding scale. */
tcks_status tcks_params_create(uint32_t log_n, const uint32_t* bit_sizes, uint32_t n_primes, double scale,
                               tcks_params** out);
/* The same chain given explicitly: n_primes primes (data primes, then P), each a prime below 2^61,
 * == 1 (mod 2N) and distinct. One chain of primes == 1 (mod 2^17) serves every N <= 2^16. Errors:
 * BAD_PARAMS when a prime fails a condition. */
tcks_status tcks_params_create_primes(uint32_t log_n, const uint64_t* primes, uint32_t n_primes, double scale,
                                      tcks_params** out);
/* Parameters for hybrid key switching (the generalisation of the context's relinearization and
 * Galois keys of §2.1 to fewer, wider digits; the paper has no parameter for it): primes[0..L-1] are
 * the data primes q_i and the last n_special are the special primes p_k, P their product; a
 * key-switching digit covers `alpha` consecutive data primes, so a key switch at level ell has
 * ceil(ell / alpha) digits instead of ell. ModUp lifts each digit's residues to the other data
 * primes and the special primes by an exact balanced base conversion, D_j = sum_{i in digit j}
 * bal(x_i (Q_j/q_i)^-1 mod q_i) (Q_j/q_i); ModDown divides by P with the same conversion from the
 * special primes. Keys of level Kt are [ceil(Kt/alpha)][2][Kt + n_special][N]. n_special and alpha in
 * [1, 8]; every digit's product must stay below P (BAD_PARAMS otherwise). With n_special = alpha = 1
 * this is tcks_params_create_primes. On such a context relinearization, rotation (single, hoisted,
 * batched), sum, dot, power and polyval use the hybrid key switch; the fused vector x matrix
 * products, hoisted rotation sums, the im2col convolution's fused sums and the CNN return
 * UNSUPPORTED. */
tcks_status tcks_params_create_hybrid(uint32_t log_n, const uint64_t* primes, uint32_t n_primes, uint32_t n_special,
                                      uint32_t alpha, double scale, tcks_params** out);
void tcks_params_free(tcks_params* p);
/* Writes the n_primes chosen primes (data primes, then P) to host `primes`. */
tcks_status tcks_params_primes(const tcks_params* p, uint64_t* primes, uint32_t capacity);

/* ------------------------------------------------------------------------------- context ---- */
/* TenSEAL context (§2.1): generates the secret key (ternary), the public key and the
 * relinearization key from `seed` with the library's counter-based sampler (Philox4x64-10), on
 * the device. flags: TCKS_AUTO_RELIN | TCKS_AUTO_RESCALE (the context's automatic policies).
 * cuda_stream: a cudaStream_t the context works on (NULL = a stream the context creates).
 * The context copies `params`. */
/* TCKS_DOUBLE_HOIST: every vector x plain matrix product of the context (tcks_vecmat_plain,
 * tcks_vecmat_plain_batch, the CNN's fully connected layers, serving lanes) takes the key switch's
 * division by P once, after the sum over rotations, instead of once per rotation (the diagonal
 * method of §3.1 with the same rotations and the same hoisted decomposition; the result decrypts to
 * the same product with less rounding noise, but its limbs differ from the per-rotation schedule).
 * The matrix must carry its diagonals modulo P (tcks_matrix_encode does; see tcks_matrix_import_ext). */
/* TCKS_RECT_DIAG, read by tcks_cnn_create: the network's two fully connected layers use rectangular
 * diagonals (tcks_matrix_encode_rect): FC1 takes 63 hoisted rotations and 2 rotate-and-adds instead
 * of 255 rotations, its output comes out replicated with period 64 and feeds FC2 without the
 * replication rotations, and FC2 takes 15 + 2. The biases are laid out replicated to match; the
 * network needs the Galois steps tcks_cnn_galois_steps reports for this layout. */
/* TCKS_CONV_HOIST, read by tcks_cnn_create: the convolution's rotate-and-add chain over the
 * 2^ceil(log2 taps) tap positions becomes two hoisted rotation sums (tcks_rotate_sum_hoisted), first
 * over the baby steps windows*b (b < B), then over the giant steps windows*B*g (g < G), B G = 2^e,
 * B = 2^floor(e/2): 14 key switches with one ModUp and one ModDown per sum instead of 6 full ones.
 * TCKS_CONV_SHARED (implies the giant-step sum above): the baby-step sum of every kernel k is taken over
 * the input's own rotations, sum_b rot(ct, windows*b) * rot(kernel_k, windows*b) (rot(x * K) =
 * rot(x) * rot(K) slot by slot), with the rotated kernels pre-encoded over the extended basis: one
 * ModUp per request for all kernels, the key-switch sums formed once per rotation, one ModDown per
 * kernel, then the rescale; 1 or 4 kernels. The baby-step keys must cover level L.
 * TCKS_CONV_PACK (implies the baby/giant split): after the baby-step sums the channels are masked to
 * the windows-blocks k + B g (g < G) instead of block k, packed into one ciphertext per request, and
 * one giant-step sum gathers each kernel's full tap sum into its block k: one giant-step sum per
 * request instead of one per kernel, at level L-2. The packed vector repeats every B windows, so the
 * first fully connected layer replicates it from that period (one rotation instead of four at the
 * paper's sizes). Needs kernels <= B and 2^ceil(log2 taps) windows == N/2. */
enum {
  TCKS_AUTO_RELIN = 1u,
  TCKS_AUTO_RESCALE = 2u,
  TCKS_DOUBLE_HOIST = 4u,
  TCKS_RECT_DIAG = 8u,
  TCKS_CONV_HOIST = 16u,
  TCKS_CONV_SHARED = 32u,
  TCKS_CONV_PACK = 64u,
  TCKS_MERGED_RESCALE = 128u,
  TCKS_CONV_FOLD = 256u
};
/* TCKS_CONV_FOLD (with TCKS_CONV_SHARED and TCKS_CONV_PACK): the network's pack masks are folded into
 * the shared baby-step diagonals. A slot-wise mask commutes with the slot-wise diagonal products, so
 * sum_k mask_k * sum_b rot(x, W b) * d_kb = sum_b rot(x, W b) * (sum_k mask_k * d_kb): one
 * diagonal-method sum per request (one ModUp, one ModDown) gives the packed vector, without the
 * per-kernel sums, the masks' products or the pack's rescale; a modulus switch then drops the limb
 * that rescale would have dropped, so every later level and key is unchanged (§5 network; a reading
 * of this library, not the paper's schedule). UNSUPPORTED at model creation without the other two. */
/* TCKS_MERGED_RESCALE: wherever a key switch's ModDown is followed by a rescale (enc x enc multiply
 * with AUTO_RESCALE, the double-hoisted vector x matrix products, the CNN's squares, products and
 * shared convolution sums) the two divisions, by P and by q_last, are one rounding:
 * round((P d + u) / (P q_last)) with the balanced residue modulo P q_last composed from the two
 * dropped limbs. About half the transforms of the ModDown + rescale pair; the limbs equal the two
 * separate roundings' except where those land within 1/q_last of a rounding boundary (a difference of
 * 1 in that integer coefficient). */
tcks_status tcks_context_create(const tcks_params* params, uint64_t seed, uint32_t flags,
                                const tcks_allocator* allocator, void* cuda_stream, tcks_ctx** out);
void tcks_ctx_free(tcks_ctx* ctx);
tcks_status tcks_ctx_info(const tcks_ctx* ctx, uint32_t* log_n, uint32_t* n_data_primes, double* scale);
/* Device bytes held by the context's keys and tables. */
tcks_status tcks_ctx_key_bytes(const tcks_ctx* ctx, uint64_t* bytes);
/* Wait for all work queued on the context's stream. A kernel whose bounded wait for its staged
 * operands ran out (results invalid) is reported here, and by tcks_ct_export, as TCKS_ERR_TIMEOUT. */
tcks_status tcks_ctx_synchronize(tcks_ctx* ctx);
/* Launch shape of the context's kernels (results are bit-identical for every shape): limb_threads =
 * threads per CTA of the limb kernels (0: the default for N; else a multiple of 32 the kernels
 * accept), accum_rpt = requests per thread of the double-hoisted accumulation with 32-bit words (1 or
 * 2: that many everywhere; 0 (default): 4 where every key of a plan sits at its level 4 or 5 at N = 2^13
 * (each key word then serves four requests), 2 elsewhere; 4: 4 wherever every key of a plan sits at its
 * level (levels 1..8, N = 2^13), 2 elsewhere), accum_form = 0 (default): that accumulation loads its
 * operands thread by
 * thread; 1, 2, 3, 4: it stages each rotation's operands in shared memory with bulk copies where the
 * layout allows (32-bit words, level <= 8, 16-byte aligned operands), with 256 x 2, 256 x 3, 128 x 3
 * or 128 x 4 elements per CTA x stages. Set by the autotuners; get reads it back. */
tcks_status tcks_ctx_set_launch_shape(tcks_ctx* ctx, uint32_t limb_threads, uint32_t accum_rpt, uint32_t accum_form);
tcks_status tcks_ctx_get_launch_shape(const tcks_ctx* ctx, uint32_t* limb_threads, uint32_t* accum_rpt,
                                      uint32_t* accum_form);
/* Replace the context's flags (any of the TCKS_* flags above) for the calls
 * that follow; work already queued or captured in a graph keeps the flags it was issued with. */
tcks_status tcks_ctx_set_flags(tcks_ctx* ctx, uint32_t flags);

/* Galois keys for left rotations by `steps` (§2.1, used by rotate / sum / dot / matmul_plain /
 * conv2d_im2col). A step is taken modulo N/2; step 0 needs no key. max_level in [1, L] trims each
 * key to the digits and limbs needed by ciphertexts at levels <= max_level (0 = L). A step that already
 * has a key of at least that level keeps it (a trimmed key holds exactly the first digits and limbs of
 * the longer one); a shorter existing key is replaced. */
tcks_status tcks_gen_galois_keys(tcks_ctx* ctx, const int32_t* steps, uint32_t n_steps, uint32_t max_level);
tcks_status tcks_has_galois_key(const tcks_ctx* ctx, int32_t step, uint32_t* key_level);

/* Key export / import as raw u64 limbs (host). kinds and layouts:
 *   TCKS_KEY_SECRET [L+1][N]; TCKS_KEY_PUBLIC [2][L][N]; TCKS_KEY_RELIN [L][2][L+1][N];
 *   TCKS_KEY_GALOIS [K][2][K+1][N] for the key of `step` (K = its level; limb K is P).
 * n_words must equal the layout size. Import replaces the context's key (for Galois keys, the key
 * of `step` at level `key_level`). */
enum { TCKS_KEY_SECRET = 0, TCKS_KEY_PUBLIC = 1, TCKS_KEY_RELIN = 2, TCKS_KEY_GALOIS = 3 };
tcks_status tcks_export_key(tcks_ctx* ctx, uint32_t kind, int32_t step, uint64_t* host, size_t n_words);
tcks_status tcks_import_key(tcks_ctx* ctx, uint32_t kind, int32_t step, uint32_t key_level, const uint64_t* host,
                            size_t n_words);

/* ---------------------------------------------------------------- encode / encrypt (§3) ---- */
/* Encode n <= N/2 real values (zero-padded) at `scale` (<= 0: the context scale) on limbs
 * q_0..q_{level-1} (level 0 = L): inverse canonical embedding with slot j at zeta^(5^j), FP64 FFT on
 * the device, rounding half away from zero, RNS reduction, NTT. VALUE_OVERFLOW if some
 * |scale * m_i| >= 2^62. v is a host array. */
tcks_status tcks_encode(tcks_ctx* ctx, const double* v, size_t n, double scale, uint32_t level, tcks_pt** out);
/* The same from a device array of n doubles. */
tcks_status tcks_encode_device(tcks_ctx* ctx, const double* d_v, size_t n, double scale, uint32_t level,
                               tcks_pt** out);
/* Decode the first n slots into host `out` (exact CRT to the centred integer, rounded to double,
 * FP64 FFT). Synchronises. */
tcks_status tcks_decode(tcks_ctx* ctx, const tcks_pt* pt, double* out, size_t n);
/* Public-key encryption at the plaintext's level: c0 = u*pk0 + e0 + m, c1 = u*pk1 + e1 with u
 * ternary and e0, e1 centred-binomial, all drawn from `seed`. */
tcks_status tcks_encrypt(tcks_ctx* ctx, const tcks_pt* pt, uint64_t seed, tcks_ct** out);
/* m = c0 + c1*s; for a three-component ciphertext (an unrelinearized product) m = c0 + c1 s + c2 s^2. */
tcks_status tcks_decrypt(tcks_ctx* ctx, const tcks_ct* ct, tcks_pt** out);

/* Raw import / export (host u64, layouts above). Import copies host -> device (asynchronously,
 * then synchronises so `limbs` may be reused). Export synchronises. */
tcks_status tcks_ct_import(tcks_ctx* ctx, const uint64_t* limbs, uint32_t level, double scale, tcks_ct** out);
/* n_words = size * level * N: the export of a three-component ciphertext is [3][level][N]. */
tcks_status tcks_ct_export(const tcks_ct* ct, uint64_t* limbs, size_t n_words);
/* Import of a ciphertext of `size` = 2 or 3 components, host limbs [size][level][N] (NTT form). */
tcks_status tcks_ct_import_sized(tcks_ctx* ctx, const uint64_t* limbs, uint32_t size, uint32_t level, double scale,
                                 tcks_ct** out);
/* Number of components: 2, or 3 for the product of tcks_mul without TCKS_AUTO_RELIN until it is
 * relinearized (§2.1: relinearization is automatic only when the context asks for it). */
tcks_status tcks_ct_size(const tcks_ct* ct, uint32_t* size);
/* The same for a batch: host limbs [count][2][level][N] contiguous; all copies are queued before one
 * wait (use pinned host memory for overlap). export_batch requires one context, one level and
 * two-component ciphertexts. */
tcks_status tcks_ct_import_batch(tcks_ctx* ctx, const uint64_t* limbs, uint32_t count, uint32_t level, double scale,
                                 tcks_ct** outs);
tcks_status tcks_ct_export_batch(const tcks_ct* const* cts, uint32_t count, uint64_t* limbs, size_t n_words);
/* Wire format (the communication of one encrypted inference, §5): a 16-byte header (b"TCKS",
 * version 1, kind 0, log2 N, level, scale as f64, little-endian) and, for component b = 0, 1 and limb
 * i < level, the N NTT-form residues packed with exactly bit_length(q_i) bits each (residue k in bits
 * [k w, (k+1) w) of the limb's ceil(N w / 8)-byte segment, least significant bit first). Packing and
 * unpacking run on the device. serialize writes *written bytes to host `out` (INVALID_ARG when cap is
 * too small); deserialize checks the header against the context and every residue against its prime
 * (INVALID_ARG otherwise). */
tcks_status tcks_ct_serialized_size(const tcks_ct* ct, uint64_t* bytes);
tcks_status tcks_ct_serialize(const tcks_ct* ct, uint8_t* out, uint64_t cap, uint64_t* written);
/* deserialize also reads kind 1 (below) and regenerates c1 from the seed on the device. */
tcks_status tcks_ct_deserialize(tcks_ctx* ctx, const uint8_t* in, uint64_t size, tcks_ct** out);
/* Secret-key encryption of a plaintext at its level (the client holds the secret key): c1 = a, the
 * uniform polynomial drawn from the public seed seed_a (sampler stream 7, NTT form), c0 = -a s + e + m
 * with e drawn from the private seed seed_e (stream 8). seed_e must stay secret; seed_a travels. */
tcks_status tcks_encrypt_symmetric(tcks_ctx* ctx, const tcks_pt* pt, uint64_t seed_a, uint64_t seed_e,
                                   tcks_ct** out);
/* Wire kind 1, the seeded form of such a ciphertext: the header with kind 1, seed_a as a little-endian
 * u64, then component 0 only, packed as in kind 0 (half the bytes of kind 0 plus 8). serialize_seeded
 * checks on the device that c1 is the uniform polynomial of seed_a (INVALID_ARG otherwise, so a
 * ciphertext that has been computed on cannot be sent this way). */
tcks_status tcks_ct_serialized_size_seeded(const tcks_ct* ct, uint64_t* bytes);
tcks_status tcks_ct_serialize_seeded(const tcks_ct* ct, uint64_t seed_a, uint8_t* out, uint64_t cap,
                                     uint64_t* written);
tcks_status tcks_pt_import(tcks_ctx* ctx, const uint64_t* limbs, uint32_t level, double scale, tcks_pt** out);
tcks_status tcks_pt_export(const tcks_pt* pt, uint64_t* limbs, size_t n_words);
tcks_status tcks_ct_info(const tcks_ct* ct, uint32_t* level, double* scale);
tcks_status tcks_pt_info(const tcks_pt* pt, uint32_t* level, double* scale);
/* Device pointer of the [size][level][N] limbs (valid until the ciphertext is freed). */
tcks_status tcks_ct_device_ptr(const tcks_ct* ct, uint64_t** d_limbs);
void tcks_ct_free(tcks_ct* ct);
void tcks_pt_free(tcks_pt* pt);

/* --------------------------------------------------------- element-wise ops (§3, Table 3) ---- */
/* These, tcks_decrypt, tcks_rescale, tcks_mod_switch and tcks_ct_export also take three-component
 * ciphertexts: add / sub give three components when either operand has them (a missing component is
 * zero), negate and mul_plain act on every component, add_plain / sub_plain on c0 only. Every other
 * operation (rotations, sums, products, the vector x matrix product, the convolution, the network,
 * power, polyval, tensors, serving, serialization) refuses them with INVALID_ARG: relinearize first. */
tcks_status tcks_add(const tcks_ct* a, const tcks_ct* b, tcks_ct** out);
tcks_status tcks_sub(const tcks_ct* a, const tcks_ct* b, tcks_ct** out);
tcks_status tcks_negate(const tcks_ct* a, tcks_ct** out);
/* Plain operand: its first level(ct) limbs are used; add / sub need the plaintext at the
 * ciphertext's scale. mul_plain multiplies the scales. */
tcks_status tcks_add_plain(const tcks_ct* a, const tcks_pt* p, tcks_ct** out);
tcks_status tcks_sub_plain(const tcks_ct* a, const tcks_pt* p, tcks_ct** out);
tcks_status tcks_mul_plain(const tcks_ct* a, const tcks_pt* p, tcks_ct** out);
/* enc x enc (§3, Table 3 "mul"; both operands two-component): tensor product (d0, d1, d2) = (a0b0,
 * a0b1 + a1b0, a1b1), then relinearize and rescale as the context's AUTO flags say (§2.1). Without
 * TCKS_AUTO_RELIN the result is the three-component ciphertext (d0, d1, d2), rescaled component by
 * component under TCKS_AUTO_RESCALE; tcks_relinearize turns it into the two-component one. */
tcks_status tcks_mul(const tcks_ct* a, const tcks_ct* b, tcks_ct** out);
tcks_status tcks_square(const tcks_ct* a, tcks_ct** out);
/* Element-wise power x^k (§3, "power" with a circuit of minimum multiplicative depth), k >= 1:
 * x^(2m) = (x^m)^2, and for i not a power of two x^i = x^(2^m) x^(i - 2^m) with 2^m the largest power
 * of two below i. Each product takes both operands to the lower of their levels (limbs dropped),
 * then tensor product, relinearization and rescale, whatever the context's AUTO flags. Result at
 * level(x) - ceil(log2 k) with the product of the scales over the dropped primes; k = 1 copies x.
 * Errors: INVALID_ARG (k = 0, null), LEVEL_EXHAUSTED (level(x) < ceil(log2 k) + 1). The result is a
 * new ciphertext owned by the caller. */
tcks_status tcks_power(const tcks_ct* x, uint32_t k, tcks_ct** out);
/* The same for `count` ciphertexts of one level and scale in batched launches; outs[count]. */
tcks_status tcks_power_batch(const tcks_ct* const* x, uint32_t count, uint32_t k, tcks_ct** outs);
/* Element-wise polynomial p(x) = sum_{i < n_coeffs} coeffs[i] x^i (§3, "polyval"; coeffs host,
 * lowest degree first, trailing zeros ignored, degree d >= 1). The powers with a non-zero
 * coefficient come from one minimum-depth power table (as tcks_power). With l their lowest level,
 * S the context scale and q = q_{l-1}: term i is multiplied by the integer rint(a_i S q / s_i) (s_i
 * its scale, round half to even), the terms are added with rint(a_0 S) q, and one rescale gives
 * the result at level l - 1 = level(x) - ceil(log2 d) - 1 and scale exactly S. Errors:
 * INVALID_ARG (no non-zero coefficient of degree >= 1), LEVEL_EXHAUSTED (level(x) < ceil(log2 d) + 2),
 * VALUE_OVERFLOW (a scaled coefficient of magnitude >= 2^62). */
tcks_status tcks_polyval(const tcks_ct* x, const double* coeffs, uint32_t n_coeffs, tcks_ct** out);
/* The same for `count` ciphertexts of one level and scale (LEVEL_MISMATCH / SCALE_MISMATCH
 * otherwise) in batched launches; outs[count]. */
tcks_status tcks_polyval_batch(const tcks_ct* const* x, uint32_t count, const double* coeffs, uint32_t n_coeffs,
                               tcks_ct** outs);
/* Relinearization in place (§2.1, the relinearization keys; the step TCKS_AUTO_RELIN runs inside
 * tcks_mul): a three-component ciphertext (c0, c1, c2) becomes (c0, c1) + KS(c2) with the
 * relinearization key (one ModUp of c2, the inner product with the key's digits, one ModDown by P), the
 * same result, bit for bit, as tcks_mul with TCKS_AUTO_RELIN and without TCKS_AUTO_RESCALE. A
 * two-component ciphertext is left as it is. Errors: INVALID_ARG (null), OUT_OF_MEMORY, CUDA_ERROR;
 * the ciphertext is unchanged on error. */
tcks_status tcks_relinearize(tcks_ct* ct);
/* Rescale in place: divide by the last prime with rounding (level - 1, scale / q_last); a
 * three-component ciphertext is rescaled component by component. */
tcks_status tcks_rescale(tcks_ct* ct);
/* Drop limbs level..ell-1 in place (scale unchanged), of every component. */
tcks_status tcks_mod_switch(tcks_ct* ct, uint32_t level);
/* Rescale that allocates no memory, for callers that must not allocate at all while they run: for
 * example a serving loop that reserves all of its device memory when it starts and admits work
 * against that fixed budget, so a library call that grows the allocator's pool (or blocks inside
 * it) would break its accounting. The paper has no counterpart; this is a variant of tcks_rescale
 * with the same result, bit for bit.
 * d_in: device [2][level][N] ciphertext limbs (NTT form) of `ctx`; d_out: device [2][level-1][N],
 * not overlapping d_in; both owned by the caller. The output's scale is the input's divided by
 * q_{level-1}, which the caller tracks. Its only scratch (two limbs) is a static device array of
 * 2 x 2^14 u64 words (256 KB), which every GPU that loads the library holds until the process
 * exits; N above 2^14 is rejected with TCKS_ERR_INVALID_ARG. The first call on a device looks up
 * that array's address, so make one call on each device before any stream capture. Every call
 * raises, where needed, the shared-memory limit of its two kernels (a host-side function
 * attribute that only ever grows; no memory is allocated). All calls share the one array: calls that can overlap on
 * the GPU (different streams, or different contexts on the same device) race on it and must be
 * serialised by the caller. Nothing in the array needs to start at zero. Asynchronous on the
 * context's stream; errors: INVALID_ARG, LEVEL_EXHAUSTED (level < 2), CUDA_ERROR. */
tcks_status tcks_rescale_noalloc(tcks_ctx* ctx, const uint64_t* d_in, uint32_t level, uint64_t* d_out);

/* Negacyclic NTT (inverse = 0) or INTT (inverse = 1), in place, of `polys` polynomials of `level`
 * limbs laid out [polys][level][N] in device memory: limb l of every polynomial is transformed
 * modulo q_l. Forward: natural order in, bit-reversed order out, out_j = sum_i a_i
 * psi_l^((2 brv(j) + 1) i) with psi_l the smallest primitive 2N-th root of unity mod q_l; the
 * inverse undoes it exactly. Inputs must be canonical residues. Asynchronous on the context stream.
 * (The transform CKKS uses for every polynomial product, implied by §2's CKKS backend.) */
tcks_status tcks_ntt_inplace(tcks_ctx* ctx, uint64_t* d_limbs, uint32_t polys, uint32_t level, int32_t inverse);

/* ------------------------------------------------------------------------------ rotations ---- */
/* Left rotation of the N/2 slots by `step` (Galois automorphism 5^step mod 2N + key switch). */
tcks_status tcks_rotate(const tcks_ct* a, int32_t step, tcks_ct** out);
/* Several rotations of one ciphertext sharing one decomposition of c1 (hoisting). outs[i] receives
 * the rotation by steps[i]; results are bit-identical to tcks_rotate. */
tcks_status tcks_rotate_hoisted(const tcks_ct* a, const int32_t* steps, uint32_t n_steps, tcks_ct** outs);

/* a + sum over steps of rot(a, steps[i]) with the rotations hoisted and the key switch's division by P
 * taken once, after the sum (one ModUp and one ModDown for all the steps). Every step needs its Galois
 * key; step 0 is rejected (the identity term is always included). The scale is unchanged. */
tcks_status tcks_rotate_sum_hoisted(const tcks_ct* a, const int32_t* steps, uint32_t n_steps, tcks_ct** out);

/* ----------------------------------------------------------------- composite ops (§3.1) ---- */
/* Rotate-and-add over all N/2 slots (slots >= n must be zero): every slot receives the total.
 * Needs Galois keys for steps 1, 2, 4, ..., N/4. */
tcks_status tcks_sum(const tcks_ct* a, uint32_t n, tcks_ct** out);
/* dot(a, b) = sum(mul(a, b)); dot_plain(a, w) = sum(rescale(a * encode(w))) with w (host, n values)
 * encoded at the context scale and a's level. */
tcks_status tcks_dot(const tcks_ct* a, const tcks_ct* b, uint32_t n, tcks_ct** out);
tcks_status tcks_dot_plain(const tcks_ct* a, const double* w, uint32_t n, tcks_ct** out);

/* Plain matrix for the vector x matrix product y = v M (M is rows x cols, rows = n inputs,
 * cols = m outputs, m <= n, n a power of two dividing N/2), stored as its n generalised diagonals
 * d_k[s] = M[(s+k) mod n][s] (s < m), each encoded at `level` and the context scale.
 * From host doubles (row-major M; each diagonal is also kept modulo P for the double-hoisted
 * product) or from pre-encoded host limbs [n][level][N]. */
tcks_status tcks_matrix_encode(tcks_ctx* ctx, const double* M, uint32_t rows, uint32_t cols, uint32_t level,
                               tcks_matrix** out);
tcks_status tcks_matrix_import(tcks_ctx* ctx, const uint64_t* diag_limbs, uint32_t rows, uint32_t cols,
                               uint32_t level, double scale, tcks_matrix** out);
/* Rectangular (hybrid) form of the same rows x cols matrix: m' = the smallest power of two >= cols
 * diagonals d_k[t] = M[(t' + k) mod rows][t' mod m'] (t' = t mod rows; zero where t' mod m' >= cols),
 * each over the extended basis. The product then takes m' - 1 hoisted rotations instead of rows - 1,
 * rescales, and finishes with log2(rows / m') rotate-and-adds by m' 2^j: slots s < cols hold
 * y_s = sum_i v_i M[i][s], the other slots partial sums (mask them before reusing the ciphertext as a
 * zero-padded vector). Galois keys needed: steps 1..m'-1, m' 2^j, and the replication steps. */
tcks_status tcks_matrix_encode_rect(tcks_ctx* ctx, const double* M, uint32_t rows, uint32_t cols, uint32_t level,
                                    tcks_matrix** out);
/* A rectangular-form matrix from pre-encoded host limbs over the extended basis: [m'][level+1][N]. */
tcks_status tcks_matrix_import_rect(tcks_ctx* ctx, const uint64_t* diag_limbs, uint32_t rows, uint32_t cols,
                                    uint32_t level, double scale, tcks_matrix** out);
/* The same with each diagonal also given modulo the special prime P: [rows][level+1][N], limb
 * `level` of each diagonal modulo P (the same integer polynomial as the data limbs). Needed by the
 * double-hoisted product (TCKS_DOUBLE_HOIST). */
tcks_status tcks_matrix_import_ext(tcks_ctx* ctx, const uint64_t* diag_limbs, uint32_t rows, uint32_t cols,
                                   uint32_t level, double scale, tcks_matrix** out);
void tcks_matrix_free(tcks_matrix* m);
/* Encrypted vector (slots [0, n), zeros elsewhere) times plain matrix (§3.1): replicate the input
 * over the N/2 slots with left rotations (if n < N/2), y = sum_k rot(ct, k) * d_k with hoisted
 * rotations, then rescale. Result: y in slots [0, m), zeros elsewhere. Needs Galois keys for the
 * replication steps N/2 - n*2^i and for steps 1..n-1. */
tcks_status tcks_vecmat_plain(const tcks_ct* a, const tcks_matrix* M, tcks_ct** out);
/* `count` ciphertexts of one level and scale times the same matrix in one batched pass: ModUp
 * once per ciphertext, every rotation's key read once for the whole batch. outs[i] is
 * bit-identical to tcks_vecmat_plain(in[i], M). */
tcks_status tcks_vecmat_plain_batch(const tcks_ct* const* in, uint32_t count, const tcks_matrix* M, tcks_ct** outs);

/* Client-side im2col (§3.2, host only, no context): windows of a kh x kw kernel sliding with
 * `stride` over an H x W image (row-major), windows ordered row-major, taps row-major; slot
 * t*n_windows + w receives tap t of window w (the vertical scan of the windows-as-rows matrix).
 * Fills out_slots[0..cap) (zeros after the last tap). */
tcks_status tcks_im2col_encode(const double* img, uint32_t H, uint32_t W, uint32_t kh, uint32_t kw, uint32_t stride,
                               double* out_slots, size_t cap, uint32_t* n_windows);
/* Encrypted im2col input times one plain kernel (§3.2): one multiplication by the kernel laid out
 * as the input (slot t*windows + w = kernel[t]), rescale, then ceil(log2(taps)) left rotate-and-adds
 * by windows*2^i. Every block of `windows` slots then holds the convolution output. */
tcks_status tcks_conv2d_im2col(const tcks_ct* a, const double* kernel, uint32_t taps, uint32_t windows,
                               tcks_ct** out);
/* The same with the laid-out kernel already encoded (at the input's level). */
tcks_status tcks_conv2d_im2col_pt(const tcks_ct* a, const tcks_pt* kernel, uint32_t taps, uint32_t windows,
                                  tcks_ct** out);

/* Autotuner: picks the CTA size of the limb kernels (transforms and their fused key-switch,
 * rescale and ModUp work) for this context's N and word type by timing a batched transform at each
 * candidate, and applies it to the context. With a cache_path (JSON, keyed by GPU name, log N and
 * word size) a stored choice is reused and a new one recorded. Results are unchanged (bit-exact);
 * only the launch shape moves. *chosen_threads may be NULL. */
tcks_status tcks_autotune(tcks_ctx* ctx, const char* cache_path, uint32_t* chosen_threads);
/* Autotuner of the batched encrypted network (declared here, takes the model of tcks_cnn_create): times
 * a whole batched forward pass of `batch` requests for every combination of limb-kernel CTA size
 * (N/64, N/32, N/16 threads per slice), double-hoisted accumulation requests per thread (0, 2, 4 or 1) and
 * accumulation form (per-thread loads, or operands staged by bulk copies in one of four shapes; see
 * tcks_ctx_set_launch_shape; the last two for 32-bit words), keeps the fastest on the model's context (tcks_ctx_set_launch_shape) and, with a cache_path,
 * records it under the GPU name, log N, word size and batch (a later call reads it back). Results are
 * bit-identical for every shape. The chosen_* pointers may be NULL. Synchronises. */
typedef struct tcks_cnn tcks_cnn;
tcks_status tcks_cnn_autotune(const tcks_cnn* m, uint32_t batch, const char* cache_path, uint32_t* chosen_threads,
                              uint32_t* chosen_rpt, uint32_t* chosen_form);

/* --------------------------------------------------- batched launches (descriptor table) ---- */
/* A batch of independent jobs over raw device buffers, possibly of several contexts (different N)
 * and levels, run as one unit: the NTT/INTT jobs of a context go out as ONE launch over a
 * descriptor table (mixed levels and buffers), the key-switch jobs of a context as one batched
 * launch sequence per (level, op), and the contexts' streams run concurrently (forked from and
 * joined back into the first job's context stream). Results are bit-identical to the single
 * calls (tcks_ntt_inplace, tcks_relinearize, tcks_rotate). The batching of homomorphic work on
 * the device is this library's replacement for the CPU thread pool of §2; the paper has no
 * counterpart for the call itself.
 *   TCKS_JOB_NTT / TCKS_JOB_INTT: count polynomials [count][level][N] from d_in to d_out (equal
 *     pointers transform in place); canonical residues in, forward output bit-reversed.
 *   TCKS_JOB_RELIN: count size-3 ciphertexts d_in [count][3][level][N] (NTT form) to d_out
 *     [count][2][level][N] with the relinearization key.
 *   TCKS_JOB_ROTATE: count ciphertexts d_in [count][2][level][N] rotated left by `step` slots to
 *     d_out (same shape; must not overlap d_in); needs the Galois key for `step`.
 * The jobs are independent: no job reads another's output, and they may run in any order or at
 * once. Pointers may be NULL when count is 0 (the job is skipped).
 * Buffers are the caller's; they must stay valid until the work completes. Asynchronous: wait
 * with tcks_ctx_synchronize on jobs[0].ctx. Errors: INVALID_ARG (null pointer, unknown op, level
 * out of range), NO_GALOIS_KEY, LEVEL_EXHAUSTED (key trimmed below the level), OUT_OF_MEMORY, CUDA;
 * nothing is launched when validation fails. */
enum { TCKS_JOB_NTT = 0, TCKS_JOB_INTT = 1, TCKS_JOB_RELIN = 2, TCKS_JOB_ROTATE = 3 };
typedef struct {
  tcks_ctx* ctx;
  uint32_t op;
  int32_t step;
  uint32_t count;
  uint32_t level;
  const uint64_t* d_in;
  uint64_t* d_out;
} tcks_batch_job;
tcks_status tcks_batch_run(const tcks_batch_job* jobs, uint32_t n_jobs);
/* The same batch submitted with a handle to wait on (the paper has no
 * counterpart): tcks_batch_submit validates and queues the jobs exactly as tcks_batch_run does, then
 * records a completion point on jobs[0].ctx's stream (after every context's work has joined it) and
 * returns *out, owned by the caller. tcks_batch_wait waits on the host for that point: TCKS_OK once
 * every job has completed; TCKS_ERR_TIMEOUT when timeout_ns nanoseconds passed first (0 polls once;
 * a negative timeout waits without limit) -- the handle stays valid and the work keeps running, so
 * wait again or free it; TCKS_ERR_CUDA when the device reported an error. tcks_batch_free waits for
 * the work (without limit) before it releases the handle and the contexts it retains. */
typedef struct tcks_batch tcks_batch;
tcks_status tcks_batch_submit(const tcks_batch_job* jobs, uint32_t n_jobs, tcks_batch** out);
tcks_status tcks_batch_wait(tcks_batch* b, int64_t timeout_ns);
void tcks_batch_free(tcks_batch* b);
/* The batch captured once as a CUDA graph (after one eager run that builds the key tables) and
 * replayed by tcks_batch_graph_run on jobs[0].ctx's stream over the same buffers. With the library's
 * pool allocator the graph holds stream-ordered allocation nodes; a context with a caller allocator
 * (whose callbacks cannot run inside a capture) gets one scratch block from its allocator, sized by a
 * second uncaptured pass, which the graph holds until tcks_batch_graph_free. launches: kernels per
 * replay. */
typedef struct tcks_batch_graph tcks_batch_graph;
tcks_status tcks_batch_graph_create(const tcks_batch_job* jobs, uint32_t n_jobs, tcks_batch_graph** out);
tcks_status tcks_batch_graph_run(tcks_batch_graph* g);
tcks_status tcks_batch_graph_launches(const tcks_batch_graph* g, uint64_t* launches);
void tcks_batch_graph_free(tcks_batch_graph* g);

/* -------------------------------------------- persistent executor (device work queue) ---- */
/* A kernel that stays resident and takes NTT / INTT work from a queue instead of one launch per job
 * (for streams of small transforms, such as a serving loop's, where a launch costs as much as the
 * work; the paper has no counterpart). tcks_executor_start launches it on a stream of its own (one CTA
 * per SM; N <= 2^13, one CTA per limb) with a ring of `capacity` one-limb tasks in pinned, mapped host
 * memory. tcks_executor_post queues a job: polys polynomials [polys][level][N] from d_in to d_out
 * (device buffers of the executor's context that stay valid until the ticket completes; limb l of
 * each polynomial modulo q_l; forward: natural order in, bit-reversed out; results equal
 * tcks_ntt_inplace), and returns a ticket. tcks_executor_wait waits on the host for the ticket (a
 * negative timeout waits without limit; TCKS_ERR_TIMEOUT when timeout_ns passes first). Every wait
 * inside the kernel is bounded: when no task is published for idle_timeout_ns (the GPU's global timer,
 * with an iteration cap as well), the kernel writes TCKS_ERR_TIMEOUT to its status word and every CTA
 * leaves; later posts and waits then return that status. tcks_executor_close stops the kernel (and
 * waits, bounded, for it to leave) and returns the status word (0, TCKS_ERR_TIMEOUT, or in a debug
 * build TCKS_ERR_DEBUG_CHECK for a task that failed its range check); tcks_executor_free closes if needed and releases everything. While the kernel is resident, a
 * device-wide synchronize (cudaDeviceSynchronize, and calls that imply one such as cudaFree) waits
 * for it to leave, i.e. until close or the idle limit: synchronize streams instead, and have d_in
 * written (its stream synchronized) before the post. Errors: INVALID_ARG, UNSUPPORTED (N > 2^13),
 * TIMEOUT, CUDA_ERROR. */
typedef struct tcks_executor tcks_executor;
enum { TCKS_EXEC_NTT = 0, TCKS_EXEC_INTT = 1 };
tcks_status tcks_executor_start(tcks_ctx* ctx, uint32_t capacity, int64_t idle_timeout_ns, tcks_executor** out);
tcks_status tcks_executor_post(tcks_executor* e, uint32_t op, const uint64_t* d_in, uint64_t* d_out, uint32_t polys,
                               uint32_t level, uint64_t* ticket);
tcks_status tcks_executor_wait(tcks_executor* e, uint64_t ticket, int64_t timeout_ns);
tcks_status tcks_executor_close(tcks_executor* e, int32_t* device_status);
void tcks_executor_free(tcks_executor* e);

/* ------------------------------------------------------------------ launch accounting ---- */
/* Integer-pipe ceiling for the roofline of the ALU-bound kernels: modular butterflies per second
 * (the library's Cooley-Tukey butterfly with a Shoup twiddle product, registers only, every SM
 * busy) on the current device for 64-bit (q < 2^62) or 32-bit (q < 2^31) words. A measurement aid
 * with no counterpart in the paper. Synchronous; errors: INVALID_ARG, CUDA. */
tcks_status tcks_calibrate_butterflies(uint32_t word_bits, double* per_second);
/* The same for modular multiply-accumulates in the form of the key-switch sums (products summed lazily,
 * one reduction per eight products; for 32-bit words in plain 64-bit sums of four): product-accumulates
 * per second, the ceiling of the kernels whose work is sums of products rather than transforms. */
tcks_status tcks_calibrate_macs(uint32_t word_bits, double* per_second);
/* The product-accumulate rate of the double-hoisted vector x matrix accumulation in its own form at
 * level ell (1..8; 32-bit words, two requests per thread): the unreduced key-switch sums over ell
 * digits, their carry-chain products with the diagonal and the c0 product, from registers, each of
 * the kernel's loads replaced by one logic op. The measured ceiling of that kernel's roofline, in the
 * unit it counts (one modular product-accumulate). Uses the current device; a measurement aid. */
tcks_status tcks_calibrate_dh_macs(uint32_t ell, double* per_second);
/* Number of kernel launches the library has issued since it was loaded. */
uint64_t tcks_launch_count(void);
/* Debug build (compiled with TCKS_DEBUG_CHECKS): 1, else 0. A debug build asserts the invariants of
 * every descriptor table a batched launch builds and of the job list it comes from (no job's buffer
 * overlapping another job's output), and its descriptor-driven kernels check each index they take
 * from a descriptor (context, limb within the descriptor's declared range, prime within the chain)
 * before using it: a failed check sets a bit of the context's error word and skips that work item
 * (no trap). Batch runs, graph replays and batch waits then synchronize, read the word of every
 * context involved and return TCKS_ERR_DEBUG_CHECK when a bit is set (clearing it). */
int32_t tcks_debug_checks(void);
/* Debug builds' self-test of the device range checks: transforms (forward NTT, in place) the
 * device buffer d_buf [polys][level][N] of ctx (N in [2^13, 2^16]) through the multi-context
 * descriptor launch with the descriptor declaring `understate` limbs fewer than the grid covers, so
 * that the kernels must skip the last `understate` limbs (left as they were) and report them;
 * *word receives the error word's bits (then cleared). UNSUPPORTED in the default build or for N
 * outside the range. */
tcks_status tcks_debug_selftest(tcks_ctx* ctx, uint64_t* d_buf, uint32_t polys, uint32_t level, uint32_t understate,
                                uint32_t* word);
/* Kernel profiler: while on, every launch is bracketed by CUDA events on its stream and carries its
 * algorithmic bytes (each operand read once, each result written once, each distinct key once).
 * start clears earlier records. read() reports, for kernel family idx < tcks_profile_count(), its
 * name, launches, summed device milliseconds and summed algorithmic bytes (waits for the events). */
tcks_status tcks_profile_start(void);
tcks_status tcks_profile_stop(void);
uint32_t tcks_profile_count(void);
tcks_status tcks_profile_read(uint32_t idx, const char** name, uint64_t* launches, double* ms, double* algo_bytes);
/* Algorithmic integer work of family idx over the profiled launches: modular butterflies of its
 * transforms plus its modular multiplies and multiply-accumulates, one unit each (the unit of
 * tcks_calibrate_butterflies). */
tcks_status tcks_profile_read_ops(uint32_t idx, double* algo_ops);
/* The profiled launches of family idx one by one, in launch order: up to `capacity` records of
 * (shape tag, device ms, algorithmic ops); *count receives the number of launches. The double-hoisted
 * accumulation tags a launch with its level | outputs << 8 | (unit diagonals) << 16. */
tcks_status tcks_profile_records(uint32_t idx, uint32_t capacity, uint32_t* tags, double* ms, double* algo_ops,
                                 uint32_t* count);

/* ---------------------------------------- ciphertext arrays: CKKSTensor storage (§2.3) ---- */
/* TenSEAL's CKKSTensor holds an N-dimensional tensor as a tensor of ciphertexts, with optionally one
 * axis batched into the slots (§2.3). A tcks_cta is the storage of such a tensor: `count`
 * ciphertexts of one level and scale in one device allocation [count][2][level][N] (ciphertext i at
 * i * 2 * level * N words), so that each operation below is one batched pass over all of them. The
 * tensor's shape, broadcasting and axes are the caller's (the Python CKKSTensor). Every array
 * returned is new and owned by the caller (tcks_cta_free); inputs are not modified except by
 * tcks_cta_rescale / tcks_cta_mod_switch. Empty arrays are rejected (INVALID_ARG). */
typedef struct tcks_cta tcks_cta;
enum { TCKS_CTA_ADD = 0u, TCKS_CTA_SUB = 1u, TCKS_CTA_MUL = 2u };
void tcks_cta_free(tcks_cta* a);
tcks_status tcks_cta_info(const tcks_cta* a, uint32_t* count, uint32_t* level, double* scale);
/* Host [count][2][level][N] limbs (NTT form) in and out; n_words must equal count * 2 * level * N. */
tcks_status tcks_cta_import(tcks_ctx* ctx, const uint64_t* limbs, uint32_t count, uint32_t level, double scale,
                            tcks_cta** out);
tcks_status tcks_cta_export(const tcks_cta* a, uint64_t* limbs, size_t n_words);
/* Gather ciphertexts of one level and scale into an array (LEVEL_MISMATCH / SCALE_MISMATCH), and copy
 * ciphertext i out of one. */
tcks_status tcks_cta_from_cts(const tcks_ct* const* cts, uint32_t count, tcks_cta** out);
tcks_status tcks_cta_get(const tcks_cta* a, uint32_t i, tcks_ct** out);
/* Ciphertext i encrypts host values[i*n .. i*n+n) (n <= N/2, the other slots zero) encoded at the
 * context scale on `level` limbs (0: L), with encryption seed seed + i. */
tcks_status tcks_cta_encrypt(tcks_ctx* ctx, const double* values, uint32_t count, uint32_t n, uint32_t level,
                             uint64_t seed, tcks_cta** out);
/* Slots [0, n) of every ciphertext into host values [count][n]. */
tcks_status tcks_cta_decrypt(const tcks_cta* a, double* values, uint32_t n);
/* Element-wise a op b over two arrays of one length and level (add / sub: one scale): one launch;
 * MUL is tensor product + relinearization (+ rescale under TCKS_AUTO_RESCALE) of all pairs. */
tcks_status tcks_cta_binary(uint32_t op, const tcks_cta* a, const tcks_cta* b, tcks_cta** out);
tcks_status tcks_cta_negate(const tcks_cta* a, tcks_cta** out);
/* a op plain, the plaintext of ciphertext i being host values[i*n .. i*n+n) encoded on a's level at
 * a's scale (ADD, SUB) or the context scale (MUL, then rescale under TCKS_AUTO_RESCALE). */
tcks_status tcks_cta_plain(uint32_t op, const tcks_cta* a, const double* values, uint32_t n, tcks_cta** out);
/* Gathered combination: out[o] = sum_{t < terms} c[o][t] * a[idx[o][t]] for o < outputs (host idx,
 * w [outputs][terms]). mode 0: c = w, which must be integers of magnitude below 2^53 (gathers,
 * transposes and sums along tensor axes use w = 1); the scale is a's. mode 1: c = rint(w * S), the
 * constant polynomial of w at the context scale S (products with a plain matrix, scalars per
 * ciphertext); the scale is a's times S, then rescale under TCKS_AUTO_RESCALE. One launch.
 * Errors: INVALID_ARG (index >= count, a non-integer weight in mode 0), VALUE_OVERFLOW (|w S| >= 2^62). */
tcks_status tcks_cta_combine(const tcks_cta* a, const uint32_t* idx, const double* w, uint32_t outputs,
                             uint32_t terms, int32_t mode, tcks_cta** out);
/* Rotate-and-add within every ciphertext by 1, 2, 4, ... below n (n in [1, N/2]): slot 0 then holds the
 * sum of slots [0, 2^ceil(log2 n)), which is the sum of the first n when the slots from n up to that
 * power of two are zero. Needs the Galois keys of those steps (NO_GALOIS_KEY before any launch). */
tcks_status tcks_cta_sum_slots(const tcks_cta* a, uint32_t n, tcks_cta** out);
/* tcks_power / tcks_polyval on every ciphertext of the array (the same circuits, batched). */
tcks_status tcks_cta_power(const tcks_cta* a, uint32_t k, tcks_cta** out);
tcks_status tcks_cta_polyval(const tcks_cta* a, const double* coeffs, uint32_t n_coeffs, tcks_cta** out);
/* In place: rescale every ciphertext (level - 1, scale / q_last); drop limbs down to `level`. */
tcks_status tcks_cta_rescale(tcks_cta* a);
tcks_status tcks_cta_mod_switch(tcks_cta* a, uint32_t level);

/* ------------------------------------------------------------- the encrypted CNN (§5) ---- */
/* The MNIST-shaped network of the paper's evaluation (§5, Table 2): im2col conv with `kernels`
 * kernels of `taps` taps over `windows` windows (§3.2), square, FC (kernels*windows) -> hidden
 * (§3.1), square, FC hidden -> classes. Weights are host doubles: conv_w [kernels][taps], conv_b
 * [kernels], fc1_w [hidden][kernels*windows], fc1_b [hidden], fc2_w [classes][hidden], fc2_b
 * [classes]. All plaintexts are encoded on the device at creation: kernels at level L, channel
 * masks at L-1, FC1 diagonals at L-3, FC2 diagonals at L-5, biases at the scales the schedule
 * reaches from an input at the context scale. Needs L >= 7 data primes (six levels are consumed,
 * the six multiplications the paper counts), power-of-two FC sizes, classes <= hidden <= kernels*windows. */
typedef struct tcks_cnn tcks_cnn;
tcks_status tcks_cnn_create(tcks_ctx* ctx, const double* conv_w, const double* conv_b, uint32_t kernels,
                            uint32_t taps, uint32_t windows, const double* fc1_w, const double* fc1_b, uint32_t hidden,
                            const double* fc2_w, const double* fc2_b, uint32_t classes, tcks_cnn** out);
void tcks_cnn_free(tcks_cnn* m);
/* Rotation steps the forward pass uses and the level each key must cover: (steps[i], levels[i]),
 * i < *count. With steps == NULL only *count is written. */
tcks_status tcks_cnn_galois_steps(const tcks_cnn* m, int32_t* steps, uint32_t* levels, uint32_t cap,
                                  uint32_t* count);
/* One encrypted inference: input = the im2col-encoded image encrypted at level L and the context
 * scale; output at level L-6 with the logits in slots [0, classes). */
tcks_status tcks_cnn_forward(const tcks_cnn* m, const tcks_ct* in, tcks_ct** out);
/* `count` inferences in one pass (the batched path): every stage of the schedule runs once for
 * the whole batch (rotations of all requests share key-switch launches). outs[i] is bit-identical
 * to tcks_cnn_forward(in[i]). */
tcks_status tcks_cnn_forward_batch(const tcks_cnn* m, const tcks_ct* const* in, uint32_t count, tcks_ct** outs);
/* The batched forward pass on device buffers: d_in [count][2][L][N] (level L, the context scale),
 * d_out [count][2][L-6][N], both contiguous, owned by the caller and not overlapping. Enqueued on the
 * context's stream; returns without waiting for it. */
tcks_status tcks_cnn_forward_device(const tcks_cnn* m, const uint64_t* d_in, uint32_t count, uint64_t* d_out);
/* The batched forward pass straight from and to host memory: host_in [count][2][L][N] input limbs
 * (NTT form, level L, the context scale; pinned memory copies fastest), host_out [count][2][L-6][N]
 * receives the outputs (their scale is the model's output scale, as tcks_cnn_forward reports). One
 * host-to-device copy, the batched schedule on one contiguous device batch, one device-to-host copy;
 * returns when host_out is written. */
tcks_status tcks_cnn_forward_host(const tcks_cnn* m, const uint64_t* host_in, uint32_t count, uint64_t* host_out);
/* Sizes of one serialized input of the network (level L; in_full: both components, in_seeded: c0 and
 * the seed of c1) and of one serialized output (level L-6), in bytes: the wire form of
 * tcks_ct_serialize / tcks_ct_serialize_seeded. */
tcks_status tcks_cnn_wire_sizes(const tcks_cnn* m, uint64_t* in_full, uint64_t* in_seeded, uint64_t* out_size);
/* The batched forward pass on serialized ciphertexts, the client-server exchange of an encrypted
 * evaluation (§5): host_in holds count inputs back to back, each in_size bytes (in_full or in_seeded of
 * tcks_cnn_wire_sizes; all of that one kind, level L, the context scale); host_out receives count
 * serialized outputs, each out_size bytes (kind 0, level L-6, the model's output scale). One
 * host-to-device copy of the bytes, the residues unpacked and c1 regenerated from its seed on the
 * device, the batched schedule, the outputs packed on the device, one device-to-host copy; returns when
 * host_out is written. Errors: INVALID_ARG for a size, header or residue (>= its prime) that does not
 * fit, SCALE_MISMATCH for an input scale; after a residue error host_out is unspecified. */
tcks_status tcks_cnn_forward_wire(const tcks_cnn* m, const uint8_t* host_in, uint64_t in_size, uint32_t count,
                                  uint8_t* host_out, uint64_t out_size);
/* The same exchange for a stream of batches, pipelined (§5's client-server evaluation served batch
 * after batch; the paper has no pipeline): a pipe holds two slots of device buffers for batches of
 * `count` serialized inputs of in_size bytes (in_full or in_seeded). submit checks the headers,
 * queues the batch and returns a ticket without waiting. The input copy runs on the pipe's own copy
 * stream as soon as the batch's slot is free; the unpacking, the network and the packing run on the
 * model's stream after it. So the input copy of one batch overlaps the network of the one before.
 * wait(ticket) returns when that batch's outputs are in its host_out (serialized as in
 * tcks_cnn_forward_wire). host_in and host_out must stay valid (and host_in unchanged) until the
 * batch completes; pinned memory lets the copies run asynchronously. A submit first completes the
 * batch two submits earlier, whose slot it takes. A batch's errors (INVALID_ARG for a residue >= its
 * prime: its host_out is then not written; TIMEOUT or CUDA_ERROR for a kernel error) are reported by
 * the call that completes it: its wait, or that later submit. wait on a ticket already completed
 * returns OK. free waits for the work in flight. */
typedef struct tcks_cnn_pipe tcks_cnn_pipe;
tcks_status tcks_cnn_pipe_create(const tcks_cnn* m, uint32_t count, uint64_t in_size, tcks_cnn_pipe** out);
tcks_status tcks_cnn_pipe_submit(tcks_cnn_pipe* p, const uint8_t* host_in, uint8_t* host_out, uint64_t* ticket);
tcks_status tcks_cnn_pipe_wait(tcks_cnn_pipe* p, uint64_t ticket);
void tcks_cnn_pipe_free(tcks_cnn_pipe* p);
/* CUDA graph of the batched forward for a fixed batch size (the schedule is captured once with its
 * stream-ordered scratch allocations, then replayed): create captures it (after one eager pass that
 * warms the key tables), run copies the inputs into the graph's staging buffers, replays and returns
 * new output ciphertexts, bit-identical to tcks_cnn_forward. With a caller allocator the scratch
 * is one block from it, sized by a second uncaptured pass and held by the graph. */
typedef struct tcks_cnn_graph tcks_cnn_graph;
tcks_status tcks_cnn_graph_create(const tcks_cnn* m, uint32_t count, tcks_cnn_graph** out);
tcks_status tcks_cnn_graph_run(tcks_cnn_graph* g, const tcks_ct* const* in, tcks_ct** outs);
void tcks_cnn_graph_free(tcks_cnn_graph* g);
/* Export one of the model's encoded plaintexts (kind 0 conv kernel, 1 channel mask, 2 bias
 * (index 0..2), 3 FC1 diagonal, 4 FC2 diagonal, 5 / 6 the FC1 / FC2 diagonal over the extended basis,
 * its limb modulo P last, 7 the baby-step diagonal kernel * B + b of TCKS_CONV_SHARED over the
 * extended basis, 8 the folded baby-step diagonal b of TCKS_CONV_FOLD over the extended basis) to
 * host [level][N] ([level+1][N] for kinds 5 to 8); level / scale are reported. */
tcks_status tcks_cnn_export_plaintext(const tcks_cnn* m, uint32_t kind, uint32_t index, uint64_t* host,
                                      size_t n_words, uint32_t* level, double* scale);

/* ------------------------------------------------------------------------------ serving ---- */
/* A serving loop for encrypted inference requests (the paper's client-server setting, §2 and §5,
 * with requests of several parameter sizes on one GPU). Lanes are models on their contexts: a CNN
 * (five stages) or a vector x plain matrix (one stage). Requests are queued on submit (the server
 * keeps a device copy of the input) and admitted in arrival order while the HBM budget (every
 * lane's resident keys, tables and model plaintexts, plus a per-request allowance of 65 top-level
 * ciphertexts for the live state and the stage scratch) and the in-flight cap allow. A step groups
 * admitted requests by (lane, stage), runs each group's stage as one batched pass of up to max_batch
 * requests (all lanes' work is launched before the step waits), and advances each request by one
 * stage; requests submitted while a step runs join stage 0 at the next step (continuous batching).
 * Results are bit-identical to the single-request path. submit fails with BUDGET_EXCEEDED for a
 * request that could never fit; take returns NOT_READY for a request still queued or running. */
typedef struct tcks_server tcks_server;
tcks_status tcks_server_create(uint64_t hbm_budget_bytes, uint32_t max_in_flight, uint32_t max_batch,
                               tcks_server** out);
void tcks_server_free(tcks_server* s);
tcks_status tcks_server_add_cnn(tcks_server* s, const tcks_cnn* m, uint32_t* lane);
tcks_status tcks_server_add_vecmat(tcks_server* s, const tcks_matrix* M, uint32_t* lane);
tcks_status tcks_server_submit(tcks_server* s, uint32_t lane, const tcks_ct* in, uint64_t* id);
/* Runs one step and waits for it; *completed = requests that finished in it. */
tcks_status tcks_server_step(tcks_server* s, uint32_t* completed);
/* Ids completed since the last poll (up to cap). */
tcks_status tcks_server_poll(tcks_server* s, uint64_t* ids, uint32_t cap, uint32_t* n);
tcks_status tcks_server_take(tcks_server* s, uint64_t id, tcks_ct** out);
tcks_status tcks_server_stats(const tcks_server* s, uint64_t* queued, uint64_t* in_flight, uint64_t* finished,
                              uint64_t* bytes_in_use, uint64_t* bytes_resident);

#ifdef __cplusplus
}
#endif
#endif /* TCKS_H */

// Core RNS kernels: batched NTT / INTT, element-wise ops, the tensor product, rescale and the
// key-switching pipeline (ModUp, inner product with the key, ModDown), with the Galois
// automorphism folded into the inner product's reads.
//
// Every kernel that transforms a limb stages it in shared memory (one CTA per limb, N <= 2^14),
// so a limb crosses HBM once per kernel; the prologue that fills shared memory and the epilogue
// that drains it carry the surrounding element-wise work (lifts, products, combines).
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>

#include "context.h"
#include "kernels.h"
#include "ntt.cuh"

namespace tcks {

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per kernel and size (the
// attribute is per function, so the registry is keyed by the kernel's address).
void ensure_smem(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  static std::mutex mu;
  static std::map<const void*, size_t> granted;
  std::lock_guard<std::mutex> lock(mu);
  size_t& g = granted[kernel];
  if (bytes > g) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    g = bytes;
  }
}

// --------------------------------------------------------------------------- batched NTT ----
// Job b (blockIdx.x): src + b*src_stride -> dst + b*dst_stride, prime = mod_base + b % mod_period.
template <bool INVERSE>
__global__ void k_ntt(DevTables T, const u64* __restrict__ src, u64 src_stride, u64* __restrict__ dst,
                      u64 dst_stride, u32 mod_base, u32 mod_period) {
  extern __shared__ u64 s[];
  const u32 n = 1u << T.log_n;
  const u32 b = blockIdx.x;
  const u32 mod = mod_base + b % mod_period;
  const ModConst m = T.mods[mod];
  const u64* in = src + (u64)b * src_stride;
  u64* out = dst + (u64)b * dst_stride;
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) s[k] = in[k];
  __syncthreads();
  if (INVERSE) {
    ntt_inv_smem(s, T, mod);
    for (u32 k = threadIdx.x; k < n; k += blockDim.x) out[k] = inv_final(s[k], m);
  } else {
    ntt_fwd_smem(s, T, mod);
    for (u32 k = threadIdx.x; k < n; k += blockDim.x) out[k] = fwd_final(s[k], m.q);
  }
}

u32 ntt_threads(u32 log_n) {
  const u32 n = 1u << log_n;
  u32 t = n / 8;
  if (t < 32) t = 32;
  if (t > 1024) t = 1024;
  return t;
}

static size_t smem_bytes(u32 log_n) { return ((size_t)8) << log_n; }

template <typename K>
static void allow_smem(K kernel, size_t bytes) {
  ensure_smem((const void*)kernel, bytes);
}

void launch_ntt(const DevTables& T, bool inverse, const u64* src, u64 src_stride, u64* dst, u64 dst_stride,
                u32 count, u32 mod_base, u32 mod_period, cudaStream_t st) {
  if (!count) return;
  const size_t sm = smem_bytes(T.log_n);
  Launch L(inverse ? K_NTT_INV : K_NTT_FWD, st, 16.0 * count * (1u << T.log_n));
  if (inverse) {
    allow_smem(k_ntt<true>, sm);
    k_ntt<true><<<count, ntt_threads(T.log_n), sm, st>>>(T, src, src_stride, dst, dst_stride, mod_base, mod_period);
  } else {
    allow_smem(k_ntt<false>, sm);
    k_ntt<false><<<count, ntt_threads(T.log_n), sm, st>>>(T, src, src_stride, dst, dst_stride, mod_base, mod_period);
  }
}

// ------------------------------------------------------------------------ element-wise ops ----
// Operands laid out [polys][ell][N]; element e belongs to limb (e >> log_n) % ell.
enum : u32 { EW_ADD = OP_ADD, EW_SUB = OP_SUB, EW_NEG = OP_NEG, EW_MUL_PLAIN = OP_MUL_PLAIN, EW_ADD_PLAIN = OP_ADD_PLAIN,
             EW_SUB_PLAIN = OP_SUB_PLAIN };

__global__ void k_elementwise(DevTables T, u32 op, const u64* __restrict__ a, const u64* __restrict__ b,
                              u64* __restrict__ out, u32 ell, u32 polys) {
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u64 total2 = ((u64)polys * ell * n) >> 1;
  for (u64 e2 = (u64)blockIdx.x * blockDim.x + threadIdx.x; e2 < total2; e2 += (u64)gridDim.x * blockDim.x) {
    const u64 e = e2 << 1;
    const u64 row = e >> log_n;  // poly * ell + limb
    const u32 limb = (u32)(row % ell);
    const u32 poly = (u32)(row / ell);
    const ModConst m = T.mods[limb];
    const ulonglong2 x = reinterpret_cast<const ulonglong2*>(a)[e2];
    ulonglong2 r;
    switch (op) {
      case EW_ADD: {
        const ulonglong2 y = reinterpret_cast<const ulonglong2*>(b)[e2];
        r.x = add_mod(x.x, y.x, m.q);
        r.y = add_mod(x.y, y.y, m.q);
        break;
      }
      case EW_SUB: {
        const ulonglong2 y = reinterpret_cast<const ulonglong2*>(b)[e2];
        r.x = sub_mod(x.x, y.x, m.q);
        r.y = sub_mod(x.y, y.y, m.q);
        break;
      }
      case EW_NEG:
        r.x = neg_mod(x.x, m.q);
        r.y = neg_mod(x.y, m.q);
        break;
      case EW_MUL_PLAIN: {  // b is a plaintext [ell][N]
        const ulonglong2 y = reinterpret_cast<const ulonglong2*>(b + (u64)limb * n)[(e & (n - 1)) >> 1];
        r.x = mul_mod(x.x, y.x, m);
        r.y = mul_mod(x.y, y.y, m);
        break;
      }
      default: {  // EW_ADD_PLAIN / EW_SUB_PLAIN: only component 0 changes
        if (poly == 0) {
          const ulonglong2 y = reinterpret_cast<const ulonglong2*>(b + (u64)limb * n)[(e & (n - 1)) >> 1];
          if (op == EW_ADD_PLAIN) {
            r.x = add_mod(x.x, y.x, m.q);
            r.y = add_mod(x.y, y.y, m.q);
          } else {
            r.x = sub_mod(x.x, y.x, m.q);
            r.y = sub_mod(x.y, y.y, m.q);
          }
        } else {
          r = x;
        }
      }
    }
    reinterpret_cast<ulonglong2*>(out)[e2] = r;
  }
}

static u32 ew_blocks(u64 elems2) {
  u64 b = (elems2 + 255) / 256;
  const u64 cap = 152ull * 16;
  return (u32)(b < cap ? (b ? b : 1) : cap);
}

void launch_elementwise(const DevTables& T, u32 op, const u64* a, const u64* b, u64* out, u32 ell, u32 polys,
                        cudaStream_t st) {
  const u64 e2 = ((u64)polys * ell << T.log_n) >> 1;
  const double limb = 8.0 * ell * (1u << T.log_n);  // bytes of one [ell][N] polynomial
  const double by = op == OP_NEG ? 2.0 * polys * limb
                    : (op == OP_ADD || op == OP_SUB) ? 3.0 * polys * limb
                                                     : (2.0 * polys + 1.0) * limb;  // plaintext operand
  Launch L(K_ELEMENTWISE, st, by);
  k_elementwise<<<ew_blocks(e2), 256, 0, st>>>(T, op, a, b, out, ell, polys);
}

// Tensor product: (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1), out [3][ell][N].
__global__ void k_tensor(DevTables T, const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out,
                         u32 ell) {
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u64 per_poly = (u64)ell * n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < per_poly; e += (u64)gridDim.x * blockDim.x) {
    const ModConst m = T.mods[e >> log_n];
    const u64 a0 = a[e], a1 = a[per_poly + e], b0 = b[e], b1 = b[per_poly + e];
    out[e] = mul_mod(a0, b0, m);
    Acc128 acc{0, 0};
    mac128(acc, a0, b1);
    mac128(acc, a1, b0);
    out[per_poly + e] = reduce128(acc.hi, acc.lo, m);
    out[2 * per_poly + e] = mul_mod(a1, b1, m);
  }
}

void launch_tensor(const DevTables& T, const u64* a, const u64* b, u64* out, u32 ell, cudaStream_t st) {
  const u64 e = (u64)ell << T.log_n;
  Launch L(K_TENSOR, st, 7.0 * 8.0 * e);
  k_tensor<<<ew_blocks(e / 2 + 1), 256, 0, st>>>(T, a, b, out, ell);
}

// Decryption kernel: m = c0 + c1 * s over limbs < ell (s has L+1 limbs, chain order).
__global__ void k_decrypt(DevTables T, const u64* __restrict__ ct, const u64* __restrict__ s, u64* __restrict__ pt,
                          u32 ell) {
  const u32 log_n = T.log_n;
  const u64 per_poly = (u64)ell << log_n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < per_poly; e += (u64)gridDim.x * blockDim.x) {
    const ModConst m = T.mods[e >> log_n];
    pt[e] = add_mod(ct[e], mul_mod(ct[per_poly + e], s[e], m), m.q);
  }
}

void launch_decrypt(const DevTables& T, const u64* ct, const u64* s, u64* pt, u32 ell, cudaStream_t st) {
  const u64 e = (u64)ell << T.log_n;
  Launch L(K_DECRYPT, st, 4.0 * 8.0 * e);
  k_decrypt<<<ew_blocks(e / 2 + 1), 256, 0, st>>>(T, ct, s, pt, ell);
}

// ---------------------------------------------------------------- drop the last prime ----
// Rescale (drop = q_{ell-1}) and ModDown (drop = P) share this combine:
//   out[p][i] = (in[p][i] - NTT_i(bal(top[p]) mod q_i)) * drop^-1 mod q_i,  i < n_out,
// with top[p] the coefficient-domain limb of the dropped prime. One CTA per (p, i).
__global__ void k_drop_combine(DevTables T, const u64* __restrict__ in, u64 in_poly_stride,
                               const u64* __restrict__ top, u32 drop_mod, u32 n_out, u64* __restrict__ out) {
  extern __shared__ u64 s[];
  const u32 n = 1u << T.log_n;
  const u32 p = blockIdx.x / n_out, i = blockIdx.x % n_out;
  const ModConst mi = T.mods[i];
  const ModConst md = T.mods[drop_mod];
  const PairConst pc = T.pairs[(u64)drop_mod * T.n_mods + i];
  const u64* tp = top + (u64)p * n;
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) s[k] = lift_balanced(tp[k], md.half, pc.qa_mod_b, mi);
  __syncthreads();
  ntt_fwd_smem(s, T, i);
  const u64* src = in + (u64)p * in_poly_stride + (u64)i * n;
  u64* dst = out + ((u64)p * n_out + i) * n;
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) {
    const u64 c = sub_mod(src[k], fwd_final(s[k], mi.q), mi.q);
    dst[k] = mul_shoup(c, pc.inv_qa, pc.inv_qa_sh, mi.q);
  }
}

void launch_rescale(const DevTables& T, const u64* ct, u32 ell, u64* top_tmp, u64* out, cudaStream_t st) {
  const u64 n = 1ull << T.log_n;
  // INTT of the last limb of each component
  launch_ntt(T, true, ct + (u64)(ell - 1) * n, (u64)ell * n, top_tmp, n, 2, ell - 1, 1, st);
  const size_t sm = smem_bytes(T.log_n);
  allow_smem(k_drop_combine, sm);
  Launch L(K_DROP, st, 8.0 * (1u << T.log_n) * (4.0 * (ell - 1) + 2.0));
  k_drop_combine<<<2 * (ell - 1), ntt_threads(T.log_n), sm, st>>>(T, ct, (u64)ell * n, top_tmp, ell - 1, ell - 1,
                                                                   out);
}

// ------------------------------------------------------------------------ key switching ----
// ModUp (one digit per prime): digit j = bal_{q_j}(x_j) lifted to slot i (prime q_i for i < ell,
// P for i = ell) and NTT'd; digits [ell][ell+1][N]. Slot i == j is x_j itself.
__global__ void k_modup(DevTables T, const u64* __restrict__ x_ntt, const u64* __restrict__ x_coef, u32 ell,
                        u64* __restrict__ digits) {
  extern __shared__ u64 s[];
  const u32 n = 1u << T.log_n;
  const u32 j = blockIdx.x / (ell + 1), slot = blockIdx.x % (ell + 1);
  u64* out = digits + ((u64)j * (ell + 1) + slot) * n;
  if (slot == j) {
    const u64* in = x_ntt + (u64)j * n;
    for (u32 k = threadIdx.x; k < n; k += blockDim.x) out[k] = in[k];
    return;
  }
  const u32 tmod = slot < ell ? slot : T.L;
  const ModConst mt = T.mods[tmod];
  const u64 half_j = T.mods[j].half;
  const u64 qj_mod_t = T.pairs[(u64)j * T.n_mods + tmod].qa_mod_b;
  const u64* in = x_coef + (u64)j * n;
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) s[k] = lift_balanced(in[k], half_j, qj_mod_t, mt);
  __syncthreads();
  ntt_fwd_smem(s, T, tmod);
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) out[k] = fwd_final(s[k], mt.q);
}

void launch_modup(const DevTables& T, const u64* x_ntt, u32 ell, u64* x_coef_tmp, u64* digits, cudaStream_t st) {
  const u64 n = 1ull << T.log_n;
  launch_ntt(T, true, x_ntt, n, x_coef_tmp, n, ell, 0, ell, st);
  const size_t sm = smem_bytes(T.log_n);
  allow_smem(k_modup, sm);
  Launch L(K_MODUP, st, 8.0 * (1u << T.log_n) * (2.0 * ell + (double)ell * (ell + 1)));
  k_modup<<<ell * (ell + 1), ntt_threads(T.log_n), sm, st>>>(T, x_ntt, x_coef_tmp, ell, digits);
}

// Inner product of (automorphed) digits with one key component on slot `slot`:
//   sum_j D_j[slot][src(k)] * key_j[b][key_slot][k], 128-bit lazy accumulation, one reduction.
__device__ __forceinline__ u64 ks_inner(const u64* __restrict__ digits, u32 ell, u32 slot, const u64* __restrict__ key,
                                        u32 K, u32 key_slot, u32 b, u32 k, u32 src, u32 n, const ModConst& m) {
  Acc128 acc{0, 0};
  for (u32 j = 0; j < ell; ++j) {
    const u64 d = digits[((u64)j * (ell + 1) + slot) * n + src];
    const u64 w = key[(((u64)j * 2 + b) * (K + 1) + key_slot) * n + k];
    mac128(acc, d, w);
  }
  return reduce128(acc.hi, acc.lo, m);
}


// Stage 1: u_b[P] = sum_j tau_g(D_j)[P] * key_j[b][P], then INTT mod P -> top[b]. grid (2, jobs).
__global__ void k_ks_inner_p(DevTables T, u32 ell, const __grid_constant__ KsBatch jobs) {
  extern __shared__ u64 s[];
  const u32 log_n = T.log_n, n = 1u << log_n;
  const KsJob& J = jobs.job[blockIdx.y];
  const u64* __restrict__ digits = J.digits;
  const u32 b = blockIdx.x;
  const ModConst mp = T.mods[T.L];
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) {
    const u32 src = J.g == 1 ? k : galois_src(k, J.g, log_n);
    s[k] = ks_inner(digits, ell, ell, J.key, J.K, J.K, b, k, src, n, mp);
  }
  __syncthreads();
  ntt_inv_smem(s, T, T.L);
  u64* top = J.top + (u64)b * n;
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) top[k] = inv_final(s[k], mp);
}

// Stage 2 (ModDown): out_b[i] = (u_b[i] - NTT_i(bal_P(top_b) mod q_i)) * P^-1 + addend_b[i].
// grid (2 * ell, jobs).
__global__ void k_ks_moddown(DevTables T, u32 ell, const __grid_constant__ KsBatch jobs) {
  extern __shared__ u64 s[];
  const u32 log_n = T.log_n, n = 1u << log_n;
  const KsJob& J = jobs.job[blockIdx.y];
  const u64* __restrict__ digits = J.digits;
  const u32 b = blockIdx.x / ell, i = blockIdx.x % ell;
  const ModConst mi = T.mods[i];
  const ModConst mp = T.mods[T.L];
  const PairConst pc = T.pairs[(u64)T.L * T.n_mods + i];
  const u64* top = J.top + (u64)b * n;
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) s[k] = lift_balanced(top[k], mp.half, pc.qa_mod_b, mi);
  __syncthreads();
  ntt_fwd_smem(s, T, i);
  const u64* add = b == 0 ? J.add0 : J.add1;
  u64* dst = J.out + ((u64)b * ell + i) * n;
  for (u32 k = threadIdx.x; k < n; k += blockDim.x) {
    const u32 src = J.g == 1 ? k : galois_src(k, J.g, log_n);
    const u64 u = ks_inner(digits, ell, i, J.key, J.K, i, b, k, src, n, mi);
    u64 v = mul_shoup(sub_mod(u, fwd_final(s[k], mi.q), mi.q), pc.inv_qa, pc.inv_qa_sh, mi.q);
    if (add) v = add_mod(v, add[(u64)i * n + (J.add_perm ? src : k)], mi.q);
    dst[k] = v;
  }
}

void launch_keyswitch(const DevTables& T, u32 ell, const KsBatch& jobs, cudaStream_t st) {
  if (!jobs.count) return;
  const size_t sm = smem_bytes(T.log_n);
  allow_smem(k_ks_inner_p, sm);
  allow_smem(k_ks_moddown, sm);
  // algorithmic bytes: distinct digit sets and keys once, scratch and outputs once
  const double n = (double)(1u << T.log_n);
  double digits = 0, keys_p = 0, keys_q = 0, adds = 0;
  for (u32 j = 0; j < jobs.count; ++j) {
    bool new_digits = true, new_key = true, new_add = true;
    for (u32 i = 0; i < j; ++i) {
      new_digits &= jobs.job[i].digits != jobs.job[j].digits;
      new_key &= jobs.job[i].key != jobs.job[j].key;
      new_add &= jobs.job[i].add0 != jobs.job[j].add0;
    }
    if (new_digits) digits += 1;
    if (new_key) keys_p += 2.0 * ell, keys_q += 2.0 * ell * ell;
    if (new_add && jobs.job[j].add0) adds += jobs.job[j].add1 ? 2.0 * ell : ell;
  }
  {
    Launch L(K_KS_P, st, 8.0 * n * (digits * ell + keys_p + 2.0 * jobs.count));
    k_ks_inner_p<<<dim3(2, jobs.count), ntt_threads(T.log_n), sm, st>>>(T, ell, jobs);
  }
  {
    Launch L(K_KS_MODDOWN, st,
             8.0 * n * (digits * ell * ell + keys_q + 2.0 * jobs.count + adds + 2.0 * ell * jobs.count));
    k_ks_moddown<<<dim3(2 * ell, jobs.count), ntt_threads(T.log_n), sm, st>>>(T, ell, jobs);
  }
}

// acc += sum_c rots[c] * diag[c]: one pass over acc, lazy 128-bit accumulation (count <= 64 keeps
// the sum below 2^128 for q < 2^61), one reduction per element.
__global__ void k_mulacc(DevTables T, u64* __restrict__ acc, const u64* __restrict__ rots, u64 rot_stride,
                         const u64* __restrict__ diag, u64 diag_stride, u32 count, u32 ell) {
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u64 per_poly = (u64)ell * n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < 2 * per_poly; e += (u64)gridDim.x * blockDim.x) {
    const u64 pe = e < per_poly ? e : e - per_poly;  // offset inside the component
    const ModConst m = T.mods[pe >> log_n];
    Acc128 a{acc[e], 0};
    for (u32 c = 0; c < count; ++c) mac128(a, rots[c * rot_stride + e], diag[c * diag_stride + pe]);
    acc[e] = reduce128(a.hi, a.lo, m);
  }
}

void launch_mulacc(const DevTables& T, u64* acc, const u64* rots, u64 rot_stride, const u64* diag, u64 diag_stride,
                   u32 count, u32 ell, cudaStream_t st) {
  if (!count) return;
  const u64 e = (u64)2 * ell << T.log_n;
  Launch L(K_MULACC, st, 8.0 * ((double)e * (2.0 + count) + (double)count * ell * (1u << T.log_n)));
  k_mulacc<<<ew_blocks(e / 2 + 1), 256, 0, st>>>(T, acc, rots, rot_stride, diag, diag_stride, count, ell);
}

}  // namespace tcks

// ------------------------------------------------------------- allocation-free rescale ----
// A variant of the rescale for callers that cannot allocate device memory. Its only scratch (the
// coefficient-domain top limb of both components, [2][N] words) lives in the static array below,
// which every GPU that loads the library holds until the process exits.
namespace tcks {
tcks_status abi_record(tcks_status code, const std::string& msg);
void abi_clear();
void count_launch();

namespace {
constexpr u32 kNoAllocMaxLogN = 14;                           // N <= 16384
constexpr size_t kNoAllocWords = (size_t)2 << kNoAllocMaxLogN;  // 256 KB
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) u64 g_rescale_scratch[kNoAllocWords];
u64* g_scratch_ptr[kNoAllocMaxDevices];  // device address of g_rescale_scratch per device, set up once
bool g_scratch_ready[kNoAllocMaxDevices];
std::mutex g_scratch_mu;

// Once per device, with that device current: resolve the scratch array's device address and raise
// the shared-memory limit of the two kernels the rescale launches. Returns nullptr on failure.
u64* noalloc_setup(int device, std::string* why) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ready[device]) return g_scratch_ptr[device];
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    *why = "cudaGetDevice failed";
    return nullptr;
  }
  if (prev != device && cudaSetDevice(device) != cudaSuccess) {
    *why = "cudaSetDevice failed";
    return nullptr;
  }
  u64* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_rescale_scratch);
  const int bytes = (int)(((size_t)8) << kNoAllocMaxLogN);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ntt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_drop_combine, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    *why = std::string("scratch set-up failed: ") + cudaGetErrorString(e);
    return nullptr;
  }
  g_scratch_ptr[device] = ptr;
  g_scratch_ready[device] = true;
  return ptr;
}
}  // namespace
}  // namespace tcks

extern "C" tcks_status tcks_rescale_noalloc(tcks_ctx* ctx, const uint64_t* d_in, uint32_t level, uint64_t* d_out) {
  using namespace tcks;
  if (!ctx || !d_in || !d_out) return abi_record(TCKS_ERR_INVALID_ARG, "rescale_noalloc: null argument");
  if (level < 2) return abi_record(TCKS_ERR_LEVEL_EXHAUSTED, "rescale_noalloc: needs level >= 2");
  if (level > ctx->L) return abi_record(TCKS_ERR_INVALID_ARG, "rescale_noalloc: level exceeds the chain");
  const u32 log_n = ctx->params.log_n;
  if (log_n > kNoAllocMaxLogN)
    return abi_record(TCKS_ERR_INVALID_ARG,
                      "rescale_noalloc: N = 2^" + std::to_string(log_n) +
                          " exceeds the static scratch, which holds two limbs of at most N = 2^14");
  if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
    return abi_record(TCKS_ERR_INVALID_ARG, "rescale_noalloc: device index out of range");
  std::string why;
  u64* scratch = noalloc_setup(ctx->device, &why);
  if (!scratch) return abi_record(TCKS_ERR_CUDA, "rescale_noalloc: " + why);
  const DevTables& T = ctx->T;
  const u64 n = 1ull << log_n;
  const size_t sm = ((size_t)8) << log_n;
  // the two launches of launch_rescale, without its allocating bookkeeping
  count_launch();
  k_ntt<true><<<2, ntt_threads(log_n), sm, ctx->stream>>>(T, d_in + (u64)(level - 1) * n, (u64)level * n, scratch, n,
                                                           level - 1, 1);
  count_launch();
  k_drop_combine<<<2 * (level - 1), ntt_threads(log_n), sm, ctx->stream>>>(T, d_in, (u64)level * n, scratch,
                                                                             level - 1, level - 1, d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return abi_record(TCKS_ERR_CUDA, std::string("rescale_noalloc: ") + cudaGetErrorString(e));
  abi_clear();
  return TCKS_OK;
}

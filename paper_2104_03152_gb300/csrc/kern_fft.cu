// CKKS encoding and decoding (the canonical embedding, slot j <-> zeta^(5^j), zeta = exp(i pi/N)),
// the only FP64 step of the library.
//
// With n = N/2 and w_k = m_k + i m_{k+n}, the embedding is
//   z_j = m(zeta^(5^j)) = sum_k (w_k zeta^k) omega^(t_j k),  omega = zeta^4, t_j = (5^j mod 2N - 1)/4,
// because zeta^(5^j) = zeta * omega^(t_j) and zeta^(N/2) = i. Encoding inverts it:
//   w_k = zeta^-k * (1/n) sum_t y_t omega^(-t k),  y_(t_j) = z_j,
// one complex FFT of size n in shared memory (radix-2, decimation in time). Decoding composes each
// coefficient exactly from its residues (Garner mixed radix in multiword integers), rounds it once to
// double, then runs the forward FFT.
#include <cuda_runtime.h>

#include "kernels.h"
#include "limb_launch.cuh"
#include "ntt.cuh"

namespace tcks {

namespace {

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csubc(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }

// zeta^e for any integer e (taken mod 2N).
__device__ __forceinline__ cplx zeta_pow(const double* zeta, long long e, u32 log_n) {
  const unsigned long long r = (unsigned long long)e & ((2ull << log_n) - 1ull);  // 2N is a power of two
  return {zeta[2 * r], zeta[2 * r + 1]};
}

// In-place size-n FFT of y in shared memory; sign -1: sum y_t omega^(-tk), +1: omega^(+tk).
__device__ void fft_smem(cplx* y, u32 log_half, int sign, const double* zeta, u32 log_n) {
  const u32 n = 1u << log_half;
  // bit-reversal permutation
  for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
    const u32 r = __brev(i) >> (32 - log_half);
    if (r > i) {
      const cplx t = y[i];
      y[i] = y[r];
      y[r] = t;
    }
  }
  __syncthreads();
  for (u32 s = 1; s <= log_half; ++s) {
    const u32 half = 1u << (s - 1);
    // twiddle omega^(pos * n / len) = zeta^(4 * pos * 2^(log_half - s))
    for (u32 b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const u32 blk = b >> (s - 1), pos = b & (half - 1);
      const u32 i0 = (blk << s) + pos, i1 = i0 + half;
      const long long e = (long long)4 * pos * (1ll << (log_half - s));
      const cplx w = zeta_pow(zeta, sign > 0 ? e : -e, log_n);
      const cplx u = y[i0], v = cmul(y[i1], w);
      y[i0] = cadd(u, v);
      y[i1] = csubc(u, v);
    }
    __syncthreads();
  }
}

}  // namespace

// One CTA: z (n_in <= N/2 doubles, device) -> coefficients round(scale * m_i) as int64 [N].
__global__ void k_encode_coeffs(DevTables T, FftTables F, const double* __restrict__ z, u32 n_in, double scale,
                                i64* __restrict__ coeffs, int* __restrict__ status) {
  extern __shared__ cplx y[];
  const u32 log_n = T.log_n, log_half = log_n - 1;
  const u32 half = 1u << log_half;
  for (u32 t = threadIdx.x; t < half; t += blockDim.x) y[t] = {0.0, 0.0};
  __syncthreads();
  for (u32 j = threadIdx.x; j < n_in; j += blockDim.x) y[F.slot_index[j]] = {z[j], 0.0};
  __syncthreads();
  fft_smem(y, log_half, -1, F.zeta, log_n);
  const double inv_half = 1.0 / (double)half;
  int overflow = 0;
  for (u32 k = threadIdx.x; k < half; k += blockDim.x) {
    const cplx w = cmul({y[k].re * inv_half, y[k].im * inv_half}, zeta_pow(F.zeta, -(long long)k, log_n));
    const double x0 = scale * w.re, x1 = scale * w.im;
    const double lim = 4611686018427387904.0;  // 2^62
    if (!(fabs(x0) < lim) || !(fabs(x1) < lim)) {
      overflow = 1;
      coeffs[k] = 0;
      coeffs[k + half] = 0;
    } else {
      coeffs[k] = llround(x0);  // round half away from zero
      coeffs[k + half] = llround(x1);
    }
  }
  if (overflow) atomicExch(status, 1);
}

// int64 coefficients -> NTT-form limbs, one limb job per prime: limb j modulo q_j, and limb p_slot
// (when the launch includes it) modulo the special prime P.
template <typename W, int LC>
__global__ void k_coeffs_to_ntt(DevTables T, const i64* __restrict__ coeffs, u32 p_slot, u64* __restrict__ pt) {
  TCKS_SMEM(W);
  const Slice P = slice_of<LC>(T);
  const u32 rank = P.rank, j = P.job, ns = P.ns, off = P.off;
  const u32 l = j == p_slot ? T.L : j;
  const ModConst m = T.mods[l];
  for (u32 k = threadIdx.x; k < ns; k += blockDim.x) {
    const i64 v = coeffs[off + k];
    const u64 a = v >= 0 ? (u64)v : (u64)(-(v + 1)) + 1;  // |v|
    const u64 r = reduce64(a, m);
    s[sw(k)] = (W)(v >= 0 ? r : neg_mod(r, m.q));
  }
  __syncthreads();
  ntt_fwd_slice<W, LC>(s, T, l, rank);
  u64* out = pt + ((u64)j << T.log_n) + off;
  for (u32 k = threadIdx.x; k < ns; k += blockDim.x) out[k] = Ar<W>::fwd_out(s[sw(k)], m);
}

// Exact CRT of one coefficient: Garner digits v_i (x = v_0 + v_1 q_0 + v_2 q_0 q_1 + ...), the
// multiword integer, its centred value, and the double nearest to it (sticky-bit rounding).
__global__ void k_crt_compose(DevTables T, const u64* __restrict__ coef, u32 ell, const u64* __restrict__ qwords,
                              double* __restrict__ out) {
  const u32 log_n = T.log_n, n = 1u << log_n;
  const u32 k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  u64 v[CRT_MAXW];
  for (u32 i = 0; i < ell; ++i) {
    const ModConst mi = T.mods[i];
    u64 t = coef[(u64)i * n + k];
    for (u32 j = 0; j < i; ++j) {
      const PairConst pc = T.pairs[(u64)j * T.n_mods + i];
      t = mul_shoup(sub_mod(t, reduce64(v[j], mi), mi.q), pc.inv_qa, pc.inv_qa_sh, mi.q);
    }
    v[i] = t;
  }
  // Horner from the top digit: X = (...(v_{l-1} q_{l-2} + v_{l-2}) q_{l-3} + ...) + v_0
  u64 X[CRT_MAXW];
  u32 words = 1;
  X[0] = v[ell - 1];
  for (int i = (int)ell - 2; i >= 0; --i) {
    const u64 q = T.mods[i].q;
    u64 carry = v[i];
    for (u32 w = 0; w < words; ++w) {
      const u64 lo = X[w] * q, hi = __umul64hi(X[w], q);
      const u64 s = lo + carry;
      carry = hi + (s < lo);
      X[w] = s;
    }
    if (carry) X[words++] = carry;
  }
  for (u32 w = words; w < ell + 1; ++w) X[w] = 0;
  // centre: compare with (Q - 1)/2
  const u64* Q = qwords + (u64)(ell - 1) * CRT_MAXW;
  const u64* H = qwords + ((u64)T.L + ell - 1) * CRT_MAXW;
  bool greater = false;
  for (int w = (int)ell; w >= 0; --w) {
    if (X[w] != H[w]) {
      greater = X[w] > H[w];
      break;
    }
  }
  double sign = 1.0;
  if (greater) {  // X <- Q - X
    u64 borrow = 0;
    for (u32 w = 0; w <= ell; ++w) {
      const u64 a = Q[w], b = X[w];
      const u64 d = a - b - borrow;
      borrow = (a < b) || (a - b < borrow);
      X[w] = d;
    }
    sign = -1.0;
  }
  int top = (int)ell;
  while (top > 0 && X[top] == 0) --top;
  double val;
  if (top == 0) {
    val = (double)X[0];
  } else {
    const int lz = __clzll(X[top]);
    // leading 64 bits starting at the top set bit, plus a sticky bit for everything below
    const u64 lead = lz ? (X[top] << lz) | (X[top - 1] >> (64 - lz)) : X[top];
    bool sticky = lz ? (X[top - 1] << lz) != 0 : X[top - 1] != 0;
    for (int w = top - 2; w >= 0 && !sticky; --w) sticky = X[w] != 0;
    val = ldexp(__ull2double_rn(lead | (sticky ? 1ull : 0ull)), 64 * top - lz);
  }
  out[k] = sign * val;
}

// One CTA: p (centred coefficients as doubles, [N]) -> slot values z_j, j < n_out.
__global__ void k_decode_slots(DevTables T, FftTables F, const double* __restrict__ p, double scale, u32 n_out,
                               double* __restrict__ z) {
  extern __shared__ cplx y[];
  const u32 log_n = T.log_n, log_half = log_n - 1;
  const u32 half = 1u << log_half;
  for (u32 k = threadIdx.x; k < half; k += blockDim.x)
    y[k] = cmul({p[k] / scale, p[k + half] / scale}, zeta_pow(F.zeta, (long long)k, log_n));
  __syncthreads();
  fft_smem(y, log_half, +1, F.zeta, log_n);
  for (u32 j = threadIdx.x; j < n_out; j += blockDim.x) z[j] = y[F.slot_index[j]].re;
}

static void allow(const void* k, size_t bytes) { ensure_smem(k, bytes); }

void launch_encode_coeffs(const DevTables& T, const FftTables& F, const double* d_z, u32 n_in, double scale,
                          i64* d_coeffs, int* d_status, cudaStream_t st) {
  const size_t sm = (size_t)16 << (T.log_n - 1);
  allow((const void*)k_encode_coeffs, sm);
  Launch L(K_ENCODE, st, 8.0 * n_in + 8.0 * (1u << T.log_n));
  k_encode_coeffs<<<1, 1024, sm, st>>>(T, F, d_z, n_in, scale, d_coeffs, d_status);
}

static decltype(&k_coeffs_to_ntt<u64, 0>) const K6_k_coeffs_to_ntt[6] = TCKS_K6(k_coeffs_to_ntt);

// Largest CTA size the limb kernel of this file accepts for the word type and cluster split.
u32 limb_threads_cap_fft(bool narrow, u32 log_c) {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, (const void*)K6_k_coeffs_to_ntt[(narrow ? 3 : 0) + log_c]) != cudaSuccess) return 0;
  return (u32)a.maxThreadsPerBlock;
}

void launch_coeffs_to_ntt(const DevTables& T, const i64* d_coeffs, u32 ell, u64* pt, cudaStream_t st, bool ext) {
  const u32 limbs = ell + (ext ? 1 : 0);
  Launch L(K_ENCODE, st, 8.0 * (1.0 + limbs) * (1u << T.log_n));
  launch_limb(K6_k_coeffs_to_ntt, T.narrow, limbs, 1, T.log_n, st, T.limb_threads, T, d_coeffs,
              ext ? ell : 0xffffffffu, pt);
}

void launch_crt_compose(const DevTables& T, const u64* coef, u32 ell, const u64* d_qwords, double* out,
                        cudaStream_t st) {
  const u32 n = 1u << T.log_n;
  Launch L(K_DECODE, st, 8.0 * (ell + 1.0) * (1u << T.log_n));
  k_crt_compose<<<(n + 127) / 128, 128, 0, st>>>(T, coef, ell, d_qwords, out);
}

void launch_decode_slots(const DevTables& T, const FftTables& F, const double* p, double scale, u32 n_out,
                         double* out, cudaStream_t st) {
  const size_t sm = (size_t)16 << (T.log_n - 1);
  allow((const void*)k_decode_slots, sm);
  Launch L(K_DECODE, st, 8.0 * (1u << T.log_n) + 8.0 * n_out);
  k_decode_slots<<<1, 1024, sm, st>>>(T, F, p, scale, n_out, out);
}

}  // namespace tcks

// Integer-pipe calibration: the rate of the library's own NTT butterfly (Cooley-Tukey, Shoup
// twiddle product) when nothing but registers is involved. It is the ALU ceiling the transforms,
// key switching and the fused vector x matrix kernel are measured against: their algorithmic work is
// counted in the same unit (one modular butterfly or one modular multiply-accumulate each).
#include <cuda_runtime.h>

#include "../../include/tcks.h"
#include "kernels.h"
#include "ntt.cuh"

namespace tcks {

namespace {

constexpr int kChains = 8;  // independent butterflies per thread (instruction-level parallelism)

template <typename W>
__global__ void k_butterfly_peak(u64 q, u64 w, u64 wsh, u32 iters, u64* __restrict__ sink) {
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  W x[kChains], y[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    x[j] = (W)((tid * 7 + j) % q);
    y[j] = (W)((tid * 13 + j + 1) % q);
  }
  for (u32 it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) Ar<W>::ct(x[j], y[j], (W)w, (W)wsh, (W)q);
  }
  u64 h = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) h ^= (u64)x[j] * 3 + (u64)y[j];
  sink[tid] = h;
}

// Modular multiply-accumulate in the form of the key-switch sums (KsSum with the level known): eight
// products of residues summed lazily (32-bit words: plain 64-bit sums of four, folded into a
// carry-counted sum; 64-bit words: a 128-bit sum), one reduction per eight, the result fed back into
// every operand (one logic op each) so that nothing is loop-invariant. One op = one product-accumulate.
template <typename W>
__global__ void k_mac_peak(ModConst m, u32 iters, u64* __restrict__ sink) {
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 mask = sizeof(W) == 4 ? 0x7FFFFFFFull : ((1ull << 61) - 1);
  u64 x[kChains], y[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    x[j] = (tid * 7 + j) & mask;
    y[j] = (tid * 13 + j + 1) & mask;
  }
  u64 h = 0;
  for (u32 it = 0; it < iters; ++it) {
    KsSum<W, kChains> s;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s.mac(x[j], y[j], (u32)j);
    const u64 v = s.get(m);
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (x[j] ^ v) & mask;
    h ^= v;
  }
  sink[tid] = h;
}

}  // namespace

}  // namespace tcks

using namespace tcks;

extern "C" tcks_status tcks_calibrate_macs(uint32_t word_bits, double* per_second) {
  if (!per_second || (word_bits != 32 && word_bits != 64)) return TCKS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TCKS_ERR_CUDA;
  const u32 threads = 256, blocks = (u32)sms * 8, iters = 4096;
  const u64 total = (u64)threads * blocks;
  const u64 q = word_bits == 64 ? 576460752308273153ull : 1073479681ull;
  ModConst m{};
  m.q = q;
  m.mu64 = ~0ull / q;
  const unsigned __int128 mu = ~(unsigned __int128)0 / q;
  m.mu_hi = (u64)(mu >> 64);
  m.mu_lo = (u64)mu;
  m.r64 = (u64)(((unsigned __int128)1 << 64) % q);
  u64* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  double best = 0;
  tcks_status st = TCKS_OK;
  if (cudaMalloc(&sink, total * 8) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess) {
    st = TCKS_ERR_CUDA;
  } else {
    for (int rep = 0; rep < 4 && st == TCKS_OK; ++rep) {
      cudaEventRecord(a, 0);
      if (word_bits == 64)
        k_mac_peak<u64><<<blocks, threads>>>(m, iters, sink);
      else
        k_mac_peak<u32><<<blocks, threads>>>(m, iters, sink);
      cudaEventRecord(b, 0);
      if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        st = TCKS_ERR_CUDA;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms > 0) best = std::max(best, (double)total * kChains * iters / (ms * 1e-3));
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  *per_second = best;
  return st;
}

extern "C" tcks_status tcks_calibrate_butterflies(uint32_t word_bits, double* per_second) {
  if (!per_second || (word_bits != 32 && word_bits != 64)) return TCKS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TCKS_ERR_CUDA;
  const u32 threads = 256, blocks = (u32)sms * 8, iters = 4096;
  const u64 total = (u64)threads * blocks;
  // a 59-bit (or 30-bit) prime == 1 mod 2^17 and a twiddle with its Shoup companion
  const u64 q = word_bits == 64 ? 576460752308273153ull : 1073479681ull;
  const u64 w = q / 3 + 12345;
  const u64 wsh = word_bits == 64 ? (u64)(((unsigned __int128)w << 64) / q) : (u64)(((unsigned __int128)w << 32) / q);
  u64* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  double best = 0;
  tcks_status st = TCKS_OK;
  if (cudaMalloc(&sink, total * 8) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess) {
    st = TCKS_ERR_CUDA;
  } else {
    for (int rep = 0; rep < 4 && st == TCKS_OK; ++rep) {
      cudaEventRecord(a, 0);
      if (word_bits == 64)
        k_butterfly_peak<u64><<<blocks, threads>>>(q, w, wsh, iters, sink);
      else
        k_butterfly_peak<u32><<<blocks, threads>>>(q, w, wsh, iters, sink);
      cudaEventRecord(b, 0);
      if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        st = TCKS_ERR_CUDA;
        break;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms > 0) best = std::max(best, (double)total * kChains * iters / (ms * 1e-3));
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  *per_second = best;
  return st;
}

// Bit-packed ciphertext wire format (the communication of §5's encrypted inference): every residue of
// limb i travels in exactly w_i = bit_length(q_i) bits. A limb's segment is ceil(N w_i / 8) bytes,
// residue k in bits [k w_i, (k + 1) w_i), least significant bit first. One thread per output byte
// packs (a byte touches at most two residues, w_i >= 8); one thread per residue unpacks and checks
// that the residue is below q_i.
#include <cuda_runtime.h>

#include "context.h"
#include "kernels.h"

namespace tcks {

namespace {

__device__ __forceinline__ u32 width_of(u64 q) { return 64 - __clzll(q); }

// Byte offset of segment (b, i) inside the payload.
__device__ __forceinline__ u64 seg_off(const DevTables& T, u32 level, u32 b, u32 i) {
  const u64 n = 1ull << T.log_n;
  u64 per_comp = 0, before = 0;
  for (u32 l = 0; l < level; ++l) {
    const u64 bytes = (n * width_of(T.mods[l].q) + 7) / 8;
    per_comp += bytes;
    if (l < i) before += bytes;
  }
  return (u64)b * per_comp + before;
}

// blockIdx.z = request * comps + component; request r's ciphertext at ct + r ct_stride (words), its
// payload at out + r out_stride (bytes)
__global__ void k_pack(DevTables T, const u64* __restrict__ ct, u64 ct_stride, u32 level, u32 comps,
                       unsigned char* __restrict__ out, u64 out_stride) {
  const u32 b = blockIdx.z % comps, r = blockIdx.z / comps, i = blockIdx.y;
  const u64 n = 1ull << T.log_n;
  const u32 w = width_of(T.mods[i].q);
  const u64 seg = (n * w + 7) / 8;
  const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= seg) return;
  const u64* x = ct + r * ct_stride + ((u64)b * level + i) * n;
  const u64 bit = t * 8;
  const u64 k = bit / w;
  const u32 o = (u32)(bit - k * w);
  u64 v = x[k] >> o;  // the rest of residue k
  if (w - o < 8 && k + 1 < n) v |= x[k + 1] << (w - o);
  out[r * out_stride + seg_off(T, level, b, i) + t] = (unsigned char)v;
}

__global__ void k_unpack(DevTables T, const unsigned char* __restrict__ in, u64 in_stride, u32 level, u32 comps,
                         u64* __restrict__ ct, u64 ct_stride, int* __restrict__ status) {
  const u32 b = blockIdx.z % comps, r = blockIdx.z / comps, i = blockIdx.y;
  const u64 n = 1ull << T.log_n;
  const u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const u32 w = width_of(T.mods[i].q);
  const unsigned char* seg = in + r * in_stride + seg_off(T, level, b, i);
  const u64 seg_bytes = (n * w + 7) / 8;
  const u64 bit = k * w;
  const u64 byte0 = bit / 8;
  const u32 o = (u32)(bit % 8);
  // w + o <= 68 bits: up to 9 bytes
  u64 lo = 0;
  for (u32 j = 0; j < 8 && byte0 + j < seg_bytes; ++j) lo |= (u64)seg[byte0 + j] << (8 * j);
  u64 v = lo >> o;
  if (o && byte0 + 8 < seg_bytes) v |= (u64)seg[byte0 + 8] << (64 - o);
  if (w < 64) v &= (1ull << w) - 1;
  if (v >= T.mods[i].q) {
    atomicExch(status, 1);
    v = 0;
  }
  ct[r * ct_stride + ((u64)b * level + i) * n + k] = v;
}

}  // namespace

u64 wire_payload_bytes(const DevTables& T, const u64* host_primes, u32 level) {
  const u64 n = 1ull << T.log_n;
  u64 bytes = 0;
  for (u32 l = 0; l < level; ++l) {
    u32 w = 0;
    while (w < 64 && (host_primes[l] >> w)) ++w;
    bytes += (n * w + 7) / 8;
  }
  return 2 * bytes;
}

void launch_pack_batch(const DevTables& T, const u64* ct, u64 ct_stride, u32 level, unsigned char* out, u64 out_stride,
                       u32 count, cudaStream_t st, u32 comps) {
  const u64 n = 1ull << T.log_n;
  const u64 max_seg = (n * 64 + 7) / 8;
  Launch L(K_ELEMENTWISE, st, 8.0 * count * comps * level * n * 1.9);
  k_pack<<<dim3((unsigned)((max_seg + 255) / 256), level, count * comps), 256, 0, st>>>(T, ct, ct_stride, level, comps,
                                                                                        out, out_stride);
}

void launch_unpack_batch(const DevTables& T, const unsigned char* in, u64 in_stride, u32 level, u64* ct, u64 ct_stride,
                         u32 count, int* status, cudaStream_t st, u32 comps) {
  const u64 n = 1ull << T.log_n;
  Launch L(K_ELEMENTWISE, st, 8.0 * count * comps * level * n * 1.9);
  k_unpack<<<dim3((unsigned)((n + 255) / 256), level, count * comps), 256, 0, st>>>(T, in, in_stride, level, comps, ct,
                                                                                    ct_stride, status);
}

void launch_pack(const DevTables& T, const u64* ct, u32 level, unsigned char* out, cudaStream_t st, u32 comps) {
  launch_pack_batch(T, ct, 0, level, out, 0, 1, st, comps);
}

void launch_unpack(const DevTables& T, const unsigned char* in, u32 level, u64* ct, int* status, cudaStream_t st,
                   u32 comps) {
  launch_unpack_batch(T, in, 0, level, ct, 0, 1, status, st, comps);
}

}  // namespace tcks

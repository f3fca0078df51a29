// Core RNS kernels: batched NTT / INTT (one context, a descriptor table, several contexts),
// element-wise ops, the tensor product, decryption and rescale (the key-switching kernels are in
// kern_keyswitch.cu).
//
// Every kernel that transforms a limb stages it in shared memory: one CTA per limb for N <= 2^14, a
// cluster of 2 or 4 CTAs (each holding a contiguous slice, cross-slice stages over DSMEM) for
// N = 2^15, 2^16. A limb crosses HBM once per kernel; the prologue that fills shared memory and the
// epilogue that drains it carry the surrounding element-wise work (lifts, products, combines).
// Jobs are laid out on blockIdx.x (limb jobs, clusters along x) and blockIdx.y / z (requests and
// rotations), so one launch carries a whole batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>

#include "context.h"
#include "kernels.h"
#include "limb_launch.cuh"
#include "debug_checks.cuh"
#include "ntt.cuh"

namespace tcks {

// Opt a kernel in to more than 48 KB of dynamic shared memory and to the largest shared-memory
// carveout, once per kernel (the attributes are per function, so the registry is keyed by address).
void ensure_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<const void*, size_t> granted;
  std::lock_guard<std::mutex> lock(mu);
  auto it = granted.find(kernel);
  if (it == granted.end()) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    // the default dynamic allowance is 48 KB less the kernel's static shared memory
    cudaFuncAttributes fa{};
    const size_t start = cudaFuncGetAttributes(&fa, kernel) == cudaSuccess ? (size_t)fa.maxDynamicSharedSizeBytes : 0;
    cudaGetLastError();
    it = granted.emplace(kernel, start).first;
  }
  if (bytes > it->second) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(TCKS_ERR_CUDA, "raising a kernel's dynamic shared memory to " + std::to_string(bytes) +
                              " bytes failed: " + cudaGetErrorString(e));
    }
    it->second = bytes;
  }
}

u32 ntt_threads(u32 log_n) { return limb_shape(log_n).threads; }

// Modular butterflies of one length-N transform: (N / 2) log2 N.
static double bfly_per_limb(u32 log_n) { return 0.5 * (double)(1u << log_n) * log_n; }

// --------------------------------------------------------------------------- batched NTT ----
// Job j: limb (j % per) of entry (j / per): src + (j/per)*src_outer + (j%per)*N, prime mod_base + j%per.
template <bool INVERSE, typename W, int LC>
__global__ void k_ntt(DevTables T, const u64* __restrict__ src, u64 src_outer, u64* __restrict__ dst, u64 dst_outer,
                      u32 mod_base, u32 per, u64 src_y, u64 dst_y) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 jo = sl.job / per, ji = sl.job % per;
  const u32 mod = mod_base + ji;
  const ModConst m = T.mods[mod];
  const u64* in = src + sl.y * src_y + jo * src_outer + ji * n + sl.off;
  u64* out = dst + sl.y * dst_y + jo * dst_outer + ji * n + sl.off;
  for (u32 k = 2 * threadIdx.x; k < sl.ns; k += 2 * blockDim.x) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(in + k);
    s[sw(k)] = (W)v.x;
    s[sw(k + 1)] = (W)v.y;
  }
  __syncthreads();
  if (INVERSE) {
    ntt_inv_slice<W, LC>(s, T, mod, sl.rank);
    for (u32 k = 2 * threadIdx.x; k < sl.ns; k += 2 * blockDim.x)
      *reinterpret_cast<ulonglong2*>(out + k) = make_ulonglong2(Ar<W>::inv_out(s[sw(k)], m), Ar<W>::inv_out(s[sw(k + 1)], m));
  } else {
    ntt_fwd_slice<W, LC>(s, T, mod, sl.rank);
    for (u32 k = 2 * threadIdx.x; k < sl.ns; k += 2 * blockDim.x)
      *reinterpret_cast<ulonglong2*>(out + k) = make_ulonglong2(Ar<W>::fwd_out(s[sw(k)], m), Ar<W>::fwd_out(s[sw(k + 1)], m));
  }
}

static void (*const kNttInv[6])(DevTables, const u64*, u64, u64*, u64, u32, u32, u64, u64) = {
    k_ntt<true, u64, 0>, k_ntt<true, u64, 1>, k_ntt<true, u64, 2>,
    k_ntt<true, u32, 0>, k_ntt<true, u32, 1>, k_ntt<true, u32, 2>};
static void (*const kNttFwd[6])(DevTables, const u64*, u64, u64*, u64, u32, u32, u64, u64) = {
    k_ntt<false, u64, 0>, k_ntt<false, u64, 1>, k_ntt<false, u64, 2>,
    k_ntt<false, u32, 0>, k_ntt<false, u32, 1>, k_ntt<false, u32, 2>};

// ------------------------------------------------------ NTT of N >= 2^14 in two passes ----
// A limb of N = 2^(13 + k) elements is transformed in two passes over memory instead of one
// cluster of 2^k CTAs: the first k forward stages pair elements 2^(13) apart and run on columns
// {j + m 2^13 : m < 2^k} in registers; the other 13 stages run on 2^k independent 8192-element
// slices in shared memory (three 64 KB CTAs per SM rather than one 128 KB CTA or a cluster). The
// inverse runs the mirror order, the N^-1 scaling last. Every element meets the same butterflies
// in the same order as in the one-pass transform, so results are identical. Both passes work in
// place on the destination. The transform is integer-pipe bound, so the extra pass over HBM is
// cheaper than the lost occupancy.
constexpr u32 kSplitLogNs = 13;

// Limb job -> (input, output, prime): the strided batch of launch_ntt ...
struct NttJobsStrided {
  const u64* src;
  u64* dst;
  u64 src_outer, dst_outer;
  u32 mod_base, per;
  __device__ __forceinline__ void locate(u32 job, u32 log_n, const u64*& in, u64*& out, u32& mod) const {
    const u32 jo = job / per, ji = job % per;
    mod = mod_base + ji;
    in = src + jo * src_outer + ((u64)ji << log_n);
    out = dst + jo * dst_outer + ((u64)ji << log_n);
  }
};
// ... or a descriptor table (see k_ntt_desc).
struct NttJobsTable {
  NttDescTable tab;
  __device__ __forceinline__ void locate(u32 job, u32 log_n, const u64*& in, u64*& out, u32& mod) const {
    u32 lo = 0, hi = tab.n;
    while (hi - lo > 1) {
      const u32 mid = (lo + hi) >> 1;
      if (tab.d[mid].first <= job)
        lo = mid;
      else
        hi = mid;
    }
    const NttDesc& d = tab.d[lo];
    const u32 local = job - d.first;
    mod = local % d.level;
    in = d.src + ((u64)local << log_n);
    out = d.dst + ((u64)local << log_n);
  }
};

// Columns pass: forward stages 0..K-1 (src -> dst), or inverse stages log_n-K..log_n-1 plus N^-1
// (dst -> dst). Item = (limb job, column j), grid-stride.
template <bool INVERSE, typename W, int K, typename Jobs>
__global__ void k_ntt_columns(DevTables T, const __grid_constant__ Jobs jobs, u32 n_jobs) {
  const u32 log_n = T.log_n, log_cols = log_n - K;
  const u64 items = (u64)n_jobs << log_cols;
  for (u64 it = (u64)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (u64)gridDim.x * blockDim.x) {
    const u32 job = (u32)(it >> log_cols), j = (u32)(it & ((1u << log_cols) - 1));
    const u64* in;
    u64* out;
    u32 mod;
    jobs.locate(job, log_n, in, out, mod);
    const ModConst m = T.mods[mod];
    const W q = (W)m.q;
    W x[1 << K];
    const u64* from = INVERSE ? out : in;
#pragma unroll
    for (int c = 0; c < (1 << K); ++c) x[c] = (W)from[j + ((u64)c << log_cols)];
    if (INVERSE) {
      inv_group<W, K>(x, log_n, log_cols, 0, Ar<W>::tw(T, mod, 2), Ar<W>::tw(T, mod, 3), q);
#pragma unroll
      for (int c = 0; c < (1 << K); ++c) out[j + ((u64)c << log_cols)] = Ar<W>::inv_out(x[c], m);
    } else {
      fwd_group<W, K>(x, 0, 0, Ar<W>::tw(T, mod, 0), Ar<W>::tw(T, mod, 1), q);
#pragma unroll
      for (int c = 0; c < (1 << K); ++c) out[j + ((u64)c << log_cols)] = (u64)x[c];
    }
  }
}

// Slices pass: CTA = slice `rank` of a limb job; forward stages k..log_n-1 (dst -> dst, canonical
// out), or inverse stages 0..12 (src -> dst, unscaled).
template <bool INVERSE, typename W, typename Jobs>
__global__ void k_ntt_slices(DevTables T, const __grid_constant__ Jobs jobs, u32 log_k) {
  TCKS_SMEM(W);
  const u32 log_n = T.log_n, log_ns = log_n - log_k;
  const u32 rank = blockIdx.x & ((1u << log_k) - 1), job = blockIdx.x >> log_k;
  const u64* in;
  u64* out;
  u32 mod;
  jobs.locate(job, log_n, in, out, mod);
  const ModConst m = T.mods[mod];
  const W q = (W)m.q;
  const u32 ns = 1u << log_ns;
  const u64 off = (u64)rank << log_ns;
  const u64* from = (INVERSE ? in : out) + off;
  u64* to = out + off;
  for (u32 k = 2 * threadIdx.x; k < ns; k += 2 * blockDim.x) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(from + k);
    s[sw(k)] = (W)v.x;
    s[sw(k + 1)] = (W)v.y;
  }
  __syncthreads();
  if (INVERSE) {
    ntt_inv_local_rounds<W>(s, log_n, log_ns, rank, Ar<W>::tw(T, mod, 2), Ar<W>::tw(T, mod, 3), q);
    for (u32 k = 2 * threadIdx.x; k < ns; k += 2 * blockDim.x)
      *reinterpret_cast<ulonglong2*>(to + k) = make_ulonglong2(s[sw(k)], s[sw(k + 1)]);
  } else {
    ntt_fwd_local_rounds<W>(s, log_n, log_ns, rank, Ar<W>::tw(T, mod, 0), Ar<W>::tw(T, mod, 1), q);
    for (u32 k = 2 * threadIdx.x; k < ns; k += 2 * blockDim.x)
      *reinterpret_cast<ulonglong2*>(to + k) = make_ulonglong2(Ar<W>::fwd_out(s[sw(k)], m), Ar<W>::fwd_out(s[sw(k + 1)], m));
  }
}

template <bool INVERSE, typename W, typename Jobs>
static void launch_columns(const DevTables& T, const Jobs& jobs, u32 n_jobs, u32 k, cudaStream_t st) {
  const u64 items = (u64)n_jobs << (T.log_n - k);
  const u32 blocks = (u32)std::min<u64>((items + 255) / 256, 152ull * 16);
  if (k == 1) k_ntt_columns<INVERSE, W, 1, Jobs><<<blocks, 256, 0, st>>>(T, jobs, n_jobs);
  if (k == 2) k_ntt_columns<INVERSE, W, 2, Jobs><<<blocks, 256, 0, st>>>(T, jobs, n_jobs);
  if (k == 3) k_ntt_columns<INVERSE, W, 3, Jobs><<<blocks, 256, 0, st>>>(T, jobs, n_jobs);
}

template <bool INVERSE, typename W, typename Jobs>
static void launch_slices(const DevTables& T, const Jobs& jobs, u32 n_jobs, u32 k, cudaStream_t st) {
  const size_t smem = sizeof(W) << kSplitLogNs;
  const void* kern = (const void*)k_ntt_slices<INVERSE, W, Jobs>;
  ensure_smem(kern, smem);
  k_ntt_slices<INVERSE, W, Jobs><<<n_jobs << k, 256, smem, st>>>(T, jobs, k);
}

// The two-pass transform of n_jobs limbs; algorithmic bytes and butterflies go to the slices pass.
template <typename Jobs>
static void launch_ntt_split(const DevTables& T, bool inverse, const Jobs& jobs, u32 n_jobs, cudaStream_t st) {
  const u32 k = T.log_n - kSplitLogNs;
  const double n = (double)(1u << T.log_n);
  const double cols_ops = n_jobs * 0.5 * n * k, slice_ops = n_jobs * 0.5 * n * kSplitLogNs;
  const KernelId id = inverse ? K_NTT_INV : K_NTT_FWD;
  if (!inverse) {
    {
      Launch L(id, st, 0.0, cols_ops);
      if (T.narrow) launch_columns<false, u32>(T, jobs, n_jobs, k, st); else launch_columns<false, u64>(T, jobs, n_jobs, k, st);
    }
    Launch L(id, st, 16.0 * n * n_jobs, slice_ops);
    if (T.narrow) launch_slices<false, u32>(T, jobs, n_jobs, k, st); else launch_slices<false, u64>(T, jobs, n_jobs, k, st);
  } else {
    {
      Launch L(id, st, 16.0 * n * n_jobs, slice_ops);
      if (T.narrow) launch_slices<true, u32>(T, jobs, n_jobs, k, st); else launch_slices<true, u64>(T, jobs, n_jobs, k, st);
    }
    Launch L(id, st, 0.0, cols_ops);
    if (T.narrow) launch_columns<true, u32>(T, jobs, n_jobs, k, st); else launch_columns<true, u64>(T, jobs, n_jobs, k, st);
  }
}

// ------------------------------------------- NTT over several contexts (mixed N and level) ----
// Every N = 2^(13 + k), k = 0..3, is the k column stages (columns of 2^k elements 2^13 apart) plus the
// other 13 stages on 2^k slices of 8192 elements, so batches of different contexts share one columns
// launch (batches with k > 0) and one slices launch: each CTA / item finds its batch in the table
// (binary search on the first job, then a forward walk in the grid-stride loop) and takes that
// batch's context tables. The butterflies and their order are those of the single-context
// transforms, so the results are identical.
__device__ __forceinline__ u32 multi_desc_slice(const MultiNttTable& tab, u64 job) {
  u32 lo = 0, hi = tab.n;
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    if (tab.d[mid].first <= job) lo = mid; else hi = mid;
  }
  return lo;
}

template <bool INVERSE, typename W>
__global__ void k_ntt_slices_multi(const __grid_constant__ MultiNttTable tab) {
  TCKS_SMEM(W);
  const MultiNttDesc& d = tab.d[multi_desc_slice(tab, blockIdx.x)];
  if (dbg_fail(tab.T[0].dbg, d.ctx < tab.n_ctx, DBG_CTX_INDEX)) return;
  const DevTables& T = tab.T[d.ctx];
  const u32 log_n = T.log_n, log_k = log_n - kSplitLogNs;
  const u64 local = blockIdx.x - d.first;
  const u64 limb = local >> log_k;
  if (dbg_fail(T.dbg, limb < d.limbs && d.level > 0, DBG_LIMB_RANGE)) return;  // uniform over the CTA
  const u32 rank = (u32)(local & ((1u << log_k) - 1)), mod = (u32)(limb % d.level);
  if (dbg_fail(T.dbg, mod < T.n_mods, DBG_MOD_INDEX) || dbg_fail(T.dbg, d.src && d.dst, DBG_NULL)) return;
  const ModConst m = T.mods[mod];
  const W q = (W)m.q;
  const u32 ns = 1u << kSplitLogNs;
  const u64 off = (limb << log_n) + ((u64)rank << kSplitLogNs);
  const u64* from = (INVERSE || log_k == 0 ? d.src : d.dst) + off;
  u64* to = d.dst + off;
  for (u32 k = 2 * threadIdx.x; k < ns; k += 2 * blockDim.x) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(from + k);
    s[sw(k)] = (W)v.x;
    s[sw(k + 1)] = (W)v.y;
  }
  __syncthreads();
  if (INVERSE) {
    ntt_inv_local_rounds<W>(s, log_n, kSplitLogNs, rank, Ar<W>::tw(T, mod, 2), Ar<W>::tw(T, mod, 3), q);
    for (u32 k = 2 * threadIdx.x; k < ns; k += 2 * blockDim.x) {  // without columns the N^-1 is taken here
      const u64 a = log_k ? (u64)s[sw(k)] : Ar<W>::inv_out(s[sw(k)], m);
      const u64 b = log_k ? (u64)s[sw(k + 1)] : Ar<W>::inv_out(s[sw(k + 1)], m);
      *reinterpret_cast<ulonglong2*>(to + k) = make_ulonglong2(a, b);
    }
  } else {
    ntt_fwd_local_rounds<W>(s, log_n, kSplitLogNs, rank, Ar<W>::tw(T, mod, 0), Ar<W>::tw(T, mod, 1), q);
    for (u32 k = 2 * threadIdx.x; k < ns; k += 2 * blockDim.x)
      *reinterpret_cast<ulonglong2*>(to + k) = make_ulonglong2(Ar<W>::fwd_out(s[sw(k)], m), Ar<W>::fwd_out(s[sw(k + 1)], m));
  }
}

template <bool INVERSE, typename W, int K>
__device__ __forceinline__ void multi_column(const DevTables& T, const MultiNttDesc& d, u64 local) {
  const u32 log_n = T.log_n;
  const u64 job = local >> kSplitLogNs;
  const u32 j = (u32)(local & ((1u << kSplitLogNs) - 1)), mod = (u32)(job % d.level);
  const ModConst m = T.mods[mod];
  const W q = (W)m.q;
  const u64* in = d.src + (job << log_n);
  u64* out = d.dst + (job << log_n);
  W x[1 << K];
  const u64* from = INVERSE ? out : in;
#pragma unroll
  for (int c = 0; c < (1 << K); ++c) x[c] = (W)from[j + ((u64)c << kSplitLogNs)];
  if (INVERSE) {
    inv_group<W, K>(x, log_n, kSplitLogNs, 0, Ar<W>::tw(T, mod, 2), Ar<W>::tw(T, mod, 3), q);
#pragma unroll
    for (int c = 0; c < (1 << K); ++c) out[j + ((u64)c << kSplitLogNs)] = Ar<W>::inv_out(x[c], m);
  } else {
    fwd_group<W, K>(x, 0, 0, Ar<W>::tw(T, mod, 0), Ar<W>::tw(T, mod, 1), q);
#pragma unroll
    for (int c = 0; c < (1 << K); ++c) out[j + ((u64)c << kSplitLogNs)] = (u64)x[c];
  }
}

template <bool INVERSE, typename W>
__global__ void k_ntt_columns_multi(const __grid_constant__ MultiNttTable tab) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  u64 it = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= tab.col_items) return;
  u32 di = 0;
  {  // the batch of the first item, then walk forward (items only grow)
    u32 lo = 0, hi = tab.n;
    while (hi - lo > 1) {
      const u32 mid = (lo + hi) >> 1;
      if (tab.d[mid].col_first <= it) lo = mid; else hi = mid;
    }
    di = lo;
  }
  for (; it < tab.col_items; it += stride) {
    while (di + 1 < tab.n && tab.d[di + 1].col_first <= it) ++di;
    const MultiNttDesc& d = tab.d[di];
    if (dbg_fail(tab.T[0].dbg, d.ctx < tab.n_ctx, DBG_CTX_INDEX)) continue;
    const DevTables& T = tab.T[d.ctx];
    const u64 local = it - d.col_first;
    if (dbg_fail(T.dbg, (local >> kSplitLogNs) < d.limbs && d.level > 0, DBG_LIMB_RANGE) ||
        dbg_fail(T.dbg, (u32)((local >> kSplitLogNs) % d.level) < T.n_mods, DBG_MOD_INDEX) ||
        dbg_fail(T.dbg, d.src && d.dst, DBG_NULL))
      continue;
    switch (T.log_n - kSplitLogNs) {
      case 1: multi_column<INVERSE, W, 1>(T, d, local); break;
      case 2: multi_column<INVERSE, W, 2>(T, d, local); break;
      case 3: multi_column<INVERSE, W, 3>(T, d, local); break;
      default: break;  // N = 2^13 batches have no columns (and no items)
    }
  }
}

u32 launch_ntt_multi(bool inverse, const MultiNttBatch* batches, u32 n, cudaStream_t st, u32 understate) {
  if (!n || n > kMultiDescMax) return 0;
  MultiNttTable tab{};
  const bool narrow = batches[0].T->narrow != 0;
  double bytes = 0, slice_ops = 0, col_ops = 0;
  for (u32 i = 0; i < n; ++i) {
    const MultiNttBatch& b = batches[i];
    if (b.T->log_n < kSplitLogNs || b.T->log_n > kSplitLogNs + 3 || (b.T->narrow != 0) != narrow) return 0;
    u32 c = 0;
    while (c < tab.n_ctx && tab.T[c].mods != b.T->mods) ++c;  // contexts told apart by their tables
    if (c == tab.n_ctx) {
      if (tab.n_ctx == kMultiCtxMax) return 0;
      tab.T[tab.n_ctx++] = *b.T;
    }
    const u64 limbs = (u64)b.polys * b.level;
    const u32 log_k = b.T->log_n - kSplitLogNs;
    MultiNttDesc& d = tab.d[tab.n];
    d.src = b.src;
    d.dst = b.dst;
    d.level = b.level;
    d.limbs = (u32)limbs;
    d.ctx = c;
    d.first = tab.slice_jobs;
    d.col_first = tab.col_items;
    ++tab.n;
    tab.slice_jobs += limbs << log_k;
    if (log_k) tab.col_items += limbs << kSplitLogNs;
    const double nn = (double)(1u << b.T->log_n);
    bytes += 16.0 * nn * limbs;
    slice_ops += limbs * 0.5 * nn * kSplitLogNs;
    col_ops += limbs * 0.5 * nn * log_k;
  }
  if (!tab.slice_jobs || tab.slice_jobs > 0x7fffffffull) return 0;
  if (kDebugChecks) {  // the table's invariants: offsets from 0, monotone, adding up to the launch
    u64 slices = 0, cols = 0;
    for (u32 i = 0; i < tab.n; ++i) {
      const MultiNttDesc& d = tab.d[i];
      const u32 log_k = tab.T[d.ctx].log_n - kSplitLogNs;
      if (d.ctx >= tab.n_ctx || d.first != slices || d.col_first != cols || !d.level || d.limbs % d.level)
        fail(TCKS_ERR_DEBUG_CHECK, "multi-context NTT table: descriptor " + std::to_string(i) + " out of order or range");
      slices += (u64)d.limbs << log_k;
      if (log_k) cols += (u64)d.limbs << kSplitLogNs;
    }
    if (slices != tab.slice_jobs || cols != tab.col_items)
      fail(TCKS_ERR_DEBUG_CHECK, "multi-context NTT table: descriptors do not add up to the launch");
    if (understate) tab.d[tab.n - 1].limbs -= std::min(understate, tab.d[tab.n - 1].limbs);
  }
  const KernelId id = inverse ? K_NTT_INV : K_NTT_FWD;
  const size_t smem = (narrow ? 4 : 8) << kSplitLogNs;
  auto slices = [&]() {
    Launch L(id, st, bytes, slice_ops);
    const void* k = narrow ? (inverse ? (const void*)k_ntt_slices_multi<true, u32> : (const void*)k_ntt_slices_multi<false, u32>)
                           : (inverse ? (const void*)k_ntt_slices_multi<true, u64> : (const void*)k_ntt_slices_multi<false, u64>);
    ensure_smem(k, smem);
    const u32 grid = (u32)tab.slice_jobs;
    if (narrow) {
      if (inverse) k_ntt_slices_multi<true, u32><<<grid, 256, smem, st>>>(tab);
      else k_ntt_slices_multi<false, u32><<<grid, 256, smem, st>>>(tab);
    } else {
      if (inverse) k_ntt_slices_multi<true, u64><<<grid, 256, smem, st>>>(tab);
      else k_ntt_slices_multi<false, u64><<<grid, 256, smem, st>>>(tab);
    }
  };
  auto columns = [&]() {
    if (!tab.col_items) return;
    Launch L(id, st, 0.0, col_ops);
    const u32 blocks = (u32)std::min<u64>((tab.col_items + 255) / 256, 152ull * 16);
    if (narrow) {
      if (inverse) k_ntt_columns_multi<true, u32><<<blocks, 256, 0, st>>>(tab);
      else k_ntt_columns_multi<false, u32><<<blocks, 256, 0, st>>>(tab);
    } else {
      if (inverse) k_ntt_columns_multi<true, u64><<<blocks, 256, 0, st>>>(tab);
      else k_ntt_columns_multi<false, u64><<<blocks, 256, 0, st>>>(tab);
    }
  };
  if (inverse) {
    slices();
    columns();
  } else {
    columns();
    slices();
  }
  return tab.col_items ? 2 : 1;
}

// ------------------------------------------------------- NTT over a descriptor table ----
// One launch over several polynomial batches of the same N and chain but their own levels and
// buffers: CTA job j belongs to the last descriptor whose first job is <= j, and is limb
// (j - first) of that batch laid out [polys][level][N] (prime (j - first) % level).
template <bool INVERSE, typename W, int LC>
__global__ void k_ntt_desc(DevTables T, const __grid_constant__ NttDescTable tab) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  u32 lo = 0, hi = tab.n;
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    if (tab.d[mid].first <= sl.job)
      lo = mid;
    else
      hi = mid;
  }
  const NttDesc& d = tab.d[lo];
  const u32 local = sl.job - d.first;
  // the same for every CTA of the limb (cluster), so a skip reaches no barrier
  if (dbg_fail(T.dbg, local < d.limbs && d.level > 0, DBG_LIMB_RANGE)) return;
  const u32 mod = local % d.level;
  if (dbg_fail(T.dbg, mod < T.n_mods, DBG_MOD_INDEX) || dbg_fail(T.dbg, d.src && d.dst, DBG_NULL)) return;
  const ModConst m = T.mods[mod];
  const u64* in = d.src + ((u64)local << T.log_n) + sl.off;
  u64* out = d.dst + ((u64)local << T.log_n) + sl.off;
  for (u32 k = 2 * threadIdx.x; k < sl.ns; k += 2 * blockDim.x) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(in + k);
    s[sw(k)] = (W)v.x;
    s[sw(k + 1)] = (W)v.y;
  }
  __syncthreads();
  if (INVERSE) {
    ntt_inv_slice<W, LC>(s, T, mod, sl.rank);
    for (u32 k = 2 * threadIdx.x; k < sl.ns; k += 2 * blockDim.x)
      *reinterpret_cast<ulonglong2*>(out + k) = make_ulonglong2(Ar<W>::inv_out(s[sw(k)], m), Ar<W>::inv_out(s[sw(k + 1)], m));
  } else {
    ntt_fwd_slice<W, LC>(s, T, mod, sl.rank);
    for (u32 k = 2 * threadIdx.x; k < sl.ns; k += 2 * blockDim.x)
      *reinterpret_cast<ulonglong2*>(out + k) = make_ulonglong2(Ar<W>::fwd_out(s[sw(k)], m), Ar<W>::fwd_out(s[sw(k + 1)], m));
  }
}

static void (*const kNttDescInv[6])(DevTables, NttDescTable) = {
    k_ntt_desc<true, u64, 0>, k_ntt_desc<true, u64, 1>, k_ntt_desc<true, u64, 2>,
    k_ntt_desc<true, u32, 0>, k_ntt_desc<true, u32, 1>, k_ntt_desc<true, u32, 2>};
static void (*const kNttDescFwd[6])(DevTables, NttDescTable) = {
    k_ntt_desc<false, u64, 0>, k_ntt_desc<false, u64, 1>, k_ntt_desc<false, u64, 2>,
    k_ntt_desc<false, u32, 0>, k_ntt_desc<false, u32, 1>, k_ntt_desc<false, u32, 2>};

void launch_ntt_desc(const DevTables& T, bool inverse, const NttDescTable& tab, u32 total_jobs, cudaStream_t st) {
  if (!total_jobs || !tab.n) return;
  if (T.log_n > kSplitLogNs) {
    NttJobsTable jobs;
    jobs.tab = tab;
    launch_ntt_split(T, inverse, jobs, total_jobs, st);
    return;
  }
  Launch L(inverse ? K_NTT_INV : K_NTT_FWD, st, 16.0 * total_jobs * (1u << T.log_n), total_jobs * bfly_per_limb(T.log_n));
  if (inverse)
    launch_limb(kNttDescInv, T.narrow, total_jobs, 1, T.log_n, st, T.limb_threads, T, tab);
  else
    launch_limb(kNttDescFwd, T.narrow, total_jobs, 1, T.log_n, st, T.limb_threads, T, tab);
}

void launch_ntt(const DevTables& T, bool inverse, const u64* src, u64 src_outer, u64* dst, u64 dst_outer, u32 count,
                u32 mod_base, u32 per, cudaStream_t st, u32 ny, u64 src_y, u64 dst_y) {
  if (!count || !ny) return;
  if (T.log_n > kSplitLogNs) {
    for (u32 y = 0; y < ny; ++y) {
      const NttJobsStrided jobs{src + y * src_y, dst + y * dst_y, src_outer, dst_outer, mod_base, per};
      launch_ntt_split(T, inverse, jobs, count, st);
    }
    return;
  }
  const double jobs = (double)count * ny;
  Launch L(inverse ? K_NTT_INV : K_NTT_FWD, st, 16.0 * jobs * (1u << T.log_n), jobs * bfly_per_limb(T.log_n));
  if (inverse)
    launch_limb(kNttInv, T.narrow, count, ny, T.log_n, st, T.limb_threads, T, src, src_outer, dst, dst_outer, mod_base, per,
                src_y, dst_y);
  else
    launch_limb(kNttFwd, T.narrow, count, ny, T.log_n, st, T.limb_threads, T, src, src_outer, dst, dst_outer, mod_base, per,
                src_y, dst_y);
}

// a * b mod q: the 64-bit Barrett of the product when every prime is below 2^31, else the 128-bit one
__device__ __forceinline__ u64 mulq(u64 a, u64 b, const ModConst& m, u32 narrow) {
  return narrow ? reduce64(a * b, m) : mul_mod(a, b, m);
}

// ------------------------------------------------------------------ 32-bit copies of keys ----
void count_launch();

__global__ void k_narrow_copy(const u64* __restrict__ src, u32* __restrict__ dst, u64 n) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) dst[i] = (u32)src[i];
}

void launch_narrow_copy(const u64* src, u32* dst, u64 n, cudaStream_t st) {
  if (!n) return;
  const u64 blocks = std::min<u64>((n + 255) / 256, 152ull * 16);
  count_launch();
  k_narrow_copy<<<(u32)blocks, 256, 0, st>>>(src, dst, n);
}

// ------------------------------------------------------------------------ element-wise ops ----
// Operands laid out [polys][ell][N] (a batch of ciphertexts is [2B][ell][N]); element e belongs to
// limb (e >> log_n) % ell and component ((e >> log_n) / ell) % 2. A plain operand b is shared by every
// polynomial (b_stride = 0) or is one plaintext per ciphertext, b_stride words apart.
__global__ void k_elementwise(DevTables T, u32 op, const u64* __restrict__ a, const u64* __restrict__ b,
                              u64* __restrict__ out, u32 ell, u32 polys, u64 b_stride) {
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
      case OP_ADD: {
        const ulonglong2 y = reinterpret_cast<const ulonglong2*>(b)[e2];
        r.x = add_mod(x.x, y.x, m.q);
        r.y = add_mod(x.y, y.y, m.q);
        break;
      }
      case OP_SUB: {
        const ulonglong2 y = reinterpret_cast<const ulonglong2*>(b)[e2];
        r.x = sub_mod(x.x, y.x, m.q);
        r.y = sub_mod(x.y, y.y, m.q);
        break;
      }
      case OP_NEG:
        r.x = neg_mod(x.x, m.q);
        r.y = neg_mod(x.y, m.q);
        break;
      case OP_MUL_PLAIN: {  // b is a plaintext [>= ell][N] (per ciphertext when b_stride != 0)
        const ulonglong2 y =
            reinterpret_cast<const ulonglong2*>(b + (poly >> 1) * b_stride + (u64)limb * n)[(e & (n - 1)) >> 1];
        r.x = mulq(x.x, y.x, m, T.narrow);
        r.y = mulq(x.y, y.y, m, T.narrow);
        break;
      }
      default: {  // OP_ADD_PLAIN / OP_SUB_PLAIN: only component 0 of each ciphertext changes
        if ((poly & 1u) == 0) {
          const ulonglong2 y =
              reinterpret_cast<const ulonglong2*>(b + (poly >> 1) * b_stride + (u64)limb * n)[(e & (n - 1)) >> 1];
          if (op == OP_ADD_PLAIN) {
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
                        cudaStream_t st, u64 b_stride) {
  const u64 e2 = ((u64)polys * ell << T.log_n) >> 1;
  const double limb = 8.0 * ell * (1u << T.log_n);  // bytes of one [ell][N] polynomial
  const double by = op == OP_NEG ? 2.0 * polys * limb
                    : (op == OP_ADD || op == OP_SUB) ? 3.0 * polys * limb
                    : b_stride ? 2.5 * polys * limb                                  // a plaintext per ciphertext
                               : (2.0 * polys + 1.0) * limb;  // shared plaintext operand
  Launch L(K_ELEMENTWISE, st, by);
  k_elementwise<<<ew_blocks(e2), 256, 0, st>>>(T, op, a, b, out, ell, polys, b_stride);
}

// Tensor product of `count` pairs: (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1); a, b [count][2][ell][N],
// out [count][3][ell][N].
__global__ void k_tensor(DevTables T, const u64* __restrict__ a, const u64* __restrict__ b, u64* __restrict__ out,
                         u32 ell, u32 count) {
  const u32 log_n = T.log_n;
  const u64 per_poly = (u64)ell << log_n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < per_poly * count; e += (u64)gridDim.x * blockDim.x) {
    const u64 c = e / per_poly, o = e - c * per_poly;
    const ModConst m = T.mods[o >> log_n];
    const u64* ac = a + c * 2 * per_poly;
    const u64* bc = b + c * 2 * per_poly;
    u64* oc = out + c * 3 * per_poly;
    const u64 a0 = ac[o], a1 = ac[per_poly + o], b0 = bc[o], b1 = bc[per_poly + o];
    oc[o] = mulq(a0, b0, m, T.narrow);
    Acc128 acc{0, 0};
    mac128(acc, a0, b1);
    mac128(acc, a1, b0);
    oc[per_poly + o] = reduce128(acc.hi, acc.lo, m);
    oc[2 * per_poly + o] = mulq(a1, b1, m, T.narrow);
  }
}

void launch_tensor(const DevTables& T, const u64* a, const u64* b, u64* out, u32 ell, u32 count, cudaStream_t st) {
  const u64 e = ((u64)ell << T.log_n) * count;
  Launch L(K_TENSOR, st, 7.0 * 8.0 * e, 4.0 * e);
  k_tensor<<<ew_blocks(e / 2 + 1), 256, 0, st>>>(T, a, b, out, ell, count);
}

// Decryption kernel: m = c0 + c1 * s (+ c2 * s^2 for a three-component product) over limbs < ell (s
// has L+1 limbs, chain order).
__global__ void k_decrypt(DevTables T, const u64* __restrict__ ct, const u64* __restrict__ s, u64* __restrict__ pt,
                          u32 ell, u32 size) {
  const u32 log_n = T.log_n;
  const u64 per_poly = (u64)ell << log_n;
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < per_poly; e += (u64)gridDim.x * blockDim.x) {
    const ModConst m = T.mods[e >> log_n];
    u64 v = add_mod(ct[e], mulq(ct[per_poly + e], s[e], m, T.narrow), m.q);
    if (size == 3) v = add_mod(v, mulq(ct[2 * per_poly + e], mulq(s[e], s[e], m, T.narrow), m, T.narrow), m.q);
    pt[e] = v;
  }
}

void launch_decrypt(const DevTables& T, const u64* ct, const u64* s, u64* pt, u32 ell, cudaStream_t st, u32 size) {
  const u64 e = (u64)ell << T.log_n;
  Launch L(K_DECRYPT, st, (size + 2.0) * 8.0 * e);
  k_decrypt<<<ew_blocks(e / 2 + 1), 256, 0, st>>>(T, ct, s, pt, ell, size);
}

// ---------------------------------------------------------------- drop the last prime ----
// Rescale (drop = q_{ell-1}) and ModDown (drop = P) share this combine:
//   out[p][i] = (in[p][i] - NTT_i(bal(top[p]) mod q_i)) * drop^-1 mod q_i,  i < n_out,
// with top[p] the coefficient-domain limb of the dropped prime. Limb job = p * n_out + i.
template <typename W, int LC>
__global__ void k_drop_combine(DevTables T, const u64* __restrict__ in, u64 in_poly_stride,
                               const u64* __restrict__ top, u32 drop_mod, u32 n_out, u64* __restrict__ out) {
  TCKS_SMEM(W);
  const Slice sl = slice_of<LC>(T);
  const u64 n = 1ull << T.log_n;
  const u32 p = sl.job / n_out, i = sl.job % n_out;
  const ModConst mi = T.mods[i];
  const ModConst md = T.mods[drop_mod];
  const PairConst pc = T.pairs[(u64)drop_mod * T.n_mods + i];
  const u64* tp = top + (u64)p * n + sl.off;
  if constexpr (LC == 0) {
    ntt_fwd_limb_load<W>(s, T, i, [&](u32 k) { return lift_balanced_w<W>(tp[k], md.half, pc.qa_mod_b, mi); });
  } else {
    for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) s[sw(k)] = lift_balanced_w<W>(tp[k], md.half, pc.qa_mod_b, mi);
    __syncthreads();
    ntt_fwd_slice<W, LC>(s, T, i, sl.rank);
  }
  const u64* src = in + (u64)p * in_poly_stride + (u64)i * n + sl.off;
  u64* dst = out + ((u64)p * n_out + i) * n + sl.off;
  for (u32 k = threadIdx.x; k < sl.ns; k += blockDim.x) {
    const u64 c = sub_mod(src[k], fwd_fin(s[sw(k)], mi), mi.q);
    dst[k] = Ew<W>::shoup_inv(c, pc, mi);
  }
}

static decltype(&k_drop_combine<u64, 0>) const K6_k_drop_combine[6] = TCKS_K6(k_drop_combine);

void launch_rescale(const DevTables& T, const u64* ct, u32 ell, u32 polys, u64* top_tmp, u64* out, cudaStream_t st) {
  const u64 n = 1ull << T.log_n;
  // INTT of the last limb of each polynomial
  launch_ntt(T, true, ct + (u64)(ell - 1) * n, (u64)ell * n, top_tmp, n, polys, ell - 1, 1, st);
  Launch L(K_DROP, st, 8.0 * n * polys * (2.0 * (ell - 1) + 1.0), (double)polys * (ell - 1) * (bfly_per_limb(T.log_n) + n));
  launch_limb(K6_k_drop_combine, T.narrow, polys * (ell - 1), 1, T.log_n, st, T.limb_threads, T, ct, (u64)ell * n, (const u64*)top_tmp, ell - 1,
              ell - 1, out);
}

// ------------------------------------------------------------ launch-shape limits (autotune) ----
// Largest CTA size every limb kernel of this file accepts for the word type and cluster split.
template <typename F>
static u32 max_threads_of(F k) {
  cudaFuncAttributes a{};
  if (cudaFuncGetAttributes(&a, (const void*)k) != cudaSuccess) return 0;
  return (u32)a.maxThreadsPerBlock;
}
u32 limb_threads_cap_core(bool narrow, u32 log_c) {
  const u32 i = (narrow ? 3 : 0) + log_c;
  u32 cap = 1024;
  for (u32 t : {max_threads_of(kNttFwd[i]), max_threads_of(kNttInv[i]), max_threads_of(kNttDescFwd[i]),
                max_threads_of(kNttDescInv[i]), max_threads_of(K6_k_drop_combine[i]),
                limb_threads_cap_keyswitch(narrow, log_c)})
    cap = t < cap ? t : cap;
  return cap;
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

// Once per device, with that device current: resolve the scratch array's device address. Returns
// nullptr on failure. (The shared-memory limits of the two kernels are raised on every call through
// ensure_smem, whose registry only ever raises a limit; setting them here behind its back would let a
// later ordinary launch of the same kernel at a smaller N lower the limit again.)
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
  const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_rescale_scratch);
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
  drop_stale_cuda_error();  // report only this call's launches
  std::string why;
  u64* scratch = noalloc_setup(ctx->device, &why);
  if (!scratch) return abi_record(TCKS_ERR_CUDA, "rescale_noalloc: " + why);
  const DevTables& T = ctx->T;
  const u64 n = 1ull << log_n;
  const LimbShape sh = limb_shape(log_n);  // one CTA per limb at these sizes
  // the two launches of launch_rescale, without its allocating bookkeeping
  const size_t smem = T.narrow ? sh.smem / 2 : sh.smem;
  auto ntt = T.narrow ? k_ntt<true, u32, 0> : k_ntt<true, u64, 0>;
  auto drop = T.narrow ? k_drop_combine<u32, 0> : k_drop_combine<u64, 0>;
  ensure_smem((const void*)ntt, smem);  // allocates no device memory
  ensure_smem((const void*)drop, smem);
  count_launch();
  ntt<<<2, sh.threads, smem, ctx->stream>>>(T, d_in + (u64)(level - 1) * n, (u64)level * n, scratch, n, level - 1, 1,
                                            0, 0);
  count_launch();
  drop<<<2 * (level - 1), sh.threads, smem, ctx->stream>>>(T, d_in, (u64)level * n, scratch, level - 1, level - 1,
                                                             d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return abi_record(TCKS_ERR_CUDA, std::string("rescale_noalloc: ") + cudaGetErrorString(e));
  abi_clear();
  return TCKS_OK;
}

// The double-hoisted accumulation of the vector x matrix product (see kern_vecmat.cu) with each
// rotation's operands staged in shared memory by bulk (TMA engine) copies, for 32-bit words.
//
// A CTA owns EB consecutive elements of one slot i and RPT requests per thread; per rotation it needs
// the CTA's block of the 2 ELL key limbs and of the KO diagonals, and, per request, one block of each
// of the ELL digit limbs and of c0: the NTT-domain automorphism maps an aligned block of EB elements
// onto an aligned block, so the sources of the CTA's elements fill exactly one block. The lanes of warp
// 0 issue the rotation's copies in parallel into one of S stage buffers (one mbarrier each), S
// rotations ahead of the computing threads, which then read the keys and diagonals at their own
// element and the digits and c0 at their source's place in the block (an in-block permutation; an
// aligned block of 32 elements maps onto one, so the reads are free of bank conflicts). The arithmetic
// and the partial layout are those of the per-thread kernel, so the results are the same bits.
//
// Every wait is bounded (bulk_copy.cuh). A wait that runs out, or a source off its 16-byte alignment
// (no copy is then issued for that rotation), sets a bit of the context's kernel error word, which
// the host reads after synchronizing; a CTA that finds the timeout bit already set leaves at once.
#include <cuda_runtime.h>

#include <string>

#include "../../include/tcks.h"
#include "bulk_copy.cuh"
#include "context.h"
#include "dh_acc.cuh"
#include "kernels.h"
#include "ntt.cuh"

namespace tcks {

namespace {

// Bits of a context's kernel error word (DevTables::kerr).
constexpr u32 kErrWaitTimeout = 1u, kErrCopyAlign = 2u;

// One rotation's operands, byte offsets into a stage buffer: the 2 ELL key words [2j + b][EB] (u64),
// the digits [rr][j][EB] of the source block (u32), the c0 words [rr][EB] of the source block (u64)
// and KO diagonal blocks [o][EB] (u64).
template <int ELL, int RPT, int KO, int EB>
struct DhStage {
  static constexpr u32 kKey = 0;
  static constexpr u32 kDig = kKey + 16u * ELL * EB;
  static constexpr u32 kC0 = kDig + 4u * RPT * ELL * EB;
  static constexpr u32 kDiag = kC0 + 8u * RPT * EB;
  static constexpr u32 kBytes = kDiag + 8u * KO * EB;
  static constexpr u32 kCopiesMax = 2 * ELL + RPT * ELL + RPT + KO;
};

__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Copy c of a rotation (keys, then digits request by request, then c0 per request, then diagonals):
// its destination offset in the stage, source and size. False when c is past the rotation's copies.
template <int ELL, int RPT, int KO, int EB>
struct DhCopies {
  using St = DhStage<ELL, RPT, KO, EB>;
  const u64* k0;      // the CTA's block of key limb 0 of the rotation
  u64 kstep;          // words between key limbs
  const u32* dig[RPT];  // request rr's source block of digit limb 0 (slot i)
  const u64* c0[RPT];   // request rr's source block of c0 (slot i < ell)
  const u64* dk;      // the CTA's block of diagonal 0 (null: unit diagonals)
  u64 diag_set, dig_step;
  bool has_c0;

  __device__ __forceinline__ bool get(u32 c, u32& dst, const void*& src, u32& bytes) const {
    if (c < 2u * ELL) {
      dst = St::kKey + c * EB * 8u;
      src = k0 + c * kstep;
      bytes = EB * 8u;
      return true;
    }
    c -= 2u * ELL;
    if (c < (u32)(RPT * ELL)) {
      dst = St::kDig + c * EB * 4u;
      src = dig[c / ELL] + (u64)(c % ELL) * dig_step;
      bytes = EB * 4u;
      return true;
    }
    c -= RPT * ELL;
    if (has_c0) {
      if (c < (u32)RPT) {
        dst = St::kC0 + c * EB * 8u;
        src = c0[c];
        bytes = EB * 8u;
        return true;
      }
      c -= RPT;
    }
    if (dk && c < (u32)KO) {
      dst = St::kDiag + c * EB * 8u;
      src = dk + (u64)c * diag_set;
      bytes = EB * 8u;
      return true;
    }
    return false;
  }
};

template <int ELL, int RPT, int KO, int EB, int S>
__global__ void __launch_bounds__(EB, KO > 1 ? 2 : (EB >= 256 ? 3 : 6))
    k_vecmat_dh_acc_bulk(DevTables T, const __grid_constant__ VecmatDhPlan p) {
  using St = DhStage<ELL, RPT, KO, EB>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) u64 full[S];
  __shared__ u32 stage_g[S];  // Galois element of the rotation a stage holds
  __shared__ int abort_flag;
  constexpr u32 ell = ELL, slots = ELL + 1;
  const u32 log_n = T.log_n;
  const u64 n = 1ull << log_n;
  const u32 groups = (p.B + RPT - 1) / RPT;
  const u32 eblocks = (u32)(n / EB);
  const u32 rg = blockIdx.x % groups;  // requests fastest, then element blocks, then the slot
  const u32 rest = blockIdx.x / groups;
  const u32 eb = rest % eblocks, i = rest / eblocks;
  const u32 chunk = blockIdx.y;
  const u32 mod = i < ell ? i : T.L;
  const ModConst m = T.mods[mod];
  const u32 t = threadIdx.x, lane = t & 31u;
  const bool issuer = t < 32;  // warp 0 issues the copies
  const u32 r0 = chunk * p.chunk, r1 = min(p.R, r0 + p.chunk);
  const bool unit = p.diag == nullptr;  // a hoisted rotation sum: every diagonal is 1
  const bool has_c0 = i < ell;
  u32 n_issued = 0;  // warp 0: rotations staged so far (stage k holds those with index k mod S)

  // warp 0: rotation r's operands into stage s, one copy per lane (all sources 16-byte aligned, or none)
  auto issue = [&](u32 r, u32 s) {
    const KsKey kk = p.keys[r];
    DhCopies<ELL, RPT, KO, EB> cp;
    const u32 key_slot = i < ell ? i : kk.K;
    cp.k0 = kk.key + (u64)key_slot * n + (u64)eb * EB;
    cp.kstep = (u64)(kk.K + 1) * n;
    const u64 sbase = (u64)(galois_src(eb * EB, kk.g, log_n) / EB) * EB;  // first source element
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const u32 rq = min(rg * RPT + rr, p.B - 1);  // a short last group repeats a request, never stored
      cp.dig[rr] = reinterpret_cast<const u32*>(p.digits) + rq * p.digits_b + (u64)i * n + sbase;
      cp.c0[rr] = p.ct + rq * p.ct_b + (u64)i * n + sbase;
    }
    cp.dk = unit ? nullptr
                 : p.diag + (u64)(r + 1) * p.diag_stride + (u64)(i < ell ? i : p.p_limb) * n + (u64)eb * EB;
    cp.diag_set = p.diag_set;
    cp.dig_step = (u64)slots * n;
    cp.has_c0 = has_c0;
    ++n_issued;
    u32 dst[2], bytes[2];
    const void* src[2];
    bool mine[2], ok = true;
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // at most 2 * 8 + 2 * 8 + 2 + 4 = 38 copies: two per lane
      mine[k] = cp.get(lane + 32u * k, dst[k], src[k], bytes[k]);
      if (mine[k]) ok = ok && aligned16(src[k]);
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) {
      stage_g[s] = kk.g;
      const u32 total = 16u * ELL * EB + 4u * RPT * ELL * EB + (has_c0 ? 8u * RPT * EB : 0u) + (unit ? 0u : 8u * KO * EB);
      if (!ok) atomicOr(T.kerr, kErrCopyAlign);
      mbar_arrive_expect_tx(&full[s], ok ? total : 0u);
    }
    if (!ok) return;
    unsigned char* st = dsm + (size_t)s * St::kBytes;
    fence_proxy_async_smem();  // this stage was read through the generic proxy before
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (mine[k]) bulk_g2s(st + dst[k], src[k], bytes[k], &full[s]);
  };

  if (t == 0) {
#pragma unroll
    for (int k = 0; k < S; ++k) mbar_init(&full[k], 1);
    mbar_init_fence();
    // a wait of another CTA already ran out: the launch's results are invalid, leave at once
    abort_flag = (*(volatile u32*)T.kerr & kErrWaitTimeout) ? 1 : 0;
  }
  __syncthreads();
  if (abort_flag) return;
  if (issuer)
    for (u32 k = 0; k < (u32)S && r0 + k < r1; ++k) issue(r0 + k, k);
  __syncthreads();  // stage_g of the first stages

  const u32 kb = 2u * brv(eb * EB + t, log_n) + 1u;  // the element's exponent; a rotation multiplies it by g
  const u32 emask = (2u << log_n) - 1u;
  DhAcc<u32> u0[RPT * KO], u1[RPT * KO], a0[RPT * KO];
  u32 it = 0;
  for (u32 r = r0; r < r1; ++r, ++it) {
    const u32 s = it % S;
    if (!mbar_wait_bounded(&full[s], (it / S) & 1u)) {
      abort_flag = 1;
    } else {
      const unsigned char* st = dsm + (size_t)s * St::kBytes;
      const u64* ks = reinterpret_cast<const u64*>(st + St::kKey);
      const u32* ds = reinterpret_cast<const u32*>(st + St::kDig);
      const u64* cs = reinterpret_cast<const u64*>(st + St::kC0);
      const u64* dg = reinterpret_cast<const u64*>(st + St::kDiag);
      const u32 e = (kb * stage_g[s]) & emask;
      const u32 ls = brv((e - 1u) >> 1, log_n) & (EB - 1);  // the source's place in its block
      KsSum<u32, ELL> s0[RPT], s1[RPT];
#pragma unroll
      for (int j = 0; j < ELL; ++j) {
        const u64 w0 = ks[(2 * j) * EB + t], w1 = ks[(2 * j + 1) * EB + t];
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) {
          const u64 d = ds[(rr * ELL + j) * EB + ls];
          s0[rr].mac(d, w0, j);
          s1[rr].mac(d, w1, j);
        }
      }
      constexpr bool kCarry = ELL > 4;
      if (unit) {
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) {
          u32 c;
          u64 v = s0[rr].raw(c);
          u0[rr].add_wide(v, c);
          v = s1[rr].raw(c);
          u1[rr].add_wide(v, c);
          if (has_c0) a0[rr].add(cs[rr * EB + ls]);
        }
      } else if (KO == 1) {
        const u64 dv = dg[t];
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) {
          u32 c;
          u64 v = s0[rr].raw(c);
          u0[rr].template mac_wide<kCarry>(v, c, dv);
          v = s1[rr].raw(c);
          u1[rr].template mac_wide<kCarry>(v, c, dv);
          if (has_c0) a0[rr].mac(cs[rr * EB + ls], dv);
        }
      } else {
        const u64 v0 = s0[0].get(m), v1 = s1[0].get(m), x0 = has_c0 ? cs[ls] : 0;
#pragma unroll
        for (int o = 0; o < KO; ++o) {
          const u64 dv = dg[o * EB + t];
          u0[o].mac(v0, dv);
          u1[o].mac(v1, dv);
          if (has_c0) a0[o].mac(x0, dv);
        }
      }
    }
    __syncthreads();  // every thread is done with stage s (and abort_flag is settled)
    if (abort_flag) {
      if (t == 0) {
        atomicOr(T.kerr, kErrWaitTimeout);
        // copies still in flight land in this CTA's shared memory: wait for them (bounded)
#pragma unroll
        for (u32 k = 0; k < (u32)S; ++k)
          if (n_issued > k) mbar_wait_bounded(&full[k], ((n_issued - 1 - k) / S) & 1u);
      }
      __syncthreads();
      return;
    }
    if (issuer && r + S < r1) issue(r + S, s);
  }
  const u32 g = eb * EB + t;
#pragma unroll
  for (int rr = 0; rr < RPT * KO; ++rr) {
    const u32 rq = KO == 1 ? rg * RPT + rr : rg;  // KO > 1: rr is the output
    const u32 ro = KO == 1 ? rq : rq * KO + rr;   // index of the partial
    if (rq < p.B) {
      p.partial[dh_off(ro, chunk, p.chunks, 0, i, ell, log_n) + g] = u0[rr].get(m);
      p.partial[dh_off(ro, chunk, p.chunks, 1, i, ell, log_n) + g] = u1[rr].get(m);
      if (has_c0) p.partial[dh_off(ro, chunk, p.chunks, 2, i, ell, log_n) + g] = a0[rr].get(m);
    }
  }
}

// A launch error of the staged form, reported with its shape and the kernel's attributes.
void dh_bulk_launched(const void* k, int ell, int rpt, int ko, int eb, int stages, size_t smem, dim3 grid) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return;
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, k);
  cudaGetLastError();
  fail(TCKS_ERR_CUDA, "staged accumulation (level " + std::to_string(ell) + ", " + std::to_string(rpt) +
                          " requests per thread, " + std::to_string(ko) + " outputs, " + std::to_string(eb) +
                          " elements per CTA, " + std::to_string(stages) + " stages, grid " + std::to_string(grid.x) +
                          " x " + std::to_string(grid.y) + ", dynamic shared memory " + std::to_string(smem) + " of " +
                          std::to_string(fa.maxDynamicSharedSizeBytes) + " allowed, " + std::to_string(fa.numRegs) +
                          " registers): " + cudaGetErrorString(e));
}

template <int RPT, int KO, int EB, int S>
void launch_shape(const DevTables& T, u32 ell, const VecmatDhPlan& p, cudaStream_t st) {
  const u64 n = 1ull << T.log_n;
  const dim3 grid((u32)((n / EB) * (ell + 1) * ((p.B + RPT - 1) / RPT)), p.chunks);
  switch (ell) {
#define TCKS_DHB_CASE(E)                                                      \
  case E: {                                                                   \
    const auto k = k_vecmat_dh_acc_bulk<E, RPT, KO, EB, S>;                  \
    const size_t smem = (size_t)S * DhStage<E, RPT, KO, EB>::kBytes;         \
    ensure_smem((const void*)k, smem);                                        \
    k<<<grid, EB, smem, st>>>(T, p);                                          \
    dh_bulk_launched((const void*)k, E, RPT, KO, EB, S, smem, grid);          \
    return;                                                                   \
  }
    TCKS_DHB_CASE(1) TCKS_DHB_CASE(2) TCKS_DHB_CASE(3) TCKS_DHB_CASE(4)
    TCKS_DHB_CASE(5) TCKS_DHB_CASE(6) TCKS_DHB_CASE(7) TCKS_DHB_CASE(8)
#undef TCKS_DHB_CASE
    default:
      fail(TCKS_ERR_UNSUPPORTED, "the staged accumulation takes levels 1..8");
  }
}

// Elements per CTA and stages of each staged form (DevTables::dh_form 1..4).
template <int RPT, int KO>
void launch_form(const DevTables& T, u32 ell, const VecmatDhPlan& p, cudaStream_t st) {
  switch (T.dh_form) {
    case 2: launch_shape<RPT, KO, 256, 3>(T, ell, p, st); return;
    case 3: launch_shape<RPT, KO, 128, 3>(T, ell, p, st); return;
    case 4: launch_shape<RPT, KO, 128, 4>(T, ell, p, st); return;
    default: launch_shape<RPT, KO, 256, 2>(T, ell, p, st); return;  // 1
  }
}

}  // namespace

bool dh_bulk_applies(const DevTables& T, u32 ell, const VecmatDhPlan& p) {
  auto al = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  if (!T.narrow || T.dh_form == 0 || T.dh_form > 4 || ell < 1 || ell > 8 || T.log_n < 8 || !p.keys_aligned) return false;
  if (!al(p.digits) || (p.digits_b & 3) || !al(p.ct) || (p.ct_b & 1)) return false;
  if (p.diag && (!al(p.diag) || (p.diag_stride & 1) || (p.diag_set & 1))) return false;
  return true;
}

void launch_vecmat_dh_acc_bulk(const DevTables& T, u32 ell, const VecmatDhPlan& p, u32 rpt, cudaStream_t st) {
  if (dh_outs(p) == 4)
    launch_form<1, 4>(T, ell, p, st);
  else if (rpt == 1)
    launch_form<1, 1>(T, ell, p, st);
  else
    launch_form<2, 1>(T, ell, p, st);
}

}  // namespace tcks

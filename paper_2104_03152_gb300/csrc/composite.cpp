// Composite operations of TenSEAL's CKKSVector (§3.1 dot product / vector x plain matrix, §3.2
// im2col convolution) as schedules of the library's kernels.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

using namespace tcks;

namespace tcks {

// ct <- ct + rot(ct, step), on device buffers at level ell.
static void rotate_add(tcks_ctx* c, u64* ct, u32 ell, int32_t step, u64* tmp) {
  op_rotate_hoisted(c, ct, ell, &step, 1, &tmp);
  launch_elementwise(c->T, OP_ADD, ct, tmp, ct, ell, 2, c->stream);
  check_launch("rotate-add");
}

static int ilog2(u64 x) {
  int r = 0;
  while ((1ull << r) < x) ++r;
  return r;
}

void op_sum(tcks_ctx* c, u64* ct, u32 ell) {
  DevBuf tmp(c, ct_words(c, ell));
  for (u32 m = 0; m + 1 < c->params.log_n; ++m) rotate_add(c, ct, ell, (int32_t)(1u << m), tmp.p);
}

// y = v M by the diagonal method with a replicated input (O21 of the hot-path reading).
void op_vecmat(tcks_ctx* c, const u64* ct_in, u32 ell, const tcks_matrix* M, u64* out) {
  const size_t n = c->N;
  const u32 rows = M->rows;
  const u32 slots = c->N / 2;
  // validate keys first
  std::vector<int32_t> rep;
  for (u32 m = 0; ((u64)rows << m) < slots; ++m) rep.push_back((int32_t)(slots - (rows << m)));
  for (int32_t s : rep) galois_key_for(c, s, ell);
  for (u32 k = 1; k < rows; ++k) galois_key_for(c, (int32_t)k, ell);
  DevBuf ct(c, ct_words(c, ell));
  check_cuda(cudaMemcpyAsync(ct.p, ct_in, ct_words(c, ell) * 8, cudaMemcpyDeviceToDevice, c->stream), "vecmat copy");
  {
    DevBuf tmp(c, ct_words(c, ell));
    for (int32_t s : rep) rotate_add(c, ct.p, ell, s, tmp.p);
  }
  const u64 diag_stride = (u64)M->level * n;
  DevBuf acc(c, ct_words(c, ell));
  launch_elementwise(c->T, OP_MUL_PLAIN, ct.p, M->d, acc.p, ell, 2, c->stream);  // k = 0
  // hoisted rotations k = 1..rows-1, KS_BATCH_MAX per launch, each chunk multiply-accumulated
  DevBuf coef(c, (size_t)ell * n), digits(c, (size_t)ell * (ell + 1) * n);
  launch_modup(c->T, ct.p + (size_t)ell * n, ell, coef.p, digits.p, c->stream);
  const u32 chunk = KS_BATCH_MAX;
  DevBuf rots(c, (size_t)chunk * ct_words(c, ell)), top(c, (size_t)chunk * 2 * n);
  for (u32 k0 = 1; k0 < rows; k0 += chunk) {
    const u32 cnt = (rows - k0) < chunk ? (rows - k0) : chunk;
    KsBatch b{};
    b.count = cnt;
    for (u32 t = 0; t < cnt; ++t) {
      const u32 k = k0 + t;
      const GaloisKey& gk = galois_key_for(c, (int32_t)k, ell);
      b.job[t] = KsJob{digits.p,
                       gk.d,
                       rots.p + (size_t)t * ct_words(c, ell),
                       top.p + (size_t)t * 2 * n,
                       ct.p,
                       nullptr,
                       gk.K,
                       (u32)galois_element(c->params.log_n, k),
                       1u,
                       0u};
    }
    launch_keyswitch(c->T, ell, b, c->stream);
    launch_mulacc(c->T, acc.p, rots.p, ct_words(c, ell), M->d + (size_t)k0 * diag_stride, diag_stride, cnt, ell,
                  c->stream);
    check_launch("vecmat chunk");
  }
  op_rescale(c, acc.p, ell, out);
}

// One im2col convolution kernel (§3.2): rescale(ct * kernel), then rotate-and-add by windows*2^i.
void op_conv(tcks_ctx* c, const u64* ct, u32 ell, const u64* kernel_pt, u32 taps, u32 windows, u64* out) {
  const int steps = ilog2(taps);
  for (int m = 0; m < steps; ++m) galois_key_for(c, (int32_t)(windows << m), ell - 1);
  DevBuf prod(c, ct_words(c, ell));
  launch_elementwise(c->T, OP_MUL_PLAIN, ct, kernel_pt, prod.p, ell, 2, c->stream);
  op_rescale(c, prod.p, ell, out);
  DevBuf tmp(c, ct_words(c, ell - 1));
  for (int m = 0; m < steps; ++m) rotate_add(c, out, ell - 1, (int32_t)(windows << m), tmp.p);
}

}  // namespace tcks

// The encrypted MNIST-shaped CNN of the paper's evaluation (§5, Table 2): conv (4 kernels 7x7,
// stride 3, im2col, §3.2) -> square -> FC 256->64 (§3.1) -> square -> FC 64->10, six multiplicative
// levels, on one CKKSVector.
//
// Schedule (levels in brackets, L = input level):
//   conv: per kernel k, rescale(ct * kernel_k) [L-1], then log2(taps) left rotate-and-adds by
//         windows * 2^i — the four channels rotate together, one key-switch launch per step;
//         (TCKS_CONV_HOIST) the sum as a baby-step and a giant-step hoisted rotation sum;
//         (TCKS_CONV_SHARED) the baby steps as a diagonal-method sum over the input's own rotations,
//         sum_b rot(ct, W b) * rot(kernel_k, W b), one ModUp per request for all kernels and one
//         ModDown per kernel, rescaled [L-1], then the giant steps;
//         (TCKS_CONV_PACK) after the baby steps the channels are masked to the windows-blocks k + B g
//         and packed [L-2], then one giant-step sum per request gathers block k's full tap sum; the
//         packed vector repeats every B blocks, so FC1 replicates it from that period;
//         (TCKS_CONV_FOLD) the masks folded into the shared baby-step diagonals, sum_k mask_k * rot(
//         kernel_k, W b): one diagonal-method sum per request gives the packed vector [L-1] (one ModUp,
//         one ModDown, no pack), and a modulus switch drops the limb the pack's rescale would have
//         dropped [L-2], so every later level is the same;
//   pack: v = sum_k rescale(conv_k * mask_k) [L-2], mask_k = 1 on slots [k*W, (k+1)*W); + conv bias;
//   square: rescale(relin(v * v)) [L-3];
//   FC1: vector x plain matrix (replicate, hoisted diagonal method, rescale) [L-4]; + bias;
//   square [L-5]; FC2 [L-6]; + bias. Logits sit in slots [0, classes).
// Biases are encoded once, at the scales the schedule reaches from an input at the context scale
// (the same double operations the forward pass performs), so the forward pass needs no encoding.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

using namespace tcks;

struct tcks_cnn {
  tcks_ctx* ctx;
  u32 kernels, taps, windows, hidden, classes;
  u32 L;                     // input level
  double in_scale;           // expected input scale
  std::vector<u64*> conv;    // per kernel, [L][N]
  std::vector<u64*> masks;   // per kernel, [L-1][N]
  u64* bias[3];              // [L-2], [L-4], [L-6]
  double bias_scale[3];
  tcks_matrix* fc1;          // level L-3
  tcks_matrix* fc2;          // level L-5
  double out_scale;
  bool rect;                 // rectangular FC layers: FC1's output comes replicated and feeds FC2 as is
  bool conv_hoist;           // the convolution sums as two hoisted rotation sums (baby and giant steps)
  bool conv_shared;          // baby steps on the input's own rotations, shared by every kernel
  bool pack_first;           // channels packed after the baby steps, one giant-step sum per request
  u32 period = 0;            // pack_first: the packed vector repeats every B windows (0 otherwise)
  std::vector<int32_t> baby, giant;
  u64* baby_ext = nullptr;   // conv_shared: per kernel k and baby step b (0 first), the kernel rotated
                             // left by windows * b over the extended basis, [kernels][B][L+1][N]
  bool fold = false;         // the masks folded into the baby-step diagonals (one sum, no pack)
  u64* fold_ext = nullptr;   // fold: per baby step b, sum_k mask_k * (kernel k rotated left by windows * b)
                             // over the extended basis, [B][L+1][N]
  int* h_wire_status = nullptr;  // pinned host word: the residue check of tcks_cnn_forward_wire's inputs
};

namespace tcks {

int ceil_log2(u32 x) {
  int r = 0;
  while ((1u << r) < x) ++r;
  return r;
}

// Scale after each stage, from the input scale (identical double operations to the forward pass).
static void schedule_scales(const tcks_cnn* m, double s_in, double delta, double* s_pack, double* s_fc1,
                            double* s_fc2) {
  const std::vector<u64>& q = m->ctx->host.chain;
  const u32 L = m->L;
  double s = s_in * delta / (double)q[L - 1];  // conv: mul_plain + rescale
  if (!m->fold) s = s * delta / (double)q[L - 2];  // pack: mul_plain(mask) + rescale (folded: a modulus switch)
  *s_pack = s;
  s = s * s / (double)q[L - 3];                 // square
  s = s * m->fc1->scale / (double)q[L - 4];     // FC1
  *s_fc1 = s;
  s = s * s / (double)q[L - 5];                 // square
  s = s * m->fc2->scale / (double)q[L - 6];     // FC2
  *s_fc2 = s;
}

u64 cnn_resident_bytes(const tcks_cnn* m) {
  const tcks_ctx* c = m->ctx;
  const u64 n = c->N, L = m->L;
  u64 b = (u64)m->kernels * (L + (L - 1)) * n * 8;          // conv kernels and masks
  if (m->baby_ext) b += (u64)m->kernels * (m->baby.size() + 1) * (L + 1) * n * 8;
  if (m->fold_ext) b += (u64)(m->baby.size() + 1) * (L + 1) * n * 8;
  b += ((L - 2) + (L - 4) + (L - 6)) * n * 8;                  // biases
  b += (u64)m->fc1->diags * m->fc1->limbs() * n * 8 + (u64)m->fc2->diags * m->fc2->limbs() * n * 8;
  return b;
}

tcks_ctx* cnn_context(const tcks_cnn* m) { return m->ctx; }

// Scale after stage `stage` for an input scale s (the double operations of the forward pass).
double cnn_out_scale(const tcks_cnn* m, u32 stage, double s) {
  const std::vector<u64>& q = m->ctx->host.chain;
  const u32 L = m->L;
  const double delta = m->ctx->params.scale;
  switch (stage) {
    case 0:
      s = s * delta / (double)q[L - 1];
      return m->fold ? s : s * delta / (double)q[L - 2];  // folded masks: no pack, a modulus switch
    case 1: return s * s / (double)q[L - 3];
    case 2: return s * m->fc1->scale / (double)q[L - 4];
    case 3: return s * s / (double)q[L - 5];
    default: return s * m->fc2->scale / (double)q[L - 6];
  }
}

// Stages of the schedule, each on a contiguous batch [count][2][level][N]:
//   0: conv + pack + conv bias   (L   -> L-2)
//   1: square                    (L-2 -> L-3)
//   2: FC1 + bias                (L-3 -> L-4)
//   3: square                    (L-4 -> L-5)
//   4: FC2 + bias                (L-5 -> L-6)
// Every stage runs once for the whole batch: the 4 * count channel ciphertexts rotate together, the
// relinearizations and rescales take the batch in one launch each, and the vector x matrix products
// process every request's rotations in shared launches.
u32 cnn_stage_level(const tcks_cnn* m, u32 stage) {  // input level of a stage (stage 5 = output)
  static const u32 drop[6] = {0, 2, 3, 4, 5, 6};
  return m->L - drop[stage];
}

static void square_stage(tcks_ctx* c, const u64* in, u32 ell, u32 count, u64* out) {
  const size_t n = c->N;
  DevBuf d3(c, (size_t)count * 3 * ell * n);
  launch_tensor(c->T, in, in, d3.p, ell, count, c->stream);
  if (c->flags & TCKS_MERGED_RESCALE) {
    op_relin_rescale(c, d3.p, ell, out, count);
    return;
  }
  DevBuf rel(c, (size_t)count * ct_words(c, ell));
  op_relinearize(c, d3.p, ell, rel.p, count);
  op_rescale(c, rel.p, ell, out, count);
}

void cnn_stage(const tcks_cnn* m, u32 stage, const u64* x, u32 count, u64* out) {
  tcks_ctx* c = m->ctx;
  const u32 L = m->L, K = m->kernels;
  switch (stage) {
    case 0: {
      const u64 w_in = ct_words(c, L), w1 = ct_words(c, L - 1), w2 = ct_words(c, L - 2);
      if (m->fold) {  // one sum over the folded diagonals is the packed vector [L-1]
        const u32 nb = (u32)m->baby.size() + 1;
        const u64 dstride = (u64)(L + 1) * c->N;
        if (c->flags & TCKS_MERGED_RESCALE) {
          // the ModDown, the rescale and the modulus switch [L-2] in one pass: the limb the switch
          // drops is never formed
          op_dh_sum_multi(c, x, w_in, count, L, m->baby, m->fold_ext, dstride, dstride * nb, L, 1, out, w2,
                          (u64)count * w2, true, L - 2);
        } else {
          DevBuf z(c, (size_t)count * w1), zz(c, (size_t)count * w_in);
          op_dh_sum_multi(c, x, w_in, count, L, m->baby, m->fold_ext, dstride, dstride * nb, L, 1, zz.p, w_in,
                          (u64)count * w_in);
          op_rescale(c, zz.p, L, z.p, count);
          // modulus switch [L-2]: each polynomial keeps its first L-2 limbs
          const size_t limb = (size_t)c->N * 8;
          check_cuda(cudaMemcpy2DAsync(out, (L - 2) * limb, z.p, (L - 1) * limb, (L - 2) * limb, 2 * (size_t)count,
                                       cudaMemcpyDeviceToDevice, c->stream),
                     "modulus switch");
        }
        op_rotsum_hoisted(c, out, w2, count, L - 2, m->giant, out, m->bias[0]);  // + bias in the ModDown
        break;
      }
      // conv [L-1]: channel k of request r at chans + (k * count + r) * w1
      DevBuf chans(c, (size_t)K * count * w1);
      if (m->conv_shared) {
        const u32 nb = (u32)m->baby.size() + 1;
        const u64 dstride = (u64)(L + 1) * c->N;
        if (c->flags & TCKS_MERGED_RESCALE) {  // ModDown and rescale in one rounding, straight into chans
          op_dh_sum_multi(c, x, w_in, count, L, m->baby, m->baby_ext, dstride, dstride * nb, L, K, chans.p, w1,
                          (u64)count * w1, true);
        } else {
          DevBuf z(c, (size_t)K * count * w_in);  // [kernel][request][2][L][N] before the rescale
          op_dh_sum_multi(c, x, w_in, count, L, m->baby, m->baby_ext, dstride, dstride * nb, L, K, z.p, w_in,
                          (u64)count * w_in);
          op_rescale(c, z.p, L, chans.p, K * count);
        }
        if (!m->pack_first) op_rotsum_hoisted(c, chans.p, w1, K * count, L - 1, m->giant, chans.p);
      } else {
        {
          DevBuf prod(c, (size_t)count * w_in);
          for (u32 k = 0; k < K; ++k) {
            launch_elementwise(c->T, OP_MUL_PLAIN, x, m->conv[k], prod.p, L, 2 * count, c->stream);
            op_rescale(c, prod.p, L, chans.p + (size_t)k * count * w1, count);
          }
        }
        if (m->conv_hoist) {
          op_rotsum_hoisted(c, chans.p, w1, K * count, L - 1, m->baby, chans.p);
          if (!m->pack_first) op_rotsum_hoisted(c, chans.p, w1, K * count, L - 1, m->giant, chans.p);
        } else {
          const int rsteps = ceil_log2(m->taps);
          for (int i = 0; i < rsteps; ++i)
            op_rotate_add(c, chans.p, w1, K * count, L - 1, (int32_t)(m->windows << i));
        }
      }
      // pack [L-2] + bias
      if ((c->flags & TCKS_MERGED_RESCALE) && K <= kLincombMax) {
        // the masked channels summed before one rescale (one rounding instead of K)
        MulSumArgs a{};
        a.x = chans.p;
        a.x_stride = (u64)count * w1;
        for (u32 k = 0; k < K; ++k) a.m[k] = m->masks[k];
        a.terms = K;
        a.ell = L - 1;
        a.count = count;
        DevBuf packed(c, (size_t)count * w1);
        launch_mulsum(c->T, a, packed.p, c->stream);
        op_rescale(c, packed.p, L - 1, out, count);
      } else {
        DevBuf prod(c, (size_t)count * w1), t(c, (size_t)count * w2);
        for (u32 k = 0; k < K; ++k) {
          launch_elementwise(c->T, OP_MUL_PLAIN, chans.p + (size_t)k * count * w1, m->masks[k], prod.p, L - 1,
                             2 * count, c->stream);
          op_rescale(c, prod.p, L - 1, k == 0 ? out : t.p, count);
          if (k) launch_elementwise(c->T, OP_ADD, out, t.p, out, L - 2, 2 * count, c->stream);
        }
      }
      if (m->pack_first)
        op_rotsum_hoisted(c, out, w2, count, L - 2, m->giant, out, m->bias[0]);
      else
        launch_elementwise(c->T, OP_ADD_PLAIN, out, m->bias[0], out, L - 2, 2 * count, c->stream);
      break;
    }
    case 1:
      square_stage(c, x, L - 2, count, out);
      break;
    case 2:
      op_vecmat(c, x, ct_words(c, L - 3), count, L - 3, m->fc1, out, m->period, m->bias[1]);
      break;
    case 3:
      square_stage(c, x, L - 4, count, out);
      break;
    case 4:
      op_vecmat(c, x, ct_words(c, L - 5), count, L - 5, m->fc2, out, m->rect ? m->fc2->rows : 0, m->bias[2]);
      break;
    default:
      fail(TCKS_ERR_INVALID_ARG, "no such stage");
  }
  check_launch("cnn stage");
}

// Forward pass of `count` requests at once: inputs in + r * in_stride ([2][L][N] each), outputs
// out [count][2][L-6][N].
u32 cnn_input_level(const tcks_cnn* m) { return m->L; }

void cnn_forward_dev(const tcks_cnn* m, const u64* in, u64 in_stride, u32 count, u64* out) {
  tcks_ctx* c = m->ctx;
  const u64 w_in = ct_words(c, m->L);
  DevBuf xin;
  const u64* x = in;
  if (count > 1 && in_stride != w_in) {  // gather the inputs into one contiguous batch
    xin = DevBuf(c, (size_t)count * w_in);
    for (u32 r = 0; r < count; ++r)
      check_cuda(cudaMemcpyAsync(xin.p + r * w_in, in + r * in_stride, w_in * 8, cudaMemcpyDeviceToDevice, c->stream),
                 "gather");
    x = xin.p;
  }
  DevBuf cur;
  for (u32 st = 0; st < 5; ++st) {
    if (st == 4) {
      cnn_stage(m, st, x, count, out);
      break;
    }
    DevBuf next(c, (size_t)count * ct_words(c, cnn_stage_level(m, st + 1)));
    cnn_stage(m, st, x, count, next.p);
    cur = std::move(next);
    x = cur.p;
  }
}

}  // namespace tcks

#define CNN_BEGIN \
  try {                 \
    tcks::NvtxRange tcks_nvtx_range_(__func__); \
    tcks::drop_stale_cuda_error();
#define CNN_END                                                       \
  }                                                                   \
  catch (const tcks::Error& e) {                                      \
    return tcks::abi_record(e.code, e.msg);                           \
  }                                                                   \
  catch (const std::bad_alloc&) {                                     \
    return tcks::abi_record(TCKS_ERR_OUT_OF_MEMORY, "host allocation failed"); \
  }                                                                   \
  tcks::abi_clear();                                                  \
  return TCKS_OK;

extern "C" {

void tcks_cnn_free(tcks_cnn* m) {
  if (!m) return;
  tcks_ctx* c = m->ctx;
  for (u64* p : m->conv) c->dev_free(p);
  for (u64* p : m->masks) c->dev_free(p);
  for (u64* p : m->bias) c->dev_free(p);
  if (m->baby_ext) c->dev_free(m->baby_ext);
  if (m->fold_ext) c->dev_free(m->fold_ext);
  if (m->h_wire_status) cudaFreeHost(m->h_wire_status);
  tcks_matrix_free(m->fc1);
  tcks_matrix_free(m->fc2);
  delete m;
  ctx_release(c);
}

tcks_status tcks_cnn_create(tcks_ctx* c, const double* conv_w, const double* conv_b, uint32_t kernels, uint32_t taps,
                            uint32_t windows, const double* fc1_w, const double* fc1_b, uint32_t hidden,
                            const double* fc2_w, const double* fc2_b, uint32_t classes, tcks_cnn** out) {
  struct Guard {  // frees a partly built model when creation fails
    tcks_cnn* m = nullptr;
    ~Guard() { tcks_cnn_free(m); }
  } guard;
  tcks_cnn*& m = guard.m;
  CNN_BEGIN
  if (!c || !conv_w || !conv_b || !fc1_w || !fc1_b || !fc2_w || !fc2_b || !out)
    fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  const u32 slots = c->N / 2, L = c->L;
  need_one_prime_ks(c, "the encrypted network");
  if (L < 7) fail(TCKS_ERR_BAD_PARAMS, "the network needs at least 7 data primes (6 levels + 1)");
  if (!kernels || !taps || !windows || (u64)taps * windows > slots || (u64)kernels * windows > slots)
    fail(TCKS_ERR_INVALID_ARG, "bad conv geometry");
  const u32 n1 = kernels * windows;
  if ((n1 & (n1 - 1)) || (hidden & (hidden - 1)) || hidden > n1 || classes > hidden || slots % n1)
    fail(TCKS_ERR_INVALID_ARG, "FC sizes must be powers of two with classes <= hidden <= kernels*windows");
  m = new tcks_cnn();
  m->ctx = c;
  ctx_retain(c);
  check_cuda(cudaHostAlloc((void**)&m->h_wire_status, sizeof(int), cudaHostAllocDefault), "pinned status word");
  m->kernels = kernels;
  m->taps = taps;
  m->windows = windows;
  m->hidden = hidden;
  m->classes = classes;
  m->L = L;
  m->in_scale = c->params.scale;
  m->rect = (c->flags & TCKS_RECT_DIAG) != 0;
  m->conv_shared = (c->flags & TCKS_CONV_SHARED) != 0;
  m->pack_first = (c->flags & TCKS_CONV_PACK) != 0;
  m->conv_hoist = m->conv_shared || m->pack_first || (c->flags & TCKS_CONV_HOIST) != 0;
  m->fold = (c->flags & TCKS_CONV_FOLD) != 0;
  if (m->fold && !(m->conv_shared && m->pack_first))
    fail(TCKS_ERR_UNSUPPORTED, "folding the masks needs TCKS_CONV_SHARED and TCKS_CONV_PACK");
  if (m->conv_shared && kernels != 4 && kernels != 1)
    fail(TCKS_ERR_UNSUPPORTED, "the shared convolution sum takes 1 or 4 kernels");
  {
    // tap positions t = b + B g over 2^ceil(log2 taps): B = 2^floor(e/2) baby steps, G = 2^ceil(e/2)
    const int e = ceil_log2(taps);
    const u32 nb = 1u << (e / 2), ng = 1u << (e - e / 2);
    for (u32 b = 1; b < nb; ++b) m->baby.push_back((int32_t)(windows * b));
    for (u32 g = 1; g < ng; ++g) m->giant.push_back((int32_t)(windows * nb * g));
    if (m->pack_first) {
      // block k of the giant-step sum gathers the blocks k + B g: kernels <= B, and the 2^e tap
      // positions must wrap around the whole slot vector (as the tap sums themselves do)
      if (kernels > nb || (u64)nb * ng * windows != slots)
        fail(TCKS_ERR_UNSUPPORTED, "packing before the giant steps needs kernels <= B and 2^e windows == N/2");
      m->period = nb * windows;
    }
  }
  m->bias[0] = m->bias[1] = m->bias[2] = nullptr;
  m->fc1 = m->fc2 = nullptr;
  const double delta = c->params.scale;
  std::vector<double> lay(slots);
  DevBuf dv(c, slots);
  auto encode_host = [&](const std::vector<double>& v, double scale, u32 level) -> u64* {
    DevBuf p(c, (size_t)level * c->N);
    check_cuda(cudaMemcpyAsync(dv.p, v.data(), (size_t)slots * 8, cudaMemcpyHostToDevice, c->stream), "H2D");
    encode_into(c, (const double*)dv.p, slots, scale, level, p.p);
    return p.release();
  };
  std::vector<std::vector<double>> kern_lay, mask_lay;  // slot layouts, kept for the folded diagonals
  for (u32 k = 0; k < kernels; ++k) {
    std::fill(lay.begin(), lay.end(), 0.0);
    for (u32 t = 0; t < taps; ++t)
      for (u32 w = 0; w < windows; ++w) lay[(size_t)t * windows + w] = conv_w[(size_t)k * taps + t];
    if (m->fold) kern_lay.push_back(lay);
    m->conv.push_back(encode_host(lay, delta, L));
    if (m->conv_shared) {
      const u32 nb = (u32)m->baby.size() + 1;
      const u64 per = (u64)(L + 1) * c->N;
      if (!m->baby_ext) m->baby_ext = (u64*)c->dev_alloc((size_t)kernels * nb * per * 8);
      std::vector<double> rot(slots);
      for (u32 b = 0; b < nb; ++b) {
        const u32 sh = b ? (u32)m->baby[b - 1] : 0;  // left rotation by sh: rot[i] = lay[i + sh]
        for (u32 i = 0; i < slots; ++i) rot[i] = lay[(i + sh) % slots];
        check_cuda(cudaMemcpyAsync(dv.p, rot.data(), (size_t)slots * 8, cudaMemcpyHostToDevice, c->stream), "H2D");
        encode_into(c, (const double*)dv.p, slots, delta, L, m->baby_ext + ((u64)k * nb + b) * per, true);
      }
    }
    std::fill(lay.begin(), lay.end(), 0.0);
    if (m->pack_first) {  // the windows-blocks k + B g
      for (u32 i = 0; i < slots; ++i) lay[i] = (i / windows) % (m->period / windows) == k ? 1.0 : 0.0;
    } else {
      for (u32 w = 0; w < windows; ++w) lay[(size_t)k * windows + w] = 1.0;
    }
    m->masks.push_back(encode_host(lay, delta, L - 1));
    if (m->fold) mask_lay.push_back(lay);
  }
  if (m->fold) {  // reading A27: sum_k mask_k * rot(kernel_k, W b), slot by slot
    const u32 nb = (u32)m->baby.size() + 1;
    const u64 per = (u64)(L + 1) * c->N;
    m->fold_ext = (u64*)c->dev_alloc((size_t)nb * per * 8);
    std::vector<double> f(slots);
    for (u32 b = 0; b < nb; ++b) {
      const u32 sh = b ? (u32)m->baby[b - 1] : 0;
      for (u32 i = 0; i < slots; ++i) {
        double v = 0.0;
        for (u32 k = 0; k < kernels; ++k) v += mask_lay[k][i] * kern_lay[k][(i + sh) % slots];
        f[i] = v;
      }
      check_cuda(cudaMemcpyAsync(dv.p, f.data(), (size_t)slots * 8, cudaMemcpyHostToDevice, c->stream), "H2D");
      encode_into(c, (const double*)dv.p, slots, delta, L, m->fold_ext + (u64)b * per, true);
    }
  }
  // FC weights W [out][in] act as M = W^T [in][out]
  std::vector<double> M1((size_t)n1 * hidden), M2((size_t)hidden * classes);
  for (u32 i = 0; i < n1; ++i)
    for (u32 o = 0; o < hidden; ++o) M1[(size_t)i * hidden + o] = fc1_w[(size_t)o * n1 + i];
  for (u32 i = 0; i < hidden; ++i)
    for (u32 o = 0; o < classes; ++o) M2[(size_t)i * classes + o] = fc2_w[(size_t)o * hidden + i];
  auto enc_m = m->rect ? tcks_matrix_encode_rect : tcks_matrix_encode;
  tcks_status st = enc_m(c, M1.data(), n1, hidden, L - 3, &m->fc1);
  if (st != TCKS_OK) fail(st, tcks_last_error_detail());
  st = enc_m(c, M2.data(), hidden, classes, L - 5, &m->fc2);
  if (st != TCKS_OK) fail(st, tcks_last_error_detail());
  double s_pack, s_fc1, s_fc2;
  schedule_scales(m, m->in_scale, delta, &s_pack, &s_fc1, &s_fc2);
  m->bias_scale[0] = s_pack;
  m->bias_scale[1] = s_fc1;
  m->bias_scale[2] = s_fc2;
  m->out_scale = s_fc2;
  std::fill(lay.begin(), lay.end(), 0.0);
  for (u32 r = 0; r < (m->period ? slots / m->period : 1); ++r)  // the packed layout's period
    for (u32 k = 0; k < kernels; ++k)
      for (u32 w = 0; w < windows; ++w) lay[(size_t)r * m->period + (size_t)k * windows + w] = conv_b[k];
  m->bias[0] = encode_host(lay, s_pack, L - 2);
  // rectangular layers leave their outputs replicated with period m' (hidden, then the power of two
  // above classes): the biases are laid out the same way
  const u32 p1 = m->rect ? m->fc1->diags : slots, p2 = m->rect ? m->fc2->diags : slots;
  std::fill(lay.begin(), lay.end(), 0.0);
  for (u32 t = 0; t < slots; ++t) lay[t] = t % p1 < hidden && t < (m->rect ? slots : hidden) ? fc1_b[t % p1] : 0.0;
  m->bias[1] = encode_host(lay, s_fc1, L - 4);
  std::fill(lay.begin(), lay.end(), 0.0);
  for (u32 t = 0; t < slots; ++t) lay[t] = t % p2 < classes && t < (m->rect ? slots : classes) ? fc2_b[t % p2] : 0.0;
  m->bias[2] = encode_host(lay, s_fc2, L - 6);
  *out = m;
  m = nullptr;
  CNN_END
}

// Galois steps the forward pass needs, with the level each must reach (for key trimming):
// writes up to `cap` (step, level) pairs and the count.
tcks_status tcks_cnn_galois_steps(const tcks_cnn* m, int32_t* steps, uint32_t* levels, uint32_t cap,
                                  uint32_t* count) {
  CNN_BEGIN
  if (!m || !count) fail(TCKS_ERR_INVALID_ARG, "null argument");
  const u32 slots = m->ctx->N / 2, L = m->L;
  std::vector<std::pair<u32, u32>> need;  // (step, level)
  auto use = [&](u32 s, u32 lv) {
    s %= slots;
    if (!s) return;
    for (auto& p : need)
      if (p.first == s) {
        if (lv > p.second) p.second = lv;
        return;
      }
    need.push_back({s, lv});
  };
  if (m->conv_hoist) {  // shared: the baby steps rotate the input, at level L; packed first: giant at L-2
    for (int32_t s : m->baby) use((u32)s, m->conv_shared ? L : L - 1);
    for (int32_t s : m->giant) use((u32)s, m->pack_first ? L - 2 : L - 1);
  } else {
    for (int i = 0; i < ceil_log2(m->taps); ++i) use(m->windows << i, L - 1);
  }
  const u32 n1 = m->kernels * m->windows, n2 = m->hidden;
  for (u32 r = 0; ((u64)n1 << r) < (m->period ? m->period : slots); ++r) use(slots - (n1 << r), L - 3);
  if (m->rect) {  // m' - 1 rotations, then the rotate-and-add chain after the rescale; FC2 unreplicated
    for (u32 k = 1; k < m->fc1->diags; ++k) use(k, L - 3);
    for (u32 w = m->fc1->diags; w < n1; w <<= 1) use(w, L - 4);
    for (u32 k = 1; k < m->fc2->diags; ++k) use(k, L - 5);
    for (u32 w = m->fc2->diags; w < n2; w <<= 1) use(w, L - 6);
  } else {
    for (u32 k = 1; k < n1; ++k) use(k, L - 3);
    for (u32 r = 0; ((u64)n2 << r) < slots; ++r) use(slots - (n2 << r), L - 5);
    for (u32 k = 1; k < n2; ++k) use(k, L - 5);
  }
  *count = (u32)need.size();
  if (steps && levels) {
    if (cap < need.size()) fail(TCKS_ERR_INVALID_ARG, "capacity too small");
    for (size_t i = 0; i < need.size(); ++i) {
      steps[i] = (int32_t)need[i].first;
      levels[i] = need[i].second;
    }
  }
  CNN_END
}

tcks_status tcks_cnn_forward(const tcks_cnn* m, const tcks_ct* in, tcks_ct** out) {
  CNN_BEGIN
  if (!m || !in || !out) fail(TCKS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  tcks_ctx* c = m->ctx;
  if (in->ctx != c) fail(TCKS_ERR_INVALID_ARG, "ciphertext belongs to another context");
  need_relinearized(in);
  if (in->level != m->L) fail(TCKS_ERR_LEVEL_MISMATCH, "the network takes a ciphertext at the top level");
  if (in->scale != m->in_scale) fail(TCKS_ERR_SCALE_MISMATCH, "the network takes a ciphertext at the context scale");
  tcks_ct* r = new_ct(c, m->L - 6, m->out_scale);
  try {
    cnn_forward_dev(m, in->d, 0, 1, r->d);
  } catch (...) {
    free_ct(r);
    throw;
  }
  *out = r;
  CNN_END
}

tcks_status tcks_cnn_forward_batch(const tcks_cnn* m, const tcks_ct* const* in, uint32_t count, tcks_ct** outs) {
  struct Made {  // outputs created so far, freed unless handed to the caller
    std::vector<tcks_ct*> v;
    ~Made() {
      for (tcks_ct* x : v) free_ct(x);
    }
  } owned;
  std::vector<tcks_ct*>& made = owned.v;
  CNN_BEGIN
  if (!m || !outs || (count && !in)) fail(TCKS_ERR_INVALID_ARG, "null argument");
  for (u32 i = 0; i < count; ++i) outs[i] = nullptr;
  if (!count) return TCKS_OK;
  tcks_ctx* c = m->ctx;
  for (u32 i = 0; i < count; ++i) {
    if (!in[i] || in[i]->ctx != c) fail(TCKS_ERR_INVALID_ARG, "ciphertext missing or of another context");
    need_relinearized(in[i]);
    if (in[i]->level != m->L) fail(TCKS_ERR_LEVEL_MISMATCH, "the network takes ciphertexts at the top level");
    if (in[i]->scale != m->in_scale) fail(TCKS_ERR_SCALE_MISMATCH, "the network takes ciphertexts at the context scale");
  }
  const u64 w_in = ct_words(c, m->L), w_out = ct_words(c, m->L - 6);
  DevBuf xin(c, (size_t)count * w_in), yout(c, (size_t)count * w_out);
  for (u32 i = 0; i < count; ++i)
    check_cuda(cudaMemcpyAsync(xin.p + i * w_in, in[i]->d, w_in * 8, cudaMemcpyDeviceToDevice, c->stream), "gather");
  cnn_forward_dev(m, xin.p, w_in, count, yout.p);
  for (u32 i = 0; i < count; ++i) {
    made.push_back(new_ct(c, m->L - 6, m->out_scale));
    check_cuda(cudaMemcpyAsync(made.back()->d, yout.p + i * w_out, w_out * 8, cudaMemcpyDeviceToDevice, c->stream),
               "scatter");
  }
  for (u32 i = 0; i < count; ++i) outs[i] = made[i];
  made.clear();
  CNN_END
}

tcks_status tcks_cnn_forward_device(const tcks_cnn* m, const uint64_t* d_in, uint32_t count, uint64_t* d_out) {
  CNN_BEGIN
  if (!m || (count && (!d_in || !d_out))) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (!count) return TCKS_OK;
  cnn_forward_dev(m, d_in, ct_words(m->ctx, m->L), count, d_out);
  CNN_END
}

tcks_status tcks_cnn_forward_host(const tcks_cnn* m, const uint64_t* host_in, uint32_t count, uint64_t* host_out) {
  CNN_BEGIN
  if (!m || (count && (!host_in || !host_out))) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (!count) return TCKS_OK;
  tcks_ctx* c = m->ctx;
  const u64 w_in = ct_words(c, m->L), w_out = ct_words(c, m->L - 6);
  DevBuf xin(c, (size_t)count * w_in), yout(c, (size_t)count * w_out);
  check_cuda(cudaMemcpyAsync(xin.p, host_in, (size_t)count * w_in * 8, cudaMemcpyHostToDevice, c->stream), "H2D");
  cnn_forward_dev(m, xin.p, w_in, count, yout.p);
  check_cuda(cudaMemcpyAsync(host_out, yout.p, (size_t)count * w_out * 8, cudaMemcpyDeviceToHost, c->stream), "D2H");
  check_cuda(cudaStreamSynchronize(c->stream), "forward");
  kernel_error_check(c);
  CNN_END
}

tcks_status tcks_cnn_wire_sizes(const tcks_cnn* m, uint64_t* in_full, uint64_t* in_seeded, uint64_t* out_size) {
  CNN_BEGIN
  if (!m || !in_full || !in_seeded || !out_size) fail(TCKS_ERR_INVALID_ARG, "null argument");
  tcks_ctx* c = m->ctx;
  const u64 pin = wire_payload_bytes(c->T, c->host.chain.data(), m->L);
  *in_full = kWireHeader + pin;
  *in_seeded = kWireHeader + 8 + pin / 2;
  *out_size = kWireHeader + wire_payload_bytes(c->T, c->host.chain.data(), m->L - 6);
  CNN_END
}

tcks_status tcks_cnn_forward_wire(const tcks_cnn* m, const uint8_t* host_in, uint64_t in_size, uint32_t count,
                                  uint8_t* host_out, uint64_t out_size) {
  CNN_BEGIN
  if (!m || (count && (!host_in || !host_out))) fail(TCKS_ERR_INVALID_ARG, "null argument");
  if (!count) return TCKS_OK;
  tcks_ctx* c = m->ctx;
  const u32 L = m->L, Lo = m->L - 6;
  const u64 pin = wire_payload_bytes(c->T, c->host.chain.data(), L);
  const u64 pout = wire_payload_bytes(c->T, c->host.chain.data(), Lo);
  const bool seeded = in_size == kWireHeader + 8 + pin / 2;
  if (!seeded && in_size != kWireHeader + pin) fail(TCKS_ERR_INVALID_ARG, "input size is not a serialized input");
  if (out_size != kWireHeader + pout) fail(TCKS_ERR_INVALID_ARG, "output size is not the serialized output");
  // headers on the host: every input of the announced kind, ring, level and scale
  std::vector<u64> seeds(seeded ? count : 0);
  for (u32 r = 0; r < count; ++r) {
    const uint8_t* h = host_in + (u64)r * in_size;
    double sc;
    std::memcpy(&sc, h + 8, 8);
    if (std::memcmp(h, kWireMagic, 4) != 0 || h[4] != 1 || h[5] != (seeded ? 1 : 0) || h[6] != c->params.log_n ||
        h[7] != L)
      fail(TCKS_ERR_INVALID_ARG, "an input header does not match the model's input");
    if (sc != m->in_scale) fail(TCKS_ERR_SCALE_MISMATCH, "the network takes ciphertexts at the context scale");
    if (seeded)
      for (int b = 0; b < 8; ++b) seeds[r] |= (u64)h[kWireHeader + b] << (8 * b);
  }
  const u64 w_in = ct_words(c, L), w_out = ct_words(c, Lo);
  DevBuf raw(c, ((u64)count * in_size + 7) / 8), xin(c, (size_t)count * w_in), yout(c, (size_t)count * w_out);
  DevBuf packed(c, ((u64)count * out_size + 7) / 8), dseeds(c, seeded ? count : 1);
  unsigned char* rb = (unsigned char*)raw.p;
  unsigned char* pb = (unsigned char*)packed.p;
  check_cuda(cudaMemcpyAsync(rb, host_in, (size_t)count * in_size, cudaMemcpyHostToDevice, c->stream), "H2D");
  if (seeded)
    check_cuda(cudaMemcpyAsync(dseeds.p, seeds.data(), (size_t)count * 8, cudaMemcpyHostToDevice, c->stream), "H2D");
  check_cuda(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream), "wire status");
  const u64 head = kWireHeader + (seeded ? 8 : 0);
  constexpr u32 kChunk = 16384;  // grid z = requests x components <= 65535
  for (u32 r0 = 0; r0 < count; r0 += kChunk) {
    const u32 k = std::min(kChunk, count - r0);
    launch_unpack_batch(c->T, rb + (u64)r0 * in_size + head, in_size, L, xin.p + (u64)r0 * w_in, w_in, k, c->d_status,
                        c->stream, seeded ? 1 : 2);
    if (seeded)
      launch_sym_a_batch(c->T, dseeds.p + r0, L, xin.p + (u64)r0 * w_in + (u64)L * c->N, w_in, k, c->stream);
  }
  check_launch("wire input");
  // The residue check's verdict travels to a pinned host word right behind the unpacking; the host
  // reads it while the network runs and only then lets the outputs reach host_out, so a refused batch
  // leaves the caller's buffer untouched.
  struct Event {
    cudaEvent_t e = nullptr;
    ~Event() {
      if (e) cudaEventDestroy(e);
    }
  } checked;
  check_cuda(cudaMemcpyAsync(m->h_wire_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
             "wire status");
  check_cuda(cudaEventCreateWithFlags(&checked.e, cudaEventDisableTiming), "event");
  check_cuda(cudaEventRecord(checked.e, c->stream), "event");
  cnn_forward_dev(m, xin.p, w_in, count, yout.p);
  for (u32 r0 = 0; r0 < count; r0 += kChunk) {
    const u32 k = std::min(kChunk, count - r0);
    launch_pack_batch(c->T, yout.p + (u64)r0 * w_out, w_out, Lo, pb + (u64)r0 * out_size + kWireHeader, out_size, k,
                      c->stream);
  }
  check_launch("wire output");
  check_cuda(cudaEventSynchronize(checked.e), "wire status");
  if (*m->h_wire_status) {
    check_cuda(cudaStreamSynchronize(c->stream), "forward");  // the scratch is released only after the network
    fail(TCKS_ERR_INVALID_ARG, "an input residue is not below its prime");
  }
  check_cuda(cudaMemcpyAsync(host_out, pb, (size_t)count * out_size, cudaMemcpyDeviceToHost, c->stream), "D2H");
  check_cuda(cudaStreamSynchronize(c->stream), "forward");
  kernel_error_check(c);
  for (u32 r = 0; r < count; ++r) {
    uint8_t* h = host_out + (u64)r * out_size;
    std::memcpy(h, kWireMagic, 4);
    h[4] = 1;
    h[5] = 0;
    h[6] = (uint8_t)c->params.log_n;
    h[7] = (uint8_t)Lo;
    std::memcpy(h + 8, &m->out_scale, 8);
  }
  CNN_END
}

// ------------------------------------------------------------- pipelined serialized batches ----
// Two slots of device buffers for batches of `count` serialized inputs of one size. A batch's input copy
// runs on the pipe's copy stream as soon as its slot is free, and its unpacking, network and packing on
// the model's stream after that copy; its output copy waits for the residue check on the host (in
// wait), so a refused batch never reaches its output buffer. With two batches in flight the next
// batch's input copy overlaps the current batch's network.
struct tcks_cnn_pipe {
  const tcks_cnn* m = nullptr;
  tcks_ctx* c = nullptr;  // retained
  u32 count = 0;
  u64 in_size = 0, out_size = 0;
  bool seeded = false;
  cudaStream_t copy = nullptr;
  struct Slot {
    unsigned char* raw = nullptr;  // [count][in_size]
    u64* seeds = nullptr;          // [count] (seeded inputs)
    u64* xin = nullptr;            // [count][2][L][N]
    u64* yout = nullptr;           // [count][2][L-6][N]
    unsigned char* packed = nullptr;  // [count][out_size]
    int* d_status = nullptr;
    int* h_status = nullptr;          // pinned
    u32* h_kerr = nullptr;            // pinned: the context's kernel error word after the batch
    u64* h_seeds = nullptr;           // pinned staging of the seeds
    cudaEvent_t in_copied = nullptr, checked = nullptr, packed_ev = nullptr, out_copied = nullptr, consumed = nullptr;
    uint8_t* host_out = nullptr;      // the batch in flight, or null
    u64 ticket = 0;
    bool used = false;                // out_copied has been recorded once
  } slot[2];
  u64 next = 1;  // ticket of the next submit
};

namespace {

void pipe_release(tcks_cnn_pipe* p) {
  if (!p) return;
  tcks_ctx* c = p->c;
  if (c) cudaStreamSynchronize(c->stream);
  if (p->copy) {
    cudaStreamSynchronize(p->copy);
    cudaStreamDestroy(p->copy);
  }
  for (auto& s : p->slot) {
    if (c) {
      c->dev_free(s.raw);
      c->dev_free(s.seeds);
      c->dev_free(s.xin);
      c->dev_free(s.yout);
      c->dev_free(s.packed);
      c->dev_free(s.d_status);
    }
    if (s.h_status) cudaFreeHost(s.h_status);
    if (s.h_kerr) cudaFreeHost(s.h_kerr);
    if (s.h_seeds) cudaFreeHost(s.h_seeds);
    for (cudaEvent_t e : {s.in_copied, s.checked, s.packed_ev, s.out_copied, s.consumed})
      if (e) cudaEventDestroy(e);
  }
  if (c) {
    cudaStreamSynchronize(c->stream);
    ctx_release(c);
  }
  delete p;
  cudaGetLastError();  // clean-up statuses are not reported
}

// Wait for slot s's batch: its residue check, then (if it passed) its output copy; the slot is free after.
void pipe_finish(tcks_cnn_pipe* p, tcks_cnn_pipe::Slot& s) {
  if (!s.host_out) return;
  tcks_ctx* c = p->c;
  uint8_t* host_out = s.host_out;
  s.host_out = nullptr;
  check_cuda(cudaEventSynchronize(s.checked), "pipe residue check");
  if (*s.h_status) {
    check_cuda(cudaEventSynchronize(s.packed_ev), "pipe");
    fail(TCKS_ERR_INVALID_ARG, "an input residue is not below its prime");
  }
  check_cuda(cudaStreamWaitEvent(p->copy, s.packed_ev, 0), "pipe");
  check_cuda(cudaMemcpyAsync(host_out, s.packed, (size_t)p->count * p->out_size, cudaMemcpyDeviceToHost, p->copy),
             "D2H");
  check_cuda(cudaEventRecord(s.out_copied, p->copy), "pipe");
  s.used = true;
  check_cuda(cudaEventSynchronize(s.out_copied), "pipe output");
  if (*s.h_kerr) {  // a kernel's bounded wait gave up (or refused a copy): the results are invalid
    check_cuda(cudaMemsetAsync(c->T.kerr, 0, sizeof(u32), c->stream), "kernel error word");
    fail((*s.h_kerr & 1u) ? TCKS_ERR_TIMEOUT : TCKS_ERR_CUDA, "a kernel of this batch recorded an error");
  }
  const u32 Lo = p->m->L - 6;
  for (u32 r = 0; r < p->count; ++r) {
    uint8_t* h = host_out + (u64)r * p->out_size;
    std::memcpy(h, kWireMagic, 4);
    h[4] = 1;
    h[5] = 0;
    h[6] = (uint8_t)c->params.log_n;
    h[7] = (uint8_t)Lo;
    std::memcpy(h + 8, &p->m->out_scale, 8);
  }
}

}  // namespace

extern "C" {

tcks_status tcks_cnn_pipe_create(const tcks_cnn* m, uint32_t count, uint64_t in_size, tcks_cnn_pipe** out) {
  struct Guard {
    tcks_cnn_pipe* p = nullptr;
    ~Guard() { pipe_release(p); }
  } guard;
  CNN_BEGIN
  if (!m || !out || !count) fail(TCKS_ERR_INVALID_ARG, "null argument or empty batch");
  *out = nullptr;
  tcks_ctx* c = m->ctx;
  const u32 L = m->L, Lo = m->L - 6;
  const u64 pin = wire_payload_bytes(c->T, c->host.chain.data(), L);
  const u64 pout = wire_payload_bytes(c->T, c->host.chain.data(), Lo);
  const bool seeded = in_size == kWireHeader + 8 + pin / 2;
  if (!seeded && in_size != kWireHeader + pin) fail(TCKS_ERR_INVALID_ARG, "input size is not a serialized input");
  guard.p = new tcks_cnn_pipe();
  tcks_cnn_pipe* p = guard.p;
  p->m = m;
  p->c = c;
  ctx_retain(c);
  p->count = count;
  p->in_size = in_size;
  p->out_size = kWireHeader + pout;
  p->seeded = seeded;
  check_cuda(cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking), "pipe copy stream");
  const u64 w_in = ct_words(c, L), w_out = ct_words(c, Lo);
  for (auto& s : p->slot) {
    s.raw = (unsigned char*)c->dev_alloc((size_t)count * in_size);
    s.seeds = (u64*)c->dev_alloc((size_t)count * 8);
    s.xin = (u64*)c->dev_alloc((size_t)count * w_in * 8);
    s.yout = (u64*)c->dev_alloc((size_t)count * w_out * 8);
    s.packed = (unsigned char*)c->dev_alloc((size_t)count * p->out_size);
    s.d_status = (int*)c->dev_alloc(sizeof(int));
    check_cuda(cudaHostAlloc((void**)&s.h_status, sizeof(int), cudaHostAllocDefault), "pinned status word");
    check_cuda(cudaHostAlloc((void**)&s.h_kerr, sizeof(u32), cudaHostAllocDefault), "pinned status word");
    check_cuda(cudaHostAlloc((void**)&s.h_seeds, (size_t)count * 8, cudaHostAllocDefault), "pinned seeds");
    for (cudaEvent_t* e : {&s.in_copied, &s.checked, &s.packed_ev, &s.out_copied, &s.consumed})
      check_cuda(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "pipe event");
  }
  // the buffers come from the model stream's pool: ready before the copy stream touches them
  check_cuda(cudaStreamSynchronize(c->stream), "pipe buffers");
  *out = p;
  guard.p = nullptr;
  CNN_END
}

tcks_status tcks_cnn_pipe_submit(tcks_cnn_pipe* p, const uint8_t* host_in, uint8_t* host_out, uint64_t* ticket) {
  CNN_BEGIN
  if (!p || !host_in || !host_out || !ticket) fail(TCKS_ERR_INVALID_ARG, "null argument");
  const tcks_cnn* m = p->m;
  tcks_ctx* c = p->c;
  const u32 L = m->L, Lo = m->L - 6, count = p->count;
  const u64 in_size = p->in_size;
  tcks_cnn_pipe::Slot& s = p->slot[p->next & 1];
  pipe_finish(p, s);  // the slot's previous batch (two submits ago) completes first
  for (u32 r = 0; r < count; ++r) {
    const uint8_t* h = host_in + (u64)r * in_size;
    double sc;
    std::memcpy(&sc, h + 8, 8);
    if (std::memcmp(h, kWireMagic, 4) != 0 || h[4] != 1 || h[5] != (p->seeded ? 1 : 0) || h[6] != c->params.log_n ||
        h[7] != L)
      fail(TCKS_ERR_INVALID_ARG, "an input header does not match the model's input");
    if (sc != m->in_scale) fail(TCKS_ERR_SCALE_MISMATCH, "the network takes ciphertexts at the context scale");
  }
  // the input copy may start once the slot's previous batch has been unpacked
  if (s.used) check_cuda(cudaStreamWaitEvent(p->copy, s.consumed, 0), "pipe");
  check_cuda(cudaMemcpyAsync(s.raw, host_in, (size_t)count * in_size, cudaMemcpyHostToDevice, p->copy), "H2D");
  if (p->seeded) {
    for (u32 r = 0; r < count; ++r) {
      u64 v = 0;
      for (int b = 0; b < 8; ++b) v |= (u64)host_in[(u64)r * in_size + kWireHeader + b] << (8 * b);
      s.h_seeds[r] = v;
    }
    check_cuda(cudaMemcpyAsync(s.seeds, s.h_seeds, (size_t)count * 8, cudaMemcpyHostToDevice, p->copy), "H2D");
  }
  check_cuda(cudaEventRecord(s.in_copied, p->copy), "pipe");
  // the model's stream: unpack after the copy, the network, then pack once the slot's last output copy is done
  const u64 w_in = ct_words(c, L), w_out = ct_words(c, Lo);
  check_cuda(cudaStreamWaitEvent(c->stream, s.in_copied, 0), "pipe");
  check_cuda(cudaMemsetAsync(s.d_status, 0, sizeof(int), c->stream), "pipe status");
  const u64 head = kWireHeader + (p->seeded ? 8 : 0);
  constexpr u32 kChunk = 16384;  // grid z = requests x components <= 65535
  for (u32 r0 = 0; r0 < count; r0 += kChunk) {
    const u32 k = std::min(kChunk, count - r0);
    launch_unpack_batch(c->T, s.raw + (u64)r0 * in_size + head, in_size, L, s.xin + (u64)r0 * w_in, w_in, k,
                        s.d_status, c->stream, p->seeded ? 1 : 2);
    if (p->seeded) launch_sym_a_batch(c->T, s.seeds + r0, L, s.xin + (u64)r0 * w_in + (u64)L * c->N, w_in, k, c->stream);
  }
  check_launch("pipe input");
  check_cuda(cudaEventRecord(s.consumed, c->stream), "pipe");
  check_cuda(cudaMemcpyAsync(s.h_status, s.d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "pipe status");
  check_cuda(cudaEventRecord(s.checked, c->stream), "pipe");
  cnn_forward_dev(m, s.xin, w_in, count, s.yout);
  if (s.used) check_cuda(cudaStreamWaitEvent(c->stream, s.out_copied, 0), "pipe");
  for (u32 r0 = 0; r0 < count; r0 += kChunk) {
    const u32 k = std::min(kChunk, count - r0);
    launch_pack_batch(c->T, s.yout + (u64)r0 * w_out, w_out, Lo, s.packed + (u64)r0 * p->out_size + kWireHeader,
                      p->out_size, k, c->stream);
  }
  check_launch("pipe output");
  check_cuda(cudaMemcpyAsync(s.h_kerr, c->T.kerr, sizeof(u32), cudaMemcpyDeviceToHost, c->stream), "pipe status");
  check_cuda(cudaEventRecord(s.packed_ev, c->stream), "pipe");
  s.host_out = host_out;
  s.ticket = p->next++;
  *ticket = s.ticket;
  CNN_END
}

tcks_status tcks_cnn_pipe_wait(tcks_cnn_pipe* p, uint64_t ticket) {
  CNN_BEGIN
  if (!p) fail(TCKS_ERR_INVALID_ARG, "null pipe");
  tcks_cnn_pipe::Slot& s = p->slot[ticket & 1];
  if (ticket == 0 || ticket >= p->next) fail(TCKS_ERR_INVALID_ARG, "unknown ticket");
  if (s.ticket != ticket) return TCKS_OK;  // completed and reported already (its slot holds a later batch)
  pipe_finish(p, s);
  CNN_END
}

void tcks_cnn_pipe_free(tcks_cnn_pipe* p) { pipe_release(p); }

}  // extern "C"

// -------------------------------------------------------------------------- CUDA graphs ----
struct tcks_cnn_graph {
  tcks_ctx* ctx;  // retained: the graph's buffers belong to it
  const tcks_cnn* m;
  u32 count;
  u64* in;   // staging [count][2][L][N]
  u64* out;  // staging [count][2][L-6][N]
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  u64 launches;  // kernel launches in one replay
  std::vector<std::pair<tcks_ctx*, char*>> blocks;  // the capture arena with a caller allocator
};

void tcks_cnn_graph_free(tcks_cnn_graph* g) {
  if (!g) return;
  tcks_ctx* c = g->ctx;
  cudaStreamSynchronize(c->stream);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (const auto& b : g->blocks) arena_release(b.first, b.second);
  c->dev_free(g->in);
  c->dev_free(g->out);
  delete g;
  ctx_release(c);
  cudaGetLastError();  // clean-up statuses are not reported
}

tcks_status tcks_cnn_graph_create(const tcks_cnn* m, uint32_t count, tcks_cnn_graph** out) {
  struct Guard {
    tcks_cnn_graph* g = nullptr;
    ~Guard() { tcks_cnn_graph_free(g); }
  } guard;
  CNN_BEGIN
  if (!m || !out || !count) fail(TCKS_ERR_INVALID_ARG, "null argument or zero batch");
  *out = nullptr;
  tcks_ctx* c = m->ctx;
  const u64 w_in = ct_words(c, m->L), w_out = ct_words(c, m->L - 6);
  guard.g = new tcks_cnn_graph{c, m, count, nullptr, nullptr, nullptr, nullptr, 0};
  ctx_retain(c);
  tcks_cnn_graph* g = guard.g;
  g->in = (u64*)c->dev_alloc((size_t)count * w_in * 8);
  g->out = (u64*)c->dev_alloc((size_t)count * w_out * 8);
  check_cuda(cudaMemsetAsync(g->in, 0, (size_t)count * w_in * 8, c->stream), "graph staging");
  // one eager pass builds every cached key table (their host copies cannot run inside a capture)
  cnn_forward_dev(m, g->in, w_in, count, g->out);
  check_cuda(cudaStreamSynchronize(c->stream), "graph warm-up");
  // a caller allocator: a second uncaptured pass measures the scratch the capture takes
  const std::vector<tcks_ctx*> ctxs{c};
  struct ArenaGuard {
    const std::vector<tcks_ctx*>& ctxs;
    ~ArenaGuard() { arena_off(ctxs); }
  } arena_guard{ctxs};
  if (c->has_alloc) {
    arena_record(ctxs);
    cnn_forward_dev(m, g->in, w_in, count, g->out);
    check_cuda(cudaStreamSynchronize(c->stream), "graph scratch pass");
    arena_serve(ctxs, g->blocks);
  }
  const u64 n0 = tcks_launch_count();
  check_cuda(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  try {
    cnn_forward_dev(m, g->in, w_in, count, g->out);
  } catch (...) {
    cudaGraph_t dead = nullptr;
    cudaStreamEndCapture(c->stream, &dead);
    if (dead) cudaGraphDestroy(dead);
    throw;
  }
  check_cuda(cudaStreamEndCapture(c->stream, &g->graph), "end capture");
  arena_off(ctxs);
  g->launches = tcks_launch_count() - n0;
  check_cuda(cudaGraphInstantiate(&g->exec, g->graph, 0), "graph instantiate");
  *out = g;
  guard.g = nullptr;
  CNN_END
}

tcks_status tcks_cnn_graph_run(tcks_cnn_graph* g, const tcks_ct* const* in, tcks_ct** outs) {
  struct Made {
    std::vector<tcks_ct*> v;
    ~Made() {
      for (tcks_ct* x : v) free_ct(x);
    }
  } owned;
  CNN_BEGIN
  if (!g || !in || !outs) fail(TCKS_ERR_INVALID_ARG, "null argument");
  const tcks_cnn* m = g->m;
  tcks_ctx* c = m->ctx;
  for (u32 i = 0; i < g->count; ++i) {
    outs[i] = nullptr;
    if (!in[i] || in[i]->ctx != c) fail(TCKS_ERR_INVALID_ARG, "ciphertext missing or of another context");
    need_relinearized(in[i]);
    if (in[i]->level != m->L || in[i]->scale != m->in_scale)
      fail(TCKS_ERR_LEVEL_MISMATCH, "the network takes ciphertexts at the top level and the context scale");
  }
  const u64 w_in = ct_words(c, m->L), w_out = ct_words(c, m->L - 6);
  for (u32 i = 0; i < g->count; ++i)
    check_cuda(cudaMemcpyAsync(g->in + i * w_in, in[i]->d, w_in * 8, cudaMemcpyDeviceToDevice, c->stream), "stage in");
  check_cuda(cudaGraphLaunch(g->exec, c->stream), "graph launch");
  count_launches(g->launches);
  for (u32 i = 0; i < g->count; ++i) {
    owned.v.push_back(new_ct(c, m->L - 6, m->out_scale));
    check_cuda(cudaMemcpyAsync(owned.v.back()->d, g->out + i * w_out, w_out * 8, cudaMemcpyDeviceToDevice, c->stream),
               "stage out");
  }
  for (u32 i = 0; i < g->count; ++i) outs[i] = owned.v[i];
  owned.v.clear();
  CNN_END
}

// Plaintexts of the model for inspection: kind 0 conv kernel, 1 mask (index = kernel), 2 bias
// (index 0..2), 3 FC1 diagonal, 4 FC2 diagonal (index = diagonal); host [level][N]. Kinds 5, 6: the
// FC diagonals over the extended basis; 7: baby-step diagonal (index = kernel * B + b) of the shared
// convolution, [L+1][N]; 8: folded baby-step diagonal b (TCKS_CONV_FOLD), [L+1][N].
tcks_status tcks_cnn_export_plaintext(const tcks_cnn* m, uint32_t kind, uint32_t index, uint64_t* host,
                                      size_t n_words, uint32_t* level, double* scale) {
  CNN_BEGIN
  if (!m || !host) fail(TCKS_ERR_INVALID_ARG, "null argument");
  tcks_ctx* c = m->ctx;
  const u64* src = nullptr;
  u32 lv = 0;
  double sc = 0;
  switch (kind) {
    case 0:
      if (index >= m->kernels) fail(TCKS_ERR_INVALID_ARG, "index");
      src = m->conv[index], lv = m->L, sc = c->params.scale;
      break;
    case 1:
      if (index >= m->kernels) fail(TCKS_ERR_INVALID_ARG, "index");
      src = m->masks[index], lv = m->L - 1, sc = c->params.scale;
      break;
    case 2:
      if (index >= 3) fail(TCKS_ERR_INVALID_ARG, "index");
      src = m->bias[index], lv = m->L - 2 - 2 * index, sc = m->bias_scale[index];
      break;
    case 3:
    case 4:
    case 5:
    case 6: {
      const tcks_matrix* M = (kind == 3 || kind == 5) ? m->fc1 : m->fc2;
      if (index >= M->diags) fail(TCKS_ERR_INVALID_ARG, "index");
      src = M->d + (size_t)index * M->limbs() * c->N, lv = kind >= 5 ? M->limbs() : M->level, sc = M->scale;
      break;
    }
    case 7: {
      const u32 nb = (u32)m->baby.size() + 1;
      if (!m->baby_ext || index >= m->kernels * nb) fail(TCKS_ERR_INVALID_ARG, "index");
      src = m->baby_ext + (size_t)index * (m->L + 1) * c->N, lv = m->L + 1, sc = c->params.scale;
      break;
    }
    case 8: {
      const u32 nb = (u32)m->baby.size() + 1;
      if (!m->fold_ext || index >= nb) fail(TCKS_ERR_INVALID_ARG, "index");
      src = m->fold_ext + (size_t)index * (m->L + 1) * c->N, lv = m->L + 1, sc = c->params.scale;
      break;
    }
    default: fail(TCKS_ERR_INVALID_ARG, "kind");
  }
  if (n_words != (size_t)lv * c->N) fail(TCKS_ERR_INVALID_ARG, "n_words does not match [level][N]");
  check_cuda(cudaMemcpyAsync(host, src, n_words * 8, cudaMemcpyDeviceToHost, c->stream), "export");
  check_cuda(cudaStreamSynchronize(c->stream), "export");
  if (level) *level = lv;
  if (scale) *scale = sc;
  CNN_END
}

}  // extern "C"

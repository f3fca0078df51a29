// Autotuners: the limb kernels' CTA size (tcks_autotune), and the launch shape of the batched
// encrypted network (tcks_cnn_autotune).
//
// Every limb kernel (transforms with their fused prologues and epilogues) strides its work over
// the CTA's threads, so any multiple of 32 up to the slice size is correct; the best size depends
// on the GPU, N and the word type. The tuner times a batched forward + inverse transform of 256 limbs
// for each candidate (N/64, N/32, N/16 threads per slice, clamped to [32, 1024]), keeps the fastest,
// and records it in a small JSON file keyed by "<GPU name>|<log N>|<word bits>", so a later context
// with the same key reads the choice instead of measuring again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "context.h"

using namespace tcks;

namespace {

// The cache: a flat JSON object {"key": threads, ...}.
std::map<std::string, u32> read_cache(const std::string& path) {
  std::map<std::string, u32> out;
  std::ifstream f(path);
  if (!f) return out;
  std::stringstream ss;
  ss << f.rdbuf();
  const std::string t = ss.str();
  size_t i = 0;
  while ((i = t.find('"', i)) != std::string::npos) {
    const size_t j = t.find('"', i + 1);
    if (j == std::string::npos) break;
    const std::string key = t.substr(i + 1, j - i - 1);
    size_t k = t.find(':', j);
    if (k == std::string::npos) break;
    out[key] = (u32)std::strtoul(t.c_str() + k + 1, nullptr, 10);
    i = t.find_first_of(",}", k);
    if (i == std::string::npos) break;
  }
  return out;
}

void write_cache(const std::string& path, const std::map<std::string, u32>& c) {
  const std::string tmp = path + ".tmp";
  {
    std::ofstream f(tmp);
    f << "{";
    bool first = true;
    for (const auto& kv : c) {
      f << (first ? "\n  " : ",\n  ") << '"' << kv.first << "\": " << kv.second;
      first = false;
    }
    f << "\n}\n";
  }
  std::rename(tmp.c_str(), path.c_str());
}

}  // namespace

namespace tcks {
void cnn_forward_dev(const tcks_cnn* m, const u64* x, u64 x_stride, u32 count, u64* out);
tcks_ctx* cnn_context(const tcks_cnn* m);
u32 cnn_input_level(const tcks_cnn* m);
}  // namespace tcks

// The batched network's launch shape: the limb kernels' CTA size (N/64, N/32, N/16 threads per slice)
// times the double-hoisted accumulation's requests per thread (1 or 2) times its form (0 per-thread
// loads, or 1..4 operands staged by bulk copies with 256 x 2, 256 x 3, 128 x 3 or 128 x 4 elements per
// CTA x stages; 32-bit words), each timed on a whole batched forward pass of
// `batch` requests (the median of three after one warm-up); the fastest shape is kept on the context
// and recorded under "<GPU>|cnn2|<log N>|<word bits>|<batch>" (threads * 100 + form * 10 + requests
// per thread). Results are bit-identical for every shape.
extern "C" tcks_status tcks_cnn_autotune(const tcks_cnn* m, uint32_t batch, const char* cache_path,
                                         uint32_t* chosen_threads, uint32_t* chosen_rpt, uint32_t* chosen_form) {
  try {
    tcks::NvtxRange nvtx(__func__);
    drop_stale_cuda_error();
    if (!m || !batch) fail(TCKS_ERR_INVALID_ARG, "null model or empty batch");
    tcks_ctx* c = cnn_context(m);
    cudaDeviceProp prop;
    check_cuda(cudaGetDeviceProperties(&prop, c->device), "device properties");
    const u32 log_n = c->params.log_n, log_c = log_n > 14 ? log_n - 14 : 0, ns = 1u << (log_n - log_c);
    const std::string key = std::string(prop.name) + "|cnn3|" + std::to_string(log_n) + "|" +
                            (c->T.narrow ? "32" : "64") + "|" + std::to_string(batch);
    std::map<std::string, u32> cache;
    if (cache_path && *cache_path) cache = read_cache(cache_path);
    u32 cap = 1024;
    for (u32 t : {limb_threads_cap_core(c->T.narrow, log_c), limb_threads_cap_sample(c->T.narrow, log_c),
                  limb_threads_cap_fft(c->T.narrow, log_c)})
      cap = std::min(cap, t);
    cap &= ~31u;
    u32 best_t = 0, best_r = 0, best_f = 0;
    auto it = cache.find(key);
    const u32 cv = it != cache.end() ? it->second : 0;
    if (cv / 100 >= 32 && cv / 100 <= cap && (cv / 10) % 10 <= 4 && (cv % 10 <= 2 || cv % 10 == 4)) {
      best_t = cv / 100;
      best_f = (cv / 10) % 10;
      best_r = cv % 10;
    } else {
      std::vector<u32> threads;
      for (u32 div : {64u, 32u, 16u}) {
        u32 t = std::max<u32>(32, std::min(cap, ns / div));
        if (std::find(threads.begin(), threads.end(), t) == threads.end()) threads.push_back(t);
      }
      const std::vector<u32> rpts = c->T.narrow ? std::vector<u32>{0, 2, 4, 1} : std::vector<u32>{0};
      const std::vector<u32> forms = c->T.narrow ? std::vector<u32>{0, 1, 2, 3, 4} : std::vector<u32>{0};
      const u32 L = cnn_input_level(m);
      const u64 win = ct_words(c, L), wout = ct_words(c, L - 6);
      DevBuf x(c, (size_t)batch * win), y(c, (size_t)batch * wout);
      check_cuda(cudaMemsetAsync(x.p, 0, (size_t)batch * win * 8, c->stream), "tune input");
      cudaEvent_t ev[4];
      for (cudaEvent_t& e : ev) check_cuda(cudaEventCreate(&e), "event");
      const u32 saved_t = c->T.limb_threads, saved_r = c->T.dh_rpt, saved_f = c->T.dh_form;
      float best_ms = 1e30f;
      for (u32 t : threads)
        for (u32 r : rpts)
          for (u32 f : forms) {
          c->T.limb_threads = t;
          c->T.dh_rpt = r;
          c->T.dh_form = f;
          cnn_forward_dev(m, x.p, win, batch, y.p);  // warm-up
          float ms[3];
          for (int k = 0; k < 3; ++k) {
            check_cuda(cudaEventRecord(ev[0], c->stream), "event");
            cnn_forward_dev(m, x.p, win, batch, y.p);
            check_cuda(cudaEventRecord(ev[1], c->stream), "event");
            check_cuda(cudaEventSynchronize(ev[1]), "tune");
            cudaEventElapsedTime(&ms[k], ev[0], ev[1]);
          }
          std::sort(ms, ms + 3);
          if (ms[1] < best_ms) {
            best_ms = ms[1];
            best_t = t;
            best_r = r;
            best_f = f;
          }
        }
      c->T.limb_threads = saved_t;
      c->T.dh_rpt = saved_r;
      c->T.dh_form = saved_f;
      for (cudaEvent_t& e : ev) cudaEventDestroy(e);
      check_launch("cnn autotune");
      if (cache_path && *cache_path) {
        cache[key] = best_t * 100 + best_f * 10 + best_r;
        write_cache(cache_path, cache);
      }
    }
    c->T.limb_threads = best_t;
    c->T.dh_rpt = best_r;
    c->T.dh_form = best_f;
    if (chosen_threads) *chosen_threads = best_t;
    if (chosen_rpt) *chosen_rpt = best_r;
    if (chosen_form) *chosen_form = best_f;
  } catch (const tcks::Error& e) {
    return abi_record(e.code, e.msg);
  }
  abi_clear();
  return TCKS_OK;
}

extern "C" tcks_status tcks_autotune(tcks_ctx* c, const char* cache_path, uint32_t* chosen_threads) {
  try {
    drop_stale_cuda_error();
    if (!c) fail(TCKS_ERR_INVALID_ARG, "null context");
    cudaDeviceProp prop;
    check_cuda(cudaGetDeviceProperties(&prop, c->device), "device properties");
    const u32 log_n = c->params.log_n;
    const u32 log_c = log_n > 14 ? log_n - 14 : 0;  // the cluster split of a limb (see ntt.cuh)
    const u32 ns = 1u << (log_n - log_c);
    const std::string key =
        std::string(prop.name) + "|" + std::to_string(log_n) + "|" + (c->T.narrow ? "32" : "64");
    std::map<std::string, u32> cache;
    if (cache_path && *cache_path) cache = read_cache(cache_path);
    // every kernel that runs with the tuned CTA size must accept it (registers bound the size)
    u32 cap = 1024;
    for (u32 t : {limb_threads_cap_core(c->T.narrow, log_c), limb_threads_cap_sample(c->T.narrow, log_c),
                  limb_threads_cap_fft(c->T.narrow, log_c)})
      cap = std::min(cap, t);
    cap &= ~31u;
    if (cap < 32) fail(TCKS_ERR_CUDA, "autotune: cannot read the limb kernels' launch limits");
    u32 best = 0;
    auto it = cache.find(key);
    if (it != cache.end() && it->second >= 32 && it->second <= cap && it->second % 32 == 0) {
      best = it->second;
    } else {
      std::vector<u32> cand;
      for (u32 div : {64u, 32u, 16u}) {
        u32 t = ns / div;
        t = t < 32 ? 32 : (t > cap ? cap : t);
        if (std::find(cand.begin(), cand.end(), t) == cand.end()) cand.push_back(t);
      }
      // timed work: batched transforms up to N = 2^13; above that the plain transforms run in two
      // passes of fixed shape and the tuned size only reaches the fused kernels, so batched rescales
      // (lift + transform + combine per limb) are timed instead
      const u32 limbs = 256, lv = c->L + 1;
      DevBuf buf(c, (size_t)limbs * c->N), out(c, (size_t)limbs * c->N), top(c, (size_t)limbs * c->N);
      check_cuda(cudaMemsetAsync(buf.p, 0, (size_t)limbs * c->N * 8, c->stream), "tune buffer");
      const u32 ell = c->L;
      const bool fused = log_n > 13 && ell >= 2;
      const u32 polys = fused ? std::max<u32>(1, limbs / ell) : 0;
      cudaEvent_t a, b;
      check_cuda(cudaEventCreate(&a), "event");
      check_cuda(cudaEventCreate(&b), "event");
      float best_ms = 1e30f;
      const u32 saved = c->T.limb_threads;
      for (u32 t : cand) {
        c->T.limb_threads = t;
        for (int rep = 0; rep < 2; ++rep) {  // warm-up, then timed
          cudaEventRecord(a, c->stream);
          for (int it2 = 0; it2 < 3; ++it2) {
            if (fused) {
              launch_rescale(c->T, buf.p, ell, polys, top.p, out.p, c->stream);
            } else {
              launch_ntt(c->T, false, buf.p, (u64)lv * c->N, buf.p, (u64)lv * c->N, limbs, 0, lv, c->stream);
              launch_ntt(c->T, true, buf.p, (u64)lv * c->N, buf.p, (u64)lv * c->N, limbs, 0, lv, c->stream);
            }
          }
          cudaEventRecord(b, c->stream);
        }
        check_cuda(cudaEventSynchronize(b), "tune");
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
      c->T.limb_threads = saved;
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      check_launch("autotune");
      if (cache_path && *cache_path) {
        cache[key] = best;
        write_cache(cache_path, cache);
      }
    }
    c->T.limb_threads = best;
    if (chosen_threads) *chosen_threads = best;
  } catch (const tcks::Error& e) {
    return abi_record(e.code, e.msg);
  }
  abi_clear();
  return TCKS_OK;
}

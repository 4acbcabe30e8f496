// Autotuner of the FFT radix schedule of pass B (the y/z transforms of the local-potential path,
// §5.1 batched FFTs).  For a box length N = N2 = N3 the candidates are the CTA-wide form with
// every compile-time split N = A * B at 256 and 384 threads per CTA (and 128 in single precision),
// and the per-warp form.  Each
// candidate runs one warm-up and three timed launches (the fastest counts) on a zero-filled
// scratch slab of the same window and of the production chunk size (CUDA events on the context's
// stream); the fastest candidate is kept for the process in a table keyed by device, precision,
// box and window.  All candidates compute the same transform; they differ only in rounding order.
#include <map>
#include <mutex>
#include <tuple>

#include "gemm_tune.h"
#include "local_wide.h"
#include "tune.h"

namespace kss {

namespace {

using Key = std::tuple<int, int, int, int, int, int, int>;  // device, bytes/real, N1, N2, N3, W3 (rounded), 0

struct Entry {
  PassBSched s;
  int device, prec, N1, N, W3, W2;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;
std::vector<Key> g_order;  // insertion order (for listing)

template <typename T>
PassBSched builtin(const lk::LocalArgs<T>& a, const fftr::Split& s2) {
  PassBSched s;
  s.A = s2.A;
  s.B = s2.B;
  s.threads = wide_pass_b<T>(a, s2.A, s2.B, lk::kWideThreads, 0, nullptr, true) ? lk::kWideThreads : 0;
  return s;
}

}  // namespace

template <typename T>
PassBSched pass_b_schedule(kss_ctx ctx, const lk::LocalArgs<T>& a, const fftr::Split& s2, bool may_tune) {
  // Configurations are keyed by box and the window height W3 rounded up to a multiple of 8 (the
  // y-stage task count); a schedule tuned at the rounded height fits every smaller one.
  const int W3b = std::min(a.N3, (a.W3 + 7) / 8 * 8);
  const Key key{ctx->device, (int)sizeof(T), a.N1, a.N2, a.N3, W3b, 0};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(key);
    if (it != g_table.end()) return it->second.s;
  }
  if (!may_tune || !ctx->autotune) return builtin<T>(a, s2);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  KSS_CHECK_CUDA(cudaStreamIsCapturing(ctx->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return builtin<T>(a, s2);

  using C = typename lk::CT<T>::C;
  lk::LocalArgs<T> t = a;
  t.W3 = W3b;
  // candidates: CTA-wide splits x threads, then the per-warp form
  std::vector<PassBSched> cand;
  if (a.N2 == a.N3)
    for (const auto& ab : wide_splits())
      for (int nt : {128, 256, 384})  // 128: single precision only (the dry check says which exist)
        if (ab.first * ab.second == a.N2 && wide_pass_b<T>(t, ab.first, ab.second, nt, 0, nullptr, true))
          cand.push_back(PassBSched{ab.first, ab.second, nt, 0, 0});
  cand.push_back(PassBSched{s2.A, s2.B, 0, 0, 0});
  // scratch slab of the production chunk size (the local passes keep kSlabChunkBytes of slab per
  // launch), so that candidates are timed at the launch shape they will run at
  const size_t per_band = (size_t)t.N1 * t.W3 * t.W2 * sizeof(C);
  const int nbt = (int)std::max<size_t>(1, std::min<size_t>(64, kSlabChunkBytes / per_band));
  const size_t elems = (size_t)t.N1 * t.W3 * t.W2 * nbt;
  ctx->ws_tune.ensure(elems * sizeof(C));
  KSS_CHECK_CUDA(cudaMemsetAsync(ctx->ws_tune.p, 0, elems * sizeof(C), ctx->stream));
  t.work = ctx->ws_tune.as<C>();
  t.Vpi = t.Vx;  // any N1 x N x N array: the values do not matter for timing
  t.n0 = 0;
  cudaEvent_t e0, e1;
  KSS_CHECK_CUDA(cudaEventCreate(&e0));
  KSS_CHECK_CUDA(cudaEventCreate(&e1));
  auto launch = [&](const PassBSched& c) {
    if (c.threads) wide_pass_b<T>(t, c.A, c.B, c.threads, nbt, ctx->stream, false);
    else warp_pass_b<T>(ctx, t, nbt);
  };
  int best = -1;
  for (size_t i = 0; i < cand.size(); ++i) {
    launch(cand[i]);  // warm-up (and shared-memory attribute)
    double tmin = 1e300;
    for (int r = 0; r < 3; ++r) {  // the fastest of three timed launches
      KSS_CHECK_CUDA(cudaEventRecord(e0, ctx->stream));
      launch(cand[i]);
      KSS_CHECK_CUDA(cudaEventRecord(e1, ctx->stream));
      KSS_CHECK_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      KSS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      tmin = std::min(tmin, (double)ms);
    }
    cand[i].ms = tmin;
    if (best < 0 || cand[i].ms < cand[best].ms) best = (int)i;
  }
  KSS_CHECK_CUDA(cudaEventDestroy(e0));
  KSS_CHECK_CUDA(cudaEventDestroy(e1));
  KSS_CHECK_CUDA(cudaGetLastError());
  PassBSched s = cand[best];
  s.ncand = (int)cand.size();
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_table.count(key)) {
    g_table[key] = Entry{s, ctx->device, sizeof(T) == 8 ? KSS_PREC_FP64 : KSS_PREC_MIXED, a.N1, a.N2, W3b, a.W2};
    g_order.push_back(key);
  }
  return g_table[key].s;
}

template PassBSched pass_b_schedule<double>(kss_ctx, const lk::LocalArgs<double>&, const fftr::Split&, bool);
template PassBSched pass_b_schedule<float>(kss_ctx, const lk::LocalArgs<float>&, const fftr::Split&, bool);

}  // namespace kss

using namespace kss;

extern "C" {

kss_status kss_autotune_set(kss_ctx ctx, int mode) {
  if (!ctx || (mode != 0 && mode != 1)) return KSS_EINVAL;
  ctx->autotune = mode;
  return KSS_OK;
}

kss_status kss_autotune_count(int* n) {
  if (!n) return KSS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  *n = (int)g_order.size();
  return KSS_OK;
}

kss_status kss_autotune_get(int i, kss_tune_entry* out) {
  if (!out) return KSS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (i < 0 || i >= (int)g_order.size()) return KSS_EINVAL;
  const Entry& e = g_table.at(g_order[i]);
  out->device = e.device;
  out->precision = e.prec;
  out->N1 = e.N1;
  out->N = e.N;
  out->W3 = e.W3;
  out->W2 = e.W2;
  out->A = e.s.A;
  out->B = e.s.B;
  out->threads = e.s.threads;
  out->ms = e.s.ms;
  out->ncand = e.s.ncand;
  return KSS_OK;
}

kss_status kss_autotune_put(const kss_tune_entry* e) {
  if (!e || e->N1 < 2 || e->N < 2 || e->W3 < 1 || e->W3 > e->N ||
      (e->precision != KSS_PREC_FP64 && e->precision != KSS_PREC_MIXED) ||
      (e->threads != 0 && e->threads != 128 && e->threads != 256 && e->threads != 384) || e->A * e->B != e->N)
    return KSS_EINVAL;
  const int bytes = e->precision == KSS_PREC_FP64 ? 8 : 4;
  const int W3b = std::min(e->N, (e->W3 + 7) / 8 * 8);
  const Key key{e->device, bytes, e->N1, e->N, e->N, W3b, 0};
  PassBSched s;
  s.A = e->A;
  s.B = e->B;
  s.threads = e->threads;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_table.count(key)) g_order.push_back(key);
  g_table[key] = Entry{s, e->device, e->precision, e->N1, e->N, W3b, e->W2};
  return KSS_OK;
}

kss_status kss_autotune_clear(void) {
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table.clear();
    g_order.clear();
  }
  gemm_tune_clear();
  return KSS_OK;
}

}  // extern "C"

// Autotuner of the schedule of the tensor-core GEMMs: the kernel form (for the split-BF16 products:
// one CTA per output tile, or persistent CTAs with two TMEM accumulators and 128- or 64-column
// tiles) and the K-split.  Splitting K across CTAs fills the SMs when a
// product has few output tiles (the Gram matrices, the projector coefficients), at the price of one
// set of partial sums per split written and added back; the best split depends on the shape, the
// operand sizes in L2 and the per-CTA fixed cost, so it is timed on the device at first use per
// shape and kept for the process (the FFT schedule tuner of tune.cu does the same for the FFT).
// Every split computes the same product (the K ranges are summed in a fixed order by the combine
// kernels); results differ only in rounding order.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "gemm_tune.h"

namespace kss {

namespace {

using Key = std::tuple<int, int, int, int, int>;  // device, kind, Mr, Nr, kb_total

struct Entry {
  int device, kind, Mr, Nr, kb_total;
  int splits;
  double ms;
  int ncand;
  int form;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;
std::vector<Key> g_order;

}  // namespace

GemmChoice tuned_gemm(kss_ctx ctx, int kind, int Mr, int Nr, int kb_total, std::vector<GemmChoice> cand,
                      GemmChoice plan, const std::function<void(GemmChoice)>& run) {
  const Key key{ctx->device, kind, Mr, Nr, kb_total};
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(key);
    if (it != g_table.end()) return GemmChoice{it->second.form, it->second.splits};
  }
  if (!ctx->autotune) return plan;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  KSS_CHECK_CUDA(cudaStreamIsCapturing(ctx->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return plan;
  cand.push_back(plan);
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  cudaEvent_t e0, e1;
  KSS_CHECK_CUDA(cudaEventCreate(&e0));
  KSS_CHECK_CUDA(cudaEventCreate(&e1));
  GemmChoice best = plan;
  double tbest = 1e300;
  for (const GemmChoice& c : cand) {
    run(c);  // warm-up
    double tmin = 1e300;
    for (int r = 0; r < 3; ++r) {
      KSS_CHECK_CUDA(cudaEventRecord(e0, ctx->stream));
      run(c);
      KSS_CHECK_CUDA(cudaEventRecord(e1, ctx->stream));
      KSS_CHECK_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      KSS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      tmin = std::min(tmin, (double)ms);
    }
    if (tmin < tbest) {
      tbest = tmin;
      best = c;
    }
  }
  KSS_CHECK_CUDA(cudaEventDestroy(e0));
  KSS_CHECK_CUDA(cudaEventDestroy(e1));
  KSS_CHECK_CUDA(cudaGetLastError());
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_table.count(key)) {
    g_table[key] = Entry{ctx->device, kind, Mr, Nr, kb_total, best.splits, tbest, (int)cand.size(), best.form};
    g_order.push_back(key);
  }
  const Entry& e = g_table[key];
  return GemmChoice{e.form, e.splits};
}

int tuned_split(kss_ctx ctx, int kind, int Mr, int Nr, int kb_total, long long tiles, int min_kb, int plan,
                const std::function<void(int)>& run) {
  const int smax = std::max(1, kb_total / std::max(1, min_kb));
  const int nsm = std::max(1, ctx->nsm);
  std::vector<GemmChoice> cand{{0, plan}, {0, 1}};
  for (int w = 1; w <= 3; ++w)
    cand.push_back({0, (int)std::max(1LL, (long long)w * nsm / std::max(1LL, tiles))});
  for (auto& c : cand) c.splits = std::max(1, std::min(c.splits, smax));
  const GemmChoice g = tuned_gemm(ctx, kind, Mr, Nr, kb_total, cand, GemmChoice{0, std::max(1, std::min(plan, smax))},
                                  [&](GemmChoice c) { run(c.splits); });
  return std::max(1, std::min(g.splits, smax));
}

void gemm_tune_clear() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.clear();
  g_order.clear();
}

}  // namespace kss

using namespace kss;

extern "C" {

kss_status kss_autotune_gemm_count(int* n) {
  if (!n) return KSS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  *n = (int)g_order.size();
  return KSS_OK;
}

kss_status kss_autotune_gemm_get(int i, kss_gemm_tune_entry* out) {
  if (!out) return KSS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (i < 0 || i >= (int)g_order.size()) return KSS_EINVAL;
  const Entry& e = g_table[g_order[i]];
  out->device = e.device;
  out->kind = e.kind;
  out->Mr = e.Mr;
  out->Nr = e.Nr;
  out->kblocks = e.kb_total;
  out->splits = e.splits;
  out->ms = e.ms;
  out->ncand = e.ncand;
  out->form = e.form;
  return KSS_OK;
}

kss_status kss_autotune_gemm_put(const kss_gemm_tune_entry* e) {
  if (!e || e->kind < 0 || e->kind > 3 || e->Mr < 1 || e->Nr < 1 || e->kblocks < 1 || e->splits < 1 ||
      e->splits > e->kblocks || e->form < 0 || e->form > (e->kind == GT_BF16X3 ? 2 : 0))
    return KSS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  const Key key{e->device, e->kind, e->Mr, e->Nr, e->kblocks};
  if (!g_table.count(key)) g_order.push_back(key);
  g_table[key] = Entry{e->device, e->kind, e->Mr, e->Nr, e->kblocks, e->splits, 0.0, 0, e->form};
  return KSS_OK;
}

}  // extern "C"

// Launch accounting and optional per-kernel CUDA-event timing on the context stream.
#include <mutex>
#include <string>
#include <unordered_map>

#include "kss_internal.h"

namespace kss {

namespace {
std::mutex g_mu;
std::vector<std::string>& names() {
  static std::vector<std::string> n;
  return n;
}
std::unordered_map<std::string, int>& index() {
  static std::unordered_map<std::string, int> m;
  return m;
}
}  // namespace

int prof_register(const char* name) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto& m = index();
  auto it = m.find(name);
  if (it != m.end()) return it->second;
  const int id = (int)names().size();
  names().push_back(name);
  m.emplace(name, id);
  return id;
}

const char* prof_name(int id) {
  std::lock_guard<std::mutex> lk(g_mu);
  return (id >= 0 && id < (int)names().size()) ? names()[id].c_str() : "";
}

int prof_names() {
  std::lock_guard<std::mutex> lk(g_mu);
  return (int)names().size();
}

static cudaEvent_t take_event(Prof& p) {
  if (!p.free_ev.empty()) {
    cudaEvent_t e = p.free_ev.back();
    p.free_ev.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

ProfScope::ProfScope(kss_ctx c, int id_) : ctx(c), id(id_) {
  ctx->prof.launches += 1;
  if ((int)ctx->prof.count.size() <= id) {
    ctx->prof.count.resize(id + 1, 0);
    ctx->prof.ms.resize(id + 1, 0.0);
  }
  ctx->prof.count[id] += 1;
  if (ctx->prof.on) {
    if (ctx->prof.pending.size() >= 16384) prof_resolve(ctx);
    a = take_event(ctx->prof);
    b = take_event(ctx->prof);
    if (a && b) cudaEventRecord(a, ctx->stream);
  }
}

ProfScope::~ProfScope() {
  if (a && b) {
    cudaEventRecord(b, ctx->stream);
    ctx->prof.pending.push_back({a, b, id});
  } else {
    if (a) ctx->prof.free_ev.push_back(a);
    if (b) ctx->prof.free_ev.push_back(b);
  }
}

void prof_resolve(kss_ctx ctx) {
  Prof& p = ctx->prof;
  if (p.pending.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& e : p.pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess && e.id < (int)p.ms.size())
      p.ms[e.id] += ms;
    else
      cudaGetLastError();
    p.free_ev.push_back(e.a);
    p.free_ev.push_back(e.b);
  }
  p.pending.clear();
}

void prof_fold(kss_ctx ctx) {
  for (kss_ctx w : ctx->aux) {
    prof_resolve(w);
    Prof& a = w->prof;
    if (ctx->prof.count.size() < a.count.size()) {
      ctx->prof.count.resize(a.count.size(), 0);
      ctx->prof.ms.resize(a.count.size(), 0.0);
    }
    for (size_t i = 0; i < a.count.size(); ++i) {
      ctx->prof.count[i] += a.count[i];
      ctx->prof.ms[i] += a.ms[i];
    }
    ctx->prof.launches += a.launches;
    a.launches = 0;
    std::fill(a.count.begin(), a.count.end(), 0);
    std::fill(a.ms.begin(), a.ms.end(), 0.0);
  }
}

void prof_release(kss_ctx ctx) {
  prof_resolve(ctx);
  for (auto e : ctx->prof.free_ev) cudaEventDestroy(e);
  ctx->prof.free_ev.clear();
}

}  // namespace kss

using namespace kss;

extern "C" {

kss_status kss_profile_enable(kss_ctx ctx, int enable) {
  if (!ctx) return KSS_EINVAL;
  prof_resolve(ctx);
  prof_fold(ctx);
  ctx->prof.on = enable != 0;
  ctx->prof.launches = 0;
  std::fill(ctx->prof.count.begin(), ctx->prof.count.end(), 0);
  std::fill(ctx->prof.ms.begin(), ctx->prof.ms.end(), 0.0);
  return KSS_OK;
}

kss_status kss_profile_count(kss_ctx ctx, int* nkernels, long long* launches) {
  if (!ctx) return KSS_EINVAL;
  prof_resolve(ctx);
  prof_fold(ctx);
  if (nkernels) *nkernels = (int)ctx->prof.count.size();
  if (launches) *launches = ctx->prof.launches;
  return KSS_OK;
}

kss_status kss_profile_entry(kss_ctx ctx, int i, const char** name, long long* launches,
                             double* total_ms) {
  if (!ctx) return KSS_EINVAL;
  prof_resolve(ctx);
  prof_fold(ctx);
  if (i < 0 || i >= (int)ctx->prof.count.size()) return KSS_EINVAL;
  if (name) *name = prof_name(i);
  if (launches) *launches = ctx->prof.count[i];
  if (total_ms) *total_ms = ctx->prof.ms[i];
  return KSS_OK;
}

}  // extern "C"

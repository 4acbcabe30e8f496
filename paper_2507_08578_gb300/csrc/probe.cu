// Throughput probes of the CUDA cores' fused multiply-add pipes (FP64 and FP32): the denominators
// of the ALU rooflines of the FFT passes, measured on the device the context runs on instead of
// taken from a datasheet.  Every thread runs kChains independent FMA chains (enough independent
// work per SM to cover the pipe latency), the grid is a whole number of CTAs per SM, and the rate
// is the best of three timed launches (CUDA events on the context stream).
#include <algorithm>

#include "kss_internal.h"

namespace kss {

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe(const T* __restrict__ seed, T* __restrict__ out, int iters) {
  T a[kChains];
  const T b = seed[0], c = seed[1];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed[2] + (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == (T)12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
double run_probe(kss_ctx ctx, int iters) {
  const int nsm = std::max(1, ctx->nsm);
  const int blocks = nsm * 8;
  DevBuf seed, out;
  seed.alloc(3 * sizeof(T));
  out.alloc((size_t)blocks * kProbeThreads * sizeof(T));
  // b slightly below 1 and c small: the chains stay finite for any iteration count
  const T h[3] = {(T)0.999999, (T)1e-7, (T)0.5};
  KSS_CHECK_CUDA(cudaMemcpyAsync(seed.p, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
  cudaEvent_t e0, e1;
  KSS_CHECK_CUDA(cudaEventCreate(&e0));
  KSS_CHECK_CUDA(cudaEventCreate(&e1));
  double best = 0;
  fma_probe<T><<<blocks, kProbeThreads, 0, ctx->stream>>>(seed.as<T>(), out.as<T>(), iters);  // warm-up
  for (int r = 0; r < 3; ++r) {
    KSS_CHECK_CUDA(cudaEventRecord(e0, ctx->stream));
    fma_probe<T><<<blocks, kProbeThreads, 0, ctx->stream>>>(seed.as<T>(), out.as<T>(), iters);
    KSS_CHECK_CUDA(cudaEventRecord(e1, ctx->stream));
    KSS_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    KSS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double flops = 2.0 * kChains * (double)iters * blocks * kProbeThreads;
    best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  KSS_CHECK_CUDA(cudaEventDestroy(e0));
  KSS_CHECK_CUDA(cudaEventDestroy(e1));
  KSS_CHECK_CUDA(cudaGetLastError());
  return best;
}

}  // namespace

}  // namespace kss

using namespace kss;

extern "C" kss_status kss_peak_probe(kss_ctx ctx, int pipe, double* tflops) {
  if (!ctx || !tflops || pipe < 0 || pipe > 1) return KSS_EINVAL;
  try {
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    *tflops = pipe == 0 ? run_probe<double>(ctx, 4096) : run_probe<float>(ctx, 65536);
    ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    ctx->err = e.msg;
    return e.st;
  }
}

// Kernel instances of the CTA-wide pass B (local_kernels.cuh, pass_bw_body) for one precision:
// every split of KSS_WIDE_SPLITS at 256 and 384 threads per CTA (and 128 in single precision).  Included by one translation
// unit per precision (local_wide_f32.cu, local_wide_f64.cu) so the build compiles them in parallel.
#pragma once

#include "local_kernels.cuh"
#include "local_wide.h"

namespace kss {
namespace wide_detail {

using namespace lk;

template <typename T, int A, int B, int NT, int CW = 0>
__global__ void __launch_bounds__(NT) pass_bw(LocalArgs<T> a) {
  pass_bw_body<T, A, B, NT, CW>(a, blockIdx.x, blockIdx.y);
}

// Splits with a pruned instance and its edge width: the 96-point splits, with the widths that the
// sphere window of the config-2 box (|m| <= 20 along y and z) needs; a window that needs no more
// than that width runs the pruned instance, any other the full one.
constexpr int pruned_cw(int A, int B) {
  return A == 8 && B == 12 ? 2 : A == 12 && B == 8 ? 3 : A == 6 && B == 16 ? 2 : A == 16 && B == 6 ? 4 : 0;
}

template <typename T, int A, int B, int NT>
bool launch_one(const LocalArgs<T>& a, int nbands, cudaStream_t st, bool dry) {
  const size_t sm = WideB<T, A, B>::smem(a.W3);
  if (sm > kWideSmemMax) return false;
  if (dry) return true;
  constexpr int PC = pruned_cw(A, B);
  if constexpr (PC > 0) {
    const int cw = wide_prune_cw(A, B, a.lo2, a.W2, a.lo3, a.W3);
    if (cw > 0 && cw <= PC) {
      KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_bw<T, A, B, NT, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      pass_bw<T, A, B, NT, PC><<<dim3(a.N1, nbands), NT, sm, st>>>(a);
      return true;
    }
  }
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_bw<T, A, B, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  pass_bw<T, A, B, NT><<<dim3(a.N1, nbands), NT, sm, st>>>(a);
  return true;
}

// 128-thread instances in single precision only: for the small boxes of batched systems a stage's
// tasks fill a 128-thread CTA better, and four-warp barriers idle fewer warps.
template <typename T, int A, int B>
bool launch_small(const LocalArgs<T>& a, int nbands, cudaStream_t st, bool dry) {
  if constexpr (sizeof(T) == 4) return launch_one<T, A, B, 128>(a, nbands, st, dry);
  else return false;
}

template <typename T>
bool dispatch(const LocalArgs<T>& a, int A, int B, int nt, int nbands, cudaStream_t st, bool dry) {
  if (a.N2 != a.N3 || A * B != a.N2 || (nt != 128 && nt != 256 && nt != 384)) return false;
  switch (A * 32 + B) {
#define KSS_CASE(x, y)                                                                \
  case x * 32 + y:                                                                    \
    return nt == 128   ? launch_small<T, x, y>(a, nbands, st, dry)                    \
           : nt == 256 ? launch_one<T, x, y, 256>(a, nbands, st, dry)                 \
                       : launch_one<T, x, y, 384>(a, nbands, st, dry);
    KSS_WIDE_SPLITS(KSS_CASE)
#undef KSS_CASE
    default:
      return false;
  }
}

}  // namespace wide_detail
}  // namespace kss

// Kernel instances of the CTA-wide pass B (local_kernels.cuh, pass_bw_body): the y/z transforms
// of one x-plane with every lane of the CTA busy in each transform stage (§5.1 batched FFTs).
// Kept in a translation unit of their own so that the build compiles them in parallel with the
// per-warp forms.
#include "local_kernels.cuh"
#include "local_wide.h"

namespace kss {
namespace {

using namespace lk;

template <typename T, int A, int B>
__global__ void __launch_bounds__(kWideThreads) pass_bw(LocalArgs<T> a) {
  pass_bw_body<T, A, B>(a, blockIdx.x, blockIdx.y);
}

template <typename T, int A, int B>
bool launch_one(const LocalArgs<T>& a, int nbands, cudaStream_t st, bool dry) {
  const size_t sm = WideB<T, A, B>::smem(a.W3);
  if (sm > kWideSmemMax) return false;
  if (dry) return true;
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_bw<T, A, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  pass_bw<T, A, B><<<dim3(a.N1, nbands), kWideThreads, sm, st>>>(a);
  return true;
}

}  // namespace

template <typename T>
bool wide_pass_b(const LocalArgs<T>& a, int A, int B, int nbands, cudaStream_t st, bool dry) {
  if (a.N2 != a.N3 || A * B != a.N2) return false;
  switch (A * 32 + B) {
#define KSS_CASE(x, y) \
  case x * 32 + y:     \
    return launch_one<T, x, y>(a, nbands, st, dry);
    KSS_SPLITS(KSS_CASE)
#undef KSS_CASE
    default:
      return false;
  }
}

template bool wide_pass_b<double>(const LocalArgs<double>&, int, int, int, cudaStream_t, bool);
template bool wide_pass_b<float>(const LocalArgs<float>&, int, int, int, cudaStream_t, bool);

}  // namespace kss

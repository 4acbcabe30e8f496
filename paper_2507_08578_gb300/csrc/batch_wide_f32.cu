// Grouped CTA-wide pass B instances of the batch engine, single precision: every split
// of KSS_WIDE_SPLITS at 128, 256 and 384 threads per CTA.
#include "batch_kernels.cuh"

namespace kss {
namespace bk {

template <>
GroupKernel<float> group_kernel_w<float>(int A, int B, int nt) {
  if (nt != 128 && nt != 256 && nt != 384) return nullptr;
  switch (A * 32 + B) {
#define KSS_CASE(x, y) \
  case x * 32 + y:     \
    return nt == 128 ? group_passw<float, x, y, 128> : nt == 256 ? group_passw<float, x, y, 256> : group_passw<float, x, y, 384>;
    KSS_WIDE_SPLITS(KSS_CASE)
#undef KSS_CASE
    default:
      return nullptr;
  }
}

}  // namespace bk
}  // namespace kss

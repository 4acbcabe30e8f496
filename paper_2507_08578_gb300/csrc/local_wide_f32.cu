// CTA-wide pass B instances, single precision (see local_wide_impl.cuh).
#include "local_wide_impl.cuh"

namespace kss {

template <>
bool wide_pass_b<float>(const lk::LocalArgs<float>& a, int A, int B, int nt, int nbands, cudaStream_t st,
                        bool dry) {
  return wide_detail::dispatch<float>(a, A, B, nt, nbands, st, dry);
}

template <>
bool wide_pass_x<float>(const lk::LocalArgs<float>& a, int which, int nbands, cudaStream_t st, bool dry) {
  return wide_detail::dispatch_x<float>(a, which, nbands, st, dry);
}

}  // namespace kss

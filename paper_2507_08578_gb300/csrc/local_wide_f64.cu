// CTA-wide pass B instances, double precision (see local_wide_impl.cuh).
#include "local_wide_impl.cuh"

namespace kss {

template <>
bool wide_pass_b<double>(const lk::LocalArgs<double>& a, int A, int B, int nt, int nbands, cudaStream_t st,
                         bool dry) {
  return wide_detail::dispatch<double>(a, A, B, nt, nbands, st, dry);
}

template <>
bool wide_pass_x<double>(const lk::LocalArgs<double>& a, int which, int nbands, cudaStream_t st, bool dry) {
  return wide_detail::dispatch_x<double>(a, which, nbands, st, dry);
}

}  // namespace kss

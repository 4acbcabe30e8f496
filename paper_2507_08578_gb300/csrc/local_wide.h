// Host entry of the CTA-wide pass B instances (local_wide_impl.cuh).
#pragma once

#include "local_kernels.cuh"

namespace kss {

constexpr size_t kWideSmemMax = 227 * 1024;

// Launches pass B for nbands bands (grid N1 x nbands, nt = 256 or 384 threads per CTA) with the
// CTA-wide transform stages for the split N2 == N3 == A * B.  Returns false (and launches
// nothing) when no instance exists for (A, B, nt) or its shared memory does not fit.
// dry = true only checks availability.
template <typename T>
bool wide_pass_b(const lk::LocalArgs<T>& a, int A, int B, int nt, int nbands, cudaStream_t st, bool dry);

// Launches pass A (which = 0) or pass C (which = 1) for nbands bands (grid W3 x nbands) with the
// CTA-wide x transforms (lk::pass_aw_body, lk::pass_cw_body), pruned to the sphere's x window when
// an instance covers it.  Returns false (and launches nothing) when no instance exists for N1 or
// its shared memory does not fit; dry = true only checks availability.
template <typename T>
bool wide_pass_x(const lk::LocalArgs<T>& a, int which, int nbands, cudaStream_t st, bool dry);

// The (A, B) pairs with instances, in KSS_WIDE_SPLITS order.
inline const std::vector<std::pair<int, int>>& wide_splits() {
  static const std::vector<std::pair<int, int>> v = {
#define KSS_PAIR(x, y) {x, y},
      KSS_WIDE_SPLITS(KSS_PAIR)
#undef KSS_PAIR
  };
  return v;
}

}  // namespace kss

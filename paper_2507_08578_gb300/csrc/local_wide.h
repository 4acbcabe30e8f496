// Host entry of the CTA-wide pass B instances (local_wide.cu).
#pragma once

#include "local_kernels.cuh"

namespace kss {

constexpr size_t kWideSmemMax = 227 * 1024;

// Launches pass B for nbands bands (grid N1 x nbands) with the CTA-wide transform stages when a
// compile-time instance exists for the split (A, B) of N2 == N3 and its shared memory fits.
// Returns false (and launches nothing) otherwise.  dry = true only checks availability.
template <typename T>
bool wide_pass_b(const lk::LocalArgs<T>& a, int A, int B, int nbands, cudaStream_t st, bool dry);

}  // namespace kss

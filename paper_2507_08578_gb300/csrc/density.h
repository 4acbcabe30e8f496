// Shared by the density build (density.cu) and the local passes (local_apply.cu).
#pragma once

#include <functional>

#include "local_kernels.cuh"

namespace kss {

// Pass A (sphere -> slab: scatter and inverse x transform) of nb bands of psi (band-major,
// leading dimension ld) in chunks that keep the slab L2-resident; after(a, m) is called once per
// chunk with a.work holding the slabs of bands a.n0 .. a.n0 + m - 1.  KSS_ENOTSUP for FFT
// lengths without a two-codelet split.
template <typename T>
void pass_a_chunks(kss_sys s, int ik, int nb, const void* psi, int ld,
                   const std::function<void(const lk::LocalArgs<T>&, int)>& after);

}  // namespace kss

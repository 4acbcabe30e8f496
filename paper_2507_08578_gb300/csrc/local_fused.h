// Host entry of the fused single-kernel local part for small cubic boxes (local_fused.cu).
#pragma once

#include "local_kernels.cuh"

namespace kss {

// Runs the local part of H (scatter, 3D FFTs, x V, gather and the epilogue of a) for `units` bands
// of a.psi, or band pairs when a.packed, in one persistent kernel per call.  Single precision,
// cubic boxes N1 = N2 = N3 with an instance (10, 12, 15, 16, 18, 20, 24, 25) whose box and
// potential fit in shared memory.  Returns false, launching nothing, otherwise.
bool fused_local_apply(kss_sys s, const lk::LocalArgs<float>& a, int units);

// True when fused_local_apply would run for this system's box.
bool fused_local_available(kss_sys s);

}  // namespace kss

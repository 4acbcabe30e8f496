// Host entry of the fused single-kernel local part for small cubic boxes (local_fused.cu).
#pragma once

#include "batch_kernels.cuh"

namespace kss {

// Runs the local part of H (scatter, 3D FFTs, x V, gather and the epilogue of a) for `units` bands
// of a.psi, or band pairs when a.packed, in one persistent kernel per call.  Single precision,
// cubic boxes N1 = N2 = N3 with an instance (10, 12, 15, 16, 18, 20, 24, 25) whose box and
// potential fit in shared memory.  Returns false, launching nothing, otherwise.
bool fused_local_apply(kss_sys s, const lk::LocalArgs<float>& a, int units);

// True when fused_local_apply would run for this system's box.
bool fused_local_available(kss_sys s);

// For the batch engine (grouped form, one persistent launch per box class):
// split code A*32+B of the system's fused instance, 0 when none;
int fused_code(kss_sys s);
// V/N^3 in the fused kernel's digit-reversed order (built on first use, kept with the system);
const float* fused_potential_view(kss_sys s);
// dynamic shared memory of the system's fused kernel;
size_t fused_smem_bytes(kss_sys s);
// the local part of all tasks of a class: items[i] (i < n) is a unit whose a.Vpi holds its
// fused_potential_view, a.nbands its band count, blk_ac its first task, tasks the total.
// fused_group_prepare (outside any stream capture: kernel attribute, error word) before the first
// fused_group_launch of a class.
void fused_group_prepare(kss_ctx ctx, int code, size_t smem);
void fused_group_launch(kss_ctx ctx, int code, const bk::LocalItem<float>* d_items, int n, int tasks, size_t smem);

}  // namespace kss

// Autotuner of the FFT pass-B schedule (tune.cu).
#pragma once

#include "local_kernels.cuh"

namespace kss {

// Pass-B schedule: the CTA-wide form with split N = A * B at `threads` threads per CTA, or the
// per-warp two-level form (threads == 0; A, B then give the cost-model split it uses).
struct PassBSched {
  int A = 0, B = 0, threads = 0;
  double ms = 0;  // measured time of one tuning launch (0 when not timed)
  int ncand = 0;  // candidates timed
};

// Schedule for the pass-B configuration of `a` (box N1 x N2 x N3, sphere window W2 x W3).
// From the process-wide table if present; else, when tuning is allowed (ctx->autotune, not inside
// a stream capture), by timing every candidate on a scratch slab; else the built-in choice (the
// CTA-wide form with the cost-model split at 384 threads when it exists, else the per-warp form).
// Candidates are timed at the window height rounded up to a multiple of 8, each launch sizing its
// shared memory from the arguments it is given (the per-warp form through warp_pass_b).
template <typename T>
PassBSched pass_b_schedule(kss_ctx ctx, const lk::LocalArgs<T>& a, const fftr::Split& s2, bool may_tune);

// The per-warp pass B (compile-time split when available) for args a over nbands bands on the
// context stream; used by the tuner as that form's timing (local_apply.cu).
template <typename T>
void warp_pass_b(kss_ctx ctx, const lk::LocalArgs<T>& a, int nbands);

}  // namespace kss

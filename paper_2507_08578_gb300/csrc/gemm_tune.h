// Autotuner of the schedule (kernel form and K-split) of the tensor-core GEMMs (gemm_tc.cu,
// gemm_oz.cu).
#pragma once

#include <functional>
#include <vector>

#include "kss_internal.h"

namespace kss {

// The tensor-core GEMM kinds with a tuned K-split.
enum GemmTuneKind { GT_BF16X3 = 0, GT_OZ77 = 1, GT_OZ77_C64OUT = 2, GT_OZ44 = 3 };

// A schedule of one product: the kernel form (kind-specific; 0 for the digit products, which have
// one form) and the K-split.
struct GemmChoice {
  int form, splits;
  bool operator==(const GemmChoice& o) const { return form == o.form && splits == o.splits; }
  bool operator<(const GemmChoice& o) const { return form != o.form ? form < o.form : splits < o.splits; }
};
// Schedule for a (kind, Mr, Nr, kb_total) product: the process-wide table entry if present; else,
// when tuning is allowed (ctx->autotune, not inside a stream capture), the fastest of `cand`, each
// timed by `run(choice)` (one warm-up and the fastest of three timed runs, CUDA events on the
// context stream); else `plan`.  The caller clamps a pinned entry to what its kernels accept.
GemmChoice tuned_gemm(kss_ctx ctx, int kind, int Mr, int Nr, int kb_total, std::vector<GemmChoice> cand,
                      GemmChoice plan, const std::function<void(GemmChoice)>& run);
// K-split for a (kind, Mr real rows, Nr columns, kb_total k-blocks) product: the process-wide table
// entry if present; else, when tuning is allowed (ctx->autotune, not inside a stream capture), the
// fastest of the candidates, each timed by `run(splits)` (which launches the product with that
// split into scratch outputs: one warm-up and the fastest of three timed runs, CUDA events on the
// context stream); else `plan` (the closed-form choice).  Candidates: the closed-form plan, no
// split, and the splits that fill the SMs in one, two or three waves, each keeping at least
// `min_kb` k-blocks per CTA.  Returns a split in [1, kb_total / min_kb] (at least 1).
int tuned_split(kss_ctx ctx, int kind, int Mr, int Nr, int kb_total, long long tiles, int min_kb, int plan,
                const std::function<void(int)>& run);
// Empty the K-split table (kss_autotune_clear).
void gemm_tune_clear();

}  // namespace kss

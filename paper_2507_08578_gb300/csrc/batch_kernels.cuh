// Grouped local-pass kernels of the batch engine (batch.cu): one launch covers the blocks of
// many (system, k-point) units, each block finding its unit by binary search over the item table.
#pragma once

#include "local_kernels.cuh"

namespace kss {
namespace bk {

using namespace lk;

template <typename T>
struct LocalItem {
  LocalArgs<T> a;
  RegPlan rp;
  int blk_ac;  // first block of this item in the pass A / pass C launches
  int blk_b;   // first block in the pass B launch
  int idle;    // unit past its own filter degree: its blocks return at once
};

template <typename T>
__device__ __forceinline__ int find_local(const LocalItem<T>* it, int n, int b, bool pb) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((pb ? it[mid].blk_b : it[mid].blk_ac) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T, int PASS, class Pol>
__global__ void __launch_bounds__(kThreads) group_pass(const LocalItem<T>* __restrict__ items, int n,
                                                       int scr_warp) {
  __shared__ LocalArgs<T> sa;
  __shared__ RegPlan srp;
  __shared__ int s_local, s_idle;
  if (threadIdx.x == 0) {
    const int i = find_local(items, n, blockIdx.x, PASS == 1);
    s_idle = items[i].idle;
    if (!s_idle) {
      sa = items[i].a;
      srp = items[i].rp;
    }
    s_local = blockIdx.x - (PASS == 1 ? items[i].blk_b : items[i].blk_ac);
  }
  __syncthreads();
  if (s_idle) return;
  const int local = s_local;
  if (PASS == 0) pass_a_body<T, Pol>(sa, srp, scr_warp, local % sa.W3, local / sa.W3);
  else if (PASS == 1) pass_b_body<T, Pol>(sa, srp, scr_warp, local % sa.N1, local / sa.N1);
  else pass_c_body<T, Pol>(sa, srp, scr_warp, local % sa.W3, local / sa.W3);
}

// Pass B of a class with a common compile-time y/z split, in the CTA-wide form.
template <typename T, int A, int B, int NT>
__global__ void __launch_bounds__(NT) group_passw(const LocalItem<T>* __restrict__ items, int n, int) {
  __shared__ LocalArgs<T> sa;
  __shared__ int s_local, s_idle;
  if (threadIdx.x == 0) {
    const int i = find_local(items, n, blockIdx.x, true);
    s_idle = items[i].idle;
    if (!s_idle) sa = items[i].a;
    s_local = blockIdx.x - items[i].blk_b;
  }
  __syncthreads();
  if (s_idle) return;
  const int local = s_local;
  pass_bw_body<T, A, B, NT>(sa, local % sa.N1, local / sa.N1);
}

template <typename T>
using GroupKernel = void (*)(const LocalItem<T>*, int, int);

// Grouped CTA-wide pass B for split (A, B) at nt threads (128 in single precision, 256 or 384);
// nullptr when no instance
// exists.  Instances live in batch_wide_f32.cu / batch_wide_f64.cu.
template <typename T>
GroupKernel<T> group_kernel_w(int A, int B, int nt);

}  // namespace bk
}  // namespace kss

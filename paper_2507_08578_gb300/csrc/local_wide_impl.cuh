// Kernel instances of the CTA-wide passes (local_kernels.cuh) for one precision: pass B
// (pass_bw_body) for every split of KSS_WIDE_SPLITS at 256 and 384 threads per CTA (and 128 in
// single precision), passes A and C (pass_aw_body, pass_cw_body) for the x splits of
// KSS_WIDEX_SPLITS.  Included by one translation unit per precision (local_wide_f32.cu,
// local_wide_f64.cu) so the build compiles them in parallel.
#pragma once

#include "local_kernels.cuh"
#include "local_wide.h"

namespace kss {
namespace wide_detail {

using namespace lk;

template <typename T, int A, int B, int NT, int CW = 0>
__global__ void __launch_bounds__(NT) pass_bw(LocalArgs<T> a) {
  pass_bw_body<T, A, B, NT, CW>(a, blockIdx.x, blockIdx.y);
}

// Splits with a pruned instance and its edge width: the 96-point splits, with the widths that the
// sphere window of a 96^3 box at a = 20 bohr, Ecut = 20 Ha (|m| <= 20 along y and z) needs; a
// window that needs no more than that width runs the pruned instance, any other the full one.
constexpr int pruned_cw(int A, int B) {
  return A == 8 && B == 12 ? 2 : A == 12 && B == 8 ? 3 : A == 6 && B == 16 ? 2 : A == 16 && B == 6 ? 4 : 0;
}

template <typename T, int A, int B, int NT>
bool launch_one(const LocalArgs<T>& a, int nbands, cudaStream_t st, bool dry) {
  const size_t sm = WideB<T, A, B>::smem(a.W3);
  if (sm > kWideSmemMax) return false;
  if (dry) return true;
  constexpr int PC = pruned_cw(A, B);
  if constexpr (PC > 0) {
    const int cw = wide_prune_cw(A, B, a.lo2, a.W2, a.lo3, a.W3);
    if (cw > 0 && cw <= PC) {
      KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_bw<T, A, B, NT, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      pass_bw<T, A, B, NT, PC><<<dim3(a.N1, nbands), NT, sm, st>>>(a);
      return true;
    }
  }
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_bw<T, A, B, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  pass_bw<T, A, B, NT><<<dim3(a.N1, nbands), NT, sm, st>>>(a);
  return true;
}

// 128-thread instances in single precision only: for the small boxes of batched systems a stage's
// tasks fill a 128-thread CTA better, and four-warp barriers idle fewer warps.
template <typename T, int A, int B>
bool launch_small(const LocalArgs<T>& a, int nbands, cudaStream_t st, bool dry) {
  if constexpr (sizeof(T) == 4) return launch_one<T, A, B, 128>(a, nbands, st, dry);
  else return false;
}

template <typename T>
bool dispatch(const LocalArgs<T>& a, int A, int B, int nt, int nbands, cudaStream_t st, bool dry) {
  if (a.N2 != a.N3 || A * B != a.N2 || (nt != 128 && nt != 256 && nt != 384)) return false;
  switch (A * 32 + B) {
#define KSS_CASE(x, y)                                                                \
  case x * 32 + y:                                                                    \
    return nt == 128   ? launch_small<T, x, y>(a, nbands, st, dry)                    \
           : nt == 256 ? launch_one<T, x, y, 256>(a, nbands, st, dry)                 \
                       : launch_one<T, x, y, 384>(a, nbands, st, dry);
    KSS_WIDE_SPLITS(KSS_CASE)
#undef KSS_CASE
    default:
      return false;
  }
}

// ---- passes A and C ----
// x splits with CTA-wide instances (N1 = A * B even) for pass A and for pass C, and the edge width
// of their pruned instances (the widths that the x window of the same sphere, |m| <= 20, needs).
// Each pass puts the stage with the twiddle multiply on the 8-point transforms (pass A inverts
// 8 x 12, pass C forwards 12 x 8): the 12-point stage then runs without the 11 twiddle values,
// which keeps double precision at 64 / 80 registers (three CTAs per SM).  The slab between the
// passes is in natural x order, so the two passes need not share a split.
#define KSS_WIDEX_SPLITS(X) X(8, 12, 12, 8)
constexpr int x_pruned_cw(int A, int B) { return A == 8 && B == 12 ? 2 : A == 12 && B == 8 ? 3 : 0; }
constexpr int kWideXThreads = 256;

template <typename T, int A, int B, int NT, int CW = 0>
__global__ void __launch_bounds__(NT) pass_aw(LocalArgs<T> a) {
  pass_aw_body<T, A, B, NT, CW>(a, blockIdx.x, blockIdx.y);
}
template <typename T, int A, int B, int NT, int CW = 0>
__global__ void __launch_bounds__(NT) pass_cw(LocalArgs<T> a) {
  pass_cw_body<T, A, B, NT, CW>(a, blockIdx.x, blockIdx.y);
}

template <typename T, int NT, class K>
void launch_x1(K kern, const LocalArgs<T>& a, size_t sm, int nbands, cudaStream_t st) {
  KSS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<dim3(a.W3, nbands), NT, sm, st>>>(a);
}

// which = 0: pass A (inverse transforms), 1: pass C (forward transforms)
template <typename T, int A, int B, int NT, int which>
bool launch_x(const LocalArgs<T>& a, int nbands, cudaStream_t st, bool dry) {
  using G = WideX<T, A, B>;
  if (a.N1p != G::P) return false;  // the tile index table's pitch
  const size_t sm = G::smem(a.W2);
  if (sm > kWideSmemMax) return false;
  if (dry) return true;
  constexpr int PC = x_pruned_cw(A, B);
  const bool pruned = PC > 0 && axis_prune_cw(B, a.lo1, a.W1) <= PC;
  if constexpr (which == 0) {
    if (pruned) launch_x1<T, NT>(pass_aw<T, A, B, NT, PC>, a, sm, nbands, st);
    else launch_x1<T, NT>(pass_aw<T, A, B, NT>, a, sm, nbands, st);
  } else {
    if (pruned) launch_x1<T, NT>(pass_cw<T, A, B, NT, PC>, a, sm, nbands, st);
    else launch_x1<T, NT>(pass_cw<T, A, B, NT>, a, sm, nbands, st);
  }
  return true;
}

template <typename T>
bool dispatch_x(const LocalArgs<T>& a, int which, int nbands, cudaStream_t st, bool dry) {
  switch (a.N1) {
#define KSS_CASE(xa, ya, xc, yc)                                                           \
  case xa * ya:                                                                            \
    static_assert(xa * ya == xc * yc, "passes A and C split the same length");            \
    return which == 0 ? launch_x<T, xa, ya, kWideXThreads, 0>(a, nbands, st, dry)          \
                      : launch_x<T, xc, yc, kWideXThreads, 1>(a, nbands, st, dry);
    KSS_WIDEX_SPLITS(KSS_CASE)
#undef KSS_CASE
    default:
      return false;
  }
}

}  // namespace wide_detail
}  // namespace kss

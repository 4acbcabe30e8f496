// Complex GEMMs on the CUDA cores (FP64 and FP32), for the shapes of the eigensolver:
//   gemm_cn: C = alpha A^H B + beta C   (projector coefficients beta^H psi, Gram and projected-H
//            matrices Y^H Y, Y^H HY; K = npw is long, so K is split across CTAs and the partial
//            sums are reduced in a fixed order, which keeps results bitwise reproducible)
//   gemm_nn: C = alpha A B + beta C     (nonlocal accumulation beta C', subspace rotations Y Q)
// All matrices are column-major; a band block [nb][ld] is an npw x nb matrix with leading
// dimension ld.  On GB300 the FP64 pipe (about 1.2 TFLOP/s) bounds these kernels long before
// shared memory or HBM does; the FP32 instantiation is the CUDA-core form of the mixed path.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>

#include "kss_internal.h"

namespace kss {

namespace {

constexpr int BM = 64, BN = 64, BK = 8;

template <typename T> struct CT;
template <> struct CT<double> { using C = double2; };
template <> struct CT<float> { using C = float2; };

// Complex multiply-accumulate.  FP64 uses the three-multiplication (Gauss) form with the operand
// sums formed once per staged element: for p = x + iy (from A) and q = u + iv (from B),
//   k1 = u (x + y),  k2 = x (v - u),  k3 = y (u + v);   Re pq = k1 - k3,  Im pq = k1 + k2,
// so each complex term costs three fused multiply-adds instead of four (the FP64 pipe bounds
// these GEMMs; the rounding error stays a small multiple of eps * sum |p||q|).  FP32 keeps the
// four-multiplication form, whose error bound is tighter, for the mixed path's Gram matrices.
template <typename T>
struct Cmac {
  static constexpr bool G = sizeof(T) == 8;
  static constexpr int NS = G ? 3 : 2;  // staged values per element and accumulators per output
  // staged values of p = x + iy (A side) and q = u + iv (B side)
  static __device__ __forceinline__ void stage_a(T (*dst)[BK][BM], int k, int i, T x, T y) {
    if constexpr (G) {
      dst[0][k][i] = x + y;
      dst[1][k][i] = x;
      dst[2][k][i] = y;
    } else {
      dst[0][k][i] = x;
      dst[1][k][i] = y;
    }
  }
  static __device__ __forceinline__ void stage_b(T (*dst)[BK][BN], int k, int j, T u, T v) {
    if constexpr (G) {
      dst[0][k][j] = u;
      dst[1][k][j] = v - u;
      dst[2][k][j] = u + v;
    } else {
      dst[0][k][j] = u;
      dst[1][k][j] = v;
    }
  }
  static __device__ __forceinline__ void mac(T (&acc)[NS], const T (&a)[NS], const T (&b)[NS]) {
    if constexpr (G) {
      acc[0] = fma(a[0], b[0], acc[0]);
      acc[1] = fma(a[1], b[1], acc[1]);
      acc[2] = fma(a[2], b[2], acc[2]);
    } else {
      acc[0] = fma(a[0], b[0], acc[0]);
      acc[0] = fma(-a[1], b[1], acc[0]);
      acc[1] = fma(a[0], b[1], acc[1]);
      acc[1] = fma(a[1], b[0], acc[1]);
    }
  }
  static __device__ __forceinline__ T re(const T (&acc)[NS]) {
    if constexpr (G) return acc[0] - acc[2];
    else return acc[0];
  }
  static __device__ __forceinline__ T im(const T (&acc)[NS]) {
    if constexpr (G) return acc[0] + acc[1];
    else return acc[1];
  }
};

// Inputs of type TI (complex64 or complex128), accumulation and partial sums in T.  The next
// K tile is fetched into registers while the current one is multiplied.
template <typename T, typename TI = T>
__device__ __forceinline__ void cn_partial_body(int M, int N, int K, const typename CT<TI>::C* __restrict__ A,
                                                long long lda, const typename CT<TI>::C* __restrict__ B,
                                                long long ldb, typename CT<T>::C* __restrict__ P,
                                                int kchunk, int bx, int by, int bz) {
  using C = typename CT<T>::C;
  using CI = typename CT<TI>::C;
  using X = Cmac<T>;
  constexpr int NS = X::NS;
  __shared__ T As[NS][BK][BM];
  __shared__ T Bs[NS][BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = bx * BM, j0 = by * BN;
  const int kbeg = bz * kchunk;
  const int kend = min(K, kbeg + kchunk);
  T acc[4][4][NS];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < NS; ++q) acc[r][c][q] = 0;
  const int li = tid >> 2, lk = (tid & 3) * 2;
  const int gi = i0 + li, gj = j0 + li;
  CI ra[2], rb[2];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = k0 + lk + e;
      ra[e] = (k < kend && gi < M) ? A[gi * lda + k] : CI{0, 0};
      rb[e] = (k < kend && gj < N) ? B[gj * ldb + k] : CI{0, 0};
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      X::stage_a(As, lk + e, li, (T)ra[e].x, -(T)ra[e].y);  // conj(a)
      X::stage_b(Bs, lk + e, li, (T)rb[e].x, (T)rb[e].y);
    }
    __syncthreads();
    if (k0 + BK < kend) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4][NS], bv[4][NS];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < NS; ++q) av[r][q] = As[q][kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int q = 0; q < NS; ++q) bv[c][q] = Bs[q][kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) X::mac(acc[r][c], av[r], bv[c]);
    }
    __syncthreads();
  }
  C* Pz = P + (size_t)bz * M * N;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
      if (i < M && j < N) Pz[(size_t)j * M + i] = C{X::re(acc[r][c]), X::im(acc[r][c])};
    }
}

template <typename T>
__global__ void __launch_bounds__(256) gemm_cn_partial(int M, int N, int K, const typename CT<T>::C* __restrict__ A,
                                                       long long lda, const typename CT<T>::C* __restrict__ B,
                                                       long long ldb, typename CT<T>::C* __restrict__ P,
                                                       int kchunk) {
  cn_partial_body<T>(M, N, K, A, lda, B, ldb, P, kchunk, blockIdx.x, blockIdx.y, blockIdx.z);
}

// complex64 inputs, FP64 accumulation (Gram matrices of ill-conditioned complex64 blocks)
__global__ void __launch_bounds__(256) gemm_cn_partial_f32in(int M, int N, int K, const float2* __restrict__ A,
                                                             long long lda, const float2* __restrict__ B,
                                                             long long ldb, double2* __restrict__ P, int kchunk) {
  cn_partial_body<double, float>(M, N, K, A, lda, B, ldb, P, kchunk, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Lower-triangle form for Hermitian products C = A^H B (M x M): block t of the grid's x
// dimension is tile (bx, by) with bx >= by (row-major over the lower triangle of tiles).
__device__ __forceinline__ void lower_tile(int t, int& bx, int& by) {
  int r = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  bx = r;
  by = t - r * (r + 1) / 2;
}

template <typename T, typename TI>
__global__ void __launch_bounds__(256) gemm_cn_partial_lower(int M, int K, const typename CT<TI>::C* __restrict__ A,
                                                             long long lda, const typename CT<TI>::C* __restrict__ B,
                                                             long long ldb, typename CT<T>::C* __restrict__ P,
                                                             int kchunk) {
  int bx, by;
  lower_tile(blockIdx.x, bx, by);
  cn_partial_body<T, TI>(M, M, K, A, lda, B, ldb, P, kchunk, bx, by, blockIdx.z);
}

// Sum of the partials on and below the diagonal tiles; strictly upper tiles of C are set to 0.
template <typename T>
__global__ void gemm_reduce_lower(int M, int nsplit, const typename CT<T>::C* __restrict__ P,
                                  typename CT<T>::C* __restrict__ Cm, long long ldc) {
  using C = typename CT<T>::C;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)M * M) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  C out = {0, 0};
  if (i / BM >= j / BN) {
    for (int z = 0; z < nsplit; ++z) {
      const C p = P[(size_t)z * M * M + idx];
      out.x += p.x;
      out.y += p.y;
    }
  }
  Cm[(size_t)j * ldc + i] = out;
}

template <typename T>
__global__ void gemm_reduce(int M, int N, int nsplit, const typename CT<T>::C* __restrict__ P,
                            typename CT<T>::C* __restrict__ Cm, long long ldc, T ar, T ai, T br,
                            T bi) {
  using C = typename CT<T>::C;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  T sr = 0, si = 0;
  for (int z = 0; z < nsplit; ++z) {
    const C p = P[(size_t)z * M * N + idx];
    sr += p.x;
    si += p.y;
  }
  C out;
  out.x = ar * sr - ai * si;
  out.y = ar * si + ai * sr;
  C* dst = Cm + (size_t)j * ldc + i;
  if (br != 0 || bi != 0) {
    const C o = *dst;
    out.x += br * o.x - bi * o.y;
    out.y += br * o.y + bi * o.x;
  }
  *dst = out;
}

template <typename T>
__device__ __forceinline__ void nn_body(int M, int N, int K, const typename CT<T>::C* __restrict__ A,
                                        long long lda, const typename CT<T>::C* __restrict__ B,
                                        long long ldb, typename CT<T>::C* __restrict__ Cm,
                                        long long ldc, T ar, T ai, T br, T bi, int bx, int by) {
  using C = typename CT<T>::C;
  using X = Cmac<T>;
  constexpr int NS = X::NS;
  __shared__ T As[NS][BK][BM];
  __shared__ T Bs[NS][BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = bx * BM, j0 = by * BN;
  T acc[4][4][NS];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < NS; ++q) acc[r][c][q] = 0;
  const int ai_ = tid & 63, ak = tid >> 6;           // A tile: i fastest
  const int bj = tid >> 2, bk = (tid & 3) * 2;       // B tile: k fastest
  const int gi = i0 + ai_, gj = j0 + bj;
  C ra[2], rb[2];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int ka = k0 + ak + 4 * e, kb = k0 + bk + e;
      ra[e] = (ka < K && gi < M) ? A[(size_t)ka * lda + gi] : C{0, 0};
      rb[e] = (kb < K && gj < N) ? B[(size_t)gj * ldb + kb] : C{0, 0};
    }
  };
  if (K > 0) fetch(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      X::stage_a(As, ak + 4 * e, ai_, ra[e].x, ra[e].y);
      X::stage_b(Bs, bk + e, bj, rb[e].x, rb[e].y);
    }
    __syncthreads();
    if (k0 + BK < K) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[4][NS], bv[4][NS];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < NS; ++q) av[r][q] = As[q][kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int q = 0; q < NS; ++q) bv[c][q] = Bs[q][kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) X::mac(acc[r][c], av[r], bv[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = i0 + tx + 16 * r, j = j0 + ty + 16 * c;
      if (i < M && j < N) {
        C* dst = Cm + (size_t)j * ldc + i;
        const T sr = X::re(acc[r][c]), si = X::im(acc[r][c]);
        C out;
        out.x = ar * sr - ai * si;
        out.y = ar * si + ai * sr;
        if (br != 0 || bi != 0) {
          const C o = *dst;
          out.x += br * o.x - bi * o.y;
          out.y += br * o.y + bi * o.x;
        }
        *dst = out;
      }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) gemm_nn_kernel(int M, int N, int K, const typename CT<T>::C* __restrict__ A,
                                                      long long lda, const typename CT<T>::C* __restrict__ B,
                                                      long long ldb, typename CT<T>::C* __restrict__ Cm,
                                                      long long ldc, T ar, T ai, T br, T bi) {
  nn_body<T>(M, N, K, A, lda, B, ldb, Cm, ldc, ar, ai, br, bi, blockIdx.x, blockIdx.y);
}

// ---- grouped forms: one launch over many independent products (batched solves) ------------
__device__ __forceinline__ int find_item(const GemmItem* it, int n, int b, bool reduce) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((reduce ? it[mid].rblk0 : it[mid].blk0) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) gg_cn_partial(const GemmItem* __restrict__ items, int n) {
  using C = typename CT<T>::C;
  const int i = find_item(items, n, blockIdx.x, false);
  const GemmItem& g = items[i];
  if (g.idle) return;
  const int local = blockIdx.x - g.blk0;
  const int per = g.tm * g.tn;
  const int bz = local / per, r = local - bz * per;
  cn_partial_body<T>(g.M, g.N, g.K, (const C*)g.A, g.lda, (const C*)g.B, g.ldb, (C*)g.P, g.kchunk,
                     r % g.tm, r / g.tm, bz);
}

template <typename T>
__global__ void gg_reduce(const GemmItem* __restrict__ items, int n) {
  using C = typename CT<T>::C;
  const int it = find_item(items, n, blockIdx.x, true);
  const GemmItem& g = items[it];
  if (g.idle) return;
  const long long idx = (long long)(blockIdx.x - g.rblk0) * blockDim.x + threadIdx.x;
  if (idx >= (long long)g.M * g.N) return;
  const int i = (int)(idx % g.M), j = (int)(idx / g.M);
  T sr = 0, si = 0;
  const C* P = (const C*)g.P;
  for (int z = 0; z < g.splits; ++z) {
    const C p = P[(size_t)z * g.M * g.N + idx];
    sr += p.x;
    si += p.y;
  }
  // C = s * D * (sum), the nonlocal scaling alpha * D folded in (D may be null: plain product)
  const T f = g.d ? (T)(((const T*)g.d)[i] * (T)g.s) : (T)1;
  C out;
  out.x = f * sr;
  out.y = f * si;
  ((C*)g.C)[(size_t)j * g.ldc + i] = out;
}

// The same reduction for complex64 products delivered in complex128 (the batched Gram matrices of
// the mixed form): the FP32 partial sums of each K chunk added in FP64.
__global__ void gg_reduce_c64_to_c128(const GemmItem* __restrict__ items, int n) {
  const int it = find_item(items, n, blockIdx.x, true);
  const GemmItem& g = items[it];
  if (g.idle) return;
  const long long idx = (long long)(blockIdx.x - g.rblk0) * blockDim.x + threadIdx.x;
  if (idx >= (long long)g.M * g.N) return;
  const int i = (int)(idx % g.M), j = (int)(idx / g.M);
  double sr = 0, si = 0;
  const float2* P = (const float2*)g.P;
  for (int z = 0; z < g.splits; ++z) {
    const float2 p = P[(size_t)z * g.M * g.N + idx];
    sr += p.x;
    si += p.y;
  }
  ((double2*)g.C)[(size_t)j * g.ldc + i] = make_double2(sr, si);
}

template <typename T>
__global__ void __launch_bounds__(256) gg_nn(const GemmItem* __restrict__ items, int n) {
  using C = typename CT<T>::C;
  const int i = find_item(items, n, blockIdx.x, false);
  const GemmItem& g = items[i];
  if (g.idle) return;
  const int local = blockIdx.x - g.blk0;
  nn_body<T>(g.M, g.N, g.K, (const C*)g.A, g.lda, (const C*)g.B, g.ldb, (C*)g.C, g.ldc, (T)g.ar,
             (T)0, (T)g.br, (T)0, local % g.tm, local / g.tm);
}

template <typename T>
__global__ void scale_rows_kernel(int M, int N, typename CT<T>::C* __restrict__ Cm, long long ldc,
                                  const T* __restrict__ d, T s) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  const T f = d[i] * s;
  typename CT<T>::C& e = Cm[(size_t)j * ldc + i];
  e.x *= f;
  e.y *= f;
}

int sm_count(kss_ctx ctx) {
  if (!ctx->nsm) {  // normally set when the context is created
    int v = 0;
    KSS_CHECK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device));
    ctx->nsm = v > 0 ? v : 1;
  }
  return ctx->nsm;
}

// Resident CTAs per SM of a 256-thread kernel without dynamic shared memory.
template <class F>
int resident_ctas(F f) {
  static std::mutex mu;
  static std::map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find((const void*)f);
  if (it != cache.end()) return it->second;
  int b = 0;
  KSS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, 256, 0));
  b = std::max(b, 1);
  cache[(const void*)f] = b;
  return b;
}

// Split count s of a split-K product over `tiles` output tiles: the smallest s <= smax that
// minimises the wave-quantised time ceil(tiles * s / cap) / s (cap = resident CTAs on the GPU),
// with at least 64 K values per split.
int pick_splits(int tiles, int K, int cap, int smax) {
  smax = std::max(1, std::min(smax, (K + 63) / 64));
  int best = 1;
  double bt = 1e300;
  for (int s = 1; s <= smax; ++s) {
    const double t = (double)((tiles * (long long)s + cap - 1) / cap) / s;
    if (t < bt * (1.0 - 1e-9)) {
      bt = t;
      best = s;
    }
  }
  return best;
}

// Splits, K chunk (a multiple of BK) and partial-sum count for a split-K launch.
struct SplitK {
  int splits, kchunk;
};
template <class F>
SplitK plan_splitk(kss_ctx ctx, F kernel, int tiles, int K, size_t partial_bytes_each, size_t max_bytes) {
  const int cap = sm_count(ctx) * resident_ctas(kernel);
  const int smax = (int)std::max<size_t>(1, std::min<size_t>(128, max_bytes / partial_bytes_each));
  int splits = pick_splits(tiles, K, cap, smax);
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = (K + kchunk - 1) / kchunk;
  return {splits, kchunk};
}

int tag_id(const char* kernel, bool f64, const char* tag) {
  std::string n = std::string(kernel) + (f64 ? "<f64>:" : "<f32>:") + (tag ? tag : "");
  return prof_register(n.c_str());
}

template <typename T>
void run_cn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
            void* Cm, int ldc, double ar, double ai, double br, double bi, const char* tag) {
  using C = typename CT<T>::C;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const SplitK sk = plan_splitk(ctx, gemm_cn_partial<T>, tm * tn, K, (size_t)M * N * sizeof(C), 512ull << 20);
  const int splits = sk.splits, kchunk = sk.kchunk;
  ctx->ws_gemm.ensure((size_t)splits * M * N * sizeof(C));
  const bool f64 = sizeof(T) == 8;
  {
    ProfScope ps(ctx, tag_id("gemm_cn_partial", f64, tag));
    gemm_cn_partial<T><<<dim3(tm, tn, splits), 256, 0, ctx->stream>>>(
        M, N, K, (const C*)A, lda, (const C*)B, ldb, ctx->ws_gemm.as<C>(), kchunk);
  }
  const long long mn = (long long)M * N;
  {
    ProfScope ps(ctx, tag_id("gemm_reduce", f64, tag));
    gemm_reduce<T><<<(unsigned)((mn + 255) / 256), 256, 0, ctx->stream>>>(
        M, N, splits, ctx->ws_gemm.as<C>(), (C*)Cm, ldc, (T)ar, (T)ai, (T)br, (T)bi);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

template <typename T>
void run_nn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
            void* Cm, int ldc, double ar, double ai, double br, double bi, const char* tag) {
  using C = typename CT<T>::C;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  ProfScope ps(ctx, tag_id("gemm_nn", sizeof(T) == 8, tag));
  gemm_nn_kernel<T><<<dim3(tm, tn), 256, 0, ctx->stream>>>(M, N, K, (const C*)A, lda, (const C*)B,
                                                           ldb, (C*)Cm, ldc, (T)ar, (T)ai, (T)br, (T)bi);
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

void gemm_cn(kss_ctx ctx, bool fp64, int M, int N, int K, const void* A, int lda, const void* B,
             int ldb, void* C, int ldc, double ar, double ai, double br, double bi, const char* tag) {
  if (M <= 0 || N <= 0) return;
  KSS_REQUIRE(K >= 0 && lda >= K && ldb >= K && ldc >= M, "gemm_cn: bad leading dimension");
  if (K == 0) {
    // C = beta C
    KSS_REQUIRE(br == 0 && bi == 0, "gemm_cn: K == 0 with beta != 0 is not supported");
    const size_t es = fp64 ? 16 : 8;
    KSS_CHECK_CUDA(cudaMemset2DAsync(C, (size_t)ldc * es, 0, (size_t)M * es, N, ctx->stream));
    return;
  }
  if (fp64) run_cn<double>(ctx, M, N, K, A, lda, B, ldb, C, ldc, ar, ai, br, bi, tag);
  else run_cn<float>(ctx, M, N, K, A, lda, B, ldb, C, ldc, ar, ai, br, bi, tag);
}

// C (complex128, M x N) = A^H B for complex64 A (K x M) and B (K x N), accumulated in FP64.
void gemm_cn_c64_acc64(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B,
                       int ldb, void* C, int ldc, const char* tag) {
  if (M <= 0 || N <= 0) return;
  KSS_REQUIRE(K > 0 && lda >= K && ldb >= K && ldc >= M, "gemm_cn_c64_acc64: bad leading dimension");
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const SplitK sk = plan_splitk(ctx, gemm_cn_partial_f32in, tm * tn, K, (size_t)M * N * sizeof(double2),
                                512ull << 20);
  const int splits = sk.splits, kchunk = sk.kchunk;
  ctx->ws_gemm.ensure((size_t)splits * M * N * sizeof(double2));
  {
    ProfScope ps(ctx, tag_id("gemm_cn_partial_c64in", true, tag));
    gemm_cn_partial_f32in<<<dim3(tm, tn, splits), 256, 0, ctx->stream>>>(
        M, N, K, (const float2*)A, lda, (const float2*)B, ldb, ctx->ws_gemm.as<double2>(), kchunk);
  }
  const long long mn = (long long)M * N;
  {
    ProfScope ps(ctx, tag_id("gemm_reduce", true, tag));
    gemm_reduce<double><<<(unsigned)((mn + 255) / 256), 256, 0, ctx->stream>>>(
        M, N, splits, ctx->ws_gemm.as<double2>(), (double2*)C, ldc, 1.0, 0.0, 0.0, 0.0);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

// Lower triangle (tiles on or below the diagonal) of a Hermitian product C = A^H B, M x M, with
// A and B K x M of element type TI (complex64 / complex128) and accumulation in T; the strictly
// upper tiles of C are zeroed.  For Gram matrices read through one triangle by the eigensolver.
template <typename T, typename TI>
void run_cn_lower(kss_ctx ctx, int M, int K, const void* A, int lda, const void* B, int ldb, void* Cm,
                  int ldc, const char* name, const char* tag) {
  using C = typename CT<T>::C;
  using CI = typename CT<TI>::C;
  const int tm = (M + BM - 1) / BM;
  const int tiles = tm * (tm + 1) / 2;
  const SplitK sk = plan_splitk(ctx, gemm_cn_partial_lower<T, TI>, tiles, K, (size_t)M * M * sizeof(C), 512ull << 20);
  ctx->ws_gemm.ensure((size_t)sk.splits * M * M * sizeof(C));
  const bool f64 = sizeof(T) == 8;
  {
    ProfScope ps(ctx, tag_id(name, f64, tag));
    gemm_cn_partial_lower<T, TI><<<dim3(tiles, 1, sk.splits), 256, 0, ctx->stream>>>(
        M, K, (const CI*)A, lda, (const CI*)B, ldb, ctx->ws_gemm.as<C>(), sk.kchunk);
  }
  const long long mm = (long long)M * M;
  {
    ProfScope ps(ctx, tag_id("gemm_reduce", f64, tag));
    gemm_reduce_lower<T><<<(unsigned)((mm + 255) / 256), 256, 0, ctx->stream>>>(M, sk.splits, ctx->ws_gemm.as<C>(),
                                                                              (C*)Cm, ldc);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

void gemm_cn_lower(kss_ctx ctx, bool fp64, int M, int K, const void* A, int lda, const void* B, int ldb,
                   void* C, int ldc, const char* tag) {
  if (M <= 0) return;
  KSS_REQUIRE(K > 0 && lda >= K && ldb >= K && ldc >= M, "gemm_cn_lower: bad size");
  if (fp64) run_cn_lower<double, double>(ctx, M, K, A, lda, B, ldb, C, ldc, "gemm_cn_partial", tag);
  else run_cn_lower<float, float>(ctx, M, K, A, lda, B, ldb, C, ldc, "gemm_cn_partial", tag);
}

void gemm_cn_c64_acc64_lower(kss_ctx ctx, int M, int K, const void* A, int lda, const void* B, int ldb,
                             void* C, int ldc, const char* tag) {
  if (M <= 0) return;
  KSS_REQUIRE(K > 0 && lda >= K && ldb >= K && ldc >= M, "gemm_cn_c64_acc64_lower: bad size");
  run_cn_lower<double, float>(ctx, M, K, A, lda, B, ldb, C, ldc, "gemm_cn_partial_c64in", tag);
}

// gemm_cn with a caller-provided partial-sum buffer (no allocation, no profiling events): the
// K split is limited to what fits in partial_bytes.  Returns false if even one split does not fit.
bool gemm_cn_ws(kss_ctx ctx, bool fp64, int M, int N, int K, const void* A, int lda, const void* B,
                int ldb, void* C, int ldc, void* partials, size_t partial_bytes) {
  if (M <= 0 || N <= 0) return true;
  KSS_REQUIRE(K > 0 && lda >= K && ldb >= K && ldc >= M, "gemm_cn_ws: bad size");
  const size_t es = fp64 ? 16 : 8;
  const size_t per = (size_t)M * N * es;
  const int maxs = (int)std::min<size_t>(partial_bytes / per, 1 << 20);
  if (maxs < 1) return false;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const SplitK sk = fp64 ? plan_splitk(ctx, gemm_cn_partial<double>, tm * tn, K, per, (size_t)maxs * per)
                         : plan_splitk(ctx, gemm_cn_partial<float>, tm * tn, K, per, (size_t)maxs * per);
  const int splits = sk.splits, kchunk = sk.kchunk;
  const long long mn = (long long)M * N;
  if (fp64) {
    gemm_cn_partial<double><<<dim3(tm, tn, splits), 256, 0, ctx->stream>>>(
        M, N, K, (const double2*)A, lda, (const double2*)B, ldb, (double2*)partials, kchunk);
    gemm_reduce<double><<<(unsigned)((mn + 255) / 256), 256, 0, ctx->stream>>>(
        M, N, splits, (const double2*)partials, (double2*)C, ldc, 1.0, 0.0, 0.0, 0.0);
  } else {
    gemm_cn_partial<float><<<dim3(tm, tn, splits), 256, 0, ctx->stream>>>(
        M, N, K, (const float2*)A, lda, (const float2*)B, ldb, (float2*)partials, kchunk);
    gemm_reduce<float><<<(unsigned)((mn + 255) / 256), 256, 0, ctx->stream>>>(
        M, N, splits, (const float2*)partials, (float2*)C, ldc, 1.f, 0.f, 0.f, 0.f);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
  return true;
}

void scale_rows_noprof(bool fp64, int M, int N, void* C, int ldc, const void* d, double s,
                       cudaStream_t st) {
  const long long mn = (long long)M * N;
  if (!mn) return;
  if (fp64)
    scale_rows_kernel<double><<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(M, N, (double2*)C, ldc,
                                                                            (const double*)d, s);
  else
    scale_rows_kernel<float><<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(M, N, (float2*)C, ldc,
                                                                          (const float*)d, (float)s);
  KSS_CHECK_CUDA(cudaGetLastError());
}

void gemm_nn_noprof(bool fp64, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                    void* C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  const int tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  if (fp64)
    gemm_nn_kernel<double><<<dim3(tm, tn), 256, 0, st>>>(M, N, K, (const double2*)A, lda, (const double2*)B,
                                                         ldb, (double2*)C, ldc, 1.0, 0.0, 1.0, 0.0);
  else
    gemm_nn_kernel<float><<<dim3(tm, tn), 256, 0, st>>>(M, N, K, (const float2*)A, lda, (const float2*)B,
                                                        ldb, (float2*)C, ldc, 1.f, 0.f, 1.f, 0.f);
  KSS_CHECK_CUDA(cudaGetLastError());
}

// Fill the launch bookkeeping of grouped items (tiles, splits, block offsets) and return the
// block counts of the partial/product and reduce launches.
void group_plan(kss_ctx ctx, std::vector<GemmItem>& items, bool cn, int* blocks, int* rblocks) {
  int b = 0, rb = 0;
  for (auto& g : items) {
    g.tm = (g.M + BM - 1) / BM;
    g.tn = (g.N + BN - 1) / BN;
    g.blk0 = b;
    g.rblk0 = rb;
    if (cn) {
      g.splits = std::max(1, std::min(16, (g.K + 2047) / 2048));
      g.kchunk = ((g.K + g.splits - 1) / g.splits + BK - 1) / BK * BK;
      g.splits = (g.K + g.kchunk - 1) / g.kchunk;
      b += g.tm * g.tn * g.splits;
      rb += (int)(((long long)g.M * g.N + 255) / 256);
    } else {
      g.splits = 1;
      b += g.tm * g.tn;
    }
  }
  *blocks = b;
  *rblocks = rb;
}

void group_gemm_cn(kss_ctx ctx, bool fp64, const GemmItem* d_items, int n, int blocks, int rblocks) {
  if (!n || !blocks) return;
  static const int idp = prof_register("group_gemm_cn_partial"), idr = prof_register("group_gemm_reduce");
  {
    ProfScope ps(ctx, idp);
    if (fp64) gg_cn_partial<double><<<blocks, 256, 0, ctx->stream>>>(d_items, n);
    else gg_cn_partial<float><<<blocks, 256, 0, ctx->stream>>>(d_items, n);
  }
  {
    ProfScope ps(ctx, idr);
    if (fp64) gg_reduce<double><<<rblocks, 256, 0, ctx->stream>>>(d_items, n);
    else gg_reduce<float><<<rblocks, 256, 0, ctx->stream>>>(d_items, n);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

void group_gemm_cn_c64_to_c128(kss_ctx ctx, const GemmItem* d_items, int n, int blocks, int rblocks) {
  if (!n || !blocks) return;
  static const int idp = prof_register("group_gemm_cn_partial:gram"), idr = prof_register("group_reduce64:gram");
  {
    ProfScope ps(ctx, idp);
    gg_cn_partial<float><<<blocks, 256, 0, ctx->stream>>>(d_items, n);
  }
  {
    ProfScope ps(ctx, idr);
    gg_reduce_c64_to_c128<<<rblocks, 256, 0, ctx->stream>>>(d_items, n);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

void group_gemm_nn(kss_ctx ctx, bool fp64, const GemmItem* d_items, int n, int blocks) {
  if (!n || !blocks) return;
  static const int id = prof_register("group_gemm_nn");
  ProfScope ps(ctx, id);
  if (fp64) gg_nn<double><<<blocks, 256, 0, ctx->stream>>>(d_items, n);
  else gg_nn<float><<<blocks, 256, 0, ctx->stream>>>(d_items, n);
  KSS_CHECK_CUDA(cudaGetLastError());
}

void gemm_nn(kss_ctx ctx, bool fp64, int M, int N, int K, const void* A, int lda, const void* B,
             int ldb, void* C, int ldc, double ar, double ai, double br, double bi, const char* tag) {
  if (M <= 0 || N <= 0) return;
  KSS_REQUIRE(K >= 0 && lda >= M && ldb >= K && ldc >= M, "gemm_nn: bad leading dimension");
  if (fp64) run_nn<double>(ctx, M, N, K, A, lda, B, ldb, C, ldc, ar, ai, br, bi, tag);
  else run_nn<float>(ctx, M, N, K, A, lda, B, ldb, C, ldc, ar, ai, br, bi, tag);
}

void scale_rows(kss_ctx ctx, bool fp64, int M, int N, void* C, int ldc, const void* d, double s) {
  const long long mn = (long long)M * N;
  if (!mn) return;
  cudaStream_t st = ctx->stream;
  static const int id = prof_register("scale_rows");
  ProfScope ps(ctx, id);
  if (fp64)
    scale_rows_kernel<double><<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(M, N, (double2*)C, ldc,
                                                                            (const double*)d, s);
  else
    scale_rows_kernel<float><<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(M, N, (float2*)C, ldc,
                                                                          (const float*)d, (float)s);
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace kss

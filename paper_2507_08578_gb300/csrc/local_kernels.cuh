// Shared device code of the local-potential passes (register-codelet form): argument block,
// two-level pencil transforms and the bodies of passes A, B and C.  Included by the per-system
// launcher (local_apply.cu) and by the grouped multi-system launcher (batch.cu).
#pragma once

#include <algorithm>

#include "fft_reg.cuh"
#include "kss_internal.h"

namespace kss {
namespace lk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename T> struct CT;
template <> struct CT<double> { using C = double2; };
template <> struct CT<float> { using C = float2; };


template <typename T>
struct LocalArgs {
  using C = typename CT<T>::C;
  int N1, N2, N3, N1p, N2p, N3p;
  int W2, W3, lo2, lo3;
  int W1, lo1;    // the sphere's x window (0, 0 when unknown: no pruning of the x transforms)
  FftDim d1, d2, d3;
  int pw1, pw2, pw3;  // pencils per warp call along x, y, z
  const C* tw1;
  const C* tw2;
  const C* tw3;
  const int* zstart;
  const int* rowrange;
  const int* tileidx;
  const T* kin;
  const T* Vx;
  const T* Vpi;   // CTA-wide pass B: V/N^3 as [x][z][p], p the y position of the stages' digit-reversed
                  // order for the split in use (so the middle z stage reads it coalesced)
  const C* psi;
  const C* psi_prev;
  C* out;
  long long ld;
  C* work;  // [nc][N1][W3][W2]
  int n0;
  T alpha, beta, gamma;
  const T* coef;  // when set: alpha, beta, gamma read from device memory (graph replays)
  int packed;     // Gamma point: "band" n of the passes is the pair (2n, 2n+1) packed as
                  // psi_2n + i psi_2n+1 (real-space-real bands); pass C then stores the raw
                  // transform (no epilogue) and a separate kernel unpacks
  int nbands;     // bands in psi (packed mode: the last pair may hold one band)
};

template <typename C>
__device__ __forceinline__ void copy_table(C* dst, const C* src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// ---------------------------------------------------------------------------------------------
// Register-codelet form of the three passes (two-level pencil FFTs, see fft_reg.cuh).
// ---------------------------------------------------------------------------------------------
using fftr::Split;
using fftr::kMaxR;

struct RegPlan {
  Split s1, s2, s3;  // x, y, z
};

// Transform np (<= sp.PP) pencils with one warp.  in(p, e) returns element e of pencil p, out(p,
// e, v) receives output element e.  s = +1 inverse, -1 forward.  scr: sp.PP * sp.scr elements.
template <typename C, typename T, class In, class Out>
__device__ __forceinline__ void pencil_fft_rt(const Split& sp, int np, const C* tw, T s, C* scr,
                                           int lane, In in, Out out) {
  const int p = lane / sp.L, r = lane - p * sp.L;
  const bool act = p < np;
  C* sc = scr + p * sp.scr;
  C v[kMaxR];
  if (act && r < sp.B) {
#pragma unroll
    for (int i = 0; i < kMaxR; ++i)
      if (i < sp.A) v[i] = in(p, r + sp.B * i);
    fftr::rdft_rt(sp.A, v, s);
#pragma unroll
    for (int k = 1; k < kMaxR; ++k)
      if (k < sp.A) {
        C w = tw[r * k];
        if (s > (T)0) w.y = -w.y;  // table holds e^{-2 pi i m/N}; conjugate for the inverse
        v[k] = fftr::mul(v[k], w);
      }
#pragma unroll
    for (int k = 0; k < kMaxR; ++k)
      if (k < sp.A) sc[k * (sp.B + 1) + r] = v[k];
  }
  __syncwarp();
  if (act && r < sp.A) {
#pragma unroll
    for (int j = 0; j < kMaxR; ++j)
      if (j < sp.B) v[j] = sc[r * (sp.B + 1) + j];
    fftr::rdft_rt(sp.B, v, s);
#pragma unroll
    for (int k = 0; k < kMaxR; ++k)
      if (k < sp.B) out(p, r + sp.A * k, v[k]);
  }
  __syncwarp();
}

// z-column: inverse FFT, x V(z), forward FFT, with the data kept in registers between the two
// transforms.  in(p, z) / out(p, z, v) address the sphere-range part of the column; vz(p, z) is
// the (scaled) potential.
template <typename C, typename T, class In, class Out, class Vf>
__device__ __forceinline__ void zcolumn_rt(const Split& sp, int np, const C* tw, C* scr, int lane,
                                        In in, Out out, Vf vz) {
  const int p = lane / sp.L, r = lane - p * sp.L;
  const bool act = p < np;
  C* sc = scr + p * sp.scr;
  C v[kMaxR];
  // inverse, stage 1
  if (act && r < sp.B) {
#pragma unroll
    for (int i = 0; i < kMaxR; ++i)
      if (i < sp.A) v[i] = in(p, r + sp.B * i);
    fftr::rdft_rt(sp.A, v, (T)1);
#pragma unroll
    for (int k = 1; k < kMaxR; ++k)
      if (k < sp.A) {
        C w = tw[r * k];
        w.y = -w.y;
        v[k] = fftr::mul(v[k], w);
      }
#pragma unroll
    for (int k = 0; k < kMaxR; ++k)
      if (k < sp.A) sc[k * (sp.B + 1) + r] = v[k];
  }
  __syncwarp();
  if (act && r < sp.A) {
#pragma unroll
    for (int j = 0; j < kMaxR; ++j)
      if (j < sp.B) v[j] = sc[r * (sp.B + 1) + j];
  }
  __syncwarp();
  if (act && r < sp.A) {
    // inverse, stage 2: v[k2] = psi(z = r + A k2); multiply by V; forward stage 1 (DFT-B)
    fftr::rdft_rt(sp.B, v, (T)1);
#pragma unroll
    for (int k = 0; k < kMaxR; ++k)
      if (k < sp.B) {
        const T vv = vz(p, r + sp.A * k);
        v[k].x *= vv;
        v[k].y *= vv;
      }
    fftr::rdft_rt(sp.B, v, (T)-1);
#pragma unroll
    for (int q = 1; q < kMaxR; ++q)
      if (q < sp.B) v[q] = fftr::mul(v[q], tw[r * q]);
#pragma unroll
    for (int q = 0; q < kMaxR; ++q)
      if (q < sp.B) sc[q * (sp.A + 1) + r] = v[q];
  }
  __syncwarp();
  if (act && r < sp.B) {
#pragma unroll
    for (int k = 0; k < kMaxR; ++k)
      if (k < sp.A) v[k] = sc[r * (sp.A + 1) + k];
    fftr::rdft_rt(sp.A, v, (T)-1);
#pragma unroll
    for (int k = 0; k < kMaxR; ++k)
      if (k < sp.A) out(p, r + sp.B * k, v[k]);
  }
  __syncwarp();
}

// Compile-time forms of the two transforms above for the (A, B) splits the common FFT lengths
// use: loops fully unrolled with constant shared-memory offsets and no per-element guards.
template <int A, int B, typename C, typename T, class In, class Out>
__device__ __forceinline__ void pencil_fft_ct(int np, int scrsz, const C* tw, T s, C* scr, int lane,
                                              In in, Out out) {
  constexpr int L = A > B ? A : B;
  const int p = lane / L, r = lane - p * L;
  const bool act = p < np;
  C* sc = scr + p * scrsz;
  C v[L];
  if (act && r < B) {
#pragma unroll
    for (int i = 0; i < A; ++i) v[i] = in(p, r + B * i);
    fftr::rdft<A>(v, s);
#pragma unroll
    for (int k = 1; k < A; ++k) {
      C w = tw[r * k];
      if (s > (T)0) w.y = -w.y;  // conjugate for the inverse
      v[k] = fftr::mul(v[k], w);
    }
#pragma unroll
    for (int k = 0; k < A; ++k) sc[k * (B + 1) + r] = v[k];
  }
  __syncwarp();
  if (act && r < A) {
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = sc[r * (B + 1) + j];
    fftr::rdft<B>(v, s);
#pragma unroll
    for (int k = 0; k < B; ++k) out(p, r + A * k, v[k]);
  }
  __syncwarp();
}

template <int A, int B, typename C, typename T, class In, class Out, class Vf>
__device__ __forceinline__ void zcolumn_ct(int np, int scrsz, const C* tw, C* scr, int lane, In in,
                                           Out out, Vf vz) {
  constexpr int L = A > B ? A : B;
  const int p = lane / L, r = lane - p * L;
  const bool act = p < np;
  C* sc = scr + p * scrsz;
  C v[L];
  if (act && r < B) {
#pragma unroll
    for (int i = 0; i < A; ++i) v[i] = in(p, r + B * i);
    fftr::rdft<A>(v, (T)1);
#pragma unroll
    for (int k = 1; k < A; ++k) {
      C w = tw[r * k];
      w.y = -w.y;
      v[k] = fftr::mul(v[k], w);
    }
#pragma unroll
    for (int k = 0; k < A; ++k) sc[k * (B + 1) + r] = v[k];
  }
  __syncwarp();
  if (act && r < A) {
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = sc[r * (B + 1) + j];
  }
  __syncwarp();
  if (act && r < A) {
    fftr::rdft<B>(v, (T)1);
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const T vv = vz(p, r + A * k);
      v[k].x *= vv;
      v[k].y *= vv;
    }
    fftr::rdft<B>(v, (T)-1);
#pragma unroll
    for (int q = 1; q < B; ++q) v[q] = fftr::mul(v[q], tw[r * q]);
#pragma unroll
    for (int q = 0; q < B; ++q) sc[q * (A + 1) + r] = v[q];
  }
  __syncwarp();
  if (act && r < B) {
#pragma unroll
    for (int k = 0; k < A; ++k) v[k] = sc[r * (A + 1) + k];
    fftr::rdft<A>(v, (T)-1);
#pragma unroll
    for (int k = 0; k < A; ++k) out(p, r + B * k, v[k]);
  }
  __syncwarp();
}

// FFT policies of the pass bodies: runtime-sized transforms (any split) or the compile-time
// forms for one (A, B) split.  Each kernel instance uses one policy, so it gets a register
// allocation for its own split only.
struct RtPol {
  template <typename C, typename T, class In, class Out>
  static __device__ __forceinline__ void pencil(const Split& sp, int np, const C* tw, T s, C* scr,
                                                int lane, In in, Out out) {
    pencil_fft_rt<C, T>(sp, np, tw, s, scr, lane, in, out);
  }
  template <typename C, typename T, class In, class Out, class Vf>
  static __device__ __forceinline__ void zcol(const Split& sp, int np, const C* tw, C* scr, int lane,
                                              In in, Out out, Vf vz) {
    zcolumn_rt<C, T>(sp, np, tw, scr, lane, in, out, vz);
  }
};
template <int A, int B>
struct CtPol {
  template <typename C, typename T, class In, class Out>
  static __device__ __forceinline__ void pencil(const Split& sp, int np, const C* tw, T s, C* scr,
                                                int lane, In in, Out out) {
    pencil_fft_ct<A, B, C, T>(np, sp.scr, tw, s, scr, lane, in, out);
  }
  template <typename C, typename T, class In, class Out, class Vf>
  static __device__ __forceinline__ void zcol(const Split& sp, int np, const C* tw, C* scr, int lane,
                                              In in, Out out, Vf vz) {
    zcolumn_ct<A, B, C, T>(np, sp.scr, tw, scr, lane, in, out, vz);
  }
};

// Splits with compile-time kernel instances (the FFT lengths 15..60 and 96 of the workloads).
#define KSS_SPLITS(X) X(3, 5) X(4, 4) X(3, 6) X(4, 5) X(4, 6) X(5, 5) X(3, 9) X(5, 6) X(6, 6) \
                      X(5, 8) X(5, 9) X(6, 8) X(5, 10) X(6, 9) X(6, 10) X(8, 12)

// Splits (A, B) with CTA-wide pass B instances: both orientations of the FFT lengths the workloads
// use (24 .. 60 and 96) plus a second factorisation of 96, so the autotuner can choose the radix
// schedule; one orientation for the small test lengths.
#define KSS_WIDE_SPLITS(X)                                                                        \
  X(3, 5) X(4, 4) X(3, 6) X(4, 5) X(5, 5) X(3, 9)                                                 \
  X(4, 6) X(6, 4) X(3, 8) X(8, 3) X(5, 6) X(6, 5) X(3, 10) X(10, 3) X(6, 6) X(4, 9) X(9, 4)       \
  X(5, 8) X(8, 5) X(4, 10) X(10, 4) X(5, 9) X(9, 5) X(6, 8) X(8, 6) X(5, 10) X(10, 5) X(6, 9)     \
  X(9, 6) X(6, 10) X(10, 6) X(5, 12) X(12, 5) X(8, 12) X(12, 8) X(6, 16) X(16, 6)

// Scatter of band n's sphere coefficients on z-plane u3 into the x-row tile (row u2 at u2 * N1p,
// x in natural order, as the tile index table holds them).  Packed mode forms psi_2n + i psi_2n+1.
template <int NT, typename T, typename C>
__device__ __forceinline__ void scatter_plane(const LocalArgs<T>& a, C* tile, int u3, int n) {
  const int g0 = a.zstart[u3], g1 = a.zstart[u3 + 1];
  if (a.packed) {
    const C* pa = a.psi + (size_t)(2 * n) * a.ld;
    const C* pb = 2 * n + 1 < a.nbands ? pa + a.ld : nullptr;
    for (int g = g0 + (int)threadIdx.x; g < g1; g += NT) {
      C x = pa[g];
      if (pb) {
        const C y = pb[g];  // x + i y
        x.x -= y.y;
        x.y += y.x;
      }
      tile[a.tileidx[g]] = x;
    }
  } else {
    const C* ps = a.psi + n * a.ld;
    for (int g = g0 + (int)threadIdx.x; g < g1; g += NT) tile[a.tileidx[g]] = ps[g];
  }
}

// Gather of z-plane u3 from the x-row tile and the epilogue of pass C: out = alpha (T psi + V
// psi) + beta psi + gamma psi_prev (coefficients from device memory when coef is set).  Packed
// mode stores the raw transform of the pair (unpacked and finished by gamma_unpack).
template <int NT, typename T, typename C>
__device__ __forceinline__ void gather_plane(const LocalArgs<T>& a, const C* tile, int u3, int n) {
  const int g0 = a.zstart[u3], g1 = a.zstart[u3 + 1];
  C* po = a.out + n * a.ld;
  if (a.packed) {
    for (int g = g0 + (int)threadIdx.x; g < g1; g += NT) po[g] = tile[a.tileidx[g]];
    return;
  }
  const C* ps = a.psi + n * a.ld;
  const C* pp = a.psi_prev ? a.psi_prev + n * a.ld : nullptr;
  const T al = a.coef ? a.coef[0] : a.alpha;
  const T be = a.coef ? a.coef[1] : a.beta;
  const T ga = a.coef ? a.coef[2] : a.gamma;
  for (int g = g0 + (int)threadIdx.x; g < g1; g += NT) {
    const C v = tile[a.tileidx[g]];
    const C p = ps[g];
    const T t = a.kin[g];
    C o;
    o.x = al * (t * p.x + v.x) + be * p.x;
    o.y = al * (t * p.y + v.y) + be * p.y;
    if (pp) {
      const C q = pp[g];
      o.x += ga * q.x;
      o.y += ga * q.y;
    }
    po[g] = o;
  }
}

template <typename T, class Pol = RtPol>
__device__ __forceinline__ void pass_a_body(const LocalArgs<T>& a, const RegPlan& rp, int scr_warp,
                                            int u3, int nl) {
  using C = typename CT<T>::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  C* tile = tw + a.N1;
  C* scr = tile + a.W2 * a.N1p + (threadIdx.x >> 5) * scr_warp;
  const int n = a.n0 + nl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  copy_table(tw, a.tw1, a.N1);
  const int tsz = a.W2 * a.N1p;
  for (int i = threadIdx.x; i < tsz; i += kThreads) tile[i] = C{0, 0};
  __syncthreads();
  scatter_plane<kThreads>(a, tile, u3, n);
  __syncthreads();
  const int r0 = a.rowrange[2 * u3], r1 = a.rowrange[2 * u3 + 1];
  const int nrows = r1 - r0 + 1;
  const Split sp = rp.s1;
  for (int r = warp * sp.PP; r < nrows; r += kWarps * sp.PP) {
    C* rows = tile + (r0 + r) * a.N1p;
    const int ld = a.N1p;
    Pol::template pencil<C, T>(sp, min(sp.PP, nrows - r), tw, (T)1, scr, lane,
                     [&](int p, int e) { return rows[p * ld + e]; },
                     [&](int p, int e, C v) { rows[p * ld + e] = v; });
  }
  __syncthreads();
  C* dst = a.work + ((size_t)nl * a.N1 * a.W3 + u3) * a.W2;
  const size_t xs = (size_t)a.W3 * a.W2;
  const fftr::FastDiv dw2(a.W2);
  for (int i = threadIdx.x; i < a.N1 * a.W2; i += kThreads) {
    const int x = dw2(i), u2 = i - x * a.W2;
    dst[x * xs + u2] = tile[u2 * a.N1p + x];
  }
}

template <typename T, class Pol = RtPol>
__device__ __forceinline__ void pass_b_body(const LocalArgs<T>& a, const RegPlan& rp, int scr_warp,
                                            int x, int nl) {
  using C = typename CT<T>::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw2 = reinterpret_cast<C*>(smraw);
  C* tw3 = tw2 + a.N2;
  C* Q = tw3 + a.N3;                           // W3 x N2p
  C* scr = Q + a.W3 * a.N2p + (threadIdx.x >> 5) * scr_warp;
  int* zmap = reinterpret_cast<int*>(Q + a.W3 * a.N2p + kWarps * scr_warp);  // N3
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  copy_table(tw2, a.tw2, a.N2);
  copy_table(tw3, a.tw3, a.N3);
  for (int z = threadIdx.x; z < a.N3; z += kThreads) {
    int u = (z - a.lo3) % a.N3;
    if (u < 0) u += a.N3;
    zmap[z] = u < a.W3 ? u : -1;
  }
  for (int i = threadIdx.x; i < a.W3 * a.N2p; i += kThreads) Q[i] = C{0, 0};
  __syncthreads();
  C* slab = a.work + ((size_t)nl * a.N1 + x) * a.W3 * a.W2;
  const fftr::FastDiv dw2(a.W2);
  for (int i = threadIdx.x; i < a.W3 * a.W2; i += kThreads) {
    const int u3 = dw2(i), u2 = i - u3 * a.W2;
    Q[u3 * a.N2p + fftr::wrap_add(a.lo2, u2, a.N2)] = slab[i];
  }
  __syncthreads();
  const int N2p = a.N2p;
  {
    const Split sp = rp.s2;
    for (int r = warp * sp.PP; r < a.W3; r += kWarps * sp.PP) {
      C* rows = Q + r * N2p;
      Pol::template pencil<C, T>(sp, min(sp.PP, a.W3 - r), tw2, (T)1, scr, lane,
                       [&](int p, int e) { return rows[p * N2p + e]; },
                       [&](int p, int e, C v) { rows[p * N2p + e] = v; });
    }
  }
  __syncthreads();
  {
    const Split sp = rp.s3;
    const T* vx = a.Vx + (size_t)x * a.N2 * a.N3;
    const int N3 = a.N3;
    for (int y0 = warp * sp.PP; y0 < a.N2; y0 += kWarps * sp.PP) {
      Pol::template zcol<C, T>(sp, min(sp.PP, a.N2 - y0), tw3, scr, lane,
                    [&](int p, int z) {
                      const int u = zmap[z];
                      return u >= 0 ? Q[u * N2p + y0 + p] : C{0, 0};
                    },
                    [&](int p, int z, C v) {
                      const int u = zmap[z];
                      if (u >= 0) Q[u * N2p + y0 + p] = v;
                    },
                    [&](int p, int z) { return vx[(size_t)(y0 + p) * N3 + z]; });
    }
  }
  __syncthreads();
  {
    const Split sp = rp.s2;
    for (int r = warp * sp.PP; r < a.W3; r += kWarps * sp.PP) {
      C* rows = Q + r * N2p;
      Pol::template pencil<C, T>(sp, min(sp.PP, a.W3 - r), tw2, (T)-1, scr, lane,
                       [&](int p, int e) { return rows[p * N2p + e]; },
                       [&](int p, int e, C v) { rows[p * N2p + e] = v; });
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.W3 * a.W2; i += kThreads) {
    const int u3 = dw2(i), u2 = i - u3 * a.W2;
    slab[i] = Q[u3 * a.N2p + fftr::wrap_add(a.lo2, u2, a.N2)];
  }
}

template <typename T, class Pol = RtPol>
__device__ __forceinline__ void pass_c_body(const LocalArgs<T>& a, const RegPlan& rp, int scr_warp,
                                            int u3, int nl) {
  using C = typename CT<T>::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  C* tile = tw + a.N1;
  C* scr = tile + a.W2 * a.N1p + (threadIdx.x >> 5) * scr_warp;
  const int n = a.n0 + nl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  copy_table(tw, a.tw1, a.N1);
  const int r0 = a.rowrange[2 * u3], r1 = a.rowrange[2 * u3 + 1];
  const int nrows = r1 - r0 + 1;
  const C* src = a.work + ((size_t)nl * a.N1 * a.W3 + u3) * a.W2;
  const size_t xs = (size_t)a.W3 * a.W2;
  const fftr::FastDiv dnr(nrows);
  for (int i = threadIdx.x; i < a.N1 * nrows; i += kThreads) {
    const int x = dnr(i), u2 = r0 + (i - x * nrows);
    tile[u2 * a.N1p + x] = src[x * xs + u2];
  }
  __syncthreads();
  const Split sp = rp.s1;
  for (int r = warp * sp.PP; r < nrows; r += kWarps * sp.PP) {
    C* rows = tile + (r0 + r) * a.N1p;
    const int ld = a.N1p;
    Pol::template pencil<C, T>(sp, min(sp.PP, nrows - r), tw, (T)-1, scr, lane,
                     [&](int p, int e) { return rows[p * ld + e]; },
                     [&](int p, int e, C v) { rows[p * ld + e] = v; });
  }
  __syncthreads();
  gather_plane<kThreads>(a, tile, u3, n);
}

// Pass B with every transform stage spread over the whole CTA.  The per-warp pencil forms above
// give each pencil max(A, B) lanes, so a stage of size min(A, B) leaves lanes idle (for 96 = 8 x
// 12, a third of the lanes in stage 1 and half in stage 2).  Here each stage is one loop over all
// (pencil, sub-transform) tasks of the x-plane, and every stage works in place:
//   inverse, stage 1: task (pencil, r < B) reads elements r + B i (i < A), DFT-A, twiddle, writes
//                     them back; stage 2: task (pencil, k < A) reads the B contiguous elements
//                     j + B k, DFT-B, writes back, so that position k2 + B k holds the transform
//                     at index k + A k2 (digit-reversed order);
//   forward,  stage 1: task (pencil, r < A) reads the B contiguous elements at positions k2 + B r
//                     (input index r + A k2), DFT-B, twiddle, writes back; stage 2: task (pencil,
//                     q < B) reads positions q + B m (m < A), DFT-A, writes index q + B k at
//                     position q + B k (natural order).
// The y rows stay in digit-reversed order through the z stages, which only need to know which y
// a column holds (to read V).  The z columns of the whole plane live in a second buffer Z, so the
// inverse z transform reads the sphere window rows of Q (zeros elsewhere) and the forward one
// writes only the window rows back.  Requires N2 == N3 == A * B.
constexpr int kWideThreads = 384;  // 12 warps: 96-point stages split into whole rounds of tasks

template <typename T, int A, int B>
struct WideB {
  static constexpr int N = A * B;
  static constexpr int QS = (N + 1) | 1;  // odd row / column pitches: with the index along the
  static constexpr int ZS = (N + 1) | 1;  // pitch fastest across lanes, no shared-memory bank conflicts
  static size_t smem(int W3) {
    return sizeof(typename CT<T>::C) * ((size_t)N + (size_t)W3 * QS + (size_t)N * ZS) + sizeof(int) * N;
  }
};

// Pruned stages (CW > 0): the window rows of y and z (the sphere's extent, about 0.4 N) occupy,
// in the strided index r + B i of a DFT-A stage, only the first CW and the last CW values of i, so
// the first inverse stages read only those inputs (the others are zero) and the last forward
// stages compute only those outputs (the others are discarded): fftr::rdft_m with the edge mask.
// Valid when B CW exceeds the window's largest index and is at least its most negative index's
// magnitude along both y and z (wide_prune_cw); CW = 0 is the full transform.
template <typename T, int A, int B, int NT = kWideThreads, int CW = 0>
__device__ __forceinline__ void pass_bw_body(const LocalArgs<T>& a, int x, int nl) {
  using C = typename CT<T>::C;
  using G = WideB<T, A, B>;
  constexpr int N = G::N, QS = G::QS, ZS = G::ZS;
  constexpr unsigned MW = fftr::edge_mask<A, CW>(), MF = fftr::full_mask<A>();
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);  // e^{-2 pi i m / N}, m < N
  C* Q = tw + N;                        // W3 rows (z in the sphere window) x N (y)
  C* Z = Q + a.W3 * QS;                 // N columns (y position) x N (z)
  int* zmap = reinterpret_cast<int*>(Z + N * ZS);
  const int tid = threadIdx.x;
  const int W3 = a.W3, W2 = a.W2;
  for (int i = tid; i < N; i += NT) tw[i] = a.tw2[i];
  for (int z = tid; z < N; z += NT) {
    int u = (z - a.lo3) % N;
    if (u < 0) u += N;
    zmap[z] = u < W3 ? u : -1;
  }
  for (int i = tid; i < W3 * QS; i += NT) Q[i] = C{0, 0};
  __syncthreads();
  C* slab = a.work + ((size_t)nl * a.N1 + x) * W3 * W2;
  const fftr::FastDiv dw2(W2), dw3(W3);
  for (int i = tid; i < W3 * W2; i += NT) {
    const int u3 = dw2(i), u2 = i - u3 * W2;
    Q[u3 * QS + fftr::wrap_add(a.lo2, u2, N)] = slab[i];
  }
  __syncthreads();
  // ---- y, inverse ----
  for (int t = tid; t < W3 * B; t += NT) {
    const int r = dw3(t), u = t - r * W3;  // rows fastest across lanes
    C* row = Q + u * QS + r;
    C v[A];
    fftr::static_for<0, A>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      if constexpr (MW >> i & 1u) v[i] = row[B * i];
    });
    fftr::rdft_m<A, MW, MF>(v, (T)1);
#pragma unroll
    for (int k = 1; k < A; ++k) {
      C w = tw[r * k];
      w.y = -w.y;
      v[k] = fftr::mul(v[k], w);
    }
#pragma unroll
    for (int k = 0; k < A; ++k) row[B * k] = v[k];
  }
  __syncthreads();
  for (int t = tid; t < W3 * A; t += NT) {
    const int k = dw3(t), u = t - k * W3;
    C* row = Q + u * QS + B * k;
    C v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = row[j];
    fftr::rdft<B>(v, (T)1);
#pragma unroll
    for (int j = 0; j < B; ++j) row[j] = v[j];
  }
  __syncthreads();
  // ---- z, inverse stage 1 (column p of the plane; only window rows are nonzero) ----
  for (int t = tid; t < N * B; t += NT) {
    const int r = t / N, p = t - r * N;
    C v[A];
    fftr::static_for<0, A>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      if constexpr (MW >> i & 1u) {
        const int u = zmap[r + B * i];
        v[i] = u >= 0 ? Q[u * QS + p] : C{0, 0};
      }
    });
    fftr::rdft_m<A, MW, MF>(v, (T)1);
#pragma unroll
    for (int k = 1; k < A; ++k) {
      C w = tw[r * k];
      w.y = -w.y;
      v[k] = fftr::mul(v[k], w);
    }
    C* col = Z + p * ZS + r;
#pragma unroll
    for (int k = 0; k < A; ++k) col[B * k] = v[k];
  }
  __syncthreads();
  // ---- z, inverse stage 2, x V, forward stage 1 ----
  // columns fastest across lanes; V from the [x][z][p] view (coalesced in p)
  const T* vp = a.Vpi + (size_t)x * N * N;
  for (int t = tid; t < N * A; t += NT) {
    const int k = t / N, p = t - k * N;
    const T* vrow = vp + (size_t)k * N + p;  // (z = k + A k2, p) at vrow[A k2 N]
    C* col = Z + p * ZS + B * k;
    C v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = col[j];
    fftr::rdft<B>(v, (T)1);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) {
      const T vv = vrow[(size_t)A * k2 * N];  // z = k + A k2
      v[k2].x *= vv;
      v[k2].y *= vv;
    }
    fftr::rdft<B>(v, (T)-1);
#pragma unroll
    for (int q = 1; q < B; ++q) v[q] = fftr::mul(v[q], tw[k * q]);
#pragma unroll
    for (int q = 0; q < B; ++q) col[q] = v[q];
  }
  __syncthreads();
  // ---- z, forward stage 2: keep the window rows ----
  for (int t = tid; t < N * B; t += NT) {
    const int q = t / N, p = t - q * N;
    const C* col = Z + p * ZS + q;
    C v[A];
#pragma unroll
    for (int m = 0; m < A; ++m) v[m] = col[B * m];
    fftr::rdft_m<A, MF, MW>(v, (T)-1);
    fftr::static_for<0, A>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (MW >> k & 1u) {
        const int u = zmap[q + B * k];
        if (u >= 0) Q[u * QS + p] = v[k];
      }
    });
  }
  __syncthreads();
  // ---- y, forward ----
  for (int t = tid; t < W3 * A; t += NT) {
    const int r = dw3(t), u = t - r * W3;
    C* row = Q + u * QS + B * r;
    C v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = row[j];
    fftr::rdft<B>(v, (T)-1);
#pragma unroll
    for (int q = 1; q < B; ++q) v[q] = fftr::mul(v[q], tw[r * q]);
#pragma unroll
    for (int q = 0; q < B; ++q) row[q] = v[q];
  }
  __syncthreads();
  for (int t = tid; t < W3 * B; t += NT) {
    const int q = dw3(t), u = t - q * W3;
    C* row = Q + u * QS + q;
    C v[A];
#pragma unroll
    for (int m = 0; m < A; ++m) v[m] = row[B * m];
    fftr::rdft_m<A, MF, MW>(v, (T)-1);
    fftr::static_for<0, A>([&](auto kc) {  // rows outside the window are not read again
      constexpr int k = decltype(kc)::value;
      if constexpr (MW >> k & 1u) row[B * k] = v[k];
    });
  }
  __syncthreads();
  for (int i = tid; i < W3 * W2; i += NT) {
    const int u3 = dw2(i), u2 = i - u3 * W2;
    slab[i] = Q[u3 * QS + fftr::wrap_add(a.lo2, u2, N)];
  }
}

// Passes A and C with the x transforms spread over the CTA, in the manner of pass_bw_body: each
// stage is one loop over the (row, sub-transform) tasks of the rows r0..r1 of z-plane u3 that hold
// sphere points, in place in the tile (rows fastest across lanes, odd pitch N + 1).  The tile
// holds x in natural order for the scatter (pass A) and the gather (pass C); between the
// transform stages and the slab it is in the stages' digit-reversed order, position x / A +
// B (x % A) holding index x, so pass A's inverse ends and pass C's forward starts there, and the
// slab keeps natural x order for pass B.  CW > 0: the sphere's x window occupies only the first
// and last CW values of the strided index r + B i, so pass A's first stage reads only those
// inputs and pass C's last stage computes only those outputs (fftr::rdft_m with the edge mask).
// Requires N1 == A * B, even, so that the tile index table's pitch N1 + 1 is odd.
template <typename T, int A, int B>
struct WideX {
  static constexpr int N = A * B, P = N + 1;
  static_assert(N % 2 == 0, "the tile pitch N + 1 must be odd");
  static size_t smem(int W2) { return sizeof(typename CT<T>::C) * ((size_t)N + (size_t)W2 * P); }
  __device__ static int pos(int x) { return x / A + B * (x % A); }
};

template <typename T, int A, int B, int NT, int CW = 0>
__device__ __forceinline__ void pass_aw_body(const LocalArgs<T>& a, int u3, int nl) {
  using C = typename CT<T>::C;
  using G = WideX<T, A, B>;
  constexpr int N = G::N, P = G::P;
  constexpr unsigned MW = fftr::edge_mask<A, CW>(), MF = fftr::full_mask<A>();
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);  // e^{-2 pi i m / N}, m < N
  C* tile = tw + N;                     // W2 rows (y in the sphere window) x N (x)
  const int tid = threadIdx.x;
  const int n = a.n0 + nl;
  int r0 = a.rowrange[2 * u3];
  const int r1 = a.rowrange[2 * u3 + 1];
  const int nrows = r1 >= r0 ? r1 - r0 + 1 : 0;
  if (!nrows) r0 = 0;
  C* rows = tile + r0 * P;
  for (int i = tid; i < N; i += NT) tw[i] = a.tw1[i];
  for (int i = tid; i < nrows * P; i += NT) rows[i] = C{0, 0};
  __syncthreads();
  scatter_plane<NT>(a, tile, u3, n);
  __syncthreads();
  const fftr::FastDiv dnr(nrows > 0 ? nrows : 1);
  // inverse, stage 1: task (row, r < B) on the elements r + B i
  for (int t = tid; t < nrows * B; t += NT) {
    const int r = dnr(t), u = t - r * nrows;
    C* row = rows + u * P + r;
    C v[A];
    fftr::static_for<0, A>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      if constexpr (MW >> i & 1u) v[i] = row[B * i];
    });
    fftr::rdft_m<A, MW, MF>(v, (T)1);
#pragma unroll
    for (int k = 1; k < A; ++k) {
      C w = tw[r * k];
      w.y = -w.y;
      v[k] = fftr::mul(v[k], w);
    }
#pragma unroll
    for (int k = 0; k < A; ++k) row[B * k] = v[k];
  }
  __syncthreads();
  // inverse, stage 2: task (row, k < A) on the B contiguous elements j + B k
  for (int t = tid; t < nrows * A; t += NT) {
    const int k = dnr(t), u = t - k * nrows;
    C* row = rows + u * P + B * k;
    C v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = row[j];
    fftr::rdft<B>(v, (T)1);
#pragma unroll
    for (int j = 0; j < B; ++j) row[j] = v[j];
  }
  __syncthreads();
  // slab [x][u3][u2] in natural x order; rows outside r0..r1 hold no sphere point (zero)
  C* dst = a.work + ((size_t)nl * N * a.W3 + u3) * a.W2;
  const size_t xs = (size_t)a.W3 * a.W2;
  const fftr::FastDiv dw2(a.W2);
  for (int i = tid; i < N * a.W2; i += NT) {
    const int x = dw2(i), u2 = i - x * a.W2;
    const int u = u2 - r0;
    dst[x * xs + u2] = (u >= 0 && u < nrows) ? rows[u * P + G::pos(x)] : C{0, 0};
  }
}

template <typename T, int A, int B, int NT, int CW = 0>
__device__ __forceinline__ void pass_cw_body(const LocalArgs<T>& a, int u3, int nl) {
  using C = typename CT<T>::C;
  using G = WideX<T, A, B>;
  constexpr int N = G::N, P = G::P;
  constexpr unsigned MW = fftr::edge_mask<A, CW>(), MF = fftr::full_mask<A>();
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  C* tile = tw + N;
  const int tid = threadIdx.x;
  const int n = a.n0 + nl;
  int r0 = a.rowrange[2 * u3];
  const int r1 = a.rowrange[2 * u3 + 1];
  const int nrows = r1 >= r0 ? r1 - r0 + 1 : 0;
  if (!nrows) r0 = 0;
  C* rows = tile + r0 * P;
  for (int i = tid; i < N; i += NT) tw[i] = a.tw1[i];
  const C* src = a.work + ((size_t)nl * N * a.W3 + u3) * a.W2;
  const size_t xs = (size_t)a.W3 * a.W2;
  const fftr::FastDiv dnr(nrows > 0 ? nrows : 1);
  for (int i = tid; i < N * nrows; i += NT) {
    const int x = dnr(i), u = i - x * nrows;
    rows[u * P + G::pos(x)] = src[x * xs + r0 + u];
  }
  __syncthreads();
  // forward, stage 1: task (row, r < A) on the B contiguous positions k2 + B r (index r + A k2)
  for (int t = tid; t < nrows * A; t += NT) {
    const int r = dnr(t), u = t - r * nrows;
    C* row = rows + u * P + B * r;
    C v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = row[j];
    fftr::rdft<B>(v, (T)-1);
#pragma unroll
    for (int q = 1; q < B; ++q) v[q] = fftr::mul(v[q], tw[r * q]);
#pragma unroll
    for (int q = 0; q < B; ++q) row[q] = v[q];
  }
  __syncthreads();
  // forward, stage 2: task (row, q < B) on the positions q + B m; index q + B k lands at
  // position q + B k (natural order); only the window's outputs are formed
  for (int t = tid; t < nrows * B; t += NT) {
    const int q = dnr(t), u = t - q * nrows;
    C* row = rows + u * P + q;
    C v[A];
#pragma unroll
    for (int m = 0; m < A; ++m) v[m] = row[B * m];
    fftr::rdft_m<A, MF, MW>(v, (T)-1);
    fftr::static_for<0, A>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr (MW >> k & 1u) row[B * k] = v[k];
    });
  }
  __syncthreads();
  gather_plane<NT>(a, tile, u3, n);
}

// Smallest edge width CW of split N = A * B whose strided index r + B i covers every position of
// the window [lo, lo + W - 1] (B CW > largest index, B CW >= magnitude of the most negative one);
// 1 << 20 when the window does not straddle 0.
inline int axis_prune_cw(int B, int lo, int W) {
  const int hi = lo + W - 1;
  if (lo > 0 || hi < 0) return 1 << 20;
  const int c1 = hi / B + 1, c2 = (-lo + B - 1) / B;
  return c1 > c2 ? c1 : c2;
}

// Pruning width of the CTA-wide pass B for split N = A * B and the sphere windows of y (lo2, W2)
// and z (lo3, W3): the width covering both axes, or 0 when the windows do not straddle 0 or leave
// nothing to prune (2 CW >= A).
inline int wide_prune_cw(int A, int B, int lo2, int W2, int lo3, int W3) {
  const int c = std::max(axis_prune_cw(B, lo2, W2), axis_prune_cw(B, lo3, W3));
  return 2 * c < A ? c : 0;
}

// Best two-factor split N = A*B over the codelet sizes (fewest warp instructions per pencil).
inline bool choose_split(int N, Split& out) {
  static const int S[] = {1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16};
  double best = 1e30;
  bool ok = false;
  for (int A : S)
    for (int B : S) {
      if (A * B != N) continue;
      const int L = std::max(A, B);
      const int PP = 32 / L;
      auto cost = [](int n) { double c = 2.0; for (int m = n; m > 1; m >>= 1) c += n; return c; };
      const double sc = (cost(A) + cost(B)) / PP;
      if (sc < best) {
        best = sc;
        out.N = N;
        out.A = A;
        out.B = B;
        out.L = L;
        out.PP = PP;
        out.scr = std::max(A * (B + 1), B * (A + 1));
        ok = true;
      }
    }
  return ok;
}


}  // namespace lk
}  // namespace kss

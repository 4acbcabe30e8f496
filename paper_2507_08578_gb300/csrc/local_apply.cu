// H application on a band block: kinetic + local potential through pruned 3D FFTs (batched over
// bands, §5.1) + the separable nonlocal operator as two matrix products with the projector table
// and the projector coefficients held in memory (Eq. ham-nl, §5.2).
//
// Local part, per band (box N1 x N2 x N3, sphere bounding box W1 x W2 x W3 starting at lo):
//   pass A  (one CTA per z-slice u3):   scatter the slice's plane waves into a W2 x N1 tile,
//                                       inverse FFT along x, store the slab T[x][u3][u2]
//   pass B  (one CTA per x-plane):      inverse FFT along y (W3 rows), then per y-column:
//                                       inverse FFT along z, x V(r)/N^3, forward FFT along z;
//                                       forward FFT along y; store back in place
//   pass C  (one CTA per z-slice u3):   forward FFT along x, gather the slice's plane waves and
//                                       finish the Chebyshev epilogue
//     out = alpha*(T psi + V psi) + beta*psi + gamma*psi_prev
// Only pencils that can hold sphere data are transformed (the slab keeps W2 x W3 of the N2 x N3
// (y, z) cross-section), so the executed FFT work is about half of the dense 3D transform.
// Kernel forms, best first:
//   * pass B with a common y/z length A*B that has a compile-time instance: the CTA-wide form
//     (local_wide.cu), every transform stage spread over all lanes of the CTA;
//   * passes A/C (and pass B otherwise) with a compile-time split: per-warp two-level register
//     codelets (fft_reg.cuh, CtPol), else the same with runtime sizes (RtPol);
//   * lengths that do not split into two codelets of size <= 16: warp-level Stockham FFTs
//     (radix 4/2/3/5) on contiguous pencils in shared memory (the kernels in this file).
// The slab lives in a workspace of nc bands (chunked so that it stays L2-resident).
#include <algorithm>

#include "local_fused.h"
#include "local_kernels.cuh"
#include "density.h"
#include "local_wide.h"
#include "tune.h"

namespace kss {

namespace {

using namespace lk;
using fftr::Split;
constexpr int kMaxB = 4;  // butterflies per lane held in registers by one Stockham stage

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// multiply by s*i (s = +-1)
template <typename C, typename T> __device__ __forceinline__ C cmuli(C a, T s) { C r; r.x = -s * a.y; r.y = s * a.x; return r; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { C r; r.x = s * a.x; r.y = s * a.y; return r; }

// y_q = sum_t v_t exp(dir * 2 pi i t q / R), in place (radix-R DFT kernels).
template <int R, typename C, typename T> struct Dft;
template <typename C, typename T> struct Dft<2, C, T> {
  static __device__ __forceinline__ void run(C* v, T) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <typename C, typename T> struct Dft<3, C, T> {
  static __device__ __forceinline__ void run(C* v, T dir) {
    const T h = (T)0.5, s3 = (T)0.86602540378443864676;  // cos(pi/3), sin(pi/3)
    const C t1 = cadd(v[1], v[2]);
    const C t2 = csub(v[0], cscale(t1, h));
    const C t3 = cmuli(csub(v[1], v[2]), dir * s3);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  }
};
template <typename C, typename T> struct Dft<4, C, T> {
  static __device__ __forceinline__ void run(C* v, T dir) {
    const C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const C c = cadd(v[1], v[3]), d = cmuli(csub(v[1], v[3]), dir);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};
template <typename C, typename T> struct Dft<5, C, T> {
  static __device__ __forceinline__ void run(C* v, T dir) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;  // cos(2pi/5), cos(4pi/5)
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;   // sin(2pi/5), sin(4pi/5)
    const C a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
    const C b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
    C r1, r2, i1, i2;
    r1.x = v[0].x + c1 * a1.x + c2 * a2.x;  r1.y = v[0].y + c1 * a1.y + c2 * a2.y;
    r2.x = v[0].x + c2 * a1.x + c1 * a2.x;  r2.y = v[0].y + c2 * a1.y + c1 * a2.y;
    C w1, w2;
    w1.x = s1 * b1.x + s2 * b2.x;  w1.y = s1 * b1.y + s2 * b2.y;
    w2.x = s2 * b1.x - s1 * b2.x;  w2.y = s2 * b1.y - s1 * b2.y;
    i1 = cmuli(w1, dir);
    i2 = cmuli(w2, dir);
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(r1, i1);
    v[4] = csub(r1, i1);
    v[2] = cadd(r2, i2);
    v[3] = csub(r2, i2);
  }
};

// One radix-R Stockham stage over np contiguous pencils (pencil p at x + p*ps) of length N whose
// sub-transforms have span Ns.  In place: every lane loads all its butterflies into registers,
// the warp synchronises, then the results are stored.  Requires np*N/R <= 32*kMaxB.
template <int R, typename C, typename T>
__device__ __forceinline__ void stage(C* x, int np, int ps, int N, int Ns, const C* tw, T dir, int lane) {
  const int nbf = N / R;
  const int tot = np * nbf;
  const int tws = N / (Ns * R);
  C v[kMaxB][R];
#pragma unroll
  for (int b = 0; b < kMaxB; ++b) {
    const int it = lane + 32 * b;
    if (it < tot) {
      const int p = it / nbf, j = it - p * nbf;
      const C* xp = x + p * ps;
      const int k = j % Ns;
#pragma unroll
      for (int t = 0; t < R; ++t) v[b][t] = xp[j + t * nbf];
      if (Ns > 1) {
#pragma unroll
        for (int t = 1; t < R; ++t) {
          C w = tw[(t * k * tws) % N];
          w.y = -dir * w.y;  // table holds e^{-2 pi i m/N}; conjugate for the inverse
          v[b][t] = cmul(v[b][t], w);
        }
      }
      Dft<R, C, T>::run(v[b], dir);
    }
  }
  __syncwarp();
#pragma unroll
  for (int b = 0; b < kMaxB; ++b) {
    const int it = lane + 32 * b;
    if (it < tot) {
      const int p = it / nbf, j = it - p * nbf;
      C* xp = x + p * ps;
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int t = 0; t < R; ++t) xp[base + t * Ns] = v[b][t];
    }
  }
  __syncwarp();
}

// Full transform of np pencils: dir = -1 forward (e^{-i}), +1 inverse (e^{+i}), unnormalised.
template <typename C, typename T>
__device__ __noinline__ void warp_fft(C* x, int np, int ps, const FftDim& d, const C* tw, T dir, int lane) {
  int Ns = 1;
  for (int s = 0; s < d.nst; ++s) {
    const int R = d.rad[s];
    if (R == 4) stage<4, C, T>(x, np, ps, d.N, Ns, tw, dir, lane);
    else if (R == 2) stage<2, C, T>(x, np, ps, d.N, Ns, tw, dir, lane);
    else if (R == 3) stage<3, C, T>(x, np, ps, d.N, Ns, tw, dir, lane);
    else stage<5, C, T>(x, np, ps, d.N, Ns, tw, dir, lane);
    Ns *= R;
  }
}


// Pass A: scatter a z-slice of the sphere, inverse FFT along x, store slab rows.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_a(LocalArgs<T> a) {
  using C = typename CT<T>::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  C* tile = tw + a.N1;
  const int u3 = blockIdx.x, nl = blockIdx.y, n = a.n0 + nl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  copy_table(tw, a.tw1, a.N1);
  const int tsz = a.W2 * a.N1p;
  for (int i = threadIdx.x; i < tsz; i += kThreads) tile[i] = C{0, 0};
  __syncthreads();
  const int g0 = a.zstart[u3], g1 = a.zstart[u3 + 1];
  const C* ps = a.psi + n * a.ld;
  for (int g = g0 + threadIdx.x; g < g1; g += kThreads) tile[a.tileidx[g]] = ps[g];
  __syncthreads();
  const int r0 = a.rowrange[2 * u3], r1 = a.rowrange[2 * u3 + 1];
  const int nrows = r1 - r0 + 1;
  for (int r = warp * a.pw1; r < nrows; r += kWarps * a.pw1)
    warp_fft<C, T>(tile + (r0 + r) * a.N1p, min(a.pw1, nrows - r), a.N1p, a.d1, tw, (T)1, lane);
  __syncthreads();
  C* dst = a.work + ((size_t)nl * a.N1 * a.W3 + u3) * a.W2;
  const size_t xs = (size_t)a.W3 * a.W2;
  for (int i = threadIdx.x; i < a.N1 * a.W2; i += kThreads) {
    const int x = i / a.W2, u2 = i - x * a.W2;
    dst[x * xs + u2] = tile[u2 * a.N1p + x];
  }
}

// Pass B: one x-plane of the slab: y inverse FFT, z inverse FFT, x V, z forward FFT, y forward FFT.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_b(LocalArgs<T> a) {
  using C = typename CT<T>::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw2 = reinterpret_cast<C*>(smraw);
  C* tw3 = tw2 + a.N2;
  C* Q = tw3 + a.N3;                 // W3 x N2p
  C* Z = Q + a.W3 * a.N2p;           // kWarps x pw3 x N3p
  const int x = blockIdx.x, nl = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  copy_table(tw2, a.tw2, a.N2);
  copy_table(tw3, a.tw3, a.N3);
  for (int i = threadIdx.x; i < a.W3 * a.N2p; i += kThreads) Q[i] = C{0, 0};
  __syncthreads();
  C* slab = a.work + ((size_t)nl * a.N1 + x) * a.W3 * a.W2;
  for (int i = threadIdx.x; i < a.W3 * a.W2; i += kThreads) {
    const int u3 = i / a.W2, u2 = i - u3 * a.W2;
    int y = (a.lo2 + u2) % a.N2;
    if (y < 0) y += a.N2;
    Q[u3 * a.N2p + y] = slab[i];
  }
  __syncthreads();
  for (int r = warp * a.pw2; r < a.W3; r += kWarps * a.pw2)
    warp_fft<C, T>(Q + r * a.N2p, min(a.pw2, a.W3 - r), a.N2p, a.d2, tw2, (T)1, lane);
  __syncthreads();
  C* Zw = Z + warp * a.pw3 * a.N3p;
  const T* vx = a.Vx + (size_t)x * a.N2 * a.N3;
  for (int y0 = warp * a.pw3; y0 < a.N2; y0 += kWarps * a.pw3) {
    const int np = min(a.pw3, a.N2 - y0);
    for (int i = lane; i < np * a.N3p; i += 32) Zw[i] = C{0, 0};
    __syncwarp();
    for (int i = lane; i < np * a.W3; i += 32) {
      const int p = i / a.W3, u3 = i - p * a.W3;
      int z = (a.lo3 + u3) % a.N3;
      if (z < 0) z += a.N3;
      Zw[p * a.N3p + z] = Q[u3 * a.N2p + y0 + p];
    }
    __syncwarp();
    warp_fft<C, T>(Zw, np, a.N3p, a.d3, tw3, (T)1, lane);
    for (int i = lane; i < np * a.N3; i += 32) {
      const int p = i / a.N3, z = i - p * a.N3;
      const T v = vx[(size_t)(y0 + p) * a.N3 + z];
      C& e = Zw[p * a.N3p + z];
      e.x *= v;
      e.y *= v;
    }
    __syncwarp();
    warp_fft<C, T>(Zw, np, a.N3p, a.d3, tw3, (T)-1, lane);
    for (int i = lane; i < np * a.W3; i += 32) {
      const int p = i / a.W3, u3 = i - p * a.W3;
      int z = (a.lo3 + u3) % a.N3;
      if (z < 0) z += a.N3;
      Q[u3 * a.N2p + y0 + p] = Zw[p * a.N3p + z];
    }
    __syncwarp();
  }
  __syncthreads();
  for (int r = warp * a.pw2; r < a.W3; r += kWarps * a.pw2)
    warp_fft<C, T>(Q + r * a.N2p, min(a.pw2, a.W3 - r), a.N2p, a.d2, tw2, (T)-1, lane);
  __syncthreads();
  for (int i = threadIdx.x; i < a.W3 * a.W2; i += kThreads) {
    const int u3 = i / a.W2, u2 = i - u3 * a.W2;
    int y = (a.lo2 + u2) % a.N2;
    if (y < 0) y += a.N2;
    slab[i] = Q[u3 * a.N2p + y];
  }
}

// Pass C: forward FFT along x of the slice's rows, gather, kinetic term and Chebyshev epilogue.
template <typename T>
__global__ void __launch_bounds__(kThreads) pass_c(LocalArgs<T> a) {
  using C = typename CT<T>::C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  C* tile = tw + a.N1;
  const int u3 = blockIdx.x, nl = blockIdx.y, n = a.n0 + nl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  copy_table(tw, a.tw1, a.N1);
  const int r0 = a.rowrange[2 * u3], r1 = a.rowrange[2 * u3 + 1];
  const int nrows = r1 - r0 + 1;
  const C* src = a.work + ((size_t)nl * a.N1 * a.W3 + u3) * a.W2;
  const size_t xs = (size_t)a.W3 * a.W2;
  for (int i = threadIdx.x; i < a.N1 * nrows; i += kThreads) {
    const int x = i / nrows, u2 = r0 + (i - x * nrows);
    tile[u2 * a.N1p + x] = src[x * xs + u2];
  }
  __syncthreads();
  for (int r = warp * a.pw1; r < nrows; r += kWarps * a.pw1)
    warp_fft<C, T>(tile + (r0 + r) * a.N1p, min(a.pw1, nrows - r), a.N1p, a.d1, tw, (T)-1, lane);
  __syncthreads();
  const int g0 = a.zstart[u3], g1 = a.zstart[u3 + 1];
  const C* ps = a.psi + n * a.ld;
  const C* pp = a.psi_prev ? a.psi_prev + n * a.ld : nullptr;
  C* po = a.out + n * a.ld;
  for (int g = g0 + threadIdx.x; g < g1; g += kThreads) {
    const C v = tile[a.tileidx[g]];
    const C p = ps[g];
    const T t = a.kin[g];
    C o;
    o.x = a.alpha * (t * p.x + v.x) + a.beta * p.x;
    o.y = a.alpha * (t * p.y + v.y) + a.beta * p.y;
    if (pp) {
      const C q = pp[g];
      o.x += a.gamma * q.x;
      o.y += a.gamma * q.y;
    }
    po[g] = o;
  }
}

// Gamma point: F = FT(V psi_a) + i FT(V psi_b) for the pair (a, b) = (2p, 2p+1) of real-space-real
// bands; the two transforms of real functions separate as
//   V psi_a(G) = (F(G) + conj F(-G)) / 2,   V psi_b(G) = (F(G) - conj F(-G)) / (2i),
// then out = alpha (T psi + V psi) + beta psi + gamma psi_prev (psi_prev may alias out).
template <typename C, typename T>
__global__ void gamma_unpack(const C* __restrict__ F, long long ld, const int* __restrict__ mirror,
                             const C* __restrict__ psi, const C* psi_prev, C* out, const T* __restrict__ kin,
                             int npw, int nb, T al, T be, T ga) {
  const long long n = (long long)npw * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / npw), g = (int)(i - (long long)b * npw);
    const C* f = F + (size_t)(b >> 1) * ld;
    const C x = f[g], y = f[mirror[g]];
    C v;
    if ((b & 1) == 0) {
      v.x = (T)0.5 * (x.x + y.x);
      v.y = (T)0.5 * (x.y - y.y);
    } else {
      v.x = (T)0.5 * (x.y + y.y);
      v.y = (T)0.5 * (y.x - x.x);
    }
    const C p = psi[(size_t)b * ld + g];
    const T t = kin[g];
    C o;
    o.x = al * (t * p.x + v.x) + be * p.x;
    o.y = al * (t * p.y + v.y) + be * p.y;
    if (psi_prev) {
      const C q = psi_prev[(size_t)b * ld + g];
      o.x += ga * q.x;
      o.y += ga * q.y;
    }
    out[(size_t)b * ld + g] = o;
  }
}

template <typename T, class Pol = RtPol>
__global__ void __launch_bounds__(kThreads) pass_a_r(LocalArgs<T> a, RegPlan rp, int scr_warp) {
  pass_a_body<T, Pol>(a, rp, scr_warp, blockIdx.x, blockIdx.y);
}
template <typename T, class Pol = RtPol>
__global__ void __launch_bounds__(kThreads) pass_b_r(LocalArgs<T> a, RegPlan rp, int scr_warp) {
  pass_b_body<T, Pol>(a, rp, scr_warp, blockIdx.x, blockIdx.y);
}
template <typename T, class Pol = RtPol>
__global__ void __launch_bounds__(kThreads) pass_c_r(LocalArgs<T> a, RegPlan rp, int scr_warp) {
  pass_c_body<T, Pol>(a, rp, scr_warp, blockIdx.x, blockIdx.y);
}

template <typename T>
struct PassKernels {
  void (*a)(LocalArgs<T>, RegPlan, int);
  void (*b)(LocalArgs<T>, RegPlan, int);
  void (*c)(LocalArgs<T>, RegPlan, int);
};

// Kernel instances for a plan: the compile-time transforms when the x split (passes A, C) or,
// in single precision, the common y/z split (pass B) has an instance.  (Double-precision pass B
// with a common y/z split runs the CTA-wide form of local_wide.cu.)
template <typename T>
PassKernels<T> pick_kernels(const RegPlan& rp) {
  PassKernels<T> k{pass_a_r<T, RtPol>, pass_b_r<T, RtPol>, pass_c_r<T, RtPol>};
  {
    const int c1 = rp.s1.A * 32 + rp.s1.B;
    const int c23 = (rp.s2.A == rp.s3.A && rp.s2.B == rp.s3.B) ? rp.s2.A * 32 + rp.s2.B : -1;
    switch (c1) {
#define KSS_CASE(x, y)                    \
  case x * 32 + y:                        \
    k.a = pass_a_r<T, CtPol<x, y>>;        \
    k.c = pass_c_r<T, CtPol<x, y>>;        \
    break;
      KSS_SPLITS(KSS_CASE)
#undef KSS_CASE
      default:
        break;
    }
    if constexpr (sizeof(T) == 4) {
      switch (c23) {
#define KSS_CASE(x, y)                    \
  case x * 32 + y:                        \
    k.b = pass_b_r<T, CtPol<x, y>>;        \
    break;
        KSS_SPLITS(KSS_CASE)
#undef KSS_CASE
        default:
          break;
      }
    }
  }
  return k;
}


int pencils_per_call(const FftDim& d) {
  int rmin = 5;
  for (int s = 0; s < d.nst; ++s) rmin = std::min(rmin, d.rad[s]);
  return std::max(1, (32 * kMaxB * rmin) / d.N);
}

template <typename T>
size_t smem_a(const LocalArgs<T>& a) {
  return sizeof(typename CT<T>::C) * ((size_t)a.N1 + (size_t)a.W2 * a.N1p);
}
template <typename T>
size_t smem_b(const LocalArgs<T>& a) {
  return sizeof(typename CT<T>::C) *
         ((size_t)a.N2 + a.N3 + (size_t)a.W3 * a.N2p + (size_t)kWarps * a.pw3 * a.N3p);
}

size_t slab_elems(kss_sys s, int ik) {
  const KData& kd = s->k[ik];
  return (size_t)s->N[0] * kd.W[2] * kd.W[1];
}

int chunk_bands(kss_sys s, int ik, int nb, size_t es) {
  const size_t per = slab_elems(s, ik) * es;
  const size_t target = kSlabChunkBytes;  // keep the slab chunk L2-resident
  return (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, target / per));
}

// Kernel arguments of the local passes for (system, k-point, band block).
template <typename T>
LocalArgs<T> local_args(kss_sys s, int ik, const void* psi, const void* psi_prev, void* out, int ld,
                        ChebCoef c) {
  using C = typename CT<T>::C;
  const bool f64 = sizeof(T) == 8;
  KData& kd = s->k[ik];
  LocalArgs<T> a{};
  a.N1 = s->N[0];
  a.N2 = s->N[1];
  a.N3 = s->N[2];
  a.N1p = a.N1 + 1;
  a.N2p = a.N2 + 1;
  a.N3p = a.N3 + 1;
  a.W2 = kd.W[1];
  a.W3 = kd.W[2];
  a.lo2 = kd.lo[1];
  a.lo3 = kd.lo[2];
  a.W1 = kd.W[0];
  a.lo1 = kd.lo[0];
  a.d1 = s->dim[0];
  a.d2 = s->dim[1];
  a.d3 = s->dim[2];
  a.pw1 = pencils_per_call(a.d1);
  a.pw2 = pencils_per_call(a.d2);
  a.pw3 = pencils_per_call(a.d3);
  a.tw1 = (const C*)(f64 ? s->d_tw64[0].p : s->d_tw32[0].p);
  a.tw2 = (const C*)(f64 ? s->d_tw64[1].p : s->d_tw32[1].p);
  a.tw3 = (const C*)(f64 ? s->d_tw64[2].p : s->d_tw32[2].p);
  a.zstart = kd.d_zstart.as<int>();
  a.rowrange = kd.d_rowrange.as<int>();
  a.tileidx = kd.d_tileidx.as<int>();
  a.kin = (const T*)(f64 ? kd.d_kin64.p : kd.d_kin32.p);
  a.Vx = (const T*)(f64 ? s->d_Vx64.p : s->d_Vx32.p);
  a.psi = (const C*)psi;
  a.psi_prev = (const C*)psi_prev;
  a.out = (C*)out;
  a.ld = ld;
  a.alpha = (T)c.alpha;
  a.beta = (T)c.beta;
  a.gamma = (T)c.gamma;
  return a;
}

// Gamma point: unpack the pair transforms in the context's pair workspace and finish the epilogue.
template <typename T>
void gamma_finish(kss_sys s, int ik, int nb, const void* psi, const void* psi_prev, void* out, int ld,
                  ChebCoef c) {
  using C = typename CT<T>::C;
  const bool f64 = sizeof(T) == 8;
  kss_ctx ctx = s->ctx;
  const KData& kd = s->k[ik];
  static const int idu = prof_register(f64 ? "gamma_unpack<f64>" : "gamma_unpack<f32>");
  ProfScope ps(ctx, idu);
  const long long n = (long long)kd.npw * nb;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32);
  gamma_unpack<C, T><<<blocks, 256, 0, ctx->stream>>>(
      ctx->ws_gpack.as<C>(), ld, kd.d_mirror.as<int>(), (const C*)psi, (const C*)psi_prev, (C*)out,
      (const T*)(f64 ? kd.d_kin64.p : kd.d_kin32.p), kd.npw, nb, (T)c.alpha, (T)c.beta, (T)c.gamma);
}

template <typename T>
void run_local(kss_sys s, int ik, int nb, const void* psi, const void* psi_prev, void* out,
               int ld, ChebCoef c) {
  using C = typename CT<T>::C;
  const bool f64 = sizeof(T) == 8;
  kss_ctx ctx = s->ctx;
  LocalArgs<T> a = local_args<T>(s, ik, psi, psi_prev, out, ld, c);
  if constexpr (sizeof(T) == 4) {
    // small cubic boxes: the whole local part in one kernel (local_fused.cu)
    if (fused_local_available(s)) {
      const bool packed = c.packed && s->k[ik].gamma && nb >= 2;
      int units = nb;
      if (packed) {
        units = (nb + 1) / 2;
        ctx->ws_gpack.ensure((size_t)units * ld * sizeof(C));
        a.packed = 1;
        a.nbands = nb;
        a.out = ctx->ws_gpack.as<C>();
        a.psi_prev = nullptr;
      }
      if (fused_local_apply(s, a, units)) {
        if (packed) gamma_finish<T>(s, ik, nb, psi, psi_prev, out, ld, c);
        KSS_CHECK_CUDA(cudaGetLastError());
        return;
      }
      a = local_args<T>(s, ik, psi, psi_prev, out, ld, c);
    }
  }
  const size_t sa = smem_a(a), sb = smem_b(a);
  const size_t smax = 227 * 1024;
  if (sa > smax || sb > smax)
    fail(KSS_ENOTSUP, "FFT box too large for the shared-memory pencil tiles of this build");
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_a<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
  const int nc = chunk_bands(s, ik, nb, sizeof(C));
  ctx->ws_local.ensure(slab_elems(s, ik) * nc * sizeof(C));
  a.work = ctx->ws_local.as<C>();
  RegPlan rp;
  if (choose_split(a.N1, rp.s1) && choose_split(a.N2, rp.s2) && choose_split(a.N3, rp.s3)) {
    const int scr_warp = std::max(rp.s1.PP * rp.s1.scr, std::max(rp.s2.PP * rp.s2.scr, rp.s3.PP * rp.s3.scr));
    const size_t es = sizeof(C);
    const size_t ra = es * ((size_t)a.N1 + (size_t)a.W2 * a.N1p + (size_t)kWarps * scr_warp);
    const size_t rb = es * ((size_t)a.N2 + a.N3 + (size_t)a.W3 * a.N2p + (size_t)kWarps * scr_warp) +
                      sizeof(int) * a.N3;
    if (ra <= smax && rb <= smax) {
      const PassKernels<T> kk = pick_kernels<T>(rp);
      KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ra));
      KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rb));
      KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ra));
      auto warp_b = [&](const LocalArgs<T>& t, int m) {
        kk.b<<<dim3(t.N1, m), kThreads, rb, ctx->stream>>>(t, rp, scr_warp);
      };
      const PassBSched sb = pass_b_schedule<T>(ctx, a, rp.s2, true);
      const bool wx = wide_pass_x<T>(a, 0, 0, nullptr, true);
      if (sb.threads) a.Vpi = (const T*)vpi_view(s, sb.A, sb.B, f64);
      static const int ida = prof_register(f64 ? "local_pass_a<f64>" : "local_pass_a<f32>");
      static const int idb = prof_register(f64 ? "local_pass_b<f64>" : "local_pass_b<f32>");
      static const int idc = prof_register(f64 ? "local_pass_c<f64>" : "local_pass_c<f32>");
      // Gamma point with real-space-real bands: the passes run over band pairs
      const KData& kd = s->k[ik];
      const bool packed = c.packed && kd.gamma && nb >= 2;
      int units = nb;
      if (packed) {
        units = (nb + 1) / 2;
        ctx->ws_gpack.ensure((size_t)units * ld * sizeof(C));
        a.packed = 1;
        a.nbands = nb;
        a.out = ctx->ws_gpack.as<C>();
        a.psi_prev = nullptr;
      }
      for (int n0 = 0; n0 < units; n0 += nc) {
        const int m = std::min(nc, units - n0);
        a.n0 = n0;
        {
          ProfScope ps(ctx, ida);
          if (!(wx && wide_pass_x<T>(a, 0, m, ctx->stream, false)))
            kk.a<<<dim3(a.W3, m), kThreads, ra, ctx->stream>>>(a, rp, scr_warp);
        }
        {
          ProfScope ps(ctx, idb);
          if (!(sb.threads && wide_pass_b<T>(a, sb.A, sb.B, sb.threads, m, ctx->stream, false))) warp_b(a, m);
        }
        {
          ProfScope ps(ctx, idc);
          if (!(wx && wide_pass_x<T>(a, 1, m, ctx->stream, false)))
            kk.c<<<dim3(a.W3, m), kThreads, ra, ctx->stream>>>(a, rp, scr_warp);
        }
      }
      if (packed) gamma_finish<T>(s, ik, nb, psi, psi_prev, out, ld, c);
      KSS_CHECK_CUDA(cudaGetLastError());
      return;
    }
  }
  static const int ida = prof_register(f64 ? "local_pass_a<f64>" : "local_pass_a<f32>");
  static const int idb = prof_register(f64 ? "local_pass_b<f64>" : "local_pass_b<f32>");
  static const int idc = prof_register(f64 ? "local_pass_c<f64>" : "local_pass_c<f32>");
  for (int n0 = 0; n0 < nb; n0 += nc) {
    const int m = std::min(nc, nb - n0);
    a.n0 = n0;
    {
      ProfScope ps(ctx, ida);
      pass_a<T><<<dim3(a.W3, m), kThreads, sa, ctx->stream>>>(a);
    }
    {
      ProfScope ps(ctx, idb);
      pass_b<T><<<dim3(a.N1, m), kThreads, sb, ctx->stream>>>(a);
    }
    {
      ProfScope ps(ctx, idc);
      pass_c<T><<<dim3(a.W3, m), kThreads, sa, ctx->stream>>>(a);
    }
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

// The local passes on a caller-provided slab workspace of nc bands (no allocation, no profiling
// events).  Same kernels as run_local; the pass-B schedule comes from the autotuner's table or
// the built-in choice (no tuning, which would allocate a scratch slab).
template <typename T>
void run_local_ws(kss_sys s, int ik, int nb, const void* psi, void* out, int ld, void* work, int nc) {
  using C = typename CT<T>::C;
  const bool f64 = sizeof(T) == 8;
  kss_ctx ctx = s->ctx;
  KData& kd = s->k[ik];
  LocalArgs<T> a{};
  a.N1 = s->N[0];
  a.N2 = s->N[1];
  a.N3 = s->N[2];
  a.N1p = a.N1 + 1;
  a.N2p = a.N2 + 1;
  a.N3p = a.N3 + 1;
  a.W2 = kd.W[1];
  a.W3 = kd.W[2];
  a.lo2 = kd.lo[1];
  a.lo3 = kd.lo[2];
  a.W1 = kd.W[0];
  a.lo1 = kd.lo[0];
  a.d1 = s->dim[0];
  a.d2 = s->dim[1];
  a.d3 = s->dim[2];
  a.pw1 = pencils_per_call(a.d1);
  a.pw2 = pencils_per_call(a.d2);
  a.pw3 = pencils_per_call(a.d3);
  a.tw1 = (const C*)(f64 ? s->d_tw64[0].p : s->d_tw32[0].p);
  a.tw2 = (const C*)(f64 ? s->d_tw64[1].p : s->d_tw32[1].p);
  a.tw3 = (const C*)(f64 ? s->d_tw64[2].p : s->d_tw32[2].p);
  a.zstart = kd.d_zstart.as<int>();
  a.rowrange = kd.d_rowrange.as<int>();
  a.tileidx = kd.d_tileidx.as<int>();
  a.kin = (const T*)(f64 ? kd.d_kin64.p : kd.d_kin32.p);
  a.Vx = (const T*)(f64 ? s->d_Vx64.p : s->d_Vx32.p);
  a.psi = (const C*)psi;
  a.psi_prev = nullptr;
  a.out = (C*)out;
  a.ld = ld;
  a.alpha = (T)1;
  a.beta = (T)0;
  a.gamma = (T)0;
  a.work = (C*)work;
  const size_t smax = 227 * 1024;
  RegPlan rp;
  if (choose_split(a.N1, rp.s1) && choose_split(a.N2, rp.s2) && choose_split(a.N3, rp.s3)) {
    const int scr_warp = std::max(rp.s1.PP * rp.s1.scr, std::max(rp.s2.PP * rp.s2.scr, rp.s3.PP * rp.s3.scr));
    const size_t es = sizeof(C);
    const size_t ra = es * ((size_t)a.N1 + (size_t)a.W2 * a.N1p + (size_t)kWarps * scr_warp);
    const size_t rb = es * ((size_t)a.N2 + a.N3 + (size_t)a.W3 * a.N2p + (size_t)kWarps * scr_warp) +
                      sizeof(int) * a.N3;
    if (ra <= smax && rb <= smax) {
      const PassKernels<T> kk = pick_kernels<T>(rp);
      KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ra));
      KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rb));
      KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ra));
      auto warp_b = [&](const LocalArgs<T>& t, int m) {
        kk.b<<<dim3(t.N1, m), kThreads, rb, ctx->stream>>>(t, rp, scr_warp);
      };
      PassBSched sb = pass_b_schedule<T>(ctx, a, rp.s2, false);  // no tuning here
      const bool wx = wide_pass_x<T>(a, 0, 0, nullptr, true);
      // The CTA-wide form needs V in its split's layout; that view is built (allocated) by the
      // first ordinary application, and without it this path takes the per-warp form.
      if (sb.threads) {
        auto& cache = f64 ? s->vpi64 : s->vpi32;
        auto it = cache.find(sb.A * 32 + sb.B);
        if (it != cache.end()) a.Vpi = (const T*)it->second.p;
        else sb.threads = 0;
      }
      for (int n0 = 0; n0 < nb; n0 += nc) {
        const int m = std::min(nc, nb - n0);
        a.n0 = n0;
        if (!(wx && wide_pass_x<T>(a, 0, m, ctx->stream, false)))
          kk.a<<<dim3(a.W3, m), kThreads, ra, ctx->stream>>>(a, rp, scr_warp);
        if (!(sb.threads && wide_pass_b<T>(a, sb.A, sb.B, sb.threads, m, ctx->stream, false))) warp_b(a, m);
        if (!(wx && wide_pass_x<T>(a, 1, m, ctx->stream, false)))
          kk.c<<<dim3(a.W3, m), kThreads, ra, ctx->stream>>>(a, rp, scr_warp);
      }
      KSS_CHECK_CUDA(cudaGetLastError());
      return;
    }
  }
  const size_t sa = smem_a(a), sb = smem_b(a);
  if (sa > smax || sb > smax)
    fail(KSS_ENOTSUP, "FFT box too large for the shared-memory pencil tiles of this build");
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_a<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
  for (int n0 = 0; n0 < nb; n0 += nc) {
    const int m = std::min(nc, nb - n0);
    a.n0 = n0;
    pass_a<T><<<dim3(a.W3, m), kThreads, sa, ctx->stream>>>(a);
    pass_b<T><<<dim3(a.N1, m), kThreads, sb, ctx->stream>>>(a);
    pass_c<T><<<dim3(a.W3, m), kThreads, sa, ctx->stream>>>(a);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

template <typename T>
void warp_pass_b(kss_ctx ctx, const LocalArgs<T>& a, int nbands) {
  RegPlan rp;
  if (!(choose_split(a.N1, rp.s1) && choose_split(a.N2, rp.s2) && choose_split(a.N3, rp.s3)))
    fail(KSS_ENOTSUP, "FFT length without a two-codelet split");
  const int scr_warp = std::max(rp.s1.PP * rp.s1.scr, std::max(rp.s2.PP * rp.s2.scr, rp.s3.PP * rp.s3.scr));
  const size_t es = sizeof(typename CT<T>::C);
  const size_t rb = es * ((size_t)a.N2 + a.N3 + (size_t)a.W3 * a.N2p + (size_t)kWarps * scr_warp) +
                    sizeof(int) * a.N3;
  const PassKernels<T> kk = pick_kernels<T>(rp);
  KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rb));
  kk.b<<<dim3(a.N1, nbands), kThreads, rb, ctx->stream>>>(a, rp, scr_warp);
}
template void warp_pass_b<double>(kss_ctx, const LocalArgs<double>&, int);
template void warp_pass_b<float>(kss_ctx, const LocalArgs<float>&, int);

template <typename T>
void pass_a_chunks(kss_sys s, int ik, int nb, const void* psi, int ld,
                   const std::function<void(const LocalArgs<T>&, int)>& after) {
  using C = typename CT<T>::C;
  kss_ctx ctx = s->ctx;
  LocalArgs<T> a = local_args<T>(s, ik, psi, nullptr, nullptr, ld, ChebCoef{1.0, 0.0, 0.0});
  RegPlan rp;
  if (!(choose_split(a.N1, rp.s1) && choose_split(a.N2, rp.s2) && choose_split(a.N3, rp.s3)))
    fail(KSS_ENOTSUP, "FFT length without a two-codelet split");
  const int scr_warp = std::max(rp.s1.PP * rp.s1.scr, std::max(rp.s2.PP * rp.s2.scr, rp.s3.PP * rp.s3.scr));
  const size_t ra = sizeof(C) * ((size_t)a.N1 + (size_t)a.W2 * a.N1p + (size_t)kWarps * scr_warp);
  if (ra > 227 * 1024) fail(KSS_ENOTSUP, "FFT box too large for the shared-memory pencil tiles");
  const PassKernels<T> kk = pick_kernels<T>(rp);
  KSS_CHECK_CUDA(cudaFuncSetAttribute(kk.a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ra));
  const int nc = chunk_bands(s, ik, nb, sizeof(C));
  ctx->ws_local.ensure(slab_elems(s, ik) * nc * sizeof(C));
  a.work = ctx->ws_local.as<C>();
  static const int ida = prof_register(sizeof(T) == 8 ? "local_pass_a<f64>" : "local_pass_a<f32>");
  for (int n0 = 0; n0 < nb; n0 += nc) {
    const int m = std::min(nc, nb - n0);
    a.n0 = n0;
    {
      ProfScope ps(ctx, ida);
      kk.a<<<dim3(a.W3, m), kThreads, ra, ctx->stream>>>(a, rp, scr_warp);
    }
    after(a, m);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}
template void pass_a_chunks<double>(kss_sys, int, int, const void*, int,
                                    const std::function<void(const LocalArgs<double>&, int)>&);
template void pass_a_chunks<float>(kss_sys, int, int, const void*, int,
                                   const std::function<void(const LocalArgs<float>&, int)>&);

size_t local_slab_bytes_per_band(kss_sys s, int ik, kss_precision prec) {
  return slab_elems(s, ik) * (prec == KSS_PREC_FP64 ? 16 : 8);
}

void local_apply_ws(kss_sys s, int ik, int nb, const void* psi, void* out, int ld,
                    kss_precision prec, void* work, int nc) {
  if (prec == KSS_PREC_FP64)
    run_local_ws<double>(s, ik, nb, psi, out, ld, work, nc);
  else
    run_local_ws<float>(s, ik, nb, psi, out, ld, work, nc);
}

size_t local_workspace_bytes(kss_sys s, int ik, int nb, kss_precision prec) {
  const size_t es = prec == KSS_PREC_FP64 ? 16 : 8;
  return slab_elems(s, ik) * chunk_bands(s, ik, nb, es) * es;
}

template <typename T>
__global__ void vpi_gather(const T* __restrict__ vx, T* __restrict__ out, int N1, int N, int A, int B) {
  const long long n = (long long)N1 * N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % N);
    const long long r = i / N;
    const int z = (int)(r % N), x = (int)(r / N);
    const int k = p / B, k2 = p - k * B;
    const int y = k + A * k2;
    out[i] = vx[((size_t)x * N + y) * N + z];
  }
}

const void* vpi_view(kss_sys s, int A, int B, bool f64) {
  const int code = A * 32 + B;
  auto& cache = f64 ? s->vpi64 : s->vpi32;
  auto it = cache.find(code);
  if (it != cache.end()) return it->second.p;
  KSS_REQUIRE(s->N[1] == s->N[2] && A * B == s->N[1], "V view: split does not match the box");
  const int N1 = s->N[0], N = s->N[1];
  const long long n = (long long)N1 * N * N;
  DevBuf& d = cache[code];
  d.alloc((size_t)n * (f64 ? 8 : 4));
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32);
  if (f64)
    vpi_gather<double><<<blocks, 256, 0, s->ctx->stream>>>(s->d_Vx64.as<double>(), d.as<double>(), N1, N, A, B);
  else
    vpi_gather<float><<<blocks, 256, 0, s->ctx->stream>>>(s->d_Vx32.as<float>(), d.as<float>(), N1, N, A, B);
  KSS_CHECK_CUDA(cudaGetLastError());
  return d.p;
}

// Split-BF16 forms of the (static) complex64 projector table, built on first use per k-point.
const void* beta_split_cn(kss_sys s, int ik) {
  KData& kd = s->k[ik];
  if (!kd.d_btc_cn.p) {
    kd.d_btc_cn.alloc(tc_split_cn_bytes(s->nproj, kd.npw));
    tc_split_cn(s->ctx, s->nproj, kd.npw, kd.d_beta32.p, kd.npw, kd.d_btc_cn.p);
  }
  return kd.d_btc_cn.p;
}
const void* beta_split_nn(kss_sys s, int ik) {
  KData& kd = s->k[ik];
  if (!kd.d_btc_nn.p) {
    kd.d_btc_nn.alloc(tc_split_nn_bytes(kd.npw, s->nproj));
    tc_split_nn(s->ctx, kd.npw, s->nproj, kd.d_beta32.p, kd.npw, kd.d_btc_nn.p);
  }
  return kd.d_btc_nn.p;
}

const OzOperand& beta_oz_cn(kss_sys s, int ik) {
  KData& kd = s->k[ik];
  if (!kd.d_oz_cn.p) {
    kd.d_oz_cn.alloc(oz_operand_bytes(2 * s->nproj, kd.npw));
    kd.oz_cn = oz_prepare(s->ctx, OZ_CN_A, s->nproj, kd.npw, kd.d_beta64.p, kd.npw, kd.d_oz_cn.p);
  }
  return kd.oz_cn;
}
const OzOperand& beta_oz_nn(kss_sys s, int ik) {
  KData& kd = s->k[ik];
  if (!kd.d_oz_nn.p) {
    kd.d_oz_nn.alloc(oz_operand_bytes(2 * kd.npw, s->nproj));
    kd.oz_nn = oz_prepare(s->ctx, OZ_MMAJOR_A, kd.npw, s->nproj, kd.d_beta64.p, kd.npw, kd.d_oz_nn.p);
  }
  return kd.oz_nn;
}

void apply_local(kss_sys s, int ik, int nb, const void* psi, void* out, int ld, kss_precision prec) {
  if (nb == 0) return;
  if (prec == KSS_PREC_FP64)
    run_local<double>(s, ik, nb, psi, nullptr, out, ld, ChebCoef{1.0, 0.0, 0.0});
  else
    run_local<float>(s, ik, nb, psi, nullptr, out, ld, ChebCoef{1.0, 0.0, 0.0});
}

void apply_h(kss_sys s, int ik, int nb, const void* psi, const void* psi_prev, void* out, int ld,
             ChebCoef c, kss_precision prec) {
  KSS_REQUIRE(ik >= 0 && ik < (int)s->k.size(), "k-point index out of range");
  KSS_REQUIRE(nb >= 0, "nb < 0");
  KSS_REQUIRE(prec == KSS_PREC_FP64 || prec == KSS_PREC_MIXED, "unknown precision");
  const KData& kd = s->k[ik];
  KSS_REQUIRE(ld >= kd.npw, "ld < npw");
  if (nb == 0) return;
  KSS_REQUIRE(psi && out, "null psi or out");
  KSS_REQUIRE(psi != out, "psi and out must not overlap");
  kss_ctx ctx = s->ctx;
  const bool f64 = prec == KSS_PREC_FP64;
  const size_t es = f64 ? 16 : 8;
  // Nonlocal, first half: projector coefficients C = beta^H psi, scaled to alpha * D * C.
  if (s->nproj) {
    ctx->ws_cprj.ensure((size_t)s->nproj * nb * es);
    if (f64)
      oz_gemm_cn(ctx, s->nproj, nb, kd.npw, kd.d_beta64.p, kd.npw, psi, ld, ctx->ws_cprj.p, s->nproj, 1.0, 0.0,
                 0.0, 0.0, "cprj", &beta_oz_cn(s, ik));
    else if (c.fp32_proj)
      gemm_cn(ctx, false, s->nproj, nb, kd.npw, kd.d_beta32.p, kd.npw, psi, ld, ctx->ws_cprj.p, s->nproj, 1.0, 0.0,
              0.0, 0.0, "cprj");
    else
      tc_gemm_cn_split(ctx, s->nproj, nb, kd.npw, beta_split_cn(s, ik), psi, ld, ctx->ws_cprj.p, s->nproj,
                       1.0, 0.0, 0.0, 0.0, "cprj");
    scale_rows(ctx, f64, s->nproj, nb, ctx->ws_cprj.p, s->nproj, f64 ? s->d_D64.p : s->d_D32.p,
               c.alpha);
  }
  if (f64)
    run_local<double>(s, ik, nb, psi, psi_prev, out, ld, c);
  else
    run_local<float>(s, ik, nb, psi, psi_prev, out, ld, c);
  // Nonlocal, second half: out += beta (alpha D C).
  if (s->nproj) {
    if (f64)
      oz_gemm_nn(ctx, kd.npw, nb, s->nproj, kd.d_beta64.p, kd.npw, ctx->ws_cprj.p, s->nproj, out, ld, 1.0, 0.0,
                 1.0, 0.0, "nonlocal", &beta_oz_nn(s, ik));
    else if (c.fp32_proj)
      gemm_nn(ctx, false, kd.npw, nb, s->nproj, kd.d_beta32.p, kd.npw, ctx->ws_cprj.p, s->nproj, out, ld, 1.0, 0.0,
              1.0, 0.0, "nonlocal");
    else
      tc_gemm_nn_split(ctx, kd.npw, nb, s->nproj, beta_split_nn(s, ik), ctx->ws_cprj.p, s->nproj, out, ld,
                       1.0, 0.0, 1.0, 0.0, "nonlocal");
  }
}

}  // namespace kss

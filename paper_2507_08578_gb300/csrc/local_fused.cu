// Local part of the H application for small cubic FFT boxes in single precision, in one kernel
// (kinetic + local potential through 3D FFTs batched over bands, §5.1): scatter of the band's
// plane waves -> inverse FFT along x, y, z -> x V(r) -> forward FFT along z, y, x -> gather and
// Chebyshev epilogue, with the whole N^3 box of one band held in shared memory.  When the box
// and the potential fit in one SM (complex64 box + FP32 V: N <= 25), this replaces the three-pass
// slab pipeline: no slab in global memory, so the band's coefficients are read and its result
// written once (DRAM bytes per band = the algorithmic 2 npw words, plus psi_prev).
//
// Organisation.  A persistent grid (one CTA per SM) loops over bands.  At start each CTA stages
// the potential (V/N^3, FP32) into shared memory with one bulk copy of the TMA engine
// (cp.async.bulk, completion on an mbarrier, bounded wait) and keeps it for all its bands.  The
// transforms are two-level (N = A x B register codelets of fft_reg.cuh); every stage is one
// CTA-wide loop over (pencil, sub-transform) tasks with the pencil index fastest across lanes:
//   inverse, stage 1: task (pencil, r < B) reads elements r + B i (i < A), DFT-A, twiddle, and
//                     writes them back; stage 2: task (pencil, k < A) reads the B contiguous
//                     positions j + B k, DFT-B, writes back: position j + B k then holds index
//                     k + A j (digit-reversed order);
//   forward,  stage 1: task (pencil, r < A) reads the B contiguous positions (digit-reversed
//                     input), DFT-B, twiddle; stage 2: task (pencil, q < B) reads q + B m, DFT-A,
//                     writes index q + B k in natural order.
// Between the inverse and forward transforms every dimension is in digit-reversed order, so V is
// staged in that order (a permuted copy built once per system).  Pruning by the sphere window:
// only the W2 x W3 x-pencils that can hold plane waves are transformed along x, only the W3 z
// planes along y; inverse loads outside the window read zero and forward stores outside it are
// skipped, so no zero-fill of the box is needed beyond the x-pencils the scatter writes into.
// Row pitch N | 1 (odd) keeps lanes that step through pencils on distinct shared-memory banks.
#include <cstdint>

#include "batch_kernels.cuh"
#include "fft_reg.cuh"
#include "kss_internal.h"
#include "local_fused.h"
#include "tc_common.cuh"

namespace kss {

namespace {

constexpr int kFusedThreads = 512;
constexpr unsigned long long kStageWaitNs = 2000000000ull;  // bounded wait for the V copy

struct FusedArgs {
  int W2, W3, lo2, lo3, N1p;
  int units;     // bands, or band pairs in packed (Gamma) mode
  int nbands;    // bands in psi (packed: the last pair may hold one band)
  int packed;    // Gamma point: unit n is the pair (2n, 2n+1) as psi_2n + i psi_2n+1; the raw
                 // transform goes to out and a separate kernel unpacks and finishes
  int vbytes;    // bytes of the staged potential (a multiple of 16)
  const float2* tw;   // e^{-2 pi i m / N}, m < N
  const float* vdr;   // V / N^3 at the digit-reversed box positions (padded)
  const int* zstart;  // sphere points of z-slice u3: [zstart[u3], zstart[u3 + 1])
  const int* tileidx; // u2 * N1p + x of each sphere point
  const float* kin;
  const float2* psi;
  const float2* psi_prev;
  float2* out;
  long long ld;
  float alpha, beta, gamma;
  const float* coef;  // when set: alpha, beta, gamma read from device memory (graph replays)
  int* err;           // raised when the staging wait gives up
};

// Shared-memory layout: [V][twiddles][box][maps][mbarrier].  Maps (N + 1 ints each): y and z
// coordinate -> window index or -1, window index -> coordinate for y and z, and the slice starts
// of the sphere points (W3 + 1 <= N + 1 entries).
struct FusedLayout {
  size_t tw, box, maps, bar, total;
};
__host__ __device__ inline FusedLayout fused_layout(int N, int vbytes) {
  const int P1 = N | 1;
  FusedLayout L;
  L.tw = (size_t)vbytes;
  L.box = L.tw + sizeof(float2) * (size_t)N;
  L.maps = L.box + sizeof(float2) * (size_t)N * N * P1;
  L.bar = (L.maps + sizeof(int) * 5 * (size_t)(N + 1) + 7) & ~(size_t)7;
  L.total = L.bar + 8;
  return L;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"((unsigned long long)src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ float2 conjf2(float2 w) { return make_float2(w.x, -w.y); }

// Shared-memory views of one CTA.
struct FusedSmem {
  const float* V;
  float2* tw;
  float2* box;
  int *ymap, *zmap, *ywin, *zwin, *zst;
  uint32_t bar;
};
template <int N>
__device__ __forceinline__ FusedSmem fused_smem(unsigned char* fsm, int vbytes) {
  const FusedLayout L = fused_layout(N, vbytes);
  FusedSmem m;
  m.V = reinterpret_cast<const float*>(fsm);
  m.tw = reinterpret_cast<float2*>(fsm + L.tw);
  m.box = reinterpret_cast<float2*>(fsm + L.box);
  m.ymap = reinterpret_cast<int*>(fsm + L.maps);
  m.zmap = m.ymap + (N + 1);
  m.ywin = m.zmap + (N + 1);
  m.zwin = m.ywin + (N + 1);
  m.zst = m.zwin + (N + 1);
  m.bar = tc::smem_u32(fsm + L.bar);
  return m;
}

// Once per kernel, thread 0: the mbarrier of the potential copies.
__device__ __forceinline__ void fused_init(const FusedSmem& m) {
  if (threadIdx.x == 0) {
    tc::mbar_init(m.bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
}

// Stage one unit: its potential (bulk copy, completion phase `parity` of the mbarrier), twiddles,
// window maps and slice starts.  Called by every thread after the previous band's last read of
// shared memory; returns false (every thread) when the copy's bounded wait gave up.
template <int N>
__device__ bool fused_stage(unsigned char* fsm, const FusedSmem& m, const FusedArgs& a, uint32_t parity) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic reads of V first
    tc::mbar_expect_tx(m.bar, (uint32_t)a.vbytes);
    bulk_load(tc::smem_u32(fsm), a.vdr, (uint32_t)a.vbytes, m.bar);
  }
  for (int i = threadIdx.x; i < N; i += kFusedThreads) {
    m.tw[i] = a.tw[i];
    int u = (i - a.lo2) % N;
    if (u < 0) u += N;
    m.ymap[i] = u < a.W2 ? u : -1;
    int w = (i - a.lo3) % N;
    if (w < 0) w += N;
    m.zmap[i] = w < a.W3 ? w : -1;
    int yy = (a.lo2 + i) % N;
    if (yy < 0) yy += N;
    m.ywin[i] = yy;
    int zz = (a.lo3 + i) % N;
    if (zz < 0) zz += N;
    m.zwin[i] = zz;
  }
  for (int i = threadIdx.x; i <= a.W3; i += kFusedThreads) m.zst[i] = a.zstart[i];
  if (threadIdx.x == 0) {
    int ok = tc::mbar_wait(m.bar, parity, kStageWaitNs) ? 1 : 0;
    if (!ok) {
      atomicExch(a.err, 1);
      tc::mbar_wait(m.bar, parity, kStageWaitNs);  // the copy still in flight, once more (bounded)
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The local part for band (or pair) n of the staged unit.
template <int A, int B>
__device__ void fused_band(const FusedSmem& m, const FusedArgs& a, int n) {
  constexpr int N = A * B, P1 = N | 1, P2 = N * P1, NN = N * N, NT = kFusedThreads;
  const float* V = m.V;
  const float2* tw = m.tw;
  float2* box = m.box;
  const int* ymap = m.ymap;
  const int* zmap = m.zmap;
  const int* ywin = m.ywin;
  const int* zwin = m.zwin;
  const int* zst = m.zst;
  const int tid = threadIdx.x;
  const int W2 = a.W2, W3 = a.W3;
  const int npx = W2 * W3;  // x pencils: (y, z) in the sphere window
  const int npy = N * W3;   // y pencils: (x position, z in the window)
  const fftr::FastDiv dw2(W2), dnpx(npx), dnpy(npy), dn1p(a.N1p);
  const int g0 = zst[0], g1 = zst[W3];
  // slice of a sphere point: the last u3 with zst[u3] <= g
  auto slice_of = [&](int g) {
    int lo = 0, hi = W3;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (zst[mid] <= g) lo = mid;
      else hi = mid;
    }
    return lo;
  };
  // ---- zero the window's x pencils, scatter the plane waves ----
  for (int i = tid; i < npx * N; i += NT) {
    const int p = i / N, x = i - p * N;
    const int u3 = dw2(p), u2 = p - u3 * W2;
    box[zwin[u3] * P2 + ywin[u2] * P1 + x] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  {
    const float2* pa = a.psi + (size_t)(a.packed ? 2 * n : n) * a.ld;
    const float2* pb = a.packed && 2 * n + 1 < a.nbands ? pa + a.ld : nullptr;
    for (int g = g0 + tid; g < g1; g += NT) {
      const int u3 = slice_of(g);
      const int t = a.tileidx[g];
      const int u2 = dn1p(t), x = t - u2 * a.N1p;
      float2 v = pa[g];
      if (pb) {  // psi_2n + i psi_2n+1
        const float2 w = pb[g];
        v.x -= w.y;
        v.y += w.x;
      }
      box[zwin[u3] * P2 + ywin[u2] * P1 + x] = v;
    }
  }
  __syncthreads();
  // ---- x, inverse ----
  for (int t = tid; t < npx * B; t += NT) {
    const int r = dnpx(t), p = t - r * npx;
    const int u3 = dw2(p), u2 = p - u3 * W2;
    float2* row = box + zwin[u3] * P2 + ywin[u2] * P1;
    float2 v[A];
#pragma unroll
    for (int i = 0; i < A; ++i) v[i] = row[r + B * i];
    fftr::rdft<A>(v, 1.f);
#pragma unroll
    for (int k = 1; k < A; ++k) v[k] = fftr::mul(v[k], conjf2(tw[r * k]));
#pragma unroll
    for (int k = 0; k < A; ++k) row[r + B * k] = v[k];
  }
  __syncthreads();
  for (int t = tid; t < npx * A; t += NT) {
    const int k = dnpx(t), p = t - k * npx;
    const int u3 = dw2(p), u2 = p - u3 * W2;
    float2* row = box + zwin[u3] * P2 + ywin[u2] * P1 + B * k;
    float2 v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = row[j];
    fftr::rdft<B>(v, 1.f);
#pragma unroll
    for (int j = 0; j < B; ++j) row[j] = v[j];
  }
  __syncthreads();
  // ---- y, inverse (the W3 window planes; rows outside the y window read as zero) ----
  for (int t = tid; t < npy * B; t += NT) {
    const int r = dnpy(t), p = t - r * npy;
    const int u3 = p / N, x = p - u3 * N;
    float2* col = box + zwin[u3] * P2 + x;
    float2 v[A];
#pragma unroll
    for (int i = 0; i < A; ++i) v[i] = ymap[r + B * i] >= 0 ? col[(r + B * i) * P1] : make_float2(0.f, 0.f);
    fftr::rdft<A>(v, 1.f);
#pragma unroll
    for (int k = 1; k < A; ++k) v[k] = fftr::mul(v[k], conjf2(tw[r * k]));
#pragma unroll
    for (int k = 0; k < A; ++k) col[(r + B * k) * P1] = v[k];
  }
  __syncthreads();
  for (int t = tid; t < npy * A; t += NT) {
    const int k = dnpy(t), p = t - k * npy;
    const int u3 = p / N, x = p - u3 * N;
    float2* col = box + zwin[u3] * P2 + x + (B * k) * P1;
    float2 v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = col[j * P1];
    fftr::rdft<B>(v, 1.f);
#pragma unroll
    for (int j = 0; j < B; ++j) col[j * P1] = v[j];
  }
  __syncthreads();
  // ---- z, inverse stage 1 (every (x, y) column; planes outside the z window read as zero) ----
  for (int t = tid; t < NN * B; t += NT) {
    const int r = t / NN, p = t - r * NN;
    float2* col = box + (p / N) * P1 + (p % N);
    float2 v[A];
#pragma unroll
    for (int i = 0; i < A; ++i) v[i] = zmap[r + B * i] >= 0 ? col[(r + B * i) * P2] : make_float2(0.f, 0.f);
    fftr::rdft<A>(v, 1.f);
#pragma unroll
    for (int k = 1; k < A; ++k) v[k] = fftr::mul(v[k], conjf2(tw[r * k]));
#pragma unroll
    for (int k = 0; k < A; ++k) col[(r + B * k) * P2] = v[k];
  }
  __syncthreads();
  // ---- z, inverse stage 2, x V, forward stage 1 (in registers) ----
  for (int t = tid; t < NN * A; t += NT) {
    const int k = t / NN, p = t - k * NN;
    float2* col = box + (p / N) * P1 + (p % N) + (B * k) * P2;
    const float* vz = V + (size_t)(B * k) * NN + p;  // position z' = B k + j at vz[j NN]
    float2 v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = col[j * P2];
    fftr::rdft<B>(v, 1.f);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const float vv = vz[j * NN];
      v[j].x *= vv;
      v[j].y *= vv;
    }
    fftr::rdft<B>(v, -1.f);
#pragma unroll
    for (int q = 1; q < B; ++q) v[q] = fftr::mul(v[q], tw[k * q]);
#pragma unroll
    for (int q = 0; q < B; ++q) col[q * P2] = v[q];
  }
  __syncthreads();
  // ---- z, forward stage 2: only the window planes are kept ----
  for (int t = tid; t < NN * B; t += NT) {
    const int q = t / NN, p = t - q * NN;
    float2* col = box + (p / N) * P1 + (p % N);
    float2 v[A];
#pragma unroll
    for (int m = 0; m < A; ++m) v[m] = col[(q + B * m) * P2];
    fftr::rdft<A>(v, -1.f);
#pragma unroll
    for (int k = 0; k < A; ++k)
      if (zmap[q + B * k] >= 0) col[(q + B * k) * P2] = v[k];
  }
  __syncthreads();
  // ---- y, forward (window planes; only the window rows are kept) ----
  for (int t = tid; t < npy * A; t += NT) {
    const int r = dnpy(t), p = t - r * npy;
    const int u3 = p / N, x = p - u3 * N;
    float2* col = box + zwin[u3] * P2 + x + (B * r) * P1;
    float2 v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = col[j * P1];
    fftr::rdft<B>(v, -1.f);
#pragma unroll
    for (int q = 1; q < B; ++q) v[q] = fftr::mul(v[q], tw[r * q]);
#pragma unroll
    for (int q = 0; q < B; ++q) col[q * P1] = v[q];
  }
  __syncthreads();
  for (int t = tid; t < npy * B; t += NT) {
    const int q = dnpy(t), p = t - q * npy;
    const int u3 = p / N, x = p - u3 * N;
    float2* col = box + zwin[u3] * P2 + x;
    float2 v[A];
#pragma unroll
    for (int m = 0; m < A; ++m) v[m] = col[(q + B * m) * P1];
    fftr::rdft<A>(v, -1.f);
#pragma unroll
    for (int k = 0; k < A; ++k)
      if (ymap[q + B * k] >= 0) col[(q + B * k) * P1] = v[k];
  }
  __syncthreads();
  // ---- x, forward (window pencils) ----
  for (int t = tid; t < npx * A; t += NT) {
    const int r = dnpx(t), p = t - r * npx;
    const int u3 = dw2(p), u2 = p - u3 * W2;
    float2* row = box + zwin[u3] * P2 + ywin[u2] * P1 + B * r;
    float2 v[B];
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = row[j];
    fftr::rdft<B>(v, -1.f);
#pragma unroll
    for (int q = 1; q < B; ++q) v[q] = fftr::mul(v[q], tw[r * q]);
#pragma unroll
    for (int q = 0; q < B; ++q) row[q] = v[q];
  }
  __syncthreads();
  for (int t = tid; t < npx * B; t += NT) {
    const int q = dnpx(t), p = t - q * npx;
    const int u3 = dw2(p), u2 = p - u3 * W2;
    float2* row = box + zwin[u3] * P2 + ywin[u2] * P1;
    float2 v[A];
#pragma unroll
    for (int m = 0; m < A; ++m) v[m] = row[q + B * m];
    fftr::rdft<A>(v, -1.f);
#pragma unroll
    for (int k = 0; k < A; ++k) row[q + B * k] = v[k];
  }
  __syncthreads();
  // ---- gather and epilogue: out = alpha (T psi + V psi) + beta psi + gamma psi_prev ----
  {
    float2* po = a.out + (size_t)n * a.ld;
    const float2* ps = a.psi + (size_t)n * a.ld;
    const float2* pp = a.psi_prev ? a.psi_prev + (size_t)n * a.ld : nullptr;
    const float al = a.coef ? a.coef[0] : a.alpha;
    const float be = a.coef ? a.coef[1] : a.beta;
    const float ga = a.coef ? a.coef[2] : a.gamma;
    for (int g = g0 + tid; g < g1; g += NT) {
      const int u3 = slice_of(g);
      const int t = a.tileidx[g];
      const int u2 = dn1p(t), x = t - u2 * a.N1p;
      const float2 v = box[zwin[u3] * P2 + ywin[u2] * P1 + x];
      if (a.packed) {  // raw transform of the pair; unpacked and finished by gamma_unpack
        po[g] = v;
        continue;
      }
      const float2 p = ps[g];
      const float k = a.kin[g];
      float2 o;
      o.x = al * (k * p.x + v.x) + be * p.x;
      o.y = al * (k * p.y + v.y) + be * p.y;
      if (pp) {
        const float2 q = pp[g];
        o.x += ga * q.x;
        o.y += ga * q.y;
      }
      po[g] = o;
    }
  }
  __syncthreads();  // the next band reuses the box
}

template <int A, int B>
__global__ void __launch_bounds__(kFusedThreads, 1) fused_local_kernel(FusedArgs args) {
  constexpr int N = A * B;
  extern __shared__ __align__(128) unsigned char fsm[];
  __shared__ FusedArgs a;
  if (threadIdx.x == 0) a = args;
  const FusedSmem m = fused_smem<N>(fsm, args.vbytes);
  fused_init(m);
  if (!fused_stage<N>(fsm, m, a, 0)) return;
  for (int n = blockIdx.x; n < a.units; n += gridDim.x) fused_band<A, B>(m, a, n);
}

// Grouped form for the batch engine: one persistent launch covers the bands of many units of one
// box class (same N = A x B).  The (unit, band) tasks are numbered unit by unit (items[i].blk_ac is
// the first task of item i) and every CTA takes one contiguous range of them, so that it restages
// the potential and tables only when its range crosses into the next unit.
template <int A, int B>
__global__ void __launch_bounds__(kFusedThreads, 1) fused_group_kernel(const bk::LocalItem<float>* __restrict__ items,
                                                                       int n, int tasks, int* err) {
  constexpr int N = A * B;
  constexpr int vbytes = (int)(((size_t)N * N * N * sizeof(float) + 15) & ~(size_t)15);
  extern __shared__ __align__(128) unsigned char fsm[];
  __shared__ FusedArgs a;
  __shared__ int s_item;
  const FusedSmem m = fused_smem<N>(fsm, vbytes);
  fused_init(m);
  const int per = (tasks + (int)gridDim.x - 1) / (int)gridDim.x;
  const int t0 = (int)blockIdx.x * per, t1 = min(tasks, t0 + per);
  int cur = -1;
  uint32_t stages = 0;
  for (int t = t0; t < t1; ++t) {
    if (threadIdx.x == 0) {  // the last item whose first task is <= t
      int lo = 0, hi = n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].blk_ac <= t) lo = mid;
        else hi = mid - 1;
      }
      s_item = lo;
    }
    __syncthreads();
    const int i = s_item;
    if (items[i].idle) {  // unit past its own filter degree
      __syncthreads();
      continue;
    }
    if (i != cur) {
      if (threadIdx.x == 0) {
        const lk::LocalArgs<float>& la = items[i].a;
        a.W2 = la.W2;
        a.W3 = la.W3;
        a.lo2 = la.lo2;
        a.lo3 = la.lo3;
        a.N1p = la.N1p;
        a.units = la.nbands;
        a.nbands = la.nbands;
        a.packed = 0;
        a.vbytes = vbytes;
        a.tw = la.tw1;
        a.vdr = la.Vpi;
        a.zstart = la.zstart;
        a.tileidx = la.tileidx;
        a.kin = la.kin;
        a.psi = la.psi;
        a.psi_prev = la.psi_prev;
        a.out = la.out;
        a.ld = la.ld;
        a.alpha = la.alpha;
        a.beta = la.beta;
        a.gamma = la.gamma;
        a.coef = la.coef;
        a.err = err;
      }
      if (!fused_stage<N>(fsm, m, a, stages & 1u)) return;
      ++stages;
      cur = i;
    }
    fused_band<A, B>(m, a, t - items[i].blk_ac);
  }
}

// V / N^3 at the digit-reversed positions of the fused kernel: position p of a dimension holds
// index p / B + A (p % B); entries past N^3 (padding to 16 bytes) are zero.
__global__ void vdr_gather(const float* __restrict__ vx, float* __restrict__ out, int A, int B, int total) {
  const int N = A * B;
  const int n3 = N * N * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i >= n3) {
      out[i] = 0.f;
      continue;
    }
    const int zp = i / (N * N), rem = i - zp * N * N;
    const int yp = rem / N, xp = rem - yp * N;
    const int x = xp / B + A * (xp % B), y = yp / B + A * (yp % B), z = zp / B + A * (zp % B);
    out[i] = vx[((size_t)x * N + y) * N + z];  // vx: [x][y][z]
  }
}

// (A, B) split of each box length with an instance.
bool fused_split(int N, int* A, int* B) {
  switch (N) {
#define KSS_FUSED(n, x, y) \
  case n:                  \
    *A = x;                \
    *B = y;                \
    return true;
    KSS_FUSED(10, 2, 5) KSS_FUSED(12, 3, 4) KSS_FUSED(15, 3, 5) KSS_FUSED(16, 4, 4)
    KSS_FUSED(18, 3, 6) KSS_FUSED(20, 4, 5) KSS_FUSED(24, 4, 6) KSS_FUSED(25, 5, 5)
#undef KSS_FUSED
    default:
      return false;
  }
}

int vdr_bytes(int N) { return (int)(((size_t)N * N * N * sizeof(float) + 15) & ~(size_t)15); }

template <int A, int B>
void launch_fused(const FusedArgs& fa, int grid, size_t smem, cudaStream_t st) {
  KSS_CHECK_CUDA(cudaFuncSetAttribute(fused_local_kernel<A, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fused_local_kernel<A, B><<<grid, kFusedThreads, smem, st>>>(fa);
}


int* fused_err(kss_ctx ctx) {
  if (!ctx->tc_err.p) {
    ctx->tc_err.alloc(sizeof(int));
    KSS_CHECK_CUDA(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), ctx->stream));
  }
  return ctx->tc_err.as<int>();
}

}  // namespace

const float* fused_potential_view(kss_sys s) {
  int A = 0, B = 0;
  KSS_REQUIRE(fused_split(s->N[0], &A, &B), "fused local part: no instance for this box");
  DevBuf& vd = s->vfused32[A * 32 + B];
  if (!vd.p) {  // built once per system
    const int vbytes = vdr_bytes(s->N[0]);
    vd.alloc((size_t)vbytes);
    const int total = vbytes / (int)sizeof(float);
    vdr_gather<<<(total + 255) / 256, 256, 0, s->ctx->stream>>>(s->d_Vx32.as<float>(), vd.as<float>(), A, B, total);
    KSS_CHECK_CUDA(cudaGetLastError());
  }
  return vd.as<float>();
}

size_t fused_smem_bytes(kss_sys s) { return fused_layout(s->N[0], vdr_bytes(s->N[0])).total; }

int fused_code(kss_sys s) {
  int A = 0, B = 0;
  return fused_local_available(s) && fused_split(s->N[0], &A, &B) ? A * 32 + B : 0;
}

void fused_group_prepare(kss_ctx ctx, int code, size_t smem) {
  fused_err(ctx);
  switch (code) {
#define KSS_FUSED_ATTR(x, y)                                                                        \
  case x * 32 + y:                                                                                  \
    KSS_CHECK_CUDA(cudaFuncSetAttribute(fused_group_kernel<x, y>,                                   \
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));   \
    break;
    KSS_FUSED_ATTR(2, 5) KSS_FUSED_ATTR(3, 4) KSS_FUSED_ATTR(3, 5) KSS_FUSED_ATTR(4, 4)
    KSS_FUSED_ATTR(3, 6) KSS_FUSED_ATTR(4, 5) KSS_FUSED_ATTR(4, 6) KSS_FUSED_ATTR(5, 5)
#undef KSS_FUSED_ATTR
    default:
      fail(KSS_ENOTSUP, "fused local part: no grouped instance for this split");
  }
}

void fused_group_launch(kss_ctx ctx, int code, const bk::LocalItem<float>* d_items, int n, int tasks, size_t smem) {
  KSS_REQUIRE(ctx->tc_err.p, "fused_group_prepare first");
  int* err = ctx->tc_err.as<int>();
  const int grid = std::max(1, std::min(tasks, std::max(1, ctx->nsm)));
  switch (code) {
#define KSS_FUSED_GROUP(x, y)                                                                       \
  case x * 32 + y:                                                                                  \
    fused_group_kernel<x, y><<<grid, kFusedThreads, smem, ctx->stream>>>(d_items, n, tasks, err);   \
    break;
    KSS_FUSED_GROUP(2, 5) KSS_FUSED_GROUP(3, 4) KSS_FUSED_GROUP(3, 5) KSS_FUSED_GROUP(4, 4)
    KSS_FUSED_GROUP(3, 6) KSS_FUSED_GROUP(4, 5) KSS_FUSED_GROUP(4, 6) KSS_FUSED_GROUP(5, 5)
#undef KSS_FUSED_GROUP
    default:
      fail(KSS_ENOTSUP, "fused local part: no grouped instance for this split");
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

bool fused_local_available(kss_sys s) {
  int A = 0, B = 0;
  const int N = s->N[0];
  if (s->N[1] != N || s->N[2] != N || !fused_split(N, &A, &B)) return false;
  return fused_layout(N, vdr_bytes(N)).total <= 227u * 1024u;
}

bool fused_local_apply(kss_sys s, const lk::LocalArgs<float>& a, int units) {
  if (!fused_local_available(s)) return false;
  kss_ctx ctx = s->ctx;
  const int N = s->N[0];
  int A = 0, B = 0;
  fused_split(N, &A, &B);
  const int vbytes = vdr_bytes(N);
  const float* vdr = fused_potential_view(s);
  int* err = fused_err(ctx);
  FusedArgs fa{};
  fa.W2 = a.W2;
  fa.W3 = a.W3;
  fa.lo2 = a.lo2;
  fa.lo3 = a.lo3;
  fa.N1p = a.N1p;
  fa.units = units;
  fa.nbands = a.nbands;
  fa.packed = a.packed;
  fa.vbytes = vbytes;
  fa.tw = a.tw1;
  fa.vdr = vdr;
  fa.zstart = a.zstart;
  fa.tileidx = a.tileidx;
  fa.kin = a.kin;
  fa.psi = a.psi;
  fa.psi_prev = a.psi_prev;
  fa.out = a.out;
  fa.ld = a.ld;
  fa.alpha = a.alpha;
  fa.beta = a.beta;
  fa.gamma = a.gamma;
  fa.coef = a.coef;
  fa.err = err;
  const size_t smem = fused_layout(N, vbytes).total;
  const int grid = std::max(1, std::min(units, std::max(1, ctx->nsm)));
  static const int id = prof_register("local_fused<f32>");
  ProfScope ps(ctx, id);
  switch (A * 32 + B) {
#define KSS_FUSED_CASE(x, y) \
  case x * 32 + y:           \
    launch_fused<x, y>(fa, grid, smem, ctx->stream); \
    break;
    KSS_FUSED_CASE(2, 5) KSS_FUSED_CASE(3, 4) KSS_FUSED_CASE(3, 5) KSS_FUSED_CASE(4, 4)
    KSS_FUSED_CASE(3, 6) KSS_FUSED_CASE(4, 5) KSS_FUSED_CASE(4, 6) KSS_FUSED_CASE(5, 5)
#undef KSS_FUSED_CASE
    default:
      return false;
  }
  KSS_CHECK_CUDA(cudaGetLastError());
  return true;
}

}  // namespace kss

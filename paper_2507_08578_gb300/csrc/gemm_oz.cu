// FP64-accurate complex GEMMs on the BF16 tensor cores (tcgen05 + TMEM + TMA): the FP64 form's
// projector products (Eq. ham-nl with projectors and coefficients in memory, §5.2) and the Gram,
// projected-H and rotation products of Rayleigh-Ritz (§5.1).
//
// GB300 retires about two FP64 fused multiply-adds per SM and clock, against thousands of BF16
// multiply-adds on the tensor cores, so the FP64 products run as sums of exact BF16 products
// (the error-free splitting of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication", 2012):
//
//   * every row of both operands gets an exponent e with |x| < 2^e for all its entries, and every
//     entry is written as 2^e sum_p d_p 2^{-7p}, p = 1..7, with balanced integer digits
//     (|d_1| <= 128, |d_p| <= 64 otherwise) taken exactly from the FP64 bit pattern (49 bits,
//     truncation below); each digit is exact in BF16;
//   * a product x y is 2^{ex+ey} sum_{p,q} d_p d'_q 2^{-7(p+q)}; the pairs with p + q <= 8 are kept
//     (28 of 49; the dropped terms are below 2^{-56} of the row scales), and the pairs with the
//     same p + q form one "group" whose weight is a single power of two;
//   * within a chunk of 384 BF16 along K every group sum is an integer below 2^24 (at most 7
//     pairs of |d d'| <= 2^13 per K entry), so FP32 accumulation in TMEM is exact; after each
//     chunk the seven group sums are read back, combined in double-float (two FP32 words) and
//     added to FP64 accumulators in registers; the row exponents are applied at the end.
//
// Complex -> real as in the split-BF16 kernel: the B rows hold interleaved (re, im) pairs along K
// and each complex row of A becomes two real rows on the A side ((re, im) and (-im, re) for
// A^H B; (re, -im) and (im, re) for A B), the real and imaginary parts of one output row in
// adjacent accumulator rows.
//
// Kernel: one CTA per 128 x 64 tile of real output rows x complex columns (K split across CTAs
// when the tiles do not fill the SMs); warp 0 lane 0 feeds a 2-stage TMA ring (each stage the 7
// digit tiles of A, 128 x 32 BF16, and of B, 64 x 32 BF16, 64-byte swizzle), warp 1 lane 0
// issues tcgen05.mma (M = 128, N = 64, K = 16; 28 per 16-wide slice) into 7 TMEM accumulators of
// 64 columns, warps 2-5 drain the accumulators chunk by chunk.  Every wait is bounded; on time-out
// the kernel raises the error flag shared with the split-BF16 kernel, drains its own copies,
// frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "gemm_tune.h"
#include "tc_common.cuh"

namespace kss {

namespace {

constexpr int TM = 128;                              // real A rows per tile (UMMA M)
constexpr int TN = 64;                               // B rows (complex columns) per tile (UMMA N)
constexpr int TK = 32;                               // BF16 per k-block: one 64-byte swizzle row
constexpr int NG = 7;                                // digit-pair groups g = p + q <= 6 (TMEM: 7 x 64 columns)
constexpr uint32_t ATILE = TM * TK * 2;              // 8 KB
constexpr uint32_t BTILE = TN * TK * 2;              // 4 KB
constexpr int CHUNK = 12;                            // k-blocks per exact chunk (384 BF16 of K)
constexpr int kOzThreads = 192;
constexpr uint32_t kTmemCols = 512;                  // 7 groups x 64 columns, rounded up
constexpr unsigned long long kWaitNs = 2000000000ull;

// Digits per value: 7 for FP64 data (49 bits), 4 for FP32 data (28 bits: every FP32 value of a
// row whose scale is within 2^4 of it is represented exactly).  The ring holds SA + SB digit tiles
// per stage: 2 stages of 84 KB for 7 + 7, 4 stages of 48 KB for 4 + 4.
template <int SA, int SB>
struct OzCfg {
  static constexpr uint32_t STAGE = SA * ATILE + SB * BTILE;
  static constexpr int STAGES = (SA + SB) > 8 ? 2 : 4;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE + 256;
};

using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_try;
using tc::smem_u32;
using tc::tma_load_2d;

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t desc64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)4 << 61;                   // 64-byte swizzle
  return d;
}
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major, M = TM, N = TN.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

// Bounded wait that also gives up as soon as another role of the CTA has failed.
__device__ __forceinline__ bool wait_or_fail(uint32_t bar, uint32_t parity, const volatile int* fail) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = tc::globaltimer();
  while (!mbar_try(bar, parity)) {
    if (*fail) return false;
    if (tc::globaltimer() - t0 > kWaitNs) return false;
  }
  return true;
}

__device__ __forceinline__ double pow2(int e) {  // 2^e for |e| < 1000, exactly
  return __longlong_as_double((long long)(1023 + e) << 52);
}

template <int SA, int SB, typename CT>
__global__ void __launch_bounds__(kOzThreads, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int rowsA,
               int rowsB, int Mr, int Nr, int tnn, int kb_per_split, int kb_total, const int* __restrict__ ea,
               const int* __restrict__ eb, int* __restrict__ err, double* __restrict__ part,
               CT* __restrict__ C, long long ldc, double ar, double ai, double br, double bi) {
  constexpr uint32_t STAGE = OzCfg<SA, SB>::STAGE;
  constexpr int STAGES = OzCfg<SA, SB>::STAGES;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* accf = bars + 2 * STAGES;  // a chunk's accumulators are complete (MMA -> epilogue)
  uint64_t* acce = accf + 1;           // the accumulators have been read (epilogue -> MMA)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 1);
  __shared__ int fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tm = blockIdx.x / tnn, tn = blockIdx.x - tm * tnn;
  const int kb0 = blockIdx.y * kb_per_split;
  const int nkb = max(0, min(kb_total, kb0 + kb_per_split) - kb0);
  const int nchunks = (nkb + CHUNK - 1) / CHUNK;

  if (tid == 0) {
    fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accf), 1);
    mbar_init(smem_u32(acce), 4);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const volatile int* vfail = &fail;

  if (warp == 0 && lane == 0) {
    // TMA producer: every stage carries the 7 digit tiles of A and of B for one k-block.
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !wait_or_fail(smem_u32(&empty[s]), ((kb / STAGES) & 1) ^ 1, vfail)) {
        atomicExch(&fail, 1);
        break;
      }
      if (*vfail) break;
      mbar_expect_tx(smem_u32(&full[s]), STAGE);
      const int x = (kb0 + kb) * TK;
      const uint32_t st = smem_u32(base + s * STAGE), fb = smem_u32(&full[s]);
      for (int p = 0; p < SA; ++p) tma_load_2d(st + p * ATILE, &tmA, x, p * rowsA + tm * TM, fb);
      for (int q = 0; q < SB; ++q) tma_load_2d(st + SA * ATILE + q * BTILE, &tmB, x, q * rowsB + tn * TN, fb);
      ++issued;
    }
    // Drain: every issued copy has landed before the CTA can leave (bounded).
    for (int kb = max(0, issued - STAGES); kb < issued; ++kb)
      if (!tc::mbar_wait(smem_u32(&full[kb % STAGES]), (kb / STAGES) & 1, kWaitNs)) atomicExch(&fail, 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: group g = p + q (0-based digit indices) accumulates in TMEM columns [64 g, 64 g + 64).
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, kc = kb % CHUNK, c = kb / CHUNK;
      if (kc == 0 && c > 0) {
        if (!wait_or_fail(smem_u32(acce), (c - 1) & 1, vfail)) {
          atomicExch(&fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      if (!wait_or_fail(smem_u32(&full[s]), (kb / STAGES) & 1, vfail)) {
        atomicExch(&fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(base + s * STAGE), b0 = a0 + SA * ATILE;
#pragma unroll
      for (int k16 = 0; k16 < TK / 16; ++k16) {
#pragma unroll
        for (int p = 0; p < SA; ++p) {
          const uint64_t da = desc64(a0 + p * ATILE + 32 * k16);
#pragma unroll
          for (int q = 0; q < SB && p + q < NG; ++q) {
            const uint64_t db = desc64(b0 + q * BTILE + 32 * k16);
            // the first product of every group in a chunk overwrites: in issue order that is the
            // pair with the smallest p, p = max(0, g - (SB - 1))
            const int g = p + q;
            const int pfirst = g > SB - 1 ? g - (SB - 1) : 0;
            const uint32_t acc = (kc == 0 && k16 == 0 && p == pfirst) ? 0u : 1u;
            const uint32_t dcol = tmem + (uint32_t)((p + q) * TN);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&empty[s]))
                   : "memory");
      if (kc == CHUNK - 1 || kb == nkb - 1)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(accf))
                     : "memory");
    }
  } else if (warp >= 2) {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (accumulator rows).
    const int quarter = warp & 3;
    const int row = tm * TM + quarter * 32 + lane;
    double acc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[j] = 0.0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      ok = wait_or_fail(smem_u32(accf), c & 1, vfail);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicExch(&fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < TN; c0 += 16) {
        float hi[16], lo[16];
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          uint32_t r[16];
          const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * TN + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          // group g weighs 2^{-7 g} relative to group 0 (exact in FP32); double-float sum
          const float sc = __int_as_float((127 - 7 * g) << 23);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float v = __uint_as_float(r[j]) * sc;
            if (g == 0) {
              hi[j] = v;
              lo[j] = 0.f;
            } else {
              const float s = hi[j] + v;
              const float bb = s - hi[j];
              const float e = (hi[j] - (s - bb)) + (v - bb);
              hi[j] = s;
              lo[j] += e;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[c0 + j] += (double)hi[j] + (double)lo[j];
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(acce));
    }
    if (ok && nkb > 0) {
      // value = acc * 2^{ea + eb - 14} (the 2^-14 of group 0)
      const int er = row < Mr ? ea[row] - 14 : 0;
      const int col0 = tn * TN;
      if (part) {
        double* P = part + (size_t)blockIdx.y * Nr * Mr;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int col = col0 + j;
          if (row < Mr && col < Nr) P[(size_t)col * Mr + row] = acc[j] * pow2(er + eb[col]);
        }
      } else {
        // fused complex result: accumulator row 2i is Re C(i, col), row 2i + 1 is Im C(i, col)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int col = col0 + j;
          const double v = (row < Mr && col < Nr) ? acc[j] * pow2(er + eb[col]) : 0.0;
          const double w = __shfl_down_sync(0xffffffffu, v, 1);
          if (!(lane & 1) && row < Mr && col < Nr) {
            CT* dst = C + (size_t)col * ldc + (row >> 1);
            double ox = ar * v - ai * w, oy = ar * w + ai * v;
            if (br != 0.0 || bi != 0.0) {
              const CT q = *dst;
              ox += br * (double)q.x - bi * (double)q.y;
              oy += br * (double)q.y + bi * (double)q.x;
            }
            CT o;
            o.x = ox;
            o.y = oy;
            *dst = o;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  if (tid == 0 && fail) atomicExch(err, 1);
}

// ---- operand preparation (digit planes) --------------------------------------------------------
// IEEE layout of the source precision.
template <typename R> struct Bits;
template <> struct Bits<double> {
  using U = unsigned long long;
  static constexpr int kFrac = 52, kBias = 1023, kExpMask = 0x7FF;
  static constexpr U kAbs = 0x7FFFFFFFFFFFFFFFull;
  __device__ static U of(double v) { return (U)__double_as_longlong(v); }
};
template <> struct Bits<float> {
  using U = unsigned int;
  static constexpr int kFrac = 23, kBias = 127, kExpMask = 0xFF;
  static constexpr U kAbs = 0x7FFFFFFFu;
  __device__ static U of(float v) { return (U)__float_as_uint(v); }
};

// Exponent e with every |x| of the row below 2^e, from the largest magnitude's bit pattern
// (for non-negative IEEE values the integer order of the bit patterns is the numeric order).
template <typename R>
__device__ __forceinline__ int row_exponent(unsigned long long maxbits) {
  const int ev = (int)(maxbits >> Bits<R>::kFrac);
  return ev ? ev - Bits<R>::kBias + 1 : 0;
}

// The S balanced base-128 digits of v 2^{7S - e} (|v| < 2^e), most significant first, taken from
// the bit pattern with integer operations only (bits below 2^{e - 7S} truncated).
template <int S, typename R>
__device__ __forceinline__ void digits(R v, int e, float d[S]) {
  const auto bits = Bits<R>::of(v);
  const int ev = (int)((bits >> Bits<R>::kFrac) & Bits<R>::kExpMask);
  long long N = 0;
  if (ev != 0) {
    const unsigned long long mant =
        (unsigned long long)(bits & ((((decltype(bits))1) << Bits<R>::kFrac) - 1)) | (1ull << Bits<R>::kFrac);
    // v 2^{7S-e} = mant 2^{ev - bias - frac + 7S - e}; the shift is at most 7S - frac - 1 + ... so
    // that the result stays below 2^{7S}
    const int sh = ev - Bits<R>::kBias - Bits<R>::kFrac + 7 * S - e;
    N = sh >= 0 ? (long long)(mant << sh) : (sh <= -64 ? 0 : (long long)(mant >> -sh));
  }
  int u[S];
#pragma unroll
  for (int p = 0; p < S; ++p) u[p] = (int)((N >> (7 * (S - 1 - p))) & 127);
#pragma unroll
  for (int p = S - 1; p > 0; --p)
    if (u[p] >= 64) {
      u[p] -= 128;
      u[p - 1] += 1;
    }
  const bool neg = (bits >> (8 * sizeof(bits) - 1)) != 0;
#pragma unroll
  for (int p = 0; p < S; ++p) d[p] = (float)(neg ? -u[p] : u[p]);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

template <typename CS> struct Real;
template <> struct Real<double2> { using T = double; };
template <> struct Real<float2> { using T = float; };

// K-major complex source (column c: K values at src + c ld) -> digit planes [S][rows][KT] of
// interleaved (re, im) pairs, one warp per column.  pair = 1 (the A operand of A^H B): row 2c holds
// (re, im) and row 2c + 1 (-im, re), both with the column's exponent.
template <int S, typename CS>
__global__ void oz_prep_k(const CS* __restrict__ src, long long ld, int K, int ncols, int KT,
                          __nv_bfloat16* __restrict__ dst, int rows, int* __restrict__ erow, int pair) {
  using R = typename Real<CS>::T;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= ncols) return;
  const CS* x = src + (size_t)c * ld;
  unsigned long long mx = 0;
  for (int k = lane; k < K; k += 32) {
    const CS v = x[k];
    const unsigned long long a = Bits<R>::of(v.x) & Bits<R>::kAbs;
    const unsigned long long b = Bits<R>::of(v.y) & Bits<R>::kAbs;
    mx = a > mx ? a : mx;
    mx = b > mx ? b : mx;
  }
  const int e = row_exponent<R>(warp_max_u64(mx));
  const int r0 = pair ? 2 * c : c;
  if (lane == 0) {
    erow[r0] = e;
    if (pair) erow[r0 + 1] = e;
  }
  const size_t plane = (size_t)rows * KT;
  for (int k = lane; k < KT / 2; k += 32) {
    R re = 0, im = 0;
    if (k < K) {
      const CS v = x[k];
      re = v.x;
      im = v.y;
    }
    float dr[S], di[S];
    digits<S>(re, e, dr);
    digits<S>(im, e, di);
#pragma unroll
    for (int p = 0; p < S; ++p) {
      __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(dst + p * plane + (size_t)r0 * KT);
      o[k] = __floats2bfloat162_rn(dr[p], di[p]);
      if (pair) {
        __nv_bfloat162* o1 = reinterpret_cast<__nv_bfloat162*>(dst + p * plane + (size_t)(r0 + 1) * KT);
        o1[k] = __floats2bfloat162_rn(-di[p], dr[p]);
      }
    }
  }
}

// Exponents of the rows of an M-major complex A (element (i, k) at src[k ld + i]), one thread per i.
template <typename CS>
__global__ void oz_exp_m(const CS* __restrict__ src, long long ld, int M, int K, int* __restrict__ erow) {
  using R = typename Real<CS>::T;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  unsigned long long mx = 0;
  for (int k = 0; k < K; ++k) {
    const CS v = src[(size_t)k * ld + i];
    const unsigned long long a = Bits<R>::of(v.x) & Bits<R>::kAbs;
    const unsigned long long b = Bits<R>::of(v.y) & Bits<R>::kAbs;
    mx = a > mx ? a : mx;
    mx = b > mx ? b : mx;
  }
  const int e = row_exponent<R>(mx);
  erow[2 * i] = e;
  erow[2 * i + 1] = e;
}

// M-major complex A -> digit planes of the A operand of C = A B: row 2i holds (re, -im) pairs,
// row 2i + 1 (im, re); a 32 x 32 transpose through shared memory.
template <int S, typename CS>
__global__ void oz_prep_m(const CS* __restrict__ src, long long ld, int M, int K, int KT,
                          __nv_bfloat16* __restrict__ dst, int rows, const int* __restrict__ erow) {
  __shared__ CS t[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, i = i0 + threadIdx.x;
    CS z;
    z.x = 0;
    z.y = 0;
    t[r][threadIdx.x] = (k < K && i < M) ? src[(size_t)k * ld + i] : z;
  }
  __syncthreads();
  const size_t plane = (size_t)rows * KT;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, k = k0 + threadIdx.x;
    if (i >= M || k >= KT / 2) continue;
    const CS v = t[threadIdx.x][r];
    const int e = erow[2 * i];
    float dr[S], di[S];
    digits<S>(v.x, e, dr);
    digits<S>(v.y, e, di);
#pragma unroll
    for (int p = 0; p < S; ++p) {
      __nv_bfloat162* ra = reinterpret_cast<__nv_bfloat162*>(dst + p * plane + (size_t)(2 * i) * KT);
      __nv_bfloat162* rb = reinterpret_cast<__nv_bfloat162*>(dst + p * plane + (size_t)(2 * i + 1) * KT);
      ra[k] = __floats2bfloat162_rn(dr[p], -di[p]);
      rb[k] = __floats2bfloat162_rn(di[p], dr[p]);
    }
  }
}

// C (complex, col-major ldc) = alpha * D + beta * C from the FP64 K-split partials (col-major
// Mr x Nr each, Mr = 2M): re = D(2i, j), im = D(2i + 1, j), splits added in a fixed order.
template <typename CT>
__global__ void oz_combine(const double* __restrict__ P, int nsplit, int Mr, int Nr, int M, int N,
                           CT* __restrict__ C, long long ldc, double ar, double ai, double br, double bi) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  const size_t o = (size_t)j * Mr + 2 * i;
  const size_t stride = (size_t)Mr * Nr;
  double sr = 0.0, si = 0.0;
  for (int z = 0; z < nsplit; ++z) {
    sr += P[z * stride + o];
    si += P[z * stride + o + 1];
  }
  double ox = ar * sr - ai * si, oy = ar * si + ai * sr;
  CT* dst = C + (size_t)j * ldc + i;
  if (br != 0.0 || bi != 0.0) {
    const CT q = *dst;
    ox += br * (double)q.x - bi * (double)q.y;
    oy += br * (double)q.y + bi * (double)q.x;
  }
  CT r;
  r.x = ox;
  r.y = oy;
  *dst = r;
}

CUtensorMap make_map(const void* base, long long rows, int kt, int box_rows) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[2] = {(cuuint64_t)kt, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kt * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = tc::encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(KSS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

int ktile(int K) { return ((2 * K + TK - 1) / TK) * TK; }

int* err_flag(kss_ctx ctx) {
  if (!ctx->tc_err.p) {
    ctx->tc_err.alloc(sizeof(int));
    KSS_CHECK_CUDA(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), ctx->stream));
  }
  return ctx->tc_err.as<int>();
}

// C (M x N complex) = alpha * A_op (2M real rows) * B_op (N rows)^T + beta * C.
template <int SA, int SB, typename CT>
void launch_oz(kss_ctx ctx, const OzOperand& a, const OzOperand& b, int M, int N, CT* C, int ldc, double ar,
               double ai, double br, double bi, const char* tag) {
  using Cfg = OzCfg<SA, SB>;
  const int Mr = 2 * M, Nr = N;
  const int tmn = (Mr + TM - 1) / TM, tnn = (Nr + TN - 1) / TN;
  const int kb_total = a.KT / TK;
  const long long tiles = (long long)tmn * tnn;
  if (tiles > 0x7fffffffLL) fail(KSS_EINVAL, "digit-product GEMM: too many output tiles");
  // K-split plan: one CTA per SM (the ring takes 169 / 193 KB of shared memory); with fewer tiles
  // than SMs, split K so that the grid fills the SMs in one wave, keeping at least two exact
  // chunks per CTA.
  int nsm = ctx->nsm;
  if (!nsm) {
    KSS_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    ctx->nsm = nsm = std::max(nsm, 1);
  }
  // closed-form plan; the autotuner times it against other splits at first use of the shape
  int plan = 1;
  if (tiles < nsm) plan = (int)std::max(1LL, std::min<long long>(nsm / tiles, kb_total / (2 * CHUNK)));
  const CUtensorMap ma = make_map(a.planes, (long long)SA * a.rows, a.KT, TM);
  const CUtensorMap mb = make_map(b.planes, (long long)SB * b.rows, b.KT, TN);
  auto kern = oz_gemm_kernel<SA, SB, CT>;
  KSS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
  const std::string name = std::string(SA == 7 ? "tc_gemm_oz7:" : "tc_gemm_oz4:") + tag;
  const std::string cname = std::string("oz_combine:") + tag;
  // One product with `splits` K-splits into C (ldc, alpha, beta).
  auto launch = [&](int splits, CT* Cd, int ldd, double br_, double bi_, bool prof) {
    int kps = (kb_total + splits - 1) / splits;
    kps = ((kps + CHUNK - 1) / CHUNK) * CHUNK;
    splits = (kb_total + kps - 1) / kps;
    if (splits > 1) ctx->oz_part.ensure((size_t)splits * Mr * Nr * sizeof(double));
    const bool fused = splits == 1;
    {
      ProfScope ps(ctx, prof ? prof_register(name.c_str()) : prof_register("gemm_tuning"));
      kern<<<dim3((unsigned)tiles, splits, 1), kOzThreads, Cfg::SMEM, ctx->stream>>>(
          ma, mb, a.rows, b.rows, Mr, Nr, tnn, kps, kb_total, a.e, b.e, err_flag(ctx),
          fused ? nullptr : ctx->oz_part.as<double>(), Cd, ldd, ar, ai, br_, bi_);
    }
    KSS_CHECK_CUDA(cudaGetLastError());
    if (fused) return;
    const long long mn = (long long)M * N;
    ProfScope ps(ctx, prof ? prof_register(cname.c_str()) : prof_register("gemm_tuning"));
    oz_combine<CT><<<(unsigned)((mn + 255) / 256), 256, 0, ctx->stream>>>(ctx->oz_part.as<double>(), splits, Mr,
                                                                          Nr, M, N, Cd, ldd, ar, ai, br_, bi_);
    KSS_CHECK_CUDA(cudaGetLastError());
  };
  const int kind = SA == 4 ? GT_OZ44 : (sizeof(CT) == sizeof(double2) ? GT_OZ77 : GT_OZ77_C64OUT);
  const int splits = tuned_split(ctx, kind, Mr, Nr, kb_total, tiles, 2 * CHUNK, plan, [&](int sp) {
    ctx->tune_c.ensure((size_t)M * N * sizeof(CT));
    launch(sp, ctx->tune_c.as<CT>(), M, 0.0, 0.0, false);
  });
  launch(splits, C, ldc, br, bi, true);
}

void run_oz(kss_ctx ctx, const OzOperand& a, const OzOperand& b, int M, int N, void* C, bool c128out, int ldc,
            double ar, double ai, double br, double bi, const char* tag) {
  KSS_REQUIRE(a.KT == b.KT && a.rows == 2 * M && b.rows == N, "digit-product GEMM: operand shapes differ");
  if (a.S == 7 && b.S == 7 && c128out)
    launch_oz<7, 7>(ctx, a, b, M, N, (double2*)C, ldc, ar, ai, br, bi, tag);
  else if (a.S == 7 && b.S == 7)
    launch_oz<7, 7>(ctx, a, b, M, N, (float2*)C, ldc, ar, ai, br, bi, tag);
  else if (a.S == 4 && b.S == 4 && c128out)
    launch_oz<4, 4>(ctx, a, b, M, N, (double2*)C, ldc, ar, ai, br, bi, tag);
  else
    fail(KSS_EINVAL, "digit-product GEMM: unsupported digit counts");
}

}  // namespace

size_t oz_operand_bytes(int rows, int K, int S) {
  return (size_t)S * rows * ktile(K) * 2 + (size_t)rows * sizeof(int) + 256;
}

OzOperand oz_operand_at(void* mem, int rows, int K, int S) {
  OzOperand o;
  o.rows = rows;
  o.KT = ktile(K);
  o.S = S;
  o.planes = static_cast<__nv_bfloat16*>(mem);
  const size_t pb = ((size_t)S * rows * o.KT * 2 + 255) & ~(size_t)255;
  o.e = reinterpret_cast<int*>(static_cast<unsigned char*>(mem) + pb);
  return o;
}

// Digit planes of an operand: cn_a (A of A^H B, K-major, 2 rows per column), kmajor (B, K-major, one
// row per column), mmajor (A of A B, M-major, 2 rows per row); S = 7 or 4 digits per value from
// complex128 (f64src) or complex64 data.
template <int S, typename CS>
void prepare_as(kss_ctx ctx, OzKind kind, int n, int K, const CS* src, long long ld, const OzOperand& o) {
  if (kind == OZ_MMAJOR_A) {
    dim3 g((n + 31) / 32, (o.KT / 2 + 31) / 32);
    oz_exp_m<CS><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(src, ld, n, K, o.e);
    oz_prep_m<S, CS><<<g, dim3(32, 8), 0, ctx->stream>>>(src, ld, n, K, o.KT, o.planes, o.rows, o.e);
  } else {
    oz_prep_k<S, CS><<<(unsigned)((n + 7) / 8), 256, 0, ctx->stream>>>(src, ld, K, n, o.KT, o.planes, o.rows, o.e,
                                                                      kind == OZ_CN_A ? 1 : 0);
  }
}

OzOperand oz_prepare(kss_ctx ctx, OzKind kind, int n, int K, const void* src, long long ld, void* mem, bool f64src,
                     int S) {
  if (S <= 0) S = f64src ? 7 : 4;
  KSS_REQUIRE(S == 7 || (S == 4 && !f64src), "digit-product GEMM: 7 digits (complex128 or complex64 data) or 4 "
                                             "(complex64 data)");
  const int rows = kind == OZ_B ? n : 2 * n;
  OzOperand o = oz_operand_at(mem, rows, K, S);
  ProfScope ps(ctx, prof_register("oz_prep"));
  if (f64src) prepare_as<7, double2>(ctx, kind, n, K, (const double2*)src, ld, o);
  else if (S == 7) prepare_as<7, float2>(ctx, kind, n, K, (const float2*)src, ld, o);
  else prepare_as<4, float2>(ctx, kind, n, K, (const float2*)src, ld, o);
  KSS_CHECK_CUDA(cudaGetLastError());
  return o;
}

// C (M x N) = alpha A^H B + beta C; A: K x M (lda), B: K x N (ldb).  f64in: complex128 operands,
// else complex64; f64out: complex128 C, else complex64; digits: per value (0: 7 for complex128, 4
// for complex64 data).
void oz_gemm_cn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C, int ldc,
                double ar, double ai, double br, double bi, const char* tag, const OzOperand* a_pre, bool f64in,
                bool f64out, int digits) {
  if (M <= 0 || N <= 0) return;
  KSS_REQUIRE(K > 0, "digit-product GEMM: K = 0");
  const int S = digits > 0 ? digits : (f64in ? 7 : 4);
  OzOperand a;
  if (a_pre) {
    a = *a_pre;
  } else {
    ctx->oz_a.ensure(oz_operand_bytes(2 * M, K, S));
    a = oz_prepare(ctx, OZ_CN_A, M, K, A, lda, ctx->oz_a.p, f64in, S);
  }
  ctx->oz_b.ensure(oz_operand_bytes(N, K, S));
  const OzOperand b = oz_prepare(ctx, OZ_B, N, K, B, ldb, ctx->oz_b.p, f64in, S);
  run_oz(ctx, a, b, M, N, C, f64out, ldc, ar, ai, br, bi, tag);
}

// C (M x N) = alpha A B + beta C; A: M x K (lda, M contiguous), B: K x N (ldb).
void oz_gemm_nn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C, int ldc,
                double ar, double ai, double br, double bi, const char* tag, const OzOperand* a_pre, bool f64in,
                bool f64out, int digits) {
  if (M <= 0 || N <= 0) return;
  KSS_REQUIRE(K > 0, "digit-product GEMM: K = 0");
  const int S = digits > 0 ? digits : (f64in ? 7 : 4);
  OzOperand a;
  if (a_pre) {
    a = *a_pre;
  } else {
    ctx->oz_a.ensure(oz_operand_bytes(2 * M, K, S));
    a = oz_prepare(ctx, OZ_MMAJOR_A, M, K, A, lda, ctx->oz_a.p, f64in, S);
  }
  ctx->oz_b.ensure(oz_operand_bytes(N, K, S));
  const OzOperand b = oz_prepare(ctx, OZ_B, N, K, B, ldb, ctx->oz_b.p, f64in, S);
  run_oz(ctx, a, b, M, N, C, f64out, ldc, ar, ai, br, bi, tag);
}

}  // namespace kss

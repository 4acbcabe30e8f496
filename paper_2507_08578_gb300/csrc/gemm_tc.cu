// Split-precision complex GEMMs on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// Mixed-precision form of the projector products C = beta^H psi and H psi += beta C' (Eq. ham-nl
// with the projectors and their coefficients in memory, §5.2) and of the subspace Gram / projected
// H / rotation products of Rayleigh-Ritz (§5.1).
//
// Each complex product is written as one real GEMM D = A_tc * B_tc^T with both operands K-major
// in BF16:
//   * complex -> real: the B rows hold interleaved (re, im) pairs along K; every complex row i of
//     A becomes two real rows, 2i giving the real and 2i + 1 the imaginary part of output row i
//     ((re, im) and (-im, re) for A^H B; (re, -im) and (im, re) for A B), so the extra rows sit on
//     the A side, which for the projector products is the static table prepared once;
//   * split precision: every FP32 value x = hi + lo with hi = bf16(x), lo = bf16(x - hi); each
//     operand row holds its hi copy followed by its lo copy, and for every k-block the kernel
//     accumulates hi*hi + hi*lo + lo*hi in FP32 (TMEM) from the same four staged tiles.
// Two kernel forms, chosen per shape by the autotuner (gemm_tune.cu): the persistent form (one CTA
// per SM walking output tiles with two TMEM accumulators, described below at tc_persist_kernel,
// also the grouped products of the batch engine), and the one-CTA-per-tile form:
// one CTA per 128 x 128 output tile (tiles with the same A rows adjacent in
// launch order, so A is fetched from HBM once and re-read from L2) and K split across CTAs so
// that the grid fills the SMs in as few waves as possible; a TMA producer thread fills a 3-stage
// ring, each stage holding the hi and lo 128B-swizzled 128 x 64 BF16 tiles of both operands; one
// thread issues tcgen05.mma (M=128, N=128, K=16; three per 16-wide slice) into a TMEM
// accumulator, and four warps read TMEM back with tcgen05.ld and store FP32 partial sums.  A
// reduction kernel adds the K-splits in a fixed order and forms the complex result.  Every
// mbarrier wait is bounded; on time-out the kernel raises an error flag, drains its own copies,
// frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "gemm_tune.h"
#include "tc_common.cuh"

namespace kss {

namespace {

constexpr int TM = 128;   // UMMA M (rows of A_tc per tile)
constexpr int TN = 128;   // UMMA N (rows of B_tc per tile)
constexpr int TK = 64;    // BF16 per k-block: one 128-byte swizzle row
constexpr int STAGES = 3;
constexpr int kTcThreads = 128;
constexpr uint32_t kTileBytes = TM * TK * 2;  // 16 KB (A and B tiles are the same size)
constexpr uint32_t kStageBytes = 4 * kTileBytes;  // A hi, A lo, B hi, B lo
constexpr size_t kTcSmem = 1024 + (size_t)STAGES * kStageBytes + 256;
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded waits: 2 s

using tc::globaltimer;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_try;
using tc::smem_u32;
using tc::tma_load_2d;
// Wait for the phase of the given parity to complete, at most kWaitNs; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) { return tc::mbar_wait(bar, parity, kWaitNs); }
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major, M = TM, N = TN.
__host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__global__ void __launch_bounds__(kTcThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               float* __restrict__ D, int Mr, int Nr, int tnn, int kb_per_split, int kb_total, int kp,
               int* __restrict__ err, float2* __restrict__ Cf, long long ldc, float ar, float ai, float br,
               float bi) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  // stage s: A hi, A lo, B hi, B lo tiles at base + s * kStageBytes
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * kStageBytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* done = bars + 2 * STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  __shared__ int fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tm = blockIdx.x / tnn, tn = blockIdx.x - tm * tnn;
  const int kb0 = blockIdx.y * kb_per_split;
  const int nkb = max(0, min(kb_total, kb0 + kb_per_split) - kb0);

  if (tid == 0) {
    fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(smem_u32(&empty[s]), ((kb / STAGES) & 1) ^ 1)) {
        atomicExch(&fail, 1);
        break;
      }
      if (*(volatile int*)&fail) break;
      mbar_expect_tx(smem_u32(&full[s]), kStageBytes);
      const int x = (kb0 + kb) * TK;  // hi copy at x, lo copy at x + kp (both multiples of 64)
      const uint32_t st = smem_u32(base + s * kStageBytes), fb = smem_u32(&full[s]);
      tma_load_2d(st, &tmA, x, tm * TM, fb);
      tma_load_2d(st + kTileBytes, &tmA, x + kp, tm * TM, fb);
      tma_load_2d(st + 2 * kTileBytes, &tmB, x, tn * TN, fb);
      tma_load_2d(st + 3 * kTileBytes, &tmB, x + kp, tn * TN, fb);
      ++issued;
    }
    // Drain: every issued copy has landed before the CTA can leave (bounded).
    for (int kb = max(0, issued - STAGES); kb < issued; ++kb)
      if (!mbar_wait(smem_u32(&full[kb % STAGES]), (kb / STAGES) & 1)) atomicExch(&fail, 1);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = instr_desc();
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(smem_u32(&full[s]), (kb / STAGES) & 1)) {
        atomicExch(&fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(base + s * kStageBytes), al = ah + kTileBytes;
      const uint32_t bh = ah + 2 * kTileBytes, bl = ah + 3 * kTileBytes;
#pragma unroll
      for (int k = 0; k < TK / 16; ++k) {
        // hi*hi, hi*lo, lo*hi for this 16-wide slice (32 bytes into each swizzled row)
        const uint64_t dah = smem_desc(ah + 32 * k), dal = smem_desc(al + 32 * k);
        const uint64_t dbh = smem_desc(bh + 32 * k), dbl = smem_desc(bl + 32 * k);
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p, q;\n setp.ne.b32 p, %6, 0;\n setp.eq.b32 q, %6, %6;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %5, p;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %5, q;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %2, %5, q;\n}\n" ::"r"(tmem),
            "l"(dah), "l"(dbh), "l"(dbl), "l"(dal), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(done)) : "memory");
  }
  __syncwarp();
  // Epilogue: warp w owns TMEM lanes 32w..32w+31 (accumulator rows).
  bool ok = mbar_wait(smem_u32(done), 0);
  ok = __all_sync(0xffffffffu, ok);
  if (!ok) atomicExch(&fail, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = tm * TM + warp * 32 + lane;
  float* Dz = D + (size_t)blockIdx.y * Mr * Nr;
  if (ok && nkb > 0) {
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (Cf) {
        // Fused complex epilogue (no K-split; interleaved A rows): accumulator row 2i
        // holds Re C(i, col), row 2i+1 Im C(i, col); the pair sits in adjacent lanes of this warp.
        float w[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) w[j] = __shfl_down_sync(0xffffffffu, __uint_as_float(r[j]), 1);
        if (row < Mr && !(lane & 1)) {
          const int ncol = min(32, Nr - (tn * TN + c0));
          float2* dst0 = Cf + (size_t)(tn * TN + c0) * ldc + (row >> 1);
          float2 q[32];
          // all loads of the old values first (independent), then the stores
#pragma unroll
          for (int j = 0; j < 32; ++j)
            q[j] = (j < ncol && (br != 0.f || bi != 0.f)) ? dst0[(size_t)j * ldc] : make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < ncol) {
              const float v = __uint_as_float(r[j]);
              float2 o;
              o.x = ar * v - ai * w[j] + br * q[j].x - bi * q[j].y;
              o.y = ar * w[j] + ai * v + br * q[j].y + bi * q[j].x;
              dst0[(size_t)j * ldc] = o;
            }
          }
        }
      } else if (row < Mr) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = tn * TN + c0 + j;
          if (col < Nr) Dz[(size_t)col * Mr + row] = __uint_as_float(r[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
  if (tid == 0 && fail) atomicExch(err, 1);
}

// ---- persistent form --------------------------------------------------------------------------
// One CTA per SM walks a list of works (output tile x K range) of one or more products: the works
// of the whole launch are numbered product by product (tiles sharing A rows adjacent) and CTA c
// takes works c, c + G, c + 2G, ...  Roles: warp 0 (one thread) fills the stage ring with TMA
// across work boundaries, warp 1 (one thread) issues the MMAs into one of two TMEM accumulators
// (alternating per work), and eight epilogue warps drain the other accumulator meanwhile: warp w
// reads TMEM lanes 32 (w mod 4) .. + 31 and one half of the tile's columns.  Accumulator handoff:
// acc_full[a] (committed by the MMA thread after a work's last MMA) and acc_empty[a] (one arrival
// per epilogue warp after its last TMEM read).  Every wait is bounded; on time-out the kernel
// raises the error flag, every role leaves its loop, the MMA thread waits (bounded) for its
// MMAs in flight and the producer for its copies in flight, and TMEM is freed.
constexpr int kPEpiWarps = 8;
constexpr int kMaxKbSplit = 128;  // k-blocks one split accumulates in FP32 (8192 BF16 of K)
constexpr int kPThreads = 64 + 32 * kPEpiWarps;

struct TcProd {          // one product of a persistent launch (split-BF16 operands, see above)
  int Mr, Nr, tmn, tnn;  // accumulator rows and columns; row and column tiles
  int kb_total, kbs;     // k-blocks of K; k-blocks per split
  int kp;                // BF16 offset of the lo copy within an operand row
  int w0;                // first work of this product in the launch
  int idle;              // the product's works do nothing (a unit past its own filter degree)
  float2* C;             // complex result when the product is not split
  long long ldc;
  float ar, ai, br, bi;  // C = (alpha * rs[i]) * A_tc B_tc^T + beta * C
  const float* rs;       // real scale of complex output row i, or null (1)
  float* P;              // partial sums [split][Nr][Mr] when the product is split
  long long cb0;         // first block of the product in the grouped combine launch
};

struct TcPersistArgs {
  CUtensorMap ma, mb;        // operands of the single product (prods == null)
  TcProd one;                // the single product
  const TcProd* prods;       // grouped launch: product table in device memory
  const CUtensorMap* maps;   // grouped launch: maps[2 i] (A) and maps[2 i + 1] (B) of product i
  int nprod, nwork;
  int* err;
};

struct TcWorkPos {
  const TcProd* p;
  const CUtensorMap *ma, *mb;
  int tm, tn, z, kb0, nkb;
};

__device__ __forceinline__ TcWorkPos tc_decode(const TcPersistArgs& a, int x) {
  TcWorkPos w;
  if (a.prods) {
    int lo = 0, hi = a.nprod;  // the last product with w0 <= x
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.prods[mid].w0 <= x) lo = mid;
      else hi = mid;
    }
    w.p = a.prods + lo;
    w.ma = a.maps + 2 * lo;
    w.mb = w.ma + 1;
  } else {
    w.p = &a.one;
    w.ma = &a.ma;
    w.mb = &a.mb;
  }
  const TcProd& p = *w.p;
  const int l = x - p.w0;
  w.tn = l % p.tnn;
  const int r = l / p.tnn;
  w.tm = r % p.tmn;
  w.z = r / p.tmn;
  w.kb0 = w.z * p.kbs;
  w.nkb = max(0, min(p.kb_total, w.kb0 + p.kbs) - w.kb0);
  return w;
}

template <int TNP>
__host__ __device__ constexpr uint32_t instr_desc_n() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TNP >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}
template <int TNP> __host__ __device__ constexpr int p_stages() { return TNP == 128 ? 3 : 4; }
template <int TNP> __host__ __device__ constexpr uint32_t p_stage_bytes() { return 2u * TM * TK * 2 + 2u * TNP * TK * 2; }
template <int TNP> constexpr size_t p_smem() { return 1024 + (size_t)p_stages<TNP>() * p_stage_bytes<TNP>() + 256; }

template <int TNP>
__global__ void __launch_bounds__(kPThreads, 1) tc_persist_kernel(const __grid_constant__ TcPersistArgs a) {
  constexpr int S = p_stages<TNP>();
  constexpr uint32_t kA = TM * TK * 2, kB = TNP * TK * 2, kSt = p_stage_bytes<TNP>();
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + S * kSt);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = bars + 2 * S + 2;
  uint64_t* done = bars + 2 * S + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 5);
  __shared__ int fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    fail = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), kPEpiWarps);
    }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TNP));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      long long g = 0;  // k-blocks issued by this CTA
      for (int x = blockIdx.x; x < a.nwork; x += gridDim.x) {
        if (*(volatile int*)&fail) break;
        const TcWorkPos w = tc_decode(a, x);
        if (w.p->idle) continue;
        const int kp = w.p->kp;
        bool ok = true;
        for (int kb = 0; kb < w.nkb; ++kb, ++g) {
          const int s = (int)(g % S);
          if (g >= S && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((g / S) & 1) ^ 1u)) {
            ok = false;
            break;
          }
          mbar_expect_tx(smem_u32(&full[s]), kSt);
          const int xk = (w.kb0 + kb) * TK;
          const uint32_t st = smem_u32(base + s * kSt), fb = smem_u32(&full[s]);
          tma_load_2d(st, w.ma, xk, w.tm * TM, fb);
          tma_load_2d(st + kA, w.ma, xk + kp, w.tm * TM, fb);
          tma_load_2d(st + 2 * kA, w.mb, xk, w.tn * TNP, fb);
          tma_load_2d(st + 2 * kA + kB, w.mb, xk + kp, w.tn * TNP, fb);
        }
        if (!ok) {
          atomicExch(&fail, 1);
          break;
        }
      }
      // Drain: the copies of the last S issued k-blocks have landed before the CTA can leave.
      for (long long q = g > S ? g - S : 0; q < g; ++q)
        if (!mbar_wait(smem_u32(&full[q % S]), (uint32_t)((q / S) & 1))) atomicExch(&fail, 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = instr_desc_n<TNP>();
      long long g = 0;
      int u = 0;  // works accumulated by this CTA
      for (int x = blockIdx.x; x < a.nwork; x += gridDim.x) {
        if (*(volatile int*)&fail) break;
        const TcWorkPos w = tc_decode(a, x);
        if (w.p->idle) continue;
        const int acc = u & 1, use = u >> 1;
        if (use > 0 && !mbar_wait(smem_u32(&acce[acc]), (uint32_t)((use - 1) & 1))) {
          atomicExch(&fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dt = tmem + (uint32_t)(acc * TNP);
        bool ok = true;
        for (int kb = 0; kb < w.nkb; ++kb, ++g) {
          const int s = (int)(g % S);
          if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((g / S) & 1))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = smem_u32(base + s * kSt), al = ah + kA;
          const uint32_t bh = ah + 2 * kA, bl = bh + kB;
#pragma unroll
          for (int k = 0; k < TK / 16; ++k) {
            const uint64_t dah = smem_desc(ah + 32 * k), dal = smem_desc(al + 32 * k);
            const uint64_t dbh = smem_desc(bh + 32 * k), dbl = smem_desc(bl + 32 * k);
            const uint32_t accf_ = (kb > 0 || k > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.b32 p, %6, 0;\n setp.eq.b32 q, %6, %6;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %5, p;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %3, %5, q;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %2, %5, q;\n}\n" ::"r"(dt),
                "l"(dah), "l"(dbh), "l"(dbl), "l"(dal), "r"(idesc), "r"(accf_));
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&empty[s]))
                       : "memory");
        }
        if (!ok) {
          atomicExch(&fail, 1);
          break;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&accf[acc]))
                     : "memory");
        ++u;
      }
      // every MMA issued by this thread has completed before TMEM and the ring are released
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(done))
                   : "memory");
      if (!mbar_wait(smem_u32(done), 0)) atomicExch(&fail, 1);
    }
  } else {  // epilogue warps
    const int q = warp & 3, h = (warp - 2) >> 2;
    int u = 0;
    for (int x = blockIdx.x; x < a.nwork; x += gridDim.x) {
      if (__any_sync(0xffffffffu, *(volatile int*)&fail)) break;  // warp-uniform exit
      const TcWorkPos w = tc_decode(a, x);
      const TcProd& p = *w.p;
      if (p.idle) continue;
      const int acc = u & 1, use = u >> 1;
      bool ok = mbar_wait(smem_u32(&accf[acc]), (uint32_t)(use & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) atomicExch(&fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = w.tm * TM + q * 32 + lane;
      const bool split = p.kb_total > p.kbs;
      float* Pz = split ? p.P + (size_t)w.z * p.Mr * p.Nr : nullptr;
#pragma unroll 1
      for (int c0 = h * (TNP / 2); c0 < (h + 1) * (TNP / 2); c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * TNP + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int col0 = w.tn * TNP + c0;
        const int ncol = min(32, p.Nr - col0);
        if (!split) {
          // accumulator row 2i: Re C(i, col), row 2i + 1: Im C(i, col), in adjacent lanes
          float wv[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) wv[j] = __shfl_down_sync(0xffffffffu, __uint_as_float(r[j]), 1);
          if (row < p.Mr && !(lane & 1) && ncol > 0) {
            const float sr = p.rs ? p.rs[row >> 1] : 1.f;
            const float ar = p.ar * sr, ai = p.ai * sr;
            float2* dst0 = p.C + (size_t)col0 * p.ldc + (row >> 1);
            const bool rd = p.br != 0.f || p.bi != 0.f;
#pragma unroll
            for (int j0 = 0; j0 < 32; j0 += 16) {  // old values in two groups (register pressure)
              float2 old[16];
#pragma unroll
              for (int j = 0; j < 16; ++j)
                old[j] = (j0 + j < ncol && rd) ? dst0[(size_t)(j0 + j) * p.ldc] : make_float2(0.f, 0.f);
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                if (j0 + j < ncol) {
                  const float v = __uint_as_float(r[j0 + j]), wi = wv[j0 + j];
                  float2 o;
                  o.x = ar * v - ai * wi + p.br * old[j].x - p.bi * old[j].y;
                  o.y = ar * wi + ai * v + p.br * old[j].y + p.bi * old[j].x;
                  dst0[(size_t)(j0 + j) * p.ldc] = o;
                }
              }
            }
          }
        } else if (row < p.Mr) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (j < ncol) Pz[(size_t)(col0 + j) * p.Mr + row] = __uint_as_float(r[j]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(smem_u32(&acce[acc]));
      ++u;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TNP));
  if (tid == 0 && fail) atomicExch(a.err, 1);
}

// Grouped combine of the split products of a persistent launch: C = (alpha rs[i]) sum_z P_z +
// beta C, the K ranges added in a fixed order.  Block b belongs to the last product with cb0 <= b.
__global__ void tc_group_combine(const TcProd* __restrict__ prods, int nprod) {
  int lo = 0, hi = nprod;
  const long long b = blockIdx.x;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prods[mid].cb0 <= b) lo = mid;
    else hi = mid;
  }
  const TcProd& p = prods[lo];
  if (p.idle || p.kb_total <= p.kbs) return;
  const int M = p.Mr / 2;
  const long long idx = (b - p.cb0) * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * p.Nr) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  const int splits = (p.kb_total + p.kbs - 1) / p.kbs;
  const size_t o = (size_t)j * p.Mr + 2 * i, stride = (size_t)p.Mr * p.Nr;
  float sr = 0.f, si = 0.f;
  for (int z = 0; z < splits; ++z) {
    const float2 v = *reinterpret_cast<const float2*>(p.P + z * stride + o);
    sr += v.x;
    si += v.y;
  }
  const float sc = p.rs ? p.rs[i] : 1.f;
  const float ar = p.ar * sc, ai = p.ai * sc;
  float2* dst = p.C + (size_t)j * p.ldc + i;
  float2 out = make_float2(ar * sr - ai * si, ar * si + ai * sr);
  if (p.br != 0.f || p.bi != 0.f) {
    const float2 o2 = *dst;
    out.x += p.br * o2.x - p.bi * o2.y;
    out.y += p.br * o2.y + p.bi * o2.x;
  }
  *dst = out;
}

// ---- operand preparation -------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// K-major complex source (column c has K complex values at src + c*ld) -> BF16 rows of length
// 2*Kp, [hi | lo] of interleaved pairs.  pair = 0: row c holds (re, im).  pair = 1 (the A operand
// of A^H B): row 2c holds (re, im) and row 2c + 1 holds (-im, re).  One (column c, pair k) element.
__device__ __forceinline__ void prep_kmajor_elem(const float2* __restrict__ src, long long ld, int K, int Kp,
                                                 __nv_bfloat16* __restrict__ dst, int pair, int c, int k) {
  const int half = Kp / 2;
  float re = 0.f, im = 0.f;
  if (k < K) {
    const float2 v = src[(size_t)c * ld + k];
    re = v.x;
    im = v.y;
  }
  __nv_bfloat16 hr, lr, hi_, li_;
  split_bf16(re, hr, lr);
  split_bf16(im, hi_, li_);
  const size_t rowlen = 2 * (size_t)Kp;
  __nv_bfloat162* r0 = reinterpret_cast<__nv_bfloat162*>(dst + (size_t)(pair ? 2 * c : c) * rowlen);
  r0[k] = __halves2bfloat162(hr, hi_);
  r0[half + k] = __halves2bfloat162(lr, li_);
  if (pair) {
    __nv_bfloat16 hmi, lmi;
    split_bf16(-im, hmi, lmi);
    __nv_bfloat162* r1 = reinterpret_cast<__nv_bfloat162*>(dst + (size_t)(2 * c + 1) * rowlen);
    r1[k] = __halves2bfloat162(hmi, hr);
    r1[half + k] = __halves2bfloat162(lmi, lr);
  }
}

__global__ void prep_kmajor(const float2* __restrict__ src, long long ld, int K, int ncols, int Kp,
                            __nv_bfloat16* __restrict__ dst, int pair) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int half = Kp / 2;
  if (idx >= (long long)ncols * half) return;
  const int c = (int)(idx / half), k = (int)(idx - (long long)c * half);
  prep_kmajor_elem(src, ld, K, Kp, dst, pair, c, k);
}

// Grouped form (B operands of a grouped product, pair = 0): block b belongs to the last item with
// b0 <= b.
struct TcPrepItem {
  const float2* src;
  long long ld;
  int K, ncols, Kp, idle;
  __nv_bfloat16* dst;
  long long b0;
};
__global__ void prep_kmajor_group(const TcPrepItem* __restrict__ items, int n) {
  int lo = 0, hi = n;
  const long long b = blockIdx.x;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (items[mid].b0 <= b) lo = mid;
    else hi = mid;
  }
  const TcPrepItem& it = items[lo];
  if (it.idle) return;
  const long long idx = (b - it.b0) * blockDim.x + threadIdx.x;
  const int half = it.Kp / 2;
  if (idx >= (long long)it.ncols * half) return;
  const int c = (int)(idx / half), k = (int)(idx - (long long)c * half);
  prep_kmajor_elem(it.src, it.ld, it.K, it.Kp, it.dst, 0, c, k);
}

// M-major complex A (element (i, k) at src[k*ld + i]) -> BF16 K-major rows for C = A B:
// row 2i: (re, -im) pairs, row 2i + 1: (im, re) pairs (so the real and imaginary parts of output
// row i are adjacent accumulator rows), each row [hi | lo].  32x32 smem transpose.
__global__ void prep_mmajor(const float2* __restrict__ src, long long ld, int M, int K, int Kp,
                            __nv_bfloat16* __restrict__ dst) {
  __shared__ float2 t[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r, i = i0 + threadIdx.x;
    t[r][threadIdx.x] = (k < K && i < M) ? src[(size_t)k * ld + i] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int half = Kp / 2;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, k = k0 + threadIdx.x;
    if (i >= M || k >= half) continue;
    const float2 v = t[threadIdx.x][r];
    __nv_bfloat16 hr, lr, hi_, li_, hmi, lmi;
    split_bf16(v.x, hr, lr);
    split_bf16(v.y, hi_, li_);
    split_bf16(-v.y, hmi, lmi);
    __nv_bfloat162* ra = reinterpret_cast<__nv_bfloat162*>(dst + (size_t)(2 * i) * (2 * (size_t)Kp));
    __nv_bfloat162* rb = reinterpret_cast<__nv_bfloat162*>(dst + (size_t)(2 * i + 1) * (2 * (size_t)Kp));
    ra[k] = __halves2bfloat162(hr, hmi);
    ra[half + k] = __halves2bfloat162(lr, lmi);
    rb[k] = __halves2bfloat162(hi_, hr);
    rb[half + k] = __halves2bfloat162(li_, lr);
  }
}

// C (complex, col-major ldc) = alpha * D + beta * C with D assembled from the K-split partials
// (col-major Mr x Nr, Mr = 2M): re = D(2i, j), im = D(2i + 1, j).
__global__ void tc_combine(const float* __restrict__ P, int nsplit, int Mr, int Nr, int M, int N,
                           float2* __restrict__ C, long long ldc, float ar, float ai, float br, float bi) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int i = (int)(idx % M), j = (int)(idx / M);
  const size_t o = (size_t)j * Mr + 2 * i;
  float sr = 0.f, si = 0.f;
  const size_t stride = (size_t)Mr * Nr;
  for (int z = 0; z < nsplit; ++z) {
    const float2 v = *reinterpret_cast<const float2*>(P + z * stride + o);
    sr += v.x;
    si += v.y;
  }
  float2 out;
  out.x = ar * sr - ai * si;
  out.y = ar * si + ai * sr;
  float2* dst = C + (size_t)j * ldc + i;
  if (br != 0.f || bi != 0.f) {
    const float2 o2 = *dst;
    out.x += br * o2.x - bi * o2.y;
    out.y += br * o2.y + bi * o2.x;
  }
  *dst = out;
}

using tc::encode_fn;

CUtensorMap make_map(const void* base, int rows, int kt, int box_rows = TM) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[2] = {(cuuint64_t)kt, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kt * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                                 strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(KSS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

int sms(kss_ctx ctx) {
  if (!ctx->nsm) {
    int v = 0;
    KSS_CHECK_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device));
    ctx->nsm = v > 0 ? v : 1;
  }
  return ctx->nsm;
}

template <int TNP>
void launch_persist(kss_ctx ctx, const TcPersistArgs& args, int grid) {
  // per device (the attribute belongs to the current device): set at every launch
  KSS_CHECK_CUDA(cudaFuncSetAttribute(tc_persist_kernel<TNP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)p_smem<TNP>()));
  tc_persist_kernel<TNP><<<grid, kPThreads, p_smem<TNP>(), ctx->stream>>>(args);
  KSS_CHECK_CUDA(cudaGetLastError());
}

void ensure_err(kss_ctx ctx) {
  if (!ctx->tc_err.p) {
    ctx->tc_err.alloc(sizeof(int));
    KSS_CHECK_CUDA(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), ctx->stream));
  }
}

// C (M x N complex) = alpha * A_tc (2M x 2Kp) * B_tc (N x 2Kp)^T + beta * C over the three hi/lo
// products: written by the GEMM kernel itself without a K-split, else through partial sums.
// Schedule: form 0 (one CTA per 128 x 128 tile and split, tc_gemm_kernel) or the persistent
// kernel on 128- (form 1) or 64-column (form 2) tiles, and the K-split; autotuned per shape.
void run_tc(kss_ctx ctx, const __nv_bfloat16* Atc, const __nv_bfloat16* Btc, int Kp, int M, int N,
            float2* C, int ldc, double ar, double ai, double br, double bi, const char* tag) {
  const int Mr = 2 * M, Nr = N;
  const int tmn = (Mr + TM - 1) / TM, tnn = (Nr + TN - 1) / TN;
  const int kb_total = Kp / TK;
  const long long tiles = (long long)tmn * tnn;
  if (tiles > 0x7fffffffLL / 2) fail(KSS_EINVAL, "tensor-core GEMM: too many output tiles");
  // K-split plan.  One CTA fits per SM (the ring takes ~194 KB of shared memory).  With at least
  // as many output tiles as SMs there is no split (the kernel writes the complex result itself);
  // otherwise split K so that the grid fills the SMs in one wave, keeping at least 8 k-blocks per
  // CTA.  Every extra split costs a CTA's fixed work (TMEM allocation, pipeline fill, epilogue)
  // and one more set of FP32 partial sums written and read back, so more than one wave of split
  // CTAs does not pay.
  // This is the closed-form plan; the autotuner times it against the other forms and splits at
  // first use of the shape.
  const int nsm = sms(ctx);
  int plan = 1;
  if (tiles < nsm) plan = (int)std::max(1LL, std::min<long long>(nsm / tiles, kb_total / 8));
  ensure_err(ctx);
  const CUtensorMap ma = make_map(Atc, Mr, 2 * Kp), mb = make_map(Btc, Nr, 2 * Kp);
  const CUtensorMap mb64 = make_map(Btc, Nr, 2 * Kp, 64);
  // per device (the attribute belongs to the current device): set at every launch, as the
  // other kernels of the path do
  KSS_CHECK_CUDA(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  const std::string name = std::string("tc_gemm_bf16x3:") + tag, cname = std::string("tc_combine:") + tag;
  // One product with schedule ch into Cd (ldd, alpha, beta).
  auto launch = [&](GemmChoice ch, float2* Cd, int ldd, double br_, double bi_, bool prof) {
    int splits = std::max(1, std::min(ch.splits, kb_total));
    const int kps = (kb_total + splits - 1) / splits;
    splits = (kb_total + kps - 1) / kps;
    if (splits > 1) ctx->tc_part.ensure((size_t)splits * Mr * Nr * sizeof(float));
    const bool fused = splits == 1;
    {
      ProfScope ps(ctx, prof_register(prof ? name.c_str() : "gemm_tuning"));
      if (ch.form == 0) {
        tc_gemm_kernel<<<dim3((unsigned)tiles, splits, 1), kTcThreads, kTcSmem, ctx->stream>>>(
            ma, mb, ctx->tc_part.as<float>(), Mr, Nr, tnn, kps, kb_total, Kp, ctx->tc_err.as<int>(),
            fused ? Cd : nullptr, ldd, (float)ar, (float)ai, (float)br_, (float)bi_);
        KSS_CHECK_CUDA(cudaGetLastError());
      } else {
        const int tnp = ch.form == 2 ? 64 : 128;
        TcPersistArgs args;
        std::memset(&args, 0, sizeof(args));
        args.ma = ma;
        args.mb = ch.form == 2 ? mb64 : mb;
        TcProd& p = args.one;
        p.Mr = Mr;
        p.Nr = Nr;
        p.tmn = tmn;
        p.tnn = (Nr + tnp - 1) / tnp;
        p.kb_total = kb_total;
        p.kbs = kps;
        p.kp = Kp;
        p.C = Cd;
        p.ldc = ldd;
        p.ar = (float)ar;
        p.ai = (float)ai;
        p.br = (float)br_;
        p.bi = (float)bi_;
        p.P = ctx->tc_part.as<float>();
        args.nprod = 1;
        args.nwork = p.tmn * p.tnn * splits;
        args.err = ctx->tc_err.as<int>();
        const int grid = std::max(1, std::min(args.nwork, nsm));
        if (ch.form == 2) launch_persist<64>(ctx, args, grid);
        else launch_persist<128>(ctx, args, grid);
      }
    }
    if (fused) return;
    const long long mn = (long long)M * N;
    ProfScope ps(ctx, prof_register(prof ? cname.c_str() : "gemm_tuning"));
    tc_combine<<<(unsigned)((mn + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->tc_part.as<float>(), splits, Mr, Nr, M, N, Cd, ldd, (float)ar, (float)ai, (float)br_, (float)bi_);
    KSS_CHECK_CUDA(cudaGetLastError());
  };
  // Candidates: every form with no split, the plan and the splits filling one to three waves.  Each
  // split accumulates at most kMaxKbSplit k-blocks in FP32 (TMEM), which bounds the rounding of
  // the accumulation chain for long K; the partial sums of the splits are added by the combine.
  const int smin = (kb_total + kMaxKbSplit - 1) / kMaxKbSplit;
  const int smax = std::max(smin, kb_total / 4);
  auto fmax = [&](int form) { return form == 0 ? std::max(smin, kb_total / 8) : smax; };
  std::vector<GemmChoice> cand;
  for (int form = 0; form < 3; ++form) {
    const long long t = (long long)tmn * ((Nr + (form == 2 ? 63 : 127)) / (form == 2 ? 64 : 128));
    std::vector<int> sp{1, plan};
    for (int w = 1; w <= 3; ++w) sp.push_back((int)std::max(1LL, (long long)w * nsm / std::max(1LL, t)));
    for (int x : sp) cand.push_back(GemmChoice{form, std::max(smin, std::min(x, fmax(form)))});
  }
  GemmChoice ch = tuned_gemm(ctx, GT_BF16X3, Mr, Nr, kb_total, cand, GemmChoice{0, std::max(smin, std::min(plan, fmax(0)))},
                             [&](GemmChoice c) {
                               ctx->tune_c.ensure((size_t)M * N * sizeof(float2));
                               launch(c, ctx->tune_c.as<float2>(), M, 0.0, 0.0, false);
                             });
  ch.form = std::max(0, std::min(ch.form, 2));
  ch.splits = std::max(smin, std::min(ch.splits, fmax(ch.form)));
  launch(ch, C, ldc, br, bi, true);
}

int kpad(int K) { return ((2 * K + TK - 1) / TK) * TK; }

}  // namespace

// C (M x N) = alpha A^H B + beta C, complex64; A: K x M (lda), B: K x N (ldb).
void tc_gemm_cn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                void* C, int ldc, double ar, double ai, double br, double bi, const char* tag) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  const int Kp = kpad(K);
  ctx->tc_a.ensure(tc_split_cn_bytes(M, K));
  ctx->tc_b.ensure((size_t)N * 2 * Kp * 2);
  __nv_bfloat16* Atc = ctx->tc_a.as<__nv_bfloat16>();
  {
    ProfScope ps(ctx, prof_register("tc_prep"));
    const long long na = (long long)M * (Kp / 2);
    prep_kmajor<<<(unsigned)((na + 255) / 256), 256, 0, ctx->stream>>>((const float2*)A, lda, K, M, Kp, Atc, 1);
  }
  tc_gemm_cn_split(ctx, M, N, K, Atc, B, ldb, C, ldc, ar, ai, br, bi, tag);
}

// C (M x N) = alpha A B + beta C, complex64; A: M x K (lda, M contiguous), B: K x N (ldb).
void tc_gemm_nn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                void* C, int ldc, double ar, double ai, double br, double bi, const char* tag) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  const int Kp = kpad(K);
  ctx->tc_a.ensure(tc_split_nn_bytes(M, K));
  __nv_bfloat16* Atc = ctx->tc_a.as<__nv_bfloat16>();
  {
    ProfScope ps(ctx, prof_register("tc_prep"));
    dim3 g((M + 31) / 32, (Kp / 2 + 31) / 32);
    prep_mmajor<<<g, dim3(32, 8), 0, ctx->stream>>>((const float2*)A, lda, M, K, Kp, Atc);
  }
  tc_gemm_nn_split(ctx, M, N, K, Atc, B, ldb, C, ldc, ar, ai, br, bi, tag);
}

// Forms with A already split (static operands such as the projector table, prepared once with
// tc_split_* and kept): only B is prepared per call.  Both split forms of an M x K complex A hold
// 2M rows of 2 * kpad(K) BF16 values.
size_t tc_split_cn_bytes(int M, int K) { return (size_t)2 * M * 2 * kpad(K) * 2; }
size_t tc_split_nn_bytes(int M, int K) { return (size_t)2 * M * 2 * kpad(K) * 2; }

void tc_split_cn(kss_ctx ctx, int M, int K, const void* A, int lda, void* Atc) {
  const int Kp = kpad(K);
  const long long na = (long long)M * (Kp / 2);
  prep_kmajor<<<(unsigned)((na + 255) / 256), 256, 0, ctx->stream>>>((const float2*)A, lda, K, M, Kp,
                                                                    (__nv_bfloat16*)Atc, 1);
  KSS_CHECK_CUDA(cudaGetLastError());
}

void tc_split_nn(kss_ctx ctx, int M, int K, const void* A, int lda, void* Atc) {
  const int Kp = kpad(K);
  dim3 g((M + 31) / 32, (Kp / 2 + 31) / 32);
  prep_mmajor<<<g, dim3(32, 8), 0, ctx->stream>>>((const float2*)A, lda, M, K, Kp, (__nv_bfloat16*)Atc);
  KSS_CHECK_CUDA(cudaGetLastError());
}

namespace {
// B operand (K x N complex, ldb) -> N BF16 rows [hi | lo] of (re, im) pairs in the context buffer.
const __nv_bfloat16* prep_b(kss_ctx ctx, int N, int K, const void* B, int ldb) {
  const int Kp = kpad(K);
  ctx->tc_b.ensure((size_t)N * 2 * Kp * 2);
  __nv_bfloat16* Btc = ctx->tc_b.as<__nv_bfloat16>();
  ProfScope ps(ctx, prof_register("tc_prep"));
  const long long nb = (long long)N * (Kp / 2);
  prep_kmajor<<<(unsigned)((nb + 255) / 256), 256, 0, ctx->stream>>>((const float2*)B, ldb, K, N, Kp, Btc, 0);
  return Btc;
}
}  // namespace

void tc_gemm_cn_split(kss_ctx ctx, int M, int N, int K, const void* Atc, const void* B, int ldb, void* C, int ldc,
                      double ar, double ai, double br, double bi, const char* tag) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  const __nv_bfloat16* Btc = prep_b(ctx, N, K, B, ldb);
  run_tc(ctx, (const __nv_bfloat16*)Atc, Btc, kpad(K), M, N, (float2*)C, ldc, ar, ai, br, bi, tag);
}

void tc_gemm_nn_split(kss_ctx ctx, int M, int N, int K, const void* Atc, const void* B, int ldb, void* C, int ldc,
                      double ar, double ai, double br, double bi, const char* tag) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  const __nv_bfloat16* Btc = prep_b(ctx, N, K, B, ldb);
  run_tc(ctx, (const __nv_bfloat16*)Atc, Btc, kpad(K), M, N, (float2*)C, ldc, ar, ai, br, bi, tag);
}

// ---- grouped products (batch engine) ----------------------------------------------------------
void TcGroupPlan::build(kss_ctx ctx, const std::vector<TcGroupSpec>& specs, int steps) {
  n_ = (int)specs.size();
  steps_ = std::max(1, steps);
  prod_bytes_ = sizeof(TcProd);
  prep_bytes_ = sizeof(TcPrepItem);
  if (!n_) return;
  const int nsm = sms(ctx);
  ensure_err(ctx);
  // Column tile: 64 or 128, whichever wastes less MMA work on the products' column counts (a
  // tile's A operand costs about as much to stage as 64 of its columns).
  long long c64 = 0, c128 = 0;
  for (const auto& sp : specs) {
    const long long tm = (2LL * sp.M + TM - 1) / TM;
    c64 += tm * ((sp.N + 63) / 64) * (64 + 64);
    c128 += tm * ((sp.N + 127) / 128) * (128 + 64);
  }
  tnp_ = c64 <= c128 ? 64 : 128;
  // K-split: none when the launch has at least two waves of tiles; otherwise splits of about
  // equal k-block counts (at least 8) giving about four works per SM, so that the static
  // round-robin assignment of works to CTAs stays balanced.
  long long tiles = 0, tkb = 0;
  for (const auto& sp : specs) {
    const long long t = ((2LL * sp.M + TM - 1) / TM) * ((sp.N + tnp_ - 1) / tnp_);
    tiles += t;
    tkb += t * (kpad(sp.K) / TK);
  }
  int kbs = kMaxKbSplit;
  if (tiles < 2LL * nsm) kbs = (int)std::min<long long>(kMaxKbSplit, std::max(8LL, (tkb + 4LL * nsm - 1) / (4LL * nsm)));
  std::vector<TcProd> prods(n_);
  std::vector<TcPrepItem> preps(n_);
  std::vector<CUtensorMap> maps(2 * (size_t)n_);
  size_t btc = 0, part = 0;
  std::vector<size_t> boff(n_), poff(n_);
  long long w = 0, cb = 0, pb = 0;
  any_split_ = false;
  for (int i = 0; i < n_; ++i) {
    const TcGroupSpec& sp = specs[i];
    KSS_REQUIRE(sp.M > 0 && sp.N > 0 && sp.K > 0 && sp.Atc, "grouped product: empty operand");
    const int Kp = kpad(sp.K);
    TcProd& p = prods[i];
    std::memset(&p, 0, sizeof(p));
    p.Mr = 2 * sp.M;
    p.Nr = sp.N;
    p.tmn = (p.Mr + TM - 1) / TM;
    p.tnn = (p.Nr + tnp_ - 1) / tnp_;
    p.kb_total = Kp / TK;
    p.kbs = std::min(p.kb_total, kbs);
    const int splits = (p.kb_total + p.kbs - 1) / p.kbs;
    p.kp = Kp;
    p.w0 = (int)w;
    w += (long long)p.tmn * p.tnn * splits;
    p.ldc = sp.ldc;
    p.rs = sp.rs;
    p.cb0 = cb;
    if (splits > 1) {
      any_split_ = true;
      poff[i] = part;
      part += (size_t)splits * p.Mr * p.Nr;
      cb += ((long long)sp.M * sp.N + 255) / 256;
    }
    boff[i] = btc;
    btc += (size_t)sp.N * 2 * Kp;
    TcPrepItem& q = preps[i];
    std::memset(&q, 0, sizeof(q));
    q.ld = sp.ldb;
    q.K = sp.K;
    q.ncols = sp.N;
    q.Kp = Kp;
    q.b0 = pb;
    pb += ((long long)sp.N * (Kp / 2) + 255) / 256;
  }
  KSS_REQUIRE(w < 0x7fffffffLL && pb < 0x7fffffffLL && cb < 0x7fffffffLL, "grouped product: too many tiles");
  nwork_ = (int)w;
  prep_blocks_ = (int)pb;
  comb_blocks_ = cb;
  d_btc_.ensure(btc * sizeof(__nv_bfloat16));
  if (part) d_part_.ensure(part * sizeof(float));
  for (int i = 0; i < n_; ++i) {
    const TcGroupSpec& sp = specs[i];
    const int Kp = kpad(sp.K);
    __nv_bfloat16* b = d_btc_.as<__nv_bfloat16>() + boff[i];
    preps[i].dst = b;
    if (prods[i].kb_total > prods[i].kbs) prods[i].P = d_part_.as<float>() + poff[i];
    maps[2 * i] = make_map(sp.Atc, 2 * sp.M, 2 * Kp);
    maps[2 * i + 1] = make_map(b, sp.N, 2 * Kp, tnp_);
  }
  h_prod_.resize((size_t)steps_ * n_ * prod_bytes_);
  h_prep_.resize((size_t)steps_ * n_ * prep_bytes_);
  for (int j = 0; j < steps_; ++j) {
    std::memcpy(h_prod_.data() + (size_t)j * n_ * prod_bytes_, prods.data(), n_ * prod_bytes_);
    std::memcpy(h_prep_.data() + (size_t)j * n_ * prep_bytes_, preps.data(), n_ * prep_bytes_);
  }
  d_maps_.ensure(maps.size() * sizeof(CUtensorMap));
  d_prod_.ensure(h_prod_.size());
  d_prep_.ensure(h_prep_.size());
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_maps_.p, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                                 ctx->stream));
  KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  // per device (this context's): set here, outside any stream capture of the launches
  if (tnp_ == 64)
    KSS_CHECK_CUDA(cudaFuncSetAttribute(tc_persist_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)p_smem<64>()));
  else
    KSS_CHECK_CUDA(cudaFuncSetAttribute(tc_persist_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)p_smem<128>()));
}

void TcGroupPlan::set(int step, int i, const void* Bsrc, void* C, float ar, float br, bool idle) {
  KSS_REQUIRE(step >= 0 && step < steps_ && i >= 0 && i < n_, "grouped product: index out of range");
  TcProd* p = reinterpret_cast<TcProd*>(h_prod_.data() + ((size_t)step * n_ + i) * prod_bytes_);
  TcPrepItem* q = reinterpret_cast<TcPrepItem*>(h_prep_.data() + ((size_t)step * n_ + i) * prep_bytes_);
  q->src = (const float2*)Bsrc;
  q->idle = idle ? 1 : 0;
  p->C = (float2*)C;
  p->ar = ar;
  p->ai = 0.f;
  p->br = br;
  p->bi = 0.f;
  p->idle = idle ? 1 : 0;
}

void TcGroupPlan::upload(cudaStream_t st) {
  if (!n_) return;
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_prod_.p, h_prod_.data(), h_prod_.size(), cudaMemcpyHostToDevice, st));
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_prep_.p, h_prep_.data(), h_prep_.size(), cudaMemcpyHostToDevice, st));
}

void TcGroupPlan::launch(kss_ctx ctx, int step, const char* tag) const {
  if (!n_) return;
  KSS_REQUIRE(step >= 0 && step < steps_, "grouped product: step out of range");
  const TcProd* prods = reinterpret_cast<const TcProd*>(d_prod_.as<unsigned char>() + (size_t)step * n_ * prod_bytes_);
  const TcPrepItem* preps =
      reinterpret_cast<const TcPrepItem*>(d_prep_.as<unsigned char>() + (size_t)step * n_ * prep_bytes_);
  {
    static const int id = prof_register("tc_prep_group");
    ProfScope ps(ctx, id);
    prep_kmajor_group<<<prep_blocks_, 256, 0, ctx->stream>>>(preps, n_);
    KSS_CHECK_CUDA(cudaGetLastError());
  }
  {
    ProfScope ps(ctx, prof_register((std::string("tc_group_bf16x3:") + tag).c_str()));
    TcPersistArgs args;
    std::memset(&args, 0, sizeof(args));
    args.prods = prods;
    args.maps = d_maps_.as<CUtensorMap>();
    args.nprod = n_;
    args.nwork = nwork_;
    args.err = ctx->tc_err.as<int>();
    const int grid = std::max(1, std::min(nwork_, sms(ctx)));
    if (tnp_ == 64)
      tc_persist_kernel<64><<<grid, kPThreads, p_smem<64>(), ctx->stream>>>(args);
    else
      tc_persist_kernel<128><<<grid, kPThreads, p_smem<128>(), ctx->stream>>>(args);
    KSS_CHECK_CUDA(cudaGetLastError());
  }
  if (any_split_) {
    ProfScope ps(ctx, prof_register((std::string("tc_group_combine:") + tag).c_str()));
    tc_group_combine<<<(unsigned)comb_blocks_, 256, 0, ctx->stream>>>(prods, n_);
    KSS_CHECK_CUDA(cudaGetLastError());
  }
}

// ---- the failure path of the bounded waits, exercised without a fault --------------------------
namespace {
// One thread waits on a device word that nothing writes, with the pipeline waits' %globaltimer
// limit pattern, and then raises the tensor-core error flag as a pipeline wait that gave up does.
__global__ void bounded_wait_probe(const int* __restrict__ word, unsigned long long limit_ns, int* __restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long t0 = globaltimer();
  while (*(const volatile int*)word == 0)
    if (globaltimer() - t0 > limit_ns) {
      atomicExch(err, 1);
      return;
    }
}
}  // namespace

void tc_wait_selftest(kss_ctx ctx, double limit_ms) {
  KSS_REQUIRE(limit_ms > 0 && limit_ms <= 1000, "limit_ms must be in (0, 1000]");
  if (!ctx->tc_err.p) {
    ctx->tc_err.alloc(sizeof(int));
    KSS_CHECK_CUDA(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), ctx->stream));
  }
  DevBuf word;
  word.alloc(sizeof(int));
  KSS_CHECK_CUDA(cudaMemsetAsync(word.p, 0, sizeof(int), ctx->stream));
  bounded_wait_probe<<<1, 32, 0, ctx->stream>>>(word.as<int>(), (unsigned long long)(limit_ms * 1e6),
                                                ctx->tc_err.as<int>());
  KSS_CHECK_CUDA(cudaGetLastError());
  KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
}

// Device-side failure flag of the tensor-core kernels (bounded waits that gave up).
int tc_error_flag(kss_ctx ctx, bool reset) {
  if (!ctx->tc_err.p) return 0;
  int v = 0;
  KSS_CHECK_CUDA(cudaMemcpyAsync(&v, ctx->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  if (reset && v) KSS_CHECK_CUDA(cudaMemsetAsync(ctx->tc_err.p, 0, sizeof(int), ctx->stream));
  return v;
}

}  // namespace kss

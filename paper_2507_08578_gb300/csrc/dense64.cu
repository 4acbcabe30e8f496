// FP64 dense generalised Hermitian eigensolver for the Rayleigh-Ritz step (§5.1: the subspace
// problem of the Chebyshev-filtered iteration, "less efficient on GPU" and called rarely).
//
// Solves A x = lambda B x for Hermitian A and Hermitian positive definite B (n x n, complex128,
// column-major, lower triangles read), returning all eigenvalues ascending and B-orthonormal
// eigenvectors, in five phases written out here:
//
//   1. Cholesky B = L L^H (blocked right-looking: a 16-column panel at a time, its diagonal block
//      factored in shared memory, the rows below solved against it, then a rank-16 update of the
//      trailing lower triangle).
//   2. Reduction to standard form C = L^{-1} A L^{-H}: two forward substitutions with n
//      right-hand sides each (X = L^{-1} A, then C = L^{-1} X^H, using A = A^H).
//   3. Householder tridiagonalisation C = Q T Q^H (unblocked, on the full Hermitian matrix):
//      per column, the reflector H = I - tau v v^H with a real subdiagonal (beta = -sign(Re
//      alpha) |x|), p = tau C v, w = p - (tau/2)(p^H v) v, C <- C - v w^H - w v^H.
//   4. Eigenpairs of the real symmetric tridiagonal T: every eigenvalue by bisection on the
//      Sturm count (the number of negative pivots of the LDL^T factorisation of T - sigma I),
//      every eigenvector by inverse iteration with the partially pivoted LU of T - lambda I;
//      eigenvalues closer than 1e-5 |T| form a cluster whose vectors are orthogonalised against
//      each other (modified Gram-Schmidt) in every iteration.
//   5. Back-transformation x = L^{-H} Q z (the reflectors applied to each column of Z in
//      reverse order, then a backward substitution with L^H).
//
// Real symmetric pencils (the Gamma point) run the same phases in real arithmetic on compact real
// copies of the lower triangles: a quarter of the FP64 operations of the O(n^3) phases.
//
// Parallel organisation.  The same phase code runs on a "team": either one CTA (many small
// pencils, one CTA each, barrier = __syncthreads) or a whole cooperative grid (one large pencil,
// barrier = a grid barrier of this file with a bounded wait).  Work that is independent per
// column (the triangular solves, the reflector applications, the inverse iterations) needs no
// team barrier: one warp owns a column and each lane owns the rows r = lane (mod 32), so values
// written by one lane are read back only by that lane and everything else travels by shuffles.
// The barrier count is about n + n/8 per pencil (one per tridiagonalisation step, two per 16-column
// Cholesky panel).
//
// Every grid-barrier wait gives up after a time limit; the kernel then raises the control
// block's error word, sets the pencil's info to -1, and every thread leaves at its next barrier;
// callers report KSS_ETIMEOUT.  A non-positive Cholesky pivot at column j stops the solve with
// info = j + 1 (the LAPACK convention) and leaves the outputs undefined.
#include <cuda/atomic>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kss_internal.h"

namespace kss {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
static_assert((kWarps & (kWarps - 1)) == 0, "the CTA reductions take a power-of-two warp count");

// ---- complex helpers ---------------------------------------------------------------------------
// On GB300 an SM retires about two FP64 fused multiply-adds per clock, so every FP64 instruction
// counts: complex products are written as chains of fused multiply-adds (4 per complex
// multiply-accumulate) and scalars a whole warp or CTA needs are computed once and broadcast.
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // c + a b
  return make_double2(fma(-a.y, b.y, fma(a.x, b.x, c.x)), fma(a.y, b.x, fma(a.x, b.y, c.y)));
}
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {  // c - a b
  return make_double2(fma(a.y, b.y, fma(-a.x, b.x, c.x)), fma(-a.y, b.x, fma(-a.x, b.y, c.y)));
}
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 c) {  // c + conj(a) b
  return make_double2(fma(a.y, b.y, fma(a.x, b.x, c.x)), fma(-a.y, b.x, fma(a.x, b.y, c.y)));
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 shfl_c(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ double2 warp_sum_c(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The same operations on real scalars: the phases are templates on the scalar type S (double2 for
// Hermitian pencils, double for real symmetric ones, which then take a quarter of the FP64 work of
// the O(n^3) phases and half the memory traffic).
__device__ __forceinline__ double cmul(double a, double b) { return a * b; }
__device__ __forceinline__ double cmulc(double a, double b) { return a * b; }
__device__ __forceinline__ double cfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double cfms(double a, double b, double c) { return fma(-a, b, c); }
__device__ __forceinline__ double cfmac(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double conjd(double a) { return a; }
__device__ __forceinline__ double cadd(double a, double b) { return a + b; }
__device__ __forceinline__ double csub(double a, double b) { return a - b; }
__device__ __forceinline__ double cscale(double a, double s) { return a * s; }
__device__ __forceinline__ double shfl_c(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double warp_sum_c(double v) { return warp_sum(v); }
__device__ __forceinline__ double shfl_xor_c(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double2 shfl_xor_c(double2 v, int o) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

__device__ __forceinline__ double re(double a) { return a; }
__device__ __forceinline__ double re(double2 a) { return a.x; }
__device__ __forceinline__ double im(double) { return 0.0; }
__device__ __forceinline__ double im(double2 a) { return a.y; }
template <class S>
__device__ __forceinline__ S mk(double x, double y);
template <>
__device__ __forceinline__ double mk<double>(double x, double) { return x; }
template <>
__device__ __forceinline__ double2 mk<double2>(double x, double y) { return make_double2(x, y); }
// s + |a|^2
__device__ __forceinline__ double abs2_acc(double a, double s) { return fma(a, a, s); }
__device__ __forceinline__ double abs2_acc(double2 a, double s) { return fma(a.x, a.x, fma(a.y, a.y, s)); }
// 1 / a
__device__ __forceinline__ double cinv(double a) { return 1.0 / a; }
__device__ __forceinline__ double2 cinv(double2 a) {
  const double r = 1.0 / (a.x * a.x + a.y * a.y);
  return make_double2(a.x * r, -a.y * r);
}
// complex128 value of a scalar (the caller's matrices are complex128 in both cases)
__device__ __forceinline__ double2 widen(double a) { return make_double2(a, 0.0); }
__device__ __forceinline__ double2 widen(double2 a) { return a; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Control block of one grid-team solve (zeroed before the launch).
struct Ctl {
  unsigned count;  // barrier arrivals (monotonic)
  unsigned pad0;
  int err;  // 1: a barrier wait gave up
  int pad1;
  unsigned long long t[8];  // %globaltimer at the start and after each phase (measurement)
};

struct CtaTeam {
  __device__ int rank() const { return threadIdx.x; }
  // rank for per-thread independent work (the same as rank() on one CTA)
  __device__ int srank() const { return threadIdx.x; }
  __device__ int swrank() const { return threadIdx.x >> 5; }  // the same for per-warp work
  __device__ int size() const { return blockDim.x; }
  __device__ int wsize() const { return blockDim.x >> 5; }
  __device__ bool sync() const {
    __syncthreads();
    return true;
  }
  __device__ void stamp(int) const {}
};

struct GridTeam {
  Ctl* ctl;
  int* info;  // the pencil's status word: -1 when a barrier wait gave up
  unsigned long long limit_ns;
  __device__ int rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  // rank for per-thread independent work, spread over the CTAs first so that n work items use
  // every SM's FP64 units instead of the first few CTAs'
  __device__ int srank() const { return threadIdx.x * gridDim.x + blockIdx.x; }
  __device__ int swrank() const { return (threadIdx.x >> 5) * gridDim.x + blockIdx.x; }
  __device__ int size() const { return gridDim.x * blockDim.x; }
  __device__ int wsize() const { return (gridDim.x * blockDim.x) >> 5; }
  // time stamp k (by one thread, after the barrier that ends a phase)
  __device__ void stamp(int k) const {
    if (rank() == 0) ctl->t[k] = global_ns();
  }
  // Grid barrier (all CTAs are resident: cooperative launch).  The counter only grows: barrier
  // number b (counted by every thread in its own copy of the team) is passed once it reaches
  // b x gridDim.x.  Each CTA arrives with one release add, which makes the writes of all its
  // threads (ordered before it by __syncthreads) visible to any thread that acquires the counter,
  // and waits with acquire loads in a bounded spin.  Returns false when the solve has been
  // abandoned.
  mutable unsigned epoch = 0;
  __device__ bool sync() const {
    __shared__ int s_ok;
    __syncthreads();
    const unsigned target = ++epoch * gridDim.x;
    if (threadIdx.x == 0) {
      cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(ctl->count);
      cuda::atomic_ref<int, cuda::thread_scope_device> err(ctl->err);
      int ok = err.load(cuda::memory_order_relaxed) == 0;
      if (ok) {
        cnt.fetch_add(1u, cuda::memory_order_release);
        const unsigned long long t0 = global_ns();
        unsigned spins = 0;
        while (cnt.load(cuda::memory_order_acquire) < target) {
          if (err.load(cuda::memory_order_relaxed)) {
            ok = 0;
            break;
          }
          if ((++spins & 63u) == 0 && global_ns() - t0 > limit_ns) {
            err.store(1, cuda::memory_order_relaxed);
            *info = -1;
            ok = 0;
            break;
          }
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  }
};

// One pencil and its workspace.  For a complex pencil (S = double2) A and B are the caller's
// matrices, worked on in place; for a real one (S = double) they are compact real copies (ld n) in
// the workspace, and the results are written back to the caller's complex matrices at the end.
template <class S>
struct Pencil {
  S* A;         // n x n (lda): in A, out eigenvectors
  S* B;         // n x n (ldb): in B, out Cholesky factor L (lower)
  double* w;    // n eigenvalues (out)
  int* info;    // out: 0, or j + 1 for a non-positive pivot at column j
  int n, lda, ldb;
  S* R;         // n x n (ld n): reduction workspace, then the reflector vectors
  double* Z;    // n x n (ld n): eigenvectors of T
  double* wk;   // 7 n^2 doubles: inverse-iteration arrays
  double* vec;  // 11 n + 8 doubles: d, e, tau (S), p (2 x S), 1/L_jj, e^2, FP32 d and e^2
  int smem_cols;  // 1: the launch gives every warp n words of S of dynamic shared memory
  double2* outA;  // the caller's A and B (complex128; the same as A and B when S = double2)
  double2* outB;
  int ldoa, ldob;
};

// ---- phase 0: inputs ---------------------------------------------------------------------------
// Real pencils: the real parts of the lower triangles into the compact copies.
template <class Team>
__device__ bool prepare(const Team& T, const Pencil<double>& P) {
  const int n = P.n, lane = threadIdx.x & 31;
  for (int c = T.swrank(); c < n; c += T.wsize()) {
    const double2* __restrict__ ia = P.outA + (size_t)c * P.ldoa;
    const double2* __restrict__ ib = P.outB + (size_t)c * P.ldob;
    double* __restrict__ a = P.A + (size_t)c * P.lda;
    double* __restrict__ b = P.B + (size_t)c * P.ldb;
    for (int i = c + lane; i < n; i += 32) {
      a[i] = ia[i].x;
      b[i] = ib[i].x;
    }
  }
  return T.sync();
}
template <class Team>
__device__ bool prepare(const Team&, const Pencil<double2>&) {
  return true;  // worked on in place
}

// Real pencils: L (lower triangle) back into the caller's B.
template <class Team>
__device__ void finish(const Team& T, const Pencil<double>& P) {
  const int n = P.n, lane = threadIdx.x & 31;
  for (int c = T.swrank(); c < n; c += T.wsize()) {
    const double* __restrict__ b = P.B + (size_t)c * P.ldb;
    double2* __restrict__ ob = P.outB + (size_t)c * P.ldob;
    for (int i = c + lane; i < n; i += 32) ob[i] = make_double2(b[i], 0.0);
  }
}
template <class Team>
__device__ void finish(const Team&, const Pencil<double2>&) {}

// ---- phase 1: Cholesky B = L L^H -----------------------------------------------------------------
template <class S>
__device__ __forceinline__ double* vrdiag(const Pencil<S>& P) { return P.vec + 8 * P.n; }

// Panel width of the blocked Cholesky: 16 columns (one row of the panel lives in a thread's
// registers while it is solved against the diagonal block).
template <class S> __host__ __device__ constexpr int chol_panel() { return 16; }
// Shared memory of the blocked Cholesky: the diagonal block (pitch panel + 1) and its 1 / L[j][j].
template <class S> __host__ __device__ constexpr size_t chol_smem() {
  return sizeof(S) * (size_t)chol_panel<S>() * (chol_panel<S>() + 1) + sizeof(double) * chol_panel<S>();
}

// Blocked right-looking Cholesky B = L L^H in panels of W columns, two team barriers per panel:
//   1. every CTA factors the W x W diagonal block in its own shared memory (the same arithmetic
//      in every CTA, so the copies agree bit for bit; the team's first CTA writes it back);
//   2. the rows below it are solved against it, L21 = A21 L11^{-H} (one warp per 32 rows, one
//      row per lane, its W entries in registers): no barrier between the rows;
//   3. barrier; the trailing lower triangle is updated, A22 -= L21 L21^H (one warp per column,
//      one row per lane, the column's W factors broadcast once); barrier.
// Returns false when the solve stops (non-positive pivot: *info set; or an abandoned barrier).
template <class Team, class S>
__device__ bool cholesky(const Team& T, const Pencil<S>& P, S* smem) {
  constexpr int W = chol_panel<S>(), LP = W + 1;
  const int n = P.n, ld = P.ldb;
  S* B = P.B;
  double* rd = vrdiag(P);
  S* Lb = smem;  // diagonal block, column-major with pitch LP
  double* rdb = reinterpret_cast<double*>(Lb + W * LP);
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool first_cta = T.rank() < (int)blockDim.x;
  for (int p0 = 0; p0 < n; p0 += W) {
    const int w = min(W, n - p0);
    // 1. the diagonal block
    for (int e = tid; e < W * W; e += blockDim.x) {
      const int c = e / W, r = e - c * W;
      Lb[c * LP + r] = (r < w && c < w && r >= c) ? B[(p0 + r) + (size_t)(p0 + c) * ld] : mk<S>(0.0, 0.0);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (warp == 0) {  // unblocked right-looking on the block, lane = row
      for (int j = 0; j < w; ++j) {
        const double d = re(Lb[j * LP + j]);
        if (!(d > 0.0) || !isfinite(d)) {
          if (lane == 0) s_bad = p0 + j + 1;
          break;
        }
        const double sd = sqrt(d), r = 1.0 / sd;
        if (lane > j && lane < w) Lb[j * LP + lane] = cscale(Lb[j * LP + lane], r);
        if (lane == j) {
          Lb[j * LP + j] = mk<S>(sd, 0.0);
          rdb[j] = r;
        }
        __syncwarp();
        for (int k = j + 1; k < w; ++k) {
          const S lkj = conjd(Lb[j * LP + k]);
          if (lane >= k && lane < w) Lb[k * LP + lane] = cfms(Lb[j * LP + lane], lkj, Lb[k * LP + lane]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (s_bad) {
      if (T.rank() == 0) *P.info = s_bad;
      return false;
    }
    if (first_cta) {
      for (int e = tid; e < w * w; e += blockDim.x) {
        const int c = e / w, r = e - c * w;
        if (r >= c) B[(p0 + r) + (size_t)(p0 + c) * ld] = Lb[c * LP + r];
      }
      for (int j = tid; j < w; j += blockDim.x) rd[p0 + j] = rdb[j];
    }
    // 2. the rows below: l_ij = (a_ij - sum_{k<j} l_ik conj(L11[j][k])) / L11[j][j]
    for (int rb = p0 + w + 32 * T.swrank(); rb < n; rb += 32 * T.wsize()) {
      const int i = rb + lane;
      if (i < n) {
        S row[W];
#pragma unroll
        for (int j = 0; j < W; ++j) row[j] = j < w ? B[i + (size_t)(p0 + j) * ld] : mk<S>(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < W; ++j) {
          S v = row[j];
#pragma unroll
          for (int k = 0; k < j; ++k) v = cfms(row[k], conjd(Lb[k * LP + j]), v);
          row[j] = cscale(v, rdb[j]);
        }
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w) B[i + (size_t)(p0 + j) * ld] = row[j];
      }
    }
    if (!T.sync()) return false;
    // 3. the trailing lower triangle
    if (p0 + w < n) {
      for (int k = p0 + w + T.swrank(); k < n; k += T.wsize()) {
        S f[W];
        const S mine = lane < w ? conjd(B[k + (size_t)(p0 + lane) * ld]) : mk<S>(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < W; ++j) f[j] = shfl_c(mine, j);
        S* __restrict__ ck = B + (size_t)k * ld;
        // two rows per lane and two partial sums per row: four independent accumulation chains
        for (int i = k + lane; i < n; i += 64) {
          const int i2 = i + 32;
          S a0 = mk<S>(0.0, 0.0), a1 = a0, c0 = a0, c1 = a0;
#pragma unroll
          for (int j = 0; j < W; j += 2) {
            const S* pj = B + (size_t)(p0 + j) * ld;
            const S* pk = pj + ld;
            if (j < w) a0 = cfma(pj[i], f[j], a0);
            if (j + 1 < w) a1 = cfma(pk[i], f[j + 1], a1);
            if (i2 < n) {
              if (j < w) c0 = cfma(pj[i2], f[j], c0);
              if (j + 1 < w) c1 = cfma(pk[i2], f[j + 1], c1);
            }
          }
          ck[i] = csub(ck[i], cadd(a0, a1));
          if (i2 < n) ck[i2] = csub(ck[i2], cadd(c0, c1));
        }
      }
      if (!T.sync()) return false;
    }
  }
  return T.sync();
}

// x <- L^{-1} x for one column x (stride 1) by the calling warp, in blocks of 32 rows: the
// diagonal block is solved in registers (lane l holds row b0 + l, values pass by shuffles), then the
// rows below are updated by a block product whose loads are all independent.  rd: 1 / L[i][i].
template <class S>
__device__ __forceinline__ void forward_subst(const S* __restrict__ L, const double* __restrict__ rd,
                                              int ld, int n, S* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int bn = min(32, n - b0);
    S xl = lane < bn ? x[b0 + lane] : mk<S>(0.0, 0.0);
    const double rl = lane < bn ? rd[b0 + lane] : 0.0;
    for (int i = 0; i < bn; ++i) {
      if (lane == i) xl = cscale(xl, rl);
      const S xi = shfl_c(xl, i);
      if (lane > i && lane < bn) xl = cfms(L[(size_t)(b0 + i) * ld + b0 + lane], xi, xl);
    }
    if (lane < bn) x[b0 + lane] = xl;
    // rows below, two 32-row blocks per pass and two partial sums per row (four independent
    // accumulation chains per lane; every broadcast x_i serves both blocks)
    for (int r0 = b0 + bn; r0 < n; r0 += 64) {
      const int r = r0 + lane, r2 = r + 32;
      S a0 = mk<S>(0.0, 0.0), a1 = a0, c0 = a0, c1 = a0;
      int i = 0;
      for (; i + 1 < bn; i += 2) {
        const S xi = shfl_c(xl, i), xj = shfl_c(xl, i + 1);
        const S* li = L + (size_t)(b0 + i) * ld;
        const S* lj = li + ld;
        if (r < n) {
          a0 = cfma(li[r], xi, a0);
          a1 = cfma(lj[r], xj, a1);
        }
        if (r2 < n) {
          c0 = cfma(li[r2], xi, c0);
          c1 = cfma(lj[r2], xj, c1);
        }
      }
      if (i < bn) {
        const S xi = shfl_c(xl, i);
        const S* li = L + (size_t)(b0 + i) * ld;
        if (r < n) a0 = cfma(li[r], xi, a0);
        if (r2 < n) c0 = cfma(li[r2], xi, c0);
      }
      if (r < n) x[r] = csub(x[r], cadd(a0, a1));
      if (r2 < n) x[r2] = csub(x[r2], cadd(c0, c1));
    }
  }
}

// x <- L^{-H} x for one column x by the calling warp, in blocks of 32 rows from the bottom: the
// diagonal block of L^H is solved in registers, then the rows above are updated (lane i reads the
// contiguous segment L[b0..b1), i] of column i).
template <class S>
__device__ __forceinline__ void backward_subst_h(const S* __restrict__ L, const double* __restrict__ rd,
                                                 int ld, int n, S* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int b1 = n; b1 > 0; b1 -= 32) {
    const int b0 = max(0, b1 - 32), bn = b1 - b0;
    S xl = lane < bn ? x[b0 + lane] : mk<S>(0.0, 0.0);
    const double rl = lane < bn ? rd[b0 + lane] : 0.0;
    for (int i = bn - 1; i >= 0; --i) {
      if (lane == i) xl = cscale(xl, rl);
      const S xi = shfl_c(xl, i);
      if (lane < i) xl = csub(xl, cmulc(L[(size_t)(b0 + lane) * ld + b0 + i], xi));
    }
    if (lane < bn) x[b0 + lane] = xl;
    // rows above, two 32-row blocks per pass and two partial sums per row
    for (int r0 = 0; r0 < b0; r0 += 64) {
      const int r = r0 + lane, r2 = r + 32;
      S a0 = mk<S>(0.0, 0.0), a1 = a0, c0 = a0, c1 = a0;
      const S* lr = L + (size_t)r * ld + b0;
      const S* lr2 = lr + (size_t)32 * ld;
      int t = 0;
      for (; t + 1 < bn; t += 2) {
        const S xt = shfl_c(xl, t), xu = shfl_c(xl, t + 1);
        if (r < b0) {
          a0 = cfmac(lr[t], xt, a0);
          a1 = cfmac(lr[t + 1], xu, a1);
        }
        if (r2 < b0) {
          c0 = cfmac(lr2[t], xt, c0);
          c1 = cfmac(lr2[t + 1], xu, c1);
        }
      }
      if (t < bn) {
        const S xt = shfl_c(xl, t);
        if (r < b0) a0 = cfmac(lr[t], xt, a0);
        if (r2 < b0) c0 = cfmac(lr2[t], xt, c0);
      }
      if (r < b0) x[r] = csub(x[r], cadd(a0, a1));
      if (r2 < b0) x[r2] = csub(x[r2], cadd(c0, c1));
    }
  }
}

// ---- phase 2: C = L^{-1} A L^{-H} ---------------------------------------------------------------
template <class Team, class S>
__device__ bool reduce_standard(const Team& T, const Pencil<S>& P) {
  const int n = P.n, la = P.lda;
  S* A = P.A;
  S* R = P.R;
  const int lane = threadIdx.x & 31;
  // full Hermitian A from its lower triangle
  for (int i = T.swrank(); i < n; i += T.wsize()) {
    S* ci = A + (size_t)i * la;
    for (int j = lane; j < i; j += 32) ci[j] = conjd(A[i + (size_t)j * la]);
    if (lane == 0) ci[i] = mk<S>(re(ci[i]), 0.0);
  }
  if (!T.sync()) return false;
  // X = L^{-1} A, column by column, in place in A
  for (int c = T.swrank(); c < n; c += T.wsize()) forward_subst(P.B, vrdiag(P), P.ldb, n, A + (size_t)c * la);
  if (!T.sync()) return false;
  // R = X^H
  for (int r = T.swrank(); r < n; r += T.wsize()) {
    S* cr = R + (size_t)r * n;
    for (int c = lane; c < n; c += 32) cr[c] = conjd(A[r + (size_t)c * la]);
  }
  if (!T.sync()) return false;
  // C = L^{-1} X^H = L^{-1} A L^{-H}, in place in R
  for (int c = T.swrank(); c < n; c += T.wsize()) forward_subst(P.B, vrdiag(P), P.ldb, n, R + (size_t)c * n);
  if (!T.sync()) return false;
  // A = C, made exactly Hermitian (lower triangle kept, upper = its conjugate, real diagonal)
  for (int c = T.swrank(); c < n; c += T.wsize()) {
    S* ac = A + (size_t)c * la;
    for (int r = lane; r < n; r += 32) {
      S v;
      if (r > c) v = R[r + (size_t)c * n];
      else if (r < c) v = conjd(R[c + (size_t)r * n]);
      else v = mk<S>(re(R[c + (size_t)c * n]), 0.0);
      ac[r] = v;
    }
  }
  return T.sync();
}

// ---- phase 3: Householder tridiagonalisation ------------------------------------------------------
// vec layout: d[n], e[n], tau[2n] (n words of S), p[4n] (2 n words of S: p of two consecutive
// steps), 1/L_jj[n], e^2[n], FP32 d and e^2[n]
template <class S>
__device__ __forceinline__ double* vd(const Pencil<S>& P) { return P.vec; }
template <class S>
__device__ __forceinline__ double* ve(const Pencil<S>& P) { return P.vec + P.n; }
template <class S>
__device__ __forceinline__ S* vtau(const Pencil<S>& P) { return reinterpret_cast<S*>(P.vec + 2 * P.n); }
template <class S>
__device__ __forceinline__ S* vp(const Pencil<S>& P) { return reinterpret_cast<S*>(P.vec + 4 * P.n); }
template <class S>
__device__ __forceinline__ double* ve2(const Pencil<S>& P) { return P.vec + 9 * P.n; }   // e^2
template <class S>
__device__ __forceinline__ float* vd32(const Pencil<S>& P) { return reinterpret_cast<float*>(P.vec + 10 * P.n); }
template <class S>
__device__ __forceinline__ float* ve232(const Pencil<S>& P) { return vd32(P) + P.n; }   // e^2 in FP32

// Sum over the CTA (every thread passes a value; every thread gets the same total, reduced in a
// fixed order so that all CTAs of a grid team obtain bit-identical results).
template <class S>
__device__ __forceinline__ S cta_sum_c(S v) {
  __shared__ S red[kWarps];
  v = warp_sum_c(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  // second level: the kWarps warp totals in every group of kWarps lanes, a butterfly within the
  // group (every lane ends with the same value: each level adds the same two operands, in either
  // order); the launch has kThreads threads
  S s = red[threadIdx.x & (kWarps - 1)];
#pragma unroll
  for (int o = kWarps / 2; o > 0; o >>= 1) s = cadd(s, shfl_xor_c(s, o));
  return s;
}

// Reflector j from x = column j of the updated matrix, rows j+1..n-1, staged in sx[j+1..n-1] by the
// whole CTA: beta = -sign(Re x_0) |x| (the real subdiagonal e_j), tau = (beta - x_0) / beta and
// v = x / (x_0 - beta) with v_{j+1} = 1, left in sx.  Every CTA of a grid team computes it the same
// way (fixed-order sums); the writer CTA also stores e_j, tau_j and v (column j of R).
template <class S>
__device__ S cta_reflector(const Pencil<S>& P, int j, S* sx, bool writer) {
  __shared__ S s_tau, s_vs;
  const int n = P.n, tid = threadIdx.x;
  __syncthreads();  // sx was staged by other threads
  double s = 0.0;
  for (int i = j + 2 + tid; i < n; i += blockDim.x) s = abs2_acc(sx[i], s);
  s = cta_sum_c(s);  // (its barriers also publish sx)
  if (tid == 0) {
    const S alpha = sx[j + 1];
    double beta;
    S tj = mk<S>(0.0, 0.0), vs = mk<S>(0.0, 0.0);
    if (s == 0.0 && im(alpha) == 0.0) {
      beta = re(alpha);  // nothing to annihilate: H = I
    } else {
      const double an = sqrt(abs2_acc(alpha, s));
      beta = re(alpha) >= 0.0 ? -an : an;
      const double rb = 1.0 / beta;
      tj = mk<S>((beta - re(alpha)) * rb, -im(alpha) * rb);
      vs = cinv(csub(alpha, mk<S>(beta, 0.0)));  // v_i = x_i / (alpha - beta)
    }
    s_tau = tj;
    s_vs = vs;
    if (writer) {
      ve(P)[j] = beta;
      vtau(P)[j] = tj;
    }
  }
  __syncthreads();
  const S vs = s_vs, tj = s_tau;
  S* __restrict__ rj = P.R + (size_t)j * n;
  for (int i = j + 1 + tid; i < n; i += blockDim.x) {
    const S v = i == j + 1 ? mk<S>(1.0, 0.0) : cmul(sx[i], vs);
    sx[i] = v;
    if (writer) rj[i] = v;
  }
  __syncthreads();
  return tj;
}

// One team barrier per column.  Step j applies reflector j (v_j, tau_j, and p_j = tau_j C v_j from
// the previous step) to the trailing matrix: gamma = -(tau_j / 2) p_j^H v_j, w = p_j + gamma v_j,
// C <- C - v w^H - w v^H.  Every CTA forms column j+1 of the updated matrix and reflector j+1 from
// it in shared memory (the same values in every CTA), then each warp updates its columns k >= j+2
// and, in the same pass over the column, accumulates p_{j+1}[k] = tau_{j+1} (column k)^H v_{j+1}
// (C is Hermitian, so that is row k of C v_{j+1}).  Rows < j+2 of those columns are never read
// again and are not updated.  p of consecutive steps alternate between two buffers, so that a
// CTA still reading p_j never meets the p_{j+1} that faster CTAs write.
// sbuf: 3 n words of S of shared memory per CTA (v_j, w and v_{j+1}, indexed by row).
template <class Team, class S>
__device__ bool tridiagonalise(const Team& T, const Pencil<S>& P, S* sbuf) {
  const int n = P.n, la = P.lda;
  S* A = P.A;
  const int tid = threadIdx.x, lane = tid & 31;
  const bool writer = T.rank() < (int)blockDim.x;  // the first CTA writes d, e, tau and R
  if (n == 1) {
    if (T.rank() == 0) vd(P)[0] = re(A[0]);
    return T.sync();
  }
  S* sv = sbuf;
  S* sw = sbuf + n;
  S* sn = sbuf + 2 * n;
  // reflector 0 from column 0, and p_0 = tau_0 C v_0 (rows 1..n-1)
  for (int i = 1 + tid; i < n; i += blockDim.x) sv[i] = A[i];
  if (writer && tid == 0) vd(P)[0] = re(A[0]);
  S tau = cta_reflector(P, 0, sv, writer);
  {
    S* __restrict__ p0 = vp(P);
    for (int k = 1 + T.swrank(); k < n; k += T.wsize()) {
      const S* __restrict__ ck = A + (size_t)k * la;
      S acc = mk<S>(0.0, 0.0);
      for (int i = 1 + lane; i < n; i += 32) acc = cfmac(ck[i], sv[i], acc);
      acc = warp_sum_c(acc);
      if (lane == 0) p0[k] = cmul(tau, acc);
    }
  }
  if (!T.sync()) return false;
  for (int j = 0; j <= n - 2; ++j) {
    const S* __restrict__ pj = vp(P) + (size_t)(j & 1) * n;
    S* __restrict__ pn = vp(P) + (size_t)((j + 1) & 1) * n;
    // p_j and column j+1 of C are read together (one round trip to L2), staged raw in sw and sn;
    // then w = p_j + gamma v_j and column j+1 of the updated matrix, x - v conj(w_{j+1}) - w (the
    // entry of v_j in row j+1 is 1), each thread on its own rows
    const S* __restrict__ c1 = A + (size_t)(j + 1) * la;
    S g = mk<S>(0.0, 0.0);
    for (int i = j + 1 + tid; i < n; i += blockDim.x) {
      const S pi = pj[i];
      sn[i] = c1[i];
      sw[i] = pi;
      g = cfmac(pi, sv[i], g);
    }
    g = cta_sum_c(g);
    const S gamma = cscale(cmul(tau, g), -0.5);
    const S cw1 = conjd(cadd(pj[j + 1], gamma));
    for (int i = j + 1 + tid; i < n; i += blockDim.x) {
      const S wi = cfma(gamma, sv[i], sw[i]);
      const S x = csub(cfms(sv[i], cw1, sn[i]), wi);
      sw[i] = wi;
      sn[i] = x;
      if (i == j + 1 && writer) vd(P)[j + 1] = re(x);
    }
    if (j + 1 <= n - 2) {
      const S tn = cta_reflector(P, j + 1, sn, writer);
      // columns k >= j+2: rank-2 update of rows j+2..n-1 fused with p_{j+1}[k]
      for (int k = j + 2 + T.swrank(); k < n; k += T.wsize()) {
        const S cvk = conjd(sv[k]), cwk = conjd(sw[k]);
        S* __restrict__ ck = A + (size_t)k * la;
        S acc = mk<S>(0.0, 0.0), acc2 = acc;  // two partial sums: shorter dependent chains
        int i = j + 2 + lane;
        for (; i + 96 < n; i += 128) {
          S a[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = ck[i + 32 * u];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = i + 32 * u;
            a[u] = cfms(sw[r], cvk, cfms(sv[r], cwk, a[u]));
            ck[r] = a[u];
            if (u & 1) acc2 = cfmac(a[u], sn[r], acc2);
            else acc = cfmac(a[u], sn[r], acc);
          }
        }
        for (; i < n; i += 32) {
          const S a = cfms(sw[i], cvk, cfms(sv[i], cwk, ck[i]));
          ck[i] = a;
          acc = cfmac(a, sn[i], acc);
        }
        acc = warp_sum_c(cadd(acc, acc2));
        if (lane == 0) pn[k] = cmul(tn, acc);
      }
      tau = tn;
    }
    if (!T.sync()) return false;
    S* t = sv;  // v_{j+1} becomes the current reflector
    sv = sn;
    sn = t;
  }
  return true;
}

// ---- phase 4: eigenpairs of the symmetric tridiagonal T (d, e) -----------------------------------
// Number of eigenvalues of T below s, from the signs of the leading principal minors p_i of
// T - s I (a Sturm sequence): p_0 = 1, p_1 = d_0 - s, p_{i+1} = (d_i - s) p_i - e_{i-1}^2 p_{i-1};
// the count is the number of sign changes between consecutive minors, i.e. of negative pivots
// p_{i+1} / p_i of the LDL^T factorisation (Sylvester's law of inertia).  Division-free: one fused
// multiply-add per row on the dependent chain (an FP64 division has about seven times the latency
// of a fused multiply-add on GB300, where that latency is already 64 cycles).  The pair
// (p_i, p_{i+1}) is rescaled by an exact power of two when p_{i+1} leaves [2^-600, 2^600]; an
// exactly zero minor is replaced by -2^-600 times the previous one (a tiny negative pivot, the
// guard of the pivot form), which also carries the sequence across a split (e_i = 0).  e2 = e^2.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// |x| as an integer: ordered like |x| for all non-NaN doubles
__device__ __forceinline__ unsigned long long dmag(double x) {
  return (unsigned long long)dbits(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double s) {
  double pm = 1.0, p = d[0] - s;
  if (((unsigned long long)dbits(p) << 1) == 0) p = -0x1p-600;
  int c = (int)((unsigned long long)dbits(p) >> 63);
  for (int i = 1; i < n; ++i) {
    double pn = fma(d[i] - s, p, -e2[i - 1] * pm);
    if (((unsigned long long)dbits(pn) << 1) == 0) pn = -0x1p-600 * p;
    c += (int)((unsigned long long)(dbits(pn) ^ dbits(p)) >> 63);
    pm = p;
    p = pn;
    const int ex = (int)((dbits(p) >> 52) & 0x7FF);  // biased exponent of |p|
    if (ex > 1023 + 600) {
      p *= 0x1p-600;
      pm *= 0x1p-600;
    } else if (ex < 1023 - 600 && (int)((dbits(pm) >> 52) & 0x7FF) < 1023 + 400) {
      p *= 0x1p+600;
      pm *= 0x1p+600;
    }
  }
  return c;
}
// The same count in FP32 (about 64 times cheaper on GB300), used only to narrow the bracket.
__device__ __forceinline__ int sturm_count32(const float* __restrict__ d, const float* __restrict__ e2, int n,
                                             float s, float pivmin) {
  int c = 0;
  float q = d[0] - s;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - s) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// Deterministic start vector entry in (-1, 1) for eigenvector k, row i.
__device__ __forceinline__ double start_entry(int k, int i) {
  unsigned h = (unsigned)k * 0x9E3779B1u ^ ((unsigned)i + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return ((double)(h >> 8) + 0.5) * (2.0 / 16777216.0) - 1.0;
}

template <class Team, class S>
__device__ bool tridiagonal_eig(const Team& T, const Pencil<S>& P) {
  const int n = P.n;
  const double* d = vd(P);
  const double* e = ve(P);
  double* e2 = ve2(P);
  float* d32 = vd32(P);
  float* e232 = ve232(P);
  double* w = P.w;
  for (int i = T.rank(); i < n; i += T.size()) {
    const double ei = i < n - 1 ? e[i] : 0.0;
    e2[i] = ei * ei;
    d32[i] = (float)d[i];
    e232[i] = (float)(ei * ei);
  }
  // norms and Gershgorin interval (every thread computes them the same way)
  double tn = 0.0, glo = 0.0, gu = 0.0, emax2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    tn = fmax(tn, fabs(d[i]) + r);
    glo = i ? fmin(glo, d[i] - r) : d[i] - r;
    gu = i ? fmax(gu, d[i] + r) : d[i] + r;
    if (i < n - 1) emax2 = fmax(emax2, e[i] * e[i]);
  }
  const double eps = 2.220446049250313e-16;
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax2);
  tn = fmax(tn, 1e-300);
  glo -= 2.0 * eps * tn + 2.0 * pivmin;
  gu += 2.0 * eps * tn + 2.0 * pivmin;
  if (!T.sync()) return false;
  // Eigenvalue k by multisection, one group of kSect lanes per eigenvalue (32 / kSect eigenvalues
  // per warp, kSect = 8, 16 or 32): in every round the group's lanes count at kSect interior points of the bracket
  // [lo, hi] (count(lo) <= k < count(hi)) and the bracket shrinks to the 1/(kSect+1) between the
  // last point below eigenvalue k and the first above it.  The bracket is first narrowed with FP32
  // counts (about 64 times cheaper than FP64 on GB300) to 1e-6 |T|, widened by 2e-6 |T| and
  // accepted only if the FP64 counts at both ends confirm it (else the Gershgorin interval is
  // used); FP64 rounds then take it to 2 eps |lambda|.  The rounds are a sequence of dependent
  // Sturm counts, so the lane groups trade a few times more FP64 work than plain bisection for a
  // sequence about three times shorter.
  const float pivmin32 = 1e-30f * (float)fmax(1.0, emax2);
  const int lane = threadIdx.x & 31;
  // lanes per eigenvalue: a 32-section shrinks the bracket by 33 per round, an 8-section by 9, at
  // four times the Sturm counts per round; wider sections pay while they keep the busy warps at
  // no more than half of the team's (beyond that the FP64 pipe, not the chain, is the limit)
  const int kSect = T.wsize() >= 2 * n ? 32 : T.wsize() >= n ? 16 : 8;
  const int kGroups = 32 / kSect;
  if (T.wsize() * kGroups >= n) {
    const int grp = lane / kSect, gi = lane % kSect;
    const unsigned gmask = kSect == 32 ? 0xffffffffu : ((1u << kSect) - 1u) << (grp * kSect);
    for (int k0 = T.swrank() * kGroups; k0 < n; k0 += T.wsize() * kGroups) {
      const int k = k0 + grp;
      const bool act = k < n;
      float l32 = (float)glo, h32 = (float)gu;
      const float wid = (float)(1e-6 * tn);
      bool open = act;
      for (int it = 0; it < 16; ++it) {
        open = open && h32 - l32 > wid;
        if (!__any_sync(0xffffffffu, open)) break;
        const float step = (h32 - l32) * (1.0f / (float)(kSect + 1));
        const float pt = l32 + (float)(gi + 1) * step;
        const bool above = open && pt < h32 && sturm_count32(d32, e232, n, pt, pivmin32) > k;
        const unsigned bits = (__ballot_sync(0xffffffffu, above) & gmask) >> (grp * kSect);
        const int f = bits ? __ffs(bits) - 1 : kSect;
        if (open) {
          const float nl = f == 0 ? l32 : l32 + (float)f * step;
          const float nh = f == kSect ? h32 : l32 + (float)(f + 1) * step;
          if (nh > nl) {
            l32 = nl;
            h32 = fminf(nh, h32);
          } else {
            open = false;
          }
        }
      }
      double lo = fmax(glo, (double)l32 - 2e-6 * tn), hi = fmin(gu, (double)h32 + 2e-6 * tn);
      {
        const int c = !act ? 0 : gi == 0 ? sturm_count(d, e2, n, lo) : (gi == 1 ? sturm_count(d, e2, n, hi) : 0);
        const int c0 = __shfl_sync(0xffffffffu, c, grp * kSect), c1 = __shfl_sync(0xffffffffu, c, grp * kSect + 1);
        if (!(c0 <= k && c1 > k)) {
          lo = glo;
          hi = gu;
        }
      }
      open = act;
      for (int it = 0; it < 64; ++it) {
        open = open && !(hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + pivmin);
        if (!__any_sync(0xffffffffu, open)) break;
        const double step = (hi - lo) * (1.0 / (double)(kSect + 1));
        const double pt = lo + (double)(gi + 1) * step;
        const bool above = open && pt < hi && sturm_count(d, e2, n, pt) > k;
        const unsigned bits = (__ballot_sync(0xffffffffu, above) & gmask) >> (grp * kSect);
        const int f = bits ? __ffs(bits) - 1 : kSect;
        if (open) {
          const double nl = f == 0 ? lo : lo + (double)f * step;
          const double nh = f == kSect ? hi : lo + (double)(f + 1) * step;
          if (!(nh > nl) || (nl == lo && nh >= hi)) {
            open = false;
          } else {
            lo = nl;
            hi = fmin(nh, hi);
          }
        }
      }
      if (act && gi == 0) w[k] = 0.5 * (lo + hi);
    }
  } else {
    // fewer warps than eigenvalues (one CTA per pencil): plain bisection, one thread per
    // eigenvalue, with the same FP32 narrowing and FP64 confirmation of the bracket
    for (int k = T.srank(); k < n; k += T.size()) {
      float l32 = (float)glo, h32 = (float)gu;
      const float wid = (float)(1e-5 * tn);
      for (int it = 0; it < 64 && h32 - l32 > wid; ++it) {
        const float mid = 0.5f * (l32 + h32);
        if (mid <= l32 || mid >= h32) break;
        if (sturm_count32(d32, e232, n, mid, pivmin32) > k) h32 = mid;
        else l32 = mid;
      }
      double lo = fmax(glo, (double)l32 - 1e-5 * tn), hi = fmin(gu, (double)h32 + 1e-5 * tn);
      if (!(sturm_count(d, e2, n, lo) <= k && sturm_count(d, e2, n, hi) > k)) {
        lo = glo;
        hi = gu;
      }
      for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + pivmin || mid <= lo || mid >= hi) break;
        if (sturm_count(d, e2, n, mid) > k) hi = mid;
        else lo = mid;
      }
      w[k] = 0.5 * (lo + hi);
    }
  }
  if (!T.sync()) return false;
  T.stamp(4);
  // eigenvectors by inverse iteration, one cluster per thread
  const double ortol = 1e-5 * tn;
  const double tiny = eps * tn;
  const size_t nn = (size_t)n * n;
  // (separate input and output arrays in every sweep, so that the loads of later rows can be
  // issued ahead of the dependent arithmetic)
  double* __restrict__ ua = P.wk;           // reciprocals of U's diagonal
  double* __restrict__ ub = P.wk + nn;      // U first superdiagonal
  double* __restrict__ uc = P.wk + 2 * nn;  // U second superdiagonal (fill-in of row swaps)
  double* __restrict__ ml = P.wk + 3 * nn;  // multipliers
  double* __restrict__ sw = P.wk + 4 * nn;  // 1: rows i, i+1 swapped
  double* __restrict__ x = P.wk + 5 * nn;   // iterate
  double* __restrict__ y = P.wk + 6 * nn;   // L^{-1} P x
  // 32 consecutive eigenvalues per warp (the interleaved arrays are then read in full 256-byte
  // rows), the warps spread over the CTAs
  for (int k0 = T.swrank() * 32 + (threadIdx.x & 31); k0 < n; k0 += T.size()) {
    if (k0 > 0 && w[k0] - w[k0 - 1] <= ortol) continue;  // not the first of its cluster
    int k1 = k0 + 1;
    while (k1 < n && w[k1] - w[k1 - 1] <= ortol) ++k1;
    double sprev = 0.0;
    for (int m = k0; m < k1; ++m) {
      // slot m of the interleaved arrays: element i at [i * n + m]
      double s = w[m];
      const double pert = 10.0 * eps * fmax(fabs(s), tn);
      if (m > k0 && s - sprev < pert) s = sprev + pert;
      sprev = s;
      // factor T - s I = P L U with partial pivoting
      {
        double a = d[0] - s, b = n > 1 ? e[0] : 0.0;
        for (int i = 0; i < n - 1; ++i) {
          const double sub = e[i];
          const double nd = d[i + 1] - s;
          const double ns = i + 1 < n - 1 ? e[i + 1] : 0.0;
          const size_t o = (size_t)i * n + m;
          // ua holds the reciprocal pivot: one division per row, none in the solves; the pivot
          // choice compares magnitudes as integers (the FP64 compare would add 64 cycles a row)
          if (dmag(a) >= dmag(sub)) {
            if (dmag(a) == 0) a = tiny;
            const double r = 1.0 / a;
            const double l = sub * r;
            ua[o] = r;
            ub[o] = b;
            uc[o] = 0.0;
            ml[o] = l;
            sw[o] = 0.0;
            a = nd - l * b;
            b = ns;
          } else {
            const double r = 1.0 / sub;
            const double l = a * r;
            ua[o] = r;
            ub[o] = nd;
            uc[o] = ns;
            ml[o] = l;
            sw[o] = 1.0;
            a = b - l * nd;
            b = -l * ns;
          }
        }
        if (dmag(a) == 0) a = tiny;
        ua[(size_t)(n - 1) * n + m] = 1.0 / a;
      }
      for (int i = 0; i < n; ++i) x[(size_t)i * n + m] = start_entry(m, i);
      const int iters = (k1 - k0 > 1) ? 4 : 3;
      for (int it = 0; it < iters; ++it) {
        // forward: y = L^{-1} P x, the row operations of the factorisation (running row in a register)
        {
          double cur = x[m];
#pragma unroll 4
          for (int i = 0; i < n - 1; ++i) {
            const size_t o = (size_t)i * n + m;
            double nxt = x[o + n];
            if (dmag(sw[o]) != 0) {
              const double t = cur;
              cur = nxt;
              nxt = t;
            }
            y[o] = cur;
            cur = fma(-ml[o], cur, nxt);
          }
          y[(size_t)(n - 1) * n + m] = cur;
        }
        // backward: x = U^{-1} y (the two solved rows below in registers; the iterate and the rows
        // still to solve are scaled down together when it grows)
        {
          double x1 = 0.0, x2 = 0.0;
#pragma unroll 4
          for (int i = n - 1; i >= 0; --i) {
            const size_t o = (size_t)i * n + m;
            double v = y[o];
            if (i + 2 < n) v = fma(-uc[o], x2, v);
            if (i + 1 < n) v = fma(-ub[o], x1, v);
            v *= ua[o];
            x[o] = v;
            x2 = x1;
            x1 = v;
            if (dmag(v) > dmag(1e100)) {
              for (int r = 0; r < n; ++r) {
                x[(size_t)r * n + m] *= 1e-100;
                y[(size_t)r * n + m] *= 1e-100;
              }
              x1 *= 1e-100;
              x2 *= 1e-100;
            }
          }
        }
        // orthogonalise against the cluster's earlier vectors, then normalise
        for (int q = k0; q < m; ++q) {
          const double* zq = P.Z + (size_t)q * n;
          double s2 = 0.0;
          for (int i = 0; i < n; ++i) s2 += zq[i] * x[(size_t)i * n + m];
          for (int i = 0; i < n; ++i) x[(size_t)i * n + m] -= s2 * zq[i];
        }
        double n0 = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0;  // four independent chains
        int i = 0;
        for (; i + 3 < n; i += 4) {
          const double v0 = x[(size_t)i * n + m], v1 = x[(size_t)(i + 1) * n + m];
          const double v2 = x[(size_t)(i + 2) * n + m], v3 = x[(size_t)(i + 3) * n + m];
          n0 = fma(v0, v0, n0);
          n1 = fma(v1, v1, n1);
          n2 = fma(v2, v2, n2);
          n3 = fma(v3, v3, n3);
        }
        for (; i < n; ++i) {
          const double v = x[(size_t)i * n + m];
          n0 = fma(v, v, n0);
        }
        const double nrm = sqrt((n0 + n1) + (n2 + n3));
        const double r = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int i = 0; i < n; ++i) x[(size_t)i * n + m] *= r;
      }
      double* zm = P.Z + (size_t)m * n;
      for (int i = 0; i < n; ++i) zm[i] = x[(size_t)i * n + m];
    }
  }
  return T.sync();
}

// ---- phase 5: x = L^{-H} Q z ------------------------------------------------------------------
template <class Team, class S>
__device__ bool back_transform(const Team& T, const Pencil<S>& P, S* smem) {
  const int n = P.n;
  const int lane = threadIdx.x & 31;
  const S* tau = vtau(P);
  for (int c = T.swrank(); c < n; c += T.wsize()) {
    // The column is built in this warp's shared-memory slot when the launch provided one, else in
    // place in A's column c (A is free: the reflectors live in R, L in B).
    S* ac = P.A + (size_t)c * P.lda;
    S* vc = smem ? smem + (size_t)(threadIdx.x >> 5) * n : ac;
    const double* zc = P.Z + (size_t)c * n;
    for (int i = lane; i < n; i += 32) vc[i] = mk<S>(zc[i], 0.0);
    __syncwarp();
    // V = H_0 H_1 ... H_{n-2} Z: reflector j (rows j+1..n-1, stored in column j of R) applied last-first
    for (int j = n - 2; j >= 0; --j) {
      const S tj = tau[j];
      if (re(tj) == 0.0 && im(tj) == 0.0) continue;
      const S* __restrict__ rj = P.R + (size_t)j * n;
      const int r0 = j + 1 + ((lane - j - 1) & 31);
      S s = mk<S>(0.0, 0.0);
      for (int i = r0; i < n; i += 32) s = cfmac(rj[i], vc[i], s);
      s = cmul(tj, warp_sum_c(s));
      for (int i = r0; i < n; i += 32) vc[i] = cfms(rj[i], s, vc[i]);
    }
    __syncwarp();
    backward_subst_h(P.B, vrdiag(P), P.ldb, n, vc);
    __syncwarp();
    // into the caller's complex A (in place for a complex pencil: the same lane, the same element)
    double2* oc = P.outA + (size_t)c * P.ldoa;
    for (int i = lane; i < n; i += 32) oc[i] = widen(vc[i]);
    __syncwarp();
  }
  return T.sync();
}

template <class Team, class S>
__device__ void solve_pencil(const Team& T, const Pencil<S>& P) {
  extern __shared__ double2 dyn_smem[];
  S* smem = reinterpret_cast<S*>(dyn_smem);
  if (T.rank() == 0) *P.info = 0;
  if (P.n <= 0) return;
  T.stamp(0);
  if (!prepare(T, P)) return;
  if (!cholesky(T, P, smem)) return;
  T.stamp(1);
  if (!reduce_standard(T, P)) return;
  T.stamp(2);
  if (!tridiagonalise(T, P, smem)) return;
  T.stamp(3);
  if (!tridiagonal_eig(T, P)) return;
  T.stamp(5);
  if (!back_transform(T, P, P.smem_cols ? smem : nullptr)) return;
  finish(T, P);
  T.stamp(6);
}

template <class S>
__global__ void __launch_bounds__(kThreads, 2) hegv_grid_kernel(Pencil<S> P, Ctl* ctl, unsigned long long limit_ns) {
  GridTeam T{ctl, P.info, limit_ns};
  solve_pencil(T, P);
}

template <class S>
__global__ void __launch_bounds__(kThreads, 2) hegv_cta_kernel(const Pencil<S>* __restrict__ items, int count) {
  if ((int)blockIdx.x >= count) return;
  const Pencil<S> P = items[blockIdx.x];
  CtaTeam T;
  solve_pencil(T, P);
}

size_t pad32(size_t x) { return (x + 31) & ~(size_t)31; }

// Workspace doubles of one pencil, each array padded to 32 doubles: complex, R (complex n^2);
// real, the compact A, B and R (n^2 each); then Z (n^2), wk (7 n^2) and vec (11 n + 8).
size_t work_doubles(int n, bool real) {
  const size_t nn = (size_t)n * n;
  const size_t own = real ? 3 * pad32(nn) : pad32(2 * nn);
  return own + pad32(nn) + pad32(7 * nn) + pad32(11 * (size_t)n + 8);
}

template <class S>
Pencil<S> make_pencil(double2* A, int lda, double2* B, int ldb, double* w, int* info, int n, double* ws) {
  const size_t nn = (size_t)n * n;
  Pencil<S> P;
  P.w = w;
  P.info = info;
  P.n = n;
  P.outA = A;
  P.outB = B;
  P.ldoa = lda;
  P.ldob = ldb;
  double* rest;
  if constexpr (sizeof(S) == sizeof(double)) {  // real: compact copies in the workspace
    P.A = reinterpret_cast<S*>(ws);
    P.B = reinterpret_cast<S*>(ws + pad32(nn));
    P.R = reinterpret_cast<S*>(ws + 2 * pad32(nn));
    P.lda = P.ldb = n;
    rest = ws + 3 * pad32(nn);
  } else {
    P.A = reinterpret_cast<S*>(A);
    P.B = reinterpret_cast<S*>(B);
    P.lda = lda;
    P.ldb = ldb;
    P.R = reinterpret_cast<S*>(ws);
    rest = ws + pad32(2 * nn);
  }
  P.Z = rest;
  P.wk = P.Z + pad32(nn);
  P.vec = P.wk + pad32(7 * nn);
  P.smem_cols = 0;
  return P;
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per grid-barrier wait
constexpr int kGridMinN = 32;  // a single pencil at least this large runs on a cooperative grid

// Dynamic shared memory: 3 n words of S for the tridiagonalisation's v_j, w and v_{j+1}, and, when
// it fits in 200 KB, one column of n words of S per warp for the back-transformation.
size_t col_smem_bytes(int n, size_t ws) {
  const size_t b = (size_t)kWarps * (size_t)std::max(n, 1) * ws;
  return b <= 200u * 1024u ? b : 0;
}
size_t dyn_smem_bytes(int n, size_t ws) {
  const size_t chol = ws == 8 ? chol_smem<double>() : chol_smem<double2>();
  return std::max({col_smem_bytes(n, ws), (size_t)3 * std::max(n, 1) * ws, chol});
}
constexpr int kMaxN = 4608;  // 3 n complex words must fit in shared memory (221 KB)

template <class S>
void launch_cta(kss_ctx ctx, std::vector<Pencil<S>>& small, size_t items_offset, const char* name) {
  if (small.empty()) return;
  // largest pencils first: the CTAs start in launch order, so the long solves begin on their own
  // SMs and the short ones fill in behind them (each CTA reads its own self-contained item)
  std::stable_sort(small.begin(), small.end(), [](const Pencil<S>& a, const Pencil<S>& b) { return a.n > b.n; });
  cudaStream_t st = ctx->stream;
  int nmax = 1;
  for (const auto& P : small) nmax = std::max(nmax, P.n);
  const size_t sm = dyn_smem_bytes(nmax, sizeof(S));
  for (auto& P : small) P.smem_cols = col_smem_bytes(nmax, sizeof(S)) ? 1 : 0;
  Pencil<S>* d_items = reinterpret_cast<Pencil<S>*>(static_cast<char*>(ctx->dense_items.p) + items_offset);
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_items, small.data(), small.size() * sizeof(Pencil<S>), cudaMemcpyHostToDevice, st));
  KSS_CHECK_CUDA(cudaFuncSetAttribute(hegv_cta_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  ProfScope ps(ctx, prof_register(name));
  hegv_cta_kernel<S><<<(unsigned)small.size(), kThreads, sm, st>>>(d_items, (int)small.size());
  KSS_CHECK_CUDA(cudaGetLastError());
}

template <class S>
void launch_grid(kss_ctx ctx, Pencil<S> P, const char* name) {
  cudaStream_t st = ctx->stream;
  const int n = P.n;
  const size_t sm = dyn_smem_bytes(n, sizeof(S));
  KSS_CHECK_CUDA(cudaFuncSetAttribute(hegv_grid_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  KSS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hegv_grid_kernel<S>, kThreads, sm));
  const int coop = std::max(1, per_sm) * std::max(1, ctx->nsm);
  const int G = std::max(1, std::min({(n + 3) / 4, ctx->nsm > 0 ? ctx->nsm : 1, coop}));
  ctx->dense_ctl.ensure(sizeof(Ctl));
  KSS_CHECK_CUDA(cudaMemsetAsync(ctx->dense_ctl.p, 0, sizeof(Ctl), st));
  P.smem_cols = col_smem_bytes(n, sizeof(S)) ? 1 : 0;
  Ctl* ctl = ctx->dense_ctl.as<Ctl>();
  unsigned long long lim = kWaitLimitNs;
  void* args[] = {&P, &ctl, &lim};
  ProfScope ps(ctx, prof_register(name));
  KSS_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)hegv_grid_kernel<S>, dim3(G), dim3(kThreads), args, sm, st));
}

}  // namespace

void hegv_batched(kss_ctx ctx, const std::vector<HegvItem>& items) {
  if (items.empty()) return;
  size_t total = 0;
  for (const auto& it : items) total += work_doubles(std::max(it.n, 1), it.real);
  ctx->dense_ws.ensure(total * sizeof(double));
  // one CTA per pencil, real and complex pencils in separate launches; a single large pencil on a
  // cooperative grid
  std::vector<Pencil<double>> small_r;
  std::vector<Pencil<double2>> small_c;
  double* p = ctx->dense_ws.as<double>();
  const bool alone = items.size() == 1;
  for (const auto& it : items) {
    KSS_REQUIRE(it.n >= 0 && it.lda >= std::max(it.n, 1) && it.ldb >= std::max(it.n, 1), "hegv: bad sizes");
    KSS_REQUIRE(it.n <= kMaxN, "hegv: order above " + std::to_string(kMaxN));
    double2* A = (double2*)it.A;
    double2* B = (double2*)it.B;
    const bool large = alone && it.n >= kGridMinN;
    if (it.real) {
      const Pencil<double> P = make_pencil<double>(A, it.lda, B, it.ldb, it.w, it.info, it.n, p);
      if (large) launch_grid(ctx, P, "dense_hegv_grid_real");
      else small_r.push_back(P);
    } else {
      const Pencil<double2> P = make_pencil<double2>(A, it.lda, B, it.ldb, it.w, it.info, it.n, p);
      if (large) launch_grid(ctx, P, "dense_hegv_grid");
      else small_c.push_back(P);
    }
    p += work_doubles(std::max(it.n, 1), it.real);
  }
  const size_t off_c = (small_r.size() * sizeof(Pencil<double>) + 255) & ~(size_t)255;
  ctx->dense_items.ensure(off_c + small_c.size() * sizeof(Pencil<double2>) + 1);
  launch_cta(ctx, small_r, 0, "dense_hegv_cta_real");
  launch_cta(ctx, small_c, off_c, "dense_hegv_cta");
}

void hegv(kss_ctx ctx, int n, void* A, int lda, void* B, int ldb, double* w, int* info, bool real) {
  hegv_batched(ctx, {HegvItem{A, B, w, info, n, lda, ldb, real}});
}

}  // namespace kss

using namespace kss;

extern "C" kss_status kss_dense_hegv(kss_ctx ctx, int count, const int* n, void* const* A, const int* lda,
                                     void* const* B, const int* ldb, double* const* w, int* info, int real) {
  if (!ctx) return KSS_EINVAL;
  try {
    KSS_REQUIRE(count >= 0, "count < 0");
    if (count == 0) {
      ctx->err.clear();
      return KSS_OK;
    }
    KSS_REQUIRE(n && A && lda && B && ldb && w && info, "NULL argument");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    std::vector<HegvItem> items(count);
    DevBuf dinfo;
    dinfo.alloc((size_t)count * sizeof(int));
    for (int i = 0; i < count; ++i) {
      KSS_REQUIRE(n[i] >= 0 && lda[i] >= std::max(1, n[i]) && ldb[i] >= std::max(1, n[i]), "bad order or leading dimension");
      KSS_REQUIRE(n[i] == 0 || (A[i] && B[i] && w[i]), "NULL matrix");
      items[i] = HegvItem{A[i], B[i], w[i], dinfo.as<int>() + i, n[i], lda[i], ldb[i], real != 0};
    }
    hegv_batched(ctx, items);
    KSS_CHECK_CUDA(cudaMemcpyAsync(info, dinfo.p, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    KSS_CHECK_CUDA(cudaGetLastError());
    for (int i = 0; i < count; ++i)
      if (info[i] < 0) fail(KSS_ETIMEOUT, "kss_dense_hegv: a bounded grid-barrier wait gave up");
    ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    ctx->err = e.msg;
    return e.st;
  } catch (...) {
    ctx->err = "unexpected internal error";
    return KSS_ECUDA;
  }
}

extern "C" kss_status kss_dense_hegv_phase_ms(kss_ctx ctx, double* ms) {
  if (!ctx || !ms) return KSS_EINVAL;
  try {
    for (int k = 0; k < 6; ++k) ms[k] = 0.0;
    if (!ctx->dense_ctl.p) {
      ctx->err.clear();
      return KSS_OK;
    }
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    Ctl c;
    KSS_CHECK_CUDA(cudaMemcpyAsync(&c, ctx->dense_ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    if (c.t[6] > c.t[0])
      for (int k = 0; k < 6; ++k) ms[k] = c.t[k + 1] > c.t[k] ? 1e-6 * (double)(c.t[k + 1] - c.t[k]) : 0.0;
    ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    ctx->err = e.msg;
    return e.st;
  }
}

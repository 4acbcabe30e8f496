// Chebyshev-filtered subspace iteration with Rayleigh-Ritz (§5.1: spectral filtering keeps the
// number of Rayleigh-Ritz calls low and spends the time in H applications).
//
// One iteration on the block X (npw x nb, orthonormal Ritz vectors with Ritz values lambda):
//   bounds   a = lambda_max(block), lambda_lo = lambda_min(block), b = rigorous upper bound of H
//   filter   scaled Chebyshev three-term recurrence of degree m on [a, b] (each term one fused
//            H application, the recurrence folded into the application's epilogue)
//   HY       one more H application on the filtered block Y
//   RR       S = Y^H Y and H_s = Y^H (HY) on the GPU, then the FP64 generalised Hermitian
//            eigensolve H_s q = lambda S q (Cholesky factorisation of S, reduction, eigensolve)
//            on the GPU; X = Y Q, HX = (HY) Q.  Because Q^H S Q = I this is Cholesky
//            orthonormalisation of Y followed by Rayleigh-Ritz, with the Y L^{-H} product folded
//            into the rotation.
//   resid    r_n = |HX_n - lambda_n X_n|_2 (FP64 accumulation), copied to the host.
// Mixed precision keeps the blocks, the filter and the rotations in complex64; S and H_s are
// promoted to FP64 for the eigensolve; a converged FP32 subspace is finished by one FP64
// H application and an FP64 Rayleigh-Ritz (Ritz values are quadratically accurate in the
// subspace error), whose eigenvalues and residuals are what the solver returns.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>

#include "kss_internal.h"

namespace kss {

namespace {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (g, band, 0, 0), key = seed.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double u01_sym(uint32_t v) {  // uniform in (-1, 1)
  return ((double)(v >> 8) + 0.5) * (2.0 / 16777216.0) - 1.0;
}

template <typename C>
__global__ void random_kernel(C* X, int npw, int nb, long long ld, uint2 key, int band0) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)npw * nb) return;
  const int g = (int)(idx % npw), n = (int)(idx / npw);
  const uint4 r = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)(band0 + n), 0u, 0u), key);
  C v;
  v.x = u01_sym(r.x);
  v.y = u01_sym(r.y);
  X[(size_t)n * ld + g] = v;
}

template <typename C>
__global__ void residual_kernel(const C* __restrict__ X, const C* __restrict__ HX, int npw,
                                long long ld, const double* __restrict__ w, double* __restrict__ r) {
  __shared__ double red[256];
  const int n = blockIdx.x;
  const double lam = w[n];
  const C* x = X + (size_t)n * ld;
  const C* h = HX + (size_t)n * ld;
  double s = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double dr = (double)h[g].x - lam * (double)x[g].x;
    const double di = (double)h[g].y - lam * (double)x[g].y;
    s += dr * dr + di * di;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) r[n] = sqrt(red[0]);
}

// Gamma point: c(G) <- (c(G) + conj c(-G)) / 2 for every band (the component at G = 0 made real);
// the thread of the smaller index of each pair writes both.
template <typename C>
__global__ void gamma_symmetrize(C* X, const int* __restrict__ mirror, int npw, int nb, long long ld) {
  const long long n = (long long)npw * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / npw), g = (int)(i - (long long)b * npw);
    const int m = mirror[g];
    C* x = X + (size_t)b * ld;
    if (g < m) {
      const C p = x[g], q = x[m];
      C r;
      r.x = (p.x + q.x) * 0.5f;
      r.y = (p.y - q.y) * 0.5f;
      x[g] = r;
      r.y = -r.y;
      x[m] = r;
    } else if (g == m) {
      x[g].y = 0;
    }
  }
}

__global__ void real_part(const double2* __restrict__ in, double* __restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i].x;
}
__global__ void real_to_complex(const double* __restrict__ in, double2* __restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2(in[i], 0.0);
}

__global__ void c64_to_c128(const float2* __restrict__ in, double2* __restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2(in[i].x, in[i].y);
}
__global__ void c128_to_c64(const double2* __restrict__ in, float2* __restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// Block copy between band-major layouts with independent leading dimensions (and precisions).
template <typename Ci, typename Co>
__global__ void copy_block(const Ci* __restrict__ in, long long ldi, Co* __restrict__ out, long long ldo,
                           int npw, int nb) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)npw * nb) return;
  const int g = (int)(idx % npw), n = (int)(idx / npw);
  const Ci v = in[(size_t)n * ldi + g];
  Co o;
  o.x = v.x;
  o.y = v.y;
  out[(size_t)n * ldo + g] = o;
}

unsigned blocks_for(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Helper contexts: same device and settings, own non-blocking stream, own workspaces and
// dense-eigensolver workspace, so that work issued on them can run beside the context stream's.
kss_ctx aux_ctx(kss_ctx ctx, int i) {
  while ((int)ctx->aux.size() <= i) {
    std::unique_ptr<kss_ctx_s> w(new kss_ctx_s());
    w->device = ctx->device;
    w->nsm = ctx->nsm;
    w->autotune = ctx->autotune;
    cudaStream_t st = nullptr;
    KSS_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    w->stream = st;
    w->own_stream = true;
    ctx->aux.push_back(w.release());
  }
  return ctx->aux[i];
}

void aux_release(kss_ctx ctx) {
  prof_fold(ctx);
  for (kss_ctx w : ctx->aux) {
    cudaStreamSynchronize(w->stream);
    prof_release(w);
    cudaStreamDestroy(w->stream);
    delete w;
  }
  ctx->aux.clear();
}

void random_block(kss_ctx ctx, bool fp64, void* X, int npw, int nb, int ld, uint64_t seed,
                  int band0) {
  const long long n = (long long)npw * nb;
  if (!n) return;
  cudaStream_t st = ctx->stream;
  static const int id = prof_register("random_block");
  ProfScope ps(ctx, id);
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  if (fp64) random_kernel<double2><<<blocks_for(n), 256, 0, st>>>((double2*)X, npw, nb, ld, key, band0);
  else random_kernel<float2><<<blocks_for(n), 256, 0, st>>>((float2*)X, npw, nb, ld, key, band0);
  KSS_CHECK_CUDA(cudaGetLastError());
}

void residual_norms(kss_ctx ctx, bool fp64, const void* X, const void* HX, int npw, int nb, int ld,
                    const double* w, double* r) {
  cudaStream_t st = ctx->stream;
  static const int id = prof_register("residual_norms");
  ProfScope ps(ctx, id);
  if (fp64) residual_kernel<double2><<<nb, 256, 0, st>>>((const double2*)X, (const double2*)HX, npw, ld, w, r);
  else residual_kernel<float2><<<nb, 256, 0, st>>>((const float2*)X, (const float2*)HX, npw, ld, w, r);
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace kss

using namespace kss;

kss_solver_s::~kss_solver_s() {
  if (hpin) cudaFreeHost(hpin);
}

namespace kss {
double max_wanted(const kss_solver_s* s) {
  double m = 0;
  for (int n = 0; n < s->nband; ++n) m = std::max(m, s->resid[n]);
  return m;
}
}  // namespace kss

namespace {

size_t esize(bool f64) { return f64 ? 16 : 8; }

// FP64 generalised eigensolve of (Hs, S) in place: Hs <- Q with Q^H S Q = I, W <- eigenvalues,
// info <- status.  At Gamma the pencil of real-space-real blocks is real symmetric and is solved
// as such: a real rotation Q keeps the rotated bands real in real space (a complex eigensolver
// may return each eigenvector with an arbitrary complex phase).
void subspace_eig(kss_solver_s* s, kss_ctx ctx) {
  hegv(ctx, s->nb, s->Hs.p, s->nb, s->S.p, s->nb, s->W.as<double>(), s->info.as<int>(), s->gamma);
}

}  // namespace

namespace kss {

// Rayleigh-Ritz on (Y, HY) -> (Xo, HXo): everything is queued on the stream; eigenvalues,
// residuals and the eigensolver status land in pinned host memory (read by rr_finish).
void rr_issue(kss_solver_s* s, bool f64, const void* Y, const void* HY, void* Xo, void* HXo,
              kss_ctx on) {
  kss_ctx ctx = on ? on : s->sys->ctx;
  const int nb = s->nb, npw = s->npw;
  const long long nn = (long long)nb * nb;
  // With an overlap the metric is Y^H S Y (S Y kept in sb, later overwritten by S X).
  const bool gen = s->sys->has_S;
  DevBuf& sb = (f64 && !s->f64) ? s->sblk64 : s->sblk;
  const void* MY = Y;
  if (gen) {
    sb.ensure((size_t)npw * nb * (f64 ? 16 : 8));
    apply_s(ctx, s->sys, s->ik, nb, Y, sb.p, npw, f64 ? KSS_PREC_FP64 : KSS_PREC_MIXED);
    MY = sb.p;
  }
  // The generalised eigensolve reads the lower triangles of S and Hs only: the Gram products
  // compute the tiles on and below the diagonal (about half the work) and zero the rest.
  if (f64) {
    // FP64 Gram matrices on the tensor cores (FP64-accurate digit products, full matrices)
    oz_gemm_cn(ctx, nb, nb, npw, Y, npw, MY, npw, s->S.p, nb, 1, 0, 0, 0, "gram");
    oz_gemm_cn(ctx, nb, nb, npw, Y, npw, HY, npw, s->Hs.p, nb, 1, 0, 0, 0, "gram");
  } else if (s->gram64) {
    gemm_cn_c64_acc64_lower(ctx, nb, npw, Y, npw, MY, npw, s->S.p, nb, "gram");
    gemm_cn_c64_acc64_lower(ctx, nb, npw, Y, npw, HY, npw, s->Hs.p, nb, "gram");
  } else {
    // Gram matrices of the complex64 block on the tensor cores: exact products of the FP32 values
    // (4 digits each), summed exactly per chunk and in FP64 across chunks, delivered in FP64
    oz_gemm_cn(ctx, nb, nb, npw, Y, npw, MY, npw, s->S.p, nb, 1, 0, 0, 0, "gram", nullptr, false, true);
    oz_gemm_cn(ctx, nb, nb, npw, Y, npw, HY, npw, s->Hs.p, nb, 1, 0, 0, 0, "gram", nullptr, false, true);
  }
  subspace_eig(s, ctx);  // real symmetric at Gamma (real-space-real blocks)
  if (f64) {
    oz_gemm_nn(ctx, npw, nb, nb, Y, npw, s->Hs.p, nb, Xo, npw, 1, 0, 0, 0, "rotate");
    oz_gemm_nn(ctx, npw, nb, nb, HY, npw, s->Hs.p, nb, HXo, npw, 1, 0, 0, 0, "rotate");
  } else {
    {
      static const int idq = prof_register("convert_c128_c64");
      ProfScope ps(ctx, idq);
      c128_to_c64<<<blocks_for(nn), 256, 0, ctx->stream>>>(s->Hs.as<double2>(), s->Q32.as<float2>(), nn);
    }
    // complex64 rotations on the FP32 pipe: the filtered block's columns span up to 2^12 in scale,
    // which digit products would have to cover with 7 digits per value (measured slower here)
    gemm_nn(ctx, false, npw, nb, nb, Y, npw, s->Q32.p, nb, Xo, npw, 1, 0, 0, 0, "rotate");
    gemm_nn(ctx, false, npw, nb, nb, HY, npw, s->Q32.p, nb, HXo, npw, 1, 0, 0, 0, "rotate");
  }
  // residuals |H x - lambda S x| (S x = x without an overlap)
  if (gen) apply_s(ctx, s->sys, s->ik, nb, Xo, sb.p, npw, f64 ? KSS_PREC_FP64 : KSS_PREC_MIXED);
  residual_norms(ctx, f64, gen ? sb.p : Xo, HXo, npw, nb, npw, s->W.as<double>(), s->resid_d.as<double>());
  if (!s->hpin) {
    KSS_CHECK_CUDA(cudaMallocHost((void**)&s->hpin, (2 * (size_t)nb + 1) * sizeof(double)));
  }
  KSS_CHECK_CUDA(cudaMemcpyAsync(s->hpin, s->W.p, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KSS_CHECK_CUDA(cudaMemcpyAsync(s->hpin + nb, s->resid_d.p, nb * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KSS_CHECK_CUDA(cudaMemcpyAsync(s->hpin + 2 * nb, s->info.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KSS_CHECK_CUDA(cudaGetLastError());
}

// rr_finish; in mixed precision a failed Cholesky of the FP32-accumulated Gram matrix (a
// numerically rank-deficient filtered block) is retried once with FP64 accumulation, and the
// solver keeps FP64 accumulation from then on.  Y and HY are untouched by the first attempt.
void rr_finish_or_retry(kss_solver_s* s, bool f64, const void* Y, const void* HY, void* Xo, void* HXo) {
  try {
    rr_finish(s);
  } catch (const KssError& e) {
    if (e.st != KSS_ENUMERIC || f64 || s->gram64) throw;
    s->gram64 = true;
    rr_issue(s, f64, Y, HY, Xo, HXo);
    KSS_CHECK_CUDA(cudaStreamSynchronize(s->sys->ctx->stream));
    KSS_CHECK_CUDA(cudaGetLastError());
    rr_finish(s);
  }
}

void rr_finish(kss_solver_s* s) {
  const int nb = s->nb;
  int info = 0;
  std::memcpy(&info, s->hpin + 2 * nb, sizeof(int));
  s->evals.assign(s->hpin, s->hpin + nb);
  s->resid.assign(s->hpin + nb, s->hpin + 2 * nb);
  if (info < 0) fail(KSS_ETIMEOUT, "subspace eigensolve: a bounded grid-barrier wait gave up");
  if (info != 0)
    fail(KSS_ENUMERIC, "subspace eigensolve failed (info = " + std::to_string(info) +
                           "): the Gram matrix is not numerically positive definite");
  for (int n = 0; n < nb; ++n)
    if (!std::isfinite(s->evals[n]) || !std::isfinite(s->resid[n]))
      fail(KSS_ENUMERIC, "non-finite Ritz value or residual");
}

}  // namespace kss

namespace {

void rayleigh_ritz(kss_solver_s* s, bool f64, const void* Y, const void* HY, void* Xo, void* HXo) {
  rr_issue(s, f64, Y, HY, Xo, HXo);
  KSS_CHECK_CUDA(cudaStreamSynchronize(s->sys->ctx->stream));
  KSS_CHECK_CUDA(cudaGetLastError());
  rr_finish_or_retry(s, f64, Y, HY, Xo, HXo);
}

// Gamma point: re-project X and H X onto real-space-real bands after every Rayleigh-Ritz.  The
// packed local part returns exactly symmetric output, but the nonlocal products and the
// recurrence carry the rounding-level asymmetry of their inputs forward and the filter amplifies
// it (about 5x per iteration); without the projection it reaches the residual level and stalls
// convergence.
void gamma_fix(kss_solver_s* s, bool f64, void* X, void* HX) {
  if (!s->gamma) return;
  kss_ctx ctx = s->sys->ctx;
  const long long n = (long long)s->npw * s->nb;
  const unsigned bl = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32);
  const int* mir = s->sys->k[s->ik].d_mirror.as<int>();
  for (void* b : {X, HX}) {
    if (f64) gamma_symmetrize<double2><<<bl, 256, 0, ctx->stream>>>((double2*)b, mir, s->npw, s->nb, s->npw);
    else gamma_symmetrize<float2><<<bl, 256, 0, ctx->stream>>>((float2*)b, mir, s->npw, s->nb, s->npw);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

void apply_block(kss_solver_s* s, bool f64, const void* psi, void* out) {
  apply_h(s->sys, s->ik, s->nb, psi, nullptr, out, s->npw, ChebCoef{1, 0, 0, s->gamma, s->proj32},
          f64 ? KSS_PREC_FP64 : KSS_PREC_MIXED);
  s->napply += s->nb;
}

}  // namespace

namespace kss {
ChebParams cheb_params(const kss_solver_s* s) {
  const int nb = s->nb;
  const double lam_lo = s->evals[0];
  double a = s->evals[nb - 1];
  const double b = s->sys->k[s->ik].bound_f;  // bound of the filter operator (H or S^-1 H)
  if (!(b - a > 1e-3 * (b - lam_lo))) a = lam_lo + 0.5 * (b - lam_lo);
  ChebParams p;
  p.e = 0.5 * (b - a);
  p.c = 0.5 * (b + a);
  p.sigma1 = p.e / (lam_lo - p.c);
  p.degree = s->o.degree;
  if (!s->f64) {
    // The scaled filter amplifies the lowest Ritz direction by T_m(|x_lo|) relative to the top of
    // the block, x_lo = (lambda_lo - c) / e.  A complex64 block resolves about seven digits, so in
    // mixed precision the degree is capped to keep that ratio below 2^12 and leave the top
    // columns about twelve significant bits.
    const double xl = std::fabs((lam_lo - p.c) / p.e);
    if (xl > 1.0) {
      const int m = (int)std::floor(std::acosh(4096.0) / std::acosh(xl));
      p.degree = std::max(2, std::min(p.degree, m));
    }
  }
  return p;
}
}  // namespace kss

namespace {

// Scaled Chebyshev filter of degree m on X (in blk[ix]); returns the buffer holding Y_m and, in
// *prev_out, the buffer holding Y_{m-1} (free for reuse).
int chebyshev_filter(kss_solver_s* s, int f1, int* prev_out) {
  const int nb = s->nb;
  const ChebParams cp = cheb_params(s);
  const double e = cp.e, c = cp.c;
  const double sigma1 = cp.sigma1;
  const double tau = 2.0 / sigma1;
  const kss_precision p = s->f64 ? KSS_PREC_FP64 : KSS_PREC_MIXED;
  int cur = s->ix, prev = f1;
  // Y_1 = (sigma1/e)(H - c) X
  {
    const double al = sigma1 / e;
    apply_filter_op(s->sys, s->ik, nb, s->blk[cur].p, nullptr, s->blk[prev].p, s->npw,
                    ChebCoef{al, -al * c, 0.0, s->gamma, s->proj32}, p);
    s->napply += nb;
    std::swap(cur, prev);  // cur = Y_1, prev = X
  }
  double sigma = sigma1;
  const int m = cp.degree;
  for (int j = 2; j <= m; ++j) {
    const double sn = 1.0 / (tau - sigma);
    const double al = 2.0 * sn / e;
    // Y_j = (2 sn / e)(H - c) Y_{j-1} - sigma sn Y_{j-2}, written over Y_{j-2}
    apply_filter_op(s->sys, s->ik, nb, s->blk[cur].p, s->blk[prev].p, s->blk[prev].p, s->npw,
                    ChebCoef{al, -al * c, -sigma * sn, s->gamma, s->proj32}, p);
    s->napply += nb;
    std::swap(cur, prev);
    sigma = sn;
  }
  *prev_out = prev;
  return cur;
}

}  // namespace

namespace kss {
void refine_fp64(kss_solver_s* s) {
  kss_ctx ctx = s->sys->ctx;
  const size_t bytes = (size_t)s->npw * s->nb * 16;
  for (int i = 0; i < 4; ++i) s->r64[i].ensure(bytes);
  const long long n = (long long)s->npw * s->nb;
  static const int idp = prof_register("copy_block");
  {
    ProfScope ps(ctx, idp);
    copy_block<float2, double2><<<blocks_for(n), 256, 0, ctx->stream>>>(
        s->blk[s->ix].as<float2>(), s->npw, s->r64[0].as<double2>(), s->npw, s->npw, s->nb);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
  apply_block(s, true, s->r64[0].p, s->r64[1].p);
  rayleigh_ritz(s, true, s->r64[0].p, s->r64[1].p, s->r64[2].p, s->r64[3].p);
  // Keep the refined vectors as the current iterate (demoted to complex64).
  {
    ProfScope ps(ctx, idp);
    copy_block<double2, float2><<<blocks_for(n), 256, 0, ctx->stream>>>(
        s->r64[2].as<double2>(), s->npw, s->blk[s->ix].as<float2>(), s->npw, s->npw, s->nb);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}
}  // namespace kss

namespace {

void after_iterate(kss_solver_s* s);

void solver_step(kss_solver_s* s) {
  kss_ctx ctx = s->sys->ctx;
  const auto t0 = std::chrono::steady_clock::now();
  if (!s->started) {
    {
      KSS_NVTX("apply_H");
      apply_block(s, s->f64, s->blk[0].p, s->blk[1].p);
    }
    const auto t1 = std::chrono::steady_clock::now();
    {
      KSS_NVTX("rayleigh_ritz");
      rayleigh_ritz(s, s->f64, s->blk[0].p, s->blk[1].p, s->blk[2].p, s->blk[3].p);
      gamma_fix(s, s->f64, s->blk[2].p, s->blk[3].p);
    }
    s->ix = 2;
    s->ihx = 3;
    s->started = true;
    s->ms_rr += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  } else {
    int fr[2], nf = 0;
    for (int i = 0; i < 4; ++i)
      if (i != s->ix && i != s->ihx) fr[nf++] = i;
    int prev = -1, y = -1;
    {
      KSS_NVTX("filter");
      y = chebyshev_filter(s, fr[0], &prev);
      // y and prev are two of {ix, fr[0]}; the HY block reuses prev.
      apply_block(s, s->f64, s->blk[y].p, s->blk[prev].p);
      KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    const auto t1 = std::chrono::steady_clock::now();
    s->ms_filter += std::chrono::duration<double, std::milli>(t1 - t0).count();
    {
      KSS_NVTX("rayleigh_ritz");
      rayleigh_ritz(s, s->f64, s->blk[y].p, s->blk[prev].p, s->blk[fr[1]].p, s->blk[s->ihx].p);
      gamma_fix(s, s->f64, s->blk[fr[1]].p, s->blk[s->ihx].p);
    }
    s->ix = fr[1];
    s->iter += 1;
    s->ms_rr += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
  }
  after_iterate(s);
  s->ms_total += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Convergence bookkeeping after a Rayleigh-Ritz (and the FP64 refinement that ends a mixed solve).
void after_iterate(kss_solver_s* s) {
  // A tensor-core projector product whose bounded wait gave up left wrong values behind.
  if (tc_error_flag(s->sys->ctx, true)) fail(KSS_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up");
  const double r = max_wanted(s);
  s->hist.push_back(r);
  if (s->f64) {
    s->converged = r <= s->tol;
    s->done = s->converged;
  } else {
    bool stalled = false;
    const size_t h = s->hist.size();
    // stalled at the single-precision floor: no 10% progress in three iterations near tol
    if (h >= 4) stalled = s->hist[h - 1] > 0.9 * s->hist[h - 4] && s->hist[h - 1] < 100.0 * s->tol;
    if (r <= s->tol || stalled || s->iter >= s->o.max_iter) {
      refine_fp64(s);
      s->converged = max_wanted(s) <= s->tol;
      // The split-BF16 projector products bound the residual the single-precision filter can
      // reach; a block that misses the tolerance in the FP64 check continues with FP32 products.
      if (!s->converged && !s->proj32 && s->sys->nproj && s->iter < s->o.max_iter) {
        s->proj32 = true;
        s->hist.clear();
        return;
      }
      s->done = true;
    }
  }
}

// One pipelined iteration of several solvers of one context: the filter of solver u+1 is queued
// on the context stream before the Rayleigh-Ritz of solver u is issued on a helper stream (the
// eigensolver may block the host until its input is ready, and the queued filter keeps the GPU
// busy meanwhile).  Every solver's blocks and the workspaces of each stream are disjoint; the
// context stream waits for the helpers before the results are read.
void step_many(kss_ctx ctx, const std::vector<kss_solver_s*>& us) {
  const auto t0 = std::chrono::steady_clock::now();
  const int n = (int)us.size();
  constexpr int kAux = 2;
  struct Roles { int y, prev, f1; };
  std::vector<Roles> ro(n);
  std::vector<cudaEvent_t> ev(n, nullptr);
  std::vector<cudaEvent_t> jev(kAux, nullptr);
  auto destroy = [&] {
    for (auto e : ev) if (e) cudaEventDestroy(e);
    for (auto e : jev) if (e) cudaEventDestroy(e);
  };
  try {
    auto filter = [&](int u) {
      kss_solver_s* s = us[u];
      int fr[2], nf = 0;
      for (int i = 0; i < 4; ++i)
        if (i != s->ix && i != s->ihx) fr[nf++] = i;
      KSS_NVTX("filter");
      int prev = -1;
      const int y = chebyshev_filter(s, fr[0], &prev);
      apply_block(s, s->f64, s->blk[y].p, s->blk[prev].p);
      ro[u] = Roles{y, prev, fr[1]};
      KSS_CHECK_CUDA(cudaEventCreateWithFlags(&ev[u], cudaEventDisableTiming));
      KSS_CHECK_CUDA(cudaEventRecord(ev[u], ctx->stream));
    };
    auto rr = [&](int u) {
      KSS_NVTX("rayleigh_ritz");
      kss_solver_s* s = us[u];
      kss_ctx w = aux_ctx(ctx, u % kAux);
      w->prof.on = ctx->prof.on;
      KSS_CHECK_CUDA(cudaStreamWaitEvent(w->stream, ev[u], 0));
      rr_issue(s, s->f64, s->blk[ro[u].y].p, s->blk[ro[u].prev].p, s->blk[ro[u].f1].p, s->blk[s->ihx].p, w);
    };
    if (n > 0) filter(0);
    for (int u = 0; u < n; ++u) {
      if (u + 1 < n) filter(u + 1);
      rr(u);
    }
    for (int i = 0; i < std::min(n, kAux); ++i) {
      KSS_CHECK_CUDA(cudaEventCreateWithFlags(&jev[i], cudaEventDisableTiming));
      KSS_CHECK_CUDA(cudaEventRecord(jev[i], ctx->aux[i]->stream));
      KSS_CHECK_CUDA(cudaStreamWaitEvent(ctx->stream, jev[i], 0));
    }
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    KSS_CHECK_CUDA(cudaGetLastError());
  } catch (...) {
    for (kss_ctx w : ctx->aux) cudaStreamSynchronize(w->stream);
    destroy();
    throw;
  }
  destroy();
  const double share =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() / std::max(n, 1);
  for (int u = 0; u < n; ++u) {
    kss_solver_s* s = us[u];
    const auto t1 = std::chrono::steady_clock::now();
    rr_finish_or_retry(s, s->f64, s->blk[ro[u].y].p, s->blk[ro[u].prev].p, s->blk[ro[u].f1].p, s->blk[s->ihx].p);
    gamma_fix(s, s->f64, s->blk[ro[u].f1].p, s->blk[s->ihx].p);
    s->ix = ro[u].f1;
    s->iter += 1;
    after_iterate(s);
    const double own = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count();
    s->ms_filter += 0.5 * share;
    s->ms_rr += 0.5 * share + own;
    s->ms_total += share + own;
  }
}

template <typename F>
kss_status guard(kss_ctx ctx, F&& f) {
  try {
    f();
    ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    ctx->err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return KSS_ENOMEM;
  } catch (...) {
    ctx->err = "unexpected internal error";
    return KSS_ECUDA;
  }
}

}  // namespace

extern "C" {

kss_status kss_solver_create(kss_sys sys, int ik, int nband, const kss_solve_opts* opts,
                             kss_solver* out) {
  if (!sys || !out) return KSS_EINVAL;
  kss_ctx ctx = sys->ctx;
  return guard(ctx, [&] {
    *out = nullptr;
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(nband >= 1, "nband must be >= 1");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    std::unique_ptr<kss_solver_s> s(new kss_solver_s());
    s->sys = sys;
    s->ik = ik;
    s->nband = nband;
    s->npw = sys->k[ik].npw;
    kss_solve_opts o{};
    if (opts) o = *opts;
    if (o.degree <= 0) o.degree = 10;
    if (o.max_iter <= 0) o.max_iter = 200;
    if (o.nbuffer < 0) o.nbuffer = std::max(4, (nband + 9) / 10);
    KSS_REQUIRE(o.prec == KSS_PREC_FP64 || o.prec == KSS_PREC_MIXED, "unknown precision");
    s->f64 = o.prec == KSS_PREC_FP64;
    // Default tolerances: 1e-8 Ha in FP64; in the mixed form twice the single-precision floor of
    // the residual, which grows with the spectral range (about 1e-6 of the upper bound of H:
    // complex64 carries ~7 digits of H x), and never below 1e-5 Ha.
    s->tol = o.tol > 0 ? o.tol : (s->f64 ? 1e-8 : std::max(1e-5, 2e-6 * std::fabs(sys->k[ik].bound_f)));
    s->nb = nband + o.nbuffer;
    KSS_REQUIRE(s->nb <= s->npw, "nband + nbuffer exceeds the number of plane waves");
    s->o = o;
    const size_t bytes = (size_t)s->npw * s->nb * esize(s->f64);
    for (int i = 0; i < 4; ++i) s->blk[i].alloc(bytes);
    const size_t nn = (size_t)s->nb * s->nb;
    s->S.alloc(nn * 16);
    s->Hs.alloc(nn * 16);
    s->W.alloc(s->nb * sizeof(double));
    s->resid_d.alloc(s->nb * sizeof(double));
    s->info.alloc(sizeof(int));
    if (!s->f64) {
      s->S32.alloc(nn * 8);
      s->Hs32.alloc(nn * 8);
      s->Q32.alloc(nn * 8);
    }
    int nx = 0;
    if (o.x0) {
      KSS_REQUIRE(o.x0_nb >= 0 && o.x0_nb <= s->nb && o.x0_ld >= s->npw, "bad x0_nb or x0_ld");
      nx = o.x0_nb;
      if (nx)
        KSS_CHECK_CUDA(cudaMemcpy2DAsync(s->blk[0].p, (size_t)s->npw * esize(s->f64), o.x0,
                                         (size_t)o.x0_ld * esize(s->f64), (size_t)s->npw * esize(s->f64),
                                         nx, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (nx < s->nb)
      random_block(ctx, s->f64, (char*)s->blk[0].p + (size_t)nx * s->npw * esize(s->f64), s->npw,
                   s->nb - nx, s->npw, o.seed, nx);
    s->gamma = sys->k[ik].gamma && !sys->has_S && !(o.flags & KSS_SOLVE_NO_GAMMA_REAL);
    if (s->gamma) {
      const long long n = (long long)s->npw * s->nb;
      const unsigned bl = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32);
      if (s->f64)
        gamma_symmetrize<double2><<<bl, 256, 0, ctx->stream>>>(s->blk[0].as<double2>(),
                                                               sys->k[ik].d_mirror.as<int>(), s->npw, s->nb, s->npw);
      else
        gamma_symmetrize<float2><<<bl, 256, 0, ctx->stream>>>(s->blk[0].as<float2>(),
                                                              sys->k[ik].d_mirror.as<int>(), s->npw, s->nb, s->npw);
      KSS_CHECK_CUDA(cudaGetLastError());
    }
    s->o.x0 = nullptr;  // copied; the caller's buffer is not referenced again
    sys->nsolvers += 1;
    *out = s.release();
  });
}

kss_status kss_solver_destroy(kss_solver s) {
  if (!s) return KSS_EINVAL;
  cudaSetDevice(s->sys->ctx->device);
  cudaStreamSynchronize(s->sys->ctx->stream);
  s->sys->nsolvers -= 1;
  delete s;
  return KSS_OK;
}

kss_status kss_solver_step(kss_solver s, int* converged) {
  if (!s) return KSS_EINVAL;
  kss_ctx ctx = s->sys->ctx;
  return guard(ctx, [&] {
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    if (!s->done) solver_step(s);
    if (converged) *converged = s->converged ? 1 : 0;
  });
}

kss_status kss_solver_step_many(int n, kss_solver const* solvers, int* converged) {
  if (n < 0 || (n > 0 && !solvers)) return KSS_EINVAL;
  if (n == 0) return KSS_OK;
  for (int u = 0; u < n; ++u)
    if (!solvers[u]) return KSS_EINVAL;
  kss_ctx ctx = solvers[0]->sys->ctx;
  for (int u = 1; u < n; ++u)
    if (solvers[u]->sys->ctx != ctx) {
      ctx->err = "kss_solver_step_many: the solvers belong to different contexts";
      return KSS_EINVAL;
    }
  return guard(ctx, [&] {
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    std::vector<kss_solver_s*> uniq, iter;
    for (int u = 0; u < n; ++u)
      if (std::find(uniq.begin(), uniq.end(), solvers[u]) == uniq.end()) uniq.push_back(solvers[u]);
    for (kss_solver_s* s : uniq) {
      if (s->done) continue;
      if (!s->started) solver_step(s);  // the initial Rayleigh-Ritz is this call's step
      else iter.push_back(s);
    }
    step_many(ctx, iter);
    if (converged)
      for (int u = 0; u < n; ++u) converged[u] = solvers[u]->converged ? 1 : 0;
  });
}

kss_status kss_solver_results(kss_solver s, double* evals, double* resid, void* evecs, int ld,
                              kss_solve_stats* stats) {
  if (!s) return KSS_EINVAL;
  kss_ctx ctx = s->sys->ctx;
  return guard(ctx, [&] {
    KSS_REQUIRE(s->started, "no iterate yet: call kss_solver_step first");
    if (evals) std::memcpy(evals, s->evals.data(), s->nband * sizeof(double));
    if (resid) std::memcpy(resid, s->resid.data(), s->nband * sizeof(double));
    if (evecs) {
      KSS_REQUIRE(ld >= s->npw, "ld < npw");
      const size_t es = esize(s->f64);
      KSS_CHECK_CUDA(cudaMemcpy2DAsync(evecs, (size_t)ld * es, s->blk[s->ix].p, (size_t)s->npw * es,
                                       (size_t)s->npw * es, s->nband, cudaMemcpyDeviceToDevice,
                                       ctx->stream));
      KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    if (stats) {
      stats->iters = s->iter;
      stats->napply = s->napply;
      stats->max_resid = max_wanted(s);
      stats->ms_filter = s->ms_filter;
      stats->ms_rr = s->ms_rr;
      stats->ms_total = s->ms_total;
      stats->nb = s->nb;
    }
  });
}

kss_status kss_chebfi_solve(kss_sys sys, int ik, int nband, const kss_solve_opts* opts,
                            double* evals, void* evecs, int ld, double* resid,
                            kss_solve_stats* stats) {
  if (!sys) return KSS_EINVAL;
  kss_solver s = nullptr;
  kss_status st = kss_solver_create(sys, ik, nband, opts, &s);
  if (st != KSS_OK) return st;
  int conv = 0;
  while (st == KSS_OK && !conv && !s->done && s->iter < s->o.max_iter) st = kss_solver_step(s, &conv);
  if (st == KSS_OK && !s->started) st = kss_solver_step(s, &conv);
  kss_status st2 = KSS_OK;
  if (s->started) st2 = kss_solver_results(s, evals, resid, evecs, ld, stats);
  std::string msg = sys->ctx->err;
  kss_solver_destroy(s);
  sys->ctx->err = msg;
  if (st != KSS_OK) return st;
  if (st2 != KSS_OK) return st2;
  if (!conv) {
    sys->ctx->err = "not converged within max_iter";
    return KSS_ENOCONV;
  }
  return KSS_OK;
}

}  // extern "C"

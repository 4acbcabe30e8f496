// The generalised eigenproblem H psi = lambda S psi with the nonlocal overlap
// S = 1 + sum_i |beta_i> q_i <beta_i| (§5.2: the nonlocal part of the overlap operator has the
// structure of Eq. ham-nl).  With the projector Gram matrix G = beta^H beta (nproj x nproj, per
// k-point) the push-through identity gives
//   S^-1 = 1 - beta W beta^H,   W = Q (1 + G Q)^-1,
// so that S^-1 costs two projector products.  For the Chebyshev filter the operator S^-1 H is
// applied as
//   C = beta^H psi;  L psi (the local part);  E = beta^H (L psi) + G (D C);
//   S^-1 H psi = L psi + beta (D C - W E)
// (three projector products per band block instead of two).
#include <cmath>
#include <complex>
#include <vector>

#include "kss_internal.h"

namespace kss {

namespace {

template <typename C, typename T>
__global__ void cheb_combine(const C* __restrict__ f, long long ldf, const C* __restrict__ psi,
                             const C* psi_prev, C* out, long long ld, int npw, int nb, T al, T be, T ga) {
  const long long n = (long long)npw * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / npw), g = (int)(i - (long long)b * npw);
    const C x = f[(size_t)b * ldf + g];
    const C p = psi[(size_t)b * ld + g];
    C o;
    o.x = al * x.x + be * p.x;
    o.y = al * x.y + be * p.y;
    if (psi_prev) {
      const C q = psi_prev[(size_t)b * ld + g];  // read before the write of the same element
      o.x += ga * q.x;
      o.y += ga * q.y;
    }
    out[(size_t)b * ld + g] = o;
  }
}

// Projector products at the precision of the path: FP64-accurate digit products or split-BF16
// products on the tensor cores (the same kernels as the H application).
void proj_cn(kss_ctx ctx, bool f64, kss_sys s, int ik, int nb, const void* psi, int ld, void* out,
             const char* tag) {
  const KData& kd = s->k[ik];
  const int nproj = s->nproj;
  if (f64)
    oz_gemm_cn(ctx, nproj, nb, kd.npw, kd.d_beta64.p, kd.npw, psi, ld, out, nproj, 1, 0, 0, 0, tag,
               &beta_oz_cn(s, ik));
  else
    tc_gemm_cn_split(ctx, nproj, nb, kd.npw, beta_split_cn(s, ik), psi, ld, out, nproj, 1, 0, 0, 0, tag);
}
void proj_nn(kss_ctx ctx, bool f64, kss_sys s, int ik, int nb, const void* coef, void* out, int ld,
             const char* tag) {
  const KData& kd = s->k[ik];
  const int nproj = s->nproj;
  if (f64)
    oz_gemm_nn(ctx, kd.npw, nb, nproj, kd.d_beta64.p, kd.npw, coef, nproj, out, ld, 1, 0, 1, 0, tag,
               &beta_oz_nn(s, ik));
  else
    tc_gemm_nn_split(ctx, kd.npw, nb, nproj, beta_split_nn(s, ik), coef, nproj, out, ld, 1, 0, 1, 0, tag);
}

unsigned grid_for(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 32));
}

}  // namespace

// Per-k overlap tables and the filter bound (called by kss_setup once the projector table of
// every k-point is on the device).  s_min >= 1 + min(0, min q) * g, g = the Gershgorin bound of
// the largest eigenvalue of G; the filter operator's spectrum lies below bound(H) / s_min.
void overlap_setup(kss_sys s) {
  kss_ctx ctx = s->ctx;
  const int np = s->nproj;
  double qmin = 0;
  for (double q : s->Q) qmin = std::min(qmin, q);
  for (auto& kd : s->k) {
    kd.bound_f = kd.bound;
    if (!s->has_S || np == 0) continue;
    DevBuf g64;
    g64.alloc((size_t)np * np * 16);
    gemm_cn(ctx, true, np, np, kd.npw, kd.d_beta64.p, kd.npw, kd.d_beta64.p, kd.npw, g64.p, np, 1, 0,
            0, 0, "overlap_gram");
    std::vector<std::complex<double>> G((size_t)np * np);
    KSS_CHECK_CUDA(cudaMemcpyAsync(G.data(), g64.p, G.size() * 16, cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    double gersh = 0;  // max row sum of |G_ij| bounds the largest eigenvalue of G
    for (int i = 0; i < np; ++i) {
      double r = 0;
      for (int j = 0; j < np; ++j) r += std::abs(G[(size_t)j * np + i]);
      gersh = std::max(gersh, r);
    }
    const double smin = 1.0 + qmin * gersh;
    KSS_REQUIRE(smin > 1e-6, "the overlap S = 1 + beta Q beta^H is not provably positive definite "
                             "(1 + min(q) * |G| <= 0)");
    kd.bound_f = kd.bound > 0 ? kd.bound / smin : kd.bound;
    // W = Q (1 + G Q)^-1 by Gauss-Jordan elimination with partial pivoting on [A | 1], A = 1 + G Q.
    std::vector<std::complex<double>> A((size_t)np * np), Inv((size_t)np * np, 0.0);
    for (int j = 0; j < np; ++j)
      for (int i = 0; i < np; ++i) A[(size_t)j * np + i] = G[(size_t)j * np + i] * s->Q[j] + (i == j ? 1.0 : 0.0);
    for (int i = 0; i < np; ++i) Inv[(size_t)i * np + i] = 1.0;
    auto at = [&](std::vector<std::complex<double>>& M, int i, int j) -> std::complex<double>& {
      return M[(size_t)j * np + i];
    };
    for (int c = 0; c < np; ++c) {
      int piv = c;
      for (int i = c + 1; i < np; ++i)
        if (std::abs(at(A, i, c)) > std::abs(at(A, piv, c))) piv = i;
      KSS_REQUIRE(std::abs(at(A, piv, c)) > 1e-300, "1 + G Q is singular");
      if (piv != c)
        for (int j = 0; j < np; ++j) {
          std::swap(at(A, c, j), at(A, piv, j));
          std::swap(at(Inv, c, j), at(Inv, piv, j));
        }
      const std::complex<double> d = 1.0 / at(A, c, c);
      for (int j = 0; j < np; ++j) {
        at(A, c, j) *= d;
        at(Inv, c, j) *= d;
      }
      for (int i = 0; i < np; ++i) {
        if (i == c) continue;
        const std::complex<double> f = at(A, i, c);
        if (f == 0.0) continue;
        for (int j = 0; j < np; ++j) {
          at(A, i, j) -= f * at(A, c, j);
          at(Inv, i, j) -= f * at(Inv, c, j);
        }
      }
    }
    std::vector<std::complex<double>> W((size_t)np * np);
    std::vector<std::complex<float>> W32((size_t)np * np), G32((size_t)np * np);
    for (int j = 0; j < np; ++j)
      for (int i = 0; i < np; ++i) {
        W[(size_t)j * np + i] = s->Q[i] * at(Inv, i, j);
        W32[(size_t)j * np + i] = std::complex<float>(W[(size_t)j * np + i]);
        G32[(size_t)j * np + i] = std::complex<float>(G[(size_t)j * np + i]);
      }
    kd.d_W64.alloc(W.size() * 16);
    kd.d_W32.alloc(W.size() * 8);
    kd.d_G64.alloc(G.size() * 16);
    kd.d_G32.alloc(G.size() * 8);
    KSS_CHECK_CUDA(cudaMemcpy(kd.d_W64.p, W.data(), W.size() * 16, cudaMemcpyHostToDevice));
    KSS_CHECK_CUDA(cudaMemcpy(kd.d_W32.p, W32.data(), W32.size() * 8, cudaMemcpyHostToDevice));
    KSS_CHECK_CUDA(cudaMemcpyAsync(kd.d_G64.p, g64.p, G.size() * 16, cudaMemcpyDeviceToDevice, ctx->stream));
    KSS_CHECK_CUDA(cudaMemcpy(kd.d_G32.p, G32.data(), G32.size() * 8, cudaMemcpyHostToDevice));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  }
}

// out = S psi = psi + beta (Q (beta^H psi)) on ctx's stream; psi and out must not overlap.
void apply_s(kss_ctx ctx, kss_sys s, int ik, int nb, const void* psi, void* out, int ld, kss_precision prec) {
  const KData& kd = s->k[ik];
  const bool f64 = prec == KSS_PREC_FP64;
  const size_t es = f64 ? 16 : 8;
  KSS_CHECK_CUDA(cudaMemcpy2DAsync(out, (size_t)ld * es, psi, (size_t)ld * es, (size_t)kd.npw * es, nb,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
  if (!s->has_S || s->nproj == 0 || nb == 0) return;
  ctx->ws_cprj.ensure((size_t)s->nproj * nb * es);
  proj_cn(ctx, f64, s, ik, nb, psi, ld, ctx->ws_cprj.p, "overlap_cprj");
  scale_rows(ctx, f64, s->nproj, nb, ctx->ws_cprj.p, s->nproj, f64 ? s->d_Q64.p : s->d_Q32.p, 1.0);
  proj_nn(ctx, f64, s, ik, nb, ctx->ws_cprj.p, out, ld, "overlap_nonlocal");
}

// out = alpha * F psi + beta * psi + gamma * psi_prev with the filter operator F = H, or S^-1 H
// for a system with an overlap.  psi_prev may alias out.
void apply_filter_op(kss_sys s, int ik, int nb, const void* psi, const void* psi_prev, void* out, int ld,
                     ChebCoef c, kss_precision prec) {
  if (!s->has_S || s->nproj == 0) {
    apply_h(s, ik, nb, psi, psi_prev, out, ld, c, prec);
    return;
  }
  KSS_REQUIRE(ik >= 0 && ik < (int)s->k.size(), "k-point index out of range");
  KSS_REQUIRE(nb >= 0, "nb < 0");
  const KData& kd = s->k[ik];
  KSS_REQUIRE(ld >= kd.npw, "ld < npw");
  if (nb == 0) return;
  KSS_REQUIRE(psi && out && psi != out, "null or overlapping psi / out");
  kss_ctx ctx = s->ctx;
  const bool f64 = prec == KSS_PREC_FP64;
  const size_t es = f64 ? 16 : 8;
  const int np = s->nproj;
  ctx->ws_sapply.ensure((size_t)nb * ld * es);
  ctx->ws_e.ensure((size_t)np * nb * es);
  ctx->ws_f.ensure((size_t)np * nb * es);
  void* lpsi = ctx->ws_sapply.p;
  // D C (kept in ws_f; apply_local uses ws_cprj for nothing)
  proj_cn(ctx, f64, s, ik, nb, psi, ld, ctx->ws_f.p, "cprj");
  scale_rows(ctx, f64, np, nb, ctx->ws_f.p, np, f64 ? s->d_D64.p : s->d_D32.p, 1.0);
  // L psi = T psi + V psi
  apply_local(s, ik, nb, psi, lpsi, ld, prec);
  // E = beta^H (L psi) + G (D C)
  proj_cn(ctx, f64, s, ik, nb, lpsi, ld, ctx->ws_e.p, "overlap_cprj");
  gemm_nn(ctx, f64, np, nb, np, f64 ? kd.d_G64.p : kd.d_G32.p, np, ctx->ws_f.p, np, ctx->ws_e.p, np, 1, 0, 1, 0,
          "overlap_small");
  // F = D C - W E
  gemm_nn(ctx, f64, np, nb, np, f64 ? kd.d_W64.p : kd.d_W32.p, np, ctx->ws_e.p, np, ctx->ws_f.p, np, -1, 0, 1, 0,
          "overlap_small");
  // S^-1 H psi = L psi + beta F
  proj_nn(ctx, f64, s, ik, nb, ctx->ws_f.p, lpsi, ld, "nonlocal");
  static const int idc = prof_register("cheb_combine");
  const long long n = (long long)kd.npw * nb;
  {
    ProfScope ps(ctx, idc);
    if (f64)
      cheb_combine<double2, double><<<grid_for(n), 256, 0, ctx->stream>>>(
          (const double2*)lpsi, ld, (const double2*)psi, (const double2*)psi_prev, (double2*)out, ld, kd.npw, nb,
          c.alpha, c.beta, c.gamma);
    else
      cheb_combine<float2, float><<<grid_for(n), 256, 0, ctx->stream>>>(
          (const float2*)lpsi, ld, (const float2*)psi, (const float2*)psi_prev, (float2*)out, ld, kd.npw, nb,
          (float)c.alpha, (float)c.beta, (float)c.gamma);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace kss

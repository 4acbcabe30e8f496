// LOBPCG, the paper's second GPU eigensolver (§5.1; Knyazev's locally optimal block
// preconditioned conjugate gradient, the blocked form of Bottin et al.): the lowest m = nband +
// nbuffer eigenpairs of H, FP64, one block.  Each iteration:
//   R = H X - X Lambda;  W = K R with the Teter-Payne-Allan preconditioner
//       K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4),  x = T_G / Ekin_n
//       (Ekin_n the kinetic energy of band n);
//   W and P orthogonalised against X and normalised band by band (a well-conditioned basis);
//   H W (the iteration's only H application);
//   Rayleigh-Ritz in span[X W P]: A = Z^H HZ, B = Z^H Z (lower-triangle blocks), FP64
//   generalised eigensolve, X <- Z C, HX <- HZ C, P <- [W P] C_wp, HP <- [HW HP] C_wp
// (the products H X, H P are carried along by linear combination, the "projections in memory"
// idea of §5.2: no H application for X or P).  If [X W P] is numerically dependent the
// iteration falls back to [X W].
#include <chrono>
#include <cmath>
#include <memory>
#include <vector>


#include "kss_internal.h"

namespace kss {
}

namespace kss {

namespace {

__global__ void band_ekin(const double2* __restrict__ X, const double* __restrict__ kin, int npw,
                          double* __restrict__ ek) {
  __shared__ double s_t[256], s_n[256];
  const double2* x = X + (size_t)blockIdx.x * npw;
  double t = 0, n = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double a = x[g].x * x[g].x + x[g].y * x[g].y;
    t += kin[g] * a;
    n += a;
  }
  s_t[threadIdx.x] = t;
  s_n[threadIdx.x] = n;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      s_t[threadIdx.x] += s_t[threadIdx.x + k];
      s_n[threadIdx.x] += s_n[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) ek[blockIdx.x] = s_n[0] > 0 ? s_t[0] / s_n[0] : 1.0;
}

// W = K(T_G / ek_n) (HX - lambda_n X)
__global__ void precond_resid(const double2* __restrict__ X, const double2* __restrict__ HX,
                              const double* __restrict__ kin, const double* __restrict__ lam,
                              const double* __restrict__ ek, int npw, int nb, double2* __restrict__ W) {
  const long long n = (long long)npw * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / npw), g = (int)(i - (long long)b * npw);
    const double x = kin[g] / fmax(ek[b], 1e-12);
    const double p = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
    const double k = p / (p + 16.0 * x * x * x * x);
    const double2 h = HX[i], v = X[i];
    W[i] = make_double2(k * (h.x - lam[b] * v.x), k * (h.y - lam[b] * v.y));
  }
}

// Scale band n of A (and of B, when given) by 1 / |A_n| (bands of zero norm are left as they are).
__global__ void normalize_bands(double2* __restrict__ A, double2* __restrict__ B, int npw) {
  __shared__ double red[256];
  double2* a = A + (size_t)blockIdx.x * npw;
  double s = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s += a[g].x * a[g].x + a[g].y * a[g].y;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  const double nrm = sqrt(red[0]);
  if (!(nrm > 0)) return;
  const double f = 1.0 / nrm;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    a[g].x *= f;
    a[g].y *= f;
  }
  if (B) {
    double2* b = B + (size_t)blockIdx.x * npw;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
      b[g].x *= f;
      b[g].y *= f;
    }
  }
}

// Per-band sums for RMM-DIIS, one block per band n, residuals formed on the fly as
// R_i = H psi_i - e_i psi_i:
//   mode 0: out[n] = Re <psi_a|H psi_a>, out[nb + n] = <psi_a|psi_a>           (Rayleigh quotient)
//   mode 1: out[n] = Re <R_a|R_b>                                               (DIIS matrix entry)
//   mode 2: out[n] = Re <(H - e_a) w|R_a>, out[nb + n] = |(H - e_a) w|^2 with w = c, Hw = d
//           (the optimal step length along w)
__global__ void band_sums(int mode, int npw, int nb, const double2* __restrict__ pa, const double2* __restrict__ ha,
                          const double* __restrict__ ea, const double2* __restrict__ pb,
                          const double2* __restrict__ hb, const double* __restrict__ eb,
                          const double2* __restrict__ c, const double2* __restrict__ d, double* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  const int n = blockIdx.x;
  const size_t o = (size_t)n * npw;
  double u = 0, v = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 x = pa[o + g], hx = ha[o + g];
    if (mode == 0) {
      u += x.x * hx.x + x.y * hx.y;
      v += x.x * x.x + x.y * x.y;
    } else if (mode == 1) {
      const double2 y = pb[o + g], hy = hb[o + g];
      const double rx = hx.x - ea[n] * x.x, ix = hx.y - ea[n] * x.y;
      const double ry = hy.x - eb[n] * y.x, iy = hy.y - eb[n] * y.y;
      u += rx * ry + ix * iy;
    } else {
      const double2 w = c[o + g], hw = d[o + g];
      const double tr = hw.x - ea[n] * w.x, ti = hw.y - ea[n] * w.y;
      const double rr = hx.x - ea[n] * x.x, ri = hx.y - ea[n] * x.y;
      u += tr * rr + ti * ri;
      v += tr * tr + ti * ti;
    }
  }
  s0[threadIdx.x] = u;
  s1[threadIdx.x] = v;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) {
      s0[threadIdx.x] += s0[threadIdx.x + k];
      s1[threadIdx.x] += s1[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[n] = s0[0];
    if (mode != 1) out[nb + n] = s1[0];
  }
}

// out_n = sum_{i < q} coef[n * q + i] * v_i,n  (q <= 4 vectors; out may alias none of them)
__global__ void band_combine(int q, int npw, int nb, const double2* __restrict__ v0, const double2* __restrict__ v1,
                             const double2* __restrict__ v2, const double2* __restrict__ v3,
                             const double* __restrict__ coef, double2* __restrict__ out) {
  const long long n = (long long)npw * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / npw);
    const double* c = coef + (size_t)b * q;
    double2 s = make_double2(c[0] * v0[i].x, c[0] * v0[i].y);
    if (q > 1) { s.x += c[1] * v1[i].x; s.y += c[1] * v1[i].y; }
    if (q > 2) { s.x += c[2] * v2[i].x; s.y += c[2] * v2[i].y; }
    if (q > 3) { s.x += c[3] * v3[i].x; s.y += c[3] * v3[i].y; }
    out[i] = s;
  }
}

unsigned grid_for(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 32));
}

struct Lobpcg {
  kss_sys sys = nullptr;
  kss_ctx ctx = nullptr;
  int ik = 0, nband = 0, m = 0, npw = 0;
  double tol = 1e-8;
  int max_iter = 500;
  DevBuf X, HX, W, HW, P, HP, T1, T2, T3, T4;
  DevBuf A, B, ev, info, lam, ek, resid, M;
  bool have_p = false;
  int iters = 0;
  long long napply = 0;
  std::vector<double> evals, res;

  double2* d(DevBuf& b) { return b.as<double2>(); }
  size_t blk() const { return (size_t)npw * m * 16; }

  void apply(const void* psi, void* out) {
    apply_h(sys, ik, m, psi, nullptr, out, npw, ChebCoef{1, 0, 0}, KSS_PREC_FP64);
    napply += m;
  }

  // Lower-triangle blocks of A = Z^H HZ and B = Z^H Z for Z = [Z_0 .. Z_q-1] (each npw x m).
  void gram(const std::vector<const void*>& Z, const std::vector<const void*>& HZ, int k) {
    const int q = (int)Z.size();
    // the strictly upper blocks are never written (the eigensolve reads the lower triangle)
    KSS_CHECK_CUDA(cudaMemsetAsync(A.p, 0, (size_t)k * k * 16, ctx->stream));
    KSS_CHECK_CUDA(cudaMemsetAsync(B.p, 0, (size_t)k * k * 16, ctx->stream));
    for (int i = 0; i < q; ++i)
      for (int j = 0; j <= i; ++j) {
        double2* a = d(A) + (size_t)j * m * k + (size_t)i * m;
        double2* b = d(B) + (size_t)j * m * k + (size_t)i * m;
        if (i == j) {
          gemm_cn_lower(ctx, true, m, npw, Z[i], npw, HZ[j], npw, a, k, "lobpcg_gram");
          gemm_cn_lower(ctx, true, m, npw, Z[i], npw, Z[j], npw, b, k, "lobpcg_gram");
        } else {
          gemm_cn(ctx, true, m, m, npw, Z[i], npw, HZ[j], npw, a, k, 1, 0, 0, 0, "lobpcg_gram");
          gemm_cn(ctx, true, m, m, npw, Z[i], npw, Z[j], npw, b, k, 1, 0, 0, 0, "lobpcg_gram");
        }
      }
  }

  // Generalised eigensolve of the k x k pencil (A, B); returns the status word (0 = success,
  // j + 1 = the metric is not positive definite at column j).
  int eig(int k) {
    hegv(ctx, k, A.p, k, B.p, k, ev.as<double>(), info.as<int>(), false);
    int inf = 0;
    KSS_CHECK_CUDA(cudaMemcpyAsync(&inf, info.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    if (inf < 0) fail(KSS_ETIMEOUT, "LOBPCG Rayleigh-Ritz: a bounded grid-barrier wait gave up");
    return inf;
  }

  // out = sum_i Z_i C_i with C_i the rows [i m, (i+1) m) of the first m eigenvector columns.
  void combine(const std::vector<const void*>& Z, int k, int first, void* out) {
    for (size_t i = first; i < Z.size(); ++i)
      gemm_nn(ctx, true, npw, m, m, Z[i], npw, d(A) + i * m, k, out, npw, 1, 0, i == (size_t)first ? 0 : 1, 0,
              "lobpcg_rotate");
  }

  // Rayleigh-Ritz in span(Z); false if the pencil is not numerically positive definite.
  bool rayleigh_ritz(const std::vector<const void*>& Z, const std::vector<const void*>& HZ) {
    const int k = (int)Z.size() * m;
    gram(Z, HZ, k);
    if (eig(k) != 0) return false;
    combine(Z, k, 0, T1.p);
    combine(HZ, k, 0, T2.p);
    if (Z.size() > 1) {
      combine(Z, k, 1, T3.p);   // P <- W C_w (+ P C_p)
      combine(HZ, k, 1, T4.p);
      std::swap(P, T3);
      std::swap(HP, T4);
      have_p = true;
    }
    std::swap(X, T1);
    std::swap(HX, T2);
    KSS_CHECK_CUDA(cudaMemcpyAsync(lam.p, ev.p, (size_t)m * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    residual_norms(ctx, true, X.p, HX.p, npw, m, npw, lam.as<double>(), resid.as<double>());
    evals.resize(m);
    res.resize(m);
    KSS_CHECK_CUDA(cudaMemcpyAsync(evals.data(), lam.p, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaMemcpyAsync(res.data(), resid.p, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    if (tc_error_flag(ctx, true)) fail(KSS_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up");
    for (int n = 0; n < m; ++n)
      if (!std::isfinite(evals[n]) || !std::isfinite(res[n])) fail(KSS_ENUMERIC, "non-finite Ritz value or residual");
    return true;
  }

  // Y <- Y - X (X^H Y) (and HY <- HY - HX (X^H Y) when given), then unit-norm bands.
  void orth_normalize(void* Y, void* HY) {
    gemm_cn(ctx, true, m, m, npw, X.p, npw, Y, npw, M.p, m, 1, 0, 0, 0, "lobpcg_orth");
    gemm_nn(ctx, true, npw, m, m, X.p, npw, M.p, m, Y, npw, -1, 0, 1, 0, "lobpcg_orth");
    if (HY) gemm_nn(ctx, true, npw, m, m, HX.p, npw, M.p, m, HY, npw, -1, 0, 1, 0, "lobpcg_orth");
    static const int idn = prof_register("lobpcg_normalize");
    ProfScope ps(ctx, idn);
    normalize_bands<<<m, 256, 0, ctx->stream>>>((double2*)Y, (double2*)HY, npw);
    KSS_CHECK_CUDA(cudaGetLastError());
  }

  // ---- RMM-DIIS (Kresse & Furthmueller): per-band residual minimisation from the Ritz block ----
  DevBuf eps, sums, coef;
  std::vector<double> h_sums, h_step;

  // Rayleigh quotients of the bands of (v, hv) -> e (device, m values)
  void rayleigh(const void* v, const void* hv, double* e) {
    band_sums<<<m, 256, 0, ctx->stream>>>(0, npw, m, (const double2*)v, (const double2*)hv, nullptr, nullptr,
                                          nullptr, nullptr, nullptr, nullptr, sums.as<double>());
    h_sums.resize(2 * (size_t)m);
    KSS_CHECK_CUDA(cudaMemcpyAsync(h_sums.data(), sums.p, 2 * (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<double> q(m);
    for (int n = 0; n < m; ++n) q[n] = h_sums[m + n] > 0 ? h_sums[n] / h_sums[m + n] : 0.0;
    KSS_CHECK_CUDA(cudaMemcpyAsync(e, q.data(), (size_t)m * 8, cudaMemcpyHostToDevice, ctx->stream));
  }

  // W = K R(v) with R(v) = hv - e v (Teter-Payne-Allan preconditioner)
  void precondition(const void* v, const void* hv, const double* e) {
    const KData& kd = sys->k[ik];
    band_ekin<<<m, 256, 0, ctx->stream>>>((const double2*)v, kd.d_kin64.as<double>(), npw, ek.as<double>());
    precond_resid<<<grid_for((long long)npw * m), 256, 0, ctx->stream>>>(
        (const double2*)v, (const double2*)hv, kd.d_kin64.as<double>(), e, ek.as<double>(), npw, m, d(W));
    KSS_CHECK_CUDA(cudaGetLastError());
  }

  // out = base + step_n * W, hout = hbase + step_n * HW (per-band step)
  void advance(const void* base, const void* hbase, void* out, void* hout) {
    std::vector<double> c(2 * (size_t)m);
    for (int n = 0; n < m; ++n) {
      c[2 * n] = 1.0;
      c[2 * n + 1] = h_step[n];
    }
    KSS_CHECK_CUDA(cudaMemcpyAsync(coef.p, c.data(), c.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    const unsigned gb = grid_for((long long)npw * m);
    band_combine<<<gb, 256, 0, ctx->stream>>>(2, npw, m, (const double2*)base, d(W), nullptr, nullptr,
                                              coef.as<double>(), (double2*)out);
    band_combine<<<gb, 256, 0, ctx->stream>>>(2, npw, m, (const double2*)hbase, d(HW), nullptr, nullptr,
                                              coef.as<double>(), (double2*)hout);
    KSS_CHECK_CUDA(cudaGetLastError());
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));  // c lives on the host stack
  }

  // One sweep of nstep trial updates per band from (X, HX, Ritz values); leaves the last trial in
  // (X, HX) (not orthonormal: the next Rayleigh-Ritz orthonormalises).
  void rmm_sweep(int nstep) {
    static const int idr = prof_register("rmmdiis_band_ops");
    ProfScope ps(ctx, idr);
    DevBuf* pv[3] = {&X, &T1, &T3};
    DevBuf* hv[3] = {&HX, &T2, &T4};
    double* e[3] = {eps.as<double>(), eps.as<double>() + m, eps.as<double>() + 2 * m};
    KSS_CHECK_CUDA(cudaMemcpyAsync(e[0], lam.p, (size_t)m * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    // step 1: optimal step length along W = K R(psi_0), psi_1 = psi_0 + lambda W
    precondition(X.p, HX.p, e[0]);
    apply(W.p, HW.p);
    band_sums<<<m, 256, 0, ctx->stream>>>(2, npw, m, d(X), d(HX), e[0], nullptr, nullptr, nullptr, d(W), d(HW),
                                          sums.as<double>());
    h_sums.resize(2 * (size_t)m);
    KSS_CHECK_CUDA(cudaMemcpyAsync(h_sums.data(), sums.p, 2 * (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    h_step.assign(m, 0.0);
    for (int n = 0; n < m; ++n) {
      const double v = h_sums[m + n];
      double l = v > 0 ? -h_sums[n] / v : 0.0;
      if (!std::isfinite(l)) l = 0.0;
      h_step[n] = std::max(-3.0, std::min(3.0, l));
    }
    if (nstep == 1) {
      advance(X.p, HX.p, T1.p, T2.p);
      std::swap(X, T1);
      std::swap(HX, T2);
      return;
    }
    advance(X.p, HX.p, T1.p, T2.p);
    rayleigh(T1.p, T2.p, e[1]);
    for (int j = 1; j < nstep; ++j) {
      const int q = j + 1;  // history psi_0 .. psi_j
      // DIIS: minimise |sum a_i R_i| with sum a_i = 1, per band (matrix M_ik = Re <R_i|R_k>)
      std::vector<double> M((size_t)q * q * m);
      for (int i = 0; i < q; ++i)
        for (int k = 0; k <= i; ++k) {
          band_sums<<<m, 256, 0, ctx->stream>>>(1, npw, m, d(*pv[i]), d(*hv[i]), e[i], d(*pv[k]), d(*hv[k]), e[k],
                                                nullptr, nullptr, sums.as<double>());
          h_sums.resize(m);
          KSS_CHECK_CUDA(cudaMemcpyAsync(h_sums.data(), sums.p, (size_t)m * 8, cudaMemcpyDeviceToHost, ctx->stream));
          KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
          for (int n = 0; n < m; ++n) M[((size_t)n * q + i) * q + k] = M[((size_t)n * q + k) * q + i] = h_sums[n];
        }
      std::vector<double> a((size_t)m * q);
      for (int n = 0; n < m; ++n) diis_coefficients(q, &M[(size_t)n * q * q], &a[(size_t)n * q]);
      KSS_CHECK_CUDA(cudaMemcpyAsync(coef.p, a.data(), a.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
      const unsigned gb = grid_for((long long)npw * m);
      band_combine<<<gb, 256, 0, ctx->stream>>>(q, npw, m, d(*pv[0]), d(*pv[1]), q > 2 ? d(*pv[2]) : nullptr,
                                                nullptr, coef.as<double>(), d(P));
      band_combine<<<gb, 256, 0, ctx->stream>>>(q, npw, m, d(*hv[0]), d(*hv[1]), q > 2 ? d(*hv[2]) : nullptr,
                                                nullptr, coef.as<double>(), d(HP));
      KSS_CHECK_CUDA(cudaGetLastError());
      KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));  // a lives on the host
      // next trial from the extrapolated vector: psi_(j+1) = psibar + lambda K R(psibar)
      rayleigh(P.p, HP.p, lam.as<double>());
      precondition(P.p, HP.p, lam.as<double>());
      apply(W.p, HW.p);
      if (j + 1 < nstep) {
        advance(P.p, HP.p, pv[j + 1]->p, hv[j + 1]->p);
        rayleigh(pv[j + 1]->p, hv[j + 1]->p, e[j + 1]);
      } else {
        advance(P.p, HP.p, X.p, HX.p);  // psi_0 (in X) is no longer needed
      }
    }
  }

  // Coefficients a (sum 1) minimising a^T M a for a q x q Gram matrix M of residuals: the
  // bordered system [M 1; 1^T 0][a; mu] = [0; 1] by Gaussian elimination with partial pivoting;
  // the latest vector alone when it is singular.
  static void diis_coefficients(int q, const double* M, double* a) {
    double s = 0;
    for (int i = 0; i < q; ++i) s = std::max(s, std::fabs(M[i * q + i]));
    const int n = q + 1;
    double A[5][6];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= n; ++j) A[i][j] = 0;
    for (int i = 0; i < q; ++i) {
      for (int j = 0; j < q; ++j) A[i][j] = s > 0 ? M[i * q + j] / s : 0.0;
      A[i][q] = 1.0;
      A[q][i] = 1.0;
    }
    A[q][n] = 1.0;
    bool ok = s > 0;
    for (int c = 0; c < n && ok; ++c) {
      int p = c;
      for (int r = c + 1; r < n; ++r)
        if (std::fabs(A[r][c]) > std::fabs(A[p][c])) p = r;
      if (std::fabs(A[p][c]) < 1e-14) {
        ok = false;
        break;
      }
      if (p != c)
        for (int j = 0; j <= n; ++j) std::swap(A[c][j], A[p][j]);
      for (int r = 0; r < n; ++r) {
        if (r == c) continue;
        const double f = A[r][c] / A[c][c];
        for (int j = c; j <= n; ++j) A[r][j] -= f * A[c][j];
      }
    }
    for (int i = 0; i < q; ++i) a[i] = ok ? A[i][n] / A[i][i] : (i == q - 1 ? 1.0 : 0.0);
    for (int i = 0; i < q; ++i)
      if (!std::isfinite(a[i])) {
        for (int k = 0; k < q; ++k) a[k] = k == q - 1 ? 1.0 : 0.0;
        break;
      }
  }

  double max_wanted() const {
    double r = 0;
    for (int n = 0; n < nband; ++n) r = std::max(r, res[n]);
    return r;
  }

  // One LOBPCG step from (X, HX, Lambda, residuals): W, then Rayleigh-Ritz in [X W P].
  void step() {
    const KData& kd = sys->k[ik];
    static const int idp = prof_register("lobpcg_precond");
    {
      ProfScope ps(ctx, idp);
      band_ekin<<<m, 256, 0, ctx->stream>>>(d(X), kd.d_kin64.as<double>(), npw, ek.as<double>());
      precond_resid<<<grid_for((long long)npw * m), 256, 0, ctx->stream>>>(
          d(X), d(HX), kd.d_kin64.as<double>(), lam.as<double>(), ek.as<double>(), npw, m, d(W));
    }
    KSS_CHECK_CUDA(cudaGetLastError());
    orth_normalize(W.p, nullptr);
    if (have_p) orth_normalize(P.p, HP.p);
    apply(W.p, HW.p);
    bool ok = false;
    if (have_p) ok = rayleigh_ritz({X.p, W.p, P.p}, {HX.p, HW.p, HP.p});
    if (!ok) ok = rayleigh_ritz({X.p, W.p}, {HX.p, HW.p});
    if (!ok) fail(KSS_ENUMERIC, "LOBPCG: the Rayleigh-Ritz pencil is not numerically positive definite");
    iters += 1;
  }
};

}  // namespace

}  // namespace kss

using namespace kss;

extern "C" kss_status kss_rmmdiis_solve(kss_sys sys, int ik, int nband, const kss_solve_opts* opts, double* evals,
                                        void* evecs, int ld, double* resid, kss_solve_stats* stats) {
  if (!sys) return KSS_EINVAL;
  kss_ctx ctx = sys->ctx;
  try {
    KSS_NVTX("rmmdiis_solve");
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(nband >= 1, "nband must be >= 1");
    KSS_REQUIRE(opts && opts->x0 && opts->x0_nb >= nband,
                "kss_rmmdiis_solve refines trial vectors: opts->x0 with at least nband bands is required");
    const kss_solve_opts o = *opts;
    if (o.prec != KSS_PREC_FP64) fail(KSS_ENOTSUP, "kss_rmmdiis_solve runs in FP64 only");
    if (sys->has_S) fail(KSS_ENOTSUP, "kss_rmmdiis_solve takes systems without an overlap");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<Lobpcg> L(new Lobpcg());
    L->sys = sys;
    L->ctx = ctx;
    L->ik = ik;
    L->nband = nband;
    L->npw = sys->k[ik].npw;
    const int nbuf = o.nbuffer >= 0 ? o.nbuffer : std::max(4, (nband + 9) / 10);
    L->m = std::max(nband + nbuf, std::min(o.x0_nb, nband + nbuf));
    KSS_REQUIRE(L->m <= L->npw, "nband + nbuffer > npw");
    KSS_REQUIRE(o.x0_ld >= L->npw, "x0_ld < npw");
    L->tol = o.tol > 0 ? o.tol : 1e-8;
    L->max_iter = o.max_iter > 0 ? o.max_iter : 100;
    const int m = L->m;
    for (DevBuf* b : {&L->X, &L->HX, &L->W, &L->HW, &L->P, &L->HP, &L->T1, &L->T2, &L->T3, &L->T4})
      b->alloc(L->blk());
    L->A.alloc((size_t)m * m * 16);
    L->B.alloc((size_t)m * m * 16);
    L->ev.alloc((size_t)m * 8);
    L->info.alloc(sizeof(int));
    L->lam.alloc((size_t)m * 8);
    L->ek.alloc((size_t)m * 8);
    L->resid.alloc((size_t)m * 8);
    L->eps.alloc(3 * (size_t)m * 8);
    L->sums.alloc(2 * (size_t)m * 8);
    L->coef.alloc(4 * (size_t)m * 8);
    const int nx = std::min(o.x0_nb, m);
    KSS_CHECK_CUDA(cudaMemcpy2DAsync(L->X.p, (size_t)L->npw * 16, o.x0, (size_t)o.x0_ld * 16, (size_t)L->npw * 16,
                                     nx, cudaMemcpyDeviceToDevice, ctx->stream));
    if (nx < m)
      random_block(ctx, true, (char*)L->X.p + (size_t)nx * L->npw * 16, L->npw, m - nx, L->npw, o.seed, nx);
    L->apply(L->X.p, L->HX.p);
    if (!L->rayleigh_ritz({L->X.p}, {L->HX.p}))
      fail(KSS_ENUMERIC, "RMM-DIIS: the trial block is numerically rank-deficient");
    bool conv = L->max_wanted() <= L->tol;
    while (!conv && L->iters < L->max_iter) {
      L->rmm_sweep(3);
      if (!L->rayleigh_ritz({L->X.p}, {L->HX.p}))
        fail(KSS_ENUMERIC, "RMM-DIIS: the refined block lost rank (Cholesky failed)");
      L->iters += 1;
      conv = L->max_wanted() <= L->tol;
    }
    if (evals) std::copy(L->evals.begin(), L->evals.begin() + nband, evals);
    if (resid) std::copy(L->res.begin(), L->res.begin() + nband, resid);
    if (evecs) {
      KSS_REQUIRE(ld >= L->npw, "ld < npw");
      KSS_CHECK_CUDA(cudaMemcpy2DAsync(evecs, (size_t)ld * 16, L->X.p, (size_t)L->npw * 16, (size_t)L->npw * 16,
                                       nband, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    if (stats) {
      *stats = kss_solve_stats{};
      stats->iters = L->iters;
      stats->napply = L->napply;
      stats->max_resid = L->max_wanted();
      stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      stats->nb = m;
    }
    if (!conv) {
      ctx->err = "not converged within max_iter";
      return KSS_ENOCONV;
    }
    ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    ctx->err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return KSS_ENOMEM;
  }
}

extern "C" kss_status kss_lobpcg_solve(kss_sys sys, int ik, int nband, const kss_solve_opts* opts, double* evals,
                                       void* evecs, int ld, double* resid, kss_solve_stats* stats) {
  if (!sys) return KSS_EINVAL;
  kss_ctx ctx = sys->ctx;
  try {
    KSS_NVTX("lobpcg_solve");
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(nband >= 1, "nband must be >= 1");
    kss_solve_opts o{};
    if (opts) o = *opts;
    if (o.prec != KSS_PREC_FP64) fail(KSS_ENOTSUP, "kss_lobpcg_solve runs in FP64 only");
    if (sys->has_S) fail(KSS_ENOTSUP, "kss_lobpcg_solve takes systems without an overlap");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<Lobpcg> L(new Lobpcg());
    L->sys = sys;
    L->ctx = ctx;
    L->ik = ik;
    L->nband = nband;
    L->npw = sys->k[ik].npw;
    const int nbuf = o.nbuffer >= 0 ? o.nbuffer : std::max(4, (nband + 9) / 10);
    L->m = nband + nbuf;
    KSS_REQUIRE(3 * L->m <= L->npw, "LOBPCG needs 3 (nband + nbuffer) <= npw");
    L->tol = o.tol > 0 ? o.tol : 1e-8;
    L->max_iter = o.max_iter > 0 ? o.max_iter : 500;
    const int m = L->m;
    for (DevBuf* b : {&L->X, &L->HX, &L->W, &L->HW, &L->P, &L->HP, &L->T1, &L->T2, &L->T3, &L->T4})
      b->alloc(L->blk());
    const size_t k3 = 3 * (size_t)m;
    L->A.alloc(k3 * k3 * 16);
    L->B.alloc(k3 * k3 * 16);
    L->ev.alloc(k3 * 8);
    L->info.alloc(sizeof(int));
    L->lam.alloc((size_t)m * 8);
    L->ek.alloc((size_t)m * 8);
    L->resid.alloc((size_t)m * 8);
    L->M.alloc((size_t)m * m * 16);
    // starting block: the caller's warm start, then Philox random bands
    int nx = 0;
    if (o.x0) {
      KSS_REQUIRE(o.x0_nb >= 0 && o.x0_nb <= m && o.x0_ld >= L->npw, "bad warm start");
      nx = o.x0_nb;
      if (nx)
        KSS_CHECK_CUDA(cudaMemcpy2DAsync(L->X.p, (size_t)L->npw * 16, o.x0, (size_t)o.x0_ld * 16,
                                         (size_t)L->npw * 16, nx, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (nx < m)
      random_block(ctx, true, (char*)L->X.p + (size_t)nx * L->npw * 16, L->npw, m - nx, L->npw, o.seed, nx);
    L->apply(L->X.p, L->HX.p);
    if (!L->rayleigh_ritz({L->X.p}, {L->HX.p}))
      fail(KSS_ENUMERIC, "LOBPCG: the starting block is numerically rank-deficient");
    bool conv = L->max_wanted() <= L->tol;
    while (!conv && L->iters < L->max_iter) {
      L->step();
      conv = L->max_wanted() <= L->tol;
    }
    if (evals) std::copy(L->evals.begin(), L->evals.begin() + nband, evals);
    if (resid) std::copy(L->res.begin(), L->res.begin() + nband, resid);
    if (evecs) {
      KSS_REQUIRE(ld >= L->npw, "ld < npw");
      KSS_CHECK_CUDA(cudaMemcpy2DAsync(evecs, (size_t)ld * 16, L->X.p, (size_t)L->npw * 16, (size_t)L->npw * 16,
                                       nband, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    if (stats) {
      *stats = kss_solve_stats{};
      stats->iters = L->iters;
      stats->napply = L->napply;
      stats->max_resid = L->max_wanted();
      stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      stats->nb = m;
    }
    if (!conv) {
      ctx->err = "not converged within max_iter";
      return KSS_ENOCONV;
    }
    ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    ctx->err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    ctx->err = "host allocation failed";
    return KSS_ENOMEM;
  }
}

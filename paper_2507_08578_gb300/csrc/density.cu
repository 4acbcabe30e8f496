// Electron density after the solve, n(r_j) = sum_n w_n |psi_n(r_j)|^2 (Eq. nandtau, §2; w the
// occupancy times the k-point weight), psi_n(r) = Omega^-1/2 sum_G c_n(G) e^{i(k+G).r}.
//
// Per chunk of bands: pass A (scatter + inverse x transform into the slab, shared with the H
// application), then one CTA per (x-plane, band group g) runs the inverse y and z transforms of
// its plane for the group's bands with every transform stage spread over the CTA (the layout of
// the CTA-wide middle pass, local_kernels.cuh) and accumulates w |psi|^2 in FP64 registers.  Each
// (g, x) owns one plane of a partial-sum buffer [G][N1][N2][N3], so the accumulation over chunks
// is deterministic; a last kernel sums the groups into rho ([N3][N2][N1], x fastest) times 1/Omega.
#include <algorithm>

#include "density.h"
#include "kss_internal.h"

namespace kss {

namespace {

using namespace lk;

constexpr int kDensThreads = 384;
constexpr int kMaxGroups = 16;  // band groups per chunk (partial-density planes)

template <typename T, int A, int B, int NT>
__global__ void __launch_bounds__(NT) pass_dw(LocalArgs<T> a, int m, int G, const double* __restrict__ occ,
                                              double* __restrict__ part) {
  using C = typename CT<T>::C;
  constexpr int N = A * B, QS = (N + 1) | 1, ZS = (N + 1) | 1;  // odd pitches (as the CTA-wide pass B)
  constexpr int R = (N * A + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tw = reinterpret_cast<C*>(smraw);
  C* Q = tw + N;
  C* Z = Q + a.W3 * QS;
  int* zmap = reinterpret_cast<int*>(Z + N * ZS);
  const int x = blockIdx.x, g = blockIdx.y;
  const int tid = threadIdx.x, W3 = a.W3, W2 = a.W2;
  for (int i = tid; i < N; i += NT) tw[i] = a.tw2[i];
  for (int z = tid; z < N; z += NT) {
    int u = (z - a.lo3) % N;
    if (u < 0) u += N;
    zmap[z] = u < W3 ? u : -1;
  }
  double acc[R][B];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < B; ++j) acc[r][j] = 0;
  const fftr::FastDiv dw2(W2), dw3(W3);
  for (int b = g; b < m; b += G) {
    __syncthreads();  // the previous band's reads of Q and Z are done
    for (int i = tid; i < W3 * QS; i += NT) Q[i] = C{0, 0};
    __syncthreads();
    const C* slab = a.work + ((size_t)b * a.N1 + x) * W3 * W2;
    for (int i = tid; i < W3 * W2; i += NT) {
      const int u3 = dw2(i), u2 = i - u3 * W2;
      Q[u3 * QS + fftr::wrap_add(a.lo2, u2, N)] = slab[i];
    }
    __syncthreads();
    // y inverse (two stages, in place; leaves position k2 + B k holding y = k + A k2)
    for (int t = tid; t < W3 * B; t += NT) {
      const int r = dw3(t), u = t - r * W3;  // rows fastest across lanes
      C* row = Q + u * QS + r;
      C v[A];
#pragma unroll
      for (int i = 0; i < A; ++i) v[i] = row[B * i];
      fftr::rdft<A>(v, (T)1);
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
    // z inverse, stage 1 (window rows of Q -> full columns of Z)
    for (int t = tid; t < N * B; t += NT) {
      const int r = t / N, p = t - r * N;
      C v[A];
#pragma unroll
      for (int i = 0; i < A; ++i) {
        const int u = zmap[r + B * i];
        v[i] = u >= 0 ? Q[u * QS + p] : C{0, 0};
      }
      fftr::rdft<A>(v, (T)1);
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
    // z inverse, stage 2: psi(x, y, z = k + A k2); accumulate w |psi|^2 (fixed task -> thread map)
    const double wb = occ[a.n0 + b];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = tid + NT * r;
      if (t < N * A) {
        const int k = t / N, p = t - k * N;  // columns fastest across lanes
        const C* col = Z + p * ZS + B * k;
        C v[B];
#pragma unroll
        for (int j = 0; j < B; ++j) v[j] = col[j];
        fftr::rdft<B>(v, (T)1);
#pragma unroll
        for (int j = 0; j < B; ++j) {
          const double re = (double)v[j].x, im = (double)v[j].y;
          acc[r][j] = fma(wb, fma(re, re, im * im), acc[r][j]);
        }
      }
    }
  }
  // Through shared memory to the partial plane: the accumulators sit in column (y position) order,
  // so stage them as [p][z] (the odd pitch ZS, in doubles: Z holds at least N ZS of them) and write
  // the plane out row by row in natural y.
  __syncthreads();  // the last band's reads of Z are done
  double* st = reinterpret_cast<double*>(Z);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = tid + NT * r;
    if (t < N * A) {
      const int k = t / N, p = t - k * N;  // the accumulation's task -> thread map
#pragma unroll
      for (int j = 0; j < B; ++j) st[p * ZS + k + A * j] = acc[r][j];
    }
  }
  __syncthreads();
  double* pg = part + ((size_t)g * a.N1 + x) * N * N;
  for (int i = tid; i < N * N; i += NT) {
    const int y = i / N, z = i - y * N;
    const int k2 = y / A, k = y - k2 * A;  // y = k + A k2 sits at position k2 + B k
    pg[i] += st[(k2 + B * k) * ZS + z];
  }
}

// rho[z][y][x] += inv_vol * sum_g part[g][x][y][z]
__global__ void density_reduce(int N1, int N2, int N3, int G, const double* __restrict__ part, double* rho,
                               double inv_vol) {
  const long long n = (long long)N1 * N2 * N3;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(idx % N1);
    const long long r = idx / N1;
    const int y = (int)(r % N2), z = (int)(r / N2);
    double sum = 0;
    for (int g = 0; g < G; ++g) sum += part[(((size_t)g * N1 + x) * N2 + y) * N3 + z];
    rho[idx] += inv_vol * sum;
  }
}

// dry: only check that the instance exists and fits; *resident (when given) receives the
// resident CTAs per SM of the instance at this shared-memory size.
template <typename T, int A, int B>
bool launch_d(const LocalArgs<T>& a, int m, int G, const double* occ, double* part, cudaStream_t st, bool dry,
              int* resident) {
  using C = typename CT<T>::C;
  constexpr int N = A * B;
  constexpr int P = (N + 1) | 1;
  const size_t sm = sizeof(C) * ((size_t)N + (size_t)a.W3 * P + (size_t)N * P) + sizeof(int) * N;
  if (sm > 227 * 1024) return false;
  if (resident) {
    KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_dw<T, A, B, kDensThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sm));
    KSS_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(resident, pass_dw<T, A, B, kDensThreads>,
                                                                 kDensThreads, sm));
  }
  if (dry) return true;
  KSS_CHECK_CUDA(cudaFuncSetAttribute(pass_dw<T, A, B, kDensThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm));
  pass_dw<T, A, B, kDensThreads><<<dim3(a.N1, G), kDensThreads, sm, st>>>(a, m, G, occ, part);
  return true;
}

template <typename T>
bool pass_d(const LocalArgs<T>& a, int A, int B, int m, int G, const double* occ, double* part, cudaStream_t st,
            bool dry, int* resident = nullptr) {
  if (a.N2 != a.N3 || A * B != a.N2) return false;
  switch (A * 32 + B) {
#define KSS_CASE(x, y) \
  case x * 32 + y:     \
    return launch_d<T, x, y>(a, m, G, occ, part, st, dry, resident);
    KSS_SPLITS(KSS_CASE)
#undef KSS_CASE
    default:
      return false;
  }
}

template <typename T>
void density_t(kss_sys s, int ik, int nb, const void* psi, int ld, const double* occ_host, double* rho) {
  kss_ctx ctx = s->ctx;
  fftr::Split sp;
  int resident = 1;
  if (!(s->N[1] == s->N[2] && choose_split(s->N[1], sp)))
    fail(KSS_ENOTSUP, "kss_density_accumulate needs N2 == N3 with a two-codelet split");
  {
    LocalArgs<T> probe{};
    probe.N1 = s->N[0];
    probe.N2 = s->N[1];
    probe.N3 = s->N[2];
    probe.W3 = s->k[ik].W[2];
    if (!pass_d<T>(probe, sp.A, sp.B, 0, 1, nullptr, nullptr, nullptr, true, &resident))
      fail(KSS_ENOTSUP, "no density kernel instance for this FFT length / window");
  }
  const int N1 = s->N[0], N2 = s->N[1], N3 = s->N[2];
  const int cap = std::max(1, ctx->nsm) * std::max(1, resident);
  // Band groups of a chunk of m bands: G maximising (fill of the last wave of N1*G CTAs) x
  // (balance of ceil(m/G) bands per CTA), the larger G on ties.
  auto groups = [&](int m) {
    int best = 1;
    double be = -1;
    for (int g = 1; g <= std::min(kMaxGroups, m); ++g) {
      const long long ctas = (long long)N1 * g;
      const double fill = (double)ctas / (double)(((ctas + cap - 1) / cap) * cap);
      const double bal = (double)m / (double)(g * ((m + g - 1) / g));
      if (fill * bal >= be - 1e-12) {
        be = fill * bal;
        best = g;
      }
    }
    return best;
  };
  const int G = kMaxGroups;  // partial planes allocated for the largest grouping
  ctx->ws_occ.ensure((size_t)nb * sizeof(double));
  ctx->ws_rho.ensure((size_t)G * N1 * N2 * N3 * sizeof(double));
  KSS_CHECK_CUDA(cudaMemcpyAsync(ctx->ws_occ.p, occ_host, (size_t)nb * sizeof(double), cudaMemcpyHostToDevice,
                                 ctx->stream));
  KSS_CHECK_CUDA(cudaMemsetAsync(ctx->ws_rho.p, 0, (size_t)G * N1 * N2 * N3 * sizeof(double), ctx->stream));
  static const int idd = prof_register(sizeof(T) == 8 ? "density_pass<f64>" : "density_pass<f32>");
  pass_a_chunks<T>(s, ik, nb, psi, ld, [&](const LocalArgs<T>& a, int m) {
    ProfScope ps(ctx, idd);
    pass_d<T>(a, sp.A, sp.B, m, groups(m), ctx->ws_occ.as<double>(), ctx->ws_rho.as<double>(), ctx->stream, false);
  });
  static const int idr = prof_register("density_reduce");
  {
    ProfScope ps(ctx, idr);
    const long long n = (long long)N1 * N2 * N3;
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16);
    density_reduce<<<blocks, 256, 0, ctx->stream>>>(N1, N2, N3, G, ctx->ws_rho.as<double>(), rho, 1.0 / s->vol);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace

}  // namespace kss

using namespace kss;

extern "C" kss_status kss_density_accumulate(kss_sys sys, int ik, int nb, const void* psi, int ld,
                                             const double* occ, double* rho, kss_precision prec) {
  if (!sys) return KSS_EINVAL;
  kss_ctx ctx = sys->ctx;
  try {
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(nb >= 0, "nb < 0");
    KSS_REQUIRE(prec == KSS_PREC_FP64 || prec == KSS_PREC_MIXED, "unknown precision");
    KSS_REQUIRE(ld >= sys->k[ik].npw, "ld < npw");
    if (nb == 0) {
      ctx->err.clear();
      return KSS_OK;
    }
    KSS_REQUIRE(psi && occ && rho, "null psi, occ or rho");
    for (int n = 0; n < nb; ++n) KSS_REQUIRE(std::isfinite(occ[n]), "non-finite occupation");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    if (prec == KSS_PREC_FP64) density_t<double>(sys, ik, nb, psi, ld, occ, rho);
    else density_t<float>(sys, ik, nb, psi, ld, occ, rho);
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

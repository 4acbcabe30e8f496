// Host side of the C ABI: contexts, system setup (G-sphere, index maps, tables), queries.
//
// Built with -ffp-contract=off: the G-sphere inclusion test below must round exactly as the
// written expression (no fused multiply-add), so that every implementation that evaluates the
// same expression in IEEE double selects the same plane waves.
#include <cmath>
#include <cstring>
#include <new>
#include <algorithm>
#include <memory>
#include <unordered_map>

#include "kss_internal.h"

namespace kss {

void fail(kss_status st, const std::string& msg) { throw KssError{st, msg}; }

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

void DevBuf::alloc(size_t n) {
  release();
  if (n == 0) return;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    fail(KSS_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed: " +
                         cudaGetErrorString(e));
  }
  bytes = n;
}

void DevBuf::ensure(size_t n) {
  if (n > bytes) alloc(n);
}

static bool smooth235(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Default FFT box edge along one axis: the smallest {2,3,5}-smooth N >= 4 max|m| + 1 (no aliasing
// of products of two band functions).
static int default_box_edge(int mmax) {
  int n = 4 * mmax + 1;
  while (!smooth235(n)) ++n;
  return n;
}

FftDim make_fft_dim(int N) {
  FftDim d{};
  d.N = N;
  int n = N;
  // Radix-4 stages first (fewest passes), then 2, 3, 5.
  while (n % 4 == 0) { d.rad[d.nst++] = 4; n /= 4; }
  while (n % 2 == 0) { d.rad[d.nst++] = 2; n /= 2; }
  while (n % 3 == 0) { d.rad[d.nst++] = 3; n /= 3; }
  while (n % 5 == 0) { d.rad[d.nst++] = 5; n /= 5; }
  if (n != 1 || d.nst > 10) fail(KSS_EINVAL, "FFT length " + std::to_string(N) + " is not {2,3,5}-smooth");
  return d;
}

// Reciprocal rows b_i = (2 pi / vol) (a_j x a_k), scalar formula in a fixed order.
static void reciprocal(const double* a, double* B, double* vol) {
  const double a1x = a[0], a1y = a[1], a1z = a[2];
  const double a2x = a[3], a2y = a[4], a2z = a[5];
  const double a3x = a[6], a3y = a[7], a3z = a[8];
  const double c23[3] = {a2y * a3z - a2z * a3y, a2z * a3x - a2x * a3z, a2x * a3y - a2y * a3x};
  const double c31[3] = {a3y * a1z - a3z * a1y, a3z * a1x - a3x * a1z, a3x * a1y - a3y * a1x};
  const double c12[3] = {a1y * a2z - a1z * a2y, a1z * a2x - a1x * a2z, a1x * a2y - a1y * a2x};
  const double v = a1x * c23[0] + a1y * c23[1] + a1z * c23[2];
  const double f = (2.0 * 3.141592653589793) / v;  // 2 pi in double
  for (int i = 0; i < 3; ++i) {
    B[0 + i] = f * c23[i];
    B[3 + i] = f * c31[i];
    B[6 + i] = f * c12[i];
  }
  *vol = v;
}

// q = sum_i (m_i + kappa_i) b_i, each Cartesian component summed left to right.
static inline void qvec(const double* B, const double* kr, int m1, int m2, int m3, double* q) {
  const double u1 = (double)m1 + kr[0];
  const double u2 = (double)m2 + kr[1];
  const double u3 = (double)m3 + kr[2];
  q[0] = u1 * B[0] + u2 * B[3] + u3 * B[6];
  q[1] = u1 * B[1] + u2 * B[4] + u3 * B[7];
  q[2] = u1 * B[2] + u2 * B[5] + u3 * B[8];
}

static inline double half_q2(const double* q) {
  return 0.5 * ((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]);
}

// Enumerate the sphere in canonical order (m3, m2, m1 ascending).  Loops visit m3, then m2, then
// m1 in ascending order; the m1 loop is limited to a window around the row's closest approach
// (widened by 2) and every candidate passes the exact inclusion test.
static void enumerate_sphere(const double* lat, const double* B, double ecut, const double* kr,
                             std::vector<int32_t>& miller) {
  miller.clear();
  const double gmax = std::sqrt(2.0 * ecut);
  int lo[3], hi[3];
  for (int i = 0; i < 3; ++i) {
    const double an = std::sqrt(lat[3 * i] * lat[3 * i] + lat[3 * i + 1] * lat[3 * i + 1] +
                                lat[3 * i + 2] * lat[3 * i + 2]);
    const double R = gmax * an / (2.0 * 3.141592653589793);
    lo[i] = (int)std::floor(-R - kr[i]) - 1;
    hi[i] = (int)std::ceil(R - kr[i]) + 1;
  }
  // Along b1, |q| is minimised at u1 = -(w . b1)/|b1|^2 where w is the (m2,m3) part of q.
  const double b1n2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  const double b1n = std::sqrt(b1n2);
  for (int m3 = lo[2]; m3 <= hi[2]; ++m3) {
    for (int m2 = lo[1]; m2 <= hi[1]; ++m2) {
      const double u2 = (double)m2 + kr[1], u3 = (double)m3 + kr[2];
      const double w[3] = {u2 * B[3] + u3 * B[6], u2 * B[4] + u3 * B[7], u2 * B[5] + u3 * B[8]};
      const double t = -(w[0] * B[0] + w[1] * B[1] + w[2] * B[2]) / b1n2;  // u1 at closest approach
      const double perp2 = (w[0] + t * B[0]) * (w[0] + t * B[0]) +
                           (w[1] + t * B[1]) * (w[1] + t * B[1]) +
                           (w[2] + t * B[2]) * (w[2] + t * B[2]);
      const double rem = 2.0 * ecut - perp2;
      if (rem < -1e-6 * (2.0 * ecut + 1.0)) continue;  // row entirely outside (with margin)
      const double half = std::sqrt(std::max(rem, 0.0)) / b1n;
      int a = (int)std::floor(t - half - kr[0]) - 2, b = (int)std::ceil(t + half - kr[0]) + 2;
      a = std::max(a, lo[0]);
      b = std::min(b, hi[0]);
      for (int m1 = a; m1 <= b; ++m1) {
        double q[3];
        qvec(B, kr, m1, m2, m3, q);
        if (half_q2(q) <= ecut) {
          miller.push_back(m1);
          miller.push_back(m2);
          miller.push_back(m3);
        }
      }
    }
  }
}

template <typename F>
static kss_status guard(kss_ctx ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    if (ctx) ctx->err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed";
    return KSS_ENOMEM;
  } catch (...) {
    if (ctx) ctx->err = "unexpected internal error";
    return KSS_ECUDA;
  }
}

}  // namespace kss

using namespace kss;

namespace kss {
}

extern "C" {

int kss_version(void) { return KSS_VERSION_MAJOR * 1000 + KSS_VERSION_MINOR; }

const char* kss_last_error(kss_ctx ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

kss_status kss_create(kss_ctx* out, int device, void* cuda_stream) {
  if (!out) return KSS_EINVAL;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return KSS_ECUDA;
  }
  if (device < 0 || device >= n) return KSS_ECUDA;
  kss_ctx ctx = new (std::nothrow) kss_ctx_s();
  if (!ctx) return KSS_ENOMEM;
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return KSS_ECUDA;
  }
  ctx->stream = (cudaStream_t)cuda_stream;  // NULL: legacy default stream
  ctx->own_stream = false;
  {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && v > 0) ctx->nsm = v;
  }
  *out = ctx;
  return KSS_OK;
}

kss_status kss_destroy(kss_ctx ctx) {
  if (!ctx) return KSS_EINVAL;
  if (ctx->server) {
    ctx->err = "stop the request server (kss_server_stop) before destroying its context";
    return KSS_EINVAL;
  }
  if (ctx->nsys > 0) {
    ctx->err = "destroy every system before its context";
    return KSS_EINVAL;
  }
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  aux_release(ctx);
  prof_release(ctx);
  ctx->ws_local.release();
  ctx->ws_gemm.release();
  ctx->ws_cprj.release();
  ctx->stage_in.release();
  ctx->stage_out.release();
  ctx->tc_a.release();
  ctx->tc_b.release();
  ctx->tc_part.release();
  ctx->tc_err.release();
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return KSS_OK;
}

kss_status kss_setup(kss_ctx ctx, const kss_cell* cell, const kss_atoms* atoms, kss_sys* out) {
  if (!ctx) return KSS_EINVAL;
  return guard(ctx, [&] {
    KSS_NVTX("setup");
    KSS_REQUIRE(cell && atoms && out, "kss_setup: null argument");
    *out = nullptr;
    KSS_REQUIRE(cell->ecut > 0 && std::isfinite(cell->ecut), "ecut must be positive");
    KSS_REQUIRE(cell->nk >= 1 && cell->kpts_red, "need at least one k-point");
    KSS_REQUIRE(atoms->natom >= 0, "natom < 0");
    KSS_REQUIRE(atoms->natom == 0 || atoms->pos_cart, "pos_cart is null");
    KSS_REQUIRE(atoms->nproj_per_atom == 0 || atoms->nproj_per_atom == 1 ||
                    atoms->nproj_per_atom == 4,
                "nproj_per_atom must be 0, 1 or 4");
    KSS_REQUIRE(atoms->vloc_sigma > 0 && std::isfinite(atoms->vloc_sigma), "vloc_sigma must be positive");
    KSS_REQUIRE(std::isfinite(atoms->vloc_amp), "non-finite vloc_amp");
    KSS_REQUIRE(atoms->nproj_per_atom == 0 || atoms->natom == 0 ||
                    (atoms->D && atoms->proj_alpha > 0 && std::isfinite(atoms->proj_alpha)),
                "projectors need D and proj_alpha > 0");
    for (int i = 0; i < 9; ++i) KSS_REQUIRE(std::isfinite(cell->lattice[i]), "non-finite lattice vector");
    for (int i = 0; i < 3 * cell->nk; ++i) KSS_REQUIRE(std::isfinite(cell->kpts_red[i]), "non-finite k-point");
    for (int i = 0; i < 3 * atoms->natom; ++i)
      KSS_REQUIRE(std::isfinite(atoms->pos_cart[i]), "non-finite atom position");
    if (atoms->natom && atoms->nproj_per_atom)
      for (int i = 0; i < atoms->natom * atoms->nproj_per_atom; ++i)
        KSS_REQUIRE(std::isfinite(atoms->D[i]), "non-finite projector coefficient D");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    std::unique_ptr<kss_sys_s> s(new kss_sys_s());
    s->ctx = ctx;
    std::memcpy(s->lat, cell->lattice, sizeof(s->lat));
    reciprocal(s->lat, s->B, &s->vol);
    KSS_REQUIRE(std::isfinite(s->vol) && s->vol > 0, "lattice must be right-handed and non-singular");
    s->ecut = cell->ecut;
    s->natom = atoms->natom;
    s->nppa = atoms->natom ? atoms->nproj_per_atom : 0;
    s->nproj = s->natom * s->nppa;
    s->pos.assign(atoms->pos_cart, atoms->pos_cart + 3 * s->natom);
    if (s->nproj) s->D.assign(atoms->D, atoms->D + s->nproj);
    if (s->nproj && atoms->Q) {
      s->Q.assign(atoms->Q, atoms->Q + s->nproj);
      for (double q : s->Q) {
        KSS_REQUIRE(std::isfinite(q), "non-finite overlap coefficient");
        s->has_S |= q != 0.0;
      }
      if (!s->has_S) s->Q.clear();
    }
    s->vamp = atoms->vloc_amp;
    s->vsig = atoms->vloc_sigma;
    s->alpha = atoms->proj_alpha;

    // G-spheres.
    s->k.resize(cell->nk);
    int mmax[3] = {0, 0, 0};
    for (int ik = 0; ik < cell->nk; ++ik) {
      KData& kd = s->k[ik];
      for (int i = 0; i < 3; ++i) kd.kred[i] = cell->kpts_red[3 * ik + i];
      enumerate_sphere(s->lat, s->B, s->ecut, kd.kred, kd.miller);
      kd.npw = (int)(kd.miller.size() / 3);
      KSS_REQUIRE(kd.npw > 0, "empty G-sphere");
      for (int i = 0; i < 3; ++i) {
        int lo = 1 << 30, hi = -(1 << 30);
        for (int g = 0; g < kd.npw; ++g) {
          lo = std::min(lo, kd.miller[3 * g + i]);
          hi = std::max(hi, kd.miller[3 * g + i]);
          mmax[i] = std::max(mmax[i], std::abs(kd.miller[3 * g + i]));
        }
        kd.lo[i] = lo;
        kd.W[i] = hi - lo + 1;
      }
    }
    // FFT box.
    const bool dflt = cell->fft_box[0] == 0 && cell->fft_box[1] == 0 && cell->fft_box[2] == 0;
    for (int i = 0; i < 3; ++i) {
      if (dflt) {
        s->N[i] = default_box_edge(mmax[i]);
      } else {
        s->N[i] = cell->fft_box[i];
      }
      KSS_REQUIRE(s->N[i] >= 2 && s->N[i] <= 256 && smooth235(s->N[i]),
                  "FFT box dimensions must be {2,3,5}-smooth and in [2, 256]");
      for (auto& kd : s->k)
        KSS_REQUIRE(kd.W[i] <= s->N[i], "FFT box does not hold the G-sphere");
      s->dim[i] = make_fft_dim(s->N[i]);
    }
    const int N1 = s->N[0], N2 = s->N[1], N3 = s->N[2];
    const int N1p = N1 + 1;  // padded row stride of the x-pencil tiles

    // Twiddles e^{-2 pi i k / N} (long double angles, rounded once).
    for (int d = 0; d < 3; ++d) {
      const int N = s->N[d];
      std::vector<double> tw(2 * N);
      std::vector<float> tw32(2 * N);
      for (int kk = 0; kk < N; ++kk) {
        const long double ang = -2.0L * 3.141592653589793238462643383279502884L * kk / N;
        tw[2 * kk] = (double)cosl(ang);
        tw[2 * kk + 1] = (double)sinl(ang);
        tw32[2 * kk] = (float)cosl(ang);
        tw32[2 * kk + 1] = (float)sinl(ang);
      }
      s->d_tw64[d].alloc(tw.size() * sizeof(double));
      s->d_tw32[d].alloc(tw32.size() * sizeof(float));
      KSS_CHECK_CUDA(cudaMemcpy(s->d_tw64[d].p, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(s->d_tw32[d].p, tw32.data(), tw32.size() * sizeof(float), cudaMemcpyHostToDevice));
    }

    // Local potential.
    const size_t nr = (size_t)N1 * N2 * N3;
    s->d_V64.alloc(nr * sizeof(double));
    s->d_Vx64.alloc(nr * sizeof(double));
    s->d_Vx32.alloc(nr * sizeof(float));
    launch_vloc(s.get(), ctx->stream);
    launch_vloc_views(s.get(), ctx->stream);
    s->vmax = device_max(s->d_V64.as<double>(), nr, ctx->stream);

    if (s->nproj) {
      s->d_D64.alloc(s->nproj * sizeof(double));
      s->d_D32.alloc(s->nproj * sizeof(float));
      std::vector<float> d32(s->D.begin(), s->D.end());
      KSS_CHECK_CUDA(cudaMemcpy(s->d_D64.p, s->D.data(), s->nproj * sizeof(double), cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(s->d_D32.p, d32.data(), s->nproj * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (s->has_S) {
      s->d_Q64.alloc(s->nproj * sizeof(double));
      s->d_Q32.alloc(s->nproj * sizeof(float));
      std::vector<float> q32(s->Q.begin(), s->Q.end());
      KSS_CHECK_CUDA(cudaMemcpy(s->d_Q64.p, s->Q.data(), s->nproj * sizeof(double), cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(s->d_Q32.p, q32.data(), s->nproj * sizeof(float), cudaMemcpyHostToDevice));
    }

    // Per-k tables.
    for (auto& kd : s->k) {
      const int npw = kd.npw;
      // Gamma point: the sphere is symmetric under m -> -m (q -> -q exactly); the index of -m
      // lets real-space-real bands be packed two per complex FFT
      kd.gamma = kd.kred[0] == 0.0 && kd.kred[1] == 0.0 && kd.kred[2] == 0.0;
      if (kd.gamma) {
        std::unordered_map<long long, int> at;
        auto key = [](int a, int b, int c) {
          return ((long long)(a + 4096) << 26) | ((long long)(b + 4096) << 13) | (long long)(c + 4096);
        };
        for (int g = 0; g < npw; ++g) at[key(kd.miller[3 * g], kd.miller[3 * g + 1], kd.miller[3 * g + 2])] = g;
        std::vector<int32_t> mir(npw);
        for (int g = 0; g < npw; ++g) {
          auto it = at.find(key(-kd.miller[3 * g], -kd.miller[3 * g + 1], -kd.miller[3 * g + 2]));
          KSS_REQUIRE(it != at.end(), "Gamma-point sphere not symmetric (internal)");
          mir[g] = it->second;
        }
        kd.d_mirror.alloc((size_t)npw * 4);
        KSS_CHECK_CUDA(cudaMemcpy(kd.d_mirror.p, mir.data(), (size_t)npw * 4, cudaMemcpyHostToDevice));
      }
      std::vector<int32_t> off(npw), tile(npw);
      std::vector<double> kin(npw), q(3 * npw);
      std::vector<float> kin32(npw);
      kd.zstart.assign(kd.W[2] + 1, 0);
      kd.rowrange.assign(2 * kd.W[2], 0);
      for (int u3 = 0; u3 < kd.W[2]; ++u3) { kd.rowrange[2 * u3] = 1 << 30; kd.rowrange[2 * u3 + 1] = -1; }
      kd.tmax = 0;
      for (int g = 0; g < npw; ++g) {
        const int m1 = kd.miller[3 * g], m2 = kd.miller[3 * g + 1], m3 = kd.miller[3 * g + 2];
        const int j1 = ((m1 % N1) + N1) % N1, j2 = ((m2 % N2) + N2) % N2, j3 = ((m3 % N3) + N3) % N3;
        off[g] = j1 + N1 * (j2 + N2 * j3);
        const int u2 = m2 - kd.lo[1], u3 = m3 - kd.lo[2];
        tile[g] = u2 * N1p + j1;
        kd.zstart[u3 + 1] += 1;
        kd.rowrange[2 * u3] = std::min(kd.rowrange[2 * u3], u2);
        kd.rowrange[2 * u3 + 1] = std::max(kd.rowrange[2 * u3 + 1], u2);
        double qq[3];
        qvec(s->B, kd.kred, m1, m2, m3, qq);
        kin[g] = half_q2(qq);
        kin32[g] = (float)kin[g];
        kd.tmax = std::max(kd.tmax, kin[g]);
        q[3 * g] = qq[0];
        q[3 * g + 1] = qq[1];
        q[3 * g + 2] = qq[2];
      }
      for (int u3 = 0; u3 < kd.W[2]; ++u3) kd.zstart[u3 + 1] += kd.zstart[u3];
      kd.d_miller.alloc(kd.miller.size() * 4);
      kd.d_offset.alloc(npw * 4);
      kd.d_tileidx.alloc(npw * 4);
      kd.d_zstart.alloc(kd.zstart.size() * 4);
      kd.d_rowrange.alloc(kd.rowrange.size() * 4);
      kd.d_kin64.alloc(npw * 8);
      kd.d_kin32.alloc(npw * 4);
      kd.d_q.alloc(3 * npw * 8);
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_miller.p, kd.miller.data(), kd.miller.size() * 4, cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_offset.p, off.data(), npw * 4, cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_tileidx.p, tile.data(), npw * 4, cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_zstart.p, kd.zstart.data(), kd.zstart.size() * 4, cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_rowrange.p, kd.rowrange.data(), kd.rowrange.size() * 4, cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_kin64.p, kin.data(), npw * 8, cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_kin32.p, kin32.data(), npw * 4, cudaMemcpyHostToDevice));
      KSS_CHECK_CUDA(cudaMemcpy(kd.d_q.p, q.data(), 3 * npw * 8, cudaMemcpyHostToDevice));
      double nl = 0;
      if (s->nproj) {
        kd.d_beta64.alloc((size_t)npw * s->nproj * 16);
        kd.d_beta32.alloc((size_t)npw * s->nproj * 8);
        launch_projectors(s.get(), kd, ctx->stream);
        convert_f64_to_f32(kd.d_beta64.as<double>(), kd.d_beta32.as<float>(),
                           (size_t)npw * s->nproj * 2, ctx->stream);
        projector_norms(kd.d_beta64.as<double>(), npw, s->nproj, kd.beta_norm2, ctx->stream);
        for (int i = 0; i < s->nproj; ++i) nl += std::max(s->D[i], 0.0) * kd.beta_norm2[i];
      }
      kd.bound = kd.tmax + std::max(s->vmax, 0.0) + nl;
    }
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    overlap_setup(s.get());  // per-k W = Q (1 + G Q)^-1 and the filter bound (bound_f = bound without Q)
    KSS_CHECK_CUDA(cudaGetLastError());
    ctx->nsys += 1;
    *out = s.release();
  });
}

kss_status kss_sys_destroy(kss_sys sys) {
  if (!sys) return KSS_EINVAL;
  kss_ctx ctx = sys->ctx;
  if (sys->nsolvers > 0) {
    ctx->err = "destroy every solver of a system before the system";
    return KSS_EINVAL;
  }
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  delete sys;
  ctx->nsys -= 1;
  return KSS_OK;
}

kss_status kss_sys_info_get(kss_sys sys, kss_sys_info* out) {
  if (!sys || !out) return KSS_EINVAL;
  out->nk = (int)sys->k.size();
  for (int i = 0; i < 3; ++i) out->fft_box[i] = sys->N[i];
  out->nproj = sys->nproj;
  int m = 0;
  for (auto& kd : sys->k) m = std::max(m, kd.npw);
  out->npw_max = m;
  out->volume = sys->vol;
  out->vloc_max = sys->vmax;
  return KSS_OK;
}

kss_status kss_sphere(kss_sys sys, int ik, int* npw, const int32_t** miller_host) {
  if (!sys || !npw) return KSS_EINVAL;
  if (ik < 0 || ik >= (int)sys->k.size()) {
    sys->ctx->err = "k-point index out of range";
    return KSS_EINVAL;
  }
  *npw = sys->k[ik].npw;
  if (miller_host) *miller_host = sys->k[ik].miller.data();
  return KSS_OK;
}

kss_status kss_get_maps(kss_sys sys, int ik, int32_t* miller_out, int32_t* offset_out) {
  if (!sys) return KSS_EINVAL;
  return guard(sys->ctx, [&] {
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KData& kd = sys->k[ik];
    KSS_CHECK_CUDA(cudaSetDevice(sys->ctx->device));
    KSS_CHECK_CUDA(cudaStreamSynchronize(sys->ctx->stream));
    if (miller_out)
      KSS_CHECK_CUDA(cudaMemcpy(miller_out, kd.d_miller.p, (size_t)kd.npw * 12, cudaMemcpyDeviceToHost));
    if (offset_out)
      KSS_CHECK_CUDA(cudaMemcpy(offset_out, kd.d_offset.p, (size_t)kd.npw * 4, cudaMemcpyDeviceToHost));
  });
}

kss_status kss_get_tables(kss_sys sys, int ik, double* vloc_out, double* kinetic_out,
                          double* beta_out) {
  if (!sys) return KSS_EINVAL;
  return guard(sys->ctx, [&] {
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KData& kd = sys->k[ik];
    KSS_CHECK_CUDA(cudaSetDevice(sys->ctx->device));
    KSS_CHECK_CUDA(cudaStreamSynchronize(sys->ctx->stream));
    if (vloc_out)
      KSS_CHECK_CUDA(cudaMemcpy(vloc_out, sys->d_V64.p, sys->d_V64.bytes, cudaMemcpyDeviceToHost));
    if (kinetic_out)
      KSS_CHECK_CUDA(cudaMemcpy(kinetic_out, kd.d_kin64.p, (size_t)kd.npw * 8, cudaMemcpyDeviceToHost));
    if (beta_out && sys->nproj)
      KSS_CHECK_CUDA(cudaMemcpy(beta_out, kd.d_beta64.p, kd.d_beta64.bytes, cudaMemcpyDeviceToHost));
  });
}

kss_status kss_upper_bound(kss_sys sys, int ik, double* bound) {
  if (!sys || !bound) return KSS_EINVAL;
  if (ik < 0 || ik >= (int)sys->k.size()) return KSS_EINVAL;
  *bound = sys->k[ik].bound;
  return KSS_OK;
}

kss_status kss_apply_H(kss_sys sys, int ik, int nb, const void* psi, void* hpsi, int ld,
                       kss_precision prec) {
  if (!sys) return KSS_EINVAL;
  return guard(sys->ctx, [&] {
    KSS_NVTX("apply_H");
    KSS_CHECK_CUDA(cudaSetDevice(sys->ctx->device));
    apply_h(sys, ik, nb, psi, nullptr, hpsi, ld, ChebCoef{1.0, 0.0, 0.0}, prec);
  });
}

kss_status kss_cheb_step(kss_sys sys, int ik, int nb, const void* psi, const void* psi_prev,
                         void* out, int ld, double alpha, double beta, double gamma,
                         kss_precision prec) {
  if (!sys) return KSS_EINVAL;
  return guard(sys->ctx, [&] {
    KSS_CHECK_CUDA(cudaSetDevice(sys->ctx->device));
    apply_filter_op(sys, ik, nb, psi, psi_prev, out, ld, ChebCoef{alpha, beta, psi_prev ? gamma : 0.0},
                    prec);
  });
}

kss_status kss_apply_H_gamma(kss_sys sys, int ik, int nb, const void* psi, void* hpsi, int ld,
                             kss_precision prec) {
  if (!sys) return KSS_EINVAL;
  return guard(sys->ctx, [&] {
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(sys->k[ik].gamma, "kss_apply_H_gamma needs the Gamma point");
    KSS_CHECK_CUDA(cudaSetDevice(sys->ctx->device));
    ChebCoef c{1.0, 0.0, 0.0};
    c.packed = true;
    apply_h(sys, ik, nb, psi, nullptr, hpsi, ld, c, prec);
  });
}

kss_status kss_apply_S(kss_sys sys, int ik, int nb, const void* psi, void* spsi, int ld,
                       kss_precision prec) {
  if (!sys) return KSS_EINVAL;
  return guard(sys->ctx, [&] {
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(nb >= 0, "nb < 0");
    KSS_REQUIRE(prec == KSS_PREC_FP64 || prec == KSS_PREC_MIXED, "unknown precision");
    KSS_REQUIRE(ld >= sys->k[ik].npw, "ld < npw");
    if (nb == 0) return;
    KSS_REQUIRE(psi && spsi && psi != spsi, "null or overlapping psi / spsi");
    KSS_CHECK_CUDA(cudaSetDevice(sys->ctx->device));
    apply_s(sys->ctx, sys, ik, nb, psi, spsi, ld, prec);
  });
}

kss_status kss_apply_H_host(kss_sys sys, int ik, int nb, const void* psi_host, void* hpsi_host,
                            int ld, kss_precision prec) {
  if (!sys) return KSS_EINVAL;
  kss_ctx ctx = sys->ctx;
  return guard(ctx, [&] {
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(nb >= 0 && ld >= sys->k[ik].npw, "bad nb or ld");
    if (nb == 0) return;
    KSS_REQUIRE(psi_host && hpsi_host, "null buffer");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    const size_t bytes = (size_t)nb * ld * (prec == KSS_PREC_FP64 ? 16 : 8);
    ctx->stage_in.ensure(bytes);
    ctx->stage_out.ensure(bytes);
    KSS_CHECK_CUDA(cudaMemcpyAsync(ctx->stage_in.p, psi_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    apply_h(sys, ik, nb, ctx->stage_in.p, nullptr, ctx->stage_out.p, ld, ChebCoef{1.0, 0.0, 0.0},
            prec);
    KSS_CHECK_CUDA(cudaMemcpyAsync(hpsi_host, ctx->stage_out.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  });
}

kss_status kss_gemm(kss_ctx ctx, int op, int M, int N, int K, const void* A, int lda, const void* B,
                    int ldb, void* C, int ldc, double alpha_re, double alpha_im, double beta_re,
                    double beta_im, kss_precision prec) {
  if (!ctx) return KSS_EINVAL;
  return guard(ctx, [&] {
    KSS_REQUIRE(op == 0 || op == 1, "op must be 0 (A^H B) or 1 (A B)");
    KSS_REQUIRE(M >= 0 && N >= 0 && K >= 0, "negative size");
    KSS_REQUIRE(prec == KSS_PREC_FP64 || prec == KSS_PREC_MIXED, "unknown precision");
    if (M == 0 || N == 0) return;
    KSS_REQUIRE(A && B && C, "null matrix");
    KSS_REQUIRE(ldc >= M && (op == 0 ? (lda >= K && ldb >= K) : (lda >= M && ldb >= K)),
                "bad leading dimension");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    if (prec == KSS_PREC_FP64) {
      if (K == 0) {  // C = beta C
        gemm_cn(ctx, true, M, N, K, A, lda, B, ldb, C, ldc, alpha_re, alpha_im, beta_re, beta_im, "user");
        return;
      }
      if (op == 0) oz_gemm_cn(ctx, M, N, K, A, lda, B, ldb, C, ldc, alpha_re, alpha_im, beta_re, beta_im, "user");
      else oz_gemm_nn(ctx, M, N, K, A, lda, B, ldb, C, ldc, alpha_re, alpha_im, beta_re, beta_im, "user");
      if (tc_error_flag(ctx, true)) fail(KSS_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up");
    } else {
      KSS_REQUIRE(K > 0 || (beta_re == 0 && beta_im == 0), "K == 0 with beta != 0 is not supported");
      if (K == 0) {
        KSS_CHECK_CUDA(cudaMemset2DAsync(C, (size_t)ldc * 8, 0, (size_t)M * 8, N, ctx->stream));
        return;
      }
      if (op == 0) tc_gemm_cn(ctx, M, N, K, A, lda, B, ldb, C, ldc, alpha_re, alpha_im, beta_re, beta_im, "user");
      else tc_gemm_nn(ctx, M, N, K, A, lda, B, ldb, C, ldc, alpha_re, alpha_im, beta_re, beta_im, "user");
      if (tc_error_flag(ctx, true)) fail(KSS_ETIMEOUT, "tensor-core GEMM: a bounded wait gave up");
    }
  });
}

// ---- host-only queries (no context, no device) ----

static bool host_cell_ok(const double* lattice, double ecut, double* B) {
  if (!lattice || !(ecut > 0) || !std::isfinite(ecut)) return false;
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(lattice[i])) return false;
  double vol = 0.0;
  reciprocal(lattice, B, &vol);
  return std::isfinite(vol) && vol > 0;
}

kss_status kss_sphere_host(const double* lattice, double ecut, const double* kred, int cap, int* npw,
                           int32_t* miller) {
  if (!npw || !kred) return KSS_EINVAL;
  double B[9];
  if (!host_cell_ok(lattice, ecut, B)) return KSS_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(kred[i])) return KSS_EINVAL;
  try {
    std::vector<int32_t> m;
    enumerate_sphere(lattice, B, ecut, kred, m);
    *npw = (int)(m.size() / 3);
    if (miller) {
      if (cap < *npw) return KSS_EINVAL;
      std::memcpy(miller, m.data(), m.size() * sizeof(int32_t));
    }
    return KSS_OK;
  } catch (const std::bad_alloc&) {
    return KSS_ENOMEM;
  }
}

kss_status kss_default_box(const double* lattice, double ecut, int nk, const double* kpts_red, int* box) {
  if (!box || nk < 1 || !kpts_red) return KSS_EINVAL;
  double B[9];
  if (!host_cell_ok(lattice, ecut, B)) return KSS_EINVAL;
  try {
    int mmax[3] = {0, 0, 0};
    std::vector<int32_t> m;
    for (int ik = 0; ik < nk; ++ik) {
      for (int i = 0; i < 3; ++i)
        if (!std::isfinite(kpts_red[3 * ik + i])) return KSS_EINVAL;
      enumerate_sphere(lattice, B, ecut, kpts_red + 3 * ik, m);
      for (size_t g = 0; g < m.size(); ++g) mmax[g % 3] = std::max(mmax[g % 3], std::abs(m[g]));
    }
    for (int i = 0; i < 3; ++i) box[i] = default_box_edge(mmax[i]);
    return KSS_OK;
  } catch (const std::bad_alloc&) {
    return KSS_ENOMEM;
  }
}

kss_status kss_selftest_bounded_wait(kss_ctx ctx, double limit_ms) {
  if (!ctx) return KSS_EINVAL;
  return guard(ctx, [&] {
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    tc_wait_selftest(ctx, limit_ms);
    if (tc_error_flag(ctx, true)) fail(KSS_ETIMEOUT, "bounded device wait gave up (self-test)");
  });
}

}  // extern "C"

namespace kss {
// Device bytes held by a system's tables (V grids and views, twiddles, D, and every k-point's
// sphere maps, kinetic energies and projector tables, including the lazily built split forms
// present so far).
size_t sys_device_bytes(kss_sys s) {
  size_t b = s->d_V64.bytes + s->d_Vx64.bytes + s->d_Vx32.bytes + s->d_D64.bytes + s->d_D32.bytes +
             s->d_Q64.bytes + s->d_Q32.bytes;
  for (int i = 0; i < 3; ++i) b += s->d_tw64[i].bytes + s->d_tw32[i].bytes;
  for (const auto& kv : s->vpi64) b += kv.second.bytes;
  for (const auto& kv : s->vpi32) b += kv.second.bytes;
  for (const auto& kv : s->vfused32) b += kv.second.bytes;
  for (const KData& kd : s->k) {
    const DevBuf* bufs[] = {&kd.d_miller, &kd.d_offset, &kd.d_tileidx, &kd.d_zstart, &kd.d_rowrange,
                            &kd.d_kin64,  &kd.d_kin32,  &kd.d_beta64,  &kd.d_beta32, &kd.d_btc_cn,
                            &kd.d_btc_nn, &kd.d_oz_cn,  &kd.d_oz_nn,   &kd.d_q,      &kd.d_mirror,
                            &kd.d_G64,    &kd.d_G32,    &kd.d_W64,     &kd.d_W32};
    for (const DevBuf* d : bufs) b += d->bytes;
  }
  return b;
}
}  // namespace kss

extern "C" {

kss_status kss_footprint(kss_sys sys, int nband, kss_precision prec, size_t* bytes) {
  if (!sys || !bytes || nband < 1) return KSS_EINVAL;
  size_t m = 0;
  const size_t es = prec == KSS_PREC_FP64 ? 16 : 8;
  for (size_t ik = 0; ik < sys->k.size(); ++ik) {
    const int npw = sys->k[ik].npw;
    const int nb = std::min(npw, nband + std::max(4, (nband + 9) / 10));
    size_t b = 4 * (size_t)npw * nb * es;                       // four band blocks
    if (prec == KSS_PREC_MIXED) b += 2 * (size_t)npw * nb * 16; // FP64 refinement blocks
    b += 3 * (size_t)nb * nb * 16;                              // Gram / projected H / work
    if (sys->has_S) b += 2 * (size_t)npw * nb * es;             // S Y / S X block, L psi scratch
    if (prec == KSS_PREC_MIXED && sys->nproj)                   // split-BF16 projector tables
      b += tc_split_cn_bytes(sys->nproj, npw) + tc_split_nn_bytes(npw, sys->nproj);
    b += local_workspace_bytes(sys, (int)ik, nb, prec);
    // V in the CTA-wide pass B's layout (one split per precision in use)
    b += (size_t)sys->N[0] * sys->N[1] * sys->N[2] * (prec == KSS_PREC_FP64 ? 8 : 12);
    m = std::max(m, b);
  }
  *bytes = m;
  return KSS_OK;
}

}  // extern "C"

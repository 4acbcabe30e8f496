// Device-side setup: local potential on the FFT grid, its plane-kernel views, the projector
// table (Eq. ham-nl of §5.2 with projectors kept in memory) and small reductions.
#include <cmath>

#include "kss_internal.h"

namespace kss {

namespace {

struct Lat {
  double a[9];  // rows a1, a2, a3
  double b[9];  // rows b1, b2, b3 (a_i . b_j = 2 pi delta_ij)
};

// V(r_j) = A sum_a sum_L exp(-|r_j - R_a - L|^2 / (2 sigma^2)).  For every atom the images are
// enumerated around the nearest one, far enough along each lattice direction to reach every
// image within rcut; images farther than rcut (terms < 1e-20 |A|) are skipped.
__global__ void vloc_kernel(Lat L, int N1, int N2, int N3, const double* __restrict__ pos,
                            int natom, double amp, double inv2s2, double rcut2, int e1, int e2,
                            int e3, double* __restrict__ V) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)N1 * N2 * N3;
  if (idx >= n) return;
  const int j1 = (int)(idx % N1);
  const int j2 = (int)((idx / N1) % N2);
  const int j3 = (int)(idx / ((long long)N1 * N2));
  const double f1 = (double)j1 / N1, f2 = (double)j2 / N2, f3 = (double)j3 / N3;
  const double rx = f1 * L.a[0] + f2 * L.a[3] + f3 * L.a[6];
  const double ry = f1 * L.a[1] + f2 * L.a[4] + f3 * L.a[7];
  const double rz = f1 * L.a[2] + f2 * L.a[5] + f3 * L.a[8];
  const double inv2pi = 0.15915494309189535;
  double sum = 0.0;
  for (int at = 0; at < natom; ++at) {
    const double dx = rx - pos[3 * at], dy = ry - pos[3 * at + 1], dz = rz - pos[3 * at + 2];
    const double s1 = (dx * L.b[0] + dy * L.b[1] + dz * L.b[2]) * inv2pi;
    const double s2 = (dx * L.b[3] + dy * L.b[4] + dz * L.b[5]) * inv2pi;
    const double s3 = (dx * L.b[6] + dy * L.b[7] + dz * L.b[8]) * inv2pi;
    const int c1 = (int)rint(s1), c2 = (int)rint(s2), c3 = (int)rint(s3);
    for (int n1 = c1 - e1; n1 <= c1 + e1; ++n1)
      for (int n2 = c2 - e2; n2 <= c2 + e2; ++n2)
        for (int n3 = c3 - e3; n3 <= c3 + e3; ++n3) {
          const double ex = dx - (n1 * L.a[0] + n2 * L.a[3] + n3 * L.a[6]);
          const double ey = dy - (n1 * L.a[1] + n2 * L.a[4] + n3 * L.a[7]);
          const double ez = dz - (n1 * L.a[2] + n2 * L.a[5] + n3 * L.a[8]);
          const double d2 = ex * ex + ey * ey + ez * ez;
          if (d2 <= rcut2) sum += exp(-d2 * inv2s2);
        }
  }
  V[idx] = amp * sum;
}

// Vx[(j1*N2 + j2)*N3 + j3] = V[(j3*N2 + j2)*N1 + j1] * scale  (x-major view for the plane kernel)
template <typename T>
__global__ void vloc_view_kernel(const double* __restrict__ V, T* __restrict__ Vx, int N1, int N2,
                                 int N3, double scale) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)N1 * N2 * N3;
  if (idx >= n) return;
  const int j3 = (int)(idx % N3);
  const int j2 = (int)((idx / N3) % N2);
  const int j1 = (int)(idx / ((long long)N3 * N2));
  Vx[idx] = (T)(V[((long long)j3 * N2 + j2) * N1 + j1] * scale);
}

__global__ void max_kernel(const double* __restrict__ x, long long n, double* out) {
  __shared__ double red[1024];
  double m = -INFINITY;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// beta_{a,l}(g) = c_l q_l exp(-alpha |q|^2) exp(-i q.R_a), projector-major [4a+l][g].
__global__ void projector_kernel(const double* __restrict__ q, int npw, const double* __restrict__ pos,
                                 int natom, int nppa, double alpha, double cs, double cp,
                                 double2* __restrict__ beta) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int at = blockIdx.y;
  if (g >= npw) return;
  const double qx = q[3 * g], qy = q[3 * g + 1], qz = q[3 * g + 2];
  const double q2 = qx * qx + qy * qy + qz * qz;
  const double gs = exp(-alpha * q2);
  const double ph = qx * pos[3 * at] + qy * pos[3 * at + 1] + qz * pos[3 * at + 2];
  double sn, cn;
  sincos(ph, &sn, &cn);
  const double re = cn, im = -sn;  // e^{-i q.R}
  const long long base = (long long)(nppa * at) * npw + g;
  const double s0 = cs * gs;
  beta[base] = make_double2(s0 * re, s0 * im);
  if (nppa == 4) {
    const double p = cp * gs;
    beta[base + npw] = make_double2(p * qx * re, p * qx * im);
    beta[base + 2LL * npw] = make_double2(p * qy * re, p * qy * im);
    beta[base + 3LL * npw] = make_double2(p * qz * re, p * qz * im);
  }
}

__global__ void norm2_kernel(const double2* __restrict__ beta, int npw, double* __restrict__ out) {
  __shared__ double red[256];
  const double2* b = beta + (long long)blockIdx.x * npw;
  double s = 0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s += b[g].x * b[g].x + b[g].y * b[g].y;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

}  // namespace

void launch_vloc(kss_sys s, cudaStream_t st) {
  Lat L;
  for (int i = 0; i < 9; ++i) {
    L.a[i] = s->lat[i];
    L.b[i] = s->B[i];
  }
  const double rcut = s->vsig * std::sqrt(2.0 * std::log(1e20));
  int e[3];
  for (int i = 0; i < 3; ++i) {
    const double bn = std::sqrt(s->B[3 * i] * s->B[3 * i] + s->B[3 * i + 1] * s->B[3 * i + 1] +
                                s->B[3 * i + 2] * s->B[3 * i + 2]);
    const double h = 2.0 * 3.141592653589793 / bn;  // spacing of lattice planes
    e[i] = (int)std::ceil(rcut / h + 0.5);
  }
  DevBuf dpos;
  if (s->natom) {
    dpos.alloc(s->pos.size() * sizeof(double));
    KSS_CHECK_CUDA(cudaMemcpy(dpos.p, s->pos.data(), s->pos.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  const long long n = (long long)s->N[0] * s->N[1] * s->N[2];
  vloc_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      L, s->N[0], s->N[1], s->N[2], dpos.as<double>(), s->natom, s->vamp,
      1.0 / (2.0 * s->vsig * s->vsig), rcut * rcut, e[0], e[1], e[2], s->d_V64.as<double>());
  KSS_CHECK_CUDA(cudaGetLastError());
  KSS_CHECK_CUDA(cudaStreamSynchronize(st));  // dpos is freed on return
}

void launch_vloc_views(kss_sys s, cudaStream_t st) {
  const long long n = (long long)s->N[0] * s->N[1] * s->N[2];
  const double scale = 1.0 / (double)n;
  vloc_view_kernel<double><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      s->d_V64.as<double>(), s->d_Vx64.as<double>(), s->N[0], s->N[1], s->N[2], scale);
  vloc_view_kernel<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      s->d_V64.as<double>(), s->d_Vx32.as<float>(), s->N[0], s->N[1], s->N[2], scale);
  KSS_CHECK_CUDA(cudaGetLastError());
}

double device_max(const double* x, size_t n, cudaStream_t st) {
  DevBuf out;
  out.alloc(sizeof(double));
  max_kernel<<<1, 1024, 0, st>>>(x, (long long)n, out.as<double>());
  KSS_CHECK_CUDA(cudaGetLastError());
  double h = 0;
  KSS_CHECK_CUDA(cudaMemcpyAsync(&h, out.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  KSS_CHECK_CUDA(cudaStreamSynchronize(st));
  return h;
}

void launch_projectors(kss_sys s, KData& kd, cudaStream_t st) {
  const double pi = 3.141592653589793;
  const double cs = std::sqrt(std::pow(2.0 * pi, 3.0) * std::pow(2.0 * s->alpha / pi, 1.5) / s->vol);
  const double cp = cs * std::sqrt(4.0 * s->alpha);
  DevBuf dpos;
  dpos.alloc(s->pos.size() * sizeof(double));
  KSS_CHECK_CUDA(cudaMemcpy(dpos.p, s->pos.data(), s->pos.size() * sizeof(double), cudaMemcpyHostToDevice));
  dim3 grid((kd.npw + 127) / 128, s->natom);
  projector_kernel<<<grid, 128, 0, st>>>(kd.d_q.as<double>(), kd.npw, dpos.as<double>(), s->natom,
                                         s->nppa, s->alpha, cs, cp, kd.d_beta64.as<double2>());
  KSS_CHECK_CUDA(cudaGetLastError());
  KSS_CHECK_CUDA(cudaStreamSynchronize(st));
}

void projector_norms(const double* beta, int npw, int nproj, std::vector<double>& out,
                     cudaStream_t st) {
  DevBuf d;
  d.alloc(nproj * sizeof(double));
  norm2_kernel<<<nproj, 256, 0, st>>>((const double2*)beta, npw, d.as<double>());
  KSS_CHECK_CUDA(cudaGetLastError());
  out.assign(nproj, 0.0);
  KSS_CHECK_CUDA(cudaMemcpyAsync(out.data(), d.p, nproj * sizeof(double), cudaMemcpyDeviceToHost, st));
  KSS_CHECK_CUDA(cudaStreamSynchronize(st));
}

void convert_f64_to_f32(const double* in, float* out, size_t n, cudaStream_t st) {
  if (!n) return;
  f64_to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, (long long)n);
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace kss

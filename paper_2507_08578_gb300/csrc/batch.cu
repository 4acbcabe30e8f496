// Batched Chebyshev-filtered solves: many (system, k-point) units of uneven sizes advanced in
// lockstep, the local passes and the projector products of all units issued as single grouped
// launches, and the whole filter of one iteration (degree m applications plus H on the filtered
// block) captured once into a CUDA graph and replayed every iteration.  The paper batches many
// FFTs and products per call over bands (§5.1); here the batch extends to independent problems
// (k-points and systems share nothing, §5.3 notes the trivial parallelism in k).
//
// Per iteration and unit the filter reads its coefficients and buffer roles from device tables
// that the host rewrites before each replay; Rayleigh-Ritz (FP64 eigensolve) is then issued for
// every unit with a single host synchronisation for the convergence decisions.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>


#include "batch.h"
#include "batch_kernels.cuh"
#include "local_fused.h"
#include "local_kernels.cuh"
#include "tune.h"

namespace kss {

namespace {

using namespace lk;
using namespace bk;
using fftr::Split;

// Shared memory of the CTA-wide pass B for box length N and sphere window W3.
size_t wide_b_smem(int N, int W3, size_t es) {
  const size_t P = (size_t)((N + 1) | 1);  // the odd pitches of the CTA-wide form
  return es * ((size_t)N + (size_t)W3 * P + (size_t)N * P) + sizeof(int) * N;
}

bool has_ct(int code) {
  switch (code) {
#define KSS_CASE(x, y) case x * 32 + y:
    KSS_SPLITS(KSS_CASE)
#undef KSS_CASE
    return true;
    default:
      return false;
  }
}

// Kernel instance of one grouped pass for a split code (-1: runtime-sized transforms).
template <typename T, int PASS>
GroupKernel<T> group_kernel(int code) {
  if constexpr (sizeof(T) == 4) {
    switch (code) {
#define KSS_CASE(x, y) \
  case x * 32 + y:     \
    return group_pass<T, PASS, CtPol<x, y>>;
      KSS_SPLITS(KSS_CASE)
#undef KSS_CASE
      default:
        break;
    }
  }
  return group_pass<T, PASS, RtPol>;
}

template <typename T>
void fill_args(kss_sys s, int ik, LocalArgs<T>& a) {
  using C = typename CT<T>::C;
  const bool f64 = sizeof(T) == 8;
  KData& kd = s->k[ik];
  a = LocalArgs<T>{};
  a.N1 = s->N[0];
  a.N2 = s->N[1];
  a.N3 = s->N[2];
  a.N1p = a.N1 + 1;
  a.N2p = a.N2 + 1;
  a.N3p = a.N3 + 1;
  a.W2 = kd.W[1];
  a.W3 = kd.W[2];
  a.lo2 = kd.lo[1];
  a.lo3 = kd.lo[2];
  a.d1 = s->dim[0];
  a.d2 = s->dim[1];
  a.d3 = s->dim[2];
  a.tw1 = (const C*)(f64 ? s->d_tw64[0].p : s->d_tw32[0].p);
  a.tw2 = (const C*)(f64 ? s->d_tw64[1].p : s->d_tw32[1].p);
  a.tw3 = (const C*)(f64 ? s->d_tw64[2].p : s->d_tw32[2].p);
  a.zstart = kd.d_zstart.as<int>();
  a.rowrange = kd.d_rowrange.as<int>();
  a.tileidx = kd.d_tileidx.as<int>();
  a.kin = (const T*)(f64 ? kd.d_kin64.p : kd.d_kin32.p);
  a.Vx = (const T*)(f64 ? s->d_Vx64.p : s->d_Vx32.p);
  a.ld = kd.npw;
  a.n0 = 0;
}

size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }

// Copy the leading m x m block of a complex64 matrix (ld m) into a complex128 matrix (ld np).
__global__ void c64_to_c128_ld(const float2* __restrict__ in, int m, double2* __restrict__ out, int np) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)m * m) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  const float2 v = in[idx];
  out[(size_t)j * np + i] = make_double2(v.x, v.y);
}
__global__ void c128_ld_to_c64(const double2* __restrict__ in, int np, float2* __restrict__ out, int m) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)m * m) return;
  const int i = (int)(idx % m), j = (int)(idx / m);
  const double2 v = in[(size_t)j * np + i];
  out[idx] = make_float2((float)v.x, (float)v.y);
}

// One unit of the grouped Rayleigh-Ritz epilogue (single precision): eigenvectors to complex64,
// residual norms of the rotated block.
struct RrItem {
  const double2* Q;  // eigenvectors: leading nb x nb block, ld np
  float2* Q32;       // complex64 copy, ld nb
  const float2* X;   // rotated block and H times it, ld npw
  const float2* HX;
  const double* w;   // eigenvalues
  double* r;         // residual norms |H x - lambda x|
  int np, nb, npw;
  long long q0, r0;  // first block of the unit in the conversion and residual launches
};

__device__ __forceinline__ int rr_find(const RrItem* it, int n, long long b, bool res) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((res ? it[mid].r0 : it[mid].q0) <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void rr_q_to_c64(const RrItem* __restrict__ items, int n) {
  const RrItem& t = items[rr_find(items, n, blockIdx.x, false)];
  const long long idx = (blockIdx.x - t.q0) * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)t.nb * t.nb) return;
  const int i = (int)(idx % t.nb), j = (int)(idx / t.nb);
  const double2 v = t.Q[(size_t)j * t.np + i];
  t.Q32[idx] = make_float2((float)v.x, (float)v.y);
}

// One block per band: |H x_n - lambda_n x_n| with FP64 accumulation.
__global__ void rr_residuals(const RrItem* __restrict__ items, int n) {
  __shared__ double red[256];
  const RrItem& t = items[rr_find(items, n, blockIdx.x, true)];
  const int band = (int)(blockIdx.x - t.r0);
  const double lam = t.w[band];
  const float2* x = t.X + (size_t)band * t.npw;
  const float2* h = t.HX + (size_t)band * t.npw;
  double s = 0;
  for (int g = threadIdx.x; g < t.npw; g += blockDim.x) {
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
  if (threadIdx.x == 0) t.r[band] = sqrt(red[0]);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// BatchEngine
// ---------------------------------------------------------------------------------------------

BatchEngine::~BatchEngine() {
  drop_graph();
  if (hstage) cudaFreeHost(hstage);
  if (cap) cudaStreamDestroy((cudaStream_t)cap);
  for (auto w : workers) {
    cudaStreamSynchronize(w->stream);
    cudaStreamDestroy(w->stream);
    delete w;
  }
  for (auto e : wev) cudaEventDestroy((cudaEvent_t)e);
  if (fork_ev) cudaEventDestroy((cudaEvent_t)fork_ev);
}

// Issue every unit's Rayleigh-Ritz on the worker streams after the work already queued on the
// context stream, then make the context stream wait for all of them.
void BatchEngine::rr_all(const std::vector<kss_solver_s*>& us, const std::vector<int>& y,
                         const std::vector<int>& hy, const std::vector<int>& xo,
                         const std::vector<int>& hxo) {
  const int kW = 8;
  if (workers.empty()) {
    for (int i = 0; i < kW; ++i) {
      kss_ctx w = new kss_ctx_s();
      w->device = ctx->device;
      cudaStream_t st = nullptr;
      KSS_CHECK_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      w->stream = st;
      workers.push_back(w);
      cudaEvent_t e = nullptr;
      KSS_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      wev.push_back(e);
    }
    cudaEvent_t f = nullptr;
    KSS_CHECK_CUDA(cudaEventCreateWithFlags(&f, cudaEventDisableTiming));
    fork_ev = f;
  }
  KSS_CHECK_CUDA(cudaEventRecord((cudaEvent_t)fork_ev, ctx->stream));
  for (auto w : workers) KSS_CHECK_CUDA(cudaStreamWaitEvent(w->stream, (cudaEvent_t)fork_ev, 0));
  for (size_t u = 0; u < us.size(); ++u) {
    kss_ctx w = workers[u % workers.size()];
    kss_solver_s* s = us[u];
    w->prof.on = false;
    rr_issue(s, s->f64, s->blk[y[u]].p, s->blk[hy[u]].p, s->blk[xo[u]].p, s->blk[hxo[u]].p, w);
  }
  for (size_t i = 0; i < workers.size(); ++i) {
    KSS_CHECK_CUDA(cudaEventRecord((cudaEvent_t)wev[i], workers[i]->stream));
    KSS_CHECK_CUDA(cudaStreamWaitEvent(ctx->stream, (cudaEvent_t)wev[i], 0));
  }
  ctx->prof.launches += 0;
}

void* BatchEngine::stage(size_t bytes) {
  if (bytes > hstage_bytes) {
    if (hstage) KSS_CHECK_CUDA(cudaFreeHost(hstage));
    hstage = nullptr;
    hstage_bytes = 0;
    KSS_CHECK_CUDA(cudaMallocHost(&hstage, bytes));
    hstage_bytes = bytes;
  }
  return hstage;
}

void BatchEngine::drop_graph() {
  if (gexec) cudaGraphExecDestroy((cudaGraphExec_t)gexec);
  gexec = nullptr;
}

void BatchEngine::set_units(const std::vector<kss_solver_s*>& us) {
  bool same = us.size() == units.size();
  for (size_t i = 0; same && i < us.size(); ++i) same = us[i] == units[i];
  if (same && prepared) return;
  units = us;
  prepared = false;
  drop_graph();
}

template <typename T>
void BatchEngine::prepare_t() {
  using C = typename CT<T>::C;
  const size_t es = sizeof(C);
  const int n = (int)units.size();
  plans.assign(n, RegPlanHost{});
  ws_off.assign(n, {0, 0, 0});
  size_t off = 0;
  scr_warp = 0;
  smem_ac = smem_b = 0;
  blocks_ac = blocks_b = 0;
  for (int u = 0; u < n; ++u) {
    kss_solver_s* s = units[u];
    kss_sys sy = s->sys;
    const KData& kd = sy->k[s->ik];
    RegPlan rp;
    if (!(choose_split(sy->N[0], rp.s1) && choose_split(sy->N[1], rp.s2) && choose_split(sy->N[2], rp.s3)))
      fail(KSS_ENOTSUP, "batched solves need FFT lengths that split into two codelets (<= 16 each)");
    static_assert(sizeof(RegPlanHost) == sizeof(RegPlan), "plan layouts differ");
    std::memcpy(&plans[u], &rp, sizeof(RegPlan));
    const int sw = std::max(rp.s1.PP * rp.s1.scr, std::max(rp.s2.PP * rp.s2.scr, rp.s3.PP * rp.s3.scr));
    scr_warp = std::max(scr_warp, sw);
    const size_t plane = (size_t)sy->N[0] * kd.W[2] * kd.W[1] * es;
    ws_off[u].cprj = off;
    off += al256((size_t)std::max(sy->nproj, 1) * s->nb * es);
    ws_off[u].part = off;
    off += al256((size_t)16 * std::max(sy->nproj, 1) * s->nb * es);
    ws_off[u].slab = off;
    off += al256(plane * s->nb);
    blocks_ac += kd.W[2] * s->nb;
    blocks_b += sy->N[0] * s->nb;
  }
  // Units grouped by kernel instance: the x split code of passes A/C and the pass-B schedule the
  // autotuner picks for the unit's box and window (CTA-wide split and threads, or the per-warp
  // form with its split code).
  std::vector<std::pair<long long, int>> key(n);
  std::vector<PassBSched> bs(n);
  for (int u = 0; u < n; ++u) {
    const RegPlanHost& p = plans[u];
    int c1 = -1, c23 = -1;
    c1 = has_ct(p.s1.A * 32 + p.s1.B) ? p.s1.A * 32 + p.s1.B : -1;
    if (p.s2.A == p.s3.A && p.s2.B == p.s3.B && has_ct(p.s2.A * 32 + p.s2.B)) c23 = p.s2.A * 32 + p.s2.B;
    LocalArgs<T> au;
    fill_args<T>(units[u]->sys, units[u]->ik, au);
    RegPlan rp;
    std::memcpy(&rp, &p, sizeof(RegPlan));
    bs[u] = pass_b_schedule<T>(ctx, au, rp.s2, true);
    if (bs[u].threads && (!group_kernel_w<T>(bs[u].A, bs[u].B, bs[u].threads) ||
                          wide_b_smem(au.N2, au.W3, es) > 227 * 1024 || au.N2 != au.N3))
      bs[u].threads = 0;
    const long long k2 = bs[u].threads ? 10001 + (long long)(bs[u].A * 32 + bs[u].B) * 3 + bs[u].threads / 128 - 1
                                       : (long long)(c23 + 1);
    key[u] = {(long long)(c1 + 1) * 100000 + k2, u};
    if (sizeof(T) == 4 && fused_code(units[u]->sys)) key[u].first = -100000 + fused_code(units[u]->sys);
  }
  vpi.assign(n, nullptr);
  for (int u = 0; u < n; ++u) {
    if (key[u].first < 0) vpi[u] = fused_potential_view(units[u]->sys);
    else if (bs[u].threads) vpi[u] = vpi_view(units[u]->sys, bs[u].A, bs[u].B, sizeof(T) == 8);
  }
  std::stable_sort(key.begin(), key.end());
  pos.assign(n, 0);
  classes.clear();
  for (int i = 0; i < n; ++i) {
    const int u = key[i].second;
    pos[u] = i;
    const RegPlanHost& p = plans[u];
    const int c1 = (int)(key[i].first / 100000) - 1;
    const int c23 = (p.s2.A == p.s3.A && p.s2.B == p.s3.B && has_ct(p.s2.A * 32 + p.s2.B)) ? p.s2.A * 32 + p.s2.B : -1;
    const PassBSched& b = bs[u];
    if (classes.empty() || i == 0 || key[i].first != key[i - 1].first) {
      classes.push_back(PassClass{c1, b.threads ? -1 : c23, i, 0, 0, 0, 0, 0, 0, b.A, b.B, b.threads});
      if (key[i].first < 0) classes.back().fcode = (int)(key[i].first + 100000);
    }
    PassClass& pc = classes.back();
    kss_sys sy = units[u]->sys;
    const KData& kd = sy->k[units[u]->ik];
    pc.count += 1;
    if (pc.fcode) {  // the fused class launches none of the three passes
      pc.ftasks += units[u]->nb;
      pc.smem_f = std::max(pc.smem_f, fused_smem_bytes(sy));
      continue;
    }
    pc.blocks_ac += kd.W[2] * units[u]->nb;
    pc.blocks_b += sy->N[0] * units[u]->nb;
    pc.smem_ac = std::max(pc.smem_ac, es * ((size_t)sy->N[0] + (size_t)kd.W[1] * (sy->N[0] + 1) + (size_t)kWarps * scr_warp));
    if (pc.wnt)
      pc.smem_bw = std::max(pc.smem_bw, wide_b_smem(sy->N[1], kd.W[2], es));
    else
      pc.smem_b = std::max(pc.smem_b, es * ((size_t)sy->N[1] + sy->N[2] + (size_t)kd.W[2] * (sy->N[1] + 1) +
                                            (size_t)kWarps * scr_warp) + sizeof(int) * sy->N[2]);
    smem_ac = std::max(smem_ac, pc.smem_ac);
    smem_b = std::max(smem_b, std::max(pc.smem_b, pc.smem_bw));
  }
  if (smem_ac > 227 * 1024 || smem_b > 227 * 1024)
    fail(KSS_ENOTSUP, "a batched unit's FFT tiles do not fit in shared memory");
  ws.ensure(off);
  steps = cur_degree + 1;
  litem_bytes = sizeof(LocalItem<T>);
  h_local.assign((size_t)steps * n * litem_bytes, 0);
  h_cn.assign((size_t)steps * n, GemmItem{});
  h_nn.assign((size_t)steps * n, GemmItem{});
  d_local.ensure(h_local.size());
  d_cn.ensure(h_cn.size() * sizeof(GemmItem));
  d_nn.ensure(h_nn.size() * sizeof(GemmItem));
  // Several classes can share a kernel instance (same x split, different pass-B schedule): each
  // instance's dynamic shared-memory limit is the largest any of its classes launches with.
  std::map<const void*, size_t> need;
  auto want = [&](GroupKernel<T> k, size_t bytes) {
    size_t& v = need[(const void*)k];
    v = std::max(v, bytes);
  };
  for (const PassClass& pc : classes) {
    if (pc.fcode) {
      fused_group_prepare(ctx, pc.fcode, pc.smem_f);
      continue;
    }
    want(group_kernel<T, 0>(pc.code1), pc.smem_ac);
    want(group_kernel<T, 2>(pc.code1), pc.smem_ac);
    if (pc.wnt) want(group_kernel_w<T>(pc.wa, pc.wb, pc.wnt), pc.smem_bw);
    else want(group_kernel<T, 1>(pc.code23), pc.smem_b);
  }
  for (const auto& kv : need)
    KSS_CHECK_CUDA(cudaFuncSetAttribute(kv.first, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kv.second));
  // Single precision: the projector products as grouped split-BF16 tensor-core products.
  tc_on = false;
  tc_i.assign(n, -1);
  if (sizeof(T) == 4 && use_tc_gemm) {
    std::vector<TcGroupSpec> cs, ns;
    for (int u = 0; u < n; ++u) {
      kss_solver_s* s = units[u];
      kss_sys sy = s->sys;
      const KData& kd = sy->k[s->ik];
      if (!sy->nproj) continue;
      tc_i[u] = (int)cs.size();
      cs.push_back(TcGroupSpec{beta_split_cn(sy, s->ik), sy->nproj, s->nb, kd.npw, kd.npw, sy->nproj,
                               sy->d_D32.as<float>()});
      ns.push_back(TcGroupSpec{beta_split_nn(sy, s->ik), kd.npw, s->nb, sy->nproj, sy->nproj, kd.npw, nullptr});
    }
    tc_cn.build(ctx, cs, steps);
    tc_nn.build(ctx, ns, steps);
    tc_on = !cs.empty();
  }
  prepared = true;
}

// Buffer roles and coefficients of every unit for the m filter steps and the H-on-Y step.
template <typename T>
void BatchEngine::fill_tables_t() {
  using C = typename CT<T>::C;
  const bool f64 = sizeof(T) == 8;
  const int n = (int)units.size();
  roles.assign(n, Roles{});
  std::vector<int> cur(n), prev(n);
  std::vector<double> sigma(n), tau(n), e(n), c(n);
  udeg.assign(n, 0);
  for (int u = 0; u < n; ++u) {
    kss_solver_s* s = units[u];
    int fr[2], nf = 0;
    for (int i = 0; i < 4; ++i)
      if (i != s->ix && i != s->ihx) fr[nf++] = i;
    cur[u] = s->ix;
    prev[u] = fr[0];
    roles[u].free2 = fr[1];
    const ChebParams cp = cheb_params(s);
    udeg[u] = std::min(cp.degree, steps - 1);
    e[u] = cp.e;
    c[u] = cp.c;
    sigma[u] = cp.sigma1;
    tau[u] = 2.0 / cp.sigma1;
  }
  // Units whose FP64 check missed the tolerance with the split-BF16 products (proj32) take the
  // FP32 CUDA-core products; the graph holds those launches only while such units exist.
  bool need_simt = !tc_on;
  for (auto* s : units) need_simt |= s->proj32 && s->sys->nproj;
  if (need_simt != simt_on) {
    simt_on = need_simt;
    drop_graph();
  }
  // block offsets restart for every class (each class is its own launch)
  std::vector<int> off_ac(n), off_b(n);
  for (const PassClass& pc : classes) {
    int bac = 0, bb = 0;
    for (int i = pc.first; i < pc.first + pc.count; ++i) {
      int u = 0;
      while (pos[u] != i) ++u;
      off_ac[u] = bac;
      off_b[u] = bb;
      if (pc.fcode) {  // the fused class numbers (unit, band) tasks
        bac += units[u]->nb;
        continue;
      }
      bac += units[u]->sys->k[units[u]->ik].W[2] * units[u]->nb;
      bb += units[u]->sys->N[0] * units[u]->nb;
    }
  }
  for (int j = 0; j < steps; ++j) {
    std::vector<GemmItem> cn(n), nn(n);
    for (int u = 0; u < n; ++u) {
      kss_solver_s* s = units[u];
      kss_sys sy = s->sys;
      const KData& kd = sy->k[s->ik];
      double al = 0, be = 0, ga = 0;
      const void* psi = nullptr;
      const void* pp = nullptr;
      void* out = nullptr;
      const int mu = udeg[u];
      const bool idle = j > mu;
      if (idle) {
        // past this unit's degree: nothing to do in this step
      } else if (j == 0) {  // Y_1 = (sigma1/e)(H - c) X
        al = sigma[u] / e[u];
        be = -al * c[u];
        ga = 0;
        psi = s->blk[cur[u]].p;
        pp = nullptr;
        out = s->blk[prev[u]].p;
        std::swap(cur[u], prev[u]);
      } else if (j < mu) {  // Y_j from Y_{j-1}, Y_{j-2}, written over Y_{j-2}
        const double sn = 1.0 / (tau[u] - sigma[u]);
        al = 2.0 * sn / e[u];
        be = -al * c[u];
        ga = -sigma[u] * sn;
        psi = s->blk[cur[u]].p;
        pp = s->blk[prev[u]].p;
        out = s->blk[prev[u]].p;
        std::swap(cur[u], prev[u]);
        sigma[u] = sn;
      } else {  // HY = H Y_m into the Y_{m-1} buffer
        al = 1.0;
        be = 0.0;
        ga = 0.0;
        psi = s->blk[cur[u]].p;
        pp = nullptr;
        out = s->blk[prev[u]].p;
        roles[u].y = cur[u];
        roles[u].hy = prev[u];
      }
      LocalItem<T> it;
      fill_args<T>(sy, s->ik, it.a);
      it.a.Vpi = (const T*)vpi[u];
      it.a.nbands = s->nb;
      it.a.psi = (const C*)psi;
      it.a.psi_prev = (const C*)pp;
      it.a.out = (C*)out;
      it.a.alpha = (T)al;
      it.a.beta = (T)be;
      it.a.gamma = (T)ga;
      it.a.work = (C*)((char*)ws.p + ws_off[u].slab);
      std::memcpy(&it.rp, &plans[u], sizeof(RegPlan));
      it.blk_ac = off_ac[u];
      it.blk_b = off_b[u];
      it.idle = idle ? 1 : 0;
      std::memcpy(&h_local[((size_t)j * n + pos[u]) * litem_bytes], &it, sizeof(it));
      GemmItem& g = cn[u];
      g = GemmItem{};
      GemmItem& h = nn[u];
      h = GemmItem{};
      const bool on_tc = tc_on && tc_i[u] >= 0 && !s->proj32;
      g.idle = h.idle = (idle || on_tc) ? 1 : 0;
      if (sy->nproj) {
        g.M = sy->nproj;
        g.N = s->nb;
        g.K = kd.npw;
        g.A = f64 ? kd.d_beta64.p : kd.d_beta32.p;
        g.lda = kd.npw;
        g.B = psi;
        g.ldb = kd.npw;
        g.C = (char*)ws.p + ws_off[u].cprj;
        g.ldc = sy->nproj;
        g.P = (char*)ws.p + ws_off[u].part;
        g.d = f64 ? sy->d_D64.p : sy->d_D32.p;
        g.s = al;
        h.M = kd.npw;
        h.N = s->nb;
        h.K = sy->nproj;
        h.A = g.A;
        h.lda = kd.npw;
        h.B = g.C;
        h.ldb = sy->nproj;
        h.C = out;
        h.ldc = kd.npw;
        h.ar = 1.0;
        h.br = 1.0;
        if (tc_on) {
          void* cprj = (char*)ws.p + ws_off[u].cprj;
          tc_cn.set(j, tc_i[u], psi, cprj, (float)al, 0.f, idle || !on_tc);
          tc_nn.set(j, tc_i[u], cprj, out, 1.f, 1.f, idle || !on_tc);
        }
      }
    }
    int b1, r1, b2, r2;
    group_plan(ctx, cn, true, &b1, &r1);
    group_plan(ctx, nn, false, &b2, &r2);
    std::copy(cn.begin(), cn.end(), h_cn.begin() + (size_t)j * n);
    std::copy(nn.begin(), nn.end(), h_nn.begin() + (size_t)j * n);
    if (j == 0) {
      cn_blocks = b1;
      cn_rblocks = r1;
      nn_blocks = b2;
    }
  }
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_local.p, h_local.data(), h_local.size(), cudaMemcpyHostToDevice, ctx->stream));
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_cn.p, h_cn.data(), h_cn.size() * sizeof(GemmItem), cudaMemcpyHostToDevice, ctx->stream));
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_nn.p, h_nn.data(), h_nn.size() * sizeof(GemmItem), cudaMemcpyHostToDevice, ctx->stream));
  if (tc_on) {
    tc_cn.upload(ctx->stream);
    tc_nn.upload(ctx->stream);
  }
}

template <typename T>
void BatchEngine::launch_filter_t() {
  const bool f64 = sizeof(T) == 8;
  const int n = (int)units.size();
  const LocalItem<T>* dl = (const LocalItem<T>*)d_local.p;
  for (int j = 0; j < steps; ++j) {
    const GemmItem* cn = d_cn.as<GemmItem>() + (size_t)j * n;
    const GemmItem* nn = d_nn.as<GemmItem>() + (size_t)j * n;
    if (tc_on) tc_cn.launch(ctx, j, "cprj");
    if (simt_on && cn_blocks) group_gemm_cn(ctx, f64, cn, n, cn_blocks, cn_rblocks);
    static const int ida = prof_register(f64 ? "group_pass_a<f64>" : "group_pass_a<f32>");
    static const int idb = prof_register(f64 ? "group_pass_b<f64>" : "group_pass_b<f32>");
    static const int idc = prof_register(f64 ? "group_pass_c<f64>" : "group_pass_c<f32>");
    for (const PassClass& pc : classes) {
      const LocalItem<T>* it = dl + (size_t)j * n + pc.first;
      if (pc.fcode) {
        static const int idf = prof_register("group_fused<f32>");
        ProfScope ps(ctx, idf);
        if constexpr (sizeof(T) == 4) fused_group_launch(ctx, pc.fcode, it, pc.count, pc.ftasks, pc.smem_f);
        continue;
      }
      ProfScope ps(ctx, ida);
      group_kernel<T, 0>(pc.code1)<<<pc.blocks_ac, kThreads, pc.smem_ac, ctx->stream>>>(it, pc.count, scr_warp);
    }
    for (const PassClass& pc : classes) {
      const LocalItem<T>* it = dl + (size_t)j * n + pc.first;
      if (pc.fcode) continue;
      ProfScope ps(ctx, idb);
      if (pc.wnt)
        group_kernel_w<T>(pc.wa, pc.wb, pc.wnt)<<<pc.blocks_b, pc.wnt, pc.smem_bw, ctx->stream>>>(it, pc.count, scr_warp);
      else
        group_kernel<T, 1>(pc.code23)<<<pc.blocks_b, kThreads, pc.smem_b, ctx->stream>>>(it, pc.count, scr_warp);
    }
    for (const PassClass& pc : classes) {
      const LocalItem<T>* it = dl + (size_t)j * n + pc.first;
      if (pc.fcode) continue;
      ProfScope ps(ctx, idc);
      group_kernel<T, 2>(pc.code1)<<<pc.blocks_ac, kThreads, pc.smem_ac, ctx->stream>>>(it, pc.count, scr_warp);
    }
    if (tc_on) tc_nn.launch(ctx, j, "nonlocal");
    if (simt_on && nn_blocks) group_gemm_nn(ctx, f64, nn, n, nn_blocks);
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

void BatchEngine::run_filter() {
  KSS_NVTX("batch_filter");
  // The graph runs the largest effective degree among the units; a unit with a smaller one sits
  // out the remaining steps (its items are marked idle).  A change of that largest degree
  // changes the launch sequence and re-captures the graph.
  int m = 2;
  for (auto* s : units) m = std::max(m, cheb_params(s).degree);
  if (prepared && m + 1 != steps) {
    prepared = false;
    drop_graph();
  }
  cur_degree = m;
  if (!prepared) {
    if (f64) prepare_t<double>();
    else prepare_t<float>();
  }
  if (f64) fill_tables_t<double>();
  else fill_tables_t<float>();
  int per_step = (tc_on ? 4 + (tc_cn.split() ? 1 : 0) + (tc_nn.split() ? 1 : 0) : 0) +
                 (simt_on ? (cn_blocks ? 2 : 0) + (nn_blocks ? 1 : 0) : 0);
  for (const PassClass& pc : classes) per_step += pc.fcode ? 1 : 3;
  if (use_graph) {
    if (!gexec) {
      // Capture the filter launches once for this set of units; later iterations only rewrite
      // the device tables the kernels read.
      // Capture on a private stream (the legacy default stream cannot be captured); the graph
      // is then launched on the context stream, which keeps it ordered with everything else.
      if (!cap) {
        cudaStream_t cs = nullptr;
        KSS_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cap = cs;
      }
      const bool prof_on = ctx->prof.on;
      ctx->prof.on = false;  // no event records inside the captured region
      cudaStream_t home = ctx->stream;
      ctx->stream = (cudaStream_t)cap;
      KSS_CHECK_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      try {
        if (f64) launch_filter_t<double>();
        else launch_filter_t<float>();
      } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(ctx->stream, &g);
        if (g) cudaGraphDestroy(g);
        ctx->stream = home;
        ctx->prof.on = prof_on;
        throw;
      }
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g);
      ctx->stream = home;
      if (ec != cudaSuccess) {
        ctx->prof.on = prof_on;
        KSS_CHECK_CUDA(ec);
      }
      cudaGraphExec_t ex = nullptr;
      const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      ctx->prof.on = prof_on;
      KSS_CHECK_CUDA(e);
      gexec = ex;
      // launches recorded during capture are not executions
      ctx->prof.launches -= (long long)per_step * steps;
    }
    static const int idg = prof_register("batch_filter_graph");
    {
      ProfScope ps(ctx, idg);
      KSS_CHECK_CUDA(cudaGraphLaunch((cudaGraphExec_t)gexec, ctx->stream));
    }
    ctx->prof.launches += (long long)per_step * steps - 1;
  } else {
    if (f64) launch_filter_t<double>();
    else launch_filter_t<float>();
  }
}

// One lockstep iteration over every unit that is not done.
void BatchEngine::iterate(std::vector<kss_solver_s*>& all) {
  // Units that have not started: initial Rayleigh-Ritz on their starting block.
  std::vector<kss_solver_s*> fresh, active;
  for (auto* s : all) {
    if (s->done) continue;
    (s->started ? active : fresh).push_back(s);
  }
  std::vector<kss_solver_s*> rr_units;
  std::vector<int> ry, rhy, rxo, rhxo;
  for (auto* s : fresh) {
    apply_h(s->sys, s->ik, s->nb, s->blk[0].p, nullptr, s->blk[1].p, s->npw, ChebCoef{1, 0, 0},
            s->f64 ? KSS_PREC_FP64 : KSS_PREC_MIXED);
    s->napply += s->nb;
    rr_units.push_back(s);
    ry.push_back(0);
    rhy.push_back(1);
    rxo.push_back(2);
    rhxo.push_back(3);
  }
  if (!active.empty()) {
    set_units(active);
    run_filter();
    for (size_t u = 0; u < active.size(); ++u) {
      kss_solver_s* s = active[u];
      s->napply += (long long)s->nb * (udeg[u] + 1);
      rr_units.push_back(s);
      ry.push_back(roles[u].y);
      rhy.push_back(roles[u].hy);
      rxo.push_back(roles[u].free2);
      rhxo.push_back(s->ihx);
    }
  }
  if (!rr_units.empty()) {
    bool gram64_any = false;
    for (auto* s : rr_units) gram64_any |= s->gram64;
    if (use_batched_rr && !gram64_any) rr_batched(rr_units, ry, rhy, rxo, rhxo);
    else rr_all(rr_units, ry, rhy, rxo, rhxo);
  }
  KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  KSS_CHECK_CUDA(cudaGetLastError());
  for (auto* s : fresh) {
    rr_finish_or_retry(s, s->f64, s->blk[0].p, s->blk[1].p, s->blk[2].p, s->blk[3].p);
    s->ix = 2;
    s->ihx = 3;
    s->started = true;
    decide(s);
  }
  for (size_t u = 0; u < active.size(); ++u) {
    kss_solver_s* s = active[u];
    rr_finish_or_retry(s, s->f64, s->blk[roles[u].y].p, s->blk[roles[u].hy].p, s->blk[roles[u].free2].p,
                       s->blk[s->ihx].p);
    s->ix = roles[u].free2;
    s->iter += 1;
    decide(s);
  }
}

void BatchEngine::decide(kss_solver_s* s) {
  const double r = max_wanted(s);
  s->hist.push_back(r);
  if (s->f64) {
    s->converged = r <= s->tol;
    s->done = s->converged || s->iter >= s->o.max_iter;
  } else {
    bool stalled = false;
    const size_t h = s->hist.size();
    if (h >= 4) stalled = s->hist[h - 1] > 0.9 * s->hist[h - 4] && s->hist[h - 1] < 100.0 * s->tol;
    if (r <= s->tol || stalled || s->iter >= s->o.max_iter) {
      refine_fp64(s);
      s->converged = max_wanted(s) <= s->tol;
      // as in the single-system solver: a block that misses the tolerance in the FP64 check with
      // the split-BF16 projector products continues with FP32 products
      if (!s->converged && !s->proj32 && s->sys->nproj && s->iter < s->o.max_iter) {
        s->proj32 = true;
        s->hist.clear();
        return;
      }
      s->done = true;
    }
  }
}

void BatchEngine::rr_batched(const std::vector<kss_solver_s*>& us, const std::vector<int>& y,
                             const std::vector<int>& hy, const std::vector<int>& xo,
                             const std::vector<int>& hxo) {
  KSS_NVTX("batch_rayleigh_ritz");
  const int U = (int)us.size();
  int np = 0;
  for (auto* s : us) np = std::max(np, s->nb);
  cudaStream_t st = ctx->stream;
  const size_t mat = (size_t)np * np;
  Sb.ensure((size_t)U * mat * sizeof(double2));
  Hb.ensure((size_t)U * mat * sizeof(double2));
  Wb.ensure((size_t)U * np * sizeof(double));
  binfo.ensure((size_t)U * sizeof(int));
  double2* S = Sb.as<double2>();
  double2* H = Hb.as<double2>();
  bool any64 = false;
  for (auto* s : us) any64 |= s->f64;
  if (!any64) {
    rr_batched_grouped(us, y, hy, xo, hxo, np);
    return;
  }
  // Gram and projected-H matrices of every unit, into the leading nb x nb blocks.  The batch's
  // units are small (16-141 bands): one SIMT product per unit beats the tensor-core digit products,
  // whose operand preparation and 128 x 64 tiles do not pay at these sizes (measured).
  for (int u = 0; u < U; ++u) {
    kss_solver_s* s = us[u];
    const int nb = s->nb, npw = s->npw;
    const void* Y = s->blk[y[u]].p;
    const void* HY = s->blk[hy[u]].p;
    if (s->f64) {
      gemm_cn(ctx, true, nb, nb, npw, Y, npw, Y, npw, S + u * mat, np, 1, 0, 0, 0, "gram");
      gemm_cn(ctx, true, nb, nb, npw, Y, npw, HY, npw, H + u * mat, np, 1, 0, 0, 0, "gram");
    } else {
      gemm_cn(ctx, false, nb, nb, npw, Y, npw, Y, npw, s->S32.p, nb, 1, 0, 0, 0, "gram");
      gemm_cn(ctx, false, nb, nb, npw, Y, npw, HY, npw, s->Hs32.p, nb, 1, 0, 0, 0, "gram");
      const long long nn = (long long)nb * nb;
      c64_to_c128_ld<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(s->S32.as<float2>(), nb, S + u * mat, np);
      c64_to_c128_ld<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(s->Hs32.as<float2>(), nb, H + u * mat, np);
    }
  }
  // every unit's FP64 generalised eigensolve (H_s q = lambda S q) in one launch, one CTA per unit
  int* dinfo = binfo.as<int>();
  std::vector<HegvItem> items(U);
  for (int u = 0; u < U; ++u)
    items[u] = HegvItem{H + u * mat, S + u * mat, Wb.as<double>() + (size_t)u * np, dinfo + u, us[u]->nb, np, np, false};
  hegv_batched(ctx, items);
  // rotations, residuals and results of every unit
  for (int u = 0; u < U; ++u) {
    kss_solver_s* s = us[u];
    const int nb = s->nb, npw = s->npw;
    const void* Y = s->blk[y[u]].p;
    const void* HY = s->blk[hy[u]].p;
    void* Xo = s->blk[xo[u]].p;
    void* HXo = s->blk[hxo[u]].p;
    const double2* Q = H + u * mat;
    if (s->f64) {
      gemm_nn(ctx, true, npw, nb, nb, Y, npw, Q, np, Xo, npw, 1, 0, 0, 0, "rotate");
      gemm_nn(ctx, true, npw, nb, nb, HY, npw, Q, np, HXo, npw, 1, 0, 0, 0, "rotate");
    } else {
      const long long nn = (long long)nb * nb;
      c128_ld_to_c64<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Q, np, s->Q32.as<float2>(), nb);
      gemm_nn(ctx, false, npw, nb, nb, Y, npw, s->Q32.p, nb, Xo, npw, 1, 0, 0, 0, "rotate");
      gemm_nn(ctx, false, npw, nb, nb, HY, npw, s->Q32.p, nb, HXo, npw, 1, 0, 0, 0, "rotate");
    }
    const double* W = Wb.as<double>() + (size_t)u * np;
    residual_norms(ctx, s->f64, Xo, HXo, npw, nb, npw, W, s->resid_d.as<double>());
    if (!s->hpin) KSS_CHECK_CUDA(cudaMallocHost((void**)&s->hpin, (2 * (size_t)nb + 1) * sizeof(double)));
    KSS_CHECK_CUDA(cudaMemcpyAsync(s->hpin, W, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    KSS_CHECK_CUDA(cudaMemcpyAsync(s->hpin + nb, s->resid_d.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  binfo_h.assign(U, 0);
  KSS_CHECK_CUDA(cudaMemcpyAsync(binfo_h.data(), dinfo, U * sizeof(int), cudaMemcpyDeviceToHost, st));
  KSS_CHECK_CUDA(cudaStreamSynchronize(st));
  for (int u = 0; u < U; ++u) {
    // status word read by rr_finish
    const int info = binfo_h[u];
    std::memcpy(us[u]->hpin + 2 * us[u]->nb, &info, sizeof(int));
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

// Single precision: the Rayleigh-Ritz of every unit in a fixed number of grouped launches (the
// Gram and projected-H products of all units in one SIMT launch with FP32 partial sums added in
// FP64, the batched FP64 eigensolve, the eigenvectors to complex64, the rotations of all units in
// one launch, the residuals of all bands in one launch) instead of about twenty launches per unit.
void BatchEngine::rr_batched_grouped(const std::vector<kss_solver_s*>& us, const std::vector<int>& y,
                                     const std::vector<int>& hy, const std::vector<int>& xo,
                                     const std::vector<int>& hxo, int np) {
  const int U = (int)us.size();
  cudaStream_t st = ctx->stream;
  const size_t mat = (size_t)np * np;
  double2* S = Sb.as<double2>();
  double2* H = Hb.as<double2>();
  // Gram (Y^H Y) and projected H (Y^H HY) of every unit
  std::vector<GemmItem> g(2 * (size_t)U);
  for (int u = 0; u < U; ++u) {
    kss_solver_s* s = us[u];
    for (int k = 0; k < 2; ++k) {
      GemmItem& e = g[2 * u + k];
      e = GemmItem{};
      e.M = e.N = s->nb;
      e.K = s->npw;
      e.A = s->blk[y[u]].p;
      e.lda = s->npw;
      e.B = k ? s->blk[hy[u]].p : s->blk[y[u]].p;
      e.ldb = s->npw;
      e.C = (k ? H : S) + u * mat;
      e.ldc = np;
      e.s = 1.0;
    }
  }
  int gb = 0, grb = 0;
  group_plan(ctx, g, true, &gb, &grb);
  size_t part = 0;
  for (auto& e : g) part += (size_t)e.splits * e.M * e.N;
  rr_part.ensure(part * sizeof(float2));
  part = 0;
  for (auto& e : g) {
    e.P = rr_part.as<float2>() + part;
    part += (size_t)e.splits * e.M * e.N;
  }
  // rotations X = Y Q, HX = HY Q and the per-unit conversion / residual items
  std::vector<GemmItem> rot(2 * (size_t)U);
  std::vector<RrItem> it(U);
  long long qb = 0, rb = 0;
  for (int u = 0; u < U; ++u) {
    kss_solver_s* s = us[u];
    const int nb = s->nb, npw = s->npw;
    s->Q32.ensure((size_t)nb * nb * sizeof(float2));
    for (int k = 0; k < 2; ++k) {
      GemmItem& e = rot[2 * u + k];
      e = GemmItem{};
      e.M = npw;
      e.N = nb;
      e.K = nb;
      e.A = k ? s->blk[hy[u]].p : s->blk[y[u]].p;
      e.lda = npw;
      e.B = s->Q32.p;
      e.ldb = nb;
      e.C = k ? s->blk[hxo[u]].p : s->blk[xo[u]].p;
      e.ldc = npw;
      e.ar = 1.0;
      e.br = 0.0;
    }
    RrItem& t = it[u];
    t.Q = H + u * mat;
    t.Q32 = s->Q32.as<float2>();
    t.X = s->blk[xo[u]].as<float2>();
    t.HX = s->blk[hxo[u]].as<float2>();
    t.w = Wb.as<double>() + (size_t)u * np;
    t.r = s->resid_d.as<double>();
    t.np = np;
    t.nb = nb;
    t.npw = npw;
    t.q0 = qb;
    t.r0 = rb;
    qb += ((long long)nb * nb + 255) / 256;
    rb += nb;
  }
  int rotb = 0, rotrb = 0;
  group_plan(ctx, rot, false, &rotb, &rotrb);
  // tables through one pinned staging buffer (rewritten only after this call's synchronisation)
  const size_t bg = g.size() * sizeof(GemmItem), br = rot.size() * sizeof(GemmItem), bi = it.size() * sizeof(RrItem);
  unsigned char* h = (unsigned char*)stage(bg + br + bi);
  std::memcpy(h, g.data(), bg);
  std::memcpy(h + bg, rot.data(), br);
  std::memcpy(h + bg + br, it.data(), bi);
  d_rr_g.ensure(bg);
  d_rr_rot.ensure(br);
  d_rr_it.ensure(bi);
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_rr_g.p, h, bg, cudaMemcpyHostToDevice, st));
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_rr_rot.p, h + bg, br, cudaMemcpyHostToDevice, st));
  KSS_CHECK_CUDA(cudaMemcpyAsync(d_rr_it.p, h + bg + br, bi, cudaMemcpyHostToDevice, st));
  group_gemm_cn_c64_to_c128(ctx, d_rr_g.as<GemmItem>(), 2 * U, gb, grb);
  // every unit's FP64 generalised eigensolve (H_s q = lambda S q) in one launch, one CTA per unit
  int* dinfo = binfo.as<int>();
  std::vector<HegvItem> items(U);
  for (int u = 0; u < U; ++u)
    items[u] = HegvItem{H + u * mat, S + u * mat, Wb.as<double>() + (size_t)u * np, dinfo + u, us[u]->nb, np, np, false};
  hegv_batched(ctx, items);
  {
    static const int id = prof_register("group_q_to_c64");
    ProfScope ps(ctx, id);
    rr_q_to_c64<<<(unsigned)qb, 256, 0, st>>>(d_rr_it.as<RrItem>(), U);
    KSS_CHECK_CUDA(cudaGetLastError());
  }
  group_gemm_nn(ctx, false, d_rr_rot.as<GemmItem>(), 2 * U, rotb);
  {
    static const int id = prof_register("group_residuals");
    ProfScope ps(ctx, id);
    rr_residuals<<<(unsigned)rb, 256, 0, st>>>(d_rr_it.as<RrItem>(), U);
    KSS_CHECK_CUDA(cudaGetLastError());
  }
  for (int u = 0; u < U; ++u) {
    kss_solver_s* s = us[u];
    const int nb = s->nb;
    const double* W = Wb.as<double>() + (size_t)u * np;
    if (!s->hpin) KSS_CHECK_CUDA(cudaMallocHost((void**)&s->hpin, (2 * (size_t)nb + 1) * sizeof(double)));
    KSS_CHECK_CUDA(cudaMemcpyAsync(s->hpin, W, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    KSS_CHECK_CUDA(cudaMemcpyAsync(s->hpin + nb, s->resid_d.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  binfo_h.assign(U, 0);
  KSS_CHECK_CUDA(cudaMemcpyAsync(binfo_h.data(), dinfo, U * sizeof(int), cudaMemcpyDeviceToHost, st));
  KSS_CHECK_CUDA(cudaStreamSynchronize(st));
  for (int u = 0; u < U; ++u) {
    const int info = binfo_h[u];
    std::memcpy(us[u]->hpin + 2 * us[u]->nb, &info, sizeof(int));
  }
  KSS_CHECK_CUDA(cudaGetLastError());
}

}  // namespace kss

using namespace kss;

extern "C" kss_status kss_solve_batch(kss_ctx ctx, int n, const kss_sys* sys, const int* ik,
                                      const int* nband, const kss_solve_opts* opts,
                                      double* const* evals, double* const* resid,
                                      kss_solve_stats* stats) {
  if (!ctx) return KSS_EINVAL;
  std::vector<kss_solver> made;
  try {
    KSS_REQUIRE(n >= 0 && (n == 0 || (sys && ik && nband)), "kss_solve_batch: bad arguments");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    kss_solve_opts o{};
    if (opts) o = *opts;
    KSS_REQUIRE(o.x0 == nullptr, "kss_solve_batch takes no warm start (use the server or solvers)");
    for (int u = 0; u < n; ++u) {
      KSS_REQUIRE(sys[u] && sys[u]->ctx == ctx, "every system must belong to this context");
      if (sys[u]->has_S)
        fail(KSS_ENOTSUP, "batched solves take systems without an overlap (solve generalised problems per system)");
      kss_solve_opts ou = o;
      ou.seed = o.seed + (uint64_t)u;
      ou.flags |= KSS_SOLVE_NO_GAMMA_REAL;  // the grouped passes do not pack Gamma bands
      kss_solver s = nullptr;
      const kss_status st = kss_solver_create(sys[u], ik[u], nband[u], &ou, &s);
      if (st != KSS_OK) fail(st, ctx->err);
      made.push_back(s);
    }
    BatchEngine eng;
    eng.ctx = ctx;
    eng.use_graph = !(o.flags & KSS_SOLVE_BATCH_NO_GRAPH);
    eng.use_tc_gemm = !(o.flags & KSS_SOLVE_BATCH_FP32_PROJ);
    eng.f64 = n ? made[0]->f64 : true;
    for (auto* s : made)
      KSS_REQUIRE(s->f64 == eng.f64 && s->o.degree == made[0]->o.degree,
                  "batched units share precision and filter degree");
    eng.degree = n ? made[0]->o.degree : 10;
    std::vector<kss_solver_s*> all(made.begin(), made.end());
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      bool any = false;
      for (auto* s : all) any |= !s->done;
      if (!any) break;
      eng.iterate(all);
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool allconv = true;
    for (int u = 0; u < n; ++u) {
      kss_solver_s* s = made[u];
      allconv &= s->converged;
      if (evals && evals[u]) std::memcpy(evals[u], s->evals.data(), s->nband * sizeof(double));
      if (resid && resid[u]) std::memcpy(resid[u], s->resid.data(), s->nband * sizeof(double));
      if (stats) {
        stats[u].iters = s->iter;
        stats[u].napply = s->napply;
        stats[u].max_resid = max_wanted(s);
        stats[u].ms_filter = 0;
        stats[u].ms_rr = 0;
        stats[u].ms_total = ms;
        stats[u].nb = s->nb;
      }
    }
    for (auto s : made) kss_solver_destroy(s);
    made.clear();
    if (!allconv) {
      ctx->err = "at least one unit did not converge within max_iter";
      return KSS_ENOCONV;
    }
    ctx->err.clear();
    return KSS_OK;
  } catch (const KssError& e) {
    for (auto s : made) kss_solver_destroy(s);
    ctx->err = e.msg;
    return e.st;
  } catch (...) {
    for (auto s : made) kss_solver_destroy(s);
    ctx->err = "unexpected internal error";
    return KSS_ECUDA;
  }
}

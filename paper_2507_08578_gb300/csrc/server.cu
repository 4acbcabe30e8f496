// Request server: eigensolves of different cells, cutoffs and band counts taken as they arrive,
// the way high-throughput campaigns feed many independent calculations (§7), served by
// continuous batching on the lockstep engine.
//
// Every pump tick (1) admits queued requests in arrival order while the HBM budget and the slot
// limit allow (a request's k-points become units of the engine; its tables and blocks stay
// resident on the device until it completes), (2) runs one lockstep iteration over every unit in
// flight -- new units do their initial Rayleigh-Ritz in the same tick as the others filter --
// and (3) retires finished requests: results to host memory, the converged subspace of each
// k-point into a warm-start cache keyed by the request's content (a repeated cell starts from
// it), device memory back to the budget, latency recorded.  Work of one unit never depends on
// which other units share the launch, so a result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <unordered_map>

#include "batch.h"

namespace kss {

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Request {
  uint64_t id = 0;
  double lattice[9];
  double ecut = 0;
  std::vector<double> kpts, pos, D;
  int fft_box[3] = {0, 0, 0};
  double vamp = 0, vsig = 1, alpha = 0.25;
  int nppa = 0;
  int nband = 0;
  uint64_t key = 0;
  double t_submit = 0, t_done = 0;
  bool admitted = false, done = false, warm = false;
  kss_status status = KSS_OK;
  std::string err;
  kss_sys sys = nullptr;
  std::vector<kss_solver> solvers;
  size_t bytes = 0;
  std::vector<double> evals, resid;  // nk * nband, k-major
  int iters = 0;
};

struct WarmEntry {
  std::vector<DevBuf> x;  // per k-point: nband x npw block of the request's precision
  std::vector<int> npw;
  size_t bytes = 0;
};

}  // namespace

struct Server {
  kss_ctx ctx = nullptr;
  size_t budget = 0, used = 0, peak = 0;
  int max_slots = 0, slots = 0;
  kss_solve_opts opts{};
  BatchEngine eng;
  uint64_t next_id = 1;
  std::map<uint64_t, Request> reqs;
  std::deque<uint64_t> pending;
  std::list<uint64_t> lru;  // warm-start cache order (front = newest)
  std::unordered_map<uint64_t, WarmEntry> cache;
  size_t cache_bytes = 0, cache_cap = 0;
  std::vector<double> lat;
  long long warm_hits = 0, rejected = 0, completed = 0;
  double t_first = -1, t_last = 0;

  size_t estimate(const Request& r) const {
    // Plane waves per k from the sphere volume (4/3 pi (2 Ecut)^{3/2} Omega / (2 pi)^3), +15%.
    double vol = std::fabs(r.lattice[0] * (r.lattice[4] * r.lattice[8] - r.lattice[5] * r.lattice[7]) -
                           r.lattice[1] * (r.lattice[3] * r.lattice[8] - r.lattice[5] * r.lattice[6]) +
                           r.lattice[2] * (r.lattice[3] * r.lattice[7] - r.lattice[4] * r.lattice[6]));
    const double npw = 1.15 * vol * std::pow(2.0 * r.ecut, 1.5) / (6.0 * M_PI * M_PI) + 64;
    const int nk = (int)(r.kpts.size() / 3);
    const size_t es = opts.prec == KSS_PREC_FP64 ? 16 : 8;
    const int nb = r.nband + std::max(4, (r.nband + 9) / 10);
    const size_t nproj = (r.pos.size() / 3) * r.nppa;
    size_t per_k = (size_t)(4 * npw * nb * es + npw * nproj * 24 + 3.0 * nb * nb * 16 + npw * 64);
    if (opts.prec == KSS_PREC_MIXED) per_k += (size_t)(4 * npw * nb * 16);
    const double box = 4.0 * std::pow(npw, 1.0 / 3.0) * 1.6;  // default-rule box edge, generous
    per_k += (size_t)(box * npw * 0.6 * nb * es);            // FFT slab of the batched launch
    return (size_t)nk * per_k + (size_t)(box * box * box * 16);
  }

  void admit() {
    while (!pending.empty()) {
      Request& r = reqs[pending.front()];
      const int nk = (int)(r.kpts.size() / 3);
      size_t need = estimate(r);
      const bool first = slots == 0 && used == 0;
      if (!first && (slots + nk > max_slots || used + need > budget)) break;
      pending.pop_front();
      try {
        kss_cell cell{};
        std::memcpy(cell.lattice, r.lattice, sizeof(cell.lattice));
        cell.ecut = r.ecut;
        cell.nk = nk;
        cell.kpts_red = r.kpts.data();
        std::memcpy(cell.fft_box, r.fft_box, sizeof(cell.fft_box));
        kss_atoms at{};
        at.natom = (int)(r.pos.size() / 3);
        at.pos_cart = r.pos.data();
        at.vloc_amp = r.vamp;
        at.vloc_sigma = r.vsig;
        at.nproj_per_atom = r.nppa;
        at.proj_alpha = r.alpha;
        at.D = r.D.data();
        kss_status st = kss_setup(ctx, &cell, &at, &r.sys);
        if (st != KSS_OK) fail(st, ctx->err);
        auto hit = cache.find(r.key);
        for (int ik = 0; ik < nk; ++ik) {
          kss_solve_opts o = opts;
          // The start block depends on the request's content (its cache key), not on when it
          // arrived: the same cell starts from the same block alone or in any mix.
          o.seed = opts.seed + r.key * 16 + (uint64_t)ik;
          if (hit != cache.end() && hit->second.npw[ik] == r.sys->k[ik].npw) {
            o.x0 = hit->second.x[ik].p;
            o.x0_nb = r.nband;
            o.x0_ld = r.sys->k[ik].npw;
            r.warm = true;
          }
          kss_solver s = nullptr;
          o.flags |= KSS_SOLVE_NO_GAMMA_REAL;  // the lockstep engine does not pack Gamma bands
          st = kss_solver_create(r.sys, ik, r.nband, &o, &s);
          if (st != KSS_OK) fail(st, ctx->err);
          r.solvers.push_back(s);
        }
        if (r.warm) {
          warm_hits += 1;
          lru.remove(r.key);
          lru.push_front(r.key);
        }
        r.admitted = true;
        // Charged from here on: what the request holds, its system's tables plus one solver per
        // k-point (kss_footprint: blocks, Rayleigh-Ritz matrices, workspaces, split projector
        // tables); the estimate above only decided the admission.
        size_t fp = 0;
        if (kss_footprint(r.sys, r.nband, opts.prec, &fp) == KSS_OK) need = sys_device_bytes(r.sys) + (size_t)nk * fp;
        r.bytes = need;
        used += need;
        slots += nk;
        peak = std::max(peak, used);
      } catch (const KssError& e) {
        for (auto s : r.solvers) kss_solver_destroy(s);
        r.solvers.clear();
        if (r.sys) kss_sys_destroy(r.sys);
        r.sys = nullptr;
        r.done = true;
        r.status = e.st;
        r.err = e.msg;
        r.t_done = now_ms();
        rejected += 1;
      }
    }
  }

  void remember(Request& r) {
    // Keep the converged subspace of every k-point for a later request with the same content.
    if (cache.count(r.key) || cache_cap == 0) return;
    WarmEntry w;
    const size_t es = opts.prec == KSS_PREC_FP64 ? 16 : 8;
    for (auto s : r.solvers) w.bytes += (size_t)s->npw * r.nband * es;
    if (w.bytes > cache_cap) return;
    while (cache_bytes + w.bytes > cache_cap && !lru.empty()) {
      const uint64_t old = lru.back();
      lru.pop_back();
      cache_bytes -= cache[old].bytes;
      cache.erase(old);
    }
    for (auto s : r.solvers) {
      DevBuf b;
      b.alloc((size_t)s->npw * r.nband * es);
      kss_solver_results(s, nullptr, nullptr, b.p, s->npw, nullptr);
      w.npw.push_back(s->npw);
      w.x.push_back(std::move(b));
    }
    cache_bytes += w.bytes;
    lru.push_front(r.key);
    cache.emplace(r.key, std::move(w));
  }

  void retire() {
    for (auto& kv : reqs) {
      Request& r = kv.second;
      if (!r.admitted || r.done) continue;
      bool all = true;
      for (auto s : r.solvers) all &= s->done;
      if (!all) continue;
      const int nk = (int)r.solvers.size();
      r.evals.assign((size_t)nk * r.nband, 0.0);
      r.resid.assign((size_t)nk * r.nband, 0.0);
      bool conv = true;
      for (int ik = 0; ik < nk; ++ik) {
        kss_solver_s* s = r.solvers[ik];
        std::memcpy(&r.evals[(size_t)ik * r.nband], s->evals.data(), r.nband * sizeof(double));
        std::memcpy(&r.resid[(size_t)ik * r.nband], s->resid.data(), r.nband * sizeof(double));
        conv &= s->converged;
        r.iters = std::max(r.iters, s->iter);
      }
      r.status = conv ? KSS_OK : KSS_ENOCONV;
      remember(r);
      for (auto s : r.solvers) kss_solver_destroy(s);
      r.solvers.clear();
      kss_sys_destroy(r.sys);
      r.sys = nullptr;
      used -= r.bytes;
      slots -= nk;
      r.done = true;
      r.t_done = now_ms();
      t_last = r.t_done;
      lat.push_back(r.t_done - r.t_submit);
      completed += 1;
    }
  }

  void tick() {
    admit();
    std::vector<kss_solver_s*> units;
    for (auto& kv : reqs)
      if (kv.second.admitted && !kv.second.done)
        for (auto s : kv.second.solvers)
          if (!s->done) units.push_back(s);
    if (!units.empty()) eng.iterate(units);
    retire();
  }

  ~Server() {
    for (auto& kv : reqs) {
      for (auto s : kv.second.solvers) kss_solver_destroy(s);
      if (kv.second.sys) kss_sys_destroy(kv.second.sys);
    }
  }
};

}  // namespace kss

using namespace kss;

namespace {
template <typename F>
kss_status sguard(kss_ctx ctx, F&& f) {
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
Server* srv(kss_ctx ctx) {
  if (!ctx->server) fail(KSS_EINVAL, "no server running on this context (kss_server_start)");
  return static_cast<Server*>(ctx->server);
}
}  // namespace

extern "C" {

kss_status kss_server_start(kss_ctx ctx, size_t hbm_budget_bytes, int max_slots,
                            const kss_solve_opts* opts) {
  if (!ctx) return KSS_EINVAL;
  return sguard(ctx, [&] {
    KSS_REQUIRE(!ctx->server, "a server is already running on this context");
    KSS_REQUIRE(hbm_budget_bytes > 0 && max_slots > 0, "budget and slot limit must be positive");
    std::unique_ptr<Server> s(new Server());
    s->ctx = ctx;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    if (opts) s->opts = *opts;
    KSS_REQUIRE(s->opts.x0 == nullptr, "server options take no warm start");
    KSS_REQUIRE(s->opts.prec == KSS_PREC_FP64 || s->opts.prec == KSS_PREC_MIXED, "unknown precision");
    if (s->opts.degree <= 0) s->opts.degree = 10;
    s->eng.ctx = ctx;
    s->eng.f64 = s->opts.prec == KSS_PREC_FP64;
    s->eng.degree = s->opts.degree;
    s->eng.use_graph = !(s->opts.flags & KSS_SOLVE_BATCH_NO_GRAPH);
    s->eng.use_tc_gemm = !(s->opts.flags & KSS_SOLVE_BATCH_FP32_PROJ);
    s->cache_cap = hbm_budget_bytes / 10;
    ctx->server = s.release();
  });
}

kss_status kss_server_submit(kss_ctx ctx, const kss_cell* cell, const kss_atoms* atoms, int nband,
                             uint64_t* ticket) {
  if (!ctx) return KSS_EINVAL;
  return sguard(ctx, [&] {
    Server* s = srv(ctx);
    KSS_REQUIRE(cell && atoms && ticket && nband >= 1, "kss_server_submit: bad arguments");
    KSS_REQUIRE(cell->nk >= 1 && cell->kpts_red, "need at least one k-point");
    KSS_REQUIRE(atoms->natom >= 0 && (atoms->natom == 0 || atoms->pos_cart), "bad atoms");
    if (atoms->Q && atoms->natom && atoms->nproj_per_atom)
      for (int i = 0; i < atoms->natom * atoms->nproj_per_atom; ++i)
        if (atoms->Q[i] != 0.0) fail(KSS_ENOTSUP, "the server takes atoms without an overlap");
    if (s->pending.size() >= 65536) fail(KSS_EBUSY, "server queue is full");
    Request r;
    r.id = s->next_id++;
    std::memcpy(r.lattice, cell->lattice, sizeof(r.lattice));
    r.ecut = cell->ecut;
    r.kpts.assign(cell->kpts_red, cell->kpts_red + 3 * cell->nk);
    std::memcpy(r.fft_box, cell->fft_box, sizeof(r.fft_box));
    r.pos.assign(atoms->pos_cart, atoms->pos_cart + 3 * atoms->natom);
    r.nppa = atoms->natom ? atoms->nproj_per_atom : 0;
    if (r.nppa) r.D.assign(atoms->D, atoms->D + (size_t)atoms->natom * r.nppa);
    r.vamp = atoms->vloc_amp;
    r.vsig = atoms->vloc_sigma;
    r.alpha = atoms->proj_alpha;
    r.nband = nband;
    if (s->estimate(r) > s->budget) fail(KSS_EBUSY, "request alone exceeds the server's HBM budget");
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, r.lattice, sizeof(r.lattice));
    h = fnv(h, &r.ecut, sizeof(r.ecut));
    h = fnv(h, r.kpts.data(), r.kpts.size() * sizeof(double));
    h = fnv(h, r.pos.data(), r.pos.size() * sizeof(double));
    h = fnv(h, r.D.data(), r.D.size() * sizeof(double));
    h = fnv(h, r.fft_box, sizeof(r.fft_box));
    h = fnv(h, &r.vamp, sizeof(double));
    h = fnv(h, &r.vsig, sizeof(double));
    h = fnv(h, &r.alpha, sizeof(double));
    h = fnv(h, &r.nppa, sizeof(int));
    h = fnv(h, &r.nband, sizeof(int));
    r.key = h;
    r.t_submit = now_ms();
    if (s->t_first < 0) s->t_first = r.t_submit;
    *ticket = r.id;
    s->pending.push_back(r.id);
    s->reqs.emplace(r.id, std::move(r));
  });
}

kss_status kss_server_pump(kss_ctx ctx, double max_ms, int* in_flight, int* queued) {
  if (!ctx) return KSS_EINVAL;
  return sguard(ctx, [&] {
    Server* s = srv(ctx);
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    const double t0 = now_ms();
    do {
      s->tick();
      bool busy = !s->pending.empty();
      for (auto& kv : s->reqs) busy |= kv.second.admitted && !kv.second.done;
      if (!busy) break;
    } while (now_ms() - t0 < max_ms);
    int fl = 0;
    for (auto& kv : s->reqs) fl += kv.second.admitted && !kv.second.done;
    if (in_flight) *in_flight = fl;
    if (queued) *queued = (int)s->pending.size();
  });
}

kss_status kss_server_poll(kss_ctx ctx, uint64_t ticket, int* done, double* evals, double* resid,
                           double* latency_ms) {
  if (!ctx) return KSS_EINVAL;
  kss_status st = KSS_OK;
  kss_status g = sguard(ctx, [&] {
    Server* s = srv(ctx);
    auto it = s->reqs.find(ticket);
    KSS_REQUIRE(it != s->reqs.end(), "unknown or already collected ticket");
    Request& r = it->second;
    if (done) *done = r.done ? 1 : 0;
    if (!r.done) return;
    if (evals && !r.evals.empty()) std::memcpy(evals, r.evals.data(), r.evals.size() * sizeof(double));
    if (resid && !r.resid.empty()) std::memcpy(resid, r.resid.data(), r.resid.size() * sizeof(double));
    if (latency_ms) *latency_ms = r.t_done - r.t_submit;
    st = r.status;
    const std::string msg = r.err;
    s->reqs.erase(it);
    if (st != KSS_OK && st != KSS_ENOCONV) fail(st, msg);
  });
  if (g != KSS_OK) return g;
  return st;
}

kss_status kss_server_get_stats(kss_ctx ctx, kss_server_stats* out) {
  if (!ctx || !out) return KSS_EINVAL;
  return sguard(ctx, [&] {
    Server* s = srv(ctx);
    std::vector<double> l = s->lat;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
      if (l.empty()) return 0.0;
      const size_t i = (size_t)std::min<double>(l.size() - 1, std::ceil(p * l.size()) - 1);
      return l[i];
    };
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->warm_hits = s->warm_hits;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double m = 0;
    for (double v : l) m += v;
    out->mean_ms = l.empty() ? 0 : m / l.size();
    const double span = s->t_last - s->t_first;
    out->solves_per_s = span > 0 ? 1000.0 * s->completed / span : 0;
    out->peak_bytes = s->peak;
    out->in_flight_bytes = s->used;
  });
}

kss_status kss_server_stop(kss_ctx ctx) {
  if (!ctx) return KSS_EINVAL;
  return sguard(ctx, [&] {
    Server* s = srv(ctx);
    KSS_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
    delete s;
    ctx->server = nullptr;
  });
}

}  // extern "C"

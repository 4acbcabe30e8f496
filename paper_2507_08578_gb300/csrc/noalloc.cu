// kss_apply_H_noalloc: H psi for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need H psi: code running while a
// CUDA graph is being captured, a host whose allocator is owned by another runtime (a framework's
// caching allocator or a pool with a fixed budget), or a real-time loop where an allocation (and
// the device synchronisation cudaFree implies) is not allowed.  kss_apply_H may grow the
// context's workspaces; this entry point never allocates.  Every temporary it needs -- the FFT
// slab of a band chunk, the projector coefficients and the split-K partial sums of the
// coefficient product -- lives in one file-scope device array of KSS_NOALLOC_SCRATCH_BYTES that
// every GPU which loads the library holds until the process exits.
#include "kss_internal.h"

namespace {

// The scratch array.  In host code `g_noalloc_scratch` is only a host-side stand-in for the
// symbol, never a device address: host code must use the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KSS_NOALLOC_SCRATCH_BYTES];

// The address is looked up once per context, on that context's first call, with its device
// current, and kept in the context.  A context made after the CUDA context of its device was torn
// down and rebuilt (cudaDeviceReset, or a runtime that released the primary context) looks the
// symbol up again, so no call ever uses an address from an earlier CUDA context.
void* scratch_address(kss_ctx ctx) {
  if (!ctx->noalloc_scratch) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      kss::fail(KSS_ECUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                               cudaGetErrorString(e));
    }
    ctx->noalloc_scratch = p;
  }
  return ctx->noalloc_scratch;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

using namespace kss;

extern "C" kss_status kss_apply_H_noalloc(kss_sys sys, int ik, int nb, const void* psi, void* hpsi,
                                          int ld, kss_precision prec) {
  if (!sys) return KSS_EINVAL;
  kss_ctx ctx = sys->ctx;
  try {
    KSS_REQUIRE(ik >= 0 && ik < (int)sys->k.size(), "k-point index out of range");
    KSS_REQUIRE(nb >= 0, "nb < 0");
    KSS_REQUIRE(prec == KSS_PREC_FP64 || prec == KSS_PREC_MIXED, "unknown precision");
    const KData& kd = sys->k[ik];
    KSS_REQUIRE(ld >= kd.npw, "ld < npw");
    if (nb == 0) {
      ctx->err.clear();
      return KSS_OK;
    }
    KSS_REQUIRE(psi && hpsi, "null psi or hpsi");
    KSS_REQUIRE(psi != hpsi, "psi and hpsi must not overlap");
    const bool f64 = prec == KSS_PREC_FP64;
    const size_t es = f64 ? 16 : 8;
    // Scratch plan: [projector coefficients | split-K partial sums | slab chunk].
    const size_t cprj = sys->nproj ? align256((size_t)sys->nproj * nb * es) : 0;
    const size_t plane = local_slab_bytes_per_band(sys, ik, prec);
    const size_t cap = KSS_NOALLOC_SCRATCH_BYTES;
    const size_t need_min = cprj + cprj + align256(plane);  // one split of partials, one band
    if (need_min > cap)
      fail(KSS_EINVAL, "kss_apply_H_noalloc: this request needs at least " + std::to_string(need_min) +
                           " bytes of scratch (nproj=" + std::to_string(sys->nproj) + ", nb=" +
                           std::to_string(nb) + ", one FFT slab of " + std::to_string(plane) +
                           " bytes) but the static scratch holds " + std::to_string(cap) +
                           " bytes; split the band block");
    KSS_CHECK_CUDA(cudaSetDevice(ctx->device));
    unsigned char* base = static_cast<unsigned char*>(scratch_address(ctx));
    // Partial sums get up to half of what the slab does not need for one band.
    size_t part = 0;
    if (sys->nproj) {
      const size_t free_after = cap - cprj - align256(plane);
      part = std::max(cprj, (free_after / 2) / cprj * cprj);
    }
    const size_t slab_off = cprj + align256(part);
    const int nc = (int)std::max<size_t>(1, std::min<size_t>((size_t)nb, (cap - slab_off) / plane));
    if (sys->nproj) {
      void* C = base;
      const bool ok = gemm_cn_ws(ctx, f64, sys->nproj, nb, kd.npw, f64 ? kd.d_beta64.p : kd.d_beta32.p,
                                 kd.npw, psi, ld, C, sys->nproj, base + cprj, part);
      if (!ok) fail(KSS_EINVAL, "kss_apply_H_noalloc: partial sums do not fit the static scratch");
      scale_rows_noprof(f64, sys->nproj, nb, C, sys->nproj, f64 ? sys->d_D64.p : sys->d_D32.p, 1.0,
                        ctx->stream);
    }
    local_apply_ws(sys, ik, nb, psi, hpsi, ld, prec, base + slab_off, nc);
    if (sys->nproj)
      gemm_nn_noprof(f64, kd.npw, nb, sys->nproj, f64 ? kd.d_beta64.p : kd.d_beta32.p, kd.npw, base,
                     sys->nproj, hpsi, ld, ctx->stream);
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

// Internal declarations shared by the library's translation units.  Not part of the ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <map>
#include <vector>

#include "../../include/kss.h"

namespace kss {

// Errors are thrown as KssError inside the library and turned into a kss_status (with the
// message stored in the context) at the ABI edge.  Nothing throws across extern "C".
struct KssError {
  kss_status st;
  std::string msg;
};

[[noreturn]] void fail(kss_status st, const std::string& msg);

#define KSS_CHECK_CUDA(call)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      ::kss::fail(KSS_ECUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_));  \
  } while (0)

#define KSS_REQUIRE(cond, msg)                          \
  do {                                                  \
    if (!(cond)) ::kss::fail(KSS_EINVAL, (msg));        \
  } while (0)

// Owning device allocation (cudaMalloc / cudaFree).  Move-only.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release();
  void alloc(size_t n);           // exact size, discards contents
  void ensure(size_t n);          // grow-only, discards contents when it grows
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// One radix-{2,3,4,5} factorisation of a transform length (Stockham stages in order).
struct FftDim {
  int N;
  int nst;
  int rad[10];
};
FftDim make_fft_dim(int N);  // N must be {2,3,5}-smooth, 1 < N <= 256

// An operand of the FP64 tensor-core GEMMs (gemm_oz.cu) in digit form: 7 planes [rows][KT] of
// BF16 digits (KT = 2K rounded up to 32, the (re, im) pairs interleaved along K) and one exponent
// per row.
struct OzOperand {
  __nv_bfloat16* planes = nullptr;
  int* e = nullptr;
  int rows = 0, KT = 0;
  int S = 7;                       // digits per value: 7 (complex128 data) or 4 (complex64 data)
};

// Per-k-point data.
struct KData {
  double kred[3];
  int npw = 0;
  int lo[3], W[3];                 // sphere bounding box: m_i in [lo_i, lo_i + W_i)
  std::vector<int32_t> miller;     // host copy, npw*3
  std::vector<int32_t> zstart;     // W3 + 1: sphere index range of each z-slice
  std::vector<int32_t> rowrange;   // 2*W3: [first, last] row u2 present in each z-slice
  DevBuf d_miller, d_offset, d_tileidx, d_zstart, d_rowrange;
  DevBuf d_kin64, d_kin32;         // 0.5 |k+G|^2
  DevBuf d_beta64, d_beta32;       // projector-major [nproj][npw] complex
  DevBuf d_btc_cn, d_btc_nn;       // mixed: split-BF16 forms of beta for beta^H psi and beta C (lazy)
  DevBuf d_oz_cn, d_oz_nn;         // FP64: digit planes of beta for beta^H psi and beta C (lazy)
  OzOperand oz_cn, oz_nn;          //   and their descriptions
  DevBuf d_q;                      // Cartesian k+G, npw*3 doubles (setup only)
  double tmax = 0;
  double bound = 0;                // rigorous spectral upper bound of H
  double bound_f = 0;              // same for the filter operator (H, or S^-1 H with an overlap)
  std::vector<double> beta_norm2;  // |beta_i|^2 per projector
  bool gamma = false;              // k = 0: the sphere is symmetric under G -> -G
  DevBuf d_mirror;                 // Gamma only: sphere index of -G for every G
  DevBuf d_G64, d_G32;             // overlap only: projector Gram matrix beta^H beta, nproj^2
  DevBuf d_W64, d_W32;             // overlap only: W = Q (1 + G Q)^-1, so S^-1 = 1 - beta W beta^H
};

// Kernel launch accounting: every launch of the library's kernels is counted; when profiling
// is enabled a pair of CUDA events brackets each launch on the context stream.
struct Prof {
  bool on = false;
  long long launches = 0;
  std::vector<long long> count;  // per registered kernel name
  std::vector<double> ms;
  std::vector<cudaEvent_t> free_ev;
  struct Pending { cudaEvent_t a, b; int id; };
  std::vector<Pending> pending;
};
int prof_register(const char* name);   // process-wide id of a kernel name
const char* prof_name(int id);
int prof_names();

}  // namespace kss

struct kss_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int nsys = 0;
  kss::DevBuf ws_local;            // FFT plane workspace
  kss::DevBuf ws_gemm;             // split-K partial sums
  kss::DevBuf ws_cprj;             // projector coefficients
  kss::DevBuf stage_in, stage_out; // host-buffer entry point staging
  kss::DevBuf tc_a, tc_b, tc_part;  // tensor-core GEMM operands (BF16 split) and partial sums
  kss::DevBuf tc_err;               // device failure flag of the tensor-core kernels
  kss::Prof prof;
  int nsm = 0;
  void* server = nullptr;          // request server (server.cu), NULL when not running
  int autotune = 1;                // 1: time FFT schedule candidates at first use (tune.cu)
  kss::DevBuf ws_sapply, ws_e, ws_f; // overlap: L psi block, E = beta^H H psi, F (nproj x nb)
  kss::DevBuf ws_occ, ws_rho;      // density build: occupations, per-group partial densities
  kss::DevBuf ws_gpack;            // Gamma-packed raw transforms (pairs x ld)
  kss::DevBuf ws_tune;             // scratch slab of the autotuner
  std::vector<kss_ctx_s*> aux;     // helper contexts on their own streams (concurrent Rayleigh-Ritz)
  kss::DevBuf oz_a, oz_b, oz_part;  // FP64 tensor-core GEMMs: digit planes of A and B, partial sums
  kss::DevBuf tune_c;              // scratch output of the GEMM K-split tuner
  kss::DevBuf dense_ws, dense_ctl, dense_items;  // dense FP64 eigensolver: workspace, grid
                                   // barrier control block, pencil table
  void* noalloc_scratch = nullptr; // device address of the no-alloc scratch array, looked up on
                                   // this context's first kss_apply_H_noalloc call (noalloc.cu)
};

struct kss_sys_s {
  kss_ctx ctx = nullptr;
  double lat[9];
  double B[9];
  double vol = 0;
  double ecut = 0;
  int N[3];
  int natom = 0, nppa = 0, nproj = 0;
  std::vector<double> pos, D;
  double vamp = 0, vsig = 1, alpha = 0.25;
  double vmax = 0;
  kss::FftDim dim[3];
  kss::DevBuf d_V64;               // V(r_j), [j3][j2][j1], unscaled
  kss::DevBuf d_Vx64, d_Vx32;      // V(r_j)/(N1 N2 N3) in [j1][j2][j3] order (plane kernel)
  kss::DevBuf d_tw64[3], d_tw32[3];// e^{-2 pi i k/N_d}, k < N_d
  kss::DevBuf d_D64, d_D32;
  std::map<int, kss::DevBuf> vpi64, vpi32;  // V/N^3 as [x][z][p] per split code A*32+B (lazy)
  std::map<int, kss::DevBuf> vfused32;       // V/N^3 in the fused kernel's digit-reversed order (lazy)
  bool has_S = false;              // generalised problem: S = 1 + sum_i |beta_i> q_i <beta_i|
  std::vector<double> Q;           // overlap coefficients (nproj), empty without an overlap
  kss::DevBuf d_Q64, d_Q32;
  std::vector<kss::KData> k;
  int nsolvers = 0;
};

struct kss_solver_s {
  kss_sys sys = nullptr;
  int ik = 0, nband = 0, nb = 0, npw = 0;
  kss_solve_opts o{};
  bool f64 = true;
  double tol = 1e-8;
  kss::DevBuf blk[4];
  int ix = 0, ihx = 1;
  kss::DevBuf S, Hs, W, work, info, resid_d;
  kss::DevBuf S32, Hs32, Q32;
  kss::DevBuf r64[4];  // FP64 refinement blocks (mixed precision)
  kss::DevBuf sblk, sblk64;  // overlap only: S Y, then S X (solver precision / FP64 refinement)
  int lwork = 0;
  std::vector<double> evals, resid;
  int iter = 0;
  bool started = false, done = false, converged = false;
  long long napply = 0;
  double ms_filter = 0, ms_rr = 0, ms_total = 0;
  std::vector<double> hist;  // max wanted residual per iteration
  double* hpin = nullptr;    // pinned host: evals[nb], resid[nb], info (as double) for async RR
  bool gamma = false;        // Gamma point with real-space-real bands (packed FFTs, real RR)
  bool gram64 = false;       // mixed precision: Gram matrices accumulated in FP64 (after a failed
                             // Cholesky of the FP32-accumulated ones)
  bool proj32 = false;       // mixed precision: projector products on the FP32 CUDA cores (after the
                             // FP64 check of a block filtered with the split-BF16 products missed
                             // the tolerance)
  ~kss_solver_s();
};


namespace kss {

// RAII bracket around one kernel launch (count + optional CUDA events on ctx->stream).
struct ProfScope {
  kss_ctx ctx;
  int id;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(kss_ctx c, int id_);
  ~ProfScope();
};
void prof_resolve(kss_ctx ctx);  // synchronise and fold pending event pairs into totals
void prof_fold(kss_ctx ctx);     // add the helper contexts' counts and times into ctx's
kss_ctx aux_ctx(kss_ctx ctx, int i);  // helper context i of ctx (created on first use)
void aux_release(kss_ctx ctx);
void prof_release(kss_ctx ctx);
// Host-side NVTX range over one phase of the path (setup, H application, filter, Rayleigh-Ritz),
// in an NVTX domain "kss" of its own so that a caller's ranges in the default domain keep their
// nesting; profilers that read NVTX show it on the timeline, and it costs a few ns when none is
// attached.
inline nvtxDomainHandle_t nvtx_domain() {
  static const nvtxDomainHandle_t d = nvtxDomainCreateA("kss");
  return d;
}
struct NvtxRange {
  explicit NvtxRange(const char* name) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(nvtx_domain(), &a);
  }
  ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define KSS_NVTX(name) ::kss::NvtxRange kss_nvtx_range_(name)
#define KSS_PROF(ctx, name)                                   \
  static const int kss_prof_id_ = ::kss::prof_register(name); \
  ::kss::ProfScope kss_prof_scope_((ctx), kss_prof_id_)

// ---- setup kernels (setup_kernels.cu) ----
void launch_vloc(kss_sys s, cudaStream_t st);
void launch_projectors(kss_sys s, KData& kd, cudaStream_t st);
void launch_vloc_views(kss_sys s, cudaStream_t st);
double device_max(const double* x, size_t n, cudaStream_t st);
void projector_norms(const double* beta, int npw, int nproj, std::vector<double>& out,
                     cudaStream_t st);
void convert_f64_to_f32(const double* in, float* out, size_t n, cudaStream_t st);

// ---- local part + H application (local_apply.cu) ----
struct ChebCoef {
  double alpha, beta, gamma;
  bool packed = false;  // Gamma point, real-space-real bands: two bands per complex FFT
  bool fp32_proj = false;  // mixed precision: projector products on the FP32 CUDA cores instead of
                           // the split-BF16 tensor-core products
};
// out = alpha*(T psi + V psi + nonlocal psi) + beta*psi + gamma*psi_prev (psi_prev may be null)
void apply_h(kss_sys s, int ik, int nb, const void* psi, const void* psi_prev, void* out, int ld,
             ChebCoef c, kss_precision prec);
// Split-BF16 forms of a k-point's complex64 projector table for the tensor-core products
// beta^H psi and beta C (built on first use and kept with the system).
const void* beta_split_cn(kss_sys s, int ik);
const void* beta_split_nn(kss_sys s, int ik);
// V/N^3 of the system in the [x][z][p] layout of the CTA-wide pass B for split N2 = N3 = A*B (p the
// digit-reversed y position k2 + B k of y = k + A k2), built on first use and kept.
const void* vpi_view(kss_sys s, int A, int B, bool f64);
// out = T psi + V psi (the local part only)
void apply_local(kss_sys s, int ik, int nb, const void* psi, void* out, int ld, kss_precision prec);
// ---- generalised problem with a nonlocal overlap (overlap.cu) ----
void overlap_setup(kss_sys s);
// out = S psi on ctx's stream (out = psi without an overlap)
void apply_s(kss_ctx ctx, kss_sys s, int ik, int nb, const void* psi, void* out, int ld, kss_precision prec);
// out = alpha * F psi + beta * psi + gamma * psi_prev, F = H or S^-1 H (with an overlap)
void apply_filter_op(kss_sys s, int ik, int nb, const void* psi, const void* psi_prev, void* out, int ld,
                     ChebCoef c, kss_precision prec);
size_t local_workspace_bytes(kss_sys s, int ik, int nb, kss_precision prec);
// Bytes of y-z slab one launch of the local passes covers: small enough that the slab written by
// pass A is still in L2 when passes B and C read it (with V, psi and the projector operands
// streaming through the same L2).
constexpr size_t kSlabChunkBytes = 64ull << 20;
size_t sys_device_bytes(kss_sys s);  // device bytes of a system's tables (api.cpp)
// Caller-provided workspace forms (used by the entry point that allocates nothing).
size_t local_slab_bytes_per_band(kss_sys s, int ik, kss_precision prec);
void local_apply_ws(kss_sys s, int ik, int nb, const void* psi, void* out, int ld,
                    kss_precision prec, void* work, int nc);
bool gemm_cn_ws(kss_ctx ctx, bool fp64, int M, int N, int K, const void* A, int lda, const void* B,
                int ldb, void* C, int ldc, void* partials, size_t partial_bytes);
void scale_rows_noprof(bool fp64, int M, int N, void* C, int ldc, const void* d, double s,
                       cudaStream_t st);
void gemm_nn_noprof(bool fp64, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                    void* C, int ldc, cudaStream_t st);

// ---- complex GEMMs (gemm_simt.cu) ----
// C (M x N, col-major ldc) = alpha * A^H B + beta * C; A: K x M (lda), B: K x N (ldb)
void gemm_cn(kss_ctx ctx, bool fp64, int M, int N, int K, const void* A, int lda, const void* B,
             int ldb, void* C, int ldc, double alpha_re, double alpha_im, double beta_re,
             double beta_im, const char* tag);
// C (M x N) = alpha * A B + beta * C; A: M x K (lda), B: K x N (ldb)
void gemm_nn(kss_ctx ctx, bool fp64, int M, int N, int K, const void* A, int lda, const void* B,
             int ldb, void* C, int ldc, double alpha_re, double alpha_im, double beta_re,
             double beta_im, const char* tag);
// Grouped products for batched solves: one launch over many independent (M, N, K) items.
// Device-resident item table; group_plan fills tm/tn/splits/kchunk/blk0/rblk0.
struct GemmItem {
  int M, N, K;
  const void* A;
  long long lda;
  const void* B;
  long long ldb;
  void* C;
  long long ldc;
  void* P;          // split-K partial sums (cn form)
  const void* d;    // optional row scale d[i] (real, precision type), applied as s * d[i] (cn form)
  double s;
  double ar, br;    // nn form: C = ar * A B + br * C (real coefficients)
  int tm, tn, splits, kchunk, blk0, rblk0;
  int idle;         // the item's blocks return at once (unit past its own filter degree)
};
void group_plan(kss_ctx ctx, std::vector<GemmItem>& items, bool cn, int* blocks, int* rblocks);
void group_gemm_cn(kss_ctx ctx, bool fp64, const GemmItem* d_items, int n, int blocks, int rblocks);
void group_gemm_nn(kss_ctx ctx, bool fp64, const GemmItem* d_items, int n, int blocks);
// Grouped complex64 A^H B products (d null, s = 1) delivered in complex128 at C (ldc): FP32 partial
// sums per K chunk, added in FP64.
void group_gemm_cn_c64_to_c128(kss_ctx ctx, const GemmItem* d_items, int n, int blocks, int rblocks);

// Grouped split-BF16 complex64 products on the tensor cores (gemm_tc.cu), for the batch engine:
// the same product of every unit in one persistent launch (plus one launch that splits the B
// operands into BF16 hi/lo rows, and one that adds K-split partial sums when any product is split).
// Product i: C_i = ar * rs[r] * op(A_i) B_i + br * C_i with A_i given in split form (tc_split_cn /
// tc_split_nn: 2 M rows of 2 kpad(K) BF16) and B_i a K x N complex64 block (column j has K values
// at Bsrc + j ldb).  Shapes and the A operands are fixed by build(); B sources, outputs,
// coefficients and idle flags are per step (set(), uploaded with upload(), read by the launches,
// so a CUDA graph of the launches follows later uploads).
struct TcGroupSpec {
  const void* Atc;
  int M, N, K;
  long long ldb, ldc;
  const float* rs;  // real scale of output row i (null: 1)
};
class TcGroupPlan {
 public:
  void build(kss_ctx ctx, const std::vector<TcGroupSpec>& specs, int steps);
  void set(int step, int i, const void* Bsrc, void* C, float ar, float br, bool idle);
  void upload(cudaStream_t st);
  void launch(kss_ctx ctx, int step, const char* tag) const;
  int nprod() const { return n_; }
  int tile_cols() const { return tnp_; }
  int works() const { return nwork_; }
  bool split() const { return any_split_; }

 private:
  int n_ = 0, steps_ = 0, tnp_ = 128, nwork_ = 0, prep_blocks_ = 0;
  long long comb_blocks_ = 0;
  bool any_split_ = false;
  size_t prod_bytes_ = 0, prep_bytes_ = 0;
  std::vector<unsigned char> h_prod_, h_prep_;
  DevBuf d_maps_, d_prod_, d_prep_, d_btc_, d_part_;
};

// Complex64 GEMMs on the tensor cores (BF16 hi/lo split, FP32 accumulation in TMEM).
void tc_gemm_cn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                void* C, int ldc, double ar, double ai, double br, double bi, const char* tag);
void tc_gemm_nn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb,
                void* C, int ldc, double ar, double ai, double br, double bi, const char* tag);
int tc_error_flag(kss_ctx ctx, bool reset);
// Runs one bounded wait on a word that nothing writes (it gives up after limit_ms and raises the
// flag read by tc_error_flag): the failure path of the pipeline waits, without a fault.
void tc_wait_selftest(kss_ctx ctx, double limit_ms);
// The same products with the A operand split once in advance (static operands): tc_split_cn /
// tc_split_nn write the split form of A (tc_split_*_bytes) for tc_gemm_cn_split / tc_gemm_nn_split.
size_t tc_split_cn_bytes(int M, int K);
size_t tc_split_nn_bytes(int M, int K);
void tc_split_cn(kss_ctx ctx, int M, int K, const void* A, int lda, void* Atc);
void tc_split_nn(kss_ctx ctx, int M, int K, const void* A, int lda, void* Atc);
void tc_gemm_cn_split(kss_ctx ctx, int M, int N, int K, const void* Atc, const void* B, int ldb, void* C, int ldc,
                      double ar, double ai, double br, double bi, const char* tag);
void tc_gemm_nn_split(kss_ctx ctx, int M, int N, int K, const void* Atc, const void* B, int ldb, void* C, int ldc,
                      double ar, double ai, double br, double bi, const char* tag);
// C (complex128) = A^H B for complex64 A, B with FP64 accumulation.
void gemm_cn_c64_acc64(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B,
                       int ldb, void* C, int ldc, const char* tag);
// Lower triangle of the Hermitian product C = A^H B (M x M; A, B: K x M), strictly upper tiles
// zeroed: FP64 / FP32 (gemm_cn_lower) and complex64 inputs with FP64 accumulation.
void gemm_cn_lower(kss_ctx ctx, bool fp64, int M, int K, const void* A, int lda, const void* B, int ldb,
                   void* C, int ldc, const char* tag);
void gemm_cn_c64_acc64_lower(kss_ctx ctx, int M, int K, const void* A, int lda, const void* B, int ldb,
                             void* C, int ldc, const char* tag);
// Scale row i of a complex (M x N, col-major) matrix by real d[i] * s.
void scale_rows(kss_ctx ctx, bool fp64, int M, int N, void* C, int ldc, const void* d, double s);

// ---- FP64-accurate complex GEMMs on the BF16 tensor cores (gemm_oz.cu) ----
enum OzKind { OZ_CN_A = 0, OZ_B = 1, OZ_MMAJOR_A = 2 };
size_t oz_operand_bytes(int rows, int K, int S = 7);
OzOperand oz_operand_at(void* mem, int rows, int K, int S = 7);
// Digit planes of an n-column (K-major: OZ_CN_A, OZ_B) or n-row (M-major: OZ_MMAJOR_A) complex
// matrix into mem (oz_operand_bytes(rows, K, S) bytes, rows = 2n for the A kinds, n for OZ_B):
// S digits per value (0: 7 from complex128 data, 4 from complex64 data; 7 from complex64 data
// keeps 49 bits below each row's largest entry, for rows whose entries span many scales).
OzOperand oz_prepare(kss_ctx ctx, OzKind kind, int n, int K, const void* src, long long ld, void* mem,
                     bool f64src = true, int S = 0);
// C = alpha A^H B + beta C (A: K x M) and C = alpha A B + beta C (A: M x K, M contiguous),
// column-major; f64in: complex128 operands (FP64-accurate products), else complex64 (with 4
// digits: exact products of the FP32 values to 28 bits of the row scales; with 7: to 49 bits);
// f64out: complex128 C, else complex64.  a_pre: A already in digit form (static operands), else
// prepared here.
void oz_gemm_cn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C, int ldc,
                double ar, double ai, double br, double bi, const char* tag, const OzOperand* a_pre = nullptr,
                bool f64in = true, bool f64out = true, int digits = 0);
void oz_gemm_nn(kss_ctx ctx, int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C, int ldc,
                double ar, double ai, double br, double bi, const char* tag, const OzOperand* a_pre = nullptr,
                bool f64in = true, bool f64out = true, int digits = 0);
// Digit forms of a k-point's FP64 projector table for beta^H psi and beta C (built on first use).
const OzOperand& beta_oz_cn(kss_sys s, int ik);
const OzOperand& beta_oz_nn(kss_sys s, int ik);

// ---- dense FP64 generalised Hermitian eigensolver (dense64.cu) ----
// A x = lambda B x: A, B complex128 column-major (lower triangles read); on return the leading
// n x n block of A holds B-orthonormal eigenvectors (columns, eigenvalues ascending), w[n] the
// eigenvalues, B its Cholesky factor, *info 0, j + 1 (B not positive definite at column j) or -1
// (a bounded grid-barrier wait gave up);
// real: the pencil is real symmetric (imaginary parts ignored, real eigenvectors).  All device
// pointers; queued on ctx's stream.
struct HegvItem {
  void* A;
  void* B;
  double* w;
  int* info;
  int n, lda, ldb;
  bool real;
};
void hegv(kss_ctx ctx, int n, void* A, int lda, void* B, int ldb, double* w, int* info, bool real);
void hegv_batched(kss_ctx ctx, const std::vector<HegvItem>& items);

// ---- solver pieces (solver.cu) ----
void random_block(kss_ctx ctx, bool fp64, void* X, int npw, int nb, int ld, uint64_t seed,
                  int band0);
void residual_norms(kss_ctx ctx, bool fp64, const void* X, const void* HX, int npw, int nb, int ld,
                    const double* w, double* r);
// Solver internals shared with the batched / served engine (batch.cu).
struct ChebParams {
  double e, c, sigma1;
  int degree;  // effective filter degree of this iteration
};
ChebParams cheb_params(const kss_solver_s* s);
// Rayleigh-Ritz in two halves: issue (GEMMs, FP64 eigensolve, rotations, residuals, async copy of
// eigenvalues/residuals/info to pinned host memory) and finish (after the stream is synchronised).
void rr_issue(kss_solver_s* s, bool f64, const void* Y, const void* HY, void* Xo, void* HXo,
              kss_ctx on = nullptr);  // on: queue on another (worker) context's stream
void rr_finish(kss_solver_s* s);
void rr_finish_or_retry(kss_solver_s* s, bool f64, const void* Y, const void* HY, void* Xo, void* HXo);
void refine_fp64(kss_solver_s* s);
double max_wanted(const kss_solver_s* s);

}  // namespace kss
